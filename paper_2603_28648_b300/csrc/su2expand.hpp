// M-expansion of an SU(2) MPS into the U(1)xU(1) form (su2expand.cpp).
#pragma once
#include <map>
#include <utility>
#include <vector>

#include "core.hpp"

namespace qd {

// Clebsch-Gordan coefficient <j1 m1; j2 m2 | J M>, all arguments doubled.
double cg2(int j1, int m1, int j2, int m2, int J, int M);

// A bond's U(1) sectors (n, 2M) and, per (SU(2) sector, 2M), the offset of that
// sector's multiplets inside its U(1) sector.
struct ExpandedBond {
  Basis u1;
  std::map<std::pair<int, int>, int> off;
};
ExpandedBond expand_bond(const Basis& b);

// An MPS around the two-site centre (center, center+1) in the engine's layout,
// host arrays: site tensors per product sector (offsets site_off, target
// sectors site_nb), the two-site state in the psi layout.
struct SU2Mps {
  int L = 0, center = 0, N = 0, two_s = 0;
  std::vector<Basis> bonds;
  std::vector<std::vector<double>> site;
  std::vector<std::vector<int64_t>> site_off;
  std::vector<std::vector<int>> site_nb;
  std::vector<double> psi;
};
struct U1Mps {
  int L = 0, center = 0;
  std::vector<Basis> bonds;
  std::vector<std::vector<double>> site;
  std::vector<std::vector<int64_t>> site_off;
  std::vector<std::vector<int>> site_nb;
  std::vector<double> psi;
};
// The state at M = S as a U(1) MPS with 2Sz = two_s.
void expand_mps_su2(const SU2Mps& in, U1Mps& out);
// the same with the two-site state coupled to the component 2M = two_m
// (-two_s <= two_m <= two_s, two_m = two_s mod 2) instead of M = S
void expand_mps_su2(const SU2Mps& in, U1Mps& out, int two_m);

}  // namespace qd

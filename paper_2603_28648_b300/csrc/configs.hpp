// Configuration-space warm start (configs.cpp): the MPS spanned by a set of
// configurations, and the selection of configurations near an aufbau
// reference. Host code, no device.
//
// A configuration is a step vector of L entries, one per orbital in chain
// order, with the site-state indices of the library: U(1) 0 = |0>,
// 1 = a+_up|0>, 2 = a+_dn|0>, 3 = a+_up a+_dn|0> (a determinant); SU(2)
// 0 = empty, 1 = singly occupied with the spin of the orbitals so far raised
// by 1/2, 2 = singly occupied with it lowered by 1/2, 3 = doubly occupied (a
// configuration state function coupled left to right, the genealogical
// coupling).
#pragma once

#include <cstdint>
#include <vector>

namespace qd {

struct ImportArrays {
  int L = 0, center = 0;
  std::vector<int> nsec, sec;   // the import layout's bond_nsec and (n, two_s, dim) triples
  std::vector<double> data;
};

// The MPS of sum_k coef[k] |config_k> with the centre at (L-2, L-1): bond b
// (b <= L-2) holds every distinct prefix of length b as one state (sectors by
// label, prefixes in lexicographic order inside a sector), the left site
// tensors are 0/1 selectors (orthonormal columns), the two-site wavefunction
// holds the coefficients (repeated configurations add). Throws
// std::invalid_argument for steps outside 0..3, a configuration whose labels
// miss the target (N, two_s), an SU(2) spin that would turn negative, and an
// all-zero coefficient vector.
void configs_to_mps(int L, bool su2, int N, int two_s, int n, const uint8_t* steps, const double* coef,
                    ImportArrays& out);

// Up to nmax configurations of the target ranked by energy: the aufbau
// reference (U(1): the n_up and n_dn orbitals of lowest h_pp; SU(2): doubly
// occupied the (N - 2S)/2 orbitals of lowest h_pp, singly occupied the next
// 2S, all spin steps up) and every configuration at most two electrons away
// from it (determinants; SU(2): spatial occupations with each of their
// genealogical spin couplings). Energy: U(1) the diagonal element <D|H|D>;
// SU(2) the average of <D|H|D> over the determinants of the spatial
// occupation (shared by its couplings). Ties: fewer electrons moved, then
// the step vector in lexicographic order. steps (count * L) and energy
// (count) are filled; returns count.
int select_configs(int L, bool su2, int N, int two_s, const double* h, const double* V, int nmax,
                   std::vector<uint8_t>& steps, std::vector<double>& energy);

}  // namespace qd

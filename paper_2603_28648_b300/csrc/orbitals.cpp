// Orbital-optimisation pieces of DMRG-SCF (host code, no device): the paper
// couples its spin-adapted DMRG to a CAS-SCF orbital optimisation (New benchmark
// system section) in which the DMRG density matrices give the orbital gradient
// and the rotated orbitals give new active-space integrals.
//
// Orbital spaces: core 0..ncore-1 (doubly occupied), active ncore..ncore+nact-1
// (the DMRG active space), virtual the rest. Orbitals rotate as the columns of
// U = exp(kappa), kappa antisymmetric:
//   h'_pq = sum_ab U_ap h_ab U_bq,  (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd).
// The energy at fixed density matrices, E = sum h D + 1/2 sum (pq|rs) P with the
// full-space D (2 on core orbitals, gamma on the active block) and P (the
// product of the core determinant and the active state), changes to first
// order in kappa by dE/dkappa_pq = 2 (F_pq - F_qp) (one parameter per pair,
// kappa_qp = -kappa_pq), with the generalised Fock matrix
//   F_pq = sum_r h_pr D_rq + sum_rst (pr|st) P_qrst,
// which for the three kinds of second index is
//   q core    : F_pq = 2 (IF_pq + AF_pq)
//   q active  : F_pq = sum_v IF_pv gamma_vq + sum_vwx (pv|wx) Gamma_qvwx
//   q virtual : F_pq = 0
// with IF_pq = h_pq + sum_c (2 (pq|cc) - (pc|cq)) (core Fock) and
// AF_pq = sum_tu gamma_tu ((pq|tu) - 1/2 (pt|uq)) (active Fock). The derivation
// takes dh = h kappa - kappa h and the four first-order terms of the two-electron
// integrals, which are equal for the 8-fold symmetric (pq|rs) and a real state.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "orbitals.hpp"

namespace qd {

namespace {

inline size_t I4(int n, int p, int q, int r, int s) { return (((size_t)p * n + q) * n + r) * n + s; }

// C = A B for n x n row-major matrices
void matmul(int n, const double* A, const double* B, double* C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += A[(size_t)i * n + k] * B[(size_t)k * n + j];
      C[(size_t)i * n + j] = s;
    }
}

}  // namespace

void core_fock(int n, int ncore, const double* h, const double* V, double* IF) {
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double s = h[(size_t)p * n + q];
      for (int c = 0; c < ncore; ++c) s += 2.0 * V[I4(n, p, q, c, c)] - V[I4(n, p, c, c, q)];
      IF[(size_t)p * n + q] = s;
    }
}

void active_space(int n, int ncore, int nact, const double* h, const double* V, double* e_core, double* h_act,
                  double* V_act) {
  std::vector<double> IF((size_t)n * n);
  core_fock(n, ncore, h, V, IF.data());
  // E_core = sum_c (h_cc + IF_cc) = sum_c 2 h_cc + sum_cd (2 (cc|dd) - (cd|dc))
  double e = 0.0;
  for (int c = 0; c < ncore; ++c) e += h[(size_t)c * n + c] + IF[(size_t)c * n + c];
  if (e_core) *e_core = e;
  for (int t = 0; t < nact; ++t)
    for (int u = 0; u < nact; ++u) h_act[(size_t)t * nact + u] = IF[(size_t)(ncore + t) * n + ncore + u];
  if (V_act)
    for (int t = 0; t < nact; ++t)
      for (int u = 0; u < nact; ++u)
        for (int v = 0; v < nact; ++v)
          for (int w = 0; w < nact; ++w)
            V_act[I4(nact, t, u, v, w)] = V[I4(n, ncore + t, ncore + u, ncore + v, ncore + w)];
}

void orbital_gradient(int n, int ncore, int nact, const double* h, const double* V, const double* gamma,
                      const double* Gamma, double* G) {
  const int a0 = ncore;
  std::vector<double> IF((size_t)n * n), AF((size_t)n * n, 0.0), F((size_t)n * n, 0.0);
  core_fock(n, ncore, h, V, IF.data());
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double s = 0.0;
      for (int t = 0; t < nact; ++t)
        for (int u = 0; u < nact; ++u) {
          const double g = gamma[(size_t)t * nact + u];
          if (g == 0.0) continue;
          s += g * (V[I4(n, p, q, a0 + t, a0 + u)] - 0.5 * V[I4(n, p, a0 + t, a0 + u, q)]);
        }
      AF[(size_t)p * n + q] = s;
    }
  for (int p = 0; p < n; ++p) {
    for (int c = 0; c < ncore; ++c) F[(size_t)p * n + c] = 2.0 * (IF[(size_t)p * n + c] + AF[(size_t)p * n + c]);
    for (int u = 0; u < nact; ++u) {
      double s = 0.0;
      for (int v = 0; v < nact; ++v) s += IF[(size_t)p * n + a0 + v] * gamma[(size_t)v * nact + u];
      for (int v = 0; v < nact; ++v)
        for (int w = 0; w < nact; ++w)
          for (int x = 0; x < nact; ++x)
            s += V[I4(n, p, a0 + v, a0 + w, a0 + x)] * Gamma[I4(nact, u, v, w, x)];
      F[(size_t)p * n + a0 + u] = s;
    }
  }
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) G[(size_t)p * n + q] = 2.0 * (F[(size_t)p * n + q] - F[(size_t)q * n + p]);
}

void expm_antisym(int n, const double* kappa, double* U) {
  // scaling and squaring: exp(K) = exp(K / 2^s)^(2^s) with ||K / 2^s||_1 <= 1/2,
  // the scaled exponential by its Taylor series to 20 terms (remainder below
  // 2^-20 / 20!, far under the double rounding)
  double nrm = 0.0;
  for (int j = 0; j < n; ++j) {
    double col = 0.0;
    for (int i = 0; i < n; ++i) col += std::fabs(kappa[(size_t)i * n + j]);
    nrm = std::max(nrm, col);
  }
  int s = 0;
  while (nrm > 0.5 && s < 60) {
    nrm *= 0.5;
    ++s;
  }
  const double sc = std::ldexp(1.0, -s);
  std::vector<double> K((size_t)n * n), term((size_t)n * n, 0.0), next((size_t)n * n), E((size_t)n * n, 0.0);
  for (size_t i = 0; i < K.size(); ++i) K[i] = kappa[i] * sc;
  for (int i = 0; i < n; ++i) {
    term[(size_t)i * n + i] = 1.0;
    E[(size_t)i * n + i] = 1.0;
  }
  for (int k = 1; k <= 20; ++k) {
    matmul(n, term.data(), K.data(), next.data());
    for (size_t i = 0; i < next.size(); ++i) {
      term[i] = next[i] / k;
      E[i] += term[i];
    }
  }
  for (int k = 0; k < s; ++k) {
    matmul(n, E.data(), E.data(), next.data());
    E.swap(next);
  }
  for (size_t i = 0; i < E.size(); ++i) U[i] = E[i];
}

void rotate_integrals(int n, const double* U, const double* h, const double* V, double* h_out, double* V_out) {
  // h' = U^T h U
  std::vector<double> t((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int q = 0; q < n; ++q) {
      double s = 0.0;
      for (int b = 0; b < n; ++b) s += h[(size_t)a * n + b] * U[(size_t)b * n + q];
      t[(size_t)a * n + q] = s;
    }
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double s = 0.0;
      for (int a = 0; a < n; ++a) s += U[(size_t)a * n + p] * t[(size_t)a * n + q];
      h_out[(size_t)p * n + q] = s;
    }
  // (pq|rs)' by four quarter transformations, one index at a time
  const size_t n4 = (size_t)n * n * n * n, n3 = (size_t)n * n * n;
  std::vector<double> A(V, V + n4), B(n4);
  for (int pass = 0; pass < 4; ++pass) {
    // transform the last index of A into the first index of B: B[p][...] = sum_a A[...][a] U_ap,
    // so that after four passes the indices are back in order
    for (size_t m = 0; m < n3; ++m)
      for (int p = 0; p < n; ++p) {
        double s = 0.0;
        const double* row = &A[m * n];
        for (int a = 0; a < n; ++a) s += row[a] * U[(size_t)a * n + p];
        B[(size_t)p * n3 + m] = s;
      }
    A.swap(B);
  }
  for (size_t i = 0; i < n4; ++i) V_out[i] = A[i];
}

double fixed_density_energy(int n, int ncore, int nact, const double* h, const double* V, const double* gamma,
                            const double* Gamma) {
  // the frozen-core energy and the active terms of active_space, read straight
  // from V (no active-space copy)
  double e = 0.0;
  for (int c = 0; c < ncore; ++c) {
    e += 2.0 * h[(size_t)c * n + c];
    for (int d = 0; d < ncore; ++d) e += 2.0 * V[I4(n, c, c, d, d)] - V[I4(n, c, d, d, c)];
  }
  const int a0 = ncore;
  for (int t = 0; t < nact; ++t)
    for (int u = 0; u < nact; ++u) {
      double hv = h[(size_t)(a0 + t) * n + a0 + u];
      for (int c = 0; c < ncore; ++c) hv += 2.0 * V[I4(n, a0 + t, a0 + u, c, c)] - V[I4(n, a0 + t, c, c, a0 + u)];
      e += hv * gamma[(size_t)t * nact + u];
    }
  double g = 0.0;
  for (int t = 0; t < nact; ++t)
    for (int u = 0; u < nact; ++u)
      for (int v = 0; v < nact; ++v) {
        const double* row = V + I4(n, a0 + t, a0 + u, a0 + v, a0);
        const double* G = Gamma + (((size_t)t * nact + u) * nact + v) * nact;
        for (int w = 0; w < nact; ++w) g += row[w] * G[w];
      }
  return e + 0.5 * g;
}

void orbital_hessian_diag(int n, int ncore, int nact, const double* h, const double* V, const double* gamma,
                          const double* Gamma, double* H) {
  // Along U(t) = exp(t (e_pq - e_qp)) only orbitals p and q mix,
  //   phi_p' = cos t phi_p - sin t phi_q,  phi_q' = sin t phi_p + cos t phi_q,
  // and the energy at fixed density matrices is a trigonometric polynomial of
  // degree 4 in t (the two-electron integrals are quartic in U). Its values at
  // t_j = 2 pi j / 9, j = 0..8, fix it exactly: a_k = (2/9) sum_j E_j cos(k t_j)
  // and E''(0) = -sum_k k^2 a_k. Each sample rotates the integral slices with an
  // index on p or q in place and puts them back from a copy afterwards.
  const double PI = 3.14159265358979323846;
  std::vector<double> hw(h, h + (size_t)n * n), Vw(V, V + (size_t)n * n * n * n);
  std::fill(H, H + (size_t)n * n, 0.0);
  std::vector<std::pair<size_t, double>> saved;
  auto rot = [&](double* x, double* y, double c, double sn) {   // (x, y) <- (c x - s y, s x + c y)
    const double a = *x, b = *y;
    *x = c * a - sn * b;
    *y = sn * a + c * b;
  };
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < p; ++q) {
      // every entry with an index on p or q (the slices of each position; an
      // entry in several slices is saved more than once, always with its
      // original value)
      saved.clear();
      for (int o : {p, q})
        for (int x = 0; x < n; ++x)
          for (int y = 0; y < n; ++y)
            for (int z = 0; z < n; ++z)
              for (size_t at : {I4(n, o, x, y, z), I4(n, x, o, y, z), I4(n, x, y, o, z), I4(n, x, y, z, o)})
                saved.emplace_back(at, Vw[at]);
      std::vector<double> hsave(hw);
      double a[5] = {0, 0, 0, 0, 0};
      for (int jt = 0; jt < 9; ++jt) {
        const double t = 2.0 * PI * jt / 9.0, c = std::cos(t), sn = std::sin(t);
        for (int i = 0; i < n; ++i) rot(&hw[(size_t)p * n + i], &hw[(size_t)q * n + i], c, sn);
        for (int i = 0; i < n; ++i) rot(&hw[(size_t)i * n + p], &hw[(size_t)i * n + q], c, sn);
        for (int x = 0; x < n; ++x)
          for (int y = 0; y < n; ++y)
            for (int z = 0; z < n; ++z) rot(&Vw[I4(n, p, x, y, z)], &Vw[I4(n, q, x, y, z)], c, sn);
        for (int x = 0; x < n; ++x)
          for (int y = 0; y < n; ++y)
            for (int z = 0; z < n; ++z) rot(&Vw[I4(n, x, p, y, z)], &Vw[I4(n, x, q, y, z)], c, sn);
        for (int x = 0; x < n; ++x)
          for (int y = 0; y < n; ++y)
            for (int z = 0; z < n; ++z) rot(&Vw[I4(n, x, y, p, z)], &Vw[I4(n, x, y, q, z)], c, sn);
        for (int x = 0; x < n; ++x)
          for (int y = 0; y < n; ++y)
            for (int z = 0; z < n; ++z) rot(&Vw[I4(n, x, y, z, p)], &Vw[I4(n, x, y, z, q)], c, sn);
        const double e = fixed_density_energy(n, ncore, nact, hw.data(), Vw.data(), gamma, Gamma);
        for (int k = 1; k <= 4; ++k) a[k] += (2.0 / 9.0) * e * std::cos(k * t);
        hw = hsave;
        for (const auto& sv : saved) Vw[sv.first] = sv.second;
      }
      const double d2 = -(a[1] + 4.0 * a[2] + 9.0 * a[3] + 16.0 * a[4]);
      H[(size_t)p * n + q] = H[(size_t)q * n + p] = d2;
    }
}

}  // namespace qd

// Orbital entanglement and the chain ordering derived from it (host code, no
// device). The paper pre-optimises its chain topology with the
// quantum-information protocols of Barcza et al. (2011) and Szalay et al.
// (2015) (Numerical procedure section): from the two-orbital reduced density
// matrices rho_ij of an approximate state,
//   S_i  = -Tr rho_i ln rho_i     (rho_i = Tr_j rho_ij),
//   S_ij = -Tr rho_ij ln rho_ij,
//   I_ij = S_i + S_j - S_ij       (i != j; 0 on the diagonal),
// and the orbitals are ordered along the chain by the components of the
// Fiedler vector (eigenvector of the second smallest eigenvalue) of the
// weighted graph Laplacian diag(sum_j I_ij) - I, which minimises
// sum_ij I_ij (x_i - x_j)^2 over unit vectors orthogonal to the constant one,
// so that strongly entangled orbitals land close to each other.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <stdexcept>

#include "entanglement.hpp"

namespace qd {

void jacobi_eigh(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>* v) {
  // cyclic-by-row Jacobi (Golub and Van Loan, Matrix Computations, Sec. 8.5):
  // each rotation J in the (p, q) plane, A <- J^T A J, zeroes a_pq; the
  // off-diagonal norm falls quadratically once small
  auto A = [&](int r, int c) -> double& { return a[(size_t)r * n + c]; };
  std::vector<double> V;
  if (v) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  }
  double fro = 0.0;
  for (double x : a) fro += x * x;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += 2.0 * A(p, q) * A(p, q);
    if (!(off > 1e-32 * fro)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A(p, q);
        if (apq == 0.0) continue;
        const double tau = (A(q, q) - A(p, p)) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q of A J
          const double x = A(k, p), y = A(k, q);
          A(k, p) = c * x - s * y;
          A(k, q) = s * x + c * y;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q of J^T (A J)
          const double x = A(p, k), y = A(q, k);
          A(p, k) = c * x - s * y;
          A(q, k) = s * x + c * y;
        }
        A(p, q) = A(q, p) = 0.0;
        if (v)
          for (int k = 0; k < n; ++k) {
            double& x = V[(size_t)k * n + p];
            double& y = V[(size_t)k * n + q];
            const double vx = x, vy = y;
            x = c * vx - s * vy;
            y = s * vx + c * vy;
          }
      }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return A(x, x) < A(y, y); });
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A(idx[i], idx[i]);
  if (v) {
    v->assign((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k)
      for (int i = 0; i < n; ++i) (*v)[(size_t)k * n + i] = V[(size_t)k * n + idx[i]];
  }
}

namespace {

double entropy(int n, const double* rho) {
  // -sum lambda ln lambda over the eigenvalues of the symmetric part; the
  // eigenvalues at or below zero (rounding noise of a PSD matrix) add nothing
  std::vector<double> a((size_t)n * n), w;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) a[(size_t)r * n + c] = 0.5 * (rho[r * n + c] + rho[c * n + r]);
  jacobi_eigh(n, a, w, nullptr);
  double s = 0.0;
  for (double l : w)
    if (l > 0) s -= l * std::log(l);
  return s;
}

}  // namespace

void orbital_entanglement(int L, const double* rho, double* s1, double* mutual) {
  if (L < 2) throw std::invalid_argument("two orbitals at least");
  auto blk = [&](int i, int j) { return rho + ((size_t)i * L + j) * 256; };
  std::vector<double> S(L);
  for (int i = 0; i < L; ++i) {
    // rho_i from the pair with the next orbital (the previous one for the last)
    const bool first = i + 1 < L;
    const double* r = first ? blk(i, i + 1) : blk(i - 1, i);
    double one[16] = {};
    for (int x = 0; x < 4; ++x)
      for (int z = 0; z < 4; ++z)
        for (int y = 0; y < 4; ++y)
          one[x * 4 + z] += first ? r[(4 * x + y) * 16 + 4 * z + y] : r[(4 * y + x) * 16 + 4 * y + z];
    S[i] = entropy(4, one);
  }
  for (int i = 0; i < L; ++i) {
    mutual[(size_t)i * L + i] = 0.0;
    for (int j = i + 1; j < L; ++j) {
      const double m = S[i] + S[j] - entropy(16, blk(i, j));
      mutual[(size_t)i * L + j] = mutual[(size_t)j * L + i] = m;
    }
  }
  if (s1) std::copy(S.begin(), S.end(), s1);
}

void fiedler_order(int L, const double* mutual, int* order, double* fiedler) {
  if (L < 2) throw std::invalid_argument("two orbitals at least");
  std::vector<double> lap((size_t)L * L), w, v;
  for (int i = 0; i < L; ++i) {
    double d = 0.0;
    for (int j = 0; j < L; ++j)
      if (j != i) {
        d += mutual[(size_t)i * L + j];
        lap[(size_t)i * L + j] = -mutual[(size_t)i * L + j];
      }
    lap[(size_t)i * L + i] = d;
  }
  jacobi_eigh(L, lap, w, &v);
  std::vector<double> f(L);
  double big = 0.0, nrm = 0.0;
  for (int i = 0; i < L; ++i) {
    f[i] = v[(size_t)i * L + 1];
    big = std::max(big, std::fabs(f[i]));
    nrm += f[i] * f[i];
  }
  nrm = std::sqrt(nrm);
  double sg = 1.0;
  for (int i = 0; i < L; ++i)
    if (std::fabs(f[i]) > 1e-8 * big) {
      sg = f[i] < 0 ? 1.0 : -1.0;
      break;
    }
  for (double& x : f) x *= sg / nrm;
  std::vector<int> idx(L);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return f[a] < f[b]; });
  std::copy(idx.begin(), idx.end(), order);
  if (fiedler) std::copy(f.begin(), f.end(), fiedler);
}

double ordering_cost(int L, const double* mutual, const int* order, double eta) {
  std::vector<int> pos(L);
  for (int k = 0; k < L; ++k) pos[order[k]] = k;
  double c = 0.0;
  for (int i = 0; i < L; ++i)
    for (int j = i + 1; j < L; ++j) c += mutual[(size_t)i * L + j] * std::pow(std::abs(pos[i] - pos[j]), eta);
  return c;
}

int refine_order(int L, const double* mutual, double eta, int* order, int max_passes) {
  // steepest descent over position exchanges: each candidate exchange of the
  // orbitals at positions a < b is scored by the change of the terms that
  // involve them (O(L) each), the best improving one is taken
  std::vector<int> pos(L);
  for (int k = 0; k < L; ++k) pos[order[k]] = k;
  auto M = [&](int i, int j) { return mutual[(size_t)i * L + j]; };
  std::vector<double> dpow(L);   // |x|^eta for the distances 0..L-1
  for (int x = 0; x < L; ++x) dpow[x] = std::pow((double)x, eta);
  auto d = [&](int x) { return dpow[std::abs(x)]; };
  int made = 0;
  while (made < max_passes) {
    double best = 0.0;
    int ba = -1, bb = -1;
    for (int a = 0; a < L; ++a)
      for (int b = a + 1; b < L; ++b) {
        const int oa = order[a], ob = order[b];
        double delta = 0.0;
        for (int k = 0; k < L; ++k) {
          if (k == oa || k == ob) continue;
          const int pk = pos[k];
          delta += M(oa, k) * (d(b - pk) - d(a - pk)) + M(ob, k) * (d(a - pk) - d(b - pk));
        }
        if (delta < best - 1e-12 * (1.0 + std::fabs(best))) {
          best = delta;
          ba = a;
          bb = b;
        }
      }
    if (ba < 0) break;
    std::swap(order[ba], order[bb]);
    pos[order[ba]] = ba;
    pos[order[bb]] = bb;
    ++made;
  }
  return made;
}

}  // namespace qd

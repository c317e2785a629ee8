// Orbital entanglement and the chain ordering derived from it (entanglement.cpp):
// one-orbital entropies, mutual information of orbital pairs from the
// two-orbital density matrices, and the ordering by the Fiedler vector of the
// mutual-information Laplacian. Host code, row-major arrays.
#pragma once

#include <vector>

namespace qd {

// Symmetric eigenproblem by cyclic Jacobi rotations: a (n*n) is destroyed,
// w gets the eigenvalues ascending, v (if not null) the eigenvectors as the
// columns of an n*n row-major matrix in the same order.
void jacobi_eigh(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>* v);

// rho: L*L blocks of 256, block (i, j) (i < j) the 16 x 16 density matrix of
// orbitals i, j (row 4 x + y). s1 (L) and mutual (L*L, symmetric, zero
// diagonal) are written; s1 may be null.
void orbital_entanglement(int L, const double* rho, double* s1, double* mutual);

// order (L): orbitals sorted by their Fiedler-vector component (ties by
// index); fiedler (L, may be null): that vector, unit length, its first
// component of magnitude above 1e-8 of the largest made negative.
void fiedler_order(int L, const double* mutual, int* order, double* fiedler);

// sum_{i<j} mutual_ij |pos_i - pos_j|^eta for the chain order (order[k] = the
// orbital at position k)
double ordering_cost(int L, const double* mutual, const int* order, double eta);

// order improved in place by exchanging the positions of two orbitals while an
// exchange lowers ordering_cost (best exchange first, at most max_passes
// exchanges); returns the exchanges made
int refine_order(int L, const double* mutual, double eta, int* order, int max_passes);

}  // namespace qd

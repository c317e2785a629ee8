// Orbital-optimisation pieces of DMRG-SCF (orbitals.cpp): core Fock matrix,
// frozen-core active-space integrals, orbital gradient from the active density
// matrices, exp of an antisymmetric generator and the integral rotation.
// Row-major arrays; n orbitals, (pq|rs) at ((p n + q) n + r) n + s.
#pragma once

namespace qd {

void core_fock(int n, int ncore, const double* h, const double* V, double* IF);
void active_space(int n, int ncore, int nact, const double* h, const double* V, double* e_core, double* h_act,
                  double* V_act);
void orbital_gradient(int n, int ncore, int nact, const double* h, const double* V, const double* gamma,
                      const double* Gamma, double* G);
void expm_antisym(int n, const double* kappa, double* U);
void rotate_integrals(int n, const double* U, const double* h, const double* V, double* h_out, double* V_out);
// E = e_core + sum h_act gamma + 1/2 sum V_act Gamma of the given orbitals
double fixed_density_energy(int n, int ncore, int nact, const double* h, const double* V, const double* gamma,
                            const double* Gamma);
// H (n*n, symmetric, zero diagonal): H_pq = d^2 E / d kappa_pq^2 at kappa = 0
// for the rotation exp(kappa_pq (e_pq - e_qp)), E at fixed density matrices
void orbital_hessian_diag(int n, int ncore, int nact, const double* h, const double* V, const double* gamma,
                          const double* Gamma, double* H);

}  // namespace qd

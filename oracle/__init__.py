"""FP64 CPU oracle for the two-site DMRG H_eff.psi hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this
package: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
use it. It shares no code with the CUDA library.

Modules
  fci        determinant-space Hamiltonian built from E_pq (plain definition of H)
  mpsu1      dense U(1)xU(1) MPS with quantum-number labels, canonical forms,
             expansion to the determinant vector, projection definition of H_eff
  dmrgu1     operator-based two-site DMRG with normal and complementary
             renormalized operators (dense blocks), Lanczos, SVD truncation
  mpssu2     SU(2) spin-adapted two-site tangent space (multiplets coupled with
             Clebsch-Gordan coefficients, expanded to determinants) and the
             plain definition H_eff = P^T H_FCI P in that space; the same space
             written as a U(1) MPS with the Clebsch-Gordan map of the
             two-site coefficients
  su2alg     Clebsch-Gordan coefficients, 6j and 9j symbols, recoupling factors
  dmrgsu2    operator-based SU(2) two-site DMRG with reduced operators
  casscf     orbital rotation, frozen-core active space and the energy of
             rotated orbitals at fixed density matrices (DMRG-SCF pieces)
  orbital_qi two-orbital reduced density matrices of a determinant vector,
             orbital entropies, mutual information, Fiedler ordering
  configs    configuration selection near the aufbau reference and the
             determinant expansion of determinants and genealogical spin states

Conventions (the paper states none; fixed here and used by both sides):
  H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps) + e_core,
  E_pq = sum_sigma a+_{p sigma} a_{q sigma}; spin-orbitals ordered 1up,1dn,2up,...
  along the chain; site basis |0>, a+_up|0>, a+_dn|0>, a+_up a+_dn|0>.
"""

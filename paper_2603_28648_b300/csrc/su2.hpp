// SU(2) algebra of the spin-adapted path: Wigner 6j and 9j symbols (Racah
// formula), the reduced matrix element of a coupled product of two tensor
// operators acting on two parts of a coupled basis, the adjoint tensor and
// products of two tensor operators on one site.
//
// Angular momenta are passed doubled (2j). Reduced matrix elements follow the
// Wigner-Eckart convention <j m|T^k_q|j' m'> = <j' m'; k q|j m> <j||T^k||j'>
// (Condon-Shortley Clebsch-Gordan coefficients).
#pragma once
#include <cstdint>

namespace qd {
namespace su2 {

double sixj(int a, int b, int c, int d, int e, int f);
double ninej(int a, int b, int c, int d, int e, int f, int g, int h, int i);

// <(j1 j2)J || [T^k1(1) x U^k2(2)]^k || (j1' j2')J'> / (<j1||T||j1'> <j2||U||j2'>)
//   = sqrt((2J'+1)(2k+1)(2j1+1)(2j2+1)) {j1 j1' k1; j2 j2' k2; J J' k}
// (part 1 first in the fermion order; fermion signs are applied by the caller).
// Cached per thread.
double coupled(int j1, int j2, int J, int j1p, int j2p, int Jp, int k1, int k2, int k);

// reduced element of the adjoint tensor T~_q = (-1)^(k-q) (T_-q)^+ between
// (j' <- j) relative to <j||T||j'> (j: row spin of T, j': column spin):
// (-1)^(j + k - j') sqrt((2j+1)/(2j'+1))
double adjoint(int jr, int jc, int k);

// <j||[T^k1 x U^k2]^k||j'> on one space = sum_j'' same_space(j, j'', j', k1, k2, k)
// <j||T||j''> <j''||U||j'>, with same_space = (-1)^(k+j+j') sqrt((2k+1)(2j''+1))
// {k1 k2 k; j' j j''}
double same_space(int j, int jm, int jp, int k1, int k2, int k);

// recoupling of three angular momenta j1, j2, j3 (all 1/2 here):
// <((j1 j3)J13, j2) J | ((j1 j2)J12, j3) J>
//   = (-1)^(j2 + j3 + J12 + J13) sqrt((2J12+1)(2J13+1)) {j2 j1 J12; j3 J J13}
double swap23(int j1, int j2, int j3, int J12, int J13, int J);
// <(j1, (j2 j3)J23) J | ((j1 j2)J12, j3) J>
//   = (-1)^(j1 + j2 + j3 + J) sqrt((2J12+1)(2J23+1)) {j1 j2 J12; j3 J J23}
double assoc(int j1, int j2, int j3, int J12, int J23, int J);

}  // namespace su2
}  // namespace qd

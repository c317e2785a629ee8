// SU(2) recoupling coefficients of the spin-adapted path (see su2.hpp).
#include "su2.hpp"

#include <cmath>
#include <cstdlib>
#include <unordered_map>

namespace qd {
namespace su2 {

namespace {

// log n! for the factorials of the Racah formulas (arguments stay below 512)
struct LogFact {
  double t[512];
  LogFact() {
    t[0] = 0.0;
    for (int i = 1; i < 512; ++i) t[i] = t[i - 1] + std::log((double)i);
  }
};
double lfact(int n) {
  static const LogFact f;   // initialised once, thread-safe
  return f.t[n];
}

bool tri(int a, int b, int c) { return std::abs(a - b) <= c && c <= a + b && ((a + b + c) & 1) == 0; }

// log Delta(abc) (doubled arguments)
double ldelta(int a, int b, int c) {
  return 0.5 * (lfact((a + b - c) / 2) + lfact((a - b + c) / 2) + lfact((-a + b + c) / 2) - lfact((a + b + c) / 2 + 1));
}

}  // namespace

double sixj(int a, int b, int c, int d, int e, int f) {
  if (!tri(a, b, c) || !tri(a, e, f) || !tri(d, b, f) || !tri(d, e, c)) return 0.0;
  const double pre = ldelta(a, b, c) + ldelta(a, e, f) + ldelta(d, b, f) + ldelta(d, e, c);
  const int a1 = (a + b + c) / 2, a2 = (a + e + f) / 2, a3 = (d + b + f) / 2, a4 = (d + e + c) / 2;
  const int b1 = (a + b + d + e) / 2, b2 = (a + c + d + f) / 2, b3 = (b + c + e + f) / 2;
  int lo = a1;
  if (a2 > lo) lo = a2;
  if (a3 > lo) lo = a3;
  if (a4 > lo) lo = a4;
  int hi = b1;
  if (b2 < hi) hi = b2;
  if (b3 < hi) hi = b3;
  double s = 0.0;
  for (int t = lo; t <= hi; ++t) {
    const double l = lfact(t + 1) - lfact(t - a1) - lfact(t - a2) - lfact(t - a3) - lfact(t - a4) - lfact(b1 - t) -
                     lfact(b2 - t) - lfact(b3 - t) + pre;
    s += ((t & 1) ? -1.0 : 1.0) * std::exp(l);
  }
  return s;
}

double ninej(int a, int b, int c, int d, int e, int f, int g, int h, int i) {
  // sum_x (-1)^(2x) (2x+1) {a b c; f i x} {d e f; b x h} {g h i; x a d}
  int lo = std::abs(a - i), hi = a + i;
  if (std::abs(d - h) > lo) lo = std::abs(d - h);
  if (std::abs(b - f) > lo) lo = std::abs(b - f);
  if (d + h < hi) hi = d + h;
  if (b + f < hi) hi = b + f;
  double s = 0.0;
  for (int x = lo; x <= hi; x += 2)
    s += (x + 1) * sixj(a, b, c, f, i, x) * sixj(d, e, f, b, x, h) * sixj(g, h, i, x, a, d);
  return (lo & 1) ? -s : s;
}

double coupled(int j1, int j2, int J, int j1p, int j2p, int Jp, int k1, int k2, int k) {
  if (!tri(j1p, k1, j1) || !tri(j2p, k2, j2) || !tri(Jp, k, J) || !tri(j1, j2, J) || !tri(j1p, j2p, Jp)) return 0.0;
  // 7 bits per argument (doubled spins up to 127)
  uint64_t key = 0;
  for (int v : {j1, j2, J, j1p, j2p, Jp, k1, k2, k}) key = (key << 7) | (uint64_t)(v & 127);
  thread_local std::unordered_map<uint64_t, double> cache;
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const double v = std::sqrt((double)(Jp + 1) * (k + 1) * (j1 + 1) * (j2 + 1)) * ninej(j1, j1p, k1, j2, j2p, k2, J, Jp, k);
  cache.emplace(key, v);
  return v;
}

double adjoint(int jr, int jc, int k) {
  const int e = (jr + k - jc) / 2;
  return ((e & 1) ? -1.0 : 1.0) * std::sqrt((double)(jr + 1) / (double)(jc + 1));
}

double same_space(int j, int jm, int jp, int k1, int k2, int k) {
  const int e = (k + j + jp) / 2;
  return ((e & 1) ? -1.0 : 1.0) * std::sqrt((double)(k + 1) * (jm + 1)) * sixj(k1, k2, k, jp, j, jm);
}

double swap23(int j1, int j2, int j3, int J12, int J13, int J) {
  const int e = (j2 + j3 + J12 + J13) / 2;
  return ((e & 1) ? -1.0 : 1.0) * std::sqrt((double)(J12 + 1) * (J13 + 1)) * sixj(j2, j1, J12, j3, J, J13);
}

double assoc(int j1, int j2, int j3, int J12, int J23, int J) {
  const int e = (j1 + j2 + j3 + J) / 2;
  return ((e & 1) ? -1.0 : 1.0) * std::sqrt((double)(J12 + 1) * (J23 + 1)) * sixj(j1, j2, J12, j3, J, J23);
}

}  // namespace su2
}  // namespace qd

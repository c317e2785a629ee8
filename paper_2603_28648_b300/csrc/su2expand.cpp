// M-expansion of an SU(2) MPS: the same state written as a U(1)xU(1) MPS whose
// bond states are all M components of the multiplets. Used to measure the
// spin-summed two-particle density matrix of an SU(2) state element by element
// with the U(1) walk of the centre.
//
// Conventions (those of the SU(2) rules): a left product multiplet couples the
// block first, |(x a, s) J m> = sum <S_x m_x; s m_s | J m> |x a m_x> |s m_s>,
// a right one the site first, |(s, y b) J m> = sum <s m_s; S_y m_y | J m>
// |s m_s> |y b m_y>; the site doublet's components are m = +1/2 <-> a+_up|0>
// and m = -1/2 <-> a+_dn|0>; the two-site state holds the reduced elements of
// its M = S component, |((x s1) J_a, (s2 y) J_b) S, S>. Condon-Shortley
// Clebsch-Gordan coefficients throughout. Expanded bond states of a U(1)
// sector (n, 2M) list the SU(2) sectors (n, 2S) with S >= |M| in label order,
// each with its multiplets in order.
#include <cmath>
#include <map>
#include <stdexcept>
#include <vector>

#include "su2expand.hpp"

namespace qd {

namespace {

double lfact(int n) { return std::lgamma((double)n + 1.0); }

// SU(2) channel of a product sub-block -> (doubled spin of the site multiplet)
inline int chan_spin(int ch) { return (ch == 1 || ch == 2) ? 1 : 0; }

// U(1) site states of the multiplet a channel couples, with their doubled m
void chan_states(int ch, int* st, int* m2, int* n) {
  if (ch == 0 || ch == 3) {
    st[0] = ch;
    m2[0] = 0;
    *n = 1;
  } else {
    st[0] = 1;
    m2[0] = 1;
    st[1] = 2;
    m2[1] = -1;
    *n = 2;
  }
}

}  // namespace

double cg2(int j1, int m1, int j2, int m2, int J, int M) {
  // Racah's closed form, angular momenta and projections doubled
  if (m1 + m2 != M) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(M) > J) return 0.0;
  if ((j1 + m1) & 1 || (j2 + m2) & 1 || (J + M) & 1) return 0.0;
  if (J < std::abs(j1 - j2) || J > j1 + j2 || (j1 + j2 + J) & 1) return 0.0;
  const int a = (J + j1 - j2) / 2, b = (J - j1 + j2) / 2, c = (j1 + j2 - J) / 2, d = (j1 + j2 + J) / 2 + 1;
  const double pre = 0.5 * (std::log((double)J + 1.0) + lfact(a) + lfact(b) + lfact(c) - lfact(d) +
                            lfact((J + M) / 2) + lfact((J - M) / 2) + lfact((j1 - m1) / 2) + lfact((j1 + m1) / 2) +
                            lfact((j2 - m2) / 2) + lfact((j2 + m2) / 2));
  double s = 0.0;
  for (int k = 0;; ++k) {
    const int t1 = c - k, t2 = (j1 - m1) / 2 - k, t3 = (j2 + m2) / 2 - k;
    const int t4 = (J - j2 + m1) / 2 + k, t5 = (J - j1 - m2) / 2 + k;
    if (t1 < 0 || t2 < 0 || t3 < 0) break;
    if (t4 < 0 || t5 < 0) continue;
    const double lt = lfact(k) + lfact(t1) + lfact(t2) + lfact(t3) + lfact(t4) + lfact(t5);
    s += ((k & 1) ? -1.0 : 1.0) * std::exp(pre - lt);
  }
  return s;
}

ExpandedBond expand_bond(const Basis& b) {
  ExpandedBond e;
  std::map<QN, int> dims;
  for (int x = 0; x < b.nsec(); ++x)
    for (int m2 = -b.q[x].s; m2 <= b.q[x].s; m2 += 2) dims[QN{b.q[x].n, m2}] += b.dim[x];
  for (auto& kv : dims) e.u1.add(kv.first, kv.second);
  std::map<QN, int> fill;
  for (int x = 0; x < b.nsec(); ++x)
    for (int m2 = -b.q[x].s; m2 <= b.q[x].s; m2 += 2) {
      const QN q{b.q[x].n, m2};
      e.off[{x, m2}] = fill[q];
      fill[q] += b.dim[x];
    }
  return e;
}

void expand_mps_su2(const SU2Mps& in, U1Mps& out) { expand_mps_su2(in, out, in.two_s); }

void expand_mps_su2(const SU2Mps& in, U1Mps& out, int two_m) {
  if (std::abs(two_m) > in.two_s || ((in.two_s - two_m) & 1))
    throw std::invalid_argument("expand_mps_su2: M outside the multiplet");
  const int L = in.L, c = in.center;
  std::vector<ExpandedBond> eb(L + 1);
  out.bonds.assign(L + 1, Basis());
  for (int b = 0; b <= L; ++b) {
    if (b == c + 1) continue;
    eb[b] = expand_bond(in.bonds[b]);
    out.bonds[b] = eb[b].u1;
  }
  out.L = L;
  out.center = c;
  out.site.assign(L, {});
  out.site_off.assign(L, {});
  out.site_nb.assign(L, {});
  int st[2], sm[2], ns = 0;
  for (int p = 0; p < L; ++p) {
    if (p == c || p == c + 1) continue;
    const bool left = p < c;
    const int fb = left ? p : p + 1, tb = left ? p + 1 : p;
    const Basis& F2 = in.bonds[fb];
    const Basis& T2 = in.bonds[tb];
    const Basis& F1 = out.bonds[fb];
    const Basis& T1 = out.bonds[tb];
    ProdBasis pb2 = make_prod(F2, left), pb1 = make_prod(F1, left);
    // U(1) layout of the site tensor (as the import reads it)
    std::vector<int64_t>& so = out.site_off[p];
    std::vector<int>& nb = out.site_nb[p];
    so.assign(pb1.prod.nsec(), -1);
    nb.assign(pb1.prod.nsec(), -1);
    int64_t tot = 0;
    for (int q = 0; q < pb1.prod.nsec(); ++q) {
      const int t = T1.find(pb1.prod.q[q]);
      if (t < 0) continue;
      so[q] = tot;
      nb[q] = t;
      tot += (int64_t)pb1.prod.dim[q] * T1.dim[t];
    }
    std::vector<double>& A = out.site[p];
    A.assign((size_t)std::max<int64_t>(tot, 1), 0.0);
    const std::vector<double>& U = in.site[p];
    for (int s2 = 0; s2 < pb2.nsub(); ++s2) {
      const int q2 = pb2.subs[s2].prod;
      const int t2 = in.site_nb[p][q2];
      if (t2 < 0) continue;
      const int x = pb2.subs[s2].blk, ch = pb2.subs[s2].st;
      const int Sx = F2.q[x].s, J = T2.q[t2].s, sS = chan_spin(ch);
      const int dx = F2.dim[x], dk = T2.dim[t2];
      const int ncol2 = left ? dk : pb2.prod.dim[q2];   // row-major width of the SU(2) matrix
      chan_states(ch, st, sm, &ns);
      for (int mx = -Sx; mx <= Sx; mx += 2)
        for (int u = 0; u < ns; ++u) {
          const int m = mx + sm[u];
          if (std::abs(m) > J) continue;
          const double w = left ? cg2(Sx, mx, sS, sm[u], J, m) : cg2(sS, sm[u], Sx, mx, J, m);
          if (w == 0.0) continue;
          const int x1 = F1.find(QN{F2.q[x].n, mx});
          const int s1 = pb1.find(x1, st[u]);
          const int q1 = pb1.subs[s1].prod;
          const int t1 = nb[q1];
          if (t1 < 0 || T1.q[t1] != QN{T2.q[t2].n, m}) throw std::logic_error("expand_mps_su2: sector mismatch");
          const int ox = eb[fb].off.at({x, mx}), ok = eb[tb].off.at({t2, m});
          const int ncol1 = left ? T1.dim[t1] : pb1.prod.dim[q1];
          for (int a = 0; a < dx; ++a)
            for (int k = 0; k < dk; ++k) {
              const int64_t i2 = left ? (int64_t)(pb2.subs[s2].off + a) * ncol2 + k
                                      : (int64_t)k * ncol2 + pb2.subs[s2].off + a;
              const int64_t i1 = left ? (int64_t)(pb1.subs[s1].off + ox + a) * ncol1 + ok + k
                                      : (int64_t)(ok + k) * ncol1 + pb1.subs[s1].off + ox + a;
              A[(size_t)(so[q1] + i1)] += w * U[(size_t)(in.site_off[p][q2] + i2)];
            }
        }
    }
  }
  // the two-site state: ((x s1) J_a, (s2 y) J_b) S at the component M
  ProdBasis L2 = make_prod(in.bonds[c], true), R2 = make_prod(in.bonds[c + 2], false);
  ProdBasis L1 = make_prod(out.bonds[c], true), R1 = make_prod(out.bonds[c + 2], false);
  const PsiLayout lay2 = make_psi_layout(L2, R2, QN{in.N, in.two_s});
  const PsiLayout lay1 = make_psi_layout(L1, R1, QN{in.N, two_m});
  out.psi.assign((size_t)lay1.size, 0.0);
  const int S = in.two_s, M = two_m;
  int st2[2], sm2[2], ns2 = 0;
  for (const auto& b2 : lay2.blks) {
    const int Ja = L2.sub_qn(b2.lsub).s, Jb = R2.sub_qn(b2.rsub).s;
    const int Sx = in.bonds[c].q[b2.x].s, Sy = in.bonds[c + 2].q[b2.y].s;
    const int sa = chan_spin(b2.i), sb = chan_spin(b2.j);
    chan_states(b2.i, st, sm, &ns);
    chan_states(b2.j, st2, sm2, &ns2);
    for (int ma = -Ja; ma <= Ja; ma += 2) {
      const int mb = M - ma;
      if (std::abs(mb) > Jb) continue;
      const double c0 = cg2(Ja, ma, Jb, mb, S, M);
      if (c0 == 0.0) continue;
      for (int u = 0; u < ns; ++u) {
        const int mx = ma - sm[u];
        if (std::abs(mx) > Sx || ((Sx + mx) & 1)) continue;
        const double c1 = cg2(Sx, mx, sa, sm[u], Ja, ma);
        if (c1 == 0.0) continue;
        for (int v = 0; v < ns2; ++v) {
          const int my = mb - sm2[v];
          if (std::abs(my) > Sy || ((Sy + my) & 1)) continue;
          const double c2 = cg2(sb, sm2[v], Sy, my, Jb, mb);
          if (c2 == 0.0) continue;
          const int x1 = out.bonds[c].find(QN{in.bonds[c].q[b2.x].n, mx});
          const int y1 = out.bonds[c + 2].find(QN{in.bonds[c + 2].q[b2.y].n, my});
          const int bi = lay1.find(L1.find(x1, st[u]), R1.find(y1, st2[v]));
          if (bi < 0) throw std::logic_error("expand_mps_su2: psi block missing");
          const auto& b1 = lay1.blks[bi];
          const int ox = eb[c].off.at({b2.x, mx}), oy = eb[c + 2].off.at({b2.y, my});
          const double w = c0 * c1 * c2;
          for (int a = 0; a < b2.rows; ++a)
            for (int bb = 0; bb < b2.cols; ++bb)
              out.psi[(size_t)(b1.off + (int64_t)(ox + a) * b1.cols + oy + bb)] +=
                  w * in.psi[(size_t)(b2.off + (int64_t)a * b2.cols + bb)];
        }
      }
    }
  }
}

}  // namespace qd

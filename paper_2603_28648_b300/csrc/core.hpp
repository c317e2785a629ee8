// Host-side core of the two-site DMRG hot path: quantum-number layout,
// operator views, complementary-operator rules and segmented-GEMM task lists.
//
// The renormalized-operator formulation is the quantum-chemical DMRG of the
// paper's Method section (memory O(N^2 D^2), compute O(N^4 D^3)): normal
// operators a+_k, a+_k a+_l, a+_k a_l of a block and complementary operators
// S_m, P_ij, Q_il and the block Hamiltonian, built from h_pq and V_pqrs. The
// paper gives no formulas of its own; the ones used are written out next to
// each rule in rules.cpp.
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <vector>

namespace qd {

struct QN {
  int n = 0, s = 0;  // particle number, 2Sz (U(1)) or 2S (SU(2))
  bool operator<(const QN& o) const { return n != o.n ? n < o.n : s < o.s; }
  bool operator==(const QN& o) const { return n == o.n && s == o.s; }
  bool operator!=(const QN& o) const { return !(*this == o); }
  QN operator+(const QN& o) const { return {n + o.n, s + o.s}; }
  QN operator-(const QN& o) const { return {n - o.n, s - o.s}; }
};

// Site basis: 0 = |0>, 1 = a+_up|0>, 2 = a+_dn|0>, 3 = a+_up a+_dn|0>.
// In SU(2) mode the four indices are coupling channels of a block multiplet
// with a site multiplet: 0 = |0>, 1 = the doublet coupled to S + 1/2, 2 = the
// doublet coupled to S - 1/2, 3 = a+_up a+_dn|0>; their label shifts (n, 2S)
// are the same four as the U(1) shifts (n, 2Sz).
constexpr int NSITE = 4;
extern const QN SITE_QN[NSITE];

// Sectors of a block basis, sorted by label.
struct Basis {
  bool su2 = false;          // labels are (n, 2S) of SU(2) multiplets
  std::vector<QN> q;
  std::vector<int> dim;
  std::map<QN, int> idx;
  void add(QN qq, int d);   // call with increasing labels
  int find(QN qq) const {
    auto it = idx.find(qq);
    return it == idx.end() ? -1 : it->second;
  }
  int nsec() const { return (int)q.size(); }
  int64_t total() const;
};

// Enlarged basis of a block and one site. Left: X (x) site, sub-block (x, i).
// Right: site (x) Y, sub-block (j, y). Product sectors group the sub-blocks;
// inside a product sector sub-blocks follow (x, i) (left) or (j, y) (right).
struct Sub {
  int blk, st;   // block sector, site state
  int prod;      // product sector id
  int off;       // row offset inside the product sector
  int dim;
};
struct ProdBasis {
  bool left = true;
  const Basis* blk = nullptr;
  std::vector<Sub> subs;
  Basis prod;
  std::vector<std::vector<int>> prod_subs;  // sub ids of each product sector
  std::vector<int> subidx;                  // blk * NSITE + st -> sub id
  int find(int b, int st) const { return subidx[b * NSITE + st]; }
  int nsub() const { return (int)subs.size(); }
  QN sub_qn(int s) const;
  int blk_parity(int s) const;   // (-1)^n of the block part
  int site_parity(int s) const;  // (-1)^n of the site part
};
ProdBasis make_prod(const Basis& blk, bool left);

// Reference to one dense block of an operator. ptr == 0: identity block.
struct BRef {
  int r = 0, c = 0;        // row / column sector (or sub-block) ids
  uint64_t ptr = 0;        // device address of the stored block
  int rows = 0, cols = 0;  // logical shape
  int ld = 0;              // leading dimension of the stored block
  bool tr = false;         // logical block = stored^T
  double sc = 1.0;
  bool ident() const { return ptr == 0; }
};
struct OpView {
  bool odd = false;
  int k2 = 0;               // SU(2): twice the rank of the tensor operator
  std::vector<BRef> blocks;
  bool empty() const { return blocks.empty(); }
};
OpView transpose(const OpView& o);

// Operator keys.
enum Fam : int { F_I = 0, F_C, F_A, F_B, F_S, F_P, F_Q, F_H,
                 F_L };  // F_L: matrix unit |a><b| of one spatial orbital (index a, unit 4a + b)
struct Key {
  int f, a, b, k;   // family, indices, twice the SU(2) rank (0 in U(1))
  Key(int f_ = 0, int a_ = -1, int b_ = -1, int k_ = 0) : f(f_), a(a_), b(b_), k(k_) {}
  bool operator<(const Key& o) const {
    if (f != o.f) return f < o.f;
    if (a != o.a) return a < o.a;
    if (b != o.b) return b < o.b;
    return k < o.k;
  }
};

// Segmented GEMM task lists. Address fields name a buffer (0 = absolute
// device address, 1 = psi, 2 = sigma, 3 = scratch) plus an element offset,
// so that one list can be replayed on any psi / sigma.
enum Buf : int { B_ABS = 0, B_PSI = 1, B_SIG = 2, B_TMP = 3 };
struct Seg {
  uint64_t a = 0, b = 0;   // a == 0 && abuf == 0: A is the identity
  int abuf = 0, bbuf = 0;  // b == 0 && bbuf == 0: B is the identity too
  int lda = 0, ldb = 0, k = 0;
  int ta = 0, tb = 0;
  double sc = 1.0;
  // H_eff stage-2 segments: sc = asc * bsc, asc from the left block reference,
  // bsc = term coefficient x right reference scalar x fermion parity
  double asc = 1.0, bsc = 1.0;
};
struct Prob {
  uint64_t c = 0;
  int cbuf = 0;
  int m = 0, n = 0, ldc = 0;
  int beta = 0;             // 1: accumulate into C
  int seg0 = 0, nseg = 0;
  double osc = 1.0;         // H_eff stage 1: scalar the stage-2 users of C carry (bsc)
};
struct Launch {
  std::vector<Prob> probs;
  std::vector<Seg> segs;
  double flops = 0;         // algorithmic 2mnk over GEMM segments
  void clear() { probs.clear(); segs.clear(); flops = 0; }
  bool empty() const { return probs.empty(); }
};

// Memory and execution backend.
struct Executor {
  virtual ~Executor() {}
  virtual uint64_t alloc(int64_t nelem) = 0;          // zero-initialised doubles
  virtual void release(uint64_t p) = 0;
  virtual uint64_t tmp(int64_t nelem) = 0;            // scratch buffer base (grows)
  virtual void run(const Launch& l, uint64_t psi, uint64_t sig) = 0;
  virtual void upload(uint64_t dst, const double* h, int64_t n) = 0;
  virtual void download(double* h, uint64_t src, int64_t n) = 0;
  virtual void zero(uint64_t p, int64_t n) = 0;
  // i.i.d. N(0,1) numbers from a counter-based generator (splitmix64 of
  // seed and element index, Box-Muller)
  virtual void randn(uint64_t p, int64_t n, uint64_t seed) = 0;
  // in place: the column-major rows x cols matrix gets orthonormal columns
  // (QR, rows >= cols)
  virtual void orthonormal_cols(uint64_t p, int rows, int cols) = 0;
  virtual double dot(uint64_t x, uint64_t y, int64_t n) = 0;
  virtual void scale(uint64_t x, double a, int64_t n) = 0;
  // y = a x + b y
  virtual void axpby(uint64_t y, double a, uint64_t x, double b, int64_t n) = 0;
  // out[k] = xs[k] . y for k < m (host results; one round trip on a device)
  virtual void mdot(const uint64_t* xs, int m, uint64_t y, int64_t n, double* out) {
    for (int k = 0; k < m; ++k) out[k] = dot(xs[k], y, n);
  }
  // y = sum_k c[k] xs[k] + b y (b = 0: y is not read)
  virtual void mcombine(uint64_t y, const uint64_t* xs, const double* c, int m, double b, int64_t n) {
    if (b == 0.0) zero(y, n);
    else if (b != 1.0) scale(y, b, n);
    for (int k = 0; k < m; ++k) axpby(y, c[k], xs[k], 1.0, n);
  }
  // t = r / max(|d - theta|, floor) (Davidson preconditioner)
  virtual void precond(uint64_t t, uint64_t r, uint64_t d, double theta, double floor, int64_t n) = 0;
  // symmetric eigendecomposition in place: A (n x n, column-major) -> eigenvectors,
  // w (host) -> ascending eigenvalues
  virtual void eigh(uint64_t A, int n, double* w) = 0;
  virtual void copy(uint64_t dst, uint64_t src, int64_t n) = 0;
  // out-of-core store: pinned host buffers and copies on a second stream
  virtual uint64_t host_alloc(int64_t nelem) = 0;
  virtual void host_free(uint64_t h) = 0;
  virtual void d2h(uint64_t h, uint64_t d, int64_t n) = 0;        // synchronous
  virtual void h2d_async(uint64_t d, uint64_t h, int64_t n) = 0;  // on the copy stream
  virtual void copies_join() = 0;      // compute stream waits for the copy stream
  virtual double copies_wait_seconds() = 0;  // host time spent waiting in copies_join so far
  virtual int64_t live_bytes() const = 0;
};

// Integrals; spin-orbital form t_kl, w_ijkl with k = 2p + sigma.
struct Integrals {
  int L = 0;
  std::vector<double> h, V;
  double ecore = 0;
  double t(int k, int l) const;
  double w(int i, int j, int k, int l) const;
  double q(int i, int j, int k, int l) const { return w(i, j, k, l) - w(i, j, l, k); }
};

struct Mat4 {
  double v[16];
  Mat4() { for (double& x : v) x = 0; }
  static Mat4 id();
  double& operator()(int i, int j) { return v[i * 4 + j]; }
  double operator()(int i, int j) const { return v[i * 4 + j]; }
  Mat4 operator*(const Mat4& o) const;
  Mat4 operator+(const Mat4& o) const;
  Mat4 operator*(double s) const;
  Mat4 T() const;
  bool zero() const;
};
Mat4 cre(int sigma);
Mat4 ann(int sigma);

// One term of an enlarged operator:
//   left  (L' = X (x) s): coef * (O_X P_X^par) (x) o
//   right (R' = s (x) Y): coef * (o P_s^par)   (x) O_Y
// src == nullptr: O is the block identity.
struct Contrib {
  const OpView* src = nullptr;
  bool srcT = false;
  Mat4 o;
  double coef = 1.0;
  bool par = false;
};

// Which side of a cut holds the two-index operators of its own modes. A block
// with normal pairs keeps A_kl = a+_k a+_l and B_kl = a+_k a_l for k, l in the
// block; a block with complementary pairs keeps P_ij and Q_il for i, j, l on
// the other side of the cut. A left block at cut c has normal pairs while
// c <= mid and a right block while c > mid, so that at every centre cut
// exactly one of the two enlarged blocks holds normal pairs; mid = L keeps
// them on the left everywhere, mid near L/2 puts them on the side with fewer
// modes (the N/2 rule of the complementary-operator method).
inline bool normal_pairs(bool left, int cut, int mid) { return left ? cut <= mid : cut > mid; }

// Enlarged block: product basis and the views of its operators.
struct Enlarged {
  bool left = true;
  bool normal = true;       // pair operators: normal (A, B) or complementary (P, Q)
  bool local = false;       // set by the caller: a right block also keeps the 16 matrix units
                            // |a><b| of each of its orbitals (F_L), for orbital density matrices
  bool batched = false;     // set by the caller: wide sums of block operators run as GEMMs
                            // over a coefficient matrix, and renormalized operators store
                            // their blocks in sector order (equal strides across operators)
  int cut = 0;              // the enlarged block covers [0, cut) or [cut, L)
  ProdBasis pb;
  std::map<Key, OpView> ops;
  std::vector<uint64_t> owned;   // materialized storage
};

// Renormalized block. Left block at cut c: sites [0, c); right: [c, L).
struct EnvBlock {
  bool left = true;
  bool normal = true;              // pair operators, as in Enlarged
  int cut = 0;
  Basis basis;
  std::map<Key, OpView> ops;
  std::vector<uint64_t> owned;     // device storage (released when evicted)
  std::vector<int64_t> owned_n;    // elements of each owned allocation
  std::vector<uint64_t> host;      // pinned host copies while evicted
  bool evicted = false;
};

// Sector rule of the initial MPS (left labels, bonds 0..L).
std::vector<std::map<QN, int>> mps_structure(int L, int N, int two_s, int D, bool su2 = false);

// Op-key list of a block at a cut with normal or complementary pairs.
std::vector<Key> block_keys(bool left, bool normal, int cut, int L);

// Build the enlarged views from a renormalized block and one site. The
// enlarged block holds normal pairs if `normal`; a block with normal pairs
// can become complementary here (the switch), the reverse is not possible.
void enlarge(const EnvBlock& B, const Integrals& I, Executor& ex, Enlarged& out, double* flops,
             bool normal);

// An operator of the enlarged block E (built from B and one site) given as a
// sum of block-operator (x) site-operator products, each in operator order
// (left: O_B O_s; right: O_s O_B) as the enlargement rules write them.
OpView product_view(const EnvBlock& B, const Integrals& I, Enlarged& E, const std::vector<Contrib>& cs, bool odd);

// Renormalize enlarged operators with the new site tensor: for each product
// sector that is kept, a dense matrix (left: [dim_prod x d_new], right:
// [d_new x dim_prod]) at device address tensor + off[prod sector].
void renormalize(const Enlarged& E, const Basis& nb, const std::vector<int>& nb_of_prod,
                 uint64_t tensor, const std::vector<int64_t>& tensor_off, Executor& ex,
                 EnvBlock& out, int64_t tmp_budget, double* flops);

// Two-site wavefunction layout: sub-blocks (x, i, j, y), sorted, row-major.
struct PsiLayout {
  struct Blk { int x, i, j, y, lsub, rsub; int64_t off; int rows, cols; };
  bool su2 = false;              // blocks couple L' and R' multiplets to total spin target.s / 2
  QN target;
  std::vector<Blk> blks;
  int nl = 0, nr = 0;            // sub-blocks of the left and right enlarged bases
  std::vector<int> by_sub;       // lsub * nr + rsub -> block index, -1: no block
  int64_t size = 0;
  int find(int lsub, int rsub) const {
    if (lsub < 0 || rsub < 0 || lsub >= nl || rsub >= nr) return -1;
    return by_sub[(size_t)lsub * nr + rsub];
  }
};
PsiLayout make_psi_layout(const ProdBasis& Lp, const ProdBasis& Rp, QN target);

// Operator-product terms of H at the centre cut: coef * L op (x) R op.
// SU(2): LT / RT select the adjoint tensor, and the pair is the scalar
// coupling [L^k x R^k]^0 of two rank-k operators (k2 = 2k).
struct CenterTerm {
  const OpView* L;
  bool LT;
  const OpView* R;
  bool RT;
  double coef;
  int k2 = 0;
};
std::vector<CenterTerm> center_terms(const Enlarged& Lp, const Enlarged& Rp, const Integrals& I);

// Diagonal of H_eff as rank-1 segments into the sigma buffer (ones: device
// vector of 1.0 at least as long as the largest sector).
Launch plan_diag(const Enlarged& Lp, const Enlarged& Rp, const PsiLayout& lay, const Integrals& I,
                 uint64_t ones);

// H_eff psi task lists (chunks of stage-1 / stage-2 launches).
struct HeffPlan {
  std::vector<Launch> stage1, stage2;
  double flops = 0;
  // algorithmic minimum traffic of one product: every operator block the terms
  // reference read once, psi read once, sigma written once (FP64 elements)
  double bytes = 0;
  int64_t tmp_elems = 0;
  int nterms = 0;
};
HeffPlan plan_heff(const Enlarged& Lp, const Enlarged& Rp, const PsiLayout& lay,
                   const Integrals& I, int64_t tmp_budget);
// Same for an arbitrary list of operator-product terms (expectation values).
HeffPlan plan_terms(const Enlarged& Lp, const Enlarged& Rp, const PsiLayout& lay,
                    const std::vector<CenterTerm>& terms, int64_t tmp_budget);
// SU(2) spin-adapted rules (rules_su2.cpp). Every block keeps c_p of its own
// orbitals, T_m of the orbitals outside it and its Hamiltonian; the pair
// operators are the normal A^k_pq, B^k_pq (p <= q) of its own orbitals or the
// complementary P^k_pq, Q^k_pq (p <= q) of the orbitals outside it, on the
// side normal_pairs() gives (as in the U(1) rules; a block with normal pairs
// can become complementary when enlarged, the reverse is not possible).
void enlarge_su2(const EnvBlock& B, const Integrals& I, Executor& ex, Enlarged& out, bool normal);
std::vector<CenterTerm> center_terms_su2(const Enlarged& Lp, const Enlarged& Rp, const Integrals& I);
// SU(2) adjoint tensor of a view whose references index sub-blocks of pb
// (enlarged) or sectors of basis (renormalized): transposed references with
// the reduced-element factor of the adjoint
OpView adjoint_su2(const OpView& o, const ProdBasis* pb, const Basis* basis);

// identity of the block part (x) a single-site operator, on an enlarged basis;
// par applies the fermion parity of the block (left) or site (right) ket part
OpView site_op_view(const Enlarged& E, const Mat4& o, bool par);

}  // namespace qd

// Sweep engine: MPS, renormalized blocks, H_eff plan, Davidson, truncation.
#pragma once
#include <climits>
#include <functional>
#include <map>
#include <stdexcept>
#include <vector>

#include "core.hpp"
#include "kernels.hpp"

namespace qd {

// A call made in a state that does not allow it (maps to QCDMRG_ESTATE).
struct StateError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

struct DavOpts {
  double tol = 1e-6;        // residual 2-norm (normalised vector), Numerical procedure section
  int max_iter = 300;
  int m_max = 32;           // subspace size before restart
  int policy = 0;           // 0: fixed precision, 1: BF16 -> BF16x3 -> FP64 correction
  int precision = 0;        // fixed precision (policy 0)
  double tau1 = 1e-2, tau2 = 1e-5;
  double floor = 1e-8;      // |diag - theta| floor of the preconditioner
};

struct DavResult {
  double energy = 0, resid = 0;
  double energy_mixed = 0;  // last Ritz value before the FP64 correction (policy 1)
  int iters = 0;
  int hpsi[4] = {0, 0, 0, 0};  // H psi products per precision
  bool converged = false;
};

struct Engine {
  Executor* ex = nullptr;
  PreparedRunner* pr = nullptr;
  Integrals I;
  int N = 0, two_s = 0, L = 0, center = -1;
  // SU(2) spin adaptation: bond labels (n, 2S) of multiplets, reduced
  // operators (rules_su2.cpp); two_s is then twice the total spin
  bool su2 = false;
  int device = 0;           // CUDA ordinal (autotuner cache key)
  int64_t tmp_budget = 0;
  // cut of the normal/complementary switch: left blocks at cuts <= pair_switch
  // and right blocks at cuts > pair_switch hold normal pairs (0: normal pairs
  // on the left at every cut)
  int pair_switch = 0;
  bool normal_at(bool left, int cut) const { return normal_pairs(left, cut, pair_switch > 0 ? pair_switch : L); }
  // wide sums of stored operators as GEMMs: 1 on, -1 off, 0 on with the switch
  // (the switching enlargement sums every pair operator of a block into each P', Q')
  int sum_gemm = 0;
  bool batched_sums() const { return sum_gemm > 0 || (sum_gemm == 0 && pair_switch > 0); }
  // MPS: bonds (left labels for b <= center, right labels for b >= center+2),
  // site tensors (product-sector matrices) for every site except the centre pair
  std::vector<Basis> bonds;
  std::vector<uint64_t> site;
  std::vector<std::vector<int64_t>> site_off;
  std::vector<std::vector<int>> site_nb;
  // renormalized blocks by cut
  std::map<int, EnvBlock> lenv, renv;
  // centre
  bool have_env = false;
  Enlarged Lp, Rp;
  PsiLayout lay;
  HeffPlan plan;
  std::vector<std::pair<int, int>> prepared;
  Launch diag_launch;
  uint64_t dpsi = 0, ddiag = 0, dones = 0;
  int64_t ones_n = 0;
  double env_flops = 0, env_seconds = 0;
  // out-of-core operator store: renormalized blocks away from the centre move
  // to pinned host memory when the device footprint exceeds hbm_budget bytes
  int64_t hbm_budget = 0;          // 0: unlimited
  int64_t h2d_bytes = 0, d2h_bytes = 0;
  int evictions = 0, restores = 0;
  // work-item shape of the bf16 tensor-core path and its autotuner
  TileCfg tcfg;
  int64_t tiled_tbudget = 0;       // T arena bytes per plane of the prepared centre (0: one pass)
  int tiled_passes = 1;
  int64_t tiled_t_plane = 0;       // bytes of one plane of the T arena in use
  int64_t tiled_t_bytes(int planes, const TiledPlan& full);   // budget for a prepared centre
  bool autotune = true;
  bool mixed_planes = false;       // prepare the three bf16 planes even for the BF16 form
  double tune_seconds = 0;
  int tunes = 0;
  void tune_tiled(uint64_t psi, uint64_t sig, int prec);
  void evict(EnvBlock& b);
  void restore_async(EnvBlock& b);  // H2D on the copy stream, references remapped
  void ensure_resident(EnvBlock& b);
  void enforce_budget();
  void enforce_budget_build(int cut, bool left);

  ~Engine() { clear(); }
  void clear();
  void clear_env();
  void free_block(EnvBlock& b);
  void free_enlarged(Enlarged& e);
  void set_psi_host(const std::vector<double>& h);
  std::vector<double> get_psi_host();

  // blocks [0, center) and [center+2, L), then the centre plan
  void build_env();
  void prepare_center();
  void heff(uint64_t psi, uint64_t sig, void* stream, int prec);
  DavResult davidson(const DavOpts& o);
  // truncate the centre to D states (drop weights <= drop_below, at least the
  // rounding floor 1e-14; a negative drop_below keeps every positive weight),
  // renormalize and move the centre by dir (+1 right, -1 left); returns the
  // discarded weight
  // eps > 0: dynamic block-state selection, the bond dimension is the smallest
  // D' in [Dmin, D] whose discarded weight (all weights beyond the D' largest)
  // is at most eps, then the selection above runs with D'; *kept (if given)
  // receives the number of states kept
  double truncate_move(int D, int dir, double drop_below, double eps = 0.0, int Dmin = 1, int* kept = nullptr);
  // <psi| sum_t c_t O_L (x) O_R |psi> for a list of centre terms
  double expect(const std::vector<CenterTerm>& terms);
  // spin-summed one-particle density matrix gamma_pq = <E_pq> of the
  // normalised state; needs the centre at (L-2, L-1)
  std::vector<double> rdm1();
  std::vector<double> rdm1_su2();   // the same for an SU(2) state (reduced operators)
  // spin-summed two-particle density matrix Gamma_pqrs = <E_pq E_rs - delta_qr E_ps>
  // of the normalised state, averaged over the 8 permutations that leave (pq|rs)
  // invariant; by exact linearity in V (one environment build per permutation
  // orbit, L^4/8 of them); the integrals and the environment are restored
  std::vector<double> rdm2();
  // the same matrix without the permutation average, every element measured
  // once while the centre walks the chain (O(L^4) single-term products at the
  // centres instead of L^4/8 environment builds); the MPS is restored
  // afterwards and its environment rebuilt
  std::vector<double> rdm2_sweep();
  // SU(2): the same by the walk of a U(1) engine holding the M = S expansion of
  // the state (its bond states are all M components of the multiplets); this
  // engine's MPS is untouched and its centre prepared again afterwards
  std::vector<double> rdm2_sweep_su2();
  // two-orbital reduced density matrices rho_ij (16 x 16 in the site basis of
  // orbitals i < j, row (x_i, y_j) = 4 x + y) of the normalised state for every
  // pair, as L*L blocks of 256 (i >= j left zero): the centre walks the chain
  // once by exact moves, right blocks keep the matrix units of their orbitals;
  // the MPS is restored afterwards. SU(2): the average over the multiplet's
  // 2S + 1 components (one walk of each component's expansion).
  bool keep_local = false;
  std::vector<double> orbital_rdm2();

  // Host copy of the MPS (centre, bases, site tensors, two-site state): the
  // walks above re-gauge the MPS and put it back exactly from one of these.
  struct MpsSnapshot {
    int center = -1;
    std::vector<Basis> bonds;
    std::vector<std::vector<int64_t>> off;
    std::vector<std::vector<int>> nb;
    std::vector<std::vector<double>> site;   // empty for the two centre sites
    std::vector<double> psi;
  };
  MpsSnapshot snapshot();
  void restore(const MpsSnapshot& s);   // uploads the tensors and rebuilds the environment
  // f run on a U(1) engine (same executor, integrals, particle number and
  // centre) that holds this SU(2) state's expansion at the component 2M = two_m
  // (M = S when two_m is the default); this engine's centre is prepared again
  // afterwards
  std::vector<double> on_m_expansion(const std::function<std::vector<double>(Engine&)>& f, int two_m = INT_MIN);
};

}  // namespace qd

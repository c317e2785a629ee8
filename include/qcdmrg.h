/*
 * qcdmrg: C ABI of the two-site DMRG H_eff.psi hot path on B300 (sm_103a).
 *
 * The method is the ab initio DMRG of arXiv 2603.28648 (Method section,
 * Eq. (mps)): a matrix product state of L spatial orbitals with the local
 * basis {|0>, |up>, |dn>, |updn>} is optimised site pair by site pair; the
 * Davidson / Lanczos sigma step H_eff psi contracts the renormalized
 * operators of the left and right blocks (normal and complementary
 * operators built from h_pq and V_pqrs) with the two-site wavefunction,
 * one quantum-number block at a time (Method and Numerical procedure
 * sections; the cost model O(N^2 D^2) memory, O(N^4 D^3) compute is the
 * Method section's).
 *
 * Conventions
 *   - Every call returns an int status: QCDMRG_OK (0) or a negative code.
 *     qcdmrg_last_error() gives the message of the last failure on a context.
 *     No C++ exception leaves a call: a failed internal consistency check
 *     returns QCDMRG_EINTERNAL.
 *   - The library owns all device memory, the operators and the MPS. Caller
 *     arrays are copied on input; output arrays are caller-allocated.
 *   - Pointers are host pointers unless the function name ends in _dev; _dev
 *     functions take device pointers and a cudaStream_t on which the work is
 *     enqueued (NULL is the CUDA legacy default stream, as everywhere in CUDA).
 *   - Dense arrays are row-major FP64. A context is not thread-safe;
 *     separate contexts are independent.
 *   - Hamiltonian: H = sum_pq h_pq E_pq + 1/2 sum_pqrs V_pqrs (E_pq E_rs -
 *     d_qr E_ps) + e_core with chemist-notation V_pqrs = (pq|rs).
 */
#ifndef QCDMRG_H
#define QCDMRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QCDMRG_OK 0
#define QCDMRG_EINVAL (-1)   /* bad argument or inconsistent input */
#define QCDMRG_ENOMEM (-2)   /* device or host allocation failed */
#define QCDMRG_ECUDA (-3)    /* CUDA runtime error */
#define QCDMRG_ESTATE (-4)   /* call out of order (e.g. apply before build_env) */
#define QCDMRG_ENOTCONV (-5) /* iteration limit reached; results are still written */
#define QCDMRG_ETIMEOUT (-6) /* a bounded device wait gave up */
#define QCDMRG_EIO (-7)      /* file error */
#define QCDMRG_EINTERNAL (-8) /* an internal consistency check of the library failed (a bug) */

/* symmetry */
#define QCDMRG_U1 0  /* U(1)xU(1): sector labels (N, 2Sz), bond dimensions count states */
#define QCDMRG_SU2 1 /* SU(2) spin adaptation (the paper's spin-adapted DMRG, Method section;
                        bond dimensions D_SU(2) count multiplets, Numerical procedure section):
                        sector labels (N, 2S), operators stored as reduced matrix elements
                        between multiplets, the target's two_s is 2S */

/* precision of the block contractions (all accumulate sigma in FP64 across
 * problems; inside one output tile the tensor-core forms accumulate in FP32) */
#define QCDMRG_FP64 0   /* FP64 FMA on CUDA cores */
#define QCDMRG_TF32 1   /* tcgen05 kind::tf32, FP32 accumulation in tensor memory */
#define QCDMRG_BF16 2   /* tcgen05 kind::f16 with bf16 inputs, FP32 accumulation */
#define QCDMRG_BF16X3 3 /* three-term bf16 split of both operands, six products, FP32 accumulation */

typedef struct qcdmrg_ctx qcdmrg_ctx;

typedef struct {
  int symmetry;         /* QCDMRG_U1 */
  int device;           /* CUDA device ordinal */
  double tmp_budget_gb; /* scratch for stage-1 intermediates (0: 2 GB) */
  double hbm_budget_gb; /* device memory for renormalized blocks before the ones away from the
                           centre move to pinned host memory (0: unlimited); the block the next
                           move needs is copied back on a second stream during the current
                           step (the host-device transfer of the paper's Unexploited power
                           section) */
  int autotune_off;     /* 1: the BF16 forms keep the default work-item shape instead of timing
                           the candidates on the first product of each problem-size class */
  int pair_switch;      /* cut of the normal/complementary switch (0: off). Left blocks at cuts
                           <= pair_switch and right blocks at cuts > pair_switch keep the normal
                           pair operators A_kl, B_kl of their own modes; the others keep the
                           complementary P_ij, Q_il of the modes across the cut. At L/2 this is
                           the N/2 rule: the pairs are stored on the side with fewer modes,
                           which halves the operator volume of a sweep environment (SU(2),
                           CAS(54,36) shape: 2.1-2.4x less environment, 3.1-3.9x fewer
                           environment-build flops). Both symmetries. A switch one cut past
                           the centre keeps the centre's complementary pairs as references
                           instead of sums. 0 keeps normal pairs on the left at every cut.
                           Negative: QCDMRG_EINVAL */
  int sum_gemm;         /* renormalization-side sums of many stored operators (the S', H', P',
                           Q' of an enlarged block): 1 runs each group of at least 8 as a GEMM of
                           a coefficient matrix with the operators' blocks, -1 sums them block
                           by block, 0 (default) takes the GEMM form when pair_switch is set */
  int tile_chunk;       /* with autotune_off = 1: chunk byte target of the BF16 forms (0: a fixed
                           K depth per chunk; 1..65536: chunks of small operand panels deepened
                           to about that many bytes). Outside 0..65536: QCDMRG_EINVAL */
} qcdmrg_config;

/*
 * MPS description for import. Bond b (0..L) separates sites [0,b) and [b,L).
 * Bonds b <= center carry the (N, 2Sz) labels of the block on their left,
 * bonds b >= center+2 those of the block on their right; bond center+1 is
 * not used (give 0 sectors). bond_nsec[b] sectors of bond b are listed in
 * bond_sec as (n, two_sz, dim) triples, bonds concatenated, labels strictly
 * increasing by (n, two_sz) inside a bond.
 *
 * Data layout (FP64, concatenated in this order):
 *   left sites p = 0 .. center-1: for each sector q of the product basis
 *     (bond p) x site, in label order, that is present in bond p+1: the
 *     matrix U_q [rows = product rows, cols = dim_q] row-major; product rows
 *     run over (x, i) pairs (x = sector of bond p, i = site state) in
 *     (x, i) order, each x contributing dim_x rows;
 *   right sites p = center+2 .. L-1: for each sector q of site x (bond p+1)
 *     in label order present in bond p: the matrix V_q [dim_q x product
 *     cols], product columns over (j, y) pairs in (j, y) order;
 *   the two-site wavefunction: sub-blocks (x, i, j, y) with x a sector of
 *     bond center, y a sector of bond center+2, labels adding up to the
 *     target, sorted by (x, i, j, y); each sub-block dim_x x dim_y row-major.
 * Site states: 0 = |0>, 1 = a+_up|0>, 2 = a+_dn|0>, 3 = a+_up a+_dn|0>.
 */
typedef struct {
  int L;
  int center; /* two-site centre: sites (center, center+1) */
  const int* bond_nsec;
  const int* bond_sec;
} qcdmrg_mps_desc;

typedef struct {
  double heff_flops;     /* algorithmic 2mnk of one H_eff psi (all block GEMMs) */
  double heff_seconds;   /* device time of the last H_eff psi */
  double env_flops;      /* flops of the last environment build */
  double env_seconds;    /* wall time of the last environment build */
  int64_t psi_size;      /* elements of the two-site wavefunction */
  int64_t device_bytes;  /* peak bytes allocated on the device by the context */
  int64_t live_bytes;    /* bytes allocated on the device by the context now */
  int nterms;            /* operator-product terms of H_eff */
  int nlaunch;           /* kernel launches per H_eff psi */
  int64_t h2d_bytes;     /* out-of-core store: bytes copied back to the device */
  int64_t d2h_bytes;     /* bytes moved to pinned host memory */
  int evictions, restores;
  double copy_wait_seconds; /* host time the compute stream waited for copies */
  double heff_bytes;     /* algorithmic minimum traffic of one H_eff psi: every operator block
                            it references read once, psi read once, sigma written once (FP64) */
  int tile_kmax;         /* work-item shape of the BF16 forms in use: summed K per stage-2 item */
  int tile_width;        /* and accumulator columns per stage-1 item */
  int tunes;             /* autotuner runs of this context */
  double tune_seconds;   /* wall time spent in them */
  int64_t f64_tiles[4];  /* FP64 form of H_eff psi: work items (tiles) per tile shape 64x64, 64x32,
                            32x64, 32x32 over the prepared task lists of the current centre */
  int64_t f64_split_tiles; /* of those, tiles of problems whose summed K exceeds one work item
                            (split over several tiles that add with FP64 atomics) */
  int dav_hpsi[4];       /* last qcdmrg_davidson call: H psi products per precision (FP64, TF32,
                            BF16, BF16x3) */
  double dav_seconds;    /* its wall time */
  double dav_energy_mixed; /* its last Ritz value before the FP64 correction (policy 1) */
  int tile_chunk;        /* chunk byte target of the BF16 forms in use (0: fixed K depth) */
  int tile_passes;       /* passes of the BF16 forms' stage-1 intermediates: 1 when every T_t
                            of the product fits the device next to the operand mirrors,
                            more when they are split (QCDMRG_TILED_T_BYTES in the environment
                            sets the bytes of one pass's plane instead) */
  int64_t tile_t_bytes;  /* bytes of one plane of the T arena in use */
} qcdmrg_stats_t;

/* Davidson options (zero fields take the defaults in brackets). */
typedef struct {
  double tol;     /* residual 2-norm of the normalised vector [1e-6, the paper's Lanczos
                     residual, Numerical procedure section] */
  int max_iter;   /* [300] */
  int m_max;      /* subspace size before a restart [32] */
  int policy;     /* 0: every H psi in `precision`; 1: mixed precision with FP64 residual
                     correction: BF16 H psi while the residual is above tau1, BF16x3 while
                     above tau2 (a phase also ends at its rounding floor, 2^-6 |E| for BF16
                     and 2^-14 |E| for BF16x3, or when its residual has not fallen by 10 % in
                     8 iterations), then outer checks: one FP64 H psi of the normalised Ritz
                     vector gives the energy and the residual; if the residual is above tol,
                     that exact pair restarts the subspace and BF16x3 products expand it
                     until the residual has fallen 30-fold (or m_max - 2 products), then the
                     next check. The final energy and residual are always from an FP64
                     product */
  int precision;  /* QCDMRG_FP64 / _TF32 / _BF16 / _BF16X3 for policy 0 */
  double tau1;    /* [1e-2] */
  double tau2;    /* [1e-5] */
} qcdmrg_dav_opts;

typedef struct {
  int D;                 /* bond dimension kept by every truncation (U(1) states, SU(2)
                            multiplets); with trunc_eps > 0 the largest one */
  qcdmrg_dav_opts dav;
  double trunc_eps;      /* > 0: dynamic block-state selection, each truncation keeps the
                            smallest bond dimension in [D_min, D] whose discarded weight is at
                            most trunc_eps (the fixed-truncation-error alternative the paper's
                            Numerical procedure section mentions); 0: fixed D */
  int D_min;             /* smallest bond dimension of the dynamic selection */
} qcdmrg_sweep_opts;

typedef struct {
  double energy;         /* energy of the last optimisation of the sweep */
  double energy_mixed;   /* last Ritz value before the FP64 correction (policy 1) */
  double max_trunc_err;  /* largest discarded weight of the sweep */
  double seconds;        /* wall time of the sweep */
  int n_hpsi[4];         /* H psi products per precision (FP64, TF32, BF16, BF16x3) */
  int n_steps;           /* two-site optimisations (2L-4) */
  int max_D;             /* largest bond dimension kept by the sweep's truncations */
} qcdmrg_sweep_report;

/* Create a context on cfg->device: one solver of the paper's spin-adapted DMRG
 * (Method section) on one GPU (Hardware specific implementations section).
 * *out receives the handle (owned by the caller, released by
 * qcdmrg_destroy). Errors: EINVAL (unknown symmetry, negative budgets,
 * pair_switch < 0, sum_gemm outside -1..1, an SU(2) context with
 * pair_switch; checked before any CUDA call), ECUDA, ENOMEM. */
int qcdmrg_create(qcdmrg_ctx** out, const qcdmrg_config* cfg);
int qcdmrg_destroy(qcdmrg_ctx* ctx);
/* Message of the last failed call (empty if none); owned by the context. */
const char* qcdmrg_last_error(const qcdmrg_ctx* ctx);

/*
 * Load the active-space integrals: h (L*L) and V (L^4, (pq|rs) at
 * ((p*L+q)*L+r)*L+s), the one- and two-electron integrals of the model
 * Hamiltonian of the Method section over the L orbitals of the active space
 * (CAS(54,36): L = 36, Model system section). The arrays are copied.
 * Errors: EINVAL for L < 2, non-finite values or a non-symmetric h.
 */
int qcdmrg_load_integrals(qcdmrg_ctx* ctx, int L, const double* h, const double* V,
                          double e_core);

/* Target particle number N and two_s: 2S for QCDMRG_SU2 (the spin of the
 * multiplet, S = 0 for the CAS(54,36) ground state of the Model system
 * section), 2Sz for QCDMRG_U1. Errors: EINVAL on parity mismatch, a negative
 * 2S, or a target outside the Fock space of the loaded L. */
int qcdmrg_set_target(qcdmrg_ctx* ctx, int N, int two_s);

/*
 * Import a mixed-canonical MPS (Eq. (mps) of the Method section) around a
 * two-site centre (layout above). The tensors must be canonical (left tensors U_q with orthonormal columns,
 * right tensors V_q with orthonormal rows); they are copied to the device.
 * n is the number of doubles in data. Errors: EINVAL (layout mismatch),
 * ESTATE (integrals or target missing).
 */
int qcdmrg_import_mps(qcdmrg_ctx* ctx, const qcdmrg_mps_desc* desc, const double* data,
                      size_t n);

/*
 * Random initial MPS at bond dimension D around the centre (center,
 * center+1): sector dimensions from the sector rule (block-state counts,
 * Gaussian weights around N b / L and Sz = 0, water filling with caps), i.i.d.
 * normal entries from a counter-based generator (splitmix64 of seed and
 * element index, Box-Muller), each product-sector matrix made orthonormal by
 * QR on the device, and a normalised random two-site wavefunction. Errors:
 * ESTATE (integrals or target missing), EINVAL.
 */
int qcdmrg_init_mps(qcdmrg_ctx* ctx, int D, uint64_t seed, int center);

/*
 * Copy the current MPS out in the layout qcdmrg_import_mps reads (after sweeps
 * and centre moves too): *L, *center, bond_nsec (L+1 ints; bond center+1 has
 * no sectors), bond_sec ((n, two_sz, dim) triples, *n_sec of them), data (the
 * left site tensors U_q [(x, i) rows, kept states], the right site tensors V_q
 * [kept states, (j, y) columns], each site's product sectors in label order,
 * then the two-site wavefunction; *n_data doubles). Every output pointer may
 * be NULL; call once with bond_sec and data NULL to learn *n_sec and *n_data.
 * The MPS of the paper's Method section (Eq. (mps)) around its two-site
 * centre; no counterpart of the file format in the paper. Errors: ESTATE (no
 * MPS), EINVAL (a buffer shorter than needed: sec_cap ints, cap doubles).
 */
int qcdmrg_export_mps(qcdmrg_ctx* ctx, int* L, int* center, int* bond_nsec, int* bond_sec, int sec_cap,
                      double* data, size_t cap, int* n_sec, size_t* n_data);

/*
 * Checkpoint: write the integrals, the target and the MPS (export layout) to
 * a binary file (magic "QCDMRGC1", seven int64 sizes, e_core, h, V, bond
 * sector counts and triples, data; native byte order). Restore: read such a
 * file into a context, replacing its integrals, target and MPS; call
 * qcdmrg_build_env afterwards. Errors: EIO (open, short read or write, not a
 * checkpoint), ESTATE (checkpoint without integrals or target), and those of
 * qcdmrg_load_integrals / qcdmrg_import_mps on restore.
 */
int qcdmrg_checkpoint(qcdmrg_ctx* ctx, const char* path);
int qcdmrg_restore(qcdmrg_ctx* ctx, const char* path);

/* Sectors of bond b of the current MPS as (n, two_sz, dim) triples; sec may be
 * NULL to query *nsec only; cap is the length of sec in ints. */
int qcdmrg_get_bond(const qcdmrg_ctx* ctx, int bond, int* nsec, int* sec, int cap);

/* Copy the current two-site wavefunction (n = its size). */
int qcdmrg_get_psi(const qcdmrg_ctx* ctx, double* out, size_t n);

/* Replace the current two-site wavefunction (n = its size, host array). */
int qcdmrg_set_psi(qcdmrg_ctx* ctx, const double* psi, size_t n);

/*
 * Renormalize the left block up to the centre and the right block down to
 * it (the operator renormalization of every truncation step, replayed for
 * the imported tensors), enlarge both by their dot site and build the
 * H_eff task list. These renormalized operators are the O(N^2 D^2) memory of
 * the Method section's cost model. Renormalization has no entry point of its
 * own: this call runs it from both ends, and qcdmrg_truncate runs it for the
 * grown block of each step. Errors: ESTATE (no MPS), ECUDA, ENOMEM.
 */
int qcdmrg_build_env(qcdmrg_ctx* ctx);

/* Number of elements of the two-site wavefunction (after build_env). */
int qcdmrg_psi_size(const qcdmrg_ctx* ctx, size_t* n);

/*
 * Block layout of the two-site wavefunction psi[x, i, j, y] (the flat order of
 * every psi and sigma array of this interface): for each sub-block, in order,
 * 8 ints (x n, x two_sz, i, j, y n, y two_sz, rows = dim x, cols = dim y);
 * sub-blocks follow each other, each rows x cols row-major. blocks may be NULL
 * to query *nblocks and *nelem only; cap is its length in ints. The centre of
 * the MPS of the paper's Method section (Eq. (mps)). Errors: ESTATE, EINVAL.
 */
int qcdmrg_psi_layout(const qcdmrg_ctx* ctx, int* blocks, int cap, int* nblocks, size_t* nelem);

/*
 * Energy of the current two-site wavefunction at fixed MPS and its gradients
 * (host arrays, any of them NULL to skip): E = <psi|H_eff|psi>/<psi|psi> (FP64
 * product), dpsi = dE/dpsi = 2 (H_eff psi - E psi)/<psi|psi> (psi size),
 * gamma1 = dE/dh (L*L, as qcdmrg_rdm1: needs the centre at (L-2, L-1)),
 * gamma2 = 2 dE/dV for 8-fold symmetric V (L^4, as qcdmrg_rdm2: L^4/8
 * environment builds, for L <= 10; beyond, the permutation average of
 * qcdmrg_rdm2_sweep; either symmetry). The derivatives the paper's DMRG-SCF needs (New
 * benchmark system section). Errors: ESTATE, EINVAL, ENOMEM, ECUDA.
 */
int qcdmrg_energy_grad(qcdmrg_ctx* ctx, double* energy, double* dpsi, double* gamma1, double* gamma2);

/*
 * sigma = H_eff psi on host arrays of psi_size elements (layout above): the
 * sigma step of the iterative diagonalization (Numerical procedure section),
 * whose block contractions are the O(N^4 D^3) compute of the Method section's
 * cost model and the FLOP rate of the Numerical results. precision: one of
 * QCDMRG_FP64, _TF32, _BF16, _BF16X3 (the mixed-precision forms stand where
 * the paper emulates FP64 on tensor cores, Hardware specific implementations
 * section). The copies between host and device are part of the call. Errors:
 * ESTATE (no environment), EINVAL, ETIMEOUT (a bounded wait of a tensor-core
 * kernel gave up; sigma is then not valid).
 */
int qcdmrg_apply_heff(qcdmrg_ctx* ctx, int precision, const double* psi, double* sigma);

/* Same on device arrays, enqueued on stream (a cudaStream_t; NULL is the
 * legacy default stream); returns after enqueueing. psi and sigma must not
 * overlap and must stay alive until the stream reaches the work. A bounded
 * device wait that gave up is reported by qcdmrg_check_device. */
int qcdmrg_apply_heff_dev(qcdmrg_ctx* ctx, int precision, const void* psi, void* sigma,
                          void* stream);

/*
 * No counterpart in the paper: an H_eff psi that allocates nothing, for
 * callers that cannot allocate device memory when they need the product
 * (work being captured into a CUDA graph, a GPU whose free memory is held by
 * another framework's caching allocator, solvers with a fixed memory budget).
 * FP64 form only. The stage-1 intermediates go to a fixed 32 MiB device array
 * (QCDMRG_NOALLOC_SCRATCH_DOUBLES doubles) compiled into the library, which
 * every GPU that loads the library holds until exit; a problem whose
 * intermediates need more is rejected with QCDMRG_EINVAL (a smaller
 * tmp_budget_gb at qcdmrg_create makes the chunks fit). The first call on a
 * device looks up the array's address with that device current; make that
 * first call before any stream capture. All calls share the array and it
 * keeps the last call's contents: calls whose work overlaps on the GPU race.
 * psi, sigma: device arrays of psi_size doubles; stream: cudaStream_t (NULL is
 * the legacy default stream). The call makes the context's device current
 * while it enqueues and restores the caller's current device before it
 * returns; a launch error left pending by earlier work on the calling thread
 * is cleared first, so that ECUDA always reports this call's own launches.
 * Errors: ESTATE, EINVAL, ECUDA.
 */
#define QCDMRG_NOALLOC_SCRATCH_DOUBLES (4 * 1024 * 1024)
int qcdmrg_apply_heff_noalloc(qcdmrg_ctx* ctx, const void* psi, void* sigma, void* stream);

/*
 * Spin-summed one-particle density matrix gamma_pq = <Psi|E_pq|Psi>/<Psi|Psi>
 * (L*L row-major) of the current MPS state, which is the gradient dE/dh_pq of
 * the energy at fixed wavefunction (the 1-RDM CASSCF orbital optimisation
 * needs, DMRG-SCF of the paper's New benchmark system section). Measured with
 * the stored operators at the centre (L-2, L-1), where the left enlarged
 * block holds a+_k a_l for every orbital but the last: move the centre there
 * first (qcdmrg_move_center(ctx, L-2)). With pair_switch set, the blocks at
 * that centre hold complementary pairs on the left; the call then rebuilds the
 * environment with normal pairs on the left, measures, and rebuilds the
 * switched environment (two environment builds; the MPS is unchanged).
 * Errors: ESTATE.
 */
int qcdmrg_rdm1(qcdmrg_ctx* ctx, double* gamma);

/*
 * Spin-summed two-particle density matrix of the current MPS state,
 *   Gamma_pqrs = <Psi|E_pq E_rs - delta_qr E_ps|Psi> / <Psi|Psi>
 * (L^4 row-major, caller-allocated), averaged over the 8 index permutations
 * that leave a chemist-notation integral (pq|rs) invariant. With the
 * Hamiltonian's 1/2 sum V_pqrs (E_pq E_rs - delta_qr E_ps), 1/2 Gamma is the
 * gradient dE/dV at fixed wavefunction for an 8-fold symmetric V, the 2-RDM
 * CASSCF orbital optimisation needs (DMRG-SCF of the paper's New benchmark
 * system section). Computed by exact linearity in V: for each permutation
 * orbit the environment is rebuilt with h = 0 and unit integrals on that
 * orbit, and <H_eff> at the centre gives half the orbit's sum of Gamma; that
 * is L^4/8 environment builds, meant for small active spaces. Any centre,
 * either symmetry (with QCDMRG_SU2 the spin-free Gamma of the multiplet).
 * The context's integrals and environment are restored before returning.
 * Errors: ESTATE (no environment), EINVAL, ENOMEM, ECUDA.
 */
int qcdmrg_rdm2(qcdmrg_ctx* ctx, double* gamma2);

/*
 * The same two-particle density matrix element by element, without the
 * permutation average: Gamma_pqrs = sum over spins s, t of
 * <a+_{p,s} a+_{r,t} a_{s,t} a_{q,s}> / <Psi|Psi> (orbital indices p, q, r, s;
 * L^4 row-major, caller-allocated). Each element is measured once, at the
 * centre (o3 - 1, o3) for its sorted orbitals o1 <= o2 <= o3 <= o4 (o3 >= 1),
 * where at most two of its operators fall on the left block (stored a+, A, B
 * operators), any number on the two sites and at most one on the right block:
 * O(L^4) single-term products at the centres instead of L^4/8 environment
 * builds, so that active spaces of the paper's size are in reach. The centre
 * walks the chain once by exact moves (every state above the rounding noise of
 * its sector's density-matrix eigenvalues is kept); afterwards the MPS (site
 * tensors, bonds, psi at its centre) is restored as it was and the environment
 * rebuilt once. With QCDMRG_SU2 the walk runs on the state's M = S expansion (the
 * same state as a U(1) MPS whose bond states are all M components of the
 * multiplets, about 2-3 times as many states), in a temporary U(1) engine; the
 * SU(2) context is unchanged and its centre prepared again afterwards. With
 * pair_switch set, the environment is rebuilt with normal pairs on the left
 * for the walk and the switched one restored afterwards.
 * Errors: ESTATE (no environment), EINVAL, ENOMEM, ECUDA.
 */
int qcdmrg_rdm2_sweep(qcdmrg_ctx* ctx, double* gamma2);

/* Diagonal of H_eff at the centre (psi layout, n = psi size), as used by the
 * Davidson preconditioner: sum over terms of c_t diag(O_L) (x) diag(O_R)
 * restricted to diagonal quantum-number blocks. The paper names Lanczos
 * (Numerical procedure section), which needs no preconditioner: this call has
 * no counterpart there. Errors: ESTATE, EINVAL (n differs from the psi size). */
int qcdmrg_heff_diag(qcdmrg_ctx* ctx, double* out, size_t n);

/*
 * Davidson solve of the two-site problem at the centre (FP64 vectors, FP64
 * Gram-Schmidt and subspace eigenproblem; H psi in the precision the policy
 * selects), starting from the current wavefunction; the converged Ritz vector
 * replaces it. The iterative diagonalization of the Numerical procedure
 * section (residual 1e-6); its mixed policy stands for the emulated FP64 of
 * the Mixed precision and hardware section, with the final energy from an
 * FP64 product. Preconditioner (diag(H_eff) - theta)^-1 with |.| floored at
 * 1e-8; restart keeps the Ritz vector. Any pointer may be NULL. Errors:
 * ESTATE, ENOTCONV (results still written), ETIMEOUT.
 */
int qcdmrg_davidson(qcdmrg_ctx* ctx, const qcdmrg_dav_opts* opts, double* energy, double* resid,
                    int* iters);

/*
 * Truncation step of the sweep (the truncation error of the Method section:
 * the discarded Schmidt weight; D fixed per run as in the Numerical
 * procedure section, counted in multiplets for QCDMRG_SU2): density matrix of the two-site wavefunction
 * per quantum-number sector (rho = Psi Psi^T for dir = +1, Psi^T Psi for
 * dir = -1), FP64 eigendecomposition, the D states of largest weight kept
 * across sectors (ties: weight, then label, then in-sector order; weights
 * equal to 1e-8 relative that straddle the cut are dropped together, and
 * weights <= 1e-14, rounding noise of the eigenvalues, are always dropped), new site
 * tensor, renormalization of every operator of the grown block, and the
 * transformed wavefunction as the guess at the moved centre. trunc_err gets
 * the discarded weight. Errors: ESTATE, EINVAL.
 */
int qcdmrg_truncate(qcdmrg_ctx* ctx, int D, int dir, double* trunc_err);

/*
 * Truncation step with dynamic block-state selection: the bond dimension is
 * the smallest D in [D_min, D_max] whose discarded weight (the sum of all
 * density-matrix weights beyond the D largest) is at most eps, after which the
 * selection of qcdmrg_truncate runs with that D (a group of weights tied at the
 * cut is dropped as a whole, which can leave the discarded weight a little
 * above eps). The fixed-truncation-error alternative to a fixed D that the
 * paper's Numerical procedure section mentions. *kept receives the number of
 * states (SU(2): multiplets) kept; trunc_err and kept may be NULL. Errors:
 * ESTATE, EINVAL (1 <= D_min <= D_max, eps > 0, dir +1 or -1, a move off the
 * chain).
 */
int qcdmrg_truncate_dbss(qcdmrg_ctx* ctx, int D_min, int D_max, double eps, int dir, double* trunc_err,
                         int* kept);

/*
 * Extrapolation of energies to the truncation-free limit: the least-squares
 * polynomial E(x) = coef[0] + coef[1] x + ... + coef[degree] x^degree (degree
 * 1..3) through n points (x[i], energy[i]); coef[0] is the extrapolated energy.
 * The paper's Numerical benchmark section extrapolates its fixed-D series in
 * two ways: a second-order polynomial in x = 1/D, and the energy against the
 * largest truncation error of the last sweep (x = that error; the fit's form is
 * not stated there, degree 1 is the usual choice). Host arrays, coef holds
 * degree + 1 doubles. No context, no device. Errors: EINVAL (degree outside
 * 1..3, n < degree + 1, NULL arrays, non-finite values, points that do not fix
 * the polynomial).
 */
int qcdmrg_extrapolate(const double* x, const double* energy, int n, int degree, double* coef);

/*
 * DMRG-SCF orbital step, host arrays, no context and no device (the paper's
 * CAS-SCF orbital optimisation around its DMRG, New benchmark system section).
 * n orbitals: core 0..ncore-1 doubly occupied, active ncore..ncore+nact-1 (the
 * DMRG active space, in chain order), virtual the rest; h n*n, V n^4 as in
 * qcdmrg_load_integrals. Errors: EINVAL (sizes, NULL arrays).
 *
 * qcdmrg_active_space: the frozen-core energy e_core = sum_c 2 h_cc +
 * sum_cd (2 (cc|dd) - (cd|dc)), the active one-electron integrals h_act
 * (nact*nact) = h_tu + sum_c (2 (tu|cc) - (tc|cu)) and V_act (nact^4) = (tu|vw),
 * ready for qcdmrg_load_integrals(ctx, nact, h_act, V_act, e_core).
 *
 * qcdmrg_orbital_gradient: grad (n*n, antisymmetric) = dE/dkappa_pq of
 * E = e_core + sum h_act gamma1 + 1/2 sum V_act gamma2 at fixed density matrices
 * (gamma1 nact*nact as qcdmrg_rdm1, gamma2 nact^4 as qcdmrg_rdm2) when the
 * orbitals rotate as the columns of exp(kappa), one parameter per pair p > q;
 * grad = 2 (F - F^T) with the generalised Fock matrix F.
 *
 * qcdmrg_rotate_orbitals: U = exp(kappa) for an antisymmetric kappa (n*n; EINVAL
 * otherwise), h_out = U^T h U, V_out = (pq|rs) in the rotated orbitals; U may be
 * NULL. A steepest-descent step is kappa = -step * grad.
 */
int qcdmrg_active_space(int n, int ncore, int nact, const double* h, const double* V, double* e_core,
                        double* h_act, double* V_act);
int qcdmrg_orbital_gradient(int n, int ncore, int nact, const double* h, const double* V, const double* gamma1,
                            const double* gamma2, double* grad);
int qcdmrg_rotate_orbitals(int n, const double* kappa, const double* h, const double* V, double* U, double* h_out,
                           double* V_out);
/*
 * qcdmrg_orbital_hessian_diag (host only): hdiag (n*n, symmetric, zero
 * diagonal) = d^2 E / d kappa_pq^2 at kappa = 0 for the one-pair rotation
 * exp(kappa_pq (e_pq - e_qp)), E and the arguments as qcdmrg_orbital_gradient.
 * Along that rotation E is a trigonometric polynomial of degree 4, so nine
 * samples give the value exactly (no finite-difference error); O(n^3 + nact^4)
 * per sample. With the gradient it gives the diagonal-Newton step
 * kappa_pq = -grad_pq / hdiag_pq where hdiag_pq > 0. Errors: EINVAL.
 */
int qcdmrg_orbital_hessian_diag(int n, int ncore, int nact, const double* h, const double* V, const double* gamma1,
                                const double* gamma2, double* hdiag);

/*
 * Orbital entanglement for the chain ordering: the paper pre-optimises its
 * chain topology with the quantum-information protocols of Barcza et al.
 * (2011) and Szalay et al. (2015) (Numerical procedure section).
 *
 * qcdmrg_orbital_rdm: the two-orbital reduced density matrices rho_ij of the
 * normalised state, the partial trace of |Psi><Psi| over every orbital other
 * than i and j, with the creation operators of orbitals i and j moved to the
 * front of each determinant (sign of that reordering included). rho: host
 * array of L*L*256 doubles, block (i, j) at (i*L + j)*256 for i < j, a
 * row-major 16 x 16 matrix with row (and column) 4 x + y, x the state of
 * orbital i and y that of orbital j (0 empty, 1 up, 2 down, 3 a+_up a+_dn|0>);
 * blocks with i >= j are written as zeros. QCDMRG_SU2: the average over the
 * multiplet's 2S + 1 components (one component's rho_ij depends on M when
 * S > 0; the average does not), one walk per component. The centre walks the
 * chain once from bond 0 by exact moves (no
 * truncation) and every right block holds the 16 matrix units of each of its
 * orbitals (16 (L - p) extra operators in the block at site p); the MPS, its
 * centre and the environment are restored afterwards. Errors: ESTATE (no
 * environment), EINVAL (NULL), ENOMEM, ECUDA.
 *
 * qcdmrg_orbital_entanglement (host only, no context): from those blocks,
 * s1[i] = -Tr rho_i ln rho_i (rho_i = Tr_j rho_ij from the pair (i, i+1), or
 * (i-1, i) for the last orbital; s1 may be NULL) and mutual (L*L, symmetric,
 * zero diagonal) I_ij = s1[i] + s1[j] + Tr rho_ij ln rho_ij. Eigenvalues at or
 * below zero add nothing. Errors: EINVAL (L < 2, NULL rho or mutual,
 * non-finite entries).
 *
 * qcdmrg_fiedler_order (host only): order (L, a permutation of 0..L-1) sorts
 * the orbitals by their component of the Fiedler vector (eigenvector of the
 * second smallest eigenvalue) of the Laplacian diag(sum_j I_ij) - I; ties keep
 * index order. fiedler (L, may be NULL) gets the vector, unit length, its first
 * component of magnitude above 1e-8 of the largest made negative. When the
 * second eigenvalue is degenerate (a mutual-information graph in several
 * disconnected parts, or a symmetric one) the vector is one of several and so
 * is the order. Reordering the integrals as h[order][order], V likewise, puts
 * strongly entangled orbitals next to each other on the chain. Errors: EINVAL
 * (L < 2, NULL, mutual not symmetric to 1e-12 or not finite).
 */
int qcdmrg_orbital_rdm(qcdmrg_ctx* ctx, double* rho);
int qcdmrg_orbital_entanglement(int L, const double* rho, double* s1, double* mutual);
int qcdmrg_fiedler_order(int L, const double* mutual, int* order, double* fiedler);

/*
 * qcdmrg_ordering_cost (host only): *cost = sum_{i<j} mutual_ij |pos_i - pos_j|^eta
 * with pos_i the position of orbital i in order (order[k] = the orbital at
 * position k, a permutation of 0..L-1): the distance cost of entangled orbitals
 * along the chain of Barcza et al. (2011); the Fiedler vector minimises its
 * eta = 2 form relaxed to real positions.
 * qcdmrg_refine_order (host only): order improved in place by exchanging the
 * positions of two orbitals, the best exchange first, while one lowers the cost
 * (at most max_swaps exchanges); *swaps (may be NULL) gets the number made.
 * Errors: EINVAL (L < 2, NULL, order not a permutation, eta not finite or <= 0,
 * mutual not symmetric to 1e-12 or not finite, max_swaps < 0).
 */
int qcdmrg_ordering_cost(int L, const double* mutual, const int* order, double eta, double* cost);
int qcdmrg_refine_order(int L, const double* mutual, double eta, int* order, int max_swaps, int* swaps);

/*
 * Configuration-space warm start: the paper converges its runs with an
 * SU(2)-aware dynamically extended active space procedure (SU(2)-DEAS, Legeza
 * et al. 2003; Numerical benchmark section), whose warm-up sweep takes the
 * environment of each step from a small configuration space rather than from
 * a previous sweep. Here: select configurations, write them as an MPS whose
 * left bond bases are exactly their prefixes (centre at the right end), import
 * it, and run one right-to-left half sweep before the full sweeps.
 *
 * Configurations are step vectors of L bytes in chain order, the site-state
 * indices of the import layout: U(1) 0 = |0>, 1 = a+_up|0>, 2 = a+_dn|0>,
 * 3 = a+_up a+_dn|0> (a determinant); QCDMRG_SU2 0 = empty, 1 = singly
 * occupied raising the spin of the orbitals so far by 1/2, 2 = singly occupied
 * lowering it by 1/2, 3 = doubly occupied (a configuration state function in
 * the left-to-right, genealogical coupling; the spin so far never negative).
 *
 * qcdmrg_select_configs (host only): up to nmax configurations of the target
 * (N, two_s) ranked by energy, from the aufbau reference (U(1): the orbitals of
 * lowest h_pp filled with (N + two_s)/2 up and (N - two_s)/2 down electrons;
 * SU(2): (N - two_s)/2 doubly occupied, the next two_s singly occupied with
 * all steps up) and every configuration at most two electrons away from it
 * (SU(2): spatial occupations, each with all of its couplings). Energy: U(1)
 * <D|H|D>; SU(2) the average of <D|H|D> over the determinants of the spatial
 * occupation (e_core excluded). Ties: fewer electrons moved, then the step
 * vector in lexicographic order. steps: nmax * L bytes, energy: nmax doubles
 * (may be NULL), *count: configurations written. Errors: EINVAL (L < 2,
 * nmax < 1, NULL, a target outside the Fock space).
 *
 * qcdmrg_config_mps (host only): the import description (qcdmrg_import_mps)
 * of the MPS sum_k coef[k] |config_k> with centre L-2: bond b <= L-2 holds one
 * state per distinct prefix of length b, the left site tensors are 0/1
 * selectors, the two-site wavefunction holds the coefficients (repeated
 * configurations add); bond L-1 has no sectors, bond L is the vacuum. Sizes
 * as for qcdmrg_export_mps: call with NULL bond_sec and data to get *n_sec
 * (triples) and *n_data; bond_nsec takes L+1 ints, sec_cap counts ints (3 per
 * triple), cap doubles. Errors: EINVAL (steps outside 0..3, a configuration
 * outside the target or with a negative SU(2) spin, all coefficients zero,
 * buffers too small).
 *
 * qcdmrg_sweep_left: from the current centre, one Davidson solve and one
 * truncation (as in qcdmrg_sweep) per step, moving left until the centre is
 * at sites (0, 1); no exact move first. After an import of qcdmrg_config_mps
 * this is the warm-up half sweep: each step's left block is the span of the
 * configurations' prefixes. report->n_steps = the steps taken. Errors: as
 * qcdmrg_sweep.
 */
int qcdmrg_select_configs(int symmetry, int L, int N, int two_s, const double* h, const double* V, int nmax,
                          uint8_t* steps, double* energy, int* count);
int qcdmrg_config_mps(int symmetry, int L, int N, int two_s, int n, const uint8_t* steps, const double* coef,
                      int* center, int* bond_nsec, int* bond_sec, int sec_cap, double* data, size_t cap,
                      int* n_sec, size_t* n_data);
int qcdmrg_sweep_left(qcdmrg_ctx* ctx, const qcdmrg_sweep_opts* opts, qcdmrg_sweep_report* report);

/* Move the centre to sites (target, target+1) without truncation (only
 * weights <= 1e-14, rounding noise, dropped), renormalizing each grown
 * block (Method section). Errors: ESTATE, EINVAL (target outside 0..L-2). */
int qcdmrg_move_center(qcdmrg_ctx* ctx, int target);

/*
 * One full sweep of the Numerical procedure section (the paper sweeps until
 * the energy of three sweeps agrees to 1e-5; the caller repeats this call):
 * the centre is first moved (exactly) to sites (0, 1), then
 * optimised and moved right to (L-2, L-1), then back to (0, 1): 2L-4 two-site
 * optimisations, each a Davidson solve followed by qcdmrg_truncate. Errors:
 * ESTATE, EINVAL, ENOTCONV (a Davidson solve hit max_iter; the sweep completes).
 */
int qcdmrg_sweep(qcdmrg_ctx* ctx, const qcdmrg_sweep_opts* opts, qcdmrg_sweep_report* report);

/* Reads and clears the device error flag of the tensor-core kernels after
 * _dev calls (synchronous). Errors: ETIMEOUT if a bounded wait gave up. */
int qcdmrg_check_device(qcdmrg_ctx* ctx);

/*
 * Batched H_eff psi in one CUDA graph: all quantum-number blocks of one or
 * several independent H_eff psi products in one replay, instead of one
 * product after another. The paper runs one problem at a time and names no
 * batching; this is the launch-side form of its GPU-accelerated sigma step
 * (Hardware specific implementations section). The H_eff psi of each context (memset of sigma plus its
 * grouped-GEMM launches) is captured once, contexts as parallel branches,
 * with psi[i] and sigma[i] (device arrays of each context's psi size) baked
 * into the graph; qcdmrg_graph_launch replays it on a stream. The contexts'
 * environments must stay unchanged while the graph is used (build_env,
 * truncate or sweep invalidate it). All contexts on one device. Errors:
 * EINVAL, ESTATE (a context without environment), ECUDA (message in the first
 * context).
 */
typedef struct qcdmrg_graph qcdmrg_graph;
int qcdmrg_graph_create(qcdmrg_ctx* const* ctxs, int n, int precision, const void* const* psi,
                        void* const* sigma, qcdmrg_graph** out);
int qcdmrg_graph_launch(qcdmrg_graph* graph, void* stream);
/* Algorithmic flops of one replay and number of graph nodes. */
int qcdmrg_graph_info(const qcdmrg_graph* graph, double* flops, int* nodes);
int qcdmrg_graph_destroy(qcdmrg_graph* graph);

/* Counters of the last calls (flop counts, device times, bytes): the FLOP
 * rate and wall times the Numerical results section reports. */
int qcdmrg_stats(const qcdmrg_ctx* ctx, qcdmrg_stats_t* out);

#ifdef __cplusplus
}
#endif
#endif

// CUDA backend: device memory, task-list upload and the FP64 segmented
// grouped GEMM that executes every block contraction of H_eff psi,
// renormalization and complementary-operator materialization.
//
// One launch runs a list of output problems; problem p owns C_p (m x n) and
// computes C_p = beta*C_p + sum_s sc_s op(A_s) op(B_s) over its segments.
// Identity segments (A = I, or A = B = I) implement gather-AXPY. Each CTA
// owns one 64x64 output tile and loops over all segments of its problem, so
// no output is written by two CTAs and no atomics are needed.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdio>
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "core.hpp"
#include "kernels.hpp"
#include "tc_gemm.hpp"
#include "tc_tiled.hpp"

namespace qd {

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess)                                                         \
      throw std::runtime_error(std::string("CUDA: ") + cudaGetErrorString(e_) +    \
                               " at " + __FILE__ + ":" + std::to_string(__LINE__)); \
  } while (0)

constexpr int TK = 16;   // FP64 kernel: K step of a tile
constexpr int KMAX_F64 = 1024;   // summed K per work item before splitting (FP64 kernel)
constexpr int KMAX_TC = 4096;    // same for the tensor-core kernel

__device__ __forceinline__ const double* res(unsigned long long v, int buf, const Bases& B) {
  return buf == 0 ? reinterpret_cast<const double*>(v)
                  : reinterpret_cast<const double*>(B.b[buf] + v * 8ull);
}

// One CTA per TM x TN output tile of a problem (TM, TN in {32, 64}, the
// smallest padding of each problem's rows and columns), summing every segment
// of its range. Each warp owns a 16 x 32 region of the tile and each of its
// threads a 4 x 4 sub-tile of that region (rows 4 apart, columns 8 apart, so
// that shared-memory reads are conflict-free); a warp whose region lies
// outside the problem takes part in the loads but issues no FMA, and the K
// loop of a chunk stops at the segment's K: the FP64 pipe, the bound of this
// kernel, only runs on the problem's rows up to a multiple of 16, its
// columns up to a multiple of 32 and its exact K.
template <int TM, int TN>
__global__ void __launch_bounds__(TM * TN / 16, TM * TN == 4096 ? 2 : (TM * TN == 2048 ? 3 : 4)) seg_gemm_f64_t(const GProb* __restrict__ probs,
                                                               const GSeg* __restrict__ segs,
                                                               const GTile* __restrict__ tiles, int ntiles,
                                                               Bases bases) {
  const int t = blockIdx.x;
  if (t >= ntiles) return;
  const GTile tl = tiles[t];
  const GProb p = probs[tl.prob];
  constexpr int NT = TM * TN / 16;  // threads; each computes 4 x 4 outputs
  constexpr int WRM = TM / 16;      // warp regions along the rows
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31;
  const int rb = 16 * (w % WRM), cb = 32 * (w / WRM);   // the warp's region in the tile
  const int ty = lane >> 3, tx = lane & 7;               // rows rb + ty + 4r, columns cb + tx + 8c
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  const int m0 = tl.m0, n0 = tl.n0;
  const bool active = m0 + rb < p.m && n0 + cb < p.n;   // uniform in the warp
  for (int s = tl.s0; s < tl.s1; ++s) {
    const GSeg g = segs[p.seg0 + s];
    const bool aid = (g.a == 0ull && g.abuf == 0);
    const bool bid = (g.b == 0ull && g.bbuf == 0);
    if (aid) {
      if (bid) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (m0 + rb + ty + 4 * r == n0 + cb + tx + 8 * c) acc[r][c] += g.sc;
      } else {
        const double* Bp = res(g.b, g.bbuf, bases);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int row = m0 + rb + ty + 4 * r;
          if (row >= p.m) continue;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int col = n0 + cb + tx + 8 * c;
            if (col >= p.n) continue;
            const double v = g.tb ? Bp[(size_t)col * g.ldb + row] : Bp[(size_t)row * g.ldb + col];
            acc[r][c] += g.sc * v;
          }
        }
      }
      continue;
    }
    const double* Ap = res(g.a, g.abuf, bases);
    const double* Bp = res(g.b, g.bbuf, bases);
    for (int k0 = 0; k0 < g.k; k0 += TK) {
#pragma unroll
      for (int e = 0; e < TM * TK / NT; ++e) {
        const int idx = tid + NT * e;
        int row, kk;
        if (g.ta) { kk = idx / TM; row = idx % TM; }
        else { row = idx / TK; kk = idx % TK; }
        const int gr = m0 + row, gk = k0 + kk;
        double v = 0.0;
        if (gr < p.m && gk < g.k)
          v = g.ta ? Ap[(size_t)gk * g.lda + gr] : Ap[(size_t)gr * g.lda + gk];
        As[kk][row] = v * g.sc;
      }
#pragma unroll
      for (int e = 0; e < TN * TK / NT; ++e) {
        const int idx = tid + NT * e;
        int col, kk;
        if (g.tb) { col = idx / TK; kk = idx % TK; }
        else { kk = idx / TN; col = idx % TN; }
        const int gc = n0 + col, gk = k0 + kk;
        double v = 0.0;
        if (gc < p.n && gk < g.k)
          v = g.tb ? Bp[(size_t)gc * g.ldb + gk] : Bp[(size_t)gk * g.ldb + gc];
        Bs[kk][col] = v;
      }
      __syncthreads();
      if (active) {
        const int kn = g.k - k0 < TK ? g.k - k0 : TK;   // uniform in the CTA
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
          if (kk < kn) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][rb + ty + 4 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][cb + tx + 8 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
          }
        }
      }
      __syncthreads();
    }
  }
  double* Cp = const_cast<double*>(res(p.c, p.cbuf, bases));
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int row = m0 + rb + ty + 4 * r;
    if (row >= p.m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = n0 + cb + tx + 8 * c;
      if (col >= p.n) continue;
      double* dst = Cp + (size_t)row * p.ldc + col;
      if (tl.split) atomicAdd(dst, acc[r][c]);
      else *dst = p.beta ? *dst + acc[r][c] : acc[r][c];
    }
  }
}

// ---------------------------------------------------------------------------
// Vector kernels (initial MPS, norms).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void randn_kernel(double* p, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z1 = splitmix64(seed ^ splitmix64((unsigned long long)i));
    unsigned long long z2 = splitmix64(z1);
    double u1 = ((z1 >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
    double u2 = (z2 >> 11) * 0x1.0p-53;           // [0, 1)
    p[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

__global__ void dot_partial(const double* x, const double* y, long long n, double* part) {
  __shared__ double sh[256];
  double s = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void scale_kernel(double* x, double a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] *= a;
}

__global__ void axpby_kernel(double* y, double a, const double* x, double b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// Batched dots and linear combinations of Davidson basis vectors: one launch
// pair and one host round trip for up to MVEC vectors instead of one per vector.
constexpr int MVEC = 64;
struct VecList {
  const double* p[MVEC];
  double c[MVEC];
};

// part[k * gridDim.x + b] = block b's contiguous share of xs[k] . y (the share
// of y stays in L1 across the m vectors)
__global__ void mdot_partial(VecList xs, int m, const double* y, long long n, double* part) {
  __shared__ double sh[256];
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = (long long)blockIdx.x * per, hi = min(n, lo + per);
  for (int k = 0; k < m; ++k) {
    const double* x = xs.p[k];
    double s = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s = fma(x[i], y[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)k * gridDim.x + blockIdx.x] = sh[0];
  }
}

// out[k] = sum of the nb block shares of vector k (block k)
__global__ void mdot_reduce(const double* part, int nb, double* out) {
  __shared__ double sh[256];
  double s = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(long long)blockIdx.x * nb + b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// y = sum_k c_k x_k + b y (b = 0: y is not read)
__global__ void mcombine_kernel(double* y, VecList xs, int m, double b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0;
    for (int k = 0; k < m; ++k) s = fma(xs.c[k], xs.p[k][i], s);
    y[i] = (b == 0.0) ? s : fma(b, y[i], s);
  }
}

__global__ void precond_kernel(double* t, const double* r, const double* d, double theta, double fl,
                               long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double den = d[i] - theta;
    if (fabs(den) < fl) den = den < 0 ? -fl : fl;
    t[i] = r[i] / den;
  }
}

// ---------------------------------------------------------------------------
// FP64 tile shapes: TM, TN in {64, 32}; class 2 * i(TM) + i(TN)
constexpr int F64_SIZES[2] = {64, 32};
constexpr int F64_CLASSES = 4;

struct DevLaunch {
  GProb* p = nullptr;
  GSeg* s = nullptr;
  GTile* t = nullptr;    // FP64 tiles, grouped by shape class
  int cls[F64_CLASSES + 1] = {};  // class c: tiles [cls[c], cls[c+1])
  GTile* t2 = nullptr;   // 128x128 tiles (tcgen05 kernel)
  int ntiles2 = 0;
  int nsplit = 0;        // FP64 tiles of split problems
  double flops = 0;
};

// Work items: every tile of every problem, with the problem's segments cut into
// ranges whose summed K stays below kmax (split-K over segments).
// sel: 0 all problems, 1 problems that fit in 32 x 32, 2 the others
static void make_tiles(const Launch& l, int tile, int kmax, std::vector<GTile>& T, int sel = 0) {
  T.clear();
  for (size_t i = 0; i < l.probs.size(); ++i) {
    const Prob& q = l.probs[i];
    const bool small = q.m <= 32 && q.n <= 32;
    if ((sel == 1 && !small) || (sel == 2 && small)) continue;
    std::vector<std::pair<int, int>> ranges;
    int s0 = 0, ksum = 0;
    for (int s = 0; s < q.nseg; ++s) {
      const Seg& g = l.segs[q.seg0 + s];
      int k = (g.a == 0 && g.abuf == 0) ? 1 : g.k;
      if (s > s0 && ksum + k > kmax) {
        ranges.push_back({s0, s});
        s0 = s;
        ksum = 0;
      }
      ksum += k;
    }
    ranges.push_back({s0, q.nseg});
    const int split = ranges.size() > 1 ? 1 : 0;
    for (int m0 = 0; m0 < q.m; m0 += tile)
      for (int n0 = 0; n0 < q.n; n0 += tile)
        for (auto& r : ranges) T.push_back({(int)i, m0, n0, r.first, r.second, split});
  }
}

// FP64 work items: each problem gets the tile shape of least padding (ties:
// the larger tile), tiles listed class by class; off gets the class offsets
static int f64_size_index(int d) {
  int best = 0;
  long long pad = 1ll << 60;
  for (int i = 0; i < 2; ++i) {
    const int t = F64_SIZES[i];
    const long long p = (long long)((d + t - 1) / t) * t;
    if (p < pad) { pad = p; best = i; }
  }
  return best;
}
static void make_tiles_f64(const Launch& l, int kmax, std::vector<GTile>& T, int off[F64_CLASSES + 1]) {
  std::vector<GTile> byc[F64_CLASSES];
  for (size_t i = 0; i < l.probs.size(); ++i) {
    const Prob& q = l.probs[i];
    const int im = f64_size_index(q.m), in = f64_size_index(q.n);
    const int tm = F64_SIZES[im], tn = F64_SIZES[in];
    std::vector<std::pair<int, int>> ranges;
    int s0 = 0, ksum = 0;
    for (int s = 0; s < q.nseg; ++s) {
      const Seg& g = l.segs[q.seg0 + s];
      int k = (g.a == 0 && g.abuf == 0) ? 1 : g.k;
      if (s > s0 && ksum + k > kmax) {
        ranges.push_back({s0, s});
        s0 = s;
        ksum = 0;
      }
      ksum += k;
    }
    ranges.push_back({s0, q.nseg});
    const int split = ranges.size() > 1 ? 1 : 0;
    for (int m0 = 0; m0 < q.m; m0 += tm)
      for (int n0 = 0; n0 < q.n; n0 += tn)
        for (auto& r : ranges) byc[2 * im + in].push_back({(int)i, m0, n0, r.first, r.second, split});
  }
  T.clear();
  for (int c = 0; c < F64_CLASSES; ++c) {
    off[c] = (int)T.size();
    T.insert(T.end(), byc[c].begin(), byc[c].end());
  }
  off[F64_CLASSES] = (int)T.size();
}

static void build_host(const Launch& l, std::vector<GProb>& P, std::vector<GSeg>& S) {
  P.resize(l.probs.size());
  S.resize(l.segs.size());
  for (size_t i = 0; i < l.probs.size(); ++i) {
    const Prob& q = l.probs[i];
    GProb& g = P[i];
    g.c = q.c; g.m = q.m; g.n = q.n; g.ldc = q.ldc; g.beta = q.beta;
    g.seg0 = q.seg0; g.nseg = q.nseg; g.cbuf = q.cbuf; g.pad = 0;
  }
  for (size_t i = 0; i < l.segs.size(); ++i) {
    const Seg& q = l.segs[i];
    GSeg& g = S[i];
    g.a = q.a; g.b = q.b; g.lda = q.lda; g.ldb = q.ldb; g.k = q.k;
    g.abuf = (unsigned char)q.abuf; g.bbuf = (unsigned char)q.bbuf;
    g.ta = (unsigned char)q.ta; g.tb = (unsigned char)q.tb; g.sc = q.sc;
  }
}

// FP64 kernel launches, one per tile-shape class
template <int TM, int TN>
static void launch_class(const GProb* P, const GSeg* S, const GTile* T, int n, const Bases& B, cudaStream_t st) {
  if (n > 0) seg_gemm_f64_t<TM, TN><<<n, TM * TN / 16, 0, st>>>(P, S, T, n, B);
}
static void launch_f64(const GProb* P, const GSeg* S, const GTile* T, const int* off, const Bases& B,
                       cudaStream_t st) {
  auto n = [&](int c) { return off[c + 1] - off[c]; };
  launch_class<64, 64>(P, S, T + off[0], n(0), B, st);
  launch_class<64, 32>(P, S, T + off[1], n(1), B, st);
  launch_class<32, 64>(P, S, T + off[2], n(2), B, st);
  launch_class<32, 32>(P, S, T + off[3], n(3), B, st);
}

class CudaExec : public Executor, public PreparedRunner {
 public:
  explicit CudaExec(int device) : dev_(device) {
    CK(cudaSetDevice(dev_));
    CK(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
    CK(cudaMalloc(&err_, sizeof(int)));
    CK(cudaMemset(err_, 0, sizeof(int)));
    CK(cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev_));
  }
  ~CudaExec() override {
    cudaSetDevice(dev_);
    cudaStreamSynchronize(st_);
    for (auto& d : prepared_) free_dev(d);
    free_tiled();
    if (tmp_) cudaFree(reinterpret_cast<void*>(tmp_));
    if (sp_) cudaFree(sp_);
    if (ss_) cudaFree(ss_);
    if (stt_) cudaFree(stt_);
    if (part_) cudaFree(part_);
    if (work_) cudaFree(work_);
    if (info_) cudaFree(info_);
    if (sol_) cusolverDnDestroy(sol_);
    if (err_) cudaFree(err_);
    if (cp_) cudaStreamDestroy(cp_);
    if (cpev_) cudaEventDestroy(cpev_);
    cudaStreamDestroy(st_);
  }
  uint64_t alloc(int64_t n) override {
    void* p = nullptr;
    if (n <= 0) n = 1;
    CK(cudaMalloc(&p, (size_t)n * 8));
    CK(cudaMemsetAsync(p, 0, (size_t)n * 8, st_));
    bytes_ += n * 8;
    live_ += n * 8;
    peak_ = std::max(peak_, live_);
    sizes_[reinterpret_cast<uint64_t>(p)] = n * 8;
    return reinterpret_cast<uint64_t>(p);
  }
  void release(uint64_t p) override {
    if (p) {
      CK(cudaStreamSynchronize(st_));
      CK(cudaFree(reinterpret_cast<void*>(p)));
      auto it = sizes_.find(p);
      if (it != sizes_.end()) {
        live_ -= it->second;
        sizes_.erase(it);
      }
    }
  }
  uint64_t host_alloc(int64_t n) override {
    void* p = nullptr;
    CK(cudaHostAlloc(&p, (size_t)std::max<int64_t>(1, n) * 8, cudaHostAllocDefault));
    return reinterpret_cast<uint64_t>(p);
  }
  void host_free(uint64_t h) override {
    if (h) CK(cudaFreeHost(reinterpret_cast<void*>(h)));
  }
  void d2h(uint64_t h, uint64_t d, int64_t n) override {
    CK(cudaStreamSynchronize(st_));
    CK(cudaMemcpy(reinterpret_cast<void*>(h), reinterpret_cast<void*>(d), (size_t)n * 8, cudaMemcpyDeviceToHost));
  }
  void h2d_async(uint64_t d, uint64_t h, int64_t n) override {
    if (!cp_) {
      CK(cudaStreamCreateWithFlags(&cp_, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&cpev_, cudaEventDisableTiming));
    }
    // the destination was allocated (and zeroed) on the compute stream
    CK(cudaEventRecord(cpev_, st_));
    CK(cudaStreamWaitEvent(cp_, cpev_, 0));
    CK(cudaMemcpyAsync(reinterpret_cast<void*>(d), reinterpret_cast<void*>(h), (size_t)n * 8,
                       cudaMemcpyHostToDevice, cp_));
  }
  void copies_join() override {
    if (!cp_) return;
    auto t0 = std::chrono::steady_clock::now();
    CK(cudaStreamSynchronize(cp_));
    wait_s_ += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  double copies_wait_seconds() override { return wait_s_; }
  int64_t live_bytes() const override { return live_; }
  uint64_t tmp(int64_t n) override {
    if (n > tmpcap_) {
      CK(cudaStreamSynchronize(st_));
      if (tmp_) CK(cudaFree(reinterpret_cast<void*>(tmp_)));
      void* p = nullptr;
      CK(cudaMalloc(&p, (size_t)n * 8));
      tmp_ = reinterpret_cast<uint64_t>(p);
      tmpcap_ = n;
    }
    return tmp_;
  }
  void run(const Launch& l, uint64_t psi, uint64_t sig) override {
    if (l.empty()) return;
    std::vector<GProb> P;
    std::vector<GSeg> S;
    std::vector<GTile> T;
    int off[F64_CLASSES + 1];
    build_host(l, P, S);
    make_tiles_f64(l, KMAX_F64, T, off);
    CK(cudaStreamSynchronize(st_));
    grow(&sp_, &spcap_, P.size() * sizeof(GProb));
    grow(&ss_, &sscap_, std::max<size_t>(1, S.size()) * sizeof(GSeg));
    grow(&stt_, &stcap_, std::max<size_t>(1, T.size()) * sizeof(GTile));
    CK(cudaMemcpyAsync(sp_, P.data(), P.size() * sizeof(GProb), cudaMemcpyHostToDevice, st_));
    if (!S.empty()) CK(cudaMemcpyAsync(ss_, S.data(), S.size() * sizeof(GSeg), cudaMemcpyHostToDevice, st_));
    if (!T.empty()) CK(cudaMemcpyAsync(stt_, T.data(), T.size() * sizeof(GTile), cudaMemcpyHostToDevice, st_));
    Bases B;
    B.b[0] = 0; B.b[1] = psi; B.b[2] = sig; B.b[3] = tmp_;
    launch_f64((GProb*)sp_, (GSeg*)ss_, (GTile*)stt_, off, B, st_);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st_));
  }
  void upload(uint64_t dst, const double* h, int64_t n) override {
    CK(cudaMemcpyAsync(reinterpret_cast<void*>(dst), h, (size_t)n * 8, cudaMemcpyHostToDevice, st_));
    CK(cudaStreamSynchronize(st_));
  }
  void download(double* h, uint64_t src, int64_t n) override {
    CK(cudaMemcpyAsync(h, reinterpret_cast<void*>(src), (size_t)n * 8, cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
  }
  void zero(uint64_t p, int64_t n) override {
    CK(cudaMemsetAsync(reinterpret_cast<void*>(p), 0, (size_t)n * 8, st_));
  }
  void randn(uint64_t p, int64_t n, uint64_t seed) override {
    if (n <= 0) return;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    randn_kernel<<<blocks, 256, 0, st_>>>(reinterpret_cast<double*>(p), n, seed);
    CK(cudaGetLastError());
  }
  void orthonormal_cols(uint64_t p, int rows, int cols) override {
    if (rows < cols) throw std::runtime_error("orthonormal_cols: rows < cols");
    solver();
    double* A = reinterpret_cast<double*>(p);
    int l1 = 0, l2 = 0;
    if (cusolverDnDgeqrf_bufferSize(sol_, rows, cols, A, rows, &l1) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDorgqr_bufferSize(sol_, rows, cols, cols, A, rows, (double*)tau_, &l2) != CUSOLVER_STATUS_SUCCESS)
      throw std::runtime_error("CUDA: cusolver buffer query failed");
    size_t need = (size_t)std::max(l1, l2) + cols;
    if (need > work_cap_) {
      CK(cudaStreamSynchronize(st_));
      if (work_) CK(cudaFree(work_));
      CK(cudaMalloc(&work_, need * 8));
      work_cap_ = need;
    }
    double* tau = (double*)work_;
    double* wk = tau + cols;
    int lw = (int)(work_cap_ - cols);
    if (cusolverDnDgeqrf(sol_, rows, cols, A, rows, tau, wk, lw, info_) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDorgqr(sol_, rows, cols, cols, A, rows, tau, wk, lw, info_) != CUSOLVER_STATUS_SUCCESS)
      throw std::runtime_error("CUDA: cusolver QR failed");
    int info = 0;
    CK(cudaMemcpyAsync(&info, info_, sizeof(int), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    if (info != 0) throw std::runtime_error("CUDA: QR reported info " + std::to_string(info));
  }
  double dot(uint64_t x, uint64_t y, int64_t n) override {
    if (n <= 0) return 0.0;
    const int nb = 1024;
    grow(&part_, &part_cap_, nb * sizeof(double));
    dot_partial<<<nb, 256, 0, st_>>>(reinterpret_cast<const double*>(x), reinterpret_cast<const double*>(y), n,
                                      (double*)part_);
    CK(cudaGetLastError());
    double h[1024];
    CK(cudaMemcpyAsync(h, part_, nb * sizeof(double), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    double s = 0;
    for (int i = 0; i < nb; ++i) s += h[i];
    return s;
  }
  void mdot(const uint64_t* xs, int m, uint64_t y, int64_t n, double* out) override {
    for (int k0 = 0; k0 < m; k0 += MVEC) {
      const int mk = std::min(MVEC, m - k0);
      if (n <= 0) {
        for (int k = 0; k < mk; ++k) out[k0 + k] = 0.0;
        continue;
      }
      VecList v{};
      for (int k = 0; k < mk; ++k) v.p[k] = reinterpret_cast<const double*>(xs[k0 + k]);
      const int nb = 2 * 148;
      grow(&part_, &part_cap_, (size_t)(mk * nb + mk) * sizeof(double));
      double* part = (double*)part_;
      mdot_partial<<<nb, 256, 0, st_>>>(v, mk, reinterpret_cast<const double*>(y), n, part);
      mdot_reduce<<<mk, 256, 0, st_>>>(part, nb, part + (size_t)mk * nb);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(out + k0, part + (size_t)mk * nb, mk * sizeof(double), cudaMemcpyDeviceToHost, st_));
      CK(cudaStreamSynchronize(st_));
    }
  }
  void mcombine(uint64_t y, const uint64_t* xs, const double* c, int m, double b, int64_t n) override {
    if (n <= 0) return;
    if (m <= 0) {
      if (b == 0.0) zero(y, n);
      else if (b != 1.0) scale(y, b, n);
      return;
    }
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    for (int k0 = 0; k0 < m; k0 += MVEC) {
      const int mk = std::min(MVEC, m - k0);
      VecList v{};
      for (int k = 0; k < mk; ++k) {
        v.p[k] = reinterpret_cast<const double*>(xs[k0 + k]);
        v.c[k] = c[k0 + k];
      }
      mcombine_kernel<<<blocks, 256, 0, st_>>>(reinterpret_cast<double*>(y), v, mk, k0 == 0 ? b : 1.0, n);
      CK(cudaGetLastError());
    }
  }
  void axpby(uint64_t y, double a, uint64_t x, double b, int64_t n) override {
    if (n <= 0) return;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    axpby_kernel<<<blocks, 256, 0, st_>>>(reinterpret_cast<double*>(y), a, reinterpret_cast<const double*>(x), b, n);
    CK(cudaGetLastError());
  }
  void precond(uint64_t t, uint64_t r, uint64_t d, double theta, double fl, int64_t n) override {
    if (n <= 0) return;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    precond_kernel<<<blocks, 256, 0, st_>>>(reinterpret_cast<double*>(t), reinterpret_cast<const double*>(r),
                                            reinterpret_cast<const double*>(d), theta, fl, n);
    CK(cudaGetLastError());
  }
  void copy(uint64_t dst, uint64_t src, int64_t n) override {
    if (n <= 0) return;
    CK(cudaMemcpyAsync(reinterpret_cast<void*>(dst), reinterpret_cast<void*>(src), (size_t)n * 8,
                       cudaMemcpyDeviceToDevice, st_));
  }
  void eigh(uint64_t A, int n, double* w) override {
    if (n <= 0) return;
    solver();
    double* dA = reinterpret_cast<double*>(A);
    int lw = 0;
    if (cusolverDnDsyevd_bufferSize(sol_, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, nullptr,
                                    &lw) != CUSOLVER_STATUS_SUCCESS)
      throw std::runtime_error("CUDA: syevd buffer query failed");
    size_t need = (size_t)lw + n;
    if (need > work_cap_) {
      CK(cudaStreamSynchronize(st_));
      if (work_) CK(cudaFree(work_));
      CK(cudaMalloc(&work_, need * 8));
      work_cap_ = need;
    }
    double* dw = (double*)work_;
    double* wk = dw + n;
    if (cusolverDnDsyevd(sol_, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dw, wk,
                         (int)(work_cap_ - n), info_) != CUSOLVER_STATUS_SUCCESS)
      throw std::runtime_error("CUDA: syevd failed");
    int info = 0;
    CK(cudaMemcpyAsync(w, dw, (size_t)n * 8, cudaMemcpyDeviceToHost, st_));
    CK(cudaMemcpyAsync(&info, info_, sizeof(int), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    if (info != 0) throw std::runtime_error("CUDA: syevd reported info " + std::to_string(info));
  }
  void scale(uint64_t x, double a, int64_t n) override {
    if (n <= 0) return;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    scale_kernel<<<blocks, 256, 0, st_>>>(reinterpret_cast<double*>(x), a, n);
    CK(cudaGetLastError());
  }

  // prepared launches (uploaded once, replayed on any psi / sigma)
  int prepare(const Launch& l) override {
    DevLaunch d;
    std::vector<GProb> P;
    std::vector<GSeg> S;
    std::vector<GTile> T, T2;
    build_host(l, P, S);
    make_tiles_f64(l, KMAX_F64, T, d.cls);
    make_tiles(l, TC_TILE, KMAX_TC, T2, 0);
    d.ntiles2 = (int)T2.size();
    for (const GTile& g : T) d.nsplit += g.split ? 1 : 0;
    d.flops = l.flops;
    auto up = [](void** dst, const void* src, size_t bytes) {
      CK(cudaMalloc(dst, std::max<size_t>(bytes, 16)));
      if (bytes) CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    };
    if (!P.empty()) {
      up((void**)&d.p, P.data(), P.size() * sizeof(GProb));
      up((void**)&d.s, S.data(), S.size() * sizeof(GSeg));
      up((void**)&d.t, T.data(), T.size() * sizeof(GTile));
      up((void**)&d.t2, T2.data(), T2.size() * sizeof(GTile));
    }
    prepared_.push_back(d);
    return (int)prepared_.size() - 1;
  }
  void drop_prepared() override {
    CK(cudaStreamSynchronize(st_));
    for (auto& d : prepared_) free_dev(d);
    prepared_.clear();
    free_tiled();
  }

  void prepare_tiled(const TiledPlan& P, int planes) override {
    CK(cudaStreamSynchronize(st_));
    free_tiled();
    TiledDev& t = td_;
    t.planes = planes;
    t.aplane = P.abytes;
    t.bplane = P.bbytes;
    t.psiplane = P.psibytes;
    t.tplane = P.tbytes;
    auto arena = [&](uint8_t** d, int64_t bytes) {
      const size_t n = std::max<size_t>(16, (size_t)bytes * planes);
      CK(cudaMalloc(reinterpret_cast<void**>(d), n));
      CK(cudaMemsetAsync(*d, 0, n, st_));  // padding stays zero for good
      t.bytes += (int64_t)n;
    };
    arena(&t.a, P.abytes);
    arena(&t.b, P.bbytes);
    arena(&t.psi, P.psibytes);
    arena(&t.t, P.tbytes);
    TView *av = nullptr, *bv = nullptr;
    upload(reinterpret_cast<void**>(&av), P.avw.data(), P.avw.size() * sizeof(TView), nullptr);
    upload(reinterpret_cast<void**>(&bv), P.bvw.data(), P.bvw.size() * sizeof(TView), nullptr);
    upload(reinterpret_cast<void**>(&t.psiv), P.psivw.data(), P.psivw.size() * sizeof(TView), &t.bytes);
    t.npsiv = (int)P.psivw.size();
    psi_elems_ = P.psi_elems;
    set_items(P);
    // operator mirrors: converted once per prepared centre
    CK(launch_tile_views(av, (int)P.avw.size(), t.a, P.abytes, planes, nullptr, st_));
    CK(launch_tile_views(bv, (int)P.bvw.size(), t.b, P.bbytes, planes, nullptr, st_));
    CK(cudaStreamSynchronize(st_));
    CK(cudaFree(av));
    CK(cudaFree(bv));
    live_ += t.bytes;
    peak_ = std::max(peak_, live_);
  }
  void set_tiled_chunk(int bytes) override { chunk_ = std::max(0, std::min(bytes, 65536)); }
  void set_tiled_items(const TiledPlan& P) override {
    if (!td_.planes) throw std::runtime_error("tiled path not prepared");
    CK(cudaStreamSynchronize(st_));
    live_ -= td_.items_bytes;
    td_.bytes -= td_.items_bytes;
    for (void* p : {(void*)td_.i1, (void*)td_.v1, (void*)td_.i2, (void*)td_.s2})
      if (p) CK(cudaFree(p));
    set_items(P);
    live_ += td_.items_bytes;
    peak_ = std::max(peak_, live_);
  }
  int tiled_planes() const override { return td_.planes; }
  int64_t free_device_bytes() const override {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return INT64_MAX;
    return (int64_t)fr + td_.bytes;
  }
  double time_tiled(uint64_t psi, uint64_t sig, int precision, int reps) override {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // sigma is zeroed before each product, as every caller of run_tiled does
    CK(cudaMemsetAsync(reinterpret_cast<void*>(sig), 0, (size_t)psi_elems_ * 8, st_));
    run_tiled(psi, sig, st_, precision);
    CK(cudaEventRecord(e0, st_));
    for (int r = 0; r < reps; ++r) {
      CK(cudaMemsetAsync(reinterpret_cast<void*>(sig), 0, (size_t)psi_elems_ * 8, st_));
      run_tiled(psi, sig, st_, precision);
    }
    CK(cudaEventRecord(e1, st_));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms * 1e-3 / std::max(1, reps);
  }
  void run_tiled(uint64_t psi, uint64_t sig, void* stream, int precision) override {
    const TiledDev& t = td_;
    const int mode = precision == 3 ? TT_BF16X3 : TT_BF16;
    if (t.planes == 0 || (mode == TT_BF16X3 && t.planes < 3) || (precision != 2 && precision != 3))
      throw std::runtime_error("tiled tensor-core path not prepared for this precision");
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_tile_views(t.psiv, t.npsiv, t.psi, t.psiplane, t.planes, reinterpret_cast<const double*>(psi), s));
    // one stage-1 and one stage-2 launch per pass of the T arena (stage-1 pads
    // of T that a pass does not write may hold an earlier pass's finite values:
    // its K pads meet the zero K pads of the left views, its row pads only reach
    // sigma columns the stage-2 epilogue discards)
    for (size_t p = 0; p + 1 < t.pass1.size(); ++p) {
      const int a1 = t.pass1[p], n1 = t.pass1[p + 1] - a1, a2 = t.pass2[p], n2 = t.pass2[p + 1] - a2;
      CK(launch_tiled_stage1(mode, t.i1 + a1, n1, t.v1, t.psi, t.psiplane, t.b, t.bplane, t.t, t.tplane, chunk_,
                             nsm_, err_, s));
      CK(launch_tiled_stage2(mode, t.i2 + a2, n2, t.s2, t.a, t.aplane, t.t, t.tplane,
                             reinterpret_cast<double*>(sig), chunk_, nsm_, err_, s));
    }
  }
  void run_prepared(int h, uint64_t psi, uint64_t sig, void* stream, int precision) override {
    const DevLaunch& d = prepared_.at(h);
    if (!d.cls[F64_CLASSES]) return;
    if (precision == 0) {
      Bases B;
      B.b[0] = 0; B.b[1] = psi; B.b[2] = sig; B.b[3] = tmp_;
      launch_f64(d.p, d.s, d.t, d.cls, B, (cudaStream_t)stream);
      CK(cudaGetLastError());
      return;
    }
    if (!err_) {
      CK(cudaMalloc(&err_, sizeof(int)));
      CK(cudaMemset(err_, 0, sizeof(int)));
    }
    Bases B;
    B.b[0] = 0; B.b[1] = psi; B.b[2] = sig; B.b[3] = tmp_;
    // the BF16 forms run on the tiled kernel (run_tiled); prepared task lists
    // reach the tensor cores in the TF32 form only
    if (precision != 1) throw std::runtime_error("run_prepared: BF16 forms use the tiled kernel");
    int mode = TC_TF32;
    CK(launch_tc(mode, d.p, d.s, d.t2, d.ntiles2, B, err_, (cudaStream_t)stream));
  }
  int take_error() override {
    if (!err_) return 0;
    int h = 0;
    CK(cudaMemcpy(&h, err_, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) CK(cudaMemset(err_, 0, sizeof(int)));
    return h;
  }
  const void* prepared_handle(int h) const override { return &prepared_.at(h); }
  void tile_counts(int h, int64_t counts[5]) const override {
    const DevLaunch& d = prepared_.at(h);
    for (int c = 0; c < F64_CLASSES; ++c) counts[c] = d.cls[c + 1] - d.cls[c];
    counts[4] = d.nsplit;
  }
  void* stream() override { return st_; }
  void sync(void* stream) override { CK(cudaStreamSynchronize((cudaStream_t)stream)); }
  void zero_async(uint64_t p, int64_t n, void* stream) override {
    CK(cudaMemsetAsync(reinterpret_cast<void*>(p), 0, (size_t)n * 8, (cudaStream_t)stream));
  }
  int64_t bytes_allocated() const override { return peak_; }

 private:
  void solver() {
    if (!sol_) {
      if (cusolverDnCreate(&sol_) != CUSOLVER_STATUS_SUCCESS) throw std::runtime_error("CUDA: cusolverDnCreate failed");
      cusolverDnSetStream(sol_, st_);
      CK(cudaMalloc(&info_, sizeof(int)));
    }
  }
  void grow(void** p, size_t* cap, size_t need) {
    if (need <= *cap) return;
    if (*p) CK(cudaFree(*p));
    CK(cudaMalloc(p, need));
    *cap = need;
  }
  struct TiledDev {
    int planes = 0;
    uint8_t *a = nullptr, *b = nullptr, *psi = nullptr, *t = nullptr;
    int64_t aplane = 0, bplane = 0, psiplane = 0, tplane = 0;
    TView* psiv = nullptr;
    K1Item* i1 = nullptr;
    K1View* v1 = nullptr;
    K2Item* i2 = nullptr;
    K2Seg* s2 = nullptr;
    int npsiv = 0, ni1 = 0, ni2 = 0;
    std::vector<int> pass1, pass2;   // item ranges of the passes (host copies)
    int64_t bytes = 0, items_bytes = 0;
  };
  void upload(void** d, const void* src, size_t bytes, int64_t* count) {
    CK(cudaMalloc(d, std::max<size_t>(bytes, 16)));
    if (bytes) CK(cudaMemcpy(*d, src, bytes, cudaMemcpyHostToDevice));
    if (count) *count += (int64_t)std::max<size_t>(bytes, 16);
  }
  void set_items(const TiledPlan& P) {
    TiledDev& t = td_;
    int64_t b = 0;
    upload(reinterpret_cast<void**>(&t.i1), P.i1.data(), P.i1.size() * sizeof(K1Item), &b);
    upload(reinterpret_cast<void**>(&t.v1), P.v1.data(), P.v1.size() * sizeof(K1View), &b);
    upload(reinterpret_cast<void**>(&t.i2), P.i2.data(), P.i2.size() * sizeof(K2Item), &b);
    upload(reinterpret_cast<void**>(&t.s2), P.s2.data(), P.s2.size() * sizeof(K2Seg), &b);
    t.ni1 = (int)P.i1.size();
    t.ni2 = (int)P.i2.size();
    t.pass1 = P.pass1;
    t.pass2 = P.pass2;
    if (t.pass1.size() < 2 || t.pass1.size() != t.pass2.size() || t.pass1.back() != t.ni1 || t.pass2.back() != t.ni2)
      throw std::runtime_error("tiled plan: inconsistent passes");
    t.items_bytes = b;
    t.bytes += b;
  }
  void free_tiled() {
    TiledDev& t = td_;
    if (!t.planes && !t.bytes) return;
    cudaStreamSynchronize(st_);
    for (void* p : {(void*)t.a, (void*)t.b, (void*)t.psi, (void*)t.t, (void*)t.psiv, (void*)t.i1, (void*)t.v1,
                    (void*)t.i2, (void*)t.s2})
      if (p) cudaFree(p);
    live_ -= t.bytes;
    t = TiledDev();
  }
  static void free_dev(DevLaunch& d) {
    if (d.p) cudaFree(d.p);
    if (d.s) cudaFree(d.s);
    if (d.t) cudaFree(d.t);
    if (d.t2) cudaFree(d.t2);
    d.p = nullptr; d.s = nullptr; d.t = nullptr; d.t2 = nullptr;
  }
  int dev_;
  int nsm_ = 148;
  TiledDev td_;
  int64_t psi_elems_ = 0;
  cudaStream_t st_ = nullptr;
  uint64_t tmp_ = 0;
  int64_t tmpcap_ = 0;
  void *sp_ = nullptr, *ss_ = nullptr, *stt_ = nullptr;
  size_t spcap_ = 0, sscap_ = 0, stcap_ = 0;
  std::vector<DevLaunch> prepared_;
  int64_t bytes_ = 0, live_ = 0, peak_ = 0;
  std::map<uint64_t, int64_t> sizes_;
  cudaStream_t cp_ = nullptr;
  cudaEvent_t cpev_ = nullptr;
  double wait_s_ = 0;
  int* err_ = nullptr;
  cusolverDnHandle_t sol_ = nullptr;
  int* info_ = nullptr;
  void* work_ = nullptr;
  size_t work_cap_ = 0;
  void* tau_ = nullptr;
  void* part_ = nullptr;
  size_t part_cap_ = 0;
  int chunk_ = 0;   // chunk byte target of the tiled kernels
};

cudaError_t launch_f64_prepared(const void* handle, uint64_t psi, uint64_t sig, uint64_t scratch,
                                cudaStream_t st) {
  const DevLaunch* d = static_cast<const DevLaunch*>(handle);
  if (!d || !d->cls[F64_CLASSES]) return cudaSuccess;
  Bases B;
  B.b[0] = 0;
  B.b[1] = psi;
  B.b[2] = sig;
  B.b[3] = scratch;
  // a launch error left pending by earlier work on this thread is not this call's:
  // clear it so that the value returned below belongs to these launches
  (void)cudaGetLastError();
  launch_f64(d->p, d->s, d->t, d->cls, B, st);
  return cudaGetLastError();
}

Backend make_backend(int device) {
  auto* e = new CudaExec(device);
  return Backend{e, e};
}

}  // namespace qd

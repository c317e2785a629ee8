// tcgen05 segmented grouped GEMM of the TF32 form for sm_103a.
//
// Same task lists as the FP64 kernel: one CTA owns a 128x128 output tile of a
// problem and accumulates sum_s sc_s op(A_s) op(B_s) over all its segments in
// one FP32 accumulator in tensor memory. Operand tiles are loaded from HBM by
// all 128 threads (coalesced along the contiguous dimension of each operand),
// scaled by the segment scalar, rounded to TF32 (round to nearest) and stored
// in shared memory in the K-major no-swizzle core-matrix layout; one thread
// then issues tcgen05.mma (kind::tf32) for the chunk and tcgen05.commit
// signals an mbarrier when the tensor core has consumed the stage (two stages
// in flight). The BF16 and three-term BF16 forms run on the tiled kernel of
// tc_tiled.cu, whose operands are converted once per prepared centre.
// Every mbarrier wait is bounded (about one second of clock64 cycles); on a
// timeout the kernel records an error code, waits once more (bounded) for its
// own MMAs, frees its tensor memory and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_gemm.hpp"

namespace qd {

namespace {

constexpr int TCM = 128, TCN = 128;
constexpr long long WAIT_CYCLES = 2000000000ll;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// shared-memory matrix descriptor, K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  // base offset 0, relative LBO, layout type 0 = no swizzle
  return d;
}

// instruction descriptor: FP32 accumulate, K-major A and B, M = 128, N = 128
__host__ __device__ constexpr uint32_t idesc(uint32_t ab_format) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(TCN >> 3) << 17) |
         ((uint32_t)(TCM >> 4) << 24);
}

template <int MODE>
struct Cfg;
template <>
struct Cfg<TC_TF32> {
  static constexpr int ES = 4, KC = 32, KS = 8, NSPLIT = 1;
  static constexpr uint32_t FMT = 2;
};

__device__ __forceinline__ const double* resolve(unsigned long long v, int buf, const TcBases& B) {
  return buf == 0 ? reinterpret_cast<const double*>(v)
                  : reinterpret_cast<const double*>(B.b[buf] + v * 8ull);
}

// byte offset of element (r, k) of a 128 x KC K-major tile (core matrices of 8 x 16 B)
template <int ES, int KC>
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  constexpr int KB = KC * ES / 16;  // 16-byte columns per row
  const int kb = (k * ES) >> 4;
  return (uint32_t)((((r >> 3) * KB + kb) << 7) + ((r & 7) << 4) + ((k * ES) & 15));
}

// FP64 -> FP32 with round-to-nearest-even using integer operations only (the
// FP64 pipe of this GPU is narrow and a hardware conversion per operand
// element would be the bottleneck of the producer). Values below the FP32
// normal range flush to zero; the operands here are far from both limits.
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  unsigned int m23 = (unsigned int)(m >> 29);
  const unsigned long long rem = m & 0x1FFFFFFFull;
  const unsigned long long half = 0x10000000ull;
  unsigned int bits = sign | ((unsigned int)e << 23);
  if (rem > half || (rem == half && (m23 & 1u))) ++m23;  // carry into the exponent is exact
  return __uint_as_float(bits + m23);
}

// FP32 -> FP64, exact, integer operations only (zero and normal numbers)
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned int e = (b >> 23) & 0xFF;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long m = (unsigned long long)(b & 0x7FFFFF) << 29;
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | m));
}

template <int MODE>
__device__ __forceinline__ void put(unsigned char* base, uint32_t off, size_t, float x) {
  static_assert(MODE == TC_TF32, "TF32 only");
  // round to nearest TF32 (the tensor core would otherwise drop the low
  // mantissa bits, a biased truncation)
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  *reinterpret_cast<uint32_t*>(base + off) = r;
}

template <int MODE>
__global__ void __launch_bounds__(128, 1)
    seg_gemm_tc(const TcProb* __restrict__ probs, const TcSeg* __restrict__ segs,
                const TcTile* __restrict__ tiles, int ntiles, TcBases bases, int* err) {
  using C = Cfg<MODE>;
  constexpr int ES = C::ES, KC = C::KC, KS = C::KS, NS = C::NSPLIT;
  constexpr uint32_t TILE = TCM * KC * ES;          // bytes of one operand split
  constexpr uint32_t STAGE = 2 * NS * TILE;         // A splits then B splits
  constexpr uint32_t LBO = 128;
  constexpr uint32_t SBO = (KC * ES / 16) * 128;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE + 16);
  volatile int* wflag = reinterpret_cast<volatile int*>(smem + 2 * STAGE + 32);

  const int t = blockIdx.x;
  if (t >= ntiles) return;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const TcTile tl = tiles[t];
  const TcProb p = probs[tl.prob];
  const int m0 = tl.m0, n0 = tl.n0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TCN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // padding rows of both stages stay zero for the whole work item: zero once
  {
    uint4* z = reinterpret_cast<uint4*>(smem);
    const uint4 zero = make_uint4(0, 0, 0, 0);
    for (uint32_t i = tid; i < 2 * STAGE / 16; i += 128) z[i] = zero;
  }
  const int mv = min(TCM, p.m - m0), nv = min(TCN, p.n - n0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  int kt = 0;
  bool ok = true;
  for (int s = tl.s0; s < tl.s1 && ok; ++s) {
    const TcSeg g = segs[p.seg0 + s];
    if (g.a == 0ull && g.abuf == 0) continue;  // identity segments: epilogue
    const double* Ap = resolve(g.a, g.abuf, bases);
    const double* Bp = resolve(g.b, g.bbuf, bases);
    const double sc = g.sc;
    for (int k0 = 0; k0 < g.k; k0 += KC) {
      const int st = kt & 1;
      if (kt >= 2) {  // thread 0 waits; the outcome is shared so the block stays uniform
        if (tid == 0) *wflag = mbar_wait(&mbar[st], ((kt - 2) >> 1) & 1) ? 1 : 0;
        __syncthreads();
        if (!*wflag) { ok = false; break; }
      }
      unsigned char* sA = smem + st * STAGE;
      unsigned char* sB = sA + NS * TILE;
      // A tile: valid rows m0 .. m0+mv-1 only (padding rows are zero), K
      // positions past the segment's end written as zero
      const int kv = min(KC, g.k - k0);
      const float scf = (float)sc;
      if (g.ta) {
        for (int idx = tid; idx < KC * mv; idx += 128) {
          const int k = idx / mv, r = idx - k * mv;
          float v = 0.f;
          if (k < kv) v = scf * f64_to_f32(Ap[(size_t)(k0 + k) * g.lda + m0 + r]);
          put<MODE>(sA, tile_off<ES, KC>(r, k), TILE, v);
        }
      } else {
        for (int idx = tid; idx < KC * mv; idx += 128) {
          const int r = idx / KC, k = idx - r * KC;
          float v = 0.f;
          if (k < kv) v = scf * f64_to_f32(Ap[(size_t)(m0 + r) * g.lda + k0 + k]);
          put<MODE>(sA, tile_off<ES, KC>(r, k), TILE, v);
        }
      }
      // B tile stored N x K (K-major): element (k, n) of op(B), valid columns only
      if (g.tb) {
        for (int idx = tid; idx < KC * nv; idx += 128) {
          const int n = idx / KC, k = idx - n * KC;
          float v = 0.f;
          if (k < kv) v = f64_to_f32(Bp[(size_t)(n0 + n) * g.ldb + k0 + k]);
          put<MODE>(sB, tile_off<ES, KC>(n, k), TILE, v);
        }
      } else {
        for (int idx = tid; idx < KC * nv; idx += 128) {
          const int k = idx / nv, n = idx - k * nv;
          float v = 0.f;
          if (k < kv) v = f64_to_f32(Bp[(size_t)(k0 + k) * g.ldb + n0 + n]);
          put<MODE>(sB, tile_off<ES, KC>(n, k), TILE, v);
        }
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
        for (int kk = 0; kk < KC / KS; ++kk) {
          const uint32_t koff = kk * 2 * 128;  // two core matrices per K step
          uint64_t da = sdesc(a0 + koff, LBO, SBO), db = sdesc(b0 + koff, LBO, SBO);
          uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc(C::FMT)), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar[st]))
                     : "memory");
      }
      ++kt;
    }
  }
  if (kt > 0) {
    if (tid == 0) {
      int w = mbar_wait(&mbar[(kt - 1) & 1], ((kt - 1) >> 1) & 1) ? 1 : 0;
      if (!w) mbar_wait(&mbar[(kt - 1) & 1], ((kt - 1) >> 1) & 1);  // second bounded wait for our own MMAs
      *wflag = w;
    }
    __syncthreads();
    if (!*wflag) ok = false;
  }
  if (!ok && err && tid == 0) atomicExch(err, 1);
  tc_fence_after();
  // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w+31
  const int row = m0 + warp * 32 + lane;
  double* Cp = const_cast<double*>(resolve(p.c, p.cbuf, bases));
  for (int c0 = 0; c0 < TCN; c0 += 16) {
    float acc[16];
    if (kt > 0 && ok) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = __uint_as_float(r[j]);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = 0.f;
    }
    if (row < p.m && n0 + c0 < p.n) {
      double out[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) out[j] = f32_to_f64(acc[j]);
      for (int s = tl.s0; s < tl.s1; ++s) {  // identity segments
        const TcSeg g = segs[p.seg0 + s];
        if (!(g.a == 0ull && g.abuf == 0)) continue;
        if (g.b == 0ull && g.bbuf == 0) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (row == n0 + c0 + j) out[j] += g.sc;
        } else {
          const double* Bp = resolve(g.b, g.bbuf, bases);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = n0 + c0 + j;
            if (col < p.n) out[j] += g.sc * (g.tb ? Bp[(size_t)col * g.ldb + row] : Bp[(size_t)row * g.ldb + col]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = n0 + c0 + j;
        if (col < p.n) {
          double* dst = Cp + (size_t)row * p.ldc + col;
          if (tl.split) atomicAdd(dst, out[j]);
          else *dst = p.beta ? *dst + out[j] : out[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCN));
  }
}

template <int MODE>
size_t smem_bytes() {
  using C = Cfg<MODE>;
  return (size_t)2 * 2 * C::NSPLIT * TCM * C::KC * C::ES + 64;
}

template <int MODE>
cudaError_t launch_mode(const TcProb* P, const TcSeg* S, const TcTile* T, int nt, TcBases B, int* err,
                        cudaStream_t st) {
  static bool init = false;
  const size_t sm = smem_bytes<MODE>();
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(seg_gemm_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    init = true;
  }
  seg_gemm_tc<MODE><<<nt, 128, sm, st>>>(P, S, T, nt, B, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc(int mode, const TcProb* P, const TcSeg* S, const TcTile* T, int nt, TcBases B, int* err,
                      cudaStream_t st) {
  if (nt <= 0) return cudaSuccess;
  switch (mode) {
    case TC_TF32: return launch_mode<TC_TF32>(P, S, T, nt, B, err, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qd

// TMA-fed tcgen05 grouped GEMM of H_eff psi (BF16 and three-term BF16) for sm_103a.
//
// Operands are pre-tiled bf16 planes (tiled.hpp): every K chunk of an operand
// panel is one contiguous range, so a single cp.async.bulk per operand and
// plane moves it into a shared-memory ring slot whose mbarrier counts the
// bytes. One persistent CTA per SM walks a static list of work items with
// three roles:
//   warp 0, one lane : producer, issues the bulk copies of every K chunk into
//                      an NS-deep ring (waits until the MMAs freed the slot);
//   warp 1, one lane : issues tcgen05.mma for each chunk into one of two
//                      accumulators in tensor memory (256 FP32 columns each),
//                      tcgen05.commit frees the ring slot and, after an item's
//                      last chunk, marks its accumulator full;
//   warps 2-5        : epilogue, tcgen05.ld of the accumulator rows (warp w
//                      reads lanes 32 (w % 4) ..), then stage 1 scales, rounds
//                      to bf16 (split into three planes for BF16x3), transposes
//                      8 x 8 groups across lanes with shuffles and stores
//                      T_t^T in the tiled layout; stage 2 adds into sigma (FP64,
//                      atomics for split items). It then frees the accumulator.
// The two accumulators let the epilogue of one item overlap the MMAs of the
// next. MMA shape: M = 128 (rows past the panel are ignored), N = the view's
// rows rounded to 16 (stage 1, several views side by side in the accumulator)
// or the sigma block's columns rounded to 16 (stage 2), K = 16 per instruction.
// The shared-memory descriptors are K-major without swizzle: K-adjacent core
// matrices LBO = (panel core rows) x 128 bytes apart, M/N-adjacent ones 128
// bytes apart, exactly the order of the tiled arenas.
// BF16x3 (Henry, Tang, Heinecke, ARITH 2019): x = x0 + x1 + x2; the six
// products a_i b_j with i + j <= 2 accumulate in FP32.
// Every wait is bounded (~1 s of clock64); on a timeout the CTA records an
// error, stops issuing work, waits (bounded) for its own copies and MMAs, frees
// its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_tiled.hpp"

namespace qd {

namespace {

constexpr long long WAIT_CYCLES = 2000000000ll;
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 512;

template <int MODE>
struct TCfg;
template <>
struct TCfg<TT_BF16> {
  static constexpr int NP = 1, KC = 64, NS = 4;
};
template <>
struct TCfg<TT_BF16X3> {
  static constexpr int NP = 3, KC = 32, NS = 3;
};

template <int MODE>
struct Ring {
  static constexpr int NP = TCfg<MODE>::NP, KC = TCfg<MODE>::KC, NS = TCfg<MODE>::NS;
  static constexpr uint32_t APL = TP_A * KC * 2;         // one A plane of a slot
  static constexpr uint32_t BPL = TP_B * KC * 2;         // one B plane of a slot
  static constexpr uint32_t SLOT = NP * (APL + BPL);
  static constexpr uint32_t RING = NS * SLOT + 256;      // slack: MMA reads of a last view's padding rows
  static constexpr uint32_t BARS = RING;                 // 2 NS ring + 4 accumulator + 1 drain mbarriers
  static constexpr uint32_t SMEM = BARS + (2 * NS + 5) * 8 + 16;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false on timeout or when another role already gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// shared-memory matrix descriptor, K-major, no swizzle: lbo = byte distance of
// K-adjacent core matrices, sbo = of M/N-adjacent ones
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}
// instruction descriptor: bf16 A and B (K-major), FP32 accumulate, M = 128, N, optional negation of A
__device__ __forceinline__ uint32_t idesc_bf16(int n, int neg) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)neg << 13) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(TP_A >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(id), "r"(acc));
}
// all planes of one K step: BF16 one product, BF16x3 a_i b_j with i + j <= 2
template <int MODE>
__device__ __forceinline__ void mma_step(uint32_t tmem, uint32_t a, uint32_t b, uint32_t lboa, uint32_t lbob,
                                         uint32_t id, bool first) {
  using R = Ring<MODE>;
  if constexpr (R::NP == 1) {
    mma_bf16(tmem, sdesc(a, lboa, 128), sdesc(b, lbob, 128), id, first ? 0u : 1u);
  } else {
    const int pi[6] = {2, 1, 0, 1, 0, 0};
    const int pj[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
    for (int q = 0; q < 6; ++q)
      mma_bf16(tmem, sdesc(a + pi[q] * R::APL, lboa, 128), sdesc(b + pj[q] * R::BPL, lbob, 128), id,
               (first && q == 0) ? 0u : 1u);
  }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// 8 x 8 transpose of packed bf16 pairs across the 8 lanes of a lane group:
// lane r holds row r (elements 2k, 2k+1 in p[k]); afterwards it holds column r
__device__ __forceinline__ void transpose8(uint32_t* p, int lane) {
  const int r = lane & 7;
  {  // element distance 4 = register distance 2
    const bool hi = (r >> 2) & 1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t send = hi ? p[k] : p[k + 2];
      const uint32_t recv = __shfl_xor_sync(0xffffffffu, send, 4);
      if (hi) p[k] = recv; else p[k + 2] = recv;
    }
  }
  {  // element distance 2 = register distance 1
    const bool hi = (r >> 1) & 1;
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      const uint32_t send = hi ? p[k] : p[k + 1];
      const uint32_t recv = __shfl_xor_sync(0xffffffffu, send, 2);
      if (hi) p[k] = recv; else p[k + 1] = recv;
    }
  }
  {  // element distance 1 = halves of a register
    const bool hi = r & 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t send = hi ? (p[k] & 0xFFFFu) : (p[k] >> 16);
      const uint32_t recv = __shfl_xor_sync(0xffffffffu, send, 1);
      p[k] = hi ? ((p[k] & 0xFFFF0000u) | recv) : ((p[k] & 0xFFFFu) | (recv << 16));
    }
  }
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

struct Stage1Args {
  const K1Item* items;
  const K1View* views;
  const uint8_t* A;
  int64_t aplane;
  const uint8_t* B;
  int64_t bplane;
  uint8_t* T;
  int64_t tplane;
};
struct Stage2Args {
  const K2Item* items;
  const K2Seg* segs;
  const uint8_t* A;
  int64_t aplane;
  const uint8_t* B;
  int64_t bplane;
  double* sig;
};

template <int MODE, int STAGE, typename Args>
__global__ void __launch_bounds__(NTHREADS, 1) tiled_gemm(Args args, int nitems, int* err) {
  using R = Ring<MODE>;
  constexpr int NP = R::NP, KC = R::KC, NS = R::NS;
  extern __shared__ __align__(1024) uint8_t smem[];
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bars = sbase + R::BARS;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (NS + s); };
  auto accf = [&](int b) { return bars + 8u * (2 * NS + b); };
  auto acce = [&](int b) { return bars + 8u * (2 * NS + 2 + b); };
  const uint32_t drain = bars + 8u * (2 * NS + 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + R::BARS + (2 * NS + 5) * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + R::BARS + (2 * NS + 5) * 8 + 8);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf(b), 1);
      mbar_init(acce(b), 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int chunk = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        if constexpr (STAGE == 1) {
          const K1Item it = args.items[item];
          const int kp = tiled_c8(it.k) * 8;
          for (int k0 = 0; k0 < kp && ok; k0 += KC) {
            const int ck = min(KC, kp - k0), cc = ck / 8;
            const int slot = chunk % NS;
            if (chunk >= NS && !mbar_wait(empty(slot), ((chunk / NS) - 1) & 1, abort_flag)) { ok = false; break; }
            uint32_t bytes = (uint32_t)it.pa8 * cc * 128;
            for (int v = it.v0; v < it.v0 + it.nv; ++v) bytes += (uint32_t)args.views[v].pb8 * cc * 128;
            mbar_expect_tx(full(slot), bytes * NP);
            const uint32_t sa = sbase + slot * R::SLOT, sb = sa + NP * R::APL;
#pragma unroll
            for (int q = 0; q < NP; ++q)
              bulk_g2s(sa + q * R::APL, args.A + q * args.aplane + it.a + (int64_t)(k0 / 8) * it.pa8 * 128,
                       (uint32_t)it.pa8 * cc * 128, full(slot));
            uint32_t boff = 0;
            for (int v = it.v0; v < it.v0 + it.nv; ++v) {
              const K1View w = args.views[v];
              const uint32_t nb = (uint32_t)w.pb8 * cc * 128;
#pragma unroll
              for (int q = 0; q < NP; ++q)
                bulk_g2s(sb + q * R::BPL + boff, args.B + q * args.bplane + w.b + (int64_t)(k0 / 8) * w.pb8 * 128, nb,
                         full(slot));
              boff += nb;
            }
            ++chunk;
          }
        } else {
          const K2Item it = args.items[item];
          const int pa8 = (it.mrows + 7) / 8, pb8 = (it.nrows + 7) / 8;
          for (int s = it.s0; s < it.s1 && ok; ++s) {
            const K2Seg g = args.segs[s];
            const int c8 = tiled_c8(g.k), kp = c8 * 8;
            const int64_t ab = g.a + (int64_t)it.mp * (TP_A / 8) * c8 * 128;
            const int64_t bb = g.b + (int64_t)it.np * (TP_B / 8) * c8 * 128;
            for (int k0 = 0; k0 < kp; k0 += KC) {
              const int ck = min(KC, kp - k0), cc = ck / 8;
              const int slot = chunk % NS;
              if (chunk >= NS && !mbar_wait(empty(slot), ((chunk / NS) - 1) & 1, abort_flag)) { ok = false; break; }
              const uint32_t na = (uint32_t)pa8 * cc * 128, nb = (uint32_t)pb8 * cc * 128;
              mbar_expect_tx(full(slot), (na + nb) * NP);
              const uint32_t sa = sbase + slot * R::SLOT, sb = sa + NP * R::APL;
#pragma unroll
              for (int q = 0; q < NP; ++q) {
                bulk_g2s(sa + q * R::APL, args.A + q * args.aplane + ab + (int64_t)(k0 / 8) * pa8 * 128, na, full(slot));
                bulk_g2s(sb + q * R::BPL, args.B + q * args.bplane + bb + (int64_t)(k0 / 8) * pb8 * 128, nb, full(slot));
              }
              ++chunk;
            }
          }
        }
      }
      if (!ok) {
        atomicExch(err, 1);
        *abort_flag = 1;
      }
      // no copy of ours may still be in flight when the CTA exits
      for (int c = chunk - 1; c >= 0 && c >= chunk - NS; --c) {
        const long long t0 = clock64();
        while (!mbar_try(full(c % NS), (c / NS) & 1) && clock64() - t0 < WAIT_CYCLES) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int chunk = 0, li = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
        const int b = li & 1;
        if (li >= 2 && !mbar_wait(acce(b), ((li >> 1) - 1) & 1, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tacc = tmem + (uint32_t)b * 256u;
        if constexpr (STAGE == 1) {
          const K1Item it = args.items[item];
          const int kp = tiled_c8(it.k) * 8;
          bool first = true;
          for (int k0 = 0; k0 < kp; k0 += KC) {
            const int ck = min(KC, kp - k0), cc = ck / 8;
            const int slot = chunk % NS;
            if (!mbar_wait(full(slot), (chunk / NS) & 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = sbase + slot * R::SLOT, sb = sa + NP * R::APL;
            const uint32_t lboa = (uint32_t)it.pa8 * 128;
            for (int kk = 0; kk < ck / 16; ++kk) {
              uint32_t boff = 0;
              for (int v = it.v0; v < it.v0 + it.nv; ++v) {
                const K1View w = args.views[v];
                const uint32_t lbob = (uint32_t)w.pb8 * 128;
                const int n = 16 * ((w.nrows + 15) / 16);
                mma_step<MODE>(tacc + (uint32_t)w.ncol, sa + kk * 2 * lboa, sb + boff + kk * 2 * lbob, lboa, lbob,
                               idesc_bf16(n, 0), first && kk == 0);
                boff += (uint32_t)w.pb8 * cc * 128;
              }
            }
            first = false;
            tc_commit(empty(slot));
            ++chunk;
          }
        } else {
          const K2Item it = args.items[item];
          const int pa8 = (it.mrows + 7) / 8, pb8 = (it.nrows + 7) / 8;
          const int n = 16 * ((it.nrows + 15) / 16);
          const uint32_t lboa = (uint32_t)pa8 * 128, lbob = (uint32_t)pb8 * 128;
          bool first = true;
          for (int s = it.s0; s < it.s1 && ok; ++s) {
            const K2Seg g = args.segs[s];
            const int kp = tiled_c8(g.k) * 8;
            const uint32_t id = idesc_bf16(n, g.neg);
            for (int k0 = 0; k0 < kp; k0 += KC) {
              const int ck = min(KC, kp - k0);
              const int slot = chunk % NS;
              if (!mbar_wait(full(slot), (chunk / NS) & 1, abort_flag)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sa = sbase + slot * R::SLOT, sb = sa + NP * R::APL;
              for (int kk = 0; kk < ck / 16; ++kk) {
                mma_step<MODE>(tacc, sa + kk * 2 * lboa, sb + kk * 2 * lbob, lboa, lbob, id, first);
                first = false;
              }
              tc_commit(empty(slot));
              ++chunk;
            }
          }
        }
        if (!ok) break;
        tc_commit(accf(b));
      }
      if (!ok) {
        atomicExch(err, 1);
        *abort_flag = 1;
      }
      // every MMA of ours completes before the tensor memory is freed
      tc_commit(drain);
      const long long t0 = clock64();
      while (!mbar_try(drain, 0) && clock64() - t0 < WAIT_CYCLES) {
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quarter = warp & 3;
    const int m = quarter * 32 + lane;  // accumulator row (lane) within the panel
    int li = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++li) {
      const int b = li & 1;
      // the warp decides together: tcgen05.ld below is warp-collective
      const bool okw = __all_sync(0xffffffffu, mbar_wait(accf(b), (li >> 1) & 1, abort_flag));
      if (!okw) {
        if (lane == 0) atomicExch(err, 1);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * 256u;
      if constexpr (STAGE == 1) {
        const K1Item it = args.items[item];
        const bool mval = m < it.mrows;
        const int c8t = tiled_c8(it.mtot);
        const int m8 = (m & ~7);
        const bool group_live = m8 < it.mrows;  // the 16-byte unit holds a valid K position
        const int jc = (it.mp * TP_A + m8) / 8;
        for (int v = it.v0; v < it.v0 + it.nv; ++v) {
          const K1View w = args.views[v];
          const float osc = (float)w.osc;
          for (int c0 = 0; c0 < w.nrows; c0 += 8) {
            float x[8];
            tmem_ld8(trow + (uint32_t)(w.ncol + c0), x);
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = mval ? osc * x[j] : 0.f;
            const int rrow = c0 + (lane & 7);          // row of T^T within this panel after the transpose
            const bool store = group_live && rrow < w.nrows;
            const int R = w.np * TP_B + rrow;
            uint8_t* dst = args.T + w.tout + (int64_t)w.np * (TP_B / 8) * c8t * 128 + (int64_t)jc * w.pb8 * 128 +
                           ((R % TP_B) / 8) * 128 + (R % 8) * 16;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              uint32_t p[4];
              float r[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const uint32_t h = bf16_bits(x[j]);
                r[j] = x[j] - __uint_as_float(h << 16);
                if (j & 1) p[j >> 1] |= h << 16; else p[j >> 1] = h;
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) x[j] = r[j];
              transpose8(p, lane);
              if (store) *reinterpret_cast<uint4*>(dst + q * args.tplane) = make_uint4(p[0], p[1], p[2], p[3]);
            }
          }
        }
      } else {
        const K2Item it = args.items[item];
        const bool mval = m < it.mrows;
        double* row = args.sig + it.out + (int64_t)(it.mp * TP_A + m) * it.ldc + it.np * TP_B;
        for (int c0 = 0; c0 < it.nrows; c0 += 8) {
          float x[8];
          tmem_ld8(trow + (uint32_t)c0, x);
          if (mval) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              if (c0 + j < it.nrows) {
                if (it.split) atomicAdd(row + c0 + j, (double)x[j]);
                else row[c0 + j] += (double)x[j];
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce(b));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// FP64 views -> tiled bf16 planes. One CTA per view; one thread per 16-byte
// row of a core matrix (8 consecutive K elements of one row).
__global__ void __launch_bounds__(256) tile_views_kernel(const TView* __restrict__ views, uint8_t* dst,
                                                         int64_t plane, int planes, const double* psi) {
  const TView v = views[blockIdx.x];
  const int c8 = tiled_c8(v.cols);
  const int P = v.panel, P8 = P / 8;
  int r8 = 0;
  for (int p = 0; p < v.rows; p += P) r8 += (min(P, v.rows - p) + 7) / 8;
  const int64_t units = (int64_t)r8 * c8 * 8;
  const double* src = v.buf ? psi + v.src : reinterpret_cast<const double*>(v.src);
  for (int64_t u = threadIdx.x; u < units; u += blockDim.x) {
    const int rr = (int)(u & 7);
    const int64_t cu = u >> 3;
    const int j = (int)(cu % c8);
    const int cr = (int)(cu / c8);                  // core row over all panels
    const int p = cr / P8, i = cr - p * P8;
    const int pr8 = (min(P, v.rows - p * P) + 7) / 8;
    const int r = p * P + i * 8 + rr;
    uint32_t w[3][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c = j * 8 + e;
      double x = 0.0;
      if (r < v.rows && c < v.cols) {
        if (v.src == 0 && v.buf == 0) x = (r == c) ? v.scale : 0.0;
        else x = v.scale * (v.tr ? src[(int64_t)c * v.ld + r] : src[(int64_t)r * v.ld + c]);
      }
      double rem = x;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const __nv_bfloat16 h = __double2bfloat16(rem);
        rem -= (double)__bfloat162float(h);
        const uint32_t hb = (uint32_t)__bfloat16_as_ushort(h);
        if (e & 1) w[q][e >> 1] |= hb << 16; else w[q][e >> 1] = hb;
      }
    }
    uint8_t* o = dst + v.dst + (int64_t)p * P8 * c8 * 128 + (int64_t)j * pr8 * 128 + i * 128 + rr * 16;
    for (int q = 0; q < planes; ++q)
      *reinterpret_cast<uint4*>(o + q * plane) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  }
}

template <int MODE, int STAGE, typename Args>
cudaError_t launch(Args a, int nitems, int grid, int* err, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  constexpr uint32_t sm = Ring<MODE>::SMEM;
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(tiled_gemm<MODE, STAGE, Args>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    init = true;
  }
  tiled_gemm<MODE, STAGE, Args><<<std::min(grid, nitems), NTHREADS, sm, st>>>(a, nitems, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_views(const TView* views, int nviews, uint8_t* dst, int64_t plane_bytes, int planes,
                              const double* psi_base, cudaStream_t st) {
  if (nviews <= 0) return cudaSuccess;
  tile_views_kernel<<<nviews, 256, 0, st>>>(views, dst, plane_bytes, planes, psi_base);
  return cudaGetLastError();
}

cudaError_t launch_tiled_stage1(int mode, const K1Item* items, int nitems, const K1View* views,
                                const uint8_t* psi_arena, int64_t psi_plane, const uint8_t* b_arena,
                                int64_t b_plane, uint8_t* t_arena, int64_t t_plane, int grid, int* err,
                                cudaStream_t st) {
  Stage1Args a{items, views, psi_arena, psi_plane, b_arena, b_plane, t_arena, t_plane};
  if (mode == TT_BF16) return launch<TT_BF16, 1>(a, nitems, grid, err, st);
  if (mode == TT_BF16X3) return launch<TT_BF16X3, 1>(a, nitems, grid, err, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tiled_stage2(int mode, const K2Item* items, int nitems, const K2Seg* segs,
                                const uint8_t* a_arena, int64_t a_plane, const uint8_t* t_arena,
                                int64_t t_plane, double* sigma, int grid, int* err, cudaStream_t st) {
  Stage2Args a{items, segs, a_arena, a_plane, t_arena, t_plane, sigma};
  if (mode == TT_BF16) return launch<TT_BF16, 2>(a, nitems, grid, err, st);
  if (mode == TT_BF16X3) return launch<TT_BF16X3, 2>(a, nitems, grid, err, st);
  return cudaErrorInvalidValue;
}

}  // namespace qd

// Bulk-copy-fed tcgen05 grouped GEMM of H_eff psi (BF16 and three-term BF16) for sm_103a.
//
// Operands are pre-tiled bf16 planes (tiled.hpp): every K chunk of an operand
// panel is one contiguous range, so a single cp.async.bulk per operand and
// plane moves it into shared memory. One persistent CTA per SM walks a static
// list of work items with three roles:
//   warp 0   : producer. Reserves each chunk in a byte ring of shared memory
//              (chunks take exactly their bytes, so many small chunks are in
//              flight), writes the chunk's MMA list (ready shared-memory
//              descriptors) into one of NR records, arms the record's mbarrier
//              with the byte count and issues the bulk copies from several
//              lanes at once (stage 1: one lane per view, the psi panel by
//              lanes 16..; stage 2: up to 16 short segments packed into one
//              chunk, A pieces by their own lanes, B pieces by lane ^ 16).
//              Work-item descriptors are prefetched two items ahead, views and
//              segment batches one step ahead.
//   warp 1   : lane 0 of the converged warp issues tcgen05.mma from the
//              records into one of two accumulators in tensor memory (256 FP32
//              columns each); every fourth chunk (and every record without
//              data) commits to its record's mbarrier, which frees the ring
//              bytes of all chunks before it; after an item's last chunk a
//              commit marks the accumulator full.
//   warps 2-9: epilogue, two warps per tensor-memory lane quarter splitting the
//              columns. Stage 1 scales T_t^T rows, rounds them to bf16 (three
//              planes for BF16x3) and stores 16-byte core-matrix rows; stage 2
//              adds into sigma (FP64, atomics for split items). Then the
//              accumulator is released.
// Stage 1 computes T_t^T = O_R psi_blk^T (accumulator lane = row of T_t^T), so
// no transposition is needed to produce the stage-2 B operand.
// MMA shape: M = 128 (rows past the panel are ignored), N = the B panel's rows
// rounded to 16, K = 16 per instruction. Shared-memory descriptors are K-major
// without swizzle: K-adjacent core matrices LBO = (panel core rows) x 128 bytes
// apart, M/N-adjacent ones 128 bytes apart, the order of the tiled arenas.
// BF16x3 (Henry, Tang, Heinecke, ARITH 2019): x = x0 + x1 + x2; the six
// products a_i b_j with i + j <= 2 accumulate in FP32.
// Every wait is bounded (~1 s of clock64); on a timeout the CTA records an
// error, stops issuing work, waits (bounded) for its own copies and MMAs, frees
// its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "tc_tiled.hpp"

namespace qd {

namespace {

constexpr long long WAIT_CYCLES = 2000000000ll;
constexpr int NEPI = 8;                     // epilogue warps
constexpr int NTHREADS = 64 + 32 * NEPI;
constexpr uint32_t TMEM_COLS = 512;

template <int MODE>
struct TCfg;
template <>
struct TCfg<TT_BF16> {
  static constexpr int NP = 1, KC = 64;   // planes, K elements per chunk
};
template <>
struct TCfg<TT_BF16X3> {
  static constexpr int NP = 3, KC = 32;
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
// bounded wait that yields the issue slots between polls (for the epilogue
// warps, which share their schedulers with the producer and MMA lanes)
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) return false;
    __nanosleep(100);
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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

struct Stage1Args {
  const K1Item* items;
  const K1View* views;
  const uint8_t* A;    // right-view arena (A operands)
  int64_t aplane;
  const uint8_t* B;    // psi arena (B operand)
  int64_t bplane;
  uint8_t* T;
  int64_t tplane;
  int kcb;             // chunk byte target (0: KC elements of K per chunk)
};
struct Stage2Args {
  const K2Item* items;
  const K2Seg* segs;
  const uint8_t* A;    // left-view arena
  int64_t aplane;
  const uint8_t* B;    // T arena
  int64_t bplane;
  double* sig;
  int kcb;             // chunk byte target (0: KC elements of K per chunk)
};

// One chunk as the MMA issuer sees it: up to MAXOPS (A, B) pairs, each over
// its own nk16 K steps into accumulator columns from tcol (stage 1: one
// column range per view; stage 2: all ops of an item add into the same
// columns, several short segments packed into one chunk). The planes of an
// operand follow each other at astride / bstride bytes; zero: the op's first
// K step overwrites the accumulator instead of adding. The producer stores
// ready shared-memory descriptors and their increments (16-byte units) per
// K step and per plane, so that the issuing thread only adds and issues.
constexpr int MAXOPS = 16;
struct Op {
  uint64_t da, db;          // descriptors of the first K step, plane 0
  uint32_t idesc, tcol, nk16, zero;
  uint32_t ka, kb;          // descriptor increment per K step
  uint32_t pa, pb;          // descriptor increment per plane
};
struct Meta {
  uint32_t nops, flags, li, pad;
  Op op[MAXOPS];
};
// F_COMMIT: the MMA issuer commits the chunk's record to its empty barrier
// (every 4th chunk and every record without data; one commit releases the
// ring bytes of all chunks before it)
constexpr uint32_t F_FIRST = 1, F_LAST = 2, F_END = 4, F_COMMIT = 8;

template <int MODE>
struct Smem {
  static constexpr int NP = TCfg<MODE>::NP, KC = TCfg<MODE>::KC;
  static constexpr uint32_t RB = 196608;      // byte ring of chunk data
  static constexpr uint32_t SLACK = 2048;     // MMA reads of padding rows past a chunk's end
  static constexpr int NR = 32;               // chunk records in flight
  static constexpr uint32_t PACK = 32768;     // bytes of one chunk of packed stage-2 segments
  static constexpr uint32_t META = RB + SLACK;
  static constexpr uint32_t BARS = META + NR * sizeof(Meta);
  static constexpr uint32_t VEND = BARS + (2 * NR + 5) * 8 + 16;  // ring ends of the records in flight
  static constexpr uint32_t ECNT = VEND + NR * 8;                  // commits consumed per record
  static constexpr uint32_t VCM = ECNT + NR * 4;                   // record holds a commit point
  static constexpr uint32_t SMEM = VCM + NR;
};

// K elements per chunk of a work item: KC, or with a byte target kcb > 0 the
// largest multiple of 16 (at most 256) whose chunk of per8 bytes per 8 K
// elements stays within kcb; never fewer than KC. Fewer, larger chunks cut the
// producer's and the MMA issuer's per-chunk work on small operand panels.
template <int KC>
__device__ __forceinline__ int chunk_depth(int kcb, int per8) {
  if (kcb <= 0) return KC;
  return min(256, max(KC, 16 * (kcb / (2 * per8))));
}

__device__ __forceinline__ void set_op(Op& o, uint32_t a, uint32_t b, uint32_t lboa, uint32_t lbob, uint32_t idesc,
                                       uint32_t tcol, uint32_t nk16, uint32_t astride, uint32_t bstride, uint32_t zero) {
  o.da = sdesc(a, lboa, 128);
  o.db = sdesc(b, lbob, 128);
  o.idesc = idesc;
  o.tcol = tcol;
  o.nk16 = nk16;
  o.zero = zero;
  o.ka = (2 * lboa) >> 4;
  o.kb = (2 * lbob) >> 4;
  o.pa = astride >> 4;
  o.pb = bstride >> 4;
}

// one K step of an op (all planes of the split form)
template <int MODE>
__device__ __forceinline__ void mma_step(uint32_t tmem, uint64_t da, uint64_t db, const Op& o, bool first) {
  if constexpr (TCfg<MODE>::NP == 1) {
    mma_bf16(tmem, da, db, o.idesc, first ? 0u : 1u);
  } else {
    const uint32_t pi[6] = {2, 1, 0, 1, 0, 0};
    const uint32_t pj[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
    for (int q = 0; q < 6; ++q)
      mma_bf16(tmem, da + pi[q] * o.pa, db + pj[q] * o.pb, o.idesc, (first && q == 0) ? 0u : 1u);
  }
}

__device__ __forceinline__ int64_t shfl64(int64_t v, int src) {
  const int lo = __shfl_sync(0xffffffffu, (int)(v & 0xffffffff), src);
  const int hi = __shfl_sync(0xffffffffu, (int)(v >> 32), src);
  return ((int64_t)hi << 32) | (uint32_t)lo;
}

// Producer-side byte ring: chunk c takes [vs, vs + size) of a virtual byte
// stream (never wrapping inside the ring) and record c % NR; both are reused
// once the MMAs of the chunks before it have completed (freed in order).
// Completion is known at commit points only (every 4th chunk); when the
// producer must wait and none of its chunks in flight is a commit point, it
// inserts a record without data that only commits.
template <int MODE>
struct RingAlloc {
  using S = Smem<MODE>;
  uint64_t vhead = 0, freed = 0;
  long long chunk = 0, oldest = 0;
  uint64_t* vend;   // NR entries in shared memory
  uint32_t* ecnt;   // commits consumed per record
  uint8_t* vcm;     // record's chunk is a commit point
  static __device__ __forceinline__ bool commit_point(long long c) { return (c & 3) == 3; }
  // lane 0 only; false on a timeout
  __device__ bool reserve(uint32_t size, uint32_t& off, uint32_t bars, volatile int* abort_flag, Meta* meta,
                          uint32_t li) {
    uint64_t vs = vhead;
    if ((vs % S::RB) + size > S::RB) vs = (vs / S::RB + 1) * S::RB;
    const uint64_t ve = vs + size;
    while (oldest < chunk && (oldest <= chunk - S::NR || ve > freed + S::RB)) {
      long long c = oldest;
      while (c < chunk && !vcm[c % S::NR]) ++c;
      if (c == chunk) {
        // fewer than 4 chunks in flight and none commits: a commit-only record
        const int r = (int)(chunk % S::NR);
        meta[r].nops = 0;
        meta[r].flags = F_COMMIT;
        meta[r].li = li;
        vend[r] = vhead;
        vcm[r] = 1;
        mbar_arrive(bars + 8u * r);
        ++chunk;
        continue;
      }
      const int r = (int)(c % S::NR);
      if (!mbar_wait(bars + 8u * (S::NR + r), ecnt[r] & 1u, abort_flag)) return false;
      ++ecnt[r];
      freed = vend[r];
      oldest = c + 1;
    }
    vend[chunk % S::NR] = ve;
    vcm[chunk % S::NR] = commit_point(chunk) ? 1 : 0;
    vhead = ve;
    off = (uint32_t)(vs % S::RB);
    return true;
  }
};

template <int MODE, int STAGE, typename Args>
__global__ void __launch_bounds__(NTHREADS, 1) tiled_gemm(Args args, int nitems, int* err) {
  using S = Smem<MODE>;
  constexpr int NP = S::NP, KC = S::KC, NR = S::NR;
  extern __shared__ __align__(1024) uint8_t smem[];
  const uint32_t sbase = smem_u32(smem);
  Meta* meta = reinterpret_cast<Meta*>(smem + S::META);
  const uint32_t bars = sbase + S::BARS;
  auto full = [&](int r) { return bars + 8u * r; };
  auto empty = [&](int r) { return bars + 8u * (NR + r); };
  auto accf = [&](int b) { return bars + 8u * (2 * NR + b); };
  auto acce = [&](int b) { return bars + 8u * (2 * NR + 2 + b); };
  const uint32_t drain = bars + 8u * (2 * NR + 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::BARS + (2 * NR + 5) * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + S::BARS + (2 * NR + 5) * 8 + 8);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int r = 0; r < NR; ++r) {
      mbar_init(full(r), 1);
      mbar_init(empty(r), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf(b), 1);
      mbar_init(acce(b), NEPI);
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
    // ---------------- producer (whole warp; lane 0 waits and signals) ----------------
    RingAlloc<MODE> ring;
    ring.vend = reinterpret_cast<uint64_t*>(smem + S::VEND);
    ring.ecnt = reinterpret_cast<uint32_t*>(smem + S::ECNT);
    ring.vcm = smem + S::VCM;
    if (lane < NR) ring.ecnt[lane] = 0;
    __syncwarp();
    bool ok = true;
    int li = 0;
    // reserve the next chunk; the outcome is shared by the warp
    auto next = [&](uint32_t size, uint32_t& off) -> bool {
      int good = 1;
      uint32_t o = 0;
      if (lane == 0) good = ring.reserve(size, o, bars, abort_flag, meta, (uint32_t)li) ? 1 : 0;
      good = __shfl_sync(0xffffffffu, good, 0);
      off = __shfl_sync(0xffffffffu, o, 0);
      ring.chunk = shfl64(ring.chunk, 0);  // lane 0 may have inserted commit-only records
      return good != 0;
    };
    // Descriptor prefetch: work-item descriptors two items ahead, the views
    // (stage 1) or the first 32 segments (stage 2) of the next item one item
    // ahead, so that no item starts with two dependent global loads.
    using Item = typename std::conditional<STAGE == 1, K1Item, K2Item>::type;
    using Sub = typename std::conditional<STAGE == 1, K1View, K2Seg>::type;
    auto load_item = [&](int i) {
      Item x{};
      if (i < nitems) x = args.items[i];
      return x;
    };
    auto load_sub = [&](const Item& x) {
      Sub y{};
      if constexpr (STAGE == 1) {
        if (lane < x.nv) y = args.views[x.v0 + lane];
      } else {
        if (lane < x.s1 - x.s0) y = args.segs[x.s0 + lane];
      }
      return y;
    };
    Item it_n = load_item(blockIdx.x);
    Sub sub_n = load_sub(it_n);
    Item it_n2 = load_item(blockIdx.x + gridDim.x);
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
      const Item it = it_n;
      const Sub sub0 = sub_n;
      it_n = it_n2;
      sub_n = load_sub(it_n);
      it_n2 = load_item(item + 2 * gridDim.x);
      if constexpr (STAGE == 1) {
        const K1View mv = sub0;
        const int kp = tiled_c8(it.k) * 8;
        const int kc = chunk_depth<KC>(
            args.kcb, NP * ((int)__reduce_add_sync(0xffffffffu, lane < it.nv ? (unsigned)mv.pa8 : 0u) + it.pb8) * 128);
        for (int k0 = 0; k0 < kp && ok; k0 += kc) {
          const int ck = min(kc, kp - k0), cc = ck / 8;
          // A parts of the views side by side (exclusive prefix over lanes), then B
          const uint32_t mine = lane < it.nv ? (uint32_t)mv.pa8 * cc * 128 : 0u;
          uint32_t pre = mine;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, pre, d);
            if (lane >= d) pre += t;
          }
          const uint32_t atot = __shfl_sync(0xffffffffu, pre, 31);
          pre -= mine;
          const uint32_t bsz = (uint32_t)it.pb8 * cc * 128;
          uint32_t off;
          if (!next(NP * (atot + bsz), off)) { ok = false; break; }
          const int r = (int)(ring.chunk % NR);
          const uint32_t ca = sbase + off, cb = ca + NP * atot;
          if (lane < it.nv) {
            Op& o = meta[r].op[lane];
            set_op(o, ca + pre, cb, (uint32_t)mv.pa8 * 128, (uint32_t)it.pb8 * 128,
                   idesc_bf16(16 * ((it.nrows + 15) / 16), 0), (uint32_t)mv.tcol, (uint32_t)(ck / 16), atot, bsz,
                   k0 == 0 ? 1u : 0u);
          }
          if (lane == 0) {
            meta[r].nops = (uint32_t)it.nv;
            meta[r].flags = (k0 == 0 ? F_FIRST : 0u) | (k0 + kc >= kp ? F_LAST : 0u) |
                            (RingAlloc<MODE>::commit_point(ring.chunk) ? F_COMMIT : 0u);
            meta[r].li = (uint32_t)li;
          }
          __syncwarp();
          if (lane == 0) mbar_expect_tx(full(r), NP * (atot + bsz));
          __syncwarp();
          if (lane < it.nv) {
#pragma unroll
            for (int q = 0; q < NP; ++q)
              bulk_g2s(ca + q * atot + pre, args.A + q * args.aplane + mv.a + (int64_t)(k0 / 8) * mv.pa8 * 128, mine,
                       full(r));
          }
          // the psi panel's planes by lanes 16.. (views use lanes < 16), so that
          // the copies issue in parallel
          if (lane >= 16 && lane < 16 + NP) {
            const int q = lane - 16;
            bulk_g2s(cb + q * bsz, args.B + q * args.bplane + it.b + (int64_t)(k0 / 8) * it.pb8 * 128, bsz, full(r));
          }
          ring.chunk++;
          __syncwarp();
        }
      } else {
        const int pa8 = (it.mrows + 7) / 8, pb8 = (it.nrows + 7) / 8;
        const uint32_t id = idesc_bf16(16 * ((it.nrows + 15) / 16), 0);
        const int kc = chunk_depth<KC>(args.kcb, NP * (pa8 + pb8) * 128);
        const uint32_t pack = max(S::PACK, (uint32_t)max(args.kcb, 0));
        bool first = true;  // no chunk of this item issued yet
        K2Seg mg_n = sub0;  // segments of the next batch (loaded one batch ahead)
        for (int sb = it.s0; sb < it.s1 && ok; sb += 32) {
          const int cnt = min(32, it.s1 - sb);
          const K2Seg mg = mg_n;
          mg_n = K2Seg{};
          if (sb + 32 + lane < it.s1) mg_n = args.segs[sb + 32 + lane];
          // this lane's segment as one piece of a packed chunk (0: K longer
          // than one chunk, or no segment)
          const int mkp = tiled_c8(mg.k) * 8;
          const uint32_t mna = (uint32_t)pa8 * (mkp / 8) * 128, mnb = (uint32_t)pb8 * (mkp / 8) * 128;
          const uint32_t msz = (lane < cnt && mkp > 0 && mkp <= kc) ? NP * (mna + mnb) : 0u;
          // inclusive prefix sum of the piece sizes over the lanes
          uint32_t cum = msz;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, cum, d);
            if (lane >= d) cum += t;
          }
          int j = 0;
          while (j < cnt && ok) {
            const int k = __shfl_sync(0xffffffffu, mg.k, j);
            const int kp = tiled_c8(k) * 8;
            if (kp == 0) {
              ++j;
              continue;
            }
            if (kp > kc) {
              // a long segment: chunks of kc along K, one op each
              const int64_t ga = shfl64(mg.a, j), gb = shfl64(mg.b, j);
              const int c8 = kp / 8;
              const int64_t ab = ga + (int64_t)it.mp * (TP_A / 8) * c8 * 128;
              const int64_t bb = gb + (int64_t)it.np * (TP_B / 8) * c8 * 128;
              for (int k0 = 0; k0 < kp; k0 += kc) {
                const int ck = min(kc, kp - k0), cc = ck / 8;
                const uint32_t na = (uint32_t)pa8 * cc * 128, nb = (uint32_t)pb8 * cc * 128;
                uint32_t off;
                if (!next(NP * (na + nb), off)) { ok = false; break; }
                const int r0 = (int)(ring.chunk % NR);
                if (lane == 0) {
                  const int r = r0;
                  const uint32_t ca = sbase + off, cb = ca + NP * na;
                  Op& o = meta[r].op[0];
                  set_op(o, ca, cb, (uint32_t)pa8 * 128, (uint32_t)pb8 * 128, id, 0u, (uint32_t)(ck / 16), na, nb,
                         first ? 1u : 0u);
                  meta[r].nops = 1;
                  meta[r].flags = (first ? F_FIRST : 0u) | (sb + j == it.s1 - 1 && k0 + kc >= kp ? F_LAST : 0u) |
                                  (RingAlloc<MODE>::commit_point(ring.chunk) ? F_COMMIT : 0u);
                  meta[r].li = (uint32_t)li;
                  mbar_expect_tx(full(r), NP * (na + nb));
                }
                __syncwarp();
                // plane q of A by lane q, of B by lane NP + q
                if (lane < 2 * NP) {
                  const int q = lane % NP;
                  const uint32_t ca = sbase + off, cb = ca + NP * na;
                  if (lane < NP)
                    bulk_g2s(ca + q * na, args.A + q * args.aplane + ab + (int64_t)(k0 / 8) * pa8 * 128, na, full(r0));
                  else
                    bulk_g2s(cb + q * nb, args.B + q * args.bplane + bb + (int64_t)(k0 / 8) * pb8 * 128, nb, full(r0));
                }
                first = false;
                ring.chunk++;
                __syncwarp();
              }
              ++j;
              continue;
            }
            // short segments j .. j2-1 packed into one chunk, one op each: the
            // group ends before the first lane whose piece is not short, would
            // overflow the pack size (PACK, or the chunk byte target when it is
            // larger), or is the (MAXOPS+1)-th
            const uint32_t base = __shfl_sync(0xffffffffu, cum - msz, j);
            const unsigned stop = __ballot_sync(0xffffffffu, lane > j && (msz == 0 || cum - base > pack ||
                                                                         lane - j >= MAXOPS));
            const int j2 = min(cnt, stop ? __ffs(stop) - 1 : 32);
            const uint32_t tot = __shfl_sync(0xffffffffu, cum, j2 - 1) - base;
            const bool in = lane >= j && lane < j2;
            uint32_t off;
            if (!next(tot, off)) { ok = false; break; }
            const int r = (int)(ring.chunk % NR);
            const uint32_t ca = sbase + off + (cum - msz - base), cb = ca + NP * mna;
            if (in) {
              Op& o = meta[r].op[lane - j];
              set_op(o, ca, cb, (uint32_t)pa8 * 128, (uint32_t)pb8 * 128, id, 0u, (uint32_t)(mkp / 16), mna, mnb,
                     (first && lane == j) ? 1u : 0u);
            }
            if (lane == 0) {
              meta[r].nops = (uint32_t)(j2 - j);
              meta[r].flags = (first ? F_FIRST : 0u) | (sb + j2 == it.s1 ? F_LAST : 0u) |
                              (RingAlloc<MODE>::commit_point(ring.chunk) ? F_COMMIT : 0u);
              meta[r].li = (uint32_t)li;
            }
            __syncwarp();
            if (lane == 0) mbar_expect_tx(full(r), tot);
            __syncwarp();
            {
              // A pieces by their own lanes, B pieces by the partner lane
              // (lane ^ 16: a group spans at most 16 lanes, so no lane issues
              // both), so that every lane issues at most one piece
              const int c8 = mkp / 8;
              const int64_t ab = mg.a + (int64_t)it.mp * (TP_A / 8) * c8 * 128;
              const int64_t bb = mg.b + (int64_t)it.np * (TP_B / 8) * c8 * 128;
              const int64_t pbb = shfl64(bb, lane ^ 16);
              const uint32_t pcb = __shfl_sync(0xffffffffu, cb, lane ^ 16);
              const uint32_t pnb = __shfl_sync(0xffffffffu, mnb, lane ^ 16);
              const bool pin = __shfl_sync(0xffffffffu, in ? 1 : 0, lane ^ 16) != 0;
              if (in) {
#pragma unroll
                for (int q = 0; q < NP; ++q) bulk_g2s(ca + q * mna, args.A + q * args.aplane + ab, mna, full(r));
              }
              if (pin) {
#pragma unroll
                for (int q = 0; q < NP; ++q) bulk_g2s(pcb + q * pnb, args.B + q * args.bplane + pbb, pnb, full(r));
              }
            }
            first = false;
            ring.chunk++;
            __syncwarp();
            j = j2;
          }
        }
      }
    }
    if (ok) {
      // end-of-work record for the MMA issuer
      uint32_t off;
      if (next(0, off)) {
        if (lane == 0) {
          const int r = (int)(ring.chunk % NR);
          meta[r].nops = 0;
          meta[r].flags = F_END;
          mbar_arrive(full(r));
        }
        ring.chunk++;
      } else {
        ok = false;
      }
    }
    if (lane == 0) {
      if (!ok) {
        atomicExch(err, 1);
        *abort_flag = 1;
      }
      // no copy of ours may still be in flight when the CTA exits
      for (long long c = ring.oldest; c < ring.chunk; ++c) {
        const long long t0 = clock64();
        while (!mbar_try(full((int)(c % NR)), (uint32_t)((c / NR) & 1)) && clock64() - t0 < WAIT_CYCLES) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // The whole warp runs the loop and lane 0 issues: a tcgen05.mma issues in
    // about half the time when the warp-mates of the issuing lane wait at a
    // nearby __syncwarp rather than at the CTA barrier. Every lane waits on
    // the barriers itself (its own acquire of the chunk record), and the warp
    // agrees on the outcome.
    bool ok = true;
    for (long long c = 0;; ++c) {
      const int r = (int)(c % NR);
      if (!__all_sync(0xffffffffu, mbar_wait(full(r), (uint32_t)((c / NR) & 1), abort_flag))) {
        ok = false;
        break;
      }
      const uint32_t flags = meta[r].flags;
      if (flags & F_END) break;
      const int li = (int)meta[r].li, b = li & 1;
      if ((flags & F_FIRST) && li >= 2 &&
          !__all_sync(0xffffffffu, mbar_wait(acce(b), (uint32_t)(((li >> 1) - 1) & 1), abort_flag))) {
        ok = false;
        break;
      }
      tc_fence_after();
      // lane 0 issues the chunk's MMAs back to back (no warp barrier between
      // them); the warp meets again after the commits
      if (lane == 0) {
        const uint32_t tacc = tmem + (uint32_t)b * 256u;
        const int nops = (int)meta[r].nops;
        for (int o = 0; o < nops; ++o) {
          const Op op = meta[r].op[o];
          uint64_t da = op.da, db = op.db;
          for (int kk = 0; kk < (int)op.nk16; ++kk) {
            mma_step<MODE>(tacc + op.tcol, da, db, op, op.zero && kk == 0);
            da += op.ka;
            db += op.kb;
          }
        }
        if (flags & F_COMMIT) tc_commit(empty(r));
        if (flags & F_LAST) tc_commit(accf(b));
      }
      __syncwarp();
    }
    if (lane == 0) {
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
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2 .. 2 + NEPI - 1) ----------------
    const int quarter = warp & 3;            // tensor-memory lanes this warp may read
    const int half = (warp - 2) >> 2;        // two warps per lane quarter split the columns
    const int m = quarter * 32 + lane;       // accumulator row
    int li = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++li) {
      const int b = li & 1;
      // descriptors are fetched before the wait, so their latency overlaps it
      // (stage 1: lane j holds view j of the item)
      using Item = typename std::conditional<STAGE == 1, K1Item, K2Item>::type;
      const Item it = args.items[item];
      K1View mv{};
      if constexpr (STAGE == 1) {
        if (lane < it.nv) mv = args.views[it.v0 + lane];
      }
      const bool okw = __all_sync(0xffffffffu, mbar_wait_sleep(accf(b), (uint32_t)((li >> 1) & 1), abort_flag));
      if (!okw) {
        if (lane == 0) atomicExch(err, 1);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * 256u;
      if constexpr (STAGE == 1) {
        const int c8t = tiled_c8(it.mtot);
        const int ng16 = (it.nrows + 15) / 16;   // 16-column groups (within the view's accumulator columns)
        for (int vi = half; vi < it.nv; vi += 2) {
          const int64_t tout = shfl64(mv.tout, vi);
          const float osc = (float)__shfl_sync(0xffffffffu, mv.osc, vi);
          const int mrows = __shfl_sync(0xffffffffu, mv.mrows, vi);
          const int tcol = __shfl_sync(0xffffffffu, mv.tcol, vi);
          const int mp = __shfl_sync(0xffffffffu, mv.mp, vi);
          const int ntot = __shfl_sync(0xffffffffu, mv.ntot, vi);
          const bool mval = m < mrows;
          const int R = mp * TP_A + m;          // row of T_t^T
          const int pr = R / TP_B;
          const int pr8 = (min(TP_B, ntot - pr * TP_B) + 7) / 8;
          uint8_t* rowp = args.T + tout + (int64_t)pr * (TP_B / 8) * c8t * 128 + ((R % TP_B) / 8) * 128 + (R % 8) * 16;
          for (int g2 = 0; g2 < ng16; ++g2) {
            float x[16];
            tmem_ld16(trow + (uint32_t)(tcol + 16 * g2), x);
            if (mval) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int g = 2 * g2 + h;
                if (8 * g >= it.nrows) break;
                float* y = x + 8 * h;
                const int jc = (it.np * TP_B) / 8 + g;   // 16-byte K unit of T_t^T
#pragma unroll
                for (int j = 0; j < 8; ++j) y[j] = (8 * g + j < it.nrows) ? osc * y[j] : 0.f;
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                  uint32_t p[4];
#pragma unroll
                  for (int j = 0; j < 8; j += 2) {
                    const uint32_t h0 = bf16_bits(y[j]), h1 = bf16_bits(y[j + 1]);
                    p[j >> 1] = h0 | (h1 << 16);
                    y[j] -= __uint_as_float(h0 << 16);
                    y[j + 1] -= __uint_as_float(h1 << 16);
                  }
                  *reinterpret_cast<uint4*>(rowp + q * args.tplane + (int64_t)jc * pr8 * 128) =
                      make_uint4(p[0], p[1], p[2], p[3]);
                }
              }
            }
          }
        }
      } else {
        const bool mval = m < it.mrows;
        double* row = args.sig + it.out + (int64_t)(it.mp * TP_A + m) * it.ldc + it.np * TP_B;
        const int ngrp = (it.nrows + 7) / 8;
        for (int g = half; g < ngrp; g += 2) {
          float x[8];
          tmem_ld8(trow + (uint32_t)(8 * g), x);
          if (mval) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int c = 8 * g + j;
              if (c < it.nrows) {
                if (it.split) atomicAdd(row + c, (double)x[j]);
                else row[c] += (double)x[j];
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
  constexpr uint32_t sm = Smem<MODE>::SMEM;
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
                                const uint8_t* psi_arena, int64_t psi_plane, const uint8_t* r_arena,
                                int64_t r_plane, uint8_t* t_arena, int64_t t_plane, int chunk_bytes, int grid,
                                int* err, cudaStream_t st) {
  // A operands: right views; B operand: psi
  Stage1Args a{items, views, r_arena, r_plane, psi_arena, psi_plane, t_arena, t_plane, chunk_bytes};
  if (mode == TT_BF16) return launch<TT_BF16, 1>(a, nitems, grid, err, st);
  if (mode == TT_BF16X3) return launch<TT_BF16X3, 1>(a, nitems, grid, err, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tiled_stage2(int mode, const K2Item* items, int nitems, const K2Seg* segs,
                                const uint8_t* a_arena, int64_t a_plane, const uint8_t* t_arena,
                                int64_t t_plane, double* sigma, int chunk_bytes, int grid, int* err,
                                cudaStream_t st) {
  Stage2Args a{items, segs, a_arena, a_plane, t_arena, t_plane, sigma, chunk_bytes};
  if (mode == TT_BF16) return launch<TT_BF16, 2>(a, nitems, grid, err, st);
  if (mode == TT_BF16X3) return launch<TT_BF16X3, 2>(a, nitems, grid, err, st);
  return cudaErrorInvalidValue;
}

}  // namespace qd

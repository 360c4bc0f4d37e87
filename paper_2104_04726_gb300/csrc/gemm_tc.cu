// Tensor-core (tcgen05) GEMM for the large contractions of the Tucker-ALS
// sweep: the mode products T x_n S^T (Eq. 8) and the factored Gram products.
//
// C(m, n) = alpha * sum_k A(m, k) B(n, k), both operands K-major, FP32
// accumulation in tensor memory (TMEM).  One CTA computes a 128 x BN tile:
//   warp 0    TMA producer: 128-byte-swizzled K slices of A and B into a
//             STAGES-deep shared-memory ring (mbarrier full/empty pairs);
//   warp 1    allocates BN TMEM columns; one thread issues tcgen05.mma
//             (M=128, N=BN, K=32 bytes per instruction) and commits each
//             stage back to its producer barrier;
//   warps 2-9 epilogue: two warps per 32-lane quarter of TMEM (the access
//             rule of tcgen05.ld), each draining half of the BN columns;
//             tcgen05.ld 32x32b, then the strided (two-level) store,
//             accumulate or fused residual.
// Kinds: kind::tf32 on FP32 data, kind::f16 on BF16 data, and the
// three-term TF32 split (KIND 2): with A = A_hi + A_lo and B = B_hi + B_lo,
// both terms exactly TF32, each K slice issues A_hi B_hi + A_hi B_lo +
// A_lo B_hi into one accumulator (the dropped A_lo B_lo is ~2^-22 of the
// product), so the result has FP32-level accuracy.  KIND 3, the six-term
// BF16 split: each operand is stored as three BF16 parts x = x1 + x2 + x3
// (24 significant bits, as many as FP32) in the K_hi planes of its tensor
// map; each K slice stages the three parts of both operands and issues the
// part pairs (1,1) (1,2) (2,1) (1,3) (3,1) (2,2) -- every product down to
// 2^-16 of the leading one -- the leading pair into one FP32 accumulator and
// the corrections into a second, summed in the epilogue, so the result has
// FP32-level accuracy at BF16 tensor-core rate (used for the Grams of the
// factor update).  Split-K over
// grid.z writes FP32 partial tiles that one fixed-order pass reduces, so the
// result is deterministic.  Every mbarrier wait is bounded (globaltimer,
// 2 s unless the caller sets a shorter bound); a timeout sets an error bit.
// Before the CTA frees its tensor memory and exits, the producer waits for
// every TMA load it issued and the MMA thread for its committed MMAs, both
// again bounded (kDrainNs), so no copy or MMA is left writing into shared or
// tensor memory the CTA no longer owns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "gemm.cuh"
#include "gemm_tc.cuh"
#include "small.cuh"

namespace {

constexpr int BM = 128;
constexpr int kThreads = 320;   // 2 control warps + 8 epilogue warps
constexpr int kEpiWarps = 8;
constexpr uint64_t kWaitNs = 2000000000ull;    // default bound of a pipeline wait
constexpr uint64_t kDrainNs = 2000000000ull;   // bound of the teardown waits for work in flight

struct TcArgs {
  int64_t M, N;
  int k_tiles_lo, k_tiles_total, kt_per_split, splits, batch;
  int a_batched, b_batched;   // 0: operand shared by all batches (coordinate 0)
  float* C;
  int64_t M_lo, c_m, c_mh, N_lo, c_n, c_nh, c_b;
  float* C2;
  int64_t c2_m, c2_mh, c2_n, c2_nh, c2_b;
  float alpha;
  int accumulate;
  int round_out;
  const float* ref;
  double* partials;
  float* split_ws;     // [split][batch][M][N] when splits > 1
  const int* skip;
  int* err;
  uint64_t wait_ns;    // bound of each pipeline wait (0: kWaitNs)
  int lower;           // skip tiles wholly above the diagonal (n0 >= m0 + BM)
  uint16_t* Cp;        // nullable: BF16 parts of C (c_m == 1), planes of cp_plane
  int64_t cp_plane;
};

// The three BF16 parts x1 = bf(x), x2 = bf(x - x1), x3 = bf(x - x1 - x2),
// each rounded to nearest even (both differences are exact in FP32).
__device__ __forceinline__ void bf16x3_parts(float x, uint16_t& b1, uint16_t& b2, uint16_t& b3) {
  b1 = mes::bf16_bits(x);
  const float r1 = x - __uint_as_float((uint32_t)b1 << 16);
  b2 = mes::bf16_bits(r1);
  b3 = mes::bf16_bits(r1 - __uint_as_float((uint32_t)b2 << 16));
}

// Element bytes of an operand kind: BF16 for kinds 1 and 3, FP32 otherwise.
__host__ __device__ constexpr int kind_bytes(int kind) { return (kind == 1 || kind == 3) ? 2 : 4; }
// KIND 3: operand part of pair q (0..5) for A and for B.
__device__ __forceinline__ int pair_a(int q) { return (0x120100 >> (4 * q)) & 0xF; }   // 0,0,1,0,2,1
__device__ __forceinline__ int pair_b(int q) { return (0x102010 >> (4 * q)) & 0xF; }   // 0,1,0,2,0,1

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after limit_ns without the phase completing.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile, 128-byte rows, 128-byte swizzle: 8-row atoms of
// 1024 bytes (stride byte offset), descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (KIND != 1 && KIND != 3) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Offsets of consecutive output columns n, n+1, ... under the two-level
// split n = n_lo + N_lo * n_hi (offset n_lo * s_n + n_hi * s_nh), walked
// without a division per column.
struct ColWalk {
  int64_t nl, nh, off, N_lo, s_n, s_nh;
  __device__ __forceinline__ ColWalk(int64_t n, int64_t N_lo_, int64_t s_n_, int64_t s_nh_)
      : N_lo(N_lo_), s_n(s_n_), s_nh(s_nh_) {
    nh = n / N_lo;
    nl = n - nh * N_lo;
    off = nl * s_n + nh * s_nh;
  }
  __device__ __forceinline__ void next() {
    if (++nl == N_lo) {
      nl = 0;
      ++nh;
      off = nh * s_nh;
    } else {
      off += s_n;
    }
  }
};

// Stores one 32-column chunk of a finished accumulator tile (this lane's row
// m, columns n0 + c0 .. + 31) to C (and C2), or to the split-K workspace.
// An output whose n index is contiguous goes through the warp's 32 x 33
// shared tile so that each store instruction writes 32 consecutive n of one
// row; an output with contiguous m is written directly (lanes = rows).
__device__ __forceinline__ void store_chunk(const TcArgs& args, const uint32_t (&v)[32], int64_t m0, int64_t n0,
                                            int b, int split, int wq, int lane, float* tile, int c0) {
  const int64_t m = m0 + wq * 32 + lane;
  const bool mok = m < args.M;
  const int64_t M_lo = args.M_lo, N_lo = args.N_lo;
  const int64_t mh = m / M_lo, ml = m - mh * M_lo;
  const int64_t moff = ml * args.c_m + mh * args.c_mh + (int64_t)b * args.c_b;
  const int64_t moff2 = ml * args.c2_m + mh * args.c2_mh + (int64_t)b * args.c2_b;
  // val (this lane's row, 32 columns) through the tile: element (row i of
  // the warp, n = n0 + c0 + lane) at base + row_off_i + col_off(n) with
  // col_off(n) = (n mod N_lo) * s_n + (n div N_lo) * s_nh
  auto store_rows = [&](const float (&val)[32], float* base, int64_t row_off, int64_t s_n, int64_t s_nh,
                        bool acc, bool rnd) {
#pragma unroll
    for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = val[j];
    __syncwarp();
    const int64_t n = n0 + c0 + lane;
    const int64_t nh = n / N_lo, nl = n - nh * N_lo;
    const int64_t col_off = nl * s_n + nh * s_nh;
    for (int i = 0; i < 32; ++i) {
      const int64_t off = __shfl_sync(0xffffffffu, row_off, i);
      const int64_t mi = m0 + wq * 32 + i;
      if (mi < args.M && n < args.N) {
        float* p = base + off + col_off;
        float x = tile[i * 33 + lane];
        if (acc) x += *p;
        if (rnd) x = mes::round_tf32(x);
        *p = x;
      }
    }
    __syncwarp();
  };
  float val[32];
  if (args.splits > 1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) val[j] = __uint_as_float(v[j]);
    const int64_t row_off = (((int64_t)split * args.batch + b) * args.M + m) * args.N;
    store_rows(val, args.split_ws, row_off, 1, N_lo, false, false);   // col_off = n
    return;
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) val[j] = args.alpha * __uint_as_float(v[j]);
  if (args.c_n == 1) {
    store_rows(val, args.C, moff, args.c_n, args.c_nh, args.accumulate != 0, args.round_out != 0);
  } else if (mok) {
    ColWalk cw(n0 + c0, N_lo, args.c_n, args.c_nh);
#pragma unroll
    for (int j = 0; j < 32; ++j, cw.next()) {
      if (n0 + c0 + j >= args.N) continue;
      float* p = args.C + moff + cw.off;
      float w = args.accumulate ? *p + val[j] : val[j];
      if (args.round_out) w = mes::round_tf32(w);
      *p = w;
      if (args.Cp) {   // lanes are consecutive m: each part store is 64 contiguous bytes
        uint16_t b1, b2, b3;
        bf16x3_parts(w, b1, b2, b3);
        uint16_t* q = args.Cp + moff + cw.off;
        q[0] = b1;
        q[args.cp_plane] = b2;
        q[2 * args.cp_plane] = b3;
      }
    }
  }
  if (args.C2) {
    if (args.c2_n == 1) {
      store_rows(val, args.C2, moff2, args.c2_n, args.c2_nh, false, args.round_out != 0);
    } else if (mok) {
      ColWalk cw(n0 + c0, N_lo, args.c2_n, args.c2_nh);
#pragma unroll
      for (int j = 0; j < 32; ++j, cw.next()) {
        if (n0 + c0 + j >= args.N) continue;
        args.C2[moff2 + cw.off] = args.round_out ? mes::round_tf32(val[j]) : val[j];
      }
    }
  }
}

template <int KIND, int BN, int STAGES>
struct Cfg {
  static constexpr int A_BYTES = BM * 128;
  static constexpr int B_BYTES = BN * 128;
  // KIND 2 stages the low parts after the high parts: A_hi, B_hi, A_lo, B_lo
  static constexpr int STAGE = (KIND == 2 ? 2 : 1) * (A_BYTES + B_BYTES);
  // the epilogue's transpose tiles (one 32 x 33 per drain warp) reuse the
  // operand ring, which is idle once the accumulator is complete
  static constexpr int EPI = kEpiWarps * 32 * 33 * 4;
  static_assert(EPI <= STAGES * STAGE, "epilogue tiles must fit in the operand ring");
  static constexpr int SMEM = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
  // KIND 0/1 fit two CTAs per SM (one CTA's epilogue overlaps the other's
  // main loop); KIND 2 stages four tiles per slice and runs one
  static constexpr int CTAS_PER_SM = KIND == 2 ? 1 : 2;
  static_assert(CTAS_PER_SM * (SMEM + 8 * kEpiWarps + 1024) <= 233472, "shared memory per SM");
  // idesc: D=F32 (bits 4-5 = 1); A/B format (bits 7-9, 10-12): TF32 = 2,
  // BF16 = 1; both K-major; N >> 3 at bit 17; M >> 4 at bit 24.
  static constexpr uint32_t FMT = KIND == 1 ? 1u : 2u;
  static constexpr uint32_t IDESC =
      (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

template <int KIND, int BN, int STAGES, bool RESID>
__global__ void __launch_bounds__(kThreads, KIND == 2 ? 1 : 2)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               const __grid_constant__ CUtensorMap mapA2, const __grid_constant__ CUtensorMap mapB2,
               const TcArgs args) {
  using C = Cfg<KIND, BN, STAGES>;
  if (args.skip && *args.skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* tiles = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(tiles + STAGES * C::STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  float* epi = reinterpret_cast<float*>(tiles);   // used only after the accumulator is complete
  __shared__ double red[kEpiWarps];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int b = (int)(blockIdx.z % args.batch);
  const int split = (int)(blockIdx.z / args.batch);
  const int kt_begin = split * args.kt_per_split;
  int kt_end = kt_begin + args.kt_per_split;
  if (kt_end > args.k_tiles_total) kt_end = args.k_tiles_total;
  const int nkt = kt_end - kt_begin;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapB) : "memory");
    if (KIND == 2) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA2) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&mapB2) : "memory");
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  const uint64_t wait_ns = args.wait_ns ? args.wait_ns : kWaitNs;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int stage = 0;
    uint32_t phase = 0;
    uint32_t issued = 0, last_phase = 0;   // per stage: loaded at least once; parity of its last load
    for (int i = 0; i < nkt; ++i) {
      if (!mbar_wait(&empty[stage], phase ^ 1u, wait_ns)) {
        ok = false;
        break;
      }
      issued |= 1u << stage;
      last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
      const int kt = kt_begin + i;
      const int kh = kt / args.k_tiles_lo;
      const int kl = (kt - kh * args.k_tiles_lo) * (128 / kind_bytes(KIND));
      uint8_t* sa = tiles + stage * C::STAGE;
      mbar_expect_tx(&full[stage], (uint32_t)C::STAGE);
      tma_load_4d(sa, &mapA, &full[stage], kl, (int)m0, kh, args.a_batched ? b : 0);
      tma_load_4d(sa + C::A_BYTES, &mapB, &full[stage], kl, (int)n0, kh, args.b_batched ? b : 0);
      if (KIND == 2) {
        uint8_t* sl = sa + C::A_BYTES + C::B_BYTES;
        tma_load_4d(sl, &mapA2, &full[stage], kl, (int)m0, kh, args.a_batched ? b : 0);
        tma_load_4d(sl + C::A_BYTES, &mapB2, &full[stage], kl, (int)n0, kh, args.b_batched ? b : 0);
      }
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
    if (!ok) atomicOr(args.err, 8);
    // teardown: every load this thread issued has landed (a stage whose last
    // phase already completed returns at once)
    for (int s2 = 0; s2 < STAGES; ++s2)
      if (((issued >> s2) & 1u) && !mbar_wait(&full[s2], (last_phase >> s2) & 1u, kDrainNs))
        atomicOr(args.err, 64);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int stage = 0;
    uint32_t phase = 0;
    for (int i = 0; i < nkt; ++i) {
      if (!mbar_wait(&full[stage], phase, wait_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = smem_u32(tiles + stage * C::STAGE);
      const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + C::A_BYTES);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)   // 4 x 32 bytes of K per 128-byte row
        mma<KIND>(tmem, da + 2 * kk, db + 2 * kk, C::IDESC, (i > 0 || kk > 0) ? 1u : 0u);
      if (KIND == 2) {
        const uint32_t sl = sa + C::A_BYTES + C::B_BYTES;
        const uint64_t dal = sw128_desc(sl), dbl = sw128_desc(sl + C::A_BYTES);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          mma<KIND>(tmem, da + 2 * kk, dbl + 2 * kk, C::IDESC, 1u);   // A_hi B_lo
          mma<KIND>(tmem, dal + 2 * kk, db + 2 * kk, C::IDESC, 1u);   // A_lo B_hi
        }
      }
      mma_commit(&empty[stage]);
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
    mma_commit(accum);
    if (!ok) atomicOr(args.err, 16);
    // teardown: the MMAs issued above are complete before TMEM is freed
    if (!mbar_wait(accum, 0, kDrainNs)) atomicOr(args.err, 64);
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int wq = warp & 3;                 // TMEM lane quarter = rows wq*32 .. wq*32+31
    const int half = (warp - 2) >> 2;        // columns half*BN/2 .. (half+1)*BN/2 - 1
    const int64_t m = m0 + wq * 32 + lane;
    // warp-uniform: the transposed stores below shuffle across the warp
    const bool waited = __all_sync(0xffffffffu, mbar_wait(accum, 0, wait_ns));
    if (!waited && lane == 0) atomicOr(args.err, 32);
    tc_fence_after();
    const bool mok = m < args.M;
    const int64_t M_lo = args.M_lo, N_lo = args.N_lo;
    const int64_t mh = m / M_lo, ml = m - mh * M_lo;
    const int64_t moff = ml * args.c_m + mh * args.c_mh + (int64_t)b * args.c_b;
    double sq = 0.0;
    float* tile = epi + (warp - 2) * 32 * 33;
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0, v);
      if (!waited) continue;
      if (RESID && args.splits == 1) {
        if (!mok) continue;
        // 32 squares summed in FP32 (relative error ~32 * 2^-24 of a
        // non-negative sum), then one FP64 add per chunk: GB300's FP64
        // rate is a small fraction of its FP32 rate
        float sqf = 0.f;
        if (N_lo >= args.N) {
          // one-level n: linear offsets, so the 32 reference loads are
          // independent and go out together
          const float* rp = args.ref + moff + (n0 + c0) * args.c_n;
          float refv[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) refv[j] = (n0 + c0 + j < args.N) ? __ldg(rp + j * args.c_n) : 0.f;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (n0 + c0 + j >= args.N) continue;
            const float val = args.alpha * __uint_as_float(v[j]);
            const float d = refv[j] - val;
            sqf = fmaf(d, d, sqf);
            if (args.C) args.C[moff + (n0 + c0 + j) * args.c_n] = val;   // the product is stored too
          }
        } else {
          ColWalk cw(n0 + c0, N_lo, args.c_n, args.c_nh);
#pragma unroll
          for (int j = 0; j < 32; ++j, cw.next()) {
            if (n0 + c0 + j >= args.N) continue;
            const float val = args.alpha * __uint_as_float(v[j]);
            const float d = __ldg(args.ref + moff + cw.off) - val;
            sqf = fmaf(d, d, sqf);
            if (args.C) args.C[moff + cw.off] = val;   // the product is stored too
          }
        }
        sq += (double)sqf;
        continue;
      }
      store_chunk(args, v, m0, n0, b, split, wq, lane, tile, c0);
    }
    if (RESID) {
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
      if (lane == 0) red[warp - 2] = sq;
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory");
      if (warp == 2 && lane == 0) {
        const int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        double tot = 0.0;
        for (int w = 0; w < kEpiWarps; ++w) tot += red[w];
        args.partials[bid] = tot;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

// --------------------------------------------------------------------------
// Persistent form of the same product (KIND 0 and 1, no residual): one CTA
// per SM walks the tiles t = blockIdx.x, + gridDim.x, ... (tile index m
// fastest, then n, batch, split, so the CTAs running side by side share an
// operand tile through L2).  Two TMEM accumulators of BN columns each: the
// MMA thread fills accumulator j & 1 for local tile j while the epilogue
// warps drain the other, and the TMA ring runs ahead across tile
// boundaries, so loads, MMAs and stores of neighbouring tiles overlap.
// Barriers: full/empty per ring stage, tfull (accumulator complete, MMA ->
// epilogue, one commit) and tempty (accumulator drained, epilogue -> MMA,
// one arrival per epilogue warp) per accumulator.  Every wait is bounded;
// on a timeout a role sets its error bit and leaves its loop, and the
// teardown drains loads and MMAs in flight as in tc_gemm_kernel.
// --------------------------------------------------------------------------
template <int KIND, int BN, int STAGES, int CTAS = 1>
struct PCfg {
  static constexpr int A_BYTES = BM * 128;
  static constexpr int B_BYTES = BN * 128;
  // KIND 3 stages the three parts of both operands of a K slice together:
  // A1 A2 A3 B1 B2 B3, each loaded once and read by the six pair products
  static constexpr int PARTS = KIND == 3 ? 3 : 1;
  static constexpr int STAGE = PARTS * (A_BYTES + B_BYTES);
  static constexpr int EPI = kEpiWarps * 32 * 33 * 4;   // per-warp transpose tiles (own region)
  static constexpr int BAR = 8 * (2 * STAGES + 5);
  static constexpr int SMEM = STAGES * STAGE + EPI + 1024 /*align*/ + BAR + 16;
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(CTAS * (SMEM + 1024) <= 233472, "shared memory per SM");
  static constexpr uint32_t FMT = (KIND == 1 || KIND == 3) ? 1u : 2u;
  static constexpr uint32_t IDESC =
      (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  // two accumulators (double buffer) of BN columns; KIND 3 gives each tile a
  // second one for the correction terms (pairs 2..6), so 4 x BN
  static constexpr int ACC_COLS = KIND == 3 ? 2 * BN : BN;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;   // 256 or 512 columns (powers of 2)
  static_assert(CTAS * TMEM_COLS <= 512, "tensor memory columns per SM");
};

template <int KIND, int BN, int STAGES, int CTAS>
__global__ void __launch_bounds__(kThreads, CTAS)
tcp_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const TcArgs args, int mt, int nt, int ntiles) {
  using C = PCfg<KIND, BN, STAGES, CTAS>;
  if (args.skip && *args.skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* epi = reinterpret_cast<float*>(ring + STAGES * C::STAGE);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + STAGES * C::STAGE + C::EPI);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;     // [2]
  uint64_t* tempty = tfull + 2;         // [2]
  uint64_t* drain = tempty + 2;         // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], kEpiWarps);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint64_t wait_ns = args.wait_ns ? args.wait_ns : kWaitNs;
  const int mn = mt * nt;
  // tile t -> (m tile, n tile, batch, split); k range of its split
  // (false: a tile wholly above the diagonal of a lower-only product; every
  // role skips the same tiles)
  auto decode = [&](int t, int64_t& m0, int64_t& n0, int& b, int& split, int& kb, int& ke) -> bool {
    const int mi = t % mt;
    const int r = t / mt;
    const int ni = r % nt;
    const int bs = r / nt;
    b = bs % args.batch;
    split = bs / args.batch;
    m0 = (int64_t)mi * BM;
    n0 = (int64_t)ni * BN;
    kb = split * args.kt_per_split;
    ke = kb + args.kt_per_split;
    if (ke > args.k_tiles_total) ke = args.k_tiles_total;
    return !(args.lower && n0 >= m0 + BM);
  };
  (void)mn;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int stage = 0;
    uint32_t phase = 0;
    uint32_t issued = 0, last_phase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int64_t m0, n0;
      int b, split, kb, ke;
      if (!decode(t, m0, n0, b, split, kb, ke)) continue;
      for (int kt = kb; kt < ke; ++kt) {
        if (!mbar_wait(&empty[stage], phase ^ 1u, wait_ns)) {
          ok = false;
          break;
        }
        issued |= 1u << stage;
        last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
        const int kh = kt / args.k_tiles_lo;
        const int kl = (kt - kh * args.k_tiles_lo) * (128 / kind_bytes(KIND));
        uint8_t* sa = ring + stage * C::STAGE;
        mbar_expect_tx(&full[stage], (uint32_t)C::STAGE);
        if (KIND == 3) {
          // the three parts (K_hi planes) of A, then of B
#pragma unroll
          for (int part = 0; part < 3; ++part) {
            tma_load_4d(sa + part * C::A_BYTES, &mapA, &full[stage], kl, (int)m0, part, args.a_batched ? b : 0);
            tma_load_4d(sa + 3 * C::A_BYTES + part * C::B_BYTES, &mapB, &full[stage], kl, (int)n0, part,
                        args.b_batched ? b : 0);
          }
        } else {
          tma_load_4d(sa, &mapA, &full[stage], kl, (int)m0, kh, args.a_batched ? b : 0);
          tma_load_4d(sa + C::A_BYTES, &mapB, &full[stage], kl, (int)n0, kh, args.b_batched ? b : 0);
        }
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (!ok) atomicOr(args.err, 8);
    for (int s2 = 0; s2 < STAGES; ++s2)
      if (((issued >> s2) & 1u) && !mbar_wait(&full[s2], (last_phase >> s2) & 1u, kDrainNs))
        atomicOr(args.err, 64);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    int j = 0;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int64_t m0, n0;
      int b, split, kb, ke;
      if (!decode(t, m0, n0, b, split, kb, ke)) continue;
      const int acc = j & 1;
      const uint32_t use = (uint32_t)(j >> 1);
      // the accumulator's previous tile has been drained by the epilogue
      if (!mbar_wait(&tempty[acc], (use & 1u) ^ 1u, wait_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d0 = tmem + (uint32_t)(acc * C::ACC_COLS);
      for (int kt = kb; kt < ke; ++kt) {
        if (!mbar_wait(&full[stage], phase, wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(ring + stage * C::STAGE);
        if (KIND == 3) {
          // the six part pairs: the leading pair (1,1) into d0, the five
          // correction pairs into d0 + BN, so the small terms are not rounded
          // against the full sum
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const uint64_t da = sw128_desc(sa + pair_a(q) * C::A_BYTES);
            const uint64_t db = sw128_desc(sa + 3 * C::A_BYTES + pair_b(q) * C::B_BYTES);
            const uint32_t d = q == 0 ? d0 : d0 + BN;
            const bool first = kt == kb && q <= 1;   // first slice of each accumulator: overwrite
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma<KIND>(d, da + 2 * kk, db + 2 * kk, C::IDESC, (!first || kk > 0) ? 1u : 0u);
          }
        } else {
          const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + C::A_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma<KIND>(d0, da + 2 * kk, db + 2 * kk, C::IDESC, (kt > kb || kk > 0) ? 1u : 0u);
        }
        mma_commit(&empty[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit(&tfull[acc]);
      ++j;
    }
    if (!ok) atomicOr(args.err, 16);
    // teardown: every MMA issued above is complete before TMEM is freed
    mma_commit(drain);
    if (!mbar_wait(drain, 0, kDrainNs)) atomicOr(args.err, 64);
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int wq = warp & 3;                 // TMEM lane quarter = rows wq*32 .. wq*32+31
    const int half = (warp - 2) >> 2;        // columns half*BN/2 .. (half+1)*BN/2 - 1
    float* tile = epi + (warp - 2) * 32 * 33;
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int64_t m0, n0;
      int b, split, kb, ke;
      if (!decode(t, m0, n0, b, split, kb, ke)) continue;
      const int acc = j & 1;
      const uint32_t use = (uint32_t)(j >> 1);
      // warp-uniform: the transposed stores shuffle across the warp
      const bool waited = __all_sync(0xffffffffu, mbar_wait(&tfull[acc], use & 1u, wait_ns));
      if (!waited) {
        if (lane == 0) atomicOr(args.err, 32);
        break;
      }
      tc_fence_after();
      // KIND 3: every K slice writes both accumulators
      const bool has_lead = true;
      const bool has_corr = KIND == 3;
      (void)kb;
      (void)ke;
      const uint32_t row = (uint32_t)(wq * 32) << 16;
      for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 32) {
        uint32_t v[32];
        if (has_lead) {
          tmem_ld32(tmem + row + (uint32_t)(acc * C::ACC_COLS + c0), v);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = 0u;
        }
        if (has_corr) {
          uint32_t w[32];
          tmem_ld32(tmem + row + (uint32_t)(acc * C::ACC_COLS + BN + c0), w);
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) + __uint_as_float(w[q]));
        }
        store_chunk(args, v, m0, n0, b, split, wq, lane, tile, c0);
      }
      // this warp's part of the accumulator is read: hand it back to the MMA
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[acc])) : "memory");
      ++j;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// Fixed-order reduction of split-K partial tiles into C (general strides).
__global__ void split_reduce_kernel(const float* __restrict__ ws, TcArgs a) {
  if (a.skip && *a.skip) return;
  const int64_t total = (int64_t)a.batch * a.M * a.N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int sp = 0; sp < a.splits; ++sp) s += ws[(int64_t)sp * total + e];
    const int64_t n = e % a.N;
    const int64_t bm = e / a.N;
    const int64_t m = bm % a.M, b = bm / a.M;
    if (a.lower && n > m) continue;   // the consumer reads the lower triangle only
    const int64_t mh = m / a.M_lo, ml = m - mh * a.M_lo, nh = n / a.N_lo, nl = n - nh * a.N_lo;
    float val = a.alpha * s;
    float* p = a.C + ml * a.c_m + mh * a.c_mh + nl * a.c_n + nh * a.c_nh + b * a.c_b;
    val = a.accumulate ? *p + val : val;
    if (a.round_out) val = mes::round_tf32(val);
    *p = val;
    if (a.Cp) {
      uint16_t b1, b2, b3;
      bf16x3_parts(val, b1, b2, b3);
      uint16_t* q = a.Cp + (p - a.C);
      q[0] = b1;
      q[a.cp_plane] = b2;
      q[2 * a.cp_plane] = b3;
    }
    if (a.C2) a.C2[ml * a.c2_m + mh * a.c2_mh + nl * a.c2_n + nh * a.c2_nh + b * a.c2_b] = val;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

mes_status get_encode() {
  if (g_encode) return MES_OK;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return mes::fail(MES_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return MES_OK;
}

// 4-D map {K_lo, rows, K_hi, batch} of a K-major operand.
bool make_map(CUtensorMap* map, const void* base, int kind, int64_t K_lo, int64_t rows, int64_t K_hi,
              int64_t batch, int64_t s_row, int64_t s_kh, int64_t s_b, int box_rows) {
  const int E = kind_bytes(kind);
  cuuint64_t dims[4] = {(cuuint64_t)K_lo, (cuuint64_t)rows, (cuuint64_t)K_hi, (cuuint64_t)batch};
  int64_t st[3] = {s_row * E, s_kh * E, s_b * E};
  // unit dims get a harmless stride that keeps the strides increasing
  if (K_hi == 1) st[1] = st[0] * rows;
  if (batch == 1) st[2] = st[1] * (K_hi > 0 ? K_hi : 1);
  for (int i = 0; i < 3; ++i)
    if (st[i] <= 0 || st[i] % 16 != 0 || st[i] >= ((int64_t)1 << 40)) return false;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
  cuuint64_t strides[3] = {(cuuint64_t)st[0], (cuuint64_t)st[1], (cuuint64_t)st[2]};
  cuuint32_t box[4] = {(cuuint32_t)(128 / E), (cuuint32_t)box_rows, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode(map, E == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                        const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int KIND, int BN, int STAGES>
mes_status launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& ma2, const CUtensorMap& mb2,
                     const TcArgs& a, dim3 grid, bool resid, cudaStream_t st) {
  using C = Cfg<KIND, BN, STAGES>;
  static bool attr = false;
  if (!attr) {
    MES_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<KIND, BN, STAGES, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    MES_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<KIND, BN, STAGES, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    attr = true;
  }
  if (resid)
    tc_gemm_kernel<KIND, BN, STAGES, true><<<grid, kThreads, C::SMEM, st>>>(ma, mb, ma2, mb2, a);
  else
    tc_gemm_kernel<KIND, BN, STAGES, false><<<grid, kThreads, C::SMEM, st>>>(ma, mb, ma2, mb2, a);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

template <int KIND, int BN, int STAGES, int CTAS = 1>
mes_status launch_tcp(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int mt, int nt, int ntiles,
                      cudaStream_t st) {
  using C = PCfg<KIND, BN, STAGES, CTAS>;
  static bool attr = false;
  if (!attr) {
    MES_CUDA_TRY(cudaFuncSetAttribute(tcp_gemm_kernel<KIND, BN, STAGES, CTAS>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    attr = true;
  }
  const int slots = CTAS * mes::sm_count();
  const int grid = ntiles < slots ? ntiles : slots;
  tcp_gemm_kernel<KIND, BN, STAGES, CTAS><<<grid, kThreads, C::SMEM, st>>>(ma, mb, a, mt, nt, ntiles);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

}  // namespace

namespace mes {

bool tc_eligible(const Gemm& g, int kind) {
  const int E = kind_bytes(kind);
  if (kind == 2 && (!g.A2 || !g.B2 || reinterpret_cast<uintptr_t>(g.A2) % 16 || reinterpret_cast<uintptr_t>(g.B2) % 16))
    return false;
  if (g.a_k != 1 || g.b_k != 1) return false;
  if ((g.a_m * E) % 16 || (g.b_n * E) % 16) return false;
  if (g.K_hi > 1 && ((g.a_kh * E) % 16 || (g.b_kh * E) % 16)) return false;
  if (g.batch > 1 && (((g.a_b * E) % 16) || ((g.b_b * E) % 16))) return false;
  if (g.a_b < 0 || g.b_b < 0 || g.a_kh < 0 || g.b_kh < 0) return false;
  if (reinterpret_cast<uintptr_t>(g.A) % 16 || reinterpret_cast<uintptr_t>(g.B) % 16) return false;
  if (g.M > INT32_MAX || g.N > INT32_MAX || g.K_lo > INT32_MAX) return false;
  return true;
}

}  // namespace mes

namespace {

// One launch of the product with tile width bn (128 or 256) and a split-K
// factor; splits <= 0 picks the factor by the fill rule (split while the
// tile grid covers less than the SMs and each split keeps >= 4 K-tiles).
mes_status gemm_tc_cfg(const mes::Gemm& g, int kind, int bn, int want_splits, float* split_ws,
                       int64_t split_ws_elems, int* err, cudaStream_t st) {
  using namespace mes;
  const int BK = 128 / kind_bytes(kind);
  if (kind >= 2 || (bn != 128 && bn != 256)) bn = 128;   // KINDs 2 and 3 have only the 128-wide tile
  CUtensorMap ma, mb, ma2, mb2;
  const bool ab = g.batch > 1 && g.a_b != 0, bb = g.batch > 1 && g.b_b != 0;
  if (!make_map(&ma, g.A, kind, g.K_lo, g.M, g.K_hi, ab ? g.batch : 1, g.a_m, g.a_kh, g.a_b, BM) ||
      !make_map(&mb, g.B, kind, g.K_lo, g.N, g.K_hi, bb ? g.batch : 1, g.b_n, g.b_kh, g.b_b, bn))
    return fail(MES_ERR_INVALID_ARG, "gemm_tc: tensor map rejected");
  if (kind == 2) {
    if (!make_map(&ma2, g.A2, kind, g.K_lo, g.M, g.K_hi, ab ? g.batch : 1, g.a_m, g.a_kh, g.a_b, BM) ||
        !make_map(&mb2, g.B2, kind, g.K_lo, g.N, g.K_hi, bb ? g.batch : 1, g.b_n, g.b_kh, g.b_b, bn))
      return fail(MES_ERR_INVALID_ARG, "gemm_tc: tensor map of a low part rejected");
  } else {
    ma2 = ma;
    mb2 = mb;
  }
  TcArgs a;
  a.M = g.M;
  a.N = g.N;
  a.k_tiles_lo = (int)((g.K_lo + BK - 1) / BK);
  // KIND 3: the K_hi planes are the three parts, all staged with each K slice
  a.k_tiles_total = a.k_tiles_lo * (kind == 3 ? 1 : (int)g.K_hi);
  a.lower = g.lower ? 1 : 0;
  a.Cp = g.Cp;
  a.cp_plane = g.cp_plane;
  if (g.Cp && (kind >= 2 || g.c_m != 1 || g.ref))
    return fail(MES_ERR_INVALID_ARG, "gemm_tc: BF16 parts need kind 0 or 1 and an m-contiguous C");
  a.batch = g.batch;
  a.a_batched = ab ? 1 : 0;
  a.b_batched = bb ? 1 : 0;
  a.C = g.C;
  a.M_lo = g.M_lo > 0 ? g.M_lo : g.M;
  a.c_m = g.c_m; a.c_mh = g.c_mh;
  a.N_lo = g.N_lo > 0 ? g.N_lo : g.N;
  a.c_n = g.c_n; a.c_nh = g.c_nh; a.c_b = g.c_b;
  a.C2 = g.C2;
  a.c2_m = g.c2_m; a.c2_mh = g.c2_mh; a.c2_n = g.c2_n; a.c2_nh = g.c2_nh; a.c2_b = g.c2_b;
  a.alpha = g.alpha;
  a.accumulate = g.accumulate ? 1 : 0;
  a.round_out = g.round_tf32 ? 1 : 0;
  a.ref = g.ref;
  a.partials = g.partials;
  a.skip = g.skip;
  a.err = err;
  a.wait_ns = g.wait_ns;
  // split K when the tile grid leaves most SMs idle
  const int64_t tiles = ((g.M + BM - 1) / BM) * ((g.N + bn - 1) / bn) * g.batch;
  int splits = 1;
  const int64_t sms = sm_count();
  const int64_t fill = g.fill > 0 ? g.fill : sms;   // CTA slots the split rule aims at
  if (want_splits > 0 && !g.ref &&
      (want_splits == 1 || (split_ws && (int64_t)want_splits * g.batch * g.M * g.N <= split_ws_elems))) {
    splits = want_splits;   // a tuned factor the workspace can hold
  } else if (!g.ref && split_ws) {
    while (tiles * splits * 2 <= fill && a.k_tiles_total / (splits * 2) >= 4 &&
           (int64_t)(splits * 2) * g.batch * g.M * g.N <= split_ws_elems)
      splits *= 2;
  }
  a.kt_per_split = (a.k_tiles_total + splits - 1) / splits;
  splits = (a.k_tiles_total + a.kt_per_split - 1) / a.kt_per_split;
  if (splits < 1) splits = 1;
  a.splits = splits;
  a.split_ws = split_ws;
  dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + bn - 1) / bn), (unsigned)(g.batch * splits));
  {
    // algorithmic work of the product itself (KIND 2 executes three MMAs
    // per K slice and reads both parts of each operand)
    const double kk = (double)g.K_lo * (kind == 3 ? 1.0 : (double)g.K_hi);   // K of the product itself
    ProfScope prof(kind == 0 ? "gemm_tf32_tc" : kind == 1 ? "gemm_bf16_tc" : kind == 2 ? "gemm_tf32x3_tc"
                                                                                    : "gemm_bf16x6_tc",
                   st, 2.0 * g.M * g.N * kk * g.batch,
                   (kind == 1 ? 2.0 : kind == 2 ? 8.0 : kind == 3 ? 6.0 : 4.0) * g.batch * ((double)g.M + g.N) * kk +
                       4.0 * g.batch * g.M * (double)g.N);
    const bool rs = g.ref != nullptr;
    const int mt = (int)((g.M + BM - 1) / BM), nt = (int)((g.N + bn - 1) / bn);
    const int64_t ntiles = (int64_t)mt * nt * g.batch * splits;
    // MES_TC_VARIANT (measurement switch for the products of kinds 0 and 1):
    // unset = one tile per CTA; "p1" = persistent, one CTA per SM; "p2" =
    // persistent, 128-wide tiles, two CTAs per SM
    static const char* variant = getenv("MES_TC_VARIANT");
    const int pv = (variant && variant[0] == 'p') ? (variant[1] == '2' ? 2 : 1) : 0;
    if (kind == 3 && (rs || g.accumulate || ntiles >= INT32_MAX))
      return fail(MES_ERR_INVALID_ARG, "gemm_tc: the six-term product has no residual or accumulate mode");
    if (kind == 3) {
      MES_TRY((launch_tcp<3, 128, 2>(ma, mb, a, mt, nt, (int)ntiles, st)));
    } else if (pv && kind != 2 && !rs && !g.accumulate && ntiles < INT32_MAX && (pv == 1 || bn == 128)) {
      // persistent kernel: tiles looped per CTA, double-buffered accumulator
      if (pv == 2) {
        if (kind == 0) MES_TRY((launch_tcp<0, 128, 2, 2>(ma, mb, a, mt, nt, (int)ntiles, st)));
        else MES_TRY((launch_tcp<1, 128, 2, 2>(ma, mb, a, mt, nt, (int)ntiles, st)));
      } else if (kind == 0) {
        if (bn == 256) MES_TRY((launch_tcp<0, 256, 4>(ma, mb, a, mt, nt, (int)ntiles, st)));
        else MES_TRY((launch_tcp<0, 128, 6>(ma, mb, a, mt, nt, (int)ntiles, st)));
      } else {
        if (bn == 256) MES_TRY((launch_tcp<1, 256, 4>(ma, mb, a, mt, nt, (int)ntiles, st)));
        else MES_TRY((launch_tcp<1, 128, 6>(ma, mb, a, mt, nt, (int)ntiles, st)));
      }
    } else if (kind == 0) {
      if (bn == 256) MES_TRY((launch_tc<0, 256, 2>(ma, mb, ma2, mb2, a, grid, rs, st)));
      else MES_TRY((launch_tc<0, 128, 3>(ma, mb, ma2, mb2, a, grid, rs, st)));
    } else if (kind == 1) {
      if (bn == 256) MES_TRY((launch_tc<1, 256, 2>(ma, mb, ma2, mb2, a, grid, rs, st)));
      else MES_TRY((launch_tc<1, 128, 3>(ma, mb, ma2, mb2, a, grid, rs, st)));
    } else {
      MES_TRY((launch_tc<2, 128, 3>(ma, mb, ma2, mb2, a, grid, rs, st)));
    }
  }
  if (splits > 1) {
    ProfScope prof("split_reduce", st, 0.0, 4.0 * splits * g.batch * g.M * (double)g.N);
    const int64_t total = (int64_t)g.batch * g.M * g.N;
    split_reduce_kernel<<<grid_for(total, 256, sms * 8), 256, 0, st>>>(split_ws, a);
    MES_LAUNCH_CHECK();
  }
  return MES_OK;
}

// --------------------------------------------------------------------------
// Tile autotuner.  Per product shape (kind, M, N, K, batch, operand
// batching, residual mode) the tile width and the split-K factor are chosen
// by timing every candidate once on the caller's stream the first time the
// shape is met; the choice is kept for the process.  Enabled by MES_TUNE=1;
// MES_TUNE_CACHE=<file> loads earlier choices and appends new ones, one
// "key = bn splits" line each.  Never inside a stream capture, never for an
// accumulating product (a candidate run would add to C) and never in
// residual mode; those use the fill rule.
// --------------------------------------------------------------------------
struct TcChoice {
  int bn, splits;
};
std::mutex g_tune_mu;
std::unordered_map<std::string, TcChoice> g_tune;
int g_tune_state = -1;   // -1 unread, 0 off, 1 on

bool tuning_on() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune_state < 0) {
    const char* e = getenv("MES_TUNE");
    g_tune_state = (e && e[0] == '1') ? 1 : 0;
    const char* path = getenv("MES_TUNE_CACHE");
    if (path) {
      if (FILE* f = fopen(path, "r")) {
        char line[256];
        while (fgets(line, sizeof line, f)) {
          char* eq = strstr(line, " = ");
          TcChoice c;
          if (eq && sscanf(eq + 3, "%d %d", &c.bn, &c.splits) == 2 && (c.bn == 128 || c.bn == 256) && c.splits >= 1)
            g_tune[std::string(line, eq)] = c;
        }
        fclose(f);
      }
    }
  }
  return g_tune_state == 1 || !g_tune.empty();
}

std::string tune_key(const mes::Gemm& g, int kind) {
  char buf[200];
  // the CTA share (concurrency hint) is part of the key: a choice tuned for
  // a product alone is not the one for a product sharing the GPU
  snprintf(buf, sizeof buf, "k%d m%lld n%lld kl%lld kh%lld b%d ab%d bb%d f%lld", kind, (long long)g.M,
           (long long)g.N, (long long)g.K_lo, (long long)g.K_hi, g.batch, g.a_b != 0 ? 1 : 0, g.b_b != 0 ? 1 : 0,
           (long long)g.fill);
  return buf;
}

}  // namespace

namespace mes {

mes_status gemm_tc(const Gemm& g, int kind, float* split_ws, int64_t split_ws_elems, int* err, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return MES_OK;
  MES_TRY(get_encode());
  if (!tc_eligible(g, kind)) return fail(MES_ERR_INVALID_ARG, "gemm_tc: operands not TMA/K-major eligible");
  // tile width: KIND 2 stages four tiles and has only N = 128; otherwise the
  // width that pads N least (ties to 256: fewer re-reads of the A tile)
  int bn0 = 128;
  static const char* variant = getenv("MES_TC_VARIANT");
  const bool p2 = variant && variant[0] == 'p' && variant[1] == '2';
  if (kind < 2 && g.N > 128 && !p2) bn0 = ((g.N + 255) / 256) * 256 <= ((g.N + 127) / 128) * 128 ? 256 : 128;
  if (g.accumulate || g.ref || !tuning_on()) return gemm_tc_cfg(g, kind, bn0, 0, split_ws, split_ws_elems, err, st);
  const std::string key = tune_key(g, kind);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end())
      return gemm_tc_cfg(g, kind, it->second.bn, it->second.splits, split_ws, split_ws_elems, err, st);
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone || g_tune_state != 1) {
    cudaGetLastError();
    return gemm_tc_cfg(g, kind, bn0, 0, split_ws, split_ws_elems, err, st);
  }
  // candidates: both tile widths (one for KIND 2) x split-K 1..16 (>= 4 K-tiles a split)
  const int BK = 128 / kind_bytes(kind);
  const int64_t kt = ((g.K_lo + BK - 1) / BK) * (kind == 3 ? 1 : g.K_hi);
  cudaEvent_t e0, e1;
  MES_CUDA_TRY(cudaEventCreate(&e0));
  MES_CUDA_TRY(cudaEventCreate(&e1));
  TcChoice best{bn0, 1};
  float best_ms = 1e30f;
  const bool was_prof = prof_on();
  for (int bn : {128, 256}) {
    if (bn == 256 && (kind >= 2 || g.N <= 128)) continue;
    for (int sp = 1; sp <= 16; sp *= 2) {
      if (sp > 1 && (!split_ws || kt / sp < 4 || (int64_t)sp * g.batch * g.M * g.N > split_ws_elems)) break;
      cudaEventRecord(e0, st);
      mes_status r = gemm_tc_cfg(g, kind, bn, sp, split_ws, split_ws_elems, err, st);
      cudaEventRecord(e1, st);
      if (r != MES_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r;
      }
      float ms = 0.f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = TcChoice{bn, sp};
      }
      cudaGetLastError();
    }
  }
  (void)was_prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    if (const char* path = getenv("MES_TUNE_CACHE"))
      if (FILE* f = fopen(path, "a")) {
        fprintf(f, "%s = %d %d\n", key.c_str(), best.bn, best.splits);
        fclose(f);
      }
  }
  // the result of the call: the chosen configuration, run last
  return gemm_tc_cfg(g, kind, best.bn, best.splits, split_ws, split_ws_elems, err, st);
}

}  // namespace mes

namespace {

__global__ void to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16_raw* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // round to nearest even on the upper 16 bits
    uint32_t u = __float_as_uint(in[i]);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    __nv_bfloat16_raw r;
    r.x = (unsigned short)(u >> 16);
    out[i] = r;
  }
}

// x -> three BF16 parts x1 = bf(x), x2 = bf(x - x1), x3 = bf(x - x1 - x2)
// (round to nearest even each; both differences are exact in FP32), written
// to out[i], out[plane + i], out[2 plane + i].
__global__ void split_bf16x3_kernel(const float* __restrict__ in, uint16_t* __restrict__ out, int64_t n,
                                    int64_t plane, const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint16_t b1, b2, b3;
    bf16x3_parts(in[i], b1, b2, b3);
    out[i] = b1;
    out[plane + i] = b2;
    out[2 * plane + i] = b3;
  }
}

}  // namespace

namespace mes {

mes_status split_bf16x3(const float* in, uint16_t* out, int64_t n, int64_t plane, const int* skip,
                        cudaStream_t st) {
  if (n <= 0) return MES_OK;
  MES_TRY(audit(in, (size_t)n * 4 - 1, "split_bf16x3 in"));
  MES_TRY(audit(out, (size_t)(2 * plane + n) * 2 - 1, "split_bf16x3 out"));
  ProfScope prof("split_bf16x3", st, 0.0, 10.0 * n);
  split_bf16x3_kernel<<<grid_for(n, 256, (int64_t)sm_count() * 8), 256, 0, st>>>(in, out, n, plane, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

}  // namespace mes

// Test hook: C[m*N + n] = sum_k A[m*K + k] * B[n*K + k] (both row-major,
// K-major), through the CUDA-core kernel (impl 0), kind::tf32 (impl 1),
// kind::f16 on BF16-rounded inputs (impl 2) or the three-term TF32 split of
// A and B (impl 3).
extern "C" mes_status mes_gemm_selftest(int impl, const float* A, const float* B, float* C, int64_t M,
                                        int64_t N, int64_t K, int batch, void* stream) {
  mes::clear_error();
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || batch < 1 || impl < 0 || impl > 4)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_gemm_selftest: bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mes::AuditScope audit_scope;
  mes::audit_register(A, (size_t)(batch * M * K) * 4);
  mes::audit_register(B, (size_t)(batch * N * K) * 4);
  mes::audit_register(C, (size_t)(batch * M * N) * 4);
  mes::Scratch scr(st);
  mes::Gemm g;
  g.M = M; g.N = N; g.K_lo = K; g.batch = batch;
  g.A = A; g.a_m = K; g.a_k = 1; g.a_b = M * K;
  g.B = B; g.b_n = K; g.b_k = 1; g.b_b = N * K;
  g.C = C; g.c_m = N; g.c_n = 1; g.c_b = M * N;
  if (impl == 0) return mes::gemm_f32(g, st);
  int* err = nullptr;
  float* ws = nullptr;
  const int64_t ws_elems = 64 * batch * M * N;
  MES_TRY(scr.alloc(&err, 1));
  MES_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  MES_TRY(scr.alloc(&ws, ws_elems));
  if (impl == 2) {
    __nv_bfloat16_raw *Ab, *Bb;
    MES_TRY(scr.alloc(&Ab, batch * M * K));
    MES_TRY(scr.alloc(&Bb, batch * N * K));
    to_bf16_kernel<<<mes::grid_for(batch * M * K, 256, 4096), 256, 0, st>>>(A, Ab, batch * M * K);
    to_bf16_kernel<<<mes::grid_for(batch * N * K, 256, 4096), 256, 0, st>>>(B, Bb, batch * N * K);
    MES_LAUNCH_CHECK();
    g.A = reinterpret_cast<const float*>(Ab);
    g.B = reinterpret_cast<const float*>(Bb);
  }
  if (impl == 3) {
    float *Ah, *Al, *Bh, *Bl;
    MES_TRY(scr.alloc(&Ah, batch * M * K));
    MES_TRY(scr.alloc(&Al, batch * M * K));
    MES_TRY(scr.alloc(&Bh, batch * N * K));
    MES_TRY(scr.alloc(&Bl, batch * N * K));
    MES_TRY(mes::split_tf32(A, Ah, Al, batch * M * K, st));
    MES_TRY(mes::split_tf32(B, Bh, Bl, batch * N * K, st));
    g.A = Ah; g.A2 = Al;
    g.B = Bh; g.B2 = Bl;
  }
  if (impl == 4) {
    // three BF16 parts of each operand as the K_hi planes (part stride = the operand's size)
    // layout [batch][part][rows][K]: part stride rows*K, batch stride 3*rows*K
    uint16_t *Ap, *Bp;
    MES_TRY(scr.alloc(&Ap, 3 * batch * M * K));
    MES_TRY(scr.alloc(&Bp, 3 * batch * N * K));
    for (int b = 0; b < batch; ++b) {
      MES_TRY(mes::split_bf16x3(A + b * M * K, Ap + 3 * b * M * K, M * K, M * K, nullptr, st));
      MES_TRY(mes::split_bf16x3(B + b * N * K, Bp + 3 * b * N * K, N * K, N * K, nullptr, st));
    }
    g.A = reinterpret_cast<const float*>(Ap); g.K_hi = 3; g.a_kh = M * K; g.a_b = 3 * M * K;
    g.B = reinterpret_cast<const float*>(Bp); g.b_kh = N * K; g.b_b = 3 * N * K;
  }
  MES_TRY(mes::gemm_tc(g, impl == 1 ? 0 : impl == 2 ? 1 : impl == 3 ? 2 : 3, ws, ws_elems, err, st));
  int herr = 0;
  MES_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  MES_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr) return mes::fail(MES_ERR_TIMEOUT, "mes_gemm_selftest: pipeline wait gave up (flags %d)", herr);
  return MES_OK;
}

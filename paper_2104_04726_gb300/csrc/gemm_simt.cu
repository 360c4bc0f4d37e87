// FP32 CUDA-core GEMM over the strided descriptor of gemm.cuh.
//
// 128x128 block tile, 16-deep K slices, 256 threads with an 8x8 register
// tile each, shared-memory double buffering with register staging.  The
// global-load mapping is chosen per operand at compile time so that a warp
// always reads contiguous runs: 16 consecutive k of two rows for a K-major
// operand, 32 consecutive m (or n) for an MN-major one.  The K loop runs over
// (k_hi, k_lo-tile) pairs, so a two-level K index never needs a division;
// only the last k_lo tile of each k_hi is ragged (zero-filled).
#include <algorithm>
#include "gemm.cuh"

namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

template <bool KMAJ, int TILE>
__device__ __forceinline__ void load_tile(const float* __restrict__ base, int64_t rows, int64_t r0,
                                          int64_t s_row, int64_t s_k, int64_t s_kh, int64_t K_lo,
                                          int64_t k_hi, int64_t k_lo0, float (&reg)[8]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int rr, kk;
    if (KMAJ) { kk = t & 15; rr = i * 16 + (t >> 4); }
    else      { rr = t & (TILE - 1); kk = i * (NT / TILE) + t / TILE; }
    int64_t r = r0 + rr, k = k_lo0 + kk;
    float v = 0.f;
    if (r < rows && k < K_lo) v = __ldg(base + r * s_row + k * s_k + k_hi * s_kh);
    reg[i] = v;
  }
}

template <bool KMAJ, int TILE>
__device__ __forceinline__ void store_tile(float (*S)[TILE + 4], const float (&reg)[8]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int rr, kk;
    if (KMAJ) { kk = t & 15; rr = i * 16 + (t >> 4); }
    else      { rr = t & (TILE - 1); kk = i * (NT / TILE) + t / TILE; }
    S[kk][rr] = reg[i];
  }
}

template <bool AK, bool BKM, bool RESID>
__global__ void __launch_bounds__(NT) gemm_kernel(const mes::Gemm g, int splits, int64_t tiles_per_split) {
  if (g.skip && *g.skip) return;
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];

  const int t = threadIdx.x;
  const int64_t bm = (int64_t)blockIdx.x * BM;
  const int64_t bn = (int64_t)blockIdx.y * BN;
  const int b = blockIdx.z % g.batch;
  const int split = blockIdx.z / g.batch;
  if (g.lower && bm + BM <= bn) return;  // wholly above the diagonal
  const float* A = g.A + (int64_t)b * g.a_b;
  const float* B = g.B + (int64_t)b * g.b_b;

  const int64_t nkl = (g.K_lo + BK - 1) / BK;
  const int64_t tt_begin = split * tiles_per_split;
  int64_t tiles = nkl * g.K_hi - tt_begin;
  if (tiles > tiles_per_split) tiles = tiles_per_split;
  int64_t kh_next = tt_begin / nkl, kl_next = (tt_begin - (tt_begin / nkl) * nkl) * BK;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float ra[8], rb[8];
  int cur = 0;
  if (tiles > 0) {
    load_tile<AK, BM>(A, g.M, bm, g.a_m, g.a_k, g.a_kh, g.K_lo, kh_next, kl_next, ra);
    load_tile<BKM, BN>(B, g.N, bn, g.b_n, g.b_k, g.b_kh, g.K_lo, kh_next, kl_next, rb);
    store_tile<AK, BM>(As[0], ra);
    store_tile<BKM, BN>(Bs[0], rb);
  }
  __syncthreads();

  const int ty = t >> 4, tx = t & 15;
  for (int64_t tt = 0; tt < tiles; ++tt) {
    const bool more = tt + 1 < tiles;
    if (more) {
      kl_next += BK;
      if (kl_next >= g.K_lo) { kl_next = 0; ++kh_next; }
      load_tile<AK, BM>(A, g.M, bm, g.a_m, g.a_k, g.a_kh, g.K_lo, kh_next, kl_next, ra);
      load_tile<BKM, BN>(B, g.N, bn, g.b_n, g.b_k, g.b_kh, g.K_lo, kh_next, kl_next, rb);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[8], bv[8];
      float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
      bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
    }
    if (more) {
      store_tile<AK, BM>(As[cur ^ 1], ra);
      store_tile<BKM, BN>(Bs[cur ^ 1], rb);
    }
    __syncthreads();
    cur ^= 1;
  }

  // epilogue
  int64_t moff[8], noff[8];
  bool mok[8], nok[8];
  const int64_t M_lo = g.M_lo > 0 ? g.M_lo : g.M;
  const int64_t N_lo = g.N_lo > 0 ? g.N_lo : g.N;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int64_t m = bm + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    mok[i] = m < g.M;
    int64_t mh = m / M_lo, ml = m - mh * M_lo;
    moff[i] = ml * g.c_m + mh * g.c_mh;
    int64_t n = bn + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
    nok[i] = n < g.N;
    int64_t nh = n / N_lo, nl = n - nh * N_lo;
    noff[i] = nl * g.c_n + nh * g.c_nh;
  }
  const int64_t cb = (int64_t)b * g.c_b;
  if (splits > 1) {
    float* ws = g.split_ws + ((int64_t)split * g.batch + b) * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (!mok[i]) continue;
      int64_t m = bm + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int64_t n = bn + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        if (nok[j]) ws[m * g.N + n] = acc[i][j];
      }
    }
    return;
  }
  if (RESID) {
    // the thread's 64 squares summed in FP32, one FP64 value per thread
    float sf = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (mok[i] && nok[j]) {
          const float v = g.alpha * acc[i][j];
          float d = __ldg(g.ref + cb + moff[i] + noff[j]) - v;
          sf = fmaf(d, d, sf);
          if (g.C) g.C[cb + moff[i] + noff[j]] = v;   // the product is stored too
        }
    double s = sf;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[NT / 32];
    if ((t & 31) == 0) red[t >> 5] = s;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
      for (int w = 0; w < NT / 32; ++w) tot += red[w];
      int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      g.partials[bid] = tot;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (mok[i] && nok[j]) {
          float* p = g.C + cb + moff[i] + noff[j];
          float v = g.alpha * acc[i][j];
          v = g.accumulate ? *p + v : v;
          *p = g.round_tf32 ? mes::round_tf32(v) : v;
        }
    if (g.C2) {
      const int64_t M_lo2 = M_lo, N_lo2 = N_lo;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (!mok[i]) continue;
        int64_t m = bm + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        int64_t mh = m / M_lo2, ml = m - mh * M_lo2;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (!nok[j]) continue;
          int64_t n = bn + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
          int64_t nh = n / N_lo2, nl = n - nh * N_lo2;
          const float v2 = g.alpha * acc[i][j];
          g.C2[(int64_t)b * g.c2_b + ml * g.c2_m + mh * g.c2_mh + nl * g.c2_n + nh * g.c2_nh] =
              g.round_tf32 ? mes::round_tf32(v2) : v2;
        }
      }
    }
  }
}

// Fixed-order sum of split-K partial tiles into C (general strides).
__global__ void split_sum_kernel(const mes::Gemm g, int splits) {
  if (g.skip && *g.skip) return;
  const int64_t total = (int64_t)g.batch * g.M * g.N;
  const int64_t M_lo = g.M_lo > 0 ? g.M_lo : g.M, N_lo = g.N_lo > 0 ? g.N_lo : g.N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float sacc = 0.f;
    for (int sp = 0; sp < splits; ++sp) sacc += g.split_ws[(int64_t)sp * total + e];
    const int64_t n = e % g.N, bm = e / g.N;
    const int64_t m = bm % g.M, b = bm / g.M;
    if (g.lower && (m / BM + 1) * BM <= (n / BN) * BN) continue;  // tile never computed
    const int64_t mh = m / M_lo, ml = m - mh * M_lo, nh = n / N_lo, nl = n - nh * N_lo;
    float v = g.alpha * sacc;
    float* p = g.C + b * g.c_b + ml * g.c_m + mh * g.c_mh + nl * g.c_n + nh * g.c_nh;
    v = g.accumulate ? *p + v : v;
    if (g.round_tf32) v = mes::round_tf32(v);
    *p = v;
    if (g.C2) g.C2[b * g.c2_b + ml * g.c2_m + mh * g.c2_mh + nl * g.c2_n + nh * g.c2_nh] = v;
  }
}

__global__ void sum_doubles_kernel(const double* __restrict__ p, int64_t n, double* __restrict__ out,
                                   const int* skip) {
  if (skip && *skip) return;
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

template <bool AK, bool BKM>
mes_status launch(const mes::Gemm& g, dim3 grid, cudaStream_t st) {
  const double K = (double)g.K_lo * g.K_hi, bt = g.batch;
  // split K when the tile grid leaves most SMs idle (not in residual mode)
  const int64_t nkt = ((g.K_lo + BK - 1) / BK) * g.K_hi;
  int64_t tiles = (int64_t)grid.x * grid.y * grid.z;
  if (g.lower) {  // tiles (i, j) with j <= i
    int64_t lt = 0;
    for (int64_t i = 0; i < (int64_t)grid.x; ++i) lt += std::min<int64_t>(i + 1, grid.y);
    tiles = lt * grid.z;
  }
  const int64_t sms = g.fill > 0 ? g.fill : mes::sm_count();
  int splits = 1;
  if (!g.ref && g.split_ws && tiles < sms) {
    // one wave of CTAs (the register tile allows one per SM), at least 8
    // K-tiles each
    int64_t want = sms / tiles;
    if (want > nkt / 8) want = nkt / 8;
    while (want > 1 && want * g.batch * g.M * g.N > g.split_elems) --want;
    splits = want > 1 ? (int)want : 1;
  }
  const int64_t per = (nkt + splits - 1) / splits;
  splits = (int)((nkt + per - 1) / per);
  grid.z *= splits;
  {
    mes::ProfScope prof("gemm_f32_simt", st, 2.0 * g.M * g.N * K * bt,
                        4.0 * bt * (g.M * K + g.N * K + g.M * (double)g.N));
    if (g.ref)
      gemm_kernel<AK, BKM, true><<<grid, NT, 0, st>>>(g, splits, per);
    else
      gemm_kernel<AK, BKM, false><<<grid, NT, 0, st>>>(g, splits, per);
    MES_LAUNCH_CHECK();
  }
  if (splits > 1) {
    mes::ProfScope prof("split_reduce", st, 0.0, 4.0 * splits * bt * g.M * (double)g.N);
    const int64_t total = (int64_t)g.batch * g.M * g.N;
    split_sum_kernel<<<mes::grid_for(total, 256, sms * 8), 256, 0, st>>>(g, splits);
    MES_LAUNCH_CHECK();
  }
  return MES_OK;
}

dim3 grid_of(const mes::Gemm& g) {
  return dim3((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + BN - 1) / BN), (unsigned)g.batch);
}

}  // namespace

namespace mes {

int64_t gemm_partials(const Gemm& g) {
  dim3 gr = grid_of(g);
  return (int64_t)gr.x * gr.y * gr.z;
}

mes_status gemm_f32(const Gemm& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return MES_OK;
  if (g.K_lo <= 0 || g.K_hi <= 0) return fail(MES_ERR_INVALID_ARG, "gemm: empty K");
  if ((g.N + BN - 1) / BN > 65535 || g.batch > 65535)
    return fail(MES_ERR_INVALID_ARG, "gemm: grid too large");
  dim3 grid = grid_of(g);
  {
    const int64_t M_lo = g.M_lo > 0 ? g.M_lo : g.M, N_lo = g.N_lo > 0 ? g.N_lo : g.N;
    const int64_t bt = g.batch - 1;
    size_t a_last = ((g.M - 1) * g.a_m + (g.K_lo - 1) * g.a_k + (g.K_hi - 1) * g.a_kh + bt * g.a_b) * 4;
    size_t b_last = ((g.N - 1) * g.b_n + (g.K_lo - 1) * g.b_k + (g.K_hi - 1) * g.b_kh + bt * g.b_b) * 4;
    int64_t mlo = g.M < M_lo ? g.M - 1 : M_lo - 1, mhi = (g.M - 1) / M_lo;
    int64_t nlo = g.N < N_lo ? g.N - 1 : N_lo - 1, nhi = (g.N - 1) / N_lo;
    size_t c_last = (mlo * g.c_m + mhi * g.c_mh + nlo * g.c_n + nhi * g.c_nh + bt * g.c_b) * 4;
    if (g.a_m < 0 || g.a_k < 0 || g.a_kh < 0 || g.a_b < 0 || g.b_n < 0 || g.b_k < 0 || g.b_kh < 0 ||
        g.b_b < 0 || g.c_m < 0 || g.c_mh < 0 || g.c_n < 0 || g.c_nh < 0 || g.c_b < 0)
      return fail(MES_ERR_INVALID_ARG, "gemm: negative stride");
    MES_TRY(audit(g.A, a_last, "gemm A"));
    MES_TRY(audit(g.B, b_last, "gemm B"));
    MES_TRY(audit(g.C, c_last, "gemm C"));
    MES_TRY(audit(g.ref, c_last, "gemm ref"));
    if (g.ref) MES_TRY(audit(g.partials, (size_t)gemm_partials(g) * 8 - 1, "gemm partials"));
  }
  // An operand is treated as K-major when its k stride is the unit one.
  const bool ak = (g.a_k == 1);
  const bool bk = (g.b_k == 1);
  if (ak && bk) return launch<true, true>(g, grid, st);
  if (ak && !bk) return launch<true, false>(g, grid, st);
  if (!ak && bk) return launch<false, true>(g, grid, st);
  return launch<false, false>(g, grid, st);
}

mes_status sum_doubles(const double* partials, int64_t n, double* out, const int* skip,
                       cudaStream_t st) {
  ProfScope prof("sum_doubles", st, 0.0, 8.0 * n);
  sum_doubles_kernel<<<1, 256, 0, st>>>(partials, n, out, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

}  // namespace mes

// Small dense solvers of the factor update (Section III-B, text after Eq. 8:
// the factor is taken from the leading eigenvectors of the Gram).
//
//  * chol + trsm: one pass of shifted CholeskyQR, V = W R^-1 with
//               R^T R = M = W^T W (equilibrated, shifted): the Cholesky on
//               one CTA, the triangular solve over all rows of W on many.
//  * eig_small: FP64 cyclic Jacobi for the Grams of the small modes
//               (colour, view x exposure; n <= 32), one warp per matrix.
//  * eig_mid:   FP32 parallel (round-robin) Jacobi for an r x r symmetric
//               matrix with r <= 128 held in shared memory; used for the
//               Rayleigh-Ritz rotation of the factors at the end.
//
// GB300's FP64 rate is a small fraction of its FP32 rate, so O(r^3) work at
// r in the hundreds runs in FP32; FP64 is used where the work is O(n^3) with
// n <= 32 and for accumulations.
#include <cooperative_groups.h>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int PB = 32;

// --------------------------------------------------------------------------
// chol: equilibrated, shifted Cholesky of a symmetric r x r Gram M (one CTA,
// 256 threads).  A = D^-1 M D^-1 + shift * r * I = L L^T with D = diag(M)^1/2.
// Outputs L (lower triangle of `L`, column-major) and dinv = 1 / diag(D).
// Blocked by 32 columns: the diagonal block is factored by one warp in
// registers, the panel below is solved by forward substitution (one row per
// thread), the trailing lower triangle is updated in 8 x 8 tiles.
// The shift starts at shift_rel and is raised tenfold (up to 1e-2) whenever a
// pivot falls below max(1e-7, 0.1 * shift): it must dominate the FP32
// rounding of the Gram, yet stay small so the next pass is well conditioned.
// --------------------------------------------------------------------------
constexpr int kChol = 256;

// One column step of the 32 x 32 factorization held one row per lane in
// registers; J is a compile-time index so row[] never spills to local memory.
// The pivot of step J+1 is formed and broadcast before the column update so
// the serial chain per step is shuffle -> rsqrt -> multiply -> FMA; the
// scaled column J goes through shared memory (colbuf row J) and is read back
// as float4 broadcasts.  rdiag[J] receives 1 / L_JJ.
template <int J>
__device__ __forceinline__ void chol_step(float (&row)[PB], float piv, int lane, int b, float floor, int* bad,
                                          float* colbuf, float* rdiag) {
  if constexpr (J < PB) {
    if (J < b) {
      if (!(piv > floor)) {
        if (lane == 0) *bad = 1;
        piv = floor;
      }
    } else {
      piv = 1.f;
    }
    const float rs = rsqrtf(piv);
    const float l = (lane == J) ? piv * rs : row[J] * rs;
    if (lane >= J) row[J] = l;
    if (lane == J) rdiag[J] = rs;
    if constexpr (J + 1 < PB) {
      // the next pivot first: lane J+1 holds it and needs only its own l
      // (the same value the column update below gives it)
      const float next = __shfl_sync(0xffffffffu, fmaf(-l, l, row[J + 1]), J + 1);
      colbuf[J * PB + lane] = (lane > J) ? l : 0.f;
      __syncwarp();
      constexpr int K0 = (J + 1) & ~3;
#pragma unroll
      for (int k4 = K0; k4 < PB; k4 += 4) {
        const float4 c = *reinterpret_cast<const float4*>(colbuf + J * PB + k4);
        const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          // lanes < k only touch the upper part, which is never read
          const int k = k4 + u;
          if (k > J) row[k] = fmaf(-l, cv[u], row[k]);
        }
      }
      chol_step<J + 1>(row, next, lane, b, floor, bad, colbuf, rdiag);
    }
  }
}

// Inverse of a 32 x 32 lower-triangular block held in shared memory with row
// stride 33: lane j computes column j of L^-1 by forward substitution (the
// rows of L are read as broadcasts); stored row-major to out[i * 32 + j].
__device__ __forceinline__ void warp_tri_inv32(const float* Ls, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  float x[PB];
#pragma unroll
  for (int i = 0; i < PB; ++i) x[i] = (i == lane) ? 1.f : 0.f;
#pragma unroll
  for (int i = 0; i < PB; ++i) {
    const float xi = x[i] / Ls[i * (PB + 1) + i];
    x[i] = xi;
#pragma unroll
    for (int m = i + 1; m < PB; ++m) x[m] = fmaf(-Ls[m * (PB + 1) + i], xi, x[m]);
  }
#pragma unroll
  for (int i = 0; i < PB; ++i) out[i * PB + lane] = x[i];
}

// One column of the forward substitution x L^T = a for a row held in
// registers: colbuf row C holds column C of L below the diagonal, rdiag the
// reciprocals of its diagonal.  C is a compile-time index (no local memory).
template <int C>
__device__ __forceinline__ void panel_step(float (&a)[PB], const float* colbuf, const float* rdiag) {
  if constexpr (C < PB) {
    const float x = a[C] * rdiag[C];
    a[C] = x;
#pragma unroll
    for (int j4 = (C + 1) & ~3; j4 < PB; j4 += 4) {
      const float4 v = *reinterpret_cast<const float4*>(colbuf + C * PB + j4);
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j4 + u > C) a[j4 + u] = fmaf(-x, vv[u], a[j4 + u]);
    }
    asm volatile("" ::: "memory");   // keep the next column's loads after this one's
    panel_step<C + 1>(a, colbuf, rdiag);
  }
}

// 32 x 32 diagonal block (rows of Dg with stride 33, lower part; rows/cols
// at and beyond b are treated as identity) -> L in place (upper part zeroed)
// and rdiag = 1 / diag(L).  colbuf: 32 x 32 floats of shared memory, 16-byte
// aligned.  One warp.
__device__ __forceinline__ void warp_chol32(float* Dg, int b, float floor, int* bad, float* colbuf, float* rdiag) {
  const int lane = threadIdx.x & 31;
  float row[PB];
#pragma unroll
  for (int k = 0; k < PB; ++k) row[k] = (k <= lane && lane < b && k < b) ? Dg[lane * (PB + 1) + k] : (k == lane ? 1.f : 0.f);
  chol_step<0>(row, __shfl_sync(0xffffffffu, row[0], 0), lane, b, floor, bad, colbuf, rdiag);
#pragma unroll
  for (int k = 0; k < PB; ++k) Dg[lane * (PB + 1) + k] = (k <= lane) ? row[k] : 0.f;
}

__global__ void __launch_bounds__(kChol)
chol_kernel(const float* __restrict__ Min, int r, float shift_rel, float* __restrict__ A,
            float* __restrict__ dinv_out, int* __restrict__ flags, const int* __restrict__ skip,
            int* __restrict__ clean) {
  if (skip && *skip) {
    if (clean && threadIdx.x == 0) *clean = 1;
    return;
  }
  int restarts = 0;
  extern __shared__ float smem[];
  float* dinv = smem;                       // 1024
  float* Dg = dinv + 1024;                  // 32 x 33
  float* Pn = Dg + PB * (PB + 1);           // up to 1024 x 33 (panel)
  __shared__ int bad;
  __shared__ float Drc[PB];                 // reciprocals of the diagonal of L_pp
  __shared__ __align__(16) float colbuf[PB * PB];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  // flags[0]: error bits; flags[1]: calls; flags[2]: shift restarts
  if (t == 0 && flags) atomicAdd(flags + 1, 1);

  for (int i = t; i < r; i += kChol) {
    float v = Min[i + (int64_t)r * i];
    bool ok = v > 0.f && isfinite(v);
    if (!ok && flags) atomicOr(flags, 2);
    float dv = 1.f / (ok ? sqrtf(v) : 1.f);
    dinv[i] = dv;
    dinv_out[i] = dv;
  }
  __syncthreads();
  float rel = shift_rel;
  for (int attempt = 0; attempt < 8; ++attempt) {
    const float shift = rel * (float)r;
    const float floor = fmaxf(1e-7f, 0.1f * shift);
    if (t == 0) bad = 0;
    // column j by warp, rows by lane: no integer division in the loop
    for (int j = warp; j < r; j += kChol / 32) {
      const float dj = dinv[j];
      for (int i = j + (t & 31); i < r; i += 32) {
        const int64_t e = i + (int64_t)r * j;
        float v = Min[e] * dinv[i] * dj;
        if (i == j) v += shift;
        A[e] = v;
      }
    }
    __syncthreads();
    for (int p0 = 0; p0 < r; p0 += PB) {
      const int b = min(PB, r - p0);
      for (int e = t; e < PB * PB; e += kChol) {
        int i = e & 31, j = e >> 5;
        Dg[i * (PB + 1) + j] = (i < b && j < b && i >= j) ? A[(p0 + i) + (int64_t)r * (p0 + j)] : 0.f;
      }
      __syncthreads();
      if (warp == 0) warp_chol32(Dg, b, floor, &bad, colbuf, Drc);
      __syncthreads();
      for (int e = t; e < b * b; e += kChol) {
        int i = e % b, j = e / b;
        if (i >= j) A[(p0 + i) + (int64_t)r * (p0 + j)] = Dg[i * (PB + 1) + j];
      }
      const int rows = r - p0 - b;
      // panel: L[i, p0:p0+b] solves x L_pp^T = A[i, p0:p0+b] (forward substitution)
      for (int ii = t; ii < rows; ii += kChol) {
        const int i = p0 + b + ii;
        float a[PB];
#pragma unroll
        for (int c = 0; c < PB; ++c) a[c] = (c < b) ? A[i + (int64_t)r * (p0 + c)] : 0.f;
#pragma unroll
        for (int c = 0; c < PB; ++c) {
          float v = a[c];
#pragma unroll
          for (int k = 0; k < c; ++k) v = fmaf(-a[k], Dg[c * (PB + 1) + k], v);
          a[c] = (c < b) ? v * Drc[c] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < PB; ++c) {
          if (c < b) A[i + (int64_t)r * (p0 + c)] = a[c];
          Pn[ii * (PB + 1) + c] = a[c];
        }
      }
      __syncthreads();
      const int nt = (rows + 7) / 8;
      const int ntiles = nt * (nt + 1) / 2;
      for (int tile = t; tile < ntiles; tile += kChol) {
        int bi = (int)((sqrtf(8.f * tile + 1.f) - 1.f) * 0.5f);
        while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
        while (bi * (bi + 1) / 2 > tile) --bi;
        int bj = tile - bi * (bi + 1) / 2;
        float acc[8][8];
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
        for (int c = 0; c < b; ++c) {
          float u[8], v[8];
#pragma unroll
          for (int x = 0; x < 8; ++x) {
            int ri = bi * 8 + x, rj = bj * 8 + x;
            u[x] = (ri < rows) ? Pn[ri * (PB + 1) + c] : 0.f;
            v[x] = (rj < rows) ? Pn[rj * (PB + 1) + c] : 0.f;
          }
#pragma unroll
          for (int x = 0; x < 8; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(u[x], v[y], acc[x][y]);
        }
        // all 64 loads first: independent, so they overlap in flight
        float old[8][8];
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) {
            int ri = bi * 8 + x, rj = bj * 8 + y;
            old[x][y] = (ri < rows && rj < rows && ri >= rj) ? A[(p0 + b + ri) + (int64_t)r * (p0 + b + rj)] : 0.f;
          }
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) {
            int ri = bi * 8 + x, rj = bj * 8 + y;
            if (ri < rows && rj < rows && ri >= rj) A[(p0 + b + ri) + (int64_t)r * (p0 + b + rj)] = old[x][y] - acc[x][y];
          }
      }
      __syncthreads();
    }
    if (!bad) break;
    if (t == 0 && flags) {
      atomicOr(flags, 1);
      atomicAdd(flags + 2, 1);
    }
    ++restarts;
    rel = (rel == 0.f) ? 1e-6f : rel * 10.f;
    if (rel > 1e-2f) rel = 1e-2f;
    __syncthreads();
  }
  if (clean && t == 0) *clean = restarts == 0;
}

// --------------------------------------------------------------------------
// chol_cluster: the same factorization spread over a cluster of kCL CTAs on
// kCL SMs (for r > 128, where one SM would need ~r^3/3 FP32 FMAs alone).
// Every CTA factors the 32 x 32 diagonal block itself (same data, same code,
// same result, so no broadcast is needed); the panel rows and the
// trailing-update tiles are split across the CTAs; cluster barriers order the
// phases.  The matrix lives in global memory (L2); it is read with
// ld.global.cg and written with st.global.cg so no CTA sees a stale L1 line.
// --------------------------------------------------------------------------
constexpr int kCL = 8;

__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kChol)
chol_cluster_kernel(const float* __restrict__ Min, int r, float shift_rel, float* __restrict__ A,
                    float* __restrict__ dinv_out, int* __restrict__ flags, const int* __restrict__ skip,
                    int* __restrict__ clean) {
  if (skip && *skip) {
    if (clean && blockIdx.x == 0 && threadIdx.x == 0) *clean = 1;
    return;
  }
  int restarts = 0;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ float smem[];
  float* dinv = smem;                       // 1024
  float* Dg = dinv + 1024;                  // 32 x 33
  float* Pn = Dg + PB * (PB + 1);           // up to 1024 x 33 (panel)
  __shared__ int bad;
  __shared__ float Drc[PB];                 // reciprocals of the diagonal of L_pp
  __shared__ __align__(16) float colbuf[PB * PB];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (rank == 0 && t == 0 && flags) atomicAdd(flags + 1, 1);

  for (int i = t; i < r; i += kChol) {
    float v = Min[i + (int64_t)r * i];
    bool ok = v > 0.f && isfinite(v);
    if (!ok && flags && rank == 0) atomicOr(flags, 2);
    float dv = 1.f / (ok ? sqrtf(v) : 1.f);
    dinv[i] = dv;
    if (rank == 0) dinv_out[i] = dv;
  }
  __syncthreads();
  float rel = shift_rel;
  for (int attempt = 0; attempt < 8; ++attempt) {
    const float shift = rel * (float)r;
    const float floor = fmaxf(1e-7f, 0.1f * shift);
    if (t == 0) bad = 0;
    for (int j = rank + kCL * warp; j < r; j += kCL * (kChol / 32)) {
      const float dj = dinv[j];
      for (int i = j + lane; i < r; i += 32) {
        const int64_t e = i + (int64_t)r * j;
        float v = Min[e] * dinv[i] * dj;
        if (i == j) v += shift;
        __stcg(A + e, v);
      }
    }
    __threadfence();
    cluster.sync();
    for (int p0 = 0; p0 < r; p0 += PB) {
      const int b = min(PB, r - p0);
      for (int e = t; e < PB * PB; e += kChol) {
        int i = e & 31, j = e >> 5;
        Dg[i * (PB + 1) + j] = (i < b && j < b && i >= j) ? __ldcg(A + (p0 + i) + (int64_t)r * (p0 + j)) : 0.f;
      }
      __syncthreads();
      if (warp == 0) warp_chol32(Dg, b, floor, &bad, colbuf, Drc);
      __syncthreads();
      if (rank == 0)
        for (int e = t; e < b * b; e += kChol) {
          int i = e % b, j = e / b;
          if (i >= j) __stcg(A + (p0 + i) + (int64_t)r * (p0 + j), Dg[i * (PB + 1) + j]);
        }
      const int rows = r - p0 - b;
      for (int ii = rank + kCL * t; ii < rows; ii += kCL * kChol) {
        const int i = p0 + b + ii;
        float a[PB];
#pragma unroll
        for (int c = 0; c < PB; ++c) a[c] = (c < b) ? __ldcg(A + i + (int64_t)r * (p0 + c)) : 0.f;
#pragma unroll
        for (int c = 0; c < PB; ++c) {
          float v = a[c];
#pragma unroll
          for (int k = 0; k < c; ++k) v = fmaf(-a[k], Dg[c * (PB + 1) + k], v);
          a[c] = (c < b) ? v * Drc[c] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < PB; ++c)
          if (c < b) __stcg(A + i + (int64_t)r * (p0 + c), a[c]);
      }
      __threadfence();
      cluster.sync();
      if (rows > 0) {
        for (int ii = t; ii < rows; ii += kChol) {
          float v[PB];
#pragma unroll
          for (int c = 0; c < PB; ++c) v[c] = (c < b) ? __ldcg(A + (p0 + b + ii) + (int64_t)r * (p0 + c)) : 0.f;
#pragma unroll
          for (int c = 0; c < PB; ++c) Pn[ii * (PB + 1) + c] = v[c];
        }
        __syncthreads();
        const int nt = (rows + 7) / 8;
        const int ntiles = nt * (nt + 1) / 2;
        for (int tile = rank + kCL * t; tile < ntiles; tile += kCL * kChol) {
          int bi = (int)((sqrtf(8.f * tile + 1.f) - 1.f) * 0.5f);
          while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
          while (bi * (bi + 1) / 2 > tile) --bi;
          int bj = tile - bi * (bi + 1) / 2;
          float acc[8][8];
#pragma unroll
          for (int x = 0; x < 8; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
          for (int c = 0; c < b; ++c) {
            float u[8], v[8];
#pragma unroll
            for (int x = 0; x < 8; ++x) {
              int ri = bi * 8 + x, rj = bj * 8 + x;
              u[x] = (ri < rows) ? Pn[ri * (PB + 1) + c] : 0.f;
              v[x] = (rj < rows) ? Pn[rj * (PB + 1) + c] : 0.f;
            }
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
              for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(u[x], v[y], acc[x][y]);
          }
          float old[8][8];
#pragma unroll
          for (int x = 0; x < 8; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) {
              int ri = bi * 8 + x, rj = bj * 8 + y;
              old[x][y] = (ri < rows && rj < rows && ri >= rj) ? __ldcg(A + (p0 + b + ri) + (int64_t)r * (p0 + b + rj)) : 0.f;
            }
#pragma unroll
          for (int x = 0; x < 8; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) {
              int ri = bi * 8 + x, rj = bj * 8 + y;
              if (ri < rows && rj < rows && ri >= rj) __stcg(A + (p0 + b + ri) + (int64_t)r * (p0 + b + rj), old[x][y] - acc[x][y]);
            }
        }
      }
      __threadfence();
      cluster.sync();
    }
    if (!bad) break;
    if (rank == 0 && t == 0 && flags) {
      atomicOr(flags, 1);
      atomicAdd(flags + 2, 1);
    }
    ++restarts;
    rel = (rel == 0.f) ? 1e-6f : rel * 10.f;
    if (rel > 1e-2f) rel = 1e-2f;
    __syncthreads();
  }
  if (clean && rank == 0 && t == 0) *clean = restarts == 0;
}

// --------------------------------------------------------------------------
// chol_dsm: the factorization for 128 < r <= 512 with the whole matrix held
// in the shared memory of a cluster of kCL CTAs.
// Block column k (rows 32k .. rp-1, rp = r rounded up to 32; rows at and
// beyond r are zero) lives in CTA k mod kCL, row-major with stride 33.
// Each column is written to L as soon as it is factored; in step p every CTA
// that owns a column right of p copies the rows of panel p it needs from L
// (through L2: measured faster here than reading the owner's shared memory
// across the cluster); the owner of column p + 1 applies panel p to that
// column first, factors its diagonal block in registers and solves its
// panel (look-ahead), then every CTA applies panel p to the rest of its
// columns.  One cluster barrier per step; a bad pivot is reported to CTA 0's
// flag for the attempt and every CTA reads it after the same barrier, so all
// restart together.
// --------------------------------------------------------------------------
constexpr int kDsmMaxR = 512;
static_assert(kChol == 256, "the diagonal-block update maps 8 warps to 32 columns");
constexpr int LD = PB + 1;

template <int CL>
__device__ __forceinline__ int dsm_slot_offset(int rank, int slot, int rp) {
  int off = 0;
  for (int q = 0; q < slot; ++q) off += rp - PB * (rank + CL * q);
  return off;  // rows
}

__host__ __device__ inline size_t chol_dsm_smem(int r, int cl) {
  const int rp = (r + PB - 1) / PB * PB, nb = rp / PB;
  int rows = 0;  // CTA 0 holds the most rows
  for (int k = 0; k < nb; k += cl) rows += rp - PB * k;
  return (size_t)((rows + rp) * LD + rp + 8) * sizeof(float);
}

// CL CTAs in the cluster (kCL; the code holds for any CL whose owned block
// columns fit one CTA's shared memory)
template <int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kChol, 1)
chol_dsm_kernel(const float* __restrict__ Min, int r, float shift_rel, float* __restrict__ Lout,
                float* __restrict__ dinv_out, float* __restrict__ Linv_blk, int* __restrict__ flags,
                const int* __restrict__ skip, int* __restrict__ clean) {
  if (skip && *skip) {
    if (clean && blockIdx.x == 0 && threadIdx.x == 0) *clean = 1;
    return;
  }
  int restarts = 0;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int rp = (r + PB - 1) / PB * PB, nb = rp / PB;
  extern __shared__ __align__(16) float smem[];
  float* dinv = smem;              // rp
  float* store = dinv + rp;        // owned block columns
  int store_rows = 0;
  for (int k = rank; k < nb; k += CL) store_rows += rp - PB * k;
  // panel rows read from L (row stride 33)
  float* Pl_alloc = smem + rp + store_rows * LD;
  // bad-pivot flags per attempt and step parity; CTA 0's copy is the
  // cluster's.  A factor in step p reports to [p & 1]; the flag is read at the
  // top of step p + 1, before anyone can reach step p + 2 and write that
  // parity again, so every CTA reads the same value.
  __shared__ int badv[8][2];
  __shared__ int lbad;
  __shared__ float Drc[PB];
  __shared__ __align__(16) float colbuf[PB * PB];
  if (t < 16) badv[t >> 1][t & 1] = 0;
  if (rank == 0 && t == 0 && flags) atomicAdd(flags + 1, 1);
  for (int i = t; i < rp; i += kChol) {
    float dv = 0.f;
    if (i < r) {
      const float v = Min[i + (int64_t)r * i];
      const bool ok = v > 0.f && isfinite(v);
      if (!ok && flags && rank == 0) atomicOr(flags, 2);
      dv = 1.f / (ok ? sqrtf(v) : 1.f);
      if (rank == 0) dinv_out[i] = dv;
    }
    dinv[i] = dv;
  }
  volatile int* bad0 = cluster.map_shared_rank(&badv[0][0], 0);
  cluster.sync();  // every badv zeroed before anyone can report

  // rows 32 .. h-1 of the owner's column k solve x L_kk^T = a (one row a
  // thread); colbuf row c holds column c of L_kk below the diagonal and is
  // read as float4 broadcasts
  auto panel_solve = [&](float* Sk, int k) {
    const int h = rp - PB * k;
    for (int i = PB + t; i < h; i += kChol) {
      float a[PB];
#pragma unroll
      for (int c = 0; c < PB; ++c) a[c] = Sk[i * LD + c];
      panel_step<0>(a, colbuf, Drc);
#pragma unroll
      for (int c = 0; c < PB; ++c) Sk[i * LD + c] = a[c];
    }
  };
  // the owner writes its factored column k (lower part) to L, where it is
  // final and where the other CTAs read it as the next panel (through L2)
  auto publish = [&](const float* Sk, int k) {
    const int hr = r - PB * k;
    const int w = min(PB, hr);
    float* Lk = Lout + (PB * k) + (int64_t)r * (PB * k);
    for (int i = t; i < hr; i += kChol)
#pragma unroll 8
      for (int c = 0; c < w; ++c)
        if (i >= c) __stcg(Lk + i + (int64_t)r * c, Sk[i * LD + c]);
  };
  // apply the copied panel (global rows g_lo .. rp-1 at P) to rows
  // [i_begin, i_end) of owned column k, by warps w0 .. w0+nw-1: items of 128
  // rows x 4 columns, lane = row (+32 x), 4 x 4 registers
  auto update_col = [&](float* Sk, int k, const float* P, int g_lo, int i_begin, int i_end, int w0, int nw) {
    const int items = ((i_end - i_begin + 127) / 128) * 8;
    const float* prow = P + (PB * k - g_lo) * LD;
    for (int it = warp - w0; it < items; it += nw) {
      const int i0 = i_begin + (it >> 3) * 128 + lane, c0 = (it & 7) * 4;
      const float* pc = prow + c0 * LD;
      float acc[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 8
      for (int q = 0; q < PB; ++q) {
        float u[4], v[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) u[x] = (i0 + 32 * x < i_end) ? prow[(i0 + 32 * x) * LD + q] : 0.f;
#pragma unroll
        for (int y = 0; y < 4; ++y) v[y] = pc[y * LD + q];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(u[x], v[y], acc[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int i = i0 + 32 * x;
        if (i < i_end)
#pragma unroll
          for (int y = 0; y < 4; ++y) Sk[i * LD + c0 + y] -= acc[x][y];
      }
    }
  };

  float rel = shift_rel;
  for (int attempt = 0; attempt < 8; ++attempt) {
    const float shift = rel * (float)r;
    const float floor = fmaxf(1e-7f, 0.1f * shift);
    if (t == 0) lbad = 0;
    // owned columns of A = D^-1 M D^-1 + shift I (lower part; rows >= r zero)
    for (int k = rank, off = 0; k < nb; off += rp - PB * k, k += CL) {
      const int h = rp - PB * k;
      float* Sk = store + off * LD;
      // eight loads in flight a thread before the stores (one at a time made
      // this a chain of h / 8 round trips to L2 or DRAM)
      for (int e0 = t; e0 < h * PB; e0 += 8 * kChol) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kChol;
          const int i = e % h, c = e / h;
          const int g = PB * k + i, j = PB * k + c;
          v[u] = (e < h * PB && g < r && j < r && g >= j) ? Min[g + (int64_t)r * j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kChol;
          if (e >= h * PB) break;
          const int i = e % h, c = e / h;
          const int g = PB * k + i, j = PB * k + c;
          float a = 0.f;
          if (g < r && j < r && g >= j) {
            a = v[u] * dinv[g] * dinv[j];
            if (g == j) a += shift;
          }
          Sk[i * LD + c] = a;
        }
      }
    }
    __syncthreads();
    if (rank == 0) {
      if (warp == 0) warp_chol32(store, min(PB, r), floor, &lbad, colbuf, Drc);
      __syncthreads();
      panel_solve(store, 0);
      __syncthreads();
      publish(store, 0);
      if (t == 0 && lbad) bad0[2 * attempt + 1] = 1;  // step -1
    }
    cluster.sync();
    bool failed = false;
    for (int p = 0; p < nb - 1; ++p) {
      if (bad0[2 * attempt + ((p - 1) & 1)]) { failed = true; break; }
      int kmin = rank;
      while (kmin <= p) kmin += CL;
      if (kmin < nb) {
        // panel p, rows g_lo .. rp-1: the owner uses its own copy, the
        // others read it from L (column-major, written before the barrier)
        const int owner = p % CL, g_lo = PB * kmin;
        const float* P;
        if (owner == rank) {
          P = store + (dsm_slot_offset<CL>(rank, p / CL, rp) + (g_lo - PB * p)) * LD;
        } else {
          const int nrows = rp - g_lo;
          const float* Lp = Lout + (int64_t)r * (PB * p) + g_lo;
          for (int i = t; i < nrows; i += kChol) {
            const bool in = g_lo + i < r;
            float v[PB];
#pragma unroll
            for (int c = 0; c < PB; ++c) v[c] = in ? __ldcg(Lp + i + (int64_t)r * c) : 0.f;
#pragma unroll
            for (int c = 0; c < PB; ++c) Pl_alloc[i * LD + c] = v[c];
          }
          P = Pl_alloc;
        }
        __syncthreads();
        int slot = (kmin - rank) / CL;
        int off = dsm_slot_offset<CL>(rank, slot, rp);
        if (kmin == p + 1) {
          // look-ahead on the next column: its diagonal block is updated
          // first and factored by warp 0 while warps 1..7 update the rows
          // below; then every thread solves the panel
          float* Sk = store + off * LD;
          const int h = rp - PB * kmin;
          {
            // diagonal block: thread t owns row t % 32, columns 4 (t / 32) + y
            const float* prow = P + (PB * kmin - g_lo) * LD;
            const int i = t & 31, c0 = (t >> 5) * 4;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
            for (int q = 0; q < PB; ++q) {
              const float u = prow[i * LD + q];
#pragma unroll
              for (int y = 0; y < 4; ++y) acc[y] = fmaf(u, prow[(c0 + y) * LD + q], acc[y]);
            }
#pragma unroll
            for (int y = 0; y < 4; ++y) Sk[i * LD + c0 + y] -= acc[y];
          }
          __syncthreads();
          if (warp == 0)
            warp_chol32(Sk, min(PB, r - PB * kmin), floor, &lbad, colbuf, Drc);
          else
            update_col(Sk, kmin, P, g_lo, PB, h, 1, kChol / 32 - 1);
          __syncthreads();
          panel_solve(Sk, kmin);
          __syncthreads();
          publish(Sk, kmin);
          if (t == 0 && lbad) bad0[2 * attempt + (p & 1)] = 1;
          off += h;
          kmin += CL;
        }
        for (int k = kmin; k < nb; off += rp - PB * k, k += CL)
          update_col(store + off * LD, k, P, g_lo, 0, rp - PB * k, 0, kChol / 32);
      }
      cluster.sync();
    }
    if (!failed && nb >= 2 && bad0[2 * attempt + ((nb - 2) & 1)]) failed = true;
    if (!failed) break;
    if (rank == 0 && t == 0 && flags) {
      atomicOr(flags, 1);
      atomicAdd(flags + 2, 1);
    }
    ++restarts;
    rel = (rel == 0.f) ? 1e-6f : rel * 10.f;
    if (rel > 1e-2f) rel = 1e-2f;
    cluster.sync();
  }
  if (clean && rank == 0 && t == 0) *clean = restarts == 0;
  // L is already in place (each column written when factored); the inverses
  // of the owned diagonal blocks, one warp each
  for (int k = rank, off = 0, q = 0; k < nb; off += rp - PB * k, k += CL, ++q)
    if (warp == q) warp_tri_inv32(store + off * LD, Linv_blk + (size_t)k * PB * PB);
}

// Inverses of the diagonal 32 x 32 blocks of L (global, column-major), one
// warp per block: for the factorizations that do not produce them.
__global__ void diag_inv_kernel(const float* __restrict__ L, int r, float* __restrict__ Linv_blk,
                                const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ float Ls[4][PB * (PB + 1)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * 4 + warp;
  const int nb = (r + PB - 1) / PB;
  if (k >= nb) return;
  const int b = min(PB, r - PB * k);
  for (int c = 0; c < PB; ++c)
    Ls[warp][lane * (PB + 1) + c] =
        (lane < b && c < b) ? (c <= lane ? L[(PB * k + lane) + (int64_t)r * (PB * k + c)] : 0.f) : (c == lane ? 1.f : 0.f);
  __syncwarp();
  warp_tri_inv32(Ls[warp], Linv_blk + (size_t)k * PB * PB);
}

// --------------------------------------------------------------------------
// trsm: V = W D^-1 L^-T for an s x r column-major W (rows independent), i.e.
// W * Rinv with Rinv = D^-1 L^-T, without forming Rinv.  ROWS rows per CTA
// live in shared memory; column blocks of 32 in order:
//   1. subtract the solved blocks times L: a ROWS x 32 x c0 product, 4-column
//      register tiles, the block row of L staged in shared memory;
//   2. multiply by the inverse of the 32 x 32 diagonal block (computed with
//      the factorization): a ROWS x 32 x 32 product, no serial chain.
// With `round`, V is stored rounded to TF32 (an operand of kind::tf32).
// --------------------------------------------------------------------------
constexpr int kTrsm = 256;

template <int ROWS, bool BLOCKROW>
__global__ void __launch_bounds__(kTrsm)
trsm_kernel(const float* __restrict__ W, int64_t s, int r, const float* __restrict__ L,
            const float* __restrict__ dinv, const float* __restrict__ Linv_blk, float* __restrict__ V, int round,
            const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ float sm[];
  const int ld = r + 1;
  float* Vs = sm;                    // ROWS x ld
  float* Lt = Vs + ROWS * ld;        // 32 x 33
  float* Lrow = Lt + PB * (PB + 1);  // 32 x ld (BLOCKROW): L[c0 + c][0:c0]
  const int t = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * ROWS;
  for (int e = t; e < ROWS * r; e += kTrsm) {
    int i = e % ROWS, c = e / ROWS;
    int64_t row = row0 + i;
    Vs[i * ld + c] = (row < s) ? W[row + s * c] * dinv[c] : 0.f;
  }
  __syncthreads();
  constexpr int TR = ROWS / 32;       // rows per thread in the update (4 x ... tiles)
  const int ty = t >> 3, tx = t & 7;  // 32 row groups x 8 column groups of 4
  const int nb = (r + PB - 1) / PB;
  for (int cb = 0; cb < nb; ++cb) {
    const int c0 = cb * PB;
    if (BLOCKROW && c0 > 0) {
      // the whole block row of L at once: every load is in flight together
      for (int e = t; e < PB * c0; e += kTrsm) {
        const int c = e & 31, k = e >> 5;
        Lrow[c * ld + k] = (c0 + c < r) ? L[(c0 + c) + (int64_t)r * k] : 0.f;
      }
      __syncthreads();
      float acc[TR][4];
#pragma unroll
      for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[a][j] = 0.f;
#pragma unroll 4
      for (int k = 0; k < c0; ++k) {
        float a[TR], bq[4];
#pragma unroll
        for (int x = 0; x < TR; ++x) a[x] = Vs[(ty + 32 * x) * ld + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) bq[j] = Lrow[(tx * 4 + j) * ld + k];
#pragma unroll
        for (int x = 0; x < TR; ++x)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[x][j] = fmaf(a[x], bq[j], acc[x][j]);
      }
      __syncthreads();
#pragma unroll
      for (int x = 0; x < TR; ++x)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int c = tx * 4 + j;
          if (c0 + c < r) Vs[(ty + 32 * x) * ld + c0 + c] -= acc[x][j];
        }
    }
    if (!BLOCKROW && c0 > 0) {
      float acc[TR][4];
#pragma unroll
      for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[a][j] = 0.f;
      // prefetch the first L tile: Lt[c][kk] = L[(c0 + c) + r (k0 + kk)]
      float pre[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int e = t + q * kTrsm, c = e & 31, kk = e >> 5;
        pre[q] = (c0 + c < r) ? L[(c0 + c) + (int64_t)r * kk] : 0.f;
      }
      for (int k0 = 0; k0 < c0; k0 += PB) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int e = t + q * kTrsm, c = e & 31, kk = e >> 5;
          Lt[c * (PB + 1) + kk] = pre[q];
        }
        __syncthreads();
        if (k0 + PB < c0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int e = t + q * kTrsm, c = e & 31, kk = e >> 5;
            pre[q] = (c0 + c < r) ? L[(c0 + c) + (int64_t)r * (k0 + PB + kk)] : 0.f;
          }
        }
#pragma unroll 4
        for (int kk = 0; kk < PB; ++kk) {
          float a[TR], bq[4];
#pragma unroll
          for (int x = 0; x < TR; ++x) a[x] = Vs[(ty + 32 * x) * ld + k0 + kk];
#pragma unroll
          for (int j = 0; j < 4; ++j) bq[j] = Lt[(tx * 4 + j) * (PB + 1) + kk];
#pragma unroll
          for (int x = 0; x < TR; ++x)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[x][j] = fmaf(a[x], bq[j], acc[x][j]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int x = 0; x < TR; ++x)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int c = tx * 4 + j;
          if (c0 + c < r) Vs[(ty + 32 * x) * ld + c0 + c] -= acc[x][j];
        }
    }
    // x_blk := x_blk Linv^T with Linv = (L_cb,cb)^-1 staged as Lt[c][k]
    for (int e = t; e < PB * PB; e += kTrsm) {
      const int c = e >> 5, k = e & 31;
      Lt[c * (PB + 1) + k] = Linv_blk[(size_t)cb * PB * PB + c * PB + k];
    }
    __syncthreads();
    {
      float acc[TR][4];
#pragma unroll
      for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[a][j] = 0.f;
      const int kmax = min(PB, r - c0);
      for (int k = 0; k < kmax; ++k) {
        float a[TR], bq[4];
#pragma unroll
        for (int x = 0; x < TR; ++x) a[x] = Vs[(ty + 32 * x) * ld + c0 + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) bq[j] = Lt[(tx * 4 + j) * (PB + 1) + k];
#pragma unroll
        for (int x = 0; x < TR; ++x)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[x][j] = fmaf(a[x], bq[j], acc[x][j]);
      }
      __syncthreads();
#pragma unroll
      for (int x = 0; x < TR; ++x)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = tx * 4 + j;
          if (c0 + c < r) Vs[(ty + 32 * x) * ld + c0 + c] = acc[x][j];
        }
    }
    __syncthreads();
  }
  for (int e = t; e < ROWS * r; e += kTrsm) {
    int ii = e % ROWS, c = e / ROWS;
    int64_t row = row0 + ii;
    if (row < s) {
      float v = Vs[ii * ld + c];
      V[row + s * c] = round ? mes::round_tf32(v) : v;
    }
  }
}

// --------------------------------------------------------------------------
// eig_small: FP64 parallel Jacobi (round-robin pairing), n <= 32, one warp:
// every step rotates n/2 disjoint pairs at once, one lane per pair.  Output
// the r leading eigenvectors (descending eigenvalue, ties by index), each
// sign-fixed so its largest-magnitude entry (lowest index on ties) is
// positive, as FP32 column-major n x r; eigenvalues optionally.
// --------------------------------------------------------------------------
__global__ void eig_small_kernel(const double* __restrict__ Gin, int n, int r, float* __restrict__ U,
                                 double* __restrict__ evals, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double A[32][33];
  __shared__ double V[32][33];
  __shared__ double cs[16][2];
  __shared__ int pr[16][2];
  __shared__ int perm[32];
  __shared__ int order[32];
  const int lane = threadIdx.x;
  const int m = n + (n & 1);            // padded to even
  const int half = m / 2;
  for (int i = 0; i < m; ++i) {
    if (lane < m) {
      A[i][lane] = (i < n && lane < n) ? Gin[i + n * lane] : 0.0;
      V[i][lane] = (i == lane) ? 1.0 : 0.0;
    }
  }
  if (lane < m) perm[lane] = lane;
  __syncwarp();
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(A[i][i]));
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0;
    if (lane < m)
      for (int j = 0; j < m; ++j)
        if (j != lane) off += A[lane][j] * A[lane][j];
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    if (off <= 1e-26 * scale * scale || scale == 0.0) break;
    for (int step = 0; step < m - 1; ++step) {
      if (lane < half) {
        int p = perm[lane], q = perm[m - 1 - lane];
        if (p > q) { int tmp = p; p = q; q = tmp; }
        const double apq = A[p][q];
        double c = 1.0, sn = 0.0;
        if (fabs(apq) > 1e-300) {
          const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
          const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(tt * tt + 1.0);
          sn = tt * c;
        }
        cs[lane][0] = c;
        cs[lane][1] = sn;
        pr[lane][0] = p;
        pr[lane][1] = q;
      }
      __syncwarp();
      if (lane < m) {   // rows p, q: lane walks column `lane`
        for (int k = 0; k < half; ++k) {
          const int p = pr[k][0], q = pr[k][1];
          const double c = cs[k][0], sn = cs[k][1];
          const double ap = A[p][lane], aq = A[q][lane];
          A[p][lane] = c * ap - sn * aq;
          A[q][lane] = sn * ap + c * aq;
        }
      }
      __syncwarp();
      if (lane < m) {   // columns p, q of A and V: lane walks row `lane`
        for (int k = 0; k < half; ++k) {
          const int p = pr[k][0], q = pr[k][1];
          const double c = cs[k][0], sn = cs[k][1];
          const double ap = A[lane][p], aq = A[lane][q];
          A[lane][p] = c * ap - sn * aq;
          A[lane][q] = sn * ap + c * aq;
          const double vp = V[lane][p], vq = V[lane][q];
          V[lane][p] = c * vp - sn * vq;
          V[lane][q] = sn * vp + c * vq;
        }
      }
      __syncwarp();
      if (lane == 0) {   // round-robin: perm[0] fixed, the rest rotate
        const int last = perm[m - 1];
        for (int i = m - 1; i > 1; --i) perm[i] = perm[i - 1];
        perm[1] = last;
      }
      __syncwarp();
    }
  }
  // order by descending eigenvalue (stable in index), real entries only
  if (lane < n) {
    const double w = mes::order_key(A[lane][lane]);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double wj = mes::order_key(A[j][j]);
      if (wj > w || (wj == w && j < lane)) ++rank;
    }
    order[rank] = lane;
  }
  __syncwarp();
  if (lane < r) {
    const int src = order[lane];
    int best = 0;
    double bv = -1.0;
    for (int i = 0; i < n; ++i) {
      const double a = fabs(V[i][src]);
      if (a > bv) { bv = a; best = i; }
    }
    const double sg = (V[best][src] < 0.0) ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) U[i + n * lane] = (float)(sg * V[i][src]);
    if (evals) evals[lane] = A[src][src];
  }
}

// --------------------------------------------------------------------------
// eig_mid: FP32 parallel Jacobi (round-robin pairing), r <= 128, one CTA.
// Z receives the eigenvectors as columns (r x r column-major), ordered by
// descending eigenvalue.
// --------------------------------------------------------------------------
constexpr int kMid = 512;

__global__ void __launch_bounds__(kMid)
eig_mid_kernel(const float* __restrict__ Hin, int r, float* __restrict__ Z, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ float sm[];
  const int n = r + (r & 1);               // padded to even
  const int ld = n + 1;
  float* A = sm;                           // n x ld
  float* V = A + n * ld;                   // n x ld
  float* cs = V + n * ld;                  // 2 * n/2
  int* perm = reinterpret_cast<int*>(cs + n);  // n
  __shared__ float offs;
  const int t = threadIdx.x;
  for (int e = t; e < n * n; e += kMid) {
    int i = e % n, j = e / n;
    float v = (i < r && j < r) ? Hin[i + r * j] : 0.f;
    A[i * ld + j] = v;
    V[i * ld + j] = (i == j) ? 1.f : 0.f;
  }
  for (int i = t; i < n; i += kMid) perm[i] = i;
  __syncthreads();
  const int half = n / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (t == 0) {
      float off = 0.f, dia = 0.f;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          float a = A[i * ld + j];
          if (i == j) dia += a * a; else off += a * a;
        }
      offs = (off <= 1e-14f * dia) ? 1.f : 0.f;
    }
    __syncthreads();
    if (offs != 0.f) break;
    for (int step = 0; step < n - 1; ++step) {
      // pairs (perm[k], perm[n-1-k])
      for (int k = t; k < half; k += kMid) {
        int p = perm[k], q = perm[n - 1 - k];
        if (p > q) { int tmp = p; p = q; q = tmp; }
        float apq = A[p * ld + q];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) > 1e-30f) {
          float theta = (A[q * ld + q] - A[p * ld + p]) / (2.f * apq);
          float tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
          c = rsqrtf(tt * tt + 1.f);
          s = tt * c;
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // rows
      for (int e = t; e < half * n; e += kMid) {
        int k = e / n, col = e % n;
        int p = perm[k], q = perm[n - 1 - k];
        if (p > q) { int tmp = p; p = q; q = tmp; }
        float c = cs[2 * k], s = cs[2 * k + 1];
        float ap = A[p * ld + col], aq = A[q * ld + col];
        A[p * ld + col] = c * ap - s * aq;
        A[q * ld + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns (A and V)
      for (int e = t; e < half * n; e += kMid) {
        int k = e / n, row = e % n;
        int p = perm[k], q = perm[n - 1 - k];
        if (p > q) { int tmp = p; p = q; q = tmp; }
        float c = cs[2 * k], s = cs[2 * k + 1];
        float ap = A[row * ld + p], aq = A[row * ld + q];
        A[row * ld + p] = c * ap - s * aq;
        A[row * ld + q] = s * ap + c * aq;
        float vp = V[row * ld + p], vq = V[row * ld + q];
        V[row * ld + p] = c * vp - s * vq;
        V[row * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
      // rotate the round-robin schedule (perm[0] fixed)
      if (t == 0) {
        int last = perm[n - 1];
        for (int i = n - 1; i > 1; --i) perm[i] = perm[i - 1];
        perm[1] = last;
      }
      __syncthreads();
    }
  }
  // sort by descending diagonal (only the r real entries)
  for (int i = t; i < r; i += kMid) {
    const float w = mes::order_key(A[i * ld + i]);
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      const float wj = mes::order_key(A[j * ld + j]);
      if (wj > w || (wj == w && j < i)) ++rank;
    }
    for (int row = 0; row < r; ++row) Z[row + r * rank] = V[row * ld + i];
  }
}

// --------------------------------------------------------------------------
// rr_update: one refinement step of approximate eigenvectors X of a symmetric
// r x r matrix A (Rayleigh-Ritz of a large factor, r > 128).  Given
// G = X^T X and S = X^T A X it writes E with X(I + E) the refined vectors.
// E follows from the first-order conditions that X(I + E) be orthonormal,
// E + E^T = I - G, and diagonalise A, S + E^T S + S E = diag (the iterative
// refinement of Ogita and Aishima, 2018): d_i = S_ii / G_ii,
//   e_ii = (1 - G_ii) / 2,
//   e_ij = (S_ij - d_j G_ij) / (d_j - d_i)   (i != j),
// Pairs whose values are closer than kRRCluster of the largest |d| form
// clusters and keep only the orthonormality part, e_ij = -G_ij / 2 (no
// rotation between them): an FP32 A resolves its eigenvalues only to about
// 2^-24 |A|, and the first-order step needs gaps well above that (in a
// float32 emulation with the 1024x768 scene's spectrum, a floor of 1e-6 made
// the iteration diverge, 1e-5 lost orthonormality to 3e-2 on the way, 1e-4
// converged in two or three steps).  A pair whose first-order rotation would
// not be small (|e_ij| >= 1/2) is treated the same way.
// --------------------------------------------------------------------------
constexpr float kRRCluster = 1e-4f;

__global__ void rr_update_kernel(const float* __restrict__ S, const float* __restrict__ G, int r,
                                 float* __restrict__ E) {
  __shared__ float dmax_s[32];
  float m = 0.f;
  for (int i = threadIdx.x; i < r; i += blockDim.x)
    m = fmaxf(m, fabsf(S[i + (int64_t)r * i] / G[i + (int64_t)r * i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) dmax_s[threadIdx.x >> 5] = m;
  __syncthreads();
  float dmax = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) dmax = fmaxf(dmax, dmax_s[w]);
  const float floor = kRRCluster * dmax;
  const int64_t n = (int64_t)r * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % r), j = (int)(e / r);   // column-major: E[i + r j]
    const float gij = G[e];
    if (i == j) {
      E[e] = 0.5f * (1.f - gij);
      continue;
    }
    const float di = S[i + (int64_t)r * i] / G[i + (int64_t)r * i];
    const float dj = S[j + (int64_t)r * j] / G[j + (int64_t)r * j];
    const float num = S[e] - dj * gij, den = dj - di;
    E[e] = (fabsf(den) > floor && fabsf(num) < 0.5f * fabsf(den)) ? num / den : -0.5f * gij;
  }
}

}  // namespace

namespace mes {

static mes_status diag_inv(const float* L, int r, float* Linv_blk, const int* skip, cudaStream_t st) {
  const int nb = (r + PB - 1) / PB;
  diag_inv_kernel<<<(nb + 3) / 4, 128, 0, st>>>(L, r, Linv_blk, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

size_t chol_smem() { return (1024 + PB * (PB + 1) + 1024 * (PB + 1)) * sizeof(float); }

mes_status chol(const float* M, int r, float shift_rel, float* L, float* dinv, float* Linv_blk, int* flags,
                const int* skip, cudaStream_t st, int* clean) {
  if (r > 1024) return fail(MES_ERR_NOT_IMPLEMENTED, "chol: rank above 1024");
  static bool attr = false;
  if (!attr) {
    MES_CUDA_TRY(cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)chol_smem()));
    attr = true;
  }
  const size_t last = (size_t)r * r * 4 - 1;
  MES_TRY(audit(M, last, "chol M"));
  MES_TRY(audit(L, last, "chol L"));
  MES_TRY(audit(dinv, (size_t)r * 4 - 1, "chol dinv"));
  MES_TRY(audit(Linv_blk, (size_t)((r + PB - 1) / PB) * PB * PB * 4 - 1, "chol Linv blocks"));
  if (clean) MES_TRY(audit(clean, sizeof(int) - 1, "chol clean"));
  ProfScope prof("chol_f32", st, r * (double)r * r / 3.0, 8.0 * r * (double)r);
  static int cluster_ok = -1;
  if (cluster_ok < 0) {
    cudaError_t e = cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chol_smem());
    cluster_ok = (e == cudaSuccess) ? 1 : 0;
    if (e != cudaSuccess && getenv("MES_DEBUG"))
      fprintf(stderr, "[mes] cluster Cholesky disabled: %s\n", cudaGetErrorString(e));
    cudaGetLastError();
  }
  static int dsm_ok = -1;
  if (dsm_ok < 0) {
    cudaError_t e = cudaFuncSetAttribute(chol_dsm_kernel<kCL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chol_dsm_smem(kDsmMaxR, kCL));
    dsm_ok = (e == cudaSuccess) ? 1 : 0;
    if (e != cudaSuccess && getenv("MES_DEBUG"))
      fprintf(stderr, "[mes] shared-memory cluster Cholesky disabled: %s\n", cudaGetErrorString(e));
    cudaGetLastError();
  }
  if (r > 128 && r <= kDsmMaxR && dsm_ok == 1) {
    // eight CTAs.  Four (half the SMs, the owned columns still fit up to
    // r = 480) were measured: 119 against 101 us per factorization in the
    // serialised launch list at 1920x1080, 75.3 against 74.2 stacks/s with
    // 16 stacks sharing the GPU -- a gain within the run-to-run spread, for a
    // longer chain per decomposition, so eight stay.  One CTA with the packed
    // lower triangle resident in its shared memory (r <= 256, no cluster
    // barrier) was measured too: 107 against 74 us at r = 256, the same
    // 75.1 stacks/s -- one SM issues too few instructions per cycle for the
    // trailing updates
    chol_dsm_kernel<kCL><<<kCL, kChol, chol_dsm_smem(r, kCL), st>>>(M, r, shift_rel, L, dinv, Linv_blk, flags,
                                                                     skip, clean);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return MES_OK;
    if (getenv("MES_DEBUG"))
      fprintf(stderr, "[mes] shared-memory cluster Cholesky launch rejected: %s\n", cudaGetErrorString(e));
    dsm_ok = 0;
  }
  if (r > 128 && cluster_ok == 1) {
    chol_cluster_kernel<<<kCL, kChol, chol_smem(), st>>>(M, r, shift_rel, L, dinv, flags, skip, clean);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return diag_inv(L, r, Linv_blk, skip, st);
    // a cluster launch the device cannot place is rejected before anything
    // runs; fall back to the one-CTA kernel from then on
    if (getenv("MES_DEBUG")) fprintf(stderr, "[mes] cluster Cholesky launch rejected: %s\n", cudaGetErrorString(e));
    cluster_ok = 0;
  }
  chol_kernel<<<1, kChol, chol_smem(), st>>>(M, r, shift_rel, L, dinv, flags, skip, clean);
  MES_LAUNCH_CHECK();
  return diag_inv(L, r, Linv_blk, skip, st);
}

// --------------------------------------------------------------------------
// trsm_wide: the same solve with NT / 2 rows per CTA (NT threads) held
// column-major in shared memory (column c of the row block contiguous), so a
// thread's 4 rows x 4 columns register tile reads its operands as two
// 16-byte loads per k (the kernel above reads five 4-byte loads per 4 FMAs).
// With NT = 128 (64 rows, 113 KB at r = 384) two CTAs share an SM, so one
// CTA's barrier and shared-memory waits overlap the other's FMAs.  Splitting
// each tile's k range over two groups of 128 threads (twice the warps, 126
// registers) was measured: 51.3 -> 50.0 us per solve alone, but 75.1 -> 73.9
// stacks/s with 16 stacks sharing the GPU, so one group stays.
// Per 32-column block: subtract the solved columns times the block row of L
// (staged 32 x 32 at a time, next tile prefetched into registers), then
// multiply by the inverted diagonal block.
// --------------------------------------------------------------------------
constexpr int kWThreads = 128;
constexpr int kWRows = kWThreads / 2;   // 4 rows per thread, 8 threads per row group
constexpr int kWLd = kWRows + 4;        // column stride of the row block (16-byte aligned)
constexpr int kTLd = PB + 4;            // row stride of a staged 32 x 32 tile
constexpr int kWMaxR = 384;             // 113 KB of shared memory at r = 384: two CTAs per SM
constexpr int kWPer = PB * PB / kWThreads;   // tile elements staged per thread
constexpr int kWF4 = kWRows / 4;             // float4s per column of the row block

size_t trsm_wide_smem(int r) { return (size_t)(r * kWLd + 2 * PB * kTLd) * sizeof(float); }

__global__ void __launch_bounds__(kWThreads, 2)
trsm_wide_kernel(const float* __restrict__ W, int64_t s, int r, const float* __restrict__ L,
                 const float* __restrict__ dinv, const float* __restrict__ Linv_blk, float* __restrict__ V, int round,
                 const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) float sm[];
  float* Vt = sm;                    // r columns x kWLd
  float* Lk = Vt + r * kWLd;         // 2 x 32 x kTLd: staged tiles, [k][c]
  const int t = threadIdx.x;
  const int rg = t >> 3, cg = t & 7;   // rows 4 rg .. 4 rg + 3, columns 4 cg .. 4 cg + 3 of the block
  const int64_t row0 = (int64_t)blockIdx.x * kWRows;
  if ((s & 3) == 0 && row0 + kWRows <= s && (reinterpret_cast<uintptr_t>(W) & 15) == 0) {
    // whole row block, 16-byte aligned: float4 loads of 4 consecutive rows,
    // eight in flight per thread (consecutive lanes read one column run)
    const int n4 = r * kWF4;
    for (int e0 = t; e0 < n4; e0 += 8 * kWThreads) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * kWThreads;
        if (e < n4) v[u] = __ldg(reinterpret_cast<const float4*>(W + row0 + s * (e / kWF4)) + (e % kWF4));
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * kWThreads;
        if (e < n4) {
          const int c = e / kWF4;
          const float d = dinv[c];
          *reinterpret_cast<float4*>(Vt + c * kWLd + 4 * (e % kWF4)) =
              make_float4(v[u].x * d, v[u].y * d, v[u].z * d, v[u].w * d);
        }
      }
    }
  } else {
    for (int e = t; e < kWRows * r; e += kWThreads) {
      const int ii = e % kWRows, c = e / kWRows;
      const int64_t row = row0 + ii;
      Vt[c * kWLd + ii] = (row < s) ? W[row + s * c] * dinv[c] : 0.f;
    }
  }
  __syncthreads();
  // The rows of the block are private to a warp (thread t owns rows
  // 4 (t >> 3) .. +3, so each warp owns 16 rows): only the staged 32 x 32
  // tiles are shared, and those go through a double buffer with one barrier
  // per tile.  Block cb consumes the tiles L[c0 .. c0+31][32 j .. 32 j + 31]
  // for j < cb, then (L_bb)^-1, all in one stream of tiles.
  const int nb = (r + PB - 1) / PB;
  // tile q of the stream: (block, j); j == block means the inverted diagonal block
  auto tile_load = [&](int cbq, int j, float (&pre)[kWPer]) {
#pragma unroll
    for (int q = 0; q < kWPer; ++q) {
      const int e = t + q * kWThreads;
      if (j < cbq) {   // Lk[k][c] = L[c0 + c][32 j + k]
        const int c = e & 31, k = e >> 5;
        pre[q] = (PB * cbq + c < r) ? L[(PB * cbq + c) + (int64_t)r * (PB * j + k)] : 0.f;
      } else {         // Li[k][c] = (L_bb^-1)[c][k]
        const int c = e >> 5, k = e & 31;
        pre[q] = Linv_blk[(size_t)cbq * PB * PB + c * PB + k];
      }
    }
  };
  auto tile_store = [&](float* buf, int cbq, int j, const float (&pre)[kWPer]) {
#pragma unroll
    for (int q = 0; q < kWPer; ++q) {
      const int e = t + q * kWThreads;
      if (j < cbq) buf[(e >> 5) * kTLd + (e & 31)] = pre[q];
      else buf[(e & 31) * kTLd + (e >> 5)] = pre[q];
    }
  };
  float pre[kWPer];
  int cbn = 0, jn = 0;   // next tile to load
  tile_load(cbn, jn, pre);
  int bsel = 0;
  for (int cb = 0; cb < nb; ++cb) {
    const int c0 = cb * PB;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int j = 0; j <= cb; ++j) {
      float* buf = Lk + bsel * (PB * kTLd);
      tile_store(buf, cb, j, pre);
      __syncthreads();   // tile visible; every thread is done with the other buffer
      // prefetch the next tile of the stream into registers
      if (++jn > cbn) { ++cbn; jn = 0; }
      if (cbn < nb) tile_load(cbn, jn, pre);
      if (j < cb) {
        const int k0 = PB * j;
#pragma unroll 8
        for (int k = 0; k < PB; ++k) {
          const float4 av = *reinterpret_cast<const float4*>(Vt + (k0 + k) * kWLd + 4 * rg);
          const float4 bv = *reinterpret_cast<const float4*>(buf + k * kTLd + 4 * cg);
          const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(a4[i], b4[jj], acc[i][jj]);
        }
      } else {
        // diagonal block: x := (x - acc) Linv^T; the rows are this warp's own
        const int kmax = min(PB, r - c0);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int c = c0 + 4 * cg + jj;
          if (c < r)
#pragma unroll
            for (int i = 0; i < 4; ++i) Vt[c * kWLd + 4 * rg + i] -= acc[i][jj];
        }
        __syncwarp();
        float x[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) x[i][jj] = 0.f;
        for (int k = 0; k < kmax; ++k) {
          const float4 av = *reinterpret_cast<const float4*>(Vt + (c0 + k) * kWLd + 4 * rg);
          const float4 bv = *reinterpret_cast<const float4*>(buf + k * kTLd + 4 * cg);
          const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) x[i][jj] = fmaf(a4[i], b4[jj], x[i][jj]);
        }
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int c = c0 + 4 * cg + jj;
          if (c < r)
#pragma unroll
            for (int i = 0; i < 4; ++i) Vt[c * kWLd + 4 * rg + i] = x[i][jj];
        }
        __syncwarp();
      }
      bsel ^= 1;
    }
  }
  __syncthreads();
  if ((s & 3) == 0 && row0 + kWRows <= s && (reinterpret_cast<uintptr_t>(V) & 15) == 0) {
    for (int e = t; e < r * kWF4; e += kWThreads) {
      const int c = e / kWF4;
      float4 v = *reinterpret_cast<const float4*>(Vt + c * kWLd + 4 * (e % kWF4));
      if (round) v = make_float4(mes::round_tf32(v.x), mes::round_tf32(v.y), mes::round_tf32(v.z), mes::round_tf32(v.w));
      reinterpret_cast<float4*>(V + row0 + s * c)[e % kWF4] = v;
    }
  } else {
    for (int e = t; e < kWRows * r; e += kWThreads) {
      const int ii = e % kWRows, c = e / kWRows;
      const int64_t row = row0 + ii;
      if (row < s) {
        const float v = Vt[c * kWLd + ii];
        V[row + s * c] = round ? mes::round_tf32(v) : v;
      }
    }
  }
}

template <int ROWS, bool BLOCKROW>
mes_status trsm_launch(const float* W, int64_t s, int r, const float* L, const float* dinv, const float* Linv_blk,
                       float* V, bool round, const int* skip, cudaStream_t st) {
  const size_t smem = (size_t)((ROWS + (BLOCKROW ? PB : 0)) * (r + 1) + PB * (PB + 1)) * sizeof(float);
  static bool attr = false;
  if (!attr) {
    MES_CUDA_TRY(cudaFuncSetAttribute(trsm_kernel<ROWS, BLOCKROW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      220 * 1024));
    attr = true;
  }
  const unsigned grid = (unsigned)((s + ROWS - 1) / ROWS);
  trsm_kernel<ROWS, BLOCKROW><<<grid, kTrsm, smem, st>>>(W, s, r, L, dinv, Linv_blk, V, round ? 1 : 0, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status trsm(const float* W, int64_t s, int r, const float* L, const float* dinv, const float* Linv_blk, float* V,
                bool round, const int* skip, cudaStream_t st) {
  if (r > 1024) return fail(MES_ERR_NOT_IMPLEMENTED, "trsm: rank above 1024");
  if (W == V) return fail(MES_ERR_INVALID_ARG, "trsm: in-place solve not supported");
  MES_TRY(audit(W, (size_t)(s * r) * 4 - 1, "trsm W"));
  MES_TRY(audit(V, (size_t)(s * r) * 4 - 1, "trsm V"));
  MES_TRY(audit(L, (size_t)r * r * 4 - 1, "trsm L"));
  MES_TRY(audit(Linv_blk, (size_t)((r + PB - 1) / PB) * PB * PB * 4 - 1, "trsm Linv blocks"));
  ProfScope prof("trsm_f32", st, s * (double)r * r, 8.0 * s * r);
  // Rows per CTA and whether a whole block row of L fits in shared memory
  // (~210 KB budget): more rows amortise the L traffic, more CTAs fill the
  // GPU (aim for ~120).
  const size_t budget = 210 * 1024;
  if (r <= kWMaxR) {   // the row block fits in shared memory
    static bool wattr = false;
    if (!wattr) {
      MES_CUDA_TRY(cudaFuncSetAttribute(trsm_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)trsm_wide_smem(kWMaxR)));
      wattr = true;
    }
    const unsigned grid = (unsigned)((s + kWRows - 1) / kWRows);
    trsm_wide_kernel<<<grid, kWThreads, trsm_wide_smem(r), st>>>(W, s, r, L, dinv, Linv_blk, V, round ? 1 : 0, skip);
    MES_LAUNCH_CHECK();
    return MES_OK;
  }
  auto fits = [&](int rows, bool br) {
    return (size_t)((rows + (br ? PB : 0)) * (r + 1) + PB * (PB + 1)) * sizeof(float) <= budget;
  };
  if (fits(64, true) && (s + 63) / 64 >= 120) return trsm_launch<64, true>(W, s, r, L, dinv, Linv_blk, V, round, skip, st);
  if (fits(32, true)) return trsm_launch<32, true>(W, s, r, L, dinv, Linv_blk, V, round, skip, st);
  return trsm_launch<32, false>(W, s, r, L, dinv, Linv_blk, V, round, skip, st);
}

mes_status eig_small(const double* G, int n, int r, float* U, double* evals, const int* skip,
                     cudaStream_t st) {
  if (n > 32) return fail(MES_ERR_NOT_IMPLEMENTED, "eig_small: n above 32");
  MES_TRY(audit(G, (size_t)n * n * 8 - 1, "eig_small G"));
  MES_TRY(audit(U, (size_t)n * r * 4 - 1, "eig_small U"));
  ProfScope prof("eig_small_f64", st, 0.0, 8.0 * n * n);
  eig_small_kernel<<<1, 32, 0, st>>>(G, n, r, U, evals, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status rr_update(const float* S, const float* G, int r, float* E, cudaStream_t st) {
  const size_t last = (size_t)r * r * 4 - 1;
  MES_TRY(audit(S, last, "rr_update S"));
  MES_TRY(audit(G, last, "rr_update G"));
  MES_TRY(audit(E, last, "rr_update E"));
  ProfScope prof("rr_update", st, 0.0, 12.0 * r * (double)r);
  rr_update_kernel<<<grid_for((int64_t)r * r, 256, (int64_t)sm_count() * 4), 256, 0, st>>>(S, G, r, E);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

size_t eig_mid_smem(int r) {
  int n = r + (r & 1);
  return (size_t)(2 * n * (n + 1) + n) * sizeof(float) + n * sizeof(int);
}

mes_status eig_mid(const float* H, int r, float* Z, const int* skip, cudaStream_t st) {
  if (r > 128) return fail(MES_ERR_NOT_IMPLEMENTED, "eig_mid: r above 128");
  static bool attr = false;
  if (!attr) {
    MES_CUDA_TRY(cudaFuncSetAttribute(eig_mid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)eig_mid_smem(128)));
    attr = true;
  }
  MES_TRY(audit(H, (size_t)r * r * 4 - 1, "eig_mid H"));
  MES_TRY(audit(Z, (size_t)r * r * 4 - 1, "eig_mid Z"));
  ProfScope prof("eig_mid_f32", st, 0.0, 8.0 * r * r);
  eig_mid_kernel<<<1, kMid, eig_mid_smem(r), st>>>(H, r, Z, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

}  // namespace mes

// Test hook: the factorization and the solve of one CholeskyQR pass on
// caller data (declared in mes.h).
extern "C" mes_status mes_solve_selftest(const float* H, int r, const float* W, int64_t s, float* L, float* dinv,
                                         float* V, int* restarts, void* stream) {
  mes::clear_error();
  if (!H || !W || !L || !dinv || !V || r < 1 || r > 1024 || s < 1 || W == V)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_solve_selftest: bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mes::AuditScope audit_scope;
  mes::audit_register(H, (size_t)r * r * 4);
  mes::audit_register(L, (size_t)r * r * 4);
  mes::audit_register(dinv, (size_t)r * 4);
  mes::audit_register(W, (size_t)(s * r) * 4);
  mes::audit_register(V, (size_t)(s * r) * 4);
  mes::Scratch scr(st);
  float* linv = nullptr;
  int* flags = nullptr;
  MES_TRY(scr.alloc(&linv, (size_t)(r + PB - 1) / PB * PB * PB));
  MES_TRY(scr.alloc(&flags, 3));
  MES_CUDA_TRY(cudaMemsetAsync(flags, 0, 3 * sizeof(int), st));
  MES_TRY(mes::chol(H, r, 0.f, L, dinv, linv, flags, nullptr, st, nullptr));
  MES_TRY(mes::trsm(W, s, r, L, dinv, linv, V, false, nullptr, st));
  int hf[3] = {0, 0, 0};
  MES_CUDA_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
  MES_CUDA_TRY(cudaStreamSynchronize(st));
  if (restarts) *restarts = hf[2];
  if (hf[0] & 2) return mes::fail(MES_ERR_NONFINITE, "mes_solve_selftest: non-positive or non-finite diagonal");
  return MES_OK;
}

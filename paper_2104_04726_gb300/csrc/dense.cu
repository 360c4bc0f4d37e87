// Small dense solvers of the factor update (Section III-B, text after Eq. 8:
// the factor is taken from the leading eigenvectors of the Gram).
//
//  * cholinv:   equilibrated, optionally shifted Cholesky of an r x r Gram
//               M = W^T W and the inverse of its factor, giving Rinv with
//               W * Rinv orthonormal (one pass of shifted CholeskyQR).  One
//               CTA of 1024 threads, FP32, blocked by 32 columns: the
//               diagonal block is factored by one warp in shared memory, the
//               panel below by one row per thread, the trailing update by
//               8x8 register tiles; the inverse is blocked the same way.
//  * eig_small: FP64 cyclic Jacobi for the Grams of the small modes
//               (colour, view x exposure; n <= 32), one warp per matrix.
//  * eig_mid:   FP32 parallel (round-robin) Jacobi for an r x r symmetric
//               matrix with r <= 128 held in shared memory; used for the
//               Rayleigh-Ritz rotation of the factors at the end.
//
// GB300's FP64 rate is a small fraction of its FP32 rate, so O(r^3) work at
// r in the hundreds runs in FP32; FP64 is used where the work is O(n^3) with
// n <= 32 and for accumulations.
#include "common.cuh"

namespace {

constexpr int kChol = 1024;
constexpr int PB = 32;

// --------------------------------------------------------------------------
// cholinv
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kChol)
cholinv_kernel(const float* __restrict__ Min, int r, float shift_rel, float* __restrict__ A,
               float* __restrict__ X, float* __restrict__ Rinv, int* __restrict__ flags,
               const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ float smem[];
  float* dinv = smem;                       // r
  float* Dg = dinv + 1024;                  // 32 x 33
  float* Pn = Dg + PB * (PB + 1);           // up to 1024 x 33 (panel) / reuse
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  // equilibration d_i = sqrt(M_ii)
  for (int i = t; i < r; i += kChol) {
    float v = Min[i + (int64_t)r * i];
    float d = (v > 0.f && isfinite(v)) ? sqrtf(v) : 1.f;
    if (!(v > 0.f && isfinite(v)) && flags) atomicOr(flags, 2);
    dinv[i] = 1.f / d;
  }
  __syncthreads();
  // Shifted Cholesky with restarts: the shift must dominate the FP32
  // rounding of the Gram (else a pivot goes non-positive) yet stay small (the
  // next unshifted pass needs W * Rinv well conditioned).  Start at
  // shift_rel and, when a pivot falls below the floor, restart with a ten
  // times larger relative shift (at most 1e-2).
  __shared__ int bad;
  float rel = shift_rel;
  for (int attempt = 0; attempt < 8; ++attempt) {
    const float shift = rel * (float)r;
    const float floor = fmaxf(1e-7f, 0.1f * shift);
    if (t == 0) bad = 0;
    // A = D^-1 M D^-1 + shift I  (lower triangle, column-major)
    for (int64_t e = t; e < (int64_t)r * r; e += kChol) {
      int j = (int)(e / r), i = (int)(e - (int64_t)j * r);
      if (i >= j) {
        float v = Min[e] * dinv[i] * dinv[j];
        if (i == j) v += shift;
        A[e] = v;
      }
    }
    __syncthreads();

    // ---- blocked right-looking Cholesky, lower, in place in A ----
    for (int p0 = 0; p0 < r; p0 += PB) {
      const int b = min(PB, r - p0);
      for (int e = t; e < b * b; e += kChol) {
        int i = e % b, j = e / b;
        Dg[i * (PB + 1) + j] = (i >= j) ? A[(p0 + i) + (int64_t)r * (p0 + j)] : 0.f;
      }
      __syncthreads();
      if (warp == 0) {
        for (int j = 0; j < b; ++j) {
          float piv = Dg[j * (PB + 1) + j];
          if (!(piv > floor)) {
            if (lane == 0) bad = 1;
            piv = floor;
          }
          piv = sqrtf(piv);
          __syncwarp();
          if (lane == j) Dg[j * (PB + 1) + j] = piv;
          if (lane > j && lane < b) Dg[lane * (PB + 1) + j] /= piv;
          __syncwarp();
          if (lane > j && lane < b) {
            float lij = Dg[lane * (PB + 1) + j];
            for (int k = j + 1; k <= lane; ++k) Dg[lane * (PB + 1) + k] -= lij * Dg[k * (PB + 1) + j];
          }
          __syncwarp();
        }
      }
      __syncthreads();
      for (int e = t; e < b * b; e += kChol) {
        int i = e % b, j = e / b;
        if (i >= j) A[(p0 + i) + (int64_t)r * (p0 + j)] = Dg[i * (PB + 1) + j];
      }
      const int rows = r - p0 - b;
      // panel: L[i, p0:p0+b] = A[i, p0:p0+b] * Dg^-T
      for (int ii = t; ii < rows; ii += kChol) {
        const int i = p0 + b + ii;
        float a[PB];
#pragma unroll
        for (int c = 0; c < PB; ++c) a[c] = (c < b) ? A[i + (int64_t)r * (p0 + c)] : 0.f;
#pragma unroll
        for (int c = 0; c < PB; ++c) {
          if (c < b) {
            float sacc = a[c];
#pragma unroll
            for (int k = 0; k < PB; ++k)
              if (k < c) sacc -= a[k] * Dg[c * (PB + 1) + k];
            a[c] = sacc / Dg[c * (PB + 1) + c];
          }
        }
#pragma unroll
        for (int c = 0; c < PB; ++c) {
          if (c < b) A[i + (int64_t)r * (p0 + c)] = a[c];
          Pn[ii * (PB + 1) + c] = (c < b) ? a[c] : 0.f;
        }
      }
      __syncthreads();
      // trailing update of the lower triangle, 8x8 tiles
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
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) {
            int ri = bi * 8 + x, rj = bj * 8 + y;
            if (ri < rows && rj < rows && ri >= rj) {
              int64_t e = (p0 + b + ri) + (int64_t)r * (p0 + b + rj);
              A[e] -= acc[x][y];
            }
          }
      }
      __syncthreads();
    }
    if (!bad) break;
    if (t == 0 && flags) atomicOr(flags, 1);
    rel = (rel == 0.f) ? 1e-6f : rel * 10.f;
    if (rel > 1e-2f) rel = 1e-2f;
    __syncthreads();
  }

  // ---- X = L^-1 (lower), blocked by 32 rows ----
  const int nb = (r + PB - 1) / PB;
  float* Di = Dg;                  // inverse of the current diagonal block, 32 x 33
  float* Ls = Pn;                  // 32 x 33 tile of L (diagonal block first)
  float* Xs = Pn + PB * (PB + 1);  // 32 x 33 tile of X
  const int ti = t >> 5, tj = t & 31;   // 32 x 32 output element per thread
  for (int ib = 0; ib < nb; ++ib) {
    const int i0 = ib * PB, bi = min(PB, r - i0);
    // stage the diagonal block of L (coalesced: lanes walk the rows)
    Ls[tj * (PB + 1) + ti] = (tj < bi && ti < bi) ? A[(i0 + tj) + (int64_t)r * (i0 + ti)] : (tj == ti ? 1.f : 0.f);
    __syncthreads();
    // its inverse, column `lane` per lane of warp 0, in registers
    if (warp == 0) {
      float col[PB];
#pragma unroll
      for (int i = 0; i < PB; ++i) {
        float sacc = (i == lane) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < i; ++k) sacc -= Ls[i * (PB + 1) + k] * col[k];
        col[i] = (i >= lane) ? sacc / Ls[i * (PB + 1) + i] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < PB; ++i) Di[i * (PB + 1) + lane] = (lane < bi && i < bi) ? col[i] : 0.f;
    }
    __syncthreads();
    // off-diagonal blocks X[ib, jb] = -Di * sum_{kb=jb}^{ib-1} L[ib,kb] X[kb,jb]
    for (int jb = 0; jb < ib; ++jb) {
      const int j0 = jb * PB;
      float sacc = 0.f;
      for (int kb = jb; kb < ib; ++kb) {
        const int k0 = kb * PB;
        // coalesced loads: consecutive lanes read consecutive rows
        Ls[tj * (PB + 1) + ti] = (tj < bi) ? A[(i0 + tj) + (int64_t)r * (k0 + ti)] : 0.f;
        Xs[tj * (PB + 1) + ti] = X[(k0 + tj) + (int64_t)r * (j0 + ti)];
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < PB; ++k) sacc += Ls[ti * (PB + 1) + k] * Xs[k * (PB + 1) + tj];
        __syncthreads();
      }
      Ls[ti * (PB + 1) + tj] = sacc;
      __syncthreads();
      float v = 0.f;
#pragma unroll 8
      for (int k = 0; k < PB; ++k) v -= Di[ti * (PB + 1) + k] * Ls[k * (PB + 1) + tj];
      Xs[ti * (PB + 1) + tj] = v;
      __syncthreads();
      // coalesced store of the block
      if (tj < bi) X[(i0 + tj) + (int64_t)r * (j0 + ti)] = Xs[tj * (PB + 1) + ti];
      __syncthreads();
    }
    // diagonal block of X, zero above it
    if (tj < bi && ti < bi) X[(i0 + tj) + (int64_t)r * (i0 + ti)] = (tj >= ti) ? Di[tj * (PB + 1) + ti] : 0.f;
    __syncthreads();
  }
  // Rinv(p, q) = Linv(q, p) / d_p for p <= q, 0 below the diagonal
  for (int64_t e = t; e < (int64_t)r * r; e += kChol) {
    int q = (int)(e / r), p = (int)(e - (int64_t)q * r);
    Rinv[e] = (p <= q) ? X[q + (int64_t)r * p] * dinv[p] : 0.f;
  }
}

// --------------------------------------------------------------------------
// eig_small: FP64 cyclic Jacobi, n <= 32, one warp.  Output the r leading
// eigenvectors (descending eigenvalue, ties by index), each sign-fixed so its
// largest-magnitude entry (lowest index on ties) is positive, as FP32
// column-major n x r; eigenvalues optionally.
// --------------------------------------------------------------------------
__global__ void eig_small_kernel(const double* __restrict__ Gin, int n, int r, float* __restrict__ U,
                                 double* __restrict__ evals, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double A[32][33];
  __shared__ double V[32][33];
  __shared__ double cs[2];
  __shared__ int order[32];
  const int lane = threadIdx.x;
  for (int i = 0; i < n; ++i)
    if (lane < n) {
      A[i][lane] = Gin[i + n * lane];
      V[i][lane] = (i == lane) ? 1.0 : 0.0;
    }
  __syncwarp();
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(A[i][i]));
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p][q] * A[p][q];
    if (off <= 1e-30 * scale * scale || scale == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (lane == 0) {
          double apq = A[p][q];
          double c = 1.0, s = 0.0;
          if (fabs(apq) > 1e-300) {
            double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
            double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
          }
          cs[0] = c;
          cs[1] = s;
        }
        __syncwarp();
        const double c = cs[0], s = cs[1];
        if (s != 0.0) {
          if (lane < n) {  // columns p, q of A
            double akp = A[lane][p], akq = A[lane][q];
            A[lane][p] = c * akp - s * akq;
            A[lane][q] = s * akp + c * akq;
          }
          __syncwarp();
          if (lane < n) {  // rows p, q
            double apk = A[p][lane], aqk = A[q][lane];
            A[p][lane] = c * apk - s * aqk;
            A[q][lane] = s * apk + c * aqk;
            double vkp = V[lane][p], vkq = V[lane][q];
            V[lane][p] = c * vkp - s * vkq;
            V[lane][q] = s * vkp + c * vkq;
          }
        }
        __syncwarp();
      }
  }
  // order by descending eigenvalue (stable in index)
  if (lane < n) {
    double w = A[lane][lane];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double wj = A[j][j];
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
      double a = fabs(V[i][src]);
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
    float w = A[i * ld + i];
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      float wj = A[j * ld + j];
      if (wj > w || (wj == w && j < i)) ++rank;
    }
    for (int row = 0; row < r; ++row) Z[row + r * rank] = V[row * ld + i];
  }
}

}  // namespace

namespace mes {

size_t cholinv_smem() { return (1024 + PB * (PB + 1) + 1024 * (PB + 1)) * sizeof(float); }

mes_status cholinv(const float* M, int r, float shift_rel, float* work, float* X, float* Rinv,
                   int* flags, const int* skip, cudaStream_t st) {
  if (r > 1024) return fail(MES_ERR_NOT_IMPLEMENTED, "cholinv: rank above 1024");
  static bool attr = false;
  if (!attr) {
    MES_CUDA_TRY(cudaFuncSetAttribute(cholinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)cholinv_smem()));
    attr = true;
  }
  const size_t last = (size_t)r * r * 4 - 1;
  MES_TRY(audit(M, last, "cholinv M"));
  MES_TRY(audit(work, last, "cholinv work"));
  MES_TRY(audit(X, last, "cholinv X"));
  MES_TRY(audit(Rinv, last, "cholinv Rinv"));
  ProfScope prof("cholinv_f32", st, 4.0 / 3.0 * r * (double)r * r, 12.0 * r * (double)r);
  cholinv_kernel<<<1, kChol, cholinv_smem(), st>>>(M, r, shift_rel, work, X, Rinv, flags, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
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

// Bandwidth kernels around the Tucker-ALS sweep (Section III-B):
//  * slice transpose of the stack (a second layout with mode 2 fastest, so
//    that the mode-2 contraction reads its operand contiguously), with
//    ||T||_F^2 fused in FP64;
//  * a counter-based uniform generator for the random start block of the
//    T-HOSVD subspace iteration;
//  * "fibre mixing": for every fibre over the trailing small modes
//    (colour, view x exposure) apply the Kronecker product of small
//    matrices, i.e. mode products with the small factors (Eq. 8 for those
//    modes, the core of Eq. 5 / Eq. 7, and reconstruction, Eq. 1);
//  * Grams of the small modes: FP32 sums over chunks of 32 fibres,
//    accumulated in FP64 in a fixed order;
//  * the per-sweep fit and stopping flag; column sign / order fixing.
#include "small.cuh"

namespace {

constexpr int kT = 256;

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

// XB[y + s2*(x + s1*l)] = X[x + s1*(y + s2*l)], 32x32 tiles; norm partials.
__global__ void __launch_bounds__(kT)
slice_transpose_kernel(const float* __restrict__ X, int64_t s1, int64_t s2, int64_t L,
                       float* __restrict__ XB, double* __restrict__ partials, float* __restrict__ Xr,
                       int round, uint16_t* __restrict__ X16, uint16_t* __restrict__ XB16) {
  __shared__ float tile[32][33];
  __shared__ double red[kT / 32];
  const int64_t tx = (s1 + 31) / 32, ty = (s2 + 31) / 32;
  const int64_t ntile = tx * ty * L;
  double acc = 0.0;
  for (int64_t tIdx = blockIdx.x; tIdx < ntile; tIdx += gridDim.x) {
    const int64_t l = tIdx / (tx * ty);
    const int64_t rem = tIdx - l * tx * ty;
    const int64_t by = rem / tx, bx = rem - by * tx;
    const float* src = X + l * s1 * s2;
    const int c = threadIdx.x & 31;
    float part = 0.f;   // this tile's squares in FP32, one FP64 add per tile
    for (int rr = threadIdx.x >> 5; rr < 32; rr += kT / 32) {
      int64_t x = bx * 32 + c, y = by * 32 + rr;
      const bool in = x < s1 && y < s2;
      float v = in ? src[x + s1 * y] : 0.f;
      part = fmaf(v, v, part);
      if (X16 && in) X16[l * s1 * s2 + x + s1 * y] = mes::bf16_bits(v);
      if (Xr && in) Xr[l * s1 * s2 + x + s1 * y] = round ? mes::round_tf32(v) : v;
      tile[rr][c] = v;   // the input value: each output rounds it its own way
    }
    acc += (double)part;
    __syncthreads();
    for (int rr = threadIdx.x >> 5; rr < 32; rr += kT / 32) {
      int64_t y = by * 32 + c, x = bx * 32 + rr;
      if (x < s1 && y < s2) {
        const float v = tile[c][rr];
        if (XB) XB[l * s1 * s2 + y + s2 * x] = round ? mes::round_tf32(v) : v;
        if (XB16) XB16[l * s1 * s2 + y + s2 * x] = mes::bf16_bits(v);
      }
    }
    __syncthreads();
  }
  double t = block_sum_d(acc, red);
  if (threadIdx.x == 0 && partials) partials[blockIdx.x] = t;
}

__global__ void split_tf32_kernel(const float* __restrict__ in, float* __restrict__ hi, float* __restrict__ lo,
                                  int64_t n, const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = in[i];
    const float h = mes::round_tf32(x);
    hi[i] = h;
    lo[i] = mes::round_tf32(x - h);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ in, uint16_t* __restrict__ out, int64_t n,
                               const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mes::bf16_bits(in[i]);
}

__global__ void __launch_bounds__(kT)
sumsq_kernel(const float* __restrict__ x, int64_t n, double* __restrict__ partials,
             const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double red[kT / 32];
  // runs of 16 squares summed in FP32, one FP64 add per run
  double acc = 0.0;
  float part = 0.f;
  int run = 0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const float v = x[i];
    part = fmaf(v, v, part);
    if (++run == 16) {
      acc += (double)part;
      part = 0.f;
      run = 0;
    }
  }
  acc += (double)part;
  double t = block_sum_d(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void uniform_kernel(float* __restrict__ out, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = splitmix64(seed * 0x100000001B3ull + (uint64_t)i);
    out[i] = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  }
}

// Fibre mixing.  Fibre f = f_lo + F_lo*f_hi has L input values at
// in + f_lo*in_lo + f_hi*in_hi + l*in_l and L2 outputs likewise; the L2 x L
// Kronecker matrix K is staged in shared memory.
__global__ void __launch_bounds__(kT)
mix_kernel(mes::Fibres fb, const float* __restrict__ Kmat, int L, int L2, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ float Ks[];
  for (int e = threadIdx.x; e < L * L2; e += kT) Ks[e] = Kmat[e];
  __syncthreads();
  const int64_t F = fb.F_lo * fb.F_hi;
  for (int64_t f = (int64_t)blockIdx.x * kT + threadIdx.x; f < F; f += (int64_t)gridDim.x * kT) {
    const int64_t fh = f / fb.F_lo, fl = f - fh * fb.F_lo;
    const float* src = fb.in + fl * fb.in_lo + fh * fb.in_hi;
    float* dst = fb.out + fl * fb.out_lo + fh * fb.out_hi;
    float v[64];
    for (int l0 = 0; l0 < L; l0 += 64) {
      // process in chunks of 64 inputs (L may exceed 64)
      int nl = min(64, L - l0);
      for (int l = 0; l < nl; ++l) v[l] = src[(int64_t)(l0 + l) * fb.in_l];
      for (int o = 0; o < L2; ++o) {
        float s = 0.f;
        const float* kr = Ks + (int64_t)o * L + l0;
        for (int l = 0; l < nl; ++l) s = fmaf(kr[l], v[l], s);
        float* d = dst + (int64_t)o * fb.out_l;
        *d = (l0 == 0) ? s : *d + s;
      }
    }
  }
}

// The same mixing with the fibre held in registers: L <= LMAX (the
// workloads have L = 3 x 6 .. 3 x 14), loops unrolled and predicated, the
// products summed in the same order as above, so the results are identical.
template <int LMAX>
__global__ void __launch_bounds__(kT)
mix_reg_kernel(mes::Fibres fb, const float* __restrict__ Kmat, int L, int L2, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) float Ks[];
  // rows of K padded to a multiple of 4 (zeros) and read as float4
  const int LP = (L + 3) & ~3;
  for (int e = threadIdx.x; e < LP * L2; e += kT) {
    const int o = e / LP, l = e - o * LP;
    Ks[e] = l < L ? Kmat[o * L + l] : 0.f;
  }
  __syncthreads();
  const int64_t F = fb.F_lo * fb.F_hi;
  for (int64_t f = (int64_t)blockIdx.x * kT + threadIdx.x; f < F; f += (int64_t)gridDim.x * kT) {
    const int64_t fh = f / fb.F_lo, fl = f - fh * fb.F_lo;
    const float* src = fb.in + fl * fb.in_lo + fh * fb.in_hi;
    float* dst = fb.out + fl * fb.out_lo + fh * fb.out_hi;
    float v[LMAX];
#pragma unroll
    for (int l = 0; l < LMAX; ++l) v[l] = l < L ? src[(int64_t)l * fb.in_l] : 0.f;
    for (int o = 0; o < L2; ++o) {
      const float4* kr = reinterpret_cast<const float4*>(Ks + o * LP);
      float acc = 0.f;
#pragma unroll
      for (int l4 = 0; l4 < LMAX / 4; ++l4) {
        if (4 * l4 < L) {
          const float4 k = kr[l4];
          // the same order as the generic kernel: l ascending, l < L only
          acc = fmaf(k.x, v[4 * l4], acc);
          if (4 * l4 + 1 < L) acc = fmaf(k.y, v[4 * l4 + 1], acc);
          if (4 * l4 + 2 < L) acc = fmaf(k.z, v[4 * l4 + 2], acc);
          if (4 * l4 + 3 < L) acc = fmaf(k.w, v[4 * l4 + 3], acc);
        }
      }
      dst[(int64_t)o * fb.out_l] = acc;
    }
  }
}

// Gram of one small mode over all fibres.  The fibre is first projected by
// the L2 x L matrix K (the other small modes' factors, identity on mode n),
// giving an s_n x (L2/s_n) block with the mode-n index at stride `inner`
// (product of the sizes of the modes before n) ... flattened as
// idx = i*inner + o_lo + inner*s_n*o_hi.  Each block stages 32 projected
// fibres in shared memory; thread e owns Gram entry e (< s_n^2) and
// accumulates in FP64 in a fixed order.
__global__ void __launch_bounds__(kT)
small_gram_kernel(mes::Fibres fb, const float* __restrict__ Kmat, int L, int L2, int sn, int inner,
                  double* __restrict__ partials, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ float sh[];
  float* Ks = sh;                    // L2 x L
  float* Ys = Ks + L * L2;           // 32 x L2
  for (int e = threadIdx.x; e < L * L2; e += kT) Ks[e] = Kmat[e];
  __syncthreads();
  const int64_t F = fb.F_lo * fb.F_hi;
  const int ent = sn * sn;
  const int rest = L2 / sn;
  double acc = 0.0;
  const int ei = threadIdx.x % sn, ej = threadIdx.x / sn;   // valid when threadIdx.x < ent
  for (int64_t f0 = (int64_t)blockIdx.x * 32; f0 < F; f0 += (int64_t)gridDim.x * 32) {
    // project 32 fibres: element (fi, o) by thread loop
    for (int e = threadIdx.x; e < 32 * L2; e += kT) {
      int fi = e / L2, o = e - fi * L2;
      int64_t f = f0 + fi;
      float s = 0.f;
      if (f < F) {
        const int64_t fh = f / fb.F_lo, fl = f - fh * fb.F_lo;
        const float* src = fb.in + fl * fb.in_lo + fh * fb.in_hi;
        const float* kr = Ks + (int64_t)o * L;
        for (int l = 0; l < L; ++l) s = fmaf(kr[l], src[(int64_t)l * fb.in_l], s);
      }
      Ys[fi * L2 + o] = s;
    }
    __syncthreads();
    if (threadIdx.x < ent) {
      // 32 fibres are summed in FP32, chunks are accumulated in FP64
      float chunk = 0.f;
      for (int fi = 0; fi < 32; ++fi) {
        const float* y = Ys + fi * L2;
        for (int o = 0; o < rest; ++o) {
          int olo = o % inner, ohi = o / inner;
          int base = olo + inner * sn * ohi;
          chunk = fmaf(y[base + inner * ei], y[base + inner * ej], chunk);
        }
      }
      acc += (double)chunk;
    }
    __syncthreads();
  }
  if (threadIdx.x < ent) partials[(int64_t)blockIdx.x * ent + threadIdx.x] = acc;
}

__global__ void reduce_cols_kernel(const double* __restrict__ partials, int nblk, int ent,
                                   double* __restrict__ out, const int* __restrict__ skip) {
  if (skip && *skip) return;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ent) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partials[(int64_t)b * ent + e];
  out[e] = s;
}

// fit_t = 1 - sqrt(max(||T||^2 - ||Q||^2, 0)) / ||T||; stop flag after sweep
// t > 1 when |fit_t - fit_{t-1}| < tol.
__global__ void fit_flag_kernel(const double* __restrict__ normX, const double* __restrict__ normQ,
                                int sweep, double tol, double* __restrict__ hist, double* __restrict__ last,
                                int* __restrict__ done, int* __restrict__ iters) {
  if (*done) return;
  double nx = *normX, nq = *normQ;
  // T = 0 fits exactly; a non-finite ||T||^2 (NaN or Inf in T) gives NaN
  double fit = (nx > 0.0 && isfinite(nx)) ? 1.0 - sqrt(fmax(nx - nq, 0.0)) / sqrt(nx) : (nx == 0.0 ? 1.0 : NAN);
  if (hist) hist[sweep - 1] = fit;
  if (iters) *iters = sweep;
  if (sweep > 1 && fabs(fit - *last) < tol) *done = 1;
  *last = fit;
}

__global__ void final_fit_kernel(const double* __restrict__ normX, const double* __restrict__ sse,
                                 double* __restrict__ fit) {
  double nx = *normX, e = *sse;
  *fit = (nx > 0.0 && isfinite(nx)) ? 1.0 - sqrt(fmax(e, 0.0)) / sqrt(nx) : (nx == 0.0 ? 1.0 : NAN);
  if (!(e == e)) *fit = NAN;   // fmax would hide a NaN residual
}

// Status of a decomposition from what the device recorded: a bounded
// tensor-core pipeline wait that gave up (error bits 8..64) is a timeout;
// a non-finite ||T||^2 or fit is NAN/Inf in the data.  On failure the fit is
// set to NaN so no caller mistakes the result for a valid one.
__global__ void finish_status_kernel(const int* __restrict__ flags, const double* __restrict__ normX,
                                     double* __restrict__ fit, int* __restrict__ status) {
  int code = MES_OK;
  if (flags[0] & (8 | 16 | 32 | 64)) code = MES_ERR_TIMEOUT;
  else if (normX && (!isfinite(*normX) || (fit && !isfinite(*fit)))) code = MES_ERR_NONFINITE;
  if (code != MES_OK && fit) *fit = NAN;
  if (status) *status = code;
}

// Per column q of U (s x r): the sign that makes its largest-magnitude entry
// (lowest index on ties) positive.
__global__ void __launch_bounds__(kT)
col_sign_kernel(const float* __restrict__ U, int64_t s, float* __restrict__ sign) {
  const int q = blockIdx.x;
  const float* u = U + (int64_t)q * s;
  float best = -1.f;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < s; i += kT) {
    float a = fabsf(u[i]);
    if (a > best) { best = a; bi = i; }
  }
  __shared__ float bv[kT];
  __shared__ int64_t bidx[kT];
  bv[threadIdx.x] = best;
  bidx[threadIdx.x] = bi;
  __syncthreads();
  for (int w = kT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      float o = bv[threadIdx.x + w];
      int64_t oi = bidx[threadIdx.x + w];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bidx[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bidx[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sign[q] = (u[bidx[0]] < 0.f) ? -1.f : 1.f;
}

// rank of each diagonal entry of H (r x r) in descending order, ties by index
__global__ void diag_order_kernel(const float* __restrict__ H, int r, int* __restrict__ src_of) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r) return;
  const float w = mes::order_key(H[i + (int64_t)r * i]);
  int rank = 0;
  for (int j = 0; j < r; ++j) {
    const float wj = mes::order_key(H[j + (int64_t)r * j]);
    if (wj > w || (wj == w && j < i)) ++rank;
  }
  src_of[rank] = i;
}

// Uout(:, q) = sign[q] * Uin(:, src_of[q]) (src_of may be null = identity)
__global__ void permute_cols_kernel(const float* __restrict__ Uin, int64_t s, int r,
                                    const int* __restrict__ src_of, const float* __restrict__ sign,
                                    float* __restrict__ Uout) {
  int64_t n = s * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = e / s, i = e - q * s;
    int src = src_of ? src_of[q] : (int)q;
    src = min(max(src, 0), r - 1);   // a gather index never leaves the matrix
    float sg = sign ? sign[q] : 1.f;
    Uout[e] = sg * Uin[i + s * src];
  }
}

// core index (first-mode fastest) along mode n with stride `stride`, size r:
// out[.., q, ..] = sign[q] * in[.., src_of[q], ..]
__global__ void permute_core_kernel(const float* __restrict__ in, int64_t total, int64_t stride, int r,
                                    const int* __restrict__ src_of, const float* __restrict__ sign,
                                    float* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = (e / stride) % r;
    int src = src_of ? src_of[q] : (int)q;
    src = min(max(src, 0), r - 1);   // a gather index never leaves the tensor
    float sg = sign ? sign[q] : 1.f;
    out[e] = sg * in[e + (src - q) * stride];
  }
}

__global__ void round_copy_kernel(const float* __restrict__ in, float* __restrict__ out, int64_t n,
                                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mes::round_tf32(in[i]);
}

__global__ void copy_kernel(const float* __restrict__ in, float* __restrict__ out, int64_t n,
                            const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

__global__ void identity_kernel(float* __restrict__ U, int64_t s, int r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s * r; i += (int64_t)gridDim.x * blockDim.x)
    U[i] = (i % s == i / s) ? 1.f : 0.f;
}

}  // namespace

namespace mes {

mes_status copy_if(const float* in, float* out, int64_t n, const int* skip, cudaStream_t st) {
  ProfScope prof("copy", st, 0.0, 8.0 * n);
  copy_kernel<<<grid_for(n, kT, 1024), kT, 0, st>>>(in, out, n, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status identity_fill(float* U, int64_t s, int r, cudaStream_t st) {
  ProfScope prof("identity", st, 0.0, 4.0 * s * r);
  identity_kernel<<<grid_for(s * r, kT, 64), kT, 0, st>>>(U, s, r);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status slice_transpose(const float* X, int64_t s1, int64_t s2, int64_t L, float* XB,
                           double* partials, int nblocks, cudaStream_t st, float* Xr, bool round,
                           uint16_t* X16, uint16_t* XB16) {
  ProfScope prof("slice_transpose", st, 0.0,
                 (4.0 + (XB ? 4 : 0) + (Xr ? 4 : 0) + (X16 ? 2 : 0) + (XB16 ? 2 : 0)) * s1 * s2 * L);
  slice_transpose_kernel<<<nblocks, kT, 0, st>>>(X, s1, s2, L, XB, partials, Xr, round ? 1 : 0, X16, XB16);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status split_tf32(const float* in, float* hi, float* lo, int64_t n, cudaStream_t st, const int* skip) {
  ProfScope prof("split_tf32", st, 0.0, 12.0 * n);
  split_tf32_kernel<<<grid_for(n, kT, 2048), kT, 0, st>>>(in, hi, lo, n, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status to_bf16(const float* in, uint16_t* out, int64_t n, const int* skip, cudaStream_t st) {
  ProfScope prof("to_bf16", st, 0.0, 6.0 * n);
  to_bf16_kernel<<<grid_for(n, kT, 2048), kT, 0, st>>>(in, out, n, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status round_copy(const float* in, float* out, int64_t n, const int* skip, cudaStream_t st) {
  ProfScope prof("round_copy", st, 0.0, 8.0 * n);
  round_copy_kernel<<<grid_for(n, kT, 1024), kT, 0, st>>>(in, out, n, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status sumsq(const float* x, int64_t n, double* partials, int nblocks, const int* skip,
                 cudaStream_t st) {
  ProfScope prof("sumsq", st, 0.0, 4.0 * n);
  sumsq_kernel<<<nblocks, kT, 0, st>>>(x, n, partials, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status uniform_fill(float* out, int64_t n, uint64_t seed, cudaStream_t st) {
  ProfScope prof("uniform", st, 0.0, 4.0 * n);
  uniform_kernel<<<grid_for(n, kT, 4096), kT, 0, st>>>(out, n, seed);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status mix_fibres(const Fibres& fb, const float* Kmat, int L, int L2, const int* skip,
                      cudaStream_t st) {
  size_t smem = (size_t)((L + 3) & ~3) * L2 * sizeof(float);   // rows padded for the register kernels
  if (smem > 64 * 1024) return fail(MES_ERR_NOT_IMPLEMENTED, "small modes too large for fibre mixing");
  static bool attr = false;
  if (!attr) {
    MES_CUDA_TRY(cudaFuncSetAttribute(mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    MES_CUDA_TRY(cudaFuncSetAttribute(mix_reg_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    MES_CUDA_TRY(cudaFuncSetAttribute(mix_reg_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    attr = true;
  }
  int64_t F = fb.F_lo * fb.F_hi;
  MES_TRY(audit(fb.in, ((fb.F_lo - 1) * fb.in_lo + (fb.F_hi - 1) * fb.in_hi + (int64_t)(L - 1) * fb.in_l) * 4,
                "mix in"));
  MES_TRY(audit(fb.out, ((fb.F_lo - 1) * fb.out_lo + (fb.F_hi - 1) * fb.out_hi + (int64_t)(L2 - 1) * fb.out_l) * 4,
                "mix out"));
  MES_TRY(audit(Kmat, (size_t)L * L2 * 4 - 1, "mix K"));
  ProfScope prof("mix_fibres", st, 2.0 * F * L * L2, 4.0 * F * (L + L2));
  const unsigned grid = grid_for(F, kT, (int64_t)sm_count() * 8);
  if (L <= 32)
    mix_reg_kernel<32><<<grid, kT, smem, st>>>(fb, Kmat, L, L2, skip);
  else if (L <= 64)
    mix_reg_kernel<64><<<grid, kT, smem, st>>>(fb, Kmat, L, L2, skip);
  else
    mix_kernel<<<grid, kT, smem, st>>>(fb, Kmat, L, L2, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

int small_gram_blocks(int64_t F) { return (int)grid_for((F + 31) / 32, 1, (int64_t)sm_count() * 4); }

mes_status small_gram(const Fibres& fb, const float* Kmat, int L, int L2, int sn, int inner,
                      double* partials, double* G, const int* skip, cudaStream_t st) {
  size_t smem = ((size_t)L * L2 + 32 * (size_t)L2) * sizeof(float);
  if (smem > 96 * 1024 || sn * sn > kT) return fail(MES_ERR_NOT_IMPLEMENTED, "small-mode Gram too large");
  static bool attr = false;
  if (!attr) {
    MES_CUDA_TRY(cudaFuncSetAttribute(small_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    attr = true;
  }
  int64_t F = fb.F_lo * fb.F_hi;
  int nb = small_gram_blocks(F);
  MES_TRY(audit(fb.in, ((fb.F_lo - 1) * fb.in_lo + (fb.F_hi - 1) * fb.in_hi + (int64_t)(L - 1) * fb.in_l) * 4,
                "gram in"));
  MES_TRY(audit(partials, (size_t)nb * sn * sn * 8 - 1, "gram partials"));
  MES_TRY(audit(G, (size_t)sn * sn * 8 - 1, "gram out"));
  MES_TRY(audit(Kmat, (size_t)L * L2 * 4 - 1, "gram K"));
  ProfScope prof("small_gram", st, 2.0 * F * L * L2, 4.0 * F * L);
  small_gram_kernel<<<nb, kT, smem, st>>>(fb, Kmat, L, L2, sn, inner, partials, skip);
  MES_LAUNCH_CHECK();
  ProfScope prof2("small_gram_reduce", st, 0.0, 8.0 * nb * sn * sn);
  reduce_cols_kernel<<<(sn * sn + 255) / 256, 256, 0, st>>>(partials, nb, sn * sn, G, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status fit_flag(const double* normX, const double* normQ, int sweep, double tol, double* hist,
                    double* last, int* done, int* iters, cudaStream_t st) {
  ProfScope prof("fit_flag", st, 0.0, 0.0);
  fit_flag_kernel<<<1, 1, 0, st>>>(normX, normQ, sweep, tol, hist, last, done, iters);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status final_fit(const double* normX, const double* sse, double* fit, cudaStream_t st) {
  ProfScope prof("fit_flag", st, 0.0, 0.0);
  final_fit_kernel<<<1, 1, 0, st>>>(normX, sse, fit);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status nan_on_timeout(const int* flags, double* x, cudaStream_t st) {
  finish_status_kernel<<<1, 1, 0, st>>>(flags, nullptr, x, nullptr);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status finish_status(const int* flags, const double* normX, double* fit, int* status, cudaStream_t st) {
  ProfScope prof("fit_flag", st, 0.0, 0.0);
  finish_status_kernel<<<1, 1, 0, st>>>(flags, normX, fit, status);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status col_signs(const float* U, int64_t s, int r, float* sign, cudaStream_t st) {
  ProfScope prof("col_sign", st, 0.0, 4.0 * s * r);
  col_sign_kernel<<<r, kT, 0, st>>>(U, s, sign);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status diag_order(const float* H, int r, int* src_of, cudaStream_t st) {
  ProfScope prof("diag_order", st, 0.0, 4.0 * r);
  diag_order_kernel<<<(r + 127) / 128, 128, 0, st>>>(H, r, src_of);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status permute_cols(const float* Uin, int64_t s, int r, const int* src_of, const float* sign,
                        float* Uout, cudaStream_t st) {
  ProfScope prof("permute", st, 0.0, 8.0 * s * r);
  permute_cols_kernel<<<grid_for(s * r, kT, 4096), kT, 0, st>>>(Uin, s, r, src_of, sign, Uout);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

mes_status permute_core(const float* in, int64_t total, int64_t stride, int r, const int* src_of,
                        const float* sign, float* out, cudaStream_t st) {
  ProfScope prof("permute", st, 0.0, 8.0 * total);
  permute_core_kernel<<<grid_for(total, kT, 4096), kT, 0, st>>>(in, total, stride, r, src_of, sign, out);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

}  // namespace mes

namespace {

__global__ void kron_kernel(mes::KronDesc d, int rows, int cols, float* __restrict__ K,
                            const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x) {
    int o = e / cols, l = e - o * cols;
    float v = 1.f;
    for (int m = 0; m < d.nm; ++m) {
      int ro = (d.op[m] == 'T') ? d.r[m] : d.s[m];      // rows of this factor
      int co = (d.op[m] == 'N') ? d.r[m] : d.s[m];      // cols of this factor
      int io = o % ro, il = l % co;
      o /= ro;
      l /= co;
      float f;
      if (d.op[m] == 'I') f = (io == il) ? 1.f : 0.f;
      else if (d.op[m] == 'T') f = d.U[m][il + (int64_t)d.s[m] * io];   // U^T(io, il) = U(il, io)
      else f = d.U[m][io + (int64_t)d.s[m] * il];                      // U(io, il)
      v *= f;
    }
    K[e] = v;
  }
}

}  // namespace

namespace mes {

int KronDesc::rows() const {
  int p = 1;
  for (int m = 0; m < nm; ++m) p *= (op[m] == 'T') ? r[m] : s[m];
  return p;
}

int KronDesc::cols() const {
  int p = 1;
  for (int m = 0; m < nm; ++m) p *= (op[m] == 'N') ? r[m] : s[m];
  return p;
}

mes_status kron_build(const KronDesc& d, float* K, const int* skip, cudaStream_t st) {
  int rows = d.rows(), cols = d.cols();
  ProfScope prof("kron_build", st, 0.0, 4.0 * rows * cols);
  kron_kernel<<<grid_for((int64_t)rows * cols, 256, 64), 256, 0, st>>>(d, rows, cols, K, skip);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

}  // namespace mes

// Colour pre-pass (Section III-A): 8-bit R'G'B' images -> Y'CbCr (BT.601)
// or IPT planes of the stacked tensor (Section III-B), with ||T||_F^2 fused.
//
// Bandwidth kernel: each thread converts 8 consecutive pixels of one image
// (24 bytes in, 96 bytes out as three float4 pairs, one per channel plane).
// The u8 -> [0,1] scaling and the IPT linearisation go through a 256-entry
// table built per block, so the only transcendental left per pixel is the
// 0.43 power of the three cone responses.  The squared norm is accumulated
// in FP64 per thread, reduced per block, and the per-block partials are
// summed by one block in a fixed order, so the result is reproducible.
#include "common.cuh"

namespace {

struct ColourParams {
  float a[9];      // R,G,B (linear) -> L,M,S  (row-major 3x3)
  float b[9];      // L',M',S' -> I,P,T       (row-major 3x3)
  float gamma;
  int space;
};

constexpr int kThreads = 256;
constexpr int kPix = 8;

__device__ __forceinline__ float signed_pow043(float v) {
  float a = fabsf(v);
  float p = (a > 0.f) ? exp2f(0.43f * __log2f(a)) : 0.f;
  return copysignf(p, v);
}

__device__ __forceinline__ void convert_pixel(const ColourParams& P, const float* lut_lin,
                                              const float* lut_p, int r8, int g8, int b8,
                                              float& c0, float& c1, float& c2) {
  if (P.space == MES_YCBCR601) {
    float r = lut_p[r8], g = lut_p[g8], b = lut_p[b8];
    float y = fmaf(0.299f, r, fmaf(0.587f, g, 0.114f * b));
    c0 = y;
    c1 = (b - y) * (1.0f / 1.772f);
    c2 = (r - y) * (1.0f / 1.402f);
  } else {
    float r = lut_lin[r8], g = lut_lin[g8], b = lut_lin[b8];
    float L = fmaf(P.a[0], r, fmaf(P.a[1], g, P.a[2] * b));
    float M = fmaf(P.a[3], r, fmaf(P.a[4], g, P.a[5] * b));
    float S = fmaf(P.a[6], r, fmaf(P.a[7], g, P.a[8] * b));
    L = signed_pow043(L);
    M = signed_pow043(M);
    S = signed_pow043(S);
    c0 = fmaf(P.b[0], L, fmaf(P.b[1], M, P.b[2] * S));
    c1 = fmaf(P.b[3], L, fmaf(P.b[4], M, P.b[5] * S));
    c2 = fmaf(P.b[6], L, fmaf(P.b[7], M, P.b[8] * S));
  }
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (l < kThreads / 32) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kThreads)
colour_kernel(const uint8_t* __restrict__ rgb8, int64_t npix, int64_t K, ColourParams P,
              float* __restrict__ out, double* __restrict__ partials) {
  __shared__ float lut_lin[256];
  __shared__ float lut_p[256];
  for (int v = threadIdx.x; v < 256; v += blockDim.x) {
    float p = (float)v / 255.0f;
    lut_p[v] = p;
    lut_lin[v] = (P.space == MES_IPT) ? powf(p, P.gamma) : p;
  }
  __syncthreads();

  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (npix % kPix == 0) {
    const int64_t groups_per_img = npix / kPix;
    const int64_t total = groups_per_img * K;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
      const int64_t k = g / groups_per_img;
      const int64_t p0 = (g - k * groups_per_img) * kPix;
      // 8 pixels = 24 bytes, 8-byte aligned because npix % 8 == 0
      const uint2* src = reinterpret_cast<const uint2*>(rgb8 + (k * npix + p0) * 3);
      uint2 w0 = __ldg(src), w1 = __ldg(src + 1), w2 = __ldg(src + 2);
      uint32_t words[6] = {w0.x, w0.y, w1.x, w1.y, w2.x, w2.y};
      float o[3][kPix];
#pragma unroll
      for (int i = 0; i < kPix; ++i) {
        int bytes[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          int bi = i * 3 + c;
          bytes[c] = (words[bi >> 2] >> ((bi & 3) * 8)) & 0xff;
        }
        convert_pixel(P, lut_lin, lut_p, bytes[0], bytes[1], bytes[2], o[0][i], o[1][i], o[2][i]);
      }
      // the 24 squares of this group summed in FP32, then one FP64 add
      // (the FP64 rate is a small fraction of the FP32 rate on this GPU)
      float part = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float4* dst = reinterpret_cast<float4*>(out + (c + 3 * k) * npix + p0);
        dst[0] = make_float4(o[c][0], o[c][1], o[c][2], o[c][3]);
        dst[1] = make_float4(o[c][4], o[c][5], o[c][6], o[c][7]);
#pragma unroll
        for (int i = 0; i < kPix; ++i) part = fmaf(o[c][i], o[c][i], part);
      }
      acc += (double)part;
    }
  } else {
    const int64_t total = npix * K;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
      const int64_t k = g / npix;
      const int64_t p = g - k * npix;
      const uint8_t* s = rgb8 + (k * npix + p) * 3;
      float c0, c1, c2;
      convert_pixel(P, lut_lin, lut_p, s[0], s[1], s[2], c0, c1, c2);
      out[(3 * k + 0) * npix + p] = c0;
      out[(3 * k + 1) * npix + p] = c1;
      out[(3 * k + 2) * npix + p] = c2;
      acc += (double)fmaf(c0, c0, fmaf(c1, c1, c2 * c2));
    }
  }
  if (partials) {
    double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

// Sums n partials in a fixed order with one block.
__global__ void __launch_bounds__(kThreads)
sum_partials_kernel(const double* __restrict__ partials, int n, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  double t = block_sum(acc);
  if (threadIdx.x == 0) *out = t;
}

void make_params(int space, float gamma, ColourParams* P) {
  // Linear sRGB (D65) -> XYZ (IEC 61966-2-1) and XYZ -> LMS (Hunt-Pointer-
  // Estevez normalised to D65), multiplied once here in double.
  const double rgb2xyz[9] = {0.4124, 0.3576, 0.1805, 0.2126, 0.7152, 0.0722, 0.0193, 0.1192, 0.9505};
  const double xyz2lms[9] = {0.4002, 0.7075, -0.0807, -0.2280, 1.1500, 0.0612, 0.0, 0.0, 0.9184};
  const double lms2ipt[9] = {0.4000, 0.4000, 0.2000, 4.4550, -4.8510, 0.3960, 0.8056, 0.3572, -1.1628};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += xyz2lms[i * 3 + k] * rgb2xyz[k * 3 + j];
      P->a[i * 3 + j] = (float)s;
      P->b[i * 3 + j] = (float)lms2ipt[i * 3 + j];
    }
  P->gamma = gamma;
  P->space = space;
}

}  // namespace

namespace mes {

// Grid used by the colour kernel: a fixed multiple of the SM count so the
// reduction order, and hence the FP64 norm, is reproducible.
unsigned colour_grid(int64_t npix, int64_t K) {
  int64_t work = (npix % kPix == 0) ? npix / kPix * K : npix * K;
  return grid_for(work, kThreads, (int64_t)sm_count() * 8);
}

mes_status colour_launch(const uint8_t* rgb8, int64_t s1, int64_t s2, int64_t K, int space,
                         float gamma, float* out, double* partials, double* norm2,
                         cudaStream_t st) {
  ColourParams P;
  make_params(space, gamma, &P);
  const int64_t npix = s1 * s2;
  unsigned grid = colour_grid(npix, K);
  {
  ProfScope prof("colour", st, 0.0, 15.0 * npix * K);
  colour_kernel<<<grid, kThreads, 0, st>>>(rgb8, npix, K, P, out, norm2 ? partials : nullptr);
  MES_LAUNCH_CHECK();
  }
  if (norm2) {
    ProfScope prof("sum_doubles", st, 0.0, 8.0 * grid);
    sum_partials_kernel<<<1, kThreads, 0, st>>>(partials, (int)grid, norm2);
    MES_LAUNCH_CHECK();
  }
  return MES_OK;
}

}  // namespace mes

extern "C" mes_status mes_colour_convert(const uint8_t* rgb8, int64_t s1, int64_t s2, int64_t K,
                                         int space, float gamma, float* out, double* norm2,
                                         void* stream) {
  mes::clear_error();
  if (!rgb8 || !out) return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_convert: null rgb8 or out");
  if (s1 < 1 || s2 < 1 || K < 1)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_convert: sizes must be >= 1 (got %lld %lld %lld)",
                     (long long)s1, (long long)s2, (long long)K);
  if (space != MES_YCBCR601 && space != MES_IPT)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_convert: unknown colour space %d", space);
  if (!(gamma > 0.f)) return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_convert: gamma must be > 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mes::Scratch scratch(st);
  double* partials = nullptr;
  if (norm2) MES_TRY(scratch.alloc(&partials, mes::colour_grid(s1 * s2, K)));
  return mes::colour_launch(rgb8, s1, s2, K, space, gamma, out, partials, norm2, st);
}

// Colour pre-pass (Section III-A): 8-bit R'G'B' images -> Y'CbCr (BT.601),
// IPT or constant-luminance Y'CbCr (BT.2020) planes of the stacked tensor
// (Section III-B), with ||T||_F^2 fused; and its inverse, tensor -> 8-bit
// images (the approximated views handed to the encoder, Section III-C).
//
// Bandwidth kernel: each thread converts 8 consecutive pixels of one image
// (24 bytes in, 96 bytes out as three float4 pairs, one per channel plane).
// The u8 -> [0,1] scaling and the linearisation go through a 256-entry
// table built per block, so the only transcendentals left per pixel are the
// 0.43 power of the three cone responses (IPT) or the transfer function of
// Yc, B and R (BT.2020 constant luminance).  The squared norm is accumulated
// in FP64 per thread, reduced per block, and the per-block partials are
// summed by one block in a fixed order, so the result is reproducible.
#include <cmath>

#include "common.cuh"

namespace {

struct ColourParams {
  float a[9];      // IPT: R,G,B (linear) -> L,M,S; BT.2020 CL: BT.709 -> BT.2020 primaries
  float b[9];      // IPT: L',M',S' -> I,P,T      (row-major 3x3)
  float gamma;
  int space;
};

// BT.2020 luminance weights, transfer function (12-bit constants) and the
// constant-luminance chroma divisors N_b, P_b, N_r, P_r
constexpr float kKr20 = 0.2627f, kKg20 = 0.6780f, kKb20 = 0.0593f;
constexpr float kAlpha = 1.0993f, kBeta = 0.0181f;
constexpr float kNb = 1.9404f, kPb = 1.5816f, kNr = 1.7184f, kPr = 0.9936f;

__device__ __forceinline__ float oetf2020(float e) {
  return e < kBeta ? 4.5f * e : fmaf(kAlpha, powf(e, 0.45f), -(kAlpha - 1.f));
}

__device__ __forceinline__ float oetf2020_inverse(float e) {
  return e < 4.5f * kBeta ? e * (1.f / 4.5f) : powf((e + (kAlpha - 1.f)) / kAlpha, 1.f / 0.45f);
}

constexpr int kThreads = 256;
constexpr int kPix = 8;

// x^0.43 of the IPT cone responses, written for this one exponent (the
// general powf made the pre-pass issue-bound: three per pixel).  With
// x = m 2^e, m in [1, 2): x^0.43 = 2^(0.43 e) m^0.43, the first factor from a
// table over the 254 normal exponents, the second on 16 sub-intervals of
// [1, 2) as c^0.43 (1 + v)^0.43 with c the sub-interval's centre, v = m/c - 1
// (|v| <= 1/32) and the binomial series to degree 4 (the first term left out
// is below 1e-9).  The tables are computed on the host in double precision
// and rounded once, so the result is within a few ulp of x^0.43: accurate
// enough that the inverse transform still recovers the 8-bit input exactly
// (the fast log2/exp2 pair, errors up to 2e-5, did not).  Zero and subnormal
// inputs (below 2^-126, so x^0.43 < 2^-54) give 0.
struct Pow043 {
  float t2[254];                 // 2^(0.43 e), e = -126 .. 127
  float ic[16], pc[16];          // 1 / c and c^0.43 for the sub-interval centres c = 1 + (j + 1/2)/16
  float a[4];                    // binomial coefficients of (1 + v)^0.43, degrees 1 .. 4
};

struct Pow043Smem {
  float t2[256];
  float4 cp[16];                 // (c, 1 / c, c^0.43, 0) per sub-interval: one 16-byte load
};

// x >= 0 (zero, subnormals and a negative zero give 0)
__device__ __forceinline__ float pow043(float x, const Pow043Smem& T, const float (&a)[4]) {
  const uint32_t u = __float_as_uint(x);
  const int eb = (int)(u >> 23);   // biased exponent
  if (eb == 0 || eb > 254) return 0.f;
  const int j = (int)((u >> 19) & 15u);
  const float m = __uint_as_float((u & 0x7FFFFFu) | 0x3F800000u);
  const float4 t = T.cp[j];
  const float v = (m - t.x) * t.y;
  const float p = fmaf(v, fmaf(v, fmaf(v, fmaf(v, a[3], a[2]), a[1]), a[0]), 1.f);
  return (t.z * T.t2[eb - 1]) * p;
}

__device__ __forceinline__ void convert_pixel(const ColourParams& P, const float* lut_lin,
                                              const float* lut_p, const Pow043Smem& T, const float (&pa)[4],
                                              int r8, int g8, int b8, float& c0, float& c1, float& c2) {
  if (P.space == MES_YCBCR601) {
    float r = lut_p[r8], g = lut_p[g8], b = lut_p[b8];
    float y = fmaf(0.299f, r, fmaf(0.587f, g, 0.114f * b));
    c0 = y;
    c1 = (b - y) * (1.0f / 1.772f);
    c2 = (r - y) * (1.0f / 1.402f);
  } else if (P.space == MES_YCBCR2020CL) {
    float r = lut_lin[r8], g = lut_lin[g8], b = lut_lin[b8];
    float R = fmaf(P.a[0], r, fmaf(P.a[1], g, P.a[2] * b));
    float G = fmaf(P.a[3], r, fmaf(P.a[4], g, P.a[5] * b));
    float B = fmaf(P.a[6], r, fmaf(P.a[7], g, P.a[8] * b));
    float yc = oetf2020(fmaf(kKr20, R, fmaf(kKg20, G, kKb20 * B)));
    float db = oetf2020(B) - yc, dr = oetf2020(R) - yc;
    c0 = yc;
    c1 = db <= 0.f ? db * (1.f / kNb) : db * (1.f / kPb);
    c2 = dr <= 0.f ? dr * (1.f / kNr) : dr * (1.f / kPr);
  } else {
    float r = lut_lin[r8], g = lut_lin[g8], b = lut_lin[b8];
    float L = fmaf(P.a[0], r, fmaf(P.a[1], g, P.a[2] * b));
    float M = fmaf(P.a[3], r, fmaf(P.a[4], g, P.a[5] * b));
    float S = fmaf(P.a[6], r, fmaf(P.a[7], g, P.a[8] * b));
    // every entry of the linear-sRGB -> LMS matrix is positive (the product
    // of the published XYZ and cone matrices), so the cone responses of
    // 8-bit input are >= 0; the clamp only absorbs a rounding to -0
    L = pow043(fmaxf(L, 0.f), T, pa);
    M = pow043(fmaxf(M, 0.f), T, pa);
    S = pow043(fmaxf(S, 0.f), T, pa);
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
colour_kernel(const uint8_t* __restrict__ rgb8, int64_t npix, int64_t K, ColourParams P, const Pow043 PT,
              float* __restrict__ out, double* __restrict__ partials) {
  __shared__ float lut_lin[256];
  __shared__ float lut_p[256];
  __shared__ Pow043Smem T;
  for (int v = threadIdx.x; v < 256; v += blockDim.x) {
    float p = (float)v / 255.0f;
    lut_p[v] = p;
    lut_lin[v] = (P.space != MES_YCBCR601) ? powf(p, P.gamma) : p;
    T.t2[v] = v < 254 ? PT.t2[v] : 0.f;
    if (v < 16) T.cp[v] = make_float4(1.f + (v + 0.5f) / 16.f, PT.ic[v], PT.pc[v], 0.f);
  }
  const float pa[4] = {PT.a[0], PT.a[1], PT.a[2], PT.a[3]};
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
        convert_pixel(P, lut_lin, lut_p, T, pa, bytes[0], bytes[1], bytes[2], o[0][i], o[1][i], o[2][i]);
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
      convert_pixel(P, lut_lin, lut_p, T, pa, s[0], s[1], s[2], c0, c1, c2);
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

// Linear sRGB (D65) -> XYZ (IEC 61966-2-1), XYZ -> LMS (Hunt-Pointer-Estevez
// normalised to D65), L'M'S' -> IPT (Ebner-Fairchild), linear BT.709 ->
// BT.2020 primaries (ITU-R BT.2087); row-major.
const double kRgb2Xyz[9] = {0.4124, 0.3576, 0.1805, 0.2126, 0.7152, 0.0722, 0.0193, 0.1192, 0.9505};
const double kXyz2Lms[9] = {0.4002, 0.7075, -0.0807, -0.2280, 1.1500, 0.0612, 0.0, 0.0, 0.9184};
const double kLms2Ipt[9] = {0.4000, 0.4000, 0.2000, 4.4550, -4.8510, 0.3960, 0.8056, 0.3572, -1.1628};
const double k709To2020[9] = {0.6274, 0.3293, 0.0433, 0.0691, 0.9195, 0.0114, 0.0164, 0.0880, 0.8956};

void mul3(const double* x, const double* y, double* out) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += x[i * 3 + k] * y[k * 3 + j];
      out[i * 3 + j] = s;
    }
}

// inverse of a 3x3 matrix by its adjugate (the matrices here are far from
// singular)
void inv3(const double* m, double* out) {
  const double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
  const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  out[0] = c00 / det;
  out[1] = (m[2] * m[7] - m[1] * m[8]) / det;
  out[2] = (m[1] * m[5] - m[2] * m[4]) / det;
  out[3] = c01 / det;
  out[4] = (m[0] * m[8] - m[2] * m[6]) / det;
  out[5] = (m[2] * m[3] - m[0] * m[5]) / det;
  out[6] = c02 / det;
  out[7] = (m[1] * m[6] - m[0] * m[7]) / det;
  out[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

// forward parameters; with `inverse` the matrices of the inverse transform
// (a: LMS -> linear RGB or BT.2020 -> BT.709 primaries, b: IPT -> L'M'S')
void make_params(int space, float gamma, ColourParams* P, bool inverse = false) {
  double a[9], b[9], t[9];
  if (space == MES_YCBCR2020CL) {
    for (int i = 0; i < 9; ++i) a[i] = k709To2020[i];
  } else {
    mul3(kXyz2Lms, kRgb2Xyz, a);
  }
  for (int i = 0; i < 9; ++i) b[i] = kLms2Ipt[i];
  if (inverse) {
    inv3(a, t);
    for (int i = 0; i < 9; ++i) a[i] = t[i];
    inv3(b, t);
    for (int i = 0; i < 9; ++i) b[i] = t[i];
  }
  for (int i = 0; i < 9; ++i) {
    P->a[i] = (float)a[i];
    P->b[i] = (float)b[i];
  }
  P->gamma = gamma;
  P->space = space;
}

__device__ __forceinline__ float signed_pow(float v, float e) {
  float a = fabsf(v);
  return copysignf(a > 0.f ? powf(a, e) : 0.f, v);
}

// one pixel of the inverse transform: tensor channels -> R'G'B'
__device__ __forceinline__ void invert_pixel(const ColourParams& P, float c0, float c1, float c2, float& r,
                                             float& g, float& b) {
  if (P.space == MES_YCBCR601) {
    r = fmaf(1.402f, c2, c0);
    b = fmaf(1.772f, c1, c0);
    g = (c0 - 0.299f * r - 0.114f * b) * (1.f / 0.587f);
    return;
  }
  float x, y, z;
  if (P.space == MES_YCBCR2020CL) {
    const float bp = fmaf(c1 <= 0.f ? kNb : kPb, c1, c0);
    const float rp = fmaf(c2 <= 0.f ? kNr : kPr, c2, c0);
    const float yc = oetf2020_inverse(c0), B = oetf2020_inverse(bp), R = oetf2020_inverse(rp);
    x = R;
    y = (yc - kKr20 * R - kKb20 * B) * (1.f / kKg20);
    z = B;
  } else {
    x = signed_pow(fmaf(P.b[0], c0, fmaf(P.b[1], c1, P.b[2] * c2)), 1.f / 0.43f);
    y = signed_pow(fmaf(P.b[3], c0, fmaf(P.b[4], c1, P.b[5] * c2)), 1.f / 0.43f);
    z = signed_pow(fmaf(P.b[6], c0, fmaf(P.b[7], c1, P.b[8] * c2)), 1.f / 0.43f);
  }
  const float ig = 1.f / P.gamma;
  r = signed_pow(fmaf(P.a[0], x, fmaf(P.a[1], y, P.a[2] * z)), ig);
  g = signed_pow(fmaf(P.a[3], x, fmaf(P.a[4], y, P.a[5] * z)), ig);
  b = signed_pow(fmaf(P.a[6], x, fmaf(P.a[7], y, P.a[8] * z)), ig);
}

__device__ __forceinline__ uint32_t to_u8(float v) {
  // fmaxf/fminf drop a NaN, which then becomes 0
  return (uint32_t)__float2int_rn(fminf(fmaxf(255.f * v, 0.f), 255.f));
}

constexpr int kInvPix = 4;

// Inverse transform.  Fast path (npix % 4 == 0): a thread takes 4
// consecutive pixels of one image, reads a float4 from each channel plane
// and writes 12 bytes (three 32-bit words) and/or 12 floats (three float4).
__global__ void __launch_bounds__(kThreads)
colour_invert_kernel(const float* __restrict__ X, int64_t npix, int64_t K, ColourParams P,
                     uint8_t* __restrict__ rgb8, float* __restrict__ rgbp, const uint8_t* __restrict__ ref8,
                     double* __restrict__ partials) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long err = 0;   // sum of squared byte differences, exact
  if (npix % kInvPix == 0) {
    const int64_t per_img = npix / kInvPix;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < per_img * K; t += stride) {
      const int64_t k = t / per_img;
      const int64_t p0 = (t - k * per_img) * kInvPix;
      const float4 a = __ldg(reinterpret_cast<const float4*>(X + (3 * k + 0) * npix + p0));
      const float4 bq = __ldg(reinterpret_cast<const float4*>(X + (3 * k + 1) * npix + p0));
      const float4 cq = __ldg(reinterpret_cast<const float4*>(X + (3 * k + 2) * npix + p0));
      const float c0[4] = {a.x, a.y, a.z, a.w}, c1[4] = {bq.x, bq.y, bq.z, bq.w}, c2[4] = {cq.x, cq.y, cq.z, cq.w};
      float o[12];
#pragma unroll
      for (int i = 0; i < kInvPix; ++i) invert_pixel(P, c0[i], c1[i], c2[i], o[3 * i], o[3 * i + 1], o[3 * i + 2]);
      const int64_t base = (k * npix + p0) * 3;   // a multiple of 12
      if (rgbp) {
        float4* dst = reinterpret_cast<float4*>(rgbp + base);
        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
        dst[2] = make_float4(o[8], o[9], o[10], o[11]);
      }
      if (rgb8 || ref8) {
        uint32_t w[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          w[j] = to_u8(o[4 * j]) | (to_u8(o[4 * j + 1]) << 8) | (to_u8(o[4 * j + 2]) << 16) |
                 (to_u8(o[4 * j + 3]) << 24);
        if (rgb8) {
          uint32_t* dst = reinterpret_cast<uint32_t*>(rgb8 + base);
          dst[0] = w[0];
          dst[1] = w[1];
          dst[2] = w[2];
        }
        if (ref8) {
          const uint32_t* r = reinterpret_cast<const uint32_t*>(ref8 + base);
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const uint32_t v = __ldg(r + j);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int d = (int)((w[j] >> (8 * q)) & 0xff) - (int)((v >> (8 * q)) & 0xff);
              err += (unsigned long long)(d * d);
            }
          }
        }
      }
    }
  } else {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npix * K; t += stride) {
      const int64_t k = t / npix;
      const int64_t p = t - k * npix;
      float r, g, b;
      invert_pixel(P, X[(3 * k) * npix + p], X[(3 * k + 1) * npix + p], X[(3 * k + 2) * npix + p], r, g, b);
      const int64_t base = (k * npix + p) * 3;
      if (rgbp) {
        rgbp[base] = r;
        rgbp[base + 1] = g;
        rgbp[base + 2] = b;
      }
      const uint32_t o8[3] = {to_u8(r), to_u8(g), to_u8(b)};
      if (rgb8) {
        rgb8[base] = (uint8_t)o8[0];
        rgb8[base + 1] = (uint8_t)o8[1];
        rgb8[base + 2] = (uint8_t)o8[2];
      }
      if (ref8) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int d = (int)o8[c] - (int)ref8[base + c];
          err += (unsigned long long)(d * d);
        }
      }
    }
  }
  if (partials) {
    // per-thread sums are below 2^53 for any image count that fits in memory,
    // so the FP64 block sum is exact and the result reproducible
    double t = block_sum((double)err);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

}  // namespace

namespace mes {

// Grid used by the colour kernel: a fixed multiple of the SM count so the
// reduction order, and hence the FP64 norm, is reproducible.
unsigned colour_grid(int64_t npix, int64_t K) {
  int64_t work = (npix % kPix == 0) ? npix / kPix * K : npix * K;
  return grid_for(work, kThreads, (int64_t)sm_count() * 8);
}

// Tables of pow043, in double precision, rounded once (built on first use).
const Pow043& pow043_tables() {
  static const Pow043 T = [] {
    Pow043 t;
    for (int i = 0; i < 254; ++i) t.t2[i] = (float)std::exp2(0.43 * (double)(i + 1 - 127));
    for (int j = 0; j < 16; ++j) {
      const double c = 1.0 + (j + 0.5) / 16.0;   // exactly representable
      t.ic[j] = (float)(1.0 / c);
      t.pc[j] = (float)std::pow(c, 0.43);
    }
    double coef = 1.0;
    for (int k = 1; k <= 4; ++k) {
      coef *= (0.43 - (k - 1)) / k;   // generalised binomial coefficient C(0.43, k)
      t.a[k - 1] = (float)coef;
    }
    return t;
  }();
  return T;
}

mes_status colour_launch(const uint8_t* rgb8, int64_t s1, int64_t s2, int64_t K, int space,
                         float gamma, float* out, double* partials, double* norm2,
                         cudaStream_t st) {
  ColourParams P;
  make_params(space, gamma, &P);
  const Pow043& PT = pow043_tables();
  const int64_t npix = s1 * s2;
  unsigned grid = colour_grid(npix, K);
  {
  ProfScope prof("colour", st, 0.0, 15.0 * npix * K);
  colour_kernel<<<grid, kThreads, 0, st>>>(rgb8, npix, K, P, PT, out, norm2 ? partials : nullptr);
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
  if (space != MES_YCBCR601 && space != MES_IPT && space != MES_YCBCR2020CL)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_convert: unknown colour space %d", space);
  if (!(gamma > 0.f)) return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_convert: gamma must be > 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mes::Trace trace("mes_colour_convert", st);
  trace.phase("colour");
  mes::Scratch scratch(st);
  double* partials = nullptr;
  if (norm2) MES_TRY(scratch.alloc(&partials, mes::colour_grid(s1 * s2, K)));
  return mes::colour_launch(rgb8, s1, s2, K, space, gamma, out, partials, norm2, st);
}

extern "C" mes_status mes_colour_invert(const float* X, int64_t s1, int64_t s2, int64_t K, int space,
                                        float gamma, uint8_t* rgb8, float* rgbp, const uint8_t* ref8,
                                        double* sse8, void* stream) {
  mes::clear_error();
  if (!X || (!rgb8 && !rgbp && !sse8))
    return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_invert: null X or no output");
  if (!ref8 != !sse8)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_invert: ref8 and sse8 go together");
  if (s1 < 1 || s2 < 1 || K < 1)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_invert: sizes must be >= 1 (got %lld %lld %lld)",
                     (long long)s1, (long long)s2, (long long)K);
  if (space != MES_YCBCR601 && space != MES_IPT && space != MES_YCBCR2020CL)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_invert: unknown colour space %d", space);
  if (!(gamma > 0.f)) return mes::fail(MES_ERR_INVALID_ARG, "mes_colour_invert: gamma must be > 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ColourParams P;
  make_params(space, gamma, &P, true);
  const int64_t npix = s1 * s2;
  const int64_t work = (npix % kInvPix == 0) ? npix / kInvPix * K : npix * K;
  const unsigned grid = mes::grid_for(work, kThreads, (int64_t)mes::sm_count() * 8);
  mes::ProfScope prof("colour_invert", st, 0.0, (12.0 + (rgb8 ? 3.0 : 0.0) + (rgbp ? 12.0 : 0.0)) * npix * K);
  double* partials = nullptr;
  mes::Scratch scratch(st);
  if (sse8) MES_TRY(scratch.alloc(&partials, grid));
  colour_invert_kernel<<<grid, kThreads, 0, st>>>(X, npix, K, P, rgb8, rgbp, ref8, partials);
  MES_LAUNCH_CHECK();
  if (sse8) {
    sum_partials_kernel<<<1, kThreads, 0, st>>>(partials, (int)grid, sse8);
    MES_LAUNCH_CHECK();
  }
  return MES_OK;
}

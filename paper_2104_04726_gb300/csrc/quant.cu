// Core quantiser (the rate knob of the scheme: the abstract and Section I set
// the bit rate through the core's ranks and the quantisation of the core, which
// the paper does not define further).  Per r1 x r2 plane of the core:
// m = max|x| (exact), scale = m / qmax, q = clamp(rint(x / scale)).
//
// Two bandwidth passes over the core:
//   1. per-(plane, chunk) block max of |x| as IEEE bit patterns (for x >= 0
//      the unsigned order of the bits is the float order, so atomicMax on the
//      bits is an exact, order-free max), into a per-plane scratch word;
//   2. quantise every element with IEEE round-to-nearest division
//      (__fdiv_rn) and round-half-even conversion (__float2int_rn).
// Built without fast-math, so both divisions are correctly rounded and the
// codes are bit-exact against any IEEE FP32 implementation of the same steps.
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kMaxPlaneElems = (int64_t)1 << 40;   // keeps grid.x and every index in range

__global__ void __launch_bounds__(kThreads)
plane_absmax_kernel(const float* __restrict__ core, int64_t plane_size, int64_t chunk,
                    unsigned* __restrict__ maxbits) {
  const int64_t p = blockIdx.y;
  const int64_t begin = (int64_t)blockIdx.x * chunk;
  int64_t end = begin + chunk;
  if (end > plane_size) end = plane_size;
  const float* src = core + p * plane_size;
  unsigned m = 0u;
  for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
    unsigned b = __float_as_uint(fabsf(__ldg(src + i)));
    m = max(m, b);
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ unsigned red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0u;
    for (int w = 0; w < kThreads / 32; ++w) t = max(t, red[w]);
    atomicMax(maxbits + p, t);
  }
}

// Grid (chunks of a plane, planes): the plane comes from blockIdx.y, so no
// element needs an integer division, and the plane's scale is one FP32
// division per thread rather than per element (the same IEEE operation, so
// the codes do not change).
__global__ void __launch_bounds__(kThreads)
quantize_kernel(const float* __restrict__ core, int64_t plane_size, int64_t chunk,
                const unsigned* __restrict__ maxbits, float qmax, int16_t* __restrict__ q,
                float* __restrict__ scales) {
  const int64_t p = blockIdx.y;
  const int64_t begin = (int64_t)blockIdx.x * chunk;
  int64_t end = begin + chunk;
  if (end > plane_size) end = plane_size;
  const float m = __uint_as_float(maxbits[p]);
  const float scale = (m != 0.f) ? __fdiv_rn(m, qmax) : 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) scales[p] = scale;
  const float* src = core + p * plane_size;
  int16_t* dst = q + p * plane_size;
  const int iq = (int)qmax;
  for (int64_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
    int16_t code = 0;
    if (m != 0.f) {
      int c = __float2int_rn(__fdiv_rn(__ldg(src + i), scale));
      c = c > iq ? iq : (c < -iq ? -iq : c);
      code = (int16_t)c;
    }
    dst[i] = code;
  }
}

__global__ void __launch_bounds__(kThreads)
dequantize_kernel(const int16_t* __restrict__ q, const float* __restrict__ scales,
                  int64_t plane_size, int64_t total, float* __restrict__ core) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t p = i / plane_size;
    core[i] = __fmul_rn((float)q[i], scales[p]);
  }
}

}  // namespace

namespace mes {

// Plane geometry: plane_size = r1 * r2 (r2 = 1 when N = 1), planes =
// prod_{n>=3} r_n.  Each factor is checked against the limit before it is
// multiplied in, so ranks whose product would wrap int64 are rejected rather
// than passing the limit test as a small or negative count.
mes_status quant_plane_shape(int N, const int64_t* ranks, int64_t max_planes, int64_t* plane_size,
                             int64_t* planes, const char* who) {
  if (N < 1 || N > 8 || !ranks) return fail(MES_ERR_INVALID_ARG, "%s: N must be 1..8", who);
  for (int n = 0; n < N; ++n)
    if (ranks[n] < 1) return fail(MES_ERR_INVALID_ARG, "%s: ranks must be >= 1", who);
  const int64_t r1 = ranks[0], r2 = N >= 2 ? ranks[1] : 1;
  if (r1 > kMaxPlaneElems || r2 > kMaxPlaneElems / r1)
    return fail(MES_ERR_INVALID_ARG, "%s: a plane of %lld x %lld elements exceeds 2^40", who, (long long)r1,
                (long long)r2);
  int64_t P = 1;
  for (int n = 2; n < N; ++n) {
    if (ranks[n] > max_planes / P)
      return fail(MES_ERR_INVALID_ARG, "%s: more than %lld planes (prod of ranks[2..])", who,
                  (long long)max_planes);
    P *= ranks[n];
  }
  *plane_size = r1 * r2;
  *planes = P;
  return MES_OK;
}

// Launches both passes; maxbits must hold `planes` words and is cleared here.
mes_status quantize_launch(const float* core, int64_t plane_size, int64_t planes, int bits,
                           int16_t* q, float* scales, unsigned* maxbits, cudaStream_t st) {
  MES_CUDA_TRY(cudaMemsetAsync(maxbits, 0, planes * sizeof(unsigned), st));
  const int64_t chunk = 8192;
  dim3 g1((unsigned)((plane_size + chunk - 1) / chunk), (unsigned)planes);
  {
  ProfScope prof("quant_absmax", st, 0.0, 4.0 * plane_size * planes);
  plane_absmax_kernel<<<g1, kThreads, 0, st>>>(core, plane_size, chunk, maxbits);
  MES_LAUNCH_CHECK();
  }
  const int64_t total = plane_size * planes;
  const float qmax = (float)((1 << (bits - 1)) - 1);
  // enough chunks per plane to give every SM a few blocks
  int64_t qchunk = (total + (int64_t)sm_count() * 8 - 1) / ((int64_t)sm_count() * 8);
  qchunk = ((qchunk + kThreads - 1) / kThreads) * kThreads;
  if (qchunk < kThreads) qchunk = kThreads;
  if (qchunk > plane_size) qchunk = ((plane_size + kThreads - 1) / kThreads) * kThreads;
  dim3 g2((unsigned)((plane_size + qchunk - 1) / qchunk), (unsigned)planes);
  ProfScope prof("quantize", st, 0.0, 6.0 * total + 4.0 * planes);
  quantize_kernel<<<g2, kThreads, 0, st>>>(core, plane_size, qchunk, maxbits, qmax, q, scales);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

}  // namespace mes

extern "C" mes_status mes_quantize_core(const float* core, int N, const int64_t* ranks, int bits,
                                        int16_t* q, float* scales, int status_host_sync,
                                        void* stream) {
  mes::clear_error();
  if (!core || !q || !scales) return mes::fail(MES_ERR_INVALID_ARG, "mes_quantize_core: null pointer");
  if (bits < 2 || bits > 16) return mes::fail(MES_ERR_INVALID_ARG, "mes_quantize_core: bits must be 2..16");
  int64_t plane_size = 0, planes = 0;
  MES_TRY(mes::quant_plane_shape(N, ranks, 65535, &plane_size, &planes, "mes_quantize_core"));   // grid.y limit
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mes::Trace trace("mes_quantize_core", st);
  trace.phase("quantize");
  mes::Scratch scratch(st);
  unsigned* maxbits = nullptr;
  MES_TRY(scratch.alloc(&maxbits, (size_t)planes));
  MES_TRY(mes::quantize_launch(core, plane_size, planes, bits, q, scales, maxbits, st));
  if (status_host_sync) {
    unsigned* host = new unsigned[planes];
    cudaError_t e = cudaMemcpyAsync(host, maxbits, planes * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      delete[] host;
      cudaGetLastError();
      return mes::fail(MES_ERR_CUDA, "mes_quantize_core: status read failed: %s", cudaGetErrorString(e));
    }
    bool finite = true;
    for (int64_t p = 0; p < planes; ++p) finite = finite && (host[p] < 0x7f800000u);
    delete[] host;
    if (!finite) return mes::fail(MES_ERR_NONFINITE, "mes_quantize_core: a core plane holds NaN or Inf");
  }
  return MES_OK;
}

extern "C" mes_status mes_dequantize_core(const int16_t* q, const float* scales, int N,
                                          const int64_t* ranks, float* core, void* stream) {
  mes::clear_error();
  if (!core || !q || !scales) return mes::fail(MES_ERR_INVALID_ARG, "mes_dequantize_core: null pointer");
  int64_t plane_size = 0, planes = 0;
  MES_TRY(mes::quant_plane_shape(N, ranks, 65535, &plane_size, &planes, "mes_dequantize_core"));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t total = plane_size * planes;
  mes::ProfScope prof("dequantize", st, 0.0, 6.0 * total);
  dequantize_kernel<<<mes::grid_for(total, kThreads, (int64_t)mes::sm_count() * 16), kThreads, 0, st>>>(
      q, scales, plane_size, total, core);
  MES_LAUNCH_CHECK();
  return MES_OK;
}

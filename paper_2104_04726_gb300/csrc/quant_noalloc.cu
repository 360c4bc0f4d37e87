// Core quantiser for callers that cannot allocate device memory.
//
// mes_quantize_core takes its per-plane scratch words from the stream-ordered
// allocator.  Some callers cannot allow that: a pipeline that must not touch
// the allocator once it is running (fixed memory budget, no allocator calls
// on the hot path), or a host program that hands the library only the buffers
// it owns.  This entry point runs the same two kernels with the scratch held
// in a fixed array in device global memory that is part of the library
// image.  That array is allocated once, when the library's module is loaded
// on a device, and stays resident on every device that loads the library
// until the process exits.
//
// The host never dereferences the array: its name in host code is only a
// handle, so the device address is looked up with cudaGetSymbolAddress, once
// per device, with that device current, and cached.
#include <mutex>

#include "small.cuh"

#define MES_NOALLOC_MAX_PLANES 4096   // 16 KiB of scratch per device

// Per-plane maxima of |x| (IEEE bit patterns) for the quantiser; shared by
// every call of the entry point below on a device.
static __device__ __align__(256) unsigned g_plane_max[MES_NOALLOC_MAX_PLANES];

namespace {

constexpr int64_t kMaxPlanes = MES_NOALLOC_MAX_PLANES;

std::mutex g_mu;
unsigned* g_addr[128] = {nullptr};

mes_status scratch_address(unsigned** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return mes::fail(MES_ERR_CUDA, "mes_quantize_core_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  }
  if (dev < 0 || dev >= 128) return mes::fail(MES_ERR_CUDA, "mes_quantize_core_noalloc: device index %d", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_plane_max);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return mes::fail(MES_ERR_CUDA, "mes_quantize_core_noalloc: cudaGetSymbolAddress: %s",
                       cudaGetErrorString(e));
    }
    g_addr[dev] = static_cast<unsigned*>(p);
  }
  *out = g_addr[dev];
  return MES_OK;
}

}  // namespace

extern "C" mes_status mes_quantize_core_noalloc(const float* core, int N, const int64_t* ranks, int bits,
                                                int16_t* q, float* scales, void* stream) {
  mes::clear_error();
  if (!core || !q || !scales || !ranks)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_quantize_core_noalloc: null pointer");
  if (bits < 2 || bits > 16)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_quantize_core_noalloc: bits must be 2..16");
  if (N < 1 || N > 8) return mes::fail(MES_ERR_INVALID_ARG, "mes_quantize_core_noalloc: N must be 1..8");
  for (int n = 0; n < N; ++n)
    if (ranks[n] < 1) return mes::fail(MES_ERR_INVALID_ARG, "mes_quantize_core_noalloc: ranks must be >= 1");
  const int64_t plane_size = ranks[0] * (N >= 2 ? ranks[1] : 1);
  int64_t planes = 1;
  for (int n = 2; n < N; ++n) planes *= ranks[n];
  if (planes > kMaxPlanes)
    return mes::fail(MES_ERR_INVALID_ARG,
                     "mes_quantize_core_noalloc: %lld planes exceed the fixed scratch of %lld planes; "
                     "use mes_quantize_core", (long long)planes, (long long)kMaxPlanes);
  unsigned* maxbits = nullptr;
  MES_TRY(scratch_address(&maxbits));
  // quantize_launch clears the `planes` words it uses before the two passes
  return mes::quantize_launch(core, plane_size, planes, bits, q, scales, maxbits,
                              static_cast<cudaStream_t>(stream));
}

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
// per device, with that device current, and cached.  The cache assumes the
// library's module stays loaded: after cudaDeviceReset on a device the cached
// address is stale, so a process that resets a device must not call this
// entry point on it again.
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
  int64_t plane_size = 0, planes = 0;
  // rejects more than kMaxPlanes planes, checking each rank before it is
  // multiplied in (a wrapped product must not pass the limit)
  MES_TRY(mes::quant_plane_shape(N, ranks, kMaxPlanes, &plane_size, &planes, "mes_quantize_core_noalloc"));
  unsigned* maxbits = nullptr;
  MES_TRY(scratch_address(&maxbits));
  // quantize_launch clears the `planes` words it uses before the two passes
  return mes::quantize_launch(core, plane_size, planes, bits, q, scales, maxbits,
                              static_cast<cudaStream_t>(stream));
}

// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "mes.h"

namespace mes {

// Round to the nearest TF32 value (10 explicit mantissa bits), ties to even.
// The tcgen05 kind::tf32 product reads FP32 operands and ignores their 13 low
// mantissa bits, i.e. truncates; operands stored pre-rounded with this
// function make its input rounding unbiased.  Inf and NaN pass unchanged.
__host__ __device__ __forceinline__ float round_tf32(float x) {
#ifdef __CUDA_ARCH__
  unsigned u = __float_as_uint(x);
#else
  unsigned u;
  memcpy(&u, &x, 4);
#endif
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
  }
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float y;
  memcpy(&y, &u, 4);
  return y;
#endif
}

// Round to the nearest BF16 value (7 explicit mantissa bits), ties to even,
// returned as its 16-bit pattern.  Inf and NaN keep their class.
__host__ __device__ __forceinline__ uint16_t bf16_bits(float x) {
#ifdef __CUDA_ARCH__
  unsigned u = __float_as_uint(x);
#else
  unsigned u;
  memcpy(&u, &x, 4);
#endif
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// Key of the rank-by-count sorts (eigenvalues, Gram diagonals): NaN maps
// below every number, so "greater, or equal with a lower index" stays a
// strict total order and the ranks form a permutation even when a failed
// step upstream has left NaN in the data.
__host__ __device__ __forceinline__ float order_key(float w) { return w == w ? w : -INFINITY; }
__host__ __device__ __forceinline__ double order_key(double w) { return w == w ? w : -(double)INFINITY; }

// Records a formatted message in the thread-local error buffer and returns s.
mes_status fail(mes_status s, const char* fmt, ...);
void clear_error();

// Host-side fault injection (environment variable MES_FAULT, read at each
// use): fault_alloc(k) is true when allocation k of the current ABI call must
// fail ("alloc:<k>"); fault_admit() when the serving loop must refuse
// admissions ("admit").
bool fault_alloc(int index);
bool fault_admit();

// Number of SMs of the current device (cached per device).
int sm_count();

// Host-side bounds audit.  Buffers of known extent (scratch allocations and
// the caller's arrays whose sizes follow from the call's arguments) are
// registered for the duration of an ABI call; every launch descriptor is
// checked against them before the launch, so an addressing mistake returns
// an error instead of touching memory out of range.
void audit_register(const void* p, size_t bytes);
void audit_clear();
// Returns MES_OK when [p, p + last_byte] lies inside the registered buffer
// that contains p (or when p is not in any registered buffer).
mes_status audit(const void* p, size_t last_byte, const char* what);

// Per-kernel-family profiler (off by default).  When on, every launch is
// bracketed by CUDA events recorded on its own stream, and the algorithmic
// flops and bytes of the launch are accumulated per family.  Not usable
// inside stream capture.
bool prof_on();
void prof_begin(cudaStream_t st);
void prof_end(const char* family, cudaStream_t st, double flops, double bytes);

struct ProfScope {
  const char* fam;
  cudaStream_t st;
  double flops, bytes;
  ProfScope(const char* f, cudaStream_t s, double fl, double by) : fam(f), st(s), flops(fl), bytes(by) {
    if (prof_on()) prof_begin(st);
  }
  ~ProfScope() {
    if (prof_on()) prof_end(fam, st, flops, bytes);
  }
};

// Phase tracing of one ABI call.  Every phase is an NVTX range (free when no
// tool is attached; ncu can filter kernels by it).  With MES_TRACE=<file> the
// phases are also timed with CUDA events on the call's stream, and the call
// appends one JSON line {"call", "phases": [[name, ms], ...], "total_ms"} to
// <file> when it returns, so a traced call waits for its stream.  A call made
// under stream capture is not timed (its NVTX ranges remain).
class Trace {
 public:
  Trace(const char* call, cudaStream_t st);   // call == nullptr: inactive
  ~Trace();
  // ends the open phase and opens `name` (with `index` >= 0 appended)
  void phase(const char* name, int index = -1);
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;

 private:
  struct Mark;
  const char* call_;
  char path_[512] = "";
  cudaStream_t st_;
  bool timed_ = false, open_ = false;
  Mark* marks_ = nullptr;
  int n_ = 0, cap_ = 0;
};

struct AuditScope {
  AuditScope() { audit_clear(); }
  ~AuditScope() { audit_clear(); }
};

// Stream-ordered scratch allocation; every allocation of one ABI call is
// released on the same stream before the call returns.
struct Scratch {
  cudaStream_t stream;
  void* ptrs[64];
  int n = 0;
  // dry: nothing is allocated; `total` sums the bytes a real run would take
  // (each request rounded up to 256 bytes) and the returned pointers are
  // placeholders that must not be used
  bool dry = false;
  size_t total = 0;
  explicit Scratch(cudaStream_t s, bool dry_run = false) : stream(s), dry(dry_run) {}
  ~Scratch() {
    for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], stream);
  }
  template <class T>
  mes_status alloc(T** out, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    const size_t rounded = (bytes + 255) & ~size_t(255);
    total += rounded;
    if (dry) {
      *out = reinterpret_cast<T*>(uintptr_t(256));
      return MES_OK;
    }
    if (n >= 64) return fail(MES_ERR_OOM, "scratch table full");
    if (fault_alloc(n)) return fail(MES_ERR_OOM, "allocation %d refused (fault injected by MES_FAULT)", n);
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, rounded, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MES_ERR_OOM, "cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    ptrs[n++] = p;
    audit_register(p, bytes);
    *out = static_cast<T*>(p);
    return MES_OK;
  }
};

inline unsigned grid_for(int64_t work, int threads, int64_t cap) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return static_cast<unsigned>(b);
}

}  // namespace mes

#define MES_TRY(expr)                      \
  do {                                     \
    mes_status s_ = (expr);                \
    if (s_ != MES_OK) return s_;           \
  } while (0)

#define MES_CUDA_TRY(expr)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cudaGetLastError();                                                                   \
      return mes::fail(MES_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),      \
                       __FILE__, __LINE__);                                                 \
    }                                                                                       \
  } while (0)

#define MES_LAUNCH_CHECK() MES_CUDA_TRY(cudaGetLastError())

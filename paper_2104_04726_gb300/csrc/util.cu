// Error buffer, device queries and the version string.
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace mes {

static thread_local char g_err[1024] = "";

mes_status fail(mes_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

void clear_error() { g_err[0] = 0; }

// Host-side fault injection for tests of the failure paths: MES_FAULT is a
// comma-separated list of "alloc:<k>" (allocation number k of each ABI call
// fails as if the device were out of memory) and "admit" (the serving loop
// refuses every admission).  Nothing here touches the GPU.
static bool fault_item(const char* name, long* arg) {
  const char* e = getenv("MES_FAULT");
  if (!e || !*e) return false;
  const size_t n = strlen(name);
  for (const char* p = e; p && *p;) {
    if (strncmp(p, name, n) == 0 && (p[n] == 0 || p[n] == ',' || p[n] == ':')) {
      if (arg) *arg = (p[n] == ':') ? strtol(p + n + 1, nullptr, 10) : 0;
      return true;
    }
    p = strchr(p, ',');
    if (p) ++p;
  }
  return false;
}

bool fault_alloc(int index) {
  long k = 0;
  return fault_item("alloc", &k) && k == index;
}

bool fault_admit() { return fault_item("admit", nullptr); }

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 148;
    }
    cached[dev] = n;
  }
  return cached[dev];
}

struct Region {
  uintptr_t lo, hi;
};
static thread_local Region g_regions[128];
static thread_local int g_nregions = 0;

void audit_register(const void* p, size_t bytes) {
  if (!p || g_nregions >= 128) return;
  g_regions[g_nregions++] = Region{(uintptr_t)p, (uintptr_t)p + bytes};
}

void audit_clear() { g_nregions = 0; }

mes_status audit(const void* p, size_t last_byte, const char* what) {
  if (!p) return MES_OK;
  const uintptr_t a = (uintptr_t)p;
  for (int i = 0; i < g_nregions; ++i) {
    if (a >= g_regions[i].lo && a < g_regions[i].hi) {
      if (a + last_byte >= g_regions[i].hi)
        return fail(MES_ERR_INVALID_ARG, "bounds audit: %s reaches byte %zu of a %zu-byte buffer", what,
                    (size_t)(a - g_regions[i].lo) + last_byte, (size_t)(g_regions[i].hi - g_regions[i].lo));
      return MES_OK;
    }
  }
  return MES_OK;
}

// ---- profiler ----
struct ProfRec {
  int fam;
  cudaEvent_t a, b;
  double flops, bytes;
};
static bool g_prof = false;
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;
static size_t g_pool_used = 0;
static std::vector<std::string> g_fams;
static cudaEvent_t g_pending = nullptr;

static cudaEvent_t pool_event() {
  if (g_pool_used == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_pool.push_back(e);
  }
  return g_pool[g_pool_used++];
}

bool prof_on() { return g_prof; }

void prof_begin(cudaStream_t st) {
  g_pending = pool_event();
  if (g_pending) cudaEventRecord(g_pending, st);
}

void prof_end(const char* family, cudaStream_t st, double flops, double bytes) {
  cudaEvent_t b = pool_event();
  if (!g_pending || !b) return;
  cudaEventRecord(b, st);
  int fam = -1;
  for (size_t i = 0; i < g_fams.size(); ++i)
    if (g_fams[i] == family) fam = (int)i;
  if (fam < 0) {
    g_fams.push_back(family);
    fam = (int)g_fams.size() - 1;
  }
  g_recs.push_back(ProfRec{fam, g_pending, b, flops, bytes});
  g_pending = nullptr;
}

// ---- phase tracing ----
struct Trace::Mark {
  char name[40];
  cudaEvent_t ev;
};

Trace::Trace(const char* call, cudaStream_t st) : call_(call), st_(st) {
  if (!call) return;   // inactive (e.g. a workspace-size query)
  nvtxRangePushA(call);
  const char* path = getenv("MES_TRACE");
  if (!path || !*path) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  if (snprintf(path_, sizeof(path_), "%s", path) >= (int)sizeof(path_)) return;
  timed_ = true;
  phase("setup");
}

void Trace::phase(const char* name, int index) {
  if (!call_) return;
  if (open_) nvtxRangePop();
  char label[40];
  if (index >= 0)
    snprintf(label, sizeof(label), "%s %d", name, index);
  else
    snprintf(label, sizeof(label), "%s", name);
  nvtxRangePushA(label);
  open_ = true;
  if (!timed_) return;
  if (n_ == cap_) {
    const int cap = cap_ ? 2 * cap_ : 32;
    Mark* m = new Mark[cap];
    for (int i = 0; i < n_; ++i) m[i] = marks_[i];
    delete[] marks_;
    marks_ = m;
    cap_ = cap;
  }
  Mark& mk = marks_[n_];
  snprintf(mk.name, sizeof(mk.name), "%s", label);
  if (cudaEventCreate(&mk.ev) != cudaSuccess || cudaEventRecord(mk.ev, st_) != cudaSuccess) {
    cudaGetLastError();
    timed_ = false;   // tracing gives up quietly; the call itself goes on
    return;
  }
  ++n_;
}

Trace::~Trace() {
  if (!call_) return;
  if (open_) nvtxRangePop();
  nvtxRangePop();
  if (!marks_) return;
  cudaEvent_t end = nullptr;
  bool ok = timed_ && n_ > 0 && cudaEventCreate(&end) == cudaSuccess && cudaEventRecord(end, st_) == cudaSuccess &&
            cudaEventSynchronize(end) == cudaSuccess;
  std::string line = std::string("{\"call\": \"") + call_ + "\", \"phases\": [";
  float total = 0.f;
  for (int i = 0; ok && i < n_; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, marks_[i].ev, i + 1 < n_ ? marks_[i + 1].ev : end) != cudaSuccess) {
      ok = false;
      break;
    }
    total += ms;
    char buf[96];
    snprintf(buf, sizeof(buf), "%s[\"%s\", %.4f]", i ? ", " : "", marks_[i].name, ms);
    line += buf;
  }
  if (ok) {
    char buf[64];
    snprintf(buf, sizeof(buf), "], \"total_ms\": %.4f}\n", total);
    line += buf;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (FILE* f = fopen(path_, "a")) {
      fputs(line.c_str(), f);
      fclose(f);
    }
  }
  cudaGetLastError();
  for (int i = 0; i < n_; ++i) cudaEventDestroy(marks_[i].ev);
  if (end) cudaEventDestroy(end);
  delete[] marks_;
}

}  // namespace mes

extern "C" void mes_profile_enable(int on) {
  mes::g_prof = on != 0;
  if (on) {
    mes::g_recs.clear();
    mes::g_fams.clear();
    mes::g_pool_used = 0;
  }
}

extern "C" int mes_profile_count(void) { return (int)mes::g_fams.size(); }

extern "C" mes_status mes_profile_get(int i, char* name, int name_len, int64_t* launches, double* ms,
                                      double* flops, double* bytes) {
  if (i < 0 || i >= (int)mes::g_fams.size() || !name || name_len < 2)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_profile_get: bad index or buffer");
  snprintf(name, (size_t)name_len, "%s", mes::g_fams[i].c_str());
  int64_t n = 0;
  double t = 0.0, f = 0.0, b = 0.0;
  for (const auto& r : mes::g_recs) {
    if (r.fam != i) continue;
    float e = 0.f;
    cudaError_t err = cudaEventSynchronize(r.b);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&e, r.a, r.b);
    if (err != cudaSuccess) {
      cudaGetLastError();
      return mes::fail(MES_ERR_CUDA, "mes_profile_get: %s", cudaGetErrorString(err));
    }
    ++n;
    t += e;
    f += r.flops;
    b += r.bytes;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (flops) *flops = f;
  if (bytes) *bytes = b;
  return MES_OK;
}

extern "C" const char* mes_last_error(void) { return mes::g_err; }

extern "C" const char* mes_version(void) { return "mes 0.1.0 sm_103a"; }

// trace.cu -- optional per-phase timing of the library's launches.
//
// When enabled (bkfac_trace_enable), every phase of an update / apply /
// reorth records a pair of CUDA events on the stream it is launched on; a
// read synchronises on them and accumulates the elapsed time per phase.
// A kernel-launch counter is always maintained.  Host-side state only; not
// used while a stream is being captured into a graph.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace bkfac {

int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    v = 148;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}
namespace {

struct Rec {
  int ph;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
std::vector<Rec> g_pending;
double g_ms[PH_COUNT];
int64_t g_cnt[PH_COUNT];
std::atomic<int64_t> g_launches{0};

const char* kNames[PH_COUNT] = {"colnorm", "proj",   "resid",       "gram",     "chol",        "trinv",
                                "trmm",    "core",   "jacobi",      "sort",     "rotate",      "finalize",
                                "dense",   "coefs",  "apply_pass1", "apply_small", "apply_pass2", "reorth",
                                "factored_thin", "factored_step", "precond"};

cudaEvent_t take() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &st);
  return st != cudaStreamCaptureStatusNone;
}

}  // namespace

TraceScope::TraceScope(int ph, cudaStream_t s) : ph_(ph), s_(s), a_(nullptr) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || capturing(s)) return;
  a_ = take();
  cudaEventRecord((cudaEvent_t)a_, s);
}

TraceScope::~TraceScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take();
  cudaEventRecord(b, s_);
  g_pending.push_back({ph_, (cudaEvent_t)a_, b});
}

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int64_t launch_count() { return g_launches.load(); }

}  // namespace bkfac

using namespace bkfac;

extern "C" {

int bkfac_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_pending) {
    cudaEventSynchronize(r.b);
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_pending.clear();
  for (int i = 0; i < PH_COUNT; ++i) {
    g_ms[i] = 0.0;
    g_cnt[i] = 0;
  }
  g_on = on != 0;
  return BKFAC_OK;
}

int bkfac_trace_read(double* ms_out, int64_t* count_out, int nmax, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = BKFAC_OK;
  for (auto& r : g_pending) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) rc = BKFAC_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_ms[r.ph] += ms;
      g_cnt[r.ph] += 1;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_pending.clear();
  for (int i = 0; i < PH_COUNT && i < nmax; ++i) {
    if (ms_out) ms_out[i] = g_ms[i];
    if (count_out) count_out[i] = g_cnt[i];
  }
  if (launches) *launches = g_launches.load();
  return rc == BKFAC_OK ? PH_COUNT : -rc;
}

const char* bkfac_trace_phase_name(int id) { return (id >= 0 && id < PH_COUNT) ? kNames[id] : "?"; }

}  // extern "C"

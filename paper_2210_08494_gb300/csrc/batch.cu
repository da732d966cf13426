// batch.cu -- bkfac_batch_*: all factors of all FC layers of a network.
//
// A batch owns, allocated once at creation: one device workspace carved into
// per-factor update workspaces and per-layer apply workspaces, one worker
// stream per factor, the fork/join events, and (after a capture) a CUDA graph
// of one full step.  A batched update forks every factor's update onto its
// worker stream from the caller's stream and joins them back, so the factors'
// kernels run concurrently; the apply does the same per layer.  Captured once,
// the whole step (every update, then every apply) replays as a single graph
// launch.
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

struct bkfac_batch {
  int nl = 0, n = 0, dtype = 0;
  std::vector<bkfac_factor> f;  // 2 * nl: layer l -> A at 2l, G at 2l + 1
  void* ws = nullptr;
  std::vector<size_t> ws_off, ws_len;        // per factor (update)
  std::vector<size_t> aws_off, aws_len;      // per layer (apply)
  std::vector<size_t> rws_off, rws_len;      // per factor (reorth)
  std::vector<cudaStream_t> streams;         // per factor
  std::vector<cudaEvent_t> done;             // per factor
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;  // kernels one replay of the graph launches
  int device = -1;
};

namespace {

void destroy(bkfac_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->done)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ws) cudaFree(b->ws);
  delete b;
}

int fork_from(bkfac_batch* b, cudaStream_t s, int count) {
  if (cudaEventRecord(b->fork, s) != cudaSuccess) return BKFAC_ECUDA;
  for (int i = 0; i < count; ++i)
    if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) return BKFAC_ECUDA;
  return BKFAC_OK;
}

int join_into(bkfac_batch* b, cudaStream_t s, int count) {
  for (int i = 0; i < count; ++i) {
    if (cudaEventRecord(b->done[i], b->streams[i]) != cudaSuccess) return BKFAC_ECUDA;
    if (cudaStreamWaitEvent(s, b->done[i], 0) != cudaSuccess) return BKFAC_ECUDA;
  }
  return BKFAC_OK;
}

// one-CTA-per-SM clusters of 16 that fit on the GPU at once
constexpr int kClustersAtOnce = 152 / 16;

int batch_update(bkfac_batch* b, const void* const* X_A, const int64_t* ldxA, const void* const* X_G,
                 const int64_t* ldxG, double rho, cudaStream_t s) {
  const int nf = 2 * b->nl;
  int rc = fork_from(b, s, nf);
  int first_err = BKFAC_OK;
  if (rc) return rc;
  bkfac::jacobi_set_many_concurrent(nf > kClustersAtOnce);
  for (int i = 0; i < nf; ++i) {
    const int l = i / 2;
    const void* X = (i & 1) ? X_G[l] : X_A[l];
    const int64_t ld = (i & 1) ? ldxG[l] : ldxA[l];
    void* ws = (char*)b->ws + b->ws_off[i];
    bkfac_factor* f = &b->f[i];
    rc = f->r_cur == 0 ? bkfac_init(f, X, ld, b->n, ws, b->ws_len[i], (bkfac_stream_t)b->streams[i])
                       : bkfac_update(f, X, ld, b->n, rho, ws, b->ws_len[i], (bkfac_stream_t)b->streams[i]);
    if (rc && !first_err) first_err = rc;
  }
  bkfac::jacobi_set_many_concurrent(false);
  rc = join_into(b, s, nf);  // always join, so the caller's stream waits for whatever was enqueued
  return first_err ? first_err : rc;
}

int batch_apply(bkfac_batch* b, const void* const* G, const int64_t* ldg, void* const* S, const int64_t* lds,
                const double* lamA, const double* lamG, uint32_t flags, cudaStream_t s) {
  int rc = fork_from(b, s, b->nl);
  int first_err = BKFAC_OK;
  if (rc) return rc;
  for (int l = 0; l < b->nl; ++l) {
    void* ws = (char*)b->ws + b->aws_off[l];
    rc = bkfac_apply(&b->f[2 * l], &b->f[2 * l + 1], lamA[l], lamG[l], G[l], ldg[l], S[l], lds[l], flags, ws,
                     b->aws_len[l], (bkfac_stream_t)b->streams[l]);
    if (rc && !first_err) first_err = rc;
  }
  rc = join_into(b, s, b->nl);
  return first_err ? first_err : rc;
}

}  // namespace

using bkfac::launch_count;
using bkfac::note_launches;

extern "C" {

bkfac_batch* bkfac_batch_create(const bkfac_layer_desc* layers, int nlayers, int n, int dtype,
                                const char* tune_cache) {
  if (!layers || nlayers < 1 || nlayers > 1024 || n < 1) return nullptr;
  bkfac_batch* b = new (std::nothrow) bkfac_batch();
  if (!b) return nullptr;
  b->nl = nlayers;
  b->n = n;
  b->dtype = dtype;
  cudaGetDevice(&b->device);
  size_t total = 0;
  auto carve = [&](size_t bytes) {
    const size_t off = total;
    total += (bytes + 255) / 256 * 256;
    return off;
  };
  for (int l = 0; l < nlayers; ++l) {
    for (int w = 0; w < 2; ++w) {
      bkfac_factor f = w ? layers[l].G : layers[l].A;
      if (f.dtype != dtype) {
        destroy(b);
        return nullptr;
      }
      const size_t sz = bkfac_workspace_size(&f, n, BKFAC_OP_UPDATE);
      if (sz == 0) {
        destroy(b);
        return nullptr;
      }
      b->f.push_back(f);
      b->ws_off.push_back(carve(sz));
      b->ws_len.push_back(sz);
    }
  }
  for (int i = 0; i < 2 * nlayers; ++i) {
    const size_t sz = bkfac_workspace_size(&b->f[i], n, BKFAC_OP_REORTH);
    if (sz == 0) {
      destroy(b);
      return nullptr;
    }
    b->rws_off.push_back(carve(sz));
    b->rws_len.push_back(sz);
  }
  for (int l = 0; l < nlayers; ++l) {
    const size_t sz = bkfac_apply_workspace_size(&b->f[2 * l], &b->f[2 * l + 1]);
    if (sz == 0) {
      destroy(b);
      return nullptr;
    }
    b->aws_off.push_back(carve(sz));
    b->aws_len.push_back(sz);
  }
  if (cudaMalloc(&b->ws, total) != cudaSuccess) {
    b->ws = nullptr;
    destroy(b);
    return nullptr;
  }
  const int nf = 2 * nlayers;
  b->streams.assign(nf, nullptr);
  b->done.assign(nf, nullptr);
  for (int i = 0; i < nf; ++i) {
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) != cudaSuccess) {
      destroy(b);
      return nullptr;
    }
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    destroy(b);
    return nullptr;
  }
  // autotune the eigensolve shapes of this batch once (cached in tune_cache when given)
  if (tune_cache) {
    for (const auto& f : b->f) bkfac_tune(&f, n, tune_cache);
  }
  return b;
}

int bkfac_batch_get_factor(const bkfac_batch* b, int layer, int which, bkfac_factor* out) {
  if (!b || !out || layer < 0 || layer >= b->nl || (which != 0 && which != 1)) return BKFAC_EINVAL;
  *out = b->f[2 * layer + which];
  return BKFAC_OK;
}

int bkfac_batch_update(bkfac_batch* b, const void* const* X_A, const int64_t* ldxA, const void* const* X_G,
                       const int64_t* ldxG, double rho, bkfac_stream_t stream) {
  if (!b || !X_A || !X_G || !ldxA || !ldxG) return BKFAC_EINVAL;
  return batch_update(b, X_A, ldxA, X_G, ldxG, rho, (cudaStream_t)stream);
}

int bkfac_batch_apply(bkfac_batch* b, const void* const* G, const int64_t* ldg, void* const* S,
                      const int64_t* lds, const double* lamA, const double* lamG, uint32_t flags,
                      bkfac_stream_t stream) {
  if (!b || !G || !S || !ldg || !lds || !lamA || !lamG) return BKFAC_EINVAL;
  return batch_apply(b, G, ldg, S, lds, lamA, lamG, flags, (cudaStream_t)stream);
}

int bkfac_batch_step_graph(bkfac_batch* b, const void* const* X_A, const int64_t* ldxA, const void* const* X_G,
                           const int64_t* ldxG, double rho, const void* const* G, const int64_t* ldg,
                           void* const* S, const int64_t* lds, const double* lamA, const double* lamG,
                           uint32_t flags, int capture, bkfac_stream_t stream) {
  if (!b) return BKFAC_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  if (capture) {
    if (!X_A || !X_G || !ldxA || !ldxG || !G || !S || !ldg || !lds || !lamA || !lamG) return BKFAC_EINVAL;
    // the captured launch shapes depend on r_cur: only a steady rank replays identically
    // (r, or min(r + r_extra, r + n, d) for a factor that keeps the rank-(r + n) modes)
    for (const auto& f : b->f)
      if (f.r_cur != std::min(std::min(bkfac::factor_r_total(&f), f.r + b->n), (int)f.d)) return BKFAC_EINVAL;
    if (s == nullptr) return BKFAC_EINVAL;  // the legacy stream cannot be captured
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (b->graph) {
      cudaGraphDestroy(b->graph);
      b->graph = nullptr;
    }
    std::vector<bkfac_factor> saved = b->f;
    const int64_t k0 = launch_count();
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BKFAC_ECUDA;
    int rc = batch_update(b, X_A, ldxA, X_G, ldxG, rho, s);
    if (rc == BKFAC_OK) rc = batch_apply(b, G, ldg, S, lds, lamA, lamG, flags, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    b->f = saved;  // the replays below advance the counters
    b->graph_kernels = launch_count() - k0;
    note_launches((int)-b->graph_kernels);  // captured, not launched
    if (rc != BKFAC_OK || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return rc != BKFAC_OK ? rc : BKFAC_ECUDA;
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      b->exec = nullptr;
      return BKFAC_ECUDA;
    }
  }
  if (!b->exec) return BKFAC_EINVAL;
  if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return BKFAC_ECUDA;
  note_launches((int)b->graph_kernels);
  for (auto& f : b->f) f.step += 1;
  return BKFAC_OK;
}

int bkfac_batch_reorth(bkfac_batch* b, bkfac_stream_t stream) {
  if (!b) return BKFAC_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  const int nf = 2 * b->nl;
  int rc = fork_from(b, s, nf);
  if (rc) return rc;
  int first_err = BKFAC_OK;
  for (int i = 0; i < nf; ++i) {
    rc = bkfac_reorth(&b->f[i], (char*)b->ws + b->rws_off[i], b->rws_len[i], (bkfac_stream_t)b->streams[i]);
    if (rc && !first_err) first_err = rc;
  }
  rc = join_into(b, s, nf);
  return first_err ? first_err : rc;
}

void bkfac_batch_destroy(bkfac_batch* b) { destroy(b); }

}  // extern "C"

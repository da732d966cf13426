// batch.cu -- bkfac_batch_*: all factors of all FC layers of a network.
//
// A batch owns, allocated once at creation: one device workspace carved into
// per-factor update workspaces and per-layer apply workspaces, one worker
// stream per factor, the fork/join events, the launch choice of each group of
// same-shape eigensolves, and (after a capture) a CUDA graph of one full step.
// A batched update runs in three stages: every factor's update up to its
// eigensolve, forked onto the factors' worker streams; the eigensolves, one
// grouped launch per group of factors with the same eigensolve shape (each
// cluster of the launch takes one factor's problem); the rest of every update
// (ordering, rotation, write-back), forked again.  The apply forks per layer.
// Captured once, the whole step (every update, then every apply) replays as a
// single graph launch.
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
  // grouped eigensolves: factors with the same eigensolve shape at the steady rank
  // (rows, columns, precision) share a launch choice, tuned per group size
  std::vector<int> group;                   // per factor: its group
  std::vector<bkfac::JacobiChoice> choice;  // per group
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

// Stage 1 forks every factor's update up to its eigensolve; stage 2 launches the
// eigensolves grouped by launch shape (b, padded rows, cluster size, precision, rows),
// one launch per group (up to kMaxJacobiProblems problems each), the groups forked
// onto worker streams so they run concurrently; stage 3 forks the rest of every
// update.  Every stage joins back into the caller's stream.
int batch_update(bkfac_batch* b, const void* const* X_A, const int64_t* ldxA, const void* const* X_G,
                 const int64_t* ldxG, double rho, cudaStream_t s) {
  const int nf = 2 * b->nl;
  std::vector<bkfac::StagedEig> st(nf);
  std::vector<char> init(nf), ok(nf, 0);
  auto X_of = [&](int i) { return (i & 1) ? X_G[i / 2] : X_A[i / 2]; };
  auto ld_of = [&](int i) { return (i & 1) ? ldxG[i / 2] : ldxA[i / 2]; };
  int first_err = BKFAC_OK;
  int rc = fork_from(b, s, nf);
  if (rc) return rc;
  for (int i = 0; i < nf; ++i) {
    init[i] = b->f[i].r_cur == 0;
    rc = bkfac::update_stage_pre(&b->f[i], X_of(i), ld_of(i), b->n, rho, init[i], (char*)b->ws + b->ws_off[i],
                                 b->ws_len[i], &b->choice[b->group[i]], b->streams[i], &st[i]);
    if (rc && !first_err) first_err = rc;
    ok[i] = rc == BKFAC_OK;
  }
  rc = join_into(b, s, nf);  // always join, so the caller's stream waits for whatever was enqueued
  if (first_err || rc) return first_err ? first_err : rc;
  // stage 2: one launch per launch shape
  struct Launch {
    std::vector<bkfac::JacobiProblem> probs;
    int C;
    bkfac::DType jt;
    double tol;
    int dsm;
  };
  std::vector<Launch> launches;
  for (int i = 0; i < nf; ++i) {
    const bkfac::JacobiProblem& jp = st[i].jp;
    Launch* hit = nullptr;
    for (auto& L : launches) {
      const bkfac::JacobiProblem& q = L.probs[0];
      if (L.C == st[i].C && L.jt == st[i].jt && q.b == jp.b && q.rows_pad == jp.rows_pad && q.rows == jp.rows &&
          (int)L.probs.size() < bkfac::kMaxJacobiProblems) {
        hit = &L;
        break;
      }
    }
    if (!hit) {
      launches.push_back(Launch{{}, st[i].C, st[i].jt, st[i].tol, b->choice[b->group[i]].dsm});
      hit = &launches.back();
    }
    hit->probs.push_back(jp);
  }
  const int ng = std::min((int)launches.size(), nf);
  rc = fork_from(b, s, ng);
  if (rc) return rc;
  for (int g = 0; g < (int)launches.size(); ++g) {
    const Launch& L = launches[g];
    rc = bkfac::launch_jacobi_mode(L.probs.data(), (int)L.probs.size(), L.C, L.jt, L.tol, bkfac::eig_sweep_cap(),
                                   L.dsm != 0, b->streams[g % ng]);
    if (rc && !first_err) first_err = BKFAC_ECUDA;
  }
  rc = join_into(b, s, ng);
  if (first_err || rc) return first_err ? first_err : rc;
  // stage 3: the rest of every update
  rc = fork_from(b, s, nf);
  if (rc) return rc;
  for (int i = 0; i < nf; ++i) {
    rc = bkfac::update_stage_post(&b->f[i], X_of(i), ld_of(i), b->n, rho, init[i], (char*)b->ws + b->ws_off[i],
                                  b->ws_len[i], &b->choice[b->group[i]], b->streams[i]);
    if (rc && !first_err) first_err = rc;
  }
  rc = join_into(b, s, nf);
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
  // eigensolve groups: factors whose eigensolve has the same shape at the steady rank
  // (rows = r + n on the Brand path, d on the dense path; columns r + n; precision)
  struct Key {
    int rows, cols, jt;
  };
  std::vector<Key> keys;
  std::vector<int> counts;
  for (const auto& f : b->f) {
    const int jt = (f.dtype == BKFAC_F64 || (f.flags & BKFAC_FLAG_EIG_FP64)) ? 0 : 1;
    const bool dense = (int64_t)f.r + n >= f.d;
    const Key k{dense ? f.d : f.r + n, f.r + n, jt};
    int g = 0;
    while (g < (int)keys.size() && !(keys[g].rows == k.rows && keys[g].cols == k.cols && keys[g].jt == k.jt)) ++g;
    if (g == (int)keys.size()) {
      keys.push_back(k);
      counts.push_back(0);
    }
    ++counts[g];
    b->group.push_back(g);
  }
  // launch choice per group: tuned for its size when a tune cache is given; otherwise the
  // shape's single-problem plan, with the block exchange over distributed shared memory
  // (one CTA per SM) while every group's clusters fit on the GPU at once, else through L2
  // (two clusters share an SM group)
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || sms <= 0) sms = 1;
  int ctas = 0;
  for (size_t g = 0; g < keys.size(); ++g) {
    int C, bb, rp, cp;
    bkfac::jacobi_plan(keys[g].rows, keys[g].cols, (bkfac::DType)keys[g].jt, &C, &bb, &rp, &cp);
    ctas += C * counts[g];
  }
  // clusters of 16 do not pack every SM (they must sit in one GPU processing cluster)
  const bool all_at_once = ctas <= sms - sms / 16;
  b->choice.assign(keys.size(), bkfac::JacobiChoice{});
  for (size_t g = 0; g < keys.size(); ++g) {
    bkfac::JacobiChoice c;
    if (tune_cache && bkfac::tune_group(keys[g].rows, keys[g].cols, (bkfac::DType)keys[g].jt, counts[g], &c) ==
                          BKFAC_OK) {
      b->choice[g] = c;
      continue;
    }
    int bt = 0, dsm = 1;
    if (bkfac::tune_lookup(keys[g].rows, keys[g].cols, (bkfac::DType)keys[g].jt, &bt, &dsm)) c.b_max = bt;
    c.dsm = all_at_once ? dsm : 0;
    b->choice[g] = c;
  }
  if (tune_cache) bkfac::tune_save(tune_cache);
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

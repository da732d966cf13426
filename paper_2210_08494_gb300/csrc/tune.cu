// tune.cu -- the autotuner: picks, per eigensolve shape, the Jacobi block
// width b (which sets the cluster size C = ceil(cols / 2b)) and the block
// exchange between rounds (through L2 or over distributed shared memory), by
// timing every candidate on a synthetic core of that shape: a Brand-like factor
// L = [[diag(sqrt(rho sigma)), sqrt(c) M], [0, sqrt(c) R]] with a power-law sigma
// and Gaussian M, upper-triangular R.  A second table holds the choice for a
// batch's grouped launch of `count` same-shape eigensolves, timed on `count`
// copies of the synthetic core in one launch: wider blocks on smaller clusters,
// or the L2 exchange (a third of the shared memory, two clusters per SM group),
// let more problems run at once, at a cost per problem.  Results live in
// process-wide tables keyed by (rows, cols, precision[, count]) and can be
// saved to / loaded from a text file ("rows cols prec b dsm ms" per line for a
// single problem, "G rows cols prec count b dsm ms" for a group).  The Jacobi
// tables only change launch shapes; every candidate computes the same
// decomposition.
//
// A third table holds the FP32 SIMT products: per shape (M, N, K0, K1, operand
// and output layouts, D term), the kernel (64 x 64 or 128 x 128 tiles) and the
// number of K splits, timed on synthetic operands of the shapes a workload
// actually launched (recorded between bkfac_gemm_tune_begin and _end).  A choice
// changes only the order in which the K terms are summed ("M M N K0 K1 bits
// kernel splits ms" per line).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <random>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace bkfac {
namespace {

struct TuneEntry {
  int b;
  int dsm;
  float ms;
};
std::mutex g_tmu;
std::map<std::tuple<int, int, int>, TuneEntry> g_table;
std::map<std::tuple<int, int, int, int>, TuneEntry> g_group_table;

// FP32 products: (M, N, K0, K1, layout bits) -> choice
using GemmKey = std::tuple<int, int, int, int, int>;
struct GemmEntry {
  int kernel;
  int splits;
  float ms;
};
std::map<GemmKey, GemmEntry> g_gemm_table;
std::map<GemmKey, int64_t> g_gemm_recorded;  // noted shapes and the least partial room seen
std::atomic<bool> g_gemm_recording{false};

constexpr int kKmajA = 1, kKmajB = 2, kRowC = 4, kHasD = 8;
GemmKey gemm_key(const GemmArgs& g) {
  const int bits = (g.a_kmaj ? kKmajA : 0) | (g.b_kmaj ? kKmajB : 0) | (g.c_rowmaj ? kRowC : 0) |
                   (g.D != nullptr ? kHasD : 0);
  return std::make_tuple(g.M, g.N, g.K0, g.K1, bits);
}

}  // namespace

void gemm_record(bool on) { g_gemm_recording.store(on); }

void gemm_note_shape(const GemmArgs& g, int64_t room) {
  if (!g_gemm_recording.load(std::memory_order_relaxed) || g.sym) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  const GemmKey k = gemm_key(g);
  auto it = g_gemm_recorded.find(k);
  if (it == g_gemm_recorded.end())
    g_gemm_recorded[k] = room;
  else
    it->second = std::min(it->second, room);
}

bool gemm_pick_lookup(const GemmArgs& g, GemmPick* out) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (g_gemm_table.empty()) return false;
  auto it = g_gemm_table.find(gemm_key(g));
  if (it == g_gemm_table.end()) return false;
  out->kernel = it->second.kernel;
  out->splits = it->second.splits;
  return true;
}

bool tune_group_lookup(int rows, int cols, DType jt, int count, JacobiChoice* out) {
  std::lock_guard<std::mutex> lk(g_tmu);
  auto it = g_group_table.find(std::make_tuple(rows, cols, (int)jt, count));
  if (it == g_group_table.end()) return false;
  out->b_max = it->second.b;
  out->dsm = it->second.dsm;
  return true;
}

bool tune_lookup(int rows, int cols, DType jt, int* b, int* dsm) {
  std::lock_guard<std::mutex> lk(g_tmu);
  auto it = g_table.find(std::make_tuple(rows, cols, (int)jt));
  if (it == g_table.end()) return false;
  *b = it->second.b;
  *dsm = it->second.dsm;
  return true;
}

namespace {

void put(int rows, int cols, DType jt, TuneEntry e) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_table[std::make_tuple(rows, cols, (int)jt)] = e;
}

int load_file(const char* path) {
  if (!path) return 0;
  FILE* f = std::fopen(path, "r");
  if (!f) return 0;
  int rows, cols, prec, b, dsm, count, n = 0;
  float ms;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == 'M') {
      int M, N, K0, K1, bits, kern, sp;
      if (std::sscanf(line + 1, "%d %d %d %d %d %d %d %f", &M, &N, &K0, &K1, &bits, &kern, &sp, &ms) == 8 &&
          M > 0 && N > 0 && K0 >= 0 && K1 >= 0 && (kern == GEMM_SMALL || kern == GEMM_LARGE) && sp >= 1 &&
          sp <= 64) {
        std::lock_guard<std::mutex> lk(g_tmu);
        g_gemm_table[std::make_tuple(M, N, K0, K1, bits)] = GemmEntry{kern, sp, ms};
        ++n;
      }
    } else if (line[0] == 'G') {
      if (std::sscanf(line + 1, "%d %d %d %d %d %d %f", &rows, &cols, &prec, &count, &b, &dsm, &ms) == 7 &&
          b >= 2 && b <= 32 && (b % 2) == 0 && (prec == 0 || prec == 1) && count >= 1) {
        std::lock_guard<std::mutex> lk(g_tmu);
        g_group_table[std::make_tuple(rows, cols, prec, count)] = TuneEntry{b, dsm ? 1 : 0, ms};
        ++n;
      }
    } else if (std::sscanf(line, "%d %d %d %d %d %f", &rows, &cols, &prec, &b, &dsm, &ms) == 6) {
      if (b >= 2 && b <= 32 && (b % 2) == 0 && (prec == 0 || prec == 1)) {
        put(rows, cols, (DType)prec, TuneEntry{b, dsm ? 1 : 0, ms});
        ++n;
      }
    }
  }
  std::fclose(f);
  return n;
}

int save_file(const char* path) {
  if (!path) return BKFAC_OK;
  FILE* f = std::fopen(path, "w");
  if (!f) return BKFAC_EINVAL;
  std::lock_guard<std::mutex> lk(g_tmu);
  for (const auto& kv : g_table)
    std::fprintf(f, "%d %d %d %d %d %.4f\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                 kv.second.b, kv.second.dsm, kv.second.ms);
  for (const auto& kv : g_group_table)
    std::fprintf(f, "G %d %d %d %d %d %d %.4f\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), std::get<3>(kv.first), kv.second.b, kv.second.dsm, kv.second.ms);
  for (const auto& kv : g_gemm_table)
    std::fprintf(f, "M %d %d %d %d %d %d %d %.4f\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), kv.second.kernel,
                 kv.second.splits, kv.second.ms);
  std::fclose(f);
  return BKFAC_OK;
}

// time one candidate: copy `count` copies of the synthetic core in, run them as one
// grouped Jacobi launch, return ms (-1 on failure)
float time_candidate(int rows, int cols, DType jt, int b, int dsm, const std::vector<double>& host_core,
                     int count = 1) {
  int C, bb, rp, cp;
  jacobi_plan_with(rows, cols, jt, b, &C, &bb, &rp, &cp);
  if (jacobi_smem_bytes(bb, rp, jt) > 200 * 1024 || count < 1 || count > kMaxJacobiProblems) return -1.f;
  const size_t es = jt == DT_F64 ? 8 : 4;
  void* W = nullptr;
  double* cn = nullptr;
  int* stamp = nullptr;
  int* sw = nullptr;
  float ms = -1.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&W, (size_t)count * rp * cp * es) != cudaSuccess ||
      cudaMalloc(&cn, (size_t)cp * 8) != cudaSuccess || cudaMalloc(&stamp, (size_t)count * cp * 4) != cudaSuccess ||
      cudaMalloc(&sw, (size_t)count * 256) != cudaSuccess)
    goto out;
  {
    // host matrix (rows x cols, column-major) -> padded device layout in the Jacobi type
    std::vector<unsigned char> buf((size_t)rp * cp * es, 0);
    std::vector<double> norms(cp, 0.0);
    for (int j = 0; j < cols; ++j)
      for (int i = 0; i < rows; ++i) {
        const double v = host_core[(size_t)i + (size_t)j * rows];
        if (jt == DT_F64)
          reinterpret_cast<double*>(buf.data())[(size_t)i + (size_t)j * rp] = v;
        else
          reinterpret_cast<float*>(buf.data())[(size_t)i + (size_t)j * rp] = (float)v;
        norms[j] += v * v;
      }
    cudaMemcpy(cn, norms.data(), (size_t)cp * 8, cudaMemcpyHostToDevice);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<JacobiProblem> ps(count);
    for (int q = 0; q < count; ++q) {
      JacobiProblem& p = ps[q];
      p.W = (char*)W + (size_t)q * rp * cp * es;
      p.rows = rows;
      p.cols = cols;
      p.rows_pad = rp;
      p.cols_pad = cp;
      p.b = bb;
      p.colnorm2 = cn;
      p.sweeps_out = sw + 64 * q;
      p.stamp = stamp + (size_t)q * cp;
    }
    const double u = jt == DT_F64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
    const double tol = std::max(4.0 * std::sqrt((double)rows), 32.0) * u;
    float best = -1.f;
    for (int rep = 0; rep < 2; ++rep) {
      for (int q = 0; q < count; ++q)
        cudaMemcpy((char*)W + (size_t)q * rp * cp * es, buf.data(), buf.size(), cudaMemcpyHostToDevice);
      cudaEventRecord(e0, 0);
      const int rc = launch_jacobi_mode(ps.data(), count, C, jt, tol, 40, dsm != 0, 0);
      cudaEventRecord(e1, 0);
      if (rc != 0 || cudaEventSynchronize(e1) != cudaSuccess) goto out;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep == 1) best = t;  // the first run pays one-time costs
    }
    ms = best;
  }
out:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (W) cudaFree(W);
  if (cn) cudaFree(cn);
  if (stamp) cudaFree(stamp);
  if (sw) cudaFree(sw);
  cudaGetLastError();  // a failed candidate must not poison later calls
  return ms;
}

}  // namespace

// synthetic core of an eigensolve shape: power-law diagonal block plus Gaussian
// update columns
static std::vector<double> synthetic_core(int rows, int cols) {
  std::mt19937_64 rng(12345u + (unsigned)rows * 7919u + (unsigned)cols);
  std::normal_distribution<double> nd(0.0, 1.0);
  const int k = cols > rows ? 0 : std::max(0, cols / 2);
  std::vector<double> core((size_t)rows * cols, 0.0);
  const double rho = 0.95, c = 0.05 / std::max(1, cols - k);
  for (int j = 0; j < k && j < rows; ++j) core[(size_t)j + (size_t)j * rows] = std::sqrt(rho * std::pow(j + 1.0, -1.2));
  for (int j = k; j < cols; ++j)
    for (int i = 0; i < rows; ++i) {
      const bool upper_tri = i >= k && (i - k) > (j - k);
      core[(size_t)i + (size_t)j * rows] = upper_tri ? 0.0 : std::sqrt(c) * nd(rng) * std::pow(i + 1.0, -0.6);
    }
  return core;
}

// tune the Jacobi of an N x N Brand core (rows = cols = N) or a dense-path factor
int tune_shape(int rows, int cols, DType jt) {
  int b0, d0;
  if (tune_lookup(rows, cols, jt, &b0, &d0)) return BKFAC_OK;
  const std::vector<double> core = synthetic_core(rows, cols);
  float best = 1e30f;
  TuneEntry pick{16, 0, -1.f};
  for (int b : {8, 16}) {
    for (int dsm : {0, 1}) {
      const float t = time_candidate(rows, cols, jt, b, dsm, core);
      if (t > 0.f && t < best) {
        best = t;
        pick = TuneEntry{b, dsm, t};
      }
    }
  }
  if (pick.ms < 0.f) return BKFAC_ECUDA;
  put(rows, cols, jt, pick);
  return BKFAC_OK;
}

// tune a batch's grouped launch of `count` eigensolves of one shape: block-width
// caps 8, 16 and 32 (cluster sizes down to 8) with either block exchange
int tune_group(int rows, int cols, DType jt, int count, JacobiChoice* out) {
  if (tune_group_lookup(rows, cols, jt, count, out)) return BKFAC_OK;
  count = std::min(std::max(count, 1), kMaxJacobiProblems);
  const std::vector<double> core = synthetic_core(rows, cols);
  float best = 1e30f;
  TuneEntry pick{16, 0, -1.f};
  for (int b : {8, 16, 32}) {
    for (int dsm : {0, 1}) {
      const float t = time_candidate(rows, cols, jt, b, dsm, core, count);
      if (t > 0.f && t < best) {
        best = t;
        pick = TuneEntry{b, dsm, t};
      }
    }
  }
  if (pick.ms < 0.f) return BKFAC_ECUDA;
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_group_table[std::make_tuple(rows, cols, (int)jt, count)] = pick;
  }
  out->b_max = pick.b;
  out->dsm = pick.dsm;
  return BKFAC_OK;
}

namespace {

// time one choice of an FP32 product on the synthetic operands in `g`: the fastest
// of three runs after one warm-up, ms (-1 on failure)
float time_gemm(const GemmArgs& g, GemmPick pick, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  if (!gemm_choice_ok(g, pick)) return -1.f;
  float best = -1.f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, s);
    const int rc = gemm_run_choice(g, pick, s);
    cudaEventRecord(e1, s);
    if (rc != 0 || cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0 && (best < 0.f || t < best)) best = t;
  }
  return best;
}

// synthetic operands of one product shape (zeros: the FP32 units' speed does not
// depend on the values), the candidates timed, the fastest recorded
int tune_gemm_shape(const GemmKey& key, int64_t room_cap, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  const int M = std::get<0>(key), N = std::get<1>(key), K0 = std::get<2>(key), K1 = std::get<3>(key);
  const int bits = std::get<4>(key);
  const int K = K0 + K1;
  GemmArgs g;
  std::memset(&g, 0, sizeof g);
  g.M = M;
  g.N = N;
  g.K0 = K0;
  g.K1 = K1;
  g.a_kmaj = (bits & kKmajA) != 0;
  g.b_kmaj = (bits & kKmajB) != 0;
  g.c_rowmaj = (bits & kRowC) != 0;
  g.alpha = 1.0;
  g.beta = (bits & kHasD) ? 1.0 : 0.0;
  g.splits = 1;
  auto pad = [](int64_t x) { return round_up(std::max<int64_t>(x, 1), 4); };
  // element counts: A segments (a_kmaj: M rows of K; else K rows of M), B alike with N, C / D
  const int64_t lda0 = g.a_kmaj ? pad(K0) : pad(M), lda1 = g.a_kmaj ? pad(K1) : pad(M);
  const int64_t ldb0 = g.b_kmaj ? pad(K0) : pad(N), ldb1 = g.b_kmaj ? pad(K1) : pad(N);
  const int64_t na0 = (g.a_kmaj ? M : std::max(K0, 1)) * lda0, na1 = (g.a_kmaj ? M : std::max(K1, 1)) * lda1;
  const int64_t nb0 = (g.b_kmaj ? N : std::max(K0, 1)) * ldb0, nb1 = (g.b_kmaj ? N : std::max(K1, 1)) * ldb1;
  const int64_t ldc = g.c_rowmaj ? pad(N) : pad(M), nc = (g.c_rowmaj ? M : N) * ldc;
  const int64_t mn = (int64_t)M * N;
  const int64_t room = std::min<int64_t>({room_cap, 32, (int64_t)(256ll << 20) / (mn * 4)});
  const int64_t counts[7] = {na0, K1 > 0 ? na1 : 0, nb0, K1 > 0 ? nb1 : 0, nc, (bits & kHasD) ? nc : 0,
                             room >= 2 ? room * mn : 0};
  size_t off[7], total = 0;
  for (int i = 0; i < 7; ++i) {
    off[i] = total;
    total += (size_t)round_up(counts[i] * 4, 256);
  }
  void* buf = nullptr;
  if (cudaMalloc(&buf, std::max<size_t>(total, 256)) != cudaSuccess) {
    cudaGetLastError();
    return BKFAC_ECUDA;
  }
  cudaMemsetAsync(buf, 0, total, s);
  char* b = (char*)buf;
  g.A0 = b + off[0];
  g.lda0 = lda0;
  g.A1 = K1 > 0 ? b + off[1] : nullptr;
  g.lda1 = lda1;
  g.B0 = b + off[2];
  g.ldb0 = ldb0;
  g.B1 = K1 > 0 ? b + off[3] : nullptr;
  g.ldb1 = ldb1;
  g.C = b + off[4];
  g.ldc = ldc;
  g.D = (bits & kHasD) ? b + off[5] : nullptr;
  g.ldd = ldc;
  g.partial = room >= 2 ? b + off[6] : nullptr;
  g.partial_bytes = room >= 2 ? (size_t)(room * mn * 4) : 0;
  GemmEntry best{0, 1, -1.f};
  for (int kern : {GEMM_SMALL, GEMM_LARGE}) {
    for (int sp : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32}) {
      if (sp > 1 && (sp > room || K / sp < 64)) continue;
      const float t = time_gemm(g, GemmPick{kern, sp}, s, e0, e1);
      if (t > 0.f && (best.ms < 0.f || t < best.ms)) best = GemmEntry{kern, sp, t};
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(buf);
  cudaGetLastError();  // a failed candidate must not poison later calls
  if (best.ms < 0.f) return BKFAC_ECUDA;
  std::lock_guard<std::mutex> lk(g_tmu);
  g_gemm_table[key] = best;
  return BKFAC_OK;
}

}  // namespace

int gemm_tune_recorded() {
  std::vector<std::pair<GemmKey, int64_t>> todo;
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    for (const auto& kv : g_gemm_recorded)
      if (g_gemm_table.find(kv.first) == g_gemm_table.end()) todo.push_back(kv);
    g_gemm_recorded.clear();
  }
  if (todo.empty()) return BKFAC_OK;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return BKFAC_ECUDA;
  }
  int rc = BKFAC_OK;
  for (const auto& kv : todo) {
    const int r = tune_gemm_shape(kv.first, kv.second, s, e0, e1);
    if (r != BKFAC_OK) rc = r;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  return rc;
}

int tune_load(const char* path) { return load_file(path); }
int tune_save(const char* path) { return save_file(path); }

}  // namespace bkfac

using namespace bkfac;

extern "C" int bkfac_tune(const bkfac_factor* f, int n, const char* cache_path) {
  if (!f || n < 1 || f->r < 1 || f->d < 1) return BKFAC_EINVAL;
  tune_load(cache_path);
  const DType jt = (f->dtype == BKFAC_F64 || (f->flags & BKFAC_FLAG_EIG_FP64)) ? DT_F64 : DT_F32;
  const bool dense = (int64_t)f->r + n >= f->d;
  const int rows = dense ? f->d : f->r + n;
  const int cols = f->r + n;
  const int rc = tune_shape(rows, cols, jt);
  if (rc != BKFAC_OK) return rc;
  return tune_save(cache_path);
}

extern "C" int bkfac_gemm_tune_begin(void) {
  gemm_record(true);
  return BKFAC_OK;
}

extern "C" int bkfac_gemm_tune_end(const char* cache_path) {
  gemm_record(false);
  tune_load(cache_path);
  const int rc = gemm_tune_recorded();
  const int rs = tune_save(cache_path);
  return rc != BKFAC_OK ? rc : rs;
}

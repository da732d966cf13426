// common.cuh -- shared definitions of libbkfac (GB300, sm_103a).
#pragma once

#include <atomic>

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bkfac.h"

namespace bkfac {

// modes a factor holds after an update: r, or r + r_extra when it keeps the
// untruncated rank-(r + n) representation until the next update (BKFAC_FLAG_KEEP_RN)
inline int factor_r_total(const bkfac_factor* f) {
  return f->r + ((f->flags & BKFAC_FLAG_KEEP_RN) && f->r_extra > 0 ? f->r_extra : 0);
}

// ---------------------------------------------------------------------------
// Device status word.  Kernels record the first error with atomicCAS and
// never trap; bkfac_status() reads and clears it.
// ---------------------------------------------------------------------------
extern __device__ int g_status;

__device__ __forceinline__ void report(int code) { atomicCAS(&g_status, 0, code); }

// ---------------------------------------------------------------------------
// Precision traits
// ---------------------------------------------------------------------------
template <typename T>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double u = 1.1102230246251565e-16;  // 2^-53
};
template <>
struct Eps<float> {
  static constexpr double u = 5.9604644775390625e-08;  // 2^-24
};

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <typename T>
__device__ __forceinline__ T ld_round(const T* p, bool rnd) {
  return *p;
}
template <>
__device__ __forceinline__ float ld_round<float>(const float* p, bool rnd) {
  float v = *p;
  return rnd ? round_bf16(v) : v;
}

__host__ __device__ __forceinline__ int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
__host__ __device__ __forceinline__ int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

// ---------------------------------------------------------------------------
// Generic SIMT GEMM description (see gemm.cu).
//   C[m, n] = sum_k A(m, k) B(k, n), k over two concatenated segments
//   A(m, k) = a_kmaj ? A[m*lda + k] : A[m + k*lda]
//   B(k, n) = b_kmaj ? B[n*ldb + k] : B[k*ldb + n]
//   epilogue: out = alpha * rs[m] * cs[n] * acc + beta * ds[n] * D(m, n)
//   (rs, cs, ds may be null = 1; beta_dev, when set, replaces beta)
//   C and D: c_rowmaj ? C[m*ldc + n] : C[m + n*ldc]
// ---------------------------------------------------------------------------
struct GemmArgs {
  int M, N, K0, K1;
  const void* A0;
  int64_t lda0;
  const void* A1;
  int64_t lda1;
  const void* B0;
  int64_t ldb0;
  const void* B1;
  int64_t ldb1;
  bool a_kmaj, b_kmaj, c_rowmaj, round_bf16;
  bool tf32x3;     // FP32 operands: products as 3xTF32 on the tensor cores
  bool sym;        // C = A^T A with M == N and B == A: only upper tiles are computed
  void* C;
  int64_t ldc;
  const void* D;
  int64_t ldd;
  double alpha, beta;
  const double* beta_dev;
  const double* rs;
  const double* cs;
  const double* ds;
  int splits;      // split-K count (1 = direct epilogue)
  int k_chunk;     // K elements per split (multiple of the tile depth)
  void* partial;   // splits * M * N accumulators when splits > 1
  size_t partial_bytes;  // size of `partial` (bounds any split count the GEMM picks itself)
};

enum DType { DT_F64 = 0, DT_F32 = 1 };

// Function attributes (shared-memory size, cluster size) are per device: a set of
// per-device bits records where a kernel's attributes were set (devices 0..63).
inline int current_device_bit() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  return dev;
}
inline bool configured_here(const std::atomic<uint64_t>& mask) {
  return (mask.load(std::memory_order_acquire) >> current_device_bit()) & 1u;
}
inline void mark_configured(std::atomic<uint64_t>& mask) {
  mask.fetch_or(uint64_t(1) << current_device_bit(), std::memory_order_release);
}

// streaming multiprocessors of the current device (queried once per device and
// cached; the split-K and grid-size heuristics size their work to it)
int sm_count();

// launchers implemented in gemm.cu; return a cudaError_t
// in_t: element type of A/B; acc_t: accumulator; out_t: C/D element type
// (the number of kernels launched is added to the launch counter)
int gemm_run(const GemmArgs& g, DType in_t, DType acc_t, DType out_t, cudaStream_t s);
// Gram A^T A of FP32 data with compensated FP32 accumulation (FP64-level accuracy),
// output FP64; uses g.A0/lda0 (K-major), g.M = g.N, g.K0, g.C/ldc, g.partial, g.splits
int gram_run_comp(const GemmArgs& g, cudaStream_t s);
// suggested split count for a long-K product with small output
int gemm_pick_splits(int M, int N, int K, int sm_count);
// BF16-operand / FP32-accumulate product on the tensor cores (tc_gemm.cu), same
// contract as gemm_run in mixed mode; split-K partials are summed by
// splitk_reduce_f32 (gemm.cu) in a fixed order
int tc_gemm_run(const GemmArgs& g, cudaStream_t s);
bool tc_gemm_enabled();
int splitk_reduce_f32(const GemmArgs& g, cudaStream_t s);
// TMA-fed tensor-core product of BF16 K-major operands (tma_gemm.cu):
// C (M x N) = alpha sum_k A[m, k] B[n, k] + the epilogue of g (g.M, g.N, g.C, g.ldc,
// g.c_rowmaj, alpha, beta / beta_dev, rs, cs, ds, D, ldd; split K into g.partial);
// A is M x K with row pitch lda, B is N x K with row pitch ldb (elements, multiples
// of 8; 16-byte aligned bases)
bool tma_gemm_available();
int64_t bf16_ld(int k);  // row pitch (elements) of a BF16 K-major copy with k columns
int tma_gemm_run(const void* A, int64_t lda, const void* B, int64_t ldb, int K, const GemmArgs& g, cudaStream_t s);
// FP32 -> BF16 (round to nearest even) copies: G (R x C row-major) and its transpose;
// k columns of length d (same layout); [X0 | X1] (dim x (k0 + k1) column-major) as a
// dim x (k0 + k1) row-major matrix
int launch_cvt_both(const float* G, int64_t ldg, int R, int C, void* Gb, int64_t ldb, void* Gt, int64_t ldt,
                    cudaStream_t s);
int launch_cvt_cols(const float* X, int64_t ld, int d, int k, void* Y, int64_t ldo, cudaStream_t s);
int launch_cvt_cat_t(const float* X0, int64_t ld0, int k0, const float* X1, int64_t ld1, int k1, int dim, void* Y,
                     int64_t ldy, cudaStream_t s);

// ---------------------------------------------------------------------------
// Small dense kernels (small.cu)
// ---------------------------------------------------------------------------
// max_j ||x_j||^2 over the n columns of a d x n column-major matrix -> *out (double)
int launch_colnorm_max(const void* X, int64_t ldx, int d, int n, DType t, double* out, cudaStream_t s);
// thresholded Cholesky of an n x n FP64 Gram (column-major, ld n): upper R (n x n, ld n);
// pivot j dropped (row j of R zero) when s_j <= thr_rel * (*scale).  scale may be null (= 1).
// With neg_rel > 0 a pivot below -neg_rel * (*scale) -- the matrix is indefinite beyond
// its rounding -- also records BKFAC_ECHOL in the status word (the pivot is dropped).
int launch_chol(const double* Gm, int n, double* R, double thr_rel, const double* scale, double neg_rel,
                cudaStream_t s);
// the same factorisation on a thread-block cluster (chol.cu); with near_tol > 0 and
// max|G - I| <= near_tol the factor is I + (strict upper part + half diagonal of G - I);
// near_out (may be null) receives 1 when that shortcut was taken, else 0
int launch_chol_cluster(const double* Gm, int n, double* R, double thr_rel, const double* scale, double near_tol,
                        int* near_out, double neg_rel, cudaStream_t s);
int chol_cluster_size(int n);  // 0 when n is too large for the cluster kernel
// blocked (2D block-cyclic, 16 x 16 blocks) FP64 Cholesky on a 16-CTA cluster with the
// near-identity shortcut of the second CholeskyQR pass (near_tol > 0); for 32 <= n <= 576
bool chol_block_ok(int n);
int launch_chol_block(const double* Gm, int n, double* R, double thr_rel, const double* scale, double near_tol,
                      int* near_out, double neg_rel, cudaStream_t s);
// FP32 Cholesky K = G G^T of an n x n symmetric positive semidefinite matrix (lower
// triangle read, column-major, ld ldk) on a 16-CTA cluster, written as the Jacobi's
// column-major rows_pad x cols_pad matrix G (zero above the diagonal and beyond n)
// with its columns' squared norms; pivot j is dropped (zero column of G) when its
// Schur complement is <= thr_rel * K_jj; for n <= 768 (chol_core_ok)
struct CoreCholArgs {
  const void* K;  // n x n symmetric (lower triangle read), column-major: float (W mode) or double (R mode)
  int64_t ldk;
  int n;
  float thr_rel;        // drop pivot j when its Schur complement <= max(thr_rel K_jj, thr_abs * scale)
  double thr_abs;
  const double* scale;  // may be null (= 1)
  float* W;             // W mode: G, column-major rows_pad x cols_pad
  int rows_pad, cols_pad;
  double* colnorm2;     // W mode: squared column norms (cols_pad)
  double* R;            // R mode: G^T, n x n column-major FP64
  double near_tol;      // R mode: near-identity shortcut when > 0
  int* near_out;        // R mode: 1 when the shortcut was taken (may be null)
};
bool chol_core_ok(int n, int rows_pad, int cols_pad);
int launch_chol_core(const float* K, int ldk, int n, float* W, int rows_pad, int cols_pad, double* colnorm2,
                     float thr_rel, cudaStream_t s);
// the same FP32 factorisation of an FP64 Gram (CholeskyQR of the FP32 and mixed
// paths): R = G^T as n x n column-major FP64, with the near-identity shortcut of
// launch_chol_cluster when near_tol > 0; for n <= 768
bool chol_r32_ok(int n);
int launch_chol_r32(const double* Gm, int n, double* R, float thr_rel, double thr_abs, const double* scale,
                    double near_tol, int* near_out, cudaStream_t s);
// inverse of the upper-triangular R (zero rows = dropped pivots -> zero rows/cols of Rinv);
// when near (may be null) points to a nonzero flag, R = I + F is near identity and
// Rinv = I - F (exact to O(|F|^2)) is written instead
int launch_trinv(const double* R, int n, void* Rinv, DType t, const int* near, cudaStream_t s);

struct CoreArgs {
  int k, n, N;            // old rank, batch width, core size N = k + n
  int rows_pad, cols_pad; // L is rows_pad x cols_pad, column-major, ld = rows_pad
  double rho, c;
  const double* sigma;    // k values
  const void* M;          // k x n, column-major, ld = ldm (type of U)
  int64_t ldm;
  const double* R1;       // n x n upper, ld n
  const double* R2;       // n x n upper, ld n
  void* L;                // output (Jacobi type)
  double* colnorm2;       // cols_pad squared column norms (output)
};
int launch_assemble_core(const CoreArgs& a, DType m_t, DType j_t, cudaStream_t s);

// dense path: F = [U diag(sqrt(rho sigma)), sqrt(c) X] (d x (k+n) into rows_pad x cols_pad)
struct DenseArgs {
  int d, k, n, rows_pad, cols_pad;
  double rho, c;
  const void* U;
  int64_t ldu;
  const double* sigma;
  const void* X;
  int64_t ldx;
  void* F;
  double* colnorm2;
};
int launch_assemble_dense(const DenseArgs& a, DType u_t, DType j_t, cudaStream_t s);

// reorth: L = R diag(sqrt(sigma)) (k x k into rows_pad x cols_pad)
int launch_assemble_reorth(const double* R, const double* sigma, int k, int rows_pad, int cols_pad, void* L,
                           double* colnorm2, DType j_t, cudaStream_t s);

// ---------------------------------------------------------------------------
// Jacobi (jacobi.cu): one-sided block Jacobi on the columns of W (rows x cols_pad,
// column-major, ld = rows_pad), one thread-block cluster per problem.
// ---------------------------------------------------------------------------
struct JacobiProblem {
  void* W;
  int rows, cols, rows_pad, cols_pad, b;   // cols_pad = 2 * C * b >= cols
  const double* colnorm2;            // cols_pad squared column norms of the input
  int* sweeps_out;                   // optional: [0] sweeps, [1 + s] rotations in sweep s (s < 48)
  int* stamp;                        // cols_pad ints of scratch (last sweep a column rotated)
};
constexpr int kMaxJacobiProblems = 64;
struct JacobiBatch {
  JacobiProblem p[kMaxJacobiProblems];
};
// probs: host array of nprob <= kMaxJacobiProblems problems sharing the cluster size C
// (passed by value as a kernel parameter, so the launch can be captured in a graph)
int launch_jacobi(const JacobiProblem* probs, int nprob, int C, DType j_t, double tol, int max_sweeps,
                  cudaStream_t s);
// explicit block-exchange mode (false: through L2, true: distributed shared memory)
int launch_jacobi_mode(const JacobiProblem* probs, int nprob, int C, DType j_t, double tol, int max_sweeps,
                       bool want_dsm, cudaStream_t s);
void jacobi_plan_with(int rows, int cols, DType j_t, int b_max, int* C, int* b, int* rows_pad, int* cols_pad);
// tuning table (tune.cu): tuned block width and exchange mode for a (rows, cols, precision)
bool tune_lookup(int rows, int cols, DType jt, int* b, int* dsm);
int tune_shape(int rows, int cols, DType jt);
int tune_load(const char* path);
int tune_save(const char* path);
// FP32 SIMT products (gemm.cu / tune.cu): a choice of kernel (GEMM_SMALL: 64 x 64
// tiles, GEMM_LARGE: 128 x 128 tiles) and K splits per product shape.  While
// recording is on, gemm_run notes every shape it dispatches (with the partial
// buffer room of the call); gemm_tune_recorded times the candidates of each noted
// shape not yet in the table on synthetic operands and keeps the fastest.
enum { GEMM_SMALL = 1, GEMM_LARGE = 2 };
struct GemmPick {
  int kernel;
  int splits;
};
void gemm_record(bool on);
void gemm_note_shape(const GemmArgs& g, int64_t room);
bool gemm_pick_lookup(const GemmArgs& g, GemmPick* out);
int gemm_tune_recorded();
// launch an FP32 product with a given choice (checked: BKFAC_EINVAL when the
// layout or the partial buffer does not allow it)
int gemm_run_choice(const GemmArgs& g, GemmPick pick, cudaStream_t s);
bool gemm_choice_ok(const GemmArgs& g, GemmPick pick);
// shared memory bytes one CTA needs for a problem
size_t jacobi_smem_bytes(int b, int rows_pad, DType j_t);
// A caller's choice of the eigensolve's launch shape: the block-width cap (0: the
// shape's tuned or default plan) and the block exchange (-1: the default, 0: through
// L2, 1: over distributed shared memory).
struct JacobiChoice {
  int b_max = 0;
  int dsm = -1;
};
// An update enqueued up to its eigensolve (api.cu): the eigensolve's problem, its
// cluster size, precision and stopping tolerance.
struct StagedEig {
  JacobiProblem jp;
  int C = 0;
  DType jt = DT_F32;
  double tol = 0.0;
};
// bkfac_init (init) / bkfac_update split at the eigensolve, for a batch that runs the
// eigensolves of many factors as grouped launches: update_stage_pre enqueues
// everything before it, update_stage_post (same arguments, after the eigensolve ran
// on the stream) everything after it and advances r_cur and step.
int update_stage_pre(bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, bool init, void* ws,
                     size_t ws_bytes, const JacobiChoice* jc, cudaStream_t s, StagedEig* out);
int update_stage_post(bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, bool init, void* ws,
                      size_t ws_bytes, const JacobiChoice* jc, cudaStream_t s);
int eig_sweep_cap();
// the tuned choice for a grouped launch of `count` same-shape eigensolves (tune.cu):
// lookup only, or timing the candidates when the table has no entry
bool tune_group_lookup(int rows, int cols, DType jt, int count, JacobiChoice* out);
int tune_group(int rows, int cols, DType jt, int count, JacobiChoice* out);
// self-test of the bounded mbarrier wait (jacobi.cu): a wait on a phase nothing
// completes gives up after limit_cycles and records BKFAC_ETIMEOUT; *out (may be
// null) receives 1 on time-out
int launch_wait_selftest(long long limit_cycles, int* out, cudaStream_t s);
// choose cluster size and block width for a problem
void jacobi_plan(int rows, int cols, DType j_t, int* C, int* b, int* rows_pad, int* cols_pad);

// sort / output: lambda_i = ||w_i||^2 for the first `cols` columns, descending;
// V[:, rank] = w_i / ||w_i|| (type out_t, rows x r_out, ld ldv) for rank < r_out,
// sig[rank] = lambda_i, lam_sorted[rank] = lambda_i (optional)
struct SortArgs {
  const void* W;
  int rows, rows_pad, cols;
  int r_out;
  void* V;
  int64_t ldv;
  double* sig;           // r_sig values written (rank < r_out), zero-filled up to r_sig
  int r_sig;
  double* lam_sorted;    // 2 cols values: the sorted eigenvalues, then scratch for the sort
  const double* colnorm2; // cols_pad squared column norms of the Jacobi input
  int cols_pad;
};
int launch_sort_output(const SortArgs& a, DType j_t, DType out_t, cudaStream_t s);

// U[:, j] = Unew[:, j] for j < r_new, zero for r_new <= j < r
int launch_finalize(void* U, int64_t ldu, const void* Unew, int64_t ldn, int d, int r_new, int r, DType t,
                    cudaStream_t s);

// apply coefficients: cA = 1/(sig+lamA') - 1/lamA' (with optional continuation shift), etc.
struct ApplyCoefArgs {
  const double* sigA;
  int kA;
  const double* sigG;
  int kG;
  double lamA, lamG;
  int continuation;
  int relative;              // lamA / lamG are multiples of each factor's largest eigenvalue
  int completeA, completeG;  // r_cur == d: the basis spans R^d and the 1/lambda complement is empty
  double* cA;        // kA: C_A
  double* cG;        // kG: C_G
  double* cA_over;   // kA: C_A / lamG'
  double* cG_over;   // kG: C_G / lamA'
  double* alpha;     // 1: 1 / (lamA' lamG')
  double* betaA;     // 1: the identity weight of the A side (1 / lamA', or 0 for a complete basis); may be null
  double* betaG;     // 1: the same for the Gamma side; may be null
};
int launch_apply_coefs(const ApplyCoefArgs& a, cudaStream_t s);

// B-KFAC-C / B-R-KFAC helpers (small.cu)
// dst[:, j] = src[:, idx[j]] for j < n (idx null: the identity)
int launch_gather_cols(const void* src, int64_t lds, void* dst, int64_t ldd, int d, int n, const int* idx, DType t,
                       cudaStream_t s);
// dst[:, idx[j]] = src[:, j], sig[idx[j]] = lam[j] for j < n
int launch_scatter_cols(const void* src, int64_t lds, void* dst, int64_t ldd, int d, int n, const int* idx,
                        const double* lam, double* sig, DType t, cudaStream_t s);
// *out = max_i G[i, i] of an n x n FP64 matrix
int launch_diag_max(const double* G, int n, double* out, cudaStream_t s);
// the Jacobi input L = R^T of an upper n x n FP64 factor (L L^T = R^T R), with column norms
int launch_assemble_transpose(const double* R, int n, int rows_pad, int cols_pad, void* L, double* colnorm2,
                              DType j_t, cudaStream_t s);
// stable order by decreasing value: perm[rank] = i, sorted[rank] = sig[i]
int launch_mode_order(const double* sig, int k, int* perm, double* sorted, cudaStream_t s);

// ---------------------------------------------------------------------------
// Tracing (trace.cu): per-phase CUDA-event timing and a launch counter
// ---------------------------------------------------------------------------
enum Phase {
  PH_COLNORM, PH_PROJ, PH_RESID, PH_GRAM, PH_CHOL, PH_TRINV, PH_TRMM, PH_CORE, PH_JACOBI, PH_SORT,
  PH_ROTATE, PH_FINALIZE, PH_DENSE, PH_COEFS, PH_APPLY1, PH_APPLY_SMALL, PH_APPLY2, PH_REORTH, PH_FACT_THIN,
  PH_FACT_STEP, PH_PRECOND, PH_COUNT
};
class TraceScope {
 public:
  TraceScope(int ph, cudaStream_t s);
  ~TraceScope();

 private:
  int ph_;
  cudaStream_t s_;
  void* a_;
};
void note_launches(int n);
int64_t launch_count();

}  // namespace bkfac

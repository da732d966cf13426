// api.cu -- the C ABI of libbkfac: argument validation, workspace layout and
// the launch sequence of each call (see include/bkfac.h).
//
// Update (Algorithm 4 via Algorithm 3), Brand path, per factor:
//   scale = max_j ||x_j||^2                                (pivot reference)
//   M = U^T X                       split-K GEMM           (Algorithm 3, first step)
//   P = X - U M                     GEMM + epilogue
//   G1 = P^T P (FP64), R1 = chol(G1), Q1 = P R1^-1          CholeskyQR2, pass 1
//   G2 = Q1^T Q1 (FP64), R2 = chol(G2), Q = Q1 R2^-1        pass 2;  R = R2 R1
//   L = [[diag(sqrt(rho sigma)), sqrt(c) M], [0, sqrt(c) R]]   (M_S = L L^T, Eq. (7))
//   one-sided Jacobi on L -> lambda, V (sorted, truncated to r)
//   U <- [U Q] V[:, :r_new], sigma <- lambda[:r_new]
// Dense path (r + n >= d): Jacobi on F = [U sqrt(rho sigma), sqrt(c) X].
#include <algorithm>
#include <atomic>
#include <vector>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace bkfac {
namespace {

constexpr size_t kAlign = 256;
constexpr int kDefaultSweepCap = 40;
// Jacobi sweep cap of every eigensolve (bkfac_set_sweep_cap); a problem that reaches
// it records BKFAC_ENOCONV
std::atomic<int> g_sweep_cap{kDefaultSweepCap};
int sweep_cap() { return g_sweep_cap.load(std::memory_order_relaxed); }

size_t es_of(DType t) { return t == DT_F64 ? 8 : 4; }
DType dt_of(int dtype) { return dtype == BKFAC_F64 ? DT_F64 : DT_F32; }

struct Layout {
  size_t total = 0;
  size_t add(size_t bytes) {
    const size_t off = total;
    total += (size_t)round_up((int64_t)std::max<size_t>(bytes, 1), kAlign);
    return off;
  }
};

int r_total(const bkfac_factor* f) { return factor_r_total(f); }

bool valid_factor(const bkfac_factor* f) {
  if (!f || f->d < 1 || f->r < 1 || f->r > f->d || f->r_cur < 0) return false;
  if ((f->flags & BKFAC_FLAG_KEEP_RN) && f->r_extra < 0) return false;
  if (f->r_cur > r_total(f)) return false;
  if (f->dtype != BKFAC_F64 && f->dtype != BKFAC_F32 && f->dtype != BKFAC_MIXED_BF16) return false;
  if (!f->U || !f->sigma || f->ldu < f->d) return false;
  const size_t es = f->dtype == BKFAC_F64 ? 8 : 4;
  if (((uintptr_t)f->U) % 16 != 0 || (f->ldu * (int64_t)es) % 16 != 0) return false;
  if (((uintptr_t)f->sigma) % 8 != 0) return false;
  return true;
}

bool dense_path(const bkfac_factor* f, int n) { return (int64_t)f->r + n >= f->d; }

// element type of U / X, Jacobi type, GEMM accumulator
struct Prec {
  DType t, jt, acc;
  bool bf16;
  bool x3;     // FP32 products as 3xTF32 on the tensor cores (BKFAC_FLAG_TF32X3)
  bool chol64;  // CholeskyQR factorisations in FP64 also on the FP32 / mixed paths
  double u_t;  // unit roundoff governing the residual threshold
};
Prec prec_of(const bkfac_factor* f) {
  Prec p;
  p.t = dt_of(f->dtype);
  p.acc = p.t;
  p.bf16 = f->dtype == BKFAC_MIXED_BF16;
  p.x3 = f->dtype == BKFAC_F32 && (f->flags & BKFAC_FLAG_TF32X3) != 0;
  p.jt = (f->dtype == BKFAC_F64 || (f->flags & BKFAC_FLAG_EIG_FP64)) ? DT_F64 : DT_F32;
  p.chol64 = f->dtype == BKFAC_F64 || (f->flags & BKFAC_FLAG_CHOL_FP64) != 0;
  p.u_t = f->dtype == BKFAC_F64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
  return p;
}

double jacobi_tol(int rows, DType jt) {
  const double u = jt == DT_F64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
  return std::max(4.0 * std::sqrt((double)std::max(rows, 1)), 32.0) * u;
}

int64_t ld_of(int d) { return round_up(d, 32); }

// ------------------------------------------------------------------ update workspace plan
struct UpdatePlan {
  bool dense;
  int d, r, k, n, N, r_new;
  Prec pr;
  int64_t ldq, ldm, ldv;
  int C, b, rows_pad, cols_pad;  // Jacobi plan of this call
  int rows_cap, cols_cap;        // capacity of L
  size_t o_scale, o_M, o_part, o_P, o_Q1, o_Q, o_G, o_R1, o_R2, o_Rinv, o_L, o_cn, o_lam, o_V, o_Un, o_sw, o_st,
      o_flag, o_K;
  size_t part_bytes;
  size_t total;
};

// split-K scratch for any product up to M x N (fewer output tiles may use more
// splits, never more than 32)
size_t partial_bytes(int M, int N, int K, size_t acc_es) {
  (void)K;
  return (size_t)32 * std::max(M, 1) * std::max(N, 1) * acc_es;
}

// the eigensolve's launch shape: the tuned one for the shape (jacobi_plan), or the
// block-width cap of a caller's choice (a batch's grouped eigensolves)
void plan_jacobi(int rows, int cols, DType jt, const JacobiChoice* jc, int* C, int* b, int* rp, int* cp) {
  if (jc && jc->b_max > 0)
    jacobi_plan_with(rows, cols, jt, jc->b_max, C, b, rp, cp);
  else
    jacobi_plan(rows, cols, jt, C, b, rp, cp);
}

UpdatePlan plan_update(const bkfac_factor* f, int n, int k, const JacobiChoice* jc = nullptr) {
  UpdatePlan p{};
  p.pr = prec_of(f);
  p.d = f->d;
  p.r = f->r;
  p.k = k;
  p.n = n;
  p.dense = dense_path(f, n);
  p.ldq = ld_of(f->d);
  const size_t es = es_of(p.pr.t), jes = es_of(p.pr.jt), aes = es_of(p.pr.acc);
  Layout L;
  int rows_cap, cols_cap;
  if (p.dense) {
    p.N = k + n;
    p.r_new = std::min(std::min(r_total(f), k + n), f->d);
    plan_jacobi(f->d, k + n, p.pr.jt, jc, &p.C, &p.b, &p.rows_pad, &p.cols_pad);
    int C2, b2, rp2, cp2;
    jacobi_plan(f->d, f->r + n, p.pr.jt, &C2, &b2, &rp2, &cp2);
    rows_cap = rp2;
    cols_cap = (int)round_up(f->r + n, 32) + 128;
    p.o_L = L.add((size_t)rows_cap * cols_cap * jes);
    p.o_cn = L.add((size_t)cols_cap * 8);
    p.o_lam = L.add((size_t)cols_cap * 16);  // eigenvalues + the sort's scratch
    p.o_sw = L.add(256);
    p.o_st = L.add((size_t)cols_cap * 4);
  } else {
    const int kmax = f->r, Nmax = f->r + n;
    p.N = k + n;
    p.r_new = std::min(r_total(f), k + n);
    p.ldm = std::max(kmax, 1);
    p.ldv = round_up(Nmax, 4);
    plan_jacobi(p.N, p.N, p.pr.jt, jc, &p.C, &p.b, &p.rows_pad, &p.cols_pad);
    int C2, b2, rp2, cp2;
    jacobi_plan(Nmax, Nmax, p.pr.jt, &C2, &b2, &rp2, &cp2);
    rows_cap = rp2;
    // the Jacobi pads the columns to 2 C b with b a multiple of the register
    // blocking width K: at most 2 C K <= 128 columns beyond N
    cols_cap = (int)round_up(Nmax, 32) + 128;
    p.o_scale = L.add(8);
    p.o_M = L.add((size_t)p.ldm * n * es);
    const size_t part = std::max(partial_bytes(kmax, n, f->d, aes), partial_bytes(n, n, f->d, 8));
    p.o_part = L.add(part);
    p.part_bytes = part;
    p.o_P = L.add((size_t)p.ldq * n * es);
    p.o_Q1 = L.add((size_t)p.ldq * n * es);
    p.o_Q = L.add((size_t)p.ldq * n * es);
    p.o_G = L.add((size_t)n * n * 8);
    p.o_R1 = L.add((size_t)n * n * 8);
    p.o_R2 = L.add((size_t)n * n * 8);
    p.o_Rinv = L.add((size_t)n * n * es);
    p.o_L = L.add((size_t)rows_cap * cols_cap * jes);
    p.o_cn = L.add((size_t)cols_cap * 8);
    p.o_lam = L.add((size_t)cols_cap * 16);  // eigenvalues + the sort's scratch
    p.o_V = L.add((size_t)p.ldv * r_total(f) * es);
    p.o_Un = L.add((size_t)p.ldq * r_total(f) * es);
    p.o_sw = L.add(256);
    p.o_st = L.add((size_t)cols_cap * 4);
    p.o_flag = L.add(16);
    // the core's Gram L L^T for the preconditioned eigensolve (FP32 eigensolves)
    if (p.pr.jt == DT_F32) p.o_K = L.add((size_t)Nmax * Nmax * sizeof(float));
  }
  p.rows_cap = rows_cap;
  p.cols_cap = cols_cap;
  p.total = L.total;
  return p;
}

// ------------------------------------------------------------------ reorth plan
struct ReorthPlan {
  int d, k;
  Prec pr;
  int64_t ldq, ldv;
  int C, b, rows_pad, cols_pad, rows_cap, cols_cap;
  size_t o_part, o_G, o_R, o_Rinv, o_Q, o_L, o_cn, o_lam, o_V, o_Un, o_sw, o_st, total;
};

ReorthPlan plan_reorth(const bkfac_factor* f, int k) {
  ReorthPlan p{};
  p.pr = prec_of(f);
  p.d = f->d;
  p.k = k;
  p.ldq = ld_of(f->d);
  const int kmax = r_total(f);
  p.ldv = round_up(std::max(kmax, 1), 4);
  const size_t es = es_of(p.pr.t), jes = es_of(p.pr.jt);
  jacobi_plan(std::max(k, 1), std::max(k, 1), p.pr.jt, &p.C, &p.b, &p.rows_pad, &p.cols_pad);
  int C2, b2, rp2, cp2;
  jacobi_plan(kmax, kmax, p.pr.jt, &C2, &b2, &rp2, &cp2);
  p.rows_cap = rp2;
  p.cols_cap = (int)round_up(kmax, 32) + 128;
  Layout L;
  p.o_part = L.add(partial_bytes(kmax, kmax, f->d, 8));
  p.o_G = L.add((size_t)kmax * kmax * 8);
  p.o_R = L.add((size_t)kmax * kmax * 8);
  p.o_Rinv = L.add((size_t)kmax * kmax * es);
  p.o_Q = L.add((size_t)p.ldq * kmax * es);
  p.o_L = L.add((size_t)p.rows_cap * p.cols_cap * jes);
  p.o_cn = L.add((size_t)p.cols_cap * 8);
  p.o_lam = L.add((size_t)p.cols_cap * 16);  // eigenvalues + the sort's scratch
  p.o_V = L.add((size_t)p.ldv * kmax * es);
  p.o_Un = L.add((size_t)p.ldq * kmax * es);
  p.o_sw = L.add(256);
  p.o_st = L.add((size_t)p.cols_cap * 4);
  p.total = L.total;
  return p;
}

// ------------------------------------------------------------------ apply plan
struct ApplyPlan {
  int dA, dG, kA, kG;
  Prec pr;
  int64_t ld1, ld2, ldw;
  size_t o_T1, o_T2, o_T3, o_W1, o_part, o_part1, o_cA, o_cG, o_cAo, o_cGo, o_alpha, total;
  size_t part1_bytes;
  // the FP32 pass 1's split-K scratch: the small products' region and part1, which
  // lie back to back and are free while pass 1 runs
  size_t o_pass1, pass1_bytes;
  // mixed path on the TMA-fed tensor cores: BF16 K-major copies of the operands
  bool tma;
  int64_t ldgb, ldgt, ldua, ldug, ld2k;  // row pitches (elements) of Gb, Gt, UAb, UGb, A2 / B2
  size_t o_Gb, o_Gt, o_UAb, o_UGb, o_A2, o_B2;
};

// the mixed path's apply runs on the TMA-fed tensor-core kernel (BF16 operands
// rounded once into K-major copies) when the driver provides tensor maps
bool apply_on_tma(const Prec& pr) { return pr.bf16 && !pr.x3 && tma_gemm_available(); }

ApplyPlan plan_apply(const bkfac_factor* fA, const bkfac_factor* fG, int kA, int kG) {
  ApplyPlan p{};
  p.pr = prec_of(fA);
  p.pr.x3 = p.pr.x3 || prec_of(fG).x3;
  p.dA = fA->d;
  p.dG = fG->d;
  p.kA = kA;
  p.kG = kG;
  const int rA = r_total(fA), rG = r_total(fG);
  p.ld1 = ld_of(p.dG);  // T1, W1: d_out x r_A column-major
  p.ld2 = ld_of(p.dA);  // T2: r_G x d_in row-major
  p.ldw = std::max(rG, 1);
  const size_t es = es_of(p.pr.t), aes = es_of(p.pr.acc);
  Layout L;
  p.o_T1 = L.add((size_t)p.ld1 * rA * es);
  p.o_W1 = L.add((size_t)p.ld1 * rA * es);
  p.o_T2 = L.add((size_t)p.ld2 * rG * es);
  p.o_T3 = L.add((size_t)p.ldw * rA * es);
  p.o_part = L.add(partial_bytes(rG, rA, p.dG, aes));
  // pass 1 may split K in two: scratch for two copies of the larger of T1 / T2
  p.part1_bytes = (size_t)2 * std::max((size_t)p.dG * rA, (size_t)p.dA * rG) * aes;
  p.o_part1 = L.add(p.part1_bytes);
  p.o_pass1 = p.o_part;
  p.pass1_bytes = p.o_part1 + p.part1_bytes - p.o_part;
  p.o_cA = L.add((size_t)rA * 8);
  p.o_cG = L.add((size_t)rG * 8);
  p.o_cAo = L.add((size_t)rA * 8);
  p.o_cGo = L.add((size_t)rG * 8);
  p.o_alpha = L.add(8);
  p.tma = apply_on_tma(p.pr);
  if (p.tma) {
    // split K of pass 1 into up to 8 pieces (T1: d_out x r_A and T2: d_in x r_G outputs)
    p.part1_bytes = (size_t)8 * std::max((size_t)p.dG * rA, (size_t)p.dA * rG) * aes;
    p.o_part1 = L.add(p.part1_bytes);
    p.ldgb = bf16_ld(p.dA);
    p.ldgt = bf16_ld(p.dG);
    p.ldua = bf16_ld(p.dA);
    p.ldug = bf16_ld(p.dG);
    p.ld2k = bf16_ld(rA + rG);
    p.o_Gb = L.add((size_t)p.dG * p.ldgb * 2);
    p.o_Gt = L.add((size_t)p.dA * p.ldgt * 2);
    p.o_UAb = L.add((size_t)std::max(rA, 1) * p.ldua * 2);
    p.o_UGb = L.add((size_t)std::max(rG, 1) * p.ldug * 2);
    p.o_A2 = L.add((size_t)p.dG * p.ld2k * 2);
    p.o_B2 = L.add((size_t)p.dA * p.ld2k * 2);
  }
  p.total = L.total;
  return p;
}

// workspace of the linear inverse application (Algorithm 8) for n columns
struct FactoredPlan {
  Prec pr;
  int64_t ldtA, ldtG;  // T_A (r_A x n), T_G (r_G x n), column-major
  size_t o_TA, o_TG, o_part, o_cA, o_cG, o_cAo, o_cGo, o_alpha, o_bA, o_bG, total;
  size_t part_bytes;
};

FactoredPlan plan_factored(const bkfac_factor* fA, const bkfac_factor* fG, int n) {
  FactoredPlan p{};
  p.pr = prec_of(fA);
  p.pr.x3 = p.pr.x3 || prec_of(fG).x3;
  const int rA = r_total(fA), rG = r_total(fG);
  p.ldtA = std::max(rA, 1);
  p.ldtG = std::max(rG, 1);
  const size_t es = es_of(p.pr.t), aes = es_of(p.pr.acc);
  Layout L;
  p.o_TA = L.add((size_t)p.ldtA * n * es);
  p.o_TG = L.add((size_t)p.ldtG * n * es);
  p.part_bytes = partial_bytes(std::max(rA, rG), n, 0, aes);
  p.o_part = L.add(p.part_bytes);
  p.o_cA = L.add((size_t)rA * 8);
  p.o_cG = L.add((size_t)rG * 8);
  p.o_cAo = L.add((size_t)rA * 8);
  p.o_cGo = L.add((size_t)rG * 8);
  p.o_alpha = L.add(8);
  p.o_bA = L.add(8);
  p.o_bG = L.add(8);
  p.total = L.total;
  return p;
}

template <typename P>
P* at(void* ws, size_t off) {
  return (P*)((char*)ws + off);
}

#define BK_TRY(expr)                     \
  do {                                   \
    int _e = (expr);                     \
    if (_e != 0) return BKFAC_ECUDA;     \
  } while (0)

// one traced phase: CUDA events around the launches when tracing is enabled
#define PHASE(ph, expr)                  \
  do {                                   \
    TraceScope _ts((ph), s);             \
    BK_TRY(expr);                        \
  } while (0)

// Cholesky: the cluster kernel when n fits it, else the single-CTA kernel
// near_out (may be null) receives whether the near-identity shortcut was taken
// neg_rel > 0: a pivot below -neg_rel * (*scale) records BKFAC_ECHOL (the matrix is
// indefinite beyond its rounding); 0 disables the check
int run_chol(const double* Gm, int n, double* R, double thr_rel, const double* scale, double near_tol,
             int* near_out, cudaStream_t s, double neg_rel = 0.0) {
  // the blocked 2D block-cyclic kernel spreads every step over the cluster
  if (chol_block_ok(n)) return launch_chol_block(Gm, n, R, thr_rel, scale, near_tol, near_out, neg_rel, s);
  if (chol_cluster_size(n) > 0)
    return launch_chol_cluster(Gm, n, R, thr_rel, scale, near_tol, near_out, neg_rel, s);
  if (near_out != nullptr && cudaMemsetAsync(near_out, 0, sizeof(int), s) != cudaSuccess) return BKFAC_ECUDA;
  return launch_chol(Gm, n, R, thr_rel, scale, neg_rel, s);
}

// second CholeskyQR pass: G2 = I + E; the near-identity factor's error is O(|E|^2)
double near_identity_tol(const Prec& pr) { return pr.t == DT_F64 ? 1e-9 : 1e-5; }

// The Cholesky factorisations of CholeskyQR2: FP64 for the FP64 path (and with
// BKFAC_FLAG_CHOL_FP64); by default the FP32 and mixed paths factor the FP64-accurate
// Gram in FP32 on the cluster (FP64 runs at 1/64 of the FP32 rate on this GPU), and a
// pivot is also dropped when its
// Schur complement is within the FP32 elimination's rounding noise of its diagonal,
// 4 sqrt(n) u_32 G_jj: such a direction is numerically dependent at FP32 precision
// and its orthogonalisation would be noise.  The second pass restores
// orthonormality to the working precision as before.
int run_chol_qr(const Prec& pr, const double* Gm, int n, double* R, double thr_abs, const double* scale,
                double near_tol, int* near, cudaStream_t s) {
  if (!pr.chol64 && chol_r32_ok(n)) {
    const float thr_rel = (float)(4.0 * std::sqrt((double)n) * 5.9604644775390625e-08);
    return launch_chol_r32(Gm, n, R, thr_rel, thr_abs, scale, near_tol, near, s);
  }
  return run_chol(Gm, n, R, thr_abs, scale, near_tol, near, s);
}

// FP32 eigensolves of Brand cores with at least this many columns run the Jacobi
// on the Cholesky factor of the core matrix instead of the core factor L (fewer
// sweeps; the factorisation costs a few percent of one sweep)
constexpr int kPrecondMinN = 128;

bool precondition_core(const UpdatePlan& p) {
  return !p.dense && p.pr.jt == DT_F32 && p.N >= kPrecondMinN && chol_core_ok(p.N, p.rows_pad, p.cols_pad);
}

GemmArgs gemm_base() {
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.alpha = 1.0;
  g.beta = 0.0;
  g.splits = 1;
  return g;
}

// Gram G = A^T A of a d x n column-major matrix (FP64 accumulation), output n x n
int run_gram(const void* A, int64_t lda, int d, int n, Prec pr, double* G, void* part, cudaStream_t s) {
  GemmArgs g = gemm_base();
  g.M = n;
  g.N = n;
  g.K0 = d;
  g.A0 = A;
  g.lda0 = lda;
  g.B0 = A;
  g.ldb0 = lda;
  g.a_kmaj = true;
  g.b_kmaj = true;
  g.C = G;
  g.ldc = n;
  g.sym = true;
  // only the upper tiles of the symmetric output are computed: split K until about
  // two CTAs per SM are busy (at most 32 partials, at least 128 rows of K each)
  const int64_t tiles = ceil_div(n, 64), active = tiles * (tiles + 1) / 2;
  int64_t splits = ceil_div(2 * sm_count(), active);
  splits = std::min<int64_t>(std::min<int64_t>(splits, 32), std::max<int64_t>(1, d / 128));
  g.splits = (int)std::max<int64_t>(2, splits);
  g.partial = part;
  // FP32 data: FP64-accurate Gram on the FP32 pipes (compensated); FP64 data: DFMA
  if (pr.t == DT_F32) return gram_run_comp(g, s);
  return gemm_run(g, pr.t, DT_F64, DT_F64, s);
}

// Q = P Rinv (d x n times n x n upper), output column-major ld ldq
int run_trmm(const void* P, int64_t ldp, int d, int n, const void* Rinv, Prec pr, void* Q, int64_t ldq,
             void* part, size_t part_bytes, cudaStream_t s) {
  GemmArgs g = gemm_base();
  g.M = d;
  g.N = n;
  g.K0 = n;
  g.A0 = P;
  g.lda0 = ldp;
  g.a_kmaj = false;
  g.B0 = Rinv;
  g.ldb0 = n;
  g.b_kmaj = true;
  g.C = Q;
  g.ldc = ldq;
  g.partial = part;
  g.partial_bytes = part_bytes;
  return gemm_run(g, pr.t, pr.acc, pr.t, s);
}

// The update of one factor up to its eigensolve (k = current rank): the Brand path's
// projection, residual, CholeskyQR2, core factor L (and on FP32 eigensolves the
// Cholesky factor of the core matrix), or the dense path's factor F; *jp_out
// receives the eigensolve's problem.
int enqueue_update_pre(const bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, void* ws,
                       const UpdatePlan& p, cudaStream_t s, JacobiProblem* jp_out) {
  const Prec& pr = p.pr;
  const int d = f->d, k = p.k;
  const double c = (1.0 - rho) / (double)n;
  if (p.dense) {
    DenseArgs a;
    a.d = d;
    a.k = k;
    a.n = n;
    a.rows_pad = p.rows_pad;
    a.cols_pad = p.cols_pad;
    a.rho = rho;
    a.c = c;
    a.U = f->U;
    a.ldu = f->ldu;
    a.sigma = f->sigma;
    a.X = X;
    a.ldx = ldx;
    a.F = at<void>(ws, p.o_L);
    a.colnorm2 = at<double>(ws, p.o_cn);
    PHASE(PH_DENSE, launch_assemble_dense(a, pr.t, pr.jt, s));
    JacobiProblem jp;
    jp.W = a.F;
    jp.rows = d;
    jp.cols = k + n;
    jp.rows_pad = p.rows_pad;
    jp.cols_pad = p.cols_pad;
    jp.b = p.b;
    jp.colnorm2 = a.colnorm2;
    jp.sweeps_out = at<int>(ws, p.o_sw);
    jp.stamp = at<int>(ws, p.o_st);
    *jp_out = jp;
    return BKFAC_OK;
  }

  double* scale = at<double>(ws, p.o_scale);
  void* M = at<void>(ws, p.o_M);
  void* part = at<void>(ws, p.o_part);
  void* P = at<void>(ws, p.o_P);
  void* Q1 = at<void>(ws, p.o_Q1);
  void* Q = at<void>(ws, p.o_Q);
  double* Gm = at<double>(ws, p.o_G);
  double* R1 = at<double>(ws, p.o_R1);
  double* R2 = at<double>(ws, p.o_R2);
  void* Rinv = at<void>(ws, p.o_Rinv);
  PHASE(PH_COLNORM, launch_colnorm_max(X, ldx, d, n, pr.t, scale, s));

  const void* Pp = X;
  int64_t ldp = ldx;
  if (k > 0) {
    // M = U^T X  (k x n, K = d)
    GemmArgs g = gemm_base();
    g.M = k;
    g.N = n;
    g.K0 = d;
    g.A0 = f->U;
    g.lda0 = f->ldu;
    g.a_kmaj = true;
    g.B0 = X;
    g.ldb0 = ldx;
    g.b_kmaj = true;
    g.round_bf16 = pr.bf16;
    g.tf32x3 = pr.x3;
    g.C = M;
    g.ldc = p.ldm;
    g.splits = gemm_pick_splits(k, n, d, sm_count());
    g.partial = part;
    g.partial_bytes = p.part_bytes;
    PHASE(PH_PROJ, gemm_run(g, pr.t, pr.acc, pr.t, s));
    // P = X - U M  (d x n, K = k)
    GemmArgs h = gemm_base();
    h.M = d;
    h.N = n;
    h.K0 = k;
    h.A0 = f->U;
    h.lda0 = f->ldu;
    h.a_kmaj = false;
    h.B0 = M;
    h.ldb0 = p.ldm;
    h.b_kmaj = true;
    h.round_bf16 = pr.bf16;
    h.tf32x3 = pr.x3;
    h.C = P;
    h.ldc = p.ldq;
    h.D = X;
    h.ldd = ldx;
    h.alpha = -1.0;
    h.beta = 1.0;
    h.partial = part;
    h.partial_bytes = p.part_bytes;
    PHASE(PH_RESID, gemm_run(h, pr.t, pr.acc, pr.t, s));
    Pp = P;
    ldp = p.ldq;
  }
  // CholeskyQR2 with FP64 Gram and Cholesky
  const double ue = pr.bf16 ? 3.90625e-3 : pr.u_t;
  const double thr1 = pr.bf16 ? (2.0 * ue) * (2.0 * ue) : (64.0 * ue) * (64.0 * ue);
  const double thr2 = (64.0 * pr.u_t) * (64.0 * pr.u_t);
  PHASE(PH_GRAM, run_gram(Pp, ldp, d, n, pr, Gm, part, s));
  PHASE(PH_CHOL, run_chol_qr(pr, Gm, n, R1, thr1, scale, 0.0, nullptr, s));
  PHASE(PH_TRINV, launch_trinv(R1, n, Rinv, pr.t, nullptr, s));
  PHASE(PH_TRMM, run_trmm(Pp, ldp, d, n, Rinv, pr, Q1, p.ldq, part, p.part_bytes, s));
  PHASE(PH_GRAM, run_gram(Q1, p.ldq, d, n, pr, Gm, part, s));
  int* near = at<int>(ws, p.o_flag);
  PHASE(PH_CHOL, run_chol_qr(pr, Gm, n, R2, thr2, nullptr, near_identity_tol(pr), near, s));
  PHASE(PH_TRINV, launch_trinv(R2, n, Rinv, pr.t, near, s));
  PHASE(PH_TRMM, run_trmm(Q1, p.ldq, d, n, Rinv, pr, Q, p.ldq, part, p.part_bytes, s));
  // core factor L and its Jacobi eigensolve
  CoreArgs ca;
  ca.k = k;
  ca.n = n;
  ca.N = k + n;
  ca.rows_pad = p.rows_pad;
  ca.cols_pad = p.cols_pad;
  ca.rho = rho;
  ca.c = c;
  ca.sigma = f->sigma;
  ca.M = M;
  ca.ldm = p.ldm;
  ca.R1 = R1;
  ca.R2 = R2;
  ca.L = at<void>(ws, p.o_L);
  ca.colnorm2 = at<double>(ws, p.o_cn);
  PHASE(PH_CORE, launch_assemble_core(ca, pr.t, pr.jt, s));
  if (precondition_core(p)) {
    // K = L L^T (FP32), then K = G G^T: G = L Z (Z orthogonal) has the left singular
    // vectors and singular values of L, and its columns are much closer to orthogonal
    float* Kc = at<float>(ws, p.o_K);
    GemmArgs kg = gemm_base();
    kg.M = p.N;
    kg.N = p.N;
    kg.K0 = p.N;
    kg.A0 = ca.L;
    kg.lda0 = p.rows_pad;
    kg.a_kmaj = false;
    kg.B0 = ca.L;
    kg.ldb0 = p.rows_pad;
    kg.b_kmaj = false;
    kg.C = Kc;
    kg.ldc = p.N;
    kg.splits = std::max(1, std::min(8, p.N / 64));  // 16 output tiles at N = 512: split K to fill the GPU
    kg.partial = part;
    kg.partial_bytes = p.part_bytes;
    PHASE(PH_PRECOND, gemm_run(kg, DT_F32, DT_F32, DT_F32, s));
    const float thr_rel = (float)(4.0 * std::sqrt((double)p.N) * 5.9604644775390625e-08);
    PHASE(PH_PRECOND, launch_chol_core(Kc, p.N, p.N, (float*)ca.L, p.rows_pad, p.cols_pad, ca.colnorm2, thr_rel, s));
  }
  JacobiProblem jp;
  jp.W = ca.L;
  jp.rows = p.N;
  jp.cols = p.N;
  jp.rows_pad = p.rows_pad;
  jp.cols_pad = p.cols_pad;
  jp.b = p.b;
  jp.colnorm2 = ca.colnorm2;
  jp.sweeps_out = at<int>(ws, p.o_sw);
  jp.stamp = at<int>(ws, p.o_st);
  *jp_out = jp;
  return BKFAC_OK;
}

// The rest of the update after its eigensolve: eigenvalues in decreasing order and
// the eigenvector matrix V (Brand path) or the new U (dense path), U' = [U Q] V[:, :r_new]
// and its write-back.  Reads the workspace the pre-eigensolve stage filled.
int enqueue_update_post(const bkfac_factor* f, int n, void* ws, const UpdatePlan& p, cudaStream_t s) {
  const Prec& pr = p.pr;
  const int d = f->d, k = p.k;
  if (p.dense) {
    SortArgs so;
    so.W = at<void>(ws, p.o_L);
    so.rows = d;
    so.rows_pad = p.rows_pad;
    so.cols = k + n;
    so.r_out = p.r_new;
    so.V = f->U;
    so.ldv = f->ldu;
    so.sig = f->sigma;
    so.r_sig = r_total(f);
    so.lam_sorted = at<double>(ws, p.o_lam);
    so.colnorm2 = at<double>(ws, p.o_cn);
    so.cols_pad = p.cols_pad;
    PHASE(PH_SORT, launch_sort_output(so, pr.jt, pr.t, s));
    // columns past r_new are cleared so U holds no stale modes
    if (p.r_new < r_total(f)) {
      PHASE(PH_FINALIZE, launch_finalize(f->U, f->ldu, f->U, f->ldu, d, p.r_new, r_total(f), pr.t, s));
    }
    return BKFAC_OK;
  }

  void* Q = at<void>(ws, p.o_Q);
  void* part = at<void>(ws, p.o_part);
  SortArgs so;
  so.W = at<void>(ws, p.o_L);
  so.rows = p.N;
  so.rows_pad = p.rows_pad;
  so.cols = p.N;
  so.r_out = p.r_new;
  so.V = at<void>(ws, p.o_V);
  so.ldv = p.ldv;
  so.sig = f->sigma;
  so.r_sig = r_total(f);
  so.lam_sorted = at<double>(ws, p.o_lam);
  so.colnorm2 = at<double>(ws, p.o_cn);
  so.cols_pad = p.cols_pad;
  // sigma is only read by the core assembly above, so it can be overwritten here
  PHASE(PH_SORT, launch_sort_output(so, pr.jt, pr.t, s));
  // U' = [U Q] V[:, :r_new]
  GemmArgs g = gemm_base();
  g.M = d;
  g.N = p.r_new;
  g.K0 = k;
  g.K1 = n;
  g.A0 = f->U;
  g.lda0 = f->ldu;
  g.A1 = Q;
  g.lda1 = p.ldq;
  g.a_kmaj = false;
  g.B0 = so.V;
  g.ldb0 = p.ldv;
  g.B1 = (const char*)so.V + (size_t)k * es_of(pr.t);
  g.ldb1 = p.ldv;
  g.b_kmaj = true;
  g.round_bf16 = pr.bf16;
  g.tf32x3 = pr.x3;
  g.C = at<void>(ws, p.o_Un);
  g.ldc = p.ldq;
  g.partial = part;
  g.partial_bytes = p.part_bytes;
  PHASE(PH_ROTATE, gemm_run(g, pr.t, pr.acc, pr.t, s));
  PHASE(PH_FINALIZE, launch_finalize(f->U, f->ldu, g.C, p.ldq, d, p.r_new, r_total(f), pr.t, s));
  return BKFAC_OK;
}

// The whole update of one factor: pre-eigensolve stage, the eigensolve, the rest.
int enqueue_update(const bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, void* ws,
                   const UpdatePlan& p, cudaStream_t s) {
  JacobiProblem jp;
  int rc = enqueue_update_pre(f, X, ldx, n, rho, ws, p, s, &jp);
  if (rc) return rc;
  PHASE(PH_JACOBI, launch_jacobi(&jp, 1, p.C, p.pr.jt, jacobi_tol(jp.rows, p.pr.jt), sweep_cap(), s));
  return enqueue_update_post(f, n, ws, p, s);
}

int check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return BKFAC_OK;
  if (!ws || ((uintptr_t)ws) % kAlign != 0 || ws_bytes < need) return BKFAC_EWORKSPACE;
  return BKFAC_OK;
}

// the eigensolve holds every row of its columns: rows <= rows_pad (at most 1024
// FP32 / 512 FP64 rows) and two blocks of b columns within 200 KB of shared memory
bool jacobi_fits(int rows, int C, int b, int rows_pad, DType jt) {
  (void)C;
  return rows <= rows_pad && b <= 32 && jacobi_smem_bytes(b, rows_pad, jt) <= 200 * 1024;
}

// argument checks and the plan of one update (k = the modes it starts from); the plan
// of the largest rank sizes the workspace
int plan_checked(const bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, void* ws, size_t ws_bytes,
                 bool init, const JacobiChoice* jc, UpdatePlan* out) {
  if (!valid_factor(f) || !X || n < 1 || ldx < f->d) return BKFAC_EINVAL;
  const size_t es = f->dtype == BKFAC_F64 ? 8 : 4;
  if (((uintptr_t)X) % 16 != 0 || (ldx * (int64_t)es) % 16 != 0) return BKFAC_EINVAL;
  if (!(rho >= 0.0 && rho < 1.0)) return BKFAC_EINVAL;
  if (!init && f->r_cur < 1) return BKFAC_EINVAL;
  // truncation to the leading r modes happens here, just before the update (with
  // BKFAC_FLAG_KEEP_RN the factor may hold more after the previous one)
  const int k = init ? 0 : std::min(f->r_cur, f->r);
  const UpdatePlan cap = plan_update(f, n, f->r);
  UpdatePlan p = plan_update(f, n, k, jc);
  p.total = cap.total;
  if (p.rows_pad > p.rows_cap || p.cols_pad > p.cols_cap) return BKFAC_EINVAL;
  if (!jacobi_fits(p.dense ? f->d : p.N, p.C, p.b, p.rows_pad, p.pr.jt)) return BKFAC_EINVAL;
  if (p.N > 8192 || (!p.dense && n > 1024)) return BKFAC_EINVAL;
  const int rc = check_ws(ws, ws_bytes, cap.total);
  if (rc) return rc;
  *out = p;
  return BKFAC_OK;
}

int update_common(bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, void* ws, size_t ws_bytes,
                  cudaStream_t s, bool init) {
  UpdatePlan p;
  int rc = plan_checked(f, X, ldx, n, rho, ws, ws_bytes, init, nullptr, &p);
  if (rc) return rc;
  rc = enqueue_update(f, X, ldx, n, init ? 0.0 : rho, ws, p, s);
  if (rc) return rc;
  f->r_cur = p.r_new;
  f->step = init ? 1 : f->step + 1;
  return BKFAC_OK;
}


// ------------------------------------------------------------------ B-KFAC-C / B-R-KFAC
// Small symmetric p.s.d. eigenproblem A = W diag(lam) W^T (A n x n FP64, its lower
// part read): FP64 Cholesky A = R^T R (pivots below thr_rel * max diag(A) dropped),
// one-sided Jacobi on L = R^T (L L^T = A), eigenpairs in decreasing order: V (n x n,
// ld ldv, element type of the factor) and lam (n doubles).
struct SmallEvd {
  int n, C, b, rows_pad, cols_pad;
  int64_t ldv;
  size_t o_R, o_scale, o_L, o_cn, o_lams, o_V, o_lam, o_sw, o_st;
};

SmallEvd plan_small_evd(int n, const Prec& pr, Layout& L) {
  SmallEvd e{};
  e.n = n;
  jacobi_plan(std::max(n, 1), std::max(n, 1), pr.jt, &e.C, &e.b, &e.rows_pad, &e.cols_pad);
  const size_t es = es_of(pr.t), jes = es_of(pr.jt);
  e.ldv = round_up(std::max(n, 1), 4);
  e.o_R = L.add((size_t)n * n * 8);
  e.o_scale = L.add(8);
  e.o_L = L.add((size_t)e.rows_pad * e.cols_pad * jes);
  e.o_cn = L.add((size_t)e.cols_pad * 8);
  e.o_lams = L.add((size_t)e.cols_pad * 16);  // eigenvalues + the sort's scratch
  e.o_V = L.add((size_t)e.ldv * n * es);
  e.o_lam = L.add((size_t)std::max(n, 1) * 8);
  e.o_sw = L.add(256);
  e.o_st = L.add((size_t)e.cols_pad * 4);
  return e;
}

bool small_evd_fits(const SmallEvd& e, const Prec& pr) {
  return e.n >= 1 && jacobi_fits(e.n, e.C, e.b, e.rows_pad, pr.jt) && (size_t)e.n * 12 <= 200 * 1024;
}

int run_small_evd(const double* A, const SmallEvd& e, const Prec& pr, double thr_rel, void* ws, cudaStream_t s) {
  double* R = at<double>(ws, e.o_R);
  double* scale = at<double>(ws, e.o_scale);
  void* L = at<void>(ws, e.o_L);
  double* cn = at<double>(ws, e.o_cn);
  PHASE(PH_CHOL, launch_diag_max(A, e.n, scale, s));
  // the matrix must be p.s.d.: a Schur complement below -1e-2 of its largest diagonal
  // entry is indefiniteness far beyond rounding (BKFAC_ECHOL; rounding in the
  // projection of an FP32 dense factor onto its tail modes stays orders of magnitude
  // below that); such a pivot is still dropped
  PHASE(PH_CHOL, run_chol(A, e.n, R, thr_rel, scale, 0.0, nullptr, s, 1e-2));
  PHASE(PH_CORE, launch_assemble_transpose(R, e.n, e.rows_pad, e.cols_pad, L, cn, pr.jt, s));
  JacobiProblem jp;
  jp.W = L;
  jp.rows = e.n;
  jp.cols = e.n;
  jp.rows_pad = e.rows_pad;
  jp.cols_pad = e.cols_pad;
  jp.b = e.b;
  jp.colnorm2 = cn;
  jp.sweeps_out = at<int>(ws, e.o_sw);
  jp.stamp = at<int>(ws, e.o_st);
  PHASE(PH_JACOBI, launch_jacobi(&jp, 1, e.C, pr.jt, jacobi_tol(e.n, pr.jt), sweep_cap(), s));
  SortArgs so;
  so.W = L;
  so.rows = e.n;
  so.rows_pad = e.rows_pad;
  so.cols = e.n;
  so.r_out = e.n;
  so.V = at<void>(ws, e.o_V);
  so.ldv = e.ldv;
  so.sig = at<double>(ws, e.o_lam);
  so.r_sig = e.n;
  so.lam_sorted = at<double>(ws, e.o_lams);
  so.colnorm2 = cn;
  so.cols_pad = e.cols_pad;
  PHASE(PH_SORT, launch_sort_output(so, pr.jt, pr.t, s));
  return BKFAC_OK;
}

// workspace of the light correction (Algorithm 6) along n_crc modes
struct CorrectPlan {
  Prec pr;
  int64_t ldq;
  SmallEvd e;
  size_t o_idx, o_Us, o_W, o_Ms, o_part, part_bytes, o_perm, o_sorted, o_Ut, total;
};

CorrectPlan plan_correct(const bkfac_factor* f, int n_crc) {
  CorrectPlan p{};
  p.pr = prec_of(f);
  p.ldq = ld_of(f->d);
  const int rt = r_total(f);
  const size_t es = es_of(p.pr.t);
  Layout L;
  p.o_idx = L.add((size_t)std::max(n_crc, 1) * 4);
  p.o_Us = L.add((size_t)p.ldq * n_crc * es);
  p.o_W = L.add((size_t)p.ldq * n_crc * es);
  p.o_Ms = L.add((size_t)n_crc * n_crc * 8);
  p.part_bytes = std::max((size_t)4 * p.ldq * n_crc * es_of(p.pr.acc), partial_bytes(n_crc, n_crc, f->d, 8));
  p.o_part = L.add(p.part_bytes);
  p.o_perm = L.add((size_t)rt * 4);
  p.o_sorted = L.add((size_t)rt * 8);
  p.o_Ut = L.add((size_t)p.ldq * rt * es);
  p.e = plan_small_evd(n_crc, p.pr, L);
  p.total = L.total;
  return p;
}

// W = M B (d x m, M d x d symmetric, B d x m, column-major), factor precision
int run_dense_times(const void* M, int64_t ldm, int d, const void* B, int64_t ldb, int m, void* W, int64_t ldw,
                    const Prec& pr, void* part, size_t part_bytes, cudaStream_t s) {
  GemmArgs g = gemm_base();
  g.M = d;
  g.N = m;
  g.K0 = d;
  g.A0 = M;
  g.lda0 = ldm;
  g.a_kmaj = false;
  g.B0 = B;
  g.ldb0 = ldb;
  g.b_kmaj = true;
  g.round_bf16 = pr.bf16;
  g.tf32x3 = pr.x3;
  g.C = W;
  g.ldc = ldw;
  g.partial = part;
  g.partial_bytes = part_bytes;
  return gemm_run(g, pr.t, pr.acc, pr.t, s);
}

// C = A^T B (m x m FP64 output, FP64 accumulation; A, B d x m column-major)
int run_cross_f64(const void* A, int64_t lda, const void* B, int64_t ldb, int d, int m, double* C, const Prec& pr,
                  void* part, cudaStream_t s) {
  GemmArgs g = gemm_base();
  g.M = m;
  g.N = m;
  g.K0 = d;
  g.A0 = A;
  g.lda0 = lda;
  g.a_kmaj = true;
  g.B0 = B;
  g.ldb0 = ldb;
  g.b_kmaj = true;
  g.C = C;
  g.ldc = m;
  g.splits = gemm_pick_splits(m, m, d, sm_count());
  g.partial = part;
  return gemm_run(g, pr.t, DT_F64, DT_F64, s);
}

// C = A B (d x m; A d x k column-major, B k x m column-major with ld ldb)
int run_rotate(const void* A, int64_t lda, int d, int k, const void* B, int64_t ldb, int m, void* C, int64_t ldc,
               const Prec& pr, void* part, size_t part_bytes, cudaStream_t s) {
  GemmArgs g = gemm_base();
  g.M = d;
  g.N = m;
  g.K0 = k;
  g.A0 = A;
  g.lda0 = lda;
  g.a_kmaj = false;
  g.B0 = B;
  g.ldb0 = ldb;
  g.b_kmaj = true;
  g.round_bf16 = pr.bf16;
  g.tf32x3 = pr.x3;
  g.C = C;
  g.ldc = ldc;
  g.partial = part;
  g.partial_bytes = part_bytes;
  return gemm_run(g, pr.t, pr.acc, pr.t, s);
}

// the factor's r_cur modes re-sorted by decreasing sigma (stable)
int resort_modes(bkfac_factor* f, int* perm, double* sorted, void* Ut, int64_t ldt, const Prec& pr,
                 cudaStream_t s) {
  const int k = f->r_cur;
  PHASE(PH_FINALIZE, launch_mode_order(f->sigma, k, perm, sorted, s));
  PHASE(PH_FINALIZE, launch_gather_cols(f->U, f->ldu, Ut, ldt, f->d, k, perm, pr.t, s));
  PHASE(PH_FINALIZE, launch_gather_cols(Ut, ldt, f->U, f->ldu, f->d, k, nullptr, pr.t, s));
  if (k > 0 && cudaMemcpyAsync(f->sigma, sorted, (size_t)k * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return BKFAC_ECUDA;
  return BKFAC_OK;
}

// workspace of the RSVD overwrite (Algorithm 5) with l test columns
struct RsvdPlan {
  Prec pr;
  int64_t ldq;
  SmallEvd e;
  size_t o_Y, o_Q1, o_Q, o_G, o_R1, o_R2, o_Rinv, o_flag, o_scale, o_part, part_bytes, total;
};

RsvdPlan plan_rsvd(const bkfac_factor* f, int l) {
  RsvdPlan p{};
  p.pr = prec_of(f);
  p.ldq = ld_of(f->d);
  const size_t es = es_of(p.pr.t);
  Layout L;
  p.o_Y = L.add((size_t)p.ldq * l * es);
  p.o_Q1 = L.add((size_t)p.ldq * l * es);
  p.o_Q = L.add((size_t)p.ldq * l * es);
  p.o_G = L.add((size_t)l * l * 8);
  p.o_R1 = L.add((size_t)l * l * 8);
  p.o_R2 = L.add((size_t)l * l * 8);
  p.o_Rinv = L.add((size_t)l * l * es);
  p.o_flag = L.add(16);
  p.o_scale = L.add(8);
  p.part_bytes = std::max((size_t)4 * p.ldq * l * es_of(p.pr.acc), partial_bytes(l, l, f->d, 8));
  p.o_part = L.add(p.part_bytes);
  p.e = plan_small_evd(l, p.pr, L);
  p.total = L.total;
  return p;
}

// Q = orth(Y) by CholeskyQR2 (FP64 Gram and Cholesky, dropped pivots give zero columns)
int run_orth(const void* Y, int d, int l, const RsvdPlan& p, void* ws, void* Q, cudaStream_t s) {
  const Prec& pr = p.pr;
  void* part = at<void>(ws, p.o_part);
  double* Gm = at<double>(ws, p.o_G);
  double* R1 = at<double>(ws, p.o_R1);
  double* R2 = at<double>(ws, p.o_R2);
  void* Rinv = at<void>(ws, p.o_Rinv);
  void* Q1 = at<void>(ws, p.o_Q1);
  double* scale = at<double>(ws, p.o_scale);
  int* near = at<int>(ws, p.o_flag);
  const double ue = pr.bf16 ? 3.90625e-3 : pr.u_t;
  const double thr1 = (64.0 * ue) * (64.0 * ue);
  const double thr2 = (64.0 * pr.u_t) * (64.0 * pr.u_t);
  PHASE(PH_COLNORM, launch_colnorm_max(Y, p.ldq, d, l, pr.t, scale, s));
  PHASE(PH_GRAM, run_gram(Y, p.ldq, d, l, pr, Gm, part, s));
  PHASE(PH_CHOL, run_chol_qr(pr, Gm, l, R1, thr1, scale, 0.0, nullptr, s));
  PHASE(PH_TRINV, launch_trinv(R1, l, Rinv, pr.t, nullptr, s));
  PHASE(PH_TRMM, run_trmm(Y, p.ldq, d, l, Rinv, pr, Q1, p.ldq, part, p.part_bytes, s));
  PHASE(PH_GRAM, run_gram(Q1, p.ldq, d, l, pr, Gm, part, s));
  PHASE(PH_CHOL, run_chol_qr(pr, Gm, l, R2, thr2, nullptr, near_identity_tol(pr), near, s));
  PHASE(PH_TRINV, launch_trinv(R2, l, Rinv, pr.t, near, s));
  PHASE(PH_TRMM, run_trmm(Q1, p.ldq, d, l, Rinv, pr, Q, p.ldq, part, p.part_bytes, s));
  return BKFAC_OK;
}

}  // namespace

// ---- staged updates for the batch: pre-eigensolve stage, grouped eigensolves, rest
int update_stage_pre(bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, bool init, void* ws,
                     size_t ws_bytes, const JacobiChoice* jc, cudaStream_t s, StagedEig* out) {
  UpdatePlan p;
  int rc = plan_checked(f, X, ldx, n, rho, ws, ws_bytes, init, jc, &p);
  if (rc) return rc;
  rc = enqueue_update_pre(f, X, ldx, n, init ? 0.0 : rho, ws, p, s, &out->jp);
  if (rc) return rc;
  out->C = p.C;
  out->jt = p.pr.jt;
  out->tol = jacobi_tol(out->jp.rows, p.pr.jt);
  return BKFAC_OK;
}

int update_stage_post(bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, bool init, void* ws,
                      size_t ws_bytes, const JacobiChoice* jc, cudaStream_t s) {
  UpdatePlan p;
  int rc = plan_checked(f, X, ldx, n, rho, ws, ws_bytes, init, jc, &p);
  if (rc) return rc;
  rc = enqueue_update_post(f, n, ws, p, s);
  if (rc) return rc;
  f->r_cur = p.r_new;
  f->step = init ? 1 : f->step + 1;
  return BKFAC_OK;
}

int eig_sweep_cap() { return sweep_cap(); }

}  // namespace bkfac

using namespace bkfac;

extern "C" {

int bkfac_version(void) { return 100; }

const char* bkfac_strerror(int code) {
  switch (code) {
    case BKFAC_OK: return "ok";
    case BKFAC_EINVAL: return "invalid argument";
    case BKFAC_ENOTAPPLICABLE: return "path not applicable to these shapes";
    case BKFAC_ECHOL: return "CholeskyQR breakdown";
    case BKFAC_ENOCONV: return "Jacobi eigensolver did not converge within its sweep cap";
    case BKFAC_ENONFINITE: return "non-finite value in an input or intermediate";
    case BKFAC_ETIMEOUT: return "bounded device wait timed out";
    case BKFAC_ECUDA: return "CUDA runtime error";
    case BKFAC_EWORKSPACE: return "workspace missing, misaligned or too small";
    case BKFAC_ENOMEM: return "host allocation failed";
    default: return "unknown error code";
  }
}

int bkfac_status(bkfac_stream_t stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BKFAC_ECUDA;
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, bkfac::g_status, sizeof(int)) != cudaSuccess) return BKFAC_ECUDA;
  const int zero = 0;
  if (cudaMemcpyToSymbol(bkfac::g_status, &zero, sizeof(int)) != cudaSuccess) return BKFAC_ECUDA;
  return v;
}

size_t bkfac_workspace_size(const bkfac_factor* f, int n, int op) {
  if (!valid_factor(f)) return 0;
  if (op == BKFAC_OP_UPDATE) {
    if (n < 1) return 0;
    const UpdatePlan cap = plan_update(f, n, f->r);
    // beyond the eigensolve's capacity at the full rank: no workspace size
    if (!jacobi_fits(cap.dense ? f->d : cap.N, cap.C, cap.b, cap.rows_pad, cap.pr.jt)) return 0;
    return cap.total;
  }
  if (op == BKFAC_OP_REORTH) {
    const ReorthPlan cap = plan_reorth(f, r_total(f));
    if (!jacobi_fits(r_total(f), cap.C, cap.b, cap.rows_pad, cap.pr.jt)) return 0;
    return cap.total;
  }
  return 0;
}

size_t bkfac_apply_workspace_size(const bkfac_factor* fA, const bkfac_factor* fG) {
  if (!valid_factor(fA) || !valid_factor(fG) || fA->dtype != fG->dtype) return 0;
  return plan_apply(fA, fG, r_total(fA), r_total(fG)).total;
}

int bkfac_init(bkfac_factor* f, const void* X, int64_t ldx, int n, void* ws, size_t ws_bytes,
               bkfac_stream_t stream) {
  return update_common(f, X, ldx, n, 0.0, ws, ws_bytes, (cudaStream_t)stream, true);
}

int bkfac_update(bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, void* ws, size_t ws_bytes,
                 bkfac_stream_t stream) {
  return update_common(f, X, ldx, n, rho, ws, ws_bytes, (cudaStream_t)stream, false);
}

int bkfac_set_sweep_cap(int cap) {
  if (cap < 0) return -BKFAC_EINVAL;
  return g_sweep_cap.exchange(cap == 0 ? kDefaultSweepCap : cap);
}

int bkfac_selftest_wait_timeout(int64_t limit_cycles, bkfac_stream_t stream) {
  if (limit_cycles < 1 || limit_cycles > (int64_t(1) << 31)) return BKFAC_EINVAL;
  return launch_wait_selftest((long long)limit_cycles, nullptr, (cudaStream_t)stream) == 0 ? BKFAC_OK : BKFAC_ECUDA;
}

int bkfac_reorth(bkfac_factor* f, void* ws, size_t ws_bytes, bkfac_stream_t stream) {
  if (!valid_factor(f)) return BKFAC_EINVAL;
  const int k = f->r_cur;
  if (k == 0) return BKFAC_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  const ReorthPlan cap = plan_reorth(f, r_total(f));
  const ReorthPlan p = plan_reorth(f, k);
  int rc = check_ws(ws, ws_bytes, cap.total);
  if (rc) return rc;
  if (p.rows_pad > cap.rows_cap || p.cols_pad > cap.cols_cap) return BKFAC_EINVAL;
  if (!jacobi_fits(k, p.C, p.b, p.rows_pad, p.pr.jt)) return BKFAC_EINVAL;
  const Prec& pr = p.pr;
  const int d = f->d;
  TraceScope _reorth_ts(PH_REORTH, s);
  double* Gm = at<double>(ws, cap.o_G);
  double* R = at<double>(ws, cap.o_R);
  void* Rinv = at<void>(ws, cap.o_Rinv);
  void* Q = at<void>(ws, cap.o_Q);
  BK_TRY(run_gram(f->U, f->ldu, d, k, pr, Gm, at<void>(ws, cap.o_part), s));
  BK_TRY(run_chol(Gm, k, R, (64.0 * pr.u_t) * (64.0 * pr.u_t), nullptr, 0.0, nullptr, s));
  BK_TRY(launch_trinv(R, k, Rinv, pr.t, nullptr, s));
  BK_TRY(run_trmm(f->U, f->ldu, d, k, Rinv, pr, Q, cap.ldq, nullptr, 0, s));
  void* Lm = at<void>(ws, cap.o_L);
  double* cn = at<double>(ws, cap.o_cn);
  BK_TRY(launch_assemble_reorth(R, f->sigma, k, p.rows_pad, p.cols_pad, Lm, cn, pr.jt, s));
  JacobiProblem jp;
  jp.W = Lm;
  jp.rows = k;
  jp.cols = k;
  jp.rows_pad = p.rows_pad;
  jp.cols_pad = p.cols_pad;
  jp.b = p.b;
  jp.colnorm2 = cn;
  jp.sweeps_out = at<int>(ws, cap.o_sw);
  jp.stamp = at<int>(ws, cap.o_st);
  BK_TRY(launch_jacobi(&jp, 1, p.C, pr.jt, jacobi_tol(k, pr.jt), sweep_cap(), s));
  SortArgs so;
  so.W = Lm;
  so.rows = k;
  so.rows_pad = p.rows_pad;
  so.cols = k;
  so.r_out = k;
  so.V = at<void>(ws, cap.o_V);
  so.ldv = cap.ldv;
  so.sig = f->sigma;
  so.r_sig = r_total(f);
  so.lam_sorted = at<double>(ws, cap.o_lam);
  so.colnorm2 = cn;
  so.cols_pad = p.cols_pad;
  BK_TRY(launch_sort_output(so, pr.jt, pr.t, s));
  GemmArgs g = gemm_base();
  g.M = d;
  g.N = k;
  g.K0 = k;
  g.A0 = Q;
  g.lda0 = cap.ldq;
  g.a_kmaj = false;
  g.B0 = so.V;
  g.ldb0 = cap.ldv;
  g.b_kmaj = true;
  g.C = at<void>(ws, cap.o_Un);
  g.ldc = cap.ldq;
  BK_TRY(gemm_run(g, pr.t, pr.acc, pr.t, s));
  BK_TRY(launch_finalize(f->U, f->ldu, g.C, cap.ldq, d, k, r_total(f), pr.t, s));
  return BKFAC_OK;
}

int bkfac_apply(const bkfac_factor* fA, const bkfac_factor* fG, double lamA, double lamG, const void* G,
                int64_t ldg, void* S, int64_t lds, uint32_t flags, void* ws, size_t ws_bytes,
                bkfac_stream_t stream) {
  if (!valid_factor(fA) || !valid_factor(fG) || fA->dtype != fG->dtype) return BKFAC_EINVAL;
  if (!G || !S || ldg < fA->d || lds < fA->d) return BKFAC_EINVAL;
  if (!(lamA > 0.0) || !(lamG > 0.0) || !std::isfinite(lamA) || !std::isfinite(lamG)) return BKFAC_EINVAL;
  if ((flags & ~(uint32_t)(BKFAC_SPECTRUM_CONTINUATION | BKFAC_DAMPING_RELATIVE)) != 0) return BKFAC_EINVAL;
  if ((flags & BKFAC_DAMPING_RELATIVE) && (fA->r_cur < 1 || fG->r_cur < 1)) return BKFAC_EINVAL;
  if (S == G && lds != ldg) return BKFAC_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  const int kA = fA->r_cur, kG = fG->r_cur;
  const ApplyPlan cap = plan_apply(fA, fG, r_total(fA), r_total(fG));
  const ApplyPlan p = plan_apply(fA, fG, kA, kG);
  int rc = check_ws(ws, ws_bytes, cap.total);
  if (rc) return rc;
  const Prec& pr = p.pr;
  const int dA = fA->d, dG = fG->d;
  void* T1 = at<void>(ws, cap.o_T1);
  void* W1 = at<void>(ws, cap.o_W1);
  void* T2 = at<void>(ws, cap.o_T2);
  void* T3 = at<void>(ws, cap.o_T3);
  double* cA = at<double>(ws, cap.o_cA);
  double* cG = at<double>(ws, cap.o_cG);
  double* cAo = at<double>(ws, cap.o_cAo);
  double* cGo = at<double>(ws, cap.o_cGo);
  double* alpha = at<double>(ws, cap.o_alpha);
  ApplyCoefArgs ca;
  ca.sigA = fA->sigma;
  ca.kA = kA;
  ca.sigG = fG->sigma;
  ca.kG = kG;
  ca.lamA = lamA;
  ca.lamG = lamG;
  ca.continuation = (flags & BKFAC_SPECTRUM_CONTINUATION) ? 1 : 0;
  ca.relative = (flags & BKFAC_DAMPING_RELATIVE) ? 1 : 0;
  ca.completeA = kA == dA ? 1 : 0;
  ca.completeG = kG == dG ? 1 : 0;
  ca.cA = cA;
  ca.cG = cG;
  ca.cA_over = cAo;
  ca.cG_over = cGo;
  ca.alpha = alpha;
  ca.betaA = nullptr;
  ca.betaG = nullptr;
  PHASE(PH_COEFS, launch_apply_coefs(ca, s));
  if (cap.tma) {
    // BF16 K-major copies: G and G^T from one read of G, the bases U_A and U_G
    void* Gb = at<void>(ws, cap.o_Gb);
    void* Gt = at<void>(ws, cap.o_Gt);
    void* UAb = at<void>(ws, cap.o_UAb);
    void* UGb = at<void>(ws, cap.o_UGb);
    PHASE(PH_APPLY1, launch_cvt_both((const float*)G, ldg, dG, dA, Gb, cap.ldgb, Gt, cap.ldgt, s));
    PHASE(PH_APPLY1, launch_cvt_cols((const float*)fA->U, fA->ldu, dA, kA, UAb, cap.ldua, s));
    PHASE(PH_APPLY1, launch_cvt_cols((const float*)fG->U, fG->ldu, dG, kG, UGb, cap.ldug, s));
    if (kA > 0) {  // T1 = G U_A: A = G (rows i, K = j), B = U_A (rows = modes, K = j)
      GemmArgs g = gemm_base();
      g.M = dG;
      g.N = kA;
      g.C = T1;
      g.ldc = cap.ld1;
      g.partial = at<void>(ws, cap.o_part1);
      g.partial_bytes = cap.part1_bytes;
      PHASE(PH_APPLY1, tma_gemm_run(Gb, cap.ldgb, UAb, cap.ldua, dA, g, s));
    }
    if (kG > 0) {  // T2 (d_in x kG column-major) = G^T U_G scaled by C_G / lamA': A = G^T, B = U_G
      GemmArgs g = gemm_base();
      g.M = dA;
      g.N = kG;
      g.C = T2;
      g.ldc = cap.ld2;
      g.cs = cGo;
      g.partial = at<void>(ws, cap.o_part1);
      g.partial_bytes = cap.part1_bytes;
      PHASE(PH_APPLY1, tma_gemm_run(Gt, cap.ldgt, UGb, cap.ldug, dG, g, s));
    }
  }
  // pass 1: T1 = G U_A (d_out x kA), T2 = diag(C_G / lamA') U_G^T G (kG x d_in, row-major)
  if (kA > 0 && !cap.tma) {
    GemmArgs g = gemm_base();
    g.M = dG;
    g.N = kA;
    g.K0 = dA;
    g.A0 = G;
    g.lda0 = ldg;
    g.a_kmaj = true;
    g.B0 = fA->U;
    g.ldb0 = fA->ldu;
    g.b_kmaj = true;
    g.round_bf16 = pr.bf16;
    g.tf32x3 = pr.x3;
    g.C = T1;
    g.ldc = cap.ld1;
    // (3xTF32 products keep pass 1's own scratch: more splits measured slower there)
    g.partial = at<void>(ws, pr.x3 ? cap.o_part1 : cap.o_pass1);
    g.partial_bytes = pr.x3 ? cap.part1_bytes : cap.pass1_bytes;
    PHASE(PH_APPLY1, gemm_run(g, pr.t, pr.acc, pr.t, s));
  }
  if (kG > 0 && !cap.tma) {
    GemmArgs g = gemm_base();
    g.M = dA;
    g.N = kG;
    g.K0 = dG;
    g.A0 = G;
    g.lda0 = ldg;
    g.a_kmaj = false;
    g.B0 = fG->U;
    g.ldb0 = fG->ldu;
    g.b_kmaj = true;
    g.round_bf16 = pr.bf16;
    g.tf32x3 = pr.x3;
    g.C = T2;  // column-major d_in x kG == row-major kG x d_in
    g.ldc = cap.ld2;
    g.cs = cGo;
    // (3xTF32 products keep pass 1's own scratch: more splits measured slower there)
    g.partial = at<void>(ws, pr.x3 ? cap.o_part1 : cap.o_pass1);
    g.partial_bytes = pr.x3 ? cap.part1_bytes : cap.pass1_bytes;
    PHASE(PH_APPLY1, gemm_run(g, pr.t, pr.acc, pr.t, s));
  }
  // small: T3' = diag(C_G) (U_G^T T1) diag(C_A);  W1 = T1 diag(C_A / lamG') + U_G T3'
  if (kA > 0) {
    if (kG > 0) {
      GemmArgs g = gemm_base();
      g.M = kG;
      g.N = kA;
      g.K0 = dG;
      g.A0 = fG->U;
      g.lda0 = fG->ldu;
      g.a_kmaj = true;
      g.B0 = T1;
      g.ldb0 = cap.ld1;
      g.b_kmaj = true;
      g.C = T3;
      g.ldc = cap.ldw;
      g.rs = cG;
      g.cs = cA;
      g.splits = gemm_pick_splits(kG, kA, dG, sm_count());
      g.partial = at<void>(ws, cap.o_part);
      g.partial_bytes = partial_bytes(r_total(fG), r_total(fA), dG, es_of(pr.acc));
      PHASE(PH_APPLY_SMALL, gemm_run(g, pr.t, pr.acc, pr.t, s));
    }
    GemmArgs g = gemm_base();
    g.M = dG;
    g.N = kA;
    g.K0 = kG;
    g.A0 = fG->U;
    g.lda0 = fG->ldu;
    g.a_kmaj = false;
    g.B0 = T3;
    g.ldb0 = cap.ldw;
    g.b_kmaj = true;
    g.C = W1;
    g.ldc = cap.ld1;
    g.D = T1;
    g.ldd = cap.ld1;
    g.beta = 1.0;
    g.ds = cAo;
    // pass 1's partial sums are reduced by now: their scratch lets this d_out x kA
    // product split its short K over more CTAs
    g.partial = at<void>(ws, cap.o_part1);
    g.partial_bytes = cap.part1_bytes;
    PHASE(PH_APPLY_SMALL, gemm_run(g, pr.t, pr.acc, pr.t, s));
  }
  // pass 2: S = alpha G + W1 U_A^T + U_G W2
  if (cap.tma) {
    // A2 = [W1 | U_G] (d_out x (kA + kG)) and B2 = [U_A | T2] (d_in x (kA + kG)), K-major BF16
    void* A2 = at<void>(ws, cap.o_A2);
    void* B2 = at<void>(ws, cap.o_B2);
    PHASE(PH_APPLY2, launch_cvt_cat_t((const float*)W1, cap.ld1, kA, (const float*)fG->U, fG->ldu, kG, dG, A2,
                                      cap.ld2k, s));
    PHASE(PH_APPLY2, launch_cvt_cat_t((const float*)fA->U, fA->ldu, kA, (const float*)T2, cap.ld2, kG, dA, B2,
                                      cap.ld2k, s));
    GemmArgs g = gemm_base();
    g.M = dG;
    g.N = dA;
    g.C = S;
    g.ldc = lds;
    g.c_rowmaj = true;
    g.D = G;
    g.ldd = ldg;
    g.beta_dev = alpha;
    g.beta = 1.0;
    PHASE(PH_APPLY2, tma_gemm_run(A2, cap.ld2k, B2, cap.ld2k, kA + kG, g, s));
  } else {
    GemmArgs g = gemm_base();
    g.M = dG;
    g.N = dA;
    g.K0 = kA;
    g.K1 = kG;
    g.A0 = W1;
    g.lda0 = cap.ld1;
    g.A1 = fG->U;
    g.lda1 = fG->ldu;
    g.a_kmaj = false;
    g.B0 = fA->U;
    g.ldb0 = fA->ldu;
    g.B1 = T2;
    g.ldb1 = cap.ld2;
    g.b_kmaj = false;
    g.round_bf16 = pr.bf16;
    g.tf32x3 = pr.x3;
    g.C = S;
    g.ldc = lds;
    g.c_rowmaj = true;
    g.D = G;
    g.ldd = ldg;
    g.beta_dev = alpha;
    g.beta = 1.0;
    PHASE(PH_APPLY2, gemm_run(g, pr.t, pr.acc, pr.t, s));
  }
  return BKFAC_OK;
}

size_t bkfac_apply_factored_workspace_size(const bkfac_factor* fA, const bkfac_factor* fG, int n) {
  if (!valid_factor(fA) || !valid_factor(fG) || fA->dtype != fG->dtype || n < 1) return 0;
  return plan_factored(fA, fG, n).total;
}

// Algorithm 8: the damped inverses on the thin factors, then (optionally) the step.
//   T = diag(C) (U^T X)  (r_cur x n, split K over d);   P = beta X + U T  (d x n)
//   S = alpha PG PA^T
int bkfac_apply_factored(const bkfac_factor* fA, const bkfac_factor* fG, double lamA, double lamG, const void* XA,
                         int64_t ldxa, const void* XG, int64_t ldxg, int n, void* PA, int64_t ldpa, void* PG,
                         int64_t ldpg, double alpha, void* S, int64_t lds, uint32_t flags, void* ws,
                         size_t ws_bytes, bkfac_stream_t stream) {
  if (!valid_factor(fA) || !valid_factor(fG) || fA->dtype != fG->dtype || n < 1) return BKFAC_EINVAL;
  if (!(lamA > 0.0) || !(lamG > 0.0) || !std::isfinite(lamA) || !std::isfinite(lamG)) return BKFAC_EINVAL;
  if ((flags & ~(uint32_t)(BKFAC_SPECTRUM_CONTINUATION | BKFAC_DAMPING_RELATIVE)) != 0) return BKFAC_EINVAL;
  if ((flags & BKFAC_DAMPING_RELATIVE) && (fA->r_cur < 1 || fG->r_cur < 1)) return BKFAC_EINVAL;
  const int dA = fA->d, dG = fG->d;
  if (!XA || !XG || !PA || !PG || ldxa < dA || ldxg < dG || ldpa < dA || ldpg < dG) return BKFAC_EINVAL;
  const size_t es = fA->dtype == BKFAC_F64 ? 8 : 4;
  for (const void* ptr : {XA, XG, (const void*)PA, (const void*)PG})
    if (((uintptr_t)ptr) % 16 != 0) return BKFAC_EINVAL;
  for (int64_t ld : {ldxa, ldxg, ldpa, ldpg})
    if ((ld * (int64_t)es) % 16 != 0) return BKFAC_EINVAL;
  if ((PA == XA && ldpa != ldxa) || (PG == XG && ldpg != ldxg)) return BKFAC_EINVAL;
  if (S && (lds < dA || !std::isfinite(alpha))) return BKFAC_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  const int kA = fA->r_cur, kG = fG->r_cur;
  const FactoredPlan p = plan_factored(fA, fG, n);
  int rc = check_ws(ws, ws_bytes, p.total);
  if (rc) return rc;
  const Prec& pr = p.pr;
  ApplyCoefArgs ca;
  ca.sigA = fA->sigma;
  ca.kA = kA;
  ca.sigG = fG->sigma;
  ca.kG = kG;
  ca.lamA = lamA;
  ca.lamG = lamG;
  ca.continuation = (flags & BKFAC_SPECTRUM_CONTINUATION) ? 1 : 0;
  ca.relative = (flags & BKFAC_DAMPING_RELATIVE) ? 1 : 0;
  ca.completeA = kA == dA ? 1 : 0;
  ca.completeG = kG == dG ? 1 : 0;
  ca.cA = at<double>(ws, p.o_cA);
  ca.cG = at<double>(ws, p.o_cG);
  ca.cA_over = at<double>(ws, p.o_cAo);
  ca.cG_over = at<double>(ws, p.o_cGo);
  ca.alpha = at<double>(ws, p.o_alpha);
  ca.betaA = at<double>(ws, p.o_bA);
  ca.betaG = at<double>(ws, p.o_bG);
  PHASE(PH_COEFS, launch_apply_coefs(ca, s));
  struct Side {
    const bkfac_factor* f;
    int k;
    const void* X;
    int64_t ldx;
    void* P;
    int64_t ldp;
    void* T;
    int64_t ldt;
    const double* c;
    const double* beta;
  };
  const Side sides[2] = {
      {fA, kA, XA, ldxa, PA, ldpa, at<void>(ws, p.o_TA), p.ldtA, ca.cA, ca.betaA},
      {fG, kG, XG, ldxg, PG, ldpg, at<void>(ws, p.o_TG), p.ldtG, ca.cG, ca.betaG},
  };
  for (const Side& sd : sides) {
    const int d = sd.f->d;
    if (sd.k > 0) {
      // T = diag(C) U^T X  (k x n, K = d)
      GemmArgs g = gemm_base();
      g.M = sd.k;
      g.N = n;
      g.K0 = d;
      g.A0 = sd.f->U;
      g.lda0 = sd.f->ldu;
      g.a_kmaj = true;
      g.B0 = sd.X;
      g.ldb0 = sd.ldx;
      g.b_kmaj = true;
      g.round_bf16 = pr.bf16;
      g.tf32x3 = pr.x3;
      g.C = sd.T;
      g.ldc = sd.ldt;
      g.rs = sd.c;
      g.splits = gemm_pick_splits(sd.k, n, d, sm_count());
      g.partial = at<void>(ws, p.o_part);
      g.partial_bytes = p.part_bytes;
      PHASE(PH_FACT_THIN, gemm_run(g, pr.t, pr.acc, pr.t, s));
    }
    // P = U T + beta X  (d x n, K = k; the epilogue reads X(i, j) before writing P(i, j),
    // so P may be X)
    GemmArgs g = gemm_base();
    g.M = d;
    g.N = n;
    g.K0 = sd.k;
    g.A0 = sd.f->U;
    g.lda0 = sd.f->ldu;
    g.a_kmaj = false;
    g.B0 = sd.T;
    g.ldb0 = sd.ldt;
    g.b_kmaj = true;
    g.round_bf16 = pr.bf16;
    g.tf32x3 = pr.x3;
    g.C = sd.P;
    g.ldc = sd.ldp;
    g.D = sd.X;
    g.ldd = sd.ldx;
    g.beta = 1.0;
    g.beta_dev = sd.beta;
    PHASE(PH_FACT_THIN, gemm_run(g, pr.t, pr.acc, pr.t, s));
  }
  if (S) {
    // S = alpha PG PA^T  (d_out x d_in row-major, K = n)
    GemmArgs g = gemm_base();
    g.M = dG;
    g.N = dA;
    g.K0 = n;
    g.A0 = PG;
    g.lda0 = ldpg;
    g.a_kmaj = false;
    g.B0 = PA;
    g.ldb0 = ldpa;
    g.b_kmaj = false;
    g.round_bf16 = pr.bf16;
    g.tf32x3 = pr.x3;
    g.C = S;
    g.ldc = lds;
    g.c_rowmaj = true;
    g.alpha = alpha;
    PHASE(PH_FACT_STEP, gemm_run(g, pr.t, pr.acc, pr.t, s));
  }
  return BKFAC_OK;
}

int bkfac_ea_update(int d, int dtype, void* M, int64_t ldm, const void* X, int64_t ldx, int n, double rho,
                    int first, bkfac_stream_t stream) {
  if (d < 1 || n < 1 || !M || !X || ldm < d || ldx < d) return BKFAC_EINVAL;
  if (dtype != BKFAC_F64 && dtype != BKFAC_F32 && dtype != BKFAC_MIXED_BF16) return BKFAC_EINVAL;
  if (!first && !(rho >= 0.0 && rho < 1.0)) return BKFAC_EINVAL;
  const size_t es = dtype == BKFAC_F64 ? 8 : 4;
  if (((uintptr_t)M) % 16 != 0 || ((uintptr_t)X) % 16 != 0 || (ldm * (int64_t)es) % 16 != 0 ||
      (ldx * (int64_t)es) % 16 != 0)
    return BKFAC_EINVAL;
  const cudaStream_t s = (cudaStream_t)stream;
  bkfac_factor probe{};
  probe.dtype = dtype;
  const Prec pr = prec_of(&probe);
  // M = keep * M + c * X X^T; the epilogue reads M(i, j) before writing it.  M is
  // symmetric, so it is written (and read) as its row-major transpose: whole rows
  // of the output tile go out coalesced
  GemmArgs g = gemm_base();
  g.M = d;
  g.N = d;
  g.K0 = n;
  g.A0 = X;
  g.lda0 = ldx;
  g.a_kmaj = false;
  g.B0 = X;
  g.ldb0 = ldx;
  g.b_kmaj = false;
  g.round_bf16 = pr.bf16;
  g.tf32x3 = pr.x3;
  g.C = M;
  g.ldc = ldm;
  g.c_rowmaj = true;
  g.D = first ? nullptr : M;
  g.ldd = ldm;
  g.alpha = first ? 1.0 / n : (1.0 - rho) / n;
  g.beta = first ? 0.0 : rho;
  PHASE(PH_DENSE, gemm_run(g, pr.t, pr.acc, pr.t, s));
  return BKFAC_OK;
}

size_t bkfac_correct_workspace_size(const bkfac_factor* f, int n_crc) {
  if (!valid_factor(f) || n_crc < 1) return 0;
  const CorrectPlan p = plan_correct(f, n_crc);
  if (!small_evd_fits(p.e, p.pr)) return 0;
  return p.total;
}

int bkfac_correct(bkfac_factor* f, const void* M, int64_t ldm, const int32_t* idx, int n_crc, void* ws,
                  size_t ws_bytes, bkfac_stream_t stream) {
  if (!valid_factor(f) || !M || !idx || n_crc < 1 || n_crc > f->r_cur || ldm < f->d) return BKFAC_EINVAL;
  const size_t es = f->dtype == BKFAC_F64 ? 8 : 4;
  if (((uintptr_t)M) % 16 != 0 || (ldm * (int64_t)es) % 16 != 0) return BKFAC_EINVAL;
  {
    std::vector<char> seen((size_t)f->r_cur, 0);
    for (int a = 0; a < n_crc; ++a) {
      if (idx[a] < 0 || idx[a] >= f->r_cur || seen[(size_t)idx[a]]) return BKFAC_EINVAL;
      seen[(size_t)idx[a]] = 1;
    }
  }
  const CorrectPlan p = plan_correct(f, n_crc);
  if (!small_evd_fits(p.e, p.pr)) return BKFAC_EINVAL;
  int rc = check_ws(ws, ws_bytes, p.total);
  if (rc) return rc;
  const cudaStream_t s = (cudaStream_t)stream;
  const Prec& pr = p.pr;
  const int d = f->d;
  int* didx = at<int>(ws, p.o_idx);
  void* Us = at<void>(ws, p.o_Us);
  void* W = at<void>(ws, p.o_W);
  double* Ms = at<double>(ws, p.o_Ms);
  void* part = at<void>(ws, p.o_part);
  if (cudaMemcpyAsync(didx, idx, (size_t)n_crc * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return BKFAC_ECUDA;
  // U_s = U[:, idx];  M_S = U_s^T (M U_s)  (FP64 accumulation)
  PHASE(PH_PROJ, launch_gather_cols(f->U, f->ldu, Us, p.ldq, d, n_crc, didx, pr.t, s));
  PHASE(PH_PROJ, run_dense_times(M, ldm, d, Us, p.ldq, n_crc, W, p.ldq, pr, part, p.part_bytes, s));
  PHASE(PH_GRAM, run_cross_f64(Us, p.ldq, W, p.ldq, d, n_crc, Ms, pr, part, s));
  // M_S = V diag(lam) V^T;  U[:, idx] = U_s V, sigma[idx] = lam
  const int erc = run_small_evd(Ms, p.e, pr, (64.0 * pr.u_t) * (64.0 * pr.u_t), ws, s);
  if (erc) return erc;
  PHASE(PH_ROTATE, run_rotate(Us, p.ldq, d, n_crc, at<void>(ws, p.e.o_V), p.e.ldv, n_crc, W, p.ldq, pr, part,
                              p.part_bytes, s));
  PHASE(PH_FINALIZE, launch_scatter_cols(W, p.ldq, f->U, f->ldu, d, n_crc, didx, at<double>(ws, p.e.o_lam),
                                         f->sigma, pr.t, s));
  return resort_modes(f, at<int>(ws, p.o_perm), at<double>(ws, p.o_sorted), at<void>(ws, p.o_Ut), p.ldq, pr, s);
}

size_t bkfac_rsvd_workspace_size(const bkfac_factor* f, int l) {
  if (!valid_factor(f) || l < f->r || l > f->d) return 0;
  const RsvdPlan p = plan_rsvd(f, l);
  if (!small_evd_fits(p.e, p.pr)) return 0;
  return p.total;
}

int bkfac_rsvd(bkfac_factor* f, const void* M, int64_t ldm, const void* Omega, int64_t ldo, int l, int q, void* ws,
               size_t ws_bytes, bkfac_stream_t stream) {
  if (!valid_factor(f) || !M || !Omega || ldm < f->d || ldo < f->d || l < f->r || l > f->d || q < 0 || q > 64)
    return BKFAC_EINVAL;
  const size_t es = f->dtype == BKFAC_F64 ? 8 : 4;
  if (((uintptr_t)M) % 16 != 0 || ((uintptr_t)Omega) % 16 != 0 || (ldm * (int64_t)es) % 16 != 0 ||
      (ldo * (int64_t)es) % 16 != 0)
    return BKFAC_EINVAL;
  const RsvdPlan p = plan_rsvd(f, l);
  if (!small_evd_fits(p.e, p.pr)) return BKFAC_EINVAL;
  int rc = check_ws(ws, ws_bytes, p.total);
  if (rc) return rc;
  const cudaStream_t s = (cudaStream_t)stream;
  const Prec& pr = p.pr;
  const int d = f->d, r = f->r;
  void* Y = at<void>(ws, p.o_Y);
  void* Q = at<void>(ws, p.o_Q);
  void* part = at<void>(ws, p.o_part);
  // Y = M Omega; q power iterations Y = M orth(Y); Q = orth(Y); B = Q^T M Q
  PHASE(PH_PROJ, run_dense_times(M, ldm, d, Omega, ldo, l, Y, p.ldq, pr, part, p.part_bytes, s));
  for (int it = 0; it < q; ++it) {
    rc = run_orth(Y, d, l, p, ws, Q, s);
    if (rc) return rc;
    PHASE(PH_PROJ, run_dense_times(M, ldm, d, Q, p.ldq, l, Y, p.ldq, pr, part, p.part_bytes, s));
  }
  rc = run_orth(Y, d, l, p, ws, Q, s);
  if (rc) return rc;
  PHASE(PH_PROJ, run_dense_times(M, ldm, d, Q, p.ldq, l, Y, p.ldq, pr, part, p.part_bytes, s));
  double* B = at<double>(ws, p.o_G);
  PHASE(PH_GRAM, run_cross_f64(Q, p.ldq, Y, p.ldq, d, l, B, pr, part, s));
  rc = run_small_evd(B, p.e, pr, (64.0 * pr.u_t) * (64.0 * pr.u_t), ws, s);
  if (rc) return rc;
  // U = Q V[:, :r], sigma = lam[:r] (the rest of the representation cleared)
  PHASE(PH_ROTATE, run_rotate(Q, p.ldq, d, l, at<void>(ws, p.e.o_V), p.e.ldv, r, Y, p.ldq, pr, part, p.part_bytes,
                              s));
  PHASE(PH_FINALIZE, launch_finalize(f->U, f->ldu, Y, p.ldq, d, r, r_total(f), pr.t, s));
  if (cudaMemsetAsync(f->sigma, 0, (size_t)r_total(f) * 8, s) != cudaSuccess ||
      cudaMemcpyAsync(f->sigma, at<double>(ws, p.e.o_lam), (size_t)r * 8, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return BKFAC_ECUDA;
  f->r_cur = r;
  return BKFAC_OK;
}

int bkfac_debug_offsets(const bkfac_factor* f, int n, int64_t out[8]) {
  if (!valid_factor(f) || n < 1 || !out) return BKFAC_EINVAL;
  if (dense_path(f, n)) return BKFAC_EINVAL;
  const UpdatePlan p = plan_update(f, n, f->r);
  out[0] = (int64_t)p.o_M;
  out[1] = (int64_t)p.o_Q;
  out[2] = (int64_t)p.o_L;
  out[3] = (int64_t)p.o_lam;
  out[4] = (int64_t)p.o_P;
  out[5] = p.ldm;
  out[6] = p.ldq;
  out[7] = (int64_t)p.o_sw;
  return BKFAC_OK;
}

}  // extern "C"

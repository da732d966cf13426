/*
 * bkfac.h -- C ABI of libbkfac, the GB300 (sm_103a) B-KFAC preconditioning
 * hot path.
 *
 * Paper: "Brand New K-FACs: Speeding up K-FAC with Online Decomposition
 * Updates", arXiv 2210.08494.
 *
 * The library keeps each exponentially averaged (EA) Kronecker factor of an FC
 * layer (Eq. (5)) as a low-rank eigendecomposition U diag(sigma) U^T and
 *   - updates it with a new batch of columns X by the symmetric Brand update
 *     (Algorithm 3) as used by B-KFAC (Algorithm 4, Sec. 3.1):
 *       K = rho * U diag(sigma) U^T + (1 - rho)/n * X X^T,
 *       (U, sigma) <- top-r eigenpairs of K;
 *   - applies the damped inverse of both factors of a layer to its weight
 *     gradient (Algorithm 1, inverse application; K-FAC identity of Eq. (4)):
 *       S = (Gamma + lam_G I)^-1 G (A + lam_A I)^-1.
 *
 * Conventions
 *   - Every pointer documented as "device" must point to memory of the
 *     current CUDA device; "host" pointers are read during the call only.
 *   - Calls are asynchronous on the caller's stream (NULL = legacy default
 *     stream).  Argument errors are returned immediately and enqueue nothing.
 *     Errors found on the device (non-convergence, non-finite data, a
 *     Cholesky breakdown) are written to a per-device status word that
 *     bkfac_status() returns; kernels never trap.
 *   - The per-factor calls allocate no memory: the caller passes a workspace
 *     of at least the size the matching *_workspace_size() function returns,
 *     256-byte aligned.  Workspace contents need not be initialised and are
 *     not meaningful after the call.  Two calls that run concurrently must not
 *     share a workspace.
 *   - Matrices: a "d x m column-major" matrix with leading dimension ld stores
 *     element (i, j) at p[i + j*ld]; this is exactly a row-major torch tensor
 *     of shape (m, ld) viewed as m columns.  The gradient G and the step S are
 *     "d_out x d_in row-major" (element (i, j) at p[i*ld + j]), the layout of
 *     torch's weight.grad with the bias column appended last.
 *   - Leading dimensions must be >= the row count and a multiple of 4
 *     elements (16 bytes for FP32) so rows can be read with vector loads;
 *     base pointers must be 16-byte aligned.
 */
#ifndef BKFAC_H
#define BKFAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st* bkfac_stream_t;

/* ---- precision modes ----------------------------------------------------
 * BKFAC_F64        U, X, G, S in double; all arithmetic in FP64.
 * BKFAC_F32        U, X, G, S in float; tall-skinny products in FP32; the
 *                  CholeskyQR Gram FP64-accurate (exact FP32 products with
 *                  compensated FP32 sums), its Cholesky factorisations in FP32
 *                  (FP64 with BKFAC_FLAG_CHOL_FP64); core eigensolve in FP32
 *                  (FP64 with BKFAC_FLAG_EIG_FP64).
 * BKFAC_MIXED_BF16 U (master copy), X, G, S in float; the tall-skinny
 *                  products (U^T X, U M, [U Q] V, G U, U^T G and the apply
 *                  expansion) take BF16-rounded operands with FP32
 *                  accumulation; Gram, Cholesky and eigensolve as in
 *                  BKFAC_F32 (the same two flags select FP64); periodic
 *                  re-orthonormalisation (bkfac_reorth: FP64-accurate Gram,
 *                  FP64 Cholesky) restores U^T U = I. */
enum { BKFAC_F64 = 0, BKFAC_F32 = 1, BKFAC_MIXED_BF16 = 2 };

/* ---- return / status codes --------------------------------------------- */
enum {
  BKFAC_OK = 0,
  BKFAC_EINVAL = 1,         /* bad argument: sizes, ld, alignment, r > d, n <= 0 */
  BKFAC_ENOTAPPLICABLE = 2, /* (reserved) a path was requested that the shapes do not allow */
  BKFAC_ECHOL = 3,          /* a matrix that must be positive semidefinite is not: a Cholesky pivot
                               below -1e-2 times its largest diagonal entry (the dense factor M of
                               bkfac_correct / bkfac_rsvd is indefinite) */
  BKFAC_ENOCONV = 4,        /* Jacobi eigensolver hit its sweep cap */
  BKFAC_ENONFINITE = 5,     /* NaN or Inf met in an input or an intermediate */
  BKFAC_ETIMEOUT = 6,       /* a bounded device-side wait gave up */
  BKFAC_ECUDA = 7,          /* a CUDA runtime call failed */
  BKFAC_EWORKSPACE = 8,     /* workspace pointer NULL, misaligned or too small */
  BKFAC_ENOMEM = 9          /* host-side allocation failed (batch handles only) */
};

/* ---- factor flags ------------------------------------------------------- */
#define BKFAC_FLAG_EIG_FP64 (1u << 0) /* core eigensolve in FP64 also in F32 / MIXED modes */
#define BKFAC_FLAG_TF32X3 (1u << 1)   /* F32 mode: the tall-skinny products (U^T X, U M, [U Q] V and
                                         the inverse application's passes) on the tensor cores as
                                         3xTF32 (hi/lo split, FP32 accumulation; relative error of a
                                         product ~1e-5 at K = 4096 instead of ~1e-7); the apply takes
                                         it when either factor carries it */
#define BKFAC_FLAG_KEEP_RN (1u << 2)  /* truncate just before the next update instead of just after
                                         this one (the order of Algorithm 4): after an update the
                                         factor keeps up to r + r_extra modes, so the inverse
                                         applications use the rank-(r + n) representation; the next
                                         update starts from the leading r of them */
#define BKFAC_FLAG_CHOL_FP64 (1u << 3) /* F32 / MIXED modes: the Cholesky factorisations of CholeskyQR2
                                          in FP64 (the FP64 path's kernel) instead of FP32 */

/* ---- apply flags -------------------------------------------------------- */
#define BKFAC_SPECTRUM_CONTINUATION (1u << 0) /* Sec. 3.5.1: lam += min sigma, sigma -= min sigma */
#define BKFAC_DAMPING_RELATIVE (1u << 1)      /* the damping schedule of the experiments (Sec. 4): lam_A,
                                                 lam_G are multiples phi of each factor's largest stored
                                                 eigenvalue, lambda = phi * max sigma (before any
                                                 continuation shift); needs r_cur >= 1 on both factors */

/* ---- the low-rank factor state (Sec. 3.1: U~ in R^{d x r}, D~ diagonal) --
 * All buffers are caller-owned device memory.
 *   d      factor size (d_in + 1 for the forward factor A, d_out for Gamma)
 *   r      target rank, 1 <= r <= d
 *   r_cur  current rank (0 before bkfac_init); maintained by the library on
 *          the host: after an update r_cur = min(r_out, k + n) (Brand path) or
 *          min(r_out, k + n, d) (dense path), with k = min(r_cur, r) the modes
 *          the update starts from and r_out = r (or r + r_extra under
 *          BKFAC_FLAG_KEEP_RN).  Modes past the numerical rank hold sigma = 0
 *          and may have a zero column in U.
 *   dtype  BKFAC_F64 (U is double) or BKFAC_F32 / BKFAC_MIXED_BF16 (U float)
 *   U      device, d x r_out column-major, leading dimension ldu
 *   sigma  device, r_out doubles, eigenvalues in descending order (zero past r_cur)
 *   step   number of updates applied so far (host counter, incremented by
 *          bkfac_init / bkfac_update)
 *   flags  BKFAC_FLAG_* bits
 *   r_extra  with BKFAC_FLAG_KEEP_RN: columns U and sigma hold beyond r (the
 *          largest n the factor is updated with keeps all r + n modes);
 *          ignored (0) otherwise
 * The dense path (explicit d x d factor, Jacobi on its Gram factor) is used
 * when r + n >= d, where the symmetric Brand update's precondition r + n < d
 * (Algorithm 3) fails. */
typedef struct bkfac_factor {
  int32_t d;
  int32_t r;
  int32_t r_cur;
  int32_t dtype;
  void* U;
  int64_t ldu;
  double* sigma;
  int64_t step;
  uint32_t flags;
  int32_t r_extra;
} bkfac_factor;

/* Library version (major * 10000 + minor * 100 + patch). */
int bkfac_version(void);

/* Human-readable text for a code above (static storage, never NULL). */
const char* bkfac_strerror(int code);

/* Synchronises `stream`, then returns and clears the current device's status
 * word: BKFAC_OK or the first device-side error code recorded since the last
 * call.  Returns BKFAC_ECUDA if the synchronisation itself fails. */
int bkfac_status(bkfac_stream_t stream);

/* ---- fault handling (not in the paper; for tests and operators) ----------
 * bkfac_set_sweep_cap(cap)  Jacobi sweep cap of every later eigensolve in the
 *     process (cap >= 1; 0 restores the default of 40).  An eigensolve that
 *     reaches the cap records BKFAC_ENOCONV in the status word and still
 *     returns its current columns.  Returns the previous cap, or
 *     -BKFAC_EINVAL for cap < 0.  Not meant to change while other host
 *     threads enqueue updates.
 * bkfac_selftest_wait_timeout(limit_cycles, stream)  launches one thread that
 *     waits, with the bounded mbarrier wait the eigensolve's block exchange
 *     uses, on a barrier phase that nothing completes; after limit_cycles SM
 *     clock cycles (1 .. 2^31) it gives up, records BKFAC_ETIMEOUT and returns,
 *     so that the context stays usable.  Returns BKFAC_EINVAL for a limit out
 *     of range. */
int bkfac_set_sweep_cap(int cap);
int bkfac_selftest_wait_timeout(int64_t limit_cycles, bkfac_stream_t stream);

/* ---- workspace sizes ----------------------------------------------------- */
enum { BKFAC_OP_UPDATE = 0, BKFAC_OP_REORTH = 1 };

/* Bytes of workspace bkfac_init / bkfac_update (op = BKFAC_OP_UPDATE, with
 * batch width n) or bkfac_reorth (op = BKFAC_OP_REORTH, n ignored) need for
 * factor f.  Returns 0 for invalid arguments and for shapes beyond the
 * eigensolve's capacity at the full rank: its matrix (N = r + n rows and
 * columns on the Brand path, d rows and r + n columns on the dense path, r x r
 * for reorth) may have at most 1024 rows with an FP32 eigensolve (768 columns
 * once there are more than 512 rows) and 512 rows with an FP64 one; the calls
 * return BKFAC_EINVAL for such shapes. */
size_t bkfac_workspace_size(const bkfac_factor* f, int n, int op);

/* Bytes of workspace bkfac_apply needs for the factor pair (fA, fG). */
size_t bkfac_apply_workspace_size(const bkfac_factor* fA, const bkfac_factor* fG);

/* ---- per-factor calls ---------------------------------------------------- */

/* First state of a factor from its first batch (kappa(0) = 1 in Eq. (5)):
 * U diag(sigma) U^T <- top-r eigenpairs of X X^T / n, i.e. the update below
 * from r_cur = 0 with rho = 0.  Sets r_cur = min(r, n) (min(r, n, d) on the
 * dense path) and step = 1.
 *   X    device, d x n column-major, leading dimension ldx >= d (the
 *        factor's dtype: double for F64, float otherwise)
 *   ws   device workspace of bkfac_workspace_size(f, n, BKFAC_OP_UPDATE) bytes */
int bkfac_init(bkfac_factor* f, const void* X, int64_t ldx, int n, void* ws, size_t ws_bytes,
               bkfac_stream_t stream);

/* One B-KFAC update (Algorithm 4 via Algorithm 3, truncation after the
 * update): with c = (1 - rho)/n,
 *   M = U^T X;  P = X - U M;  Q R = P (CholeskyQR2, pivots below a relative
 *   threshold dropped);  M_S = [[rho diag(sigma) + c M M^T, c M R^T],
 *   [c R M^T, c R R^T]] (Eq. (7) with the substitutions of Sec. 3.1);
 *   M_S = V diag(lambda) V^T;  U <- [U Q] V[:, :r_new];  sigma <- lambda[:r_new].
 * The eigensolve runs as one-sided Jacobi on the factor
 * L = [[diag(sqrt(rho sigma)), sqrt(c) M], [0, sqrt(c) R]] (M_S = L L^T).
 * U and sigma are overwritten in place; r_cur and step are advanced on the
 * host.  0 <= rho < 1.  Requires r_cur >= 1 (call bkfac_init first). */
int bkfac_update(bkfac_factor* f, const void* X, int64_t ldx, int n, double rho, void* ws, size_t ws_bytes,
                 bkfac_stream_t stream);

/* Re-orthonormalisation of U (not in the paper; numerical hygiene for the
 * mixed-precision path): Q R = U by CholeskyQR in FP64, R diag(sigma) R^T =
 * W diag(lambda) W^T by Jacobi, U <- Q W, sigma <- lambda.  The represented
 * matrix U diag(sigma) U^T is unchanged up to rounding. */
int bkfac_reorth(bkfac_factor* f, void* ws, size_t ws_bytes, bkfac_stream_t stream);

/* Damped inverse application to one layer's gradient (Algorithm 1):
 *   S = (U_G C_G U_G^T + I/lam_G) G (U_A C_A U_A^T + I/lam_A),
 *   C = diag(1/(sigma + lam) - 1/lam) over the r_cur stored modes.
 * A factor whose basis is complete (r_cur == d, e.g. a dense-path factor)
 * has no complement: its side is applied as U diag(1/(sigma + lam)) U^T, the
 * same operator in exact arithmetic, without the 1/lam identity term (whose
 * cancellation against U C U^T a rounded basis would not reproduce).
 * Computed in two passes over G:
 *   pass 1  T1 = G U_A (d_out x r_A), T2 = U_G^T G (r_G x d_in);
 *   small   T3 = U_G^T T1, W1 = T1 C_A / lam_G + U_G (C_G T3 C_A), W2 = C_G T2 / lam_A;
 *   pass 2  S = G / (lam_A lam_G) + W1 U_A^T + U_G W2.
 *   fA, fG  the layer's forward (d = d_in) and backward (d = d_out) factors,
 *           same dtype, both with r_cur >= 0
 *   G       device, d_out x d_in row-major, leading dimension ldg >= d_in
 *   S       device, same layout, lds >= d_in; S == G (in place) is allowed
 *           when lds == ldg
 *   lamA, lamG  damping, > 0
 *   flags   BKFAC_SPECTRUM_CONTINUATION, BKFAC_DAMPING_RELATIVE (either, both or 0) */
int bkfac_apply(const bkfac_factor* fA, const bkfac_factor* fG, double lamA, double lamG, const void* G,
                int64_t ldg, void* S, int64_t lds, uint32_t flags, void* ws, size_t ws_bytes,
                bkfac_stream_t stream);

/* Linear inverse application (Algorithm 8): when a layer's weight gradient
 * is alpha * G_f A_f^T -- G_f (d_out x n) the back-propagated columns and A_f
 * (d_in x n) the input columns of the batch, the same matrices whose outer
 * products feed the K-factor updates -- the damped inverses act on the thin
 * factors instead of a dense gradient:
 *   PA = (U_A C_A U_A^T + I/lam_A) A_f     (d_in x n)
 *   PG = (U_G C_G U_G^T + I/lam_G) G_f     (d_out x n)
 *   S  = alpha * PG PA^T                   (optional, d_out x d_in)
 * with C and the complete-basis rule as in bkfac_apply; S equals bkfac_apply
 * on G = alpha * G_f A_f^T.  Work is O(n r (d_in + d_out)) for PA and PG and
 * 2 n d_in d_out for S; no dense gradient is read.
 *   XA, XG  device, column-major d_in x n / d_out x n (a torch (n, d) row-major
 *           tensor), leading dimensions ldxa >= d_in, ldxg >= d_out; 16-byte
 *           aligned base and leading dimension (in bytes)
 *   PA, PG  device outputs, same layouts and alignment (ldpa >= d_in,
 *           ldpg >= d_out); PA == XA (PG == XG) in place is allowed when the
 *           leading dimensions agree
 *   alpha   scale of the step (1/n for a mean-reduced loss with unscaled
 *           columns); ignored when S is NULL
 *   S       device, d_out x d_in row-major, lds >= d_in, or NULL to return only
 *           PA and PG; must not overlap XA, XG, PA or PG
 *   ws      bkfac_apply_factored_workspace_size(fA, fG, n) bytes
 *   flags   as bkfac_apply
 * Returns BKFAC_EINVAL for n < 1, bad leading dimensions or alignment, or
 * non-positive damping. */
size_t bkfac_apply_factored_workspace_size(const bkfac_factor* fA, const bkfac_factor* fG, int n);
int bkfac_apply_factored(const bkfac_factor* fA, const bkfac_factor* fG, double lamA, double lamG, const void* XA,
                         int64_t ldxa, const void* XG, int64_t ldxg, int n, void* PA, int64_t ldpa, void* PG,
                         int64_t ldpg, double alpha, void* S, int64_t lds, uint32_t flags, void* ws,
                         size_t ws_bytes, bkfac_stream_t stream);

/* ---- B-R-KFAC and B-KFAC-C: the dense EA factor beside the representation --
 * These variants keep the dense EA K-factor M (d x d) as well, to overwrite
 * (Algorithm 5) or correct (Algorithm 6) the low-rank representation now and
 * then.  M is column-major with leading dimension ldm >= d, in the element
 * type of dtype (double for BKFAC_F64, float otherwise), 16-byte aligned base
 * and leading dimension.
 *
 * Dense EA factor update (Eq. (5) / (8)): M = rho M + (1 - rho)/n X X^T, or
 * M = X X^T / n when first != 0 (kappa(0) = 1).  X is d x n column-major
 * (the layout of bkfac_update's X).  In BKFAC_MIXED_BF16 the product takes
 * BF16-rounded operands with FP32 accumulation.  Work 2 d^2 n flops, traffic
 * 2 d^2 elements (read and write M). */
int bkfac_ea_update(int d, int dtype, void* M, int64_t ldm, const void* X, int64_t ldx, int n, double rho,
                    int first, bkfac_stream_t stream);

/* Light correction of the representation (Algorithm 6, B-KFAC-C): for the
 * n_crc distinct modes idx[0..n_crc) (0 <= idx < r_cur; a host array, drawn
 * at random by the caller -- the paper picks them without replacement),
 *   U_s = U[:, idx],  M_S = U_s^T M U_s = W diag(lam) W^T,
 *   U[:, idx] = U_s W,  sigma[idx] = lam,
 * then all r_cur modes are re-sorted by decreasing sigma (stable), so the
 * representation keeps its order for the next truncation.  M_S is
 * accumulated in FP64 and factored as M_S = R^T R (FP64 Cholesky) for the
 * one-sided Jacobi eigensolve.  The copy of idx into the workspace is a
 * host-to-device copy on `stream`.
 *   ws  bkfac_correct_workspace_size(f, n_crc) bytes (0: n_crc too large)
 * Returns BKFAC_EINVAL for repeated or out-of-range indices. */
size_t bkfac_correct_workspace_size(const bkfac_factor* f, int n_crc);
int bkfac_correct(bkfac_factor* f, const void* M, int64_t ldm, const int32_t* idx, int n_crc, void* ws,
                  size_t ws_bytes, bkfac_stream_t stream);

/* RSVD overwrite of the representation (Algorithm 5, B-R-KFAC): a randomised
 * range finder on M with the caller's test matrix Omega (d x l column-major,
 * ld ldo, r <= l <= d; the caller draws it, e.g. N(0, 1)) and q power
 * iterations (q <= 64):
 *   Y = M Omega;  q times: Q = orth(Y), Y = M Q;  Q = orth(Y);
 *   B = Q^T M Q = W diag(lam) W^T;  U = Q W[:, :r],  sigma = lam[:r],
 * with orth by CholeskyQR2 (FP64 Gram and Cholesky) and B by FP64
 * accumulation, FP64 Cholesky and the one-sided Jacobi eigensolve.  Sets
 * r_cur = r.
 *   ws  bkfac_rsvd_workspace_size(f, l) bytes (0: l out of range or too large) */
size_t bkfac_rsvd_workspace_size(const bkfac_factor* f, int l);
int bkfac_rsvd(bkfac_factor* f, const void* M, int64_t ldm, const void* Omega, int64_t ldo, int l, int q, void* ws,
               size_t ws_bytes, bkfac_stream_t stream);

/* The damped inverse application without a caller workspace.  There is no
 * counterpart in the paper: this is an interface for callers that cannot
 * allocate device memory (code running under a stream capture that forbids
 * synchronising calls, frameworks whose device memory belongs to their own
 * pool allocator, latency-critical loops that cannot afford cudaMalloc's
 * implicit synchronisation).  Same arguments and result as bkfac_apply; the
 * workspace is a fixed array of BKFAC_NOALLOC_SCRATCH_BYTES that the library
 * keeps on every device that loads it, until the process exits.
 *   - Returns BKFAC_EWORKSPACE, before enqueuing anything, when the factor
 *     pair needs more than BKFAC_NOALLOC_SCRATCH_BYTES
 *     (bkfac_apply_workspace_size(fA, fG) tells how much it needs).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *     After a device reset (a new context on the device) the next call looks
 *     it up again, so that call too must come before any capture.
 *   - All calls on a device share the one array: calls that may overlap on
 *     the GPU (different streams without ordering) race on it and give
 *     undefined results.  Order them on one stream or with events.
 *   - Allocates nothing: no cudaMalloc / cudaFree, no allocating library call. */
#define BKFAC_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int bkfac_apply_noalloc(const bkfac_factor* fA, const bkfac_factor* fG, double lamA, double lamG, const void* G,
                        int64_t ldg, void* S, int64_t lds, uint32_t flags, bkfac_stream_t stream);

/* Diagnostics for tests: byte offsets, inside an update workspace, of the
 * intermediates left by the last bkfac_init / bkfac_update that used it:
 *   out[0] M (r_cur_old x n, column-major, dtype of U)
 *   out[1] Q (d x n, column-major, ld = out[6])
 *   out[2] the eigensolve's matrix (the core factor's columns, padded, in the
 *          eigensolve's precision; after the update its converged columns)
 *   out[3] lambda (N = r_cur_old + n doubles, descending, before truncation)
 *   out[4] P (d x n, column-major, ld = out[6]: the residual before its QR)
 *   out[5] leading dimension of M, out[6] leading dimension of Q and P.
 *   out[7] the eigensolve's counters (int32): [0] the full sweeps it ran (a
 *          closing check that finds no pair left to rotate is not a sweep),
 *          [1 + s] the rotations applied in sweep s (s < 48).
 * r_cur_old is the factor's r_cur before the update.  Returns BKFAC_EINVAL
 * for the dense path (which has no M, Q, R). */
int bkfac_debug_offsets(const bkfac_factor* f, int n, int64_t out[8]);

/* ---- tracing ---------------------------------------------------------------
 * Optional per-phase timing: while enabled, each phase of every call records
 * a CUDA event pair on the call's stream (not while the stream is being
 * captured into a graph).  Host-side state shared by all streams of the
 * process; not meant for concurrent use from several host threads.
 *   bkfac_trace_enable(on)  turns tracing on/off and clears the accumulators
 *   bkfac_trace_read(ms, count, nmax, launches)  waits for the recorded
 *       events, accumulates, and copies per-phase totals (milliseconds,
 *       number of timed phase instances) for up to nmax phases; *launches
 *       receives the number of kernels the library has launched since load.
 *       Returns the number of phases, or minus an error code.
 *   bkfac_trace_phase_name(id)  static name of phase id. */
int bkfac_trace_enable(int on);
int bkfac_trace_read(double* ms, int64_t* count, int nmax, int64_t* launches);
const char* bkfac_trace_phase_name(int id);

/* ---- autotuning -------------------------------------------------------------
 * Times the candidate launch shapes of factor f's eigensolve at batch width n
 * (block width of the Jacobi blocks, hence the cluster size, and the exchange
 * of the blocks between rounds: through L2 or over distributed shared memory)
 * on a synthetic core of that shape, on the current device, and records the
 * fastest in a process-wide table that later calls use.  cache_path (may be
 * NULL): a text file read before and written after tuning.  Allocates
 * temporary device memory; call it outside any stream capture.  The choice
 * only changes launch shapes, never the decomposition computed. */
int bkfac_tune(const bkfac_factor* f, int n, const char* cache_path);

/* GEMM autotuning for the FP32 products (CUDA-core GEMMs: the projections,
 * residuals, CholeskyQR solves, rotations and apply passes of the FP32 and FP64-
 * accumulated paths, and the small products of every apply).
 *   bkfac_gemm_tune_begin()  from now on the library notes the shape of every
 *       FP32 product it launches (M, N, the K segments, the operand and output
 *       layouts, a D term, and the partial-sum buffer the call has); the calls
 *       themselves run as before.
 *   bkfac_gemm_tune_end(cache_path)  stops noting; reads cache_path if present
 *       (may be NULL); for every noted shape not yet in the process-wide table,
 *       times the candidates -- 64 x 64 or 128 x 128 output tiles, K split into
 *       1 .. 32 pieces within the partial buffer the call had -- on synthetic
 *       operands of that shape, and records the fastest; writes the table
 *       (with the eigensolve choices) to cache_path.  Later calls whose shape
 *       is in the table use its choice when their layout and partial buffer
 *       allow it, else the built-in heuristic.  Allocates temporary device
 *       memory and synchronises: call it outside any stream capture.  A choice
 *       changes the order in which K terms are summed (FP32 rounding), not the
 *       product computed.
 * Both return BKFAC_OK or an error code (BKFAC_ECUDA when a device call failed;
 * the table then keeps the shapes that were tuned). */
int bkfac_gemm_tune_begin(void);
int bkfac_gemm_tune_end(const char* cache_path);

/* ---- batched calls: all factors of all FC layers -------------------------
 * A batch groups the two factors of nlayers layers (uneven d, r) with a
 * common batch width n and dtype.  An update runs in three stages: every
 * factor's work up to its eigensolve, forked onto one worker stream per
 * factor; the eigensolves, one grouped launch per eigensolve shape (one
 * thread-block cluster per factor, the launch shape of each group tuned for
 * its size when a tune cache is given); the rest of every update, forked
 * again.  The apply forks one stream per layer.  The whole step can be
 * captured once into a CUDA graph and replayed. */
typedef struct bkfac_layer_desc {
  bkfac_factor A;  /* forward factor, d = d_in (+1 for the bias) */
  bkfac_factor G;  /* backward factor, d = d_out */
} bkfac_layer_desc;

typedef struct bkfac_batch bkfac_batch;

/* Creates a batch over caller-owned factor buffers (copied descriptors; the
 * batch advances r_cur / step of its copies).  The handle allocates its own
 * device workspace and worker streams once, here (cudaMalloc), never on the
 * per-step path.  tune_cache: path of a text file of tuned eigensolve launch
 * shapes (may be NULL; read if present).  With a cache the batch times its
 * eigensolve groups here (temporary device memory, outside any capture) and
 * writes the choices back; without one it takes each shape's tuned or
 * default plan, with the block exchange over distributed shared memory while
 * every group's clusters fit on the GPU at once and through L2 otherwise.
 * Returns NULL on error. */
bkfac_batch* bkfac_batch_create(const bkfac_layer_desc* layers, int nlayers, int n, int dtype,
                                const char* tune_cache);

/* Current descriptor of layer l's factor (which = 0: A, 1: G). */
int bkfac_batch_get_factor(const bkfac_batch* b, int layer, int which, bkfac_factor* out);

/* Updates every factor: layer l's A factor with X_A[l] (d_A x n, ld ldxA[l]),
 * its G factor with X_G[l] (d_G x n, ld ldxG[l]).  Factors with r_cur == 0
 * are initialised instead (rho ignored for them). */
int bkfac_batch_update(bkfac_batch* b, const void* const* X_A, const int64_t* ldxA, const void* const* X_G,
                       const int64_t* ldxG, double rho, bkfac_stream_t stream);

/* Applies every layer's damped inverse: S[l] = (G_l-factor)^-1 G[l] (A_l-factor)^-1
 * with per-layer damping lamA[l], lamG[l] (host arrays). */
int bkfac_batch_apply(bkfac_batch* b, const void* const* G, const int64_t* ldg, void* const* S,
                      const int64_t* lds, const double* lamA, const double* lamG, uint32_t flags,
                      bkfac_stream_t stream);

/* Captures one full step -- bkfac_batch_update(X_A, X_G, rho) followed by
 * bkfac_batch_apply(G, S, lamA, lamG, flags) with the given pointers -- into
 * a CUDA graph owned by the batch, then replays it once on `stream`.  Later
 * calls with capture == 0 replay the graph (same pointers, same rho / lam).
 * All factors must already be at steady rank (r_cur == r after this step's
 * update, i.e. no factor still growing), else BKFAC_EINVAL. */
int bkfac_batch_step_graph(bkfac_batch* b, const void* const* X_A, const int64_t* ldxA, const void* const* X_G,
                           const int64_t* ldxG, double rho, const void* const* G, const int64_t* ldg,
                           void* const* S, const int64_t* lds, const double* lamA, const double* lamG,
                           uint32_t flags, int capture, bkfac_stream_t stream);

/* Re-orthonormalises every factor of the batch (bkfac_reorth on each, forked over
 * the worker streams): the periodic accuracy recovery of the mixed-precision path,
 * e.g. every 10 steps. */
int bkfac_batch_reorth(bkfac_batch* b, bkfac_stream_t stream);

void bkfac_batch_destroy(bkfac_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* BKFAC_H */

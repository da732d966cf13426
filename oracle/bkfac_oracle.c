/*
 * bkfac_oracle.c -- plain, slow FP64 CPU oracle for the B-KFAC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code; the library's product
 * path never calls it and has no CPU fallback.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * What it computes (paper: "Brand New K-FACs", arXiv 2210.08494):
 *
 *   update  (Sec. 3.1, Algorithm 4 built on Algorithm 3 and Eq. (7)):
 *     the EA K-factor of Eq. (5)/(8), held as U diag(sigma) U^T with U d x k,
 *     receives  K = rho * U diag(sigma) U^T + c * X X^T,  c = (1 - rho) / n,
 *     and is replaced by its top-r eigenpairs (the truncation of Sec. 3.1).
 *     Steps, in the order of Algorithm 3:
 *       1. M = U^T X,  P = X - U M                       (projection, residual)
 *       2. Q R~ = P   by Householder QR with column pivoting, truncated at the
 *          numerical rank (any orthonormal factorisation is allowed, footnote
 *          to Eq. (7)); R~ is m x n with the pivoting undone
 *       3. M_S = E diag(rho*sigma, I_m) E^T,  E = [[I, sqrt(c) M], [0, sqrt(c) R~]]
 *          (Eq. (7) with B <- A, V <- U, D <- rho*D, A <- sqrt(c) X)
 *       4. M_S = V diag(lambda) V^T by the two-sided cyclic Jacobi method,
 *          eigenvalues sorted descending (ties: lower index first)
 *       5. U' = [U Q] V[:, :r_new],  sigma' = lambda[:r_new],
 *          r_new = min(r, k + n)  (zero columns / zero values past rank m+k)
 *     Initialisation (kappa(0) = 1 in Eq. (5)) is the same update from k = 0
 *     with rho = 0, i.e. the exact top-r EVD of X X^T / n.
 *
 *   dense update (the case r + n >= d, where Algorithm 3's precondition
 *     (r+n) < d fails): form K (d x d) explicitly and take its top-r
 *     eigenpairs with the same Jacobi routine.
 *
 *   apply (Algorithm 1, inverse application; K-FAC identity of Eq. (4)):
 *     S = (U_G C_G U_G^T + I/lam_G) G (U_A C_A U_A^T + I/lam_A),
 *     C = diag(1/(sigma + lam) - 1/lam), evaluated right factor first, then
 *     the left factor, in plain loops.  Optional spectrum continuation
 *     (Sec. 3.5.1): lam <- lam + min(sigma), sigma <- sigma - min(sigma).
 *
 *   apply_factored (Algorithm 8, linear inverse application): for a weight
 *     gradient alpha * G_f A_f^T given by its thin factors (the columns that
 *     also feed the K-factor updates), the damped inverses act on the factors,
 *     PA = (U_A C_A U_A^T + I/lam_A) A_f,  PG = (U_G C_G U_G^T + I/lam_G) G_f,
 *     and the step is S = alpha * PG PA^T (formed only when asked for).
 *
 *   ea_update (Eq. (5) / (8)): the dense EA K-factor that B-R-KFAC and
 *     B-KFAC-C keep beside the low-rank representation,
 *     M <- rho M + (1 - rho)/n X X^T  (M = X X^T / n at the first step).
 *
 *   correct (Algorithm 6, the light correction of B-KFAC-C): for n_crc chosen
 *     modes idx of the representation, M_S = U_s^T M U_s with U_s = U[:, idx],
 *     M_S = W diag(lam) W^T, then U[:, idx] <- U_s W and sigma[idx] <- lam;
 *     the modes are then re-sorted by decreasing sigma (stable).
 *
 *   rsvd (Algorithm 5's overwrite of B-R-KFAC): randomised range finder with
 *     a given test matrix Omega (d x l, l = r + oversampling) and q power
 *     iterations, Y = M Omega, then q times Q = orth(Y), Y = M Q; Q = orth(Y),
 *     B = Q^T M Q = W diag(lam) W^T, U = Q W[:, :r], sigma = lam[:r].
 *
 *   reorth: the top eigenpairs of U diag(sigma) U^T restricted to span(U)
 *     (Householder QR of U, Jacobi on R diag(sigma) R^T); a no-op in exact
 *     arithmetic when U is orthonormal.
 *
 * Layout: every matrix is column-major, A[i + j*lda], except the gradient G
 * and the step S of apply, which are row-major d_G x d_A (torch weight.grad
 * layout, bias column last).  All arithmetic is IEEE double, compiled with
 * -ffp-contract=off.  OpenMP (when enabled) only splits loops whose
 * iterations write disjoint outputs, so results do not depend on the thread
 * count.
 *
 * Parity status: every function here is pinned by the CPU tests against
 * closed forms, numpy's LAPACK eigh / solve on small inputs, and the
 * invariants of Propositions 3.1, 3.2, 4.1 and 4.2.  The paper prints no
 * worked numeric example, so no value here is pinned to a printed number.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define BKO_OK 0
#define BKO_EINVAL 1
#define BKO_ENOCONV 4
#define BKO_ENOMEM 9

#define AT(A, ld, i, j) ((A)[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

/* Plain column-major products: C (m x n) = A (m x k) * B (k x n), with
 * optional transposes expressed by the element accessors below. */
static void mat_tn(int m, int n, int k, const double* A, long lda, const double* B, long ldb,
                   double* C, long ldc) {
  /* C = A^T B, A is k x m, B is k x n */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += AT(A, lda, l, i) * AT(B, ldb, l, j);
      AT(C, ldc, i, j) = s;
    }
}

static void mat_nn(int m, int n, int k, const double* A, long lda, const double* B, long ldb,
                   double* C, long ldc) {
  /* C = A B, A is m x k, B is k x n */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += AT(A, lda, i, l) * AT(B, ldb, l, j);
      AT(C, ldc, i, j) = s;
    }
}

/* ---------------------------------------------------------------------------
 * Two-sided cyclic Jacobi eigensolver for a symmetric N x N matrix A
 * (column-major, lda).  A is overwritten; on return lambda holds the
 * eigenvalues sorted descending and V (N x N, ldv) the matching orthonormal
 * eigenvectors.  Rotation angles follow Rutishauser's formulas (Golub & Van
 * Loan, Sec. 8.5).  A rotation is skipped when |a_pq| is negligible against
 * sqrt(|a_pp a_qq|) or against the Frobenius norm; the loop stops after a
 * sweep with no rotation.
 * ------------------------------------------------------------------------- */
int bko_jacobi_eig(int N, double* A, long lda, double* lambda, double* V, long ldv, int max_sweeps,
                   int* sweeps_out) {
  if (N < 0) return BKO_EINVAL;
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) AT(V, ldv, i, j) = (i == j) ? 1.0 : 0.0;
  double fro2 = 0.0;
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) fro2 += AT(A, lda, i, j) * AT(A, lda, i, j);
  const double tiny = 1e-300 + 1e-17 * sqrt(fro2);
  int sweep = 0, converged = (N <= 1);
  while (!converged && sweep < max_sweeps) {
    int rotations = 0;
    for (int p = 0; p < N - 1; ++p)
      for (int q = p + 1; q < N; ++q) {
        double apq = AT(A, lda, p, q);
        double app = AT(A, lda, p, p), aqq = AT(A, lda, q, q);
        if (fabs(apq) <= tiny || fabs(apq) <= 1e-16 * sqrt(fabs(app * aqq))) continue;
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* A <- J^T A J with J the (p,q) Givens rotation [[c, s], [-s, c]] */
        for (int i = 0; i < N; ++i) {
          double aip = AT(A, lda, i, p), aiq = AT(A, lda, i, q);
          AT(A, lda, i, p) = c * aip - s * aiq;
          AT(A, lda, i, q) = s * aip + c * aiq;
        }
        for (int j = 0; j < N; ++j) {
          double apj = AT(A, lda, p, j), aqj = AT(A, lda, q, j);
          AT(A, lda, p, j) = c * apj - s * aqj;
          AT(A, lda, q, j) = s * apj + c * aqj;
        }
        AT(A, lda, p, q) = 0.0;
        AT(A, lda, q, p) = 0.0;
        for (int i = 0; i < N; ++i) {
          double vip = AT(V, ldv, i, p), viq = AT(V, ldv, i, q);
          AT(V, ldv, i, p) = c * vip - s * viq;
          AT(V, ldv, i, q) = s * vip + c * viq;
        }
        ++rotations;
      }
    ++sweep;
    if (rotations == 0) converged = 1;
  }
  if (sweeps_out) *sweeps_out = sweep;
  /* sort descending, stable: selection of the largest remaining, lowest index on ties */
  double* lam = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  double* Vs = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N + 8);
  int* used = (int*)calloc((size_t)(N > 0 ? N : 1), sizeof(int));
  if (!lam || !Vs || !used) {
    free(lam); free(Vs); free(used);
    return BKO_ENOMEM;
  }
  for (int i = 0; i < N; ++i) lam[i] = AT(A, lda, i, i);
  for (int o = 0; o < N; ++o) {
    int best = -1;
    for (int i = 0; i < N; ++i)
      if (!used[i] && (best < 0 || lam[i] > lam[best])) best = i;
    used[best] = 1;
    lambda[o] = lam[best];
    for (int i = 0; i < N; ++i) Vs[(size_t)i + (size_t)o * N] = AT(V, ldv, i, best);
  }
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) AT(V, ldv, i, j) = Vs[(size_t)i + (size_t)j * N];
  free(lam); free(Vs); free(used);
  return converged ? BKO_OK : BKO_ENOCONV;
}

/* ---------------------------------------------------------------------------
 * Householder QR with column pivoting (Golub & Van Loan, Alg. 5.4.1) of the
 * d x n matrix P.  Stops at the numerical rank m: the first step whose
 * largest remaining column norm is <= tol.  Outputs
 *   Q  (d x n, ldq): the first m columns orthonormal, the rest zero,
 *   Rt (n x n, ldr): rows 0..m-1 hold R~ with the pivoting undone, so that
 *                    P = Q Rt up to the dropped part; rows m.. are zero,
 *   *rank = m.
 * Each Householder vector is normalised so that R's diagonal is >= 0.
 * ------------------------------------------------------------------------- */
int bko_qrcp(int d, int n, const double* P, long ldp, double tol, double* Q, long ldq, double* Rt,
             long ldr, int* rank) {
  if (d < 0 || n < 0) return BKO_EINVAL;
  double* A = (double*)malloc(sizeof(double) * (size_t)d * (size_t)(n > 0 ? n : 1) + 8);
  double* vs = (double*)malloc(sizeof(double) * (size_t)d * (size_t)(n > 0 ? n : 1) + 8);
  double* beta = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int* perm = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  double* cn = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!A || !vs || !beta || !perm || !cn) {
    free(A); free(vs); free(beta); free(perm); free(cn);
    return BKO_ENOMEM;
  }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < d; ++i) A[(size_t)i + (size_t)j * d] = AT(P, ldp, i, j);
  for (int j = 0; j < n; ++j) perm[j] = j;
  int kmax = n < d ? n : d;
  int m = 0;
  for (int s = 0; s < kmax; ++s) {
    /* column norms of the trailing block, recomputed from scratch (slow, exact) */
    int piv = s;
    double best = -1.0;
    for (int j = s; j < n; ++j) {
      double t = 0.0;
      for (int i = s; i < d; ++i) t += A[(size_t)i + (size_t)j * d] * A[(size_t)i + (size_t)j * d];
      cn[j] = t;
      if (t > best) { best = t; piv = j; }
    }
    if (sqrt(best) <= tol) break;
    if (piv != s) {
      for (int i = 0; i < d; ++i) {
        double t = A[(size_t)i + (size_t)s * d];
        A[(size_t)i + (size_t)s * d] = A[(size_t)i + (size_t)piv * d];
        A[(size_t)i + (size_t)piv * d] = t;
      }
      int tp = perm[s]; perm[s] = perm[piv]; perm[piv] = tp;
    }
    /* Householder vector v with (I - beta v v^T) x = alpha e_1, alpha = +||x|| */
    double* v = vs + (size_t)s * d;
    double xnorm = sqrt(best);
    for (int i = 0; i < d; ++i) v[i] = 0.0;
    for (int i = s; i < d; ++i) v[i] = A[(size_t)i + (size_t)s * d];
    /* v = x - alpha e1 with alpha = ||x|| > 0 gives a non-negative diagonal */
    double x0 = v[s];
    double v0 = (x0 <= 0.0) ? (x0 - xnorm) : (-(best - x0 * x0) / (x0 + xnorm));
    v[s] = v0;
    double vv = 0.0;
    for (int i = s; i < d; ++i) vv += v[i] * v[i];
    beta[s] = (vv > 0.0) ? 2.0 / vv : 0.0;
    /* apply to the trailing columns */
    for (int j = s; j < n; ++j) {
      double w = 0.0;
      for (int i = s; i < d; ++i) w += v[i] * A[(size_t)i + (size_t)j * d];
      w *= beta[s];
      for (int i = s; i < d; ++i) A[(size_t)i + (size_t)j * d] -= w * v[i];
    }
    A[(size_t)s + (size_t)s * d] = xnorm;
    for (int i = s + 1; i < d; ++i) A[(size_t)i + (size_t)s * d] = 0.0;
    m = s + 1;
  }
  /* R~ with the column permutation undone: Rt[:, perm[j]] = R[:, j] */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(Rt, ldr, i, j) = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m && i <= j; ++i) AT(Rt, ldr, i, perm[j]) = A[(size_t)i + (size_t)j * d];
  /* Q = H_0 H_1 ... H_{m-1} [I_m; 0], zero beyond column m */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < d; ++i) AT(Q, ldq, i, j) = (j < m && i == j) ? 1.0 : 0.0;
  for (int s = m - 1; s >= 0; --s) {
    const double* v = vs + (size_t)s * d;
    for (int j = 0; j < m; ++j) {
      double w = 0.0;
      for (int i = s; i < d; ++i) w += v[i] * AT(Q, ldq, i, j);
      w *= beta[s];
      for (int i = s; i < d; ++i) AT(Q, ldq, i, j) -= w * v[i];
    }
  }
  if (rank) *rank = m;
  free(A); free(vs); free(beta); free(perm); free(cn);
  return BKO_OK;
}

/* ---------------------------------------------------------------------------
 * Step 1 of Algorithm 3: M = U^T X (k x n, ld k) and P = X - U M (d x n, ld d).
 * ------------------------------------------------------------------------- */
int bko_project(int d, int k, const double* U, long ldu, int n, const double* X, long ldx, double* M,
                double* P) {
  if (d < 0 || k < 0 || n < 0) return BKO_EINVAL;
  if (k > 0) mat_tn(k, n, d, U, ldu, X, ldx, M, k);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < d; ++i) {
      double s = AT(X, ldx, i, j);
      double um = 0.0;
      for (int l = 0; l < k; ++l) um += AT(U, ldu, i, l) * M[(size_t)l + (size_t)j * k];
      P[(size_t)i + (size_t)j * d] = s - um;
    }
  return BKO_OK;
}

/* ---------------------------------------------------------------------------
 * Step 3 of Algorithm 3: the core of Eq. (7) for the symmetric update with the
 * B-KFAC substitutions of Sec. 3.1 (D <- rho*diag(sigma), A <- sqrt(c) X):
 *   M_S = E diag(rho*sigma_1..rho*sigma_k, 1, .., 1) E^T,
 *   E   = [[I_k, sqrt(c) M], [0, sqrt(c) Rt]],   N = k + n.
 * Written as the product of the three factors of Eq. (7), in plain loops.
 * ------------------------------------------------------------------------- */
int bko_core(int k, int n, const double* sigma, double rho, double c, const double* M, const double* Rt,
             long ldr, double* MS, long ldm) {
  if (k < 0 || n < 0) return BKO_EINVAL;
  int N = k + n;
  double* E = (double*)calloc((size_t)N * (size_t)(N > 0 ? N : 1) + 1, sizeof(double));
  double* Dg = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  if (!E || !Dg) { free(E); free(Dg); return BKO_ENOMEM; }
  double sc = sqrt(c);
  for (int i = 0; i < k; ++i) E[(size_t)i + (size_t)i * N] = 1.0;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < k; ++i) E[(size_t)i + (size_t)(k + j) * N] = sc * M[(size_t)i + (size_t)j * k];
    for (int i = 0; i < n; ++i) E[(size_t)(k + i) + (size_t)(k + j) * N] = sc * AT(Rt, ldr, i, j);
  }
  for (int i = 0; i < k; ++i) Dg[i] = rho * sigma[i];
  for (int i = k; i < N; ++i) Dg[i] = 1.0;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
      for (int l = 0; l < N; ++l) s += E[(size_t)i + (size_t)l * N] * Dg[l] * E[(size_t)j + (size_t)l * N];
      AT(MS, ldm, i, j) = s;
    }
  free(E); free(Dg);
  return BKO_OK;
}

/* tolerance for the rank decision of the residual QR: relative to the largest
 * column norm of X (not of P), so exact dependencies are dropped while any
 * direction carrying more than ~1e-12 of the batch's scale is kept */
static double rank_tol(int d, int n, const double* X, long ldx) {
  double mx = 0.0;
  for (int j = 0; j < n; ++j) {
    double t = 0.0;
    for (int i = 0; i < d; ++i) t += AT(X, ldx, i, j) * AT(X, ldx, i, j);
    if (t > mx) mx = t;
  }
  return 1e-12 * sqrt(mx);
}

/* ---------------------------------------------------------------------------
 * One B-KFAC update of a factor (Algorithm 4 via Algorithm 3).
 *   d, r       factor size and target rank (r <= d)
 *   k          current rank (0 <= k <= r); U is d x k (ldu), sigma has k values
 *   X          d x n new columns (ldx)
 *   rho        EA decay; c = (1 - rho) / n scales X X^T
 *   U_out      d x r (ldo): columns 0..r_new-1 written, the rest zeroed
 *   sigma_out  r values, zero beyond r_new
 *   diag       optional (may be NULL), 4 ints: r_new, rank m of P, Jacobi sweeps, N
 * ------------------------------------------------------------------------- */
int bko_update(int d, int r, int k, const double* U, long ldu, const double* sigma, int n, const double* X,
               long ldx, double rho, double* U_out, long ldo, double* sigma_out, int* diag) {
  if (d <= 0 || r <= 0 || r > d || k < 0 || k > r || n <= 0 || ldu < d || ldx < d || ldo < d)
    return BKO_EINVAL;
  int N = k + n;
  double c = (1.0 - rho) / (double)n;
  double* M = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1) * (size_t)n);
  double* P = (double*)malloc(sizeof(double) * (size_t)d * (size_t)n);
  double* Q = (double*)malloc(sizeof(double) * (size_t)d * (size_t)n);
  double* Rt = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* MS = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
  double* V = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
  double* lam = (double*)malloc(sizeof(double) * (size_t)N);
  int rc = BKO_ENOMEM;
  if (!M || !P || !Q || !Rt || !MS || !V || !lam) goto done;
  rc = bko_project(d, k, U, ldu, n, X, ldx, M, P);
  if (rc) goto done;
  int m = 0;
  rc = bko_qrcp(d, n, P, d, rank_tol(d, n, X, ldx), Q, d, Rt, n, &m);
  if (rc) goto done;
  rc = bko_core(k, n, sigma, rho, c, M, Rt, n, MS, N);
  if (rc) goto done;
  int sweeps = 0;
  rc = bko_jacobi_eig(N, MS, N, lam, V, N, 100, &sweeps);
  if (rc) goto done;
  int r_new = r < N ? r : N;
  /* U' = [U Q] V[:, :r_new] */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < r; ++j)
    for (int i = 0; i < d; ++i) {
      double s = 0.0;
      if (j < r_new) {
        for (int l = 0; l < k; ++l) s += AT(U, ldu, i, l) * V[(size_t)l + (size_t)j * N];
        for (int l = 0; l < n; ++l) s += Q[(size_t)i + (size_t)l * d] * V[(size_t)(k + l) + (size_t)j * N];
      }
      AT(U_out, ldo, i, j) = s;
    }
  for (int j = 0; j < r; ++j) sigma_out[j] = (j < r_new) ? lam[j] : 0.0;
  if (diag) { diag[0] = r_new; diag[1] = m; diag[2] = sweeps; diag[3] = N; }
  rc = BKO_OK;
done:
  free(M); free(P); free(Q); free(Rt); free(MS); free(V); free(lam);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Dense update for factors where Algorithm 3's precondition (r + n) < d fails:
 *   K = rho * U diag(sigma) U^T + c X X^T   (d x d, formed explicitly),
 *   top-r_new eigenpairs by Jacobi, r_new = min(r, k + n, d).
 * Same arguments as bko_update.
 * ------------------------------------------------------------------------- */
int bko_update_dense(int d, int r, int k, const double* U, long ldu, const double* sigma, int n,
                     const double* X, long ldx, double rho, double* U_out, long ldo, double* sigma_out,
                     int* diag) {
  if (d <= 0 || r <= 0 || r > d || k < 0 || k > r || n <= 0 || ldu < d || ldx < d || ldo < d)
    return BKO_EINVAL;
  double c = (1.0 - rho) / (double)n;
  double* K = (double*)malloc(sizeof(double) * (size_t)d * (size_t)d);
  double* V = (double*)malloc(sizeof(double) * (size_t)d * (size_t)d);
  double* lam = (double*)malloc(sizeof(double) * (size_t)d);
  if (!K || !V || !lam) { free(K); free(V); free(lam); return BKO_ENOMEM; }
#pragma omp parallel for schedule(static)
  for (int j = 0; j < d; ++j)
    for (int i = 0; i < d; ++i) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += rho * AT(U, ldu, i, l) * sigma[l] * AT(U, ldu, j, l);
      double t = 0.0;
      for (int l = 0; l < n; ++l) t += AT(X, ldx, i, l) * AT(X, ldx, j, l);
      K[(size_t)i + (size_t)j * d] = s + c * t;
    }
  int sweeps = 0;
  int rc = bko_jacobi_eig(d, K, d, lam, V, d, 100, &sweeps);
  if (rc) { free(K); free(V); free(lam); return rc; }
  int r_new = r;
  if (k + n < r_new) r_new = k + n;
  for (int j = 0; j < r; ++j)
    for (int i = 0; i < d; ++i) AT(U_out, ldo, i, j) = (j < r_new) ? V[(size_t)i + (size_t)j * d] : 0.0;
  for (int j = 0; j < r; ++j) sigma_out[j] = (j < r_new) ? lam[j] : 0.0;
  if (diag) { diag[0] = r_new; diag[1] = -1; diag[2] = sweeps; diag[3] = d; }
  free(K); free(V); free(lam);
  return BKO_OK;
}

/* ---------------------------------------------------------------------------
 * Re-orthonormalisation of a low-rank representation: the top-k eigenpairs of
 * U diag(sigma) U^T within span(U).  Q R = U (Householder, no truncation
 * beyond exact zeros), then Jacobi on R diag(sigma) R^T, U' = Q W.
 * ------------------------------------------------------------------------- */
int bko_reorth(int d, int k, const double* U, long ldu, const double* sigma, double* U_out, long ldo,
               double* sigma_out) {
  if (d <= 0 || k < 0 || k > d || ldu < d || ldo < d) return BKO_EINVAL;
  if (k == 0) return BKO_OK;
  double* Q = (double*)malloc(sizeof(double) * (size_t)d * (size_t)k);
  double* R = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double* B = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double* W = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double* lam = (double*)malloc(sizeof(double) * (size_t)k);
  int rc = BKO_ENOMEM, m = 0;
  if (!Q || !R || !B || !W || !lam) goto done;
  rc = bko_qrcp(d, k, U, ldu, 0.0, Q, d, R, k, &m);
  if (rc) goto done;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += R[(size_t)i + (size_t)l * k] * sigma[l] * R[(size_t)j + (size_t)l * k];
      B[(size_t)i + (size_t)j * k] = s;
    }
  rc = bko_jacobi_eig(k, B, k, lam, W, k, 100, NULL);
  if (rc) goto done;
  mat_nn(d, k, k, Q, d, W, k, U_out, ldo);
  for (int j = 0; j < k; ++j) sigma_out[j] = lam[j];
  rc = BKO_OK;
done:
  free(Q); free(R); free(B); free(W); free(lam);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Damped inverse application (Algorithm 1, inverse application; Eq. (4)):
 *   S = L_G G R_A,   L = I/lam + U C U^T,   C = diag(1/(sigma+lam) - 1/lam).
 * G and S are row-major dG x dA (ldg, lds >= dA); S may not alias G.
 * Option bits (opt):
 *   1  spectrum continuation (Sec. 3.5.1) over the kA / kG stored modes;
 *   2  relative damping (the damping schedule of the experiments, Sec. 4):
 *      the given lam is a multiple phi of the largest eigenvalue of the
 *      represented factor, lam = phi * max_i sigma_i, taken before the
 *      continuation shift.
 * ------------------------------------------------------------------------- */
static void damped_coeffs(int k, const double* sigma, double lam, int opt, double* coef, double* lam_eff) {
  if ((opt & 2) && k > 0) {
    double top = sigma[0];
    for (int i = 1; i < k; ++i)
      if (sigma[i] > top) top = sigma[i];
    lam *= top;
  }
  double shift = 0.0;
  if ((opt & 1) && k > 0) {
    shift = sigma[0];
    for (int i = 1; i < k; ++i)
      if (sigma[i] < shift) shift = sigma[i];
  }
  double l = lam + shift;
  for (int i = 0; i < k; ++i) coef[i] = 1.0 / ((sigma[i] - shift) + l) - 1.0 / l;
  *lam_eff = l;
}

int bko_apply(int dA, int kA, const double* UA, long lduA, const double* sigA, double lamA, int dG, int kG,
              const double* UG, long lduG, const double* sigG, double lamG, const double* G, long ldg,
              double* S, long lds, int cont) {
  if (dA <= 0 || dG <= 0 || kA < 0 || kG < 0 || lduA < dA || lduG < dG || ldg < dA || lds < dA ||
      !(lamA > 0.0) || !(lamG > 0.0) || ((cont & 2) && (kA < 1 || kG < 1)))
    return BKO_EINVAL;
  double* cA = (double*)malloc(sizeof(double) * (size_t)(kA > 0 ? kA : 1));
  double* cG = (double*)malloc(sizeof(double) * (size_t)(kG > 0 ? kG : 1));
  double* T = (double*)malloc(sizeof(double) * (size_t)dG * (size_t)dA); /* row-major G R_A */
  double* Y = (double*)malloc(sizeof(double) * (size_t)(kG > 0 ? kG : 1) * (size_t)dA);
  if (!cA || !cG || !T || !Y) { free(cA); free(cG); free(T); free(Y); return BKO_ENOMEM; }
  double lA, lG;
  damped_coeffs(kA, sigA, lamA, cont, cA, &lA);
  damped_coeffs(kG, sigG, lamG, cont, cG, &lG);
  /* right factor, row by row: t = g/lA + sum_a (g . u_a) cA[a] u_a^T */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < dG; ++i) {
    const double* g = G + (size_t)i * ldg;
    double* t = T + (size_t)i * dA;
    for (int j = 0; j < dA; ++j) t[j] = g[j] / lA;
    for (int a = 0; a < kA; ++a) {
      const double* u = UA + (size_t)a * lduA;
      double s = 0.0;
      for (int j = 0; j < dA; ++j) s += g[j] * u[j];
      s *= cA[a];
      for (int j = 0; j < dA; ++j) t[j] += s * u[j];
    }
  }
  /* left factor: Y = cG .* (U_G^T T)  (kG x dA, row-major) */
#pragma omp parallel for schedule(static)
  for (int b = 0; b < kG; ++b) {
    double* y = Y + (size_t)b * dA;
    for (int j = 0; j < dA; ++j) y[j] = 0.0;
    for (int i = 0; i < dG; ++i) {
      double u = AT(UG, lduG, i, b);
      const double* t = T + (size_t)i * dA;
      for (int j = 0; j < dA; ++j) y[j] += u * t[j];
    }
    for (int j = 0; j < dA; ++j) y[j] *= cG[b];
  }
  /* S = T/lG + U_G Y */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < dG; ++i) {
    double* srow = S + (size_t)i * lds;
    const double* t = T + (size_t)i * dA;
    for (int j = 0; j < dA; ++j) srow[j] = t[j] / lG;
    for (int b = 0; b < kG; ++b) {
      double u = AT(UG, lduG, i, b);
      const double* y = Y + (size_t)b * dA;
      for (int j = 0; j < dA; ++j) srow[j] += u * y[j];
    }
  }
  free(cA); free(cG); free(T); free(Y);
  return BKO_OK;
}

/* ---------------------------------------------------------------------------
 * Linear inverse application (Algorithm 8).  The gradient of an FC layer over a
 * batch is alpha * G_f A_f^T, G_f (dG x n) the back-propagated columns and A_f
 * (dA x n) the input columns -- the same matrices whose outer products build the
 * EA K-factors.  Algorithm 8 applies the low-rank damped inverses to these thin
 * factors, column by column,
 *   PA = A_f / lam_A + U_A C_A U_A^T A_f,   PG = G_f / lam_G + U_G C_G U_G^T G_f,
 * and forms the step S = alpha * PG PA^T (dG x dA, row-major) when S != NULL.
 * A_f, G_f, PA, PG are column-major (ld >= d).  Option bits as in apply.
 * ------------------------------------------------------------------------- */
static void damped_columns(int d, int k, const double* U, long ldu, const double* coef, double l, int n,
                           const double* X, long ldx, double* P, long ldp) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    const double* x = X + (size_t)j * ldx;
    double* p = P + (size_t)j * ldp;
    for (int i = 0; i < d; ++i) p[i] = x[i] / l;
    for (int a = 0; a < k; ++a) {
      const double* u = U + (size_t)a * ldu;
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += u[i] * x[i];
      s *= coef[a];
      for (int i = 0; i < d; ++i) p[i] += s * u[i];
    }
  }
}

int bko_apply_factored(int dA, int kA, const double* UA, long lduA, const double* sigA, double lamA, int dG,
                       int kG, const double* UG, long lduG, const double* sigG, double lamG, int n,
                       const double* XA, long ldxa, const double* XG, long ldxg, double* PA, long ldpa,
                       double* PG, long ldpg, double alpha, double* S, long lds, int cont) {
  if (dA <= 0 || dG <= 0 || kA < 0 || kG < 0 || n < 0 || lduA < dA || lduG < dG || ldxa < dA || ldxg < dG ||
      ldpa < dA || ldpg < dG || (S && lds < dA) || !(lamA > 0.0) || !(lamG > 0.0) ||
      ((cont & 2) && (kA < 1 || kG < 1)))
    return BKO_EINVAL;
  double* cA = (double*)malloc(sizeof(double) * (size_t)(kA > 0 ? kA : 1));
  double* cG = (double*)malloc(sizeof(double) * (size_t)(kG > 0 ? kG : 1));
  if (!cA || !cG) { free(cA); free(cG); return BKO_ENOMEM; }
  double lA, lG;
  damped_coeffs(kA, sigA, lamA, cont, cA, &lA);
  damped_coeffs(kG, sigG, lamG, cont, cG, &lG);
  damped_columns(dA, kA, UA, lduA, cA, lA, n, XA, ldxa, PA, ldpa);
  damped_columns(dG, kG, UG, lduG, cG, lG, n, XG, ldxg, PG, ldpg);
  if (S) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < dG; ++i) {
      double* srow = S + (size_t)i * lds;
      for (int j = 0; j < dA; ++j) {
        double acc = 0.0;
        for (int t = 0; t < n; ++t) acc += PG[(size_t)i + (size_t)t * ldpg] * PA[(size_t)j + (size_t)t * ldpa];
        srow[j] = alpha * acc;
      }
    }
  }
  free(cA); free(cG);
  return BKO_OK;
}

/* ---------------------------------------------------------------------------
 * Dense EA K-factor (Eq. (5) / (8)) for B-R-KFAC and B-KFAC-C:
 *   first != 0:  M = X X^T / n     (kappa(0) = 1)
 *   otherwise:   M = rho M + (1 - rho)/n X X^T
 * M is d x d column-major (ldm >= d), X is d x n (ldx >= d).
 * ------------------------------------------------------------------------- */
int bko_ea_update(int d, double* M, long ldm, int n, const double* X, long ldx, double rho, int first) {
  if (d <= 0 || n <= 0 || ldm < d || ldx < d) return BKO_EINVAL;
  const double c = first ? 1.0 / n : (1.0 - rho) / n;
  const double keep = first ? 0.0 : rho;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < d; ++j)
    for (int i = 0; i < d; ++i) {
      double s = 0.0;
      for (int t = 0; t < n; ++t) s += AT(X, ldx, i, t) * AT(X, ldx, j, t);
      AT(M, ldm, i, j) = keep * AT(M, ldm, i, j) + c * s;
    }
  return BKO_OK;
}

/* stable re-sort of k modes by decreasing sigma (columns of U move along) */
static int sort_modes(int d, int k, double* U, long ldu, double* sigma) {
  int* order = (int*)malloc(sizeof(int) * (size_t)(k > 0 ? k : 1));
  double* Ut = (double*)malloc(sizeof(double) * (size_t)d * (size_t)(k > 0 ? k : 1));
  double* st = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  if (!order || !Ut || !st) { free(order); free(Ut); free(st); return BKO_ENOMEM; }
  for (int i = 0; i < k; ++i) order[i] = i;
  for (int i = 1; i < k; ++i) { /* insertion sort: stable */
    const int v = order[i];
    int j = i - 1;
    while (j >= 0 && sigma[order[j]] < sigma[v]) { order[j + 1] = order[j]; --j; }
    order[j + 1] = v;
  }
  for (int j = 0; j < k; ++j) {
    st[j] = sigma[order[j]];
    for (int i = 0; i < d; ++i) Ut[(size_t)i + (size_t)j * d] = AT(U, ldu, i, order[j]);
  }
  for (int j = 0; j < k; ++j) {
    sigma[j] = st[j];
    for (int i = 0; i < d; ++i) AT(U, ldu, i, j) = Ut[(size_t)i + (size_t)j * d];
  }
  free(order); free(Ut); free(st);
  return BKO_OK;
}

/* ---------------------------------------------------------------------------
 * Light correction of a B-KFAC representation (Algorithm 6).  U (d x k, ldu)
 * and sigma (k) are corrected in place along the n_crc modes idx (distinct,
 * in [0, k)), against the dense EA factor M (d x d, ldm).
 * ------------------------------------------------------------------------- */
int bko_correct(int d, int k, double* U, long ldu, double* sigma, const double* M, long ldm, int n_crc,
                const int* idx) {
  if (d <= 0 || k < 0 || ldu < d || ldm < d || n_crc < 0 || n_crc > k) return BKO_EINVAL;
  for (int a = 0; a < n_crc; ++a) {
    if (idx[a] < 0 || idx[a] >= k) return BKO_EINVAL;
    for (int b = 0; b < a; ++b)
      if (idx[a] == idx[b]) return BKO_EINVAL;
  }
  if (n_crc == 0) return BKO_OK;
  double* Us = (double*)malloc(sizeof(double) * (size_t)d * (size_t)n_crc);
  double* MU = (double*)malloc(sizeof(double) * (size_t)d * (size_t)n_crc);
  double* Ms = (double*)malloc(sizeof(double) * (size_t)n_crc * (size_t)n_crc);
  double* W = (double*)malloc(sizeof(double) * (size_t)n_crc * (size_t)n_crc);
  double* lam = (double*)malloc(sizeof(double) * (size_t)n_crc);
  double* Un = (double*)malloc(sizeof(double) * (size_t)d * (size_t)n_crc);
  int rc = BKO_ENOMEM;
  if (!Us || !MU || !Ms || !W || !lam || !Un) goto done;
  for (int a = 0; a < n_crc; ++a)
    for (int i = 0; i < d; ++i) Us[(size_t)i + (size_t)a * d] = AT(U, ldu, i, idx[a]);
  mat_nn(d, n_crc, d, M, ldm, Us, d, MU, d);          /* M U_s */
  mat_tn(n_crc, n_crc, d, Us, d, MU, d, Ms, n_crc);    /* M_S = U_s^T M U_s */
  for (int j = 0; j < n_crc; ++j)                       /* exact symmetry */
    for (int i = j + 1; i < n_crc; ++i) {
      const double v = 0.5 * (Ms[(size_t)i + (size_t)j * n_crc] + Ms[(size_t)j + (size_t)i * n_crc]);
      Ms[(size_t)i + (size_t)j * n_crc] = Ms[(size_t)j + (size_t)i * n_crc] = v;
    }
  rc = bko_jacobi_eig(n_crc, Ms, n_crc, lam, W, n_crc, 100, NULL);
  if (rc) goto done;
  mat_nn(d, n_crc, n_crc, Us, d, W, n_crc, Un, d);    /* U_s W */
  for (int a = 0; a < n_crc; ++a) {
    for (int i = 0; i < d; ++i) AT(U, ldu, i, idx[a]) = Un[(size_t)i + (size_t)a * d];
    sigma[idx[a]] = lam[a];
  }
  rc = sort_modes(d, k, U, ldu, sigma);
done:
  free(Us); free(MU); free(Ms); free(W); free(lam); free(Un);
  return rc;
}

/* ---------------------------------------------------------------------------
 * RSVD overwrite of a B-KFAC representation (Algorithm 5): randomised range
 * finder on the dense EA factor M (d x d) with the test matrix Omega (d x l,
 * ldo >= d, r <= l <= d) and q power iterations; orthonormal bases by
 * Householder QR (bko_qrcp without truncation).  Writes U (d x r) and sigma (r).
 * ------------------------------------------------------------------------- */
int bko_rsvd(int d, int r, int l, const double* M, long ldm, const double* Omega, long ldo, int q, double* U,
             long ldu, double* sigma) {
  if (d <= 0 || r < 1 || l < r || l > d || ldm < d || ldo < d || ldu < d || q < 0) return BKO_EINVAL;
  double* Y = (double*)malloc(sizeof(double) * (size_t)d * (size_t)l);
  double* Q = (double*)malloc(sizeof(double) * (size_t)d * (size_t)l);
  double* Rt = (double*)malloc(sizeof(double) * (size_t)l * (size_t)l);
  double* B = (double*)malloc(sizeof(double) * (size_t)l * (size_t)l);
  double* W = (double*)malloc(sizeof(double) * (size_t)l * (size_t)l);
  double* lam = (double*)malloc(sizeof(double) * (size_t)l);
  int rc = BKO_ENOMEM, m = 0;
  if (!Y || !Q || !Rt || !B || !W || !lam) goto done;
  mat_nn(d, l, d, M, ldm, Omega, ldo, Y, d);           /* Y = M Omega */
  for (int it = 0; it < q; ++it) {
    rc = bko_qrcp(d, l, Y, d, 0.0, Q, d, Rt, l, &m);
    if (rc) goto done;
    mat_nn(d, l, d, M, ldm, Q, d, Y, d);               /* Y = M Q */
  }
  rc = bko_qrcp(d, l, Y, d, 0.0, Q, d, Rt, l, &m);
  if (rc) goto done;
  mat_nn(d, l, d, M, ldm, Q, d, Y, d);                 /* M Q */
  mat_tn(l, l, d, Q, d, Y, d, B, l);                   /* B = Q^T M Q */
  for (int j = 0; j < l; ++j)
    for (int i = j + 1; i < l; ++i) {
      const double v = 0.5 * (B[(size_t)i + (size_t)j * l] + B[(size_t)j + (size_t)i * l]);
      B[(size_t)i + (size_t)j * l] = B[(size_t)j + (size_t)i * l] = v;
    }
  rc = bko_jacobi_eig(l, B, l, lam, W, l, 100, NULL);
  if (rc) goto done;
  mat_nn(d, r, l, Q, d, W, l, U, ldu);                 /* U = Q W[:, :r] */
  for (int j = 0; j < r; ++j) sigma[j] = lam[j];
  rc = BKO_OK;
done:
  free(Y); free(Q); free(Rt); free(B); free(W); free(lam);
  return rc;
}

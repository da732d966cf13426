// small.cu -- the small dense steps of the B-KFAC update and apply:
//   * column-norm scale of the new batch (the reference for dropped pivots),
//   * thresholded Cholesky of the CholeskyQR Gram (QR step of Algorithm 3),
//   * inverse of the triangular factor,
//   * assembly of the factor L of the Brand core (Eq. (7) with the
//     substitutions of Sec. 3.1), of the dense-path factor and of the reorth
//     factor,
//   * ordering of the Jacobi output into (V, sigma) with truncation to rank r
//     (Sec. 3.1),
//   * the damping coefficients of the inverse application (Algorithm 1) with
//     optional spectrum continuation (Sec. 3.5.1).
#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace bkfac {

__device__ int g_status = 0;

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// deterministic block sum (fixed tree), result valid in thread 0 and returned to all
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------- column norms
template <typename T>
__global__ void __launch_bounds__(256) colnorm_max_kernel(const T* X, int64_t ldx, int d, double* out) {
  __shared__ double red[32];
  const T* x = X + (int64_t)blockIdx.x * ldx;
  double s = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    double v = (double)x[i];
    s += v * v;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    if (!isfinite(s)) {
      report(BKFAC_ENONFINITE);
    } else {
      atomicMax((unsigned long long*)out, (unsigned long long)__double_as_longlong(s));
    }
  }
}

// ---------------------------------------------------------------- Cholesky
// Right-looking upper Cholesky G = R^T R in FP64, one CTA.  Pivot j is dropped
// (row j of R set to zero) when its Schur complement s_j <= thr; the matching
// direction of P is then (numerically) in the span of the kept ones.
__global__ void __launch_bounds__(1024) chol_kernel(const double* __restrict__ Gm, int n, double* R, double thr_rel,
                                                    const double* scale, double neg_rel) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const double thr = thr_rel * (scale ? *scale : 1.0);
  const double neg = neg_rel * (scale ? *scale : 1.0);  // pivots below -neg: not p.s.d.
  for (int l = 0; l < n; ++l)
    for (int i = tid; i < n; i += nt) R[i + l * n] = (i <= l) ? Gm[i + l * n] : 0.0;
  __syncthreads();
  __shared__ double s_piv[2];
  __shared__ int s_keep;
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      // one thread takes the pivot's square root and reciprocal (long FP64 sequences)
      const double s = R[j + (int64_t)j * n];
      s_keep = s > thr;  // false for NaN as well
      if (!isfinite(s)) report(BKFAC_ENONFINITE);
      if (neg_rel > 0.0 && s < -neg) report(BKFAC_ECHOL);
      if (s_keep) {
        s_piv[0] = sqrt(s);
        s_piv[1] = 1.0 / s_piv[0];
      }
    }
    __syncthreads();
    const bool keep = s_keep;
    if (keep) {
      const double rjj = s_piv[0];
      const double inv = s_piv[1];
      for (int l = j + tid; l < n; l += nt) R[j + (int64_t)l * n] = (l == j) ? rjj : R[j + (int64_t)l * n] * inv;
    } else {
      for (int l = j + tid; l < n; l += nt) R[j + (int64_t)l * n] = 0.0;
    }
    __syncthreads();
    if (keep) {
      // trailing update, a warp per column l, lanes over rows i in (j, l]
      const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
      for (int l = j + 1 + wid; l < n; l += nw) {
        const double rjl = R[j + (int64_t)l * n];
        for (int i = j + 1 + lane; i <= l; i += 32) R[i + (int64_t)l * n] -= R[j + (int64_t)i * n] * rjl;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- triangular inverse
// One warp per column j of Rinv, solving R x = e_j by column sweeps:
//   for l = j, j-1, ..., 0:  x_l = y_l / R_ll;  y_i -= R_il x_l  (i < l, lanes over i)
// so each step is a broadcast and an axpy -- no warp reduction on the critical
// path.  Zero diagonal (dropped pivot) -> zero row/column.  R's upper triangle
// is staged in shared memory packed by columns (column l holds rows 0..l), in
// the working type, when it fits; otherwise it is read from global memory.
__host__ __device__ __forceinline__ int64_t packed_col(int l) { return (int64_t)l * (l + 1) / 2; }

template <typename T, bool SMEM>
__global__ void __launch_bounds__(1024) trinv_kernel(const double* __restrict__ R, int n, T* Rinv) {
  extern __shared__ __align__(16) unsigned char tr_smem[];
  T* inv = (T*)tr_smem;                                  // reciprocal diagonal (0 for dropped pivots)
  T* Rs = inv + n;                                       // packed upper triangle by columns (SMEM only)
  T* ys = Rs + (SMEM ? packed_col(n) : 0);               // one working column per warp
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double rii = R[i + (int64_t)i * n];
    inv[i] = rii != 0.0 ? (T)(1.0 / rii) : T(0);
  }
  if (SMEM) {
    for (int l = wid; l < n; l += blockDim.x >> 5)
      for (int i = lane; i <= l; i += 32) Rs[packed_col(l) + i] = (T)R[i + (int64_t)l * n];
  }
  __syncthreads();
  const int j = blockIdx.x * 32 + wid;
  if (j >= n) return;
  T* y = ys + (int64_t)wid * n;
  for (int i = lane; i < n; i += 32) y[i] = (i == j) ? T(1) : T(0);
  __syncwarp();
  for (int l = j; l >= 0; --l) {
    const T xl = y[l] * inv[l];  // broadcast read
    __syncwarp();
    if (lane == 0) y[l] = xl;
    if (xl != T(0)) {
      if (SMEM) {
        const T* col = Rs + packed_col(l);
        for (int i = lane; i < l; i += 32) y[i] -= col[i] * xl;
      } else {
        for (int i = lane; i < l; i += 32) y[i] -= (T)R[i + (int64_t)l * n] * xl;
      }
    }
    __syncwarp();
  }
  T* out = Rinv + (int64_t)j * n;
  for (int i = lane; i < n; i += 32) out[i] = i <= j ? y[i] : T(0);
}

// Blocked inverse of the upper-triangular R for n <= 256 (at most 8 diagonal
// blocks of 32): CTA jb computes block column jb of R^-1 (32 columns) as
//   Y_B(jb) = D_jb^-1,  then for i = jb - 1, ..., 0:
//   Y_B(i) = -D_i^-1 sum_{k = i+1..jb} R_ik Y_B(k),
// organised as a block back-substitution: after Y_B(i) is final, every block
// above it receives its update -R_{i', i} Y_B(i) (i' < i) at once, so the
// sequential depth is the number of blocks, not n.  D_i^-1 (inverse of the
// 32 x 32 diagonal block) is computed first, one warp per block, one lane per
// column.  Dropped pivots (zero rows of R) give zero rows and columns.
//
// Near-identity pass (near != null and *near != 0, set by the Cholesky of the
// second CholeskyQR pass): R = I + F with |F| tiny, R^-1 = I - F + O(|F|^2),
// written directly.
template <typename T>
__global__ void __launch_bounds__(1024) trinv_blocked_kernel(const double* __restrict__ R, int n, T* Rinv,
                                                             const int* near) {
  extern __shared__ __align__(16) unsigned char tb_smem[];
  const int jb = blockIdx.x;
  const int nb = jb + 1;              // blocks 0..jb take part
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j0 = 32 * jb;
  if (near != nullptr && *near != 0) {
    for (int c = wid; c < 32; c += 32) {
      const int j = j0 + c;
      if (j >= n) break;
      for (int r = lane; r < n; r += 32) {
        const double v = R[r + (int64_t)j * n];
        Rinv[r + (int64_t)j * n] = (T)(r == j ? 2.0 - v : (r < j ? -v : 0.0));
      }
    }
    return;
  }
  T* Dinv = (T*)tb_smem;            // nb blocks, 32 x 32 column-major each
  T* Y = Dinv + nb * 1024;          // 32 nb rows x 32 columns, column-major (ld 32 nb)
  T* P = Y + nb * 1024;             // panel R[0 : 32 i, 32 i : 32 i + 32], column-major (ld 32 i)
  const int ldy = 32 * nb;
  // ---- diagonal block inverses: warp i < nb inverts D_i, staged in the Y area
  if (wid < nb) {
    T* Ds = Y + wid * 1024;
    const int o = 32 * wid;
    for (int m = 0; m < 32; ++m) {
      const int r = o + lane, c = o + m;
      Ds[lane + 32 * m] = (r < n && c < n) ? (T)R[r + (int64_t)c * n] : (lane == m ? T(1) : T(0));
    }
    __syncwarp();
    const T dll = Ds[lane + 32 * lane];
    const T inv_mine = dll != T(0) ? T(1) / dll : T(0);
    T x[32];
#pragma unroll
    for (int l = 31; l >= 0; --l) {
      T acc = (l == lane) ? T(1) : T(0);
#pragma unroll
      for (int m = l + 1; m < 32; ++m) acc -= Ds[l + 32 * m] * x[m];
      const T il = __shfl_sync(0xffffffffu, inv_mine, l);
      x[l] = (l <= lane) ? acc * il : T(0);
    }
    __syncwarp();
    T* Dw = Dinv + wid * 1024;
#pragma unroll
    for (int l = 0; l < 32; ++l) Dw[l + 32 * lane] = x[l];
  }
  __syncthreads();
  // ---- Y = e_{j0 .. j0 + 31} restricted to rows [0, 32 nb); thread (row = lane + 32 k, col = wid)
  const int c = wid;  // this warp's column of the block column
  for (int r = lane; r < ldy; r += 32) Y[r + ldy * c] = (r == j0 + c) ? T(1) : T(0);
  __syncthreads();
  for (int i = jb; i >= 0; --i) {
    // Y_B(i) <- D_i^-1 Y_B(i)
    const T* Di = Dinv + i * 1024;
    T v = T(0);
#pragma unroll 8
    for (int k = 0; k < 32; ++k) v += Di[lane + 32 * k] * Y[32 * i + k + ldy * c];
    __syncthreads();
    Y[32 * i + lane + ldy * c] = v;
    if (i == 0) break;
    // panel R[0 : 32 i, 32 i : 32 i + 32] into shared memory
    const int pr = 32 * i;
    for (int e = threadIdx.x; e < pr * 32; e += blockDim.x) {
      const int r = e % pr, k = e / pr;
      const int col = 32 * i + k;
      P[e] = (col < n) ? (T)R[r + (int64_t)col * n] : T(0);
    }
    __syncthreads();
    // Y_B(i') -= R_{i', i} Y_B(i) for every block i' < i
    for (int r = lane; r < pr; r += 32) {
      T acc = T(0);
#pragma unroll 8
      for (int k = 0; k < 32; ++k) acc += P[r + pr * k] * Y[32 * i + k + ldy * c];
      Y[r + ldy * c] -= acc;
    }
    __syncthreads();
  }
  __syncthreads();
  const int j = j0 + c;
  if (j < n)
    for (int r = lane; r < n; r += 32) Rinv[r + (int64_t)j * n] = (r < ldy && r <= j) ? Y[r + ldy * c] : T(0);
}

// ---------------------------------------------------------------- core factor L
// L = [[diag(sqrt(rho sigma)), sqrt(c) M], [0, sqrt(c) R2 R1]]  so that
// L L^T = M_S of Eq. (7) with D <- rho diag(sigma), A <- sqrt(c) X, R = R2 R1.
// One block per column of L.
template <typename TM, typename J>
__global__ void __launch_bounds__(256) assemble_core_kernel(const CoreArgs a) {
  __shared__ double red[32];
  __shared__ J s_r1[1024];  // column jj of R1 (n <= 1024)
  const int j = blockIdx.x;
  J* col = (J*)a.L + (int64_t)j * a.rows_pad;
  const double sc = sqrt(a.c);
  const int jj = j - a.k;
  if (j >= a.k && j < a.N)
    for (int l = threadIdx.x; l <= jj; l += blockDim.x) s_r1[l] = (J)a.R1[l + (int64_t)jj * a.n];
  __syncthreads();
  double ss = 0.0;
  for (int i = threadIdx.x; i < a.rows_pad; i += blockDim.x) {
    double v = 0.0;
    if (j < a.k) {
      if (i == j) v = sqrt(a.rho * a.sigma[j]);
    } else if (j < a.N && i < a.N) {
      if (i < a.k) {
        v = sc * (double)((const TM*)a.M)[i + (int64_t)jj * a.ldm];
      } else {
        const int ii = i - a.k;
        if (ii <= jj) {
          // (R2 R1)[ii, jj] = sum_{l = ii..jj} R2[ii, l] R1[l, jj]; accumulate in the Jacobi
          // type, four partial sums so that four loads of R2 are in flight
          J s0 = J(0), s1 = J(0), s2 = J(0), s3 = J(0);
          const double* r2 = a.R2 + ii;
          int l = ii;
          for (; l + 3 <= jj; l += 4) {
            const J x0 = (J)r2[(int64_t)l * a.n], x1 = (J)r2[(int64_t)(l + 1) * a.n];
            const J x2 = (J)r2[(int64_t)(l + 2) * a.n], x3 = (J)r2[(int64_t)(l + 3) * a.n];
            s0 += x0 * s_r1[l];
            s1 += x1 * s_r1[l + 1];
            s2 += x2 * s_r1[l + 2];
            s3 += x3 * s_r1[l + 3];
          }
          for (; l <= jj; ++l) s0 += (J)r2[(int64_t)l * a.n] * s_r1[l];
          v = sc * (double)((s0 + s1) + (s2 + s3));
        }
      }
    }
    const J jv = (J)v;
    col[i] = jv;
    ss += (double)jv * (double)jv;
  }
  ss = block_sum(ss, red);
  if (threadIdx.x == 0) {
    a.colnorm2[j] = ss;
    if (!isfinite(ss)) report(BKFAC_ENONFINITE);
  }
}

// ---------------------------------------------------------------- dense-path factor
// F = [U diag(sqrt(rho sigma)), sqrt(c) X]: F F^T = rho U diag(sigma) U^T + c X X^T.
template <typename TU, typename J>
__global__ void __launch_bounds__(256) assemble_dense_kernel(const DenseArgs a) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  J* col = (J*)a.F + (int64_t)j * a.rows_pad;
  double ss = 0.0;
  double scale = 0.0;
  const TU* src = nullptr;
  if (j < a.k) {
    scale = sqrt(a.rho * a.sigma[j]);
    src = (const TU*)a.U + (int64_t)j * a.ldu;
  } else if (j < a.k + a.n) {
    scale = sqrt(a.c);
    src = (const TU*)a.X + (int64_t)(j - a.k) * a.ldx;
  }
  for (int i = threadIdx.x; i < a.rows_pad; i += blockDim.x) {
    const double v = (src && i < a.d) ? scale * (double)src[i] : 0.0;
    const J jv = (J)v;
    col[i] = jv;
    ss += (double)jv * (double)jv;
  }
  ss = block_sum(ss, red);
  if (threadIdx.x == 0) {
    a.colnorm2[j] = ss;
    if (!isfinite(ss)) report(BKFAC_ENONFINITE);
  }
}

// ---------------------------------------------------------------- reorth factor
template <typename J>
__global__ void __launch_bounds__(256) assemble_reorth_kernel(const double* R, const double* sigma, int k,
                                                              int rows_pad, J* L, double* colnorm2) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  J* col = L + (int64_t)j * rows_pad;
  const double sj = j < k ? sqrt(fmax(sigma[j], 0.0)) : 0.0;
  double ss = 0.0;
  for (int i = threadIdx.x; i < rows_pad; i += blockDim.x) {
    const double v = (j < k && i <= j) ? R[i + (int64_t)j * k] * sj : 0.0;
    const J jv = (J)v;
    col[i] = jv;
    ss += (double)jv * (double)jv;
  }
  ss = block_sum(ss, red);
  if (threadIdx.x == 0) colnorm2[j] = ss;
}

// ---------------------------------------------------------------- sort / output
// lambda_i = ||w_i||^2 (the eigenvalues of W W^T), eigenvectors w_i / ||w_i||,
// ordered descending with ties broken by column index; the first r_out go to
// (V, sig).  Columns whose norm is at the rounding level of the input (relative
// to ||W||_F^2) are returned as zero vectors with sigma = 0.  Norms, ordering and
// scaling are in the Jacobi type J (FP32 arithmetic for the FP32 paths); only the
// eigenvalues handed back are widened to double.  Two kernels over many blocks (a
// warp per column), so that the loads of W overlap across the GPU.

// squared column norms (the J value, stored as double), four loads in flight per lane
template <typename J>
__global__ void __launch_bounds__(256) col_sumsq_kernel(const J* __restrict__ W, int rows, int rows_pad, int cols,
                                                        double* out) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= cols) return;
  const J* w = W + (int64_t)i * rows_pad;
  J s0 = J(0), s1 = J(0), s2 = J(0), s3 = J(0);
  int r = lane;
  for (; r + 96 < rows; r += 128) {
    const J v0 = w[r], v1 = w[r + 32], v2 = w[r + 64], v3 = w[r + 96];
    s0 += v0 * v0;
    s1 += v1 * v1;
    s2 += v2 * v2;
    s3 += v3 * v3;
  }
  for (; r < rows; r += 32) s0 += w[r] * w[r];
  J sum = (s0 + s1) + (s2 + s3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) out[i] = (double)sum;
}

// rank of each column (a warp per column, lanes over the others) and the output
template <typename J, typename TO>
__global__ void __launch_bounds__(256) sort_write_kernel(const SortArgs a, const double* __restrict__ norms) {
  extern __shared__ __align__(16) unsigned char so_smem[];
  J* lam = (J*)so_smem;  // cols
  __shared__ double s_tiny;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < a.cols; j += blockDim.x) lam[j] = (J)norms[j];
  if (wid == 0) {
    // deterministic: fixed lane assignment, fixed shuffle tree
    double f = 0.0;
    for (int j = lane; j < a.cols_pad; j += 32) f += a.colnorm2[j];
    f = warp_sum(f);
    if (lane == 0) s_tiny = 16.0 * Eps<J>::u * Eps<J>::u * f;
  }
  __syncthreads();
  if (blockIdx.x == 0 && a.sig)
    for (int j = a.r_out + threadIdx.x; j < a.r_sig; j += blockDim.x) a.sig[j] = 0.0;
  const int i = blockIdx.x * 8 + wid;
  if (i >= a.cols) return;
  const J tiny = (J)s_tiny;
  const J li = lam[i];
  int rk = 0;
  for (int j = lane; j < a.cols; j += 32) {
    const J lj = lam[j];
    rk += (lj > li) || (lj == li && j < i);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
  if (lane == 0) {
    if (!isfinite(li)) report(BKFAC_ENONFINITE);
    if (a.lam_sorted) a.lam_sorted[rk] = (double)li;
    if (rk < a.r_out && a.sig) a.sig[rk] = li > tiny ? (double)li : 0.0;
  }
  if (rk >= a.r_out) return;
  const J sc = li > tiny ? J(1) / sqrt(li) : J(0);
  const J* w = (const J*)a.W + (int64_t)i * a.rows_pad;
  TO* v = (TO*)a.V + (int64_t)rk * a.ldv;
#pragma unroll 4
  for (int r = lane; r < a.rows; r += 32) v[r] = (TO)(w[r] * sc);
}

// ---------------------------------------------------------------- finalize
template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(T* U, int64_t ldu, const T* Un, int64_t ldn, int d, int r_new,
                                                       int r) {
  // a block row of threads per column: grid.y over columns, grid.x over rows
  for (int j = blockIdx.y; j < r; j += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
      U[i + (int64_t)j * ldu] = j < r_new ? Un[i + (int64_t)j * ldn] : T(0);
}

// ---------------------------------------------------------------- apply coefficients
__global__ void __launch_bounds__(256) apply_coefs_kernel(const ApplyCoefArgs a) {
  __shared__ double smin[2], slam[2];
  if (threadIdx.x < 2) {
    const double* sg = threadIdx.x == 0 ? a.sigA : a.sigG;
    const int k = threadIdx.x == 0 ? a.kA : a.kG;
    double lam = threadIdx.x == 0 ? a.lamA : a.lamG;
    if (a.relative && k > 0) {
      // lambda = phi * (largest eigenvalue of the represented factor)
      double top = sg[0];
      for (int i = 1; i < k; ++i) top = fmax(top, sg[i]);
      lam *= top;
      if (!(lam > 0.0)) report(BKFAC_ENONFINITE);
    }
    double m = 0.0;
    if (a.continuation && k > 0) {
      m = sg[0];
      for (int i = 1; i < k; ++i) m = fmin(m, sg[i]);
    }
    smin[threadIdx.x] = m;
    slam[threadIdx.x] = lam;
  }
  __syncthreads();
  const double shA = smin[0], shG = smin[1];
  const double lA = slam[0] + shA, lG = slam[1] + shG;
  // (U Sigma U^T + lambda I)^-1 = beta I + U C U^T with beta = 1/lambda' for the
  // complement of span(U) and C = (Sigma + lambda)^-1 - beta.  A complete basis
  // (r_cur = d) leaves no complement: beta = 0 and C = (Sigma + lambda)^-1, the same
  // operator without the cancellation of beta I against U (-beta) U^T, which
  // rounded (BF16) bases do not reproduce.
  const double bA = a.completeA ? 0.0 : 1.0 / lA, bG = a.completeG ? 0.0 : 1.0 / lG;
  for (int i = threadIdx.x; i < a.kA; i += blockDim.x) {
    const double c = 1.0 / ((a.sigA[i] - shA) + lA) - bA;
    a.cA[i] = c;
    a.cA_over[i] = c * bG;
  }
  for (int i = threadIdx.x; i < a.kG; i += blockDim.x) {
    const double c = 1.0 / ((a.sigG[i] - shG) + lG) - bG;
    a.cG[i] = c;
    a.cG_over[i] = c * bA;
  }
  if (threadIdx.x == 0) {
    *a.alpha = bA * bG;
    if (a.betaA) *a.betaA = bA;
    if (a.betaG) *a.betaG = bG;
  }
}

// ---------------------------------------------------------------- B-KFAC-C / B-R-KFAC helpers
// dst[:, j] = src[:, idx[j]] (idx null: the identity), d rows, grid.y over columns
template <typename T>
__global__ void __launch_bounds__(256) gather_cols_kernel(const T* src, int64_t lds, T* dst, int64_t ldd, int d,
                                                          int n, const int* idx) {
  for (int j = blockIdx.y; j < n; j += gridDim.y) {
    const int64_t c = idx ? idx[j] : j;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
      dst[i + (int64_t)j * ldd] = src[i + c * lds];
  }
}
// dst[:, idx[j]] = src[:, j] and sig[idx[j]] = lam[j]
template <typename T>
__global__ void __launch_bounds__(256) scatter_cols_kernel(const T* src, int64_t lds, T* dst, int64_t ldd, int d,
                                                           int n, const int* idx, const double* lam, double* sig) {
  for (int j = blockIdx.y; j < n; j += gridDim.y) {
    const int64_t c = idx[j];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
      dst[i + c * ldd] = src[i + (int64_t)j * lds];
    if (blockIdx.x == 0 && threadIdx.x == 0) sig[c] = lam[j];
  }
}
// out = max_i G[i, i] (n x n, column-major ld n)
__global__ void __launch_bounds__(256) diag_max_kernel(const double* G, int n, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, G[i + (int64_t)i * n]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    *out = t;
  }
}
// Jacobi input L = R^T (R n x n upper, column-major ld n: L is lower, L L^T = R^T R),
// zero padded to rows_pad x cols_pad, with squared column norms; one block per column
template <typename J>
__global__ void __launch_bounds__(256) assemble_transpose_kernel(const double* R, int n, int rows_pad, int cols_pad,
                                                                 J* L, double* colnorm2) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  J* col = L + (int64_t)j * rows_pad;
  double ss = 0.0;
  for (int i = threadIdx.x; i < rows_pad; i += blockDim.x) {
    const J v = (j < n && i < n && i >= j) ? (J)R[j + (int64_t)i * n] : J(0);
    col[i] = v;
    ss += (double)v * (double)v;
  }
  ss = block_sum(ss, red);
  if (threadIdx.x == 0) {
    colnorm2[j] = ss;
    if (!isfinite(ss)) report(BKFAC_ENONFINITE);
  }
}
// stable order of k modes by decreasing sigma: perm[rank] = i, sorted[rank] = sigma[i]
__global__ void __launch_bounds__(1024) mode_order_kernel(const double* sig, int k, int* perm, double* sorted) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double si = sig[i];
    if (!isfinite(si)) report(BKFAC_ENONFINITE);
    int rk = 0;
    for (int j = 0; j < k; ++j) {
      const double sj = sig[j];
      rk += (sj > si) || (sj == si && j < i);
    }
    perm[rk] = i;
    sorted[rk] = si;
  }
}

}  // namespace

// ============================================================================ launchers

int launch_colnorm_max(const void* X, int64_t ldx, int d, int n, DType t, double* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(double), s);
  if (n <= 0) return (int)cudaGetLastError();
  if (t == DT_F64)
    colnorm_max_kernel<double><<<n, 256, 0, s>>>((const double*)X, ldx, d, out);
  else
    colnorm_max_kernel<float><<<n, 256, 0, s>>>((const float*)X, ldx, d, out);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_chol(const double* Gm, int n, double* R, double thr_rel, const double* scale, double neg_rel,
                cudaStream_t s) {
  if (n <= 0) return 0;
  chol_kernel<<<1, 1024, 0, s>>>(Gm, n, R, thr_rel, scale, neg_rel);
  note_launches(1);
  return (int)cudaGetLastError();
}

template <typename T>
void trinv_launch(const double* R, int n, T* Rinv, cudaStream_t s) {
  static std::atomic<uint64_t> configured{0};  // attribute set once (the call can stall the host)
  if (!configured_here(configured)) {
    cudaFuncSetAttribute(trinv_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(trinv_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    mark_configured(configured);
  }
  const int blocks = (int)ceil_div(n, 32);
  const size_t xs = (size_t)32 * n * sizeof(T) + (size_t)n * sizeof(T);
  const size_t rs = (size_t)(packed_col(n)) * sizeof(T);
  if (rs + xs <= 220 * 1024)
    trinv_kernel<T, true><<<blocks, 1024, rs + xs, s>>>(R, n, Rinv);
  else
    trinv_kernel<T, false><<<blocks, 1024, xs, s>>>(R, n, Rinv);
}

template <typename T>
void trinv_blocked_launch(const double* R, int n, T* Rinv, const int* near, cudaStream_t s) {
  static std::atomic<uint64_t> configured{0};  // attribute set once (the call can stall the host)
  if (!configured_here(configured)) {
    cudaFuncSetAttribute(trinv_blocked_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    mark_configured(configured);
  }
  const int nb = (int)ceil_div(n, 32);
  const size_t smem = (size_t)3 * nb * 1024 * sizeof(T);
  trinv_blocked_kernel<T><<<nb, 1024, smem, s>>>(R, n, Rinv, near);
}

int launch_trinv(const double* R, int n, void* Rinv, DType t, const int* near, cudaStream_t s) {
  if (n <= 0) return 0;
  if (n <= 256) {
    if (t == DT_F64)
      trinv_blocked_launch<double>(R, n, (double*)Rinv, near, s);
    else
      trinv_blocked_launch<float>(R, n, (float*)Rinv, near, s);
  } else if (t == DT_F64) {
    trinv_launch<double>(R, n, (double*)Rinv, s);
  } else {
    trinv_launch<float>(R, n, (float*)Rinv, s);
  }
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_assemble_core(const CoreArgs& a, DType m_t, DType j_t, cudaStream_t s) {
  if (m_t == DT_F64 && j_t == DT_F64)
    assemble_core_kernel<double, double><<<a.cols_pad, 256, 0, s>>>(a);
  else if (m_t == DT_F32 && j_t == DT_F32)
    assemble_core_kernel<float, float><<<a.cols_pad, 256, 0, s>>>(a);
  else if (m_t == DT_F32 && j_t == DT_F64)
    assemble_core_kernel<float, double><<<a.cols_pad, 256, 0, s>>>(a);
  else
    assemble_core_kernel<double, float><<<a.cols_pad, 256, 0, s>>>(a);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_assemble_dense(const DenseArgs& a, DType u_t, DType j_t, cudaStream_t s) {
  if (u_t == DT_F64 && j_t == DT_F64)
    assemble_dense_kernel<double, double><<<a.cols_pad, 256, 0, s>>>(a);
  else if (u_t == DT_F32 && j_t == DT_F32)
    assemble_dense_kernel<float, float><<<a.cols_pad, 256, 0, s>>>(a);
  else if (u_t == DT_F32 && j_t == DT_F64)
    assemble_dense_kernel<float, double><<<a.cols_pad, 256, 0, s>>>(a);
  else
    assemble_dense_kernel<double, float><<<a.cols_pad, 256, 0, s>>>(a);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_assemble_reorth(const double* R, const double* sigma, int k, int rows_pad, int cols_pad, void* L,
                           double* colnorm2, DType j_t, cudaStream_t s) {
  if (j_t == DT_F64)
    assemble_reorth_kernel<double><<<cols_pad, 256, 0, s>>>(R, sigma, k, rows_pad, (double*)L, colnorm2);
  else
    assemble_reorth_kernel<float><<<cols_pad, 256, 0, s>>>(R, sigma, k, rows_pad, (float*)L, colnorm2);
  note_launches(1);
  return (int)cudaGetLastError();
}

template <typename J, typename TO>
void sort_launch(const SortArgs& a, double* norms, cudaStream_t s) {
  const unsigned blocks = (unsigned)ceil_div(a.cols, 8);
  col_sumsq_kernel<J><<<blocks, 256, 0, s>>>((const J*)a.W, a.rows, a.rows_pad, a.cols, norms);
  sort_write_kernel<J, TO><<<blocks, 256, (size_t)a.cols * sizeof(J), s>>>(a, norms);
}

int launch_sort_output(const SortArgs& a, DType j_t, DType out_t, cudaStream_t s) {
  if (a.cols <= 0) return 0;
  if ((size_t)a.cols * sizeof(double) > 48 * 1024 || a.lam_sorted == nullptr) return (int)cudaErrorInvalidValue;
  double* norms = a.lam_sorted + a.cols;  // the second half of lam_sorted is scratch
  if (j_t == DT_F64 && out_t == DT_F64)
    sort_launch<double, double>(a, norms, s);
  else if (j_t == DT_F32 && out_t == DT_F32)
    sort_launch<float, float>(a, norms, s);
  else if (j_t == DT_F64 && out_t == DT_F32)
    sort_launch<double, float>(a, norms, s);
  else
    sort_launch<float, double>(a, norms, s);
  note_launches(2);
  return (int)cudaGetLastError();
}

int launch_finalize(void* U, int64_t ldu, const void* Unew, int64_t ldn, int d, int r_new, int r, DType t,
                    cudaStream_t s) {
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(d, 256), 16)),
                  (unsigned)std::max(1, std::min(r, 1024)));
  if (t == DT_F64)
    finalize_kernel<double><<<grid, 256, 0, s>>>((double*)U, ldu, (const double*)Unew, ldn, d, r_new, r);
  else
    finalize_kernel<float><<<grid, 256, 0, s>>>((float*)U, ldu, (const float*)Unew, ldn, d, r_new, r);
  note_launches(1);
  return (int)cudaGetLastError();
}

namespace {
dim3 col_grid(int d, int n) {
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(d, 256), 16)),
              (unsigned)std::max(1, std::min(n, 1024)));
}
}  // namespace

int launch_gather_cols(const void* src, int64_t lds, void* dst, int64_t ldd, int d, int n, const int* idx, DType t,
                       cudaStream_t s) {
  if (n <= 0 || d <= 0) return 0;
  if (t == DT_F64)
    gather_cols_kernel<double><<<col_grid(d, n), 256, 0, s>>>((const double*)src, lds, (double*)dst, ldd, d, n, idx);
  else
    gather_cols_kernel<float><<<col_grid(d, n), 256, 0, s>>>((const float*)src, lds, (float*)dst, ldd, d, n, idx);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_scatter_cols(const void* src, int64_t lds, void* dst, int64_t ldd, int d, int n, const int* idx,
                        const double* lam, double* sig, DType t, cudaStream_t s) {
  if (n <= 0 || d <= 0) return 0;
  if (t == DT_F64)
    scatter_cols_kernel<double><<<col_grid(d, n), 256, 0, s>>>((const double*)src, lds, (double*)dst, ldd, d, n,
                                                                idx, lam, sig);
  else
    scatter_cols_kernel<float><<<col_grid(d, n), 256, 0, s>>>((const float*)src, lds, (float*)dst, ldd, d, n, idx,
                                                               lam, sig);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_diag_max(const double* G, int n, double* out, cudaStream_t s) {
  diag_max_kernel<<<1, 256, 0, s>>>(G, n, out);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_assemble_transpose(const double* R, int n, int rows_pad, int cols_pad, void* L, double* colnorm2,
                              DType j_t, cudaStream_t s) {
  if (j_t == DT_F64)
    assemble_transpose_kernel<double><<<cols_pad, 256, 0, s>>>(R, n, rows_pad, cols_pad, (double*)L, colnorm2);
  else
    assemble_transpose_kernel<float><<<cols_pad, 256, 0, s>>>(R, n, rows_pad, cols_pad, (float*)L, colnorm2);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_mode_order(const double* sig, int k, int* perm, double* sorted, cudaStream_t s) {
  if (k <= 0) return 0;
  mode_order_kernel<<<1, 1024, 0, s>>>(sig, k, perm, sorted);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_apply_coefs(const ApplyCoefArgs& a, cudaStream_t s) {
  apply_coefs_kernel<<<1, 256, 0, s>>>(a);
  note_launches(1);
  return (int)cudaGetLastError();
}

}  // namespace bkfac

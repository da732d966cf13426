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
                                                    const double* scale) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const double thr = thr_rel * (scale ? *scale : 1.0);
  for (int e = tid; e < n * n; e += nt) {
    const int i = e % n, l = e / n;
    R[e] = (i <= l) ? Gm[e] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double s = R[j + (int64_t)j * n];
    const bool keep = s > thr;  // false for NaN as well
    if (!isfinite(s) && tid == 0) report(BKFAC_ENONFINITE);
    __syncthreads();  // everyone has read the pivot before it is overwritten
    if (keep) {
      const double rjj = sqrt(s);
      const double inv = 1.0 / rjj;
      for (int l = j + tid; l < n; l += nt) R[j + (int64_t)l * n] = (l == j) ? rjj : R[j + (int64_t)l * n] * inv;
    } else {
      for (int l = j + tid; l < n; l += nt) R[j + (int64_t)l * n] = 0.0;
    }
    __syncthreads();
    if (keep) {
      const int m = n - j - 1;
      for (int e = tid; e < m * m; e += nt) {
        const int i = j + 1 + e % m, l = j + 1 + e / m;
        if (i <= l) R[i + (int64_t)l * n] -= R[j + (int64_t)i * n] * R[j + (int64_t)l * n];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- triangular inverse
// one warp per column j of Rinv: back substitution R x = e_j, the dot products
// split over the lanes.  Zero diagonal (dropped pivot) -> zero row/column.
template <typename T>
__global__ void __launch_bounds__(1024) trinv_kernel(const double* __restrict__ R, int n, T* Rinv) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 32 + (threadIdx.x >> 5);
  if (j >= n) return;
  T* x = Rinv + (int64_t)j * n;
  for (int i = lane; i < n; i += 32) x[i] = T(0);
  __syncwarp();
  const double rjj = R[j + (int64_t)j * n];
  if (lane == 0) x[j] = rjj != 0.0 ? (T)(1.0 / rjj) : T(0);
  __syncwarp();
  for (int i = j - 1; i >= 0; --i) {
    const double rii = R[i + (int64_t)i * n];
    T s = T(0);
    for (int l = i + 1 + lane; l <= j; l += 32) s += (T)R[i + (int64_t)l * n] * x[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[i] = rii != 0.0 ? (T)(-(double)s / rii) : T(0);
    __syncwarp();
  }
}

// ---------------------------------------------------------------- core factor L
// L = [[diag(sqrt(rho sigma)), sqrt(c) M], [0, sqrt(c) R2 R1]]  so that
// L L^T = M_S of Eq. (7) with D <- rho diag(sigma), A <- sqrt(c) X, R = R2 R1.
// One block per column of L.
template <typename TM, typename J>
__global__ void __launch_bounds__(256) assemble_core_kernel(const CoreArgs a) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  J* col = (J*)a.L + (int64_t)j * a.rows_pad;
  const double sc = sqrt(a.c);
  double ss = 0.0;
  for (int i = threadIdx.x; i < a.rows_pad; i += blockDim.x) {
    double v = 0.0;
    if (j < a.k) {
      if (i == j) v = sqrt(a.rho * a.sigma[j]);
    } else if (j < a.N && i < a.N) {
      const int jj = j - a.k;
      if (i < a.k) {
        v = sc * (double)((const TM*)a.M)[i + (int64_t)jj * a.ldm];
      } else {
        const int ii = i - a.k;
        if (ii <= jj) {
          // (R2 R1)[ii, jj] = sum_{l = ii..jj} R2[ii, l] R1[l, jj]; accumulate in the Jacobi type
          J s = J(0);
          for (int l = ii; l <= jj; ++l) s += (J)a.R2[ii + (int64_t)l * a.n] * (J)a.R1[l + (int64_t)jj * a.n];
          v = sc * (double)s;
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
// to ||W||_F^2) are returned as zero vectors with sigma = 0.
template <typename J, typename TO>
__global__ void __launch_bounds__(1024) sort_output_kernel(const SortArgs a) {
  extern __shared__ double lam[];  // cols
  int* rank = (int*)(lam + a.cols);
  __shared__ double red[32];
  __shared__ double s_tiny;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const J* W = (const J*)a.W;
  if (wid == 0) {
    // deterministic: fixed lane assignment, fixed shuffle tree
    double f = 0.0;
    for (int j = lane; j < a.cols_pad; j += 32) f += a.colnorm2[j];
    f = warp_sum(f);
    if (lane == 0) s_tiny = 16.0 * Eps<J>::u * Eps<J>::u * f;
  }
  for (int i = wid; i < a.cols; i += nw) {
    const J* w = W + (int64_t)i * a.rows_pad;
    double s = 0.0;
    for (int r = lane; r < a.rows; r += 32) {
      const double v = (double)w[r];
      s += v * v;
    }
    s = warp_sum(s);
    if (lane == 0) lam[i] = s;
  }
  __syncthreads();
  const double tiny = s_tiny;
  for (int i = threadIdx.x; i < a.cols; i += blockDim.x) {
    const double li = lam[i];
    int rk = 0;
    for (int j = 0; j < a.cols; ++j) {
      const double lj = lam[j];
      rk += (lj > li) || (lj == li && j < i);
    }
    rank[i] = rk;
    if (!isfinite(li)) report(BKFAC_ENONFINITE);
    if (a.lam_sorted) a.lam_sorted[rk] = li;
    if (rk < a.r_out && a.sig) a.sig[rk] = li > tiny ? li : 0.0;
  }
  if (a.sig)
    for (int j = a.r_out + threadIdx.x; j < a.r_sig; j += blockDim.x) a.sig[j] = 0.0;
  __syncthreads();
  (void)red;
  // write the selected columns, one warp per column
  for (int i = wid; i < a.cols; i += nw) {
    const int rk = rank[i];
    if (rk >= a.r_out) continue;
    const double li = lam[i];
    const double inv = li > tiny ? 1.0 / sqrt(li) : 0.0;
    const J* w = W + (int64_t)i * a.rows_pad;
    TO* v = (TO*)a.V + (int64_t)rk * a.ldv;
    for (int r = lane; r < a.rows; r += 32) v[r] = (TO)((double)w[r] * inv);
  }
}

// ---------------------------------------------------------------- finalize
template <typename T>
__global__ void __launch_bounds__(256) finalize_kernel(T* U, int64_t ldu, const T* Un, int64_t ldn, int d, int r_new,
                                                       int r) {
  const int64_t total = (int64_t)d * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % d), j = (int)(e / d);
    U[i + (int64_t)j * ldu] = j < r_new ? Un[i + (int64_t)j * ldn] : T(0);
  }
}

// ---------------------------------------------------------------- apply coefficients
__global__ void __launch_bounds__(256) apply_coefs_kernel(const ApplyCoefArgs a) {
  __shared__ double smin[2];
  if (threadIdx.x < 2) {
    const double* sg = threadIdx.x == 0 ? a.sigA : a.sigG;
    const int k = threadIdx.x == 0 ? a.kA : a.kG;
    double m = 0.0;
    if (a.continuation && k > 0) {
      m = sg[0];
      for (int i = 1; i < k; ++i) m = fmin(m, sg[i]);
    }
    smin[threadIdx.x] = m;
  }
  __syncthreads();
  const double shA = smin[0], shG = smin[1];
  const double lA = a.lamA + shA, lG = a.lamG + shG;
  for (int i = threadIdx.x; i < a.kA; i += blockDim.x) {
    const double c = 1.0 / ((a.sigA[i] - shA) + lA) - 1.0 / lA;
    a.cA[i] = c;
    a.cA_over[i] = c / lG;
  }
  for (int i = threadIdx.x; i < a.kG; i += blockDim.x) {
    const double c = 1.0 / ((a.sigG[i] - shG) + lG) - 1.0 / lG;
    a.cG[i] = c;
    a.cG_over[i] = c / lA;
  }
  if (threadIdx.x == 0) *a.alpha = 1.0 / (lA * lG);
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

int launch_chol(const double* Gm, int n, double* R, double thr_rel, const double* scale, cudaStream_t s) {
  if (n <= 0) return 0;
  chol_kernel<<<1, 1024, 0, s>>>(Gm, n, R, thr_rel, scale);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_trinv(const double* R, int n, void* Rinv, DType t, cudaStream_t s) {
  if (n <= 0) return 0;
  const int blocks = (int)ceil_div(n, 32);
  if (t == DT_F64)
    trinv_kernel<double><<<blocks, 1024, 0, s>>>(R, n, (double*)Rinv);
  else
    trinv_kernel<float><<<blocks, 1024, 0, s>>>(R, n, (float*)Rinv);
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

int launch_sort_output(const SortArgs& a, DType j_t, DType out_t, cudaStream_t s) {
  const size_t smem = (size_t)a.cols * (sizeof(double) + sizeof(int));
  if (smem > 200 * 1024) return (int)cudaErrorInvalidValue;
  if (j_t == DT_F64 && out_t == DT_F64) {
    cudaFuncSetAttribute(sort_output_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sort_output_kernel<double, double><<<1, 1024, smem, s>>>(a);
  } else if (j_t == DT_F32 && out_t == DT_F32) {
    cudaFuncSetAttribute(sort_output_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sort_output_kernel<float, float><<<1, 1024, smem, s>>>(a);
  } else if (j_t == DT_F64 && out_t == DT_F32) {
    cudaFuncSetAttribute(sort_output_kernel<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sort_output_kernel<double, float><<<1, 1024, smem, s>>>(a);
  } else {
    cudaFuncSetAttribute(sort_output_kernel<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sort_output_kernel<float, double><<<1, 1024, smem, s>>>(a);
  }
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_finalize(void* U, int64_t ldu, const void* Unew, int64_t ldn, int d, int r_new, int r, DType t,
                    cudaStream_t s) {
  const int64_t total = (int64_t)d * r;
  const int blocks = (int)std::min<int64_t>(std::max<int64_t>(1, ceil_div(total, 256)), 2048);
  if (t == DT_F64)
    finalize_kernel<double><<<blocks, 256, 0, s>>>((double*)U, ldu, (const double*)Unew, ldn, d, r_new, r);
  else
    finalize_kernel<float><<<blocks, 256, 0, s>>>((float*)U, ldu, (const float*)Unew, ldn, d, r_new, r);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_apply_coefs(const ApplyCoefArgs& a, cudaStream_t s) {
  apply_coefs_kernel<<<1, 256, 0, s>>>(a);
  note_launches(1);
  return (int)cudaGetLastError();
}

}  // namespace bkfac

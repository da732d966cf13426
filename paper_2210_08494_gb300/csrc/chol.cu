// chol.cu -- the Cholesky factorisations of CholeskyQR2 (the QR step of
// Algorithm 3) in FP64, spread over a thread-block cluster.
//
// G = L L^T (L lower; the library stores R = L^T, n x n upper, column-major).
// CTA q of the cluster owns the column block [q w, q w + w) of L in shared
// memory.  For panel p = 0, 1, ...: the owner factors its block (right-looking,
// w columns), the cluster synchronises on the hardware barrier, and every CTA
// that owns a later block reads the panel from the owner's shared memory
// (distributed shared memory) and applies its rank-w update.  Pivots whose
// Schur complement is <= thr are dropped (the column of L is zeroed); the
// matching direction of the residual is numerically in the span of the kept
// ones.
//
// Near-identity shortcut (the second CholeskyQR pass): when G = I + E with
// max|E_ij| <= near_tol, the factor is R = I + Phi(E) with Phi(E) the strict
// upper part of E plus half its diagonal.  (I + F)^T (I + F) = I + E - F^T F,
// so the factor is exact up to O(|E|^2), below the working precision for the
// tolerances used; every CTA evaluates the same test, so the whole cluster
// takes the same branch.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bkfac {
namespace {

constexpr int CT = 512;

__global__ void __launch_bounds__(CT) chol_cluster_kernel(const double* __restrict__ Gm, int n, double* R,
                                                          double thr_rel, const double* scale, double near_tol,
                                                          int* near_out) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const int w = (n + C - 1) / C;
  const int c0 = q * w;
  const int wq = max(0, min(w, n - c0));
  extern __shared__ __align__(16) double csm[];
  double* A = csm;            // own block, n x w, column-major (ld n)
  double* Pb = csm + n * w;   // copy of the current remote panel
  __shared__ int s_flag[2];   // [0]: this CTA's columns are near identity, [1]: cluster decision
  __shared__ double s_piv[2];  // broadcast pivot: l_jj and 1 / l_jj
  __shared__ int s_keep;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  (void)lane;
  const double thr = thr_rel * (scale ? *scale : 1.0);

  // near-identity test on the CTA's own columns with integer compares of the IEEE bit
  // patterns (|g| <= tol off the diagonal, 1 - tol <= g <= 1 + tol on it; NaN fails):
  // no FP64 arithmetic, which is slow on this GPU
  if (tid == 0) s_flag[0] = 1;
  __syncthreads();
  if (near_tol > 0.0) {
    const long long tolb = __double_as_longlong(near_tol);
    const long long lob = __double_as_longlong(1.0 - near_tol), hib = __double_as_longlong(1.0 + near_tol);
    bool ok = true;
    for (int jl = 0; jl < wq; ++jl) {
      const int c = c0 + jl;
      for (int i = tid; i < n; i += CT) {
        const long long bits = __double_as_longlong(Gm[i + c * n]);
        if (i == c) {
          ok = ok && bits >= lob && bits <= hib;  // positive range: signed compare is monotone
        } else {
          ok = ok && (bits & 0x7fffffffffffffffLL) <= tolb;
        }
      }
    }
    if (!ok) s_flag[0] = 0;  // benign race: every writer stores 0
  } else if (tid == 0) {
    s_flag[0] = 0;
  }
  cluster.sync();
  if (tid == 0) {
    int all = 1;
    for (int qq = 0; qq < C; ++qq) all &= *cluster.map_shared_rank(&s_flag[0], qq);
    s_flag[1] = all;
  }
  __syncthreads();
  const int s_near = s_flag[1];
  if (near_out != nullptr && q == 0 && tid == 0) *near_out = s_near;
  if (s_near) {
    // R = I + Phi(E): row c of R holds E[c, i] for i > c and 1 + E[c, c] / 2 on the diagonal
    for (int jl = 0; jl < wq; ++jl) {
      const int c = c0 + jl;
      for (int i = tid; i < n; i += CT) {
        const double g = Gm[c + (int64_t)i * n];
        R[c + (int64_t)i * n] = i < c ? 0.0 : (i == c ? 1.0 + 0.5 * (g - 1.0) : g);
      }
    }
    cluster.sync();
    return;
  }

  // load the lower part of the own columns
  for (int jl = 0; jl < wq; ++jl) {
    const int c = c0 + jl;
    for (int i = tid; i < n; i += CT) A[i + jl * n] = i >= c ? Gm[i + c * n] : 0.0;
  }
  __syncthreads();

  for (int p = 0; p < C; ++p) {
    const int pc0 = p * w;
    const int wp = max(0, min(w, n - pc0));
    if (q == p) {
      for (int jl = 0; jl < wq; ++jl) {
        const int c = c0 + jl;
        if (tid == 0) {
          // one thread takes the pivot's square root and reciprocal (long FP64 sequences)
          const double s = A[c + jl * n];
          const int keep = s > thr;  // false for NaN as well
          if (!isfinite(s)) report(BKFAC_ENONFINITE);
          s_keep = keep;
          if (keep) {
            const double l = sqrt(s);
            s_piv[0] = l;
            s_piv[1] = 1.0 / l;
          }
        }
        __syncthreads();
        const bool keep = s_keep;
        if (keep) {
          const double ljj = s_piv[0], inv = s_piv[1];
          for (int i = c + tid; i < n; i += CT) A[i + jl * n] = (i == c) ? ljj : A[i + jl * n] * inv;
        } else {
          for (int i = c + tid; i < n; i += CT) A[i + jl * n] = 0.0;
        }
        __syncthreads();
        if (keep) {
          // rank-1 update of the remaining columns of the block: a warp per column,
          // lanes over rows (no integer division)
          for (int j2 = jl + 1 + wid; j2 < wq; j2 += CT / 32) {
            const int c2 = c0 + j2;
            const double l2 = A[c2 + jl * n];
            for (int i = c2 + lane; i < n; i += 32) A[i + j2 * n] -= A[i + jl * n] * l2;
          }
        }
        __syncthreads();
      }
    }
    cluster.sync();  // panel p is final in its owner's shared memory
    if (q > p && wq > 0 && wp > 0) {
      const double* remote = cluster.map_shared_rank(A, p);
      for (int k = 0; k < wp; ++k)
        for (int i = c0 + tid; i < n; i += CT) Pb[i + k * n] = remote[i + k * n];
      __syncthreads();
      // A[i, jl] -= sum_k L[i, k] L[c, k] over the panel's columns, i >= c = c0 + jl;
      // a warp per column, lanes over rows
      for (int jl = wid; jl < wq; jl += CT / 32) {
        const int c = c0 + jl;
        for (int i = c + lane; i < n; i += 32) {
          double acc = 0.0;
          for (int k = 0; k < wp; ++k) acc += Pb[i + k * n] * Pb[c + k * n];
          A[i + jl * n] -= acc;
        }
      }
      __syncthreads();
    }
  }
  // R = L^T: row c of R is column c of L
  for (int jl = 0; jl < wq; ++jl) {
    const int c = c0 + jl;
    for (int i = tid; i < n; i += CT) R[c + (int64_t)i * n] = i >= c ? A[i + (int64_t)jl * n] : 0.0;
  }
  cluster.sync();  // keep shared memory alive until every remote read is done
}

}  // namespace

// cluster size for an n x n factorisation (two n x w FP64 buffers per CTA)
int chol_cluster_size(int n) {
  for (int c : {1, 2, 4, 8, 16}) {
    const int w = (n + c - 1) / c;
    if (w <= 16 && (size_t)2 * n * w * 8 <= 200 * 1024) return c;
  }
  const int w = (n + 15) / 16;
  return (size_t)2 * n * w * 8 <= 200 * 1024 ? 16 : 0;
}

int launch_chol_cluster(const double* Gm, int n, double* R, double thr_rel, const double* scale, double near_tol,
                        int* near_out, cudaStream_t s) {
  if (n <= 0) return 0;
  const int C = chol_cluster_size(n);
  if (C == 0) return (int)cudaErrorInvalidValue;
  const int w = (n + C - 1) / C;
  const size_t smem = (size_t)2 * n * w * sizeof(double);
  static std::atomic<int> configured{0};  // attributes set once (the call can stall the host)
  if (!configured.load()) {
    cudaError_t e = cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    configured.store(1);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C, 1, 1);
  cfg.blockDim = dim3(CT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, chol_cluster_kernel, Gm, n, R, thr_rel, scale, near_tol, near_out);
  note_launches(1);
  return (int)e;
}

}  // namespace bkfac

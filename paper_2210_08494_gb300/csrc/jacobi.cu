// jacobi.cu -- eigendecomposition of the Brand core (Algorithm 3, EVD(M_S)).
//
// M_S = L L^T is symmetric p.s.d., so its eigenpairs are the left singular
// pairs of the factor L.  One-sided (Hestenes) Jacobi rotates pairs of columns
// of W (initially L) until all columns are mutually orthogonal; then
//   W = L V (V orthogonal),  W W^T = L L^T = M_S,
// so the eigenvalues are ||w_i||^2 and the eigenvectors w_i / ||w_i|| -- no
// accumulation of V is needed and no product L L^T is ever formed (which
// would square the condition number).  The same kernel serves the dense path
// (W = [U sqrt(rho sigma), sqrt(c) X], d rows) and re-orthonormalisation.
//
// Parallel layout: one thread-block cluster of C CTAs per problem.  The
// columns are split into 2C blocks of b columns; a round-robin tournament
// over the blocks (circle method) meets every block pair once per sweep in
// 2C - 1 rounds, CTA c working on one block pair per round in shared memory.
// Between rounds the blocks go back to global memory (L2-resident) and the
// cluster synchronises with the hardware cluster barrier; no CTA spins on a
// flag.  Inside a CTA, b disjoint column pairs per sub-round run on the warps
// (one warp per pair: the three dot products by a warp reduction, then the
// rotation).  The sweep count is capped; a problem that reaches the cap
// reports BKFAC_ENOCONV and still returns its current columns.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bkfac {

namespace {

constexpr int JT = 256;  // threads per CTA

__device__ __forceinline__ int circle_pos(int pos, int t, int m) {
  // circle method over m slots: slot 0 fixed, the others rotate with t
  return pos == 0 ? 0 : 1 + (pos - 1 + t) % (m - 1);
}

template <typename J>
__device__ __forceinline__ J warp_sum_j(J v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename J>
struct BigZeta;
template <>
struct BigZeta<float> {
  static constexpr float v = 1e18f;
};
template <>
struct BigZeta<double> {
  static constexpr double v = 1e150;
};

// Orthogonalise the column pair (x, y) (length `rows`, in shared memory).
// Returns 1 if a rotation was applied.
template <typename J>
__device__ __forceinline__ int rotate_pair(J* x, J* y, int rows, J tol2, J tiny, int lane) {
  J a = J(0), b = J(0), g = J(0);
  for (int r = lane; r < rows; r += 32) {
    const J xv = x[r], yv = y[r];
    a += xv * xv;
    b += yv * yv;
    g += xv * yv;
  }
  a = warp_sum_j(a);
  b = warp_sum_j(b);
  g = warp_sum_j(g);
  if (!(a > tiny && b > tiny && g * g > tol2 * a * b)) return 0;
  // Rutishauser: zeta = (b - a) / (2 g), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))
  const J zeta = (b - a) / (J(2) * g);
  const J az = fabs(zeta);
  J t;
  if (az > BigZeta<J>::v)
    t = J(0.5) / zeta;
  else
    t = copysign(J(1) / (az + sqrt(J(1) + az * az)), zeta);
  const J c = J(1) / sqrt(J(1) + t * t);
  const J s = c * t;
  for (int r = lane; r < rows; r += 32) {
    const J xv = x[r], yv = y[r];
    x[r] = c * xv - s * yv;
    y[r] = s * xv + c * yv;
  }
  return 1;
}

template <typename J>
__global__ void __launch_bounds__(JT) jacobi_kernel(const __grid_constant__ JacobiBatch batch, double tol,
                                                    int max_sweeps) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int pid = blockIdx.x / C;
  const JacobiProblem& P = batch.p[pid];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  J* sm = (J*)smem_raw;
  __shared__ int s_rot;
  __shared__ int s_cnt[2];
  __shared__ int s_total;
  __shared__ double s_tiny;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = JT / 32;
  const int b = P.b, rp = P.rows_pad, rows = P.rows, nblk = 2 * C;
  J* W = (J*)P.W;
  if (tid == 0) {
    double f = 0.0;
    for (int j = 0; j < P.cols_pad; ++j) f += P.colnorm2[j];
    s_tiny = Eps<J>::u * Eps<J>::u * f;
    s_cnt[0] = s_cnt[1] = 0;
  }
  __syncthreads();
  const J tiny = (J)s_tiny;
  const J tol2 = (J)(tol * tol);

  bool converged = false;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int t = 0; t < nblk - 1; ++t) {
      const int bI = circle_pos(crank, t, nblk);
      const int bJ = circle_pos(nblk - 1 - crank, t, nblk);
      // stage both blocks in shared memory: local columns [0, b) = block I, [b, 2b) = block J
      for (int e = tid; e < b * rp; e += JT) {
        const int c = e / rp, r = e % rp;
        sm[(int64_t)c * rp + r] = W[(int64_t)(bI * b + c) * rp + r];
        sm[(int64_t)(b + c) * rp + r] = W[(int64_t)(bJ * b + c) * rp + r];
      }
      __syncthreads();
      int rot = 0;
      if (t == 0) {
        // pairs inside each block, once per sweep (circle method over b slots, b even)
        const int hb = b / 2;
        for (int s = 0; s < b - 1; ++s) {
          for (int q = wid; q < b; q += nw) {
            const int blk = q / hb, i = q % hb;
            const int p0 = circle_pos(i, s, b), p1 = circle_pos(b - 1 - i, s, b);
            rot += rotate_pair<J>(sm + (int64_t)(blk * b + p0) * rp, sm + (int64_t)(blk * b + p1) * rp, rows,
                                  tol2, tiny, lane);
          }
          __syncthreads();
        }
      }
      // all b x b cross pairs between the two blocks: sub-round s pairs i with (i + s) mod b
      for (int s = 0; s < b; ++s) {
        for (int q = wid; q < b; q += nw)
          rot += rotate_pair<J>(sm + (int64_t)q * rp, sm + (int64_t)(b + (q + s) % b) * rp, rows, tol2, tiny, lane);
        __syncthreads();
      }
      for (int e = tid; e < b * rp; e += JT) {
        const int c = e / rp, r = e % rp;
        W[(int64_t)(bI * b + c) * rp + r] = sm[(int64_t)c * rp + r];
        W[(int64_t)(bJ * b + c) * rp + r] = sm[(int64_t)(b + c) * rp + r];
      }
      if (lane == 0 && rot) atomicAdd(&s_rot, rot);
      __threadfence();
      cluster.sync();  // blocks written back before any CTA loads them in the next round
    }
    if (tid == 0) s_cnt[sweep & 1] = s_rot;
    cluster.sync();
    if (tid == 0) {
      int total = 0;
      for (int q = 0; q < C; ++q) total += *cluster.map_shared_rank(&s_cnt[sweep & 1], q);
      s_total = total;
    }
    __syncthreads();
    if (s_total == 0) {  // identical in every CTA of the cluster
      converged = true;
      break;
    }
  }
  if (crank == 0 && tid == 0) {
    if (P.sweeps_out) *P.sweeps_out = converged ? sweep + 1 : sweep;
    if (!converged) report(BKFAC_ENOCONV);
  }
  cluster.sync();  // keep every CTA's shared memory alive until all remote reads are done
}

template <typename J>
int launch_typed(const JacobiProblem* probs, int nprob, int C, double tol, int max_sweeps, cudaStream_t s) {
  size_t smem = 0;
  JacobiBatch batch;
  for (int i = 0; i < nprob; ++i) {
    batch.p[i] = probs[i];
    smem = std::max(smem, (size_t)2 * probs[i].b * probs[i].rows_pad * sizeof(J));
  }
  if (smem > 227 * 1024) return (int)cudaErrorInvalidValue;
  auto kfn = jacobi_kernel<J>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nprob * C), 1, 1);
  cfg.blockDim = dim3(JT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kfn, batch, tol, max_sweeps);
  return (int)e;
}

}  // namespace

void jacobi_plan(int rows, int cols, DType j_t, int* C_out, int* b_out, int* rows_pad, int* cols_pad) {
  const int rp = (int)round_up(std::max(rows, 1), 32);
  const size_t es = j_t == DT_F64 ? 8 : 4;
  const size_t smem_cap = 200 * 1024;
  int C = 16, b = 2;
  // smallest cluster whose blocks are at most 16 columns wide and fit in shared memory;
  // fall back to wider blocks when even 16 CTAs are not enough
  for (int c : {1, 2, 4, 8, 16}) {
    const int bb = (int)round_up(ceil_div(std::max(cols, 2), 2 * c), 2);
    if (bb <= 16 && (size_t)2 * bb * rp * es <= smem_cap) {
      C = c;
      b = bb;
      break;
    }
    if (c == 16) {
      C = 16;
      b = bb;
    }
  }
  *C_out = C;
  *b_out = b;
  *rows_pad = rp;
  *cols_pad = 2 * C * b;
}

int launch_jacobi(const JacobiProblem* probs, int nprob, int C, DType j_t, double tol, int max_sweeps,
                  cudaStream_t s) {
  if (nprob <= 0) return 0;
  if (nprob > kMaxJacobiProblems) return (int)cudaErrorInvalidValue;
  if (j_t == DT_F64) return launch_typed<double>(probs, nprob, C, tol, max_sweeps, s);
  return launch_typed<float>(probs, nprob, C, tol, max_sweeps, s);
}

size_t jacobi_smem_bytes(int b, int rows_pad, DType j_t) {
  return (size_t)2 * b * rows_pad * (j_t == DT_F64 ? 8 : 4);
}

}  // namespace bkfac

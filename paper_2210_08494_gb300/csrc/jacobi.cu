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
// flag.  Inside a CTA there is one warp per column of the first block
// (blockDim = 32 b, b <= 16): in sub-round s warp q rotates its column against column
// (q + s) mod b of the second block, so all b pairs of a sub-round are in
// flight at once.  A lane holds rows {lane, lane + 32, ...} of its pair in
// registers (16-byte vector loads); the warp's own column stays in registers
// for the whole round.  The sweep count is capped; a problem that reaches the
// cap reports BKFAC_ENOCONV and still returns its current columns.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bkfac {

namespace {

template <typename J>
struct Vec;
template <>
struct Vec<float> {
  using T = float4;
  static constexpr int W = 4;
};
template <>
struct Vec<double> {
  using T = double2;
  static constexpr int W = 2;
};

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

// column <-> registers: lane owns the 16-byte vectors lane + 32 k, k < NV
template <typename J, int NV>
__device__ __forceinline__ void load_col(const J* col, J (&x)[NV * Vec<J>::W], int lane) {
  using V = typename Vec<J>::T;
  const V* c = reinterpret_cast<const V*>(col);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const V v = c[lane + 32 * k];
    const J* pv = reinterpret_cast<const J*>(&v);
#pragma unroll
    for (int w = 0; w < Vec<J>::W; ++w) x[k * Vec<J>::W + w] = pv[w];
  }
}

template <typename J, int NV>
__device__ __forceinline__ void store_col(J* col, const J (&x)[NV * Vec<J>::W], int lane) {
  using V = typename Vec<J>::T;
  V* c = reinterpret_cast<V*>(col);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    V v;
    J* pv = reinterpret_cast<J*>(&v);
#pragma unroll
    for (int w = 0; w < Vec<J>::W; ++w) pv[w] = x[k * Vec<J>::W + w];
    c[lane + 32 * k] = v;
  }
}

// Orthogonalise the column pair (x, y) held in registers by the warp.
// Returns 1 if a rotation was applied.
template <typename J, int E>
__device__ __forceinline__ int rotate_regs(J (&x)[E], J (&y)[E], J tol2, J tiny) {
  J a0 = J(0), a1 = J(0), b0 = J(0), b1 = J(0), g0 = J(0), g1 = J(0);
#pragma unroll
  for (int e = 0; e < E; e += 2) {
    a0 += x[e] * x[e];
    b0 += y[e] * y[e];
    g0 += x[e] * y[e];
    if (e + 1 < E) {
      a1 += x[e + 1] * x[e + 1];
      b1 += y[e + 1] * y[e + 1];
      g1 += x[e + 1] * y[e + 1];
    }
  }
  const J a = warp_sum_j(a0 + a1);
  const J b = warp_sum_j(b0 + b1);
  const J g = warp_sum_j(g0 + g1);
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
  // Rutishauser's form with tau = tan(theta/2) = s / (1 + c): x' = x - s (y + tau x),
  // y' = y + s (x - tau y).  It equals (c x - s y, s x + c y) but applies the O(t^2)
  // shrink of x and y as an explicit correction, so for small angles (where 1 + t^2
  // rounds to 1 and c = 1 exactly) the rotation stays orthogonal to working precision
  // instead of growing both columns by (1 + t^2) -- a bias that otherwise
  // accumulates over the thousands of rotations a column takes part in.
  const J tau = s / (J(1) + c);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const J xv = x[e], yv = y[e];
    x[e] = xv - s * (yv + tau * xv);
    y[e] = yv + s * (xv - tau * yv);
  }
  return 1;
}

template <typename J, int NV>
__global__ void __launch_bounds__(512) jacobi_kernel(const __grid_constant__ JacobiBatch batch, double tol,
                                                      int max_sweeps) {
  constexpr int E = NV * Vec<J>::W;  // rows per lane
  using V = typename Vec<J>::T;
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

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nthr = blockDim.x, nw = nthr >> 5;
  const int b = P.b, rp = P.rows_pad, nblk = 2 * C;  // rp == 32 * E
  J* W = (J*)P.W;
  if (wid == 0) {
    // deterministic: fixed lane assignment, fixed shuffle tree
    double f = 0.0;
    for (int j = lane; j < P.cols_pad; j += 32) f += P.colnorm2[j];
    f = warp_sum_j(f);
    if (lane == 0) {
      s_tiny = Eps<J>::u * Eps<J>::u * f;
      s_cnt[0] = s_cnt[1] = 0;
    }
  }
  __syncthreads();
  const J tiny = (J)s_tiny;
  const J tol2 = (J)(tol * tol);
  const int nvec = b * rp / Vec<J>::W;  // vectors per block

  bool converged = false;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int t = 0; t < nblk - 1; ++t) {
      const int bI = circle_pos(crank, t, nblk);
      const int bJ = circle_pos(nblk - 1 - crank, t, nblk);
      {
        const V* gI = reinterpret_cast<const V*>(W + (int64_t)bI * b * rp);
        const V* gJ = reinterpret_cast<const V*>(W + (int64_t)bJ * b * rp);
        V* s0 = reinterpret_cast<V*>(sm);
        V* s1 = reinterpret_cast<V*>(sm + (int64_t)b * rp);
        for (int e = tid; e < nvec; e += nthr) {
          s0[e] = gI[e];
          s1[e] = gJ[e];
        }
      }
      __syncthreads();
      int rot = 0;
      if (t == 0) {
        // pairs inside each block, once per sweep (circle method over b slots, b even)
        const int hb = b / 2;
        for (int s = 0; s < b - 1; ++s) {
          for (int q = wid; q < b; q += nw) {
            const int blk = q / hb, i = q % hb;
            J* cp = sm + (int64_t)(blk * b + circle_pos(i, s, b)) * rp;
            J* cq = sm + (int64_t)(blk * b + circle_pos(b - 1 - i, s, b)) * rp;
            J x[E], y[E];
            load_col<J, NV>(cp, x, lane);
            load_col<J, NV>(cq, y, lane);
            if (rotate_regs<J, E>(x, y, tol2, tiny)) {
              store_col<J, NV>(cp, x, lane);
              store_col<J, NV>(cq, y, lane);
              ++rot;
            }
          }
          __syncthreads();
        }
      }
      // all b x b cross pairs: in sub-round s warp q pairs column q of block I with
      // column (q + s) mod b of block J; warp q keeps its block-I column in registers
      if (b <= nw) {
        J x[E];
        J* cx = sm + (int64_t)wid * rp;
        if (wid < b) load_col<J, NV>(cx, x, lane);
        bool xdirty = false;
        for (int s = 0; s < b; ++s) {
          if (wid < b) {
            J* cy = sm + (int64_t)(b + (wid + s) % b) * rp;
            J y[E];
            load_col<J, NV>(cy, y, lane);
            if (rotate_regs<J, E>(x, y, tol2, tiny)) {
              store_col<J, NV>(cy, y, lane);
              xdirty = true;
              ++rot;
            }
          }
          __syncthreads();
        }
        if (wid < b && xdirty) store_col<J, NV>(cx, x, lane);
      } else {
        // more pairs than warps: each warp takes several pairs per sub-round
        for (int s = 0; s < b; ++s) {
          for (int q = wid; q < b; q += nw) {
            J* cx = sm + (int64_t)q * rp;
            J* cy = sm + (int64_t)(b + (q + s) % b) * rp;
            J x[E], y[E];
            load_col<J, NV>(cx, x, lane);
            load_col<J, NV>(cy, y, lane);
            if (rotate_regs<J, E>(x, y, tol2, tiny)) {
              store_col<J, NV>(cx, x, lane);
              store_col<J, NV>(cy, y, lane);
              ++rot;
            }
          }
          __syncthreads();
        }
      }
      __syncthreads();
      {
        V* gI = reinterpret_cast<V*>(W + (int64_t)bI * b * rp);
        V* gJ = reinterpret_cast<V*>(W + (int64_t)bJ * b * rp);
        const V* s0 = reinterpret_cast<const V*>(sm);
        const V* s1 = reinterpret_cast<const V*>(sm + (int64_t)b * rp);
        for (int e = tid; e < nvec; e += nthr) {
          gI[e] = s0[e];
          gJ[e] = s1[e];
        }
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

template <typename J, int NV>
int launch_typed(const JacobiBatch& batch, int nprob, int C, int b, size_t smem, double tol, int max_sweeps,
                 cudaStream_t s) {
  auto kfn = jacobi_kernel<J, NV>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nprob * C), 1, 1);
  cfg.blockDim = dim3((unsigned)(32 * std::min(b, 16)), 1, 1);
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
  note_launches(1);
  return (int)e;
}

template <typename J>
int launch_nv(const JacobiBatch& batch, int nprob, int C, int b, int rows_pad, size_t smem, double tol,
              int max_sweeps, cudaStream_t s) {
  const int nv = rows_pad / (32 * Vec<J>::W);
  switch (nv) {
    case 1: return launch_typed<J, 1>(batch, nprob, C, b, smem, tol, max_sweeps, s);
    case 2: return launch_typed<J, 2>(batch, nprob, C, b, smem, tol, max_sweeps, s);
    case 4: return launch_typed<J, 4>(batch, nprob, C, b, smem, tol, max_sweeps, s);
    case 8: return launch_typed<J, 8>(batch, nprob, C, b, smem, tol, max_sweeps, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

// rows padded to 32 lanes x (1, 2, 4 or 8) vectors of 16 bytes
int rows_pad_for(int rows, DType j_t) {
  const int unit = 32 * (j_t == DT_F64 ? 2 : 4);
  int nv = 1;
  while (nv < 8 && unit * nv < rows) nv *= 2;
  return unit * nv;
}

}  // namespace

void jacobi_plan(int rows, int cols, DType j_t, int* C_out, int* b_out, int* rows_pad, int* cols_pad) {
  const int rp = rows_pad_for(std::max(rows, 1), j_t);
  const size_t es = j_t == DT_F64 ? 8 : 4;
  const size_t smem_cap = 200 * 1024;
  int C = 16, b = 32;
  // smallest cluster whose blocks are at most 16 columns wide and fit in shared memory;
  // fall back to wider blocks (at most 32 = 1024 threads) when 16 CTAs are not enough
  bool found = false;
  for (int c : {1, 2, 4, 8, 16}) {
    const int bb = (int)round_up(ceil_div(std::max(cols, 2), 2 * c), 2);
    if (bb <= 16 && (size_t)2 * bb * rp * es <= smem_cap) {
      C = c;
      b = bb;
      found = true;
      break;
    }
  }
  if (!found) {
    C = 16;
    b = (int)round_up(ceil_div(std::max(cols, 2), 32), 2);
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
  JacobiBatch batch;
  int b = 0, rp = 0;
  size_t smem = 0;
  for (int i = 0; i < nprob; ++i) {
    batch.p[i] = probs[i];
    // one launch: every problem shares the block width (threads) and padded row count
    if (i == 0) {
      b = probs[i].b;
      rp = probs[i].rows_pad;
    } else if (probs[i].b != b || probs[i].rows_pad != rp) {
      return (int)cudaErrorInvalidValue;
    }
    smem = std::max(smem, jacobi_smem_bytes(probs[i].b, probs[i].rows_pad, j_t));
  }
  if (b < 2 || b > 32 || (b & 1) || smem > 227 * 1024) return (int)cudaErrorInvalidValue;
  if (j_t == DT_F64) return launch_nv<double>(batch, nprob, C, b, rp, smem, tol, max_sweeps, s);
  return launch_nv<float>(batch, nprob, C, b, rp, smem, tol, max_sweeps, s);
}

size_t jacobi_smem_bytes(int b, int rows_pad, DType j_t) {
  return (size_t)2 * b * rows_pad * (j_t == DT_F64 ? 8 : 4);
}

}  // namespace bkfac

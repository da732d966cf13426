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
#include <atomic>
#include <cstdint>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bkfac {

namespace {

constexpr int kSweepLog = 48;  // per-sweep rotation counts kept in sweeps_out[1..]

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

// Rotation parameters.  FP32 uses the hardware reciprocal / square-root
// approximations: the angle need not be exact, and the update below applies
// c and s in a form that stays orthogonal when c^2 + s^2 differs from 1 in the
// last bits (the energy error is second order in s).  FP64 keeps IEEE division.
__device__ __forceinline__ void rotation_params(float a, float b, float g, float& t, float& c, float& s) {
  // hardware approximations only (reciprocal square root, fast division): the
  // rotation need not be exact, only applied consistently (see rotate_regs_f2)
  const float zeta = __fdividef(b - a, 2.0f * g);
  const float az = fabsf(zeta);
  if (az > BigZeta<float>::v) {
    t = __fdividef(0.5f, zeta);
  } else {
    const float h = fmaf(az, az, 1.0f);
    t = copysignf(__fdividef(1.0f, az + h * rsqrtf(h)), zeta);
  }
  c = rsqrtf(fmaf(t, t, 1.0f));
  s = c * t;
}
__device__ __forceinline__ void rotation_params(double a, double b, double g, double& t, double& c, double& s) {
  const double zeta = (b - a) / (2.0 * g);
  const double az = fabs(zeta);
  if (az > BigZeta<double>::v)
    t = 0.5 / zeta;
  else
    t = copysign(1.0 / (az + sqrt(1.0 + az * az)), zeta);
  c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
}

// Orthogonalise the column pair (x, y) held in registers by the warp, given
// their squared norms a = ||x||^2, b = ||y||^2 (tracked by the caller).  Only
// the cross product g = x.y is reduced over the warp.  On a rotation the norms
// are updated exactly as a' = a - t g, b' = b + t g.  Returns 1 if rotated.
template <typename J, int E>
__device__ __forceinline__ int rotate_regs_generic(J (&x)[E], J (&y)[E], J& a, J& b, J tol2, J tiny) {
  J g0 = J(0), g1 = J(0);
#pragma unroll
  for (int e = 0; e < E; e += 2) {
    g0 += x[e] * y[e];
    if (e + 1 < E) g1 += x[e + 1] * y[e + 1];
  }
  const J g = warp_sum_j(g0 + g1);
  if (!(a > tiny && b > tiny && g * g > tol2 * a * b)) return 0;
  // Rutishauser: zeta = (b - a) / (2 g), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))
  J t, c, s;
  rotation_params(a, b, g, t, c, s);
  // Rutishauser's form with tau = tan(theta/2) = s / (1 + c): x' = x - s (y + tau x),
  // y' = y + s (x - tau y).  It equals (c x - s y, s x + c y) but applies the O(t^2)
  // shrink of x and y as an explicit correction, so for small angles (where 1 + t^2
  // rounds to 1 and c = 1 exactly) the rotation stays orthogonal to working precision
  // instead of growing both columns by (1 + t^2) -- a bias that otherwise
  // accumulates over the thousands of rotations a column takes part in.
  const J tau = s / (J(1) + c);  // c >= 1/sqrt(2): well conditioned
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const J xv = x[e], yv = y[e];
    x[e] = xv - s * (yv + tau * xv);
    y[e] = yv + s * (xv - tau * yv);
  }
  a -= t * g;
  b += t * g;
  return 1;
}

// FP32 specialisation with Blackwell's packed two-wide FP32 FMA (fma.rn.f32x2):
// the dot product and the rotation process two rows per instruction.
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void unpack2(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <int E>
__device__ __forceinline__ int rotate_regs_f2(float (&x)[E], float (&y)[E], float& a, float& b, float tol2,
                                              float tiny) {
  static_assert(E % 4 == 0, "two packed chains of two rows");
  uint64_t g0 = 0, g1 = 0;  // bit pattern of (0.f, 0.f)
#pragma unroll
  for (int e = 0; e < E; e += 4) {
    g0 = ffma2(pack2(x[e], x[e + 1]), pack2(y[e], y[e + 1]), g0);
    g1 = ffma2(pack2(x[e + 2], x[e + 3]), pack2(y[e + 2], y[e + 3]), g1);
  }
  float p0, p1, p2, p3;
  unpack2(g0, p0, p1);
  unpack2(g1, p2, p3);
  const float g = warp_sum_j((p0 + p1) + (p2 + p3));
  if (!(a > tiny && b > tiny && g * g > tol2 * a * b)) return 0;
  float t, c, s;
  rotation_params(a, b, g, t, c, s);
  const float tau = __fdividef(s, 1.0f + c);
  // tau form (see the generic version): x' = x - s (y + tau x), y' = y + s (x - tau y)
  const uint64_t tau2 = pack2(tau, tau), ntau2 = pack2(-tau, -tau);
  const uint64_t s2 = pack2(s, s), ns2 = pack2(-s, -s);
#pragma unroll
  for (int e = 0; e < E; e += 2) {
    const uint64_t xv = pack2(x[e], x[e + 1]), yv = pack2(y[e], y[e + 1]);
    const uint64_t u = ffma2(tau2, xv, yv);   // y + tau x
    const uint64_t v = ffma2(ntau2, yv, xv);  // x - tau y
    const uint64_t xn = ffma2(ns2, u, xv);
    const uint64_t yn = ffma2(s2, v, yv);
    unpack2(xn, x[e], x[e + 1]);
    unpack2(yn, y[e], y[e + 1]);
  }
  a -= t * g;
  b += t * g;
  return 1;
}

// FP32 takes the packed path, FP64 the generic one
template <typename J, int E>
struct RotSel {
  static __device__ __forceinline__ int run(J (&x)[E], J (&y)[E], J& a, J& b, J tol2, J tiny) {
    return rotate_regs_generic<J, E>(x, y, a, b, tol2, tiny);
  }
};
template <int E>
struct RotSel<float, E> {
  static __device__ __forceinline__ int run(float (&x)[E], float (&y)[E], float& a, float& b, float tol2,
                                            float tiny) {
    return rotate_regs_f2<E>(x, y, a, b, tol2, tiny);
  }
};
template <typename J, int E>
__device__ __forceinline__ int rotate_regs(J (&x)[E], J (&y)[E], J& a, J& b, J tol2, J tiny) {
  return RotSel<J, E>::run(x, y, a, b, tol2, tiny);
}

template <typename J, int E>
__device__ __forceinline__ J col_norm2(const J (&x)[E]) {
  J a0 = J(0), a1 = J(0);
#pragma unroll
  for (int e = 0; e < E; e += 2) {
    a0 += x[e] * x[e];
    if (e + 1 < E) a1 += x[e + 1] * x[e + 1];
  }
  return warp_sum_j(a0 + a1);
}

// One round on the 2b staged columns (local columns [0, b) = block I, [b, 2b) =
// block J): norms refreshed, then the pairs inside each block (first round of a
// sweep only) and all b x b cross pairs.  s_nrm / s_stamp hold the squared
// norms and the sweep of each column's last rotation.  Returns the number of
// rotations this warp applied (identical in every lane).
template <typename J, int NV>
__device__ __forceinline__ int process_round(J* sm, J* s_nrm, int* s_stamp, int b, int rp, int t, int sweep,
                                             J tol2, J tiny, int lane, int wid, int nw) {
  constexpr int E = NV * Vec<J>::W;
  // a pair needs a check unless neither column has rotated since the previous sweep
  // (it was then verified orthogonal and has not changed since)
  auto needs = [&](int p, int q) { return sweep == 0 || s_stamp[p] >= sweep - 1 || s_stamp[q] >= sweep - 1; };
  // fresh squared norms of the staged columns (resets the drift of the tracked values)
  for (int c = wid; c < 2 * b; c += nw) {
    J x[E];
    load_col<J, NV>(sm + (int64_t)c * rp, x, lane);
    const J a = col_norm2<J, E>(x);
    if (lane == 0) s_nrm[c] = a;
  }
  __syncthreads();
  int rot = 0;
  if (t == 0) {
    // pairs inside each block, once per sweep (circle method over b slots, b even)
    const int hb = b / 2;
    for (int s = 0; s < b - 1; ++s) {
      for (int q = wid; q < b; q += nw) {
        const int blk = q / hb, i = q % hb;
        const int p0 = blk * b + circle_pos(i, s, b), p1 = blk * b + circle_pos(b - 1 - i, s, b);
        if (!needs(p0, p1)) continue;
        J* cp = sm + (int64_t)p0 * rp;
        J* cq = sm + (int64_t)p1 * rp;
        J x[E], y[E];
        load_col<J, NV>(cp, x, lane);
        load_col<J, NV>(cq, y, lane);
        J a = s_nrm[p0], bb = s_nrm[p1];
        if (rotate_regs<J, E>(x, y, a, bb, tol2, tiny)) {
          store_col<J, NV>(cp, x, lane);
          store_col<J, NV>(cq, y, lane);
          if (lane == 0) {
            s_nrm[p0] = a;
            s_nrm[p1] = bb;
            s_stamp[p0] = sweep;
            s_stamp[p1] = sweep;
          }
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
    J a = J(0);
    if (wid < b) {
      load_col<J, NV>(cx, x, lane);
      a = s_nrm[wid];
    }
    bool xdirty = false;
    for (int s = 0; s < b; ++s) {
      if (wid < b) {
        const int qy = b + (wid + s) % b;
        if (needs(wid, qy)) {
          J* cy = sm + (int64_t)qy * rp;
          J y[E];
          load_col<J, NV>(cy, y, lane);
          J bb = s_nrm[qy];
          if (rotate_regs<J, E>(x, y, a, bb, tol2, tiny)) {
            store_col<J, NV>(cy, y, lane);
            if (lane == 0) {
              s_nrm[qy] = bb;
              s_stamp[qy] = sweep;
              s_stamp[wid] = sweep;
            }
            xdirty = true;
            ++rot;
          }
        }
      }
      __syncthreads();
    }
    if (wid < b && xdirty) {
      store_col<J, NV>(cx, x, lane);
      if (lane == 0) s_nrm[wid] = a;
    }
  } else {
    // more pairs than warps: each warp takes several pairs per sub-round
    for (int s = 0; s < b; ++s) {
      for (int q = wid; q < b; q += nw) {
        const int qy = b + (q + s) % b;
        if (!needs(q, qy)) continue;
        J* cx = sm + (int64_t)q * rp;
        J* cy = sm + (int64_t)qy * rp;
        J x[E], y[E];
        load_col<J, NV>(cx, x, lane);
        load_col<J, NV>(cy, y, lane);
        J a = s_nrm[q], bb = s_nrm[qy];
        if (rotate_regs<J, E>(x, y, a, bb, tol2, tiny)) {
          store_col<J, NV>(cx, x, lane);
          store_col<J, NV>(cy, y, lane);
          if (lane == 0) {
            s_nrm[q] = a;
            s_nrm[qy] = bb;
            s_stamp[q] = sweep;
            s_stamp[qy] = sweep;
          }
          ++rot;
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
  return rot;
}

// copy nvec 16-byte vectors (cooperatively over the CTA)
template <typename V>
__device__ __forceinline__ void copy_vecs(V* dst, const V* src, int nvec, int tid, int nthr) {
  for (int e = tid; e < nvec; e += nthr) dst[e] = src[e];
}

// DSM = true: the blocks stay in shared memory (two buffers) and move between
// neighbouring CTAs of the cluster by remote shared-memory reads after each
// cluster barrier.  Under the circle method the block at slot p >= 1 in round
// t + 1 is the block at slot 1 + (p mod (2C - 1)) in round t (slot 0 is
// fixed); slot s < C belongs to CTA s as its first block, slot s >= C to CTA
// 2C - 1 - s as its second.  DSM = false: blocks go back to global memory
// (L2) between rounds (used when two buffers do not fit).
template <typename J, int NV, bool DSM>
__global__ void __launch_bounds__(512) jacobi_kernel(const __grid_constant__ JacobiBatch batch, double tol,
                                                      int max_sweeps) {
  using V = typename Vec<J>::T;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int pid = blockIdx.x / C;
  const JacobiProblem& P = batch.p[pid];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot;
  __shared__ int s_cnt[2];
  __shared__ int s_total;
  __shared__ double s_tiny;
  __shared__ J s_nrm[64];           // squared norms of the 2b staged columns
  __shared__ int s_stamp[2][64];    // sweep in which each staged column last rotated (per buffer)

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nthr = blockDim.x, nw = nthr >> 5;
  const int b = P.b, rp = P.rows_pad, nblk = 2 * C;  // rp == 32 * E
  J* W = (J*)P.W;
  int* stamp = P.stamp;
  J* buf0 = (J*)smem_raw;
  J* buf1 = buf0 + (DSM ? (int64_t)2 * b * rp : 0);
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
  const int nvec = b * rp / Vec<J>::W;  // vectors per block
  int cur = 0;
  if (DSM) {
    // initial blocks of round 0 from global memory
    const int bI = circle_pos(crank, 0, nblk), bJ = circle_pos(nblk - 1 - crank, 0, nblk);
    copy_vecs(reinterpret_cast<V*>(buf0), reinterpret_cast<const V*>(W + (int64_t)bI * b * rp), nvec, tid, nthr);
    copy_vecs(reinterpret_cast<V*>(buf0 + (int64_t)b * rp), reinterpret_cast<const V*>(W + (int64_t)bJ * b * rp),
              nvec, tid, nthr);
    for (int c = tid; c < 2 * b; c += nthr) s_stamp[0][c] = -10;
  }
  __syncthreads();
  const J tiny = (J)s_tiny;
  const J tol2 = (J)(tol * tol);

  bool converged = false;
  int sweep = 0, last_t = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int t = 0; t < nblk - 1; ++t) {
      const int bI = circle_pos(crank, t, nblk);
      const int bJ = circle_pos(nblk - 1 - crank, t, nblk);
      J* sm = (DSM && cur) ? buf1 : buf0;
      if (!DSM) {
        copy_vecs(reinterpret_cast<V*>(sm), reinterpret_cast<const V*>(W + (int64_t)bI * b * rp), nvec, tid, nthr);
        copy_vecs(reinterpret_cast<V*>(sm + (int64_t)b * rp), reinterpret_cast<const V*>(W + (int64_t)bJ * b * rp),
                  nvec, tid, nthr);
        for (int c = tid; c < 2 * b; c += nthr) {
          const int gc = (c < b ? bI * b + c : bJ * b + (c - b));
          s_stamp[0][c] = sweep == 0 ? -10 : stamp[gc];
        }
        __syncthreads();
      }
      const int rot = process_round<J, NV>(sm, s_nrm, s_stamp[DSM ? cur : 0], b, rp, t, sweep, tol2, tiny, lane,
                                           wid, nw);
      if (lane == 0 && rot) atomicAdd(&s_rot, rot);
      last_t = t;
      if (!DSM) {
        copy_vecs(reinterpret_cast<V*>(W + (int64_t)bI * b * rp), reinterpret_cast<const V*>(sm), nvec, tid, nthr);
        copy_vecs(reinterpret_cast<V*>(W + (int64_t)bJ * b * rp), reinterpret_cast<const V*>(sm + (int64_t)b * rp),
                  nvec, tid, nthr);
        for (int c = tid; c < 2 * b; c += nthr) {
          const int gc = (c < b ? bI * b + c : bJ * b + (c - b));
          stamp[gc] = s_stamp[0][c];
        }
        // the cluster barrier's arrive (release) / wait (acquire) order these global
        // write-backs before any CTA of the cluster loads the blocks in the next round
        cluster.sync();
      } else {
        cluster.sync();  // every CTA's blocks of this round are final
        // pull the next round's two blocks (and their stamps) from their current holders
        J* nxt = cur ? buf0 : buf1;
        int* nst = s_stamp[cur ^ 1];
        for (int half = 0; half < 2; ++half) {
          const int slot = half == 0 ? crank : nblk - 1 - crank;
          const int src_slot = slot == 0 ? 0 : 1 + (slot % (nblk - 1));
          const int src_cta = src_slot < C ? src_slot : nblk - 1 - src_slot;
          const int src_half = src_slot < C ? 0 : 1;
          const J* rbuf = cluster.map_shared_rank(sm, src_cta) + (int64_t)src_half * b * rp;
          const int* rst = cluster.map_shared_rank(s_stamp[cur], src_cta) + src_half * b;
          copy_vecs(reinterpret_cast<V*>(nxt + (int64_t)half * b * rp), reinterpret_cast<const V*>(rbuf), nvec, tid,
                    nthr);
          for (int c = tid; c < b; c += nthr) nst[half * b + c] = rst[c];
        }
        cur ^= 1;
        __syncthreads();
      }
    }
    if (tid == 0) s_cnt[sweep & 1] = s_rot;
    cluster.sync();
    if (tid == 0) {
      int total = 0;
      for (int q = 0; q < C; ++q) total += *cluster.map_shared_rank(&s_cnt[sweep & 1], q);
      s_total = total;
      // diagnostics: rotations applied in each sweep
      if (crank == 0 && P.sweeps_out && sweep < kSweepLog) P.sweeps_out[1 + sweep] = total;
    }
    __syncthreads();
    if (s_total == 0) {  // identical in every CTA of the cluster
      converged = true;
      break;
    }
  }
  if (DSM) {
    // write the final blocks back: after the last round's pull, buffer `cur` holds the
    // blocks of the round after last_t
    const int tn = last_t + 1;
    const int bI = circle_pos(crank, tn, nblk), bJ = circle_pos(nblk - 1 - crank, tn, nblk);
    const J* sm = cur ? buf1 : buf0;
    copy_vecs(reinterpret_cast<V*>(W + (int64_t)bI * b * rp), reinterpret_cast<const V*>(sm), nvec, tid, nthr);
    copy_vecs(reinterpret_cast<V*>(W + (int64_t)bJ * b * rp), reinterpret_cast<const V*>(sm + (int64_t)b * rp), nvec,
              tid, nthr);
  }
  if (crank == 0 && tid == 0) {
    if (P.sweeps_out) *P.sweeps_out = converged ? sweep + 1 : sweep;
    if (!converged) report(BKFAC_ENOCONV);
  }
  cluster.sync();  // keep every CTA's shared memory alive until all remote reads are done
}

template <typename J, int NV, bool DSM>
int launch_typed(const JacobiBatch& batch, int nprob, int C, int b, size_t smem, double tol, int max_sweeps,
                 cudaStream_t s) {
  auto kfn = jacobi_kernel<J, NV, DSM>;
  // function attributes are set once per instantiation (the call can stall the host)
  static std::atomic<int> configured{0};
  cudaError_t e = cudaSuccess;
  if (!configured.load()) {
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    configured.store(1);
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

template <typename J, bool DSM>
int launch_nv(const JacobiBatch& batch, int nprob, int C, int b, int rows_pad, size_t smem, double tol,
              int max_sweeps, cudaStream_t s) {
  const int nv = rows_pad / (32 * Vec<J>::W);
  switch (nv) {
    case 1: return launch_typed<J, 1, DSM>(batch, nprob, C, b, smem, tol, max_sweeps, s);
    case 2: return launch_typed<J, 2, DSM>(batch, nprob, C, b, smem, tol, max_sweeps, s);
    case 4: return launch_typed<J, 4, DSM>(batch, nprob, C, b, smem, tol, max_sweeps, s);
    case 8: return launch_typed<J, 8, DSM>(batch, nprob, C, b, smem, tol, max_sweeps, s);
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

void jacobi_plan_with(int rows, int cols, DType j_t, int b_max, int* C_out, int* b_out, int* rows_pad,
                      int* cols_pad) {
  const int rp = rows_pad_for(std::max(rows, 1), j_t);
  const size_t es = j_t == DT_F64 ? 8 : 4;
  const size_t smem_cap = 200 * 1024;
  int C = 16, b = 32;
  // smallest cluster whose blocks are at most b_max columns wide and fit in shared
  // memory; fall back to wider blocks when 16 CTAs are not enough
  bool found = false;
  for (int c : {1, 2, 4, 8, 16}) {
    const int bb = (int)round_up(ceil_div(std::max(cols, 2), 2 * c), 2);
    if (bb <= b_max && (size_t)2 * bb * rp * es <= smem_cap) {
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

void jacobi_plan(int rows, int cols, DType j_t, int* C_out, int* b_out, int* rows_pad, int* cols_pad) {
  int b_max = 16, dsm = 0;
  if (tune_lookup(rows, cols, j_t, &b_max, &dsm)) b_max = std::min(std::max(b_max, 2), 16);
  jacobi_plan_with(rows, cols, j_t, b_max, C_out, b_out, rows_pad, cols_pad);
}

int launch_jacobi(const JacobiProblem* probs, int nprob, int C, DType j_t, double tol, int max_sweeps,
                  cudaStream_t s) {
  int b = 0, dsm = 0;
  if (nprob > 0) tune_lookup(probs[0].rows, probs[0].cols, j_t, &b, &dsm);
  return launch_jacobi_mode(probs, nprob, C, j_t, tol, max_sweeps, dsm != 0, s);
}

int launch_jacobi_mode(const JacobiProblem* probs, int nprob, int C, DType j_t, double tol, int max_sweeps,
                       bool want_dsm, cudaStream_t s) {
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
  if (b < 2 || b > 32 || (b & 1) || smem > 200 * 1024) return (int)cudaErrorInvalidValue;
  // block exchange between rounds: through L2 by default; over distributed shared
  // memory (two buffers) when the tuning table asks for it and the buffers fit
  const bool dsm = want_dsm && 2 * smem <= 200 * 1024;
  if (j_t == DT_F64)
    return dsm ? launch_nv<double, true>(batch, nprob, C, b, rp, 2 * smem, tol, max_sweeps, s)
               : launch_nv<double, false>(batch, nprob, C, b, rp, smem, tol, max_sweeps, s);
  return dsm ? launch_nv<float, true>(batch, nprob, C, b, rp, 2 * smem, tol, max_sweeps, s)
             : launch_nv<float, false>(batch, nprob, C, b, rp, smem, tol, max_sweeps, s);
}

size_t jacobi_smem_bytes(int b, int rows_pad, DType j_t) {
  return (size_t)2 * b * rows_pad * (j_t == DT_F64 ? 8 : 4);
}

}  // namespace bkfac

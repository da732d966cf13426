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
// Parallel layout: one thread-block cluster of C CTAs per problem (a grouped
// launch runs one cluster per problem).  The columns are split into 2C blocks
// of b columns; a round-robin tournament over the blocks (circle method) meets
// every block pair once per sweep in 2C - 1 rounds, CTA c holding two blocks
// per round in shared memory.  Between rounds the blocks move to their next
// holders either by bulk copies over distributed shared memory (three buffers,
// completion on the receiver's mbarrier, a split cluster barrier) or, when
// three buffers do not fit or a group runs more clusters than the GPU holds,
// through global memory (L2) and the cluster barrier.  Inside a CTA each warp
// keeps K columns of the first block in registers for the whole round (K = 4
// for FP32 up to 512 rows, else 2) and meets the K-column groups of the second
// block in turn; a lane holds the 16-byte vectors lane, lane + 32, ... of each
// column (rows 4 lane .. 4 lane + 3, + 128, ... in FP32, kept as packed pairs
// for the two-wide FMA; two rows per vector in FP64).  The
// pairs of a meeting run as steps of K disjoint pairs with one spread warp
// reduction per step (FP32, K = 4: two interleaved chains of two pairs on the
// XOR schedule).  Late sweeps skip meetings that would rotate nothing, and a
// sweep that rotated few pairs is followed by a check of the pairs it left
// open instead of a full sweep.  The sweep count is capped; a problem that
// reaches the cap reports BKFAC_ENOCONV and still returns its current columns.
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
struct BigZeta<double> {
  static constexpr double v = 1e150;
};

// A lane's slice of one column: the 16-byte vectors lane + 32 k, k < NV.  FP32
// keeps the slice as packed pairs of rows in 64-bit registers, so that every
// product and rotation runs on Blackwell's two-wide FP32 FMA (fma.rn.f32x2)
// without repacking; FP64 keeps plain doubles.
template <typename J, int NV>
struct Col;

template <int NV>
struct Col<float, NV> {
  static constexpr int P = 2 * NV;  // packed row pairs per lane
  uint64_t v[P];
  __device__ __forceinline__ void load(const float* col, int lane) {
    const ulonglong2* c = reinterpret_cast<const ulonglong2*>(col);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const ulonglong2 q = c[lane + 32 * k];
      v[2 * k] = q.x;
      v[2 * k + 1] = q.y;
    }
  }
  __device__ __forceinline__ void store(float* col, int lane) const {
    ulonglong2* c = reinterpret_cast<ulonglong2*>(col);
#pragma unroll
    for (int k = 0; k < NV; ++k) c[lane + 32 * k] = make_ulonglong2(v[2 * k], v[2 * k + 1]);
  }
};

template <int NV>
struct Col<double, NV> {
  static constexpr int P = 2 * NV;  // doubles per lane
  double v[P];
  __device__ __forceinline__ void load(const double* col, int lane) {
    const double2* c = reinterpret_cast<const double2*>(col);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double2 q = c[lane + 32 * k];
      v[2 * k] = q.x;
      v[2 * k + 1] = q.y;
    }
  }
  __device__ __forceinline__ void store(double* col, int lane) const {
    double2* c = reinterpret_cast<double2*>(col);
#pragma unroll
    for (int k = 0; k < NV; ++k) c[lane + 32 * k] = make_double2(v[2 * k], v[2 * k + 1]);
  }
};

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

// this lane's part of x . y (two independent accumulation chains)
template <int NV>
__device__ __forceinline__ float dot_lane(const Col<float, NV>& x, const Col<float, NV>& y) {
  constexpr int P = Col<float, NV>::P;
  uint64_t g0 = 0, g1 = 0;  // bit patterns of (0.f, 0.f)
#pragma unroll
  for (int e = 0; e < P; e += 2) {
    g0 = ffma2(x.v[e], y.v[e], g0);
    g1 = ffma2(x.v[e + 1], y.v[e + 1], g1);
  }
  float p0, p1, p2, p3;
  unpack2(g0, p0, p1);
  unpack2(g1, p2, p3);
  return (p0 + p1) + (p2 + p3);
}
template <int NV>
__device__ __forceinline__ double dot_lane(const Col<double, NV>& x, const Col<double, NV>& y) {
  constexpr int P = Col<double, NV>::P;
  double g0 = 0.0, g1 = 0.0;
#pragma unroll
  for (int e = 0; e < P; e += 2) {
    g0 = fma(x.v[e], y.v[e], g0);
    g1 = fma(x.v[e + 1], y.v[e + 1], g1);
  }
  return g0 + g1;
}

// Rutishauser's form with tau = tan(theta/2) = s / (1 + c):
//   x' = x - s (y + tau x),  y' = y + s (x - tau y).
// It equals (c x - s y, s x + c y) but applies the O(theta^2) shrink of x and y
// as an explicit correction, so small rotations (where c rounds to 1) stay
// orthogonal to working precision instead of growing both columns by
// (1 + t^2) -- a bias that would otherwise accumulate over the thousands of
// rotations a column takes part in.
template <int NV>
__device__ __forceinline__ void rotate_lane(Col<float, NV>& x, Col<float, NV>& y, float s, float tau) {
  const uint64_t tau2 = pack2(tau, tau), ntau2 = pack2(-tau, -tau);
  const uint64_t s2 = pack2(s, s), ns2 = pack2(-s, -s);
#pragma unroll
  for (int e = 0; e < Col<float, NV>::P; ++e) {
    const uint64_t xv = x.v[e], yv = y.v[e];
    const uint64_t u = ffma2(tau2, xv, yv);   // y + tau x
    const uint64_t w = ffma2(ntau2, yv, xv);  // x - tau y
    x.v[e] = ffma2(ns2, u, xv);
    y.v[e] = ffma2(s2, w, yv);
  }
}
template <int NV>
__device__ __forceinline__ void rotate_lane(Col<double, NV>& x, Col<double, NV>& y, double s, double tau) {
#pragma unroll
  for (int e = 0; e < Col<double, NV>::P; ++e) {
    const double xv = x.v[e], yv = y.v[e];
    x.v[e] = xv - s * (yv + tau * xv);
    y.v[e] = yv + s * (xv - tau * yv);
  }
}

// Rotation that zeroes the cross product g = x.y of two columns with squared
// norms a, b: tan(2 theta) = 2 g / (a - b) with |theta| <= pi/4.  Outputs
// s = sin(theta), tau = tan(theta / 2) and t g (t = tan(theta)), the amount by
// which the squared norms move: a' = a - t g, b' = b + t g.
//
// FP32: a scale-free closed form on the hardware approximations.  With
// d = (b - a) s and h = 2 g s for a power of two s ~ 1/(a + b) (the formulas
// below depend only on the ratio h / d), R = sqrt(d^2 + h^2)
// and u = |d| + R:  cos = u / sqrt(2 R u),  sin = sign(d) h / sqrt(2 R u),
// tan = sign(d) h / u -- three dependent approximations (rsqrt, rsqrt,
// reciprocal) where the cotangent form needs five.  The angle need not be
// exact; the tau form above keeps the applied rotation orthogonal.
__device__ __forceinline__ void rotation_params(float a, float b, float g, float& s, float& tau, float& tg) {
  // d and h scaled by a power of two (from the exponent of a + b) into [-2, 2]:
  // exact, and no reciprocal on the step's dependency chain
  const int ex = min((__float_as_int(a + b) >> 23) & 0xff, 253);
  const float rab = __int_as_float((253 - ex) << 23);  // (a + b) rab in [0.5, 1)
  const float d = (b - a) * rab, h = 2.0f * g * rab;
  const float q = fmaf(d, d, h * h);
  const float R = q * rsqrtf(q);
  const float u = fabsf(d) + R;
  const float rp = rsqrtf(2.0f * R * u);
  const float c = u * rp;
  const float sh = d < 0.0f ? -h : h;  // sign(d) h
  s = sh * rp;
  tau = __fdividef(s, 1.0f + c);
  tg = __fdividef(sh, u) * g;
}
// FP64: Rutishauser's cotangent form with IEEE division and square root.
__device__ __forceinline__ void rotation_params(double a, double b, double g, double& s, double& tau, double& tg) {
  const double zeta = (b - a) / (2.0 * g);
  const double az = fabs(zeta);
  double t;
  if (az > BigZeta<double>::v)
    t = 0.5 / zeta;
  else
    t = copysign(1.0 / (az + sqrt(1.0 + az * az)), zeta);
  const double c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
  tau = s / (1.0 + c);
  tg = t * g;
}

// "Transposed" warp reduction of K (1, 2 or 4) values: each of the first log2 K
// butterfly levels exchanges half of the values still held, so that afterwards
// every lane holds one running sum; the remaining levels are plain butterflies.
// Lane l ends with the full sum of v[l / (32 / K)] (K - 1 + 5 - log2 K shuffles
// instead of 5 K).
template <typename J, int K>
__device__ __forceinline__ J warp_sum_spread(const J (&v)[K], int lane) {
  constexpr unsigned F = 0xffffffffu;
  J t;
  if constexpr (K == 4) {
    const bool h = (lane & 16) != 0;
    const J r0 = (h ? v[2] : v[0]) + __shfl_xor_sync(F, h ? v[0] : v[2], 16);
    const J r1 = (h ? v[3] : v[1]) + __shfl_xor_sync(F, h ? v[1] : v[3], 16);
    const bool q = (lane & 8) != 0;
    t = (q ? r1 : r0) + __shfl_xor_sync(F, q ? r0 : r1, 8);
    t += __shfl_xor_sync(F, t, 4);
  } else if constexpr (K == 2) {
    const bool h = (lane & 16) != 0;
    t = (h ? v[1] : v[0]) + __shfl_xor_sync(F, h ? v[0] : v[1], 16);
    t += __shfl_xor_sync(F, t, 8);
    t += __shfl_xor_sync(F, t, 4);
  } else {
    t = v[0];
    t += __shfl_xor_sync(F, t, 16);
    t += __shfl_xor_sync(F, t, 8);
    t += __shfl_xor_sync(F, t, 4);
  }
  t += __shfl_xor_sync(F, t, 2);
  t += __shfl_xor_sync(F, t, 1);
  return t;
}

// K independent column pairs (x[i], y[(i + SH) mod K]) held in registers by the
// warp.  The K dot products are reduced with one spread reduction, after which
// the lanes of group i (lanes [i 32/K, (i + 1) 32/K)) hold pair i's cross
// product and compute that pair's rotation -- each group one pair, so the
// angle arithmetic is issued once for all K pairs; the angles are then
// broadcast and each pair whose cosine exceeds the tolerance is rotated.  a /
// bn are the tracked squared norms of x / y; xf / yf have bit i set while x[i] /
// y[i] is fresh (rotated in this or the previous sweep), and rotated columns
// become fresh.  act bit i enables pair i.  Returns the rotated pairs as a bit
// mask.
template <typename J, int NV, int K, int SH>
__device__ __forceinline__ unsigned step_pairs(Col<J, NV> (&x)[K], Col<J, NV> (&y)[K], J (&a)[K], J (&bn)[K],
                                               unsigned& xf, unsigned& yf, unsigned act, J tol2, J tiny,
                                               int lane) {
  if (act == 0) return 0;
  constexpr int GL = 32 / K;  // lanes per pair group
  J pd[K];
#pragma unroll
  for (int i = 0; i < K; ++i) pd[i] = dot_lane(x[i], y[(i + SH) % K]);
  const J g = warp_sum_spread<J, K>(pd, lane);
  const int me = lane / GL;
  J am = a[0], bm = bn[SH % K];
#pragma unroll
  for (int i = 1; i < K; ++i)
    if (me == i) {
      am = a[i];
      bm = bn[(i + SH) % K];
    }
  const bool on = ((act >> me) & 1u) && am > tiny && bm > tiny && g * g > tol2 * am * bm;
  const unsigned bal = __ballot_sync(0xffffffffu, on);
  unsigned rot = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) rot |= ((bal >> (i * GL)) & 1u) << i;
  if (rot == 0) return 0;
  J s = J(0), tau = J(0), tg = J(0);
  if constexpr (sizeof(J) == 4)
    rotation_params(am, bm, g, s, tau, tg);
  else if (on)
    rotation_params(am, bm, g, s, tau, tg);
  J si[K], ti[K], gi[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    si[i] = __shfl_sync(0xffffffffu, s, i * GL);
    ti[i] = __shfl_sync(0xffffffffu, tau, i * GL);
    gi[i] = __shfl_sync(0xffffffffu, tg, i * GL);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int j = (i + SH) % K;
    if ((rot >> i) & 1u) {  // warp-uniform
      rotate_lane(x[i], y[j], si[i], ti[i]);
      a[i] -= gi[i];
      bn[j] += gi[i];
      xf |= 1u << i;
      yf |= 1u << j;
    }
  }
  return rot;
}

// y-side mask of a step's rotations (pair i touches y[(i + SH) mod K])
template <int K, int SH>
__device__ __forceinline__ unsigned y_mask(unsigned rot) {
  unsigned m = 0;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if ((rot >> i) & 1u) m |= 1u << ((i + SH) % K);
  return m;
}

// FP32, four columns of each block per warp: a meeting's 16 cross pairs as eight
// half-steps of two pairs on the XOR schedule (step s pairs x_i with y_(i xor s)).
// In steps 0-1 the half-steps of {x0, x1, y0, y1} and of {x2, x3, y2, y3} touch
// disjoint columns, and so do those of {x0, x1, y2, y3} and {x2, x3, y0, y1} in
// steps 2-3: two independent dependency chains, which the scheduler interleaves
// (one half's rotation FMAs issue while the other waits on its reduction and
// angle).  Rotations are predicated instead of branched: a pair that does not
// rotate gets s = tau = 0, which leaves both columns exactly unchanged.
template <int NV>
__device__ __forceinline__ unsigned half_step(Col<float, NV>& xa, Col<float, NV>& yb, Col<float, NV>& xc,
                                              Col<float, NV>& yd, float& a0, float& b0, float& a1, float& b1,
                                              bool act0, bool act1, float tol2, float tiny, int lane) {
  constexpr unsigned F = 0xffffffffu;
  float pd[2] = {dot_lane(xa, yb), dot_lane(xc, yd)};
  const float g = warp_sum_spread<float, 2>(pd, lane);  // lanes 0-15: pair 0, 16-31: pair 1
  const bool hi = (lane & 16) != 0;
  const float am = hi ? a1 : a0, bm = hi ? b1 : b0;
  const bool on = (hi ? act1 : act0) && am > tiny && bm > tiny && g * g > tol2 * am * bm;
  float sn = 0.f, tau = 0.f, tg = 0.f;
  rotation_params(am, bm, g, sn, tau, tg);
  sn = on ? sn : 0.f;
  tau = on ? tau : 0.f;
  tg = on ? tg : 0.f;
  const float s0 = __shfl_sync(F, sn, 0), t0 = __shfl_sync(F, tau, 0), g0 = __shfl_sync(F, tg, 0);
  const float s1 = __shfl_sync(F, sn, 16), t1 = __shfl_sync(F, tau, 16), g1 = __shfl_sync(F, tg, 16);
  const unsigned bal = __ballot_sync(F, on);
  rotate_lane(xa, yb, s0, t0);
  rotate_lane(xc, yd, s1, t1);
  a0 -= g0;
  b0 += g0;
  a1 -= g1;
  b1 += g1;
  return (bal & 1u) | ((bal >> 15) & 2u);  // bit 0: pair 0 rotated, bit 1: pair 1
}

// The meeting of x[0..3] with y[0..3]: xf / yf fresh bits (updated as columns
// rotate), xd / yd the columns rotated here, nrot the rotation count.
template <int NV>
__device__ __forceinline__ void meet4_xor(Col<float, NV> (&x)[4], Col<float, NV> (&y)[4], float (&a)[4],
                                          float (&bn)[4], unsigned& xf, unsigned& yf, float tol2, float tiny,
                                          int lane, unsigned& xd, unsigned& yd, int& nrot) {
  auto act = [&](int i, int j) { return (((xf >> i) | (yf >> j)) & 1u) != 0; };
  auto note = [&](unsigned r, int i0, int j0, int i1, int j1) {
    const unsigned xm = ((r & 1u) << i0) | (((r >> 1) & 1u) << i1);
    const unsigned ym = ((r & 1u) << j0) | (((r >> 1) & 1u) << j1);
    xf |= xm;
    xd |= xm;
    yf |= ym;
    yd |= ym;
    nrot += __popc(r);
  };
  unsigned rA, rB;
  // steps 0 and 1: {x0, x1} with {y0, y1}, {x2, x3} with {y2, y3}
  rA = half_step(x[0], y[0], x[1], y[1], a[0], bn[0], a[1], bn[1], act(0, 0), act(1, 1), tol2, tiny, lane);
  rB = half_step(x[2], y[2], x[3], y[3], a[2], bn[2], a[3], bn[3], act(2, 2), act(3, 3), tol2, tiny, lane);
  note(rA, 0, 0, 1, 1);
  note(rB, 2, 2, 3, 3);
  rA = half_step(x[0], y[1], x[1], y[0], a[0], bn[1], a[1], bn[0], act(0, 1), act(1, 0), tol2, tiny, lane);
  rB = half_step(x[2], y[3], x[3], y[2], a[2], bn[3], a[3], bn[2], act(2, 3), act(3, 2), tol2, tiny, lane);
  note(rA, 0, 1, 1, 0);
  note(rB, 2, 3, 3, 2);
  // steps 2 and 3: {x0, x1} with {y2, y3}, {x2, x3} with {y0, y1}
  rA = half_step(x[0], y[2], x[1], y[3], a[0], bn[2], a[1], bn[3], act(0, 2), act(1, 3), tol2, tiny, lane);
  rB = half_step(x[2], y[0], x[3], y[1], a[2], bn[0], a[3], bn[1], act(2, 0), act(3, 1), tol2, tiny, lane);
  note(rA, 0, 2, 1, 3);
  note(rB, 2, 0, 3, 1);
  rA = half_step(x[0], y[3], x[1], y[2], a[0], bn[3], a[1], bn[2], act(0, 3), act(1, 2), tol2, tiny, lane);
  rB = half_step(x[2], y[1], x[3], y[0], a[2], bn[1], a[3], bn[0], act(2, 1), act(3, 0), tol2, tiny, lane);
  note(rA, 0, 3, 1, 2);
  note(rB, 2, 1, 3, 0);
}

// Sum over the warp of 16 values per lane, transposed: each butterfly level
// exchanges half of the values still held, so that lane l ends with the full sum
// of v[l >> 1] (16 values in 16 shuffles over five levels).
__device__ __forceinline__ float warp_sum_spread16(const float (&v)[16], int lane) {
  constexpr unsigned F = 0xffffffffu;
  float r8[8], r4[4], r2[2];
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0, h2 = (lane & 2) != 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) r8[k] = (h16 ? v[k + 8] : v[k]) + __shfl_xor_sync(F, h16 ? v[k] : v[k + 8], 16);
#pragma unroll
  for (int k = 0; k < 4; ++k) r4[k] = (h8 ? r8[k + 4] : r8[k]) + __shfl_xor_sync(F, h8 ? r8[k] : r8[k + 4], 8);
#pragma unroll
  for (int k = 0; k < 2; ++k) r2[k] = (h4 ? r4[k + 2] : r4[k]) + __shfl_xor_sync(F, h4 ? r4[k] : r4[k + 2], 4);
  float r = (h2 ? r2[1] : r2[0]) + __shfl_xor_sync(F, h2 ? r2[0] : r2[1], 2);
  r += __shfl_xor_sync(F, r, 1);
  return r;
}

// Late-sweep pre-check of a meeting (FP32, four columns a side): all 16 cross
// products from the columns as they are, one reduction, and each pair's rotation
// test with the tracked norms.  True when no pair passes it: the meeting's steps
// would then rotate nothing and change nothing (a rotation is the only thing
// that changes a column), so they can be skipped with the same result.
template <int NV>
__device__ __forceinline__ bool meeting_clean(const Col<float, NV> (&x)[4], const Col<float, NV> (&y)[4],
                                              const float (&a)[4], const float (&bn)[4], unsigned xf, unsigned yf,
                                              float tol2, float tiny, int lane) {
  float pd[16];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) pd[4 * i + j] = dot_lane(x[i], y[j]);
  const float g = warp_sum_spread16(pd, lane);
  const int idx = lane >> 1, me_i = idx >> 2, me_j = idx & 3;
  float am = a[0], bm = bn[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    if (me_i == k) am = a[k];
    if (me_j == k) bm = bn[k];
  }
  const bool act = (((xf >> me_i) | (yf >> me_j)) & 1u) != 0;
  const bool on = act && am > tiny && bm > tiny && g * g > tol2 * am * bm;
  return __ballot_sync(0xffffffffu, on) == 0u;
}

// The same pre-check for two columns a side (FP64, or FP32 on tall problems):
// four cross products, one reduction.
template <typename J, int NV>
__device__ __forceinline__ bool meeting_clean2(const Col<J, NV> (&x)[2], const Col<J, NV> (&y)[2],
                                               const J (&a)[2], const J (&bn)[2], unsigned xf, unsigned yf, J tol2,
                                               J tiny, int lane) {
  const J pd[4] = {dot_lane(x[0], y[0]), dot_lane(x[0], y[1]), dot_lane(x[1], y[0]), dot_lane(x[1], y[1])};
  const J g = warp_sum_spread<J, 4>(pd, lane);  // lane l: pair l / 8
  const int idx = lane >> 3, i = idx >> 1, j = idx & 1;
  const J am = i ? a[1] : a[0], bm = j ? bn[1] : bn[0];
  const bool act = (((xf >> i) | (yf >> j)) & 1u) != 0;
  const bool on = act && am > tiny && bm > tiny && g * g > tol2 * am * bm;
  return __ballot_sync(0xffffffffu, on) == 0u;
}

// Convergence check after a sweep that rotated few pairs (FP32, four columns
// per warp).  Every column of the problem is in W (global memory) and `stamp`
// holds the sweep of each column's last rotation.  The next sweep would test
// exactly the pairs with a column rotated in sweep `sweep` ("fresh" ones): this
// CTA tests its own 2b staged columns (sm, column c at sm + c rp, global index
// gidx(c)) against every fresh column, 4 x 4 products per reduction, with norms
// recomputed from the columns as the next sweep's refresh would.  Returns true
// (in every thread) when some pair would rotate.
template <int NV, typename GIdx>
__device__ bool fresh_pairs_open(const float* sm, int b, int rp, GIdx gidx, const float* W, const int* stamp,
                                 int cols, int sweep, float tol2, float tiny, int* s_list, int* s_count,
                                 float* s_own_nrm, int lane, int wid, int nwarps) {
  // the fresh columns, compacted (order does not matter)
  if (threadIdx.x == 0) *s_count = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < cols; g += blockDim.x)
    if (stamp[g] == sweep) s_list[atomicAdd(s_count, 1)] = g;
  // own column norms
  for (int c = wid; c < 2 * b; c += nwarps) {
    Col<float, NV> x;
    x.load(sm + (int64_t)c * rp, lane);
    const float t = warp_sum_j(dot_lane(x, x));
    if (lane == 0) s_own_nrm[c] = t;
  }
  __syncthreads();
  const int nf = *s_count;
  bool open = false;
  const int ngrp = (nf + 3) / 4, nown = (2 * b + 3) / 4;
  for (int q = wid; q < ngrp * nown && !open; q += nwarps) {
    const int fg = q / nown, og = q - fg * nown;
    Col<float, NV> f[4], x[4];
    float fa[4], xa[4];
    int fgi[4], xgi[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = 4 * fg + i, c = 4 * og + i;
      fgi[i] = k < nf ? s_list[k] : -1;
      xgi[i] = c < 2 * b ? gidx(c) : -2;
      if (fgi[i] >= 0) {
        f[i].load(W + (int64_t)fgi[i] * rp, lane);
      } else {
#pragma unroll
        for (int e = 0; e < Col<float, NV>::P; ++e) f[i].v[e] = 0;
      }
      if (c < 2 * b) {
        x[i].load(sm + (int64_t)c * rp, lane);
        xa[i] = s_own_nrm[c];
      } else {
#pragma unroll
        for (int e = 0; e < Col<float, NV>::P; ++e) x[i].v[e] = 0;
        xa[i] = 0.f;
      }
    }
    float fn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) fn[i] = dot_lane(f[i], f[i]);
    const float fsum = warp_sum_spread<float, 4>(fn, lane);  // lane l: fresh column l / 8
#pragma unroll
    for (int i = 0; i < 4; ++i) fa[i] = __shfl_sync(0xffffffffu, fsum, 8 * i);
    float pd[16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) pd[4 * i + j] = dot_lane(x[i], f[j]);
    const float g = warp_sum_spread16(pd, lane);
    const int idx = lane >> 1, me_i = idx >> 2, me_j = idx & 3;
    float am = xa[0], bm = fa[0];
    int gi = xgi[0], gj = fgi[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      if (me_i == k) {
        am = xa[k];
        gi = xgi[k];
      }
      if (me_j == k) {
        bm = fa[k];
        gj = fgi[k];
      }
    }
    const bool on = gj >= 0 && gi >= 0 && gi != gj && am > tiny && bm > tiny && g * g > tol2 * am * bm;
    open = __ballot_sync(0xffffffffu, on) != 0u;
  }
  return __syncthreads_or(open) != 0;
}

// One round on the 2b staged columns (local columns [0, b) = block I, [b, 2b) =
// block J), by G = b / K warps, each holding K columns of each block in
// registers:
//   norms   squared norms of the staged columns, refreshed (resets the drift of
//           the tracked values);
//   intra   (first round of a sweep only) the pairs inside each block, by the
//           circle method over its b columns: b - 1 sub-steps of b disjoint
//           pairs, K of them per warp;
//   cross   all b x b cross pairs: warp w keeps columns [wK, wK + K) of block I
//           and, in sub-round s, takes the K columns of group (w + s) mod G of
//           block J; the K x K pairs of a meeting run as K steps of K disjoint
//           pairs (x_i with y_{(i + step) mod K}).
// Each column thus crosses shared memory once per K pairs instead of once per
// pair, and each step has K independent reduction chains in flight.  s_nrm /
// s_stamp hold the squared norms and the sweep of each column's last rotation
// (block I at [0, b), block J at [32, 32 + b)).  The norms are recomputed from
// the columns when `refresh` is set (resetting the drift of the tracked values);
// otherwise the tracked values that travelled with the blocks are used.
// Returns the number of rotations this warp applied (identical in every lane).
template <typename J, int NV, int K>
__device__ __forceinline__ int process_round(J* sm, J* s_nrm, int* s_stamp, int b, int rp, int t, int sweep,
                                             J tol2, J tiny, int lane, int wid, bool refresh, bool precheck) {
  const int G = b / K;  // warps doing pair work (== warps in the block)
  auto col = [&](int c) { return sm + (int64_t)c * rp; };
  auto sidx = [&](int c) { return c < b ? c : 32 + (c - b); };
  // a pair needs a check unless neither column has rotated since the previous sweep
  // (it was then verified orthogonal and has not changed since)
  auto fresh = [&](int st) { return sweep == 0 || st >= sweep - 1; };
  // fresh squared norms, K columns per warp at a time
  for (int c0 = wid * K; refresh && c0 < 2 * b; c0 += G * K) {
    Col<J, NV> x[K];
    J nr[K];
#pragma unroll
    for (int i = 0; i < K; ++i) x[i].load(col(c0 + i), lane);
#pragma unroll
    for (int i = 0; i < K; ++i) nr[i] = dot_lane(x[i], x[i]);
    const J t = warp_sum_spread<J, K>(nr, lane);
    if ((lane & (32 / K - 1)) == 0) s_nrm[sidx(c0 + lane / (32 / K))] = t;
  }
  __syncthreads();
  int rot = 0;
  if (t == 0) {
    const int hb = b / 2;
    for (int st = 0; st < b - 1; ++st) {
      Col<J, NV> x[K], y[K];
      J a[K], bn[K];
      int p0[K], p1[K];
      unsigned act = 0, xf = 0, yf = 0;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int q = wid * K + i;  // pair q of this sub-step: block q / hb, slot q mod hb
        const int blk = q >= hb ? 1 : 0, k = q - blk * hb;
        p0[i] = blk * b + circle_pos(k, st, b);
        p1[i] = blk * b + circle_pos(b - 1 - k, st, b);
        x[i].load(col(p0[i]), lane);
        y[i].load(col(p1[i]), lane);
        a[i] = s_nrm[sidx(p0[i])];
        bn[i] = s_nrm[sidx(p1[i])];
        act |= (fresh(s_stamp[sidx(p0[i])]) || fresh(s_stamp[sidx(p1[i])])) ? (1u << i) : 0u;
      }
      const unsigned r = step_pairs<J, NV, K, 0>(x, y, a, bn, xf, yf, act, tol2, tiny, lane);
#pragma unroll
      for (int i = 0; i < K; ++i) {
        if ((r >> i) & 1u) {
          x[i].store(col(p0[i]), lane);
          y[i].store(col(p1[i]), lane);
          if (lane == 0) {
            s_nrm[sidx(p0[i])] = a[i];
            s_nrm[sidx(p1[i])] = bn[i];
            s_stamp[sidx(p0[i])] = sweep;
            s_stamp[sidx(p1[i])] = sweep;
          }
          ++rot;
        }
      }
      __syncthreads();
    }
  }
  {
    Col<J, NV> x[K];
    J a[K];
    unsigned xf = 0;  // bit i: x[i] is fresh
    const int xc = wid * K;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      x[i].load(col(xc + i), lane);
      a[i] = s_nrm[sidx(xc + i)];
      xf |= fresh(s_stamp[sidx(xc + i)]) ? 1u << i : 0u;
    }
    unsigned xdirty = 0;
    int v = wid;
    for (int s = 0; s < G; ++s) {
      Col<J, NV> y[K];
      J bn[K];
      unsigned yf = 0;  // bit i: y[i] is fresh
      const int yc = b + v * K;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        bn[i] = s_nrm[sidx(yc + i)];
        yf |= fresh(s_stamp[sidx(yc + i)]) ? 1u << i : 0u;
      }
      unsigned ydirty = 0;
      const bool any = (xf | yf) != 0;
      if (any)
#pragma unroll
        for (int i = 0; i < K; ++i) y[i].load(col(yc + i), lane);
      auto act_mask = [&](int sh) {
        unsigned m = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) m |= (((xf >> i) | (yf >> ((i + sh) % K))) & 1u) << i;
        return m;
      };
      unsigned r = 0;
      if constexpr (sizeof(J) == 4 && K == 4) {
        if (any && !(precheck && meeting_clean<NV>(x, y, a, bn, xf, yf, tol2, tiny, lane)))
          meet4_xor<NV>(x, y, a, bn, xf, yf, tol2, tiny, lane, xdirty, ydirty, rot);
      } else {
      bool live = any;
      if constexpr (K == 2) live = any && !(precheck && meeting_clean2<J, NV>(x, y, a, bn, xf, yf, tol2, tiny, lane));
      if (live) r = step_pairs<J, NV, K, 0>(x, y, a, bn, xf, yf, act_mask(0), tol2, tiny, lane);
      xdirty |= r;
      ydirty |= y_mask<K, 0>(r);
      rot += __popc(r);
      if (K > 1) {
        r = live ? step_pairs<J, NV, K, 1 % K>(x, y, a, bn, xf, yf, act_mask(1 % K), tol2, tiny, lane) : 0u;
        xdirty |= r;
        ydirty |= y_mask<K, 1 % K>(r);
        rot += __popc(r);
      }
      if (K > 2) {
        r = live ? step_pairs<J, NV, K, 2 % K>(x, y, a, bn, xf, yf, act_mask(2 % K), tol2, tiny, lane) : 0u;
        xdirty |= r;
        ydirty |= y_mask<K, 2 % K>(r);
        rot += __popc(r);
        r = live ? step_pairs<J, NV, K, 3 % K>(x, y, a, bn, xf, yf, act_mask(3 % K), tol2, tiny, lane) : 0u;
        xdirty |= r;
        ydirty |= y_mask<K, 3 % K>(r);
        rot += __popc(r);
      }
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
        if ((ydirty >> i) & 1u) {
          y[i].store(col(yc + i), lane);
          if (lane == 0) {
            s_nrm[sidx(yc + i)] = bn[i];
            s_stamp[sidx(yc + i)] = sweep;
          }
        }
      }
      __syncthreads();  // the next holder of these columns loads them in the next sub-round
      v = v + 1 == G ? 0 : v + 1;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if ((xdirty >> i) & 1u) {
        x[i].store(col(xc + i), lane);
        if (lane == 0) {
          s_nrm[sidx(xc + i)] = a[i];
          s_stamp[sidx(xc + i)] = sweep;
        }
      }
    }
  }
  __syncthreads();
  return rot;
}

// copy nvec 16-byte vectors (cooperatively over the CTA), eight loads in flight
// per thread
template <typename V>
__device__ __forceinline__ void copy_vecs(V* dst, const V* src, int nvec, int tid, int nthr) {
  int e = tid;
  for (; e + 7 * nthr < nvec; e += 8 * nthr) {
    V v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = src[e + k * nthr];
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[e + k * nthr] = v[k];
  }
  for (; e < nvec; e += nthr) dst[e] = src[e];
}

// ---- cluster shared-memory transfer primitives (PTX) ----------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for phase `parity` of a local mbarrier: false once `limit` SM clock
// cycles (by default 2^31, about a second) have passed without completion
constexpr long long kWaitLimitCycles = 1ll << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit = kWaitLimitCycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// Self-test of the bounded wait: one thread arms a barrier that needs two arrivals,
// arrives once, and waits for the phase that the missing arrival would complete --
// a flag that nothing sets.  After `limit` cycles the wait gives up, BKFAC_ETIMEOUT is
// recorded and the kernel returns, as the eigensolve does when a block exchange
// never lands.  `out` receives 1 when the wait timed out, 0 otherwise.
__global__ void wait_timeout_selftest_kernel(long long limit, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 2);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(&bar))
               : "memory");
  const bool ok = mbar_wait_bounded(&bar, 0u, limit);
  if (!ok) report(BKFAC_ETIMEOUT);
  if (out) *out = ok ? 0 : 1;
}
// bulk copy of `bytes` (multiple of 16) from this CTA's shared memory to shared
// memory of a CTA of the cluster; completion is signalled on that CTA's mbarrier
__device__ __forceinline__ void bulk_push(uint32_t dst_cluster, const void* src, uint32_t bytes,
                                          uint32_t mbar_cluster) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst_cluster),
      "r"(smem_addr(src)), "r"(bytes), "r"(mbar_cluster)
      : "memory");
}
// split cluster barrier: arrive (release) now, wait (acquire) later
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to the async proxy
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// columns per warp and block in the register-blocked rounds (K) and the largest
// block (K columns per warp, b <= 32): four FP32 columns of up to 512 rows per
// warp (8 columns x 16 registers in flight); two for longer FP32 columns and
// for FP64
template <typename J, int NV>
struct PairK {
  static constexpr int K = (sizeof(J) == 4 && NV <= 4) ? 4 : 2;
  static constexpr int kMaxThreads = 32 * (32 / K);
};

// Block exchange between rounds.
// DSM = true: the blocks stay in shared memory (three buffers) and move between
// CTAs of the cluster.  Under the circle method the block at slot q >= 1 in
// round t moves to slot q - 1 in round t + 1 (slot 1 wraps to slot 2C - 1;
// slot 0 is fixed); slot s < C belongs to CTA s as its first block, slot s >= C
// to CTA 2C - 1 - s as its second.  After a round every CTA pushes its two
// blocks (and their stamps) with bulk asynchronous copies straight into the
// next buffer of their next holders, where the copies complete on that
// buffer's mbarrier.  The buffer written at the end of round t was last used
// in round t - 2 and pushed out at its end; those pushes completed before any
// CTA started round t - 1, so it is free once every CTA has finished round
// t - 1.  That condition is a split cluster barrier: each CTA arrives after
// computing a round and waits one round later, just before its pushes, by which
// time the other CTAs have almost always arrived.  DSM = false: blocks go back
// to global memory (L2) between rounds (used when three buffers do not fit).
//
// Stamps: s_stamp[buffer][half * 32 + c] for column c of block `half` (b <= 32),
// so that each block's stamps are one 128-byte transfer.
template <typename J, int NV, bool DSM>
__global__ void __launch_bounds__(PairK<J, NV>::kMaxThreads) jacobi_kernel(const __grid_constant__ JacobiBatch batch, double tol,
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
  __shared__ int s_abort[2];
  __shared__ int s_total;
  __shared__ int s_stop;
  __shared__ int s_vopen;  // the convergence check found a pair that would rotate (this CTA)
  __shared__ int s_vany;   // ... in some CTA of the cluster
  __shared__ double s_tiny;
  __shared__ __align__(16) J s_nrm[3][64];      // tracked squared norms of the staged columns (per buffer)
  __shared__ __align__(16) int s_stamp[3][64];  // sweep of each staged column's last rotation (per buffer)
  __shared__ __align__(8) uint64_t s_full[3];   // per buffer: the incoming blocks have landed

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nthr = blockDim.x;
  const int b = P.b, rp = P.rows_pad, nblk = 2 * C;  // rp == 32 * E
  J* W = (J*)P.W;
  int* stamp = P.stamp;
  J* buf0 = (J*)smem_raw;
  auto buffer = [&](int k) { return buf0 + (DSM ? (int64_t)k * 2 * b * rp : 0); };
  const uint32_t blk_bytes = (uint32_t)((size_t)b * rp * sizeof(J));
  if (wid == 0) {
    // deterministic: fixed lane assignment, fixed shuffle tree
    double f = 0.0;
    for (int j = lane; j < P.cols_pad; j += 32) f += P.colnorm2[j];
    f = warp_sum_j(f);
    if (lane == 0) {
      s_tiny = Eps<J>::u * Eps<J>::u * f;
      s_cnt[0] = s_cnt[1] = 0;
      s_abort[0] = s_abort[1] = 0;
    }
  }
  const int nvec = b * rp / Vec<J>::W;  // vectors per block
  int cur = 0;
  uint32_t phase[3] = {0u, 0u, 0u};
  bool aborted = false;
  bool pending = false;  // this CTA has arrived on the cluster barrier and not yet waited
  if (DSM) {
    // initial blocks of round 0 from global memory
    const int bI = circle_pos(crank, 0, nblk), bJ = circle_pos(nblk - 1 - crank, 0, nblk);
    copy_vecs(reinterpret_cast<V*>(buf0), reinterpret_cast<const V*>(W + (int64_t)bI * b * rp), nvec, tid, nthr);
    copy_vecs(reinterpret_cast<V*>(buf0 + (int64_t)b * rp), reinterpret_cast<const V*>(W + (int64_t)bJ * b * rp),
              nvec, tid, nthr);
    for (int c = tid; c < 64; c += nthr) s_stamp[0][c] = -10;
    if (tid == 0) {
      mbar_init(&s_full[0], 1);
      mbar_init(&s_full[1], 1);
      mbar_init(&s_full[2], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster.sync();  // every CTA's barriers are initialised before any push targets them
  }
  __syncthreads();
  const J tiny = (J)s_tiny;
  const J tol2 = (J)(tol * tol);

  bool converged = false;
  int sweep = 0, last_t = 0;
  // late sweeps (the previous one rotated fewer than 1 in 8 pairs) pre-check
  // each meeting and skip it when it would rotate nothing
  const int64_t npairs = (int64_t)P.cols * (P.cols - 1) / 2;
  int prev_total = -1;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int t = 0; t < nblk - 1; ++t) {
      const int bI = circle_pos(crank, t, nblk);
      const int bJ = circle_pos(nblk - 1 - crank, t, nblk);
      J* sm = buffer(cur);
      int* st = s_stamp[DSM ? cur : 0];
      if (!DSM) {
        copy_vecs(reinterpret_cast<V*>(sm), reinterpret_cast<const V*>(W + (int64_t)bI * b * rp), nvec, tid, nthr);
        copy_vecs(reinterpret_cast<V*>(sm + (int64_t)b * rp), reinterpret_cast<const V*>(W + (int64_t)bJ * b * rp),
                  nvec, tid, nthr);
        for (int c = tid; c < 2 * b; c += nthr) {
          const int gc = (c < b ? bI * b + c : bJ * b + (c - b));
          st[c < b ? c : 32 + (c - b)] = sweep == 0 ? -10 : stamp[gc];
        }
        __syncthreads();
      }
      // with the DSM exchange the tracked norms travel with the blocks and are refreshed
      // once per sweep; through L2 they are recomputed every round
      const int rot = process_round<J, NV, PairK<J, NV>::K>(sm, s_nrm[DSM ? cur : 0], st, b, rp, t, sweep, tol2,
                                                            tiny, lane, wid, !DSM || t == 0,
                                                            prev_total >= 0 && (int64_t)prev_total * 8 < npairs);
      if (lane == 0 && rot) atomicAdd(&s_rot, rot);
      last_t = t;
      if (!DSM) {
        copy_vecs(reinterpret_cast<V*>(W + (int64_t)bI * b * rp), reinterpret_cast<const V*>(sm), nvec, tid, nthr);
        copy_vecs(reinterpret_cast<V*>(W + (int64_t)bJ * b * rp), reinterpret_cast<const V*>(sm + (int64_t)b * rp),
                  nvec, tid, nthr);
        for (int c = tid; c < 2 * b; c += nthr) {
          const int gc = (c < b ? bI * b + c : bJ * b + (c - b));
          stamp[gc] = st[c < b ? c : 32 + (c - b)];
        }
        // the cluster barrier's arrive (release) / wait (acquire) order these global
        // write-backs before any CTA of the cluster loads the blocks in the next round
        cluster.sync();
      } else {
        const int nxt = cur == 2 ? 0 : cur + 1;
        fence_proxy_async_smem();  // this round's rotations, visible to the bulk copies
        if (pending) cluster_wait();  // every CTA has finished the previous round: buffer nxt is free everywhere
        __syncthreads();
        if (tid == 0) {
          mbar_arrive_expect_tx(&s_full[nxt], 2u * (blk_bytes + 128u + 32u * (uint32_t)sizeof(J)));
          J* dst_buf = buffer(nxt);
          for (int half = 0; half < 2; ++half) {
            const int slot = half == 0 ? crank : nblk - 1 - crank;
            const int to = slot == 0 ? 0 : (slot >= 2 ? slot - 1 : nblk - 1);
            const int to_cta = to < C ? to : nblk - 1 - to;
            const int to_half = to < C ? 0 : 1;
            const uint32_t mbar = cluster_addr(smem_addr(&s_full[nxt]), to_cta);
            bulk_push(cluster_addr(smem_addr(dst_buf + (int64_t)to_half * b * rp), to_cta),
                      sm + (int64_t)half * b * rp, blk_bytes, mbar);
            bulk_push(cluster_addr(smem_addr(&s_stamp[nxt][to_half * 32]), to_cta), &s_stamp[cur][half * 32], 128u,
                      mbar);
            bulk_push(cluster_addr(smem_addr(&s_nrm[nxt][to_half * 32]), to_cta), &s_nrm[cur][half * 32],
                      32u * (uint32_t)sizeof(J), mbar);
          }
        }
        cluster_arrive();  // this round is computed (and its blocks are on their way)
        pending = true;
        if (!aborted && !mbar_wait_bounded(&s_full[nxt], phase[nxt])) {
          aborted = true;
          s_abort[0] = 1;  // benign race: every writer stores 1
        }
        phase[nxt] ^= 1u;
        cur = nxt;
        __syncthreads();
      }
    }
    if (tid == 0) s_cnt[sweep & 1] = s_rot;
    if (pending) {
      cluster_wait();
      pending = false;
    }
    cluster.sync();
    if (tid == 0) {
      int total = 0, abort_any = 0;
      for (int q = 0; q < C; ++q) {
        total += *cluster.map_shared_rank(&s_cnt[sweep & 1], q);
        abort_any |= *cluster.map_shared_rank(&s_abort[0], q);
      }
      s_total = total;
      s_stop = abort_any;
      // diagnostics: rotations applied in each sweep
      if (crank == 0 && P.sweeps_out && sweep < kSweepLog) P.sweeps_out[1 + sweep] = total;
    }
    __syncthreads();
    if (s_stop) {  // a transfer never completed: give up with the status set
      if (tid == 0) report(BKFAC_ETIMEOUT);
      break;
    }
    if (s_total == 0) {  // identical in every CTA of the cluster
      converged = true;
      break;
    }
    prev_total = s_total;
    // few rotations: instead of a sweep that would only confirm convergence, write
    // the columns back and test the pairs of the columns this sweep rotated
    if constexpr (sizeof(J) == 4 && PairK<J, NV>::K == 4) {
      if ((int64_t)s_total * 256 <= npairs && sweep + 1 < max_sweeps) {
        int vI, vJ;
        J* smv;
        int* s_list;
        if constexpr (DSM) {
          // this CTA's blocks (those of the round after the last) and their stamps
          // go back to global memory; scratch in the buffer after `cur` (free until
          // the next sweep's first push)
          const int tn = last_t + 1;
          vI = circle_pos(crank, tn, nblk);
          vJ = circle_pos(nblk - 1 - crank, tn, nblk);
          smv = buffer(cur);
          copy_vecs(reinterpret_cast<V*>(W + (int64_t)vI * b * rp), reinterpret_cast<const V*>(smv), nvec, tid,
                    nthr);
          copy_vecs(reinterpret_cast<V*>(W + (int64_t)vJ * b * rp),
                    reinterpret_cast<const V*>(smv + (int64_t)b * rp), nvec, tid, nthr);
          for (int c = tid; c < 2 * b; c += nthr)
            stamp[c < b ? vI * b + c : vJ * b + (c - b)] = s_stamp[cur][c < b ? c : 32 + (c - b)];
          s_list = reinterpret_cast<int*>(buffer(cur == 2 ? 0 : cur + 1));
        } else {
          // through L2 the columns and stamps are in global memory after every round:
          // stage the blocks of the next sweep's first round; scratch after the buffer
          vI = circle_pos(crank, 0, nblk);
          vJ = circle_pos(nblk - 1 - crank, 0, nblk);
          smv = buffer(0);
          copy_vecs(reinterpret_cast<V*>(smv), reinterpret_cast<const V*>(W + (int64_t)vI * b * rp), nvec, tid,
                    nthr);
          copy_vecs(reinterpret_cast<V*>(smv + (int64_t)b * rp), reinterpret_cast<const V*>(W + (int64_t)vJ * b * rp),
                    nvec, tid, nthr);
          s_list = reinterpret_cast<int*>(smv + (int64_t)2 * b * rp);
        }
        cluster.sync();  // every CTA's columns and stamps are in global memory
        int* s_cnt_f = s_list + P.cols_pad;
        float* s_own = reinterpret_cast<float*>(s_cnt_f + 32);
        auto gidx = [&](int c) { return c < b ? vI * b + c : vJ * b + (c - b); };
        const bool open = fresh_pairs_open<NV>(reinterpret_cast<const float*>(smv), b, rp, gidx,
                                               reinterpret_cast<const float*>(W), stamp, P.cols, sweep,
                                               (float)tol2, (float)tiny, s_list, s_cnt_f, s_own, lane, wid,
                                               nthr / 32);
        if (tid == 0) s_vopen = open ? 1 : 0;
        cluster.sync();
        if (tid == 0) {
          int any = 0;
          for (int q = 0; q < C; ++q) any |= *cluster.map_shared_rank(&s_vopen, q);
          s_vany = any;
        }
        __syncthreads();
        const bool still_open = s_vany != 0;
        cluster.sync();  // every CTA has read the verdicts before s_vopen changes again
        if (!still_open) {  // nothing would rotate: converged after this sweep
          converged = true;
          break;
        }
      }
    }
  }
  if (DSM && !s_stop) {
    // write the final blocks back: after the last round's exchange, buffer `cur`
    // holds the blocks of the round after last_t
    const int tn = last_t + 1;
    const int bI = circle_pos(crank, tn, nblk), bJ = circle_pos(nblk - 1 - crank, tn, nblk);
    const J* sm = buffer(cur);
    copy_vecs(reinterpret_cast<V*>(W + (int64_t)bI * b * rp), reinterpret_cast<const V*>(sm), nvec, tid, nthr);
    copy_vecs(reinterpret_cast<V*>(W + (int64_t)bJ * b * rp), reinterpret_cast<const V*>(sm + (int64_t)b * rp), nvec,
              tid, nthr);
  }
  if (crank == 0 && tid == 0) {
    if (P.sweeps_out) *P.sweeps_out = converged ? sweep + 1 : sweep;
    if (!converged && !s_stop) report(BKFAC_ENOCONV);
  }
  cluster.sync();  // keep every CTA's shared memory alive until all remote accesses are done
}

template <typename J, int NV, bool DSM>
int launch_typed(const JacobiBatch& batch, int nprob, int C, int b, size_t smem, double tol, int max_sweeps,
                 cudaStream_t s) {
  if (b % PairK<J, NV>::K != 0 || b / PairK<J, NV>::K * 32 > PairK<J, NV>::kMaxThreads)
    return (int)cudaErrorInvalidValue;
  auto kfn = jacobi_kernel<J, NV, DSM>;
  // function attributes are set once per instantiation (the call can stall the host)
  static std::atomic<uint64_t> configured{0};
  cudaError_t e = cudaSuccess;
  if (!configured_here(configured)) {
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    mark_configured(configured);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nprob * C), 1, 1);
  cfg.blockDim = dim3((unsigned)(32 * (b / PairK<J, NV>::K)), 1, 1);
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
  // block widths are multiples of the register-blocking width K (see PairK)
  const int nv = rp / (32 * (j_t == DT_F64 ? 2 : 4));
  const int K = (j_t == DT_F32 && nv <= 4) ? 4 : 2;
  const size_t smem_cap = 200 * 1024;
  int C = 16, b = 32;
  // smallest cluster whose blocks are at most b_max columns wide and fit in shared
  // memory; fall back to wider blocks when 16 CTAs are not enough
  bool found = false;
  for (int c : {1, 2, 4, 8, 16}) {
    const int bb = (int)round_up(ceil_div(std::max(cols, 2), 2 * c), K);
    if (bb <= b_max && (size_t)2 * bb * rp * es <= smem_cap) {
      C = c;
      b = bb;
      found = true;
      break;
    }
  }
  if (!found) {
    C = 16;
    b = (int)round_up(ceil_div(std::max(cols, 2), 32), K);
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
  // Block exchange over distributed shared memory (three buffers per CTA, one CTA
  // per SM) unless the tuning table says otherwise.  (A batch that runs more
  // eigensolves than such clusters fit on the GPU picks the L2 exchange for its
  // grouped launches, where a third of the shared memory lets two clusters share SMs.)
  int b = 0, dsm = 1;
  if (nprob > 0) tune_lookup(probs[0].rows, probs[0].cols, j_t, &b, &dsm);
  return launch_jacobi_mode(probs, nprob, C, j_t, tol, max_sweeps, dsm != 0, s);
}

// scratch of the few-rotation convergence check when the blocks go through L2:
// the list of rotated columns, a counter, the staged columns' norms
static size_t jacobi_check_scratch(int cols_pad) { return (size_t)(cols_pad + 32 + 64) * 4; }

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
  // block exchange between rounds: over distributed shared memory (three buffers)
  // when asked for and the buffers fit, else through L2
  const bool dsm = want_dsm && 3 * smem <= 200 * 1024;
  if (j_t == DT_F64)
    return dsm ? launch_nv<double, true>(batch, nprob, C, b, rp, 3 * smem, tol, max_sweeps, s)
               : launch_nv<double, false>(batch, nprob, C, b, rp, smem, tol, max_sweeps, s);
  int cp_max = 0;
  for (int i = 0; i < nprob; ++i) cp_max = std::max(cp_max, probs[i].cols_pad);
  return dsm ? launch_nv<float, true>(batch, nprob, C, b, rp, 3 * smem, tol, max_sweeps, s)
             : launch_nv<float, false>(batch, nprob, C, b, rp, smem + jacobi_check_scratch(cp_max), tol,
                                       max_sweeps, s);
}

int launch_wait_selftest(long long limit_cycles, int* out, cudaStream_t s) {
  wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(limit_cycles, out);
  note_launches(1);
  return (int)cudaGetLastError();
}

size_t jacobi_smem_bytes(int b, int rows_pad, DType j_t) {
  return (size_t)2 * b * rows_pad * (j_t == DT_F64 ? 8 : 4);
}


}  // namespace bkfac

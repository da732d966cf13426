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
                                                          int* near_out, double neg_rel) {
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
  const double neg = neg_rel * (scale ? *scale : 1.0);  // pivots below -neg: not p.s.d.

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
          if (neg_rel > 0.0 && s < -neg) report(BKFAC_ECHOL);
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

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky on a 4 x 4 grid of CTAs (a 16-CTA cluster),
// for the first CholeskyQR pass.  The lower triangle is cut into 16 x 16
// blocks; block (i, j) lives in CTA (i mod 4, j mod 4) (2D block-cyclic), so
// that every step spreads its work over the cluster.  Step k:
//   A  the owner of (k, k) factors it with one warp (lane = row, pivots
//      broadcast by shuffles; a pivot <= thr is dropped: its column of L is
//      zero) and keeps the reciprocals of the diagonal;
//   B  the owners of the blocks (i, k), i > k, solve L_ik L_kk^T = A_ik row by
//      row, with L_kk read from the diagonal owner's shared memory;
//   C  every CTA updates its trailing blocks, A_ij -= L_ik L_jk^T, with the
//      panel blocks it needs copied from their owners.
// Two cluster barriers per step (after A, after B); C needs none: its inputs
// are never written again, and the next diagonal block is updated by its own
// owner.  FP64 throughout.  Blocks are row-major in shared memory.
// With near_tol > 0 the kernel first applies the near-identity test of the
// second CholeskyQR pass to its blocks (all CTAs take the cluster's decision)
// and, when it holds, writes R = I + Phi(E) instead of factoring.
constexpr int CB = 16;     // block size
constexpr int CBT = 512;   // threads per CTA

__device__ __forceinline__ int blk_rank(int pr, int pc) { return pr * 4 + pc; }

__global__ void __launch_bounds__(CBT) chol_block_kernel(const double* __restrict__ Gm, int n, double* R,
                                                         double thr_rel, const double* scale, double near_tol,
                                                         int* near_out, double neg_rel) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int pr = rank / 4, pc = rank % 4;
  const int nb = (n + CB - 1) / CB, S = (nb + 3) / 4;
  extern __shared__ __align__(16) double bsm[];
  double* slots = bsm;                       // S x S blocks: block (4a + pr, 4b + pc) at slot a * S + b
  double* Li = slots + (size_t)S * S * 256;  // S cached panel blocks (rows of this CTA)
  double* Lj = Li + (size_t)S * 256;         // S cached panel blocks (columns of this CTA)
  double* Lkk = Lj + (size_t)S * 256;        // the current diagonal block
  double* inv = Lkk + 256;                   // its reciprocal diagonal (0 for dropped pivots)
  double* inv_local = inv + 16;
  auto slot = [&](int a, int b) { return slots + (size_t)(a * S + b) * 256; };
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double thr = thr_rel * (scale ? *scale : 1.0);
  const double neg = neg_rel * (scale ? *scale : 1.0);  // pivots below -neg: not p.s.d.

  // load the owned lower blocks (entries past n are zero: their pivots are dropped)
  for (int e = tid; e < S * S * 256; e += CBT) {
    const int sl = e >> 8, w = e & 255, a = sl / S, b = sl % S;
    const int i = 4 * a + pr, j = 4 * b + pc;
    const int row = CB * i + (w >> 4), col = CB * j + (w & 15);
    slots[e] = (i < nb && j <= i && row < n && col < n && row >= col) ? Gm[row + (int64_t)col * n] : 0.0;
  }
  __shared__ int s_flag[2];  // [0]: this CTA's blocks are near identity, [1]: the cluster's decision
  if (tid == 0) s_flag[0] = 1;
  __syncthreads();
  if (near_tol > 0.0) {
    // integer compares of the IEEE bit patterns (|g| <= tol off the diagonal,
    // 1 - tol <= g <= 1 + tol on it; NaN fails): no FP64 arithmetic
    const long long tolb = __double_as_longlong(near_tol);
    const long long lob = __double_as_longlong(1.0 - near_tol), hib = __double_as_longlong(1.0 + near_tol);
    bool ok = true;
    for (int e = tid; e < S * S * 256; e += CBT) {
      const int sl = e >> 8, w = e & 255, a = sl / S, b = sl % S;
      const int i = 4 * a + pr, j = 4 * b + pc;
      const int row = CB * i + (w >> 4), col = CB * j + (w & 15);
      if (i >= nb || j > i || row >= n || col >= n || row < col) continue;
      const long long bits = __double_as_longlong(slots[e]);
      ok = ok && (row == col ? (bits >= lob && bits <= hib) : (bits & 0x7fffffffffffffffLL) <= tolb);
    }
    if (!ok) s_flag[0] = 0;  // benign race: every writer stores 0
  } else if (tid == 0) {
    s_flag[0] = 0;
  }
  cluster.sync();
  if (tid == 0) {
    int all = 1;
    for (int q = 0; q < 16; ++q) all &= *cluster.map_shared_rank(&s_flag[0], q);
    s_flag[1] = all;
  }
  __syncthreads();
  const bool near = s_flag[1] != 0;
  if (near_out != nullptr && rank == 0 && tid == 0) *near_out = near ? 1 : 0;

  for (int k = 0; k < (near ? 0 : nb); ++k) {
    const int dk = k & 3, kb = k >> 2;
    // ---- A: factor the diagonal block, all warps of its owner: per column one
    // thread takes the pivot, then the column's scaling and the rank-1 update of
    // the block's trailing lower entries run in parallel (one FP64 operation each),
    // the update written with the unscaled column and 1/pivot:
    //   D[r][c] -= D[r][j] D[c][j] / p,   L[r][j] = D[r][j] / sqrt(p)
    if (pr == dk && pc == dk) {
      double* D = slot(kb, kb);
      __shared__ double s_piv[2];  // 1/sqrt(p), 1/p (0 for a dropped pivot)
      for (int j = 0; j < CB; ++j) {
        if (tid == 0) {
          const double piv = D[j * CB + j];
          const bool keep = piv > thr;  // false for NaN as well
          if (!isfinite(piv)) report(BKFAC_ENONFINITE);
          if (neg_rel > 0.0 && piv < -neg) report(BKFAC_ECHOL);
          double l = 0.0, il = 0.0;
          if (keep) {
            if (piv > 1e-30 && piv < 1e30) {
              // 1/sqrt(piv): the FP32 hardware approximation (about 2^-22 relative
              // error) refined by one Newton step for x^(-1/2),
              // y <- y + y (1 - x y^2) / 2, which squares the error (about 4e-14);
              // FP64 square root and division are long sequences on this GPU's
              // FP64 pipe, and this chain runs once per column
              double y = (double)rsqrtf((float)piv);
              const double e = fma(-piv * y, y, 1.0);
              y = fma(0.5 * y, e, y);
              l = piv * y;
              il = y;
            } else {
              l = sqrt(piv);
              il = 1.0 / l;
            }
          }
          D[j * CB + j] = l;
          inv[j] = il;
          s_piv[0] = il;
          s_piv[1] = il * il;
        }
        __syncthreads();
        const double il = s_piv[0], ip = s_piv[1];
        // trailing entries (r, c), j < c <= r < 16 (at most 120), and the column scaling
        for (int t = tid; t < CB * CB; t += CBT) {
          const int r = t >> 4, c = t & 15;
          if (c > j && c <= r) D[r * CB + c] -= D[r * CB + j] * D[c * CB + j] * ip;
        }
        __syncthreads();
        if (tid > j && tid < CB) D[tid * CB + j] *= il;
        if (tid < j) D[tid * CB + j] = 0.0;  // the strict upper part stays zero
        __syncthreads();
      }
    }
    cluster.sync();  // L_kk and its reciprocals are final
    // ---- B: the panel blocks below the diagonal, owned by the CTAs of grid column dk
    if (pc == dk) {
      const int src = blk_rank(dk, dk);
      const double* rL = cluster.map_shared_rank(slot(kb, kb), src);
      const double* rI = cluster.map_shared_rank(inv, src);
      for (int e = tid; e < 256; e += CBT) Lkk[e] = rL[e];
      if (tid < 16) inv_local[tid] = rI[tid];
      __syncthreads();
      // one thread per row of each owned block (i, k), i > k
      for (int t = tid; t < S * CB; t += CBT) {
        const int a = t / CB, r = t % CB, i = 4 * a + pr;
        if (i <= k || i >= nb) continue;
        double* B = slot(a, kb) + r * CB;
        double x[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) x[c] = B[c];
#pragma unroll
        for (int j = 0; j < CB; ++j) {
          double v = x[j];
#pragma unroll
          for (int m = 0; m < j; ++m) v -= x[m] * Lkk[j * CB + m];
          x[j] = v * inv_local[j];
        }
#pragma unroll
        for (int c = 0; c < CB; ++c) B[c] = x[c];
      }
    }
    cluster.sync();  // the panel of step k is final
    // ---- C: trailing update of the owned blocks (i, j), k < j <= i
    {
      const int rsrc = blk_rank(pr, dk), csrc = blk_rank(pc, dk);
      for (int e = tid; e < 2 * S * 256; e += CBT) {
        const int half = e / (S * 256), w = e % (S * 256), a = w >> 8, o = w & 255;
        const int g = 4 * a + (half ? pc : pr);
        if (g <= k || g >= nb) continue;
        const double* src = cluster.map_shared_rank(slot(a, kb), half ? csrc : rsrc);
        (half ? Lj : Li)[w] = src[o];
      }
      __syncthreads();
      for (int e = tid; e < S * S * 256; e += CBT) {
        const int sl = e >> 8, w = e & 255, a = sl / S, b = sl % S;
        const int i = 4 * a + pr, j = 4 * b + pc;
        if (j <= k || j > i || i >= nb) continue;
        const int r = w >> 4, c = w & 15;
        const double* li = Li + a * 256 + r * CB;
        const double* lj = Lj + b * 256 + c * CB;
        double acc = 0.0;
#pragma unroll
        for (int m = 0; m < CB; ++m) acc += li[m] * lj[m];
        slots[e] -= acc;
      }
      __syncthreads();
    }
  }
  // R = L^T (upper), or I + Phi(E) when near identity (E = G - I: its strict upper
  // part plus half its diagonal); the strictly lower part of R is zero
  for (int e = tid; e < S * S * 256; e += CBT) {
    const int sl = e >> 8, w = e & 255, a = sl / S, b = sl % S;
    const int i = 4 * a + pr, j = 4 * b + pc;
    if (i >= nb || j > i) continue;
    const int row = CB * i + (w >> 4), col = CB * j + (w & 15);
    if (row >= n || col >= n) continue;
    const double v = slots[e];
    R[col + (int64_t)row * n] = row < col ? 0.0 : (!near ? v : (row == col ? 1.0 + 0.5 * (v - 1.0) : v));
    if (row > col) R[row + (int64_t)col * n] = 0.0;
  }
  cluster.sync();  // keep shared memory alive until every remote read is done
}


// ---------------------------------------------------------------------------
// FP32 blocked Cholesky K = G G^T on a 16-CTA cluster, for two uses:
//
// (1) The eigensolve of the Brand core (W mode).  The one-sided Jacobi of the
// update orthogonalises the columns of the core factor L (N x N, K = L L^T is
// the core matrix).  With K = G G^T (G lower triangular), G = L Z for an
// orthogonal Z: G has the same left singular vectors as L -- the eigenvectors of
// K -- and the same singular values.  The Gram of G's columns, G^T G, is K after
// one step of the LR (Cholesky) iteration, much closer to diagonal than L^T L on
// the graded spectra of the EA factors, so the Jacobi run on G instead of L
// needs fewer sweeps (9-10 instead of 11-12 on a 512-column wide-layer core).
// G is written as the Jacobi's column-major rows_pad x cols_pad matrix (zero
// above the diagonal and beyond n) with its columns' squared norms (FP64 sums
// of the FP32 entries).
//
// (2) The CholeskyQR2 passes of the FP32 and mixed-precision paths (R mode): the
// FP64-accurate Gram of the residual is factored in FP32 and R = G^T is written
// as an n x n column-major FP64 upper triangle.  With near_tol > 0 the
// near-identity test of the second pass runs first (on the FP64 Gram) and, when
// every entry passes, R = I + Phi(E) is written instead of factoring (as in the
// FP64 kernels above).
//
// Layout: 4 x 4 grid of CTAs, 32 x 32 blocks of the lower triangle, block (i, j)
// in CTA (i mod 4, j mod 4).  In shared memory a block is row-major with its
// 16-byte chunks XOR-swizzled by the row, element (r, c) at
//   r * 32 + ((c / 4) ^ (r mod 8)) * 4 + c mod 4,
// so that a warp reading a column (a lane per row) or eight lanes reading eight
// rows' chunks with 128-bit accesses meet no bank conflict.  A diagonal block
// holds its full symmetric square until it is factored and then L_kk^T.
// Step k: (A) one warp of the diagonal owner factors L_kk with shuffles (lane =
// row); pivot j is dropped (its column of G is zero) when its Schur complement
// is at most max(thr_rel * K_jj, thr_abs * scale): thr_rel * K_jj is the rounding
// noise of the FP32 elimination relative to the column's own diagonal, thr_abs
// * scale the caller's absolute threshold; (B) the owners of the panel blocks
// (i, k), i > k, solve L_ik L_kk^T = A_ik, a thread per row, and also write
// them transposed to a global (L2) panel buffer; (C) every CTA applies the
// rank-32 update to its trailing blocks from transposed copies of the panel
// blocks, and the owner of block (k + 1, k + 1) updates that block first with
// one warp and factors it (step A of k + 1) while its other warps and the other
// CTAs finish the update (lookahead).  Two cluster barriers per step.  The
// panel buffer is the output buffer (written only after the last step); the
// path that reads the panel from the owners' shared memory instead is kept for
// an output too small for nb blocks (with the sizes the launchers accept this
// happens only when nb = 1, where no panel is read).
constexpr int QB = 32;           // block size
constexpr int QBT = 512;         // threads per CTA
constexpr int kCoreMaxN = 768;   // 6 x 6 blocks per CTA: the most that fit in shared memory

__device__ __forceinline__ int qsw(int r, int c) { return r * QB + ((((c >> 2) ^ r) & 7) << 2) + (c & 3); }

// Factor a 32 x 32 diagonal block in place, one warp: D holds the full symmetric
// square (swizzled) and receives L_kk^T (element (c, r) = L_kk[r][c], zero for
// c > r); inv[j] = 1 / L_kk[j][j] (0 for a dropped pivot).  Lane r keeps row r
// (read as column r of the square).  The pivot of column j + 1 comes from two
// shuffles taken as soon as column j is scaled (the same fma that lane j + 1
// applies to its own entry), so the chain between pivots holds one shuffle; the
// rest of column j reaches the lanes through shared memory (s_l, two 32-float
// buffers) as 128-bit broadcasts.
__device__ __forceinline__ void factor_diag_block(float* D, float* inv, float* s_l, float thr, int lane) {
  float d[QB];
#pragma unroll
  for (int c = 0; c < QB; ++c) d[c] = D[qsw(c, lane)];
  bool bad = false;
  float p = __shfl_sync(0xffffffffu, d[0], 0);
#pragma unroll
  for (int j = 0; j < QB; ++j) {
    bad |= !(fabsf(p) <= 3.402823466e38f);  // NaN or infinite
    const float il = p > __shfl_sync(0xffffffffu, thr, j) ? rsqrtf(p) : 0.f;
    const float l = lane >= j ? d[j] * il : 0.f;
    d[j] = l;
    if (lane == j) inv[j] = il;
    if (j + 1 < QB) {
      const float dn = __shfl_sync(0xffffffffu, d[(j + 1) % QB], (j + 1) % QB);
      const float ln = __shfl_sync(0xffffffffu, l, (j + 1) % QB);
      d[(j + 1) % QB] = fmaf(-l, ln, d[(j + 1) % QB]);
      p = fmaf(-ln, ln, dn);
    }
    if (j + 2 < QB) {
      // buffer j & 1 is rewritten two columns later, after every lane has passed the
      // next column's __syncwarp (and so finished reading it)
      float* sb = s_l + (j & 1) * QB;
      sb[lane] = l;
      __syncwarp();
#pragma unroll
      for (int q = (j + 2) >> 2; q < 8; ++q) {
        const float4 v = *(const float4*)(sb + 4 * q);
        if (4 * q + 0 >= j + 2) d[(4 * q + 0) % QB] = fmaf(-l, v.x, d[(4 * q + 0) % QB]);
        if (4 * q + 1 >= j + 2) d[(4 * q + 1) % QB] = fmaf(-l, v.y, d[(4 * q + 1) % QB]);
        if (4 * q + 2 >= j + 2) d[(4 * q + 2) % QB] = fmaf(-l, v.z, d[(4 * q + 2) % QB]);
        if (4 * q + 3 >= j + 2) d[(4 * q + 3) % QB] = fmaf(-l, v.w, d[(4 * q + 3) % QB]);
      }
    }
  }
  if (bad && lane == 0) report(BKFAC_ENONFINITE);
#pragma unroll
  for (int c = 0; c < QB; ++c) D[qsw(c, lane)] = d[c];
}

// One 4 x 4 tile t (0..63) of a trailing block: T -= L_i L_j^T over the 32 columns of
// the panel, from the transposed panel blocks li = L_i^T, lj = L_j^T ([m][row]).
__device__ __forceinline__ void trail_tile(const float* li, const float* lj, float* T, int t) {
  const int r0 = (t >> 3) << 2, c0 = (t & 7) << 2;
  li += r0;
  lj += c0;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 8
  for (int m = 0; m < QB; ++m) {
    const float4 x = *(const float4*)(li + m * QB);
    const float4 y = *(const float4*)(lj + m * QB);
    const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xs[u], ys[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int row = r0 + u;
    float4* pp = (float4*)(T + row * QB + ((((c0 >> 2) ^ row) & 7) << 2));
    float4 o = *pp;
    o.x -= acc[u][0];
    o.y -= acc[u][1];
    o.z -= acc[u][2];
    o.w -= acc[u][3];
    *pp = o;
  }
}

template <typename TK, bool RM>
__global__ void __launch_bounds__(QBT) chol_core_kernel(const CoreCholArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int pr = rank >> 2, pc = rank & 3;
  const int n = a.n, rows_pad = a.rows_pad, cols_pad = a.cols_pad;
  const int64_t ldk = a.ldk;
  const TK* __restrict__ K = (const TK*)a.K;
  const int nb = (n + QB - 1) / QB, S = (nb + 3) / 4;
  const int ncb = (cols_pad + QB - 1) / QB, Sc = (ncb + 3) / 4;
  extern __shared__ __align__(16) float qsm[];
  float* slots = qsm;                         // S x S blocks: block (4a + pr, 4b + pc) at slot a * S + b
  float* LiT = slots + (size_t)S * S * 1024;  // panel blocks (4a + pr, k), transposed: [m][r]
  float* LjT = LiT + (size_t)S * 1024;        // panel blocks (4b + pc, k), transposed: [m][c]
  float* Lkk = LjT + (size_t)S * 1024;        // L_kk^T (swizzled), copied from the diagonal owner
  float* inv = Lkk + 1024;                    // 1 / L_kk[j][j] (0 for a dropped pivot)
  float* inv_local = inv + 32;
  double* colpart = (double*)(inv_local + 32);  // this CTA's part of the columns' squared norms
  __shared__ float s_kd[kCoreMaxN];
  __shared__ int s_flag[2];  // near identity: [0] this CTA's blocks, [1] the cluster's decision
  __shared__ __align__(16) float s_l[2 * QB];  // column broadcast buffers of factor_diag_block
  auto slot = [&](int ia, int ib) { return slots + (size_t)(ia * S + ib) * 1024; };
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float thr_abs = (float)(a.thr_abs * (a.scale ? *a.scale : 1.0));

  bool near = false;
  if (RM) {
    if (tid == 0) s_flag[0] = a.near_tol > 0.0 ? 1 : 0;
    __syncthreads();
    if (a.near_tol > 0.0) {
      // |g| <= tol off the diagonal, 1 - tol <= g <= 1 + tol on it (NaN fails), on the
      // FP64 Gram, as integer compares of the IEEE bit patterns (no FP64 arithmetic)
      const long long tolb = __double_as_longlong(a.near_tol);
      const long long lob = __double_as_longlong(1.0 - a.near_tol), hib = __double_as_longlong(1.0 + a.near_tol);
      bool ok = true;
      for (int e = tid; e < S * S * 1024; e += QBT) {
        const int sl = e >> 10, w = e & 1023, ia = sl / S, ib = sl % S;
        const int i = 4 * ia + pr, j = 4 * ib + pc;
        const int row = QB * i + (w & 31), col = QB * j + (w >> 5);  // consecutive threads: consecutive rows
        if (i >= nb || j > i || row >= n || col >= n || row < col) continue;
        const long long bits = __double_as_longlong((double)K[row + ldk * col]);
        ok = ok && (row == col ? (bits >= lob && bits <= hib) : (bits & 0x7fffffffffffffffLL) <= tolb);
      }
      if (!ok) s_flag[0] = 0;  // benign race: every writer stores 0
    }
    cluster.sync();
    if (tid == 0) {
      int all = 1;
      for (int q = 0; q < 16; ++q) all &= *cluster.map_shared_rank(&s_flag[0], q);
      s_flag[1] = all;
    }
    __syncthreads();
    near = s_flag[1] != 0;
    if (a.near_out != nullptr && rank == 0 && tid == 0) *a.near_out = near ? 1 : 0;
  }

  if (!near) {
    // the original diagonal, for the relative drop threshold
    for (int i = tid; i < nb * QB; i += QBT) s_kd[i] = i < n ? (float)K[i + ldk * i] : 0.f;
    // owned lower blocks; a diagonal block as its full symmetric square read from the
    // lower triangle; entries past n are zero (their pivots are dropped)
#pragma unroll 8
    for (int e = tid; e < S * S * 1024; e += QBT) {
      const int sl = e >> 10, w = e & 1023, ia = sl / S, ib = sl % S;
      const int i = 4 * ia + pr, j = 4 * ib + pc;
      const int c = w >> 5, r = w & 31;  // consecutive threads: consecutive rows (coalesced reads)
      const int row = QB * i + r, col = QB * j + c;
      float v = 0.f;
      if (i < nb && j <= i && row < n && col < n)
        v = (float)(row >= col ? K[row + ldk * col] : K[col + ldk * row]);
      slots[(size_t)sl * 1024 + qsw(r, c)] = v;
    }
    __syncthreads();
  }

  // Panel blocks reach the trailing updates through global memory (L2) when the output
  // buffer can hold them until the output phase (nb blocks of 1024 floats, transposed):
  // one owner serving eight readers over distributed shared memory was the bottleneck.
  // The output is written only after the last step, whose cluster barriers follow every
  // read of the panel.
  float* P = nullptr;
  if (RM) {
    if ((int64_t)2 * n * n >= (int64_t)nb * 1024) P = (float*)a.R;
  } else {
    if ((int64_t)rows_pad * cols_pad >= (int64_t)nb * 1024) P = a.W;
  }
  auto thr_of = [&](int k) { return fmaxf(a.thr_rel * s_kd[k * QB + lane], thr_abs); };

  for (int k = 0; k < (near ? 0 : nb); ++k) {
    const int dk = k & 3, kb = k >> 2;
    // ---- A: the first diagonal block; later ones are factored by their owner inside the
    // previous step's trailing update (lookahead)
    if (k == 0 && pr == 0 && pc == 0 && wid == 0) factor_diag_block(slot(0, 0), inv, s_l, thr_of(0), lane);
    cluster.sync();  // L_kk and its reciprocals are final
    // ---- B: the panel blocks below the diagonal, owned by the CTAs of grid column dk
    if (pc == dk) {
      const int src = dk * 4 + dk;
      const float4* rL = (const float4*)cluster.map_shared_rank(slot(kb, kb), src);
      const float* rI = cluster.map_shared_rank(inv, src);
      for (int e = tid; e < 256; e += QBT) ((float4*)Lkk)[e] = rL[e];
      if (tid < 32) inv_local[tid] = rI[tid];
      __syncthreads();
      for (int t = tid; t < S * QB; t += QBT) {
        const int ia = t >> 5, r = t & 31, i = 4 * ia + pr;
        if (i <= k || i >= nb) continue;
        float* B = slot(ia, kb) + r * QB;
        float x[QB];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 v = *(const float4*)(B + (((q ^ r) & 7) << 2));
          x[4 * q] = v.x;
          x[4 * q + 1] = v.y;
          x[4 * q + 2] = v.z;
          x[4 * q + 3] = v.w;
        }
        // right-looking: x_j /= L_jj, then x_m -= x_j L_mj for m > j (row j of the
        // stored L_kk^T holds L_mj, m = 0..31)
#pragma unroll
        for (int j = 0; j < QB; ++j) {
          const float xj = x[j] * inv_local[j];
          x[j] = xj;
#pragma unroll
          for (int q = (j + 1) >> 2; q < 8; ++q) {
            const float4 lv = *(const float4*)(Lkk + j * QB + (((q ^ j) & 7) << 2));
            if (4 * q + 0 > j) x[4 * q + 0] = fmaf(-xj, lv.x, x[4 * q + 0]);
            if (4 * q + 1 > j) x[4 * q + 1] = fmaf(-xj, lv.y, x[4 * q + 1]);
            if (4 * q + 2 > j) x[4 * q + 2] = fmaf(-xj, lv.z, x[4 * q + 2]);
            if (4 * q + 3 > j) x[4 * q + 3] = fmaf(-xj, lv.w, x[4 * q + 3]);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *(float4*)(B + (((q ^ r) & 7) << 2)) = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        if (P != nullptr) {
          // transposed into the panel buffer: element [m][r] of block i (coalesced over r)
          float* pb = P + (size_t)i * 1024 + r;
#pragma unroll
          for (int m = 0; m < QB; ++m) pb[m * QB] = x[m];
        }
      }
    }
    cluster.sync();  // the panel of step k is final (in shared and in global memory)
    // ---- C: trailing update of the owned blocks (i, j), k < j <= i
    {
      // transposed panel blocks (4a + pr, k) -> LiT[a] and (4b + pc, k) -> LjT[b]; a batch
      // of loads first, then its stores: the generic remote pointers could alias the local
      // tiles, so interleaving them would serialise the loads
      constexpr int kMaxCopy = kCoreMaxN / 128;  // copies per thread at most (6 x 6 blocks)
      constexpr int kBatch = 3;                  // loads in flight per batch
#pragma unroll
      for (int u0 = 0; u0 < kMaxCopy; u0 += kBatch) {
        float4 cv[kBatch];
        if (P != nullptr) {
          const float4* P4 = (const float4*)P;
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int e = tid + (u0 + u) * QBT;
            cv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e >= 2 * S * 256) continue;
            const int half = e / (S * 256), w = e % (S * 256), ia = w >> 8, o = w & 255;
            const int g = 4 * ia + (half ? pc : pr);
            if (g <= k || g >= nb) continue;
            cv[u] = __ldcg(P4 + (size_t)g * 256 + o);  // L2 only: the buffer is rewritten every step
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int e = tid + (u0 + u) * QBT;
            if (e >= 2 * S * 256) continue;
            const int half = e / (S * 256), w = e % (S * 256), ia = w >> 8, o = w & 255;
            const int g = 4 * ia + (half ? pc : pr);
            if (g <= k || g >= nb) continue;
            *(float4*)((half ? LjT : LiT) + (size_t)ia * 1024 + 4 * o) = cv[u];
          }
        } else {
          const int rsrc = pr * 4 + dk, csrc = pc * 4 + dk;
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int e = tid + (u0 + u) * QBT;
            cv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e >= 2 * S * 256) continue;
            const int half = e / (S * 256), w = e % (S * 256), ia = w >> 8, o = w & 255;
            const int g = 4 * ia + (half ? pc : pr);
            if (g <= k || g >= nb) continue;
            const int r = o & 31, q = o >> 5;
            const float4* src = (const float4*)cluster.map_shared_rank(slot(ia, kb), half ? csrc : rsrc);
            cv[u] = src[(r * QB + (((q ^ r) & 7) << 2)) >> 2];
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int e = tid + (u0 + u) * QBT;
            if (e >= 2 * S * 256) continue;
            const int half = e / (S * 256), w = e % (S * 256), ia = w >> 8, o = w & 255;
            const int g = 4 * ia + (half ? pc : pr);
            if (g <= k || g >= nb) continue;
            const int r = o & 31, q = o >> 5;
            float* dst = (half ? LjT : LiT) + (size_t)ia * 1024 + r;
            dst[(4 * q + 0) * QB] = cv[u].x;
            dst[(4 * q + 1) * QB] = cv[u].y;
            dst[(4 * q + 2) * QB] = cv[u].z;
            dst[(4 * q + 3) * QB] = cv[u].w;
          }
        }
      }
      __syncthreads();
      // lookahead: the owner of diagonal block k + 1 updates it first with warp 0 and
      // factors it there, while its other warps and the other CTAs update the rest
      const int kn = k + 1;
      const bool la = kn < nb && pr == (kn & 3) && pc == (kn & 3);
      const int sl_la = la ? (kn >> 2) * S + (kn >> 2) : -1;
      if (la && wid == 0) {
        float* T = slots + (size_t)sl_la * 1024;
        const float* li = LiT + (size_t)(kn >> 2) * 1024;
        const float* lj = LjT + (size_t)(kn >> 2) * 1024;
        trail_tile(li, lj, T, lane);
        trail_tile(li, lj, T, lane + 32);
        __syncwarp();
        factor_diag_block(T, inv, s_l, thr_of(kn), lane);
      } else {
        // 4 x 4 tiles, 64 per block; a warp's 32 consecutive tiles lie in one block
        // (uniform branches), also with warp 0 left out
        const int t0 = la ? tid - 32 : tid, nt = la ? QBT - 32 : QBT;
        for (int e = t0; e < S * S * 64; e += nt) {
          const int sl = e >> 6, t = e & 63, ia = sl / S, ib = sl % S;
          const int i = 4 * ia + pr, j = 4 * ib + pc;
          if (sl == sl_la || j <= k || j > i || i >= nb) continue;
          trail_tile(LiT + (size_t)ia * 1024, LjT + (size_t)ib * 1024, slots + (size_t)sl * 1024, t);
        }
      }
      __syncthreads();
    }
  }

  if (RM) {
    // R = G^T (n x n, column-major, FP64): the owner of lower block (bi, bj) writes
    // R(col, row) = G(row, col) for row >= col and the zero R(row, col) for row > col,
    // so every entry of R is written once; near identity: R = I + Phi(E) from the
    // FP64 Gram (strict upper part of E = G - I plus half its diagonal)
    double* R = a.R;
    for (int e = tid; e < S * S * 1024; e += QBT) {
      const int sl = e >> 10, w = e & 1023, ia = sl / S, ib = sl % S;
      const int bi = 4 * ia + pr, bj = 4 * ib + pc;
      if (bi >= nb || bj > bi) continue;
      const int r = w >> 5, c = w & 31;  // consecutive threads: consecutive columns of R
      const int row = QB * bi + r, col = QB * bj + c;
      if (row >= n || col >= n || row < col) continue;
      double v;
      if (near) {
        const double g = (double)K[row + ldk * col];
        v = row == col ? 1.0 + 0.5 * (g - 1.0) : g;
      } else {
        v = (double)(bi != bj ? slots[(size_t)sl * 1024 + qsw(r, c)] : slots[(size_t)sl * 1024 + qsw(c, r)]);
      }
      R[col + (int64_t)row * n] = v;
      if (row > col) R[row + (int64_t)col * n] = 0.0;
    }
  } else {
    // W = G, column-major rows_pad x cols_pad; a warp per column of this CTA's
    // block columns, lanes over the rows of its block rows
    float* W = a.W;
    const int nrb = rows_pad / QB;
    // (the sums are FP32: the Jacobi recomputes its norms from the columns at the start of
    // every sweep and uses these only for its negligible-column threshold; FP64 arithmetic
    // runs at 1/64 of the FP32 rate)
    for (int u = wid; u < Sc * QB; u += QBT / 32) {
      const int ib = u >> 5, c = u & 31, jb = 4 * ib + pc, col = jb * QB + c;
      float ss = 0.f;
      if (col < cols_pad) {
        for (int rb = pr; rb < nrb; rb += 4) {
          float v = 0.f;
          if (rb < nb && jb <= rb) {
            const float* blk = slot(rb >> 2, ib);
            v = rb != jb ? blk[qsw(lane, c)] : (lane >= c ? blk[qsw(c, lane)] : 0.f);
          }
          W[rb * QB + lane + (int64_t)col * rows_pad] = v;
          ss = fmaf(v, v, ss);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) colpart[u] = (double)ss;
    }
    cluster.sync();
    if (pr == 0) {
      for (int u = tid; u < Sc * QB; u += QBT) {
        const int col = (4 * (u >> 5) + pc) * QB + (u & 31);
        if (col >= cols_pad) continue;
        double t = 0.0;
        for (int q = 0; q < 4; ++q) t += *cluster.map_shared_rank(colpart + u, q * 4 + pc);
        a.colnorm2[col] = t;
        if (!isfinite(t)) report(BKFAC_ENONFINITE);
      }
    }
  }
  cluster.sync();  // keep shared memory alive until every remote read is done
}

}  // namespace

// blocked cluster Cholesky: n x n with n <= 576 (at most 9 x 9 blocks per CTA)
size_t chol_block_smem(int n) {
  const int nb = (n + CB - 1) / CB, S = (nb + 3) / 4;
  return ((size_t)S * S + 2 * (size_t)S + 1) * 256 * sizeof(double) + 32 * sizeof(double);
}

bool chol_block_ok(int n) { return n >= 32 && chol_block_smem(n) <= 200 * 1024; }

int launch_chol_block(const double* Gm, int n, double* R, double thr_rel, const double* scale, double near_tol,
                      int* near_out, double neg_rel, cudaStream_t s) {
  if (!chol_block_ok(n)) return (int)cudaErrorInvalidValue;
  static std::atomic<uint64_t> configured{0};
  if (!configured_here(configured)) {
    cudaError_t e = cudaFuncSetAttribute(chol_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(chol_block_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    mark_configured(configured);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(CBT, 1, 1);
  cfg.dynamicSmemBytes = chol_block_smem(n);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, chol_block_kernel, Gm, n, R, thr_rel, scale, near_tol, near_out, neg_rel);
  note_launches(1);
  return (int)e;
}

size_t chol_core_smem(int n, int cols_pad) {
  const int nb = (n + QB - 1) / QB, S = (nb + 3) / 4;
  const int ncb = (cols_pad + QB - 1) / QB, Sc = (ncb + 3) / 4;
  return ((size_t)S * S + 2 * (size_t)S + 1) * 1024 * sizeof(float) + 64 * sizeof(float) +
         (size_t)Sc * QB * sizeof(double);
}

bool chol_core_ok(int n, int rows_pad, int cols_pad) {
  return n >= 1 && n <= kCoreMaxN && rows_pad >= n && rows_pad % QB == 0 && cols_pad >= n &&
         chol_core_smem(n, cols_pad) <= 200 * 1024;
}

namespace {
template <typename TK, bool RM>
int launch_core_typed(const CoreCholArgs& a, cudaStream_t s) {
  static std::atomic<uint64_t> configured{0};  // attributes set once (the call can stall the host)
  if (!configured_here(configured)) {
    cudaError_t e =
        cudaFuncSetAttribute(chol_core_kernel<TK, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(chol_core_kernel<TK, RM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    mark_configured(configured);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(QBT, 1, 1);
  cfg.dynamicSmemBytes = chol_core_smem(a.n, a.cols_pad);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, chol_core_kernel<TK, RM>, a);
  note_launches(1);
  return (int)e;
}
}  // namespace

int launch_chol_core(const float* K, int ldk, int n, float* W, int rows_pad, int cols_pad, double* colnorm2,
                     float thr_rel, cudaStream_t s) {
  if (!chol_core_ok(n, rows_pad, cols_pad) || ldk < n) return (int)cudaErrorInvalidValue;
  CoreCholArgs a{};
  a.K = K;
  a.ldk = ldk;
  a.n = n;
  a.thr_rel = thr_rel;
  a.W = W;
  a.rows_pad = rows_pad;
  a.cols_pad = cols_pad;
  a.colnorm2 = colnorm2;
  return launch_core_typed<float, false>(a, s);
}

bool chol_r32_ok(int n) { return n >= 1 && chol_core_ok(n, (int)round_up(n, QB), n); }

int launch_chol_r32(const double* Gm, int n, double* R, float thr_rel, double thr_abs, const double* scale,
                    double near_tol, int* near_out, cudaStream_t s) {
  if (!chol_r32_ok(n)) return (int)cudaErrorInvalidValue;
  CoreCholArgs a{};
  a.K = Gm;
  a.ldk = n;
  a.n = n;
  a.thr_rel = thr_rel;
  a.thr_abs = thr_abs;
  a.scale = scale;
  a.R = R;
  a.rows_pad = (int)round_up(n, QB);
  a.cols_pad = n;
  a.near_tol = near_tol;
  a.near_out = near_out;
  return launch_core_typed<double, true>(a, s);
}

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
                        int* near_out, double neg_rel, cudaStream_t s) {
  if (n <= 0) return 0;
  const int C = chol_cluster_size(n);
  if (C == 0) return (int)cudaErrorInvalidValue;
  const int w = (n + C - 1) / C;
  const size_t smem = (size_t)2 * n * w * sizeof(double);
  static std::atomic<uint64_t> configured{0};  // attributes set once (the call can stall the host)
  if (!configured_here(configured)) {
    cudaError_t e = cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    mark_configured(configured);
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
  const cudaError_t e = cudaLaunchKernelEx(&cfg, chol_cluster_kernel, Gm, n, R, thr_rel, scale, near_tol, near_out, neg_rel);
  note_launches(1);
  return (int)e;
}

}  // namespace bkfac

// gemm.cu -- tiled SIMT GEMM with split-K for the tall-skinny products of the
// B-KFAC update (Algorithm 3: U^T X, U M, P R^-1, [U Q] V, Gram P^T P) and the
// two passes of the damped inverse application (Algorithm 1).
//
// One kernel template covers every operand layout the hot path needs
// (K-contiguous or M/N-contiguous operands, two concatenated K segments) with a
// fused scaling epilogue.  Long-K products with a small output use split-K:
// each split writes its partial tile, and a second kernel sums the splits in a
// fixed order (deterministic, independent of scheduling) and applies the
// epilogue (tall column-major outputs through transposing 32 x 128 tiles).
// A 128 x 128 tile kernel serves the large FP32 products; the choice of kernel
// and K splits per product shape is the autotuner's when it has timed that
// shape (tune.cu), else a heuristic sized by the SM count.  The Gram of FP32
// data for CholeskyQR is FP64-accurate on the FP32 pipe (exact products and
// TwoSum compensation, summed in FP64 across splits); an FP64-accumulating
// variant of the template serves the remaining FP32-in / FP64-out products.
// Operands rounded to BF16 on load (mixed mode) when a product does not go to
// the tensor cores.
#include <algorithm>

#include "common.cuh"

namespace bkfac {

namespace {

constexpr int BM = 64, BN = 64, BKK = 16, NT = 256;

template <typename TIn>
__device__ __forceinline__ TIn load_in(const TIn* p, bool rnd) {
  return *p;
}
template <>
__device__ __forceinline__ float load_in<float>(const float* p, bool rnd) {
  float v = __ldg(p);
  return rnd ? round_bf16(v) : v;
}
template <>
__device__ __forceinline__ double load_in<double>(const double* p, bool rnd) {
  return __ldg(p);
}

template <typename TIn, bool AK>
__device__ __forceinline__ TIn load_a(const GemmArgs& g, int m, int k, bool rnd) {
  const TIn* A;
  int64_t lda;
  if (k < g.K0) {
    A = (const TIn*)g.A0;
    lda = g.lda0;
  } else {
    A = (const TIn*)g.A1;
    lda = g.lda1;
    k -= g.K0;
  }
  return AK ? load_in<TIn>(A + (int64_t)m * lda + k, rnd) : load_in<TIn>(A + m + (int64_t)k * lda, rnd);
}

template <typename TIn, bool BKM>
__device__ __forceinline__ TIn load_b(const GemmArgs& g, int k, int n, bool rnd) {
  const TIn* B;
  int64_t ldb;
  if (k < g.K0) {
    B = (const TIn*)g.B0;
    ldb = g.ldb0;
  } else {
    B = (const TIn*)g.B1;
    ldb = g.ldb1;
    k -= g.K0;
  }
  return BKM ? load_in<TIn>(B + (int64_t)n * ldb + k, rnd) : load_in<TIn>(B + (int64_t)k * ldb + n, rnd);
}

// The epilogue computes in the accumulator's precision (FP32 for the FP32 paths:
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU).
template <typename Acc, typename TOut>
__device__ __forceinline__ void epilogue_store(const GemmArgs& g, int m, int n, Acc acc) {
  Acc v = acc * (Acc)g.alpha;
  if (g.rs) v *= (Acc)g.rs[m];
  if (g.cs) v *= (Acc)g.cs[n];
  const double beta = g.beta_dev ? *g.beta_dev : g.beta;
  const int64_t off = g.c_rowmaj ? (int64_t)m * g.ldc + n : (int64_t)m + (int64_t)n * g.ldc;
  if (g.D != nullptr && beta != 0.0) {
    const int64_t doff = g.c_rowmaj ? (int64_t)m * g.ldd + n : (int64_t)m + (int64_t)n * g.ldd;
    Acc dv = (Acc)((const TOut*)g.D)[doff];
    if (g.ds) dv *= (Acc)g.ds[n];
    v += (Acc)beta * dv;
  }
  ((TOut*)g.C)[off] = (TOut)v;
}

template <typename TIn, typename Acc, typename TOut, bool AK, bool BKM>
__global__ void __launch_bounds__(NT) gemm_kernel(const GemmArgs g) {
  __shared__ Acc As[BKK][BM + 1];
  __shared__ Acc Bs[BKK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (g.sym && blockIdx.y > blockIdx.x) return;  // symmetric product: upper tiles only
  const int K = g.K0 + g.K1;
  const int kb = blockIdx.z * g.k_chunk;
  const int ke = min(K, kb + g.k_chunk);
  const bool rnd = g.round_bf16;
  Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);

  for (int kt = kb; kt < ke; kt += BKK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + NT * q;
      int mm, kk;
      if (AK) {
        kk = e % BKK;
        mm = e / BKK;
      } else {
        mm = e % BM;
        kk = e / BM;
      }
      const int m = m0 + mm, k = kt + kk;
      As[kk][mm] = (m < g.M && k < ke) ? (Acc)load_a<TIn, AK>(g, m, k, rnd) : Acc(0);
      int nn;
      if (BKM) {
        kk = e % BKK;
        nn = e / BKK;
      } else {
        nn = e % BN;
        kk = e / BN;
      }
      const int n = n0 + nn, k2 = kt + kk;
      Bs[kk][nn] = (n < g.N && k2 < ke) ? (Acc)load_b<TIn, BKM>(g, k2, n, rnd) : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKK; ++kk) {
      Acc a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }

  if (g.splits == 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < g.M && n < g.N) {
          epilogue_store<Acc, TOut>(g, m, n, acc[i][j]);
          if (g.sym && blockIdx.y != blockIdx.x) epilogue_store<Acc, TOut>(g, n, m, acc[i][j]);
        }
      }
  } else {
    Acc* P = (Acc*)g.partial + (int64_t)blockIdx.z * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < g.M && n < g.N) P[(int64_t)m * g.N + n] = acc[i][j];
      }
  }
}

// Gram C = A^T A of an FP32 matrix with FP64-level accuracy on the FP32 pipes.
// Each product is split exactly (p = a b rounded, e = fma(a, b, -p)) and the
// rounded parts are summed with Knuth's TwoSum, whose rounding errors join the
// product errors in a compensation term: s + c carries the dot product to
// about u32^2 relative to sum |a_k b_k|.  The split partials are written as
// double (s + c) and summed in FP64 by splitk_reduce.  Upper tiles only.
// Two independent accumulators at once, on the packed FP32 instructions (each
// lane rounded to nearest; explicit instructions, so no step is contracted into
// an FMA or reassociated, which would break the error-free transformation):
// s, c, a, b hold pairs; -p is formed by flipping the two sign bits (exact).
struct Comp2 {
  uint64_t s, c;
};
__device__ __forceinline__ uint64_t f2_add(uint64_t x, uint64_t y) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t x, uint64_t y) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t x, uint64_t y) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t x, uint64_t y, uint64_t z) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(x), "l"(y), "l"(z));
  return d;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void comp_fma2(Comp2& acc, uint64_t a, uint64_t b) {
  const uint64_t p = f2_mul(a, b);
  const uint64_t e = f2_fma(a, b, p ^ 0x8000000080000000ull);
  const uint64_t t = f2_add(acc.s, p);
  const uint64_t z = f2_sub(t, acc.s);
  const uint64_t err = f2_add(f2_sub(acc.s, f2_sub(t, z)), f2_sub(p, z));
  acc.s = t;
  acc.c = f2_add(acc.c, f2_add(err, e));
}

__global__ void __launch_bounds__(NT) gram_comp_kernel(const GemmArgs g) {
  __shared__ float As[BKK][BM + 1];
  __shared__ float Bs[BKK][BN + 1];
  if (blockIdx.y > blockIdx.x) return;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int K = g.K0;
  const int kb = blockIdx.z * g.k_chunk;
  const int ke = min(K, kb + g.k_chunk);
  const float* A = (const float*)g.A0;
  // acc2[i][h] carries outputs (i, j = 2h) and (i, j = 2h + 1) as packed pairs
  Comp2 acc2[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) acc2[i][h] = Comp2{0ull, 0ull};
  for (int kt = kb; kt < ke; kt += BKK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + NT * q;
      const int kk = e % BKK, mm = e / BKK;
      const int k = kt + kk;
      As[kk][mm] = (m0 + mm < g.M && k < ke) ? __ldg(A + (int64_t)(m0 + mm) * g.lda0 + k) : 0.f;
      Bs[kk][mm] = (n0 + mm < g.N && k < ke) ? __ldg(A + (int64_t)(n0 + mm) * g.lda0 + k) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
      const uint64_t b2[2] = {f2_pack(b[0], b[1]), f2_pack(b[2], b[3])};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint64_t a2 = f2_pack(a[i], a[i]);
#pragma unroll
        for (int h = 0; h < 2; ++h) comp_fma2(acc2[i][h], a2, b2[h]);
      }
    }
    __syncthreads();
  }
  double* P = (double*)g.partial + (int64_t)blockIdx.z * g.M * g.N;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      float sv, cv, s2, c2;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(sv), "=f"(s2) : "l"(acc2[i][j >> 1].s));
      asm("mov.b64 {%0, %1}, %2;" : "=f"(cv), "=f"(c2) : "l"(acc2[i][j >> 1].c));
      if (j & 1) {
        sv = s2;
        cv = c2;
      }
      if (m < g.M && n < g.N) P[(int64_t)m * g.N + n] = (double)sv + (double)cv;
    }
}

// sums the split partials in split order, then applies the epilogue
template <typename Acc, typename TOut>
__global__ void __launch_bounds__(256) splitk_reduce(const GemmArgs g) {
  const int64_t total = (int64_t)g.M * g.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const Acc* P = (const Acc*)g.partial;
    const int m = (int)(e / g.N), n = (int)(e % g.N);
    // symmetric product: only upper tiles were computed; lower entries mirror them
    const int64_t src = (g.sym && (m / BM) > (n / BN)) ? (int64_t)n * g.N + m : e;
    Acc s = Acc(0);
    for (int z = 0; z < g.splits; ++z) s += P[(int64_t)z * total + src];
    epilogue_store<Acc, TOut>(g, m, n, s);
  }
}

// The same sum for a column-major C: 32 x 128 tiles through shared memory.  Each
// warp reads partial rows along n (four consecutive values per lane, 16-byte
// loads for FP32 when the row allows it) for every split, and C (and D) are
// written along m, both contiguous.  Same summation order as splitk_reduce.
template <typename Acc>
__device__ __forceinline__ void load4(const Acc* p, int n, int N, bool vec, Acc (&v)[4]) {
  if constexpr (sizeof(Acc) == 4) {
    if (vec && n + 4 <= N) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(p));
      v[0] = q.x;
      v[1] = q.y;
      v[2] = q.z;
      v[3] = q.w;
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = n + j < N ? p[j] : Acc(0);
}

template <typename Acc, typename TOut>
__global__ void __launch_bounds__(256) splitk_reduce_cm(const GemmArgs g) {
  __shared__ Acc t[32][129];  // [m - m0][n - n0]
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 128;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 8 warps
  const int64_t total = (int64_t)g.M * g.N;
  const Acc* P = (const Acc*)g.partial;
  const bool vec = ((reinterpret_cast<uintptr_t>(P) & 15u) == 0) && (g.N & 3) == 0;
  const int n = n0 + 4 * lane;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = w + 8 * i, m = m0 + r;
    Acc sum[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
    if (m < g.M && n < g.N) {
      const Acc* row = P + (int64_t)m * g.N + n;
      for (int z = 0; z < g.splits; ++z) {
        Acc v[4];
        load4<Acc>(row + (int64_t)z * total, n, g.N, vec, v);
#pragma unroll
        for (int j = 0; j < 4; ++j) sum[j] += v[j];
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) t[r][4 * lane + j] = sum[j];
  }
  __syncthreads();
  const int m = m0 + lane;
  for (int c = w; c < 128; c += 8) {
    const int nn = n0 + c;
    if (m < g.M && nn < g.N) epilogue_store<Acc, TOut>(g, m, nn, t[lane][c]);
  }
}

// The transposing kernel pays off for tall column-major outputs (the residual, the
// CholeskyQR solve, the rotation, the apply's T1 / T2: a million elements and more);
// small outputs (U^T X, the Gram matrices) keep more blocks in flight with the flat one.
template <typename Acc, typename TOut>
void launch_splitk_reduce(const GemmArgs& a, cudaStream_t s) {
  if (a.c_rowmaj || a.sym || (int64_t)a.M * a.N < (int64_t)256 * 1024) {
    const int64_t total = (int64_t)a.M * a.N;
    const int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 4096);
    splitk_reduce<Acc, TOut><<<blocks, 256, 0, s>>>(a);
  } else {
    dim3 grid((unsigned)ceil_div(a.N, 128), (unsigned)ceil_div(a.M, 32));
    splitk_reduce_cm<Acc, TOut><<<grid, 256, 0, s>>>(a);
  }
}

// ---------------------------------------------------------------------------
// FP32 SIMT GEMM for the large products: 128 x 128 tiles, 8 x 8 outputs per
// thread (four 4 x 4 quadrants at offsets 0 / 64 so shared-memory reads are
// 16-byte and conflict-free), 16-byte global loads, two shared-memory stages
// with the next tile prefetched into registers while the current one is used.
// Requires 16-byte aligned operands with leading dimensions a multiple of 4
// and, when an operand is K-contiguous, a first K segment that is a multiple of
// 4 (checked by the caller); edges are zero-filled.
// ---------------------------------------------------------------------------
constexpr int LBM = 128, LBN = 128, LBK = 8, LNT = 256;

template <bool AK>
__device__ __forceinline__ float4 ld_a4(const GemmArgs& g, int m, int k, int ke, bool rnd) {
  // four consecutive elements along M (M-major) or along K (K-major)
  const float* A;
  int64_t lda;
  int kk = k;
  if (k < g.K0) {
    A = (const float*)g.A0;
    lda = g.lda0;
  } else {
    A = (const float*)g.A1;
    lda = g.lda1;
    kk = k - g.K0;
  }
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (AK) {
    if (m < g.M) {
      const float* p = A + (int64_t)m * lda + kk;
      if (k + 3 < ke) {
        v = __ldg(reinterpret_cast<const float4*>(p));
      } else {
        if (k < ke) v.x = __ldg(p);
        if (k + 1 < ke) v.y = __ldg(p + 1);
        if (k + 2 < ke) v.z = __ldg(p + 2);
      }
    }
  } else {
    if (k < ke) {
      const float* p = A + m + (int64_t)kk * lda;
      if (m + 3 < g.M) {
        v = __ldg(reinterpret_cast<const float4*>(p));
      } else {
        if (m < g.M) v.x = __ldg(p);
        if (m + 1 < g.M) v.y = __ldg(p + 1);
        if (m + 2 < g.M) v.z = __ldg(p + 2);
      }
    }
  }
  if (rnd) {
    v.x = round_bf16(v.x);
    v.y = round_bf16(v.y);
    v.z = round_bf16(v.z);
    v.w = round_bf16(v.w);
  }
  return v;
}

template <bool BKM>
__device__ __forceinline__ float4 ld_b4(const GemmArgs& g, int k, int n, int ke, bool rnd) {
  const float* B;
  int64_t ldb;
  int kk = k;
  if (k < g.K0) {
    B = (const float*)g.B0;
    ldb = g.ldb0;
  } else {
    B = (const float*)g.B1;
    ldb = g.ldb1;
    kk = k - g.K0;
  }
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (BKM) {
    if (n < g.N) {
      const float* p = B + (int64_t)n * ldb + kk;
      if (k + 3 < ke) {
        v = __ldg(reinterpret_cast<const float4*>(p));
      } else {
        if (k < ke) v.x = __ldg(p);
        if (k + 1 < ke) v.y = __ldg(p + 1);
        if (k + 2 < ke) v.z = __ldg(p + 2);
      }
    }
  } else {
    if (k < ke) {
      const float* p = B + (int64_t)kk * ldb + n;
      if (n + 3 < g.N) {
        v = __ldg(reinterpret_cast<const float4*>(p));
      } else {
        if (n < g.N) v.x = __ldg(p);
        if (n + 1 < g.N) v.y = __ldg(p + 1);
        if (n + 2 < g.N) v.z = __ldg(p + 2);
      }
    }
  }
  if (rnd) {
    v.x = round_bf16(v.x);
    v.y = round_bf16(v.y);
    v.z = round_bf16(v.z);
    v.w = round_bf16(v.w);
  }
  return v;
}

// two-wide FP32 FMA (fma.rn.f32x2): d = a * b + c on packed pairs
__device__ __forceinline__ uint64_t ffma2_g(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t pack2_g(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void unpack2_g(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

template <bool AK, bool BKM>
__global__ void __launch_bounds__(LNT, 2) sgemm_large_kernel(const GemmArgs g) {
  __shared__ __align__(16) float As[2][LBK][LBM];
  __shared__ __align__(16) float Bs[2][LBK][LBN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * LBM, n0 = blockIdx.x * LBN;
  const int K = g.K0 + g.K1;
  const int kb = blockIdx.z * g.k_chunk;
  const int ke = min(K, kb + g.k_chunk);
  const bool rnd = g.round_bf16;
  // global-load coordinates of this thread's 16-byte piece of each tile
  const int am = AK ? (tid >> 1) : ((tid & 31) << 2);
  const int ak = AK ? ((tid & 1) << 2) : (tid >> 5);
  const int bn = BKM ? (tid >> 1) : ((tid & 31) << 2);
  const int bk = BKM ? ((tid & 1) << 2) : (tid >> 5);

  // With both operands M/N-contiguous (16-byte tile loads, global loads well ahead of use)
  // the accumulators are packed pairs along n, acc2[i][p] = columns 2p, 2p + 1 of row i, and
  // the inner product runs on the two-wide FMA: half the issue slots of scalar FMAs.  With a
  // K-contiguous operand the shorter loop no longer hides the next tile's global loads
  // (measured slower), so those layouts keep scalar FMAs.
  constexpr bool kPair = !AK && !BKM;
  uint64_t acc2[8][4];
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      acc2[i][p] = 0ull;  // (0.f, 0.f)
      acc[i][2 * p] = acc[i][2 * p + 1] = 0.f;
    }

  auto store_tile = [&](int buf, const float4& va, const float4& vb) {
    if (AK) {
      As[buf][ak + 0][am] = va.x;
      As[buf][ak + 1][am] = va.y;
      As[buf][ak + 2][am] = va.z;
      As[buf][ak + 3][am] = va.w;
    } else {
      *reinterpret_cast<float4*>(&As[buf][ak][am]) = va;
    }
    if (BKM) {
      Bs[buf][bk + 0][bn] = vb.x;
      Bs[buf][bk + 1][bn] = vb.y;
      Bs[buf][bk + 2][bn] = vb.z;
      Bs[buf][bk + 3][bn] = vb.w;
    } else {
      *reinterpret_cast<float4*>(&Bs[buf][bk][bn]) = vb;
    }
  };

  int buf = 0;
  if (kb < ke) {
    const float4 va = ld_a4<AK>(g, m0 + am, kb + ak, ke, rnd);
    const float4 vb = ld_b4<BKM>(g, kb + bk, n0 + bn, ke, rnd);
    store_tile(0, va, vb);
  }
  __syncthreads();
  for (int kt = kb; kt < ke; kt += LBK) {
    const bool more = kt + LBK < ke;
    float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na;
    if (more) {
      na = ld_a4<AK>(g, m0 + am, kt + LBK + ak, ke, rnd);
      nb = ld_b4<BKM>(g, kt + LBK + bk, n0 + bn, ke, rnd);
    }
#pragma unroll
    for (int kk = 0; kk < LBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      if constexpr (kPair) {
        const uint64_t b2[4] = {pack2_g(b0.x, b0.y), pack2_g(b0.z, b0.w), pack2_g(b1.x, b1.y),
                                pack2_g(b1.z, b1.w)};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint64_t ai = pack2_g(a[i], a[i]);
#pragma unroll
          for (int p = 0; p < 4; ++p) acc2[i][p] = ffma2_g(ai, b2[p], acc2[i][p]);
        }
      } else {
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
    }
    if (more) store_tile(buf ^ 1, na, nb);
    __syncthreads();
    buf ^= 1;
  }

  if constexpr (kPair) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int p = 0; p < 4; ++p) unpack2_g(acc2[i][p], acc[i][2 * p], acc[i][2 * p + 1]);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (m < g.M && n < g.N) {
        if (g.splits == 1)
          epilogue_store<float, float>(g, m, n, acc[i][j]);
        else
          ((float*)g.partial)[(int64_t)blockIdx.z * g.M * g.N + (int64_t)m * g.N + n] = acc[i][j];
      }
    }
  }
}

// operand layouts and alignment the 128 x 128 kernel accepts
bool large_layout_ok(const GemmArgs& g) {
  auto al = [](const void* p) { return p == nullptr || ((uintptr_t)p % 16) == 0; };
  if (g.sym) return false;
  // a 4-wide load along K must stay inside one K segment and 16-byte aligned: the
  // seam K0 a multiple of 4 when either operand is K-contiguous (M- and N-contiguous
  // operands load one K index at a time)
  if (g.K1 > 0 && (g.a_kmaj || g.b_kmaj) && g.K0 % 4 != 0) return false;
  if (!al(g.A0) || !al(g.A1) || !al(g.B0) || !al(g.B1)) return false;
  if (g.lda0 % 4 || g.ldb0 % 4 || (g.K1 > 0 && (g.lda1 % 4 || g.ldb1 % 4))) return false;
  return true;
}

bool large_ok(const GemmArgs& g) {
  if ((int64_t)g.M * g.N < 128 * 128 * 8) return false;  // small outputs: the 64 x 64 kernel
  return large_layout_ok(g);
}

int run_large_f32(const GemmArgs& g, cudaStream_t s) {
  const int K = g.K0 + g.K1;
  GemmArgs a = g;
  if (a.splits < 1) a.splits = 1;
  if (a.splits > 1 && K > 0) {
    a.k_chunk = (int)round_up(ceil_div(K, a.splits), 16);
    a.splits = (int)ceil_div(K, a.k_chunk);
  } else {
    a.splits = 1;
    a.k_chunk = (int)round_up(std::max(K, 1), 16);
  }
  dim3 grid((unsigned)ceil_div(a.N, LBN), (unsigned)ceil_div(a.M, LBM), (unsigned)a.splits);
  if (a.a_kmaj && a.b_kmaj)
    sgemm_large_kernel<true, true><<<grid, LNT, 0, s>>>(a);
  else if (a.a_kmaj && !a.b_kmaj)
    sgemm_large_kernel<true, false><<<grid, LNT, 0, s>>>(a);
  else if (!a.a_kmaj && a.b_kmaj)
    sgemm_large_kernel<false, true><<<grid, LNT, 0, s>>>(a);
  else
    sgemm_large_kernel<false, false><<<grid, LNT, 0, s>>>(a);
  note_launches(1);
  if (a.splits > 1) {
    launch_splitk_reduce<float, float>(a, s);
    note_launches(1);
  }
  return (int)cudaGetLastError();
}

template <typename TIn, typename Acc, typename TOut>
int run_typed(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return (int)cudaSuccess;
  const int K = g.K0 + g.K1;
  GemmArgs a = g;
  if (a.splits < 1) a.splits = 1;
  if (a.splits > 1 && K > 0) {
    a.k_chunk = (int)round_up(ceil_div(K, a.splits), BKK);
    a.splits = (int)ceil_div(K, a.k_chunk);
  } else {
    a.splits = 1;
    a.k_chunk = (int)round_up(std::max(K, 1), BKK);
  }
  dim3 grid((unsigned)ceil_div(a.N, BN), (unsigned)ceil_div(a.M, BM), (unsigned)a.splits);
  if (a.a_kmaj && a.b_kmaj)
    gemm_kernel<TIn, Acc, TOut, true, true><<<grid, NT, 0, s>>>(a);
  else if (a.a_kmaj && !a.b_kmaj)
    gemm_kernel<TIn, Acc, TOut, true, false><<<grid, NT, 0, s>>>(a);
  else if (!a.a_kmaj && a.b_kmaj)
    gemm_kernel<TIn, Acc, TOut, false, true><<<grid, NT, 0, s>>>(a);
  else
    gemm_kernel<TIn, Acc, TOut, false, false><<<grid, NT, 0, s>>>(a);
  note_launches(1);
  if (a.splits > 1) {
    launch_splitk_reduce<Acc, TOut>(a, s);
    note_launches(1);
  }
  return (int)cudaGetLastError();
}

}  // namespace

int gemm_pick_splits(int M, int N, int K, int /*sm_count*/) {
  // a fixed CTA target keeps workspace sizes independent of the device
  const int64_t tiles = ceil_div(M, BM) * ceil_div(N, BN);
  const int64_t target = 2 * sm_count();
  int64_t s = std::max<int64_t>(1, target / std::max<int64_t>(tiles, 1));
  s = std::min<int64_t>(s, std::max<int64_t>(1, K / 256));
  s = std::min<int64_t>(s, 32);
  return (int)s;
}

int gram_run_comp(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0) return (int)cudaSuccess;
  GemmArgs a = g;
  const int K = a.K0;
  a.sym = true;
  a.splits = std::max(a.splits, 1);
  a.k_chunk = (int)round_up(std::max<int64_t>(ceil_div(std::max(K, 1), a.splits), 1), BKK);
  a.splits = (int)std::max<int64_t>(1, ceil_div(std::max(K, 1), a.k_chunk));
  dim3 grid((unsigned)ceil_div(a.N, BN), (unsigned)ceil_div(a.M, BM), (unsigned)a.splits);
  gram_comp_kernel<<<grid, NT, 0, s>>>(a);
  launch_splitk_reduce<double, double>(a, s);
  note_launches(2);
  return (int)cudaGetLastError();
}

int splitk_reduce_f32(const GemmArgs& g, cudaStream_t s) {
  launch_splitk_reduce<float, float>(g, s);
  note_launches(1);
  return (int)cudaGetLastError();
}

int64_t partial_room(const GemmArgs& g) {
  return g.partial ? (int64_t)(g.partial_bytes / ((size_t)std::max(g.M, 1) * std::max(g.N, 1) * sizeof(float))) : 0;
}

bool gemm_choice_ok(const GemmArgs& g, GemmPick pick) {
  if (g.sym || g.round_bf16 || g.tf32x3) return false;
  if (pick.splits < 1 || (pick.splits > 1 && pick.splits > partial_room(g))) return false;
  if (pick.kernel == GEMM_LARGE) return large_layout_ok(g);
  return pick.kernel == GEMM_SMALL;
}

int gemm_run_choice(const GemmArgs& g, GemmPick pick, cudaStream_t s) {
  if (!gemm_choice_ok(g, pick)) return BKFAC_EINVAL;
  GemmArgs a = g;
  a.splits = pick.splits;
  return pick.kernel == GEMM_LARGE ? run_large_f32(a, s) : run_typed<float, float, float>(a, s);
}

int gemm_run(const GemmArgs& g, DType in_t, DType acc_t, DType out_t, cudaStream_t s) {
  if (in_t == DT_F64 && acc_t == DT_F64 && out_t == DT_F64) return run_typed<double, double, double>(g, s);
  // mixed precision (BF16 operands, FP32 accumulation): the tensor cores
  if (in_t == DT_F32 && acc_t == DT_F32 && out_t == DT_F32 && (g.round_bf16 || g.tf32x3) && !g.sym &&
      tc_gemm_enabled())
    return tc_gemm_run(g, s);
  if (in_t == DT_F32 && acc_t == DT_F32 && out_t == DT_F32) {
    if (g.M <= 0 || g.N <= 0) return (int)cudaSuccess;
    gemm_note_shape(g, partial_room(g));
    // a tuned choice for this shape, when it fits this call
    GemmPick pick;
    if (!g.sym && gemm_pick_lookup(g, &pick) && gemm_choice_ok(g, pick)) return gemm_run_choice(g, pick, s);
    if (large_ok(g)) {
      // enough CTAs for the GPU: split K when the output has few 128 x 128 tiles
      GemmArgs a = g;
      const int64_t tiles = ceil_div(g.M, LBM) * ceil_div(g.N, LBN);
      const int64_t room = a.partial ? (int64_t)(a.partial_bytes / ((size_t)g.M * g.N * sizeof(float))) : 0;
      if (a.splits <= 1 && tiles < sm_count() && room >= 2)
        a.splits = (int)std::min<int64_t>(std::min<int64_t>(4, 2 * sm_count() / tiles), room);
      if (a.splits > 1 && room < a.splits) a.splits = (int)std::max<int64_t>(1, room);
      return run_large_f32(a, s);
    }
    // a small output over a long K (U^T X, U_G^T T1 at r = n = 256, K = d): the 128 x 128
    // kernel split along K into enough pieces to fill the GPU, when the partial buffer
    // holds them
    const int K = g.K0 + g.K1;
    if ((int64_t)g.M * g.N >= 128 * 128 * 2 && K >= 2048 && g.partial && large_layout_ok(g)) {
      const int64_t tiles = ceil_div(g.M, LBM) * ceil_div(g.N, LBN);
      const int64_t room = (int64_t)(g.partial_bytes / ((size_t)g.M * g.N * sizeof(float)));
      const int64_t sp = std::min<int64_t>(std::min<int64_t>(room, 32),
                                           std::min<int64_t>(K / 128, ceil_div(2 * sm_count(), tiles)));
      if (sp >= 8) {
        GemmArgs a = g;
        a.splits = (int)sp;
        return run_large_f32(a, s);
      }
    }
    return run_typed<float, float, float>(g, s);
  }
  if (in_t == DT_F32 && acc_t == DT_F64 && out_t == DT_F64) return run_typed<float, double, double>(g, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace bkfac

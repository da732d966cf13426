// gemm.cu -- tiled SIMT GEMM with split-K for the tall-skinny products of the
// B-KFAC update (Algorithm 3: U^T X, U M, P R^-1, [U Q] V, Gram P^T P) and the
// two passes of the damped inverse application (Algorithm 1).
//
// One kernel template covers every operand layout the hot path needs
// (K-contiguous or M/N-contiguous operands, two concatenated K segments) with a
// fused scaling epilogue.  Long-K products with a small output use split-K:
// each split writes its partial tile, and a second kernel sums the splits in a
// fixed order (deterministic, independent of scheduling) and applies the
// epilogue.  In FP32 mode the Gram takes FP32 operands and accumulates in
// FP64 (products of two floats are exact in double).  In mixed mode the
// operands are rounded to BF16 on load and accumulate in FP32.
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

template <typename Acc, typename TOut>
__device__ __forceinline__ void epilogue_store(const GemmArgs& g, int m, int n, Acc acc) {
  double v = (double)acc * g.alpha;
  if (g.rs) v *= g.rs[m];
  if (g.cs) v *= g.cs[n];
  double beta = g.beta_dev ? *g.beta_dev : g.beta;
  int64_t off = g.c_rowmaj ? (int64_t)m * g.ldc + n : (int64_t)m + (int64_t)n * g.ldc;
  if (g.D != nullptr && beta != 0.0) {
    int64_t doff = g.c_rowmaj ? (int64_t)m * g.ldd + n : (int64_t)m + (int64_t)n * g.ldd;
    double dv = (double)((const TOut*)g.D)[doff];
    if (g.ds) dv *= g.ds[n];
    v += beta * dv;
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
        if (m < g.M && n < g.N) epilogue_store<Acc, TOut>(g, m, n, acc[i][j]);
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

// sums the split partials in split order, then applies the epilogue
template <typename Acc, typename TOut>
__global__ void __launch_bounds__(256) splitk_reduce(const GemmArgs g) {
  const int64_t total = (int64_t)g.M * g.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const Acc* P = (const Acc*)g.partial;
    Acc s = Acc(0);
    for (int z = 0; z < g.splits; ++z) s += P[(int64_t)z * total + e];
    const int m = (int)(e / g.N), n = (int)(e % g.N);
    epilogue_store<Acc, TOut>(g, m, n, s);
  }
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
    int64_t total = (int64_t)a.M * a.N;
    int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 4096);
    splitk_reduce<Acc, TOut><<<blocks, 256, 0, s>>>(a);
    note_launches(1);
  }
  return (int)cudaGetLastError();
}

}  // namespace

int gemm_pick_splits(int M, int N, int K, int /*sm_count*/) {
  // a fixed CTA target keeps workspace sizes independent of the device
  const int64_t tiles = ceil_div(M, BM) * ceil_div(N, BN);
  const int64_t target = 2 * 152;
  int64_t s = std::max<int64_t>(1, target / std::max<int64_t>(tiles, 1));
  s = std::min<int64_t>(s, std::max<int64_t>(1, K / 256));
  s = std::min<int64_t>(s, 32);
  return (int)s;
}

int gemm_run(const GemmArgs& g, DType in_t, DType acc_t, DType out_t, cudaStream_t s) {
  if (in_t == DT_F64 && acc_t == DT_F64 && out_t == DT_F64) return run_typed<double, double, double>(g, s);
  if (in_t == DT_F32 && acc_t == DT_F32 && out_t == DT_F32) return run_typed<float, float, float>(g, s);
  if (in_t == DT_F32 && acc_t == DT_F64 && out_t == DT_F64) return run_typed<float, double, double>(g, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace bkfac

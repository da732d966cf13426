// tma_gemm.cu -- the damped inverse application of the mixed-precision path on
// the 5th-generation tensor cores with operands fed by the Tensor Memory
// Accelerator (TMA).
//
// The apply (Algorithm 1) in two passes over the gradient G (d_out x d_in):
//   pass 1  T1 = G U_A,  T2 = diag(c) U_G^T G,
//   pass 2  S = alpha G + [W1 | U_G] [U_A | T2]^T
// In mixed mode every operand of these products is rounded to BF16 (round to
// nearest even) with FP32 accumulation.  Instead of rounding while staging each
// tile on the CUDA cores, the operands are rounded once, in one pass each, into
// BF16 copies laid out K-major (the contraction index contiguous): G and its
// transpose (from one read of G), the bases U_A, U_G, and the concatenated
// thin operands of pass 2.  The products then run as one kernel shape,
// C[m, n] = sum_k A[m, k] B[n, k] with A, B BF16 K-major:
//
//   * one warp issues TMA tile loads (cp.async.bulk.tensor.2d, a 64 x 128 box of
//     BF16 = 128-byte rows, 128-byte swizzle) of A and B into a three-stage ring
//     in shared memory, each stage completing on its "full" mbarrier;
//   * one thread issues the tcgen05.mma (kind::f16, M = N = 128, K = 16, four
//     per stage) with shared-memory descriptors of the swizzled K-major layout,
//     and frees each stage by tcgen05.commit to its "empty" mbarrier;
//   * four warps read the FP32 accumulator back from tensor memory
//     (tcgen05.ld 32x32b, one TMEM lane quadrant per warp) into a shared tile,
//     then apply the epilogue alpha rs[m] cs[n] acc + beta ds[n] D(m, n) and
//     write C row- or column-major with coalesced accesses, or split-K partials
//     (row-major M x N per split) for splitk_reduce_f32.
//
// Every wait is bounded: a stage or accumulator that never completes records
// BKFAC_ETIMEOUT and the kernel returns.  The TMA coordinates along K are
// multiples of 64 elements (128 bytes); rows may start anywhere; the tensor
// maps bound each operand to its true extent, so edges read as zero.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace bkfac {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;       // output tile, K per stage (128 bytes of BF16 per row)
constexpr int NSTAGE = 3;
constexpr int TILE_BYTES = BM * BK * 2;          // 16 KB per operand tile
constexpr int STAGE_BYTES = 2 * TILE_BYTES;      // A + B
constexpr int THREADS = 192;                     // warp 0: TMA, warp 1: MMA, warps 2-5: epilogue
constexpr int OLD = BN + 1;                      // leading dimension of the staged output tile (floats)
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;  // + alignment slack
constexpr int TMEM_COLS = 128;
static_assert(BM * OLD * 4 <= NSTAGE * STAGE_BYTES, "the output tile reuses the stage buffers");

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(sa(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sa(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (about a second of SM clock cycles); false on time-out
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
  const long long t0 = clock64();
  while (!bar_try(b, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

// 2-D TMA tile load: box at (x = K index, y = row) of the tensor map into shared
// memory, completing `bytes` on the mbarrier
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          sa(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sa(b))
      : "memory");
}

// shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled
// layout: start address, leading byte offset 16 (unused by this layout), stride
// byte offset 1024 (eight 128-byte rows), descriptor version 1, layout 2 = 128B
// swizzle.  Advancing the start address by 32 bytes selects the next K = 16 slice
// of a 64-wide stage (the swizzle is a function of the address bits).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

// instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tfence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tfence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tcommit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(b))
               : "memory");
}
__device__ __forceinline__ void tld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// C[m, n] = sum_k A[m, k] B[n, k] over this CTA's K chunk, epilogue as in GemmArgs
__global__ void __launch_bounds__(THREADS, 2) tma_gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                              const __grid_constant__ CUtensorMap tb,
                                                              const GemmArgs g, int K) {
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], accum;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  // stages on a 1024-byte boundary (the 128-byte swizzle repeats every 8 rows of 128 bytes)
  unsigned char* sm = raw + ((1024u - (sa(raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * g.k_chunk;
  const int ke = min(K, kb + g.k_chunk);
  const int nk = ke > kb ? (ke - kb + BK - 1) / BK : 0;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    bar_init(&accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tfence_before();
  __syncthreads();
  tfence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
      for (int it = 0; it < nk; ++it) {
        const int s = it % NSTAGE;
        // the stage's previous MMAs (round it / NSTAGE - 1) have released it
        if (it >= NSTAGE && !bar_wait(&empty[s], (uint32_t)((it / NSTAGE - 1) & 1))) {
          s_fail = 1;
          break;
        }
        unsigned char* st = sm + s * STAGE_BYTES;
        bar_expect_tx(&full[s], STAGE_BYTES);
        const int k = kb + it * BK;  // a multiple of 64: 128-byte aligned inner coordinate
        tma_load(st, &ta, k, m0, &full[s]);
        tma_load(st + TILE_BYTES, &tb, k, n0, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      for (int it = 0; it < nk; ++it) {
        const int s = it % NSTAGE;
        if (!bar_wait(&full[s], (uint32_t)((it / NSTAGE) & 1))) {
          s_fail = 1;
          break;
        }
        tfence_after();
        const uint32_t a0 = sa(sm + s * STAGE_BYTES), b0 = a0 + TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          tmma(tmem, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), idesc, (it > 0 || kk > 0) ? 1u : 0u);
        tcommit(&empty[s]);  // the stage is free once these MMAs have read it
      }
      tcommit(&accum);  // arrives when every MMA issued above has completed
    }
  } else {
    // epilogue warps: TMEM lane quadrant warp mod 4 = output rows 32 q .. 32 q + 31
    const bool done = bar_wait(&accum, 0u);
    tfence_after();
    float* T = reinterpret_cast<float*>(sm);  // every TMA load landed and every MMA read it
    const int q = warp & 3, row = q * 32 + lane;
    if (done && nk > 0) {
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) T[row * OLD + c0 + i] = v[i];
      }
    } else {
      for (int c0 = 0; c0 < BN; ++c0) T[row * OLD + c0] = 0.f;
      if (!done) s_fail = 1;
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps
    const int ew = warp - 2;                        // 0..3
    const bool split = g.splits > 1;
    const float alpha = (float)g.alpha;
    const float beta = (float)(g.beta_dev ? *g.beta_dev : g.beta);
    const bool with_d = !split && g.D != nullptr && beta != 0.f;
    if (!s_fail) {
      if (g.c_rowmaj || split) {
        // rows leave whole: lane l owns columns 4 l .. 4 l + 3 of the tile (16-byte
        // accesses), and each warp keeps the D rows of eight output rows in flight
        float* out = split ? (float*)g.partial + (int64_t)blockIdx.z * g.M * g.N : (float*)g.C;
        const int64_t ldo = split ? g.N : g.ldc;
        const int n = n0 + 4 * lane;
        const bool full = n + 4 <= g.N;
        const bool vec_o = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) && (ldo & 3) == 0;
        const bool vec_d = with_d && ((reinterpret_cast<uintptr_t>(g.D) & 15u) == 0) && (g.ldd & 3) == 0;
        float csv[4], dsv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = n + j < g.N;
          csv[j] = (!split && g.cs && in) ? (float)g.cs[n + j] : 1.f;
          dsv[j] = (g.ds && in) ? (float)g.ds[n + j] : 1.f;
        }
        constexpr int RB = 8;
        for (int r0 = ew; r0 < BM; r0 += 4 * RB) {
          float4 dq[RB];
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            const int m = m0 + r0 + 4 * u;
            dq[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (with_d && m < g.M && n < g.N) {
              const float* drow = (const float*)g.D + (int64_t)m * g.ldd + n;
              if (full && vec_d) {
                dq[u] = __ldg(reinterpret_cast<const float4*>(drow));
              } else {
                dq[u].x = drow[0];
                if (n + 1 < g.N) dq[u].y = drow[1];
                if (n + 2 < g.N) dq[u].z = drow[2];
                if (n + 3 < g.N) dq[u].w = drow[3];
              }
            }
          }
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            const int r = r0 + 4 * u, m = m0 + r;
            if (m >= g.M || n >= g.N) continue;
            const float rsm = (!split && g.rs) ? (float)g.rs[m] : 1.f;
            const float dv[4] = {dq[u].x, dq[u].y, dq[u].z, dq[u].w};
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              o[j] = T[r * OLD + 4 * lane + j];
              if (!split) o[j] *= alpha * rsm * csv[j];
              if (with_d) o[j] += beta * dv[j] * dsv[j];
            }
            float* orow = out + (int64_t)m * ldo + n;
            if (full && vec_o) {
              *reinterpret_cast<float4*>(orow) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (n + j < g.N) orow[j] = o[j];
            }
          }
        }
      } else {
        for (int rb = 0; rb < BM; rb += 32) {
          const int r = rb + lane, m = m0 + r;
          const float rsm = (g.rs && m < g.M) ? (float)g.rs[m] : 1.f;
          for (int c = ew; c < BN; c += 4) {
            const int n = n0 + c;
            if (m >= g.M || n >= g.N) continue;
            float o = T[r * OLD + c] * alpha * rsm;
            if (g.cs) o *= (float)g.cs[n];
            if (with_d) {
              float dv = ((const float*)g.D)[m + (int64_t)n * g.ldd];
              if (g.ds) dv *= (float)g.ds[n];
              o += beta * dv;
            }
            ((float*)g.C)[m + (int64_t)n * g.ldc] = o;
          }
        }
      }
    } else if (ew == 0 && lane == 0) {
      report(BKFAC_ETIMEOUT);
    }
  }
  tfence_before();
  __syncthreads();
  if (warp == 1) {
    tfence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---- BF16 operand preparation (round to nearest even) -----------------------

// G (R x C row-major, ld ldg) -> Gb (R x C, ld ldb) and its transpose Gt (C x R,
// ld ldt): one read of G, 64 x 64 tiles through shared memory
__global__ void __launch_bounds__(256) cvt_both_kernel(const float* __restrict__ G, int64_t ldg, int R, int C,
                                                       __nv_bfloat16* __restrict__ Gb, int64_t ldb,
                                                       __nv_bfloat16* __restrict__ Gt, int64_t ldt) {
  __shared__ __nv_bfloat16 t[64][66];
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
  for (int y = ty; y < 64; y += 4) {
    const int r = r0 + y, c = c0 + tx;
    __nv_bfloat16 v = __float2bfloat16_rn(0.f);
    if (r < R && c < C) {
      v = __float2bfloat16_rn(__ldg(G + (int64_t)r * ldg + c));
      Gb[(int64_t)r * ldb + c] = v;
    }
    t[y][tx] = v;
  }
  __syncthreads();
  for (int y = ty; y < 64; y += 4) {
    const int c = c0 + y, r = r0 + tx;
    if (c < C && r < R) Gt[(int64_t)c * ldt + r] = t[tx][y];
  }
}

// k columns of length d (column-major, ld) -> the same layout in BF16 (ld ldo)
__global__ void __launch_bounds__(256) cvt_cols_kernel(const float* __restrict__ X, int64_t ld, int d, int k,
                                                       __nv_bfloat16* __restrict__ Y, int64_t ldo) {
  const int64_t total = (int64_t)d * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / d), i = (int)(e % d);
    Y[(int64_t)j * ldo + i] = __float2bfloat16_rn(__ldg(X + i + (int64_t)j * ld));
  }
}

// [X0 | X1] (dim x (k0 + k1), each column-major) -> Y (dim x (k0 + k1) row-major,
// ld ldy): Y[i][k] = k < k0 ? X0[i + k ld0] : X1[i + (k - k0) ld1]; 64 x 64 tiles
__global__ void __launch_bounds__(256) cvt_cat_t_kernel(const float* __restrict__ X0, int64_t ld0, int k0,
                                                        const float* __restrict__ X1, int64_t ld1, int k1, int dim,
                                                        __nv_bfloat16* __restrict__ Y, int64_t ldy) {
  __shared__ __nv_bfloat16 t[64][66];
  const int i0 = blockIdx.x * 64, kc0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int kt = k0 + k1;
  for (int y = ty; y < 64; y += 4) {  // y: column (K index) of the source, tx: row
    const int k = kc0 + y, i = i0 + tx;
    float v = 0.f;
    if (i < dim && k < kt) v = k < k0 ? __ldg(X0 + i + (int64_t)k * ld0) : __ldg(X1 + i + (int64_t)(k - k0) * ld1);
    t[y][tx] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  for (int y = ty; y < 64; y += 4) {  // y: row i of Y, tx: K index
    const int i = i0 + y, k = kc0 + tx;
    if (i < dim && k < kt) Y[(int64_t)i * ldy + k] = t[tx][y];
  }
}

// ---- tensor maps ----------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// BF16 K-major operand: `rows` rows of `k` elements, row pitch ld elements (ld a
// multiple of 8: 16-byte pitch), box 64 (K) x 128 (rows), 128-byte swizzle
bool encode_kmajor(CUtensorMap* map, const void* base, int rows, int k, int64_t ld) {
  const auto fn = encode_fn();
  if (!fn || rows < 1 || k < 1 || (ld % 8) != 0 || ((uintptr_t)base % 16) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tma_gemm_available() { return encode_fn() != nullptr; }

int64_t bf16_ld(int k) { return round_up(std::max(k, 1), 8); }

// C (M x N) = alpha sum_k A[m, k] B[n, k] (+ epilogue of g), A: M x K, B: N x K, both
// BF16 K-major with row pitches lda / ldb (multiples of 8 elements).  g supplies M,
// N, C, ldc, c_rowmaj, alpha, beta / beta_dev, rs, cs, ds, D, ldd, and partial /
// partial_bytes for split K (chosen here: about two CTAs per SM).
int tma_gemm_run(const void* A, int64_t lda, const void* B, int64_t ldb, int K, const GemmArgs& g0, cudaStream_t s) {
  GemmArgs g = g0;
  if (g.M <= 0 || g.N <= 0) return (int)cudaSuccess;
  CUtensorMap ta, tb;
  if (!encode_kmajor(&ta, A, g.M, std::max(K, 1), lda) || !encode_kmajor(&tb, B, g.N, std::max(K, 1), ldb))
    return (int)cudaErrorInvalidValue;
  const int64_t tiles = ceil_div(g.M, BM) * ceil_div(g.N, BN);
  int64_t splits = 1;
  if (g.partial != nullptr && tiles < 2 * sm_count() && K > 4 * BK) {
    const int64_t room = (int64_t)(g.partial_bytes / ((size_t)g.M * g.N * sizeof(float)));
    splits = std::min<int64_t>(std::min<int64_t>(ceil_div(2 * sm_count(), tiles), (int64_t)K / (2 * BK)), room);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, 32));
  }
  g.k_chunk = (int)round_up(ceil_div(std::max(K, 1), splits), BK);
  g.splits = (int)std::max<int64_t>(1, ceil_div(std::max(K, 1), g.k_chunk));
  static std::atomic<uint64_t> configured{0};
  if (!configured_here(configured)) {
    const cudaError_t e = cudaFuncSetAttribute(tma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return (int)e;
    mark_configured(configured);
  }
  dim3 grid((unsigned)ceil_div(g.N, BN), (unsigned)ceil_div(g.M, BM), (unsigned)g.splits);
  tma_gemm_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(ta, tb, g, K);
  note_launches(1);
  if (g.splits > 1) return splitk_reduce_f32(g, s);
  return (int)cudaGetLastError();
}

int launch_cvt_both(const float* G, int64_t ldg, int R, int C, void* Gb, int64_t ldb, void* Gt, int64_t ldt,
                    cudaStream_t s) {
  if (R <= 0 || C <= 0) return 0;
  dim3 grid((unsigned)ceil_div(C, 64), (unsigned)ceil_div(R, 64));
  cvt_both_kernel<<<grid, 256, 0, s>>>(G, ldg, R, C, (__nv_bfloat16*)Gb, ldb, (__nv_bfloat16*)Gt, ldt);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_cvt_cols(const float* X, int64_t ld, int d, int k, void* Y, int64_t ldo, cudaStream_t s) {
  if (d <= 0 || k <= 0) return 0;
  const int64_t total = (int64_t)d * k;
  const int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 8 * sm_count());
  cvt_cols_kernel<<<blocks, 256, 0, s>>>(X, ld, d, k, (__nv_bfloat16*)Y, ldo);
  note_launches(1);
  return (int)cudaGetLastError();
}

int launch_cvt_cat_t(const float* X0, int64_t ld0, int k0, const float* X1, int64_t ld1, int k1, int dim, void* Y,
                     int64_t ldy, cudaStream_t s) {
  if (dim <= 0 || k0 + k1 <= 0) return 0;
  dim3 grid((unsigned)ceil_div(dim, 64), (unsigned)ceil_div(k0 + k1, 64));
  cvt_cat_t_kernel<<<grid, 256, 0, s>>>(X0, ld0, k0, X1, ld1, k1, dim, (__nv_bfloat16*)Y, ldy);
  note_launches(1);
  return (int)cudaGetLastError();
}

}  // namespace bkfac

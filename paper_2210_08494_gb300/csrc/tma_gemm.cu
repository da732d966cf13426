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
//     BF16 = 128-byte rows, 128-byte swizzle) of A and B into a ring of stages
//     in shared memory, each stage completing on its "full" mbarrier;
//   * one thread issues the tcgen05.mma (kind::f16, M = N = 128, K = 16, four
//     per stage) with shared-memory descriptors of the swizzled K-major layout,
//     and frees each stage by tcgen05.commit to its "empty" mbarrier;
//   * eight warps read the FP32 accumulator back from tensor memory
//     (tcgen05.ld 32x32b; a TMEM lane quadrant and half the columns per warp)
//     and run the epilogue alpha rs[m] cs[n] acc + beta ds[n] D(m, n): through
//     a shared tile of its own, C leaves row- or column-major with coalesced
//     accesses (sixteen rows of D in flight per warp); split-K partials
//     (row-major M x N per split, for splitk_reduce_f32) leave straight from
//     TMEM.
//
// The kernel is persistent (one CTA per SM walks the output tiles and K splits)
// with two accumulators in TMEM: the MMAs of the next tile run while the
// epilogue warps write the previous one out.

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
constexpr int TILE_BYTES = BM * BK * 2;          // 16 KB per operand tile
constexpr int STAGE_BYTES = 2 * TILE_BYTES;      // A + B
constexpr int NEPI = 8;                          // epilogue warps
constexpr int THREADS = 64 + 32 * NEPI;          // warp 0: TMA, warp 1: MMA, warps 2-9: epilogue
constexpr int OLD = BN + 4;                      // row pitch of the staged output tile (floats, 16-byte rows)
constexpr int TMEM_COLS = 2 * BN;                // two accumulators

// Epilogue modes.
//   EPI_PARTIAL  split-K partials, each thread's accumulator row straight from TMEM
//                (whole 32-byte sectors); six operand stages.
//   EPI_STAGED   the accumulator through a shared tile, C written row- or column-
//                major by coalesced 16-byte (or 4-byte) accesses; four stages.
// (Measured on the wide layer's pass 2, 1056 tiles of K = 512: a six-stage ring
// does not beat four, and row-major stores straight from TMEM rows cost more than
// the staged tile saves in shared memory; the short-K product is bound by its
// operand traffic from L2, about 256 KB per output tile.)
enum { EPI_PARTIAL = 0, EPI_STAGED = 1 };
template <int MODE>
struct Cfg {
  static constexpr int NSTAGE = MODE == EPI_STAGED ? 4 : 6;
  static constexpr int EXTRA = MODE == EPI_STAGED ? BM * OLD * 4 : 0;
  static constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + EXTRA + 1024;  // + alignment slack
  static_assert(SMEM_BYTES <= 227 * 1024 - 512, "shared memory per CTA");
};
static_assert(BM % NEPI == 0 && NEPI % 4 == 0, "epilogue warps cover the TMEM lane quadrants evenly");

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

// Work unit u of a launch: output tile (tx, ty) of split z, tx fastest (units that
// run at the same time share their rows of A)
struct Unit {
  int m0, n0, z, kb, nk;
};
__device__ __forceinline__ Unit unit_of(int u, const GemmArgs& g, int K, int tiles_n, int tiles_mn) {
  Unit w;
  w.z = u / tiles_mn;
  const int rem = u - w.z * tiles_mn;
  w.m0 = (rem / tiles_n) * BM;
  w.n0 = (rem % tiles_n) * BN;
  w.kb = w.z * g.k_chunk;
  const int ke = min(K, w.kb + g.k_chunk);
  w.nk = ke > w.kb ? (ke - w.kb + BK - 1) / BK : 0;
  return w;
}

// the NEPI epilogue warps (named barrier 1)
__device__ __forceinline__ void epi_sync() { asm volatile("barrier.sync 1, %0;" ::"n"(NEPI * 32) : "memory"); }
// the same barrier, returning whether any epilogue thread passed `bad` (one
// verdict for all of them, so that they leave their loops together)
__device__ __forceinline__ bool epi_any(bool bad) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, p;\n\tsetp.ne.u32 q, %1, 0;\n\tbarrier.red.or.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)bad), "n"(NEPI * 32)
      : "memory");
  return r != 0;
}

// C[m, n] = sum_k A[m, k] B[n, k] per work unit, epilogue as in GemmArgs (see the
// EPI_* modes).  A persistent CTA per SM walks the units u = blockIdx.x + j
// gridDim.x.  The stage ring runs on across units (a global k-block counter gives
// each stage's phase), and the accumulator alternates between two TMEM buffers,
// so the MMAs of unit j + 1 proceed while the epilogue warps drain unit j.
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) tma_gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                              const __grid_constant__ CUtensorMap tb,
                                                              const GemmArgs g, int K, int units, int tiles_n,
                                                              int tiles_mn) {
  constexpr int NS = Cfg<MODE>::NSTAGE;
  extern __shared__ __align__(16) unsigned char raw[];
  __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[2], tempty[2], drain;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  // stages on a 1024-byte boundary (the 128-byte swizzle repeats every 8 rows of 128 bytes)
  unsigned char* sm = raw + ((1024u - (sa(raw) & 1023u)) & 1023u);
  unsigned char* extra = sm + NS * STAGE_BYTES;  // EPI_STAGED: the output tile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&tfull[b], 1);
      bar_init(&tempty[b], NEPI);
    }
    bar_init(&drain, 1);
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
      int it = 0;  // k-blocks issued by this CTA
      bool ok = true;
      for (int u = blockIdx.x; ok && u < units; u += gridDim.x) {
        const Unit w = unit_of(u, g, K, tiles_n, tiles_mn);
        for (int i = 0; i < w.nk; ++i, ++it) {
          const int s = it % NS;
          // the stage's previous MMAs (its use it - NS) have released it
          if (it >= NS && !bar_wait(&empty[s], (uint32_t)((it / NS - 1) & 1))) {
            s_fail = 1;
            ok = false;
            break;
          }
          unsigned char* st = sm + s * STAGE_BYTES;
          bar_expect_tx(&full[s], STAGE_BYTES);
          const int k = w.kb + i * BK;  // a multiple of 64: 128-byte aligned inner coordinate
          tma_load(st, &ta, k, w.m0, &full[s]);
          tma_load(st + TILE_BYTES, &tb, k, w.n0, &full[s]);
        }
      }
      // before the CTA exits, every load it issued has landed (the last use of each
      // stage; earlier uses were consumed by the MMAs)
      for (int j = max(0, it - NS); j < it; ++j)
        if (!bar_wait(&full[j % NS], (uint32_t)((j / NS) & 1))) s_fail = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      int it = 0, j = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < units; u += gridDim.x, ++j) {
        const Unit w = unit_of(u, g, K, tiles_n, tiles_mn);
        const int buf = j & 1;
        // the epilogue has read this buffer's previous unit (j - 2)
        if (j >= 2 && !bar_wait(&tempty[buf], (uint32_t)(((j >> 1) - 1) & 1))) {
          s_fail = 1;
          break;
        }
        tfence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        for (int i = 0; i < w.nk; ++i, ++it) {
          const int s = it % NS;
          if (!bar_wait(&full[s], (uint32_t)((it / NS) & 1))) {
            s_fail = 1;
            ok = false;
            break;
          }
          tfence_after();
          const uint32_t a0 = sa(sm + s * STAGE_BYTES), b0 = a0 + TILE_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            tmma(d, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
          tcommit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        tcommit(&tfull[buf]);  // arrives when every MMA issued above has completed
      }
      // every MMA this thread issued has completed before the TMEM is freed
      tcommit(&drain);
      if (!bar_wait(&drain, 0u)) s_fail = 1;
    }
  } else {
    // epilogue warps: TMEM lane quadrant warp mod 4 (output rows 32 q .. 32 q + 31)
    const int e = warp - 2, q = warp & 3, h = e >> 2;
    const int row = q * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    const float alpha = (float)g.alpha;
    const float beta = (float)(g.beta_dev ? *g.beta_dev : g.beta);
    {
      const bool split = g.splits > 1;
      const bool with_d = !split && g.D != nullptr && beta != 0.f;
      float* T = reinterpret_cast<float*>(extra);
      constexpr int RB = BM / NEPI;  // rows of the tile per warp in the row-major write-out
      int j = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x, ++j) {
        const Unit w = unit_of(u, g, K, tiles_n, tiles_mn);
        const int m0 = w.m0, n0 = w.n0;
        const int buf = j & 1;
        // row-major write-out: lane l owns columns 4 l .. 4 l + 3 of the tile; warp e
        // rows e + NEPI t.  D does not depend on the accumulator, so its loads are
        // issued before the wait and their latency hides behind the MMAs.
        const int n = n0 + 4 * lane;
        const bool fullv = n + 4 <= g.N;
        float4 dq[RB];
        if constexpr (MODE == EPI_STAGED) {
          const bool vec_d = with_d && ((reinterpret_cast<uintptr_t>(g.D) & 15u) == 0) && (g.ldd & 3) == 0;
#pragma unroll
          for (int t = 0; t < RB; ++t) {
            const int m = m0 + e + NEPI * t;
            dq[t] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g.c_rowmaj && with_d && m < g.M && n < g.N) {
              const float* drow = (const float*)g.D + (int64_t)m * g.ldd + n;
              if (fullv && vec_d) {
                dq[t] = __ldg(reinterpret_cast<const float4*>(drow));
              } else {
                dq[t].x = drow[0];
                if (n + 1 < g.N) dq[t].y = drow[1];
                if (n + 2 < g.N) dq[t].z = drow[2];
                if (n + 3 < g.N) dq[t].w = drow[3];
              }
            }
          }
        }
        const bool okt = bar_wait(&tfull[buf], (uint32_t)((j >> 1) & 1));
        tfence_after();
        // every warp has finished reading T for unit j - 1; one verdict for all
        const bool done = !epi_any(!okt);
        const bool have = done && w.nk > 0;
        if constexpr (MODE == EPI_STAGED) {
          // accumulator -> T, 16-byte stores (a quarter warp covers all banks)
#pragma unroll
          for (int c0 = h * (BN / 2); c0 < (h + 1) * (BN / 2); c0 += 16) {
            float v[16];
            if (have) {
              tld16(trow + (uint32_t)(buf * BN + c0), v);
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 16; i += 4)
              *reinterpret_cast<float4*>(&T[row * OLD + c0 + i]) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
          }
          tfence_before();
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(&tempty[buf])) : "memory");
          epi_sync();  // T holds unit j
          if (!done) {
            if (e == 0 && lane == 0) s_fail = 1;
            break;
          }
          if (g.c_rowmaj) {
            float* out = (float*)g.C;
            const int64_t ldo = g.ldc;
            const bool vec_o = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) && (ldo & 3) == 0;
            float csv[4], dsv[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const bool in = n + jj < g.N;
              csv[jj] = (g.cs && in) ? (float)g.cs[n + jj] : 1.f;
              dsv[jj] = (g.ds && in) ? (float)g.ds[n + jj] : 1.f;
            }
#pragma unroll
            for (int t = 0; t < RB; ++t) {
              const int r = e + NEPI * t, m = m0 + r;
              if (m >= g.M || n >= g.N) continue;
              const float rsm = g.rs ? (float)g.rs[m] : 1.f;
              const float4 tv = *reinterpret_cast<const float4*>(&T[r * OLD + 4 * lane]);
              const float av[4] = {tv.x, tv.y, tv.z, tv.w};
              const float dv[4] = {dq[t].x, dq[t].y, dq[t].z, dq[t].w};
              float o[4];
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                o[jj] = av[jj] * (alpha * rsm * csv[jj]);
                if (with_d) o[jj] += beta * dv[jj] * dsv[jj];
              }
              float* orow = out + (int64_t)m * ldo + n;
              if (fullv && vec_o) {
                *reinterpret_cast<float4*>(orow) = make_float4(o[0], o[1], o[2], o[3]);
              } else {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                  if (n + jj < g.N) orow[jj] = o[jj];
              }
            }
          } else {
            for (int rb = 0; rb < BM; rb += 32) {
              const int r = rb + lane, m = m0 + r;
              const float rsm = (g.rs && m < g.M) ? (float)g.rs[m] : 1.f;
              for (int c = e; c < BN; c += NEPI) {
                const int nn = n0 + c;
                if (m >= g.M || nn >= g.N) continue;
                float o = T[r * OLD + c] * alpha * rsm;
                if (g.cs) o *= (float)g.cs[nn];
                if (with_d) {
                  float dv = ((const float*)g.D)[m + (int64_t)nn * g.ldd];
                  if (g.ds) dv *= (float)g.ds[nn];
                  o += beta * dv;
                }
                ((float*)g.C)[m + (int64_t)nn * g.ldc] = o;
              }
            }
          }
        } else {
          // split-K partial (row-major M x N per split): this thread's row, straight
          // from TMEM, 16 columns at a time
          float* prow = (float*)g.partial + (int64_t)w.z * g.M * g.N + (int64_t)(m0 + row) * g.N;
          const bool in_row = m0 + row < g.M;
          const bool vec_p = ((reinterpret_cast<uintptr_t>(g.partial) & 15u) == 0) && (g.N & 3) == 0;
#pragma unroll
          for (int c0 = h * (BN / 2); c0 < (h + 1) * (BN / 2); c0 += 16) {
            float v[16];
            if (have) {
              tld16(trow + (uint32_t)(buf * BN + c0), v);
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
            const int nc = n0 + c0;
            if (in_row && nc < g.N) {
              if (vec_p && nc + 16 <= g.N) {
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                  *reinterpret_cast<float4*>(prow + nc + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
              } else {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                  if (nc + i < g.N) prow[nc + i] = v[i];
              }
            }
          }
          tfence_before();
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(&tempty[buf])) : "memory");
          if (!done) {
            if (e == 0 && lane == 0) s_fail = 1;
            break;
          }
        }
      }
    }
  }
  tfence_before();
  __syncthreads();
  if (s_fail && threadIdx.x == 0) report(BKFAC_ETIMEOUT);
  if (warp == 1) {
    tfence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---- BF16 operand preparation (round to nearest even) -----------------------

// Rows p of a strip source (row p < P0 at S0 + p ld0, else at S1 + (p - P0) ld1;
// each row `inner` contiguous FP32 values) -> BF16 in the same layout (Yb, row
// pitch ldb; may be null) and transposed (Yt: inner x P row-major, pitch ldt; may
// be null).  Tiles of 32 rows x 128 inner values: 16-byte loads along the rows,
// 8-byte stores of the copy, and the transpose through shared memory with
// 16-byte stores of eight consecutive rows.
__global__ void __launch_bounds__(256) cvt_strip_kernel(const float* __restrict__ S0, int64_t ld0, int P0,
                                                        const float* __restrict__ S1, int64_t ld1, int P, int inner,
                                                        __nv_bfloat16* __restrict__ Yb, int64_t ldb,
                                                        __nv_bfloat16* __restrict__ Yt, int64_t ldt) {
  __shared__ __align__(16) __nv_bfloat16 t[32][132];  // [row of the tile][inner]; 264-byte pitch
  const int p0 = blockIdx.y * 32, i0 = blockIdx.x * 128;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = w; r < 32; r += 8) {
    const int p = p0 + r, i = i0 + 4 * lane;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    const bool in = p < P && i < inner;
    if (in) {
      const float* row = p < P0 ? S0 + (int64_t)p * ld0 : S1 + (int64_t)(p - P0) * ld1;
      if (i + 4 <= inner && ((reinterpret_cast<uintptr_t>(row + i) & 15u) == 0)) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(row + i));
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
      } else {
        for (int e = 0; e < 4; ++e)
          if (i + e < inner) v[e] = row[i + e];
      }
    }
    __align__(8) __nv_bfloat16 b[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) b[e] = __float2bfloat16_rn(v[e]);
    *reinterpret_cast<uint2*>(&t[r][4 * lane]) = *reinterpret_cast<const uint2*>(b);
    if (Yb != nullptr && in) {
      __nv_bfloat16* y = Yb + (int64_t)p * ldb + i;
      if (i + 4 <= inner && ((reinterpret_cast<uintptr_t>(y) & 7u) == 0)) {
        *reinterpret_cast<uint2*>(y) = *reinterpret_cast<const uint2*>(b);
      } else {
        for (int e = 0; e < 4; ++e)
          if (i + e < inner) y[e] = b[e];
      }
    }
  }
  if (Yt == nullptr) return;  // block-uniform
  __syncthreads();
  // transposed: row i of Yt holds tile rows p0 .. p0 + 31 as four 16-byte pieces
  for (int q = threadIdx.x; q < 128 * 4; q += 256) {
    const int ii = q >> 2, part = q & 3;
    const int i = i0 + ii, p = p0 + 8 * part;
    if (i >= inner || p >= P) continue;
    __align__(16) __nv_bfloat16 b[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) b[e] = t[8 * part + e][ii];
    __nv_bfloat16* y = Yt + (int64_t)i * ldt + p;
    if (p + 8 <= P && ((reinterpret_cast<uintptr_t>(y) & 15u) == 0)) {
      *reinterpret_cast<uint4*>(y) = *reinterpret_cast<const uint4*>(b);
    } else {
      for (int e = 0; e < 8; ++e)
        if (p + e < P) y[e] = b[e];
    }
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

template <int MODE>
int launch_mode(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int K, int64_t units,
                int64_t tiles_n, int64_t tiles, int sms, cudaStream_t s) {
  static std::atomic<uint64_t> configured{0};
  if (!configured_here(configured)) {
    const cudaError_t e = cudaFuncSetAttribute(tma_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               Cfg<MODE>::SMEM_BYTES);
    if (e != cudaSuccess) return (int)e;
    mark_configured(configured);
  }
  const unsigned grid = (unsigned)std::min<int64_t>(units, sms);
  tma_gemm_kernel<MODE><<<grid, THREADS, Cfg<MODE>::SMEM_BYTES, s>>>(ta, tb, g, K, (int)units, (int)tiles_n,
                                                                      (int)tiles);
  note_launches(1);
  return (int)cudaGetLastError();
}

}  // namespace

bool tma_gemm_available() { return encode_fn() != nullptr; }

int64_t bf16_ld(int k) { return round_up(std::max(k, 1), 8); }

// C (M x N) = alpha sum_k A[m, k] B[n, k] (+ epilogue of g), A: M x K, B: N x K, both
// BF16 K-major with row pitches lda / ldb (multiples of 8 elements).  g supplies M,
// N, C, ldc, c_rowmaj, alpha, beta / beta_dev, rs, cs, ds, D, ldd, and partial /
// partial_bytes for split K (chosen here: an output with fewer tiles than SMs is
// split along K until the units about fill the GPU).  One persistent CTA per SM.
int tma_gemm_run(const void* A, int64_t lda, const void* B, int64_t ldb, int K, const GemmArgs& g0, cudaStream_t s) {
  GemmArgs g = g0;
  if (g.M <= 0 || g.N <= 0) return (int)cudaSuccess;
  CUtensorMap ta, tb;
  if (!encode_kmajor(&ta, A, g.M, std::max(K, 1), lda) || !encode_kmajor(&tb, B, g.N, std::max(K, 1), ldb))
    return (int)cudaErrorInvalidValue;
  const int sms = sm_count();
  const int64_t tiles_n = ceil_div(g.N, BN), tiles = ceil_div(g.M, BM) * tiles_n;
  int64_t splits = 1;
  if (g.partial != nullptr && tiles < sms && K > 4 * BK) {
    const int64_t room = (int64_t)(g.partial_bytes / ((size_t)g.M * g.N * sizeof(float)));
    splits = std::min<int64_t>(std::min<int64_t>(sms / tiles, (int64_t)K / (2 * BK)), room);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, 32));
  }
  g.k_chunk = (int)round_up(ceil_div(std::max(K, 1), splits), BK);
  g.splits = (int)std::max<int64_t>(1, ceil_div(std::max(K, 1), g.k_chunk));
  const int64_t units = tiles * g.splits;
  if (units > INT32_MAX) return (int)cudaErrorInvalidValue;
  if (g.splits > 1) {
    const int rc = launch_mode<EPI_PARTIAL>(ta, tb, g, K, units, tiles_n, tiles, sms, s);
    if (rc != 0) return rc;
    return splitk_reduce_f32(g, s);
  }
  return launch_mode<EPI_STAGED>(ta, tb, g, K, units, tiles_n, tiles, sms, s);
}

namespace {
int launch_strip(const float* S0, int64_t ld0, int P0, const float* S1, int64_t ld1, int P, int inner, void* Yb,
                 int64_t ldb, void* Yt, int64_t ldt, cudaStream_t s) {
  if (P <= 0 || inner <= 0) return 0;
  dim3 grid((unsigned)ceil_div(inner, 128), (unsigned)ceil_div(P, 32));
  cvt_strip_kernel<<<grid, 256, 0, s>>>(S0, ld0, P0, S1, ld1, P, inner, (__nv_bfloat16*)Yb, ldb,
                                        (__nv_bfloat16*)Yt, ldt);
  note_launches(1);
  return (int)cudaGetLastError();
}
}  // namespace

// G (R x C row-major, ld ldg) -> Gb (R x C, ld ldb) and its transpose Gt (C x R, ld
// ldt), from one read of G
int launch_cvt_both(const float* G, int64_t ldg, int R, int C, void* Gb, int64_t ldb, void* Gt, int64_t ldt,
                    cudaStream_t s) {
  return launch_strip(G, ldg, R, nullptr, 0, R, C, Gb, ldb, Gt, ldt, s);
}

// k columns of length d (column-major, ld) -> the same layout in BF16 (ld ldo)
int launch_cvt_cols(const float* X, int64_t ld, int d, int k, void* Y, int64_t ldo, cudaStream_t s) {
  return launch_strip(X, ld, k, nullptr, 0, k, d, Y, ldo, nullptr, 0, s);
}

// [X0 | X1] (dim x (k0 + k1), each column-major) -> Y (dim x (k0 + k1) row-major,
// ld ldy): Y[i][k] = k < k0 ? X0[i + k ld0] : X1[i + (k - k0) ld1]
int launch_cvt_cat_t(const float* X0, int64_t ld0, int k0, const float* X1, int64_t ld1, int k1, int dim, void* Y,
                     int64_t ldy, cudaStream_t s) {
  return launch_strip(X0, ld0, k0, X1, ld1, k0 + k1, dim, nullptr, 0, Y, ldy, s);
}

}  // namespace bkfac

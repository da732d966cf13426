// tc_gemm.cu -- the tall-skinny products of the mixed-precision path on the
// 5th-generation tensor cores (tcgen05): BF16 operands, FP32 accumulation in
// tensor memory (TMEM).
//
// Same contract as the SIMT GEMM (common.cuh, GemmArgs): C[m, n] = alpha rs[m]
// cs[n] sum_k A[m, k] B[k, n] + beta ds[n] D[m, n], A = [A0 | A1] and
// B = [B0 ; B1] split along K, any of the four operand layouts, FP32 in memory.
// Operands are rounded to BF16 (round to nearest even, the same rounding the
// SIMT path applies in mixed mode) while they are staged into shared memory.
//
// Tile: 128 x 128 outputs per CTA (one tcgen05.mma.cta_group::1 of M = 128,
// N = 128 per K step of 16), K staged 64 at a time in two shared-memory buffers.
// Eight warps convert and store the next K block while the tensor core works on
// the current one; one thread issues the MMAs and commits them to the buffer's
// mbarrier, which releases the buffer for reuse.  The accumulator lives in 128
// TMEM columns; the epilogue reads it back with tcgen05.ld (warp w reads TMEM
// lanes 32 (w mod 4) .. 32 (w mod 4) + 31, i.e. output rows, the two warps of a
// quadrant one half of the columns each) into a shared-memory tile, from which
// rows (row-major C, split-K partials) or columns (column-major C) leave with
// coalesced accesses after the scaling; splitk_reduce sums partials in a fixed
// order.  Two CTAs per SM (at most 128 registers per thread).

// Shared-memory operand layout: K-major, no swizzle.  Each K step of 16 is a
// 128 x 16 sub-tile (4 KB) built from 8 x 16-byte "core matrices" (8 rows of 8
// BF16): core matrices adjacent in K are 128 bytes apart (leading byte offset),
// 8-row groups 256 bytes apart (stride byte offset).
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "common.cuh"

namespace bkfac {
namespace {

constexpr int TM = 128, TN = 128;  // output tile
constexpr int TC_THREADS = 256;  // eight warps: two per TMEM lane quadrant in the epilogue
constexpr int SUB_BYTES = 4096;  // one 128-row operand sub-tile: the K of one MMA (32 bytes per row)
constexpr int TMEM_COLS = 128;
constexpr int TLD = TN + 1;  // leading dimension of the staged output tile (floats)

// Operand encodings.  BF16 (X3 = false): one operand tile per matrix, K = 16 per
// MMA.  3xTF32 (X3 = true): each FP32 value x is split into hi = tf32(x) and
// lo = tf32(x - hi); D += A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped
// A_lo B_lo term is below 2^-22 |a b|, FP32 accumulation), K = 8 per MMA.
// Either way a stage holds four MMA sub-tiles of each operand tile.
template <bool X3>
struct TcMode {
  static constexpr int EPC = X3 ? 4 : 8;       // elements per 16-byte core-matrix row
  static constexpr int KPM = X3 ? 8 : 16;      // K per MMA
  static constexpr int TK = 4 * KPM;           // K per stage
  static constexpr int TILES = X3 ? 4 : 2;     // A(hi, lo), B(hi, lo) or A, B
  static constexpr int STAGE_BYTES = TILES * 4 * SUB_BYTES;
  static constexpr int SMEM_BYTES = (2 * STAGE_BYTES > TM * TLD * 4 ? 2 * STAGE_BYTES : TM * TLD * 4) + 1024;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading / stride byte offsets
// (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor: FP32 accumulator, A and B both K-major, operand format
// 1 = BF16 (kind::f16) or 2 = TF32 (kind::tf32)
__host__ __device__ constexpr uint32_t instr_desc(int m, int n, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (about a second of clock cycles); false on time-out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <bool X3>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
  if constexpr (X3)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
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

// A[m, k] of the concatenated operand (zero outside)
__device__ __forceinline__ float ld_a(const GemmArgs& g, int m, int k, int K) {
  if (m >= g.M || k >= K) return 0.f;
  const float* A = (const float*)g.A0;
  int64_t lda = g.lda0;
  if (k >= g.K0) {
    A = (const float*)g.A1;
    lda = g.lda1;
    k -= g.K0;
  }
  return __ldg(g.a_kmaj ? A + (int64_t)m * lda + k : A + m + (int64_t)k * lda);
}
// B[k, n]: element (n, k) of the K-major view B^T
__device__ __forceinline__ float ld_b(const GemmArgs& g, int n, int k, int K) {
  if (n >= g.N || k >= K) return 0.f;
  const float* B = (const float*)g.B0;
  int64_t ldb = g.ldb0;
  if (k >= g.K0) {
    B = (const float*)g.B1;
    ldb = g.ldb1;
    k -= g.K0;
  }
  return __ldg(g.b_kmaj ? B + (int64_t)n * ldb + k : B + (int64_t)k * ldb + n);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// byte offset of the 16-byte core-matrix row holding elements (row, k .. k + EPC
// - 1) of a staged operand tile (k a multiple of EPC): MMA sub-tile k / KPM,
// then core matrix (row / 8, (k mod KPM) / EPC), then row mod 8
template <bool X3>
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  using Md = TcMode<X3>;
  return (uint32_t)((k / Md::KPM) * SUB_BYTES + (row >> 3) * 256 + ((k % Md::KPM) / Md::EPC) * 128 + (row & 7) * 16);
}

// TF32 rounding (to nearest, ties away) of an FP32 value, as FP32 bits
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// store one 16-byte group of EPC consecutive-K elements: BF16 into tile 0, or
// the TF32 hi / lo parts into tiles 0 / 1
template <bool X3>
__device__ __forceinline__ void put_group(unsigned char* t0, unsigned char* t1, uint32_t off, const float* v) {
  if constexpr (X3) {
    uint4 hi, lo;
    uint32_t* h = reinterpret_cast<uint32_t*>(&hi);
    uint32_t* l = reinterpret_cast<uint32_t*>(&lo);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = to_tf32(v[e]);
      l[e] = to_tf32(v[e] - __uint_as_float(h[e]));
    }
    *reinterpret_cast<uint4*>(t0 + off) = hi;
    *reinterpret_cast<uint4*>(t1 + off) = lo;
  } else {
    uint4 q;
    q.x = pack_bf16(v[0], v[1]);
    q.y = pack_bf16(v[2], v[3]);
    q.z = pack_bf16(v[4], v[5]);
    q.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(t0 + off) = q;
  }
}

// Segment of the concatenated operand holding K index k (k < K), the element
// pointer of (row, k), and whether 16-byte vector loads of 4 consecutive
// elements along the contiguous index are legal there.
struct Seg {
  const float* p;
  int64_t ld;
  int k;  // K index within the segment
  bool vec;
};
template <bool IS_A>
__device__ __forceinline__ Seg seg_of(const GemmArgs& g, int k) {
  const bool first = k < g.K0;
  const float* p = (const float*)(IS_A ? (first ? g.A0 : g.A1) : (first ? g.B0 : g.B1));
  const int64_t ld = IS_A ? (first ? g.lda0 : g.lda1) : (first ? g.ldb0 : g.ldb1);
  Seg s;
  s.p = p;
  s.ld = ld;
  s.k = first ? k : k - g.K0;
  s.vec = ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) && ((ld & 3) == 0);
  return s;
}

// Staging of rows [r0, r0 + 128) x K block [k0, k0 + TK) of one operand into
// its tile(s) t0 (and t1 for the TF32 lo parts), canonical layout; rows >= R
// (M or N) and K >= K read as zero.  `kmaj`: the operand's K index is
// contiguous in memory.  Work items are EPC consecutive K of one row (one
// 16-byte core-matrix row): K-contiguous operands are read along K (16-byte
// loads, 8 lanes per row segment), the others along rows (lanes over 4-row
// groups, one 16-byte load per K).  Split in two so that the kernel can issue
// the next stage's loads (up to sixteen 16-byte loads per thread in flight)
// before it waits for the tensor core to release the buffer.  Items that
// straddle an edge, the K0 seam or a misaligned start fall back to element
// loads.
template <bool X3>
struct Stage {
  static constexpr int EPC = TcMode<X3>::EPC, CH = TcMode<X3>::TK / EPC;  // 8 chunks per row either way
  static constexpr int NK = TM * CH / TC_THREADS;                          // K-contiguous items per thread (8)
  static constexpr int NR = (TM / 4) * CH / TC_THREADS;                    // row-contiguous items per thread (2)
  static constexpr int VN = NK * EPC;                                      // == NR * 4 * EPC
};

template <bool X3, bool IS_A>
__device__ __forceinline__ void load_operand(const GemmArgs& g, int r0, int k0, int K, int tid,
                                             float (&v)[Stage<X3>::VN]) {
  using S = Stage<X3>;
  constexpr int EPC = S::EPC, CH = S::CH;
  constexpr int TK = TcMode<X3>::TK;
  const bool kmaj = IS_A ? g.a_kmaj : g.b_kmaj;
  const int R = IS_A ? g.M : g.N;
  // interior block (all rows and K in range, inside one segment, vector-aligned):
  // straight-line 16-byte loads from one base pointer, all issued back to back
  {
    const Seg sg = seg_of<IS_A>(g, min(k0, max(K - 1, 0)));
    const bool interior = r0 + TM <= R && k0 + TK <= K && (k0 >= g.K0 || k0 + TK <= g.K0) && sg.vec &&
                          (sg.k & 3) == 0;
    if (interior) {
      if (kmaj) {
        const float* base = sg.p + (int64_t)r0 * sg.ld + sg.k;
#pragma unroll
        for (int q = 0; q < S::NK; ++q) {
          const int it = tid + q * TC_THREADS;
          const float4* src = reinterpret_cast<const float4*>(base + (int64_t)(it / CH) * sg.ld + (it % CH) * EPC);
#pragma unroll
          for (int h = 0; h < EPC / 4; ++h) {
            const float4 x = __ldg(src + h);
            v[q * EPC + 4 * h] = x.x; v[q * EPC + 4 * h + 1] = x.y;
            v[q * EPC + 4 * h + 2] = x.z; v[q * EPC + 4 * h + 3] = x.w;
          }
        }
      } else {
        const float* base = sg.p + r0 + (int64_t)sg.k * sg.ld;
#pragma unroll
        for (int q = 0; q < S::NR; ++q) {
          const int it = tid + q * TC_THREADS;
          const int rq = (it & 31) * 4, kc = (it >> 5) * EPC;
#pragma unroll
          for (int e = 0; e < EPC; ++e) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(base + rq + (int64_t)(kc + e) * sg.ld));
            v[(q * 4 + 0) * EPC + e] = x.x; v[(q * 4 + 1) * EPC + e] = x.y;
            v[(q * 4 + 2) * EPC + e] = x.z; v[(q * 4 + 3) * EPC + e] = x.w;
          }
        }
      }
      return;
    }
  }
  if (kmaj) {
#pragma unroll
    for (int q = 0; q < S::NK; ++q) {
      const int it = tid + q * TC_THREADS;
      const int row = it / CH, kc = (it % CH) * EPC;
      const int gr = r0 + row, gk = k0 + kc;
      const Seg sg = seg_of<IS_A>(g, min(gk, max(K - 1, 0)));
      const bool fast = gr < R && gk + EPC <= K && (gk >= g.K0 || gk + EPC <= g.K0) && sg.vec && (sg.k & 3) == 0;
      if (fast) {
        const float4* src = reinterpret_cast<const float4*>(sg.p + (int64_t)gr * sg.ld + sg.k);
#pragma unroll
        for (int h = 0; h < EPC / 4; ++h) {
          const float4 x = __ldg(src + h);
          v[q * EPC + 4 * h] = x.x; v[q * EPC + 4 * h + 1] = x.y;
          v[q * EPC + 4 * h + 2] = x.z; v[q * EPC + 4 * h + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int e = 0; e < EPC; ++e) v[q * EPC + e] = IS_A ? ld_a(g, gr, gk + e, K) : ld_b(g, gr, gk + e, K);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < S::NR; ++q) {
      const int it = tid + q * TC_THREADS;
      const int rq = (it & 31) * 4, kc = (it >> 5) * EPC;
      const int gr = r0 + rq, gk = k0 + kc;
      const bool rows_in = gr + 4 <= R;
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int k = gk + e;
        bool done = false;
        if (rows_in && k < K) {
          const Seg sg = seg_of<IS_A>(g, k);
          if (sg.vec) {  // r0 and rq are multiples of 4: the 4 rows form one aligned vector
            const float4 x = __ldg(reinterpret_cast<const float4*>(sg.p + gr + (int64_t)sg.k * sg.ld));
            v[(q * 4 + 0) * EPC + e] = x.x; v[(q * 4 + 1) * EPC + e] = x.y;
            v[(q * 4 + 2) * EPC + e] = x.z; v[(q * 4 + 3) * EPC + e] = x.w;
            done = true;
          }
        }
        if (!done)
#pragma unroll
          for (int i = 0; i < 4; ++i)
            v[(q * 4 + i) * EPC + e] = IS_A ? ld_a(g, gr + i, k, K) : ld_b(g, gr + i, k, K);
      }
    }
  }
}

template <bool X3, bool IS_A>
__device__ __forceinline__ void store_operand(const GemmArgs& g, unsigned char* t0, unsigned char* t1, int tid,
                                              const float (&v)[Stage<X3>::VN]) {
  using S = Stage<X3>;
  constexpr int EPC = S::EPC, CH = S::CH;
  const bool kmaj = IS_A ? g.a_kmaj : g.b_kmaj;
  if (kmaj) {
#pragma unroll
    for (int q = 0; q < S::NK; ++q) {
      const int it = tid + q * TC_THREADS;
      put_group<X3>(t0, t1, tile_off<X3>(it / CH, (it % CH) * EPC), v + q * EPC);
    }
  } else {
#pragma unroll
    for (int q = 0; q < S::NR; ++q) {
      const int it = tid + q * TC_THREADS;
      const int rq = (it & 31) * 4, kc = (it >> 5) * EPC;
#pragma unroll
      for (int i = 0; i < 4; ++i) put_group<X3>(t0, t1, tile_off<X3>(rq + i, kc), v + (q * 4 + i) * EPC);
    }
  }
}

template <bool X3>
__global__ void __launch_bounds__(TC_THREADS, 2) tc_gemm_kernel(const GemmArgs g) {
  using Md = TcMode<X3>;
  constexpr int TK = Md::TK, STAGE_BYTES = Md::STAGE_BYTES;
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];  // only 16 bytes are guaranteed
  __shared__ __align__(8) uint64_t s_mma_done[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int K = g.K0 + g.K1;
  const int kb = blockIdx.z * g.k_chunk;
  const int ke = min(K, kb + g.k_chunk);
  const int nk = (ke - kb + TK - 1) / TK;
  // operand tiles on a 1024-byte boundary of the shared window, computed at run
  // time: the dynamic region starts right after the static variables (measured:
  // 32 bytes past a boundary), and the tensor core reads a no-swizzle operand
  // from the 128-byte aligned address below the descriptor's start (a tile at
  // 1056 was read from 1024)
  unsigned char* tc_smem = tc_smem_raw + ((1024u - (saddr(tc_smem_raw) & 1023u)) & 1023u);

  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&s_mma_done[0], 1);
    mbar_init(&s_mma_done[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  constexpr uint32_t idesc = instr_desc(TM, TN, X3 ? 2u : 1u);

  bool failed = false;
  for (int it = 0; it < nk; ++it) {
    const int st = it & 1;
    unsigned char* sA = tc_smem + st * STAGE_BYTES;              // A (hi)
    unsigned char* sB = sA + STAGE_BYTES / Md::TILES * (X3 ? 2 : 1);  // B (hi)
    unsigned char* sAl = sA + 4 * SUB_BYTES;                       // A lo (TF32 only)
    unsigned char* sBl = sB + 4 * SUB_BYTES;                       // B lo (TF32 only)
    const int k0 = kb + it * TK;
    // K beyond this split's chunk reads as zero; loads first, then the wait for
    // the MMAs that read this buffer two iterations ago, then the stores
    float va[Stage<X3>::VN], vb[Stage<X3>::VN];
    load_operand<X3, true>(g, m0, k0, ke, tid, va);
    load_operand<X3, false>(g, n0, k0, ke, tid, vb);
    if (it >= 2 && !failed && !mbar_wait(&s_mma_done[st], (uint32_t)((it - 2) >> 1) & 1u)) failed = true;
    store_operand<X3, true>(g, sA, sAl, tid, va);
    store_operand<X3, false>(g, sB, sBl, tid, vb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic stores -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = smem_desc(saddr(sA + kk * SUB_BYTES), 128, 256);
        const uint64_t bd = smem_desc(saddr(sB + kk * SUB_BYTES), 128, 256);
        tc_mma<X3>(tmem, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
        if constexpr (X3) {
          const uint64_t adl = smem_desc(saddr(sAl + kk * SUB_BYTES), 128, 256);
          const uint64_t bdl = smem_desc(saddr(sBl + kk * SUB_BYTES), 128, 256);
          tc_mma<X3>(tmem, ad, bdl, idesc, 1u);
          tc_mma<X3>(tmem, adl, bd, idesc, 1u);
        }
      }
      tc_commit(&s_mma_done[st]);
    }
  }
  // all MMAs complete (they finish in issue order; the last commit covers them)
  if (nk > 0 && !failed && !mbar_wait(&s_mma_done[(nk - 1) & 1], (uint32_t)((nk - 1) >> 1) & 1u)) failed = true;
  if (failed) s_fail = 1;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (!s_fail) {
    // accumulator -> shared tile T (row-major, ld 129: conflict-free whether lanes
    // run over rows or over columns); the operand buffers are free now
    float* T = reinterpret_cast<float*>(tc_smem);
    {
      // a warp reaches the TMEM lanes of its quadrant (warp id mod 4): rows 32 q ..
      // 32 q + 31; the warps sharing a quadrant split the columns
      constexpr int NW = TC_THREADS / 32, CPW = TN / (NW / 4);
      const int q = wid & 3, c_begin = (wid >> 2) * CPW;
      const int row = q * 32 + lane;
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
      for (int c0 = c_begin; c0 < c_begin + CPW; c0 += 16) {
        float v[16];
        if (nk > 0) {
          tc_ld16(trow + (uint32_t)c0, v);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) T[row * TLD + c0 + i] = v[i];
      }
    }
    __syncthreads();
    const float beta = (float)(g.beta_dev ? *g.beta_dev : g.beta);
    const float alpha = (float)g.alpha;
    const bool with_d = g.D != nullptr && beta != 0.f && g.splits == 1;
    if (g.c_rowmaj || g.splits > 1) {
      // rows go out whole: lane l owns columns 4l .. 4l + 3 of the tile
      const int n = n0 + 4 * lane;
      float csv[4], dsv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool in = n + j < g.N;
        csv[j] = (g.cs && in) ? (float)g.cs[n + j] : 1.f;
        dsv[j] = (g.ds && in) ? (float)g.ds[n + j] : 1.f;
      }
      float* out = g.splits > 1 ? (float*)g.partial + (int64_t)blockIdx.z * g.M * g.N : (float*)g.C;
      const int64_t ldo = g.splits > 1 ? g.N : g.ldc;
      const bool vec_o = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) && (ldo & 3) == 0;
      const bool vec_d = with_d && ((reinterpret_cast<uintptr_t>(g.D) & 15u) == 0) && (g.ldd & 3) == 0;
      const bool full = n + 4 <= g.N;
      // eight rows per warp at a time: their D rows are all in flight before use
      constexpr int RB = 8, RS = TC_THREADS / 32;
      for (int r0b = wid; r0b < TM; r0b += RB * RS) {
        float4 dq[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const int m = m0 + r0b + u * RS;
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
          const int r = r0b + u * RS, m = m0 + r;
          if (m >= g.M || n >= g.N) continue;
          const float rsm = (g.splits == 1 && g.rs) ? (float)g.rs[m] : 1.f;
          const float dv[4] = {dq[u].x, dq[u].y, dq[u].z, dq[u].w};
          float o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            o[j] = T[r * TLD + 4 * lane + j];
            if (g.splits == 1) o[j] *= alpha * rsm * csv[j];
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
      // column-major C: lanes run over 32 consecutive rows of one column
      for (int rb = 0; rb < TM; rb += 32) {
        const int r = rb + lane, m = m0 + r;
        const float rsm = (g.rs && m < g.M) ? (float)g.rs[m] : 1.f;
        for (int c = wid; c < TN; c += TC_THREADS / 32) {
          const int n = n0 + c;
          if (m >= g.M || n >= g.N) continue;
          float o = T[r * TLD + c] * alpha * rsm;
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
  } else if (tid == 0) {
    report(BKFAC_ETIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

namespace {

template <bool X3>
int tc_launch(const GemmArgs& g, cudaStream_t s) {
  using Md = TcMode<X3>;
  GemmArgs a = g;
  const int K = a.K0 + a.K1;
  const int64_t tiles = ceil_div(a.M, TM) * ceil_div(a.N, TN);
  // split K so that about two CTAs per SM are busy, within the partial buffer
  int64_t splits = 1;
  if (a.partial != nullptr && tiles < 2 * sm_count() && K > 4 * Md::TK) {
    const int64_t room = (int64_t)(a.partial_bytes / ((size_t)a.M * a.N * sizeof(float)));
    splits = std::min<int64_t>(std::min<int64_t>(ceil_div(2 * sm_count(), tiles), (int64_t)K / (2 * Md::TK)), room);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, 32));
  }
  a.k_chunk = (int)round_up(ceil_div(std::max(K, 1), splits), Md::TK);
  a.splits = (int)std::max<int64_t>(1, ceil_div(std::max(K, 1), a.k_chunk));
  static std::atomic<uint64_t> configured{0};  // attribute set once (the call can stall the host)
  if (!configured_here(configured)) {
    const cudaError_t e =
        cudaFuncSetAttribute(tc_gemm_kernel<X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Md::SMEM_BYTES);
    if (e != cudaSuccess) return (int)e;
    mark_configured(configured);
  }
  dim3 grid((unsigned)ceil_div(a.N, TN), (unsigned)ceil_div(a.M, TM), (unsigned)a.splits);
  tc_gemm_kernel<X3><<<grid, TC_THREADS, Md::SMEM_BYTES, s>>>(a);
  note_launches(1);
  if (a.splits > 1) return splitk_reduce_f32(a, s);
  return (int)cudaGetLastError();
}

}  // namespace

bool tc_gemm_enabled() { return true; }

// BF16 operands when the arguments ask for BF16 rounding, else 3xTF32
int tc_gemm_run(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return (int)cudaSuccess;
  if (g.sym) return (int)cudaErrorInvalidValue;
  return g.round_bf16 ? tc_launch<false>(g, s) : tc_launch<true>(g, s);
}

}  // namespace bkfac

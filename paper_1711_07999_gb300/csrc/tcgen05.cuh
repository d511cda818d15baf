// tcgen05.cuh -- inline-PTX wrappers for the fifth-generation tensor cores of sm_100a / sm_103a, as used by
// the [J r]^T [J r] contraction: tensor-memory (TMEM) allocation, the shared-memory matrix descriptor,
// tcgen05.mma with FP32 accumulation in TMEM, completion through an mbarrier, and tcgen05.ld of the
// accumulator.  Only the forms this project uses: one CTA per MMA (cta_group::1), M = 128, K-major A and
// B without swizzle, BF16 (kind::f16) or TF32 (kind::tf32) operands.
//
// Operand tile layout in shared memory (K-major, no swizzle).  A tile holds K = CH * T values (T = 16 bytes
// of K: 8 BF16 or 4 TF32) for each of the 128 rows; 8-row groups are stored one after the other, and within
// a group the CH "core matrices" (8 rows x 16 bytes = 128 contiguous bytes each) follow along K:
//   byte(m, k) = (m / 8) * (CH * 128) + (k / T) * 128 + (m % 8) * 16 + (k % T) * sizeof(element).
// In descriptor terms: leading byte offset (next core matrix along K) = 128, stride byte offset (next
// 8-row group along M or N) = CH * 128.  One MMA consumes 32 bytes of K (two core matrices), so the j-th
// MMA step of a tile starts at byte 256 j.  Every address an MMA reads lies inside its tile.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace trk {
namespace tc {

constexpr int kRows = 128;                  // M of every MMA (rows beyond the used columns are padding)
constexpr uint32_t kFmtBF16 = 1;            // A/B format code of kind::f16 for BF16
constexpr uint32_t kFmtTF32 = 2;            // A/B format code of kind::tf32
constexpr uint32_t kTmemCols = 128;         // TMEM columns per CTA (N <= 80 used; power of two >= 32)
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz: bound of every mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier (one arrival per phase: the tcgen05.commit of the MMA-issuing thread) --------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the completion of the phase with the given parity; false if it has not completed within
// kWaitCycles (the caller records the failure and still releases its TMEM).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

// ---- fences ---------------------------------------------------------------------------------
// Makes this thread's generic-proxy shared-memory writes visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- TMEM allocation (executed by one whole warp) -------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- descriptors ----------------------------------------------------------------------------
// Shared-memory matrix descriptor: start address, leading (K-direction) and stride (M/N-direction)
// byte offsets, all encoded >> 4; bits 46-48 hold the fixed value 0b001; base offset 0, relative
// leading-offset mode, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}
// Descriptor of the operand for the j-th MMA step of a tile with ch core matrices along K.
__device__ __forceinline__ uint64_t tile_desc(uint32_t tile_saddr, int j, int ch) {
  return smem_desc(tile_saddr + (uint32_t)(256 * j), 128, (uint32_t)(ch * 128));
}
// Byte offset of the 16-byte piece (row m, core matrix c along K) in a tile with ch core matrices along K.
__host__ __device__ constexpr int tile_offset(int m, int c, int ch) { return (m >> 3) * (ch * 128) + c * 128 + (m & 7) * 16; }
// Instruction descriptor (kind::f16 / kind::tf32): FP32 D, A and B of format fmt, both K-major,
// no negation, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- MMA, commit ----------------------------------------------------------------------------
// D[tmem] (+)= A * B^T over 32 bytes of K; accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives once on bar when every tcgen05 operation this thread issued so far has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// ---- accumulator read-back ------------------------------------------------------------------
// Eight consecutive FP32 columns of TMEM lane (taddr >> 16) + lane of the calling warp; the warp must
// be warp (lane base / 32) mod 4 of its warpgroup.  The values are valid after ld_wait.
__device__ __forceinline__ void ld_x8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
}
// Waits for this thread's tcgen05.ld; the registers are passed through so that no use of them can be
// scheduled before the wait.
__device__ __forceinline__ void ld_wait(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7])::"memory");
}

// ---- operand splitting ------------------------------------------------------------------------
// x = hi + lo + O(2^-16 |x|) with hi, lo BF16 (x - hi is exact in FP32).
__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}
// Round to TF32 (10 stored mantissa bits, nearest, ties away from zero), kept as an FP32 bit pattern.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo + O(2^-21 |x|) with hi, lo TF32.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

// ---- split-precision operands ----------------------------------------------------------------
// PREC 1: split-BF16x3 on kind::f16; PREC 2: 3xTF32 on kind::tf32.  Each FP32 value x of [J r] is
// stored as hi + lo; a product x_a x_b is formed as hi_a hi_b + hi_a lo_b + lo_a hi_b (three MMAs into
// one FP32 accumulator; lo_a lo_b is dropped).
template <int PREC>
struct Split;

template <>
struct Split<1> {
  static constexpr int T = 8;  // values per 16 bytes of K
  static constexpr uint32_t fmt = kFmtBF16;
  __device__ static void pack(const float (&x)[8], uint4& hi, uint4& lo) {
    uint16_t h[8], l[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) split_bf16(x[t], h[t], l[t]);
    hi = make_uint4(h[0] | (uint32_t)h[1] << 16, h[2] | (uint32_t)h[3] << 16, h[4] | (uint32_t)h[5] << 16,
                    h[6] | (uint32_t)h[7] << 16);
    lo = make_uint4(l[0] | (uint32_t)l[1] << 16, l[2] | (uint32_t)l[3] << 16, l[4] | (uint32_t)l[5] << 16,
                    l[6] | (uint32_t)l[7] << 16);
  }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    mma_bf16(d, a, b, idesc, acc);
  }
};

template <>
struct Split<2> {
  static constexpr int T = 4;
  static constexpr uint32_t fmt = kFmtTF32;
  __device__ static void pack(const float (&x)[4], uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) split_tf32(x[t], h[t], l[t]);
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    mma_tf32(d, a, b, idesc, acc);
  }
};

constexpr int kChunkRows = 64;  // rows of [J r] per operand tile of the standalone contraction

// Operand tiles with CH core matrices along K (K = CH * T rows of [J r]), 128 rows (M).
template <int PREC, int CH_>
struct Tile {
  static constexpr int T = Split<PREC>::T;
  static constexpr int CH = CH_;
  static constexpr int K = CH * T;                       // rows of [J r] per tile
  static constexpr int BYTES = (kRows / 8) * CH * 128;  // one operand tile (hi or lo)
  static constexpr int STAGE = 2 * BYTES;               // hi tile, then lo tile
};

// Issues the MMAs of one staged chunk: nsteps steps of 2T rows, three products each.
template <int PREC, int CH>
__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint32_t hi, uint32_t lo, int nsteps, uint32_t idesc,
                                            bool overwrite) {
  for (int j = 0; j < nsteps; ++j) {
    const uint64_t ah = tile_desc(hi, j, CH), al = tile_desc(lo, j, CH);
    Split<PREC>::mma(tmem, ah, ah, idesc, (overwrite && j == 0) ? 0u : 1u);
    Split<PREC>::mma(tmem, ah, al, idesc, 1u);
    Split<PREC>::mma(tmem, al, ah, idesc, 1u);
  }
}

// Zeroes rows [nc, 128) of n_tiles consecutive operand tiles (the M padding; never written again).
template <int PREC, int CH, int NT>
__device__ __forceinline__ void zero_padding(unsigned char* tiles, int n_tiles, int nc) {
  const int per_tile = (kRows - nc) * CH;
  for (int e = threadIdx.x; e < n_tiles * per_tile; e += NT) {
    const int t = e / per_tile, r = e % per_tile;
    *reinterpret_cast<uint4*>(tiles + t * Tile<PREC, CH>::BYTES + tile_offset(nc + r / CH, r % CH, CH)) =
        make_uint4(0u, 0u, 0u, 0u);
  }
}

// Splits rows [0, kq) of a chunk (kq a multiple of 2T; src(k, m) = 0 for rows past the data) for the
// columns m < nc into the hi and lo tiles at stage.
template <int PREC, int CH, int NT, class Src>
__device__ __forceinline__ void stage_chunk(const Src& src, int kq, int nc, unsigned char* stage) {
  constexpr int T = Split<PREC>::T;
  const int items = nc * (kq / T);
  for (int q = threadIdx.x; q < items; q += NT) {
    const int m = q % nc, c = q / nc;
    float x[T];
#pragma unroll
    for (int t = 0; t < T; ++t) x[t] = src(c * T + t, m);
    uint4 hi, lo;
    Split<PREC>::pack(x, hi, lo);
    const int off = tile_offset(m, c, CH);
    *reinterpret_cast<uint4*>(stage + off) = hi;
    *reinterpret_cast<uint4*>(stage + Tile<PREC, CH>::BYTES + off) = lo;
  }
}

}  // namespace tc
}  // namespace trk

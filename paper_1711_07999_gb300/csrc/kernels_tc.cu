// kernels_tc.cu -- the contraction [J r]^T [J r] (Eqs. JTJ, JTr) of materialised FP32 rows on the tensor
// cores: split-BF16x3 (kind::f16) or 3xTF32 (kind::tf32) products accumulated in FP32 in tensor memory,
// the CTA partials kept with Kahan compensation and added across CTAs in FP64 in a fixed order.
//
// One CTA of 128 threads per contiguous row range.  Rows are taken 64 at a time: the threads load a
// 64 x nc block (coalesced along the columns), split every value into hi + lo and store both into a
// K-major operand tile (parameter m = MMA row, data row = K); one thread issues the MMAs of the chunk
// (A = B = the tile: D[m][n] += sum_k x_km x_kn) and commits them to the chunk's mbarrier, so the
// next chunk is staged in the other buffer while the tensor core works.  Every 8 chunks the FP32
// accumulator is drained from TMEM into per-thread Kahan sums (thread m owns row m of D).
#include <algorithm>

#include "../../include/trk.h"
#include "tcgen05.cuh"
#include "trk_internal.cuh"

namespace trk {

constexpr int kTcThreads = 128;
constexpr int kTcDrain = 8;          // chunks accumulated in TMEM between drains (512 rows)
constexpr int kTcMaxBlocks = 296;

template <int PREC, int NB>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_jtj_rows_tc(const float* __restrict__ rows, int n, int nc, int ld, int rows_per_block,
                  float* __restrict__ partial) {
  using TL = tc::Tile<PREC, tc::kChunkRows / tc::Split<PREC>::T>;
  constexpr int N = 16 * NB, T = TL::T;
  extern __shared__ __align__(1024) unsigned char smem[];  // two stages of (hi tile, lo tile)
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(n, r0 + rows_per_block);
  const int nrows = max(0, r1 - r0);
  const int nchunks = (nrows + tc::kChunkRows - 1) / tc::kChunkRows;

  tc::zero_padding<PREC, TL::CH, kTcThreads>(smem, 4, nc);
  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    tc::fence_mbar_init();
  }
  if (w == 0) tc::tmem_alloc(&tslot, tc::kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t idesc = tc::instr_desc(tc::Split<PREC>::fmt, tc::kRows, N);
  const uint32_t sbase = tc::smem_u32(smem);

  float s[N], c[N];
#pragma unroll
  for (int k = 0; k < N; ++k) s[k] = c[k] = 0.f;
  bool ok = true;
  int pending = 0;  // chunks in TMEM since the last drain
  for (int q = 0; q < nchunks; ++q) {
    const int st = q & 1;
    if (q >= 2) {  // the MMAs of chunk q - 2 read this stage
      ok &= tc::mbar_wait(&bars[st], ((q - 2) >> 1) & 1);
      tc::fence_proxy_async();
    }
    const int base = r0 + q * tc::kChunkRows;
    const int cnt = min(tc::kChunkRows, r1 - base);
    const int kq = (cnt + 2 * T - 1) / (2 * T) * (2 * T);
    const float* blk = rows + (size_t)base * ld;
    tc::stage_chunk<PREC, TL::CH, kTcThreads>(
        [&](int k, int m) { return k < cnt ? __ldg(blk + (size_t)k * ld + m) : 0.f; }, kq, nc,
        smem + st * TL::STAGE);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t hi = sbase + st * TL::STAGE;
      tc::issue_chunk<PREC, TL::CH>(tmem, hi, hi + TL::BYTES, kq / (2 * T), idesc, pending == 0);
      tc::commit(&bars[st]);
    }
    ++pending;
    if (pending == kTcDrain || q == nchunks - 1) {
      ok &= tc::mbar_wait(&bars[st], (q >> 1) & 1);
      tc::fence_after_sync();
#pragma unroll
      for (int g = 0; g < N / 8; ++g) {
        uint32_t r[8];
        tc::ld_x8(tmem + ((uint32_t)(32 * w) << 16) + 8 * g, r);
        tc::ld_wait(r);
#pragma unroll
        for (int t = 0; t < 8; ++t) {  // Kahan: s - c carries the sum
          const float y = __uint_as_float(r[t]) - c[8 * g + t];
          const float u = s[8 * g + t] + y;
          c[8 * g + t] = (u - s[8 * g + t]) - y;
          s[8 * g + t] = u;
        }
      }
      tc::fence_before_sync();
      __syncthreads();  // every warp has read D before the next chunk's first MMA overwrites it
      pending = 0;
    }
  }
  // row m of D goes to column m of the two partial slots (coalesced): sum and -compensation
  const int m = 32 * w + lane;
  if (m < nc) {
    float* o0 = partial + (size_t)(2 * blockIdx.x) * nc * nc;
    float* o1 = o0 + (size_t)nc * nc;
    const float bad = __int_as_float(0x7fc00000);
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (k < nc) {
        o0[k * nc + m] = ok ? s[k] : bad;
        o1[k * nc + m] = ok ? -c[k] : bad;
      }
  }
  if (!ok && tid == 0 && nchunks > 0) tc::mbar_wait(&bars[(nchunks - 1) & 1], ((nchunks - 1) >> 1) & 1);
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, tc::kTmemCols);
  }
}

template <int PREC>
static constexpr int tc_rows_smem() {
  return 2 * tc::Tile<PREC, tc::kChunkRows / tc::Split<PREC>::T>::STAGE;
}

template <int PREC>
static cudaError_t launch_rows_tc(const float* rows, int n, int nc, int ld, int nblk, int rpb, float* partial,
                                  cudaStream_t st) {
  const int sm = tc_rows_smem<PREC>();
  switch ((nc + 15) / 16) {
    case 1: k_jtj_rows_tc<PREC, 1><<<nblk, kTcThreads, sm, st>>>(rows, n, nc, ld, rpb, partial); break;
    case 2: k_jtj_rows_tc<PREC, 2><<<nblk, kTcThreads, sm, st>>>(rows, n, nc, ld, rpb, partial); break;
    case 3: k_jtj_rows_tc<PREC, 3><<<nblk, kTcThreads, sm, st>>>(rows, n, nc, ld, rpb, partial); break;
    case 4: k_jtj_rows_tc<PREC, 4><<<nblk, kTcThreads, sm, st>>>(rows, n, nc, ld, rpb, partial); break;
    default: k_jtj_rows_tc<PREC, 5><<<nblk, kTcThreads, sm, st>>>(rows, n, nc, ld, rpb, partial); break;
  }
  return cudaGetLastError();
}

template <int PREC>
static void configure_rows_tc() {
  const int sm = tc_rows_smem<PREC>();
  cudaFuncSetAttribute(k_jtj_rows_tc<PREC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_jtj_rows_tc<PREC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_jtj_rows_tc<PREC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_jtj_rows_tc<PREC, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_jtj_rows_tc<PREC, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

void configure_tc_kernels() {
  configure_rows_tc<1>();
  configure_rows_tc<2>();
}

cudaError_t jtj_reduce_launch(const float* partial, int nslots, int nc, double* out, cudaStream_t st);

}  // namespace trk

extern "C" trk_status trk_jtj_rows_tc(const float* d_rows, int32_t n_rows, int32_t n_cols, int32_t ld,
                                      int32_t precision, double* d_out, void* cuda_stream) {
  if (!d_out || n_cols < 1 || n_cols > trk::kMaxNP || ld < n_cols || n_rows < 0 || (n_rows > 0 && !d_rows))
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_jtj_rows_tc: bad pointer or size");
  if (precision != TRK_PRECISION_BF16X3 && precision != TRK_PRECISION_TF32X3)
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_jtj_rows_tc: precision must be BF16X3 or TF32X3");
  trk::ensure_configured();
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nblk = std::max(1, std::min(trk::kTcMaxBlocks, (n_rows + 255) / 256));
  const int rpb = (n_rows + nblk - 1) / nblk;
  float* partial = nullptr;
  cudaError_t e = cudaMallocAsync(&partial, sizeof(float) * 2 * (size_t)nblk * n_cols * n_cols, st);
  if (e != cudaSuccess) return trk::set_error(TRK_ERR_OOM, "trk_jtj_rows_tc: scratch allocation failed");
  e = precision == TRK_PRECISION_BF16X3
          ? trk::launch_rows_tc<1>(d_rows, n_rows, n_cols, ld, nblk, rpb, partial, st)
          : trk::launch_rows_tc<2>(d_rows, n_rows, n_cols, ld, nblk, rpb, partial, st);
  if (e == cudaSuccess) e = trk::jtj_reduce_launch(partial, 2 * nblk, n_cols, d_out, st);
  const cudaError_t f = cudaFreeAsync(partial, st);
  if (e == cudaSuccess) e = f;
  if (e != cudaSuccess) return trk::set_error(TRK_ERR_CUDA, cudaGetErrorString(e));
  return TRK_OK;
}

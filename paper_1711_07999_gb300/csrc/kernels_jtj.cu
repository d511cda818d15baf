// kernels_jtj.cu -- the contraction [J r]^T [J r] of materialised FP32 rows (Eqs. JTJ, JTr), as a
// standalone operation on caller device buffers.
//
// Each CTA takes a contiguous range of rows, stages them 64 at a time in shared memory and accumulates
// its (16T) x (16T) product in registers (16 x 16 threads, a T x T tile each); the per-CTA partials are
// then added in CTA order in FP64 (deterministic for a given grid).
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/trk.h"
#include "trk_internal.cuh"

namespace trk {

constexpr int kJBlock = 256;
constexpr int kJStage = 64;
constexpr int kJMaxBlocks = 296;

template <int T>
__global__ void __launch_bounds__(kJBlock) k_jtj_rows(const float* __restrict__ rows, int n, int nc, int ld,
                                                     int rows_per_block, float* __restrict__ partial) {
  constexpr int W = 16 * T, ROW = W + 1;
  __shared__ float st[kJStage * ROW];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(n, r0 + rows_per_block);
  float acc[T][T];
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) acc[a][b] = 0.f;
  for (int base = r0; base < r1; base += kJStage) {
    const int cnt = min(kJStage, r1 - base);
    __syncthreads();
    for (int e = tid; e < kJStage * W; e += kJBlock) {
      const int s = e / W, c = e % W;
      st[s * ROW + c] = (s < cnt && c < nc) ? rows[(size_t)(base + s) * ld + c] : 0.f;
    }
    __syncthreads();
    for (int s = 0; s < cnt; ++s) {
      const float* row = st + s * ROW;
      float ra[T], rb[T];
#pragma unroll
      for (int a = 0; a < T; ++a) {
        ra[a] = row[ty * T + a];
        rb[a] = row[tx * T + a];
      }
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) acc[a][b] = fmaf(ra[a], rb[b], acc[a][b]);
    }
  }
  float* out = partial + (size_t)blockIdx.x * nc * nc;
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const int r = ty * T + a, c = tx * T + b;
      if (r < nc && c < nc) out[r * nc + c] = acc[a][b];
    }
}

__global__ void __launch_bounds__(1024) k_jtj_reduce(const float* __restrict__ partial, int nblk, int nc,
                                                     double* __restrict__ out) {
  __shared__ double sm[32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n2 = nc * nc, e = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (e < n2)
    for (int b = w; b < nblk; b += 32) s += (double)partial[(size_t)b * n2 + e];
  sm[w][lane] = s;
  __syncthreads();
  if (w != 0 || e >= n2) return;
  double t = 0.0;
  for (int k = 0; k < 32; ++k) t += sm[k][lane];
  out[e] = t;
}

// Launches the two kernels with nblk CTAs and the given partial buffer (nblk * nc * nc floats).
cudaError_t jtj_rows_launch(const float* rows, int n, int nc, int ld, double* out, int nblk, float* partial,
                            cudaStream_t st) {
  const int T = (nc + 15) / 16;
  const int rpb = (n + nblk - 1) / nblk;
  switch (T) {
    case 1: k_jtj_rows<1><<<nblk, kJBlock, 0, st>>>(rows, n, nc, ld, rpb, partial); break;
    case 2: k_jtj_rows<2><<<nblk, kJBlock, 0, st>>>(rows, n, nc, ld, rpb, partial); break;
    case 3: k_jtj_rows<3><<<nblk, kJBlock, 0, st>>>(rows, n, nc, ld, rpb, partial); break;
    case 4: k_jtj_rows<4><<<nblk, kJBlock, 0, st>>>(rows, n, nc, ld, rpb, partial); break;
    default: k_jtj_rows<5><<<nblk, kJBlock, 0, st>>>(rows, n, nc, ld, rpb, partial); break;
  }
  k_jtj_reduce<<<(nc * nc + 31) / 32, 1024, 0, st>>>(partial, nblk, nc, out);
  return cudaGetLastError();
}

// Fixed-order FP64 sum of nslots partials of nc x nc floats into out.
cudaError_t jtj_reduce_launch(const float* partial, int nslots, int nc, double* out, cudaStream_t st) {
  k_jtj_reduce<<<(nc * nc + 31) / 32, 1024, 0, st>>>(partial, nslots, nc, out);
  return cudaGetLastError();
}

int jtj_rows_blocks(int n) { return std::max(1, std::min(kJMaxBlocks, (n + kJBlock - 1) / kJBlock)); }

// ---------------------------------------------------------------------------------------------
// Allocation-free variant: the per-CTA partials live in a fixed file-scope device array (at most
// kNoAllocBlocks CTAs x 80 x 80 floats, 3.9 MB held by every device that loads the library).  Each CTA
// overwrites its whole partial on every call, so nothing has to be cleared between calls.
// ---------------------------------------------------------------------------------------------
constexpr int kNoAllocBlocks = 152;
static __device__ __align__(256) float g_noalloc_partial[kNoAllocBlocks * kMaxNP * kMaxNP];

constexpr int kMaxDevices = 64;
static float* g_noalloc_ptr[kMaxDevices];
static std::mutex g_noalloc_mutex;

// Device address of g_noalloc_partial on the current device (looked up once per device).  In host code
// the symbol itself is only a host-side stand-in, never a device address.
static cudaError_t noalloc_scratch(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    float* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_partial);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace trk

extern "C" {

trk_status trk_jtj_rows(const float* d_rows, int32_t n_rows, int32_t n_cols, int32_t ld, double* d_out,
                        void* cuda_stream) {
  if (!d_rows || !d_out || n_rows < 0 || n_cols <= 0 || n_cols > trk::kMaxNP || ld < n_cols)
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_jtj_rows: bad arguments");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nblk = trk::jtj_rows_blocks(n_rows);
  float* partial = nullptr;
  cudaError_t e = cudaMallocAsync(&partial, sizeof(float) * (size_t)nblk * n_cols * n_cols, st);
  if (e != cudaSuccess)
    return trk::set_error(e == cudaErrorMemoryAllocation ? TRK_ERR_OOM : TRK_ERR_CUDA, cudaGetErrorString(e));
  e = trk::jtj_rows_launch(d_rows, n_rows, n_cols, ld, d_out, nblk, partial, st);
  const cudaError_t f = cudaFreeAsync(partial, st);
  if (e != cudaSuccess) return trk::set_error(TRK_ERR_CUDA, cudaGetErrorString(e));
  if (f != cudaSuccess) return trk::set_error(TRK_ERR_CUDA, cudaGetErrorString(f));
  return TRK_OK;
}

trk_status trk_jtj_rows_noalloc(const float* d_rows, int32_t n_rows, int32_t n_cols, int32_t ld, double* d_out,
                                void* cuda_stream) {
  if (!d_rows || !d_out || n_rows < 0 || ld < n_cols)
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_jtj_rows_noalloc: bad arguments");
  if (n_cols <= 0 || n_cols > trk::kMaxNP)
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_jtj_rows_noalloc: n_cols must be in [1, 80] (fixed scratch size)");
  float* partial = nullptr;
  cudaError_t e = trk::noalloc_scratch(&partial);
  if (e != cudaSuccess) return trk::set_error(TRK_ERR_CUDA, cudaGetErrorString(e));
  const int nblk = std::min(trk::kNoAllocBlocks, trk::jtj_rows_blocks(n_rows));
  e = trk::jtj_rows_launch(d_rows, n_rows, n_cols, ld, d_out, nblk, partial, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return trk::set_error(TRK_ERR_CUDA, cudaGetErrorString(e));
  return TRK_OK;
}

}  // extern "C"

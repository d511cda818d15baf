// kernels_solve.cu -- point-to-plane residuals and the pose Jacobian (Eq. residual, Sec. 4.2), the
// reduction [J r]^T [J r] (Eqs. JTJ, JTr), the damped least-squares step with the pose prior and its
// energy test (Sec. 4.2), and the per-vertex shape step (Eq. r_warp, Sec. 4.3).
//
// Reductions are deterministic: per-block partial sums over fixed vertex ranges, then a second pass
// that adds the partials in a fixed order (error-free FP32 within a warp, FP64 across warps).  The LM
// retries of one iteration (damping lambda, 10 lambda, ..., 10^5 lambda) are solved side by side, one CTA
// each, and their energies evaluated over the vertices; the first candidate that does not raise the
// energy is taken on the device, which gives the same result as trying them one after the other without
// any host round trip.
#include <mutex>

#include "tcgen05.cuh"
#include "trk_internal.cuh"

namespace trk {

constexpr int kBlock = 256;

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// L(c, h) = -c_w h_vec + h_w c_vec + h_vec x c_vec: for a pure quaternion (0, xi),
// <c, (0, xi) h> = xi . L(c, h).
__device__ __forceinline__ float3 Lfun(float4 c, float4 h) {
  return make_float3(-c.x * h.y + h.x * c.y + (h.z * c.w - h.w * c.z),
                     -c.x * h.z + h.x * c.z + (h.w * c.y - h.y * c.w),
                     -c.x * h.w + h.x * c.w + (h.y * c.z - h.z * c.y));
}

// ---------------------------------------------------------------------------------------------
// Residual r_i = n_i . (p~_i - v_i) and Jacobian row dr_i/dTheta for every vertex of A, followed by
// the block's partial [J r]^T [J r].
//
// Jacobian: with c = n^T dT/dH (an 8-vector: the normal pulled back through the homogeneous point map
// at H_iSigma) and dH_iSigma/dtheta_k = sum_b w_b s_b Xi_k H_{b,Delta} over the bones b below k,
//   J_ik = -sum_b w_b s_b <c, Xi_k H_{b,Delta}> = -sum_b Xi_k . e_b,
//   e_b = w_b s_b (L(c_r, h_r) + L(c_d, h_d), L(c_d, h_r)),
// so each bone costs one 6-vector and each ancestor link one 6-term dot product.
//   c_r = (-2 N a X - 2 N b - 2 (n.v) a) / |a|^2,  c_d = 2 N a / |a|^2,  N = (0, n), X = (0, x).
// The block's rows (compacted to A) are staged in shared memory; 16 x 16 threads each own a TxT tile
// of the (16T) x (16T) product and sweep the rows.
// ---------------------------------------------------------------------------------------------
// Copies the link tables this block needs (H_Delta, Xi, parents) to shared memory.
__device__ __forceinline__ void load_link_tables(const Dev& d, DQ* sHd, float* sXi, int* sPar) {
  for (int j = threadIdx.x; j < d.L; j += kBlock) {
    sHd[j] = d.Hd[j];
    for (int c = 0; c < 6; ++c) sXi[6 * j + c] = d.xi[8 * j + c];
    sPar[j] = d.links->parent[j];
  }
}

// This block's vertices in A (c_i >= 1 and a valid normal) and each one's row slot, compacted in vertex
// order, with every input of the vertex's row (all loaded at once: one round trip, the point data of
// vertices outside A read and dropped).  Contains a __syncthreads; returns the number of rows (the same
// in every thread).
struct RowSlot {
  int i, slot, base;  // vertex, its row among the vertex block's rows, the record index of row 0
  bool inA;
  Acc4 a4;
  float4 nn, v, x0, ph, bw;
  uchar4 bi;
};
__device__ __forceinline__ int block_rows(const Dev& d, int blk, int row_base, int phi_buf, int* s_warp,
                                         RowSlot& rs) {
  const int tid = threadIdx.x;
  rs.i = blk * kBlock + tid;
  rs.base = row_base;
  rs.inA = false;
  rs.a4 = Acc4{0, 0, 0, 0};
  rs.nn = make_float4(0.f, 0.f, 0.f, 0.f);
  rs.v = rs.x0 = rs.ph = rs.bw = rs.nn;
  rs.bi = make_uchar4(0, 0, 0, 0);
  if (rs.i < d.V) {
    rs.a4 = d.acc[rs.i];
    rs.nn = d.n[rs.i];
    rs.v = d.v[rs.i];
    rs.x0 = d.v0[rs.i];
    rs.ph = d.phi[phi_buf][rs.i];
    rs.bi = d.bidx[rs.i];
    rs.bw = d.bw[rs.i];
    rs.inA = rs.a4.w >= 1 && rs.nn.w > 0.f;
  }
  const unsigned m = __ballot_sync(0xffffffffu, rs.inA);
  const int lane = tid & 31, w = tid >> 5;
  if (lane == 0) s_warp[w] = __popc(m);
  __syncthreads();
  int off = 0, total = 0;
  for (int k = 0; k < kBlock / 32; ++k) {
    off += k < w ? s_warp[k] : 0;
    total += s_warp[k];
  }
  rs.slot = off + __popc(m & ((1u << lane) - 1u));
  return total;
}

// Writes this thread's [J r] row (if its vertex is in A) to Js row rs.slot (stride ROW, columns
// [0, width) with width >= NP, zero beyond NP) and sets r2 = r_i^2 (0 outside A).  The link tables must
// be in shared memory; the caller synchronises before reading Js.
__device__ __forceinline__ void jacobian_row(const Dev& d, const RowSlot& rs, int phi_buf, float* Js, int ROW,
                                             int width, const DQ* sHd, const float* sXi, const int* sPar, float& r2) {
  r2 = 0.f;
  if (!rs.inA) return;
  const Acc4 a4 = rs.a4;
  float* row = Js + rs.slot * ROW;
  if ((ROW & 3) == 0 && (width & 3) == 0) {  // 16-byte rows: 128-bit stores
    for (int k = 0; k < width; k += 4) *reinterpret_cast<float4*>(row + k) = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    for (int k = 0; k < width; ++k) row[k] = 0.f;
  }
  const float inv = 1.f / ((float)a4.w * kFix);
  const float3 pm = make_float3((float)a4.x * inv, (float)a4.y * inv, (float)a4.z * inv);
  const float3 n = f3(rs.nn);
  const float r = dot3(n, pm);
  row[d.L] = r;
  r2 = r * r;
  float sg[4];
  const uchar4 bi = rs.bi;
  const float4 bw = rs.bw;
  const DQ H = blend_bones(sHd, bi, bw, sg);
  const float4 x0 = rs.x0, ph = rs.ph, v = rs.v;
  const float4 X = make_float4(0.f, x0.x + ph.x, x0.y + ph.y, x0.z + ph.z);
  {  // the row's record for the candidate energies: p~ = v + pm, n, x = x0 + phi, bones and weights
    float4* rec = d.arec + (size_t)(rs.base + rs.slot) * 4;
    unsigned bits;
    memcpy(&bits, &bi, 4);
    rec[0] = make_float4(v.x + pm.x, v.y + pm.y, v.z + pm.z, n.x);
    rec[1] = make_float4(n.y, n.z, X.y, X.z);
    rec[2] = make_float4(X.w, bw.x, bw.y, bw.z);
    rec[3] = make_float4(bw.w, __uint_as_float(bits), 0.f, 0.f);
  }
  const float4 Np = make_float4(0.f, n.x, n.y, n.z);
  const float invN = 1.f / qdot(H.r, H.r);
  const float4 Na = qmul(Np, H.r);
  const float4 cr = qscale(qadd(qadd(qmul(Na, X), qmul(Np, H.d)), qscale(H.r, dot3(n, f3(v)))), -2.f * invN);
  const float4 cd = qscale(Na, 2.f * invN);
  const int idx[4] = {bi.x, bi.y, bi.z, bi.w};
  const float ws[4] = {bw.x, bw.y, bw.z, bw.w};
  // e_b of every weighted bone, keyed by its link (-1: no weight)
  int key[4];
  float es[4][6];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    key[s] = -1;
#pragma unroll
    for (int c = 0; c < 6; ++c) es[s][c] = 0.f;
    if (!(ws[s] > 0.f)) continue;
    key[s] = idx[s];
    const DQ h = sHd[idx[s]];
    const float sc = ws[s] * sg[s];
    const float3 e1 = Lfun(cr, h.r), e2 = Lfun(cd, h.d), e3 = Lfun(cd, h.r);
    es[s][0] = sc * (e1.x + e2.x);
    es[s][1] = sc * (e1.y + e2.y);
    es[s][2] = sc * (e1.z + e2.z);
    es[s][3] = sc * e3.x;
    es[s][4] = sc * e3.y;
    es[s][5] = sc * e3.z;
  }
  // J_ik = -Xi_k . (sum of e_b over the bones b at or below k).  The bones, sorted by link (parents
  // precede their children), are walked to the root from the deepest one; a bone met on the way joins
  // the running sum, so a link shared by several bones' chains is visited once.  A bone on another
  // branch is not met and starts its own walk afterwards (sums are linear, so every bone still reaches
  // each of its ancestors exactly once).
  auto cswap = [&](int a, int b) {
    if (key[a] < key[b]) {
      const int t = key[a];
      key[a] = key[b];
      key[b] = t;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float u = es[a][c];
        es[a][c] = es[b][c];
        es[b][c] = u;
      }
    }
  };
  cswap(0, 1);
  cswap(2, 3);
  cswap(0, 2);
  cswap(1, 3);
  cswap(1, 2);
  auto pop = [&]() {  // drops the head of the sorted queue
    key[0] = key[1];
    key[1] = key[2];
    key[2] = key[3];
    key[3] = -1;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      es[0][c] = es[1][c];
      es[1][c] = es[2][c];
      es[2][c] = es[3][c];
    }
  };
  while (key[0] >= 0) {
    int k = key[0];
    float E[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) E[c] = es[0][c];
    pop();
    for (; k >= 0; k = sPar[k]) {
      while (key[0] == k) {
#pragma unroll
        for (int c = 0; c < 6; ++c) E[c] += es[0][c];
        pop();
      }
      const float* xk = sXi + 6 * k;
      row[k] -= xk[0] * E[0] + xk[1] * E[1] + xk[2] * E[2] + xk[3] * E[3] + xk[4] * E[4] + xk[5] * E[5];
    }
  }
}

// Row stride of the staged rows: 16T columns, padded so that rows of even T start on 16 bytes (vector loads
// of a tile's T entries) and rows of odd T fall on distinct banks.
__host__ __device__ constexpr int jtj_row_stride(int T) { return 16 * T + (T % 2 == 0 ? 4 : 1); }
constexpr int kMaxRowGroups = 4;

// Packed FP32 pairs: fma.rn.f32x2 rounds each lane as fmaf does, so a tile updated pairwise holds the same
// bits as one updated entry by entry.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ void f2_fma(unsigned long long& acc, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

// One thread's T x T tile of the product: acc[a][b] += ra[a] rb[b] over the rows it sweeps.
template <int T>
struct TileAcc {
  static constexpr bool kPaired = T % 2 == 0;
  unsigned long long p[kPaired ? T : 1][kPaired ? T / 2 : 1];
  float f[kPaired ? 1 : T][kPaired ? 1 : T];
  __device__ __forceinline__ void zero() {
    if constexpr (kPaired) {
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T / 2; ++b) p[a][b] = 0ull;
    } else {
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) f[a][b] = 0.f;
    }
  }
  // adds one staged row: entries [ty T, ty T + T) and [tx T, tx T + T)
  __device__ __forceinline__ void add_row(const float* row, int ty, int tx) {
    float ra[T], rb[T];
    if constexpr (T == 4) {
      const float4 A = *reinterpret_cast<const float4*>(row + ty * 4);
      const float4 B = *reinterpret_cast<const float4*>(row + tx * 4);
      ra[0] = A.x, ra[1] = A.y, ra[2] = A.z, ra[3] = A.w;
      rb[0] = B.x, rb[1] = B.y, rb[2] = B.z, rb[3] = B.w;
    } else {
#pragma unroll
      for (int a = 0; a < T; ++a) {
        ra[a] = row[ty * T + a];
        rb[a] = row[tx * T + a];
      }
    }
    if constexpr (kPaired) {
      unsigned long long B2[T / 2];
#pragma unroll
      for (int b = 0; b < T / 2; ++b) B2[b] = f2_pack(rb[2 * b], rb[2 * b + 1]);
#pragma unroll
      for (int a = 0; a < T; ++a) {
        const unsigned long long A2 = f2_pack(ra[a], ra[a]);
#pragma unroll
        for (int b = 0; b < T / 2; ++b) f2_fma(p[a][b], A2, B2[b]);
      }
    } else {
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) f[a][b] = fmaf(ra[a], rb[b], f[a][b]);
    }
  }
  __device__ __forceinline__ float get(int a, int b) const {
    if constexpr (kPaired) {
      float lo, hi;
      f2_unpack(p[a][b / 2], lo, hi);
      return (b & 1) ? hi : lo;
    } else {
      return f[a][b];
    }
  }
  __device__ __forceinline__ void add(int a, int b, float x) {
    if constexpr (kPaired) {
      float lo, hi;
      f2_unpack(p[a][b / 2], lo, hi);
      if (b & 1) hi += x; else lo += x;
      p[a][b / 2] = f2_pack(lo, hi);
    } else {
      f[a][b] += x;
    }
  }
};

// Every input of vertex i's row (RowSlot of a vertex known to be in A; slot and base set by the caller).
__device__ __forceinline__ void row_inputs(const Dev& d, int i, int phi_buf, RowSlot& rs) {
  rs.i = i;
  rs.inA = true;
  rs.a4 = d.acc[i];
  rs.nn = d.n[i];
  rs.v = d.v[i];
  rs.x0 = d.v0[i];
  rs.ph = d.phi[phi_buf][i];
  rs.bi = d.bidx[i];
  rs.bw = d.bw[i];
}

// A [J r] block covers jtj_group consecutive blocks of 256 vertices.  Its vertices in A are listed first,
// in vertex order (a vertex's thread tests c_i >= 1 and a valid normal: two small loads), and their rows
// are then formed 256 at a time by consecutive threads -- every thread of a chunk holds a row, instead of
// the third of a vertex block's threads whose vertices are in A -- staged, and added to the same tiles,
// so the block writes one partial for up to 256 G rows.
// The symmetric product needs only the tiles (ty, tx) with ty <= tx among the nt x nt tiles that hold
// columns < NP; S groups of nt (nt + 1) / 2 threads (S = 2 for NP <= 60 at T = 4) each sweep every S-th
// staged row, and the first group adds the other groups' tiles, in group order, before the block writes
// its partial: a fixed order, so the partial is the same in any launch.
template <int T>
__device__ __forceinline__ void resid_jtj_impl(const Dev& d, BlockPos bp, int phi_buf) {
  constexpr int ROW = jtj_row_stride(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Js = reinterpret_cast<float*>(smem_raw);
  DQ* sHd = reinterpret_cast<DQ*>(Js + kBlock * ROW);
  float* sXi = reinterpret_cast<float*>(sHd + d.L);
  int* sPar = reinterpret_cast<int*>(sXi + 6 * d.L);
  __shared__ int s_cnt[kMaxJtjGroup * (kBlock / 32)];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, G = d.jtj_group;
  const int NP = d.NP;
  const int nt = (NP + T - 1) / T;
  const int ntiles = nt * (nt + 1) / 2;
  const int S = min(kMaxRowGroups, kBlock / ntiles);
  const int h = tid / ntiles;  // this thread's row group (h >= S: idle in the product)
  int ty = 0, k = tid - h * ntiles;
  while (ty < nt && k >= nt - ty) {  // the k-th tile of the upper triangle, row-major
    k -= nt - ty;
    ++ty;
  }
  const int tx = ty + k;
  // the block's rows: membership of A of vertex tid of each vertex block, counted per (block, warp)
  unsigned m[kMaxJtjGroup];
#pragma unroll
  for (int sub = 0; sub < kMaxJtjGroup; ++sub) {
    const int i = (bp.x * G + sub) * kBlock + tid;
    bool inA = false;
    if (sub < G && i < d.V) inA = d.acc[i].w >= 1 && d.n[i].w > 0.f;
    m[sub] = __ballot_sync(0xffffffffu, inA);
    if (lane == 0) s_cnt[sub * (kBlock / 32) + w] = __popc(m[sub]);
  }
  load_link_tables(d, sHd, sXi, sPar);
  __syncthreads();
  int total = 0;
  for (int q = 0; q < G * (kBlock / 32); ++q) total += s_cnt[q];
  if (total == 0) {  // nothing to add: the reduction skips this block's (unwritten) partial
    if (tid == 0) d.jtj_rows[bp.x] = 0;
    return;
  }
  {  // the list, in vertex order, staged where the rows go (each thread takes its entries before any row)
    int* s_idx = reinterpret_cast<int*>(Js);
    int off = 0;
#pragma unroll
    for (int sub = 0; sub < kMaxJtjGroup; ++sub) {
      if (sub >= G) break;
      int before = off;
      for (int q = sub * (kBlock / 32); q < sub * (kBlock / 32) + w; ++q) before += s_cnt[q];
      if ((m[sub] >> lane) & 1u) s_idx[before + __popc(m[sub] & ((1u << lane) - 1u))] = (bp.x * G + sub) * kBlock + tid;
      for (int q = 0; q < kBlock / 32; ++q) off += s_cnt[sub * (kBlock / 32) + q];
    }
  }
  __syncthreads();
  int mine[kMaxJtjGroup];
#pragma unroll
  for (int c = 0; c < kMaxJtjGroup; ++c) mine[c] = c * kBlock + tid < total ? reinterpret_cast<const int*>(Js)[c * kBlock + tid] : -1;
  __syncthreads();
  TileAcc<T> acc;
  acc.zero();
#pragma unroll
  for (int c = 0; c < kMaxJtjGroup; ++c) {
    const int c0 = c * kBlock;
    if (c0 >= total) break;
    const int rows = min(kBlock, total - c0);
    if (c > 0) __syncthreads();  // the previous chunk's rows have been added
    if (mine[c] >= 0) {
      RowSlot rs;
      row_inputs(d, mine[c], phi_buf, rs);
      rs.slot = tid;
      rs.base = bp.x * kBlock * G + c0;
      float r2;
      jacobian_row(d, rs, phi_buf, Js, ROW, 16 * T, sHd, sXi, sPar, r2);
    }
    __syncthreads();
    if (h < S)
      for (int s = h; s < rows; s += S) acc.add_row(Js + s * ROW, ty, tx);
  }
  const int done = total;
  if (S > 1) {  // the groups' tiles, added into group 0's in group order
    __syncthreads();  // every group's sweep is done: the staged rows are free
    float* red = Js;
    if (h >= 1 && h < S)
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) red[((h - 1) * T * T + a * T + b) * ntiles + (tid - h * ntiles)] = acc.get(a, b);
    __syncthreads();
    if (h == 0)
      for (int g2 = 1; g2 < S; ++g2)
#pragma unroll
        for (int a = 0; a < T; ++a)
#pragma unroll
          for (int b = 0; b < T; ++b) acc.add(a, b, red[((g2 - 1) * T * T + a * T + b) * ntiles + tid]);
  }
  if (h == 0) {
    float* out = d.partial + (size_t)bp.x * NP * NP;
#pragma unroll
    for (int a = 0; a < T; ++a)
#pragma unroll
      for (int b = 0; b < T; ++b) {
        const int r = ty * T + a, c = tx * T + b;
        if (r < NP && c < NP && r <= c) out[r * NP + c] = acc.get(a, b);  // the upper triangle (the reduction mirrors)
      }
  }
  if (tid == 0) {
    d.jtj_rows[bp.x] = done;
    atomicAdd(&d.stats[1], done);
  }
}

template <int T>
__global__ void __launch_bounds__(kBlock, 3) k_resid_jtj(BatchGrid g, Dev d0, int phi_buf) {
  if (g.map == nullptr) {
    resid_jtj_impl<T>(d0, grid_pos(), phi_buf);
    return;
  }
  __shared__ Dev sd;
  resid_jtj_impl<T>(sd, batch_block(g, sd), phi_buf);
}

// ---------------------------------------------------------------------------------------------
// The same rows contracted on the tensor cores (split-BF16x3 or 3xTF32, PREC 1 / 2): the block's rows
// are taken in chunks of TL::K (64 BF16 / 32 TF32 rows), split into hi + lo K-major tiles and multiplied
// by one issuing thread into an FP32 accumulator in tensor memory (128 lanes x N columns; lane = parameter
// a, column = parameter b).  The energy entry [r]^T [r] is summed on the FP32 cores instead, so that the
// LM acceptance test compares energies formed the same way in every precision mode.  One stage of tiles
// (the next chunk waits for the previous chunk's MMAs) keeps the block at ~105 KB of shared memory, two
// blocks per SM; their 2 x 128 TMEM columns fit the 512 of an SM, so tcgen05.alloc never waits.
// ---------------------------------------------------------------------------------------------
template <int PREC, int NB>
__device__ __forceinline__ void resid_jtj_tc_impl(const Dev& d, BlockPos bp, int phi_buf) {
  using TL = tc::Tile<PREC, 8>;
  constexpr int N = 16 * NB, ROW = N + 1, T = TL::T;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* tiles = smem_raw;  // hi tile, lo tile
  float* Js = reinterpret_cast<float*>(smem_raw + TL::STAGE);
  DQ* sHd = reinterpret_cast<DQ*>(Js + kBlock * ROW);
  float* sXi = reinterpret_cast<float*>(sHd + d.L);
  int* sPar = reinterpret_cast<int*>(sXi + 6 * d.L);
  __shared__ int s_warp[kBlock / 32];
  __shared__ float s_e[kBlock / 32];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int NP = d.NP, G = d.jtj_group;
  // The rows of the block's G vertex blocks go into the same TMEM accumulator, chunk after chunk; the
  // tensor memory is taken when the first rows appear (a block without rows takes none).
  int done = 0, gq = 0;  // rows added, chunks issued
  float E = 0.f;
  bool ok = true, taken = false;
  uint32_t tmem = 0;
  const uint32_t idesc = tc::instr_desc(tc::Split<PREC>::fmt, tc::kRows, N);
  const uint32_t hi = tc::smem_u32(tiles);
  for (int sub = 0; sub < G; ++sub) {
    const int vb = bp.x * G + sub;
    if (vb * kBlock >= d.V) break;
    RowSlot rs;
    const int total = block_rows(d, vb, bp.x * kBlock * G + done, phi_buf, s_warp, rs);
    if (total == 0) {
      __syncthreads();  // s_warp is rewritten by the next vertex block
      continue;
    }
    if (!taken) {
      tc::zero_padding<PREC, TL::CH, kBlock>(tiles, 2, NP);
      if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
      }
      if (w == 0) tc::tmem_alloc(&tslot, tc::kTmemCols);
      load_link_tables(d, sHd, sXi, sPar);
      taken = true;
    }
    __syncthreads();
    float r2;
    jacobian_row(d, rs, phi_buf, Js, ROW, NP, sHd, sXi, sPar, r2);
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if (lane == 0) s_e[w] = r2;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tmem = tslot;
    for (int k = 0; k < kBlock / 32; ++k) E += s_e[k];
    const int nchunks = (total + TL::K - 1) / TL::K;
    for (int q = 0; q < nchunks; ++q, ++gq) {
      if (gq > 0) {  // the previous chunk's MMAs read the tiles
        ok &= tc::mbar_wait(&bar, (gq - 1) & 1);
        tc::fence_proxy_async();
      }
      const int base = q * TL::K, cnt = min(TL::K, total - base);
      const int kq = (cnt + 2 * T - 1) / (2 * T) * (2 * T);
      const float* blk = Js + base * ROW;
      tc::stage_chunk<PREC, TL::CH, kBlock>([&](int k, int m) { return k < cnt ? blk[k * ROW + m] : 0.f; }, kq, NP,
                                            tiles);
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        tc::issue_chunk<PREC, TL::CH>(tmem, hi, hi + TL::BYTES, kq / (2 * T), idesc, gq == 0);
        tc::commit(&bar);
      }
    }
    done += total;
  }
  if (!taken) {  // nothing to add: no TMEM was taken and the reduction skips this block
    if (tid == 0) d.jtj_rows[bp.x] = 0;
    return;
  }
  const int nchunks = gq;
  if (nchunks > 0) {
    ok &= tc::mbar_wait(&bar, (nchunks - 1) & 1);
    tc::fence_after_sync();
  }
  // warps w and w + 4 read the same 32 TMEM lanes (parameters a), alternate 8-column groups (b)
  float* out = d.partial + (size_t)bp.x * NP * NP;
  const int a = 32 * (w & 3) + lane;
  const float bad = __int_as_float(0x7fc00000);
  for (int g = w >> 2; g < N / 8; g += 2) {
    uint32_t r[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (nchunks > 0) {
      tc::ld_x8(tmem + ((uint32_t)(32 * (w & 3)) << 16) + 8 * g, r);
      tc::ld_wait(r);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int b = 8 * g + t;
      if (a < NP && b < NP && a <= b)  // the upper triangle (the reduction mirrors)
        out[a * NP + b] = (a == NP - 1 && b == NP - 1) ? E : (ok ? __uint_as_float(r[t]) : bad);
    }
  }
  if (!ok && tid == 0) {
    atomicExch(&d.stats[3], 1);
    tc::mbar_wait(&bar, (nchunks - 1) & 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, tc::kTmemCols);
  }
  if (tid == 0) {
    d.jtj_rows[bp.x] = done;
    atomicAdd(&d.stats[1], done);
  }
}

template <int PREC, int NB>
__global__ void __launch_bounds__(kBlock) k_resid_jtj_tc(BatchGrid g, Dev d0, int phi_buf) {
  if (g.map == nullptr) {
    resid_jtj_tc_impl<PREC, NB>(d0, grid_pos(), phi_buf);
    return;
  }
  __shared__ Dev sd;
  resid_jtj_tc_impl<PREC, NB>(sd, batch_block(g, sd), phi_buf);
}

// Fixed-order sum of the block partials -> [J r]^T [J r]; the last entry gives E_pose (with the prior
// sum_k (lambda_s S_kk theta_k)^2), recorded as this iteration's energy and as the LM reference.
// A CTA owns 32 consecutive entries (coalesced lanes); its 32 warps take every 32nd partial and add them
// in FP32 with an error-free transformation (each addition's rounding error, from Knuth's TwoSum, is
// carried in a second FP32 accumulator: the compensated sum of Ogita, Rump and Oishi, accurate to about
// u |S| + (n u)^2 sum |x| in FP32 unit roundoff u, i.e. as if added in twice the precision).  The FP64
// pipe issues a small fraction of the FP32 rate on this GPU, so it is left to warp 0, which adds the 32
// warp sums (hi + lo) in FP64 in warp order.
constexpr int kReduceThreads = 1024;

__device__ __forceinline__ void sum2_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);  // exact: hi + x = s + e
  hi = s;
  lo += e;
}

__device__ __forceinline__ void reduce_jtj_impl(const Dev& d, BlockPos bp, int slot) {
  __shared__ double sm[kReduceThreads / 32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NP = d.NP, n2 = NP * NP, nu = NP * (NP + 1) / 2;
  // lane -> the u-th entry of the upper triangle, row-major: (r, c), r <= c, at e = r NP + c
  const int u = bp.x * 32 + lane;
  int r = 0, c = 0;
  if (u < nu) {
    int rest = u;
    while (rest >= NP - r) rest -= NP - r++;
    c = r + rest;
  }
  const int e = r * NP + c;
  // warp w < S takes blocks w, w + S, ... (four loads in flight together, each partial loaded with its row
  // count rather than after it); blocks that added no rows wrote no partial and count as zero.  S depends
  // on the session alone, so its sums have the same order in any launch.
  const int nb = d.nblk_rows;
  const int S = reduce_warps(nb);
  float hi = 0.f, lo = 0.f;
  if (u < nu && w < S) {
    int b = w;
    for (; b + 3 * S < nb; b += 4 * S) {
      const int r0 = d.jtj_rows[b], r1 = d.jtj_rows[b + S], r2 = d.jtj_rows[b + 2 * S], r3 = d.jtj_rows[b + 3 * S];
      const float q0 = d.partial[(size_t)b * n2 + e], q1 = d.partial[(size_t)(b + S) * n2 + e];
      const float q2 = d.partial[(size_t)(b + 2 * S) * n2 + e], q3 = d.partial[(size_t)(b + 3 * S) * n2 + e];
      sum2_add(hi, lo, r0 > 0 ? q0 : 0.f);
      sum2_add(hi, lo, r1 > 0 ? q1 : 0.f);
      sum2_add(hi, lo, r2 > 0 ? q2 : 0.f);
      sum2_add(hi, lo, r3 > 0 ? q3 : 0.f);
    }
    for (; b < nb; b += S) {
      const int rows = d.jtj_rows[b];
      const float q = d.partial[(size_t)b * n2 + e];
      if (rows > 0) sum2_add(hi, lo, q);
    }
  }
  sm[w][lane] = (double)hi + (double)lo;
  __syncthreads();
  if (w != 0 || u >= nu) return;
  double t = 0.0;
  for (int k = 0; k < S; ++k) t += sm[k][lane];
  d.A[e] = t;
  d.A[c * NP + r] = t;  // A is symmetric: the lower triangle mirrors the upper
  if (e == n2 - 1) {
    double E = t;
    for (int k = 0; k < d.L; ++k) E += d.prior2[k] * d.theta[k] * d.theta[k];
    if (slot >= 0) d.energy[slot] = E;
    d.lm_trials[6] = E;
  }
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce_jtj(BatchGrid g, Dev d0, int slot) {
  if (g.map == nullptr) {
    reduce_jtj_impl(d0, grid_pos(), slot);
    return;
  }
  __shared__ Dev sd;
  reduce_jtj_impl(sd, batch_block(g, sd), slot);
}

static int jtj_smem_bytes(int T, int L) {
  return kBlock * jtj_row_stride(T) * 4 + L * (int)sizeof(DQ) + 6 * L * 4 + L * 4;
}

template <int PREC>
static int jtj_tc_smem_bytes(int NB, int L) {
  return tc::Tile<PREC, 8>::STAGE + kBlock * (16 * NB + 1) * 4 + L * (int)sizeof(DQ) + 6 * L * 4 + L * 4;
}

template <int PREC>
static void launch_resid_jtj_tc(const Dev& d, int phi_buf, cudaStream_t st) {
  const int NB = (d.NP + 15) / 16;
  const int g = d.nblk_rows;
  const int sm = jtj_tc_smem_bytes<PREC>(NB, d.L);
  switch (NB) {
    case 1: k_resid_jtj_tc<PREC, 1><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
    case 2: k_resid_jtj_tc<PREC, 2><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
    case 3: k_resid_jtj_tc<PREC, 3><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
    case 4: k_resid_jtj_tc<PREC, 4><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
    default: k_resid_jtj_tc<PREC, 5><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
  }
}

template <int PREC>
static void configure_resid_jtj_tc() {
  cudaFuncSetAttribute(k_resid_jtj_tc<PREC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_tc_smem_bytes<PREC>(1, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj_tc<PREC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_tc_smem_bytes<PREC>(2, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj_tc<PREC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_tc_smem_bytes<PREC>(3, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj_tc<PREC, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_tc_smem_bytes<PREC>(4, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj_tc<PREC, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_tc_smem_bytes<PREC>(5, kMaxLinks));
}

void launch_resid_jtj(const Dev& d, int phi_buf, cudaStream_t st) {
  if (d.precision == 1) return launch_resid_jtj_tc<1>(d, phi_buf, st);
  if (d.precision == 2) return launch_resid_jtj_tc<2>(d, phi_buf, st);
  const int T = (d.NP + 15) / 16;
  const int g = d.nblk_rows;
  const int sm = jtj_smem_bytes(T, d.L);
  switch (T) {
    case 1: k_resid_jtj<1><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
    case 2: k_resid_jtj<2><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
    case 3: k_resid_jtj<3><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
    case 4: k_resid_jtj<4><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
    default: k_resid_jtj<5><<<g, kBlock, sm, st>>>(kSingle, d, phi_buf); break;
  }
}

void launch_reduce_jtj(const Dev& d, int slot, cudaStream_t st) {
  k_reduce_jtj<<<(d.NP * (d.NP + 1) / 2 + 31) / 32, 32 * reduce_warps(d.nblk_rows), 0, st>>>(kSingle, d, slot);
}

void launch_normal_equations(const Dev& d, int phi_buf, int slot, cudaStream_t st) {
  launch_resid_jtj(d, phi_buf, st);
  launch_reduce_jtj(d, slot, st);
}

// ---------------------------------------------------------------------------------------------
// LM candidates (Sec. 4.2): CTA c solves (A + lambda_c diag A) x = b with A = J^T J + (lambda_s S)^2,
// b = J^T r + (lambda_s S)^2 Theta and lambda_c = min(lambda 10^c, 1e7); a parameter whose diagonal is
// zero is frozen (x_k = 0).  Theta_c = Theta - x and its FK tables follow.
//
// On this GPU a dependent FP64 FMA costs ~70 cycles and an FP64 rsqrt ~440 (FP32: ~4 and ~20), and the
// FP64 pipe issues ~2 operations per cycle per SM, so the P sequential pivot steps of an FP64 Cholesky
// are latency-bound (~80 us at P = 55).  The solve therefore factors the Jacobi-scaled matrix D M D
// (unit diagonal) in FP32 (blocked Cholesky) and reaches FP64 accuracy by iterative refinement:
// x += D (D M D)^-1 D (b - M x) with the residual in FP64, until the scaled residual is below 1e-10 of
// the scaled right-hand side.  If the FP32 factorisation breaks down or the refinement stalls, the FP64
// Cholesky factorisation of M is used instead.
// ---------------------------------------------------------------------------------------------
constexpr int kSolveThreads = 256;
constexpr int kMaxRefine = 8;

__device__ void chol_solve_fp64(double* M, double* b, int P, int& fail_out) {
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < P; ++k) {
    if (tid == 0) {
      const double piv = M[k * P + k];
      if (!(piv > 0.0)) fail = 1;
      M[k * P + k] = sqrt(fmax(piv, 0.0));
    }
    __syncthreads();
    if (fail) break;
    const double ik = 1.0 / M[k * P + k];
    for (int r = k + 1 + tid; r < P; r += nt) M[r * P + k] *= ik;
    __syncthreads();
    const int n = P - k - 1;
    for (int e = tid; e < n * n; e += nt) {
      const int r = k + 1 + e / n, q = k + 1 + e % n;
      if (q <= r) M[r * P + q] -= M[r * P + k] * M[q * P + k];
    }
    __syncthreads();
  }
  if (!fail) {
    for (int k = 0; k < P; ++k) {
      if (tid == 0) b[k] /= M[k * P + k];
      __syncthreads();
      for (int r = k + 1 + tid; r < P; r += nt) b[r] -= M[r * P + k] * b[k];
      __syncthreads();
    }
    for (int k = P - 1; k >= 0; --k) {
      if (tid == 0) b[k] /= M[k * P + k];
      __syncthreads();
      for (int r = tid; r < k; r += nt) b[r] -= M[k * P + r] * b[k];
      __syncthreads();
    }
  }
  fail_out = fail;
  __syncthreads();
}

// (r, q) of the e-th lower-triangle element in row-major order (e = r (r + 1) / 2 + q, q <= r)
__device__ __forceinline__ void tri_rc(int e, int& r, int& q) {
  int rr = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
  while (rr * (rr + 1) / 2 > e) --rr;
  r = rr;
  q = e - rr * (rr + 1) / 2;
}

constexpr int kBlk = 8;         // block size of the factorisation
constexpr int kMaxPad = 80;     // P padded to a multiple of kBlk

// Blocked FP32 Cholesky of the padded matrix F (lower triangle, in place), 1/L_kk into ivd.  Per block
// column: (1) warp 0 factors the 8x8 diagonal block in registers (lane = row, shuffles for the column),
// (2) one thread per row below solves its 8 entries against that block, (3) one warp per 8x8 block of the
// trailing triangle subtracts the rank-8 product.  Returns false if a pivot is not positive.
__device__ bool chol_blocked(float (*F)[kMaxPad + 1], float* ivd, int Pp) {
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x, nw = nt >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < Pp; j += kBlk) {
    if (warp == 0) {
      const int i = lane & 7, r = j + i;
      float a[kBlk];
#pragma unroll
      for (int q = 0; q < kBlk; ++q) a[q] = F[r][j + q];
#pragma unroll
      for (int c = 0; c < kBlk; ++c) {
        const float dc = __shfl_sync(0xffffffffu, a[c], c);
        if (!(dc > 0.f)) { if (lane == 0) bad = 1; }
        const float iv = rsqrtf(fmaxf(dc, 1e-30f));
        a[c] = i > c ? a[c] * iv : (i == c ? dc * iv : a[c]);
        if (lane == 0) ivd[j + c] = iv;
#pragma unroll
        for (int q = c + 1; q < kBlk; ++q) {
          const float lqc = __shfl_sync(0xffffffffu, a[c], q);
          if (i >= q) a[q] = fmaf(-a[c], lqc, a[q]);
        }
      }
      if (lane < kBlk) {
#pragma unroll
        for (int q = 0; q < kBlk; ++q)
          if (q <= i) F[r][j + q] = a[q];
      }
    }
    __syncthreads();
    if (bad) return false;
    for (int r = j + kBlk + tid; r < Pp; r += nt) {  // panel
      float a[kBlk];
#pragma unroll
      for (int c = 0; c < kBlk; ++c) a[c] = F[r][j + c];
#pragma unroll
      for (int c = 0; c < kBlk; ++c) {
        float sacc = a[c];
#pragma unroll
        for (int q = 0; q < c; ++q) sacc = fmaf(-a[q], F[j + c][j + q], sacc);
        a[c] = sacc * ivd[j + c];
      }
#pragma unroll
      for (int c = 0; c < kBlk; ++c) F[r][j + c] = a[c];
    }
    __syncthreads();
    const int nb = (Pp - j - kBlk) / kBlk, nblocks = nb * (nb + 1) / 2;
    for (int blk = warp; blk < nblocks; blk += nw) {  // trailing update, one warp per 8x8 block
      int bi, bq;
      tri_rc(blk, bi, bq);
      const int r0 = j + kBlk + kBlk * bi, c0 = j + kBlk + kBlk * bq;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = lane + 32 * h, r = r0 + (e >> 3), q = c0 + (e & 7);
        float lr[kBlk], lq[kBlk];
#pragma unroll
        for (int c = 0; c < kBlk; ++c) { lr[c] = F[r][j + c]; lq[c] = F[q][j + c]; }
        float dot = 0.f;
#pragma unroll
        for (int c = 0; c < kBlk; ++c) dot = fmaf(lr[c], lq[c], dot);
        if (bi != bq || q <= r) F[r][q] -= dot;
      }
    }
    __syncthreads();
  }
  return true;
}

// Blocked forward and backward substitution with the factor of chol_blocked: y <- (L L^T)^-1 y.
__device__ void solve_blocked(float (*F)[kMaxPad + 1], const float* ivd, float* y, int Pp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  for (int j = 0; j < Pp; j += kBlk) {  // L z = y
    if (warp == 0) {
      const int i = lane & 7;
      float v = y[j + i];
#pragma unroll
      for (int c = 0; c < kBlk; ++c) {
        const float zc = __shfl_sync(0xffffffffu, v, c) * ivd[j + c];
        v = i == c ? zc : (i > c ? fmaf(-F[j + i][j + c], zc, v) : v);
      }
      if (lane < kBlk) y[j + lane] = v;
    }
    __syncthreads();
    for (int r = j + kBlk + tid; r < Pp; r += nt) {
      float sacc = y[r];
#pragma unroll
      for (int c = 0; c < kBlk; ++c) sacc = fmaf(-F[r][j + c], y[j + c], sacc);
      y[r] = sacc;
    }
    __syncthreads();
  }
  for (int j = Pp - kBlk; j >= 0; j -= kBlk) {  // L^T x = z
    if (warp == 0) {
      const int i = lane & 7;
      float v = y[j + i];
#pragma unroll
      for (int c = kBlk - 1; c >= 0; --c) {
        const float xc = __shfl_sync(0xffffffffu, v, c) * ivd[j + c];
        v = i == c ? xc : (i < c ? fmaf(-F[j + c][j + i], xc, v) : v);
      }
      if (lane < kBlk) y[j + lane] = v;
    }
    __syncthreads();
    for (int r = tid; r < j; r += nt) {
      float sacc = y[r];
#pragma unroll
      for (int c = 0; c < kBlk; ++c) sacc = fmaf(-F[j + c][r], y[j + c], sacc);
      y[r] = sacc;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void lm_solve_impl(const Dev& d, BlockPos bp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float F[kMaxPad][kMaxPad + 1];  // FP32 scaled system -> its Cholesky factor
  __shared__ float ivd[kMaxPad], ys[kMaxPad], sc[kMaxPad];
  const int P = d.L, NP = d.NP, c = bp.x, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int Pp = (P + kBlk - 1) / kBlk * kBlk;
  double* M = reinterpret_cast<double*>(smem_raw);  // [P][P] FP64 system for the residuals
  double* x = M + P * P;
  double* res = x + P;
  double* b = res + P;
  double* dg = b + P;
  double* p2 = dg + P;  // (lambda_s S_kk)^2
  double* th = p2 + P;  // Theta
  LinkTable* lt = reinterpret_cast<LinkTable*>(smem_raw + ((((size_t)P * P + 6 * P) * 8 + 15) & ~(size_t)15));
  DQ* H0 = reinterpret_cast<DQ*>(reinterpret_cast<unsigned char*>(lt) + ((sizeof(LinkTable) + 15) & ~(size_t)15));
  __shared__ unsigned rmax_bits, bmax_bits;
  __shared__ unsigned char frz[kMaxPad];
  // ---- inputs in one round trip: the link table, A (P x P at row stride NP), its diagonal and last column
  for (int t = tid; t < (int)(sizeof(LinkTable) / 16); t += nt)
    cp_async16(reinterpret_cast<char*>(lt) + 16 * t, reinterpret_cast<const char*>(d.links) + 16 * t);
  for (int e = tid; e < P * P; e += nt) cp_async8(M + e, d.A + (size_t)(e / P) * NP + e % P);
  for (int r = tid; r < P; r += nt) {
    cp_async8(dg + r, d.A + (size_t)r * NP + r);
    cp_async8(b + r, d.A + (size_t)r * NP + P);
    cp_async8(p2 + r, d.prior2 + r);
    cp_async8(th + r, d.theta + r);
  }
  double lam = *d.lam;
  for (int t = 0; t < c; ++t) lam = fmin(lam * 10.0, 1e7);
  if (tid == 0) bmax_bits = 0u;
  cp_async_wait_all();
  __syncthreads();
  // ---- setup: M = A + diag(prior + lambda dg) (FP64), frozen rows/columns -> identity; scale D in FP32
  for (int r = tid; r < P; r += nt) {  // each thread reads and writes only its own rows here
    const double dgr = dg[r] + p2[r];
    const bool fr = dgr == 0.0;
    dg[r] = dgr;
    frz[r] = fr;
    sc[r] = fr ? 1.f : rsqrtf((float)(dgr * (1.0 + lam)));
    b[r] = fr ? 0.0 : b[r] + p2[r] * th[r];
    x[r] = 0.0;
    res[r] = b[r];
    double& mrr = M[(size_t)r * P + r];
    mrr = fr ? 1.0 : mrr + (p2[r] + lam * dgr);
    atomicMax(&bmax_bits, __float_as_uint(fabsf((float)b[r] * sc[r])));
  }
  __syncthreads();
  // the off-diagonal of M (zero in frozen rows and columns) and, in the same pass, the FP32 lower triangle
  // of D M D; a warp per row
  for (int r = warp; r < P; r += nt >> 5) {
    const bool fr = frz[r];
    const float sr = sc[r];
    for (int q = lane; q < P; q += 32) {
      double m = M[(size_t)r * P + q];
      if (q != r && (fr || frz[q])) {
        m = 0.0;
        M[(size_t)r * P + q] = 0.0;
      }
      if (q <= r) F[r][q] = (float)m * sr * sc[q];
    }
  }
  for (int e = tid; e < (Pp - P) * Pp; e += nt) {  // identity rows padding P to a multiple of the block
    const int r = P + e / Pp, q = e % Pp;
    if (q <= r) F[r][q] = r == q ? 1.f : 0.f;
  }
  __syncthreads();
  // ---- FP32 factor of D M D, padded with identity rows to a multiple of the block size
  const bool ok32 = chol_blocked(F, ivd, Pp);
  // ---- iterative refinement: x += D (D M D)^-1 D (b - M x), residual in FP64
  int iters = 0;
  bool converged = false;
  const float bmax = __uint_as_float(bmax_bits);
  for (int it = 0; it < kMaxRefine && ok32; ++it) {
    for (int r = tid; r < Pp; r += nt) ys[r] = r < P ? (float)res[r] * sc[r] : 0.f;
    __syncthreads();
    solve_blocked(F, ivd, ys, Pp);
    for (int r = tid; r < P; r += nt) x[r] += (double)sc[r] * (double)ys[r];
    if (tid == 0) rmax_bits = 0u;
    __syncthreads();
    // res = b - M x in FP64: four threads per row (columns q = part mod 4, two accumulators each), the
    // four sums combined by shuffles in a fixed pairing
    for (int r0 = 0; r0 < P; r0 += nt / 4) {
      const int r = r0 + (tid >> 2), part = tid & 3;
      double s0 = 0.0, s1 = 0.0;
      if (r < P) {
        const double* mr = M + (size_t)r * P;
        int q = part;
        for (; q + 4 < P; q += 8) {
          s0 = fma(-mr[q], x[q], s0);
          s1 = fma(-mr[q + 4], x[q + 4], s1);
        }
        if (q < P) s0 = fma(-mr[q], x[q], s0);
      }
      double sum = s0 + s1;
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      sum += __shfl_xor_sync(0xffffffffu, sum, 2);
      if (r < P && part == 0) {
        const double rres = b[r] + sum;
        res[r] = rres;
        atomicMax(&rmax_bits, __float_as_uint(fabsf((float)rres * sc[r])));
      }
    }
    __syncthreads();
    iters = it + 1;
    if (__uint_as_float(rmax_bits) <= 1e-10f * bmax) { converged = true; break; }
  }
  int fail = 0;
  if (!converged) {  // FP64 Cholesky of the unscaled system
    for (int r = tid; r < P; r += nt) x[r] = b[r];
    __syncthreads();
    chol_solve_fp64(M, x, P, fail);
  }
  double* thc = d.theta_c + (size_t)c * P;
  for (int j = tid; j < P; j += nt) {  // the candidate, also kept in shared memory (res is free now) for FK
    const double tj = fail ? th[j] : th[j] - x[j];
    thc[j] = tj;
    res[j] = tj;
  }
  if (tid == 0) {
    d.lm_ok[c] = !fail;
    d.lm_ok[kCandidates + c] = converged ? iters : (fail ? -2 : -1);
  }
  __syncthreads();
  fk_all(*lt, res, H0, d.Hd_c + (size_t)c * P, d.xi_c + (size_t)c * P * 8, 8);
}

__global__ void __launch_bounds__(kSolveThreads) k_lm_solve(BatchGrid g, Dev d0) {
  if (g.map == nullptr) {
    lm_solve_impl(d0, grid_pos());
    return;
  }
  __shared__ Dev sd;
  lm_solve_impl(sd, batch_block(g, sd));
}

// Energy of each candidate at the fixed association (normals and p~ held), then the accept step:
// the first candidate with E_c <= E wins (lambda <- lambda_c / 10); if none, Theta stays and
// lambda <- min(lambda_5 * 10, 1e7).  The last block to finish does the selection.
//
// In two passes, so that the common case costs a third of the work: the first pass scores candidates
// 0 and 1 (the damping that almost always succeeds) and accepts one if it can; otherwise it records
// their energies and marks the step pending (lm_trials[7] = -2), and the second pass scores candidates
// 2-5 and decides over all six.  The decision sequence and every energy are those of scoring all six at
// once (each candidate's sum has the same blocks in the same order).  Candidates not scored report +inf.
constexpr double kPending = -2.0;

__device__ __forceinline__ void lm_eval_impl(const Dev& d, BlockPos bp, int c0, int c1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DQ* sH = reinterpret_cast<DQ*>(smem_raw);  // [kCandidates][L]
  __shared__ int sok[kCandidates];
  __shared__ double swarp[kBlock / 32][kCandidates];
  __shared__ bool last;
  const int L = d.L, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (c0 > 0 && d.lm_trials[7] != kPending) return;  // the first pass decided
  // the [J r] block's rows (written by the normal-equations pass of this iteration, one record per vertex
  // of A: the mean data point p~, n, x = x0 + phi, bones and weights), with the candidates' tables
  const int cnt = d.jtj_rows[bp.x];
  const float4* recs = d.arec + (size_t)bp.x * kBlock * d.jtj_group * 4;
  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
  if (tid < cnt) {
    r0 = recs[4 * tid];
    r1 = recs[4 * tid + 1];
    r2 = recs[4 * tid + 2];
    r3 = recs[4 * tid + 3];
  }
  if (cnt > 0)  // the same in every thread of the block
    for (int t = c0 * L + tid; t < c1 * L; t += kBlock) sH[t] = d.Hd_c[t];
  if (tid < kCandidates) sok[tid] = d.lm_ok[tid];
  __syncthreads();
  float e[kCandidates];
#pragma unroll
  for (int c = 0; c < kCandidates; ++c) e[c] = 0.f;
  for (int q = tid; q < cnt; q += kBlock) {
    if (q != tid) {
      r0 = recs[4 * q];
      r1 = recs[4 * q + 1];
      r2 = recs[4 * q + 2];
      r3 = recs[4 * q + 3];
    }
    const float3 pt = make_float3(r0.x, r0.y, r0.z), nn = make_float3(r0.w, r1.x, r1.y);
    const float3 x = make_float3(r1.z, r1.w, r2.x);
    const float4 bw = make_float4(r2.y, r2.z, r2.w, r3.x);
    const unsigned bits = __float_as_uint(r3.y);
    uchar4 bi;
    memcpy(&bi, &bits, 4);
#pragma unroll
    for (int c = 0; c < kCandidates; ++c) {
      if (c < c0 || c >= c1 || !sok[c]) continue;
      float sg[4];
      const DQ H = blend_bones(sH + c * L, bi, bw, sg);
      const float3 vc = dq_point(H, x);
      const float r = nn.x * (pt.x - vc.x) + nn.y * (pt.y - vc.y) + nn.z * (pt.z - vc.z);
      e[c] += r * r;
    }
  }
#pragma unroll
  for (int c = 0; c < kCandidates; ++c)
    for (int o = 16; o > 0; o >>= 1) e[c] += __shfl_xor_sync(0xffffffffu, e[c], o);
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < kCandidates; ++c) swarp[w][c] = e[c];
  }
  __syncthreads();
  if (tid >= c0 && tid < c1) {
    double s = 0.0;
    for (int k = 0; k < kBlock / 32; ++k) s += swarp[k][tid];
    d.epart[(size_t)bp.x * 8 + tid] = s;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&d.counter[0], 1u) == (unsigned)bp.gx - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the session's last block: sum of the block energies (strided over the threads, then a shuffle tree
  // and the 8 warp sums in order) plus each candidate's prior term (warp c, lanes over the links)
  __shared__ double Ec[kCandidates], pri[kCandidates];
  {
    double s6[kCandidates] = {0, 0, 0, 0, 0, 0};
    for (int b = tid; b < bp.gx; b += kBlock) {
#pragma unroll
      for (int c = 0; c < kCandidates; ++c)
        if (c >= c0 && c < c1) s6[c] += __ldcg(d.epart + (size_t)b * 8 + c);
    }
#pragma unroll
    for (int c = 0; c < kCandidates; ++c)
      for (int o = 16; o > 0; o >>= 1) s6[c] += __shfl_xor_sync(0xffffffffu, s6[c], o);
    __syncthreads();  // swarp is reused
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < kCandidates; ++c) swarp[w][c] = s6[c];
    }
    if (w >= c0 && w < c1) {
      const double* thc = d.theta_c + (size_t)w * L;
      double p = 0.0;
      for (int k = lane; k < L; k += 32) p += d.prior2[k] * thc[k] * thc[k];
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (lane == 0) pri[w] = p;
    }
  }
  __syncthreads();
  const double inf = __longlong_as_double(0x7ff0000000000000ll);
  if (tid < kCandidates) {
    if (tid >= c0 && tid < c1) {
      double s = 0.0;
      for (int k = 0; k < kBlock / 32; ++k) s += swarp[k][tid];
      Ec[tid] = sok[tid] ? s + pri[tid] : inf;
    } else {
      Ec[tid] = tid < c0 ? d.lm_trials[tid] : inf;  // the first pass's energies; later ones unscored
    }
  }
  __syncthreads();
  __shared__ int acc_c;
  if (tid == 0) {
    const double E = d.lm_trials[6];
    double lam = *d.lam;
    int a = -1;
    for (int c = 0; c < c1; ++c) {
      d.lm_trials[c] = Ec[c];
      if (a < 0 && sok[c] && Ec[c] <= E) a = c;
    }
    for (int c = c1; c < kCandidates; ++c) d.lm_trials[c] = inf;
    if (a >= 0 || c1 == kCandidates) {
      if (a >= 0) {
        for (int t = 0; t < a; ++t) lam = fmin(lam * 10.0, 1e7);
        lam = fmax(lam / 10.0, 1e-7);
      } else {
        for (int t = 0; t < kCandidates; ++t) lam = fmin(lam * 10.0, 1e7);
      }
      *d.lam = lam;
      d.lm_trials[7] = (double)a;
    } else {
      d.lm_trials[7] = kPending;
    }
    acc_c = a;
    d.counter[0] = 0;
  }
  __syncthreads();
  const int a = acc_c;
  if (a >= 0) {
    for (int j = tid; j < L; j += kBlock) {
      d.theta[j] = d.theta_c[(size_t)a * L + j];
      d.Hd[j] = d.Hd_c[(size_t)a * L + j];
      for (int q = 0; q < 8; ++q) d.xi[8 * j + q] = d.xi_c[((size_t)a * L + j) * 8 + q];
    }
  }
}

constexpr int kFirstPass = 2;  // candidates scored by the first pass

__global__ void __launch_bounds__(kBlock) k_lm_eval(BatchGrid g, Dev d0, int c0, int c1) {
  if (g.map == nullptr) {
    lm_eval_impl(d0, grid_pos(), c0, c1);
    return;
  }
  __shared__ Dev sd;
  lm_eval_impl(sd, batch_block(g, sd), c0, c1);
}

static int lm_solve_smem(int L) {
  return (int)(((((size_t)L * L + 6 * L) * 8 + 15) & ~(size_t)15) + ((sizeof(LinkTable) + 15) & ~(size_t)15) +
               (size_t)L * sizeof(DQ));
}

void launch_lm_solve(const Dev& d, cudaStream_t st) {
  k_lm_solve<<<kCandidates, kSolveThreads, lm_solve_smem(d.L), st>>>(kSingle, d);
}

void launch_lm_eval(const Dev& d, int /*phi_buf: the rows' records already hold x0 + phi*/, cudaStream_t st) {
  const size_t sm = kCandidates * d.L * sizeof(DQ);
  k_lm_eval<<<d.nblk_rows, kBlock, sm, st>>>(kSingle, d, 0, kFirstPass);
  k_lm_eval<<<d.nblk_rows, kBlock, sm, st>>>(kSingle, d, kFirstPass, kCandidates);
}

void launch_lm(const Dev& d, int phi_buf, cudaStream_t st) {
  launch_lm_solve(d, st);
  launch_lm_eval(d, phi_buf, st);
}

// ---------------------------------------------------------------------------------------------
// Sec. 4.3 shape step (per vertex, neighbours frozen): e_i = [i in A] r_i^2 + lambda_phi |phi_i|^2 +
// lambda_N sum_n |phi_i - phi_n|^2 with g_i = dr_i/dphi_i = -R(a^_i)^T n_i; one damped 3x3 Gauss-Newton
// solve (M + lambda_w diag M) delta = -(g r + lambda_phi phi_i + lambda_N sum_n (phi_i - phi_n)),
// M = g g^T + (lambda_phi + lambda_N |N(i)|) I, written to the other Jacobi buffer.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float3 solve3_damped(float3 g, float cdiag, float lw, float3 rhs) {
  // M + lw diag(M), M = g g^T + cdiag I  (Cramer's rule)
  float m00 = g.x * g.x + cdiag, m11 = g.y * g.y + cdiag, m22 = g.z * g.z + cdiag;
  const float m01 = g.x * g.y, m02 = g.x * g.z, m12 = g.y * g.z;
  m00 += lw * m00; m11 += lw * m11; m22 += lw * m22;
  const float c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
  const float det = m00 * c00 + m01 * c01 + m02 * c02;
  if (det == 0.f) return make_float3(0.f, 0.f, 0.f);
  const float c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
  const float id = 1.f / det;
  return make_float3((c00 * rhs.x + c01 * rhs.y + c02 * rhs.z) * id, (c01 * rhs.x + c11 * rhs.y + c12 * rhs.z) * id,
                     (c02 * rhs.x + c12 * rhs.y + c22 * rhs.z) * id);
}

__device__ __forceinline__ void block_energy_to_slot(const Dev& d, BlockPos bp, float e, int slot, int ticket) {
  __shared__ double sw[kBlock];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += sw[w];
    d.epart[(size_t)bp.x * 8] = s;
    __threadfence();
    last = atomicAdd(&d.counter[ticket], 1u) == (unsigned)bp.gx - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;  // fixed order: strided per thread, then a tree over the threads
  for (int b = threadIdx.x; b < bp.gx; b += kBlock) s += __ldcg(d.epart + (size_t)b * 8);
  sw[threadIdx.x] = s;
  __syncthreads();
  for (int h = kBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sw[threadIdx.x] += sw[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (slot >= 0) d.energy[slot] = sw[0];
    d.counter[ticket] = 0;
  }
}

// r_i (the mean offset of the associated pixels along n_i) and g_i = dr_i/dphi_i = -R(a^_i)^T n_i.
__device__ __forceinline__ void vertex_r_g(const DQ* sHd, uchar4 bi, float4 bw, const Acc4& a4, const float4& nn,
                                           float& r, float3& g) {
  const float inv = 1.f / ((float)a4.w * kFix);
  r = nn.x * (float)a4.x * inv + nn.y * (float)a4.y * inv + nn.z * (float)a4.z * inv;
  float sg[4];
  const DQ H = blend_bones(sHd, bi, bw, sg);
  const float4 ah = qscale(H.r, rsqrtf(qdot(H.r, H.r)));
  const float4 q = qmul(qmul(qconj(ah), make_float4(0.f, nn.x, nn.y, nn.z)), ah);  // R^T n
  g = make_float3(-q.y, -q.z, -q.w);
}

__device__ __forceinline__ void shape_impl(const Dev& d, BlockPos bp, int src, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DQ* sHd = reinterpret_cast<DQ*>(smem_raw);
  const int i = bp.x * kBlock + threadIdx.x;
  bool anyA = false;
  if (i < d.V) anyA = d.acc[i].w >= 1 && d.n[i].w > 0.f;
  if (__syncthreads_or(anyA)) {  // the pose tables are needed only where a vertex of A is
    for (int j = threadIdx.x; j < d.L; j += kBlock) sHd[j] = d.Hd[j];
    __syncthreads();
  }
  float e = 0.f;
  int inA_count = 0;
  if (i < d.V) {
    const float4* phi = d.phi[src];
    const float4 p4 = phi[i];
    const float3 pi = f3(p4);
    const Acc4 a4 = d.acc[i];
    const float4 nn = d.n[i];
    const bool inA = a4.w >= 1 && nn.w > 0.f;
    float r = 0.f;
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (inA) {
      inA_count = 1;
      vertex_r_g(sHd, d.bidx[i], d.bw[i], a4, nn, r, g);
    }
    e = r * r + d.lambda_phi * dot3(pi, pi);
    float3 sd = make_float3(0.f, 0.f, 0.f);
    int nn_count = 0;
    const int4 nb = d.nbr[i];
    const int nbs[4] = {nb.x, nb.y, nb.z, nb.w};
    float4 qn[4];  // the neighbours' offsets, all in flight before they are used
#pragma unroll
    for (int t = 0; t < 4; ++t) qn[t] = t < d.knn && nbs[t] >= 0 ? phi[nbs[t]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= d.knn || nbs[t] < 0) continue;
      const float3 q = f3(qn[t]);
      const float3 df = make_float3(pi.x - q.x, pi.y - q.y, pi.z - q.z);
      e += d.lambda_N * dot3(df, df);
      sd.x += df.x; sd.y += df.y; sd.z += df.z;
      ++nn_count;
    }
    const float3 grad = make_float3(g.x * r + d.lambda_phi * pi.x + d.lambda_N * sd.x,
                                    g.y * r + d.lambda_phi * pi.y + d.lambda_N * sd.y,
                                    g.z * r + d.lambda_phi * pi.z + d.lambda_N * sd.z);
    const float3 dl = solve3_damped(g, d.lambda_phi + d.lambda_N * nn_count, d.lambda_w,
                                    make_float3(-grad.x, -grad.y, -grad.z));
    d.phi[1 - src][i] = make_float4(pi.x + dl.x, pi.y + dl.y, pi.z + dl.z, 0.f);
    d.rg[i] = make_float4(g.x, g.y, g.z, r);
    d.phi0[i] = p4;
  }
  const unsigned m = __ballot_sync(0xffffffffu, inA_count != 0);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(&d.stats[1], __popc(m));
  block_energy_to_slot(d, bp, e, slot, 1);
}

__global__ void __launch_bounds__(kBlock) k_shape(BatchGrid g, Dev d0, int src, int slot) {
  if (g.map == nullptr) {
    shape_impl(d0, grid_pos(), src, slot);
    return;
  }
  __shared__ Dev sd;
  shape_impl(sd, batch_block(g, sd), src, slot);
}

// A batch's launch: registers sized for kBatchMinBlocks resident blocks (a few spills for occupancy).
__global__ void __launch_bounds__(kBlock, kBatchMinBlocks) k_shape_b(BatchGrid g, int src, int slot) {
  __shared__ Dev sd;
  shape_impl(sd, batch_block(g, sd), src, slot);
}

// Further Jacobi sweeps: r_i is updated linearly, r_i = r0_i + g_i . (phi_i - phi0_i).
__device__ __forceinline__ void shape_sweep_impl(const Dev& d, BlockPos bp, int src) {
  const int i = bp.x * kBlock + threadIdx.x;
  if (i >= d.V) return;
  const float4* phi = d.phi[src];
  const float3 pi = f3(phi[i]);
  const float4 rg = d.rg[i];
  const float3 g = f3(rg), p0 = f3(d.phi0[i]);
  const float r = rg.w + g.x * (pi.x - p0.x) + g.y * (pi.y - p0.y) + g.z * (pi.z - p0.z);
  float3 sd = make_float3(0.f, 0.f, 0.f);
  int nn_count = 0;
  const int4 nb = d.nbr[i];
  const int nbs[4] = {nb.x, nb.y, nb.z, nb.w};
  float4 qn[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) qn[t] = t < d.knn && nbs[t] >= 0 ? phi[nbs[t]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t >= d.knn || nbs[t] < 0) continue;
    const float3 q = f3(qn[t]);
    sd.x += pi.x - q.x; sd.y += pi.y - q.y; sd.z += pi.z - q.z;
    ++nn_count;
  }
  const float3 grad = make_float3(g.x * r + d.lambda_phi * pi.x + d.lambda_N * sd.x,
                                  g.y * r + d.lambda_phi * pi.y + d.lambda_N * sd.y,
                                  g.z * r + d.lambda_phi * pi.z + d.lambda_N * sd.z);
  const float3 dl = solve3_damped(g, d.lambda_phi + d.lambda_N * nn_count, d.lambda_w,
                                  make_float3(-grad.x, -grad.y, -grad.z));
  d.phi[1 - src][i] = make_float4(pi.x + dl.x, pi.y + dl.y, pi.z + dl.z, 0.f);
}

__global__ void __launch_bounds__(kBlock) k_shape_sweep(BatchGrid g, Dev d0, int src) {
  if (g.map == nullptr) {
    shape_sweep_impl(d0, grid_pos(), src);
    return;
  }
  __shared__ Dev sd;
  shape_sweep_impl(sd, batch_block(g, sd), src);
}

// ---------------------------------------------------------------------------------------------
// Coupled shape step (the whole shape energy of Sec. 4.3, linearised in r): (H + lambda_w diag H) delta
// = -b with H_ii = [A] g g^T + (lambda_phi + lambda_N deg_i) I and H_ij = -lambda_N I per neighbourhood
// edge (either direction), by conjugate gradients preconditioned with the 3x3 diagonal blocks.  Vectors
// in FP32, dot products in FP64 with fixed-order block sums (deterministic); a breakdown (r.z = 0 or
// p.Ap <= 0) stops the iteration as in exact arithmetic.  One kernel per CG phase.
// ---------------------------------------------------------------------------------------------
// Block sum of v (FP64) into epart[bp.x * 8 + slot]; returns true in every thread of the session's last
// block, with the fixed-order total of all its blocks in `total`.
__device__ __forceinline__ bool block_total(const Dev& d, BlockPos bp, double v, int slot, int ticket, double& total) {
  __shared__ double sw[kBlock / 32];
  __shared__ double red[kBlock];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += sw[w];
    d.epart[(size_t)bp.x * 8 + slot] = s;
    __threadfence();
    last = atomicAdd(&d.counter[ticket], 1u) == (unsigned)bp.gx - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < bp.gx; b += kBlock) s += __ldcg(d.epart + (size_t)b * 8 + slot);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  total = red[0];
  if (threadIdx.x == 0) d.counter[ticket] = 0;
  return true;
}

// B_i = M_i + lambda_w diag(M_i), M_i = g g^T + c I (g = 0 outside A): B_i p and B_i^-1 p.
__device__ __forceinline__ float3 block_apply(float3 g, float c, float lw, float3 p) {
  const float gp = g.x * p.x + g.y * p.y + g.z * p.z;
  return make_float3(g.x * gp + c * p.x + lw * (g.x * g.x + c) * p.x, g.y * gp + c * p.y + lw * (g.y * g.y + c) * p.y,
                     g.z * gp + c * p.z + lw * (g.z * g.z + c) * p.z);
}

// r_i, g_i, E_shape (energy[slot]) as the Jacobi step; b; x = 0, r = -b, z = B^-1 r, p = z, rz = r.z.
__device__ __forceinline__ void cg_init_impl(const Dev& d, BlockPos bp, int src, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DQ* sHd = reinterpret_cast<DQ*>(smem_raw);
  const int i = bp.x * kBlock + threadIdx.x;
  bool anyA = false;
  if (i < d.V) anyA = d.acc[i].w >= 1 && d.n[i].w > 0.f;
  if (__syncthreads_or(anyA)) {
    for (int j = threadIdx.x; j < d.L; j += kBlock) sHd[j] = d.Hd[j];
    __syncthreads();
  }
  float e = 0.f;
  double rz = 0.0;
  int inA_count = 0;
  if (i < d.V) {
    const float4* phi = d.phi[src];
    const float4 p4 = phi[i];
    const float3 pi = f3(p4);
    const Acc4 a4 = d.acc[i];
    const float4 nn = d.n[i];
    float r = 0.f;
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (a4.w >= 1 && nn.w > 0.f) {
      inA_count = 1;
      vertex_r_g(sHd, d.bidx[i], d.bw[i], a4, nn, r, g);
    }
    e = r * r + d.lambda_phi * dot3(pi, pi);
    const int4 nb = d.nbr[i];
    const int nbs[4] = {nb.x, nb.y, nb.z, nb.w};
    for (int t = 0; t < d.knn; ++t) {
      if (nbs[t] < 0) continue;
      const float3 q = f3(phi[nbs[t]]);
      const float3 df = make_float3(pi.x - q.x, pi.y - q.y, pi.z - q.z);
      e += d.lambda_N * dot3(df, df);
    }
    float3 sd = make_float3(0.f, 0.f, 0.f);
    const int a0 = d.adj_off[i], a1 = d.adj_off[i + 1];
    for (int t = a0; t < a1; ++t) {
      const float3 q = f3(phi[d.adj[t]]);
      sd.x += pi.x - q.x; sd.y += pi.y - q.y; sd.z += pi.z - q.z;
    }
    const float3 rr = make_float3(-(g.x * r + d.lambda_phi * pi.x + d.lambda_N * sd.x),
                                  -(g.y * r + d.lambda_phi * pi.y + d.lambda_N * sd.y),
                                  -(g.z * r + d.lambda_phi * pi.z + d.lambda_N * sd.z));
    const float3 z = solve3_damped(g, d.lambda_phi + d.lambda_N * (float)(a1 - a0), d.lambda_w, rr);
    d.rg[i] = make_float4(g.x, g.y, g.z, r);
    d.phi0[i] = p4;
    d.cg_x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    d.cg_r[i] = make_float4(rr.x, rr.y, rr.z, 0.f);
    d.cg_z[i] = make_float4(z.x, z.y, z.z, 0.f);
    d.cg_p[i] = make_float4(z.x, z.y, z.z, 0.f);
    rz = (double)rr.x * z.x + (double)rr.y * z.y + (double)rr.z * z.z;
  }
  const unsigned m = __ballot_sync(0xffffffffu, inA_count != 0);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(&d.stats[1], __popc(m));
  double tot;
  if (block_total(d, bp, rz, 1, 2, tot) && threadIdx.x == 0) {
    d.cg[0] = tot;
    d.cg[3] = tot > 0.0 ? 0.0 : 1.0;  // stopped if the preconditioned residual is already zero
  }
  block_energy_to_slot(d, bp, e, slot, 1);
}

// Ap = (B - lambda_N Adj) p; alpha = r.z / p.Ap (0 and stop on a breakdown).
__device__ __forceinline__ void cg_apply_impl(const Dev& d, BlockPos bp) {
  const int i = bp.x * kBlock + threadIdx.x;
  double pap = 0.0;
  if (i < d.V) {
    const float4 rg = d.rg[i];
    const float3 p = f3(d.cg_p[i]);
    const int a0 = d.adj_off[i], a1 = d.adj_off[i + 1];
    float3 ap = block_apply(f3(rg), d.lambda_phi + d.lambda_N * (float)(a1 - a0), d.lambda_w, p);
    for (int t = a0; t < a1; ++t) {
      const float3 q = f3(d.cg_p[d.adj[t]]);
      ap.x -= d.lambda_N * q.x; ap.y -= d.lambda_N * q.y; ap.z -= d.lambda_N * q.z;
    }
    d.cg_ap[i] = make_float4(ap.x, ap.y, ap.z, 0.f);
    pap = (double)p.x * ap.x + (double)p.y * ap.y + (double)p.z * ap.z;
  }
  double tot;
  if (block_total(d, bp, pap, 2, 3, tot) && threadIdx.x == 0) {
    const bool go = d.cg[3] == 0.0 && tot > 0.0;
    d.cg[1] = go ? d.cg[0] / tot : 0.0;
    if (!go) d.cg[3] = 1.0;
  }
}

// x += alpha p, r -= alpha Ap, z = B^-1 r; beta = r.z_new / r.z.
__device__ __forceinline__ void cg_update_impl(const Dev& d, BlockPos bp) {
  const int i = bp.x * kBlock + threadIdx.x;
  const float alpha = (float)d.cg[1];
  double rz = 0.0;
  if (i < d.V) {
    const float4 rg = d.rg[i];
    const float3 p = f3(d.cg_p[i]), ap = f3(d.cg_ap[i]);
    float3 x = f3(d.cg_x[i]), r = f3(d.cg_r[i]);
    x.x += alpha * p.x; x.y += alpha * p.y; x.z += alpha * p.z;
    r.x -= alpha * ap.x; r.y -= alpha * ap.y; r.z -= alpha * ap.z;
    const int deg = d.adj_off[i + 1] - d.adj_off[i];
    const float3 z = solve3_damped(f3(rg), d.lambda_phi + d.lambda_N * (float)deg, d.lambda_w, r);
    d.cg_x[i] = make_float4(x.x, x.y, x.z, 0.f);
    d.cg_r[i] = make_float4(r.x, r.y, r.z, 0.f);
    d.cg_z[i] = make_float4(z.x, z.y, z.z, 0.f);
    rz = (double)r.x * z.x + (double)r.y * z.y + (double)r.z * z.z;
  }
  double tot;
  if (block_total(d, bp, rz, 1, 2, tot) && threadIdx.x == 0) {
    const bool go = d.cg[3] == 0.0 && d.cg[0] > 0.0;
    d.cg[2] = go ? tot / d.cg[0] : 0.0;
    d.cg[0] = tot;
    if (!(tot > 0.0)) d.cg[3] = 1.0;
  }
}

// p = z + beta p.
__device__ __forceinline__ void cg_dir_impl(const Dev& d, BlockPos bp) {
  const int i = bp.x * kBlock + threadIdx.x;
  if (i >= d.V) return;
  const float beta = (float)d.cg[2];
  const float3 z = f3(d.cg_z[i]), p = f3(d.cg_p[i]);
  d.cg_p[i] = make_float4(z.x + beta * p.x, z.y + beta * p.y, z.z + beta * p.z, 0.f);
}

// phi[1 - src] = phi[src] + x.
__device__ __forceinline__ void cg_finish_impl(const Dev& d, BlockPos bp, int src) {
  const int i = bp.x * kBlock + threadIdx.x;
  if (i >= d.V) return;
  const float4 p = d.phi[src][i], x = d.cg_x[i];
  d.phi[1 - src][i] = make_float4(p.x + x.x, p.y + x.y, p.z + x.z, 0.f);
}

#define TRK_CG_KERNEL(name, impl, ...)                                                     \
  __global__ void __launch_bounds__(kBlock) name(BatchGrid g, Dev d0 ARGS_##name) {         \
    if (g.map == nullptr) {                                                                  \
      impl(d0, grid_pos() CALL_##name);                                                      \
      return;                                                                                \
    }                                                                                        \
    __shared__ Dev sd;                                                                       \
    impl(sd, batch_block(g, sd) CALL_##name);                                                \
  }
#define ARGS_k_cg_init , int src, int slot
#define CALL_k_cg_init , src, slot
#define ARGS_k_cg_apply
#define CALL_k_cg_apply
#define ARGS_k_cg_update
#define CALL_k_cg_update
#define ARGS_k_cg_dir
#define CALL_k_cg_dir
#define ARGS_k_cg_finish , int src
#define CALL_k_cg_finish , src
TRK_CG_KERNEL(k_cg_init, cg_init_impl)
TRK_CG_KERNEL(k_cg_apply, cg_apply_impl)
TRK_CG_KERNEL(k_cg_update, cg_update_impl)
TRK_CG_KERNEL(k_cg_dir, cg_dir_impl)
TRK_CG_KERNEL(k_cg_finish, cg_finish_impl)

// The whole coupled step (g, n: the block table and its size for a batch; kSingle and nblk_v alone).
static void launch_shape_pcg(const BatchGrid& g, int n, const Dev& d0, int max_links, int iters, int src, int slot,
                             cudaStream_t st) {
  if (n <= 0) return;
  k_cg_init<<<n, kBlock, max_links * sizeof(DQ), st>>>(g, d0, src, slot);
  for (int k = 0; k < iters; ++k) {
    k_cg_apply<<<n, kBlock, 0, st>>>(g, d0);
    k_cg_update<<<n, kBlock, 0, st>>>(g, d0);
    if (k + 1 < iters) k_cg_dir<<<n, kBlock, 0, st>>>(g, d0);
  }
  k_cg_finish<<<n, kBlock, 0, st>>>(g, d0, src);
}

// Returns the buffer that holds Phi after the step.
int launch_shape(const Dev& d, int phi_src, int slot, cudaStream_t st) {
  if (d.shape_solver == 1) {
    launch_shape_pcg(kSingle, d.nblk_v, d, d.L, d.shape_sweeps, phi_src, slot, st);
    return 1 - phi_src;
  }
  k_shape<<<d.nblk_v, kBlock, d.L * sizeof(DQ), st>>>(kSingle, d, phi_src, slot);
  int cur = 1 - phi_src;
  for (int s = 1; s < d.shape_sweeps; ++s) {
    k_shape_sweep<<<d.nblk_v, kBlock, 0, st>>>(kSingle, d, cur);
    cur = 1 - cur;
  }
  return cur;
}

// ---- batched launches ------------------------------------------------------------------------
template <int PREC>
static void launch_resid_jtj_tc_b(const BatchGrid& g, int nblk, int max_np, int max_links, int phi_buf,
                                  cudaStream_t st) {
  const int NB = (max_np + 15) / 16;
  const int sm = jtj_tc_smem_bytes<PREC>(NB, max_links);
  switch (NB) {
    case 1: k_resid_jtj_tc<PREC, 1><<<nblk, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
    case 2: k_resid_jtj_tc<PREC, 2><<<nblk, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
    case 3: k_resid_jtj_tc<PREC, 3><<<nblk, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
    case 4: k_resid_jtj_tc<PREC, 4><<<nblk, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
    default: k_resid_jtj_tc<PREC, 5><<<nblk, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
  }
}

// gj[t - 1], nj[t - 1]: the blocks of the sessions whose [J r] tile width class is t = ceil(NP / 16)
// (one launch per class, so a small skeleton does not pay for the largest one's tiles).
void launch_normal_equations_b(const BatchGrid* gj, const int* nj, const BatchGrid& gr, int nr, int max_links,
                               int precision, int phi_buf, int slot, cudaStream_t st, int reduce_threads) {
  for (int T = 1; T <= 5; ++T) {
    const BatchGrid& g = gj[T - 1];
    const int n = nj[T - 1];
    if (n == 0) continue;
    if (precision == 1) {
      launch_resid_jtj_tc_b<1>(g, n, 16 * T, max_links, phi_buf, st);
    } else if (precision == 2) {
      launch_resid_jtj_tc_b<2>(g, n, 16 * T, max_links, phi_buf, st);
    } else {
      const int sm = jtj_smem_bytes(T, max_links);
      switch (T) {
        case 1: k_resid_jtj<1><<<n, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
        case 2: k_resid_jtj<2><<<n, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
        case 3: k_resid_jtj<3><<<n, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
        case 4: k_resid_jtj<4><<<n, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
        default: k_resid_jtj<5><<<n, kBlock, sm, st>>>(g, Dev{}, phi_buf); break;
      }
    }
  }
  if (nr > 0) k_reduce_jtj<<<nr, reduce_threads, 0, st>>>(gr, Dev{}, slot);
}

void launch_lm_b(const BatchGrid& glm, int nlm, const BatchGrid& gv, int nv, int max_links, int phi_buf,
                 cudaStream_t st) {
  if (nlm > 0) k_lm_solve<<<nlm, kSolveThreads, lm_solve_smem(max_links), st>>>(glm, Dev{});
  if (nv > 0) {
    const size_t sm = kCandidates * max_links * sizeof(DQ);
    k_lm_eval<<<nv, kBlock, sm, st>>>(gv, Dev{}, 0, kFirstPass);
    k_lm_eval<<<nv, kBlock, sm, st>>>(gv, Dev{}, kFirstPass, kCandidates);
  }
}

int launch_shape_b(const BatchGrid& gv, int nv, int max_links, int sweeps, int solver, int phi_src, int slot,
                   cudaStream_t st) {
  if (solver == 1) {
    launch_shape_pcg(gv, nv, Dev{}, max_links, sweeps, phi_src, slot, st);
    return 1 - phi_src;
  }
  if (nv > 0) k_shape_b<<<nv, kBlock, max_links * sizeof(DQ), st>>>(gv, phi_src, slot);
  int cur = 1 - phi_src;
  for (int s = 1; s < sweeps; ++s) {
    if (nv > 0) k_shape_sweep<<<nv, kBlock, 0, st>>>(gv, Dev{}, cur);
    cur = 1 - cur;
  }
  return cur;
}

static void configure_batched() {
  cudaFuncSetAttribute(k_lm_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, lm_solve_smem(kMaxLinks));
}

void configure_tc_kernels();

void configure_kernels() {
  configure_tc_kernels();
  configure_batched();
  configure_resid_jtj_tc<1>();
  configure_resid_jtj_tc<2>();
  cudaFuncSetAttribute(k_resid_jtj<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(1, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(2, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(3, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(4, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(5, kMaxLinks));
  cudaFuncSetAttribute(k_lm_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, lm_solve_smem(kMaxLinks));
}

// Sets the kernels' shared-memory limits once per device (the attributes are per device).
void ensure_configured() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    configure_kernels();
    done[dev] = true;
  }
}

}  // namespace trk

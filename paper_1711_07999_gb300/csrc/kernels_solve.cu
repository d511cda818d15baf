// kernels_solve.cu -- point-to-plane residuals and the pose Jacobian (Eq. residual, Sec. 4.2), the
// reduction [J r]^T [J r] (Eqs. JTJ, JTr), the damped least-squares step with the pose prior and its
// energy test (Sec. 4.2), and the per-vertex shape step (Eq. r_warp, Sec. 4.3).
//
// Reductions are deterministic: per-block partial sums over fixed vertex ranges, then a second pass
// that adds the partials in block order in FP64.  The LM retries of one iteration (damping lambda,
// 10 lambda, ..., 10^5 lambda) are solved side by side, one CTA each, and their energies evaluated in
// one pass over the vertices; the first candidate that does not raise the energy is taken on the device,
// which gives the same result as trying them one after the other without any host round trip.
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
template <int T>
__global__ void __launch_bounds__(kBlock) k_resid_jtj(Dev d, int phi_buf) {
  constexpr int ROW = 16 * T + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Js = reinterpret_cast<float*>(smem_raw);
  DQ* sHd = reinterpret_cast<DQ*>(Js + kBlock * ROW);
  float* sXi = reinterpret_cast<float*>(sHd + d.L);
  int* sPar = reinterpret_cast<int*>(sXi + 6 * d.L);
  __shared__ int s_warp[kBlock / 32];
  const int tid = threadIdx.x;
  for (int j = tid; j < d.L; j += kBlock) {
    sHd[j] = d.Hd[j];
    for (int c = 0; c < 6; ++c) sXi[6 * j + c] = d.xi[8 * j + c];
    sPar[j] = d.links->parent[j];
  }
  const int i = blockIdx.x * kBlock + tid;
  bool inA = false;
  Acc4 a4 = Acc4{0, 0, 0, 0};
  float4 nn = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i < d.V) {
    a4 = d.acc[i];
    nn = d.n[i];
    inA = a4.w >= 1 && nn.w > 0.f;
  }
  const unsigned m = __ballot_sync(0xffffffffu, inA);
  const int lane = tid & 31, w = tid >> 5;
  if (lane == 0) s_warp[w] = __popc(m);
  __syncthreads();
  int off = 0, total = 0;
  for (int k = 0; k < kBlock / 32; ++k) {
    off += k < w ? s_warp[k] : 0;
    total += s_warp[k];
  }
  if (inA) {
    float* row = Js + (off + __popc(m & ((1u << lane) - 1u))) * ROW;
    for (int k = 0; k < 16 * T; ++k) row[k] = 0.f;
    const float inv = 1.f / ((float)a4.w * kFix);
    const float3 pm = make_float3((float)a4.x * inv, (float)a4.y * inv, (float)a4.z * inv);
    const float3 n = f3(nn);
    row[d.L] = dot3(n, pm);
    float sg[4];
    const uchar4 bi = d.bidx[i];
    const float4 bw = d.bw[i];
    const DQ H = blend_bones(sHd, bi, bw, sg);
    const float4 x0 = d.v0[i], ph = d.phi[phi_buf][i], v = d.v[i];
    const float4 X = make_float4(0.f, x0.x + ph.x, x0.y + ph.y, x0.z + ph.z);
    const float4 Np = make_float4(0.f, n.x, n.y, n.z);
    const float invN = 1.f / qdot(H.r, H.r);
    const float4 Na = qmul(Np, H.r);
    const float4 cr = qscale(qadd(qadd(qmul(Na, X), qmul(Np, H.d)), qscale(H.r, dot3(n, f3(v)))), -2.f * invN);
    const float4 cd = qscale(Na, 2.f * invN);
    const int idx[4] = {bi.x, bi.y, bi.z, bi.w};
    const float ws[4] = {bw.x, bw.y, bw.z, bw.w};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (!(ws[s] > 0.f)) continue;
      const DQ h = sHd[idx[s]];
      const float sc = ws[s] * sg[s];
      const float3 e1 = Lfun(cr, h.r), e2 = Lfun(cd, h.d), e3 = Lfun(cd, h.r);
      const float e[6] = {sc * (e1.x + e2.x), sc * (e1.y + e2.y), sc * (e1.z + e2.z), sc * e3.x, sc * e3.y, sc * e3.z};
      for (int k = idx[s]; k >= 0; k = sPar[k]) {
        const float* xk = sXi + 6 * k;
        row[k] -= xk[0] * e[0] + xk[1] * e[1] + xk[2] * e[2] + xk[3] * e[3] + xk[4] * e[4] + xk[5] * e[5];
      }
    }
  }
  __syncthreads();
  const int ty = tid >> 4, tx = tid & 15;
  float acc[T][T];
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) acc[a][b] = 0.f;
  for (int s = 0; s < total; ++s) {
    const float* row = Js + s * ROW;
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
  const int NP = d.NP;
  float* out = d.partial + (size_t)blockIdx.x * NP * NP;
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const int r = ty * T + a, c = tx * T + b;
      if (r < NP && c < NP) out[r * NP + c] = acc[a][b];
    }
  if (tid == 0 && total) atomicAdd(&d.stats[1], total);
}

// Fixed-order FP64 sum of the block partials -> [J r]^T [J r]; the last entry gives E_pose (with the
// prior sum_k (lambda_s S_kk theta_k)^2), recorded as this iteration's energy and as the LM reference.
// A CTA owns 32 consecutive entries (coalesced lanes); its 32 warps take every 32nd partial, then warp 0
// adds the 32 warp sums in order.
constexpr int kReduceThreads = 1024;

__global__ void __launch_bounds__(kReduceThreads) k_reduce_jtj(Dev d, int slot) {
  __shared__ double sm[kReduceThreads / 32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NP = d.NP, n2 = NP * NP;
  const int e = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (e < n2)
    for (int b = w; b < d.nblk_jtj; b += kReduceThreads / 32) s += (double)d.partial[(size_t)b * n2 + e];
  sm[w][lane] = s;
  __syncthreads();
  if (w != 0 || e >= n2) return;
  double t = 0.0;
  for (int k = 0; k < kReduceThreads / 32; ++k) t += sm[k][lane];
  d.A[e] = t;
  if (e == n2 - 1) {
    double E = t;
    for (int k = 0; k < d.L; ++k) E += d.prior2[k] * d.theta[k] * d.theta[k];
    if (slot >= 0) d.energy[slot] = E;
    d.lm_trials[6] = E;
  }
}

static int jtj_smem_bytes(int T, int L) {
  return kBlock * (16 * T + 1) * 4 + L * (int)sizeof(DQ) + 6 * L * 4 + L * 4;
}

void launch_resid_jtj(const Dev& d, int phi_buf, cudaStream_t st) {
  const int T = (d.NP + 15) / 16;
  const int g = d.nblk_jtj;
  const int sm = jtj_smem_bytes(T, d.L);
  switch (T) {
    case 1: k_resid_jtj<1><<<g, kBlock, sm, st>>>(d, phi_buf); break;
    case 2: k_resid_jtj<2><<<g, kBlock, sm, st>>>(d, phi_buf); break;
    case 3: k_resid_jtj<3><<<g, kBlock, sm, st>>>(d, phi_buf); break;
    case 4: k_resid_jtj<4><<<g, kBlock, sm, st>>>(d, phi_buf); break;
    default: k_resid_jtj<5><<<g, kBlock, sm, st>>>(d, phi_buf); break;
  }
}

void launch_reduce_jtj(const Dev& d, int slot, cudaStream_t st) {
  const int n2 = d.NP * d.NP;
  k_reduce_jtj<<<(n2 + 31) / 32, kReduceThreads, 0, st>>>(d, slot);
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
// FP64 Cholesky, right-looking, two block barriers per column: (1) scale column k by 1/L_kk (computed
// with one rsqrt by the thread that finished the pivot in the previous update) into a contiguous copy,
// (2) rank-1 update of the trailing triangle, one warp per row, lanes across the columns.  No FP64
// division is issued.  The two triangular solves run on one warp (warp-synchronous).
// ---------------------------------------------------------------------------------------------
constexpr int kSolveThreads = 256;

__device__ __forceinline__ bool pivot_inv(double p, double& l, double& inv) {
  if (!(p > 0.0)) return false;
  inv = rsqrt(p);
  l = p * inv;
  return true;
}

__global__ void __launch_bounds__(kSolveThreads) k_lm_solve(Dev d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = d.L, NP = d.NP, c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  const int ld = P + 1;
  double* M = reinterpret_cast<double*>(smem_raw);  // [P][P+1]
  double* b = M + (size_t)P * ld;
  double* dg = b + P;
  double* inv = dg + P;
  double* colk = inv + P;
  LinkTable* lt = reinterpret_cast<LinkTable*>(smem_raw + ((((size_t)P * ld + 4 * P) * 8 + 15) & ~(size_t)15));
  __shared__ int bad;
  for (int t = tid; t < (int)(sizeof(LinkTable) / 4); t += nt)
    reinterpret_cast<int*>(lt)[t] = reinterpret_cast<const int*>(d.links)[t];
  double lam = *d.lam;
  for (int t = 0; t < c; ++t) lam = fmin(lam * 10.0, 1e7);
  for (int r = tid; r < P; r += nt) dg[r] = d.A[r * NP + r] + d.prior2[r];
  __syncthreads();
  for (int r = tid; r < P; r += nt) b[r] = dg[r] == 0.0 ? 0.0 : d.A[r * NP + P] + d.prior2[r] * d.theta[r];
  for (int e = tid; e < P * P; e += nt) {
    const int r = e / P, q = e % P;
    const bool frozen = dg[r] == 0.0 || dg[q] == 0.0;
    M[r * ld + q] = frozen ? (r == q ? 1.0 : 0.0) : d.A[r * NP + q] + (r == q ? d.prior2[r] + lam * dg[r] : 0.0);
  }
  __syncthreads();
  if (tid == 0) {
    double l, iv;
    bad = !pivot_inv(M[0], l, iv);
    if (!bad) { M[0] = l; inv[0] = iv; }
  }
  __syncthreads();
  for (int k = 0; k < P && !bad; ++k) {
    const double ik = inv[k];
    for (int r = k + 1 + tid; r < P; r += nt) {
      const double v = M[r * ld + k] * ik;
      M[r * ld + k] = v;
      colk[r] = v;
    }
    __syncthreads();
    for (int r = k + 1 + warp; r < P; r += nwarp) {
      const double lrk = colk[r];
      double* row = M + (size_t)r * ld;
      for (int q = k + 1 + lane; q <= r; q += 32) row[q] = fma(-lrk, colk[q], row[q]);
      if (r == k + 1 && lane == 0) {  // the next pivot is final: factor it now
        double l, iv;
        if (pivot_inv(row[r], l, iv)) { row[r] = l; inv[r] = iv; } else { bad = 1; }
      }
    }
    __syncthreads();
  }
  const int fail = bad;
  if (!fail && warp == 0) {
    for (int k = 0; k < P; ++k) {  // L y = b
      __syncwarp();
      const double yk = b[k] * inv[k];
      __syncwarp();
      if (lane == 0) b[k] = yk;
      for (int r = k + 1 + lane; r < P; r += 32) b[r] = fma(-M[r * ld + k], yk, b[r]);
    }
    for (int k = P - 1; k >= 0; --k) {  // L^T x = y
      __syncwarp();
      const double xk = b[k] * inv[k];
      __syncwarp();
      if (lane == 0) b[k] = xk;
      for (int r = lane; r < k; r += 32) b[r] = fma(-M[k * ld + r], xk, b[r]);
    }
  }
  __syncthreads();
  double* thc = d.theta_c + (size_t)c * P;
  for (int j = tid; j < P; j += nt) thc[j] = fail ? d.theta[j] : d.theta[j] - b[j];
  if (tid == 0) d.lm_ok[c] = !fail;
  __syncthreads();
  for (int j = tid; j < P; j += nt) {
    DQ H;
    float xi[6];
    fk_link(*lt, thc, j, &H, xi);
    d.Hd_c[(size_t)c * P + j] = H;
    float* xo = d.xi_c + ((size_t)c * P + j) * 8;
    for (int q = 0; q < 6; ++q) xo[q] = xi[q];
    xo[6] = xo[7] = 0.f;
  }
}

// Energy of each candidate at the fixed association (normals and p~ held), then the accept step:
// the first candidate with E_c <= E wins (lambda <- lambda_c / 10); if none, Theta stays and
// lambda <- min(lambda_5 * 10, 1e7).  The last block to finish does the selection.
__global__ void __launch_bounds__(kBlock) k_lm_eval(Dev d, int phi_buf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DQ* sH = reinterpret_cast<DQ*>(smem_raw);  // [kCandidates][L]
  __shared__ int sok[kCandidates];
  __shared__ double swarp[kBlock / 32][kCandidates];
  __shared__ bool last;
  const int L = d.L, tid = threadIdx.x;
  for (int t = tid; t < kCandidates * L; t += kBlock) sH[t] = d.Hd_c[t];
  if (tid < kCandidates) sok[tid] = d.lm_ok[tid];
  __syncthreads();
  float e[kCandidates];
#pragma unroll
  for (int c = 0; c < kCandidates; ++c) e[c] = 0.f;
  const int i = blockIdx.x * kBlock + tid;
  if (i < d.V) {
    const Acc4 a4 = d.acc[i];
    const float4 nn = d.n[i];
    if (a4.w >= 1 && nn.w > 0.f) {
      const float inv = 1.f / ((float)a4.w * kFix);
      const float3 pm = make_float3((float)a4.x * inv, (float)a4.y * inv, (float)a4.z * inv);
      const float4 v = d.v[i], x0 = d.v0[i], ph = d.phi[phi_buf][i];
      const float3 x = make_float3(x0.x + ph.x, x0.y + ph.y, x0.z + ph.z);
      const uchar4 bi = d.bidx[i];
      const float4 bw = d.bw[i];
#pragma unroll
      for (int c = 0; c < kCandidates; ++c) {
        if (!sok[c]) continue;
        float sg[4];
        const DQ H = blend_bones(sH + c * L, bi, bw, sg);
        const float3 vc = dq_point(H, x);
        const float r = nn.x * (v.x - vc.x + pm.x) + nn.y * (v.y - vc.y + pm.y) + nn.z * (v.z - vc.z + pm.z);
        e[c] = r * r;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kCandidates; ++c)
    for (int o = 16; o > 0; o >>= 1) e[c] += __shfl_xor_sync(0xffffffffu, e[c], o);
  if ((tid & 31) == 0)
    for (int c = 0; c < kCandidates; ++c) swarp[tid >> 5][c] = e[c];
  __syncthreads();
  if (tid < kCandidates) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += swarp[w][tid];
    d.epart[(size_t)blockIdx.x * 8 + tid] = s;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&d.counter[0], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double red[kBlock][kCandidates];
  __shared__ double Ec[kCandidates];
  {
    double s6[kCandidates] = {0, 0, 0, 0, 0, 0};
    for (int b = tid; b < (int)gridDim.x; b += kBlock)
      for (int c = 0; c < kCandidates; ++c) s6[c] += __ldcg(d.epart + (size_t)b * 8 + c);
    for (int c = 0; c < kCandidates; ++c) red[tid][c] = s6[c];
  }
  __syncthreads();
  for (int h = kBlock / 2; h > 0; h >>= 1) {
    if (tid < h)
      for (int c = 0; c < kCandidates; ++c) red[tid][c] += red[tid + h][c];
    __syncthreads();
  }
  if (tid < kCandidates) {
    double s = red[0][tid];
    const double* thc = d.theta_c + (size_t)tid * L;
    for (int k = 0; k < L; ++k) s += d.prior2[k] * thc[k] * thc[k];
    Ec[tid] = sok[tid] ? s : __longlong_as_double(0x7ff0000000000000ll);
  }
  __syncthreads();
  __shared__ int acc_c;
  if (tid == 0) {
    const double E = d.lm_trials[6];
    double lam = *d.lam;
    int a = -1;
    for (int c = 0; c < kCandidates; ++c) {
      d.lm_trials[c] = Ec[c];
      if (a < 0 && sok[c] && Ec[c] <= E) a = c;
    }
    if (a >= 0) {
      for (int t = 0; t < a; ++t) lam = fmin(lam * 10.0, 1e7);
      lam = fmax(lam / 10.0, 1e-7);
    } else {
      for (int t = 0; t < kCandidates; ++t) lam = fmin(lam * 10.0, 1e7);
    }
    *d.lam = lam;
    d.lm_trials[7] = (double)a;
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

static int lm_solve_smem(int L) {
  return (int)(((((size_t)L * (L + 1) + 4 * L) * 8 + 15) & ~(size_t)15) + sizeof(LinkTable));
}

void launch_lm_solve(const Dev& d, cudaStream_t st) {
  k_lm_solve<<<kCandidates, kSolveThreads, lm_solve_smem(d.L), st>>>(d);
}

void launch_lm_eval(const Dev& d, int phi_buf, cudaStream_t st) {
  k_lm_eval<<<d.nblk_v, kBlock, kCandidates * d.L * sizeof(DQ), st>>>(d, phi_buf);
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

__device__ __forceinline__ void block_energy_to_slot(Dev& d, float e, int slot, int ticket) {
  __shared__ double sw[kBlock];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += sw[w];
    d.epart[(size_t)blockIdx.x * 8] = s;
    __threadfence();
    last = atomicAdd(&d.counter[ticket], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;  // fixed order: strided per thread, then a tree over the threads
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kBlock) s += __ldcg(d.epart + (size_t)b * 8);
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

__global__ void __launch_bounds__(kBlock) k_shape(Dev d, int src, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DQ* sHd = reinterpret_cast<DQ*>(smem_raw);
  for (int j = threadIdx.x; j < d.L; j += kBlock) sHd[j] = d.Hd[j];
  __syncthreads();
  const int i = blockIdx.x * kBlock + threadIdx.x;
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
      const float inv = 1.f / ((float)a4.w * kFix);
      r = nn.x * (float)a4.x * inv + nn.y * (float)a4.y * inv + nn.z * (float)a4.z * inv;
      float sg[4];
      const DQ H = blend_bones(sHd, d.bidx[i], d.bw[i], sg);
      const float4 ah = qscale(H.r, rsqrtf(qdot(H.r, H.r)));
      const float4 q = qmul(qmul(qconj(ah), make_float4(0.f, nn.x, nn.y, nn.z)), ah);  // R^T n
      g = make_float3(-q.y, -q.z, -q.w);
    }
    e = r * r + d.lambda_phi * dot3(pi, pi);
    float3 sd = make_float3(0.f, 0.f, 0.f);
    int nn_count = 0;
    const int4 nb = d.nbr[i];
    const int nbs[4] = {nb.x, nb.y, nb.z, nb.w};
    for (int t = 0; t < d.knn; ++t) {
      if (nbs[t] < 0) continue;
      const float3 q = f3(phi[nbs[t]]);
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
  block_energy_to_slot(d, e, slot, 1);
}

// Further Jacobi sweeps: r_i is updated linearly, r_i = r0_i + g_i . (phi_i - phi0_i).
__global__ void __launch_bounds__(kBlock) k_shape_sweep(Dev d, int src) {
  const int i = blockIdx.x * kBlock + threadIdx.x;
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
  for (int t = 0; t < d.knn; ++t) {
    if (nbs[t] < 0) continue;
    const float3 q = f3(phi[nbs[t]]);
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

// Returns the buffer that holds Phi after the step.
int launch_shape(const Dev& d, int phi_src, int slot, cudaStream_t st) {
  k_shape<<<d.nblk_v, kBlock, d.L * sizeof(DQ), st>>>(d, phi_src, slot);
  int cur = 1 - phi_src;
  for (int s = 1; s < d.shape_sweeps; ++s) {
    k_shape_sweep<<<d.nblk_v, kBlock, 0, st>>>(d, cur);
    cur = 1 - cur;
  }
  return cur;
}

void configure_kernels() {
  cudaFuncSetAttribute(k_resid_jtj<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(1, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(2, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(3, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(4, kMaxLinks));
  cudaFuncSetAttribute(k_resid_jtj<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, jtj_smem_bytes(5, kMaxLinks));
  cudaFuncSetAttribute(k_lm_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, lm_solve_smem(kMaxLinks));
}

}  // namespace trk

// authoring.cu -- template authoring (the template construction of the paper's Sec. 3.2 setup): a
// low-resolution polygon cage with skin weights is refined by Catmull-Clark subdivision, the weights
// interpolated with the same stencils as the positions, then each vertex keeps its 4 largest weights
// (renormalised) and every quad is split into two triangles.
//
// Each level's connectivity is combinatorial and built on the host: the new vertices are the vertex
// points of the old vertices (same indices), then the edge points in the order the edges first appear
// when the faces are walked in order, then the face points in face order; face (v_0 .. v_{k-1}) becomes
// the quads (v_i', e(v_i, v_{i+1}), f', e(v_{i-1}, v_i)).  The device computes the points of every
// attribute (x, y, z and one weight per bone), one thread per (point, attribute):
//   face point   = mean of the face's vertices;
//   edge point   = (a + b + f_a + f_b) / 4, or the midpoint on a boundary edge;
//   vertex point = (F + 2 R + (n - 3) P) / n (F: mean of the n adjacent face points, R: mean of the
//                  incident edges' midpoints), (6 P + the two boundary neighbours) / 8 on a boundary.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/trk.h"
#include "trk_internal.cuh"

namespace trk {
namespace {

constexpr int kCCBlock = 256;

struct Level {
  int V = 0, F = 0, E = 0;
  std::vector<int> face_off, face_vert;          // the polygons of this level
  std::vector<int> ea, eb, efa, efb;             // per edge: end points, adjacent faces (-1: boundary)
  std::vector<int> vf_off, vf;                   // vertex -> incident faces
  std::vector<int> ve_off, ve;                   // vertex -> incident edges
  std::vector<int> quads;                        // the next level's faces, 4 per corner
};

// Builds the edges, adjacency and the next level's quads of a polygon mesh.
void build_level(Level& L) {
  const int nc = L.face_off[L.F];
  std::vector<int> head(L.V, -1), next;
  std::vector<int> fedge(nc);
  auto find = [&](int a, int b) {
    const int lo = std::min(a, b), hi = std::max(a, b);
    for (int e = head[lo]; e >= 0; e = next[e])
      if (std::min(L.ea[e], L.eb[e]) == lo && std::max(L.ea[e], L.eb[e]) == hi) return e;
    return -1;
  };
  for (int f = 0; f < L.F; ++f) {
    const int k = L.face_off[f + 1] - L.face_off[f];
    for (int i = 0; i < k; ++i) {
      const int a = L.face_vert[L.face_off[f] + i], b = L.face_vert[L.face_off[f] + (i + 1) % k];
      int e = find(a, b);
      if (e < 0) {
        e = (int)L.ea.size();
        L.ea.push_back(a);
        L.eb.push_back(b);
        L.efa.push_back(f);
        L.efb.push_back(-1);
        next.push_back(head[std::min(a, b)]);
        head[std::min(a, b)] = e;
      } else {
        L.efb[e] = f;
      }
      fedge[L.face_off[f] + i] = e;
    }
  }
  L.E = (int)L.ea.size();
  L.vf_off.assign(L.V + 1, 0);
  for (int i = 0; i < nc; ++i) L.vf_off[L.face_vert[i] + 1]++;
  for (int v = 0; v < L.V; ++v) L.vf_off[v + 1] += L.vf_off[v];
  L.vf.resize(std::max(nc, 1));
  {
    std::vector<int> fill(L.vf_off.begin(), L.vf_off.end() - 1);
    for (int f = 0; f < L.F; ++f)
      for (int i = L.face_off[f]; i < L.face_off[f + 1]; ++i) L.vf[fill[L.face_vert[i]]++] = f;
  }
  L.ve_off.assign(L.V + 1, 0);
  for (int e = 0; e < L.E; ++e) {
    L.ve_off[L.ea[e] + 1]++;
    L.ve_off[L.eb[e] + 1]++;
  }
  for (int v = 0; v < L.V; ++v) L.ve_off[v + 1] += L.ve_off[v];
  L.ve.resize(std::max(2 * L.E, 1));
  {
    std::vector<int> fill(L.ve_off.begin(), L.ve_off.end() - 1);
    for (int e = 0; e < L.E; ++e) {
      L.ve[fill[L.ea[e]]++] = e;
      L.ve[fill[L.eb[e]]++] = e;
    }
  }
  L.quads.resize(4 * (size_t)nc);
  int q = 0;
  for (int f = 0; f < L.F; ++f) {
    const int k = L.face_off[f + 1] - L.face_off[f];
    for (int i = 0; i < k; ++i, ++q) {
      L.quads[4 * q] = L.face_vert[L.face_off[f] + i];
      L.quads[4 * q + 1] = L.V + fedge[L.face_off[f] + i];
      L.quads[4 * q + 2] = L.V + L.E + f;
      L.quads[4 * q + 3] = L.V + fedge[L.face_off[f] + (i + k - 1) % k];
    }
  }
}

__global__ void __launch_bounds__(kCCBlock) k_cc_face(const float* __restrict__ a, int A, const int* __restrict__ fo,
                                                      const int* __restrict__ fv, int F, float* __restrict__ out) {
  const long long t = (long long)blockIdx.x * kCCBlock + threadIdx.x;
  if (t >= (long long)F * A) return;
  const int f = (int)(t / A), c = (int)(t % A);
  float s = 0.f;
  for (int i = fo[f]; i < fo[f + 1]; ++i) s += a[(size_t)fv[i] * A + c];
  out[(size_t)f * A + c] = s / (float)(fo[f + 1] - fo[f]);
}

__global__ void __launch_bounds__(kCCBlock) k_cc_edge(const float* __restrict__ a, const float* __restrict__ fp, int A,
                                                      const int* __restrict__ ea, const int* __restrict__ eb,
                                                      const int* __restrict__ efa, const int* __restrict__ efb, int E,
                                                      float* __restrict__ out) {
  const long long t = (long long)blockIdx.x * kCCBlock + threadIdx.x;
  if (t >= (long long)E * A) return;
  const int e = (int)(t / A), c = (int)(t % A);
  const float pa = a[(size_t)ea[e] * A + c], pb = a[(size_t)eb[e] * A + c];
  out[(size_t)e * A + c] = efb[e] < 0 ? 0.5f * (pa + pb)
                                      : 0.25f * (pa + pb + fp[(size_t)efa[e] * A + c] + fp[(size_t)efb[e] * A + c]);
}

__global__ void __launch_bounds__(kCCBlock) k_cc_vertex(const float* __restrict__ a, const float* __restrict__ fp,
                                                        int A, const int* __restrict__ vf_off,
                                                        const int* __restrict__ vf, const int* __restrict__ ve_off,
                                                        const int* __restrict__ ve, const int* __restrict__ ea,
                                                        const int* __restrict__ eb, const int* __restrict__ efb, int V,
                                                        float* __restrict__ out) {
  const long long t = (long long)blockIdx.x * kCCBlock + threadIdx.x;
  if (t >= (long long)V * A) return;
  const int v = (int)(t / A), c = (int)(t % A);
  const float P = a[(size_t)v * A + c];
  float Fs = 0.f, Rs = 0.f, Bs = 0.f;
  int nB = 0;
  for (int i = vf_off[v]; i < vf_off[v + 1]; ++i) Fs += fp[(size_t)vf[i] * A + c];
  const int nR = ve_off[v + 1] - ve_off[v];
  for (int i = ve_off[v]; i < ve_off[v + 1]; ++i) {
    const int e = ve[i];
    const int o = ea[e] == v ? eb[e] : ea[e];
    const float po = a[(size_t)o * A + c];
    Rs += 0.5f * (P + po);
    if (efb[e] < 0) {
      Bs += po;
      ++nB;
    }
  }
  const int nF = vf_off[v + 1] - vf_off[v];
  float r;
  if (nB > 0) {
    r = nB == 2 ? (6.f * P + Bs) / 8.f : P;
  } else if (nF > 0) {
    const float n = (float)nF;
    r = (Fs / n + 2.f * Rs / (float)nR + (n - 3.f) * P) / n;
  } else {
    r = P;
  }
  out[(size_t)v * A + c] = r;
}

// The 4 largest weights of each vertex (ties to the smaller bone), renormalised to sum 1.
__global__ void __launch_bounds__(kCCBlock) k_top4(const float* __restrict__ a, int A, int nb, int V,
                                                   float* __restrict__ xyz, uchar4* __restrict__ bi,
                                                   float4* __restrict__ bw) {
  const int v = blockIdx.x * kCCBlock + threadIdx.x;
  if (v >= V) return;
  const float* w = a + (size_t)v * A + 3;
  int id[4] = {0, 0, 0, 0};
  float val[4] = {-1.f, -1.f, -1.f, -1.f};
  for (int b = 0; b < nb; ++b) {
    const float x = w[b];
    if (!(x > val[3])) continue;  // strictly larger than the fourth: an equal later bone loses the tie
    int p = 3;
    while (p > 0 && x > val[p - 1]) {
      val[p] = val[p - 1];
      id[p] = id[p - 1];
      --p;
    }
    val[p] = x;
    id[p] = b;
  }
  float s = 0.f;
  for (int k = 0; k < 4; ++k) {
    if (val[k] < 0.f) val[k] = 0.f;
    s += val[k];
  }
  const float inv = s > 0.f ? 1.f / s : 0.f;
  xyz[3 * (size_t)v] = a[(size_t)v * A];
  xyz[3 * (size_t)v + 1] = a[(size_t)v * A + 1];
  xyz[3 * (size_t)v + 2] = a[(size_t)v * A + 2];
  bi[v] = make_uchar4(id[0], id[1], id[2], id[3]);
  bw[v] = make_float4(val[0] * inv, val[1] * inv, val[2] * inv, val[3] * inv);
}

template <typename T>
cudaError_t upload(T** d, const std::vector<T>& h, std::vector<void*>& owned) {
  cudaError_t e = cudaMalloc(d, sizeof(T) * std::max<size_t>(h.size(), 1));
  if (e != cudaSuccess) return e;
  owned.push_back(*d);
  return h.empty() ? cudaSuccess : cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

bool valid_cage(const int32_t* face_off, const int32_t* face_vert, int V, int F) {
  if (!face_off || !face_vert || V < 1 || F < 1 || face_off[0] != 0) return false;
  for (int f = 0; f < F; ++f)
    if (face_off[f + 1] - face_off[f] < 3) return false;
  for (int i = 0; i < face_off[F]; ++i)
    if (face_vert[i] < 0 || face_vert[i] >= V) return false;
  return true;
}

// The topology of every level (host only).
std::vector<Level> topology(const int32_t* face_off, const int32_t* face_vert, int V, int F, int levels) {
  std::vector<Level> lv(levels);
  Level cur;
  cur.V = V;
  cur.F = F;
  cur.face_off.assign(face_off, face_off + F + 1);
  cur.face_vert.assign(face_vert, face_vert + face_off[F]);
  for (int l = 0; l < levels; ++l) {
    build_level(cur);
    Level nxt;
    nxt.V = cur.V + cur.E + cur.F;
    nxt.F = (int)(cur.quads.size() / 4);
    nxt.face_off.resize(nxt.F + 1);
    for (int i = 0; i <= nxt.F; ++i) nxt.face_off[i] = 4 * i;
    nxt.face_vert = cur.quads;
    lv[l] = std::move(cur);
    cur = std::move(nxt);
  }
  lv.push_back(std::move(cur));  // the final mesh (no edges built)
  return lv;
}

}  // namespace
}  // namespace trk

using namespace trk;

extern "C" {

trk_status trk_subdivide_counts(const int32_t* face_off, const int32_t* face_vert, int32_t n_verts, int32_t n_faces,
                                int32_t levels, int32_t* n_verts_out, int32_t* n_tris_out) {
  if (!valid_cage(face_off, face_vert, n_verts, n_faces) || levels < 1 || levels > 4 || !n_verts_out || !n_tris_out)
    return set_error(TRK_ERR_INVALID_ARG, "trk_subdivide_counts: bad cage or levels (1..4)");
  const auto lv = topology(face_off, face_vert, n_verts, n_faces, levels);
  *n_verts_out = lv.back().V;
  *n_tris_out = 2 * lv.back().F;
  return TRK_OK;
}

trk_status trk_subdivide(const float* verts, const int32_t* face_off, const int32_t* face_vert, int32_t n_verts,
                         int32_t n_faces, const uint8_t* bone_idx, const float* bone_w, int32_t n_bones, int32_t levels,
                         float* verts_out, int32_t* tris_out, uint8_t* bone_idx_out, float* bone_w_out) {
  if (!verts || !bone_idx || !bone_w || !verts_out || !tris_out || !bone_idx_out || !bone_w_out || n_bones < 1 ||
      n_bones > 255 || levels < 1 || levels > 4 || !valid_cage(face_off, face_vert, n_verts, n_faces))
    return set_error(TRK_ERR_INVALID_ARG, "trk_subdivide: bad arguments");
  for (int i = 0; i < 4 * n_verts; ++i)
    if (bone_idx[i] >= n_bones) return set_error(TRK_ERR_INVALID_ARG, "trk_subdivide: bone index out of range");
  const auto lv = topology(face_off, face_vert, n_verts, n_faces, levels);
  const int A = 3 + n_bones;
  // attributes of the cage: position, then a dense weight per bone
  std::vector<float> a0((size_t)n_verts * A, 0.f);
  for (int v = 0; v < n_verts; ++v) {
    for (int c = 0; c < 3; ++c) a0[(size_t)v * A + c] = verts[3 * v + c];
    for (int k = 0; k < 4; ++k) a0[(size_t)v * A + 3 + bone_idx[4 * v + k]] += bone_w[4 * v + k];
  }
  std::vector<void*> owned;
  cudaError_t e = cudaSuccess;
  float* cur = nullptr;
  if ((e = upload(&cur, a0, owned)) != cudaSuccess) goto done;
  for (int l = 0; l < levels; ++l) {
    const Level& L = lv[l];
    float* nxt = nullptr;
    int *fo, *fv, *ea, *eb, *efa, *efb, *vfo, *vf, *veo, *ve;
    if ((e = cudaMalloc(&nxt, sizeof(float) * (size_t)(L.V + L.E + L.F) * A)) != cudaSuccess) goto done;
    owned.push_back(nxt);
    if ((e = upload(&fo, L.face_off, owned)) || (e = upload(&fv, L.face_vert, owned)) || (e = upload(&ea, L.ea, owned)) ||
        (e = upload(&eb, L.eb, owned)) || (e = upload(&efa, L.efa, owned)) || (e = upload(&efb, L.efb, owned)) ||
        (e = upload(&vfo, L.vf_off, owned)) || (e = upload(&vf, L.vf, owned)) || (e = upload(&veo, L.ve_off, owned)) ||
        (e = upload(&ve, L.ve, owned)))
      goto done;
    {
      float* fp = nxt + (size_t)(L.V + L.E) * A;
      const long long nf = (long long)L.F * A, ne = (long long)L.E * A, nv = (long long)L.V * A;
      k_cc_face<<<(unsigned)((nf + kCCBlock - 1) / kCCBlock), kCCBlock>>>(cur, A, fo, fv, L.F, fp);
      if (ne) k_cc_edge<<<(unsigned)((ne + kCCBlock - 1) / kCCBlock), kCCBlock>>>(cur, fp, A, ea, eb, efa, efb, L.E,
                                                                                   nxt + (size_t)L.V * A);
      k_cc_vertex<<<(unsigned)((nv + kCCBlock - 1) / kCCBlock), kCCBlock>>>(cur, fp, A, vfo, vf, veo, ve, ea, eb, efb,
                                                                             L.V, nxt);
      if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    }
    cur = nxt;
  }
  {
    const int Vn = lv.back().V;
    float* dxyz;
    uchar4* dbi;
    float4* dbw;
    if ((e = cudaMalloc(&dxyz, sizeof(float) * 3 * (size_t)Vn)) != cudaSuccess) goto done;
    owned.push_back(dxyz);
    if ((e = cudaMalloc(&dbi, sizeof(uchar4) * (size_t)Vn)) != cudaSuccess) goto done;
    owned.push_back(dbi);
    if ((e = cudaMalloc(&dbw, sizeof(float4) * (size_t)Vn)) != cudaSuccess) goto done;
    owned.push_back(dbw);
    k_top4<<<(Vn + kCCBlock - 1) / kCCBlock, kCCBlock>>>(cur, A, n_bones, Vn, dxyz, dbi, dbw);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    if ((e = cudaMemcpy(verts_out, dxyz, sizeof(float) * 3 * (size_t)Vn, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(bone_idx_out, dbi, sizeof(uchar4) * (size_t)Vn, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(bone_w_out, dbw, sizeof(float4) * (size_t)Vn, cudaMemcpyDeviceToHost)))
      goto done;
    // each quad (a, b, c, d) as the triangles (a, b, c) and (a, c, d)
    const std::vector<int>& q = lv.back().face_vert;
    for (size_t i = 0; i < q.size() / 4; ++i) {
      const int* x = &q[4 * i];
      int32_t* t = tris_out + 6 * i;
      t[0] = x[0]; t[1] = x[1]; t[2] = x[2];
      t[3] = x[0]; t[4] = x[2]; t[5] = x[3];
    }
  }
done:
  for (void* p : owned) cudaFree(p);
  if (e != cudaSuccess) return set_error(e == cudaErrorMemoryAllocation ? TRK_ERR_OOM : TRK_ERR_CUDA, cudaGetErrorString(e));
  return TRK_OK;
}

}  // extern "C"

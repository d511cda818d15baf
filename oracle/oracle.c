/*
 * oracle.c -- plain, slow, single-threaded FP64 CPU implementation of one tracking frame of
 * "Dynamic High Resolution Deformable Articulated Tracking" (Walsman, Wan, Schmidt, Fox; 3DV 2017).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this file: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg use it.  It shares no code, header,
 * table or constant with the CUDA implementation.
 *
 * Every function follows the paper's section / equation in the order the paper states it.  Where the
 * paper is silent or garbled, the reading taken is named R1..R19 (the list and its justification are
 * kept with the design notes of the repository):
 *   R1  antipodality: each bone's dual quaternion is sign-aligned with that of the vertex's heaviest bone
 *   R2  the blended dual quaternion is applied with the homogeneous (normalising) point map
 *   R4  vertex normals: normalised sum of incident (unnormalised) face cross products
 *   R5  pixel (px,py) samples the ray through integer image coordinates (px,py)
 *   R6  z-buffer coverage: inclusive edge test, both windings; depth ties go to the smaller triangle
 *   R7  visibility: front-facing, rounded pixel inside the image, not behind the z-buffer by > eps_vis
 *   R8  association ties go to the smaller vertex index
 *   R9  association window half-size W and cutoff tau are parameters
 *   R10 pose prior weight S_kk = n_k/|V| (n_k = vertices weighted to the subtree of link k), times a mask
 *   R22 the coupled shape step: the whole shape energy's damped Gauss-Newton system, solved by PCG
 *   R23 raster-ID association: the nearest corner of the triangle rasterised at the pixel
 *   R12 derivative block of link j's offset w.r.t. theta_k uses the chain from k to j (no double count)
 *   R13 LM damping uses diag of the prior-augmented matrix; a parameter with zero diagonal is frozen
 *   R14 LM schedule: lambda x10 on reject (<= 5 retries, energy at fixed association), /10 on accept
 *   R15 shape step: Gauss-Newton on the per-vertex local energy with neighbours frozen (Jacobi)
 *   R16 N(i) = 4 nearest other bind-pose vertices, ties to the smaller index, directed
 * Compile with -ffp-contract=off so that the results do not depend on the host's FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------------ */
/* Quaternions and dual quaternions (Sec. 3.1; Daniilidis 1999).  Storage: (w, x, y, z).            */
/* ------------------------------------------------------------------------------------------------ */
typedef struct { double w, x, y, z; } quat;
typedef struct { quat r, d; } dquat; /* H = r + d eps, eps^2 = 0 */

static quat q_make(double w, double x, double y, double z) { quat q = {w, x, y, z}; return q; }
static quat q_mul(quat a, quat b) {
  return q_make(a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
                a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
                a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
                a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w);
}
static quat q_conj(quat a) { return q_make(a.w, -a.x, -a.y, -a.z); }
static quat q_add(quat a, quat b) { return q_make(a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z); }
static quat q_scale(quat a, double s) { return q_make(a.w * s, a.x * s, a.y * s, a.z * s); }
static double q_dot(quat a, quat b) { return a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z; }

static dquat dq_identity(void) { dquat h; h.r = q_make(1, 0, 0, 0); h.d = q_make(0, 0, 0, 0); return h; }
static dquat dq_zero(void) { dquat h; h.r = q_make(0, 0, 0, 0); h.d = q_make(0, 0, 0, 0); return h; }
/* (a | b)(c | d) = (ac | ad + bc) since eps^2 = 0 */
static dquat dq_mul(dquat a, dquat b) {
  dquat h; h.r = q_mul(a.r, b.r); h.d = q_add(q_mul(a.r, b.d), q_mul(a.d, b.r)); return h;
}
/* inverse of a unit dual quaternion: conjugate both parts */
static dquat dq_conj(dquat a) { dquat h; h.r = q_conj(a.r); h.d = q_conj(a.d); return h; }
static dquat dq_axpy(dquat acc, double s, dquat a) {
  dquat h; h.r = q_add(acc.r, q_scale(a.r, s)); h.d = q_add(acc.d, q_scale(a.d, s)); return h;
}
static dquat dq_load(const double* p) {
  dquat h; h.r = q_make(p[0], p[1], p[2], p[3]); h.d = q_make(p[4], p[5], p[6], p[7]); return h;
}
static void dq_store(dquat h, double* p) {
  p[0] = h.r.w; p[1] = h.r.x; p[2] = h.r.y; p[3] = h.r.z;
  p[4] = h.d.w; p[5] = h.d.x; p[6] = h.d.y; p[7] = h.d.z;
}

/* Eq. H_hinge: cos(theta/2) + z sin(theta/2) + 0 eps.   Eq. H_prismatic: 1 + z (theta/2) eps. */
static dquat joint_dq(int type, const double* z, double th) {
  dquat h = dq_identity();
  if (type == 0) {
    double c = cos(0.5 * th), s = sin(0.5 * th);
    h.r = q_make(c, z[0] * s, z[1] * s, z[2] * s);
  } else {
    h.d = q_make(0, z[0] * 0.5 * th, z[1] * 0.5 * th, z[2] * 0.5 * th);
  }
  return h;
}
/* Sec. 4.2: derivative of the joint transform.  Hinge: (z cos(theta/2) - sin(theta/2)) / 2.
 * Prismatic: (z / 2) eps. */
static dquat joint_dq_deriv(int type, const double* z, double th) {
  dquat h = dq_zero();
  if (type == 0) {
    double c = cos(0.5 * th), s = sin(0.5 * th);
    h.r = q_make(-0.5 * s, 0.5 * c * z[0], 0.5 * c * z[1], 0.5 * c * z[2]);
  } else {
    h.d = q_make(0, 0.5 * z[0], 0.5 * z[1], 0.5 * z[2]);
  }
  return h;
}

/* R2: point map of a (possibly non-unit) blended dual quaternion H = (a | b):
 *   T(H, x) = vec(a x a*) / |a|^2 + 2 vec(b a*) / |a|^2                                            */
static void dq_point(dquat H, const double* x, double* out) {
  quat a = H.r, b = H.d;
  double N = q_dot(a, a);
  quat X = q_make(0, x[0], x[1], x[2]);
  quat t1 = q_mul(q_mul(a, X), q_conj(a));
  quat t2 = q_mul(b, q_conj(a));
  out[0] = (t1.x + 2.0 * t2.x) / N;
  out[1] = (t1.y + 2.0 * t2.y) / N;
  out[2] = (t1.z + 2.0 * t2.z) / N;
}

/* Directional derivative of T(H, x) (R2) along dH = (da | db), at fixed x, by the product rule:
 *   dT = [vec(da X a* + a X da*) + 2 vec(db a* + b da*)] / N  -  2 T <a, da> / N,  N = |a|^2.     */
static void dq_point_dir(dquat H, const double* x, dquat dH, double* out) {
  quat a = H.r, b = H.d, da = dH.r, db = dH.d;
  double N = q_dot(a, a);
  double T[3];
  dq_point(H, x, T);
  quat X = q_make(0, x[0], x[1], x[2]);
  quat u1 = q_add(q_mul(q_mul(da, X), q_conj(a)), q_mul(q_mul(a, X), q_conj(da)));
  quat u2 = q_add(q_mul(db, q_conj(a)), q_mul(b, q_conj(da)));
  double s = 2.0 * q_dot(a, da) / N;
  out[0] = (u1.x + 2.0 * u2.x) / N - s * T[0];
  out[1] = (u1.y + 2.0 * u2.y) / N - s * T[1];
  out[2] = (u1.z + 2.0 * u2.z) / N - s * T[2];
}

/* Rotation matrix of a unit quaternion (textbook), row-major. */
static void q_to_rot(quat q, double* R) {
  double w = q.w, x = q.x, y = q.y, z = q.z;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------------------------------ */
/* Model                                                                                             */
/* ------------------------------------------------------------------------------------------------ */
typedef struct {
  int32_t pose_iters, shape_iters, shape_sweeps, window_half, knn, shape_solver; /* 0 Jacobi (R15), 1 PCG (R22) */
  double lambda_k0, lambda_s, lambda_phi, lambda_N, lambda_w, cutoff, eps_vis, z_near;
  int32_t association, pad2_; /* 0 window search (Sec. 4.1), 1 nearest corner of the rasterised triangle (R23) */
} orc_params;

typedef struct {
  int L, V, F, W, H;
  int* parent;
  int* jtype;
  double* axis;     /* [L][3] */
  dquat* off;       /* [L] H_{P(j),j} */
  double* prior_mask;
  double* v0;       /* [V][3] */
  int* tri;         /* [F][3] */
  int* bidx;        /* [V][4] */
  double* bw;       /* [V][4] */
  double fx, fy, cx, cy;
  orc_params p;
  dquat* bind;      /* [L] H^0_{0,j} */
  double* S;        /* [L] prior weights (R10) */
  int* nbr;         /* [V][knn] (-1 pads) */
  /* tracking state, carried across frames (R14, schedule) */
  double* theta;
  double* phi;      /* [V][3] */
  double lam;
} orc_model;

static void* xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

/* Sec. 3.1 forward kinematics: H_{0,j} = H_{0,P(j)} H_{P(j),j} H_j(theta_j), H_{0,world} = I.
 * Also H_{j,Delta} = H_{0,j} (H^0_{0,j})^{-1} (Sec. 4.2). */
static void fk(const orc_model* m, const double* theta, dquat* H0, dquat* Hd) {
  for (int j = 0; j < m->L; ++j) {
    dquat hp = m->parent[j] < 0 ? dq_identity() : H0[m->parent[j]];
    dquat hj = joint_dq(m->jtype[j], m->axis + 3 * j, theta[j]);
    H0[j] = dq_mul(dq_mul(hp, m->off[j]), hj);
    if (Hd) Hd[j] = dq_mul(H0[j], dq_conj(m->bind[j]));
  }
}

/* Eq. H_Sigma with R1: sum_j w_ij s_ij H_{j,Delta}; s_ij aligns each bone with the heaviest bone j*
 * (largest weight, ties to the smaller link index). */
static dquat blend(const orc_model* m, const dquat* Hd, int i, double* sgn /*[4] or NULL*/) {
  int jstar = -1;
  double wstar = -1.0;
  for (int s = 0; s < 4; ++s) {
    double w = m->bw[4 * i + s];
    int j = m->bidx[4 * i + s];
    if (w > 0 && (w > wstar || (w == wstar && j < jstar))) { wstar = w; jstar = j; }
  }
  dquat acc = dq_zero();
  for (int s = 0; s < 4; ++s) {
    double w = m->bw[4 * i + s];
    if (sgn) sgn[s] = 0;
    if (!(w > 0)) continue;
    dquat h = Hd[m->bidx[4 * i + s]];
    double sg = q_dot(h.r, Hd[jstar].r) >= 0 ? 1.0 : -1.0;
    if (sgn) sgn[s] = sg;
    acc = dq_axpy(acc, w * sg, h);
  }
  return acc;
}

static int validate_unit_dq(const float* p) {
  double n = 0, o = 0;
  for (int k = 0; k < 4; ++k) { n += (double)p[k] * p[k]; o += (double)p[k] * p[4 + k]; }
  return fabs(n - 1.0) < 1e-5 && fabs(o) < 1e-5;
}

/* R16: N(i) = the knn nearest other bind-pose vertices (squared distance in FP64 of the float
 * inputs; ties to the smaller index).  Exact search by a sweep over vertices sorted by x. */
static const double* g_sort_key;
static int cmp_by_key(const void* a, const void* b) {
  int ia = *(const int*)a, ib = *(const int*)b;
  double ka = g_sort_key[ia], kb = g_sort_key[ib];
  if (ka < kb) return -1;
  if (ka > kb) return 1;
  return ia < ib ? -1 : (ia > ib);
}
static void knn_build(orc_model* m) {
  int V = m->V, K = m->p.knn;
  int* order = (int*)xcalloc(V, sizeof(int));
  double* kx = (double*)xcalloc(V, sizeof(double));
  int* rank = (int*)xcalloc(V, sizeof(int));
  for (int i = 0; i < V; ++i) { order[i] = i; kx[i] = m->v0[3 * i]; }
  g_sort_key = kx;
  qsort(order, V, sizeof(int), cmp_by_key);
  for (int r = 0; r < V; ++r) rank[order[r]] = r;
  double bd[16];
  int bi[16];
  for (int i = 0; i < V; ++i) {
    int nb = 0;
    const double* pi = m->v0 + 3 * i;
    for (int dir = -1; dir <= 1; dir += 2) {
      for (int r = rank[i] + dir; r >= 0 && r < V; r += dir) {
        int j = order[r];
        double dx = m->v0[3 * j] - pi[0];
        if (nb == K && dx * dx > bd[K - 1]) break;
        double dy = m->v0[3 * j + 1] - pi[1], dz = m->v0[3 * j + 2] - pi[2];
        double d2 = dx * dx + dy * dy + dz * dz;
        /* insert (d2, j) into the sorted list of the K best, lexicographic order */
        if (nb == K && (d2 > bd[K - 1] || (d2 == bd[K - 1] && j > bi[K - 1]))) continue;
        int pos = nb < K ? nb : K - 1;
        while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > j))) {
          bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; --pos;
        }
        bd[pos] = d2; bi[pos] = j;
        if (nb < K) ++nb;
      }
    }
    for (int k = 0; k < K; ++k) m->nbr[K * i + k] = k < nb ? bi[k] : -1;
  }
  free(order); free(kx); free(rank);
}

void orc_destroy(void* h) {
  orc_model* m = (orc_model*)h;
  if (!m) return;
  free(m->parent); free(m->jtype); free(m->axis); free(m->off); free(m->prior_mask);
  free(m->v0); free(m->tri); free(m->bidx); free(m->bw); free(m->bind); free(m->S); free(m->nbr);
  free(m->theta); free(m->phi);
  free(m);
}

void* orc_create(int L, const int32_t* parent, const int32_t* type, const float* axis,
                 const float* offset_dq, const float* prior_mask, int V, const float* verts, int F,
                 const int32_t* tris, const uint8_t* bone_idx, const float* bone_w, int W, int H,
                 double fx, double fy, double cx, double cy, const orc_params* prm) {
  if (L <= 0 || V <= 0 || F < 0 || W <= 0 || H <= 0 || prm->knn < 0 || prm->knn > 16) return NULL;
  for (int j = 0; j < L; ++j) {
    if (parent[j] >= j || parent[j] < -1 || (type[j] != 0 && type[j] != 1)) return NULL;
    if (!validate_unit_dq(offset_dq + 8 * j)) return NULL;
  }
  for (int f = 0; f < 3 * F; ++f) if (tris[f] < 0 || tris[f] >= V) return NULL;
  for (int i = 0; i < V; ++i) {
    double sw = 0;
    for (int s = 0; s < 4; ++s) {
      if (bone_w[4 * i + s] < 0 || bone_idx[4 * i + s] >= L) return NULL;
      sw += bone_w[4 * i + s];
    }
    if (fabs(sw - 1.0) > 1e-4) return NULL;
  }
  orc_model* m = (orc_model*)xcalloc(1, sizeof(orc_model));
  m->L = L; m->V = V; m->F = F; m->W = W; m->H = H;
  m->fx = fx; m->fy = fy; m->cx = cx; m->cy = cy; m->p = *prm;
  m->parent = (int*)xcalloc(L, sizeof(int));
  m->jtype = (int*)xcalloc(L, sizeof(int));
  m->axis = (double*)xcalloc(3 * L, sizeof(double));
  m->off = (dquat*)xcalloc(L, sizeof(dquat));
  m->prior_mask = (double*)xcalloc(L, sizeof(double));
  m->bind = (dquat*)xcalloc(L, sizeof(dquat));
  m->S = (double*)xcalloc(L, sizeof(double));
  m->theta = (double*)xcalloc(L, sizeof(double));
  for (int j = 0; j < L; ++j) {
    m->parent[j] = parent[j]; m->jtype[j] = type[j]; m->prior_mask[j] = prior_mask[j];
    /* Sec. 3.1: z is a unit axis; the float input is normalised in FP64 */
    double an = sqrt((double)axis[3 * j] * axis[3 * j] + (double)axis[3 * j + 1] * axis[3 * j + 1] +
                     (double)axis[3 * j + 2] * axis[3 * j + 2]);
    if (!(an > 0.5 && an < 2.0)) { orc_destroy(m); return NULL; }
    for (int k = 0; k < 3; ++k) m->axis[3 * j + k] = axis[3 * j + k] / an;
    double t[8];
    for (int k = 0; k < 8; ++k) t[k] = offset_dq[8 * j + k];
    m->off[j] = dq_load(t);
  }
  m->v0 = (double*)xcalloc(3 * (size_t)V, sizeof(double));
  m->bidx = (int*)xcalloc(4 * (size_t)V, sizeof(int));
  m->bw = (double*)xcalloc(4 * (size_t)V, sizeof(double));
  m->phi = (double*)xcalloc(3 * (size_t)V, sizeof(double));
  m->nbr = (int*)xcalloc((size_t)(prm->knn ? prm->knn : 1) * V, sizeof(int));
  for (size_t i = 0; i < 3 * (size_t)V; ++i) m->v0[i] = verts[i];
  for (size_t i = 0; i < 4 * (size_t)V; ++i) { m->bidx[i] = bone_idx[i]; m->bw[i] = bone_w[i]; }
  m->tri = (int*)xcalloc(3 * (size_t)F, sizeof(int));
  for (size_t f = 0; f < 3 * (size_t)F; ++f) m->tri[f] = tris[f];
  /* Sec. 3.2: the bind pose is theta = 0 */
  double* zero = (double*)xcalloc(L, sizeof(double));
  dquat* H0 = (dquat*)xcalloc(L, sizeof(dquat));
  fk(m, zero, m->bind, NULL);
  free(zero); free(H0);
  /* R10: S_kk = n_k / |V|, n_k = vertices with nonzero weight on a link of subtree(k) */
  int* stamp = (int*)xcalloc(L, sizeof(int));
  double* cnt = (double*)xcalloc(L, sizeof(double));
  for (int j = 0; j < L; ++j) stamp[j] = -1;
  for (int i = 0; i < V; ++i)
    for (int s = 0; s < 4; ++s) {
      if (!(m->bw[4 * i + s] > 0)) continue;
      for (int k = m->bidx[4 * i + s]; k >= 0; k = m->parent[k]) {
        if (stamp[k] == i) continue;
        stamp[k] = i; cnt[k] += 1.0;
      }
    }
  for (int k = 0; k < L; ++k) m->S[k] = m->prior_mask[k] * cnt[k] / (double)V;
  free(stamp); free(cnt);
  if (prm->knn > 0) knn_build(m);
  m->lam = prm->lambda_k0;
  return m;
}

void orc_set_state(void* h, const double* theta, const double* phi, double lam) {
  orc_model* m = (orc_model*)h;
  memcpy(m->theta, theta, sizeof(double) * m->L);
  if (phi) memcpy(m->phi, phi, sizeof(double) * 3 * (size_t)m->V);
  else memset(m->phi, 0, sizeof(double) * 3 * (size_t)m->V);
  m->lam = lam;
}
void orc_get_state(void* h, double* theta, double* phi, double* lam) {
  orc_model* m = (orc_model*)h;
  memcpy(theta, m->theta, sizeof(double) * m->L);
  memcpy(phi, m->phi, sizeof(double) * 3 * (size_t)m->V);
  *lam = m->lam;
}
void orc_get_derived(void* h, double* bind, double* S, int32_t* nbr) {
  orc_model* m = (orc_model*)h;
  for (int j = 0; j < m->L; ++j) { dq_store(m->bind[j], bind + 8 * j); S[j] = m->S[j]; }
  for (size_t i = 0; i < (size_t)m->p.knn * m->V; ++i) nbr[i] = m->nbr[i];
}

/* exported FK: H0 and Hd as [L][8] */
void orc_fk(void* h, const double* theta, double* H0out, double* Hdout) {
  orc_model* m = (orc_model*)h;
  dquat* H0 = (dquat*)xcalloc(m->L, sizeof(dquat));
  dquat* Hd = (dquat*)xcalloc(m->L, sizeof(dquat));
  fk(m, theta, H0, Hd);
  for (int j = 0; j < m->L; ++j) { dq_store(H0[j], H0out + 8 * j); dq_store(Hd[j], Hdout + 8 * j); }
  free(H0); free(Hd);
}

/* Eq. deformation: v_i = H_{i,Sigma} (v0_i + phi_i).  Also returns the blended DQ per vertex. */
void orc_skin(void* h, const double* theta, const double* phi, double* v, double* Hs /*[V][8] or NULL*/) {
  orc_model* m = (orc_model*)h;
  dquat* Hd = (dquat*)xcalloc(m->L, sizeof(dquat));
  dquat* H0 = (dquat*)xcalloc(m->L, sizeof(dquat));
  fk(m, theta, H0, Hd);
  for (int i = 0; i < m->V; ++i) {
    dquat Hi = blend(m, Hd, i, NULL);
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = m->v0[3 * i + k] + (phi ? phi[3 * i + k] : 0.0);
    dq_point(Hi, x, v + 3 * i);
    if (Hs) dq_store(Hi, Hs + 8 * i);
  }
  free(Hd); free(H0);
}

/* R4: n_i = normalise(sum over incident faces of (v_b - v_a) x (v_c - v_a)); invalid if tiny. */
void orc_normals(int V, int F, const int32_t* tri, const double* v, double* n, int32_t* nvalid) {
  double* acc = (double*)xcalloc(3 * (size_t)V, sizeof(double));
  for (int f = 0; f < F; ++f) {
    const double* a = v + 3 * tri[3 * f];
    const double* b = v + 3 * tri[3 * f + 1];
    const double* c = v + 3 * tri[3 * f + 2];
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double fn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    for (int t = 0; t < 3; ++t)
      for (int k = 0; k < 3; ++k) acc[3 * tri[3 * f + t] + k] += fn[k];
  }
  for (int i = 0; i < V; ++i) {
    double* s = acc + 3 * i;
    double len = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (len < 1e-12) {
      nvalid[i] = 0; n[3 * i] = n[3 * i + 1] = n[3 * i + 2] = 0;
    } else {
      nvalid[i] = 1;
      for (int k = 0; k < 3; ++k) n[3 * i + k] = s[k] / len;
    }
  }
  free(acc);
}

/* Z-buffer rasterisation of the posed mesh into the camera (R5, R6).  z = +inf, tri = -1 where empty.
 * amb (optional): 1 where some triangle's edge passes within 1e-3 px of the pixel centre (a pixel whose
 * coverage is a rounding-level decision). */
void orc_raster(int W, int H, double fx, double fy, double cx, double cy, double znear, int V,
                const double* v, int F, const int32_t* tri, double* z, int32_t* ztri, int32_t* amb) {
  (void)V;
  for (int k = 0; k < W * H; ++k) { z[k] = INFINITY; ztri[k] = -1; if (amb) amb[k] = 0; }
  for (int f = 0; f < F; ++f) {
    const double* A = v + 3 * tri[3 * f];
    const double* B = v + 3 * tri[3 * f + 1];
    const double* C = v + 3 * tri[3 * f + 2];
    if (A[2] <= znear || B[2] <= znear || C[2] <= znear) continue;
    double ua = fx * A[0] / A[2] + cx, va = fy * A[1] / A[2] + cy;
    double ub = fx * B[0] / B[2] + cx, vb = fy * B[1] / B[2] + cy;
    double uc = fx * C[0] / C[2] + cx, vc = fy * C[1] / C[2] + cy;
    double area = (ub - ua) * (vc - va) - (vb - va) * (uc - ua);
    if (area == 0) continue;
    double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double NA = N[0] * A[0] + N[1] * A[1] + N[2] * A[2];
    double umin = fmin(ua, fmin(ub, uc)), umax = fmax(ua, fmax(ub, uc));
    double vmin = fmin(va, fmin(vb, vc)), vmax = fmax(va, fmax(vb, vc));
    int x0 = (int)fmax(0.0, ceil(umin - 1e-3)), x1 = (int)fmin((double)(W - 1), floor(umax + 1e-3));
    int y0 = (int)fmax(0.0, ceil(vmin - 1e-3)), y1 = (int)fmin((double)(H - 1), floor(vmax + 1e-3));
    double lab = hypot(ub - ua, vb - va), lbc = hypot(uc - ub, vc - vb), lca = hypot(ua - uc, va - vc);
    for (int py = y0; py <= y1; ++py)
      for (int px = x0; px <= x1; ++px) {
        double w0 = (uc - ub) * (py - vb) - (vc - vb) * (px - ub); /* edge b->c */
        double w1 = (ua - uc) * (py - vc) - (va - vc) * (px - uc); /* edge c->a */
        double w2 = (ub - ua) * (py - va) - (vb - va) * (px - ua); /* edge a->b */
        int k = py * W + px;
        if (amb) {
          double d0 = fabs(w0) / (lbc > 0 ? lbc : 1), d1 = fabs(w1) / (lca > 0 ? lca : 1);
          double d2 = fabs(w2) / (lab > 0 ? lab : 1);
          /* pixel within 1e-3 px of an edge line, and near the triangle itself */
          double tol = 1e-3;
          int near0 = d0 < tol && (w1 * area >= -tol * lca * fabs(area)) && (w2 * area >= -tol * lab * fabs(area));
          int near1 = d1 < tol && (w0 * area >= -tol * lbc * fabs(area)) && (w2 * area >= -tol * lab * fabs(area));
          int near2 = d2 < tol && (w0 * area >= -tol * lbc * fabs(area)) && (w1 * area >= -tol * lca * fabs(area));
          if (near0 || near1 || near2) amb[k] = 1;
        }
        int inside = (w0 >= 0 && w1 >= 0 && w2 >= 0) || (w0 <= 0 && w1 <= 0 && w2 <= 0);
        if (!inside) continue;
        double dx = (px - cx) / fx, dy = (py - cy) / fy;
        double den = N[0] * dx + N[1] * dy + N[2];
        if (den == 0) continue;
        double zt = NA / den;
        if (!(zt > 0)) continue;
        if (zt < z[k] || (zt == z[k] && f < ztri[k])) { z[k] = zt; ztri[k] = f; }
      }
  }
}

/* R7 visibility and the pixel bucket of each vertex (Sec. 4.1 "placing them into buckets").
 * marg (optional): 1 where one of the decisions is within rounding distance of its threshold. */
void orc_visibility(void* h, const double* v, const double* n, const int32_t* nvalid, const double* z,
                    const int32_t* zamb, int32_t* vis, int32_t* pix, int32_t* marg) {
  orc_model* m = (orc_model*)h;
  const double tol_m = 1e-5, tol_px = 1e-3;
  /* facing: n.p < 0 is decided on normals summed from face normals of the posed mesh; on a dense mesh
   * (edges ~1 mm long at coordinates ~1 m) an FP32 evaluation gets their direction to ~1e-5 rad, so a
   * vertex with |n.p| < 1e-4 |p| (its normal within 1e-4 rad of the view ray's normal plane) is marginal */
  const double tol_facing = 1e-4;
  for (int i = 0; i < m->V; ++i) {
    const double* p = v + 3 * i;
    vis[i] = 0; pix[i] = -1;
    if (marg) marg[i] = 0;
    if (!nvalid[i] || !(p[2] > m->p.z_near)) continue;
    double nd = n[3 * i] * p[0] + n[3 * i + 1] * p[1] + n[3 * i + 2] * p[2];
    double u = m->fx * p[0] / p[2] + m->cx, vv = m->fy * p[1] / p[2] + m->cy;
    double fu = floor(u + 0.5), fv = floor(vv + 0.5);
    if (marg) {
      double ru = u + 0.5 - fu, rv = vv + 0.5 - fv;
      const double pl = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
      if (fabs(nd) < tol_facing * pl || ru < tol_px || ru > 1 - tol_px || rv < tol_px || rv > 1 - tol_px) marg[i] = 1;
    }
    if (!(nd < 0)) continue;
    if (fu < 0 || fv < 0 || fu >= m->W || fv >= m->H) continue;
    int k = (int)fv * m->W + (int)fu;
    double Z = z[k];
    if (marg && ((isfinite(Z) && fabs(p[2] - (Z + m->p.eps_vis)) < tol_m) || (zamb && zamb[k]))) marg[i] = 1;
    if (isfinite(Z) && !(p[2] <= Z + m->p.eps_vis)) continue;
    vis[i] = 1; pix[i] = k;
  }
}

/* Sec. 4.1 projective association.  Each valid pixel back-projects to p_k; the closest visible vertex
 * whose bucket lies in the (2W+1)^2 window, within the cutoff, is its correspondence (R8, R9).
 * acc_i = sum over assigned pixels of (p_k - v_i), cnt_i = their number (the average gives p~_i).
 * tie (optional): 1 where the decision is within 1e-5 m of another outcome (the nearest two candidates, or
 * the nearest one and the cutoff), or involves a vertex whose visibility / bucket is marginal (marg from
 * orc_visibility) and that could be the nearest. */
void orc_associate(void* h, const double* v, const int32_t* vis, const int32_t* pix, const int32_t* marg,
                   const float* depth, int32_t* corr, double* acc, int32_t* cnt, int32_t* tie) {
  orc_model* m = (orc_model*)h;
  int W = m->W, H = m->H, V = m->V, R = m->p.window_half;
  double tau = m->p.cutoff, tau2 = tau * tau, tol = 1e-5;
  /* buckets: lists of visible vertices per pixel, in index order (counting sort) */
  int* start = (int*)xcalloc((size_t)W * H + 1, sizeof(int));
  int* list = (int*)xcalloc(V, sizeof(int));
  for (int i = 0; i < V; ++i) if (vis[i]) start[pix[i] + 1]++;
  for (int k = 0; k < W * H; ++k) start[k + 1] += start[k];
  int* fill = (int*)xcalloc((size_t)W * H, sizeof(int));
  for (int i = 0; i < V; ++i) if (vis[i]) { int k = pix[i]; list[start[k] + fill[k]++] = i; }
  /* marginal vertices (visible or not) in each pixel, for the tie flags */
  int* mstart = NULL; int* mlist = NULL;
  if (tie && marg) {
    mstart = (int*)xcalloc((size_t)W * H + 1, sizeof(int));
    int nm = 0;
    for (int i = 0; i < V; ++i) if (marg[i]) ++nm;
    mlist = (int*)xcalloc(nm, sizeof(int));
    int* mp = (int*)xcalloc(V, sizeof(int));
    for (int i = 0; i < V; ++i) {
      mp[i] = -1;
      if (!marg[i] || !(v[3 * i + 2] > m->p.z_near)) continue;
      double u = m->fx * v[3 * i] / v[3 * i + 2] + m->cx, vv = m->fy * v[3 * i + 1] / v[3 * i + 2] + m->cy;
      double fu = floor(u + 0.5), fv = floor(vv + 0.5);
      if (fu < 0 || fv < 0 || fu >= W || fv >= H) continue;
      mp[i] = (int)fv * W + (int)fu;
      mstart[mp[i] + 1]++;
    }
    for (int k = 0; k < W * H; ++k) mstart[k + 1] += mstart[k];
    memset(fill, 0, sizeof(int) * (size_t)W * H);
    for (int i = 0; i < V; ++i) if (mp[i] >= 0) mlist[mstart[mp[i]] + fill[mp[i]]++] = i;
    free(mp);
  }
  for (int i = 0; i < V; ++i) { acc[3 * i] = acc[3 * i + 1] = acc[3 * i + 2] = 0; cnt[i] = 0; }
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int k = py * W + px;
      corr[k] = -1;
      if (tie) tie[k] = 0;
      double d = depth[k];
      if (!(d > 0)) continue;
      double p[3] = {(px - m->cx) * d / m->fx, (py - m->cy) * d / m->fy, d};
      int best = -1;
      double bd2 = 0, d1 = INFINITY, d2nd = INFINITY; /* best / second-best distances (any range) */
      for (int qy = py - R; qy <= py + R; ++qy) {
        if (qy < 0 || qy >= H) continue;
        for (int qx = px - R; qx <= px + R; ++qx) {
          if (qx < 0 || qx >= W) continue;
          int q = qy * W + qx;
          for (int t = start[q]; t < start[q + 1]; ++t) {
            int i = list[t];
            double dx = p[0] - v[3 * i], dy = p[1] - v[3 * i + 1], dz = p[2] - v[3 * i + 2];
            double dd = dx * dx + dy * dy + dz * dz;
            double dist = sqrt(dd);
            if (dist < d1) { d2nd = d1; d1 = dist; } else if (dist < d2nd) { d2nd = dist; }
            if (dd <= tau2 && (best < 0 || dd < bd2 || (dd == bd2 && i < best))) { best = i; bd2 = dd; }
          }
        }
      }
      /* marginal vertices one pixel beyond the window too: their bucket may round either way */
      if (tie && mstart) {
        for (int qy = py - R - 1; qy <= py + R + 1; ++qy) {
          if (qy < 0 || qy >= H) continue;
          for (int qx = px - R - 1; qx <= px + R + 1; ++qx) {
            if (qx < 0 || qx >= W) continue;
            int q = qy * W + qx;
            for (int t = mstart[q]; t < mstart[q + 1]; ++t) {
              int i = mlist[t];
              double dx = p[0] - v[3 * i], dy = p[1] - v[3 * i + 1], dz = p[2] - v[3 * i + 2];
              double dist = sqrt(dx * dx + dy * dy + dz * dz);
              if (dist <= tau + tol && (best < 0 || dist <= sqrt(bd2) + tol)) tie[k] = 1;
            }
          }
        }
      }
      /* the outcome is a rounding-level one where the nearest two candidates are within tol of each other, or
       * the nearest one is within tol of the cutoff (a farther candidate's cutoff decision cannot change it) */
      if (tie && d2nd <= tau + tol && d2nd - d1 < tol) tie[k] = 1;
      if (tie && fabs(d1 - tau) < tol) tie[k] = 1;
      corr[k] = best;
      if (best >= 0) {
        acc[3 * best] += p[0] - v[3 * best];
        acc[3 * best + 1] += p[1] - v[3 * best + 1];
        acc[3 * best + 2] += p[2] - v[3 * best + 2];
        cnt[best] += 1;
      }
    }
  free(start); free(list); free(fill); free(mstart); free(mlist);
}

/* R23: the raster-ID association.  Each valid pixel back-projects to p_k and takes the nearest corner
 * (squared distance, ties to the smaller index) of the triangle the z-buffer holds at that pixel, within
 * the cutoff; a pixel the model does not cover gets none.  O(1) per pixel instead of the window search.
 * tie (optional): 1 where the z-buffer decision there is marginal (zamb from orc_raster), where two corners
 * are within 1e-5 m of each other, or where the best corner is within 1e-5 m of the cutoff. */
void orc_associate_rid(void* h, const double* v, const int32_t* ztri, const int32_t* zamb, const float* depth,
                       int32_t* corr, double* acc, int32_t* cnt, int32_t* tie) {
  orc_model* m = (orc_model*)h;
  const double tau = m->p.cutoff, tau2 = tau * tau, tol = 1e-5;
  for (int i = 0; i < m->V; ++i) { acc[3 * i] = acc[3 * i + 1] = acc[3 * i + 2] = 0; cnt[i] = 0; }
  for (int py = 0; py < m->H; ++py)
    for (int px = 0; px < m->W; ++px) {
      const int k = py * m->W + px;
      corr[k] = -1;
      if (tie) tie[k] = zamb ? zamb[k] : 0;
      const double d = depth[k];
      if (!(d > 0) || ztri[k] < 0) continue;
      const double p[3] = {(px - m->cx) * d / m->fx, (py - m->cy) * d / m->fy, d};
      const int* t = m->tri + 3 * (size_t)ztri[k];
      int best = -1;
      double bd2 = 0, dist[3];
      for (int c = 0; c < 3; ++c) {
        const int i = t[c];
        const double dx = p[0] - v[3 * i], dy = p[1] - v[3 * i + 1], dz = p[2] - v[3 * i + 2];
        const double dd = dx * dx + dy * dy + dz * dz;
        dist[c] = sqrt(dd);
        if (dd <= tau2 && (best < 0 || dd < bd2 || (dd == bd2 && i < best))) { best = i; bd2 = dd; }
      }
      if (tie) {
        for (int c = 0; c < 3; ++c) {
          if (fabs(dist[c] - tau) < tol) tie[k] = 1;
          for (int e = c + 1; e < 3; ++e)
            if (fabs(dist[c] - dist[e]) < tol && fmin(dist[c], dist[e]) <= tau + tol) tie[k] = 1;
        }
      }
      corr[k] = best;
      if (best >= 0) {
        for (int c = 0; c < 3; ++c) acc[3 * best + c] += p[c] - v[3 * best + c];
        cnt[best] += 1;
      }
    }
}

/* Given a correspondence map (from any source), the per-vertex sums of Sec. 4.1. */
void orc_accumulate(void* h, const double* v, const float* depth, const int32_t* corr, double* acc, int32_t* cnt) {
  orc_model* m = (orc_model*)h;
  for (int i = 0; i < m->V; ++i) { acc[3 * i] = acc[3 * i + 1] = acc[3 * i + 2] = 0; cnt[i] = 0; }
  for (int py = 0; py < m->H; ++py)
    for (int px = 0; px < m->W; ++px) {
      int k = py * m->W + px, i = corr[k];
      if (i < 0) continue;
      double d = depth[k];
      double p[3] = {(px - m->cx) * d / m->fx, (py - m->cy) * d / m->fy, d};
      for (int c = 0; c < 3; ++c) acc[3 * i + c] += p[c] - v[3 * i + c];
      cnt[i] += 1;
    }
}

/* Eq. residual r_i = n_i^T (p~_i - v_i) for i in A = {c_i >= 1, valid normal}; returns
 * E_pose = sum_A r_i^2 + sum_k (lambda_s S_kk theta_k)^2 (Sec. 4.2 pose prior). */
double orc_residuals(void* h, const double* theta, const double* n, const int32_t* nvalid, const double* acc,
                     const int32_t* cnt, double* r, int32_t* inA) {
  orc_model* m = (orc_model*)h;
  double E = 0;
  for (int i = 0; i < m->V; ++i) {
    r[i] = 0; inA[i] = 0;
    if (cnt[i] < 1 || !nvalid[i]) continue;
    inA[i] = 1;
    double ri = (n[3 * i] * acc[3 * i] + n[3 * i + 1] * acc[3 * i + 1] + n[3 * i + 2] * acc[3 * i + 2]) / cnt[i];
    r[i] = ri;
    E += ri * ri;
  }
  for (int k = 0; k < m->L; ++k) { double s = m->p.lambda_s * m->S[k] * theta[k]; E += s * s; }
  return E;
}

/* Sec. 4.2 block matrix dH_{j,Delta}/dtheta_k (R12):
 *   H_{0,P(k)} H_{P(k),k} (dH_k/dtheta_k) H_{k->j} (H^0_{0,j})^{-1}   for k an ancestor of j or j itself,
 * where H_{k->j} is the product of H_{P(m),m} H_m over the links m strictly below k down to j. */
static void delta_derivs(const orc_model* m, const double* theta, const dquat* H0, dquat* dHd /*[L][L]*/, char* isanc) {
  int L = m->L;
  for (int t = 0; t < L * L; ++t) { dHd[t] = dq_zero(); isanc[t] = 0; }
  for (int j = 0; j < L; ++j) {
    dquat suffix = dq_identity(); /* H_{k->j} for the current k */
    dquat tail = dq_conj(m->bind[j]);
    for (int k = j; k >= 0; k = m->parent[k]) {
      dquat pre = m->parent[k] < 0 ? dq_identity() : H0[m->parent[k]];
      dquat blk = dq_mul(dq_mul(dq_mul(pre, m->off[k]), joint_dq_deriv(m->jtype[k], m->axis + 3 * k, theta[k])),
                         dq_mul(suffix, tail));
      dHd[j * L + k] = blk;
      isanc[j * L + k] = 1;
      suffix = dq_mul(dq_mul(m->off[k], joint_dq(m->jtype[k], m->axis + 3 * k, theta[k])), suffix);
    }
  }
}

/* Sec. 4.2 pose Jacobian rows dr_i/dTheta = -n_i^T (dv_i/dH_iSigma)(dH_iSigma/dH_Delta)(dH_Delta/dTheta)
 * for i in A (zero rows elsewhere), the normal held constant.  J is [V][L]. */
void orc_jacobian(void* h, const double* theta, const double* phi, const double* n, const int32_t* inA, double* J) {
  orc_model* m = (orc_model*)h;
  int L = m->L;
  dquat* H0 = (dquat*)xcalloc(L, sizeof(dquat));
  dquat* Hd = (dquat*)xcalloc(L, sizeof(dquat));
  dquat* dHd = (dquat*)xcalloc((size_t)L * L, sizeof(dquat));
  char* isanc = (char*)xcalloc((size_t)L * L, 1);
  fk(m, theta, H0, Hd);
  delta_derivs(m, theta, H0, dHd, isanc);
  for (int i = 0; i < m->V; ++i) {
    double* row = J + (size_t)i * L;
    for (int k = 0; k < L; ++k) row[k] = 0;
    if (!inA[i]) continue;
    double sg[4];
    dquat Hi = blend(m, Hd, i, sg);
    double x[3];
    for (int c = 0; c < 3; ++c) x[c] = m->v0[3 * i + c] + (phi ? phi[3 * i + c] : 0.0);
    /* dv_i/dH_iSigma as a 3x8 matrix, one column per basis direction of the 8 DQ coefficients */
    double D[3][8];
    for (int e = 0; e < 8; ++e) {
      double basis[8] = {0, 0, 0, 0, 0, 0, 0, 0}, col[3];
      basis[e] = 1.0;
      dq_point_dir(Hi, x, dq_load(basis), col);
      for (int c = 0; c < 3; ++c) D[c][e] = col[c];
    }
    for (int k = 0; k < L; ++k) {
      /* dH_iSigma/dtheta_k = sum_j w_ij s_ij dH_{j,Delta}/dtheta_k (8x8 identity blocks scaled by w) */
      dquat dH = dq_zero();
      int any = 0;
      for (int s = 0; s < 4; ++s) {
        double w = m->bw[4 * i + s];
        int j = m->bidx[4 * i + s];
        if (!(w > 0) || !isanc[j * L + k]) continue;
        dH = dq_axpy(dH, w * sg[s], dHd[j * L + k]);
        any = 1;
      }
      if (!any) continue;
      double dd[8], dv[3] = {0, 0, 0};
      dq_store(dH, dd);
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 8; ++e) dv[c] += D[c][e] * dd[e];
      row[k] = -(n[3 * i] * dv[0] + n[3 * i + 1] * dv[1] + n[3 * i + 2] * dv[2]);
    }
  }
  free(H0); free(Hd); free(dHd); free(isanc);
}

/* Eqs. JTJ / JTr: sums over vertices of J_i^T J_i and J_i^T r_i (rows of A only). */
void orc_normal_eq(int V, int L, const double* J, const double* r, const int32_t* inA, double* JTJ, double* JTr) {
  for (int a = 0; a < L * L; ++a) JTJ[a] = 0;
  for (int a = 0; a < L; ++a) JTr[a] = 0;
  for (int i = 0; i < V; ++i) {
    if (!inA[i]) continue;
    const double* row = J + (size_t)i * L;
    for (int a = 0; a < L; ++a) {
      if (row[a] == 0) continue;
      JTr[a] += row[a] * r[i];
      for (int b = 0; b < L; ++b) JTJ[a * L + b] += row[a] * row[b];
    }
  }
}

/* Cholesky factorisation M = C C^T and the two triangular solves; returns -1 if not positive definite. */
int orc_cholesky_solve(int n, const double* M, const double* b, double* x) {
  double* C = (double*)xcalloc((size_t)n * n, sizeof(double));
  double* y = (double*)xcalloc(n, sizeof(double));
  int ok = 0;
  for (int j = 0; j < n && ok == 0; ++j) {
    double s = M[j * n + j];
    for (int k = 0; k < j; ++k) s -= C[j * n + k] * C[j * n + k];
    if (!(s > 0)) { ok = -1; break; }
    C[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (int k = 0; k < j; ++k) t -= C[i * n + k] * C[j * n + k];
      C[i * n + j] = t / C[j * n + j];
    }
  }
  if (ok == 0) {
    for (int i = 0; i < n; ++i) {
      double t = b[i];
      for (int k = 0; k < i; ++k) t -= C[i * n + k] * y[k];
      y[i] = t / C[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < n; ++k) t -= C[k * n + i] * x[k];
      x[i] = t / C[i * n + i];
    }
  }
  free(C); free(y);
  return ok;
}

/* Pose energy at candidate Theta with the association, normals and p~ held fixed (R14). */
static double pose_energy_fixed(orc_model* m, const double* theta, const double* phi, const double* n,
                                const double* ptilde, const int32_t* inA, double* vtmp) {
  orc_skin(m, theta, phi, vtmp, NULL);
  double E = 0;
  for (int i = 0; i < m->V; ++i) {
    if (!inA[i]) continue;
    double ri = 0;
    for (int c = 0; c < 3; ++c) ri += n[3 * i + c] * (ptilde[3 * i + c] - vtmp[3 * i + c]);
    E += ri * ri;
  }
  for (int k = 0; k < m->L; ++k) { double s = m->p.lambda_s * m->S[k] * theta[k]; E += s * s; }
  return E;
}

/* Sec. 4.2 damped least squares step with the pose prior and the R13/R14 readings.
 * Inputs: JTJ/JTr of the data term, the current energy E (prior included), the fixed association
 * (n, p~ = v + acc/cnt, A).  theta and lam are updated in place.  Returns the accepted attempt index
 * (0..5) or -1 when every attempt was rejected.  Ec (optional, [6]) receives each attempt's energy
 * (+inf for attempts not made or not positive definite). */
int orc_lm_step(void* h, const double* JTJ, const double* JTr, double E, const double* v, const double* n,
                const double* acc, const int32_t* cnt, const int32_t* inA, double* theta, double* lam, double* Ec) {
  orc_model* m = (orc_model*)h;
  int L = m->L, V = m->V;
  double* A = (double*)xcalloc((size_t)L * L, sizeof(double));
  double* M = (double*)xcalloc((size_t)L * L, sizeof(double));
  double* b = (double*)xcalloc(L, sizeof(double));
  double* x = (double*)xcalloc(L, sizeof(double));
  double* thc = (double*)xcalloc(L, sizeof(double));
  double* pt = (double*)xcalloc(3 * (size_t)V, sizeof(double));
  double* vtmp = (double*)xcalloc(3 * (size_t)V, sizeof(double));
  for (int i = 0; i < V; ++i)
    for (int c = 0; c < 3; ++c) pt[3 * i + c] = inA[i] ? v[3 * i + c] + acc[3 * i + c] / cnt[i] : 0.0;
  /* prior-augmented system: A = JTJ + (lambda_s S)^2, b = JTr + (lambda_s S)^2 Theta */
  for (int a = 0; a < L * L; ++a) A[a] = JTJ[a];
  for (int k = 0; k < L; ++k) {
    double s2 = (m->p.lambda_s * m->S[k]) * (m->p.lambda_s * m->S[k]);
    A[k * L + k] += s2;
    b[k] = JTr[k] + s2 * theta[k];
  }
  int accepted = -1;
  double lk = *lam;
  for (int t = 0; t < 6; ++t) if (Ec) Ec[t] = INFINITY;
  for (int t = 0; t < 6; ++t) {
    /* (A + lambda diag A) x = b; a parameter whose diagonal is zero is frozen (x_k = 0) */
    double* bb = (double*)xcalloc(L, sizeof(double));
    for (int a = 0; a < L; ++a)
      for (int c = 0; c < L; ++c) {
        int frozen = A[a * L + a] == 0 || A[c * L + c] == 0;
        M[a * L + c] = frozen ? (a == c ? 1.0 : 0.0) : A[a * L + c] + (a == c ? lk * A[a * L + a] : 0.0);
      }
    for (int a = 0; a < L; ++a) bb[a] = A[a * L + a] == 0 ? 0.0 : b[a];
    int ok = orc_cholesky_solve(L, M, bb, x);
    free(bb);
    double e = INFINITY;
    if (ok == 0) {
      for (int k = 0; k < L; ++k) thc[k] = theta[k] - x[k];
      e = pose_energy_fixed(m, thc, m->phi, n, pt, inA, vtmp);
    }
    if (Ec) Ec[t] = e;
    if (e <= E) {
      memcpy(theta, thc, sizeof(double) * L);
      lk = lk / 10.0;
      if (lk < 1e-7) lk = 1e-7;
      accepted = t;
      break;
    }
    lk = lk * 10.0;
    if (lk > 1e7) lk = 1e7;
  }
  *lam = lk;
  free(A); free(M); free(b); free(x); free(thc); free(pt); free(vtmp);
  return accepted;
}

/* 3x3 solve by Cramer's rule (used by the shape step). */
static int solve3(const double* M, const double* b, double* x) {
  double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) + M[2] * (M[3] * M[7] - M[4] * M[6]);
  if (det == 0) return -1;
  for (int c = 0; c < 3; ++c) {
    double T[9];
    memcpy(T, M, sizeof(T));
    for (int r = 0; r < 3; ++r) T[3 * r + c] = b[r];
    x[c] = (T[0] * (T[4] * T[8] - T[5] * T[7]) - T[1] * (T[3] * T[8] - T[5] * T[6]) + T[2] * (T[3] * T[7] - T[4] * T[6])) / det;
  }
  return 0;
}
int orc_solve3(const double* M, const double* b, double* x) { return solve3(M, b, x); }

/* R22: the coupled Gauss-Newton step of the whole shape energy of Sec. 4.3,
 *   E(Phi) = sum_{i in A} r_i^2 + lambda_phi sum_i |phi_i|^2 + lambda_N sum_i sum_{n in N(i)} |phi_i - phi_n|^2,
 * with r_i linearised as r_i + g_i . delta_i:  (H + lambda_w D) delta = -b, where
 *   H_ii = [i in A] g_i g_i^T + (lambda_phi + lambda_N deg_i) I,  H_ij = -lambda_N m_ij I,
 *   b_i  = [i in A] g_i r_i + lambda_phi phi_i + lambda_N sum_{j in adj(i)} (phi_i - phi_j),
 * adj(i) = the neighbourhood edges at i in either direction (the multiset of n in N(i) and of m with
 * i in N(m)), deg_i = |adj(i)|, m_ij the multiplicity of j in adj(i), D = diag(H).  Solved by conjugate
 * gradients from delta = 0, preconditioned with the 3x3 diagonal blocks of H + lambda_w D, for `iters`
 * iterations (or until r.z = 0 or p.Ap <= 0).  phi += delta. */
static int cmp_int(const void* a, const void* b) {
  const int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

static void shape_pcg(orc_model* m, double* phi, const double* r0, const double* g, const int32_t* inA, int iters) {
  const int V = m->V, K = m->p.knn;
  const double lp = m->p.lambda_phi, lN = m->p.lambda_N, lw = m->p.lambda_w;
  /* adjacency in both directions, each list sorted by vertex index */
  int* deg = (int*)xcalloc(V + 1, sizeof(int));
  for (int i = 0; i < V; ++i)
    for (int t = 0; t < K; ++t) {
      const int q = m->nbr[K * i + t];
      if (q < 0) continue;
      ++deg[i];
      ++deg[q];
    }
  int* off = (int*)xcalloc(V + 1, sizeof(int));
  for (int i = 0; i < V; ++i) off[i + 1] = off[i] + deg[i];
  int* adj = (int*)xcalloc(off[V] > 0 ? off[V] : 1, sizeof(int));
  int* fill = (int*)xcalloc(V, sizeof(int));
  for (int i = 0; i < V; ++i)
    for (int t = 0; t < K; ++t) {
      const int q = m->nbr[K * i + t];
      if (q < 0) continue;
      adj[off[i] + fill[i]++] = q;
      adj[off[q] + fill[q]++] = i;
    }
  for (int i = 0; i < V; ++i) qsort(adj + off[i], deg[i], sizeof(int), cmp_int);
  /* per-vertex damped diagonal blocks B_i = H_ii + lambda_w diag(H_ii) */
  double* Bk = (double*)xcalloc(9 * (size_t)V, sizeof(double));
  for (int i = 0; i < V; ++i) {
    const double* gi = g + 3 * i;
    const double c = lp + lN * deg[i];
    for (int a = 0; a < 3; ++a)
      for (int e = 0; e < 3; ++e) Bk[9 * i + 3 * a + e] = (inA[i] ? gi[a] * gi[e] : 0.0) + (a == e ? c : 0.0);
    for (int a = 0; a < 3; ++a) Bk[9 * i + 4 * a] += lw * Bk[9 * i + 4 * a];
  }
  const size_t n3 = 3 * (size_t)V;
  double* x = (double*)xcalloc(n3, sizeof(double));
  double* r = (double*)xcalloc(n3, sizeof(double));
  double* z = (double*)xcalloc(n3, sizeof(double));
  double* pv = (double*)xcalloc(n3, sizeof(double));
  double* Ap = (double*)xcalloc(n3, sizeof(double));
  /* r = -b */
  for (int i = 0; i < V; ++i) {
    const double* gi = g + 3 * i;
    const double* pi = phi + 3 * i;
    for (int c = 0; c < 3; ++c) {
      double bc = (inA[i] ? gi[c] * r0[i] : 0.0) + lp * pi[c];
      for (int t = off[i]; t < off[i + 1]; ++t) bc += lN * (pi[c] - phi[3 * adj[t] + c]);
      r[3 * i + c] = -bc;
    }
  }
  double rz = 0.0;
  for (int i = 0; i < V; ++i) {
    if (solve3(Bk + 9 * i, r + 3 * i, z + 3 * i) != 0) z[3 * i] = z[3 * i + 1] = z[3 * i + 2] = 0.0;
    for (int c = 0; c < 3; ++c) rz += r[3 * i + c] * z[3 * i + c];
  }
  memcpy(pv, z, n3 * sizeof(double));
  for (int it = 0; it < iters && rz > 0.0; ++it) {
    double pAp = 0.0;
    for (int i = 0; i < V; ++i) {
      const double* Bi = Bk + 9 * i;
      const double* p = pv + 3 * i;
      for (int a = 0; a < 3; ++a) {
        double s = Bi[3 * a] * p[0] + Bi[3 * a + 1] * p[1] + Bi[3 * a + 2] * p[2];
        for (int t = off[i]; t < off[i + 1]; ++t) s -= lN * pv[3 * adj[t] + a];
        Ap[3 * i + a] = s;
        pAp += p[a] * s;
      }
    }
    if (!(pAp > 0.0)) break;
    const double alpha = rz / pAp;
    double rz_new = 0.0;
    for (int i = 0; i < V; ++i) {
      for (int c = 0; c < 3; ++c) {
        x[3 * i + c] += alpha * pv[3 * i + c];
        r[3 * i + c] -= alpha * Ap[3 * i + c];
      }
      if (solve3(Bk + 9 * i, r + 3 * i, z + 3 * i) != 0) z[3 * i] = z[3 * i + 1] = z[3 * i + 2] = 0.0;
      for (int c = 0; c < 3; ++c) rz_new += r[3 * i + c] * z[3 * i + c];
    }
    const double beta = rz_new / rz;
    rz = rz_new;
    for (size_t k = 0; k < n3; ++k) pv[k] = z[k] + beta * pv[k];
  }
  for (size_t k = 0; k < n3; ++k) phi[k] += x[k];
  free(deg); free(off); free(adj); free(fill); free(Bk); free(x); free(r); free(z); free(pv); free(Ap);
}

/* Sec. 4.3 shape step (R15): per-vertex Gauss-Newton on
 *   e_i = [i in A] r_i^2 + lambda_phi |phi_i|^2 + lambda_N sum_{n in N(i)} |phi_i - phi_n|^2
 * with the neighbours frozen, one 3x3 damped system per vertex (Jacobi), shape_sweeps sweeps;
 * with shape_solver = 1 the coupled system of R22 instead, shape_sweeps PCG iterations.
 * g_i = dr_i/dphi_i = -R(a^_i)^T n_i (a^_i the normalised real part of H_iSigma).
 * Returns the shape energy sum_i e_i before the update.  phi is updated in place.
 * r_out, g_out (optional): r_i and g_i. */
double orc_shape_step(void* h, const double* theta, double* phi, const double* n, const double* acc,
                      const int32_t* cnt, const int32_t* inA, double* r_out, double* g_out) {
  orc_model* m = (orc_model*)h;
  int V = m->V, K = m->p.knn, L = m->L;
  double lp = m->p.lambda_phi, lN = m->p.lambda_N, lw = m->p.lambda_w;
  dquat* H0 = (dquat*)xcalloc(L, sizeof(dquat));
  dquat* Hd = (dquat*)xcalloc(L, sizeof(dquat));
  double* r0 = (double*)xcalloc(V, sizeof(double));
  double* g = (double*)xcalloc(3 * (size_t)V, sizeof(double));
  double* phi0 = (double*)xcalloc(3 * (size_t)V, sizeof(double));
  double* cur = (double*)xcalloc(3 * (size_t)V, sizeof(double));
  fk(m, theta, H0, Hd);
  memcpy(phi0, phi, sizeof(double) * 3 * V);
  double E = 0;
  for (int i = 0; i < V; ++i) {
    if (inA[i]) {
      r0[i] = (n[3 * i] * acc[3 * i] + n[3 * i + 1] * acc[3 * i + 1] + n[3 * i + 2] * acc[3 * i + 2]) / cnt[i];
      dquat Hi = blend(m, Hd, i, NULL);
      double an = sqrt(q_dot(Hi.r, Hi.r)), R[9];
      q_to_rot(q_scale(Hi.r, 1.0 / an), R);
      for (int c = 0; c < 3; ++c)
        g[3 * i + c] = -(R[0 * 3 + c] * n[3 * i] + R[1 * 3 + c] * n[3 * i + 1] + R[2 * 3 + c] * n[3 * i + 2]);
      E += r0[i] * r0[i];
    }
    const double* pi = phi + 3 * i;
    E += lp * (pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2]);
    for (int t = 0; t < K; ++t) {
      int q = m->nbr[K * i + t];
      if (q < 0) continue;
      for (int c = 0; c < 3; ++c) { double d = pi[c] - phi[3 * q + c]; E += lN * d * d; }
    }
  }
  if (m->p.shape_solver == 1) shape_pcg(m, phi, r0, g, inA, m->p.shape_sweeps);
  for (int sw = 0; sw < (m->p.shape_solver == 1 ? 0 : m->p.shape_sweeps); ++sw) {
    memcpy(cur, phi, sizeof(double) * 3 * V);
    for (int i = 0; i < V; ++i) {
      const double* pi = cur + 3 * i;
      const double* gi = g + 3 * i;
      double ri = 0;
      if (inA[i]) ri = r0[i] + gi[0] * (pi[0] - phi0[3 * i]) + gi[1] * (pi[1] - phi0[3 * i + 1]) + gi[2] * (pi[2] - phi0[3 * i + 2]);
      int nn = 0;
      double grad[3], Mx[9], Md[9], dlt[3];
      for (int c = 0; c < 3; ++c) grad[c] = gi[c] * ri + lp * pi[c];
      for (int t = 0; t < K; ++t) {
        int q = m->nbr[K * i + t];
        if (q < 0) continue;
        ++nn;
        for (int c = 0; c < 3; ++c) grad[c] += lN * (pi[c] - cur[3 * q + c]);
      }
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) Mx[3 * a + c] = gi[a] * gi[c] + (a == c ? lp + lN * nn : 0.0);
      memcpy(Md, Mx, sizeof(Md));
      for (int a = 0; a < 3; ++a) Md[4 * a] += lw * Mx[4 * a];
      double rhs[3] = {-grad[0], -grad[1], -grad[2]};
      if (solve3(Md, rhs, dlt) != 0) dlt[0] = dlt[1] = dlt[2] = 0;
      for (int c = 0; c < 3; ++c) phi[3 * i + c] = pi[c] + dlt[c];
    }
  }
  if (r_out) memcpy(r_out, r0, sizeof(double) * V);
  if (g_out) memcpy(g_out, g, sizeof(double) * 3 * V);
  free(H0); free(Hd); free(r0); free(g); free(phi0); free(cur);
  return E;
}

/* Render the model's depth (skin + z-buffer) at (theta, phi); 0 where the buffer is empty. */
void orc_render(void* h, const double* theta, const double* phi, double* depth) {
  orc_model* m = (orc_model*)h;
  double* v = (double*)xcalloc(3 * (size_t)m->V, sizeof(double));
  int32_t* zt = (int32_t*)xcalloc((size_t)m->W * m->H, sizeof(int32_t));
  orc_skin(m, theta, phi, v, NULL);
  orc_raster(m->W, m->H, m->fx, m->fy, m->cx, m->cy, m->p.z_near, m->V, v, m->F, m->tri, depth, zt, NULL);
  for (int k = 0; k < m->W * m->H; ++k) if (!isfinite(depth[k])) depth[k] = 0;
  free(v); free(zt);
}

/* One association pass at the current state: skin, normals, z-buffer, visibility, association. */
typedef struct {
  double *v, *n, *z, *acc, *r;
  int32_t *nvalid, *ztri, *vis, *pix, *corr, *cnt, *inA;
} orc_ws;

static void ws_alloc(orc_model* m, orc_ws* w) {
  size_t V = m->V, P = (size_t)m->W * m->H;
  w->v = (double*)xcalloc(3 * V, sizeof(double)); w->n = (double*)xcalloc(3 * V, sizeof(double));
  w->z = (double*)xcalloc(P, sizeof(double)); w->acc = (double*)xcalloc(3 * V, sizeof(double));
  w->r = (double*)xcalloc(V, sizeof(double));
  w->nvalid = (int32_t*)xcalloc(V, 4); w->ztri = (int32_t*)xcalloc(P, 4); w->vis = (int32_t*)xcalloc(V, 4);
  w->pix = (int32_t*)xcalloc(V, 4); w->corr = (int32_t*)xcalloc(P, 4); w->cnt = (int32_t*)xcalloc(V, 4);
  w->inA = (int32_t*)xcalloc(V, 4);
}
static void ws_free(orc_ws* w) {
  free(w->v); free(w->n); free(w->z); free(w->acc); free(w->r); free(w->nvalid); free(w->ztri);
  free(w->vis); free(w->pix); free(w->corr); free(w->cnt); free(w->inA);
}
static double associate_pass(orc_model* m, orc_ws* w, const float* depth) {
  orc_skin(m, m->theta, m->phi, w->v, NULL);
  orc_normals(m->V, m->F, m->tri, w->v, w->n, w->nvalid);
  orc_raster(m->W, m->H, m->fx, m->fy, m->cx, m->cy, m->p.z_near, m->V, w->v, m->F, m->tri, w->z, w->ztri, NULL);
  orc_visibility(m, w->v, w->n, w->nvalid, w->z, NULL, w->vis, w->pix, NULL);
  if (m->p.association == 1)
    orc_associate_rid(m, w->v, w->ztri, NULL, depth, w->corr, w->acc, w->cnt, NULL);
  else
    orc_associate(m, w->v, w->vis, w->pix, NULL, depth, w->corr, w->acc, w->cnt, NULL);
  return orc_residuals(m, m->theta, w->n, w->nvalid, w->acc, w->cnt, w->r, w->inA);
}

/* One frame (Sec. 4, schedule R18): pose_iters LM iterations, then shape_iters shape iterations, each
 * re-associating at the current state.  energy[pose_iters + shape_iters] receives E_pose of each pose
 * iteration and E_shape of each shape iteration; accepted[pose_iters] (optional) the LM attempt taken.
 * Returns the number of associated pixels of the last association. */
int orc_track_frame(void* h, const float* depth, double* energy, int32_t* accepted) {
  orc_model* m = (orc_model*)h;
  int L = m->L, V = m->V;
  orc_ws w;
  ws_alloc(m, &w);
  double* J = (double*)xcalloc((size_t)V * L, sizeof(double));
  double* JTJ = (double*)xcalloc((size_t)L * L, sizeof(double));
  double* JTr = (double*)xcalloc(L, sizeof(double));
  int nassoc = 0;
  for (int it = 0; it < m->p.pose_iters; ++it) {
    double E = associate_pass(m, &w, depth);
    energy[it] = E;
    orc_jacobian(m, m->theta, m->phi, w.n, w.inA, J);
    orc_normal_eq(V, L, J, w.r, w.inA, JTJ, JTr);
    int a = orc_lm_step(m, JTJ, JTr, E, w.v, w.n, w.acc, w.cnt, w.inA, m->theta, &m->lam, NULL);
    if (accepted) accepted[it] = a;
  }
  for (int s = 0; s < m->p.shape_iters; ++s) {
    associate_pass(m, &w, depth);
    energy[m->p.pose_iters + s] = orc_shape_step(m, m->theta, m->phi, w.n, w.acc, w.cnt, w.inA, NULL, NULL);
  }
  if (m->p.pose_iters + m->p.shape_iters > 0)
    for (int k = 0; k < m->W * m->H; ++k) nassoc += w.corr[k] >= 0;
  ws_free(&w);
  free(J); free(JTJ); free(JTr);
  return nassoc;
}

/* ------------------------------------------------------------------------------------------------ */
/* Template authoring (the paper's template construction): Catmull-Clark subdivision of a polygon   */
/* cage, the skin weights interpolated with the same stencils as the positions.                      */
/* ------------------------------------------------------------------------------------------------ */
/* Conventions (shared with the library's description, not its code): the new vertices of a level are
 * the vertex points of the old vertices (same indices), then the edge points in the order in which the
 * edges first appear when the faces are walked in order (face f, edges (v_i, v_{i+1})), then the face
 * points in face order.  Face f = (v_0 .. v_{k-1}) becomes the quads (v_i', e(v_i, v_{i+1}), f', e(v_{i-1}, v_i)),
 * i = 0 .. k-1.  Rules: face point = mean of the face's vertices; interior edge point = mean of its two
 * end points and the two adjacent face points, boundary edge point = the midpoint; interior vertex point =
 * (F + 2 R + (n - 3) P) / n with F the mean of the n adjacent face points, R the mean of the midpoints
 * of the n incident edges; boundary vertex point = (6 P + the two boundary neighbours) / 8. */
typedef struct { int a, b, fa, fb; } cc_edge;

static int cc_find_edge(int* head, int* next, const cc_edge* E, int a, int b) {
  int lo = a < b ? a : b, hi = a < b ? b : a;
  for (int e = head[lo]; e >= 0; e = next[e]) {
    int ea = E[e].a < E[e].b ? E[e].a : E[e].b, eb = E[e].a < E[e].b ? E[e].b : E[e].a;
    if (ea == lo && eb == hi) return e;
  }
  return -1;
}

/* One level. face_off/face_vert: the polygons (CSR). attr: [V][A] (positions and other attributes).
 * Outputs: out_attr [V + E + F][A], out_quads [sum_k][4]; returns the new vertex count (E via *nE). */
static int cc_level(int V, int F, const int* face_off, const int* face_vert, int A, const double* attr,
                    double* out_attr, int* out_quads, int* nE) {
  int nf_v = face_off[F];
  cc_edge* E = (cc_edge*)xcalloc(nf_v, sizeof(cc_edge));
  int* head = (int*)xcalloc(V, sizeof(int));
  int* next = (int*)xcalloc(nf_v, sizeof(int));
  int* fedge = (int*)xcalloc(nf_v, sizeof(int)); /* edge of (v_i, v_{i+1}) of each face corner */
  for (int i = 0; i < V; ++i) head[i] = -1;
  int ne = 0;
  for (int f = 0; f < F; ++f) {
    int k = face_off[f + 1] - face_off[f];
    for (int i = 0; i < k; ++i) {
      int a = face_vert[face_off[f] + i], b = face_vert[face_off[f] + (i + 1) % k];
      int e = cc_find_edge(head, next, E, a, b);
      if (e < 0) {
        e = ne++;
        E[e].a = a; E[e].b = b; E[e].fa = f; E[e].fb = -1;
        int lo = a < b ? a : b;
        next[e] = head[lo];
        head[lo] = e;
      } else {
        E[e].fb = f;
      }
      fedge[face_off[f] + i] = e;
    }
  }
  double* FP = out_attr + (size_t)(V + ne) * A;  /* face points */
  for (int f = 0; f < F; ++f) {
    int k = face_off[f + 1] - face_off[f];
    for (int c = 0; c < A; ++c) {
      double s = 0;
      for (int i = 0; i < k; ++i) s += attr[(size_t)face_vert[face_off[f] + i] * A + c];
      FP[(size_t)f * A + c] = s / k;
    }
  }
  double* EP = out_attr + (size_t)V * A;  /* edge points */
  for (int e = 0; e < ne; ++e)
    for (int c = 0; c < A; ++c) {
      double pa = attr[(size_t)E[e].a * A + c], pb = attr[(size_t)E[e].b * A + c];
      EP[(size_t)e * A + c] = E[e].fb < 0 ? 0.5 * (pa + pb)
                                          : 0.25 * (pa + pb + FP[(size_t)E[e].fa * A + c] + FP[(size_t)E[e].fb * A + c]);
    }
  /* vertex points: accumulate the incident faces and edges */
  double* Fs = (double*)xcalloc((size_t)V * A, sizeof(double));
  double* Rs = (double*)xcalloc((size_t)V * A, sizeof(double));
  double* Bs = (double*)xcalloc((size_t)V * A, sizeof(double));
  int* nF = (int*)xcalloc(V, sizeof(int));
  int* nR = (int*)xcalloc(V, sizeof(int));
  int* nB = (int*)xcalloc(V, sizeof(int));
  for (int f = 0; f < F; ++f)
    for (int i = face_off[f]; i < face_off[f + 1]; ++i) {
      int v = face_vert[i];
      for (int c = 0; c < A; ++c) Fs[(size_t)v * A + c] += FP[(size_t)f * A + c];
      nF[v]++;
    }
  for (int e = 0; e < ne; ++e) {
    int ends[2] = {E[e].a, E[e].b};
    for (int s = 0; s < 2; ++s) {
      int v = ends[s], o = ends[1 - s];
      for (int c = 0; c < A; ++c) Rs[(size_t)v * A + c] += 0.5 * (attr[(size_t)v * A + c] + attr[(size_t)o * A + c]);
      nR[v]++;
      if (E[e].fb < 0) {
        for (int c = 0; c < A; ++c) Bs[(size_t)v * A + c] += attr[(size_t)o * A + c];
        nB[v]++;
      }
    }
  }
  for (int v = 0; v < V; ++v)
    for (int c = 0; c < A; ++c) {
      double P = attr[(size_t)v * A + c];
      double* o = out_attr + (size_t)v * A + c;
      if (nB[v] > 0) {
        *o = nB[v] == 2 ? (6.0 * P + Bs[(size_t)v * A + c]) / 8.0 : P;
      } else if (nF[v] > 0) {
        double n = nF[v];
        *o = (Fs[(size_t)v * A + c] / n + 2.0 * Rs[(size_t)v * A + c] / nR[v] + (n - 3.0) * P) / n;
      } else {
        *o = P;
      }
    }
  int q = 0;
  for (int f = 0; f < F; ++f) {
    int k = face_off[f + 1] - face_off[f];
    for (int i = 0; i < k; ++i) {
      out_quads[4 * q] = face_vert[face_off[f] + i];
      out_quads[4 * q + 1] = V + fedge[face_off[f] + i];
      out_quads[4 * q + 2] = V + ne + f;
      out_quads[4 * q + 3] = V + fedge[face_off[f] + (i + k - 1) % k];
      ++q;
    }
  }
  *nE = ne;
  free(E); free(head); free(next); free(fedge); free(Fs); free(Rs); free(Bs); free(nF); free(nR); free(nB);
  return V + ne + F;
}

/* Counts after `levels` levels: vertices and quads (each level's faces are quads after the first). */
void orc_subdivide_counts(int V, int F, const int32_t* face_off, const int32_t* face_vert, int levels, int32_t* Vout,
                          int32_t* Qout) {
  /* the edge count needs the topology: run the levels on a zero-width attribute */
  int* fo = (int*)xcalloc(F + 1, sizeof(int));
  int* fv = (int*)xcalloc(face_off[F] > 0 ? face_off[F] : 1, sizeof(int));
  for (int f = 0; f <= F; ++f) fo[f] = face_off[f];
  for (int i = 0; i < face_off[F]; ++i) fv[i] = face_vert[i];
  int curV = V, curF = F;
  for (int l = 0; l < levels; ++l) {
    int nq = fo[curF], ne = 0;
    int* quads = (int*)xcalloc(4 * (size_t)nq, sizeof(int));
    double dummy[1];
    double* outa = (double*)xcalloc(1, sizeof(double));
    int newV = cc_level(curV, curF, fo, fv, 0, dummy, outa, quads, &ne);
    free(outa);
    free(fo); free(fv);
    fo = (int*)xcalloc(nq + 1, sizeof(int));
    for (int i = 0; i <= nq; ++i) fo[i] = 4 * i;
    fv = quads;
    curV = newV; curF = nq;
  }
  *Vout = curV;
  *Qout = curF;
  free(fo); free(fv);
}

/* `levels` levels of Catmull-Clark on attributes attr [V][A] (positions first); out_attr [Vout][A],
 * out_quads [Qout][4] (sizes from orc_subdivide_counts). */
void orc_subdivide(int V, int F, const int32_t* face_off, const int32_t* face_vert, int A, const double* attr,
                   int levels, double* out_attr, int32_t* out_quads) {
  int* fo = (int*)xcalloc(F + 1, sizeof(int));
  int* fv = (int*)xcalloc(face_off[F] > 0 ? face_off[F] : 1, sizeof(int));
  for (int f = 0; f <= F; ++f) fo[f] = face_off[f];
  for (int i = 0; i < face_off[F]; ++i) fv[i] = face_vert[i];
  double* cur = (double*)xcalloc((size_t)V * A + 1, sizeof(double));
  memcpy(cur, attr, sizeof(double) * (size_t)V * A);
  int curV = V, curF = F;
  for (int l = 0; l < levels; ++l) {
    int nq = fo[curF], ne = 0;
    int* quads = (int*)xcalloc(4 * (size_t)nq, sizeof(int));
    /* upper bound of the new vertex count: V + (corners) + F */
    double* nxt = (double*)xcalloc((size_t)(curV + fo[curF] + curF) * A + 1, sizeof(double));
    int newV = cc_level(curV, curF, fo, fv, A, cur, nxt, quads, &ne);
    free(cur); free(fo); free(fv);
    cur = nxt;
    fo = (int*)xcalloc(nq + 1, sizeof(int));
    for (int i = 0; i <= nq; ++i) fo[i] = 4 * i;
    fv = quads;
    curV = newV; curF = nq;
  }
  memcpy(out_attr, cur, sizeof(double) * (size_t)curV * A);
  for (int i = 0; i < 4 * curF; ++i) out_quads[i] = fv[i];
  free(cur); free(fo); free(fv);
}

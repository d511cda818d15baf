/*
 * trk.h -- C ABI of the GB300 tracker for "Dynamic High Resolution Deformable Articulated Tracking"
 * (Walsman, Wan, Schmidt, Fox; 3DV 2017).
 *
 * One session tracks one subject: a kinematic tree of 1-DoF links (Sec. 3.1), a triangle mesh attached
 * by dual-quaternion skinning (Sec. 3.2) with per-vertex warp offsets Phi (Sec. 3.3), and a pinhole
 * depth camera.  Each frame runs pose_iters Levenberg-Marquardt iterations on the joint values Theta
 * (Sec. 4.2) and shape_iters per-vertex shape iterations on Phi (Sec. 4.3); every iteration re-skins,
 * z-buffers and re-associates the depth pixels (Sec. 4.1).  Every step runs in CUDA kernels on the
 * current device; there is no CPU fallback.
 *
 * Conventions
 *  - Plain pointers and sizes only.  "host" pointers are CPU memory, "device" pointers CUDA memory of
 *    the device that was current when the session was created.
 *  - Inputs are copied at the call; the caller keeps ownership of every buffer it passes.
 *  - The session owns all of its device memory and frees it in trk_destroy.
 *  - Every call returns a trk_status; on failure trk_last_error() returns a message (thread-local).
 *  - Units are metres and radians; the camera looks down +z, x right, y down (world = camera).
 *  - A session is not thread-safe: calls on one session must not overlap.
 */
#ifndef TRK_H_
#define TRK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TRK_OK = 0,
  TRK_ERR_INVALID_ARG = 1, /* malformed model, sizes or pointers; nothing was changed           */
  TRK_ERR_OOM = 2,         /* device or host allocation failed                                     */
  TRK_ERR_CUDA = 3,        /* a CUDA runtime call failed (message holds cudaGetErrorString)        */
  TRK_ERR_NO_CAPACITY = 4, /* a fixed limit was exceeded (links, server budget)                    */
  TRK_ERR_TIMEOUT = 5,     /* a bounded wait ran out                                               */
  TRK_ERR_NUMERIC = 6      /* non-finite input or a non-positive-definite system                   */
} trk_status;

typedef struct trk_session trk_session;

/* Template mesh in the bind pose Theta = 0 (Sec. 3.2).  bone_idx/bone_w: the <= 4 nonzero entries of
 * the weight column omega_i (Sec. 3.2); unused slots have weight 0; weights are >= 0 and sum to 1. */
typedef struct {
  int32_t n_verts, n_tris;
  const float* verts;      /* host [n_verts][3]                                        */
  const int32_t* tris;     /* host [n_tris][3], vertex indices, counter-clockwise seen from outside */
  const uint8_t* bone_idx; /* host [n_verts][4], link indices                          */
  const float* bone_w;     /* host [n_verts][4]                                        */
} trk_mesh;

/* Kinematic tree (Sec. 3.1): link j hangs from parent[j] < j (-1 = world) through the fixed unit
 * dual quaternion offset H_{P(j),j} followed by its 1-DoF joint: a hinge (Eq. H_hinge) or a prismatic
 * joint (Eq. H_prismatic) about / along axis z_j.  Multi-DoF joints are chains of links with identity
 * offsets.  One link carries one joint value, so |Theta| = n_links (<= TRK_MAX_LINKS). */
typedef struct {
  int32_t n_links;
  const int32_t* parent;    /* host [n_links]                                                 */
  const int32_t* type;      /* host [n_links]: 0 hinge, 1 prismatic                           */
  const float* axis;        /* host [n_links][3], normalised at create                        */
  const float* offset_dq;   /* host [n_links][8]: (w,x,y,z | w,x,y,z), |real| = 1, <real,dual> = 0 */
  const float* prior_mask;  /* host [n_links]: multiplies the pose-prior weight S_kk (0 = no prior) */
} trk_skeleton;

#define TRK_MAX_LINKS 79

/* Pinhole intrinsics; pixel (px, py) samples the ray through image coordinates (px, py). */
typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
} trk_intrinsics;

/* Method constants (Secs. 4.1-4.3).  lambda_k0 starts the LM damping; lambda_s weights the pose prior
 * (lambda_s S)^2; lambda_phi and lambda_N weight the offset damping and the neighbour smoothness of
 * Eq. r_warp; lambda_w damps the per-vertex 3x3 systems; cutoff_m is the association cutoff tau;
 * window_half_px the half-size W of the (2W+1)^2 bucket window; eps_vis_m the z-buffer slack of the
 * visibility test; z_near_m the near plane; knn the neighbourhood size |N(i)| (<= 4). */
typedef struct {
  int32_t pose_iters, shape_iters, shape_sweeps;
  float lambda_k0, lambda_s, lambda_phi, lambda_N, lambda_w;
  float cutoff_m, eps_vis_m, z_near_m;
  int32_t window_half_px, knn;
  int32_t precision; /* TRK_PRECISION_*: how [J r]^T [J r] is formed in each pose iteration      */
  int32_t shape_solver; /* 0: Jacobi sweeps with the neighbours frozen (Sec. 4.3; shape_sweeps
                           sweeps); 1: the coupled damped Gauss-Newton system of the whole shape
                           energy by block-Jacobi-preconditioned conjugate gradients (shape_sweeps
                           iterations)                                                               */
  int32_t mode;         /* TRK_MODE_*: which frames run the shape iterations (the paper's experiment
                           conditions, Sec. 5)                                                       */
  int32_t association;  /* 0: the closest visible vertex in the window (Sec. 4.1); 1: the nearest
                           corner of the triangle the z-buffer holds at the pixel (O(1) per pixel)   */
  int32_t jtj_group;    /* vertices per block of the [J r]^T [J r] contraction, in units of 256: 1, 2
                           or 4 (fewer block partials to add; batches of many sessions run faster with
                           4).  0: the larger of
                           the choice by mesh size (1 up to 304 units, 2 up to 608, else 4) and by the
                           expected rows per unit r = 128 c / V, c = distinct pixels the template's
                           vertices round to at the bind pose (4 if r < 18, 2 if r < 30, else 1)      */
} trk_params;

/* TRACK: every frame estimates the shape (the full method).  SHAPE_MATCH: only the first frame after
 * trk_set_pose does; Phi is frozen afterwards.  SMOOTH_BIND: no frame does (Phi stays as set).  A frame
 * without shape iterations reports NaN for their energies. */
#define TRK_MODE_TRACK 0
#define TRK_MODE_SHAPE_MATCH 1
#define TRK_MODE_SMOOTH_BIND 2

/* Arithmetic of the contraction [J r]^T [J r] (Eqs. JTJ, JTr).  FP32: products and per-CTA sums on the
 * FP32 cores.  BF16X3 / TF32X3: every value of [J r] split as hi + lo (BF16 or TF32), the products
 * hi hi + hi lo + lo hi formed on the tensor cores (tcgen05) with FP32 accumulation; relative error of a
 * product about 2^-16 (BF16X3) or 2^-21 (TF32X3) against about 2^-24 for FP32.  In every mode the
 * per-CTA partials are added in FP64, the energy E is summed on the FP32 cores, and the LM system is
 * solved and the step accepted in FP64 (Sec. 4.2). */
#define TRK_PRECISION_FP32 0
#define TRK_PRECISION_BF16X3 1
#define TRK_PRECISION_TF32X3 2

/* Per-frame outputs, written into caller (host) buffers; any pointer may be NULL. */
typedef struct {
  double* theta;         /* [n_links] joint values after the frame                       */
  float* offsets;        /* [n_verts][3] warp offsets Phi after the frame                */
  double* energy;        /* [pose_iters + shape_iters]: E_pose per pose iteration (data + prior,
                            at that iteration's association), then E_shape per shape iteration */
  int32_t n_assoc_px;    /* pixels associated in the last association of the frame      */
  int32_t n_assoc_verts; /* vertices with at least one associated pixel, same pass      */
} trk_result;

/* The 3D position of every link's frame origin (its joint) in the camera frame for joint values theta,
 * by forward kinematics in FP64 (Sec. 3.1: H_{0,j} = H_{0,P(j)} H_{P(j),j} J_j(theta_j)).  out: [n_links][3]
 * metres.  Host only (no device call): the joint positions the pose-accuracy curves of Sec. 5 compare.
 * Errors: TRK_ERR_INVALID_ARG (NULL arguments, a parent not before its child). */
trk_status trk_fk_joint_positions(const trk_skeleton* sk, const double* theta, double* out);

/* ---- template authoring ------------------------------------------------------------------------------
 * The template's construction: a low-resolution polygon cage with skin weights is refined by `levels`
 * levels of Catmull-Clark subdivision, the weights interpolated with the same stencils as the positions
 * (face point: mean of the face; edge point: (a + b + f_a + f_b)/4, midpoint on a boundary; vertex point:
 * (F + 2R + (n - 3)P)/n, (6P + the two boundary neighbours)/8 on a boundary), then every vertex keeps its
 * 4 largest weights (ties to the smaller bone) renormalised to sum 1, and every quad (a, b, c, d) becomes
 * the triangles (a, b, c), (a, c, d).  New vertex order per level: the old vertices' points (same
 * indices), the edge points (edges in order of first appearance walking the faces in order), the face
 * points.  The cage: face_off [n_faces + 1] (face_off[0] = 0, >= 3 corners per face) and face_vert
 * [face_off[n_faces]] (polygons, consistently oriented); host buffers in and out; the points are computed
 * on the current device.  1 <= levels <= 4.  Errors: TRK_ERR_INVALID_ARG, TRK_ERR_OOM, TRK_ERR_CUDA. */
trk_status trk_subdivide_counts(const int32_t* face_off, const int32_t* face_vert, int32_t n_verts, int32_t n_faces,
                                int32_t levels, int32_t* n_verts_out, int32_t* n_tris_out);
/* verts [n_verts][3], bone_idx [n_verts][4] (< n_bones), bone_w [n_verts][4]; outputs sized by
 * trk_subdivide_counts: verts_out [V'][3], tris_out [T'][3], bone_idx_out [V'][4], bone_w_out [V'][4]. */
trk_status trk_subdivide(const float* verts, const int32_t* face_off, const int32_t* face_vert, int32_t n_verts,
                         int32_t n_faces, const uint8_t* bone_idx, const float* bone_w, int32_t n_bones, int32_t levels,
                         float* verts_out, int32_t* tris_out, uint8_t* bone_idx_out, float* bone_w_out);

/* Creates a session on the current CUDA device: validates and copies the model, derives the bind pose
 * H^0 (Sec. 3.2), the prior weights S_kk = n_k/|V| (vertices weighted to the subtree of link k), the
 * vertex-to-face lists and the neighbourhoods N(i) (the knn nearest bind-pose vertices, Sec. 4.3),
 * allocates all device state and sets Theta = 0, Phi = 0.
 * Errors: TRK_ERR_INVALID_ARG (malformed input, *out untouched), TRK_ERR_NO_CAPACITY (too many links),
 * TRK_ERR_OOM, TRK_ERR_CUDA. */
trk_status trk_create(const trk_mesh* mesh, const trk_skeleton* skel, const trk_intrinsics* cam,
                      const trk_params* params, trk_session** out);

/* Sets Theta (host [n_links]) and Phi (host [n_verts][3], NULL = zero) and resets the LM damping to
 * lambda_k0.  Synchronous.  TRK_ERR_NUMERIC on non-finite values. */
trk_status trk_set_pose(trk_session* s, const double* theta, const float* offsets);

/* Tracks one frame (Sec. 4): uploads depth (host [height][width] metres, 0 = no return), runs the
 * frame on the session's stream, waits, and fills *out.  The state carries over to the next frame. */
trk_status trk_track_frame(trk_session* s, const float* depth_m, trk_result* out);

/* Enqueues one frame on cuda_stream (a cudaStream_t; NULL = the session's own stream) reading depth
 * from device memory d_depth_m [height][width].  Returns without waiting; trk_read_result waits for
 * the frame and copies its outputs.  cuda_stream must exist until a call has waited for the frame. */
trk_status trk_track_frame_device(trk_session* s, const float* d_depth_m, void* cuda_stream);
trk_status trk_read_result(trk_session* s, trk_result* out);

/* Renders the model's z-buffer depth at (theta, offsets) (host inputs, offsets NULL = zero) into
 * depth_m (host [height][width], 0 where no triangle covers the pixel).  Does not change the state. */
trk_status trk_render_depth(trk_session* s, const double* theta, const float* offsets, float* depth_m);

/* Checkpoint of the tracking state: what one frame hands to the next (Theta, Phi, the LM damping lambda
 * of R14 and the count of frames since trk_set_pose, which shape-match mode reads), as a host byte blob.
 * A session created from the same model and parameters resumes from it and tracks the following frames
 * bit for bit as the exporting session would have.  Layout (little-endian): 8 bytes "TRKSTATE", int32
 * version (1), int32 n_links, int32 n_verts, int32 frames_done, then double Theta [n_links], double
 * lambda, float Phi [n_verts][4] (x, y, z, 0).
 * Both wait for the session's last frame on the stream it was enqueued on, which must still exist (as
 * for trk_read_result).
 * trk_session_export: blob NULL -> *size_bytes = the blob's size; otherwise writes the blob into blob
 * (host, *size_bytes bytes) and sets *size_bytes to its size.
 * trk_session_import: checks the header against the session (format, n_links, n_verts, size) and the
 * values (finite; lambda > 0; frames_done >= 0), then sets the state.  Synchronous.
 * Errors: TRK_ERR_INVALID_ARG (NULL, a buffer too small, a blob of another format, model size or length;
 * nothing was changed), TRK_ERR_NUMERIC (non-finite values), TRK_ERR_CUDA. */
trk_status trk_session_export(trk_session* s, void* blob, size_t* size_bytes);
trk_status trk_session_import(trk_session* s, const void* blob, size_t size_bytes);

/* Device residency.  A session's device state (model data, tracking state and work buffers: the
 * device_bytes of trk_info) is ONE allocation from the current device's stream-ordered allocator.  An
 * evicted session holds no device memory: its model data and tracking state (Theta, Phi, lambda, frames
 * since trk_set_pose) wait on the host.  This is what lets a frame server admit sessions under an HBM
 * budget (trk_server_attach restores an evicted session, trk_server_detach evicts it again).
 * trk_create_evicted: as trk_create, without the device allocation (Theta = 0, Phi = 0 on the host).
 * trk_session_evict: waits for the session's last frame (on the stream it was enqueued on, which must
 *   still exist), copies the tracking state to the host, frees the device state and the frame graphs.
 *   Batches and schedules built on the session become invalid (their next call fails with
 *   TRK_ERR_INVALID_ARG); a restored session needs a new batch or schedule.  No-op when evicted.
 * trk_session_restore: allocates and fills the device state again and restores the tracking state; the
 *   session then tracks bit for bit as if it had never been evicted.  No-op when resident.
 * While evicted, trk_set_pose, trk_session_export / trk_session_import and trk_get_info work on the host
 * copy; every call that runs kernels or reads device buffers fails with TRK_ERR_INVALID_ARG.
 * Errors: TRK_ERR_INVALID_ARG, TRK_ERR_OOM (restore), TRK_ERR_CUDA. */
trk_status trk_create_evicted(const trk_mesh* mesh, const trk_skeleton* skel, const trk_intrinsics* cam,
                              const trk_params* params, trk_session** out);
trk_status trk_session_evict(trk_session* s);
trk_status trk_session_restore(trk_session* s);
int32_t trk_session_is_resident(const trk_session* s); /* 1 resident, 0 evicted or NULL */

/* Releases every resource of the session.  NULL is allowed. */
void trk_destroy(trk_session* s);

/* Message of the last failing call on this thread ("" if none). */
const char* trk_last_error(void);

/* ---- Step-level calls: each runs one step of an iteration at the session's current state, so that
 * every step can be checked on its own.  They are synchronous and leave their outputs in the session,
 * readable with trk_read. ------------------------------------------------------------------------ */

/* Copies depth (host [height][width]) into the session's depth buffer. */
trk_status trk_set_depth(trk_session* s, const float* depth_m);
/* Sec. 3.1 + Eqs. H_Sigma, deformation: FK of Theta and v_i = H_iSigma (v0_i + phi_i). */
trk_status trk_step_skin(trk_session* s);
/* z-buffer of the posed mesh (packed (depth bits << 32) | triangle, min-reduced) and face normals. */
trk_status trk_step_raster(trk_session* s);
/* Vertex normals (normalised sums of incident face normals), visibility against the z-buffer, and
 * the per-pixel buckets of visible vertices (Sec. 4.1). */
trk_status trk_step_visibility(trk_session* s);
/* Sec. 4.1 association of every valid depth pixel with the closest visible vertex in the window,
 * within the cutoff, and the per-vertex sums of (p_k - v_i). */
trk_status trk_step_associate(trk_session* s);
/* Eq. residual, the pose Jacobian (Sec. 4.2) and the reduced [J r]^T [J r] (Eqs. JTJ, JTr). */
trk_status trk_step_normal_equations(trk_session* s);
/* Damped least squares step with the pose prior (Sec. 4.2): up to 6 damping values are tried in
 * order and the first one that does not raise the energy (at the fixed association) is taken. */
trk_status trk_step_lm(trk_session* s);
/* Sec. 4.3 shape iteration (residuals, per-vertex 3x3 solves, shape_sweeps Jacobi sweeps). */
trk_status trk_step_shape(trk_session* s);

typedef enum {
  TRK_FIELD_VERTS = 0,    /* float[n_verts][4]: posed v_i, camera frame (w unused)          */
  TRK_FIELD_NORMALS = 1,  /* float[n_verts][4]: n_i, w = 1 if the normal is valid           */
  TRK_FIELD_ZBUF = 2,     /* uint64[height*width]: (float bits of depth << 32) | triangle, ~0 = empty */
  TRK_FIELD_VISPIX = 3,   /* int32[n_verts]: pixel index of a visible vertex, -1 otherwise  */
  TRK_FIELD_CORR = 4,     /* int32[height*width]: associated vertex, -1 = none               */
  TRK_FIELD_ACC = 5,      /* int64[n_verts][4]: sum of (p_k - v_i) in units of 2^-30 m, count */
  TRK_FIELD_NORMAL_EQ = 6,/* double[(n_links+1)^2]: [J r]^T [J r], row-major                  */
  TRK_FIELD_THETA = 7,    /* double[n_links]                                                 */
  TRK_FIELD_PHI = 8,      /* float[n_verts][4] (w unused)                                    */
  TRK_FIELD_LAMBDA = 9,   /* double[1]: LM damping                                           */
  TRK_FIELD_ENERGY = 10,  /* double[pose_iters + shape_iters] of the last frame              */
  TRK_FIELD_LM_TRIALS = 11,/* double[8]: E of each attempted damping value (+inf if not tried), then
                              the current E, then the accepted attempt index (-1 = none)          */
  TRK_FIELD_SHAPE_RG = 12,/* float[n_verts][4]: g_i = dr_i/dphi_i and r_i of the last shape step */
  TRK_FIELD_NEIGHBOURS = 13,/* int32[n_verts][4]: N(i), -1 pads                              */
  TRK_FIELD_PRIOR = 14,   /* double[n_links]: (lambda_s S_kk)^2                              */
  TRK_FIELD_LM_SOLVER = 15,/* int32[6]: per damping candidate of the last LM step, refinement iterations
                              of the mixed-precision solve, -1 = FP64 fallback, -2 = not positive definite */
  TRK_FIELD_COUNT = 16
} trk_field;

/* Copies a session buffer to host memory; bytes must equal the field's size exactly. */
trk_status trk_read(trk_session* s, trk_field field, void* host_dst, size_t bytes);

/* ---- Introspection and timing ------------------------------------------------------------------ */
typedef struct {
  int32_t n_links, n_verts, n_tris, width, height;
  int32_t kernels_per_frame; /* kernel launches in one trk_track_frame                          */
  size_t device_bytes;       /* device memory the session holds                                  */
  int32_t jtj_group;         /* the [J r] contraction's vertices per block / 256 (trk_params)     */
} trk_info;
trk_status trk_get_info(trk_session* s, trk_info* out);

/* Stages of one iteration, in launch order, as timed by trk_profile_iteration. */
typedef enum {
  TRK_STAGE_SKIN = 0, TRK_STAGE_RASTER, TRK_STAGE_VISIBILITY, TRK_STAGE_ASSOCIATE, TRK_STAGE_RESID_JTJ,
  TRK_STAGE_REDUCE, TRK_STAGE_LM_SOLVE, TRK_STAGE_LM_EVAL, TRK_STAGE_SHAPE, TRK_STAGE_COUNT
} trk_stage;

/* Runs reps pose iterations (and reps shape steps, from the state they reach) at the session's state
 * and depth, launching each stage's kernel(s) between CUDA events recorded on the session's stream, and
 * writes the mean duration of each stage in milliseconds to ms (host [TRK_STAGE_COUNT]).  The state
 * advances as in tracking.  flush_bytes > 0 overwrites a scratch buffer of that size before each stage
 * (outside the timed interval) so that every stage starts from a cold L2. */
trk_status trk_profile_iteration(trk_session* s, int32_t reps, size_t flush_bytes, float* ms);

/* ---- Serving: continuous batching of frames from many sessions on one device -------------------- */

typedef struct trk_server trk_server;

typedef struct {
  uint64_t frames_done;     /* frames completed since the server was created            */
  int32_t in_flight;        /* frames on the GPU now                                     */
  int32_t sessions;         /* attached sessions                                         */
  size_t hbm_used_bytes;    /* what the budget counts: the attached sessions' arenas and the batched
                               steps' buffers (per slot twice the largest sum of the sessions' step
                               tables so far), all in 2 MiB units                                     */
  double latency_p50_us, latency_p99_us, latency_max_us;  /* submit -> completion, wall time; the
                               percentiles to 1.2 % (log-spaced bins), the maximum exact */
  uint64_t steps;           /* launches of frames: batched steps plus single-session frames */
  double mean_frames_per_step;
  size_t device_bytes_reserved; /* device memory the library holds now (the arenas of every resident
                                   session, any server's step buffers), in 2 MiB units                */
} trk_server_stats;

/* How the dispatcher launches ready frames.  BATCHED (the default): the ready frames of sessions that
 * share the iteration schedule, precision, association and tracking mode (TRK_MODE_TRACK) go into one
 * batched frame -- every stage one kernel launch over the blocks of all of them -- with the depth read
 * from and the results written to host-mapped pinned staging; sessions in other modes run alone.
 * SESSION: every frame runs its session's own frame graph on the session's stream. */
#define TRK_SERVER_DISPATCH_BATCHED 0
#define TRK_SERVER_DISPATCH_SESSION 1

/* Creates a frame server on the current device.  Sessions are admitted while the sum of their device
 * memory stays within hbm_budget_bytes; at most max_inflight frames run on the GPU at a time (0 admits
 * frames but never launches them).  A dispatcher thread launches a session's next frame as soon as its
 * previous frame is done and a slot is free (see TRK_SERVER_DISPATCH_*), so frames of different
 * sessions overlap on the device and one session's frames run in submission order. */
trk_status trk_server_create(size_t hbm_budget_bytes, int32_t max_inflight, trk_server** out);
/* Dispatch mode, the most frames in one batched step (1..4096, default 64), the number of batched steps
 * that may run at once (1..16, default 2, each on its own stream) and max_wait_us (default 2000): while
 * a batched step runs, ready frames wait for a fuller step until they are (compatible sessions /
 * concurrent_steps) or the oldest has waited max_wait_us; with no step running they go at once.  Only
 * before the first attach. */
trk_status trk_server_configure(trk_server* sv, int32_t dispatch, int32_t max_batch, int32_t concurrent_steps,
                                int64_t max_wait_us);
/* Admits a session (same device).  TRK_ERR_NO_CAPACITY if its device bytes (its arena and, for batched
 * dispatch, its share of the step buffers) do not fit the remaining budget.  An evicted session
 * (trk_create_evicted, trk_session_evict) is restored here -- its device state is allocated at admission
 * -- and evicted again at trk_server_detach, so the budget bounds the device memory of such sessions
 * (arenas and step buffers are counted at the 2 MiB allocation granularity); a session that is already
 * resident is counted but holds its memory
 * regardless.  While attached, the session must be driven only through the server. */
trk_status trk_server_attach(trk_server* sv, trk_session* s);
/* Releases a session's budget (evicting it if attach restored it); TRK_ERR_INVALID_ARG while it still
 * has frames queued or running. */
trk_status trk_server_detach(trk_server* sv, trk_session* s);
/* Queues one frame (host depth [height][width], copied at the call) and returns its ticket. */
trk_status trk_server_submit(trk_server* sv, trk_session* s, const float* depth_m, uint64_t* ticket);
/* Waits up to timeout_us for the frame and fills *out (host buffers, as trk_track_frame; out may be
 * NULL).  TRK_ERR_TIMEOUT if the frame is not done by then (the ticket stays valid); TRK_ERR_INVALID_ARG
 * for an unknown or already collected ticket.  Each ticket is collected once. */
trk_status trk_server_wait(trk_server* sv, uint64_t ticket, int64_t timeout_us, trk_result* out);
trk_status trk_server_get_stats(trk_server* sv, trk_server_stats* out);
/* Stops the dispatcher, waits for frames on the GPU, frees every uncollected frame and evicts the
 * sessions that attach restored. */
void trk_server_destroy(trk_server* sv);

/* ---- Standalone contraction ------------------------------------------------------------------- */

/* [J r]^T [J r] of materialised rows (Eqs. JTJ, JTr): d_rows is device FP32 [n_rows][ld], each row the
 * Jacobian entries of one residual followed by the residual itself in its first n_cols columns; d_out
 * receives device FP64 [n_cols][n_cols], row-major and symmetric (J^T J, J^T r and r^T r as blocks).
 * Products are formed in FP32 and summed per CTA in FP32, the CTA partials in FP64 in a fixed order.
 * Enqueued on cuda_stream (a cudaStream_t, NULL = the legacy default stream); returns without waiting.
 * Scratch for the per-CTA partials (at most 296 n_cols^2 floats) comes from the stream-ordered
 * allocator of the current device and is released on the stream.  1 <= n_cols <= 80, ld >= n_cols,
 * n_rows >= 0 (0 rows gives zeros).  Errors: TRK_ERR_INVALID_ARG, TRK_ERR_OOM, TRK_ERR_CUDA. */
trk_status trk_jtj_rows(const float* d_rows, int32_t n_rows, int32_t n_cols, int32_t ld, double* d_out,
                        void* cuda_stream);

/* The same contraction for callers that must not allocate device memory: a real-time frame loop that
 * may not call the CUDA allocator once running (cudaMalloc and cudaFree can synchronise the device and
 * take unbounded time), or a host whose device memory is owned by another allocator or a fixed budget
 * that forbids side allocations.  The paper has no counterpart; this is an interface for such callers.
 * Arguments, layout and tolerance are those of trk_jtj_rows; the caller passes the rows and the output
 * buffer.  It runs at most 152 CTAs (trk_jtj_rows up to 296), so its result is bitwise that of
 * trk_jtj_rows when n_rows <= 152 * 256 = 38,912 (both use ceil(n_rows / 256) CTAs) and otherwise
 * differs from it by rounding only (the CTA partials split the rows differently).
 * Scratch: a fixed array of 152 x 80 x 80 floats (3.9 MB) that every device loading this library holds
 * until the process exits, shared by all calls.  Each call overwrites the part it uses, so no clearing
 * is needed, but calls that overlap on the GPU (concurrent streams, threads) race on it: serialise them.
 * No allocation of any kind is made.  The first call on a device looks up the array's device address
 * (once per device, with that device current); make that first call before any stream capture.
 * Errors: TRK_ERR_INVALID_ARG (n_cols outside [1, 80], bad pointers or sizes), TRK_ERR_CUDA. */
trk_status trk_jtj_rows_noalloc(const float* d_rows, int32_t n_rows, int32_t n_cols, int32_t ld, double* d_out,
                                void* cuda_stream);

/* ---- batches: many sessions stepped by the same launches ------------------------------------------
 * A batch runs one frame of every member session per call, each stage of the frame (Secs. 4.1-4.3) as
 * ONE kernel launch over the blocks of all members (a block table maps each block to its session), the
 * whole frame as one CUDA graph.  Members may differ in mesh, skeleton and image size; they must share
 * the device (the current one), the iteration schedule (pose_iters, shape_iters, shape_sweeps) and the
 * precision.  Each member's results are bitwise those it computes alone.  A session may belong to
 * several batches but must not be stepped by two calls at the same time (same rule as for sessions). */
typedef struct trk_batch trk_batch;

/* Builds the block tables and captures the frame graph.  The session pointers are borrowed: destroy the
 * batch before any of its sessions.  Errors: TRK_ERR_INVALID_ARG (NULL or repeated session, members that
 * differ in device, schedule or precision), TRK_ERR_OOM, TRK_ERR_CUDA. */
trk_status trk_batch_create(trk_session* const* sessions, int32_t n_sessions, trk_batch** out);

/* One frame of every member: member k reads its depth image from the device buffer d_depths[k] (host
 * array of n_sessions device pointers, row-major float32 metres, 0 = invalid).  Enqueued on cuda_stream
 * (NULL = legacy default stream); results stay in each session's device state: trk_read_result(member)
 * reads them in stream order.  The depth buffers must stay valid until the stream reaches the frame. */
trk_status trk_batch_track_device(trk_batch* b, const float* const* d_depths, void* cuda_stream);

/* Mean CUDA-event time (ms) of each stage of one pose iteration (TRK_STAGE_*: skin ... lm_eval) and of
 * the shape step, as ONE batched launch each, over reps repetitions at the members' current state on the
 * depth images d_depths (flush_bytes > 0: that many bytes are written before each stage, so the stage
 * starts with a cold L2).  The stages run for real: the members' state advances.  Synchronises. */
trk_status trk_batch_profile(trk_batch* b, const float* const* d_depths, int32_t reps, size_t flush_bytes, float* ms);

/* Waits for the batch's outstanding work and releases its device tables and graph. */
void trk_batch_destroy(trk_batch* b);

/* ---- schedules and the autotuner --------------------------------------------------------------------
 * A schedule steps a set of sessions each frame as `groups` work-balanced groups on concurrent streams:
 * a group of several sessions as one fused batch (trk_batch), a group of one as the session's own frame
 * graph (groups = 1: one fused batch; groups = n: one graph per session).  The fused groups' association
 * launches use assoc_blocks persistent tile blocks and tail_blocks queue-draining blocks.  Every session
 * computes bitwise the same under every schedule.  The members follow the batch rules (same device,
 * schedule of iterations and precision when grouped). */
typedef struct {
  int32_t groups;        /* 1 <= groups <= n                                     */
  int32_t assoc_blocks;  /* >= 1 */
  int32_t tail_blocks;   /* >= 1 */
} trk_schedule_config;

typedef struct trk_schedule trk_schedule;

/* cfg: the schedule to use; NULL = the entry of cache_path for this size class (trk_schedule_signature)
 * if there is one, else groups = 1, assoc_blocks = 608, tail_blocks = 304.  Session pointers are
 * borrowed.  Errors: TRK_ERR_INVALID_ARG, TRK_ERR_OOM, TRK_ERR_CUDA. */
trk_status trk_schedule_create(trk_session* const* sessions, int32_t n_sessions, const trk_schedule_config* cfg,
                               const char* cache_path, trk_schedule** out);

/* One frame of every session (depth of session k from the device buffer d_depths[k]), enqueued on
 * cuda_stream; results via trk_read_result(session) in that stream's order. */
trk_status trk_schedule_track_device(trk_schedule* s, const float* const* d_depths, void* cuda_stream);

trk_status trk_schedule_get_config(const trk_schedule* s, trk_schedule_config* out);

/* Times candidate schedules (groups from {1, 2, 4, ..., 32, n}, then the association block counts around
 * the best; 1 warm-up and `reps` timed frames each, CUDA events) on the frames d_depths, keeps the
 * fastest, optionally stores it in cache_path under this size class and returns it with its time per
 * frame.  The timed frames are real: every session advances by (1 + reps) frames per candidate, so tune
 * on warm-up frames.  Synchronises the device.  Errors: as trk_schedule_create; TRK_ERR_INVALID_ARG if
 * the cache cannot be written. */
trk_status trk_schedule_autotune(trk_schedule* s, const float* const* d_depths, int32_t reps, const char* cache_path,
                                 trk_schedule_config* chosen, double* ms_per_step);

void trk_schedule_destroy(trk_schedule* s);

/* The size class a schedule is cached under: session count, precision, total vertices and pixels (two
 * significant digits) and the largest skeleton, e.g. "n16_p0_v800000_px4900000_L55".  Host only. */
trk_status trk_schedule_signature(trk_session* const* sessions, int32_t n_sessions, char* out, size_t out_size);

/* The tuning cache, a JSON object {"<size class>": {"groups": .., "assoc_blocks": .., "tail_blocks": ..,
 * "ms_per_step": ..}, ...}.  Host only (no device calls).  lookup: TRK_ERR_INVALID_ARG when the file or
 * the entry is missing or malformed; store: adds or replaces the entry (written through a temporary
 * file and a rename). */
trk_status trk_tuning_cache_lookup(const char* path, const char* signature, trk_schedule_config* out, double* ms);
trk_status trk_tuning_cache_store(const char* path, const char* signature, const trk_schedule_config* cfg, double ms);

/* The same contraction on the tensor cores (Eqs. JTJ, JTr): out = R^T R for the FP32 rows R as in
 * trk_jtj_rows, with precision TRK_PRECISION_BF16X3 or TRK_PRECISION_TF32X3.  Each CTA accumulates
 * 64-row chunks in tensor memory (FP32) and drains them every 512 rows into Kahan-compensated FP32 sums;
 * the CTA sums (value and compensation) are added in FP64 in a fixed order, so the result is
 * deterministic for given arguments.  Entry error against the exact R^T R: about 2^-16 (BF16X3) or 2^-21
 * (TF32X3) times sum_k |R_ka R_kb|.  Scratch (at most 2 x 296 n_cols^2 floats) comes from the
 * stream-ordered allocator and is released on the stream.  1 <= n_cols <= 80, ld >= n_cols, n_rows >= 0.
 * Errors: TRK_ERR_INVALID_ARG, TRK_ERR_OOM, TRK_ERR_CUDA.  Entries are NaN if a tensor-core completion
 * wait ran out (about one second; a failure of the device, not of the data). */
trk_status trk_jtj_rows_tc(const float* d_rows, int32_t n_rows, int32_t n_cols, int32_t ld, int32_t precision,
                           double* d_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TRK_H_ */

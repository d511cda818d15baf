"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in a copy of oracle/oracle.c (a
sign, an index, an operand order, a dropped term, a wrong tie rule), compiles it with the oracle's flags, points
the oracle module at the mutant library, and runs the pins named for it: at least one must fail.  Mistakes are
planted in the oracle on the CPU only."""
import concurrent.futures as cf
import contextlib
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_geometry as geo
from tests import test_oracle_kinematics as kin
from tests import test_oracle_optim as opt
from tests import test_oracle_pcg as pcg
from tests import test_oracle_rid as rid
from tests import test_oracle_subdivision as sub

# (name, text in oracle.c, replacement (first occurrence), pins of which one must fail)
MUTANTS = [
    ("quaternion product: transposed cross term",
     "a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y", "a.w * b.x + a.x * b.w - a.y * b.z + a.z * b.y",
     [kin.test_fk_equals_homogeneous_matrix_chain]),
    ("dual quaternion product: dual part in the wrong order",
     "h.d = q_add(q_mul(a.r, b.d), q_mul(a.d, b.r));", "h.d = q_add(q_mul(b.d, a.r), q_mul(a.d, b.r));",
     [kin.test_fk_equals_homogeneous_matrix_chain]),
    ("hinge: full angle instead of half angle",
     "double c = cos(0.5 * th), s = sin(0.5 * th);\n    h.r = q_make(c,", "double c = cos(th), s = sin(th);\n    h.r = q_make(c,",
     [kin.test_fk_equals_homogeneous_matrix_chain]),
    ("prismatic joint: translation not halved",
     "h.d = q_make(0, z[0] * 0.5 * th, z[1] * 0.5 * th, z[2] * 0.5 * th);", "h.d = q_make(0, z[0] * th, z[1] * th, z[2] * th);",
     [kin.test_fk_equals_homogeneous_matrix_chain, kin.test_single_bone_vertices_move_rigidly]),
    ("FK: joint applied before the link offset",
     "H0[j] = dq_mul(dq_mul(hp, m->off[j]), hj);", "H0[j] = dq_mul(dq_mul(hp, hj), m->off[j]);",
     [kin.test_fk_equals_homogeneous_matrix_chain]),
    ("H_Delta: inverse bind pose on the wrong side",
     "Hd[j] = dq_mul(H0[j], dq_conj(m->bind[j]));", "Hd[j] = dq_mul(dq_conj(m->bind[j]), H0[j]);",
     [kin.test_single_bone_vertices_move_rigidly]),
    ("point map: dual part not doubled",
     "out[0] = (t1.x + 2.0 * t2.x) / N;", "out[0] = (t1.x + t2.x) / N;",
     [kin.test_single_bone_vertices_move_rigidly]),
    ("point map: not normalised by |a|^2",
     "double N = q_dot(a, a);\n  quat X = q_make(0, x[0], x[1], x[2]);\n  quat t1",
     "double N = 1.0;\n  quat X = q_make(0, x[0], x[1], x[2]);\n  quat t1",
     [kin.test_point_map_is_scale_invariant, kin.test_blend_of_coaxial_rotations_turns_by_the_blended_half_angle]),
    ("blend: no antipodal sign alignment (R1)",
     "double sg = q_dot(h.r, Hd[jstar].r) >= 0 ? 1.0 : -1.0;", "double sg = 1.0;",
     [kin.test_antipodal_bone_is_sign_aligned]),
    ("hinge derivative: wrong sign of the scalar part",
     "h.r = q_make(-0.5 * s, 0.5 * c * z[0]", "h.r = q_make(0.5 * s, 0.5 * c * z[0]",
     [opt.test_jacobian_matches_central_differences]),
    ("point-map derivative: normalisation term dropped",
     "out[0] = (u1.x + 2.0 * u2.x) / N - s * T[0];", "out[0] = (u1.x + 2.0 * u2.x) / N;",
     [opt.test_jacobian_matches_central_differences]),
    ("Jacobian: descendant transforms multiplied in the wrong order",
     "suffix = dq_mul(dq_mul(m->off[k], joint_dq(m->jtype[k], m->axis + 3 * k, theta[k])), suffix);",
     "suffix = dq_mul(suffix, dq_mul(m->off[k], joint_dq(m->jtype[k], m->axis + 3 * k, theta[k])));",
     [opt.test_jacobian_matches_central_differences]),
    ("Jacobian: sign of the residual derivative",
     "row[k] = -(n[3 * i] * dv[0]", "row[k] = (n[3 * i] * dv[0]",
     [opt.test_jacobian_matches_central_differences]),
    ("normals: cross product operands swapped",
     "double fn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};",
     "double fn[3] = {e2[1] * e1[2] - e2[2] * e1[1], e2[2] * e1[0] - e2[0] * e1[2], e2[0] * e1[1] - e2[1] * e1[0]};",
     [geo.test_flat_grid_has_constant_normal, geo.test_capsule_normals_are_radial_within_mesh_spacing]),
    ("raster: edge function with the wrong vertex",
     "double w1 = (ua - uc) * (py - vc) - (va - vc) * (px - uc);", "double w1 = (ua - uc) * (py - vc) - (va - vc) * (px - ub);",
     [geo.test_raster_equals_brute_force_ray_casting]),
    ("raster: pixel centres at half-integer coordinates",
     "double dx = (px - cx) / fx, dy = (py - cy) / fy;", "double dx = (px + 0.5 - cx) / fx, dy = (py + 0.5 - cy) / fy;",
     [geo.test_raster_equals_brute_force_ray_casting, geo.test_tilted_plane_depth_closed_form]),
    ("visibility: back faces kept instead of front faces",
     "if (!(nd < 0)) continue;", "if (!(nd > 0)) continue;",
     [geo.test_visibility_occlusion_backface_and_image_bounds]),
    ("association: ties to the larger index",
     "(dd == bd2 && i < best))) { best = i; bd2 = dd; }", "(dd == bd2 && i > best))) { best = i; bd2 = dd; }",
     [geo.test_association_ties_go_to_smaller_index]),
    ("association: cutoff compared with the unsquared distance",
     "double tau = m->p.cutoff, tau2 = tau * tau, tol = 1e-5;\n  /* buckets",
     "double tau = m->p.cutoff, tau2 = tau, tol = 1e-5;\n  /* buckets",
     [geo.test_single_vertex_collects_every_pixel_within_cutoff, geo.test_association_equals_brute_force]),
    ("association: window one pixel short on the right",
     "for (int qx = px - R; qx <= px + R; ++qx) {\n          if (qx < 0 || qx >= W) continue;\n          int q = qy * W + qx;\n          for (int t = start[q];",
     "for (int qx = px - R; qx < px + R; ++qx) {\n          if (qx < 0 || qx >= W) continue;\n          int q = qy * W + qx;\n          for (int t = start[q];",
     [geo.test_association_equals_brute_force]),
    ("raster-ID association: ties to the larger index",
     "if (dd <= tau2 && (best < 0 || dd < bd2 || (dd == bd2 && i < best))) { best = i; bd2 = dd; }\n      }\n      if (tie) {",
     "if (dd <= tau2 && (best < 0 || dd < bd2 || (dd == bd2 && i > best))) { best = i; bd2 = dd; }\n      }\n      if (tie) {",
     [rid.test_equidistant_corners_go_to_the_smaller_index]),
    ("residual: sum of offsets not averaged",
     "n[3 * i + 2] * acc[3 * i + 2]) / cnt[i];\n    r[i] = ri;", "n[3 * i + 2] * acc[3 * i + 2]);\n    r[i] = ri;",
     [opt.test_residual_averages_the_points_a_vertex_collects]),
    ("normal equations: sign of J^T r",
     "JTr[a] += row[a] * r[i];", "JTr[a] -= row[a] * r[i];",
     [opt.test_normal_equations_equal_explicit_products]),
    ("Cholesky: back substitution with the transposed factor",
     "for (int k = i + 1; k < n; ++k) t -= C[k * n + i] * x[k];", "for (int k = i + 1; k < n; ++k) t -= C[i * n + k] * x[k];",
     [opt.test_cholesky_solve_equals_gaussian_elimination]),
    ("LM: damping lambda I instead of lambda diag A (R13)",
     "A[a * L + c] + (a == c ? lk * A[a * L + a] : 0.0);", "A[a * L + c] + (a == c ? lk : 0.0);",
     [opt.test_lm_accepts_only_descent_and_updates_lambda]),
    ("LM: lambda divided by 2 on acceptance (R14)",
     "lk = lk / 10.0;", "lk = lk / 2.0;",
     [opt.test_lm_accepts_only_descent_and_updates_lambda]),
    ("LM: pose prior missing from the right-hand side",
     "b[k] = JTr[k] + s2 * theta[k];", "b[k] = JTr[k];",
     [opt.test_lm_accepts_only_descent_and_updates_lambda]),
    ("shape step: smoothness missing from the 3x3 system",
     "Mx[3 * a + c] = gi[a] * gi[c] + (a == c ? lp + lN * nn : 0.0);", "Mx[3 * a + c] = gi[a] * gi[c] + (a == c ? lp : 0.0);",
     [opt.test_smoothness_alone_moves_each_offset_to_its_neighbours_mean]),
    ("shape step: sign of the smoothness gradient",
     "for (int c = 0; c < 3; ++c) grad[c] += lN * (pi[c] - cur[3 * q + c]);", "for (int c = 0; c < 3; ++c) grad[c] -= lN * (pi[c] - cur[3 * q + c]);",
     [opt.test_smoothness_alone_moves_each_offset_to_its_neighbours_mean]),
    ("shape step: damping lambda_w I instead of lambda_w diag",
     "for (int a = 0; a < 3; ++a) Md[4 * a] += lw * Mx[4 * a];", "for (int a = 0; a < 3; ++a) Md[4 * a] += lw;",
     [opt.test_shape_step_closed_form_without_smoothness]),
    ("PCG: off-diagonal coupling with the wrong sign",
     "for (int t = off[i]; t < off[i + 1]; ++t) s -= lN * pv[3 * adj[t] + a];", "for (int t = off[i]; t < off[i + 1]; ++t) s += lN * pv[3 * adj[t] + a];",
     [pcg.test_converged_pcg_minimises_the_quadratic_model]),
    ("PCG: preconditioner blocks not damped",
     "for (int a = 0; a < 3; ++a) Bk[9 * i + 4 * a] += lw * Bk[9 * i + 4 * a];", "for (int a = 0; a < 3; ++a) Bk[9 * i + 4 * a] += 0.0;",
     [pcg.test_without_smoothness_one_pcg_iteration_is_the_per_vertex_solve, pcg.test_converged_pcg_minimises_the_quadratic_model]),
    ("prior weights: vertices counted on their own link only (R10)",
     "for (int k = m->bidx[4 * i + s]; k >= 0; k = m->parent[k]) {", "for (int k = m->bidx[4 * i + s]; k >= 0; k = -1) {",
     [geo.test_prior_weights_count_subtree_vertices]),
    ("subdivision: vertex point with R weighted once",
     "*o = (Fs[(size_t)v * A + c] / n + 2.0 * Rs[(size_t)v * A + c] / nR[v] + (n - 3.0) * P) / n;",
     "*o = (Fs[(size_t)v * A + c] / n + Rs[(size_t)v * A + c] / nR[v] + (n - 2.0) * P) / n;",
     [sub.test_cube_closed_forms]),
    ("subdivision: interior edge point without the face points",
     ": 0.25 * (pa + pb + FP[(size_t)E[e].fa * A + c] + FP[(size_t)E[e].fb * A + c]);", ": 0.5 * (pa + pb);",
     [sub.test_cube_closed_forms]),
    ("subdivision: boundary vertex rule",
     "*o = nB[v] == 2 ? (6.0 * P + Bs[(size_t)v * A + c]) / 8.0 : P;", "*o = nB[v] == 2 ? (4.0 * P + Bs[(size_t)v * A + c]) / 6.0 : P;",
     [sub.test_triangle_cage_and_open_boundary]),
    ("FK: grandparent taken for the parent",
     "dquat hp = m->parent[j] < 0 ? dq_identity() : H0[m->parent[j]];",
     "dquat hp = m->parent[j] < 0 ? dq_identity() : H0[m->parent[j] > 0 ? m->parent[m->parent[j]] < 0 ? m->parent[j] : m->parent[m->parent[j]] : m->parent[j]];",
     [kin.test_fk_equals_homogeneous_matrix_chain]),
    ("visibility: no tolerance behind the z-buffer",
     "if (isfinite(Z) && !(p[2] <= Z + m->p.eps_vis)) continue;", "if (isfinite(Z) && !(p[2] <= Z)) continue;",
     [geo.test_visibility_rounds_to_the_nearest_pixel_and_tolerates_eps_vis]),
    ("visibility: pixel by truncation instead of rounding",
     "double fu = floor(u + 0.5), fv = floor(vv + 0.5);\n    if (marg) {", "double fu = floor(u), fv = floor(vv);\n    if (marg) {",
     [geo.test_visibility_rounds_to_the_nearest_pixel_and_tolerates_eps_vis]),
    ("visibility: image bound one pixel too wide",
     "if (fu < 0 || fv < 0 || fu >= m->W || fv >= m->H) continue;\n    int k = (int)fv * m->W + (int)fu;",
     "if (fu < 0 || fv < 0 || fu > m->W || fv >= m->H) continue;\n    int k = (int)fv * m->W + (int)fu;",
     [geo.test_visibility_rounds_to_the_nearest_pixel_and_tolerates_eps_vis]),
    ("association: back-projection not scaled by the depth",
     "double p[3] = {(px - m->cx) * d / m->fx, (py - m->cy) * d / m->fy, d};\n      int best = -1;",
     "double p[3] = {(px - m->cx) / m->fx, (py - m->cy) / m->fy, d};\n      int best = -1;",
     [geo.test_association_equals_brute_force, geo.test_single_vertex_collects_every_pixel_within_cutoff]),
    ("accumulation: offsets v - p instead of p - v",
     "acc[3 * best] += p[0] - v[3 * best];", "acc[3 * best] += v[3 * best] - p[0];",
     [geo.test_association_equals_brute_force, opt.test_residual_averages_the_points_a_vertex_collects]),
    ("knn: neighbour ties to the larger index (R16)",
     "if (nb == K && (d2 > bd[K - 1] || (d2 == bd[K - 1] && j > bi[K - 1]))) continue;",
     "if (nb == K && (d2 > bd[K - 1] || (d2 == bd[K - 1] && j < bi[K - 1]))) continue;",
     [geo.test_knn_ties_on_a_regular_grid_go_to_smaller_index]),
    ("energy: pose prior dropped",
     "for (int k = 0; k < m->L; ++k) { double s = m->p.lambda_s * m->S[k] * theta[k]; E += s * s; }\n  return E;\n}\n\n/* Sec. 4.2 block",
     "return E;\n}\n\n/* Sec. 4.2 block",
     [opt.test_energy_without_data_is_the_pose_prior]),
    ("Cholesky: forward substitution not divided by the pivot",
     "y[i] = t / C[i * n + i];", "y[i] = t;",
     [opt.test_cholesky_solve_equals_gaussian_elimination]),
    ("shape step: Gauss-Seidel instead of Jacobi (neighbours not frozen)",
     "for (int c = 0; c < 3; ++c) grad[c] += lN * (pi[c] - cur[3 * q + c]);", "for (int c = 0; c < 3; ++c) grad[c] += lN * (pi[c] - phi[3 * q + c]);",
     [opt.test_smoothness_alone_moves_each_offset_to_its_neighbours_mean]),
    ("subdivision: face point divided by 4 whatever the face size",
     "FP[(size_t)f * A + c] = s / k;", "FP[(size_t)f * A + c] = s / 4;",
     [sub.test_triangle_cage_and_open_boundary]),
    ("subdivision: quad corners in the wrong order",
     "out_quads[4 * q + 1] = V + fedge[face_off[f] + i];", "out_quads[4 * q + 1] = V + fedge[face_off[f] + (i + k - 1) % k];",
     [sub.test_counts_and_euler_characteristic]),
    ("Jacobian: bone derivatives blended without the R1 signs",
     "dH = dq_axpy(dH, w * sg[s], dHd[j * L + k]);", "dH = dq_axpy(dH, w, dHd[j * L + k]);",
     [opt.test_jacobian_matches_central_differences_across_an_antipodal_bone]),
    ("prismatic derivative: not halved",
     "h.d = q_make(0, 0.5 * z[0], 0.5 * z[1], 0.5 * z[2]);", "h.d = q_make(0, z[0], z[1], z[2]);",
     [opt.test_jacobian_matches_central_differences]),
    ("shape step: residual not re-linearised in later sweeps",
     "if (inA[i]) ri = r0[i] + gi[0] * (pi[0] - phi0[3 * i]) + gi[1] * (pi[1] - phi0[3 * i + 1]) + gi[2] * (pi[2] - phi0[3 * i + 2]);",
     "if (inA[i]) ri = r0[i];",
     [opt.test_second_sweep_is_a_fixed_point_without_smoothness_and_damping]),
    ("PCG: step length halved",
     "const double alpha = rz / pAp;", "const double alpha = 0.5 * rz / pAp;",
     [pcg.test_converged_pcg_minimises_the_quadratic_model, pcg.test_without_smoothness_one_pcg_iteration_is_the_per_vertex_solve]),
    ("PCG: search directions not conjugated",
     "for (size_t k = 0; k < n3; ++k) pv[k] = z[k] + beta * pv[k];", "for (size_t k = 0; k < n3; ++k) pv[k] = z[k];",
     [pcg.test_pcg_iterate_minimises_over_the_krylov_subspace]),
    ("raster: triangles behind the near plane not skipped",
     "if (A[2] <= znear || B[2] <= znear || C[2] <= znear) continue;\n    double ua", "double ua",
     [geo.test_triangle_crossing_the_near_plane_is_skipped]),
    ("LM: five damping attempts instead of six (R14)",
     "for (int t = 0; t < 6; ++t) {\n    /* (A + lambda diag A)", "for (int t = 0; t < 5; ++t) {\n    /* (A + lambda diag A)",
     [opt.test_lm_accepts_only_descent_and_updates_lambda]),
    ("subdivision: boundary edge point not the midpoint",
     "EP[(size_t)e * A + c] = E[e].fb < 0 ? 0.5 * (pa + pb)", "EP[(size_t)e * A + c] = E[e].fb < 0 ? (pa + pb) / 3.0",
     [sub.test_triangle_cage_and_open_boundary]),
    ("normals: a face's third corner not credited",
     "for (int t = 0; t < 3; ++t)\n      for (int k = 0; k < 3; ++k) acc[3 * tri[3 * f + t] + k] += fn[k];",
     "for (int t = 0; t < 2; ++t)\n      for (int k = 0; k < 3; ++k) acc[3 * tri[3 * f + t] + k] += fn[k];",
     [geo.test_flat_grid_has_constant_normal, geo.test_capsule_normals_are_radial_within_mesh_spacing]),
    ("visibility: front-facing judged along the optical axis instead of the view ray",
     "double nd = n[3 * i] * p[0] + n[3 * i + 1] * p[1] + n[3 * i + 2] * p[2];", "double nd = n[3 * i + 2];",
     [geo.test_back_face_is_judged_along_the_view_ray]),
    ("z-buffer: depth ties to the later triangle",
     "if (zt < z[k] || (zt == z[k] && f < ztri[k])) { z[k] = zt; ztri[k] = f; }", "if (zt <= z[k]) { z[k] = zt; ztri[k] = f; }",
     [geo.test_coincident_triangles_keep_the_smaller_index]),
    ("LM: no lower bound on lambda (R14)",
     "if (lk < 1e-7) lk = 1e-7;", "",
     [opt.test_lm_lambda_stays_within_its_bounds]),
    ("LM: no upper bound on lambda (R14)",
     "if (lk > 1e7) lk = 1e7;", "",
     [opt.test_lm_lambda_stays_within_its_bounds]),
    ("association: near-equal candidates not flagged as ties",
     "if (tie && d2nd <= tau + tol && d2nd - d1 < tol) tie[k] = 1;", "",
     [geo.test_near_ties_are_flagged]),
    ("visibility: the facing decision never marginal",
     "if (fabs(nd) < tol_facing * pl || ru < tol_px", "if (ru < tol_px",
     [geo.test_visibility_flags_exactly_its_marginal_decisions]),
    ("visibility: facing band an absolute 1e-4 m instead of 1e-4 |p|",
     "if (fabs(nd) < tol_facing * pl ||", "if (fabs(nd) < tol_facing ||",
     [geo.test_visibility_flags_exactly_its_marginal_decisions]),
    ("visibility: pixel rounding marginal on one side of the edge only",
     "|| ru < tol_px || ru > 1 - tol_px ||", "|| ru > 1 - tol_px ||",
     [geo.test_visibility_flags_exactly_its_marginal_decisions]),
    ("visibility: pixel rounding marginal in u only",
     "|| rv < tol_px || rv > 1 - tol_px) marg[i] = 1;", ") marg[i] = 1;",
     [geo.test_visibility_flags_exactly_its_marginal_decisions]),
    ("visibility: the depth test never marginal",
     "if (marg && ((isfinite(Z) && fabs(p[2] - (Z + m->p.eps_vis)) < tol_m) || (zamb && zamb[k]))) marg[i] = 1;",
     "if (marg && zamb && zamb[k]) marg[i] = 1;",
     [geo.test_visibility_flags_exactly_its_marginal_decisions]),
    ("visibility: an ambiguous z-buffer pixel not marginal",
     "|| (zamb && zamb[k]))) marg[i] = 1;", ")) marg[i] = 1;",
     [geo.test_visibility_flags_exactly_its_marginal_decisions]),
    ("visibility: every vertex flagged marginal",
     "    if (marg) marg[i] = 0;\n", "    if (marg) marg[i] = 1;\n",
     [geo.test_visibility_flags_exactly_its_marginal_decisions]),
    ("association: marginal vertices not looked for one pixel beyond the window",
     "for (int qx = px - R - 1; qx <= px + R + 1; ++qx) {", "for (int qx = px - R; qx <= px + R; ++qx) {",
     [geo.test_marginal_vertices_make_their_pixels_ties]),
    ("association: a marginal vertex makes a tie at any distance",
     "if (dist <= tau + tol && (best < 0 || dist <= sqrt(bd2) + tol)) tie[k] = 1;", "if (dist <= tau + tol) tie[k] = 1;",
     [geo.test_marginal_vertices_make_their_pixels_ties]),
    ("association: marginal vertices ignored by the tie flags",
     "if (tie && mstart) {", "if (0) {",
     [geo.test_marginal_vertices_make_their_pixels_ties]),
    ("z-buffer: every pixel of the bounding box flagged ambiguous",
     "if (near0 || near1 || near2) amb[k] = 1;", "amb[k] = 1;",
     [geo.test_zbuffer_flags_exactly_the_pixels_on_an_edge, geo.test_raster_equals_brute_force_ray_casting]),
    ("z-buffer: edge band of 1e-2 px",
     "double tol = 1e-3;\n", "double tol = 1e-2;\n",
     [geo.test_zbuffer_flags_exactly_the_pixels_on_an_edge]),
    ("z-buffer: one edge never ambiguous",
     "if (near0 || near1 || near2) amb[k] = 1;", "if (near0 || near1) amb[k] = 1;",
     [geo.test_zbuffer_flags_exactly_the_pixels_on_an_edge]),
    ("z-buffer: an edge line flagged beyond the triangle",
     "int near2 = d2 < tol && (w0 * area >= -tol * lbc * fabs(area)) && (w1 * area >= -tol * lca * fabs(area));",
     "int near2 = d2 < tol;",
     [geo.test_zbuffer_flags_exactly_the_pixels_on_an_edge]),
    ("raster-ID: a corner at the cutoff not a tie",
     "          if (fabs(dist[c] - tau) < tol) tie[k] = 1;\n", "",
     [rid.test_ties_are_flagged]),
    ("raster-ID: equidistant corners not a tie",
     "if (fabs(dist[c] - dist[e]) < tol && fmin(dist[c], dist[e]) <= tau + tol) tie[k] = 1;", ";",
     [rid.test_ties_are_flagged]),
    ("raster-ID: equidistant corners a tie beyond the cutoff too",
     "if (fabs(dist[c] - dist[e]) < tol && fmin(dist[c], dist[e]) <= tau + tol) tie[k] = 1;",
     "if (fabs(dist[c] - dist[e]) < tol) tie[k] = 1;",
     [rid.test_ties_are_flagged]),
    ("raster-ID: an ambiguous z-buffer pixel not a tie",
     "if (tie) tie[k] = zamb ? zamb[k] : 0;", "if (tie) tie[k] = 0;",
     [rid.test_ties_are_flagged]),
    ("association: a farther candidate at the cutoff makes a tie",
     "if (tie && fabs(d1 - tau) < tol) tie[k] = 1;", "if (tie && fabs(d2nd - tau) < tol) tie[k] = 1;",
     [geo.test_cutoff_ties_are_those_of_the_nearest_candidate]),
    ("association: the nearest candidate at the cutoff not a tie",
     "if (tie && fabs(d1 - tau) < tol) tie[k] = 1;", "",
     [geo.test_cutoff_ties_are_those_of_the_nearest_candidate]),
    ("frame: shape iterations without re-association (R18)",
     "    associate_pass(m, &w, depth);\n    energy[m->p.pose_iters + s]", "    energy[m->p.pose_iters + s]",
     [opt.test_frame_is_the_schedule_of_its_steps]),
    ("frame: one pose iteration fewer (R18)",
     "for (int it = 0; it < m->p.pose_iters; ++it) {\n    double E = associate_pass", "for (int it = 1; it < m->p.pose_iters; ++it) {\n    double E = associate_pass",
     [opt.test_frame_is_the_schedule_of_its_steps]),
]


def _cases(fn):
    """Every argument set a pin runs with (its parametrize values, or none)."""
    marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    if not marks:
        return [{}]
    names, values = marks[0].args[0], marks[0].args[1]
    names = [a.strip() for a in names.split(",")] if isinstance(names, str) else list(names)
    out = []
    for v in values:
        v = v.values if hasattr(v, "values") else v
        out.append(dict(zip(names, v if len(names) > 1 else (v,))))
    return out


def _build(i, name, old, new, d):
    src = open(oracle._SRC).read()
    assert src.count(old) >= 1, f"{name}: text not found in oracle.c"
    c = os.path.join(d, f"mutant{i}.c")
    so = os.path.join(d, f"mutant{i}.so")
    with open(c, "w") as f:
        f.write(src.replace(old, new, 1))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                           c, "-o", so, "-lm"])
    return c, so


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    d = str(tmp_path_factory.mktemp("oracle_mutants"))
    with cf.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        return list(ex.map(lambda a: _build(a[0], a[1][0], a[1][1], a[1][2], d), enumerate(MUTANTS)))


@contextlib.contextmanager
def _oracle_from(c, so):
    saved = (oracle._SRC, oracle._LIB, oracle._lib)
    oracle._SRC, oracle._LIB, oracle._lib = c, so, None
    try:
        yield
    finally:
        oracle._SRC, oracle._LIB, oracle._lib = saved


@pytest.mark.parametrize("i", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_a_planted_mistake_fails_a_pin(i, mutant_libs):
    name, _, _, pins = MUTANTS[i]
    c, so = mutant_libs[i]
    caught = []
    with _oracle_from(c, so):
        for pin in pins:
            for kw in _cases(pin):
                try:
                    pin(**kw)
                except Exception as e:  # an assertion of the pin, or a failure the mistake causes
                    caught.append(f"{pin.__name__}{kw}: {type(e).__name__}")
                    break
    assert caught, f"no pin caught: {name}"

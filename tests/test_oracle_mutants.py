"""The pins above are strong enough: each plausible mistake planted in a copy of
the oracle (a dropped term, a wrong sign, constant, index or operand) makes at
least one pin fail.  The mutant is compiled from a patched copy of the source
into a temporary directory; the real oracle is untouched.
"""
import os

import numpy as np
import pytest

import oracle
from tests import test_oracle_adjoint as A
from tests import test_oracle_bsdf as B
from tests import test_oracle_estimator as E
from tests import test_oracle_probe as P
from tests import test_oracle_random as R
from tests import test_oracle_shadow_grad as S
from tests import test_oracle_visibility as V


def _adjoint_fd(orc):
    A.test_adjoint_matches_central_differences(orc, A.make_frozen_case(orc))


# (what is planted, exact source text, replacement, pins expected to catch it)
MUTANTS = [
    ("philox multiplier swapped", "(uint64_t)0xD2511F53u * (uint64_t)c0", "(uint64_t)0xCD9E8D57u * (uint64_t)c0",
     [R.test_philox_matches_triton_library]),
    ("philox key bump dropped", "k1 += 0xBB67AE85u;", "k1 += 0u;", [R.test_philox_matches_triton_library]),
    ("uniform scale off by two", "(double)(x[0] >> 8)", "(double)(x[0] >> 9)", [R.test_uniforms_uniform_and_independent]),
    ("sin(theta) dropped from texel weights", "R += Y * s;", "R += Y;", [P.test_importance_is_luminance_times_solid_angle]),
    ("luminance uses one channel", "((double)t[0] + (double)t[1] + (double)t[2]) / 3.0", "(double)t[0]",
     [P.test_importance_is_luminance_times_solid_angle]),
    ("lat-long Jacobian 4 pi instead of 2 pi^2",
     "*pdf = st > 0.0 ? (W * (double)H * wr * wc) / (2.0 * ORC_PI * ORC_PI * st) : 0.0;",
     "*pdf = st > 0.0 ? (W * (double)H * wr * wc) / (4.0 * ORC_PI * st) : 0.0;",
     [lambda o: P.test_light_samples_follow_density(o)]),
    ("light pdf evaluation drops sin(theta)",
     "return st > 0.0 ? (W * (double)H * wr * wc) / (2.0 * ORC_PI * ORC_PI * st) : 0.0;",
     "return st > 0.0 ? (W * (double)H * wr * wc) / (2.0 * ORC_PI * ORC_PI) : 0.0;",
     [lambda o: P.test_light_pdf_integrates_to_one(o, 32, 16)]),
    ("azimuth operands transposed", "atan2(d[2], d[0])", "atan2(d[0], d[2])", [P.test_texel_lookup_matches_parameterisation]),
    ("cosine lift without sqrt", "sqrt(1.0 - u0)};", "(1.0 - u0)};", [lambda o: B.test_cosine_sampler_distribution(o, 3)]),
    ("frame sign term", "b2[0] = b; b2[1] = s + n[1] * n[1] * a;", "b2[0] = b; b2[1] = 1.0 + n[1] * n[1] * a;",
     [lambda o: B.test_frame_orthonormal(o, 1)]),
    ("GGX D denominator not squared", "return a2 / (ORC_PI * d * d);", "return a2 / (ORC_PI * d);",
     [lambda o: B.test_ggx_D_normalised(o, 0.4)]),
    ("Smith Lambda missing the half", "return 0.5 * (sqrt(1.0 + z) - 1.0);", "return (sqrt(1.0 + z) - 1.0);",
     [B.test_smith_G1_alpha1_closed_form]),
    ("VNDF half-disk warp sign", "double s = 0.5 * (1.0 + vh[2]);", "double s = 0.5 * (1.0 - vh[2]);",
     [lambda o: B.test_ggx_pdf_integrates_to_one_and_predicts_samples(o, 0.5, 1.1)]),
    ("GGX pdf Jacobian 1/2 instead of 1/4",
     "return orc_ggx_G1(co, alpha) * orc_ggx_D(dot3(n, h), alpha) / (4.0 * co);",
     "return orc_ggx_G1(co, alpha) * orc_ggx_D(dot3(n, h), alpha) / (2.0 * co);",
     [lambda o: B.test_ggx_pdf_integrates_to_one_and_predicts_samples(o, 0.5, 1.1)]),
    ("Fresnel exponent four", "return f0 + (1.0 - f0) * x * x * x * x * x;", "return f0 + (1.0 - f0) * x * x * x * x;",
     [B.test_schlick_spot_values]),
    ("triangle edge test drops u+v", "if (*u < 0.0 || *v < 0.0 || *u + *v > 1.0) return 0;",
     "if (*u < 0.0 || *v < 0.0 || *u > 1.0) return 0;", [V.test_ray_triangle_matches_linear_solve]),
    ("barycentrics swapped in the G-buffer normal",
     "row[4 + c] = w * vnrm[3 * (size_t)tris[3 * k] + c] + u * vnrm[3 * (size_t)tris[3 * k + 1] + c] +\n"
     "                         v * vnrm[3 * (size_t)tris[3 * k + 2] + c];",
     "row[4 + c] = w * vnrm[3 * (size_t)tris[3 * k] + c] + v * vnrm[3 * (size_t)tris[3 * k + 1] + c] +\n"
     "                         u * vnrm[3 * (size_t)tris[3 * k + 2] + c];",
     [V.test_primary_cast_interpolates_vertex_attributes]),
    ("texel-centre offset dropped", "double x = u * T - 0.5, y = v * T - 0.5;", "double x = u * T, y = v * T;",
     [V.test_bilinear_texture]),
    ("MIS drops a sample count", "nC * orc_pdf_cosine(n, wi)", "orc_pdf_cosine(n, wi)",
     [lambda o: E.test_diffuse_converges_to_closed_form(o, (4, 2, 2))]),
    ("diffuse cosine dropped", "for (int c = 0; c < 3; ++c) o[c] += L[c] * a * ci / ORC_PI;",
     "for (int c = 0; c < 3; ++c) o[c] += L[c] * a / ORC_PI;", [E.test_cosine_furnace_zero_variance]),
    ("shadow ray offset into the surface", "double so[3] = {p[0] + prm.ray_eps * n[0], p[1] + prm.ray_eps * n[1]",
     "double so[3] = {p[0] - prm.ray_eps * n[0], p[1] - prm.ray_eps * n[1]", [E.test_surface_does_not_shadow_itself]),
    ("leakage inverted", "double Hv = hit ? 1.0 - prm.tau : 1.0;", "double Hv = hit ? prm.tau : 1.0;",
     [lambda o: E.test_closed_mesh_blocks_everything(o, 0.3)]),
    ("specular cos_o missing", "o[6 + c] += L[c] * a * D * G2 * orc_schlick(F0[c], vh) / (4.0 * co);",
     "o[6 + c] += L[c] * a * D * G2 * orc_schlick(F0[c], vh) / 4.0;",
     [lambda o: E.test_specular_albedo_matches_quadrature(o, 0.25, 0.5)]),
    ("adjoint: D slope sign", "dD_dnh = -4.0 * D * nh * (a2 - 1.0) / dd;", "dD_dnh = 4.0 * D * nh * (a2 - 1.0) / dd;",
     [_adjoint_fd]),
    ("adjoint: no tangent projection of the normal grad", "out[k] = (gn[k] - A->n[k] * ng) / A->lN;",
     "out[k] = gn[k] / A->lN;",
     [_adjoint_fd]),
    ("adjoint: metallic through F0 with the wrong sign", "g_m += -gk[c] * kd[c] + gF0[c] * (kd[c] - 0.04);",
     "g_m += -gk[c] * kd[c] + gF0[c] * (0.04 - kd[c]);", [_adjoint_fd]),
    ("edge gradient: outward normal flipped", "double sg = s1 > 0.0 ? -1.0 : 1.0, nout[3], wp[3];",
     "double sg = s1 > 0.0 ? 1.0 : -1.0, nout[3], wp[3];", [lambda o: S.test_single_triangle_matches_lambert(o, 1.0)]),
    ("edge gradient: endpoint weights swapped", "g_verts[3 * (size_t)E4[0] + c] += wt * (1.0 - s) * nout[c];",
     "g_verts[3 * (size_t)E4[0] + c] += wt * s * nout[c];", [lambda o: S.test_single_triangle_matches_lambert(o, 1.0)]),
    ("edge gradient: 1/r^2 of the Jacobian dropped", "double J = norm3(wxab) / (rr * rr);",
     "double J = norm3(wxab) / rr;", [lambda o: S.test_single_triangle_matches_lambert(o, 1.0)]),
    ("edge gradient: silhouette test skipped", "if (!(s1 * s2 > 0.0)) continue;", "if (!(s1 * s1 > 0.0)) continue;",
     [S.test_quad_interior_edge_is_not_a_silhouette]),
    ("edge gradient: outer ray not checked", "if (blocked) continue;", "if (blocked && 0) continue;",
     [lambda o: S.test_hidden_occluder_edges_contribute_nothing(o, False)]),
    ("edge table: wrong opposite vertex", "edges[4 * n + 3] = tris[3 * t2 + (i2 + 2) % 3];",
     "edges[4 * n + 3] = tris[3 * t2 + (i2 + 1) % 3];", [S.test_edge_table_closed_and_open_meshes]),
    ("edge gradient: specular without cos_o", "gw += L[c] * gs[c] * D * G2 * orc_schlick(F0, vh) / (4.0 * co);",
     "gw += L[c] * gs[c] * D * G2 * orc_schlick(F0, vh) / 4.0;",
     [lambda o: S.test_matches_finite_differences_of_the_forward_estimator(o, "specular")]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pins):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site not unique/found: {name}"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = oracle.load(oracle.build(force=True, src=str(mpath), out=str(tmp_path / "libmutant.so")))
    saved = oracle._lib
    oracle._lib = lib
    caught = False
    try:
        for pin in pins:
            try:
                pin(oracle)
            except (AssertionError, FloatingPointError, ValueError, np.linalg.LinAlgError):
                caught = True
    finally:
        oracle._lib = saved
    assert caught, f"no pin caught: {name}"

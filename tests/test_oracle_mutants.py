"""The oracle's pins catch plausible mistakes in it.

Each mutant below is a copy of the oracle package (``oracle/gs_oracle.c`` and
``oracle/__init__.py``) with one slip planted in it: a flipped sign, a dropped
term, a transposed operand, a wrong index or constant, a cut-off tested on the
wrong side.  The copy is built in a temporary directory and the oracle's own
pin tests (closed forms, invariants, independent library routines, brute
force, finite differences) are run against it in a child process.  Every
mutant must make at least one pin fail; the unmodified copy must pass them
all, so a failure comes from the planted slip and not from the harness.
Nothing here touches the CUDA library.
"""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_FILES = {"c": "gs_oracle.c", "py": "__init__.py"}
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_grad_fd.py", "tests/test_oracle_depth.py",
             "tests/test_oracle_pose.py"]

# (name, exact text in gs_oracle.c, replacement).  Each text occurs exactly once.
C_MUTANTS = [
    # rotation and covariance (App. E, gradient-flow figure)
    ("rotation_sign", "R[1] = 2.0 * (x * y - w * z);", "R[1] = 2.0 * (x * y + w * z);"),
    ("rotation_index", "R[7] = 2.0 * (y * z + w * x);", "R[7] = 2.0 * (x * z + w * x);"),
    ("covariance_transposed", "matmul(g->M, Mt, g->Sig, 3, 3, 3);", "matmul(Mt, g->M, g->Sig, 3, 3, 3);"),
    ("scale_not_activated", "g->s[i] = exp(log_scale[i]);", "g->s[i] = log_scale[i];"),
    ("opacity_not_activated", "g->o = sigmoid(logit);", "g->o = logit;"),
    ("quat_not_normalised", "g->qh[i] = quat[i] / g->qn;", "g->qh[i] = quat[i];"),
    # projection (App. C.1, App. E)
    ("focal_x_for_y", "sp->mu2[1] = fy * ty / tz + cy;", "sp->mu2[1] = fx * ty / tz + cy;"),
    ("principal_point_swapped", "sp->mu2[0] = fx * tx / tz + cx;", "sp->mu2[0] = fx * tx / tz + cy;"),
    ("jacobian_sign", "sp->J[2] = -fx * tx / (tz * tz);", "sp->J[2] = fx * tx / (tz * tz);"),
    ("jacobian_power", "sp->J[5] = -fy * ty / (tz * tz);", "sp->J[5] = -fy * ty / tz;"),
    ("view_rotation_transposed", "matmul(sp->J, Wr, sp->T, 2, 3, 3);",
     "double Wq[9]; transpose(Wr, Wq, 3, 3); matmul(sp->J, Wq, sp->T, 2, 3, 3);"),
    ("lowpass_dropped", "sp->cov[2] = sp->cov0[2] + eps2d;", "sp->cov[2] = sp->cov0[2];"),
    ("conic_offdiag_sign", "sp->conic[1] = -sp->cov[1] / det;", "sp->conic[1] = sp->cov[1] / det;"),
    ("conic_diag_swapped", "sp->conic[0] = sp->cov[2] / det;", "sp->conic[0] = sp->cov[0] / det;"),
    ("lambda_min_for_max", "double lam = m + sqrt(disc > 0.0 ? disc : 0.0);",
     "double lam = m - sqrt(disc > 0.0 ? disc : 0.0);"),
    ("radius_two_sigma", "double rr = ceil(3.0 * sqrt(lam));", "double rr = ceil(2.0 * sqrt(lam));"),
    ("radius_cap_raised", "if (!(rr > 0.0) || rr > 1.0e7) return;", "if (!(rr > 0.0) || rr > 1.0e9) return;"),
    ("pixel_box_centre", "double x0 = ceil(mx - (double)r - 0.5), x1 = floor(mx + (double)r - 0.5);",
     "double x0 = ceil(mx - (double)r), x1 = floor(mx + (double)r);"),
    ("near_plane_ignored", "if (!(tz >= near_plane)) return; /* culled */", "if (!(tz > 0.0)) return;"),
    ("antialias_no_sqrt", "sp->comp = sqrt(ratio > 0.0 ? ratio : 0.0);", "sp->comp = ratio > 0.0 ? ratio : 0.0;"),
    # spherical harmonics (App. C.1)
    ("sh_deg1_sign", "Y[1] = -k1 * y;", "Y[1] = k1 * y;"),
    ("sh_deg2_sign", "Y[5] = -k2a * y * z;", "Y[5] = k2a * y * z;"),
    ("sh_deg2_constant", "const double k2b = 0.25 * sqrt(5.0 / pi);  /* m = 0 */",
     "const double k2b = 0.5 * sqrt(5.0 / pi);  /* m = 0 */"),
    ("sh_deg3_index", "Y[13] = -k3c * x * (4.0 * z * z - x * x - y * y);",
     "Y[13] = -k3c * y * (4.0 * z * z - x * x - y * y);"),
    ("sh_deg3_term", "Y[12] = k3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);",
     "Y[12] = k3d * z * (2.0 * z * z - 3.0 * x * x - y * y);"),
    ("sh_offset_dropped", "            s += 0.5;\n            raw[3 * n + ch] = s;", "            raw[3 * n + ch] = s;"),
    ("sh_no_clamp", "colors[3 * n + ch] = s > 0.0 ? s : 0.0;", "colors[3 * n + ch] = s;"),
    ("camera_centre_transposed", "c[i] = -(vm[0 + i] * vm[3] + vm[4 + i] * vm[7] + vm[8 + i] * vm[11]);",
     "c[i] = -(vm[4 * i] * vm[3] + vm[4 * i + 1] * vm[7] + vm[4 * i + 2] * vm[11]);"),
    ("sh_grad_constant", "dY[3 * 6 + 2] = 4.0 * k2b * z;", "dY[3 * 6 + 2] = 2.0 * k2b * z;"),
    ("sh_grad_deg3_term", "dY[3 * 11 + 1] = -k3c * (4.0 * z * z - x * x - 3.0 * y * y);",
     "dY[3 * 11 + 1] = -k3c * (4.0 * z * z - x * x - y * y);"),
    ("sh_bwd_clamp_mask_dropped", "g[ch] = s > 0.0 ? d_colors[3 * n + ch] : 0.0;", "g[ch] = d_colors[3 * n + ch];"),
    ("sh_bwd_direction_projection_dropped", "dv[i] = (ddir[i] - dir[i] * dd) / len;", "dv[i] = ddir[i] / len;"),
    ("sh_deg2_xy_sign", "Y[4] = k2a * x * y;", "Y[4] = -k2a * x * y;"),
    ("sh_deg2_m0_term", "Y[6] = k2b * (2.0 * z * z - x * x - y * y);", "Y[6] = k2b * (2.0 * z * z - x * x + y * y);"),
    ("sh_deg2_xz_index", "Y[7] = -k2a * x * z;", "Y[7] = -k2a * y * z;"),
    ("sh_deg2_m2_sign", "Y[8] = k2c * (x * x - y * y);", "Y[8] = k2c * (y * y - x * x);"),
    ("sh_deg3_m_minus3_term", "Y[9] = -k3a * y * (3.0 * x * x - y * y);", "Y[9] = -k3a * y * (x * x - y * y);"),
    ("sh_deg3_xyz_constant", "Y[10] = k3b * x * y * z;", "Y[10] = k3e * x * y * z;"),
    ("sh_deg3_m_minus1_index", "Y[11] = -k3c * y * (4.0 * z * z - x * x - y * y);",
     "Y[11] = -k3c * x * (4.0 * z * z - x * x - y * y);"),
    ("sh_deg3_m2_index", "Y[14] = k3e * z * (x * x - y * y);", "Y[14] = k3e * y * (x * x - y * y);"),
    ("sh_deg3_m3_term", "Y[15] = -k3a * x * (x * x - 3.0 * y * y);", "Y[15] = -k3a * x * (x * x - y * y);"),
    ("sh_grad_deg2_index", "dY[3 * 4 + 0] = k2a * y;", "dY[3 * 4 + 0] = k2a * x;"),
    ("sh_grad_deg3_factor", "dY[3 * 9 + 0] = -k3a * 6.0 * x * y;", "dY[3 * 9 + 0] = -k3a * 3.0 * x * y;"),
    ("sh_grad_deg3_last", "dY[3 * 15 + 1] = -k3a * (-6.0 * x * y);", "dY[3 * 15 + 1] = -k3a * (-3.0 * x * y);"),
    ("sh_grad_deg3_m2_z", "dY[3 * 14 + 2] = k3e * (x * x - y * y);", "dY[3 * 14 + 2] = k3e * (x * x + y * y);"),
    ("sh_bwd_projection_sign", "double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];",
     "double dd = -(dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2]);"),
    # compositing (App. C.2)
    ("depth_order_reversed", "if (da < db) return -1;\n    if (da > db) return 1;",
     "if (da > db) return -1;\n    if (da < db) return 1;"),
    ("sigma_offdiag_doubled", "double sigma = 0.5 * (Y[0] * dx * dx + Y[2] * dy * dy) + Y[1] * dx * dy;",
     "double sigma = 0.5 * (Y[0] * dx * dx + Y[2] * dy * dy) + 2.0 * Y[1] * dx * dy;"),
    ("pixel_centre_dropped", "double pxc = px + 0.5, pyc = py + 0.5;", "double pxc = px, pyc = py;"),
    ("alpha_not_clamped", "if (a > alpha_max) { a = alpha_max; clamped = 1; }", "if (a > 1.0) { a = 1.0; clamped = 1; }"),
    ("alpha_skip_stops", "if (a < alpha_min) continue;", "if (a < alpha_min) break;"),
    ("cutoff_includes_last", "if (Tn < T_min) break; /* excluded; the pixel is finished */",
     "if (T < T_min) break;"),
    ("weight_uses_next_T", "out_col[c] += colors[(size_t)n * ch + c] * a * T;",
     "out_col[c] += colors[(size_t)n * ch + c] * a * Tn;"),
    ("channels_stride_three", "for (int c = 0; c < ch; c++) out_col[c] += colors[(size_t)n * ch + c] * a * T;",
     "for (int c = 0; c < ch; c++) out_col[c] += colors[(size_t)n * 3 + c] * a * T;"),
    ("background_not_weighted", "out_col[c] += T * (bg ? bg[c] : 0.0);", "out_col[c] += (bg ? bg[c] : 0.0);"),
    ("depth_ties_descending_in_compositing", "return (ia > ib) - (ia < ib);", "return (ia < ib) - (ia > ib);"),
    # compositing backward (App. D.2)
    ("bwd_suffix_dropped", "da += g[c] * (cn[c] * T - S[c] / (1.0 - a));", "da += g[c] * (cn[c] * T);"),
    ("bwd_suffix_not_updated", "for (int c = 0; c < ch; c++) S[c] += cn[c] * a * T;", ";"),
    ("bwd_background_dropped", "S[c] = Tf * (bg ? bg[c] : 0.0);", "S[c] = 0.0;"),
    ("bwd_alpha_output_dropped", "da += gA * Tf / (1.0 - a);", ";"),
    ("bwd_clamp_passes_gradient", "if (e->clamped) da = 0.0;", ";"),
    ("bwd_mean_sign", "double gx = -d_sigma * (Y[0] * e->dx + Y[1] * e->dy);",
     "double gx = d_sigma * (Y[0] * e->dx + Y[1] * e->dy);"),
    ("bwd_conic_offdiag_halved", "atomic_add(&d_conics[3 * n + 1], d_sigma * e->dx * e->dy);",
     "atomic_add(&d_conics[3 * n + 1], 0.5 * d_sigma * e->dx * e->dy);"),
    ("bwd_color_weight", "atomic_add(&d_colors[(size_t)n * ch + c], a * T * g[c]);",
     "atomic_add(&d_colors[(size_t)n * ch + c], a * g[c]);"),
    ("bwd_absgrad_signed", "atomic_add(&absgrad[2 * n], fabs(gx));", "atomic_add(&absgrad[2 * n], gx);"),
    ("bwd_opacity_factor", "double d_o = e->G * da;", "double d_o = da;"),
    ("bwd_sigma_opacity_dropped", "double d_sigma = -opac[n] * e->G * da;", "double d_sigma = -e->G * da;"),
    # projection backward (App. D.3, D.4)
    ("bwd_inverse_sign", "for (int i = 0; i < 4; i++) G2[i] = -G2[i];", ";"),
    ("bwd_conic_offdiag_not_split", "double dYm[4] = {d_conics[3 * n], 0.5 * d_conics[3 * n + 1], 0.5 * d_conics[3 * n + 1],",
     "double dYm[4] = {d_conics[3 * n], d_conics[3 * n + 1], d_conics[3 * n + 1],"),
    ("bwd_dT_second_term_dropped", "for (int i = 0; i < 6; i++) dT[i] += tmp[i];", ";"),
    ("bwd_jacobian_tz_term", "dt[2] += dJ[0] * (-fx / tz2) + dJ[2] * (2.0 * fx * tx / tz3)",
     "dt[2] += dJ[0] * (-fx / tz2) + dJ[2] * (fx * tx / tz3)"),
    ("bwd_mean2d_tz_sign", "dt[2] += -gmx * fx * tx / tz2 - gmy * fy * ty / tz2;",
     "dt[2] += -gmx * fx * tx / tz2 + gmy * fy * ty / tz2;"),
    ("bwd_view_rotation_not_transposed",
     "d_means[3 * n + i] += Wr[0 + i] * dt[0] + Wr[3 + i] * dt[1] + Wr[6 + i] * dt[2];",
     "d_means[3 * n + i] += Wr[3 * i] * dt[0] + Wr[3 * i + 1] * dt[1] + Wr[3 * i + 2] * dt[2];"),
    ("bwd_depth_sign", "if (d_depths) dt[2] += d_depths[n];", "if (d_depths) dt[2] -= d_depths[n];"),
    ("bwd_dM_second_term_dropped", "for (int i = 0; i < 9; i++) dM[i] += t2[i];", ";"),
    ("bwd_scale_chain_dropped", "d_log_scales[3 * n + j] += dsj * g.s[j];", "d_log_scales[3 * n + j] += dsj;"),
    ("bwd_quat_normalisation_dropped", "d_quats[4 * n + k2] += (dqh[k2] - g.qh[k2] * proj) / g.qn;",
     "d_quats[4 * n + k2] += dqh[k2] / g.qn;"),
    ("bwd_sigmoid_chain", "d_logits[n] += d_o * g.o * (1.0 - g.o);", "d_logits[n] += d_o * g.o;"),
    ("drot_sign", "double Dw[9] = {0, -z, y, z, 0, -x, -y, x, 0};", "double Dw[9] = {0, z, y, z, 0, -x, -y, x, 0};"),
    ("bwd_antialias_term_sign", "double gb = k * (-2.0 * b * det1 + 2.0 * b * det0);",
     "double gb = k * (-2.0 * b * det1 - 2.0 * b * det0);"),
    ("bwd_antialias_compensation_dropped", "double d_o = d_oeff * sp.comp;", "double d_o = d_oeff;"),
    ("antialias_det_sign", "double det0 = sp->cov0[0] * sp->cov0[2] - sp->cov0[1] * sp->cov0[1];",
     "double det0 = sp->cov0[0] * sp->cov0[2] + sp->cov0[1] * sp->cov0[1];"),
    ("bwd_antialias_c_entry", "double gc = k * (a * det1 - det0 * sp.cov[0]);",
     "double gc = k * (a * det1 - det0 * sp.cov[2]);"),
    ("bwd_mean2d_y_focal", "dt[1] += gmy * fy / tz;", "dt[1] += gmy * fx / tz;"),
    ("bwd_jacobian_x_term_sign", "dt[0] += dJ[2] * (-fx / tz2);", "dt[0] += dJ[2] * (fx / tz2);"),
    ("bwd_dM_transposed", "matmul(dSig, g.M, dM, 3, 3, 3);", "matmul(g.M, dSig, dM, 3, 3, 3);"),
    ("bwd_scale_rotation_transposed", "for (int i = 0; i < 3; i++) dsj += g.R[i * 3 + j] * dM[i * 3 + j];",
     "for (int i = 0; i < 3; i++) dsj += g.R[j * 3 + i] * dM[i * 3 + j];"),
    # pose gradients (App. A)
    ("pose_sh_centre_index", "d_viewmat[4 * i + j] += viewmat[4 * i + 3] * dv[j];",
     "d_viewmat[4 * i + j] += viewmat[4 * j + 3] * dv[i];"),
    ("pose_mean_outer_transposed", "double v = dRw[3 * i + j] + dt[i] * means[3 * n + j];",
     "double v = dRw[3 * i + j] + dt[j] * means[3 * n + i];"),
    ("pose_translation_dropped", "d_viewmat[4 * i + 3] += dt[i];", "d_viewmat[4 * i + 3] += 0.0;"),
    ("camera_translation_dropped",
     "sp->t[i] = Wr[i * 3 + 0] * mean[0] + Wr[i * 3 + 1] * mean[1] + Wr[i * 3 + 2] * mean[2] + tw[i];",
     "sp->t[i] = Wr[i * 3 + 0] * mean[0] + Wr[i * 3 + 1] * mean[1] + Wr[i * 3 + 2] * mean[2];"),
    ("antialias_not_applied", "sp->opac = g->o * sp->comp;", "sp->opac = g->o;"),
    ("bwd_antialias_half_dropped", "double k = dcomp / (2.0 * sp.comp) / (det1 * det1);",
     "double k = dcomp / sp.comp / (det1 * det1);"),
    ("bwd_antialias_wrong_entry", "double ga = k * (c * det1 - det0 * sp.cov[2]);",
     "double ga = k * (c * det1 - det0 * sp.cov[0]);"),
    ("pose_sh_rotation_transposed",
     "double r = viewmat[4 * i] * dv[0] + viewmat[4 * i + 1] * dv[1] + viewmat[4 * i + 2] * dv[2];",
     "double r = viewmat[i] * dv[0] + viewmat[4 + i] * dv[1] + viewmat[8 + i] * dv[2];"),
    ("pose_jacobian_transposed", "matmul(Jt, dT, dRw, 3, 2, 3);", "matmul(Jt, dT, dRw, 3, 2, 3);\n"
     "            for (int i = 0; i < 3; i++) for (int j = 0; j < i; j++) { double u = dRw[3 * i + j]; "
     "dRw[3 * i + j] = dRw[3 * j + i]; dRw[3 * j + i] = u; }"),
    # binning and sorting (App. C.2)
    ("bins_last_row_dropped", "for (int ty = box[2] / tile; ty <= box[3] / tile; ty++)",
     "for (int ty = box[2] / tile; ty < box[3] / tile; ty++)"),
    ("bins_ties_descending", "return (x->value > y->value) - (x->value < y->value);",
     "return (x->value < y->value) - (x->value > y->value);"),
    ("ranges_start_off_by_one", "if (j == 0 || (buf[j - 1].key >> 32) != (uint64_t)t) ranges[2 * t] = (int32_t)j;",
     "if (j == 0 || (buf[j - 1].key >> 32) != (uint64_t)t) ranges[2 * t] = (int32_t)(j + 1);"),
    ("bins_tile_row_stride", "uint64_t gt = (uint64_t)(offs[c] + ty * tiles_x + tx);",
     "uint64_t gt = (uint64_t)(offs[c] + ty * (tiles_x - 1) + tx);"),
    ("bins_depth_as_integer", "buf[k].key = (gt << 32) | (uint64_t)f32_bits(depths[i]);",
     "buf[k].key = (gt << 32) | (uint64_t)(uint32_t)depths[i];"),
]

# (name, exact text in oracle/__init__.py, replacement): the whole-pipeline and depth chains
PY_MUTANTS = [
    ("camera_fx_for_fy", "_d64([cam.fx, cam.fy, cam.cx, cam.cy])", "_d64([cam.fx, cam.fx, cam.cx, cam.cy])"),
    ("pipeline_sh_mean_term_dropped",
     'd_sh, d_means_sh = sh_bwd(scene, cam, g2["d_colors"], d_viewmat=d_view)\n',
     'd_sh, d_means_sh = sh_bwd(scene, cam, g2["d_colors"], d_viewmat=d_view)\n    d_means_sh = 0.0 * d_means_sh\n'),
    ("expected_depth_not_normalised", "expected = np.where(a > 0.0, acc / np.where(a > 0.0, a, 1.0), 0.0)",
     "expected = acc"),
    ("expected_depth_grad_alpha_sign", 'gA += -dE * f["expected_depth"] * inv', 'gA += dE * f["expected_depth"] * inv'),
    ("expected_depth_grad_not_scaled", "g4[:, 3] += dE * inv", "g4[:, 3] += dE"),
    ("near_plane_float64_literal", "NEAR = _f32(0.01)", "NEAR = 0.01"),
    ("alpha_cap_float64_literal", "ALPHA_MAX = _f32(0.99)", "ALPHA_MAX = 0.99"),
    ("depth_grad_sign", 'd_depths=g2["d_colors"][:, 3]', 'd_depths=-g2["d_colors"][:, 3]'),
]

MUTANTS = [("c", *m) for m in C_MUTANTS] + [("py", *m) for m in PY_MUTANTS]

# imports the oracle copy first, so the pin modules' ``import oracle`` find it in sys.modules
_RUNNER = r"""
import sys
sys.path.insert(0, sys.argv[1])
import oracle
assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", *sys.argv[2:]]))
"""


def _run_pins(files, workdir):
    pkg = os.path.join(workdir, "oracle")
    os.makedirs(pkg, exist_ok=True)
    for fname, text in files.items():
        with open(os.path.join(pkg, fname), "w") as f:
            f.write(text)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", _RUNNER, workdir, *PIN_FILES], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    lines = (r.stdout + r.stderr).strip().splitlines()
    return r.returncode, "\n".join(lines[-12:])


@pytest.fixture(scope="module")
def outcomes():
    original = {}
    for fname in ORACLE_FILES.values():
        with open(os.path.join(ROOT, "oracle", fname)) as f:
            original[fname] = f.read()
    jobs = {"unmodified": dict(original)}
    for kind, name, old, new in MUTANTS:
        fname = ORACLE_FILES[kind]
        assert original[fname].count(old) == 1, f"{name}: the mutated text must occur exactly once in {fname}"
        jobs[name] = dict(original, **{fname: original[fname].replace(old, new)})
    with tempfile.TemporaryDirectory() as tmp, ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as pool:
        futs = {name: pool.submit(_run_pins, files, os.path.join(tmp, name)) for name, files in jobs.items()}
        return {name: fut.result() for name, fut in futs.items()}


def test_unmodified_copy_passes_every_pin(outcomes):
    rc, tail = outcomes["unmodified"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[1] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    # pytest's exit status 1 = some test failed (a crash or a build error would be another status)
    assert rc == 1, f"mutant {name} was not caught (exit {rc}):\n{tail}"

"""FP64 central finite differences against the oracle's analytic backward (App. D).

The forward oracle is differentiated numerically, coordinate by coordinate, on
tiny scenes; coordinates where a discrete decision (radius, pixel box, alpha
skip, transmittance cut-off) changes within +-h are skipped and counted.  The
pieces are also checked in isolation: compositing w.r.t. 2D splat data,
projection w.r.t. the 3D leaves and SH colour w.r.t. its coefficients and the
mean (through the view direction).
"""
import numpy as np
import pytest

import oracle
from paper_2409_06765_gb300 import synth


def _f64_scene(sc):
    f = lambda a: np.array(a, dtype=np.float64, copy=True)
    return synth.Scene(f(sc.means), f(sc.quats), f(sc.log_scales), f(sc.opacity_logits), f(sc.sh), sc.sh_degree)


def _signature(r):
    sp = r["splats"]
    return (sp["radii"].tobytes(), sp["boxes"].tobytes(), r["ncontrib"].tobytes(), r["blends"].tobytes())


def _loss(r, w, wA):
    P = w.shape[0]
    return float((r["image"].reshape(P, -1) * w).sum() + (r["alpha"].reshape(P) * wA).sum())


FIELDS = ["means", "quats", "log_scales", "opacity_logits", "sh"]
GRAD = {"means": "d_means", "quats": "d_quats", "log_scales": "d_log_scales",
        "opacity_logits": "d_opacity_logits", "sh": "d_sh"}


@pytest.mark.parametrize("seed,deg,aa,bg", [(0, 0, False, None), (1, 1, False, (0.2, 0.4, 0.1)),
                                            (2, 3, False, None), (3, 3, True, (0.3, 0.0, 0.6))])
def test_full_pipeline_gradients_match_finite_differences(seed, deg, aa, bg):
    sc0, cam = synth.random_small_scene(9, seed=seed, sh_degree=deg, width=22, height=18,
                                        log_scale_mu=-1.7, spread=0.6)
    sc = _f64_scene(sc0)
    rng = np.random.default_rng(100 + seed)
    P = cam.width * cam.height
    w = rng.normal(size=(P, 3))
    wA = rng.normal(size=P)
    bgv = None if bg is None else np.array(bg)
    g = oracle.render_grads(sc, cam, w, d_alpha=wA, bg=bgv, antialiased=aa)
    base = oracle.render(sc, cam, bg=bgv, antialiased=aa)
    sig0 = _signature(base)
    assert base["ncontrib"].sum() > 50, "scene too empty to test anything"
    h = 1e-6
    checked = skipped = 0
    for name in FIELDS:
        arr = getattr(sc, name)
        ana = g[GRAD[name]].reshape(-1)
        flat = arr.reshape(-1)
        scale = np.abs(ana).max() + 1e-12
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            rp = oracle.render(sc, cam, bg=bgv, antialiased=aa)
            flat[i] = old - h
            rm = oracle.render(sc, cam, bg=bgv, antialiased=aa)
            flat[i] = old
            if _signature(rp) != sig0 or _signature(rm) != sig0:
                skipped += 1
                continue
            fd = (_loss(rp, w, wA) - _loss(rm, w, wA)) / (2 * h)
            assert abs(fd - ana[i]) <= 1e-5 * abs(fd) + 2e-6 * scale, (name, i, fd, ana[i])
            checked += 1
    assert checked > 0.9 * (checked + skipped)


def test_compositing_gradients_wrt_splat_data():
    sc0, cam = synth.random_small_scene(12, seed=21, sh_degree=0, width=20, height=16, log_scale_mu=-1.5)
    sp = oracle.project(_f64_scene(sc0), cam)
    W, H = cam.width, cam.height
    rng = np.random.default_rng(22)
    ch = 4  # an N-D feature vector (App. C: c may be any N-dimensional vector)
    colors = rng.uniform(0, 1, (sc0.n, ch))
    bg = rng.uniform(0, 1, ch)
    P = W * H
    w = rng.normal(size=(P, ch))
    wA = rng.normal(size=P)
    ana = oracle.render_splats_bwd(sp, colors, W, H, w, d_alpha=wA, bg=bg)

    def L(s, c):
        r = oracle.render_splats(s, c, W, H, bg=bg)
        return float((r["color"] * w).sum() + ((1 - r["T"]) * wA).sum()), (r["ncontrib"].tobytes(),
                                                                          r["blends"].tobytes())
    _, sig0 = L(sp, colors)
    h = 1e-7
    n_ok = 0
    for key, gkey in [("means2d", "d_means2d"), ("conics", "d_conics"), ("opacities", "d_opacities")]:
        arr = sp[key].reshape(-1)
        for i in range(arr.size):
            old = arr[i]
            arr[i] = old + h
            lp, sp_sig = L(sp, colors)
            arr[i] = old - h
            lm, sm_sig = L(sp, colors)
            arr[i] = old
            if sp_sig != sig0 or sm_sig != sig0:
                continue
            fd = (lp - lm) / (2 * h)
            a = ana[gkey].reshape(-1)[i]
            assert abs(fd - a) <= 1e-5 * abs(fd) + 1e-6, (key, i, fd, a)
            n_ok += 1
    flat = colors.reshape(-1)
    for i in range(flat.size):
        old = flat[i]
        flat[i] = old + h
        lp, _ = L(sp, colors)
        flat[i] = old - h
        lm, _ = L(sp, colors)
        flat[i] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - ana["d_colors"].reshape(-1)[i]) <= 1e-5 * abs(fd) + 1e-6
    assert n_ok > 30


def test_projection_gradients_wrt_leaves():
    """Projection alone: random upstream weights on (mu', conic, opacity, depth)."""
    sc0, cam = synth.random_small_scene(6, seed=31, width=30, height=30, log_scale_mu=-1.8)
    sc = _f64_scene(sc0)
    rng = np.random.default_rng(32)
    N = sc.n
    wm, wc, wo, wd = rng.normal(size=(N, 2)), rng.normal(size=(N, 3)), rng.normal(size=N), rng.normal(size=N)
    # also a camera with fx != fy and cx != cy, so that every x and y term has its own intrinsics
    cam2 = synth.Camera(cam.width, cam.height, cam.viewmat, cam.fx * 1.3, cam.fy * 0.8, cam.cx + 2.0, cam.cy - 1.5)
    for aa, cam in [(False, cam), (True, cam), (False, cam2), (True, cam2)]:
        ana = oracle.project_bwd(sc, cam, wm, wc, wo, d_depths=wd, antialiased=aa)

        def L():
            p = oracle.project(sc, cam, antialiased=aa)
            vis = p["radii"] > 0
            return float(((p["means2d"] * wm).sum(1) + (p["conics"] * wc).sum(1) + p["opacities"] * wo +
                          p["depths"] * wd)[vis].sum())
        h = 1e-6
        for name, gk in [("means", "d_means"), ("quats", "d_quats"), ("log_scales", "d_log_scales"),
                         ("opacity_logits", "d_opacity_logits")]:
            flat = getattr(sc, name).reshape(-1)
            for i in range(flat.size):
                old = flat[i]
                flat[i] = old + h
                lp = L()
                flat[i] = old - h
                lm = L()
                flat[i] = old
                fd = (lp - lm) / (2 * h)
                a = ana[gk].reshape(-1)[i]
                assert abs(fd - a) <= 1e-6 * abs(fd) + 1e-6, (aa, name, i, fd, a)


def test_sh_gradients_wrt_coefficients_and_mean():
    sc0, cam = synth.random_small_scene(5, seed=41, sh_degree=3)
    sc = _f64_scene(sc0)
    rng = np.random.default_rng(42)
    wcol = rng.normal(size=(sc.n, 3))
    d_sh, d_means = oracle.sh_bwd(sc, cam, wcol)
    h = 1e-6
    for name, ana in [("sh", d_sh), ("means", d_means)]:
        flat = getattr(sc, name).reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            lp = float((oracle.sh_colors(sc, cam)[0] * wcol).sum())
            flat[i] = old - h
            lm = float((oracle.sh_colors(sc, cam)[0] * wcol).sum())
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - ana.reshape(-1)[i]) <= 1e-6 * abs(fd) + 1e-7, (name, i)


def test_jacobian_of_J_matches_printed_derivatives():
    """App. D.3 prints dJ/dt for J = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]]."""
    fx, fy = 300.0, 250.0
    t = np.array([0.3, -0.2, 2.5])

    def J(tt):
        return np.array([[fx / tt[2], 0, -fx * tt[0] / tt[2] ** 2], [0, fy / tt[2], -fy * tt[1] / tt[2] ** 2]])
    tx, ty, tz = t
    printed = [np.array([[0, 0, -fx / tz ** 2], [0, 0, 0]]),
               np.array([[0, 0, 0], [0, 0, -fy / tz ** 2]]),
               np.array([[-fx / tz ** 2, 0, 2 * fx * tx / tz ** 3], [0, -fy / tz ** 2, 2 * fy * ty / tz ** 3]])]
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        np.testing.assert_allclose((J(t + e) - J(t - e)) / (2 * h), printed[k], atol=1e-6)


def test_suffix_recurrence_equals_direct_sum():
    """App. D.2: dC/dalpha_n = c_n T_n - S_n/(1 - alpha_n) equals the derivative of the sum."""
    rng = np.random.default_rng(9)
    n = 7
    a = rng.uniform(0.05, 0.8, n)
    c = rng.uniform(0, 1, n)

    def C(al):
        T, s = 1.0, 0.0
        for k in range(n):
            s += c[k] * al[k] * T
            T *= 1 - al[k]
        return s
    T = np.concatenate([[1.0], np.cumprod(1 - a)[:-1]])
    S = np.array([sum(c[m] * a[m] * T[m] for m in range(k + 1, n)) for k in range(n)])
    rec = c * T - S / (1 - a)
    h = 1e-7
    fd = np.array([(C(a + h * np.eye(n)[k]) - C(a - h * np.eye(n)[k])) / (2 * h) for k in range(n)])
    np.testing.assert_allclose(rec, fd, atol=1e-8)

"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties one part of the oracle to a closed form, an invariant, an
independent library routine or brute force, so that a dropped term, a wrong
sign or index or a transposed operand in gs_oracle.c fails at least one of
them.  No test here needs a GPU.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2409_06765_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene(means, quats, log_scales, logits, sh, deg=0):
    f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return synth.Scene(f(means), f(quats), f(log_scales), f(logits), f(sh), deg)


def _axis_cam(d=4.0, f=64.0, W=64, H=64, cx=32.0, cy=32.0):
    return synth.make_camera(W, H, eye=(0.0, 0.0, d), f=f, cx=cx, cy=cy)


def _identity_cam(W, H, f, cx, cy):
    return synth.Camera(W, H, np.eye(4, dtype=np.float32), f, f, cx, cy)


# --------------------------------------------------------------------------- #
# rotation (App. E) and its derivative (App. D.4)                              #
# --------------------------------------------------------------------------- #

def _rodrigues(axis, angle):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) * math.cos(angle) + math.sin(angle) * K + (1 - math.cos(angle)) * np.outer(a, a)


@pytest.mark.parametrize("seed", range(5))
def test_rotation_matches_axis_angle(seed):
    rng = np.random.default_rng(seed)
    axis = rng.normal(size=3)
    angle = rng.uniform(-math.pi, math.pi)
    a = axis / np.linalg.norm(axis)
    q = np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * a])
    R = oracle.rotation(q * 3.7)  # the oracle normalises
    np.testing.assert_allclose(R, _rodrigues(axis, angle), atol=1e-13)
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
    assert abs(np.linalg.det(R) - 1.0) < 1e-13
    np.testing.assert_allclose(oracle.rotation(-q), R, atol=1e-13)


def test_rotation_derivative_matches_finite_differences():
    rng = np.random.default_rng(7)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    D = oracle.drot_dquat(q)

    def rot_unnormalised(qq):  # R as the polynomial of App. E, no normalisation
        w, x, y, z = qq
        return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                         [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                         [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    # the closed-form polynomial and the oracle agree at unit quaternions
    np.testing.assert_allclose(rot_unnormalised(q), oracle.rotation(q), atol=1e-14)
    h = 1e-6
    for k in range(4):
        e = np.zeros(4)
        e[k] = h
        fd = (rot_unnormalised(q + e) - rot_unnormalised(q - e)) / (2 * h)
        np.testing.assert_allclose(D[k], fd, atol=1e-8)


def test_covariance_is_R_S2_Rt():
    rng = np.random.default_rng(3)
    axis, angle = rng.normal(size=3), 0.7
    a = axis / np.linalg.norm(axis)
    q = np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * a])
    ls = np.array([-1.0, 0.2, 0.5])
    R = _rodrigues(axis, angle)
    expect = R @ np.diag(np.exp(2 * ls)) @ R.T
    np.testing.assert_allclose(oracle.cov3d(q, ls), expect, atol=1e-12)


# --------------------------------------------------------------------------- #
# projection: closed forms (App. C.1, App. E, App. A)                          #
# --------------------------------------------------------------------------- #

def test_isotropic_on_axis_closed_form():
    s, d, f = math.exp(-3.0), 4.0, 64.0
    sc = _scene([[0, 0, 0]], [[1, 0, 0, 0]], [[-3.0] * 3], [0.3], np.zeros((1, 1, 3)))
    p = oracle.project(sc, _axis_cam(d=d, f=f))
    v = (f * s / d) ** 2 + oracle.EPS2D
    np.testing.assert_allclose(p["means2d"][0], [32.0, 32.0], atol=1e-12)
    np.testing.assert_allclose(p["depths"][0], d, atol=1e-12)
    np.testing.assert_allclose(p["cov2d"][0], [v, 0.0, v], atol=1e-12)
    np.testing.assert_allclose(p["conics"][0], [1 / v, 0.0, 1 / v], atol=1e-12)
    assert p["radii"][0] == math.ceil(3 * math.sqrt(v))
    np.testing.assert_allclose(p["opacities"][0], 1 / (1 + math.exp(-0.3)), atol=1e-15)


def test_off_axis_isotropic_closed_form():
    # camera = identity pose, Gaussian at (x, y, z): mu' = f (x, y)/z + c and
    # Sigma' = s^2 J J^T = s^2 f^2/z^2 [[1 + x^2/z^2, xy/z^2], [xy/z^2, 1 + y^2/z^2]]
    x, y, z, s, f = 0.4, -0.3, 2.5, 0.05, 50.0
    sc = _scene([[x, y, z]], [[1, 0, 0, 0]], [[math.log(s)] * 3], [0.0], np.zeros((1, 1, 3)))
    cam = _identity_cam(64, 48, f, 30.0, 20.0)
    p = oracle.project(sc, cam)
    np.testing.assert_allclose(p["means2d"][0], [f * x / z + 30.0, f * y / z + 20.0], atol=1e-12)
    k = s * s * f * f / (z * z)
    e = oracle.EPS2D  # the low-pass s (0.3, as the float32 value the rasterizer takes)
    expect = [k * (1 + x * x / (z * z)) + e, k * x * y / (z * z), k * (1 + y * y / (z * z)) + e]
    np.testing.assert_allclose(p["cov2d"][0], expect, rtol=1e-12)


def test_unequal_focal_lengths_and_principal_point_closed_form():
    # K = [[fx, 0, cx], [0, fy, cy], [0, 0, 1]] (App. E, with the printed fy/fy, cx/cx read as
    # fx/fy, cx/cy): x uses only fx and cx, y only fy and cy.  With the identity pose and
    # J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]], an isotropic Gaussian of scale s gives
    # Sigma' = s^2 J J^T = s^2 [[fx^2 (z^2 + x^2)/z^4, fx fy x y/z^4], [., fy^2 (z^2 + y^2)/z^4]]
    x, y, z, s = 0.35, -0.2, 2.0, 0.04
    fx, fy, cx, cy = 70.0, 45.0, 31.0, 18.0
    sc = _scene([[x, y, z]], [[1, 0, 0, 0]], [[math.log(s)] * 3], [0.0], np.zeros((1, 1, 3)))
    cam = synth.Camera(64, 40, np.eye(4, dtype=np.float32), fx, fy, cx, cy)
    p = oracle.project(sc, cam)
    np.testing.assert_allclose(p["means2d"][0], [fx * x / z + cx, fy * y / z + cy], rtol=1e-14)
    z4 = z ** 4
    expect = [s * s * fx * fx * (z * z + x * x) / z4 + oracle.EPS2D, s * s * fx * fy * x * y / z4,
              s * s * fy * fy * (z * z + y * y) / z4 + oracle.EPS2D]
    np.testing.assert_allclose(p["cov2d"][0], expect, rtol=1e-12)


def test_anisotropic_axis_aligned_and_rotated_90():
    # scales (sx, sy, sz) with identity rotation: Sigma' = diag(f^2 sx^2/z^2, f^2 sy^2/z^2) + 0.3
    # rotating the Gaussian by 90 degrees about the optical axis swaps the two entries
    sx, sy, z, f = 0.1, 0.03, 3.0, 40.0
    ls = [math.log(sx), math.log(sy), math.log(0.2)]
    q90 = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]
    sc = _scene([[0, 0, z], [0, 0, z]], [[1, 0, 0, 0], q90], [ls, ls], [0.0, 0.0], np.zeros((2, 1, 3)))
    p = oracle.project(sc, _identity_cam(32, 32, f, 16.0, 16.0))
    a, b = (f * sx / z) ** 2 + oracle.EPS2D, (f * sy / z) ** 2 + oracle.EPS2D
    np.testing.assert_allclose(p["cov2d"][0], [a, 0.0, b], atol=1e-12)
    np.testing.assert_allclose(p["cov2d"][1], [b, 0.0, a], atol=1e-12)
    lam = max(a, b)
    assert p["radii"][0] == math.ceil(3 * math.sqrt(lam))


def test_projection_invariant_under_rigid_motion_of_world_and_camera():
    sc, cam = synth.random_small_scene(20, seed=11, sh_degree=0)
    sc64 = _scene(sc.means, sc.quats, sc.log_scales, sc.opacity_logits, sc.sh)
    p0 = oracle.project(sc64, cam)
    # move every Gaussian by the rigid motion (Rm, tm) and the camera with it
    Rm = _rodrigues([0.3, 1.0, -0.5], 0.8)
    tm = np.array([0.5, -1.0, 2.0])
    qm = np.concatenate([[math.cos(0.4)], math.sin(0.4) * np.array([0.3, 1.0, -0.5]) / np.linalg.norm([0.3, 1.0, -0.5])])

    def qmul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    means2 = sc64.means @ Rm.T + tm
    quats2 = np.array([qmul(qm, q) for q in sc64.quats])
    vm = np.asarray(cam.viewmat, np.float64)
    world_to_old = np.eye(4)
    world_to_old[:3, :3] = Rm.T
    world_to_old[:3, 3] = -Rm.T @ tm
    cam2 = synth.Camera(cam.width, cam.height, vm @ world_to_old, cam.fx, cam.fy, cam.cx, cam.cy)
    p1 = oracle.project(_scene(means2, quats2, sc64.log_scales, sc64.opacity_logits, sc64.sh), cam2)
    for k in ("means2d", "depths", "cov2d", "conics"):
        np.testing.assert_allclose(p1[k], p0[k], rtol=1e-9, atol=1e-9)
    np.testing.assert_array_equal(p1["radii"], p0["radii"])


def test_antialiased_compensation_closed_form():
    s, d, f = math.exp(-3.0), 4.0, 64.0
    sc = _scene([[0, 0, 0]], [[1, 0, 0, 0]], [[-3.0] * 3], [1.0], np.zeros((1, 1, 3)))
    p = oracle.project(sc, _axis_cam(d=d, f=f), antialiased=True)
    v0 = (f * s / d) ** 2
    comp = math.sqrt(v0 * v0 / ((v0 + oracle.EPS2D) ** 2))  # sqrt(|S|/|S+sI|) for S = v0 I
    np.testing.assert_allclose(p["opacities"][0], comp / (1 + math.exp(-1.0)), rtol=1e-13)


def test_culling_and_pixel_centre_convention():
    # camera at z=4 looking down -z: depth = 4 - z.  Behind, nearer than 0.01, in front.
    sc = _scene([[0, 0, 5.0], [0, 0, 3.995], [0, 0, 0.0]], [[1, 0, 0, 0]] * 3, [[-3.0] * 3] * 3,
                [0.0] * 3, np.zeros((3, 1, 3)))
    p = oracle.project(sc, _axis_cam(d=4.0))
    assert p["radii"][0] == 0 and p["radii"][1] == 0 and p["radii"][2] > 0
    # on the optical axis the mean lands on (cx, cy) = the corner shared by four pixel centres:
    # the rendered image is symmetric about that corner
    sc = _scene([[0, 0, 0]], [[1, 0, 0, 0]], [[-2.0] * 3], [2.0], np.full((1, 1, 3), 1.0))
    r = oracle.render(sc, _axis_cam(d=4.0))
    img = r["image"][..., 0]
    np.testing.assert_allclose(img, img[::-1, :], atol=1e-14)
    np.testing.assert_allclose(img, img[:, ::-1], atol=1e-14)
    np.testing.assert_allclose(img, img.T, atol=1e-14)
    assert img[31, 31] == img.max()


def test_radius_cap_culls_splats_wider_than_1e7_pixels():
    # on the optical axis of an identity camera an isotropic Gaussian of scale s at depth z has
    # Sigma' = ((f s / z)^2 + eps) I, so r = ceil(3 sqrt((f s / z)^2 + eps)).  A splat whose radius
    # exceeds 1e7 pixels is culled like an empty one; one of about 5e6 pixels is kept, its box clipped
    f, z = 100.0, 0.02
    scales = [1333.0, 333.0]
    sc = _scene([[0, 0, z]] * 2, [[1, 0, 0, 0]] * 2, [[math.log(v)] * 3 for v in scales], [0.0] * 2,
                np.zeros((2, 1, 3)))
    p = oracle.project(sc, _identity_cam(64, 64, f, 32.0, 32.0))
    r = [math.ceil(3 * math.sqrt((f * v / z) ** 2 + oracle.EPS2D)) for v in scales]
    assert r[0] > 1e7 > r[1] > 1e6
    assert p["radii"][0] == 0 and p["radii"][1] == r[1]
    np.testing.assert_array_equal(p["boxes"][1], [0, 63, 0, 63])


# --------------------------------------------------------------------------- #
# spherical harmonics (App. C.1)                                               #
# --------------------------------------------------------------------------- #

def _quadrature(n_theta=24, n_phi=48):
    x, w = np.polynomial.legendre.leggauss(n_theta)  # nodes in cos(theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).reshape(-1)
    return dirs, wts


def test_sh_orthonormal_by_quadrature():
    dirs, wts = _quadrature()
    Y = oracle.sh_basis(3, dirs)
    gram = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_matches_scipy_real_harmonics():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(5)
    dirs = rng.normal(size=(50, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    theta = np.arccos(np.clip(dirs[:, 2], -1, 1))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    Y = oracle.sh_basis(3, dirs)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            c = sp.sph_harm_y(l, abs(m), theta, phi)  # Condon-Shortley phase included
            if m > 0:
                ref = math.sqrt(2) * c.real
            elif m < 0:
                ref = math.sqrt(2) * c.imag
            else:
                ref = c.real
            np.testing.assert_allclose(Y[:, k], ref, atol=1e-12, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_basis_gradient_matches_finite_differences():
    rng = np.random.default_rng(6)
    d = rng.normal(size=(7, 3))
    dY = oracle.sh_basis_grad(3, d)
    h = 1e-6
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd = (oracle.sh_basis(3, d + e) - oracle.sh_basis(3, d - e)) / (2 * h)
        np.testing.assert_allclose(dY[:, :, ax], fd, atol=1e-8)


def test_sh_colour_degree0_and_clamp():
    # degree 0: colour = max(0, c / (2 sqrt(pi)) + 0.5)
    coeff = np.array([[[1.0, -3.0, 0.0]]])
    sc = _scene([[0, 0, 0]], [[1, 0, 0, 0]], [[-3] * 3], [0.0], coeff)
    col, raw = oracle.sh_colors(sc, _axis_cam())
    k0 = 1 / (2 * math.sqrt(math.pi))
    np.testing.assert_allclose(raw[0], [k0 + 0.5, -3 * k0 + 0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(col[0], [k0 + 0.5, 0.0, 0.5], atol=1e-15)


def test_sh_colour_uses_direction_from_camera_centre():
    # degree 1 with only the m=0 (z) coefficient: colour = k1 * dir_z * c + 0.5
    deg = 1
    sh = np.zeros((1, 4, 3))
    sh[0, 2, :] = 1.0
    cam = _axis_cam(d=4.0)   # centre (0, 0, 4)
    mu = np.array([0.3, 0.4, 1.0])
    sc = _scene([mu], [[1, 0, 0, 0]], [[-3] * 3], [0.0], sh, deg)
    col, raw = oracle.sh_colors(sc, cam)
    v = mu - np.array([0.0, 0.0, 4.0])
    k1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(raw[0], k1 * v[2] / np.linalg.norm(v) + 0.5, atol=1e-14)


# --------------------------------------------------------------------------- #
# compositing (App. C.2)                                                       #
# --------------------------------------------------------------------------- #

def _splats_isotropic(centres, variances, opacities, depths, W, H):
    """2D splats whose conic, radius and box follow from the support rule in closed form."""
    n = len(centres)
    boxes = np.zeros((n, 4), np.int32)
    radii = np.zeros(n, np.int32)
    for i, ((mx, my), v) in enumerate(zip(centres, variances)):
        r = math.ceil(3 * math.sqrt(v))
        radii[i] = r
        boxes[i] = [max(0, math.ceil(mx - r - 0.5)), min(W - 1, math.floor(mx + r - 0.5)),
                    max(0, math.ceil(my - r - 0.5)), min(H - 1, math.floor(my + r - 0.5))]
    return dict(means2d=np.array(centres, float), conics=np.array([[1 / v, 0, 1 / v] for v in variances]),
                opacities=np.array(opacities, float), depths=np.array(depths, float), radii=radii, boxes=boxes)


def test_single_gaussian_closed_form():
    W = H = 40
    mx, my, v, o = 17.3, 21.8, 9.0, 0.8
    sp = _splats_isotropic([(mx, my)], [v], [o], [2.0], W, H)
    col = np.array([[0.2, 0.5, 0.9]])
    r = oracle.render_splats(sp, col, W, H)
    img = r["color"].reshape(H, W, 3)
    rad = math.ceil(3 * math.sqrt(v))
    for y in range(H):
        for x in range(W):
            dx, dy = x + 0.5 - mx, y + 0.5 - my
            a = min(oracle.ALPHA_MAX, o * math.exp(-0.5 * (dx * dx + dy * dy) / v))
            inside = abs(dx) <= rad and abs(dy) <= rad
            expect = col[0] * a if (inside and a >= oracle.ALPHA_MIN) else np.zeros(3)
            np.testing.assert_allclose(img[y, x], expect, atol=1e-15)


def test_two_gaussians_closed_form_and_depth_order():
    W = H = 8
    sp = _splats_isotropic([(4.0, 4.0), (4.0, 4.0)], [4.0, 4.0], [0.6, 0.9], [1.0, 2.0], W, H)
    c = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    r = oracle.render_splats(sp, c, W, H, pixels=[3 * W + 3])
    g = math.exp(-0.5 * (0.25 + 0.25) / 4.0)
    a1, a2 = 0.6 * g, 0.9 * g
    np.testing.assert_allclose(r["color"][0], [a1, a2 * (1 - a1), 0.0], atol=1e-15)
    np.testing.assert_allclose(r["T"][0], (1 - a1) * (1 - a2), atol=1e-15)
    sp["depths"] = np.array([2.0, 1.0])  # swap the order
    r = oracle.render_splats(sp, c, W, H, pixels=[3 * W + 3])
    np.testing.assert_allclose(r["color"][0], [a1 * (1 - a2), a2, 0.0], atol=1e-15)
    # equal depths: ties broken by index
    sp["depths"] = np.array([1.5, 1.5])
    r = oracle.render_splats(sp, c, W, H, pixels=[3 * W + 3])
    np.testing.assert_allclose(r["color"][0], [a1, a2 * (1 - a1), 0.0], atol=1e-15)


def test_background_and_opaque_front():
    W = H = 8
    sp = _splats_isotropic([(4.0, 4.0), (4.0, 4.0)], [100.0, 100.0], [1.0, 1.0], [1.0, 2.0], W, H)
    c = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    bg = np.array([0.0, 0.0, 1.0])
    r = oracle.render_splats(sp, c, W, H, pixels=[3 * W + 3], bg=bg)
    # both capped: e^-sigma ~ 0.9975 > alpha_max.  Behind the first, T = 1 - alpha_max; the second
    # would leave (1 - alpha_max)^2, which is below T_min for the float32 parameters (1 - 0.99 in
    # float32 is 0.0099999905, squared 9.99998e-5 < 1e-4): it is excluded and the pixel stops
    a, tmin = oracle.ALPHA_MAX, oracle.T_MIN
    assert (1 - a) ** 2 < tmin <= 1 - a
    np.testing.assert_allclose(r["color"][0], [a, 0.0, 1 - a], atol=1e-15)
    assert r["ncontrib"][0] == 1 and r["blends"][0] == 2
    # a back Gaussian below the cap is blended behind the capped front one, weight alpha (1 - alpha_max)
    sp["opacities"] = np.array([1.0, 0.5])
    r = oracle.render_splats(sp, c, W, H, pixels=[3 * W + 3], bg=bg)
    a2 = 0.5 * math.exp(-0.5 * (0.25 + 0.25) / 100.0)
    np.testing.assert_allclose(r["color"][0], [a, a2 * (1 - a), (1 - a) * (1 - a2)], atol=1e-15)


def test_transmittance_cutoff_excludes_and_stops():
    # alpha = 0.95 each: T = 0.05, 0.0025, 1.25e-4, then 6.25e-6 < 1e-4 -> the 4th is excluded
    W = H = 4
    n = 6
    v = 1e6
    o = 0.95 / math.exp(-0.5 * (2 * 0.0) / v)
    sp = _splats_isotropic([(2.5, 2.5)] * n, [v] * n, [o] * n, list(range(1, n + 1)), W, H)
    c = np.eye(n, 3) if n <= 3 else np.tile(np.array([[1.0, 1.0, 1.0]]), (n, 1))
    ids, alphas, Ts = oracle.render_trace(sp, c, 2, 2)
    assert list(ids) == [0, 1, 2]
    np.testing.assert_allclose(alphas, 0.95, rtol=1e-12)
    np.testing.assert_allclose(Ts, [1.0, 0.05, 0.0025], rtol=1e-12)
    r = oracle.render_splats(sp, c, W, H, pixels=[2 * W + 2])
    assert r["ncontrib"][0] == 3
    assert r["blends"][0] == 4  # the excluded 4th was evaluated, the rest were not
    np.testing.assert_allclose(r["T"][0], 0.05 ** 3, rtol=1e-12)


def test_alpha_below_threshold_is_skipped():
    W = H = 4
    o = 0.5 / 255
    sp = _splats_isotropic([(2.0, 2.0)], [1e6], [o], [1.0], W, H)
    r = oracle.render_splats(sp, np.ones((1, 3)), W, H)
    assert np.all(r["color"] == 0.0) and np.all(r["T"] == 1.0) and np.all(r["ncontrib"] == 0)


def test_skipped_gaussian_leaves_the_ones_behind_it():
    # a faint Gaussian in front (alpha < 1/255 everywhere) is passed over, not a stop: the
    # pixel is exactly what the back Gaussian renders alone, c alpha with alpha = o e^-sigma
    W = H = 8
    v, o = 4.0, 0.7
    sp = _splats_isotropic([(4.0, 4.0), (4.0, 4.0)], [v, v], [0.5 / 255, o], [1.0, 2.0], W, H)
    c = np.array([[1.0, 1.0, 1.0], [0.2, 0.6, 0.4]])
    r = oracle.render_splats(sp, c, W, H, pixels=[3 * W + 3])
    a = o * math.exp(-0.5 * (0.25 + 0.25) / v)
    np.testing.assert_allclose(r["color"][0], c[1] * a, atol=1e-15)
    np.testing.assert_allclose(r["T"][0], 1 - a, atol=1e-15)
    assert r["ncontrib"][0] == 1 and r["blends"][0] == 2


def test_clamped_alpha_passes_no_gradient():
    # at the centre pixel o e^-sigma > 0.99, so C = 0.99 c (+ 0.01 bg) there: C does not move with
    # the opacity, the mean or the conic (a small change keeps alpha on the clamp), only with c
    W = H = 8
    sp = _splats_isotropic([(4.0, 4.0)], [100.0], [0.999], [1.0], W, H)
    c = np.array([[0.3, 0.5, 0.7]])
    g = np.array([[0.4, -1.1, 0.9]])
    f = oracle.render_splats(sp, c, W, H, pixels=[3 * W + 3])
    np.testing.assert_allclose(f["color"][0], oracle.ALPHA_MAX * c[0], atol=1e-15)
    b = oracle.render_splats_bwd(sp, c, W, H, g, pixels=[3 * W + 3])
    assert np.all(b["d_opacities"] == 0.0) and np.all(b["d_means2d"] == 0.0) and np.all(b["d_conics"] == 0.0)
    np.testing.assert_allclose(b["d_colors"][0], oracle.ALPHA_MAX * g[0], atol=1e-15)


def test_absgrad_sums_per_pixel_magnitudes():
    # absgrad (App. A) adds |dL_p/dmu'| pixel by pixel.  One Gaussian (conic I/v), two pixels
    # mirrored about its centre in x: L = sum_p <g, c> alpha_p, dL_p/dmu'_x = <g, c> alpha_p dx_p / v,
    # so the signed x gradients cancel while absgrad keeps 2 <g, c> alpha |dx| / v; in y both
    # pixels pull the same way and the two agree
    W = H = 8
    v, o = 3.0, 0.6
    sp = _splats_isotropic([(4.0, 4.0)], [v], [o], [1.0], W, H)
    c = np.array([[0.3, 0.5, 0.7]])
    g = np.array([[0.4, 1.1, 0.9], [0.4, 1.1, 0.9]])
    b = oracle.render_splats_bwd(sp, c, W, H, g, pixels=[3 * W + 3, 3 * W + 4], want_absgrad=True)
    a = o * math.exp(-0.5 * (0.25 + 0.25) / v)
    gc = float(g[0] @ c[0])
    np.testing.assert_allclose(b["d_means2d"][0, 0], 0.0, atol=1e-15)
    np.testing.assert_allclose(b["absgrad"][0, 0], 2 * gc * a * 0.5 / v, rtol=1e-13)
    np.testing.assert_allclose(b["d_means2d"][0, 1], -2 * gc * a * 0.5 / v, rtol=1e-13)
    np.testing.assert_allclose(b["absgrad"][0, 1], 2 * gc * a * 0.5 / v, rtol=1e-13)


def test_partition_of_unity_and_trace_invariants():
    sc, cam = synth.random_small_scene(40, seed=2, width=24, height=20, log_scale_mu=-1.6)
    sp = oracle.project(sc, cam)
    ones = np.ones((sc.n, 3))
    r = oracle.render_splats(sp, ones, cam.width, cam.height)
    # sum_n alpha_n T_n + T_final = 1 (telescoping product)
    np.testing.assert_allclose(r["color"][:, 0] + r["T"], 1.0, atol=1e-13)
    assert np.all(r["T"] >= oracle.T_MIN)
    checked = 0
    for y in range(0, cam.height, 3):
        for x in range(0, cam.width, 3):
            ids, al, Ts = oracle.render_trace(sp, ones, x, y)
            if len(ids) == 0:
                continue
            checked += 1
            assert np.all(al >= oracle.ALPHA_MIN) and np.all(al <= oracle.ALPHA_MAX)
            np.testing.assert_allclose(Ts[1:], Ts[:-1] * (1 - al[:-1]), rtol=1e-13)
            assert np.all(np.diff(sp["depths"][ids]) >= 0)
    assert checked > 10


def test_fig1_single_gaussian_example():
    """The paper's Fig. 1 example: one Gaussian at (0,0,0.01), identity pose, f=1, c=120, 240x240."""
    with open(os.path.join(GOLDEN, "fig1_single_gaussian.json")) as fh:
        g = json.load(fh)
    scale = g["scale_for_test"]
    sc = _scene([g["mean"]], [g["quat"]], [[math.log(scale)] * 3], [g["opacity_logit_for_test"]],
                np.full((1, 1, 3), 1.0))
    K = g["K"]
    cam = synth.Camera(g["width"], g["height"], np.eye(4, dtype=np.float32), K[0][0], K[1][1], K[0][2], K[1][2])
    r = oracle.render(sc, cam)
    img = r["image"][..., 0]
    assert img.max() > 0.5
    # the centre pixels reach the maximum (alpha is capped at 0.99 on a small plateau) and the
    # intensity-weighted centroid sits on the principal point, pixel centres being at i + 0.5
    assert img[119, 119] == img.max() == img[120, 120]
    ys, xs = np.mgrid[0:240, 0:240]
    np.testing.assert_allclose([(img * ys).sum() / img.sum(), (img * xs).sum() / img.sum()], [119.5, 119.5],
                               atol=1e-9)
    np.testing.assert_allclose(img, img[::-1, ::-1], atol=1e-14)
    # sigma' = 100 * scale (f=1, z=0.01) plus the 0.3 low-pass
    v = (scale / 0.01) ** 2 + oracle.EPS2D
    np.testing.assert_allclose(r["splats"]["cov2d"][0], [v, 0.0, v], rtol=1e-12)
    # the same example as a caller passes it, in float32: its depth is float32(0.01), the near plane
    # too, so it is not culled and renders the same blob
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    sc32 = synth.Scene(f32(sc.means), f32(sc.quats), f32(sc.log_scales), f32(sc.opacity_logits), f32(sc.sh), 0)
    r32 = oracle.render(sc32, cam)
    assert r32["splats"]["radii"][0] == r["splats"]["radii"][0] > 0
    np.testing.assert_allclose(r32["image"], r["image"], atol=1e-5)


# --------------------------------------------------------------------------- #
# tile binning + sort against brute force with exact arithmetic (App. C.2)     #
# --------------------------------------------------------------------------- #

def _brute_bins(means2d, depths, radii, widths, heights, tile):
    out = []
    toff = 0
    C, N = depths.shape
    for c in range(C):
        W, H = int(widths[c]), int(heights[c])
        tx_n, ty_n = -(-W // tile), -(-H // tile)
        for n in range(N):
            r = int(radii[c, n])
            if r <= 0:
                continue
            mx, my = Fraction(float(means2d[c, n, 0])), Fraction(float(means2d[c, n, 1]))
            # pixel i supports the Gaussian iff |i + 1/2 - mx| <= r (exactly)
            xs = [i for i in range(W) if abs(Fraction(2 * i + 1, 2) - mx) <= r]
            ys = [j for j in range(H) if abs(Fraction(2 * j + 1, 2) - my) <= r]
            tiles = sorted({(j // tile, i // tile) for i in xs for j in ys})
            bits = int(np.asarray(depths[c, n], np.float32).view(np.uint32))
            for (ty, tx) in tiles:
                out.append(((toff + ty * tx_n + tx) << 32 | bits, c * N + n))
        toff += tx_n * ty_n
    out.sort()
    return out, toff


@pytest.mark.parametrize("tile", [8, 16])
def test_bin_sort_matches_brute_force(tile):
    rng = np.random.default_rng(tile)
    C, N = 2, 60
    widths, heights = np.array([37, 50]), np.array([29, 18])
    means2d = np.stack([rng.uniform(-10, 60, (C, N)), rng.uniform(-10, 40, (C, N))], -1).astype(np.float32)
    # exact half-integers and integers to hit the box edges
    means2d[:, :10] = np.round(means2d[:, :10] * 2) / 2
    depths = rng.uniform(0.5, 3.0, (C, N)).astype(np.float32)
    depths[:, 5:9] = depths[:, 4:5]  # ties
    radii = rng.integers(0, 9, (C, N)).astype(np.int32)
    keys, values, ranges = oracle.bin_sort(means2d, depths, radii, widths, heights, tile)
    ref, ntiles = _brute_bins(means2d, depths, radii, widths, heights, tile)
    assert len(ref) == len(keys)
    assert [int(k) for k in keys] == [k for k, _ in ref]
    assert [int(v) for v in values] == [v for _, v in ref]
    assert ranges.shape == (ntiles, 2)
    for t in range(ntiles):
        idx = [i for i, (k, _) in enumerate(ref) if (k >> 32) == t]
        if idx:
            assert (ranges[t, 0], ranges[t, 1]) == (idx[0], idx[-1] + 1)
        else:
            assert (ranges[t, 0], ranges[t, 1]) == (0, 0)


def test_bin_sort_equal_depths_share_tiles_in_index_order():
    # Gaussians at one spot with one depth fall in the same tiles with the same key; the order
    # within a tile is then by c N + n ascending (stable emission in index order), against brute force
    C, N, tile = 1, 12, 8
    means2d = np.zeros((C, N, 2), np.float32)
    means2d[0, :] = [13.5, 9.5]
    means2d[0, ::3] = [30.0, 20.0]
    depths = np.full((C, N), 1.25, np.float32)
    depths[0, 7] = 0.75
    radii = np.full((C, N), 6, np.int32)
    keys, values, ranges = oracle.bin_sort(means2d, depths, radii, [40], [28], tile)
    ref, _ = _brute_bins(means2d, depths, radii, np.array([40]), np.array([28]), tile)
    assert [int(k) for k in keys] == [k for k, _ in ref]
    assert [int(v) for v in values] == [v for _, v in ref]
    lo, hi = ranges[(9 // tile) * 5 + 13 // tile]
    assert [int(v) for v in values[lo:hi]] == [7, 1, 2, 4, 5, 8, 10, 11]


def test_render_agrees_with_bins():
    """Every (pixel, Gaussian) pair the per-pixel box admits lies in a tile bin listing it."""
    sc, cam = synth.random_small_scene(30, seed=4, width=40, height=24)
    sp = oracle.project(sc, cam)
    m = sp["means2d"].astype(np.float32)[None]
    keys, values, ranges = oracle.bin_sort(m, sp["depths"].astype(np.float32)[None], sp["radii"][None],
                                           [40], [24], 8)
    listed = {(int(k >> 32), int(v)) for k, v in zip(keys, values)}
    tx_n = 5
    for n in range(sc.n):
        if sp["radii"][n] <= 0:
            continue
        x0, x1, y0, y1 = sp["boxes"][n]
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                assert ((y // 8) * tx_n + x // 8, n) in listed

"""Pins for the oracle's unscented-transform (UT) binning gate, the 3DGUT-style
backbone the paper names beside 3DGEER (Sec. 3).  Checked against what
mathematics fixes: the bounded quadratic minimum (an independent solver and a
dense grid), the UT's exactness for a projection that is linear on the
Gaussian's support, the UT definition evaluated by hand where the projections
have a closed form, and the invariant that small distant Gaussians (an affine
projection) lose no contributing pixel."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

import synthetic as S


def _sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


def _one(mu, ls, q, logit):
    n = 1
    sh = np.zeros((n, 1, 3), np.float32)
    return S.Scene(np.asarray([mu], np.float32), np.asarray([ls], np.float32), np.asarray([q], np.float32),
                   np.asarray([logit], np.float32), sh, 0, np.zeros(n, np.float32))


# ---------------------------------------------------------------- bounded quadratic minimum

def test_rect_min_matches_bounded_solver_and_grid(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(11)
    for _ in range(200):
        L = rng.normal(0, 1, (2, 2))
        M = L @ L.T + 0.05 * np.eye(2)
        A, B, C = M[0, 0], M[0, 1], M[1, 1]
        c = rng.uniform(-10, 10, 2)
        x0, y0 = rng.uniform(-12, 8, 2)
        x1, y1 = x0 + rng.uniform(0.1, 7), y0 + rng.uniform(0.1, 7)
        got = O.ut_rect_min(c, (A, B, C), (x0, x1, y0, y1))
        f = lambda y: float((y - c) @ M @ (y - c))
        best = min(minimize(f, s, method="L-BFGS-B", bounds=[(x0, x1), (y0, y1)],
                            options={"ftol": 1e-15, "gtol": 1e-12}).fun
                   for s in ([x0, y0], [x1, y1], [(x0 + x1) / 2, (y0 + y1) / 2]))
        gx, gy = np.meshgrid(np.linspace(x0, x1, 201), np.linspace(y0, y1, 201))
        d = np.stack([gx - c[0], gy - c[1]], -1)
        grid = np.einsum("...i,ij,...j->...", d, M, d).min()
        assert got <= grid + 1e-9 * (1 + grid)
        assert abs(got - best) <= 1e-7 * (1 + best), (got, best)
    # centre inside the rectangle
    assert O.ut_rect_min((1.0, 2.0), (2.0, 0.3, 1.0), (0.0, 3.0, 1.0, 4.0)) == 0.0


# ---------------------------------------------------------------- UT moments

@pytest.mark.parametrize("phi", [0.0, 0.6, -1.1])
def test_planar_gaussian_in_fronto_parallel_plane_is_exact(oracle_lib, phi):
    """A flat Gaussian lying in the plane z = z0 of a pinhole camera: the
    projection is affine on its support, u = f_x x / z0 + c_x, so the UT gives
    the exact image moments: ybar = Pi(mu), Sigma_2 = F R diag(s1^2, s2^2) R^T F
    + I/12 with F = diag(f_x, f_y) / z0 and R the in-plane rotation by phi."""
    O = oracle_lib
    cam = S.Camera(S.PINHOLE, 160, 120, 150.0, 130.0, 81.0, 57.5)
    mu = np.array([0.21, -0.13, 3.7])
    ls = [math.log(0.05), math.log(0.02), -30.0]
    q = [math.cos(phi / 2), 0.0, 0.0, math.sin(phi / 2)]
    logit = 0.5
    sc = _one(mu, ls, q, logit)
    gate, status, geo = O.ut_gate(cam, sc)
    assert status[0] == 1
    m = sc.means[0].astype(float)
    s = np.exp(sc.log_scales[0].astype(float))
    qq = sc.quats[0].astype(float)
    qq /= np.linalg.norm(qq)
    ang = 2 * math.atan2(qq[3], qq[0])
    Rp = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
    F = np.diag([cam.fx / m[2], cam.fy / m[2]])
    S2 = F @ Rp @ np.diag(s[:2] ** 2) @ Rp.T @ F + np.eye(2) / 12
    ybar = np.array([cam.fx * m[0] / m[2] + cam.cx, cam.fy * m[1] / m[2] + cam.cy])
    np.testing.assert_allclose(geo[0, :2], ybar, rtol=1e-12)
    inv = np.linalg.inv(S2)
    np.testing.assert_allclose(geo[0, 2:5], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-9,
                               atol=1e-12 * np.abs(inv).max())
    k2 = 2 * math.log(255 * _sigmoid(float(sc.opacity_logits[0])))
    assert abs(geo[0, 5] - k2) < 1e-12


def test_needle_along_depth_by_hand(oracle_lib):
    """A needle Gaussian along the optical axis at lateral offset (x_c, y_c):
    its sigma points are mu +- sqrt(3) a z-hat and four copies of mu (the two
    vanishing axes), whose images are u = f x_c / (z0 +- sqrt(3) a) + c.  The UT
    (mean weights 0 and 1/6, covariance weights 2 and 1/6) evaluated by hand on
    these closed-form images: this fixes the sigma-point spread, the weights,
    the centre point's covariance weight and the low-pass term."""
    O = oracle_lib
    cam = S.Camera(S.PINHOLE, 200, 160, 180.0, 180.0, 100.0, 80.0)
    xc, yc, z0, a = 0.4, -0.25, 2.0, 0.3
    # rotation about y by -90 deg: the first principal axis becomes +z
    q = [math.cos(-math.pi / 4), 0.0, math.sin(-math.pi / 4), 0.0]
    sc = _one([xc, yc, z0], [math.log(a), -30.0, -30.0], q, 1.0)
    gate, status, geo = O.ut_gate(cam, sc)
    assert status[0] == 1
    m = sc.means[0].astype(float)
    aa = math.exp(float(sc.log_scales[0, 0]))
    qq = sc.quats[0].astype(float)
    qq /= np.linalg.norm(qq)
    # first column of the rotation (a unit vector within FP32 rounding of +z)
    w, x, y, z = qq
    ax = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
    pts = [m] + [m + ax * math.sqrt(3) * aa, m - ax * math.sqrt(3) * aa] + [m] * 4
    ys = np.array([[cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy] for p in pts])
    wm = np.array([0] + [1 / 6] * 6)
    wc = np.array([2] + [1 / 6] * 6)
    yb = wm @ ys
    S2 = sum(wc[j] * np.outer(ys[j] - yb, ys[j] - yb) for j in range(7)) + np.eye(2) / 12
    inv = np.linalg.inv(S2)
    np.testing.assert_allclose(geo[0, :2], yb, rtol=1e-12)
    np.testing.assert_allclose(geo[0, 2:5], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-6)
    # the needle is strongly non-linear: the UT mean moves off Pi(mu)
    assert abs(yb[0] - ys[0, 0]) > 0.1


# ---------------------------------------------------------------- gate semantics

@pytest.mark.parametrize("which", ["pinhole", "kb"])
def test_small_distant_gaussians_lose_no_contributing_pixel(oracle_lib, which):
    """For Gaussians a few pixels wide far from the camera the projection is
    affine on their support and the UT ellipse contains the alpha >= 1/255 region
    of the filtered response (Eq. 9 with the footprint added as I/12): every
    (pixel, Gaussian) pair with T >= 1.05/255 lies in a kept tile."""
    O = oracle_lib
    if which == "pinhole":
        cam = S.pinhole(96, 72, 90.0)
    else:
        cam = S.c3_camera(96, 96)
    rng = np.random.default_rng(4)
    n = 300
    if which == "pinhole":
        means = np.stack([rng.uniform(-1.2, 1.2, n), rng.uniform(-0.9, 0.9, n), rng.uniform(6, 10, n)], 1)
    else:
        means = np.stack([rng.uniform(-4, 4, n), rng.uniform(-4, 4, n), rng.uniform(3, 8, n)], 1)
    sc = S.Scene(means.astype(np.float32), rng.normal(-3.5, 0.4, (n, 3)).astype(np.float32),
                 S._random_quats(rng, n), rng.normal(1.0, 1.0, n).astype(np.float32),
                 np.zeros((n, 1, 3), np.float32), 0, np.zeros(n, np.float32))
    gate, status, _ = O.ut_gate(cam, sc)
    assert (status == 1).sum() > 0.8 * n
    pix, gid = O.pairs_above(cam, sc, 1.05 / 255)
    assert pix.size > 500
    tx, _ = O.tile_grid(cam)
    tile = (pix // cam.width) // O.TILE * tx + (pix % cam.width) // O.TILE
    ut = status[gid] == 1
    assert ut.sum() > 0.8 * ut.size
    assert np.all(gate[gid[ut], tile[ut]] >= 1)


def test_fallbacks_and_culled(oracle_lib):
    """A Gaussian straddling the pinhole's side plane (a sigma point at
    p_z < 0.1 |p|) and one that can never reach 1/255 keep the angular-tile rule."""
    O = oracle_lib
    cam = S.pinhole(64, 48, 60.0)
    sc = S.Scene(np.array([[0.0, 0.0, 3.0], [3.0, 0.0, 0.2], [0.1, 0.1, 4.0]], np.float32),
                 np.array([[-2.0] * 3, [-1.0] * 3, [-3.0] * 3], np.float32),
                 np.tile(np.array([1, 0, 0, 0], np.float32), (3, 1)),
                 np.array([0.0, 0.0, -9.0], np.float32), np.zeros((3, 1, 3), np.float32), 0,
                 np.zeros(3, np.float32))
    gate, status, _ = O.ut_gate(cam, sc)
    assert list(status) == [1, 0, 0]
    assert np.all(gate[1] == 1) and np.all(gate[2] == 1)
    sure, near, st = O.ut_bin_counts(cam, sc)
    _, pg, _, _ = O.bin_counts(cam, sc)
    assert sure[1] == pg[1] and sure[2] == pg[2] == 0 and near[1] == near[2] == 0


def test_gate_render_equals_plain_when_gate_keeps_all(oracle_lib):
    """A gate of ones renders exactly what no gate renders."""
    O = oracle_lib
    cam, sc = S.c1()
    tx, ty = O.tile_grid(cam)
    a = O.render(cam, sc)
    b = O.render(cam, sc, gate=np.ones((sc.n, tx * ty), np.uint8))
    assert np.array_equal(a.rgb, b.rgb) and np.array_equal(a.T, b.T)


def test_ut_binning_study(oracle_lib):
    """What UT binning keeps and loses against the conservative angular-tile
    rule (the render without a gate is exact: every pair with alpha >= 1/255 is
    evaluated).  Asserted: it keeps fewer pairs on the pinhole scenes, and its
    render differs from the exact one by little on average (the loss sits on
    the ellipse's rim and on Gaussians the UT moments describe poorly)."""
    O = oracle_lib
    cases = {"c1": S.c1(),
             "c2_small": (S.pinhole(160, 90, 150.0),
                          S.blob_scene(3000, seed=2, cam=S.pinhole(160, 90, 150.0), sh_degree=0)),
             "fisheye": (S.c3_camera(64, 64),
                         S.blob_scene(3000, seed=5, cam=S.pinhole(64, 64, 40.0), blob_frac=0.3, shell=(1.5, 4.0),
                                      log_scale_mean=-2.5, sh_degree=0))}
    out = {}
    for name, (cam, sc) in cases.items():
        gate, status, _ = O.ut_gate(cam, sc, eps=0.0)
        total, pg, _, pas = O.bin_counts(cam, sc, dense=True)
        g = gate.copy()
        g[status == 0] = pas[status == 0]
        ut_pairs = int((g >= 1).sum())
        exact = O.render(cam, sc, eps=0.0)
        utr = O.render(cam, sc, eps=0.0, gate=gate)
        diff = np.abs(utr.rgb - exact.rgb)
        out[name] = dict(pair_ratio=ut_pairs / max(total, 1), mean=float(diff.mean()),
                         frac=float((diff.max(1) > 1 / 255).mean()), ut_share=float((status == 1).mean()))
    print(out)
    for name in ("c1", "c2_small"):
        assert out[name]["pair_ratio"] < 1.0, out
    for name in out:
        assert out[name]["mean"] < 5e-3, out

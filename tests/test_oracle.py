"""Pins for the FP64 oracle: closed forms, brute force, quadrature and invariants
fixed by the paper and by mathematics (never by the oracle's own formulas)."""
import json
import math
import os

import numpy as np
import pytest

import synthetic as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


def _rot(q):
    w, x, y, z = np.asarray(q, float) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _project(cam, X):
    """Forward camera model written independently of the oracle (test-side)."""
    R = cam.cam_to_world[:, :3].astype(float)
    o = cam.cam_to_world[:, 3].astype(float)
    v = (np.asarray(X, float) - o) @ np.linalg.inv(R).T
    if cam.model == S.PINHOLE:
        return cam.fx * v[..., 0] / v[..., 2] + cam.cx, cam.fy * v[..., 1] / v[..., 2] + cam.cy
    rho = np.hypot(v[..., 0], v[..., 1])
    th = np.arctan2(rho, v[..., 2])
    k = cam.k.astype(float)
    td = th * (1 + k[0] * th ** 2 + k[1] * th ** 4 + k[2] * th ** 6 + k[3] * th ** 8)
    return cam.fx * td * v[..., 0] / rho + cam.cx, cam.fy * td * v[..., 1] / rho + cam.cy


# ---------------------------------------------------------------- camera model

@pytest.mark.parametrize("which", ["pinhole", "kb"])
def test_unproject_round_trip(oracle_lib, which):
    O = oracle_lib
    if which == "pinhole":
        cam = S.pinhole(640, 480, 500.0, 311.3, 247.9, cam_to_world=S.look_at((0.3, -0.2, 0.1), (1, 0, 5)))
    else:
        cam = S.c3_camera(256, 256)
        cam.cam_to_world = S.look_at((0.1, 0.2, 0.0), (0.5, 0, 3))
    rng = np.random.default_rng(5)
    xs, ys = rng.uniform(0, cam.width, 2000), rng.uniform(0, cam.height, 2000)
    d, dx, dy, valid = O.rays(cam, xs, ys)
    assert valid.sum() > 1000
    X = cam.cam_to_world[:, 3].astype(float) + 3.7 * d[valid]
    px, py = _project(cam, X)
    assert np.abs(px - xs[valid]).max() < 1e-9 and np.abs(py - ys[valid]).max() < 1e-9
    np.testing.assert_allclose(np.linalg.norm(d[valid], axis=1), 1.0, atol=1e-14)


def test_kb_equidistant_theta_equals_r(oracle_lib):
    """KB with k = 0 is the equidistant model: theta = r / f exactly."""
    cam = S.Camera(S.KB_FISHEYE, 200, 200, 50.0, 50.0, 100.0, 100.0, np.zeros(4), theta_lim=math.radians(95))
    xs = np.array([100.5, 150.5, 170.5, 100.0 + 50 * 1.5])
    ys = np.array([100.5, 100.0, 140.5, 100.0])
    d, _, _, valid = oracle_lib.rays(cam, xs, ys)
    r = np.hypot((xs - 100) / 50, (ys - 100) / 50)
    np.testing.assert_allclose(np.arccos(np.clip(d[:, 2], -1, 1)), r, atol=1e-12)


def test_edge_rays_are_half_pixel_offsets(oracle_lib):
    """delta_x = Pi^-1(p + (1/2, 0)) - Pi^-1(p) with the same camera model (Eq. 6 text)."""
    cam = S.c3_camera(128, 128)
    d, dx, dy, valid = oracle_lib.rays(cam, np.array([40.5]), np.array([77.5]))
    d2, _, _, _ = oracle_lib.rays(cam, np.array([41.0, 40.5]), np.array([77.5, 78.0]))
    np.testing.assert_allclose(dx[0], d2[0] - d[0], atol=1e-15)
    np.testing.assert_allclose(dy[0], d2[1] - d[0], atol=1e-15)


# ---------------------------------------------------------------- footprint (Eq. 6-8)

def _random_pair(rng, cam):
    mu = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.3, 0.3), rng.uniform(2.5, 5)])
    px, py = _project(cam, mu[None])
    x = float(px[0] + rng.uniform(-3, 3))
    y = float(py[0] + rng.uniform(-3, 3))
    ls = rng.normal(-3, 0.5, 3)
    q = rng.standard_normal(4)
    return x, y, mu, ls, q


def test_footprint_invariants(oracle_lib):
    """Sigma_fp^u d_u = 0, PSD and rank <= 2 (Eq. 8); Sigma_render too (Eq. 12, text below it)."""
    rng = np.random.default_rng(1)
    cam = S.pinhole(64, 48, 60.0)
    for it in range(50):
        x, y, mu, ls, q = _random_pair(rng, cam)
        rho2 = 0.0 if it % 2 == 0 else float(rng.uniform(0, 1e-3))
        r = oracle_lib.pair(cam, x, y, mu, ls, q, 0.3, rho2)
        for key in ("Sfp", "Sr"):
            M = r[key]
            scale = np.abs(M).max() + 1e-300
            assert np.abs(M @ r["du"]).max() <= 1e-12 * scale * np.linalg.norm(r["du"])
            np.testing.assert_allclose(M, M.T, atol=1e-14 * scale)
            ev = np.linalg.eigvalsh(M)
            assert ev.min() >= -1e-12 * scale
        # q lies in the ray-orthogonal plane and |q|^2 = D^2 (Eq. 2)
        assert abs(r["q"] @ r["du"]) <= 1e-10 * np.linalg.norm(r["q"]) * np.linalg.norm(r["du"]) + 1e-14


@pytest.mark.parametrize("model", ["pinhole", "kb"])
def test_footprint_matches_subray_covariance(oracle_lib, model):
    """Moment matching (Eq. 7-8): Sigma_fp^u equals the covariance of the depth-local,
    whitened, projected sub-ray offsets t* M_perp W (d(xi) - d) over xi uniform in the
    pixel, computed by brute force through the inverse mapping; the ratio -> 1 as the
    pixel shrinks (finer calibration)."""
    O = oracle_lib
    errs = []
    for f in (40.0, 160.0, 640.0):
        if model == "pinhole":
            cam = S.pinhole(int(f * 1.2), int(f), f, cam_to_world=S.look_at((0, 0, 0), (0.6, 0.2, 4)))
        else:
            cam = S.Camera(S.KB_FISHEYE, int(3.2 * f), int(3.2 * f), f, f, 1.6 * f, 1.6 * f,
                           np.array([0.02, -0.01, 0.004, -0.001]), theta_lim=1.5)
        mu = np.array([0.9, 0.4, 2.5])
        px, py = _project(cam, mu[None])
        x, y = float(np.floor(px[0])) + 0.5, float(np.floor(py[0])) + 0.5
        ls, q = np.log([0.06, 0.03, 0.015]), np.array([0.9, 0.2, -0.3, 0.25])
        r = O.pair(cam, x, y, mu, ls, q, 0.0)
        n = 256
        g = (np.arange(n) + 0.5) / n - 0.5
        XI, YI = np.meshgrid(g, g, indexing="ij")
        dsub, _, _, _ = O.rays(cam, x + XI.ravel(), y + YI.ravel())
        G = O.gauss(cam, S.Scene(mu[None].astype(np.float32), ls[None].astype(np.float32),
                                 q[None].astype(np.float32), np.zeros(1, np.float32), np.zeros((1, 1, 3), np.float32),
                                 0, np.zeros(1, np.float32)))
        W = G[0, :9].reshape(3, 3)
        du = r["du"]
        Mp = np.eye(3) - np.outer(du, du) / (du @ du)
        off = r["ts"] * (Mp @ W @ (dsub - r["d"]).T).T
        cov = np.cov(off.T, bias=True)
        rel = np.abs(cov - r["Sfp"]).max() / np.abs(r["Sfp"]).max()
        errs.append(rel)
    # the whitened pixel parallelogram and the exact sub-ray set agree to first order
    assert errs[-1] < 2e-2
    assert errs[2] < errs[0]


# ---------------------------------------------------------------- response (Eq. 9)

def _gauss_hermite_2d(fun, n=150):
    x, w = np.polynomial.hermite_e.hermegauss(n)
    w = w / np.sqrt(2 * np.pi)
    A, B = np.meshgrid(x, x, indexing="ij")
    WW = np.outer(w, w)
    return float((fun(A, B) * WW).sum())


def test_closed_form_equals_gaussian_kernel_convolution(oracle_lib):
    """Eq. 9 is the exact convolution of the unit Gaussian with N(0, Sigma_fp) in the
    ray-orthogonal plane (Assumption 3): compare with Gauss-Hermite quadrature."""
    rng = np.random.default_rng(2)
    cam = S.pinhole(64, 48, 12.0)     # coarse pixels: large footprint
    for _ in range(20):
        x, y, mu, ls, q = _random_pair(rng, cam)
        r = oracle_lib.pair(cam, x, y, mu, ls, q, 0.7)
        ex, ey, qv = r["ex"], r["ey"], r["q"]

        def fun(a, b):
            z = (a[..., None] * ex + b[..., None] * ey) / np.sqrt(3.0)
            return np.exp(-0.5 * ((qv - z) ** 2).sum(-1))

        ref = r["sig_eff"] * _gauss_hermite_2d(fun)
        assert abs(r["T"] - ref) <= 1e-10 * ref


def test_closed_form_vs_uniform_parallelogram(oracle_lib):
    """Against the uniform parallelogram average (the linearised Eq. 5), moment matching
    leaves an error of order |e|^4: the ratio err/|e|^4 stays bounded as e is halved."""
    o = np.zeros(3)
    mu = np.array([0.05, -0.02, 3.0])
    ls, q = np.log([0.05, 0.03, 0.04]), np.array([0.8, 0.3, 0.1, -0.5])
    d = np.array([0.0, 0.0, 1.0])
    ratios = []
    for h in (0.004, 0.002, 0.001, 0.0005):
        dx = np.array([h, 0.0, 0.0])
        dy = np.array([0.3 * h, 0.8 * h, 0.0])
        r = oracle_lib.pair_rays(o, d, dx, dy, mu, ls, q, 2.0)
        ex, ey, qv = r["ex"], r["ey"], r["q"]
        xg, wg = np.polynomial.legendre.leggauss(40)
        A, B = np.meshgrid(xg, xg, indexing="ij")
        z = A[..., None] * ex + B[..., None] * ey
        ref = r["sig_eff"] * float((np.exp(-0.5 * ((qv + z) ** 2).sum(-1)) * np.outer(wg, wg)).sum()) / 4.0
        e2 = max(ex @ ex, ey @ ey)
        ratios.append(abs(r["T"] - ref) / e2 ** 2)
    assert max(ratios) < 10 * min(ratios) + 1e-12
    assert ratios[-1] < 1.0


def test_centre_ray_limit(oracle_lib):
    """Footprint -> 0 (f -> inf): T -> sigma e^{-D^2/2} (Eq. 3 with C = 1), error O(|e|^2)."""
    mu = np.array([0.1, 0.05, 4.0])
    ls, q = np.log([0.05, 0.02, 0.08]), np.array([0.7, -0.2, 0.4, 0.1])
    errs = []
    for f in (100.0, 1000.0, 10000.0):
        cam = S.pinhole(64, 64, f, 32.0, 32.0)
        x = float(_project(cam, mu[None])[0][0]) + 0.3
        y = float(_project(cam, mu[None])[1][0]) - 0.2
        r = oracle_lib.pair(cam, x, y, mu, ls, q, 0.0)
        c = oracle_lib.pair(cam, x, y, mu, ls, q, 0.0, filter=oracle_lib.FILTER_NONE)
        assert abs(c["T"] - c["sig_eff"] * math.exp(-0.5 * c["D2"])) < 1e-15
        errs.append(abs(r["T"] - c["T"]) / c["T"])
    assert errs[1] < errs[0] / 50 and errs[2] < errs[1] / 50


def test_on_axis_worked_example(oracle_lib):
    g = GOLD["on_axis_isotropic_response"]
    f, s, z, sig = g["f"], g["s"], g["depth"], g["sigma"]
    cam = S.pinhole(65, 49, f, 32.5, 24.5)
    logit = math.log(sig / (1 - sig))
    r = oracle_lib.pair(cam, 32.5, 24.5, [0, 0, z], np.log([s, s, s]), [1, 0, 0, 0], logit)
    assert abs(r["ex"] @ r["ex"] - g["e2"]) < 1e-7
    assert abs(np.trace(r["Sfp"]) / 2 - g["lambda"]) < 1e-7
    assert abs(r["T"] - g["T"]) < 1e-7


def test_pinhole_matches_screen_space_ewa(oracle_lib):
    """Near the axis and for s/z -> 0, the ray-native footprint filter agrees with
    screen-space EWA with a (1/12) px^2 box-variance pixel filter (Sec. 4.1 closing remark)."""
    rels = []
    for scale in (0.02, 0.005, 0.00125):
        f = 400.0
        cam = S.pinhole(400, 400, f, 200.0, 200.0)
        z = 4.0
        s = np.array([scale, 0.6 * scale, 1.3 * scale]) * z
        q = np.array([0.9, 0.1, -0.3, 0.2])
        mu = np.array([0.01, -0.02, z])
        R = _rot(q)
        Sig = R @ np.diag(s ** 2) @ R.T
        J = np.array([[f / mu[2], 0, -f * mu[0] / mu[2] ** 2], [0, f / mu[2], -f * mu[1] / mu[2] ** 2]])
        S2 = J @ Sig @ J.T
        px = f * mu[0] / mu[2] + 200.0
        py = f * mu[1] / mu[2] + 200.0
        x, y = px + 0.7 * np.sqrt(S2[0, 0] + 1 / 12), py - 0.4 * np.sqrt(S2[1, 1] + 1 / 12)
        r = oracle_lib.pair(cam, x, y, mu, np.log(s), q, 0.0)
        Sf = S2 + np.eye(2) / 12
        dlt = np.array([x - px, y - py])
        ewa = r["sig_eff"] * math.sqrt(np.linalg.det(S2) / np.linalg.det(Sf)) * math.exp(-0.5 * dlt @ np.linalg.solve(Sf, dlt))
        rels.append(abs(r["T"] - ewa) / ewa)
    assert rels[-1] < 2e-2
    assert rels[2] < rels[0]


# ---------------------------------------------------------------- floor and marginal (Eq. 10-12)

def test_floor_identities(oracle_lib):
    """Eq. 10: s_eff^2 - s^2 = rho^2 per axis and sigma_eff prod s_eff = sigma prod s."""
    sc = S.uniform_box_scene(30, seed=4)
    rho2 = np.linspace(0, 2e-3, 30).astype(np.float32)
    sc = sc.with_rho2(rho2)
    cam = S.pinhole(64, 48, 60.0)
    G = oracle_lib.gauss(cam, sc)
    for i in range(30):
        W = G[i, :9].reshape(3, 3)
        seff = 1.0 / np.linalg.norm(W, axis=1)
        s = np.exp(sc.log_scales[i].astype(float))
        np.testing.assert_allclose(seff ** 2 - s ** 2, rho2[i], atol=1e-12)
        sig = 1 / (1 + math.exp(-float(sc.opacity_logits[i])))
        assert abs(G[i, 18] * np.prod(seff) - sig * np.prod(s)) < 1e-14
        np.testing.assert_allclose(G[i, 9:18].reshape(3, 3) @ W, np.eye(3), atol=1e-12)


def test_floor_on_axis_worked_example(oracle_lib):
    g = GOLD["on_axis_floor"]
    cam = S.pinhole(65, 49, g["f"], 32.5, 24.5)
    r = oracle_lib.floor_rho2([cam], np.array([[0.0, 0.0, g["t"]]]))
    assert abs(r[0] - g["rho2"]) < 1e-9


def test_floor_is_min_over_visible_views(oracle_lib):
    mu = np.array([[0.1, 0.0, 4.0], [0.0, 0.0, -3.0]])
    fine = S.pinhole(640, 480, 600.0)
    coarse = fine.scaled(0.25)
    r_f = oracle_lib.floor_rho2([fine], mu)
    r_c = oracle_lib.floor_rho2([coarse], mu)
    r_b = oracle_lib.floor_rho2([coarse, fine], mu)
    assert r_b[0] == min(r_f[0], r_c[0]) and r_f[0] < r_c[0]
    assert r_b[1] == 0.0   # behind every camera: never visible


def test_marginal_composition(oracle_lib):
    """Eq. 12: identity at rho = 0; Sigma_render <= Sigma_fp,eff; a Gaussian rendered by
    the view its floor came from gets no extra filtering; at 1/8 resolution (f/8) the
    world footprint is ~64 rho^2 per direction and the clamp keeps ~63 rho^2."""
    O = oracle_lib
    rng = np.random.default_rng(3)
    cam = S.pinhole(64, 48, 60.0)
    for _ in range(20):
        x, y, mu, ls, q = _random_pair(rng, cam)
        r0 = O.pair(cam, x, y, mu, ls, q, 0.1, 0.0)
        np.testing.assert_allclose(r0["Sr"], r0["Sfp"], atol=1e-12 * np.abs(r0["Sfp"]).max())
        rho2 = float(rng.uniform(0, 3e-4))
        r1 = O.pair(cam, x, y, mu, ls, q, 0.1, rho2)
        ev = np.linalg.eigvalsh(r1["Sfp"] - r1["Sr"])
        assert ev.min() >= -1e-12 * np.abs(r1["Sfp"]).max()
    # isotropic on-axis Gaussian, floor from the same camera
    cam = S.pinhole(65, 49, 60.0, 32.5, 24.5)
    mu = np.array([[0.0, 0.0, 4.0]])
    rho2 = float(O.floor_rho2([cam], mu)[0])
    r = O.pair(cam, 32.5, 24.5, mu[0], np.log([0.05] * 3), [1, 0, 0, 0], 0.0, rho2)
    assert np.abs(r["Sr"]).max() < 1e-12 * np.abs(r["Sfp"]).max()
    # same camera at 1/8 resolution
    cam8 = S.pinhole(9, 7, 60.0 / 8, 4.5, 3.5)
    r8 = O.pair(cam8, 4.5, 3.5, mu[0], np.log([0.05] * 3), [1, 0, 0, 0], 0.0, rho2)
    seff2 = 0.05 ** 2 + rho2
    world_r = r8["Sr"] * seff2        # isotropic: W^-1 Sigma W^-T = s_eff^2 Sigma
    world_f = r8["Sfp"] * seff2
    lam_r = np.sort(np.linalg.eigvalsh(world_r))[1:]
    lam_f = np.sort(np.linalg.eigvalsh(world_f))[1:]
    a = 1 / 120.0                     # half-pixel offset a = 1/(2f) at f = 60
    ratio = 64 * (1 + a * a) / (1 + 64 * a * a)   # |e|^2 ratio of the two calibrations
    np.testing.assert_allclose(lam_f / rho2, ratio, rtol=1e-6)
    np.testing.assert_allclose(lam_r / rho2, ratio - 1.0, rtol=1e-6)


# ---------------------------------------------------------------- compositing (Eq. 4)

def _single_gauss_scene(mus, logits, rgbs, s=0.05):
    n = len(mus)
    sh = ((np.asarray(rgbs, float) - 0.5) / S.SH_C0).reshape(n, 1, 3)
    return S.Scene(np.asarray(mus, np.float32), np.full((n, 3), math.log(s), np.float32),
                   np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)), np.asarray(logits, np.float32),
                   sh.astype(np.float32), 0, np.zeros(n, np.float32))


def test_composite_single_and_two(oracle_lib):
    O = oracle_lib
    cam = S.pinhole(65, 49, 60.0, 32.5, 24.5)
    p = 24 * 65 + 32
    sc = _single_gauss_scene([[0, 0, 4]], [0.4], [[0.2, 0.7, 0.9]])
    r = O.render(cam, sc, pix=[p], cull=False)
    ls32 = np.full(3, math.log(0.05), np.float32).astype(float)   # the scene stores FP32 values
    T1 = O.pair(cam, 32.5, 24.5, [0, 0, 4], ls32, [1, 0, 0, 0], float(np.float32(0.4)))["T"]
    col = sc.sh[0, 0].astype(float) * S.SH_C0 + 0.5     # stored (FP32) DC term -> colour
    np.testing.assert_allclose(r.rgb[0], col * T1, rtol=1e-12)
    assert abs(r.T[0] - (1 - T1)) < 1e-14
    sc2 = _single_gauss_scene([[0, 0, 5], [0, 0, 4]], [1.0, 0.4], [[1, 0, 0], [0, 0, 1]])
    r2 = O.render(cam, sc2, pix=[p], cull=False)
    a_far = O.pair(cam, 32.5, 24.5, [0, 0, 5], ls32, [1, 0, 0, 0], 1.0)["T"]
    c2 = np.maximum(sc2.sh[:, 0].astype(float) * S.SH_C0 + 0.5, 0.0)   # colour clamp at 0
    np.testing.assert_allclose(r2.rgb[0], c2[1] * T1 + c2[0] * a_far * (1 - T1), rtol=1e-12, atol=1e-15)


def test_composite_stop_rule(oracle_lib):
    """200 stacked alpha = 0.85 Gaussians: the walk stops before pair k once
    T_acc (1 - a_k) < 1e-4, i.e. after 4 contributions (0.15^5 < 1e-4 <= 0.15^4)."""
    O = oracle_lib
    cam = S.pinhole(65, 49, 60.0, 32.5, 24.5)
    n = 200
    z = 4 + 0.01 * np.arange(n)
    ls32 = float(np.float32(math.log(0.5)))
    T0 = np.array([O.pair(cam, 32.5, 24.5, [0, 0, zz], [ls32] * 3, [1, 0, 0, 0], 0.0)["T"] for zz in z])
    sig = 0.5 * 0.85 / T0                      # sigma such that T = 0.85 on the axis pixel
    sc = _single_gauss_scene(np.stack([np.zeros(n), np.zeros(n), z], 1), np.zeros(n), np.ones((n, 3)), s=0.5)
    sc.opacity_logits = np.log(sig / (1 - sig))
    r = O.render(cam, sc, pix=[24 * 65 + 32], cull=False)
    assert r.ncontrib[0] == 4
    assert abs(r.T[0] - 0.15 ** 4) < 1e-12
    assert r.flags[0] == 0


def test_cull_is_exact(oracle_lib):
    cam, sc = S.c1()
    a = oracle_lib.render(cam, sc, cull=False)
    b = oracle_lib.render(cam, sc, cull=True)
    assert np.array_equal(a.rgb, b.rgb) and np.array_equal(a.T, b.T)


# ---------------------------------------------------------------- Fig. 2 protocol

def test_fig2_anisotropic_beats_centre_ray_offaxis_fisheye(oracle_lib):
    """Single Gaussian vs the 32x32 supersampled pixel (Fig. 2(c,d)): off-axis fisheye
    pixels, the anisotropic footprint response has lower error than the centre ray."""
    O = oracle_lib
    cam = S.Camera(S.KB_FISHEYE, 96, 96, 30.0, 30.0, 48.0, 48.0, np.array([0.01, -0.004, 0.0, 0.0]),
                   theta_lim=1.55)
    rng = np.random.default_rng(7)
    wins, trials = 0, 0
    for _ in range(40):
        th = rng.uniform(math.radians(62), math.radians(80))
        ph = rng.uniform(0, 2 * math.pi)
        dist = rng.uniform(2, 4)
        mu = dist * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        px, py = _project(cam, mu[None])
        x, y = float(np.floor(px[0])) + 0.5, float(np.floor(py[0])) + 0.5
        s = dist * 0.6 / 30.0
        ls = np.log([s, 0.5 * s, 0.8 * s])
        q = rng.standard_normal(4)
        ref = O.bundle(cam, x, y, mu, ls, q, 1.0, nsub=32)
        if ref < 1e-3:
            continue
        an = O.pair(cam, x, y, mu, ls, q, 1.0)["T"]
        ce = O.pair(cam, x, y, mu, ls, q, 1.0, filter=O.FILTER_NONE)["T"]
        trials += 1
        wins += abs(an - ref) < abs(ce - ref)
    assert trials >= 20 and wins >= 0.8 * trials


# ---------------------------------------------------------------- isotropic footprint variants

@pytest.mark.parametrize("which", ["pinhole", "kb"])
@pytest.mark.parametrize("variant", ["iso", "zf"])
def test_isotropic_variants_closed_form(oracle_lib, which, variant):
    """An isotropic Gaussian (W = I/s) under a footprint isotropic across the ray
    (half-edge a b_i, b_i orthonormal across d): Sigma_fp^u = c M_perp with
    c = t*^2 a^2 / (3 s^2) (Eq. 6, 8), so A = I + c M_perp gives
    T = sigma / (1 + c) exp(-D^2 / (2 (1 + c))) (Eq. 9), with t* = <mu - o, d> and
    D the centre ray's distance over s.  a: the pixel's own differentials
    (iso: a^2 = (|dx_perp|^2 + |dy_perp|^2)/2) or the paraxial z/f size
    (zf: a = |<d, z_cam>| / (2 f_x))."""
    O = oracle_lib
    if which == "pinhole":
        cam = S.pinhole(160, 120, 90.0, 71.3, 66.2, cam_to_world=S.look_at((0.1, 0.0, -0.2), (0.6, 0.3, 4.0)))
    else:
        cam = S.c3_camera(128, 128)
        cam.cam_to_world = S.look_at((0.0, 0.1, 0.0), (0.4, -0.2, 3.0))
    R = cam.cam_to_world[:, :3].astype(float)
    o = cam.cam_to_world[:, 3].astype(float)
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(30):
        x, y = rng.uniform(5, cam.width - 5), rng.uniform(5, cam.height - 5)
        d, dx, dy, valid = O.rays(cam, np.array([x]), np.array([y]))
        if not valid[0]:
            continue
        d, dx, dy = d[0], dx[0], dy[0]
        t_true = rng.uniform(2.0, 5.0)
        s = rng.uniform(0.01, 0.05)
        mu = o + t_true * d + rng.normal(0, 1.5 * s, 3)
        logit = 0.7
        p = O.pair(cam, x, y, mu, np.log([s, s, s]), [1.0, 0.0, 0.0, 0.0], logit,
                   filter=O.FILTER_ISO if variant == "iso" else O.FILTER_ZF, comp=O.COMP_ADDITIVE)
        v = mu - o
        ts = float(v @ d)
        D2 = float((v - ts * d) @ (v - ts * d)) / s ** 2
        if variant == "iso":
            px, py = dx - (d @ dx) * d, dy - (d @ dy) * d
            a2 = 0.5 * (px @ px + py @ py)
        else:
            a2 = float(d @ R[:, 2]) ** 2 / (4.0 * cam.fx ** 2)
        c = ts ** 2 * a2 / (3.0 * s ** 2)
        sig = 1.0 / (1.0 + math.exp(-logit))
        want = sig / (1.0 + c) * math.exp(-0.5 * D2 / (1.0 + c))
        # the camera's rotation is stored in FP32, so its rays are unit to ~1e-7
        assert abs(p["T"] - want) <= 1e-6 * want + 1e-300, (p["T"], want)
        checked += 1
    assert checked >= 15


def test_zf_sizing_over_dilates_offaxis_pinhole(oracle_lib):
    """Pinhole: a pixel at angle theta from the axis spans cos^2(theta)/f radially
    and cos(theta)/f tangentially, so the paraxial z/f size (cos(theta)/f on both
    axes) exceeds the true footprint's isotropic reduction off axis and matches
    it on axis (to O(1/f^2))."""
    O = oracle_lib
    cam = S.pinhole(801, 601, 300.0, 400.5, 300.5)
    xs = np.array([400.5, 500.5, 650.5, 790.5])
    ys = np.array([300.5, 300.5, 420.5, 590.5])
    d, dx, dy, _ = O.rays(cam, xs, ys)
    a_iso, a_zf = [], []
    for k in range(len(xs)):
        px, py = dx[k] - (d[k] @ dx[k]) * d[k], dy[k] - (d[k] @ dy[k]) * d[k]
        a_iso.append(math.sqrt(0.5 * (px @ px + py @ py)))
        a_zf.append(abs(d[k][2]) / (2.0 * cam.fx))
    assert abs(a_zf[0] - a_iso[0]) <= 1e-4 * a_iso[0]
    ratio = np.array(a_zf) / np.array(a_iso)
    assert np.all(np.diff(ratio) > 0) and ratio[-1] > 1.1


def test_fig2_variant_errors_against_supersampled_pixel(oracle_lib):
    """Fig. 2(c,d) error study over the filter variants: single anisotropic
    Gaussians seen by a fisheye, responses against the 32x32 supersampled pixel
    at three eccentricity bands.  The anisotropic footprint has the lowest mean
    error in every band; the centre ray and the paraxial z/f sizing are far
    worse, z/f increasingly so off axis; the isotropic reduction trails the
    anisotropic footprint where footprints shear (the outer band)."""
    O = oracle_lib
    cam = S.Camera(S.KB_FISHEYE, 96, 96, 30.0, 30.0, 48.0, 48.0, np.array([0.01, -0.004, 0.0, 0.0]),
                   theta_lim=1.55)
    rng = np.random.default_rng(7)
    means = {}
    for band in ((0, 30), (30, 62), (62, 80)):
        err = {k: [] for k in ("centre", "zf", "iso", "aniso")}
        for _ in range(40):
            th = rng.uniform(math.radians(band[0]), math.radians(band[1]))
            ph = rng.uniform(0, 2 * math.pi)
            dist = rng.uniform(2, 4)
            mu = dist * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            px, py = _project(cam, mu[None])
            x, y = float(np.floor(px[0])) + 0.5, float(np.floor(py[0])) + 0.5
            s = dist * 0.6 / 30.0
            ls = np.log([s, 0.5 * s, 0.8 * s])
            q = rng.standard_normal(4)
            ref = O.bundle(cam, x, y, mu, ls, q, 1.0, nsub=32)
            if ref < 1e-3:
                continue
            for k, f in (("centre", O.FILTER_NONE), ("zf", O.FILTER_ZF), ("iso", O.FILTER_ISO),
                         ("aniso", O.FILTER_ANISO)):
                err[k].append(abs(O.pair(cam, x, y, mu, ls, q, 1.0, filter=f)["T"] - ref) / ref)
        assert len(err["aniso"]) >= 25
        means[band] = {k: float(np.mean(v)) for k, v in err.items()}
    for band, m in means.items():
        assert m["aniso"] < m["zf"] and m["aniso"] < m["centre"] and m["aniso"] <= m["iso"] * 1.02, (band, m)
    assert means[(62, 80)]["aniso"] < 0.9 * means[(62, 80)]["iso"]
    assert means[(62, 80)]["zf"] > 2.0 * means[(0, 30)]["zf"]


# ---------------------------------------------------------------- order and multi-Gaussian references

def test_per_ray_order_two_gaussians(oracle_lib):
    """Two Gaussians: a wide one whose centre is farther but which the ray meets
    first (its max-response depth t* along the ray is smaller) and a small one on
    the axis.  Canonical key order composites by |mu - o|;
    the per-ray order by each pair's t* (Eq. 4 in either order, closed form)."""
    O = oracle_lib
    cam = S.pinhole(9, 9, 8.0)
    # A: small, on axis at depth 3.  B: a wide sheet thin along z at z = 2.6 whose
    # centre sits off axis (|mu_B| > |mu_A|); the ray meets the sheet at t* ~ 2.6
    means = np.array([[0.0, 0.0, 3.0], [2.0, 0.0, 2.6]], np.float32)
    ls = np.log(np.array([[0.05, 0.05, 0.05], [1.2, 1.2, 0.02]], np.float32))
    quats = np.array([[1, 0, 0, 0], [1, 0, 0, 0]], np.float64)
    sc = S.Scene(means, ls.astype(np.float32), quats, np.array([0.4, 0.9], np.float32),
                 np.zeros((2, 1, 3), np.float32), 0, np.zeros(2, np.float32))
    sc.sh[0, 0, :] = (np.array([0.9, 0.1, 0.1]) - 0.5) / S.SH_C0
    sc.sh[1, 0, :] = (np.array([0.1, 0.1, 0.9]) - 0.5) / S.SH_C0
    pix = 4 * 9 + 4                       # the centre pixel: its ray is the optical axis
    a = O.render(cam, sc, pix=[pix], filter=O.FILTER_NONE, order=0, eps=0.0)
    b = O.render(cam, sc, pix=[pix], filter=O.FILTER_NONE, order=1, eps=0.0)
    x, y = 4.5, 4.5
    d, _, _, _ = O.rays(cam, np.array([x]), np.array([y]))
    d = d[0]
    al, ts, col = [], [], []
    for k in range(2):
        p = O.pair(cam, x, y, means[k], ls[k], quats[k], float(sc.opacity_logits[k]), filter=O.FILTER_NONE)
        al.append(min(p["T"], 0.99))
        ts.append(p["ts"])
    col = [np.array([0.9, 0.1, 0.1]), np.array([0.1, 0.1, 0.9])]
    assert np.linalg.norm(means[0]) < np.linalg.norm(means[1]) and ts[1] < ts[0] and min(al) > 1 / 255
    key = col[0] * al[0] + col[1] * al[1] * (1 - al[0])
    ray = col[1] * al[1] + col[0] * al[0] * (1 - al[1])
    assert np.allclose(a.rgb[0], key, atol=1e-12) and np.allclose(b.rgb[0], ray, atol=1e-12)
    assert np.abs(key - ray).max() > 0.05


def test_subray_reference_single_gaussian_is_bundle(oracle_lib):
    """For one Gaussian (all sub-ray alphas inside [1/255, 0.99)) the dense sub-ray
    reference is its colour times the supersampled response of or_bundle."""
    O = oracle_lib
    cam = S.c3_camera(40, 40)
    mu, ls, q = np.array([0.5, 0.3, 2.5]), np.log([0.06, 0.03, 0.05]), np.array([0.9, 0.1, 0.3, 0.2])
    sc = S.Scene(mu[None].astype(np.float32), ls[None].astype(np.float32), q[None], np.array([-1.0], np.float32),
                 np.zeros((1, 1, 3), np.float32), 0, np.zeros(1, np.float32))
    sc.sh[0, 0, :] = (np.array([0.7, 0.4, 0.2]) - 0.5) / S.SH_C0
    px, py = _project(cam, mu[None])
    i, j = int(px[0]), int(py[0])
    rgb, T = O.render_subrays(cam, sc, pix=[j * cam.width + i], nsub=8)
    b = O.bundle(cam, i + 0.5, j + 0.5, sc.means[0], sc.log_scales[0], q, -1.0, nsub=8)
    assert 1 / 255 < b < 0.2
    assert np.allclose(rgb[0], np.array([0.7, 0.4, 0.2]) * b, rtol=1e-9)
    assert abs(T[0] - (1 - b)) < 1e-9


def test_order_and_subray_studies(oracle_lib):
    """NEXT-3 quantification on three synthetic scenes (C1; a close-up of large
    overlapping Gaussians; a fisheye inside a shell): (i) the canonical key vs
    the exact per-ray t* order; (ii) each filter's render against the 8x8 dense
    sub-ray reference (same order) at native resolution and at 1/4.  Asserted:
    the centre ray is the worst filter in every case and the anisotropic footprint
    is within 10% of the best; the order effect is largest for the overlapping
    close-up."""
    O = oracle_lib
    cases = {"c1": S.c1(),
             "overlap": (S.pinhole(48, 36, 40.0),
                         S.uniform_box_scene(400, seed=3, log_scale_mean=-1.6, log_scale_std=0.4, sh_degree=1)),
             "fisheye": (S.c3_camera(48, 48),
                         S.blob_scene(2000, seed=5, cam=S.pinhole(48, 48, 30.0), blob_frac=0.3, shell=(1.5, 4.0),
                                      log_scale_mean=-2.5, sh_degree=1))}
    order_err = {}
    for name, (cam, sc) in cases.items():
        a = O.render(cam, sc, order=0, eps=0.0)
        b = O.render(cam, sc, order=1, eps=0.0)
        order_err[name] = float(np.abs(a.rgb - b.rgb).mean())
        for scale in (1.0, 0.25):
            c2 = cam.scaled(scale) if scale < 1 else cam
            ref, _ = O.render_subrays(c2, sc, nsub=8)
            err = {}
            for k, f in (("centre", O.FILTER_NONE), ("zf", O.FILTER_ZF), ("iso", O.FILTER_ISO),
                         ("aniso", O.FILTER_ANISO)):
                err[k] = float(np.abs(O.render(c2, sc, filter=f, eps=0.0).rgb - ref).mean())
            assert err["centre"] == max(err.values()), (name, scale, err)
            assert err["aniso"] <= 1.1 * min(err["zf"], err["iso"]), (name, scale, err)
    assert order_err["overlap"] == max(order_err.values()) and order_err["overlap"] > 5 * order_err["c1"]


def _world_space_response(o, d, dx, dy, mu, log_scales, quat, logit):
    """Eq. 9 written in world space, with no whitening, in 50-digit arithmetic: with
    Sigma = R S^2 R^T, the max-response depth t* = d^T Sigma^-1 (mu - o) / d^T Sigma^-1 d,
    the world half-edges t* (delta_i - d (d^T Sigma^-1 delta_i) / d^T Sigma^-1 d) (Eq. 6
    mapped back by W^-1) and F their moment-matched covariance (Eq. 8),
        det A = det(Sigma + F) / det Sigma,  q^T A^-1 q = r^T (Sigma + F)^-1 r,
    r = o + t* d - mu (from W^T W = Sigma^-1)."""
    import mpmath as mp
    mp.mp.dps = 50
    v = lambda a: mp.matrix([mp.mpf(float(x)) for x in np.asarray(a).reshape(-1)])
    q = [mp.mpf(float(x)) for x in quat]
    nq = mp.sqrt(sum(x * x for x in q))
    w, x, y, z = [c / nq for c in q]
    R = mp.matrix([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                   [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                   [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    s2 = [mp.e ** (2 * mp.mpf(float(c))) for c in log_scales]
    Sig = R * mp.diag(s2) * R.T
    Sinv = R * mp.diag([1 / c for c in s2]) * R.T
    D, O, MU = v(d), v(o), v(mu)
    Sd = Sinv * D
    dSd = (D.T * Sd)[0]
    ts = (Sd.T * (MU - O))[0] / dSd
    F = mp.zeros(3, 3)
    for dl in (v(dx), v(dy)):
        e = ts * (dl - D * ((Sd.T * dl)[0] / dSd))
        F += e * e.T / 3
    r = O + ts * D - MU
    M = Sig + F
    sig = 1 / (1 + mp.e ** (-mp.mpf(float(logit))))
    return float(sig * mp.sqrt(mp.det(Sig) / mp.det(M)) * mp.e ** (-(r.T * mp.inverse(M) * r)[0] / 2))


@pytest.mark.parametrize("kind,pose", [("pinhole", (80.0, 89.5)), ("pinhole", (0.0, 30.0)), ("kb", (0.0, 30.0)),
                                       ("kb", (80.0, 89.5))])
def test_flat_gaussians_world_space_form(oracle_lib, kind, pose):
    """Near-degenerate flat Gaussians (s_max/s_min = 10^4): the oracle's whitened
    FP64 response (Eq. 9 with Eq. 12 at rho = 0) against the world-space form of the
    same equation, which never forms the 1/s_min whitening, evaluated in 50 digits,
    on the pixels around each Gaussian; it stays finite and at most sigma (det A >= 1).
    The literal 3x3 route of Eq. 12 (whiten, clamp, re-whiten) loses digits when the
    whitened footprint is huge (up to ~1e-3 relative at grazing angles, where
    det A ~ 1e9), but only on pairs whose response is then small: the absolute error
    stays below 2e-6, 50x inside the 1e-4 parity tolerance."""
    cam = S.pinhole(96, 72, 90.0) if kind == "pinhole" else S.c3_camera(96, 96)
    sc = S.flat_scene(30, seed=5, ratio=1e4, tilt_deg=pose, cam=cam, fov_deg=25.0 if kind == "pinhole" else 85.0)
    d, dx, dy, valid = oracle_lib.rays(cam)
    o = cam.cam_to_world[:, 3].astype(np.float64)
    vidx = np.nonzero(valid)[0]
    checked = 0
    for k in range(sc.n):
        u = sc.means[k].astype(np.float64) - o
        near = vidx[np.argsort(-(d[vidx] @ (u / np.linalg.norm(u))))[:80]]   # pixels around the Gaussian
        for p in near:
            r = oracle_lib.pair(cam, p % cam.width + 0.5, p // cam.width + 0.5, sc.means[k], sc.log_scales[k],
                                sc.quats[k], float(sc.opacity_logits[k]))
            if r is None or not r["valid_depth"]:
                continue
            assert np.isfinite(r["T"]) and 0.0 <= r["T"] <= r["sig_eff"] * (1 + 1e-12)
            if r["T"] < 1e-5:
                continue
            want = _world_space_response(o, d[p], dx[p], dy[p], sc.means[k], sc.log_scales[k], sc.quats[k],
                                         float(sc.opacity_logits[k]))
            assert abs(r["T"] - want) <= 2e-6 + 1e-9 * want, (k, p, r["T"], want)
            checked += 1
    assert checked > 250


def test_render_nalpha_and_tstar_tie_flag(oracle_lib):
    """nalpha counts every pair with T >= 1/255: where no pixel stops (C1 scene, T
    stays above 1e-4), that is exactly the pairs composited, in either order.  In
    the per-ray order, stacked Gaussians (identical t*) raise the tie flag; well
    separated ones do not."""
    O = oracle_lib
    cam, sc = S.c1()
    for order in (0, 1):
        r = O.render(cam, sc, order=order, eps=0.0)
        assert (r.T > 1e-3).all()
        assert np.array_equal(r.nalpha, r.ncontrib)
    cam = S.pinhole(16, 16, 20.0)

    def stack(z):
        n = len(z)
        return S.Scene(means=np.array([[0.0, 0.0, zz] for zz in z], np.float32),
                       log_scales=np.full((n, 3), np.log(0.3), np.float32),
                       quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                       opacity_logits=np.zeros(n, np.float32), sh=np.zeros((n, 1, 3), np.float32), sh_degree=0,
                       rho2=np.zeros(n, np.float32))
    c = 8 * 16 + 8
    tie = O.render(cam, stack([3.0, 3.0]), pix=[c], order=1, eps=0.0, eps_key=1e-6)
    sep = O.render(cam, stack([3.0, 3.5]), pix=[c], order=1, eps=0.0, eps_key=1e-6)
    assert tie.flags[0] & O.FL_KEY_TIE and not sep.flags[0] & O.FL_KEY_TIE
    assert tie.nalpha[0] == 2 and sep.nalpha[0] == 2

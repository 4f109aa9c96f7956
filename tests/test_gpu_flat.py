"""Near-degenerate flat Gaussians (disks with s_max/s_min from 60 to 10^4, seen
face-on and at grazing angles) through a pinhole and a Kannala-Brandt fisheye.

Their whitening W_eff has a row of length 1/s_min (Sec. 3), so the closed-form
response of Eq. 9 cancels in FP32: the library evaluates Gaussians with an
effective scale ratio above 200 in FP64 (the footprint-convolved covariance's
inverse and determinant, with t*, q and e_i feeding them) and the rest in FP32
through an orthonormal basis of the footprint.  The image must match the FP64
oracle within 1e-4 either way, the pair counts bit for bit, and the profiled
counters must show which path ran."""
import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
EPS_FLAG = 2e-4
POSES = {"face_on": (0.0, 30.0), "grazing": (80.0, 89.5)}
FLAT_RATIO = 200.0   # the library's FP64 threshold on s_eff,max / s_eff,min


@pytest.fixture(scope="module")
def cg():
    import paper_2609_13397_b300 as cg
    return cg


def _camera(kind):
    return S.pinhole(96, 72, 90.0) if kind == "pinhole" else S.c3_camera(96, 96)


def _scene(kind, ratio, pose, floor=False, seed=1):
    cam = _camera(kind)
    sc = S.flat_scene(300, seed=seed, ratio=ratio, tilt_deg=POSES[pose], cam=cam,
                      fov_deg=25.0 if kind == "pinhole" else 85.0)
    if floor:   # a floor as large as the thin scale: Eq. 10 dilates it, Eq. 12's clamp is active
        sc = sc.with_rho2(np.exp(2.0 * sc.log_scales.min(1)).astype(np.float32))
    return cam, sc


@pytest.mark.parametrize("kind", ["pinhole", "kb"])
@pytest.mark.parametrize("ratio", [60.0, 150.0, 400.0, 1e3, 1e4])
@pytest.mark.parametrize("pose", list(POSES))
def test_flat_gaussians_match_oracle(cg, oracle_lib, kind, ratio, pose):
    cam, sc = _scene(kind, ratio, pose)
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v = ctx.view()
    v.set_camera_from(cam)
    rgb, T = v.render(flags=cg.PROFILE)
    st = v.stats()
    rgb = rgb.cpu().numpy().reshape(3, -1).T
    T = T.cpu().numpy().reshape(-1)
    r = oracle_lib.render(cam, sc, eps=EPS_FLAG)
    ok = r.flags == 0
    assert ok.mean() > 0.95
    assert (r.ncontrib > 0).mean() > (0.2 if kind == "pinhole" else 0.08)   # the disks cover the image
    err = np.abs(rgb - r.rgb)[ok].max()
    errT = np.abs(T - r.T)[ok].max()
    assert err <= TOL and errT <= TOL, (err, errT)
    if ratio * 1.02 > FLAT_RATIO:       # flat_scene draws the ratio as ratio x U(1.02, 1.3)
        assert st["n_evaluated_flat"] > 0 and st["n_evaluated_flat"] == st["n_evaluated"]
    elif ratio * 1.3 < FLAT_RATIO:
        assert st["n_evaluated_flat"] == 0
    pg, pt = (t.cpu().numpy() for t in v.bin_counts())
    total, opg, opt, _ = oracle_lib.bin_counts(cam, sc)
    assert np.array_equal(pg, opg) and np.array_equal(pt, opt)


@pytest.mark.parametrize("kind", ["pinhole", "kb"])
def test_flat_gaussians_with_floor_match_oracle(cg, oracle_lib, kind):
    """A floor rho^2 = s_min^2 (ratio 10^4 -> ~7000 after Eq. 10): the marginal
    rule (Eq. 12) clamps the footprint in FP64."""
    cam, sc = _scene(kind, 1e4, "grazing", floor=True, seed=3)
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v = ctx.view()
    v.set_camera_from(cam)
    rgb, T = v.render(flags=cg.PROFILE)
    assert v.stats()["n_evaluated_flat"] > 0
    r = oracle_lib.render(cam, sc, eps=EPS_FLAG)
    ok = r.flags == 0
    assert ok.mean() > 0.95
    assert np.abs(rgb.cpu().numpy().reshape(3, -1).T - r.rgb)[ok].max() <= TOL
    assert np.abs(T.cpu().numpy().reshape(-1) - r.T)[ok].max() <= TOL

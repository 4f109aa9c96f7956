"""The rasteriser's pre-test in its two forms, and against no pre-test at all.

The pre-test skips pixel/Gaussian pairs that cannot reach alpha >= 1/255 and
changes no result.  On pinhole views the library tests each pixel centre
against the ellipse that the Gaussian's visual cone cuts from the image plane;
CONEGS_PRETEST_RAY asks for the ray-direction form instead (the only form on
fisheye views).  Both forms are conservative, so a render is bitwise the same
either way: colour, transmittance and the adjoint's per-pixel state.  The
gradients agree up to the order of their atomic sums.  CONEGS_PRETEST_OFF
evaluates every listed pair: a render equal to it bit for bit shows that the
pre-test's bounds (the footprint's largest and smallest eigenvalues over the
pixels a Gaussian can reach, the dilution of the peak, the bounds on t*) drop
no contributing pair.  The GPU renders are also checked against the FP64
oracle elsewhere, with the pixel form as the default.
"""
import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import paper_2609_13397_b300 as cg
    return cg


def _cases():
    from test_binning_rule import _random_case
    out = {"c1": S.c1()}
    bcam = S.pinhole(320, 180, 300.0)
    out["blob320"] = (bcam, S.blob_scene(20000, seed=1, cam=bcam))
    out["ragged"] = (S.pinhole(70, 45, 40.0, 33.0, 21.0, cam_to_world=S.look_at((0.1, 0.0, -0.5), (0.2, 0.1, 4.0))),
                     S.uniform_box_scene(500, seed=9, log_scale_mean=-2.5))
    wcam = S.Camera(S.PINHOLE, 96, 64, 30.0, 36.0, 50.5, 30.25,
                    cam_to_world=S.look_at((0.0, 0.1, 0.0), (1.0, 0.4, 2.0)))
    out["wide_surround"] = (wcam, S.blob_scene(3000, seed=13, cam=wcam, blob_frac=0.3, shell=(1.5, 4.0),
                                               log_scale_mean=-2.5, sh_degree=1))
    lcam = S.pinhole(24, 20, 19.0, cam_to_world=S.look_at((0.1, -0.2, 0.0), (0.4, 0.3, 2.0)))
    out["lowres_close"] = (lcam, S.blob_scene(1500, seed=31, cam=lcam, blob_frac=0.3, shell=(0.3, 3.0),
                                              log_scale_mean=-2.2, log_scale_std=1.5, sh_degree=1))
    for seed in (0, 2, 4, 6):                       # the pinhole ones among the random cases
        out[f"random{seed}"] = _random_case(seed)
    fcam = S.pinhole(96, 72, 90.0)
    for ratio in (60.0, 1e3, 1e4):
        for pose, tilt in (("face_on", (0.0, 30.0)), ("grazing", (80.0, 89.5))):
            out[f"flat{int(ratio)}_{pose}"] = (fcam, S.flat_scene(300, seed=1, ratio=ratio, tilt_deg=tilt, cam=fcam,
                                                                  fov_deg=25.0))
    return out


CASES = _cases()


def _render(cg, cam, sc, flags, rho2=None):
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, rho2=rho2)
    v = ctx.view()
    v.set_camera_from(cam)
    rgb, T = v.render(flags=flags | cg.PROFILE | cg.KEEP_FOR_BACKWARD)
    st = v.stats()
    g = v.render_backward(torch.ones_like(rgb), torch.full_like(T, 0.5))
    torch.cuda.synchronize()
    out = (rgb.cpu(), T.cpu(), {k: t.cpu() for k, t in g.items()}, st)
    ctx.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_pixel_and_ray_pretest_render_the_same(cg, name):
    cam, sc = CASES[name]
    rgb_p, T_p, g_p, st_p = _render(cg, cam, sc, 0)
    rgb_r, T_r, g_r, st_r = _render(cg, cam, sc, cg.PRETEST_RAY)
    assert torch.equal(rgb_p, rgb_r) and torch.equal(T_p, T_r)
    assert st_p["n_walked"] == st_r["n_walked"] and st_p["n_pairs"] == st_r["n_pairs"]
    assert st_p["n_evaluated"] > 0 or float(T_p.min()) == 1.0
    for k in g_p:                                   # equal up to the order of the atomic sums
        a, b = g_p[k], g_r[k]
        bound = 1e-5 * float(b.abs().max()) + 1e-4 * b.abs()
        assert bool(((a - b).abs() <= bound).all()), (k, float((a - b).abs().max()))


def test_pixel_pretest_on_c2_low_resolution_view(cg):
    """The benchmark's 160x90 view of the 500k-Gaussian scene (Eq. 11 floor from the
    1280x720 view): the same image with either form, and the pixel form evaluates no
    more pairs than the lists hold."""
    cams, sc = S.c2_cameras(), S.c2_scene()
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v0 = ctx.view()
    v0.set_camera_from(cams[0])
    rho2 = ctx.compute_floor([v0])
    ctx.close()
    outs = []
    for flags in (0, cg.PRETEST_RAY):
        ctx = cg.Context(0)
        ctx.set_scene_from(sc, rho2=rho2)
        v = ctx.view()
        v.set_camera_from(cams[1])
        rgb, T = v.render(flags=flags | cg.PROFILE)
        st = v.stats()
        outs.append((rgb.cpu(), T.cpu(), st))
        ctx.close()
    (a, ta, sa), (b, tb, sb) = outs
    assert torch.equal(a, b) and torch.equal(ta, tb)
    assert 0 < sa["n_evaluated"] <= sa["n_walked"] and 0 < sb["n_evaluated"] <= sb["n_walked"]


def _off_cases():
    """Views where the pre-test's footprint bounds bite: low-resolution views of
    scenes floored (Eq. 11) at a much sharper view, fisheyes whose footprint
    varies strongly from axis to rim, a zoomed-out fisheye and a wide pinhole."""
    from test_binning_rule import _random_case
    full = S.c4_rig()[0]                                  # 1920x1080 pinhole: the floor's view
    rig = S.c4_rig(scale_list=(0.125, 0.0625, 0.125, 0.0625))
    blobs = S.blob_scene(30000, seed=5, cam=full, shell=(2.0, 9.0))
    out = [(f"rig{k}", cam, blobs, full, 0) for k, cam in enumerate(rig)]
    kb = rig[4]
    for name, fl in (("iso", cg_flag("FILTER_ISO")), ("additive", cg_flag("COMP_ADDITIVE")),
                     ("zf", cg_flag("FILTER_ZF")), ("none", cg_flag("FILTER_NONE"))):
        out.append((f"kb240_{name}", kb, blobs, full, fl))
    box = S.uniform_box_scene(20000, seed=2, log_scale_mean=-3.5)
    out.append(("c3_256", S.c3_camera(256, 256), box, None, 0))
    k = np.random.default_rng(7).uniform(-0.05, 0.05, 4)
    look = S.look_at((0.0, 0.0, 0.0), (0.1, 0.2, 4.0))
    out.append(("kb_zoom_out", S.kb_fisheye(200, 150, k, zoom=0.5, cam_to_world=look), box,
                S.pinhole(800, 600, 700.0, cam_to_world=look), 0))
    out.append(("wide_pinhole", S.pinhole(200, 150, 40.0, cam_to_world=look), box,
                S.pinhole(800, 600, 700.0, cam_to_world=look), 0))
    for seed in (1, 3, 5):
        cam, sc = _random_case(seed)
        out.append((f"random{seed}", cam, sc, None, 0))
    return out


def cg_flag(name):
    import paper_2609_13397_b300 as cg
    return getattr(cg, name)


OFF_CASES = {c[0]: c[1:] for c in _off_cases()}


@pytest.mark.parametrize("name", list(OFF_CASES))
def test_pretest_drops_no_contributing_pair(cg, name):
    cam, sc, floor_cam, flags = OFF_CASES[name]
    rho2 = None
    if floor_cam is not None:
        ctx = cg.Context(0)
        ctx.set_scene_from(sc)
        vf = ctx.view()
        vf.set_camera_from(floor_cam)
        rho2 = ctx.compute_floor([vf])
        ctx.close()
    keep = cg.KEEP_FOR_BACKWARD
    outs = []
    for f in (flags, flags | cg.PRETEST_OFF):
        ctx = cg.Context(0)
        ctx.set_scene_from(sc, rho2=rho2)
        v = ctx.view()
        v.set_camera_from(cam)
        rgb, T = v.render(flags=f | cg.PROFILE | keep)
        st = v.stats()
        g = v.render_backward(torch.ones_like(rgb), torch.full_like(T, 0.5))
        torch.cuda.synchronize()
        outs.append((rgb.cpu(), T.cpu(), {k: t.cpu() for k, t in g.items()}, st))
        ctx.close()
    (rgb_a, T_a, g_a, st_a), (rgb_b, T_b, g_b, st_b) = outs
    assert torch.equal(rgb_a, rgb_b) and torch.equal(T_a, T_b)
    assert st_a["n_walked"] == st_b["n_walked"] and st_a["n_pairs"] == st_b["n_pairs"]
    # without the pre-test every walked entry is evaluated up to the pixel's stop
    # (walked counts whole staged batches, so a pixel that stops mid-batch has
    # walked a few entries more)
    assert st_a["n_evaluated"] <= st_b["n_evaluated"] <= st_b["n_walked"]
    # the same per-pair contributions, summed by atomics in a run-dependent order:
    # FP32 rounding of long sums with cancellation, at the scale of the largest entry
    for k in g_a:
        a, b = g_a[k], g_b[k]
        bound = 1e-4 * float(b.abs().max()) + 1e-4 * b.abs()
        assert bool(((a - b).abs() <= bound).all()), (k, float((a - b).abs().max()))

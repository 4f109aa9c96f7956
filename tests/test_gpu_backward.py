"""GPU adjoint (conegs_render_backward) vs the FP64 gradient oracle (oracle/grad.py,
itself pinned to finite differences of the C oracle), entry by entry.  Loss
L = sum w_rgb . rgb + w_T . T with seeded weights; pixels the oracle flags as
near a compositing threshold get zero weight (the render is not
differentiable there)."""
import dataclasses

import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# element-wise bound of the FP32 adjoint against the FP64 gradient oracle:
# |g - g_ref| <= ABS * max|g_ref| + REL * |g_ref| on every entry of every group
REL = 2e-3
ABS = 1e-5


def assert_grads_close(got: dict, want: dict, names=(("means", "means"), ("log_scales", "log_scales"),
                                                     ("quats", "quats"), ("opacity_logits", "logits"),
                                                     ("sh", "sh")), rel=REL, abs_=ABS):
    for gk, ok in names:
        g = np.asarray(got[gk], np.float64).reshape(want[ok].shape)
        w = want[ok]
        bound = abs_ * np.abs(w).max() + rel * np.abs(w)
        excess = np.abs(g - w) - bound
        worst = int(np.argmax(excess))
        assert excess.max() <= 0.0, (gk, worst, float(g.reshape(-1)[worst]), float(w.reshape(-1)[worst]),
                                     float(np.abs(w).max()))


@pytest.fixture(scope="module")
def cg():
    import paper_2609_13397_b300 as cg
    return cg


def _case(name):
    if name == "pinhole":
        cam = S.pinhole(40, 30, 36.0, cam_to_world=S.look_at((0.05, 0.0, 0.0), (0.1, 0.05, 4.0)))
        sc = S.uniform_box_scene(150, seed=2, log_scale_mean=-2.6, log_scale_std=0.4, sh_degree=1)
    elif name == "floor":
        cam = S.pinhole(40, 30, 36.0, cam_to_world=S.look_at((0.05, 0.0, 0.0), (0.1, 0.05, 4.0)))
        sc = S.uniform_box_scene(150, seed=4, log_scale_mean=-3.2, log_scale_std=0.5, sh_degree=2)
        import oracle
        sc = sc.with_rho2(oracle.floor_rho2([S.pinhole(160, 120, 144.0)], sc.means).astype(np.float32))
    elif name == "coarse_floor":       # footprints well above the floor: the marginal rule is active
        cam = S.pinhole(20, 15, 18.0, cam_to_world=S.look_at((0.0, 0.05, 0.0), (0.0, 0.0, 4.0)))
        sc = S.uniform_box_scene(150, seed=6, log_scale_mean=-3.0, log_scale_std=0.6, sh_degree=3)
        import oracle
        sc = sc.with_rho2(oracle.floor_rho2([S.pinhole(80, 60, 72.0)], sc.means).astype(np.float32))
    elif name == "flat":               # near-degenerate disks (s_max/s_min ~ 10^3), adjoint in FP64
        cam = S.pinhole(40, 30, 36.0)
        sc = S.flat_scene(150, seed=8, ratio=1e3, tilt_deg=(0.0, 89.0), cam=cam, fov_deg=25.0)
    elif name == "anisotropic":        # s_max/s_min ~ 100 at all angles: FP32, through the orthonormal basis
        cam = S.pinhole(40, 30, 36.0)
        sc = S.flat_scene(150, seed=9, ratio=100.0, tilt_deg=(0.0, 89.5), cam=cam, fov_deg=25.0,
                          log_scale_mean=-3.5)
    else:                              # fisheye
        cam = S.c3_camera(48, 48)
        sc = S.uniform_box_scene(150, seed=5, log_scale_mean=-2.4, log_scale_std=0.4, sh_degree=1)
    return cam, sc


@pytest.mark.parametrize("name,mode", [("pinhole", "aniso"), ("floor", "aniso"), ("coarse_floor", "aniso"),
                                       ("fisheye", "aniso"), ("flat", "aniso"), ("anisotropic", "aniso"),
                                       ("pinhole", "filter_none"),
                                       ("coarse_floor", "additive"), ("coarse_floor", "iso"), ("fisheye", "zf")])
def test_backward_matches_gradient_oracle(cg, oracle_lib, name, mode):
    from oracle import grad as G
    cam, sc = _case(name)
    filt = mode != "filter_none"
    add = mode == "additive"
    fp = mode if mode in ("iso", "zf") else "own"
    cfilt = {"own": int(filt), "iso": oracle_lib.FILTER_ISO, "zf": oracle_lib.FILTER_ZF}[fp]
    rng = np.random.default_rng(7)
    P = cam.n_pixels
    w_rgb = rng.normal(size=(P, 3))
    w_T = rng.normal(size=P)
    ref = oracle_lib.render(cam, sc, filter=cfilt, comp=int(add), eps=2e-4)
    flagged = ref.flags != 0
    w_rgb[flagged] = 0.0
    w_T[flagged] = 0.0
    _, g_ref = G.loss_and_grad(cam, sc, np.arange(P), w_rgb, w_T, filter_on=filt, additive=add, footprint=fp)

    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v = ctx.view()
    v.set_camera_from(cam)
    flags = cg.KEEP_FOR_BACKWARD | (0 if filt else cg.FILTER_NONE) | (cg.COMP_ADDITIVE if add else 0)
    flags |= {"own": 0, "iso": cg.FILTER_ISO, "zf": cg.FILTER_ZF}[fp]
    rgb, T = v.render(flags=flags)
    dL_drgb = torch.from_numpy(w_rgb.T.reshape(3, cam.height, cam.width).astype(np.float32)).cuda()
    dL_dT = torch.from_numpy(w_T.reshape(cam.height, cam.width).astype(np.float32)).cuda()
    g = v.render_backward(dL_drgb, dL_dT)
    torch.cuda.synchronize()
    assert_grads_close({k: t.cpu().numpy() for k, t in g.items()}, g_ref)


def test_backward_requires_forward_state(cg):
    cam, sc = _case("pinhole")
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v = ctx.view()
    v.set_camera_from(cam)
    rgb, _ = v.render()                                  # no KEEP_FOR_BACKWARD
    with pytest.raises(cg.ConegsError) as e:
        v.render_backward(torch.ones_like(rgb))
    assert e.value.status == 6


def test_backward_accumulates_over_views(cg):
    cam, sc = _case("pinhole")
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v = ctx.view()
    v.set_camera_from(cam)
    rgb, _ = v.render(flags=cg.KEEP_FOR_BACKWARD)
    g1 = v.render_backward(torch.ones_like(rgb))
    g2 = v.render_backward(torch.ones_like(rgb), grads={k: t.clone() for k, t in g1.items()})
    torch.cuda.synchronize()
    for k in g1:   # atomics add in any order: compare at the gradient's own scale
        scale = float(g1[k].abs().max()) + 1e-12
        assert float((g2[k] - 2 * g1[k]).abs().max()) <= 1e-5 * scale


def test_backward_split_lists_match_gradient_oracle(cg, oracle_lib):
    """Tile lists of a few thousand faint, wide Gaussians: the lists are cut into
    256-entry segments walked by separate CTAs, and pixels composite hundreds of
    pairs across segment boundaries before (or without) reaching the stop rule,
    so the adjoint walks each segment back to front from the per-segment state
    the forward leaves."""
    from oracle import grad as G
    cam = S.pinhole(16, 16, 10.0)
    sc = S.uniform_box_scene(2500, seed=21, log_scale_mean=-0.3, log_scale_std=0.3, sh_degree=1)
    rng = np.random.default_rng(22)
    sc = dataclasses.replace(sc, opacity_logits=rng.normal(-4.0, 0.5, sc.n).astype(np.float32))
    sc = sc.with_rho2(oracle_lib.floor_rho2([S.pinhole(64, 64, 40.0)], sc.means).astype(np.float32))
    P = cam.n_pixels
    ref = oracle_lib.render(cam, sc, eps=3e-5)
    assert ref.ncontrib.max() > 600                      # walks cross several 256-entry segments
    assert (ref.T < 2e-4).any() and (ref.T > 2e-4).any()   # some pixels stop, some do not
    w_rgb = rng.normal(size=(P, 3))
    w_T = rng.normal(size=P)
    flagged = ref.flags != 0
    w_rgb[flagged] = 0.0
    w_T[flagged] = 0.0
    assert flagged.mean() < 0.2
    _, g_ref = G.loss_and_grad(cam, sc, np.arange(P), w_rgb, w_T, chunk=64)

    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v = ctx.view()
    v.set_camera_from(cam)
    rgb, T = v.render(flags=cg.KEEP_FOR_BACKWARD)
    _, pt = v.bin_counts()
    assert int(pt.max()) > 4 * 256
    ok = ~flagged
    assert np.abs(rgb.cpu().numpy().reshape(3, -1).T - ref.rgb)[ok].max() <= 1e-4
    assert np.abs(T.cpu().numpy().reshape(-1) - ref.T)[ok].max() <= 1e-4
    dL_drgb = torch.from_numpy(w_rgb.T.reshape(3, cam.height, cam.width).astype(np.float32)).cuda()
    dL_dT = torch.from_numpy(w_T.reshape(cam.height, cam.width).astype(np.float32)).cuda()
    g = v.render_backward(dL_drgb, dL_dT)
    torch.cuda.synchronize()
    assert_grads_close({k: t.cpu().numpy() for k, t in g.items()}, g_ref)


def test_backward_full_size_c2_sampled(cg, oracle_lib):
    """The adjoint on the benchmark workload: the 1280x720 view of the 500k-Gaussian
    blob scene with SH degree 3 and the Eq. 11 floor, a loss on 300 sampled pixels.
    The gradient oracle runs per pixel on the Gaussians that contribute there (the
    others have no gradient through that pixel), and the sums are compared entry by
    entry with the GPU adjoint, which walks the full tile lists."""
    from oracle import grad as G
    cam = S.c2_cameras()[0]
    sc = S.c2_scene()
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v = ctx.view()
    v.set_camera_from(cam)
    rho2 = ctx.compute_floor([v])
    ctx.set_scene_from(sc, rho2=rho2)
    sc = sc.with_rho2(rho2.cpu().numpy())
    rng = np.random.default_rng(31)
    pix = rng.choice(cam.n_pixels, size=300, replace=False).astype(np.int32)
    MAXU = 512
    ref = oracle_lib.render(cam, sc, pix=pix, eps=2e-4, max_used=MAXU)
    keep = (ref.flags == 0) & (ref.ncontrib < MAXU) & (ref.ncontrib > 0)
    assert keep.sum() > 200
    w_rgb = rng.normal(size=(pix.size, 3)) * keep[:, None]
    w_T = rng.normal(size=pix.size) * keep

    dL_drgb = torch.zeros(3, cam.n_pixels, dtype=torch.float32)
    dL_T = torch.zeros(cam.n_pixels, dtype=torch.float32)
    dL_drgb[:, torch.from_numpy(pix).long()] = torch.from_numpy(w_rgb.T.astype(np.float32))
    dL_T[torch.from_numpy(pix).long()] = torch.from_numpy(w_T.astype(np.float32))
    rgb, T = v.render(flags=cg.KEEP_FOR_BACKWARD)
    g = v.render_backward(dL_drgb.reshape(3, cam.height, cam.width).cuda(), dL_T.reshape(cam.height, cam.width).cuda())
    torch.cuda.synchronize()
    got = {k: t.cpu().numpy().astype(np.float64) for k, t in g.items()}

    want = {"means": np.zeros((sc.n, 3)), "log_scales": np.zeros((sc.n, 3)), "quats": np.zeros((sc.n, 4)),
            "logits": np.zeros(sc.n), "sh": np.zeros(sc.sh.shape)}
    for t in np.nonzero(keep)[0]:
        ids = np.sort(ref.used[t][ref.used[t] >= 0])
        _, gp = G.loss_and_grad(cam, sc.subset(ids), pix[t:t + 1], w_rgb[t:t + 1], w_T[t:t + 1])
        for k in want:
            want[k][ids] += gp[k]
    touched = np.zeros(sc.n, bool)
    for t in np.nonzero(keep)[0]:
        touched[ref.used[t][ref.used[t] >= 0]] = True
    assert touched.sum() > 1000
    sub = {k: a[touched] for k, a in want.items()}
    assert_grads_close({"means": got["means"].reshape(-1, 3)[touched],
                        "log_scales": got["log_scales"].reshape(-1, 3)[touched],
                        "quats": got["quats"].reshape(-1, 4)[touched],
                        "opacity_logits": got["opacity_logits"].reshape(-1)[touched],
                        "sh": got["sh"].reshape(sc.sh.shape)[touched]}, sub)
    # Gaussians that contribute to no kept pixel get no gradient
    scale = max(np.abs(want["means"]).max(), 1e-12)
    assert np.abs(got["means"].reshape(-1, 3)[~touched]).max() <= ABS * scale


def test_backward_accumulates_views_like_the_oracle(cg, oracle_lib):
    """Gradients of a loss over several views (a pinhole and a fisheye of one scene)
    accumulated into one buffer, as a training step over a camera batch does, against
    the sum of the gradient oracle's per-view gradients."""
    from oracle import grad as G
    sc = S.uniform_box_scene(150, seed=31, log_scale_mean=-2.6, log_scale_std=0.4, sh_degree=1)
    cams = [S.pinhole(40, 30, 36.0, cam_to_world=S.look_at((0.05, 0.0, 0.0), (0.1, 0.05, 4.0))),
            S.c3_camera(48, 48)]
    sc = sc.with_rho2(oracle_lib.floor_rho2([c.scaled(2.0) for c in cams], sc.means).astype(np.float32))
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    grads = None
    total = None
    rng = np.random.default_rng(32)
    for cam in cams:
        P = cam.n_pixels
        w_rgb = rng.normal(size=(P, 3))
        w_T = rng.normal(size=P)
        ref = oracle_lib.render(cam, sc, eps=2e-4)
        w_rgb[ref.flags != 0] = 0.0
        w_T[ref.flags != 0] = 0.0
        _, g_ref = G.loss_and_grad(cam, sc, np.arange(P), w_rgb, w_T)
        total = g_ref if total is None else {k: total[k] + g_ref[k] for k in total}
        v = ctx.view()
        v.set_camera_from(cam)
        v.render(flags=cg.KEEP_FOR_BACKWARD)
        dL_drgb = torch.from_numpy(w_rgb.T.reshape(3, cam.height, cam.width).astype(np.float32)).cuda()
        dL_dT = torch.from_numpy(w_T.reshape(cam.height, cam.width).astype(np.float32)).cuda()
        grads = v.render_backward(dL_drgb, dL_dT, grads=grads)
    torch.cuda.synchronize()
    assert_grads_close({k: t.cpu().numpy() for k, t in grads.items()}, total)

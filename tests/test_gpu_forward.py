"""GPU forward path vs the FP64 oracle, through the C ABI.

Bit-exact: valid masks, tile cone tables, per-Gaussian / per-tile pair counts,
the per-tile list order, the radix sort.  Within tolerance: ray tables, the
Eq. 11 floor and the rendered image (1e-4 absolute per RGB channel and on T,
excluding the pixels the oracle flags as near a compositing threshold).
"""
import math

import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
# relative margin of the oracle's near-threshold flags (alpha vs 1/255 and 0.99, the
# 1e-4 stop test, t* vs 0.01): well above the FP32 path's relative error in T
EPS_FLAG = 2e-4


@pytest.fixture(scope="module")
def cg():
    import paper_2609_13397_b300 as cg
    return cg


def _cases():
    out = {"c1": S.c1()}
    out["kb160"] = (S.c3_camera(160, 160), S.uniform_box_scene(1500, seed=3))
    bcam = S.pinhole(320, 180, 300.0)
    out["blob320"] = (bcam, S.blob_scene(20000, seed=1, cam=bcam))
    out["ragged"] = (S.pinhole(70, 45, 40.0, 33.0, 21.0, cam_to_world=S.look_at((0.1, 0.0, -0.5), (0.2, 0.1, 4.0))),
                     S.uniform_box_scene(500, seed=9, log_scale_mean=-2.5))
    kb_pose = S.look_at((0.05, -0.1, 0.2), (0.3, 0.2, 4.0))
    kcam = S.c3_camera(96, 80)
    kcam.cam_to_world = kb_pose
    out["kb_ragged"] = (kcam, S.uniform_box_scene(800, seed=5))
    # wide, rotated pinhole with fx != fy and an off-centre principal point, inside a
    # shell of Gaussians on every side (behind, beside, near the image plane's horizon)
    wcam = S.Camera(S.PINHOLE, 96, 64, 30.0, 36.0, 50.5, 30.25,
                    cam_to_world=S.look_at((0.0, 0.1, 0.0), (1.0, 0.4, 2.0)))
    out["wide_surround"] = (wcam, S.blob_scene(3000, seed=13, cam=wcam, blob_frac=0.3, shell=(1.5, 4.0),
                                               log_scale_mean=-2.5, sh_degree=1))
    # rotated fisheye with an off-centre principal point in the same kind of shell: cones
    # that contain the optical axis, reach the valid circle's rim, or sit behind the camera
    fcam = S.c3_camera(112, 96, seed=2)
    fcam = S.Camera(fcam.model, fcam.width, fcam.height, fcam.fx, fcam.fy, 57.5, 46.0, k=fcam.k,
                    cam_to_world=S.look_at((0.1, 0.0, 0.1), (-1.0, 0.5, 2.0)), theta_lim=fcam.theta_lim)
    out["kb_surround"] = (fcam, S.blob_scene(3000, seed=17, cam=S.pinhole(112, 96, 60.0), blob_frac=0.3,
                                             shell=(1.5, 4.0), log_scale_mean=-2.5, sh_degree=1))
    # very low resolution fisheye among close, strongly anisotropic Gaussians: the
    # t* bound's anisotropy factor decides most tiles
    lcam = S.c3_camera(24, 20, seed=1)
    lcam = S.Camera(lcam.model, 24, 20, lcam.fx, lcam.fy, 12.0, 10.0, k=lcam.k,
                    cam_to_world=S.look_at((0.1, -0.2, 0.0), (0.4, 0.3, 2.0)), theta_lim=lcam.theta_lim)
    out["lowres_kb"] = (lcam, S.blob_scene(1500, seed=31, cam=S.pinhole(24, 20, 19.0), blob_frac=0.3,
                                           shell=(0.3, 3.0), log_scale_mean=-2.2, log_scale_std=1.5, sh_degree=1))
    return out


CASES = _cases()


def _with_floor(oracle, name, cam, sc):
    if name == "blob320":
        return sc.with_rho2(oracle.floor_rho2([S.pinhole(640, 360, 600.0)], sc.means).astype(np.float32))
    return sc


def _setup(cg, cam, sc, storage=None):
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, storage=storage)
    v = ctx.view()
    v.set_camera_from(cam)
    return ctx, v


@pytest.mark.parametrize("name", list(CASES))
def test_ray_table(cg, oracle_lib, name):
    cam, sc = CASES[name]
    ctx, v = _setup(cg, cam, sc)
    d, dx, dy, valid = (t.cpu().numpy() for t in v.rays())
    torch.cuda.synchronize()
    od, odx, ody, ovalid = oracle_lib.rays(cam)
    assert np.array_equal(valid.astype(bool), ovalid)
    m = ovalid
    # pinhole: a few FP32 ulps of a unit vector.  Kannala-Brandt: theta solves r(theta) =
    # |pixel offset| and r' >= 1/4 below theta_lim, so the ~2-ulp error of the FP32 radius
    # (r <= ~1.2) grows up to 4x in theta before sin/cos: about 6e-7, bound 1e-6
    tol = 4e-7 if cam.model == S.PINHOLE else 1e-6
    assert np.abs(d.T[m] - od[m]).max() < tol
    for g, o in ((dx, odx), (dy, ody)):
        err = np.linalg.norm(g.T[m] - o[m], axis=1) / np.linalg.norm(o[m], axis=1)
        assert err.max() < 2e-5, err.max()


@pytest.mark.parametrize("name", list(CASES))
def test_tile_table_bit_exact(cg, oracle_lib, name):
    cam, sc = CASES[name]
    ctx, v = _setup(cg, cam, sc)
    g = v.tile_table().cpu().numpy()
    o = oracle_lib.tile_table(cam)
    assert np.array_equal(g.view(np.uint32), o.view(np.uint32))


@pytest.mark.parametrize("name", list(CASES))
def test_pair_counts_bit_exact(cg, oracle_lib, name):
    cam, sc = CASES[name]
    sc = _with_floor(oracle_lib, name, cam, sc)
    ctx, v = _setup(cg, cam, sc)
    v.render()
    pg, pt = (t.cpu().numpy() for t in v.bin_counts())
    total, opg, opt, _ = oracle_lib.bin_counts(cam, sc)
    assert np.array_equal(pg, opg)
    assert np.array_equal(pt, opt)
    assert v.stats()["n_pairs"] == total


@pytest.mark.parametrize("name", ["c1", "blob320", "kb_ragged"])
def test_tile_lists_in_depth_order(cg, oracle_lib, name):
    """Each tile's list is the binned Gaussians sorted by (FP32 depth key, index)."""
    cam, sc = CASES[name]
    ctx, v = _setup(cg, cam, sc)
    v.render()
    gid, rng = (t.cpu().numpy() for t in v.pairs())
    _, _, _, pas = oracle_lib.bin_counts(cam, sc, dense=True)
    L = oracle_lib.bin_gauss(cam, sc)[:, 3]
    for t in range(rng.shape[0]):
        got = gid[rng[t, 0]:rng[t, 1]]
        want = np.nonzero(pas[:, t])[0]
        want = want[np.lexsort((want, L[want]))]
        assert np.array_equal(got, want), t


def _render_compare(cg, oracle_lib, cam, sc, flags=0, filt=1, comp=0, storage=None, tol=TOL, pix=None):
    ctx, v = _setup(cg, cam, sc, storage=storage)
    rgb, T = v.render(flags=flags)
    rgb = rgb.cpu().numpy().reshape(3, -1).T
    T = T.cpu().numpy().reshape(-1)
    r = oracle_lib.render(cam, sc, pix=pix, filter=filt, comp=comp, eps=EPS_FLAG)
    if pix is not None:
        rgb, T = rgb[pix], T[pix]
    ok = r.flags == 0
    err = np.abs(rgb - r.rgb)[ok].max(initial=0.0)
    errT = np.abs(T - r.T)[ok].max(initial=0.0)
    return err, errT, (~ok).sum(), ok.size


@pytest.mark.parametrize("name", list(CASES))
def test_render_matches_oracle(cg, oracle_lib, name):
    cam, sc = CASES[name]
    sc = _with_floor(oracle_lib, name, cam, sc)
    err, errT, nflag, npx = _render_compare(cg, oracle_lib, cam, sc)
    assert nflag <= 0.01 * npx
    assert err <= TOL and errT <= TOL, (err, errT)


@pytest.mark.parametrize("mode", ["filter_none", "additive"])
def test_render_variants(cg, oracle_lib, mode):
    cam, sc = CASES["blob320"]
    sc = _with_floor(oracle_lib, "blob320", cam, sc)
    if mode == "filter_none":
        err, errT, nflag, npx = _render_compare(cg, oracle_lib, cam, sc, flags=cg.FILTER_NONE, filt=0)
    else:
        err, errT, nflag, npx = _render_compare(cg, oracle_lib, cam, sc, flags=cg.COMP_ADDITIVE, comp=1)
    assert err <= TOL and errT <= TOL, (err, errT)


@pytest.mark.parametrize("name", ["blob320", "wide_surround", "kb_surround", "kb160"])
@pytest.mark.parametrize("variant", ["iso", "zf"])
def test_isotropic_footprint_variants(cg, oracle_lib, name, variant):
    """FILTER_ISO / FILTER_ZF against the oracle's variants: images within the
    FP32 tolerance; pair lists bit-exact with the binning rule (for z/f with the
    tiles' footprint bound raised to 1/(6 f_x^2), which keeps the rule conservative
    for the z/f footprint)."""
    cam, sc = CASES[name]
    sc = _with_floor(oracle_lib, name, cam, sc)
    flags, filt = ((cg.FILTER_ISO, oracle_lib.FILTER_ISO) if variant == "iso"
                   else (cg.FILTER_ZF, oracle_lib.FILTER_ZF))
    err, errT, nflag, npx = _render_compare(cg, oracle_lib, cam, sc, flags=flags, filt=filt)
    assert nflag <= 0.02 * npx
    assert err <= TOL and errT <= TOL, (err, errT)
    ctx, v = _setup(cg, cam, sc)
    v.render(flags=flags)
    pg, pt = (t.cpu().numpy() for t in v.bin_counts())
    total, opg, opt, _ = oracle_lib.bin_counts(cam, sc, zf=variant == "zf")
    assert np.array_equal(pg, opg) and np.array_equal(pt, opt)
    with pytest.raises(cg.ConegsError) as e:
        v.render(flags=cg.FILTER_ISO | cg.FILTER_ZF)
    assert e.value.status == 1


def test_render_deterministic(cg):
    cam, sc = CASES["blob320"]
    ctx, v = _setup(cg, cam, sc)
    a, ta = v.render()
    b, tb = v.render()
    assert torch.equal(a, b) and torch.equal(ta, tb)


def test_empty_scene_and_invalid_pixels(cg):
    cam = S.c3_camera(64, 64)
    sc = S.uniform_box_scene(0, seed=0)
    ctx, v = _setup(cg, cam, sc)
    rgb, T = v.render()
    assert float(rgb.abs().max()) == 0.0 and float(T.min()) == 1.0
    sc = S.uniform_box_scene(50, seed=0)
    ctx.set_scene_from(sc)
    rgb, T = v.render()
    _, _, _, valid = v.rays()
    inv = (valid == 0).reshape(64, 64)
    assert inv.any()
    assert float(rgb[:, inv].abs().max()) == 0.0 and float(T[inv].min()) == 1.0


@pytest.mark.parametrize("model", ["pinhole", "kb"])
def test_every_gaussian_outside_the_view(cg, model):
    """Gaussians all behind a pinhole (or beyond a fisheye's field of view):
    background image and a zero adjoint.  Behind the pinhole they are culled
    before binning (no pairs); a 64x64 fisheye's large footprint bound keeps a
    few conservative pairs for the close, elongated ones, which contribute
    nothing."""
    sc = S.uniform_box_scene(300, seed=4)
    sc.means[:, 2] = -sc.means[:, 2]                       # z in [-6, -2]: behind the camera
    cam = S.pinhole(64, 48, 60.0) if model == "pinhole" else S.c3_camera(64, 64)
    if model == "kb":
        sc.means[:, :2] *= 0.05                            # straight behind: beyond the 95-degree half field
    ctx, v = _setup(cg, cam, sc)
    rgb, T = v.render(flags=cg.KEEP_FOR_BACKWARD)
    assert float(rgb.abs().max()) == 0.0 and float(T.min()) == 1.0
    if model == "pinhole":
        assert v.stats()["n_pairs"] == 0 and v.stats()["n_visible"] == 0
    g = v.render_backward(torch.ones_like(rgb))
    assert all(float(t.abs().max()) == 0.0 for t in g.values())


def test_floor_matches_oracle(cg, oracle_lib):
    sc = S.blob_scene(20000, seed=2, cam=S.pinhole(320, 180, 300.0))
    views = [S.pinhole(640, 360, 600.0), S.pinhole(320, 180, 300.0, cam_to_world=S.look_at((0.3, 0, 0), (0, 0, 6))),
             S.c3_camera(200, 200)]
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    vs = []
    for c in views:
        v = ctx.view()
        v.set_camera_from(c)
        vs.append(v)
    g = ctx.compute_floor(vs).cpu().numpy()
    o = oracle_lib.floor_rho2(views, sc.means)
    both = (g > 0) & (o > 0)
    # visibility is a decision on the projected centre; it may differ only for a
    # centre within rounding of an image border or the fisheye's valid circle
    assert ((g > 0) == (o > 0)).mean() >= 1.0 - 1e-4
    rel = np.abs(g[both] - o[both]) / o[both]
    # a few FP32 roundings of a half-trace: ~1e-7 for the pinholes; the fisheye's
    # differentials come from the FP32 inverse mapping (~2e-5 relative per edge ray)
    assert np.quantile(rel, 0.999) < 1e-5 and rel.max() < 5e-5, (np.quantile(rel, 0.999), rel.max())


@pytest.mark.parametrize("n,bits", [(1, 32), (1000, 32), (4097, 12), (100003, 32), (1 << 20, 16), (3 << 20, 7)])
def test_radix_sort(cg, n, bits):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 3] = keys[n // 2]            # many ties
    vals = np.arange(n, dtype=np.uint32)
    ctx = cg.Context(0)
    k = torch.from_numpy(keys.view(np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    cg.radix_sort_pairs(ctx, k, v, 0, bits)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(k.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(v.cpu().numpy().view(np.uint32), vals[order])


def test_full_size_c2_sampled(cg, oracle_lib):
    """The 1280x720 + 160x90 workload with 500k Gaussians and the Eq. 11 floor, as
    the benchmark runs it: sampled pixels against the oracle, all pair counts of
    a sample of Gaussians bit-exact."""
    cams = S.c2_cameras()
    sc = S.c2_scene()
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    v0 = ctx.view()
    v0.set_camera_from(cams[0])
    rho2 = ctx.compute_floor([v0])
    ctx.set_scene_from(sc, rho2=rho2)
    sc = sc.with_rho2(rho2.cpu().numpy())
    rng = np.random.default_rng(0)
    for cam in cams:
        v = ctx.view()
        v.set_camera_from(cam)
        rgb, T = v.render()
        rgb = rgb.cpu().numpy().reshape(3, -1).T
        T = T.cpu().numpy().reshape(-1)
        pix = rng.choice(cam.n_pixels, size=min(600, cam.n_pixels), replace=False).astype(np.int32)
        r = oracle_lib.render(cam, sc, pix=pix, eps=EPS_FLAG)
        ok = r.flags == 0
        assert ok.mean() > 0.9, ok.mean()
        assert np.abs(rgb[pix] - r.rgb)[ok].max() <= TOL
        assert np.abs(T[pix] - r.T)[ok].max() <= TOL
        pg, _ = v.bin_counts()
        sub = rng.choice(sc.n, size=3000, replace=False)
        _, opg, _, _ = oracle_lib.bin_counts(cam, sc.subset(sub))
        assert np.array_equal(pg.cpu().numpy()[sub], opg)


def test_split_long_lists_match_oracle(cg, oracle_lib):
    """A small low-resolution view of a dense scene: every tile list spans many
    1024-entry segments processed by separate CTAs and merged front to back."""
    cam = S.pinhole(24, 16, 12.0)
    sc = S.blob_scene(40000, seed=11, cam=S.pinhole(240, 160, 120.0), n_blobs=4)
    sc = sc.with_rho2(oracle_lib.floor_rho2([S.pinhole(240, 160, 120.0)], sc.means).astype(np.float32))
    ctx, v = _setup(cg, cam, sc)
    rgb, T = v.render(flags=cg.PROFILE)
    st = v.stats()
    _, pt = v.bin_counts()
    assert int(pt.max()) > 4 * 1024                       # lists really span several segments
    rgb = rgb.cpu().numpy().reshape(3, -1).T
    T = T.cpu().numpy().reshape(-1)
    r = oracle_lib.render(cam, sc, eps=EPS_FLAG)
    ok = r.flags == 0
    assert ok.mean() > 0.8
    assert np.abs(rgb - r.rgb)[ok].max() <= TOL and np.abs(T - r.T)[ok].max() <= TOL
    assert st["n_walked"] > 0


def test_render_batch_equals_single_renders(cg):
    """conegs_render_batch overlaps the views' work but computes each view's image
    exactly as a single render does."""
    sc = S.blob_scene(20000, seed=4, cam=S.pinhole(320, 180, 300.0))
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    cams = [S.pinhole(320, 180, 300.0), S.c3_camera(96, 96), S.pinhole(40, 24, 37.5)]
    views = []
    for c in cams:
        v = ctx.view()
        v.set_camera_from(c)
        views.append(v)
    single = [v.render() for v in views]
    streams = [torch.cuda.Stream() for _ in views]
    batch = ctx.render_batch(views, streams=streams)
    torch.cuda.synchronize()
    for (r1, t1), (r2, t2) in zip(single, batch):
        assert torch.equal(r1, r2) and torch.equal(t1, t2)
    with pytest.raises(cg.ConegsError) as e:
        ctx.render_batch([views[0], views[0]])
    assert e.value.status == 1


def test_render_host_batch_equals_device_render(cg):
    sc = S.blob_scene(5000, seed=6, cam=S.pinhole(160, 90, 150.0))
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    cams = [S.pinhole(160, 90, 150.0), S.c3_camera(48, 40)]
    views = []
    for c in cams:
        v = ctx.view()
        v.set_camera_from(c)
        views.append(v)
    dev = [v.render() for v in views]
    host = [(torch.empty(3, c.height, c.width, pin_memory=True), torch.empty(c.height, c.width, pin_memory=True))
            for c in cams]
    ctx.render_host_batch(views, host, streams=[torch.cuda.Stream() for _ in views])
    for (r, t), (hr, ht) in zip(dev, host):
        assert torch.equal(r.cpu(), hr) and torch.equal(t.cpu(), ht)
    # pageable host memory: the copies complete before the call returns
    plain = [(torch.empty(3, c.height, c.width), torch.empty(c.height, c.width)) for c in cams]
    ctx.render_host_batch(views, plain, streams=[torch.cuda.Stream() for _ in views])
    for (r, t), (hr, ht) in zip(dev, plain):
        assert torch.equal(r.cpu(), hr) and torch.equal(t.cpu(), ht)


def test_pipelined_host_renders_equal_device_renders(cg):
    """render_host_batch_async: six calls in a row, the cameras changing every call,
    each into its own pinned host buffers and read only after host_wait; every image
    equals the device render of its camera (the staging images alternate, so a
    render never overwrites an image whose copy is still in flight)."""
    cams = [S.pinhole(160, 96, 150.0), S.c3_camera(128, 112)]
    sc = S.blob_scene(8000, seed=5, cam=cams[0])
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    views = [ctx.view() for _ in cams]
    streams = [torch.cuda.Stream() for _ in views]
    poses = [S.look_at((0.05 * k, 0.0, 0.0), (0.1 * k, 0.05, 4.0)) for k in range(6)]
    outs = []
    for k, pose in enumerate(poses):
        for v, c in zip(views, cams):
            c2 = S.Camera(c.model, c.width, c.height, c.fx, c.fy, c.cx, c.cy, k=c.k, cam_to_world=pose,
                          theta_lim=c.theta_lim)
            v.set_camera_from(c2)
        host = [(torch.empty(3, c.height, c.width, pin_memory=True), torch.empty(c.height, c.width, pin_memory=True))
                for c in cams]
        ctx.render_host_batch_async(views, host, streams=streams)
        outs.append(host)
    for v in views:
        v.host_wait()
    ref_view = ctx.view()
    for pose, host in zip(poses, outs):
        for c, (h_rgb, h_T) in zip(cams, host):
            ref_view.set_camera_from(S.Camera(c.model, c.width, c.height, c.fx, c.fy, c.cx, c.cy, k=c.k,
                                              cam_to_world=pose, theta_lim=c.theta_lim))
            rgb, T = ref_view.render()
            assert torch.equal(rgb.cpu(), h_rgb) and torch.equal(T.cpu(), h_T)


@pytest.mark.parametrize("seed", range(8))
def test_pair_counts_bit_exact_random(cg, oracle_lib, seed):
    """Random cameras (pinhole and Kannala-Brandt, random poses, intrinsics and
    distortion) and scenes: per-Gaussian and per-tile counts bit-exact with the
    oracle's FP32 emulation of the rule (cone and silhouette tests)."""
    from test_binning_rule import _random_case
    cam, sc = _random_case(seed)
    ctx, v = _setup(cg, cam, sc)
    v.render()
    pg, pt = (t.cpu().numpy() for t in v.bin_counts())
    total, opg, opt, _ = oracle_lib.bin_counts(cam, sc)
    assert np.array_equal(pg, opg)
    assert np.array_equal(pt, opt)


def _sampled_parity(oracle_lib, cam, sc, rgb, T, npx, seed, tol=TOL, eps=EPS_FLAG, min_ok=0.9):
    valid = oracle_lib.rays(cam)[3]
    cand = np.nonzero(valid)[0]
    rng = np.random.default_rng(seed)
    pix = rng.choice(cand, size=min(npx, cand.size), replace=False).astype(np.int32)
    r = oracle_lib.render(cam, sc, pix=pix, eps=eps)
    ok = r.flags == 0
    assert ok.mean() > min_ok, ok.mean()
    err = np.abs(rgb.reshape(3, -1).T[pix] - r.rgb)[ok].max(initial=0.0)
    errT = np.abs(T.reshape(-1)[pix] - r.T)[ok].max(initial=0.0)
    assert err <= tol and errT <= tol, (err, errT)
    return r


def test_full_size_c3_fisheye_sampled(cg, oracle_lib):
    """The differentiation workload's camera and scene at full size: a 190-degree
    Kannala-Brandt fisheye at 1024x1024 and 1M Gaussians; sampled pixels against
    the oracle, the pair counts of sampled Gaussians bit-exact."""
    cam, sc = S.c3_camera(), S.c3_scene()
    ctx, v = _setup(cg, cam, sc)
    rgb, T = v.render()
    r = _sampled_parity(oracle_lib, cam, sc, rgb.cpu().numpy(), T.cpu().numpy(), 400, seed=3)
    assert (r.ncontrib > 0).mean() > 0.2
    pg, _ = v.bin_counts()
    sub = np.random.default_rng(4).choice(sc.n, size=3000, replace=False)
    _, opg, _, _ = oracle_lib.bin_counts(cam, sc.subset(sub))
    assert np.array_equal(pg.cpu().numpy()[sub], opg)


def test_full_size_c4_rig_bf16_sampled(cg, oracle_lib):
    """The eight-camera rig (4 pinhole, 4 fisheye at 1, 1/2, 1/4, 1/8 of 1080p), 3M
    Gaussians with the Eq. 11 floor over the rig, SH and opacity stored in BF16: every
    view on sampled pixels against the oracle on the quantised values (FP32 arithmetic:
    1e-4) and on the FP32 values (the storage's budget: 2e-3, away from thresholds)."""
    rig = S.c4_rig()
    sc = S.blob_scene(3_000_000, seed=0, cam=rig[0])
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, storage=torch.bfloat16)
    views = []
    for c in rig:
        v = ctx.view()
        v.set_camera_from(c)
        views.append(v)
    rho2 = ctx.compute_floor(views)
    ctx.set_scene_from(sc, storage=torch.bfloat16, rho2=rho2)
    sc = sc.with_rho2(rho2.cpu().numpy())
    q = S.quantized(sc, "bf16")
    outs = ctx.render_batch(views, streams=[torch.cuda.Stream() for _ in views])
    torch.cuda.synchronize()
    for k, (cam, (rgb, T)) in enumerate(zip(rig, outs)):
        rgb, T = rgb.cpu().numpy(), T.cpu().numpy()
        _sampled_parity(oracle_lib, cam, q, rgb, T, 80, seed=10 + k)
        # the wide flag margin (5e-3: quantisation moves responses by ~1e-3 relative) flags
        # a good share of the rig's dense pixels; the others must stay within the budget
        _sampled_parity(oracle_lib, cam, sc, rgb, T, 80, seed=10 + k, tol=2e-3, eps=5e-3, min_ok=0.5)


def test_full_size_c5_request_4k_fp16_sampled(cg, oracle_lib):
    """The largest serving request: 3840x2160 of the 5M-Gaussian scene with SH degree 3
    stored in FP16 (floor from the rig), through a fisheye and a pinhole."""
    rig = S.c4_rig()
    sc = S.blob_scene(5_000_000, seed=0, cam=rig[0])
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, storage=torch.float16)
    vs = []
    for c in rig:
        v = ctx.view()
        v.set_camera_from(c)
        vs.append(v)
    rho2 = ctx.compute_floor(vs)
    ctx.set_scene_from(sc, storage=torch.float16, rho2=rho2)
    sc = S.quantized(sc.with_rho2(rho2.cpu().numpy()), "f16")
    pose = rig[2].cam_to_world
    for k, cam in enumerate([S.pinhole(3840, 2160, 3840 * 60.0 / 64.0, cam_to_world=pose),
                             S.kb_fisheye(3840, 2160, rig[4].k, cam_to_world=pose)]):
        v = ctx.view()
        v.set_camera_from(cam)
        rgb, T = v.render()
        _sampled_parity(oracle_lib, cam, sc, rgb.cpu().numpy(), T.cpu().numpy(), 150, seed=20 + k)

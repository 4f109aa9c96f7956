"""The hand-written adjoint behind torch.autograd (render_fn), checked two ways:

- against the FP64 gradient oracle (oracle/grad.py), entry by entry, on small
  pinhole and fisheye scenes with an L1 loss;
- the differentiation workload: a Kannala-Brandt fisheye (190 deg) at 256x256
  with a C1-distributed scene, L1 loss against the FP64 oracle's render of the
  seed-1 perturbed scene, loss.backward() through render_fn, against FP64
  central differences of the C oracle on 64 random parameters (seed 2) of
  Gaussians that contribute to some pixel.  Each difference re-renders only the
  pixels of the tiles the binning rule gives the perturbed Gaussian (no other
  pixel can change); a parameter is skipped when the differences at h and h/2
  disagree (a compositing threshold lies within h).

Pixels the oracle flags as near a threshold, and channels whose value lies
within 1e-4 of the target (where the L1 kink could fall on either side), are
left out of the loss on both sides.
"""
import dataclasses

import numpy as np
import pytest

import synthetic as S
from test_gpu_backward import assert_grads_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def cg():
    import paper_2609_13397_b300 as cg
    return cg


def _tensors(sc, dev="cuda"):
    return [torch.tensor(np.asarray(getattr(sc, k), np.float32), device=dev, requires_grad=True)
            for k in PARAMS]


def _l1_mask(ref, target, valid):
    mask = (np.abs(ref.rgb - target) > 1e-4) & (ref.flags == 0)[:, None] & valid[:, None]
    return mask


@pytest.mark.parametrize("kind", ["pinhole", "fisheye"])
def test_render_fn_matches_gradient_oracle(cg, oracle_lib, kind):
    from oracle import grad as G
    if kind == "pinhole":
        cam = S.pinhole(40, 30, 36.0, cam_to_world=S.look_at((0.05, 0.0, 0.0), (0.1, 0.05, 4.0)))
        sc = S.uniform_box_scene(150, seed=12, log_scale_mean=-2.6, log_scale_std=0.4, sh_degree=2)
    else:
        cam = S.c3_camera(48, 48)
        sc = S.uniform_box_scene(150, seed=13, log_scale_mean=-2.4, log_scale_std=0.4, sh_degree=1)
    sc = sc.with_rho2(oracle_lib.floor_rho2([cam.scaled(2.0)], sc.means).astype(np.float32))
    tgt = S.perturbed(sc, seed=1)
    P = cam.n_pixels
    target = oracle_lib.render(cam, tgt).rgb
    ref = oracle_lib.render(cam, sc, eps=2e-4)
    valid = oracle_lib.rays(cam)[3]
    mask = _l1_mask(ref, target, valid)
    nval = int(valid.sum())
    w_rgb = np.sign(ref.rgb - target) * mask / (3.0 * nval)
    _, g_ref = G.loss_and_grad(cam, sc, np.arange(P), w_rgb, np.zeros(P))

    ctx = cg.Context(0)
    v = ctx.view()
    v.set_camera_from(cam)
    params = _tensors(sc)
    rho2 = torch.tensor(sc.rho2, device="cuda")
    rgb, T = cg.render_fn(v, *params, rho2=rho2)
    tgt_t = torch.tensor(target.T.reshape(3, cam.height, cam.width), dtype=torch.float32, device="cuda")
    m_t = torch.tensor(mask.T.reshape(3, cam.height, cam.width), device="cuda")
    loss = ((rgb - tgt_t).abs() * m_t).sum() / (3.0 * nval)
    loss.backward()
    got = {k: p.grad.detach().cpu().numpy() for k, p in zip(PARAMS, params)}
    assert_grads_close(got, g_ref)
    # a second step through the same view: the scene is set again from the updated tensors
    with torch.no_grad():
        params[0].add_(0.001)
    for p in params:
        p.grad = None
    rgb2, _ = cg.render_fn(v, *params, rho2=rho2)
    (rgb2 * m_t).sum().backward()
    assert all(p.grad is not None and torch.isfinite(p.grad).all() for p in params)


def test_render_fn_backward_after_rerender_fails(cg):
    cam = S.pinhole(32, 24, 30.0)
    sc = S.uniform_box_scene(50, seed=3)
    ctx = cg.Context(0)
    v = ctx.view()
    v.set_camera_from(cam)
    params = _tensors(sc)
    rgb, _ = cg.render_fn(v, *params)
    v.render()                                      # replaces the view's adjoint state
    with pytest.raises(RuntimeError, match="adjoint state is gone"):
        rgb.sum().backward()


def _tiles_of(oracle_lib, cam, sc, k):
    """Pixels of the tiles the binning rule keeps for Gaussian k."""
    _, _, _, pas = oracle_lib.bin_counts(cam, sc.subset([k]), dense=True)
    tx, ty = oracle_lib.tile_grid(cam)
    tiles = np.nonzero(pas[0])[0]
    pix = []
    for t in tiles:
        x0, y0 = (t % tx) * oracle_lib.TILE, (t // tx) * oracle_lib.TILE
        for y in range(y0, min(y0 + oracle_lib.TILE, cam.height)):
            for x in range(x0, min(x0 + oracle_lib.TILE, cam.width)):
                pix.append(y * cam.width + x)
    return np.asarray(pix, np.int32)


def test_render_fn_finite_differences_fisheye_l1(cg, oracle_lib):
    cam = S.c3_camera(256, 256)
    sc = S.uniform_box_scene(32768, seed=0)
    tgt = S.perturbed(sc, seed=1)
    P = cam.n_pixels
    target = oracle_lib.render(cam, tgt).rgb
    ref = oracle_lib.render(cam, sc, eps=2e-4, max_used=64)
    valid = oracle_lib.rays(cam)[3]
    nval = int(valid.sum())
    mask = _l1_mask(ref, target, valid)

    # GPU: render_fn, L1 loss, loss.backward()
    ctx = cg.Context(0)
    v = ctx.view()
    v.set_camera_from(cam)
    params = _tensors(sc)
    rgb, _ = cg.render_fn(v, *params)
    tgt_t = torch.tensor(target.T.reshape(3, cam.height, cam.width), dtype=torch.float32, device="cuda")
    m_t = torch.tensor(mask.T.reshape(3, cam.height, cam.width), device="cuda")
    loss = ((rgb - tgt_t).abs() * m_t).sum() / (3.0 * nval)
    loss.backward()
    grads = [p.grad.detach().cpu().numpy().astype(np.float64) for p in params]

    # 64 random scalar parameters (seed 2) of Gaussians with a contributing pair
    contrib = np.unique(ref.used[ref.used >= 0])
    rng = np.random.default_rng(2)
    sizes = [3, 3, 4, 1, 3]              # means, log-scales, quaternion, logit, SH DC (degree 0)
    picks = []
    while len(picks) < 64:
        k = int(rng.choice(contrib))
        j = int(rng.integers(0, sum(sizes)))
        if (k, j) not in picks:
            picks.append((k, j))

    base64 = dataclasses.replace(sc, means=sc.means.astype(np.float64), log_scales=sc.log_scales.astype(np.float64),
                                 quats=sc.quats.astype(np.float64),
                                 opacity_logits=sc.opacity_logits.astype(np.float64), sh=sc.sh.astype(np.float64))

    def field(j):
        for f, (name, n) in enumerate(zip(("means", "log_scales", "quats", "opacity_logits", "sh"), sizes)):
            if j < n:
                return f, name, j
            j -= n

    def loss_at(k, name, j, delta, pix):
        arr = getattr(base64, name).copy()
        if name == "opacity_logits":
            arr[k] += delta
        elif name == "sh":
            arr[k, 0, j] += delta
        else:
            arr[k, j] += delta
        r = oracle_lib.render(cam, dataclasses.replace(base64, **{name: arr}), pix=pix)
        return float((np.abs(r.rgb - target[pix]) * mask[pix]).sum() / (3.0 * nval))

    pairs = []
    for k, jj in picks:
        f, name, j = field(jj)
        pix = _tiles_of(oracle_lib, cam, sc, k)
        p0 = float(getattr(base64, name)[k] if name == "opacity_logits" else
                   (getattr(base64, name)[k, 0, j] if name == "sh" else getattr(base64, name)[k, j]))
        h = 1e-6 * max(1.0, abs(p0))
        fd1 = (loss_at(k, name, j, h, pix) - loss_at(k, name, j, -h, pix)) / (2 * h)
        fd2 = (loss_at(k, name, j, h / 2, pix) - loss_at(k, name, j, -h / 2, pix)) / h
        if abs(fd1 - fd2) > 1e-4 * max(abs(fd1), 1e-9) + 1e-9:
            continue                     # a threshold within h: not differentiable here
        g = grads[f][k] if name == "opacity_logits" else (grads[f][k, 0, j] if name == "sh" else grads[f][k, j])
        pairs.append((name, k, j, float(g), fd1))
    assert len(pairs) >= 48
    scale = max(abs(p[4]) for p in pairs)
    for name, k, j, g, fd in pairs:
        assert abs(g - fd) <= 2e-3 * abs(fd) + 1e-5 * scale, (name, k, j, g, fd, scale)

"""Pins for the gradient oracle (oracle/grad.py): its forward equals the C
oracle's, and its autograd gradient equals FP64 central finite differences of
the C oracle's render."""
import dataclasses

import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")


def _small(seed=0, n=120, floor=False, deg=1):
    cam = S.pinhole(40, 30, 36.0, cam_to_world=S.look_at((0.05, 0.0, 0.0), (0.1, 0.05, 4.0)))
    sc = S.uniform_box_scene(n, seed=seed, log_scale_mean=-2.6, log_scale_std=0.4, sh_degree=deg)
    if floor:
        import oracle
        sc = sc.with_rho2(oracle.floor_rho2([S.pinhole(80, 60, 72.0)], sc.means).astype(np.float32))
    return cam, sc


def _as64(sc):
    return dataclasses.replace(sc, means=sc.means.astype(np.float64), log_scales=sc.log_scales.astype(np.float64),
                               quats=sc.quats.astype(np.float64),
                               opacity_logits=np.asarray(sc.opacity_logits, np.float64),
                               sh=sc.sh.astype(np.float64))


@pytest.mark.parametrize("mode", ["plain", "floor", "filter_none", "additive", "iso", "zf_floor"])
def test_torch_forward_equals_c_oracle(oracle_lib, mode):
    """The torch restatement (with its own basis for the isotropic variants)
    against the C oracle."""
    from oracle import grad as G
    cam, sc = _small(seed=1, floor=mode in ("floor", "additive", "zf_floor"))
    pix = np.arange(cam.n_pixels)
    filt = mode != "filter_none"
    add = mode == "additive"
    fp = {"iso": "iso", "zf_floor": "zf"}.get(mode, "own")
    cfilt = {"own": int(filt), "iso": oracle_lib.FILTER_ISO, "zf": oracle_lib.FILTER_ZF}[fp]
    params = {k: torch.tensor(np.asarray(getattr(sc, a), np.float64)) for k, a in
              (("means", "means"), ("log_scales", "log_scales"), ("quats", "quats"), ("logits", "opacity_logits"),
               ("sh", "sh"))}
    rgb, T = G.render_torch(cam, params, sc.sh_degree, torch.tensor(sc.rho2.astype(np.float64)), pix, filt, add,
                            footprint=fp)
    r = oracle_lib.render(cam, sc, filter=cfilt, comp=int(add), cull=False, eps=1e-9)
    ok = r.flags == 0
    tol = 1e-11 if fp == "own" else 1e-8   # the variants' bases differ; the FP32 camera rotation is unit to ~1e-7
    assert np.abs(rgb.numpy() - r.rgb)[ok].max() < tol
    assert np.abs(T.numpy() - r.T)[ok].max() < tol


def _loss_c(oracle_lib, cam, sc, pix, w_rgb, w_T, filt=1, comp=0):
    r = oracle_lib.render(cam, sc, pix=pix, filter=filt, comp=comp, cull=False)
    return float((r.rgb * w_rgb).sum() + (r.T * w_T).sum())


@pytest.mark.parametrize("floor", [False, True])
def test_gradient_equals_central_differences(oracle_lib, floor):
    from oracle import grad as G
    cam, sc = _small(seed=2, floor=floor)
    sc = _as64(sc)
    rng = np.random.default_rng(3)
    pix = np.arange(cam.n_pixels)
    w_rgb = rng.normal(size=(pix.size, 3))
    w_T = rng.normal(size=pix.size)
    L, g = G.loss_and_grad(cam, sc, pix, w_rgb, w_T)
    assert abs(L - _loss_c(oracle_lib, cam, sc, pix, w_rgb, w_T)) < 1e-9 * max(1.0, abs(L))
    fields = [("means", "means"), ("log_scales", "log_scales"), ("quats", "quats"), ("logits", "opacity_logits"),
              ("sh", "sh")]
    active = np.nonzero(np.abs(g["logits"]) > 1e-6)[0]
    checked, bad = 0, []
    for t in range(40):
        key, attr = fields[t % len(fields)]
        i = int(rng.choice(active))
        arr = getattr(sc, attr)
        idx = (i,) + tuple(rng.integers(0, s) for s in arr.shape[1:])
        base = float(arr[idx])
        fd = []
        for h in (1e-6 * max(1.0, abs(base)), 0.5e-6 * max(1.0, abs(base))):
            vals = []
            for sgn in (1, -1):
                a2 = arr.copy()
                a2[idx] = base + sgn * h
                vals.append(_loss_c(oracle_lib, cam, dataclasses.replace(sc, **{attr: a2}), pix, w_rgb, w_T))
            fd.append((vals[0] - vals[1]) / (2 * h))
        if abs(fd[0] - fd[1]) > 1e-4 * max(1.0, abs(fd[0])):
            continue                      # a compositing threshold lies within +-h: not differentiable here
        checked += 1
        an = float(g[key][idx])
        if abs(an - fd[0]) > 1e-5 * max(1.0, abs(fd[0])):
            bad.append((key, idx, an, fd[0]))
    assert checked >= 30 and not bad, bad

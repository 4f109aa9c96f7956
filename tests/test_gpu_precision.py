"""Half-precision storage: SH coefficients and opacity logits stored in BF16 or
FP16, evaluated and accumulated in FP32.  Against the FP64 oracle on the
quantised values the error stays at the FP32 level (1e-4); against the oracle
on the original FP32 values the stated budget is 2e-3 per RGB channel, away
from the compositing thresholds: quantisation moves a pair's response by up
to ~1e-3 relative, so pixels whose alpha or stop decisions lie that close to
a threshold (flag margin 5e-3) can flip a whole 1/255 contribution and are
counted separately."""
import dataclasses

import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_FLAG = 2e-4


def _quantised(sc, dtype):
    q = lambda a: torch.from_numpy(np.asarray(a, np.float32)).to(dtype).to(torch.float32).numpy()
    return dataclasses.replace(sc, sh=q(sc.sh), opacity_logits=q(sc.opacity_logits))


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_half_storage_error(oracle_lib, dtype):
    import paper_2609_13397_b300 as cg
    cam = S.pinhole(320, 180, 300.0)
    sc = S.blob_scene(20000, seed=5, cam=cam)
    sc = sc.with_rho2(oracle_lib.floor_rho2([S.pinhole(640, 360, 600.0)], sc.means).astype(np.float32))
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, storage=dtype)
    v = ctx.view()
    v.set_camera_from(cam)
    rgb, T = v.render()
    rgb = rgb.cpu().numpy().reshape(3, -1).T
    T = T.cpu().numpy().reshape(-1)
    rq = oracle_lib.render(cam, _quantised(sc, dtype), eps=EPS_FLAG)
    r0 = oracle_lib.render(cam, sc, eps=5e-3)
    okq = rq.flags == 0
    err_q = np.abs(rgb - rq.rgb)[okq].max()
    assert err_q <= 1e-4, err_q          # the arithmetic is FP32: only storage is half
    assert np.abs(T - rq.T)[okq].max() <= 1e-4
    ok0 = okq & (r0.flags == 0)
    assert ok0.mean() > 0.9
    err_0 = np.abs(rgb - r0.rgb)[ok0].max()
    assert err_0 <= 2e-3, err_0          # quantisation of SH / opacity stays within budget


def test_half_storage_adjoint(oracle_lib):
    import paper_2609_13397_b300 as cg
    from oracle import grad as G
    cam = S.pinhole(40, 30, 36.0, cam_to_world=S.look_at((0.05, 0.0, 0.0), (0.1, 0.05, 4.0)))
    sc = S.uniform_box_scene(150, seed=8, log_scale_mean=-2.6, log_scale_std=0.4, sh_degree=2)
    scq = _quantised(sc, torch.bfloat16)
    rng = np.random.default_rng(9)
    P = cam.n_pixels
    w_rgb, w_T = rng.normal(size=(P, 3)), rng.normal(size=P)
    ref = oracle_lib.render(cam, scq, eps=EPS_FLAG)
    w_rgb[ref.flags != 0] = 0.0
    w_T[ref.flags != 0] = 0.0
    _, g_ref = G.loss_and_grad(cam, scq, np.arange(P), w_rgb, w_T)
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, storage=torch.bfloat16)
    v = ctx.view()
    v.set_camera_from(cam)
    v.render(flags=cg.KEEP_FOR_BACKWARD)
    g = v.render_backward(torch.from_numpy(w_rgb.T.reshape(3, cam.height, cam.width).astype(np.float32)).cuda(),
                          torch.from_numpy(w_T.reshape(cam.height, cam.width).astype(np.float32)).cuda())
    torch.cuda.synchronize()
    for gk, ok in (("means", "means"), ("opacity_logits", "logits"), ("sh", "sh")):
        got = g[gk].cpu().numpy().astype(np.float64).reshape(g_ref[ok].shape)
        err = np.linalg.norm(got - g_ref[ok]) / np.linalg.norm(g_ref[ok])
        assert err < 2e-3, (gk, err)

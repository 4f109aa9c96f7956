"""Unscented-transform binning (CONEGS_BIN_UT, the 3DGUT-style backbone of
Sec. 3) on the GPU against the oracle's FP64 UT gate, through the C ABI.

Decisions the oracle finds within a relative 2e-3 of a threshold (the ellipse
test against k^2, the sigma points' domain limit) may go either way in FP32;
every other (Gaussian, tile) decision must match exactly, and pixels where an
ambiguous pair contributes are left out of the image comparison."""
import numpy as np
import pytest

import synthetic as S
from test_gpu_forward import CASES, EPS_FLAG, TOL, _setup, _with_floor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

UT_EPS = 2e-3
NAMES = ["c1", "kb160", "blob320", "ragged", "kb_ragged", "wide_surround", "kb_surround"]


@pytest.fixture(scope="module")
def cg():
    import paper_2609_13397_b300 as cg
    return cg


def _gate(oracle_lib, cam, sc):
    """UT gate with the angular-tile rule's FP32 pass rows for the Gaussians it keeps."""
    gate, status, _ = oracle_lib.ut_gate(cam, sc, eps=UT_EPS)
    _, _, _, pas = oracle_lib.bin_counts(cam, sc, dense=True)
    g = gate.copy()
    g[status == 0] = pas[status == 0]
    return gate, g, status


@pytest.mark.parametrize("name", NAMES)
def test_ut_pairs_match_oracle_gate(cg, oracle_lib, name):
    cam, sc = CASES[name]
    sc = _with_floor(oracle_lib, name, cam, sc)
    ctx, v = _setup(cg, cam, sc)
    v.render(flags=cg.BIN_UT)
    pg, pt = (t.cpu().numpy() for t in v.bin_counts())
    gate, g, status = _gate(oracle_lib, cam, sc)
    sure, near = (g == 1).sum(1), (g == 2).sum(1)
    assert (status == 1).sum() > 0
    assert np.all(pg >= sure) and np.all(pg <= sure + near)
    assert (near == 0).mean() > 0.9
    assert v.stats()["n_pairs"] == pg.sum()
    # every listed pair is allowed by the gate, every sure pair is listed, lists in depth order
    gid, rng = (t.cpu().numpy() for t in v.pairs())
    L = oracle_lib.bin_gauss(cam, sc)[:, 3]
    for t in range(rng.shape[0]):
        got = gid[rng[t, 0]:rng[t, 1]]
        assert np.all(g[got, t] >= 1), t
        assert np.isin(np.nonzero(g[:, t] == 1)[0], got).all(), t
        assert np.array_equal(got, got[np.lexsort((got, L[got]))]), t
    assert np.array_equal(pt, np.diff(rng, axis=1).reshape(-1))


@pytest.mark.parametrize("name", NAMES)
def test_ut_render_matches_oracle(cg, oracle_lib, name):
    cam, sc = CASES[name]
    sc = _with_floor(oracle_lib, name, cam, sc)
    gate, _, _ = _gate(oracle_lib, cam, sc)
    ctx, v = _setup(cg, cam, sc)
    rgb, T = v.render(flags=cg.BIN_UT)
    rgb = rgb.cpu().numpy().reshape(3, -1).T
    T = T.cpu().numpy().reshape(-1)
    r = oracle_lib.render(cam, sc, eps=EPS_FLAG, gate=gate)
    ok = r.flags == 0
    assert (~ok).sum() <= 0.03 * ok.size
    assert np.abs(rgb - r.rgb)[ok].max(initial=0.0) <= TOL
    assert np.abs(T - r.T)[ok].max(initial=0.0) <= TOL


def test_ut_keeps_fewer_pairs_and_loses_little(cg, oracle_lib):
    """On the 320x180 blob scene UT binning keeps fewer pairs than the
    angular-tile rule and its image stays close to the exact one."""
    cam, sc = CASES["blob320"]
    sc = _with_floor(oracle_lib, "blob320", cam, sc)
    ctx, v = _setup(cg, cam, sc)
    a, ta = v.render()
    n_rule = v.stats()["n_pairs"]
    b, tb = v.render(flags=cg.BIN_UT)
    n_ut = v.stats()["n_pairs"]
    assert n_ut < n_rule
    assert float((a - b).abs().mean()) < 1e-3


def test_ut_backward_lossless_scene(cg):
    """Small distant Gaussians: UT binning drops no contributing pair, so the UT
    render and its adjoint equal the angular-tile rule's up to FP32 rounding."""
    rng = np.random.default_rng(4)
    n = 400
    cam = S.pinhole(96, 72, 90.0)
    means = np.stack([rng.uniform(-1.2, 1.2, n), rng.uniform(-0.9, 0.9, n), rng.uniform(6, 10, n)], 1)
    sh = np.zeros((n, 4, 3), np.float32)
    sh[:, 0] = rng.uniform(-1, 1, (n, 3))
    sh[:, 1:] = rng.normal(0, 0.2, (n, 3, 3))
    sc = S.Scene(means.astype(np.float32), rng.normal(-3.5, 0.4, (n, 3)).astype(np.float32),
                 S._random_quats(rng, n), rng.normal(1.0, 1.0, n).astype(np.float32), sh, 1,
                 np.zeros(n, np.float32))
    ctx, v = _setup(cg, cam, sc)
    w = torch.randn(3, cam.height, cam.width, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    out = {}
    for flags in (0, cg.BIN_UT):
        rgb, T = v.render(flags=flags | cg.KEEP_FOR_BACKWARD)
        g = v.render_backward(w)
        torch.cuda.synchronize()
        out[flags] = (rgb.clone(), T.clone(), {k: t.clone() for k, t in g.items()}, v.stats()["n_pairs"])
    a, b = out[0], out[cg.BIN_UT]
    assert b[3] < a[3]
    assert float((a[0] - b[0]).abs().max()) < 1e-5 and float((a[1] - b[1]).abs().max()) < 1e-5
    for k in a[2]:
        scale = float(a[2][k].abs().max()) + 1e-12
        assert float((a[2][k] - b[2][k]).abs().max()) <= 1e-4 * scale, k


def test_ut_flag_combines_with_variants(cg, oracle_lib):
    """BIN_UT with FILTER_ISO: the gate is the same, the response is the variant's."""
    cam, sc = CASES["c1"]
    gate, _, _ = _gate(oracle_lib, cam, sc)
    ctx, v = _setup(cg, cam, sc)
    rgb, T = v.render(flags=cg.BIN_UT | cg.FILTER_ISO)
    rgb = rgb.cpu().numpy().reshape(3, -1).T
    r = oracle_lib.render(cam, sc, eps=EPS_FLAG, gate=gate, filter=oracle_lib.FILTER_ISO)
    ok = r.flags == 0
    assert np.abs(rgb - r.rgb)[ok].max(initial=0.0) <= TOL

"""The conservative angular-tile binning rule (FP32 emulation in the oracle) checked
against FP64 truth: no pixel-Gaussian pair that can reach alpha >= 1/255 may fall in
a tile the rule rejects, and every tile cone must contain its pixels' FP64 rays."""
import math

import numpy as np
import pytest

import synthetic as S


def _cases():
    c1cam, c1sc = S.c1()
    kb = S.c3_camera(96, 96)
    kb_sc = S.uniform_box_scene(400, seed=3)
    blob_cam = S.pinhole(160, 90, 150.0)
    blob_sc = S.blob_scene(3000, seed=1, cam=blob_cam)
    ragged = S.pinhole(70, 45, 40.0, 33.0, 21.0, cam_to_world=S.look_at((0.1, 0.0, -0.5), (0.2, 0.1, 4.0)))
    rag_sc = S.uniform_box_scene(500, seed=9, log_scale_mean=-2.5)
    # strongly anisotropic Gaussians (log-scales N(-3, 1.5) per axis) around and in front of a
    # wide, rotated pinhole with fx != fy: silhouette ellipses of every aspect, near the
    # grazing limit, and cameras close to or inside the bound
    wide = S.Camera(S.PINHOLE, 96, 64, 30.0, 36.0, 50.5, 30.25,
                    cam_to_world=S.look_at((0.0, 0.1, 0.0), (1.0, 0.4, 2.0)))
    an_sc = S.blob_scene(3000, seed=21, cam=wide, blob_frac=0.5, shell=(0.8, 4.0), log_scale_mean=-3.0,
                         log_scale_std=1.5, sh_degree=0)
    # the same kind of shell around a rotated fisheye with an off-centre principal point:
    # Gaussians behind the camera, near the valid circle's rim and across the axis
    fk = S.c3_camera(96, 80, seed=2)
    fk = S.Camera(fk.model, fk.width, fk.height, fk.fx, fk.fy, 49.0, 38.5, k=fk.k,
                  cam_to_world=S.look_at((0.1, 0.0, 0.1), (-1.0, 0.5, 2.0)), theta_lim=fk.theta_lim)
    fk_sc = S.blob_scene(3000, seed=23, cam=S.pinhole(96, 80, 50.0), blob_frac=0.3, shell=(0.8, 4.0),
                         log_scale_mean=-3.0, log_scale_std=1.2, sh_degree=0)
    return {"c1": (c1cam, c1sc), "kb96": (kb, kb_sc), "blob160": (blob_cam, blob_sc), "ragged": (ragged, rag_sc),
            "aniso_wide": (wide, an_sc), "kb_shell": (fk, fk_sc)}


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_binning_is_conservative(oracle_lib, name):
    O = oracle_lib
    cam, sc = CASES[name]
    if name == "blob160":
        floor_cam = S.pinhole(320, 180, 300.0)
        sc = sc.with_rho2(O.floor_rho2([floor_cam], sc.means).astype(np.float32))
    total, pg, pt, pas = O.bin_counts(cam, sc, dense=True)
    pix, g = O.pairs_above(cam, sc, (1.0 / 255.0) * (1 - 1e-3))
    assert pix.size > 0
    tx, _ = O.tile_grid(cam)
    tile = (pix // cam.width) // O.TILE * tx + (pix % cam.width) // O.TILE
    missed = pas[g, tile] == 0
    assert missed.sum() == 0, f"{missed.sum()} of {pix.size} contributing pairs not binned"
    # the rule should not be wildly loose either (pairs per contributing pair)
    assert total == pas.sum() and total >= np.unique(g * 100000 + tile).size


@pytest.mark.parametrize("name", list(CASES))
def test_tile_cones_contain_fp64_rays(oracle_lib, name):
    O = oracle_lib
    cam, _ = CASES[name]
    table = O.tile_table(cam)
    d, _, _, valid = O.rays(cam)
    tx, _ = O.tile_grid(cam)
    ii = np.arange(cam.width * cam.height)
    T_ = oracle_lib.TILE
    tile = (ii // cam.width) // T_ * tx + (ii % cam.width) // T_
    a = table[tile, :3].astype(float)
    sg = table[tile, 3].astype(float)
    chord = np.linalg.norm(a - d, axis=1)
    ok = ~valid | (chord <= 2 * sg)
    assert ok.all()
    # every tile with a valid pixel is non-empty; empty tiles have no valid pixel
    has_valid = np.bincount(tile[valid], minlength=table.shape[0]) > 0
    assert np.array_equal(has_valid, table[:, 3] >= 0)
    # footprint bound m >= (|dx|^2 + |dy|^2)/3 for every pixel of the tile
    _, dx, dy, _ = O.rays(cam)
    m = ((dx ** 2).sum(1) + (dy ** 2).sum(1)) / 3
    assert (m[valid] <= table[tile[valid], 5]).all()


def test_fp32_rule_directions_track_fp64(oracle_lib):
    for cam in (S.pinhole(1280, 720, 1200.0), S.c3_camera(512, 512)):
        rng = np.random.default_rng(0)
        xs = rng.uniform(0, cam.width, 4000).astype(np.float32)
        ys = rng.uniform(0, cam.height, 4000).astype(np.float32)
        f, valid = oracle_lib.fdir(cam, xs, ys)
        d, _, _, v64 = oracle_lib.rays(cam, xs.astype(float), ys.astype(float))
        assert np.array_equal(valid, v64)
        err = np.linalg.norm(f[valid] - d[valid], axis=1).max()
        assert err < 1e-6


def test_rule_culls_transparent_and_keeps_near(oracle_lib):
    cam = S.pinhole(64, 48, 60.0)
    sc = S.uniform_box_scene(3, seed=0)
    sc.opacity_logits[:] = np.array([math.log(1 / 300.0 / (1 - 1 / 300.0)), 0.0, 0.0], np.float32)
    sc.means[2] = np.array([0.0, 0.0, 0.01], np.float32)     # almost at the optical centre
    recs = oracle_lib.bin_gauss(cam, sc)
    assert recs[0, 9] == 0.0            # sigma < 1/255: can never contribute
    total, pg, pt, _ = oracle_lib.bin_counts(cam, sc)
    assert pg[0] == 0 and pg[2] == pt.size   # the near Gaussian covers every tile


def _random_case(seed):
    """A random small camera (pinhole or Kannala-Brandt, random pose, intrinsics and
    distortion) inside a random mixture of clustered and surrounding Gaussians with
    random size statistics."""
    rng = np.random.default_rng(1000 + seed)
    w, h = int(rng.integers(40, 90)), int(rng.integers(30, 70))
    eye = rng.normal(0, 0.3, 3)
    target = eye + rng.normal(0, 1, 3) + np.array([0.0, 0.0, 2.0])
    pose = S.look_at(eye, target)
    if seed % 2 == 0:
        f = float(rng.uniform(0.4, 1.5) * w)
        cam = S.Camera(S.PINHOLE, w, h, f, f * float(rng.uniform(0.8, 1.25)), w * float(rng.uniform(0.3, 0.7)),
                       h * float(rng.uniform(0.3, 0.7)), cam_to_world=pose)
    else:
        base = S.c3_camera(w, w, seed=seed)
        cam = S.Camera(base.model, w, h, base.fx, base.fy, w * float(rng.uniform(0.4, 0.6)),
                       h * float(rng.uniform(0.4, 0.6)), k=base.k, cam_to_world=pose, theta_lim=base.theta_lim)
    sc = S.blob_scene(700, seed=seed, cam=S.pinhole(w, h, 0.8 * w, cam_to_world=pose),
                      blob_frac=float(rng.uniform(0.2, 0.8)), shell=(0.6, 5.0),
                      log_scale_mean=float(rng.uniform(-4.0, -2.0)), log_scale_std=float(rng.uniform(0.3, 1.5)),
                      sh_degree=0)
    return cam, sc


@pytest.mark.parametrize("seed", range(8))
def test_binning_is_conservative_random(oracle_lib, seed):
    """Random cameras and scenes: no pair that can reach alpha >= 1/255 falls in a
    tile the rule (cone and silhouette tests) rejects."""
    O = oracle_lib
    cam, sc = _random_case(seed)
    total, pg, pt, pas = O.bin_counts(cam, sc, dense=True)
    pix, g = O.pairs_above(cam, sc, (1.0 / 255.0) * (1 - 1e-3))
    tx, _ = O.tile_grid(cam)
    tile = (pix // cam.width) // O.TILE * tx + (pix % cam.width) // O.TILE
    missed = pas[g, tile] == 0
    assert missed.sum() == 0, f"{missed.sum()} of {pix.size} contributing pairs not binned"


def _lowres_case(seed):
    """A very low-resolution camera (12-40 px wide: large footprints, so the t* bound
    and its anisotropy factor decide most tiles) inside close, strongly anisotropic
    Gaussians (log-scale std 1.5, shell from 0.3), some with the Eq. 11 floor."""
    rng = np.random.default_rng(5000 + seed)
    w = int(rng.integers(12, 40))
    h = int(w * rng.uniform(0.56, 1.0))
    eye = rng.normal(0, 0.3, 3)
    pose = S.look_at(eye, eye + rng.normal(0, 1, 3) + np.array([0.0, 0.0, 2.0]))
    if seed % 2 == 0:
        f = float(rng.uniform(0.4, 1.2) * w)
        cam = S.Camera(S.PINHOLE, w, h, f, f, w / 2, h / 2, cam_to_world=pose)
    else:
        base = S.c3_camera(w, w, seed=seed)
        cam = S.Camera(base.model, w, h, base.fx, base.fy, w / 2, h / 2, k=base.k, cam_to_world=pose,
                       theta_lim=base.theta_lim)
    sc = S.blob_scene(1500, seed=seed, cam=S.pinhole(w, h, 0.8 * w, cam_to_world=pose), blob_frac=0.3,
                      shell=(0.3, 3.0), log_scale_mean=float(rng.uniform(-3.0, -1.5)), log_scale_std=1.5,
                      sh_degree=0)
    return cam, sc


@pytest.mark.parametrize("seed", range(6))
def test_binning_is_conservative_lowres(oracle_lib, seed):
    """Where the anisotropy factor of the t* bound, r1 = (r + 1/r)/2, decides:
    no pair that can reach alpha >= 1/255 is lost."""
    O = oracle_lib
    cam, sc = _lowres_case(seed)
    if seed % 3 == 0:
        fcam = S.Camera(S.PINHOLE, 4 * cam.width, 4 * cam.height, 3.2 * cam.width, 3.2 * cam.width,
                        2.0 * cam.width, 2.0 * cam.height, cam_to_world=cam.cam_to_world)
        sc = sc.with_rho2(O.floor_rho2([fcam], sc.means).astype(np.float32))
    total, pg, pt, pas = O.bin_counts(cam, sc, dense=True)
    pix, g = O.pairs_above(cam, sc, (1.0 / 255.0) * (1 - 1e-3))
    assert pix.size > 1000
    tx, _ = O.tile_grid(cam)
    tile = (pix // cam.width) // O.TILE * tx + (pix % cam.width) // O.TILE
    missed = pas[g, tile] == 0
    assert missed.sum() == 0, f"{missed.sum()} of {pix.size} contributing pairs not binned"
    # not every Gaussian may pass every tile (the bound must decide somewhere)
    assert total < (pg > 0).sum() * pt.size

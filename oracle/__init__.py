"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It loads ``liboracle.so`` built from
``conegs_oracle.c`` (plain C, FP64, OpenMP) and shares no code with the CUDA
library in ``paper_2609_13397_b300``.

Functions follow the paper's notation; see the header of conegs_oracle.c for
the list of equations each step implements and the readings taken where the
paper is silent.  ``grad.py`` holds the gradient oracle (PyTorch FP64 CPU).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "conegs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

FILTER_NONE, FILTER_ANISO, FILTER_ISO, FILTER_ZF = 0, 1, 2, 3
COMP_MARGINAL, COMP_ADDITIVE = 0, 1
FL_ALPHA_MIN, FL_ALPHA_MAX, FL_STOP, FL_KEY_TIE, FL_TNEAR, FL_UT_NEAR = 1, 2, 4, 8, 16, 32
UT_DROP, UT_KEEP, UT_NEAR = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, FP64, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared",
               "-fPIC", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB_PATH)
        _lib.or_pair_detail.restype = ctypes.c_int
        _lib.or_pair_rays.restype = ctypes.c_double
        _lib.or_bundle.restype = ctypes.c_double
        _lib.or_pairs_above.restype = ctypes.c_long
        _lib.or_bin_counts.restype = ctypes.c_long
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_ut_rect_min.restype = ctypes.c_double
        _lib.or_ut_rect_min.argtypes = [ctypes.c_double] * 9
        for name in ("or_pair_detail", "or_bundle"):
            getattr(_lib, name).argtypes = None
    return _lib


def _p(a: np.ndarray, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, np.float64))


def _f(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, np.float32))


def pack_camera(cam) -> np.ndarray:
    c2w = np.asarray(cam.cam_to_world, np.float64).reshape(3, 4)
    return _d([cam.model, cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, *np.asarray(cam.k, np.float64),
               *c2w[:, :3].reshape(-1), *c2w[:, 3], cam.theta_lim])


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int) -> None:
    """Host threads of the oracle's parallel loops from now on (timing only)."""
    lib().or_set_threads(int(n))


def sh_basis(v) -> np.ndarray:
    """The oracle's real SH basis (degrees 0-3, 16 values) of directions v [n,3]."""
    v = _d(np.atleast_2d(v))
    out = np.zeros((v.shape[0], 16))
    lib().or_sh_basis(ctypes.c_int(v.shape[0]), _p(v), _p(out))
    return out


# ------------------------------------------------------------------ rays

def rays(cam, xs=None, ys=None):
    """FP64 d, delta_x, delta_y ([n,3] each) and the valid mask for image points
    (default: every pixel centre, row-major)."""
    if xs is None:
        jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
        xs, ys = ii.reshape(-1) + 0.5, jj.reshape(-1) + 0.5
    xs, ys = _d(xs), _d(ys)
    n = xs.size
    d, dx, dy = (np.zeros((n, 3)) for _ in range(3))
    valid = np.zeros(n, np.int32)
    lib().or_rays(_p(pack_camera(cam)), ctypes.c_int(n), _p(xs), _p(ys), _p(d), _p(dx), _p(dy),
                  _p(valid, ctypes.c_int))
    return d, dx, dy, valid.astype(bool)


def fdir(cam, xs, ys):
    """The binning rule's FP32 ray directions of image points (bit-exact emulation)."""
    xs, ys = _f(xs), _f(ys)
    n = xs.size
    out = np.zeros((n, 3), np.float32)
    valid = np.zeros(n, np.int32)
    lib().or_fdir(_p(pack_camera(cam)), ctypes.c_int(n), _p(xs, ctypes.c_float), _p(ys, ctypes.c_float),
                  _p(out, ctypes.c_float), _p(valid, ctypes.c_int))
    return out, valid.astype(bool)


# ------------------------------------------------------------------ gaussians / pairs

def gauss(cam, scene) -> np.ndarray:
    """Per-Gaussian FP64 quantities [n,24]: W(9) W^-1(9) sigma_eff rgb(3) L rho2."""
    n = scene.n
    out = np.zeros((n, 24))
    lib().or_gauss(_p(pack_camera(cam)), ctypes.c_int(n), _p(_d(scene.means)), _p(_d(scene.log_scales)),
                   _p(_d(scene.quats)), _p(_d(scene.opacity_logits)), _p(_d(scene.sh)),
                   ctypes.c_int(scene.sh_degree), _p(_d(scene.rho2)), _p(out))
    return out


DETAIL_KEYS = {"T": 0, "ts": 1, "q": slice(2, 5), "du": slice(5, 8), "ex": slice(8, 11), "ey": slice(11, 14),
               "Sfp": slice(14, 23), "Sr": slice(23, 32), "detA": 32, "Q": 33, "D2": 34, "d": slice(40, 43),
               "dx": slice(43, 46), "dy": slice(46, 49), "sig_eff": 49}


def _unpack_detail(det: np.ndarray) -> dict:
    out = {}
    for k, s in DETAIL_KEYS.items():
        v = det[s]
        if k in ("Sfp", "Sr"):
            v = v.reshape(3, 3)
        out[k] = v.copy() if isinstance(v, np.ndarray) else float(v)
    return out


def pair(cam, x: float, y: float, mu, log_scales, quat, logit: float, rho2: float = 0.0,
         filter: int = FILTER_ANISO, comp: int = COMP_MARGINAL) -> Optional[dict]:
    """One pixel-Gaussian pair at image point (x, y) with every intermediate of Eq. 2-12."""
    det = np.zeros(64)
    L = lib()
    ok = L.or_pair_detail(_p(pack_camera(cam)), ctypes.c_double(x), ctypes.c_double(y), _p(_d(mu)),
                          _p(_d(log_scales)), _p(_d(quat)), ctypes.c_double(logit), ctypes.c_double(rho2),
                          ctypes.c_int(filter), ctypes.c_int(comp), _p(det))
    if ok < 0:
        return None
    out = _unpack_detail(det)
    out["valid_depth"] = bool(ok)
    return out


def pair_rays(o, d, dx, dy, mu, log_scales, quat, logit, rho2=0.0, filter=FILTER_ANISO,
              comp=COMP_MARGINAL) -> dict:
    """Pair response for explicit rays d (unit) and differentials dx, dy."""
    det = np.zeros(64)
    L = lib()
    L.or_pair_rays.argtypes = [ctypes.POINTER(ctypes.c_double)] * 7 + [ctypes.c_double] * 2 + \
        [ctypes.c_int] * 2 + [ctypes.POINTER(ctypes.c_double)]
    L.or_pair_rays(_p(_d(o)), _p(_d(d)), _p(_d(dx)), _p(_d(dy)), _p(_d(mu)), _p(_d(log_scales)),
                   _p(_d(quat)), logit, rho2, filter, comp, _p(det))
    return _unpack_detail(det)


def bundle(cam, x, y, mu, log_scales, quat, logit, rho2=0.0, nsub=32) -> float:
    """Supersampled pixel-bundle reference (nsub x nsub sub-rays, centre-ray response each)."""
    return float(lib().or_bundle(_p(pack_camera(cam)), ctypes.c_double(x), ctypes.c_double(y), _p(_d(mu)),
                                 _p(_d(log_scales)), _p(_d(quat)), ctypes.c_double(logit),
                                 ctypes.c_double(rho2), ctypes.c_int(nsub)))


# ------------------------------------------------------------------ render

class Render:
    """Oracle render of a set of pixels: rgb [n,3], T [n], flags [n], ncontrib [n]."""

    def __init__(self, rgb, T, flags, ncontrib, pix, used=None):
        self.rgb, self.T, self.flags, self.ncontrib, self.pix, self.used = rgb, T, flags, ncontrib, pix, used


def render(cam, scene, pix: Optional[Sequence[int]] = None, filter: int = FILTER_ANISO,
           comp: int = COMP_MARGINAL, cull: bool = True, eps: float = 1e-5, eps_key: float = 0.0,
           max_used: int = 0, order: int = 0, gate: Optional[np.ndarray] = None) -> Render:
    """Render pixels (indices into the row-major W x H grid; None = all).  order: 0
    the canonical per-Gaussian key |mu - o|, 1 the exact per-ray t* order (with
    eps_key > 0, near ties in t* between pairs that may contribute set FL_KEY_TIE).
    gate: a [n, ntiles] UT gate (``ut_gate``): only kept tiles are evaluated; pixels
    where an ambiguous entry contributes get FL_UT_NEAR.  The result's ``nalpha``:
    per pixel, the pairs with T >= 1/255 (reached before the stop or not)."""
    if gate is not None:
        gate = np.ascontiguousarray(gate, np.uint8)
        tx, ty = tile_grid(cam)
        assert gate.shape == (scene.n, tx * ty)
    n = scene.n
    if pix is None:
        npix, pix_arr, pptr = cam.width * cam.height, None, None
    else:
        pix_arr = np.ascontiguousarray(np.asarray(pix, np.int32))
        npix, pptr = pix_arr.size, _p(pix_arr, ctypes.c_int)
    rgb = np.zeros((npix, 3))
    T = np.zeros(npix)
    flags = np.zeros(npix, np.int32)
    ncon = np.zeros(npix, np.int32)
    used = np.full((npix, max(max_used, 1)), -1, np.int32)
    nalpha = np.zeros(npix, np.int32)
    lib().or_render(_p(pack_camera(cam)), ctypes.c_int(n), _p(_d(scene.means)), _p(_d(scene.log_scales)),
                    _p(_d(scene.quats)), _p(_d(scene.opacity_logits)), _p(_d(scene.sh)),
                    ctypes.c_int(scene.sh_degree), _p(_d(scene.rho2)), ctypes.c_int(filter), ctypes.c_int(comp),
                    ctypes.c_int(npix), pptr, ctypes.c_int(int(cull)), ctypes.c_double(eps),
                    ctypes.c_double(eps_key), _p(rgb), _p(T), _p(flags, ctypes.c_int), _p(ncon, ctypes.c_int),
                    _p(used, ctypes.c_int) if max_used > 0 else None, ctypes.c_int(max_used), ctypes.c_int(order),
                    _p(gate, ctypes.c_ubyte) if gate is not None else None, _p(nalpha, ctypes.c_int))
    r = Render(rgb, T, flags, ncon, pix_arr, used if max_used > 0 else None)
    r.nalpha = nalpha
    return r


def render_subrays(cam, scene, pix: Optional[Sequence[int]] = None, nsub: int = 8, order: int = 0):
    """Dense sub-ray reference: nsub x nsub centre rays per pixel, each composited on
    its own (centre-ray responses), averaged.  Returns (rgb [n,3], T [n])."""
    n = scene.n
    if pix is None:
        npix, pptr = cam.width * cam.height, None
    else:
        pix_arr = np.ascontiguousarray(np.asarray(pix, np.int32))
        npix, pptr = pix_arr.size, _p(pix_arr, ctypes.c_int)
    rgb = np.zeros((npix, 3))
    T = np.zeros(npix)
    lib().or_render_subrays(_p(pack_camera(cam)), ctypes.c_int(n), _p(_d(scene.means)), _p(_d(scene.log_scales)),
                            _p(_d(scene.quats)), _p(_d(scene.opacity_logits)), _p(_d(scene.sh)),
                            ctypes.c_int(scene.sh_degree), _p(_d(scene.rho2)), ctypes.c_int(npix), pptr,
                            ctypes.c_int(nsub), ctypes.c_int(order), _p(rgb), _p(T))
    return rgb, T


def pairs_above(cam, scene, thr: float, cap: int = 10_000_000):
    """Every (pixel, Gaussian) pair with T >= thr (brute force, FP64)."""
    pix = np.zeros(cap, np.int32)
    g = np.zeros(cap, np.int32)
    cnt = lib().or_pairs_above(_p(pack_camera(cam)), ctypes.c_int(scene.n), _p(_d(scene.means)),
                               _p(_d(scene.log_scales)), _p(_d(scene.quats)), _p(_d(scene.opacity_logits)),
                               _p(_d(scene.rho2)), ctypes.c_double(thr), ctypes.c_long(cap),
                               _p(pix, ctypes.c_int), _p(g, ctypes.c_int))
    cnt = int(cnt)
    if cnt > cap:
        raise RuntimeError("pairs_above: capacity exceeded")
    return pix[:cnt].copy(), g[:cnt].copy()


def floor_rho2(cams, means) -> np.ndarray:
    """Eq. 11 training-frequency floor over the views ``cams``."""
    packed = np.ascontiguousarray(np.concatenate([pack_camera(c) for c in cams]))
    means = _d(means)
    n = means.shape[0]
    out = np.zeros(n)
    lib().or_floor(ctypes.c_int(len(cams)), _p(packed), ctypes.c_int(n), _p(means), _p(out))
    return out


# ------------------------------------------------------------------ FP32 binning emulation

TILE = 8   # tile side (pixels) of the binning rule


def tile_grid(cam):
    return (cam.width + TILE - 1) // TILE, (cam.height + TILE - 1) // TILE


def tile_table(cam) -> np.ndarray:
    tx, ty = tile_grid(cam)
    out = np.zeros((tx * ty, 6), np.float32)
    lib().or_tile_table(_p(pack_camera(cam)), _p(out, ctypes.c_float))
    return out


def bin_gauss(cam, scene) -> np.ndarray:
    """Per-Gaussian binning records [n,16]: u (3), L, kap, ks, kr, r1sq, s2, flag, Sigma_eff (6)."""
    n = scene.n
    out = np.zeros((n, 16), np.float32)
    lib().or_bin_gauss(_p(pack_camera(cam)), ctypes.c_int(n), _p(_f(scene.means), ctypes.c_float),
                       _p(_f(scene.log_scales), ctypes.c_float), _p(_f(scene.quats), ctypes.c_float),
                       _p(_f(scene.opacity_logits), ctypes.c_float), _p(_f(scene.rho2), ctypes.c_float),
                       _p(out, ctypes.c_float))
    return out


def zf_footprint_bound(cam) -> np.float32:
    """FP32 bound 1/(6 f_x^2) of the z/f pseudo-differentials' (|dx|^2 + |dy|^2)/3,
    by the op sequence the GPU rule uses (fx * fx, times 6, 1 over)."""
    fx = np.float32(cam.fx)
    return np.float32(1.0) / (np.float32(6.0) * (fx * fx))


def bin_counts(cam, scene, dense: bool = False, zf: bool = False):
    """Per-Gaussian and per-tile pair counts of the binning rule (FP32 emulation);
    with dense=True also the [n, ntiles] pass matrix.  zf=True: the rule's
    footprint bound m of every tile raised to the z/f variant's 1/(6 f_x^2)."""
    table = tile_table(cam)
    if zf:
        live = table[:, 3] >= 0
        table[live, 5] = np.maximum(table[live, 5], zf_footprint_bound(cam))
    recs = bin_gauss(cam, scene)
    n, nt = scene.n, table.shape[0]
    pg = np.zeros(n, np.int32)
    pt = np.zeros(nt, np.int32)
    pas = np.zeros((n, nt), np.uint8) if dense else None
    means = _f(scene.means)
    total = lib().or_bin_counts(_p(pack_camera(cam)), _p(table, ctypes.c_float), ctypes.c_int(n),
                                _p(recs, ctypes.c_float), _p(means, ctypes.c_float), _p(pg, ctypes.c_int),
                                _p(pt, ctypes.c_int), _p(pas, ctypes.c_ubyte) if dense else None)
    return int(total), pg, pt, pas


# ------------------------------------------------------------------ UT binning (3DGUT-style backbone)

def ut_rect_min(c, conic, rect) -> float:
    """min over the rectangle (x0, x1, y0, y1) of (y - c)^T [[A,B],[B,C]] (y - c)."""
    A, B, C = conic
    x0, x1, y0, y1 = rect
    return float(lib().or_ut_rect_min(float(c[0]), float(c[1]), float(A), float(B), float(C),
                                      float(x0), float(x1), float(y0), float(y1)))


def ut_gate(cam, scene, eps: float = 2e-3):
    """Unscented-transform binning gate (definition in conegs_oracle.c).

    Returns (gate [n, ntiles] uint8: 0 drop / 1 keep / 2 ambiguous, status [n]:
    0 the angular-tile rule decides / 1 UT / 2 ambiguous domain decision,
    geo [n, 6]: ybar, conic A B C, k^2 of status-1 Gaussians).  The angular-tile
    rule's flags come from its FP32 emulation (``bin_gauss``)."""
    n = scene.n
    tx, ty = tile_grid(cam)
    flags = np.ascontiguousarray(bin_gauss(cam, scene)[:, 9].astype(np.int32))
    gate = np.zeros((n, tx * ty), np.uint8)
    status = np.zeros(n, np.int32)
    geo = np.zeros((n, 6))
    lib().or_ut_gate(_p(pack_camera(cam)), ctypes.c_int(n), _p(_d(scene.means)), _p(_d(scene.log_scales)),
                     _p(_d(scene.quats)), _p(_d(scene.opacity_logits)), _p(_d(scene.rho2)),
                     _p(flags, ctypes.c_int), ctypes.c_double(eps), _p(gate, ctypes.c_ubyte),
                     _p(status, ctypes.c_int), _p(geo))
    return gate, status, geo


def ut_bin_counts(cam, scene, eps: float = 2e-3):
    """Per-Gaussian pair counts of UT binning: (sure [n], near [n], status [n]).
    UT Gaussians keep between sure and sure + near tiles; the others keep
    exactly their angular-tile rule count (FP32 emulation), which is ``sure``."""
    gate, status, _ = ut_gate(cam, scene, eps)
    _, _, _, pas = bin_counts(cam, scene, dense=True)
    cone = status == 0
    gate[cone] = pas[cone]
    return (gate == UT_KEEP).sum(1).astype(np.int64), (gate == UT_NEAR).sum(1).astype(np.int64), status

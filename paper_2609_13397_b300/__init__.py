"""B300 (sm_103a) ConeGaussian renderer: Python binding of include/conegs.h.

Every step of the render and its adjoint runs in the CUDA library
(libconegs.so); this module only marshals torch tensors (device memory and
streams) into the C calls.

    ctx = Context(device=0)
    ctx.set_scene(means, log_scales, quats, opacity_logits, sh, sh_degree, rho2)
    view = ctx.view()
    view.set_camera(model, width, height, (fx, fy, cx, cy), k, cam_to_world, theta_lim)
    rgb, T = view.render()

Differentiable form (the hand-written adjoint behind torch.autograd):

    rgb, T = render_fn(view, means, log_scales, quats, opacity_logits, sh)
    loss(rgb, T).backward()        # fills .grad of the five parameter tensors
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import ConegsError, check, lib

PINHOLE, KB_FISHEYE = 0, 1
F32, BF16, F16 = 0, 1, 2
(FILTER_NONE, COMP_ADDITIVE, KEEP_FOR_BACKWARD, PROFILE, FILTER_ISO, FILTER_ZF, BIN_UT, ORDER_TSTAR, PRETEST_RAY,
 PRETEST_OFF) = (1, 2, 4, 8, 16, 32, 64, 128, 256, 512)

_DTYPE_CODE = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}

__all__ = ["Context", "View", "ConegsError", "PINHOLE", "KB_FISHEYE", "FILTER_NONE", "COMP_ADDITIVE",
           "KEEP_FOR_BACKWARD", "PROFILE", "FILTER_ISO", "FILTER_ZF", "BIN_UT", "ORDER_TSTAR", "PRETEST_RAY",
           "PRETEST_OFF",
           "radix_sort_pairs", "render_fn", "measure_fp32_peak"]


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, device, dtype=torch.float32) -> torch.Tensor:
    return t.to(device=device, dtype=dtype).contiguous()


def _host_f32(x, n: int):
    if x is None:
        return None
    arr = (ctypes.c_float * n)(*[float(v) for v in list(torch.as_tensor(x, dtype=torch.float64).reshape(-1))])
    return arr


class Context:
    """A scene resident on one CUDA device plus its views."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        lib()
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        check(lib().conegs_create(ctypes.byref(h), device, mem_budget_bytes), "create")
        self._h = h
        self._scene_refs = None
        self._scene_key = None      # (data_ptr, version) of the arrays the scene was set from
        self._scene_gen = 0         # bumped by every set_scene
        self._owned_copies = False  # the scene refs include copies this binding made
        self.n = 0
        self.sh_degree = 0
        self.storage = torch.float32
        self._views = []

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize(self.device)
            lib().conegs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scene(self, means, log_scales, quats, opacity_logits, sh, sh_degree: int, rho2=None,
                  storage: Optional[torch.dtype] = None, stream=None):
        """Scene parameters (kept by reference).  SH and opacity may be stored in
        bf16/fp16 (``storage``); everything else is FP32."""
        dev = self.device
        storage = storage if storage is not None else torch.float32
        given = dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits, sh=sh,
                     rho2=rho2)
        m = _dev(torch.as_tensor(means), dev)
        n = m.shape[0]
        refs = dict(
            means=m.reshape(n, 3),
            log_scales=_dev(torch.as_tensor(log_scales), dev).reshape(n, 3),
            quats=_dev(torch.as_tensor(quats), dev).reshape(n, 4),
            opacity_logits=_dev(torch.as_tensor(opacity_logits), dev, storage).reshape(n),
            sh=_dev(torch.as_tensor(sh), dev, storage).reshape(n, (sh_degree + 1) ** 2, 3),
            rho2=None if rho2 is None else _dev(torch.as_tensor(rho2), dev).reshape(n),
        )
        if self._owned_copies:
            # the old scene arrays include copies made here: work queued on any stream
            # may still read them, so let it finish before they can be freed
            torch.cuda.synchronize(dev)
        check(lib().conegs_set_scene(self._h, n, _ptr(refs["means"]), _ptr(refs["log_scales"]), _ptr(refs["quats"]),
                                     _ptr(refs["opacity_logits"]), _ptr(refs["sh"]), sh_degree,
                                     _DTYPE_CODE[storage], _ptr(refs["rho2"]), _stream(stream)), "set_scene")
        self._scene_refs = refs
        self._owned_copies = any(refs[k] is not None and not (isinstance(given[k], torch.Tensor) and
                                                              refs[k].data_ptr() == given[k].data_ptr())
                                 for k in refs)
        self._scene_key = None
        self._scene_gen += 1
        self.n, self.sh_degree, self.storage = n, sh_degree, storage
        return refs

    def set_scene_from(self, scene, storage: Optional[torch.dtype] = None, rho2=None):
        """Convenience: a synthetic.Scene (numpy arrays)."""
        return self.set_scene(torch.from_numpy(scene.means), torch.from_numpy(scene.log_scales),
                              torch.from_numpy(scene.quats), torch.from_numpy(scene.opacity_logits),
                              torch.from_numpy(scene.sh), scene.sh_degree,
                              torch.from_numpy(scene.rho2) if rho2 is None else rho2, storage=storage)

    def view(self) -> "View":
        v = View(self)
        self._views.append(v)
        return v

    def render_batch(self, views: Sequence["View"], flags: int = 0, outs=None, streams=None):
        """Render several views in one call (their work overlaps on the device);
        returns [(rgb, T)] per view.  outs: optional [(out_rgb, out_T)] per view."""
        n = len(views)
        dev = self.device
        if outs is None:
            outs = [(torch.empty(3, v.height, v.width, device=dev, dtype=torch.float32),
                     torch.empty(v.height, v.width, device=dev, dtype=torch.float32)) for v in views]
        P = ctypes.c_void_p
        hv = (P * n)(*[v._h for v in views])
        rgb = (P * n)(*[_ptr(o[0]) for o in outs])
        Ts = (P * n)(*[_ptr(o[1]) for o in outs])
        st = (P * n)(*[_stream(None if streams is None else streams[i]) for i in range(n)])
        for v in views:
            v._bump()
        check(lib().conegs_render_batch(n, hv, rgb, Ts, flags, st), "render_batch")
        return list(outs)

    def render_host_batch(self, views: Sequence["View"], host_outs, flags: int = 0, streams=None):
        """render_batch into (pinned) host tensors [(rgb, T or None)] per view; returns
        after every copy completed."""
        n = len(views)
        P = ctypes.c_void_p
        hv = (P * n)(*[v._h for v in views])
        rgb = (P * n)(*[_ptr(o[0]) for o in host_outs])
        Ts = (P * n)(*[_ptr(o[1]) for o in host_outs])
        st = (P * n)(*[_stream(None if streams is None else streams[i]) for i in range(n)])
        for v in views:
            v._bump()
        check(lib().conegs_render_host_batch(n, hv, rgb, Ts, flags, st), "render_host_batch")
        return list(host_outs)

    def render_host_batch_async(self, views: Sequence["View"], host_outs, flags: int = 0, streams=None):
        """render_host_batch without the wait: the image copies into the (pinned) host
        tensors [(rgb, T or None)] are enqueued on each view's copy stream; read them
        only after ``view.host_wait()``.  The copy of one call overlaps the next call's
        render of the same view."""
        n = len(views)
        P = ctypes.c_void_p
        hv = (P * n)(*[v._h for v in views])
        rgb = (P * n)(*[_ptr(o[0]) for o in host_outs])
        Ts = (P * n)(*[_ptr(o[1]) for o in host_outs])
        st = (P * n)(*[_stream(None if streams is None else streams[i]) for i in range(n)])
        for v in views:
            v._bump()
            # keeps the host tensors alive while their copies may be in flight (at most
            # the last two calls' per view: a render waits for the copy of two calls back)
            v._pending = v._pending[-1:] + [host_outs]
        check(lib().conegs_render_host_batch_async(n, hv, rgb, Ts, flags, st), "render_host_batch_async")
        return list(host_outs)

    def compute_floor(self, views: Sequence["View"], stream=None) -> torch.Tensor:
        """Eq. 11 training-frequency floor of the current scene's Gaussians over ``views``."""
        out = torch.empty(self.n, device=self.device, dtype=torch.float32)
        arr = (ctypes.c_void_p * max(len(views), 1))(*[v._h for v in views])
        check(lib().conegs_compute_floor(self._h, len(views), arr, _ptr(out), _stream(stream)), "compute_floor")
        return out


class View:
    """One camera and its render scratch (see conegs_view in include/conegs.h)."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        h = ctypes.c_void_p()
        check(lib().conegs_view_create(ctx._h, ctypes.byref(h)), "view_create")
        self._h = h
        self.width = self.height = 0
        self._token = 0       # bumped by every call that replaces the view's adjoint state
        self._pending = []    # host tensors of copies in flight (render_host_batch_async)

    def _bump(self):
        self._token += 1

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value and self.ctx._h is not None:
            lib().conegs_view_destroy(self._h)
        self._h = None

    def set_camera(self, model: int, width: int, height: int, intrinsics, distortion=None, cam_to_world=None,
                   theta_lim: float = 0.0, stream=None):
        check(lib().conegs_set_camera(self._h, int(model), int(width), int(height), _host_f32(intrinsics, 4),
                                      _host_f32(distortion, 4), _host_f32(cam_to_world, 12), float(theta_lim),
                                      _stream(stream)), "set_camera")
        self._bump()
        self.width, self.height = int(width), int(height)

    def set_camera_from(self, cam, stream=None):
        """Convenience: a synthetic.Camera."""
        self.set_camera(cam.model, cam.width, cam.height, cam.intrinsics, cam.k, cam.cam_to_world, cam.theta_lim,
                        stream)

    def render(self, flags: int = 0, out_rgb: Optional[torch.Tensor] = None, out_T: Optional[torch.Tensor] = None,
               stream=None):
        dev = self.ctx.device
        if out_rgb is None:
            out_rgb = torch.empty(3, self.height, self.width, device=dev, dtype=torch.float32)
        if out_T is None:
            out_T = torch.empty(self.height, self.width, device=dev, dtype=torch.float32)
        self._bump()
        check(lib().conegs_render(self._h, _ptr(out_rgb), _ptr(out_T), flags, _stream(stream)), "render")
        return out_rgb, out_T

    def render_count(self, flags: int = 0, stream=None):
        """Run the render's count pass ahead of it: (pairs, device bytes the rest of
        the render needs).  The next render with the same flags reuses the count."""
        pairs = ctypes.c_int64()
        nbytes = ctypes.c_size_t()
        check(lib().conegs_render_count(self._h, int(flags), ctypes.byref(pairs), ctypes.byref(nbytes),
                                        _stream(stream)), "render_count")
        return pairs.value, nbytes.value

    def render_host(self, out_rgb_host: torch.Tensor, out_T_host: Optional[torch.Tensor] = None, flags: int = 0,
                    stream=None):
        """Render into (pinned) host tensors; returns after the copy completed."""
        self._bump()
        check(lib().conegs_render_host(self._h, _ptr(out_rgb_host), _ptr(out_T_host), flags, _stream(stream)),
              "render_host")
        return out_rgb_host, out_T_host

    def host_wait(self):
        """Wait until every image copy that render_host_batch_async enqueued for this view
        has reached host memory."""
        check(lib().conegs_view_host_wait(self._h), "view_host_wait")
        self._pending.clear()

    def render_backward(self, dL_drgb: torch.Tensor, dL_dT: Optional[torch.Tensor] = None, grads=None,
                        stream=None):
        """Accumulate scene gradients (dict of FP32 tensors; created if None)."""
        refs = self.ctx._scene_refs
        dev = self.ctx.device
        if grads is None:
            grads = {k: torch.zeros(refs[k].shape, device=dev, dtype=torch.float32)
                     for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        g_rgb = _dev(dL_drgb, dev)
        g_T = None if dL_dT is None else _dev(dL_dT, dev)
        check(lib().conegs_render_backward(self._h, _ptr(g_rgb), _ptr(g_T),
                                           _ptr(grads.get("means")), _ptr(grads.get("log_scales")),
                                           _ptr(grads.get("quats")), _ptr(grads.get("opacity_logits")),
                                           _ptr(grads.get("sh")), _stream(stream)), "render_backward")
        # copies made here are read asynchronously on `stream`: keep their memory from
        # being handed out again before that work has run
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        for mine, theirs in ((g_rgb, dL_drgb), (g_T, dL_dT)):
            if mine is not None and mine is not theirs:
                mine.record_stream(s)
        return grads

    def stats(self) -> dict:
        st = _lib.Stats()
        check(lib().conegs_get_stats(self._h, ctypes.byref(st)), "get_stats")
        return {k: getattr(st, k) for k, _ in _lib.Stats._fields_}

    def rays(self, stream=None):
        P = self.width * self.height
        dev = self.ctx.device
        d = torch.empty(3, P, device=dev)
        dx = torch.empty(3, P, device=dev)
        dy = torch.empty(3, P, device=dev)
        valid = torch.empty(P, device=dev, dtype=torch.uint8)
        check(lib().conegs_get_rays(self._h, _ptr(d), _ptr(dx), _ptr(dy), _ptr(valid), _stream(stream)), "get_rays")
        return d, dx, dy, valid

    def tile_table(self, stream=None) -> torch.Tensor:
        st = self.stats()
        out = torch.empty(st["tiles_x"] * st["tiles_y"], 6, device=self.ctx.device)
        check(lib().conegs_get_tile_table(self._h, _ptr(out), _stream(stream)), "get_tile_table")
        return out

    def bin_counts(self, stream=None):
        st = self.stats()
        pg = torch.empty(self.ctx.n, device=self.ctx.device, dtype=torch.int32)
        pt = torch.empty(st["tiles_x"] * st["tiles_y"], device=self.ctx.device, dtype=torch.int32)
        check(lib().conegs_get_bin_counts(self._h, _ptr(pg), _ptr(pt), _stream(stream)), "get_bin_counts")
        return pg, pt

    def pairs(self, stream=None):
        st = self.stats()
        gid = torch.empty(max(st["n_pairs"], 1), device=self.ctx.device, dtype=torch.int32)
        rng = torch.empty(st["tiles_x"] * st["tiles_y"], 2, device=self.ctx.device, dtype=torch.int32)
        check(lib().conegs_get_pairs(self._h, _ptr(gid), _ptr(rng), _stream(stream)), "get_pairs")
        return gid[: st["n_pairs"]], rng


class _Render(torch.autograd.Function):
    """Forward: conegs_render with KEEP_FOR_BACKWARD.  Backward: conegs_render_backward,
    which recomputes the transmittance back to front (no per-pair state is stored)."""

    @staticmethod
    def forward(fctx, view, flags, means, log_scales, quats, opacity_logits, sh):
        rgb, T = view.render(flags=flags | KEEP_FOR_BACKWARD)
        fctx.view = view
        fctx.token = (view._token, view.ctx._scene_gen)
        fctx.dtypes = (means.dtype, log_scales.dtype, quats.dtype, opacity_logits.dtype, sh.dtype)
        fctx.shapes = (means.shape, log_scales.shape, quats.shape, opacity_logits.shape, sh.shape)
        return rgb, T

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(fctx, g_rgb, g_T):
        view = fctx.view
        if (view._token, view.ctx._scene_gen) != fctx.token:
            raise RuntimeError("render_fn backward: the view was rendered again, or its camera or the scene "
                               "was set, after this render; its adjoint state is gone (render each view once "
                               "per backward, or use one view per render)")
        if g_rgb is None:
            g_rgb = torch.zeros(3, view.height, view.width, device=view.ctx.device)
        grads = view.render_backward(g_rgb, g_T)
        out = []
        for k, dt, shp in zip(("means", "log_scales", "quats", "opacity_logits", "sh"), fctx.dtypes, fctx.shapes):
            out.append(grads[k].reshape(shp).to(dt))
        return (None, None, *out)


def render_fn(view: View, means: torch.Tensor, log_scales: torch.Tensor, quats: torch.Tensor,
              opacity_logits: torch.Tensor, sh: torch.Tensor, rho2: Optional[torch.Tensor] = None, flags: int = 0):
    """Differentiable render of ``view`` (rgb [3,H,W], T [H,W]).

    The five parameter tensors (device tensors: means, log_scales, quats FP32;
    opacity_logits and sh FP32, BF16 or FP16 storage) become the context's
    scene unless it was already set from exactly these tensors, unchanged since
    (same storage and version).  ``loss.backward()`` then runs the library's
    adjoint for this render and returns the gradients w.r.t. those tensors;
    rho2 (the Eq. 10 floor) is not differentiated.  Each view keeps the state
    of its last render only: render a view once per backward pass."""
    ctx = view.ctx
    key = tuple((t.data_ptr(), t._version) for t in (means, log_scales, quats, opacity_logits, sh)) + \
        ((None,) if rho2 is None else ((rho2.data_ptr(), rho2._version),))
    if ctx._scene_key != key:
        k = sh.shape[1] if sh.dim() == 3 else sh.shape[-1] // 3
        deg = int(round(k ** 0.5)) - 1
        storage = sh.dtype if sh.dtype in (torch.bfloat16, torch.float16) else None
        ctx.set_scene(means.detach(), log_scales.detach(), quats.detach(), opacity_logits.detach(), sh.detach(),
                      deg, None if rho2 is None else rho2.detach(), storage=storage)
        ctx._scene_key = key
    return _Render.apply(view, int(flags), means, log_scales, quats, opacity_logits, sh)


def radix_sort_pairs(ctx: Context, keys: torch.Tensor, values: torch.Tensor, begin_bit: int = 0, end_bit: int = 32,
                     stream=None):
    """Stable in-place LSD radix sort of uint32-valued (int32 storage) key/value tensors."""
    assert keys.dtype == torch.int32 and values.dtype == torch.int32 and keys.is_contiguous()
    check(lib().conegs_radix_sort_pairs(ctx._h, _ptr(keys), _ptr(values), keys.numel(), begin_bit, end_bit,
                                        _stream(stream)), "radix_sort_pairs")
    return keys, values


def measure_fp32_peak(device: int = 0):
    """Measured FP32 FMA throughput of the device: (TFLOP/s, ms of the timed launch)."""
    t = ctypes.c_double()
    m = ctypes.c_double()
    check(lib().conegs_measure_fp32_peak(int(device), ctypes.byref(t), ctypes.byref(m)), "measure_fp32_peak")
    return t.value, m.value

"""Serving loop with continuous batching over the C ABI.

The scene stays resident in one conegs context.  Requests (a camera each) are
queued as they arrive; each slot owns a view (ray table and render scratch), a
CUDA stream and a host thread (the C calls release the GIL), so requests that
arrive while others are on the GPU start right away and their kernels overlap
on the device.  Every request's image is copied to pinned host memory;
latency is measured from arrival to the end of that copy.

Memory admission: a slot takes the next request in arrival order, sets its
camera and runs the render's count pass (conegs_render_count), which returns
the device bytes the rest of the render needs (pair lists, sort scratch,
per-pixel state); the request then waits until that, with its image, fits the
server's budget next to the requests in flight, and renders with the count it
already has.  A large request waiting for memory holds only its own slot: the
other slots keep taking later, smaller requests past it.  A render that still
exceeds the library's own budget (CONEGS_ERR_BUDGET) is retried once memory
frees up.

Start-up: Server.warm(cameras) renders the given cameras (say the largest a
stream will see) once on every slot, so that the slots' device and pinned host
buffers grow before requests arrive instead of stalling the first ones.
"""
from __future__ import annotations

import collections
import dataclasses
import statistics
import threading
import time
from typing import List, Optional

import torch

from . import ConegsError, Context

IMAGE_BYTES_PER_PIXEL = 16 + 16           # device image (rgb + T) and its pinned host copy


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    camera: object        # anything with model, width, height, intrinsics, k, cam_to_world, theta_lim
    flags: int = 0


@dataclasses.dataclass
class Result:
    rid: int
    width: int
    height: int
    rays: int
    t_arrival: float
    t_admit: float
    t_done: float
    rgb: Optional[torch.Tensor] = None
    T: Optional[torch.Tensor] = None
    error: Optional[str] = None
    need_bytes: int = 0          # the memory the request was admitted with
    t_release: float = 0.0       # when that memory went back to the gate

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.t_done - self.t_arrival)


def image_bytes(cam) -> int:
    return cam.width * cam.height * IMAGE_BYTES_PER_PIXEL


class MemoryGate:
    """Admission by memory: acquire(need) waits until the bytes in use plus `need`
    fit the budget (a request larger than the budget runs when nothing else is in
    flight).  Callers that wait do not block callers with smaller needs that fit."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.in_use = 0
        self._cv = threading.Condition()

    def acquire(self, need: int, closed=lambda: False) -> bool:
        with self._cv:
            while self.in_use > 0 and self.in_use + need > self.budget:
                if closed():
                    return False
                self._cv.wait(0.05)
            self.in_use += need
            return True

    def release(self, need: int):
        with self._cv:
            self.in_use -= need
            self._cv.notify_all()


class Server:
    def __init__(self, ctx: Context, slots: int = 4, mem_budget_bytes: int = 32 << 30, keep_images: int = 0):
        """keep_images: how many results keep a copy of their image (True: all)."""
        self.ctx = ctx
        self.gate = MemoryGate(mem_budget_bytes)
        self.keep_images = (1 << 62) if keep_images is True else int(keep_images)
        self._kept = 0
        self._slots = [(ctx.view(), torch.cuda.Stream(device=ctx.device)) for _ in range(slots)]
        self._host = [None] * slots     # per slot: pinned host buffer for images (rgb and T)
        self._queue: collections.deque = collections.deque()
        self._cv = threading.Condition()
        self._closed = False
        self._t0 = time.perf_counter()
        self.results: List[Result] = []
        self._threads = [threading.Thread(target=self._worker, args=(k,), daemon=True) for k in range(slots)]
        for t in self._threads:
            t.start()

    @property
    def budget(self) -> int:
        return self.gate.budget

    def now(self) -> float:
        return time.perf_counter() - self._t0

    def submit(self, req: Request, t_arrival: Optional[float] = None):
        with self._cv:
            self._queue.append((req, self.now() if t_arrival is None else t_arrival))
            self._cv.notify_all()

    def _take(self):
        """The next request in arrival order (memory is checked after its count pass)."""
        with self._cv:
            while not self._closed and not self._queue:
                self._cv.wait(0.05)
            if self._closed:
                return None
            return self._queue.popleft()

    def _host_images(self, k: int, cam):
        """Views (rgb, T) into slot k's pinned host buffer, grown to the largest request
        seen and reused: allocating pinned memory per request stalls every slot."""
        P = cam.height * cam.width
        host = self._host[k]
        if host is None or host.numel() < 4 * P:
            host = torch.empty(max(4 * P, 0 if host is None else host.numel() * 3 // 2), pin_memory=True)
            self._host[k] = host
        return host[:3 * P].view(3, cam.height, cam.width), host[3 * P:4 * P].view(cam.height, cam.width)

    def warm(self, cameras, flags: int = 0):
        """Render each camera once on every slot, before requests arrive: the slots' device
        buffers and pinned host buffers grow to those sizes now, not while serving."""
        with self._cv:
            if self._queue:
                raise RuntimeError("warm() runs before requests are submitted")
        for k, (view, stream) in enumerate(self._slots):
            for cam in cameras:
                h_rgb, h_T = self._host_images(k, cam)
                with torch.cuda.stream(stream):
                    view.set_camera_from(cam, stream=stream)
                    view.render_host(h_rgb, h_T, flags=flags, stream=stream)

    def _worker(self, k: int):
        view, stream = self._slots[k]
        torch.cuda.set_device(self.ctx.device)
        while True:
            item = self._take()
            if item is None:
                return
            req, ta = item
            cam = req.camera
            res = Result(req.rid, cam.width, cam.height, 0, ta, 0.0, 0.0)
            need = 0
            try:
                h_rgb, h_T = self._host_images(k, cam)
                with torch.cuda.stream(stream):
                    view.set_camera_from(cam, stream=stream)
                    _, nbytes = view.render_count(flags=req.flags, stream=stream)
                    need = nbytes + image_bytes(cam)
                    if not self.gate.acquire(need, closed=lambda: self._closed):
                        return
                    res.t_admit, res.need_bytes = self.now(), need
                    try:
                        view.render_host(h_rgb, h_T, flags=req.flags, stream=stream)
                    finally:
                        res.t_release = self.now()
                        self.gate.release(need)
                res.rays = int(view.stats()["n_valid_pixels"])
                with self._cv:
                    keep = self._kept < self.keep_images
                    self._kept += 1 if keep else 0
                if keep:
                    res.rgb, res.T = h_rgb.clone(), h_T.clone()
            except ConegsError as e:
                if e.status == 7:                       # library budget: retry when memory frees up
                    with self._cv:
                        self._queue.appendleft((req, ta))
                        self._cv.notify_all()
                    time.sleep(0.01)
                    continue
                res.error = str(e)
                res.t_admit = res.t_admit or self.now()
            res.t_done = self.now()
            with self._cv:
                self.results.append(res)
                self._cv.notify_all()

    def drain(self, n_expected: int, timeout_s: float = 600.0):
        t_end = time.perf_counter() + timeout_s
        with self._cv:
            while len(self.results) < n_expected and time.perf_counter() < t_end:
                self._cv.wait(0.05)
        return sorted(self.results, key=lambda r: r.rid)

    def close(self):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for t in self._threads:
            t.join(timeout=30)
        for view, _ in self._slots:
            view.close()

    def play(self, requests: List[Request], realtime: bool = True) -> List[Result]:
        """Submit requests at their arrival times (seconds from now) and wait for all."""
        start = self.now()
        for r in requests:
            if realtime:
                delay = start + r.arrival_s - self.now()
                if delay > 0:
                    time.sleep(delay)
            self.submit(r, start + r.arrival_s if realtime else None)
        return self.drain(len(requests))


def summarize(results: List[Result]) -> dict:
    ok = [r for r in results if r.error is None]
    lat = sorted(r.latency_ms for r in ok)
    if not lat:
        return {"requests": len(results), "errors": len(results)}
    span = max(r.t_done for r in ok) - min(r.t_arrival for r in ok)

    def pct(p):
        return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]

    return {"requests": len(results), "errors": len(results) - len(ok), "p50_ms": pct(50), "p99_ms": pct(99),
            "mean_ms": statistics.mean(lat), "rays": sum(r.rays for r in ok),
            "mrays_per_s": sum(r.rays for r in ok) / span / 1e6 if span > 0 else None, "span_s": span}

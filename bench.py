"""Benchmark: anti-aliased Mrays/s of the ConeGaussian render on one B300.

Headline workload (`value`): pinhole 1280x720 (f = 1200) and the same camera at
1/8 resolution (160x90), 500k Gaussians drawn from the clustered blob +
background-shell distribution, SH degree 3, per-Gaussian Eq. 11 floor from the
1280x720 view.  One step renders both cameras (936,000 rays).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is forward Mrays/s with inputs resident in HBM
(L2 flushed between timed steps); `fwd_bwd` the same workload with the adjoint;
`e2e` the forward through the host-buffer entry point (camera parameters in,
images copied back every step).  The other workloads ride along on one GPU:
  c3  Kannala-Brandt fisheye 190 deg 1024x1024, 1M Gaussians: forward, and
      forward + adjoint of an L1 loss against the render of the perturbed scene;
  c4  the 8-camera rig (4 pinhole, 4 fisheye at 1, 1/2, 1/4, 1/8 of 1080p), 3M
      Gaussians, SH and opacity stored in BF16: forward and forward + adjoint;
  c5  serving: 5M Gaussians resident, SH3 in FP16, a Poisson request stream at
      200 req/s: p50 / p99 latency and Mrays/s;
  c1  pinhole 64x48, 1000 Gaussians (launch bound).
Each form states its RGB error: against the FP32-storage render on the GPU
(half-storage forms), and against the FP64 oracle on a pixel sample (in the
CPU-baseline leg, which runs the oracle on the host after the timed regions).
The reference arm times the FP64 oracle on the host cores on a bounded pixel
sample of the headline workload.  Under torchrun every rank renders its own
replica of the headline workload (no collective); the value sums all ranks'
rays over the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

METRIC = "anti-aliased Mrays/s fwd & fwd+bwd at stated RGB err vs FP32 plain; p50/p99 ms"
WORKLOAD = "pinhole 1280x720 + 160x90 (1/8), 500k Gaussians (64 blobs + shell), SH3, Eq.11 floor"
# FP32 flops of one full pair evaluation past the pre-test (an FMA counts as 2, a
# reciprocal, square root or exp as 1), counted from the code of the response with a
# floor (rho^2 > 0): d_u, n, t*, q 33; the differentials g_x, g_y, c_x, c_y and the
# half-edge vectors e_x, e_y 60; the world Gram terms and H' 18; the eigenvalues
# of H' and K (Eq. 12) 22; the orthonormal basis of the footprint and q's parts 58;
# N, det A, the quadratic form, T (Eq. 9) 37; compositing (Eq. 4) 9.
FLOPS_PER_EVAL = 237
# DRAM bytes (read + write) of one 1280x720 first-segment raster launch of this
# workload, from ncu (dram__bytes_read.sum + dram__bytes_write.sum: 76.42 + 7.51 MB)
# on this kernel's current code; to be taken again whenever the kernel changes.
RASTER_MAIN_TRAFFIC_BYTES = 83.93e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the benchmark runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.rows.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if "Active" in r[3 + k]
                          and "Not" not in r[3 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def reduce_step_time(ms: float, device) -> float:
    """The slowest rank's step time: every rank waits for it, so the whole job's
    rate is all ranks' rays over this (MAX over the process group; the local time
    when not distributed)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def _timed(fn, steps, stream, flush=None):
    """Mean ms per call over `steps` calls, CUDA events on `stream`; with `flush`
    (a large buffer) L2 is flushed between calls, outside the timed spans."""
    import torch
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


class Batch:
    """Several views of one context rendered in one batch call, each on its own stream."""

    def __init__(self, ctx, cams, priorities=None):
        import torch
        dev = ctx.device
        self.ctx = ctx
        self.views = []
        for c in cams:
            v = ctx.view()
            v.set_camera_from(c)
            self.views.append(v)
        self.outs = [(torch.empty(3, c.height, c.width, device=dev), torch.empty(c.height, c.width, device=dev))
                     for c in cams]
        pr = priorities or [0] * len(cams)
        self.streams = [torch.cuda.Stream(device=dev, priority=p) for p in pr]
        self.main = torch.cuda.current_stream()

    def step(self, flags=0, grads=None, dl=None):
        import torch
        ev0 = torch.cuda.Event()
        ev0.record(self.main)
        for st in self.streams:
            st.wait_event(ev0)
        self.ctx.render_batch(self.views, flags=flags, outs=self.outs, streams=self.streams)
        if dl is not None:
            for k, (v, st) in enumerate(zip(self.views, self.streams)):
                with torch.cuda.stream(st):        # dL/drgb may read the view's image: after its render
                    v.render_backward(dl(k), grads=None if grads is None else grads[k], stream=st)
        for st in self.streams:
            self.main.wait_stream(st)

    def rays(self):
        return sum(v.stats()["n_valid_pixels"] for v in self.views)

    def close(self):
        for v in self.views:
            v.close()


def _grads_like(ctx):
    import torch
    refs = ctx._scene_refs
    return {k: torch.zeros(refs[k].shape, device=ctx.device, dtype=torch.float32)
            for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}


# ---------------------------------------------------------------- workloads (GPU, timed)

def bench_c2(args, world, local_rank, peak_tflops):
    import torch
    import paper_2609_13397_b300 as cg
    dev = torch.device("cuda", local_rank)
    cams, sc = S.c2_cameras(), S.c2_scene()
    ctx = cg.Context(local_rank)
    ctx.set_scene_from(sc)
    b = Batch(ctx, cams, priorities=[0, -1])   # the 160x90 view's chain of small launches gets priority
    rho2 = ctx.compute_floor([b.views[0]])
    ctx.set_scene_from(sc, rho2=rho2)
    rays = b.rays()
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)
    for _ in range(max(args.warmup, 3)):
        b.step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    ms = reduce_step_time(_timed(lambda: b.step(), args.steps, b.main, flush), dev)
    launches = sum(v.stats()["n_launches"] for v in b.views) * args.steps
    # stage times and counters: the same steps again with CUDA events and counters on
    # (conegs PROFILE), after the timed ones; the last step's per-view statistics
    prof = []
    for k in range(min(args.steps, 10)):
        flush.fill_(float(k))
        b.step(cg.PROFILE)
        prof.append([v.stats() for v in b.views])
    views = [dict(p) for p in prof[-1]]
    for i in range(len(views)):
        views[i]["ms_raster_main"] = statistics.median(p[i]["ms_raster_main"] for p in prof)
    out = {"rays": rays, "ms": ms, "value": rays * world / (ms * 1e-3) / 1e6, "launches": launches}
    images = [o[0].cpu().numpy() for o in b.outs]
    # forward + adjoint
    gl = [torch.ones_like(o[0]) for o in b.outs]
    grads = [_grads_like(ctx) for _ in b.views]
    fb = lambda: b.step(cg.KEEP_FOR_BACKWARD, grads=grads, dl=lambda k: gl[k])
    for _ in range(2):
        fb()
    fb_ms = reduce_step_time(_timed(fb, args.steps, b.main), dev)
    out["fwd_bwd"] = {"value": rays * world / (fb_ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": fb_ms}
    # the same forward with unscented-transform binning (approximate: fewer pairs)
    for _ in range(2):
        b.step(cg.BIN_UT)
    ut_ms = reduce_step_time(_timed(lambda: b.step(cg.BIN_UT), args.steps, b.main, flush), dev)
    ut_imgs = [o[0].clone() for o in b.outs]
    ut_pairs = [v.stats()["n_pairs"] for v in b.views]
    b.step()
    torch.cuda.synchronize()
    loss = []
    for (o, _), u in zip(b.outs, ut_imgs):
        d = (o - u).abs()
        loss.append({"mean_abs_rgb": float(d.mean()), "frac_px_over_1_255": float((d.amax(0) > 1 / 255).float().mean())})
    out["bin_ut"] = {"value": rays * world / (ut_ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": ut_ms,
                     "n_pairs": ut_pairs, "n_pairs_rule": [v["n_pairs"] for v in views], "vs_exact": loss}
    # end to end through the host-buffer entry points: every step sets both cameras from
    # host parameters and reads both images (rgb and T) back into pinned host memory.
    # Pipelined (render_host_batch_async): a step's copies overlap the next step's
    # render; every copy has landed when the clock stops.  Blocking (render_host_batch):
    # each step waits for its own copies.
    host = [[(torch.empty(3, c.height, c.width, pin_memory=True), torch.empty(c.height, c.width, pin_memory=True))
             for c in cams] for _ in range(2)]

    def set_cams():
        for v, c, st in zip(b.views, cams, b.streams):
            v.set_camera_from(c, stream=st)

    def e2e_run(steps, pipelined):
        for k in range(steps):
            set_cams()
            if pipelined:
                ctx.render_host_batch_async(b.views, host[k % 2], streams=b.streams)
            else:
                ctx.render_host_batch(b.views, host[k % 2], streams=b.streams)
        for v in b.views:
            v.host_wait()
    e2e = {}
    for pipelined in (True, False):
        e2e_run(2, pipelined)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_run(args.steps, pipelined)
        torch.cuda.synchronize()
        e2e[pipelined] = reduce_step_time((time.perf_counter() - t0) * 1e3 / args.steps, dev)
    out["e2e"] = {"value": rays * world / (e2e[True] * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": e2e[True],
                  "h2d_bytes_per_step": len(cams) * (4 + 4 + 12) * 4,
                  "d2h_bytes_per_step": sum(4 * 4 * c.width * c.height for c in cams),
                  "api": "render_host_batch_async (copies overlap the next step's render)",
                  "blocking": {"value": rays * world / (e2e[False] * 1e-3) / 1e6, "unit": "Mrays/s",
                               "ms_per_step": e2e[False], "api": "render_host_batch"}}
    # roofline of the dominant kernel: the 1280x720 view's first-segment raster launch
    # (its tile lists are all shorter than the segment length, so the launch does the
    # view's whole raster work), timed by CUDA events on its stream inside the step
    v0 = views[0]
    achieved = FLOPS_PER_EVAL * v0["n_evaluated"] / (v0["ms_raster_main"] * 1e-3) / 1e12
    out["roofline"] = {
        "bound": "alu", "kernel": "raster_seg_kernel<FILTER=1, FIRST=1, PIX=1> (1280x720 view)", "achieved": achieved,
        "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
        "traffic": RASTER_MAIN_TRAFFIC_BYTES, "traffic_unit": "bytes per launch (ncu)",
        "peak_basis": "measured FP32 FMA throughput of this device (conegs_measure_fp32_peak; FMA = 2 flops)",
        "flops_per_eval": FLOPS_PER_EVAL, "evals_per_launch": v0["n_evaluated"],
        "entries_walked_per_launch": v0["n_walked"], "ms_per_launch": v0["ms_raster_main"],
        "flat_fp64_evals_per_launch": v0["n_evaluated_flat"]}
    out["views"] = [{"camera": f"{c.width}x{c.height}",
                     **{k: v[k] for k in ("n_pairs", "n_visible", "n_flat", "n_walked", "n_evaluated",
                                          "n_evaluated_flat", "ms_preprocess", "ms_sort", "ms_raster",
                                          "ms_raster_main", "ms_total")}} for c, v in zip(cams, views)]
    out["_error_work"] = {"cams": cams, "scene": sc.with_rho2(rho2.cpu().numpy()), "images": images}
    b.close()
    ctx.close()
    return out


def bench_c3(args):
    import torch
    import paper_2609_13397_b300 as cg
    cam, sc = S.c3_camera(), S.c3_scene()
    ctx = cg.Context(0)
    ctx.set_scene_from(S.perturbed(sc, seed=1))
    b = Batch(ctx, [cam])
    b.step()
    torch.cuda.synchronize()
    target = b.outs[0][0].clone()
    ctx.set_scene_from(sc)
    valid = b.views[0].rays()[3].reshape(cam.height, cam.width).bool()
    nval = int(valid.sum())
    g = _grads_like(ctx)

    def dl(k):   # d/d rgb of the mean L1 loss over valid pixels and channels
        return torch.sign(b.outs[0][0] - target) * valid / (3.0 * nval)
    for _ in range(max(args.warmup, 2)):
        b.step(cg.KEEP_FOR_BACKWARD, grads=[g], dl=dl)
    ms_f = _timed(lambda: b.step(), args.steps, b.main)
    ms_fb = _timed(lambda: b.step(cg.KEEP_FOR_BACKWARD, grads=[g], dl=dl), args.steps, b.main)
    b.step(cg.PROFILE)
    torch.cuda.synchronize()
    st = b.views[0].stats()
    img = b.outs[0][0].cpu().numpy()
    b.close()
    ctx.close()
    return {"workload": "KB fisheye 190 deg 1024x1024, k~U(-0.05,0.05), 1M Gaussians (C1 distribution)",
            "value": nval / ms_f / 1e3, "unit": "Mrays/s", "ms_per_step": ms_f,
            "fwd_bwd": {"value": nval / ms_fb / 1e3, "unit": "Mrays/s", "ms_per_step": ms_fb,
                        "loss": "L1 vs the render of the seed-1 perturbed scene"},
            "rays_per_step": nval, "n_pairs": st["n_pairs"], "n_flat": st["n_flat"],
            "_error_work": {"cams": [cam], "scene": sc, "images": [img]}}


def bench_c4(args):
    import torch
    import paper_2609_13397_b300 as cg
    rig = S.c4_rig()
    sc = S.blob_scene(3_000_000, seed=0, cam=rig[0])
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, storage=torch.bfloat16)
    b = Batch(ctx, rig)
    rho2 = ctx.compute_floor(b.views)
    sc = sc.with_rho2(rho2.cpu().numpy())
    ctx.set_scene_from(sc, storage=torch.bfloat16)
    rays = b.rays()
    grads = [_grads_like(ctx) for _ in b.views]
    dls = [torch.full_like(o[0], 1e-3) for o in b.outs]
    for _ in range(max(args.warmup, 2)):
        b.step(cg.KEEP_FOR_BACKWARD, grads=grads, dl=lambda k: dls[k])
    ms_f = _timed(lambda: b.step(), args.steps, b.main)
    ms_fb = _timed(lambda: b.step(cg.KEEP_FOR_BACKWARD, grads=grads, dl=lambda k: dls[k]), args.steps, b.main)
    b.step(cg.PROFILE)
    torch.cuda.synchronize()
    prof = [{"camera": f"{'pinhole' if c.model == 0 else 'kb'} {c.width}x{c.height}",
             **{k: v.stats()[k] for k in ("n_pairs", "n_flat", "n_walked", "n_evaluated", "ms_preprocess",
                                          "ms_sort", "ms_raster", "ms_total")}} for c, v in zip(rig, b.views)]
    half = [o[0].clone() for o in b.outs]
    # the precision form against the plain FP32 path: the same render with FP32 storage
    ctx.set_scene_from(sc)
    b.step()
    torch.cuda.synchronize()
    d32 = max(float((o[0] - h).abs().max()) for o, h in zip(b.outs, half))
    images = [h.cpu().numpy() for h in half]
    b.close()
    ctx.close()
    q = S.quantized(sc, "bf16")
    return {"workload": "8 cameras (4 pinhole, 4 KB) at 1,1/2,1/4,1/8 of 1920x1080, 3M Gaussians, Eq.11 floor "
                        "over the rig, SH and opacity stored in BF16",
            "value": rays / ms_f / 1e3, "unit": "Mrays/s", "ms_per_step": ms_f,
            "fwd_bwd": {"value": rays / ms_fb / 1e3, "unit": "Mrays/s", "ms_per_step": ms_fb},
            "rays_per_step": rays, "dtype_storage": "bf16", "max_abs_rgb_vs_fp32_storage": d32, "views": prof,
            "_error_work": {"cams": rig, "scene": q, "scene_fp32": sc, "images": images}}


def bench_c5(args):
    import torch
    import paper_2609_13397_b300 as cg
    from paper_2609_13397_b300 import serving
    rig = S.c4_rig()
    sc = S.blob_scene(args.c5_gaussians, seed=0, cam=rig[0])
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, storage=torch.float16)
    vs = []
    for c in rig:
        v = ctx.view()
        v.set_camera_from(c)
        vs.append(v)
    rho2 = ctx.compute_floor(vs)
    for v in vs:
        v.close()
    sc = sc.with_rho2(rho2.cpu().numpy())
    ctx.set_scene_from(sc, storage=torch.float16)
    reqs = [serving.Request(r.rid, r.arrival_s, r.camera)
            for r in S.c5_requests(args.c5_requests, rate_hz=args.c5_rate, seed=0)]
    srv = serving.Server(ctx, slots=args.c5_slots, mem_budget_bytes=64 << 30)
    # the server's start-up: every slot renders the stream's largest pinhole and fisheye
    # request once (its buffers grow now), then a few requests of the stream
    srv.warm([max((r.camera for r in reqs if r.camera.model == m), key=lambda c: c.width * c.height)
              for m in (S.PINHOLE, S.KB_FISHEYE) if any(r.camera.model == m for r in reqs)])
    warm = [serving.Request(10_000 + r.rid, 0.0, r.camera) for r in reqs[:2 * args.c5_slots]]
    for r in warm:
        srv.submit(r)
    srv.drain(len(warm))
    srv.results.clear()
    srv.keep_images = 4           # the first served requests keep their images (error check)
    res = srv.play(reqs, realtime=True)
    st = serving.summarize(res)
    srv.close()
    # error of FP16 storage: a few requests again with FP32 storage (outside the served stream)
    picks = [r for r in res if r.error is None and r.rgb is not None][:4]
    ctx.set_scene_from(sc)
    v = ctx.view()
    d32 = 0.0
    for r in picks:
        cam = next(q.camera for q in reqs if q.rid == r.rid)
        v.set_camera_from(cam)
        rgb, _ = v.render()
        d32 = max(d32, float((rgb.cpu() - r.rgb).abs().max()))
    v.close()
    ctx.close()
    cams = [next(q.camera for q in reqs if q.rid == r.rid) for r in picks]
    return {"workload": f"serving: {args.c5_gaussians} Gaussians resident, SH3 FP16, Poisson {args.c5_rate} req/s, "
                        f"W=round(160*24^u) H=round(120*18^u), zoom 8^U(-1,1), pinhole/KB 50/50, "
                        f"{args.c5_slots} slots, {args.c5_requests} requests",
            "value": st.get("mrays_per_s"), "unit": "Mrays/s", "p50_ms": st.get("p50_ms"),
            "p99_ms": st.get("p99_ms"), "mean_ms": st.get("mean_ms"), "requests": st["requests"],
            "errors": st["errors"], "dtype_storage": "f16", "max_abs_rgb_vs_fp32_storage": d32,
            "_error_work": {"cams": cams, "scene": S.quantized(sc, "f16"), "scene_fp32": sc,
                            "images": [r.rgb.numpy() for r in picks]}}


def bench_c1(args):
    import torch
    import paper_2609_13397_b300 as cg
    cam, sc = S.c1()
    ctx = cg.Context(0)
    ctx.set_scene_from(sc)
    b = Batch(ctx, [cam])
    for _ in range(max(args.warmup, 3)):
        b.step()
    ms = _timed(lambda: b.step(), args.steps, b.main)
    rays = b.rays()
    img = b.outs[0][0].cpu().numpy()
    b.close()
    ctx.close()
    return {"workload": "pinhole 64x48 f=60, 1000 Gaussians, FP32", "value": rays / ms / 1e3, "unit": "Mrays/s",
            "ms_per_step": ms, "_error_work": {"cams": [cam], "scene": sc, "images": [img]}}


# ---------------------------------------------------------------- the oracle on the host (CPU leg)

def _oracle_rate(sc, cam, budget_s, seed):
    """Pixels per second of the oracle on random pixels of cam, the sample grown until
    one call takes about budget_s / 4."""
    import oracle
    rng = np.random.default_rng(seed)
    cap = min(65536, cam.n_pixels)
    npx = min(16, cap)
    while True:
        pix = rng.choice(cam.n_pixels, size=npx, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        oracle.render(cam, sc, pix=pix)
        t = time.perf_counter() - t0
        if t > budget_s / 4 or npx >= cap:
            break
        npx = int(min(cap, npx * max(2.0, min(8.0, budget_s / 4 / max(t, 1e-3)))))
    return npx / t, npx


def cpu_baseline(sc, cam, budget_s=10.0, single_thread=True):
    """The FP64 oracle as it stands, on the host cores, on a bounded pixel sample; and
    (single_thread) the same on one core."""
    import oracle
    cores = oracle.num_threads()
    rate, npx = _oracle_rate(sc, cam, budget_s, seed=1)
    out = {"value": rate / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
           "sample": f"{npx} random pixels of the 1280x720 view (same 500k-Gaussian scene, culled FP64 oracle)"}
    if single_thread:
        oracle.set_threads(1)
        try:
            rate1, npx1 = _oracle_rate(sc, cam, budget_s / 2, seed=3)
        finally:
            oracle.set_threads(cores)
        out["single_thread"] = {"value": rate1 / 1e6, "unit": "Mrays/s", "cores": 1, "sample": f"{npx1} pixels"}
    return out


def oracle_error(work, px_per_view, seed=5):
    """max |RGB - oracle| over a pixel sample of each image (pixels the oracle flags as
    within rounding of a compositing threshold excluded, and counted)."""
    import oracle
    rng = np.random.default_rng(seed)
    out = {}
    for key in ("scene", "scene_fp32"):
        if key not in work:
            continue
        err, flagged, n = 0.0, 0, 0
        for cam, img in zip(work["cams"], work["images"]):
            valid = oracle.rays(cam)[3]
            cand = np.nonzero(valid)[0]
            pix = rng.choice(cand, size=min(px_per_view, cand.size), replace=False).astype(np.int32)
            r = oracle.render(cam, work[key], pix=pix, eps=2e-4)
            ok = r.flags == 0
            got = img.reshape(3, -1).T[pix]
            err = max(err, float(np.abs(got - r.rgb)[ok].max(initial=0.0)))
            flagged += int((~ok).sum())
            n += pix.size
        out["max_abs_rgb" if key == "scene" else "max_abs_rgb_vs_fp32_values"] = err
        out["pixels"] = n
        out["flagged_pixels"] = flagged
    return out


# ---------------------------------------------------------------- arms

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    cams, sc = S.c2_cameras(), S.c2_scene()
    rho2 = oracle.floor_rho2([cams[0]], sc.means).astype(np.float32)
    scr = sc.with_rho2(rho2)
    cal = cpu_baseline(scr, cams[0], budget_s=4.0, single_thread=False)
    per_step_px = max(64, int(cal["value"] * 1e6 * 3.0))   # about 3 s of CPU work per step
    rng = np.random.default_rng(2)
    times = []
    for k in range(args.warmup + args.steps):
        pix = rng.choice(cams[0].n_pixels, size=per_step_px, replace=False).astype(np.int32)
        t0 = time.perf_counter()
        oracle.render(cams[0], scr, pix=pix)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = per_step_px * len(times) / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: pixel sample per step)", "pixels_per_step": per_step_px},
            "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{per_step_px} random pixels of the 1280x720 view per step"},
            "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2609_13397_b300 as cg
    torch.cuda.set_device(local_rank)
    peak, _ = cg.measure_fp32_peak(local_rank)
    others = {}
    with ClockSampler(local_rank) as clk:
        c2 = bench_c2(args, world, local_rank, peak)
        if world == 1 and not args.headline_only:
            extra = [w.strip() for w in args.extra.split(",") if w.strip()]
            for name, fn in (("c3", bench_c3), ("c4", bench_c4), ("c5", bench_c5), ("c1", bench_c1)):
                if name in extra:
                    others[name] = fn(args)
    line = {
        "metric": METRIC, "value": c2["value"], "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": c2["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_step": c2["rays"], "gaussians": 500_000,
                   "l2": "flushed between timed forward steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "sms": torch.cuda.get_device_properties(local_rank).multi_processor_count},
        "fwd_bwd": c2["fwd_bwd"], "e2e": c2["e2e"], "bin_ut": c2["bin_ut"], "views": c2["views"],
        "roofline": c2["roofline"], "gpu_launches": c2["launches"], "clocks": clk.summary(),
        "peak_fp32_tflops_measured": peak,
    }
    for name, blk in others.items():
        line[name] = {k: v for k, v in blk.items() if not k.startswith("_")}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on the host, after every timed region: its rate on the headline
        # workload, and each form's RGB error against it on a pixel sample
        line["cpu_baseline"] = cpu_baseline(c2["_error_work"]["scene"], c2["_error_work"]["cams"][0],
                                            budget_s=args.cpu_budget)
        errs = {"c2": oracle_error(c2["_error_work"], 240)}
        budget = {"c3": 160, "c4": 32, "c5": 40, "c1": 3072}
        for name, blk in others.items():
            errs[name] = oracle_error(blk["_error_work"], budget[name])
        line["rgb_error_vs_fp64_oracle"] = errs
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true", help="time the headline workload only")
    ap.add_argument("--extra", default="c3,c4,c5,c1", help="the other workloads timed after the headline one")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--c5-requests", type=int, default=300)
    ap.add_argument("--c5-rate", type=float, default=200.0)
    ap.add_argument("--c5-slots", type=int, default=6)
    ap.add_argument("--c5-gaussians", type=int, default=5_000_000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Serving with continuous batching: every request's image is the same alone and
in the mix (bitwise: the computation of a request does not depend on what else
is in flight), admission respects the memory budget, and a malformed request
fails alone without stopping the others."""
import dataclasses

import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests(n, seed=0):
    base = list(S.c5_requests(n, rate_hz=400.0, seed=seed))
    out = []
    for r in base:                                     # keep the test small: cap the resolution
        c = r.camera
        scale = min(1.0, 320.0 / max(c.width, c.height))
        cam = c.scaled(scale) if scale < 1.0 else c
        out.append(dataclasses.replace(r, camera=cam))
    return out


@pytest.fixture(scope="module")
def scene_ctx():
    import paper_2609_13397_b300 as cg
    sc = S.blob_scene(60000, seed=3, cam=S.c4_rig()[0])
    ctx = cg.Context(0)
    ctx.set_scene_from(sc, storage=torch.float16)
    return ctx


def test_alone_equals_mixed(scene_ctx):
    from paper_2609_13397_b300 import serving
    from paper_2609_13397_b300.serving import Request
    reqs = [Request(r.rid, r.arrival_s, r.camera) for r in _requests(24)]
    alone = serving.Server(scene_ctx, slots=1, keep_images=True)
    ra = []
    for r in reqs:                       # one at a time
        alone.submit(r)
        ra = alone.drain(len(ra) + 1)
    alone.close()
    mixed = serving.Server(scene_ctx, slots=6, keep_images=True)
    for r in reqs:                       # all at once: they overlap on the device
        mixed.submit(r)
    rm = mixed.drain(len(reqs))
    mixed.close()
    assert len(ra) == len(rm) == len(reqs)
    overlap = sum(1 for a in rm for b in rm if a.rid < b.rid and a.t_admit < b.t_done and b.t_admit < a.t_done)
    assert overlap > 0                   # requests really were in flight together
    for a, b in zip(ra, rm):
        assert a.error is None and b.error is None
        assert torch.equal(a.rgb, b.rgb) and torch.equal(a.T, b.T)
    stats = serving.summarize(rm)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0 and stats["rays"] > 0


def test_memory_admission_limits_concurrency(scene_ctx):
    """Each request is admitted with the memory its count pass reports: requests in
    flight together never exceed the budget, and that memory is what the render uses."""
    from paper_2609_13397_b300 import serving
    from paper_2609_13397_b300.serving import Request, image_bytes
    reqs = [Request(r.rid, 0.0, r.camera) for r in _requests(12, seed=1)]
    v = scene_ctx.view()
    needs = []
    for r in reqs:                       # what each request will ask for
        v.set_camera_from(r.camera)
        needs.append(v.render_count()[1] + image_bytes(r.camera))
        rgb, _ = v.render()              # the render reuses the count
    v.close()
    budget = int(max(needs) * 1.5)
    srv = serving.Server(scene_ctx, slots=6, mem_budget_bytes=budget)
    for r in reqs:
        srv.submit(r)
    res = srv.drain(len(reqs))
    srv.close()
    assert all(r.error is None for r in res)
    assert [r.need_bytes for r in res] == needs
    # memory is held from admission to release (the end of the copy, before t_done)
    for a in res:
        for b in res:
            if a.rid < b.rid and a.t_admit < b.t_release and b.t_admit < a.t_release:
                assert a.need_bytes + b.need_bytes <= budget


def test_count_then_render_equals_render(scene_ctx):
    """A render that reuses a count pass run ahead of it gives the same image."""
    r = _requests(1, seed=4)[0]
    v = scene_ctx.view()
    v.set_camera_from(r.camera)
    a, ta = (t.clone() for t in v.render())
    pairs, nbytes = v.render_count()
    assert pairs == v.stats()["n_pairs"] and nbytes > 0
    b, tb = v.render()
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(ta, tb)
    v.close()


def test_malformed_request_fails_alone(scene_ctx):
    from paper_2609_13397_b300 import serving
    from paper_2609_13397_b300.serving import Request
    reqs = [Request(r.rid, 0.0, r.camera) for r in _requests(6, seed=2)]
    bad = dataclasses.replace(reqs[2].camera, fx=-1.0)
    reqs[2] = Request(2, 0.0, bad)
    srv = serving.Server(scene_ctx, slots=3)
    for r in reqs:
        srv.submit(r)
    res = srv.drain(len(reqs))
    srv.close()
    assert res[2].error is not None and "ERR_ARG" in res[2].error
    assert all(r.error is None for k, r in enumerate(res) if k != 2)


def test_warm_slots_then_serve(scene_ctx):
    """Warming every slot with the largest cameras first changes no result: the
    requests served after it are bitwise those of a server that was not warmed."""
    from paper_2609_13397_b300 import serving
    from paper_2609_13397_b300.serving import Request
    reqs = [Request(r.rid, 0.0, r.camera) for r in _requests(10, seed=7)]
    big = [max((r.camera for r in reqs if r.camera.model == m), key=lambda c: c.width * c.height)
           for m in (S.PINHOLE, S.KB_FISHEYE) if any(r.camera.model == m for r in reqs)]
    out = []
    for warm in (False, True):
        srv = serving.Server(scene_ctx, slots=3, keep_images=True)
        if warm:
            srv.warm(big)
        for r in reqs:
            srv.submit(r)
        out.append(srv.drain(len(reqs)))
        srv.close()
    for a, b in zip(*out):
        assert a.error is None and b.error is None
        assert torch.equal(a.rgb, b.rgb) and torch.equal(a.T, b.T)

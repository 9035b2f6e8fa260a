"""Continuous-batching server (gs3_server_*): every result equals the same
frame rendered alone with gs3_render, bit for bit (each request has its own
workspace and the frame is deterministic), while requests overlap on the GPU
and queued requests are rendered together in batches (single launches of the
shadow and camera composites over a batch's frames); admission respects the
HBM budget; capacity overflows are retried; injected allocation failures fail
only their own requests; the shadow composite's chained waits are bounded."""
import numpy as np
import pytest

from paper_2410_11419_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scenes(gs3):
    from paper_2410_11419_gb300 import _native as N, render as R
    s0 = synth.object_scene(11, n=30_000)
    s1 = synth.tiny_scene(0)
    s2 = synth.paper_mlp_scene(3, n=4000)
    ds = [R.DeviceScene(s0, mlp_dtype=N.GS3_MLP_BF16), R.DeviceScene(s1),
          R.DeviceScene(s2, mlp_dtype=N.GS3_MLP_BF16)]
    yield ds
    for d in ds:
        d.close()


def alone(ds, cam, light):
    import torch
    from paper_2410_11419_gb300 import render as R
    rd = R.Renderer(ds, cam.width, cam.height, 1 << 23)
    img = rd.render(cam, light).clone()
    torch.cuda.synchronize()
    rd.check()
    return img


MIX = [(0, 256, 1), (1, 128, 2), (2, 160, 3), (0, 320, 4), (1, 96, 5), (0, 256, 6),
       (2, 200, 7), (0, 256, 1), (1, 128, 8), (0, 192, 9), (2, 144, 10), (0, 256, 12)]


def test_mixed_requests_equal_alone(scenes):
    import torch
    from paper_2410_11419_gb300 import render as R
    srv = R.Server(hbm_budget=8 << 30, max_inflight=4)
    ids = [srv.add_scene(d) for d in scenes]
    outs = [torch.full((res, res, 3), -1.0, device="cuda") for _, res, _ in MIX]
    torch.cuda.synchronize()  # the server's streams do not wait for torch's fills
    tickets = []
    for (si, res, seed), out in zip(MIX, outs):
        cam, light = synth.camera_light_pair(seed, res, res)
        tickets.append(srv.submit(ids[si], cam, light, out))
    lat = []
    for t in tickets:
        st, ms = srv.wait(t)
        assert st == 0
        lat.append(ms)
    stats = srv.stats()
    assert stats.completed == len(MIX) and stats.failed == 0
    assert stats.max_in_flight >= 2          # work overlapped on the device
    assert stats.device_span_ms > 0 and all(x > 0 for x in lat)
    for (si, res, seed), out in zip(MIX, outs):
        cam, light = synth.camera_light_pair(seed, res, res)
        want = alone(scenes[si], cam, light)
        assert torch.equal(out, want), (si, res, seed)
    srv.close()


def test_light_cache_reuses_shadow_values(scenes):
    """With a light cache, requests sharing (scene, light, size, options) with
    a completed frame copy its shadow values and run only the camera-side
    stages; every image still equals its frame rendered alone."""
    import torch
    from paper_2410_11419_gb300 import render as R
    srv = R.Server(hbm_budget=8 << 30, max_inflight=2, light_cache=4)
    sid = srv.add_scene(scenes[0])
    light = synth.camera_light_pair(21, 256, 256)[1]
    light2 = synth.camera_light_pair(22, 256, 256)[1]
    cams = [synth.camera_light_pair(s, 256, 256)[0] for s in range(30, 36)]
    first = torch.empty((256, 256, 3), device="cuda")
    torch.cuda.synchronize()
    assert srv.wait(srv.submit(sid, cams[0], light, first))[0] == 0  # fills the cache
    reqs = [(cams[1], light2)] + [(c, light) for c in cams[1:]]
    outs = [torch.full((256, 256, 3), -1.0, device="cuda") for _ in reqs]
    torch.cuda.synchronize()
    ts = [srv.submit(sid, c, l, o) for (c, l), o in zip(reqs, outs)]
    for t in ts:
        assert srv.wait(t)[0] == 0
    st = srv.stats()
    assert st.completed == len(reqs) + 1 and st.failed == 0
    assert st.light_reuse == len(cams) - 1  # every later view of the first light
    assert torch.equal(first, alone(scenes[0], cams[0], light))
    for (c, l), o in zip(reqs, outs):
        assert torch.equal(o, alone(scenes[0], c, l))
    srv.close()


def test_light_cache_evicts_least_recently_used(scenes):
    """A full light cache drops its least recently used entry for a new light;
    one request at a time, so which lights are kept is fixed: with room for
    two, A B A C B C A reuses only the third (A) and the sixth (C)."""
    import torch
    from paper_2410_11419_gb300 import render as R
    srv = R.Server(hbm_budget=8 << 30, max_inflight=2, light_cache=2)
    sid = srv.add_scene(scenes[1])
    lights = {k: synth.camera_light_pair(40 + i, 128, 128)[1] for i, k in enumerate("ABC")}
    order = "ABACBCA"
    reused = []
    for i, k in enumerate(order):
        cam = synth.camera_light_pair(50 + i, 128, 128)[0]
        out = torch.full((128, 128, 3), -1.0, device="cuda")
        torch.cuda.synchronize()
        before = srv.stats().light_reuse
        assert srv.wait(srv.submit(sid, cam, lights[k], out))[0] == 0
        reused.append(srv.stats().light_reuse - before)
        assert torch.equal(out, alone(scenes[1], cam, lights[k])), (i, k)
    assert reused == [0, 0, 1, 0, 0, 1, 0]
    srv.close()


def test_admission_respects_budget(scenes):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    cam, light = synth.camera_light_pair(1, 256, 256)
    one = N.gs3_workspace_size(scenes[0].n, 256, 256, int(scenes[0].n * (4 + 64 * 256 * 256 / 640000)))
    srv = R.Server(hbm_budget=int(one * 1.5), max_inflight=4)
    sid = srv.add_scene(scenes[0])
    outs = [torch.empty((256, 256, 3), device="cuda") for _ in range(5)]
    ts = [srv.submit(sid, cam, light, o) for o in outs]
    for t in ts:
        assert srv.wait(t)[0] == 0
    st = srv.stats()
    assert st.max_in_flight == 1 and st.peak_bytes_in_use <= int(one * 1.5)
    want = alone(scenes[0], cam, light)
    for o in outs:
        assert torch.equal(o, want)
    srv.close()


def test_capacity_retry(scenes):
    import torch
    from paper_2410_11419_gb300 import render as R
    srv = R.Server(hbm_budget=8 << 30, max_inflight=2, initial_pairs=0.01)  # far too few pairs
    sid = srv.add_scene(scenes[0])
    cam, light = synth.camera_light_pair(3, 256, 256)
    out = torch.empty((256, 256, 3), device="cuda")
    assert srv.wait(srv.submit(sid, cam, light, out))[0] == 0
    assert srv.stats().retries >= 1
    assert torch.equal(out, alone(scenes[0], cam, light))
    # the next request of the same (scene, resolution) uses the learned capacity
    out2 = torch.empty_like(out)
    srv.reset_counters()
    assert srv.wait(srv.submit(sid, cam, light, out2))[0] == 0
    assert srv.stats().retries == 0
    srv.close()


def test_injected_allocation_failures(scenes):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    srv = R.Server(hbm_budget=8 << 30, max_inflight=2, inject_alloc_failures=2)
    sid = srv.add_scene(scenes[1])
    cam, light = synth.camera_light_pair(2, 128, 128)
    outs = [torch.empty((128, 128, 3), device="cuda") for _ in range(4)]
    ts = [srv.submit(sid, cam, light, o) for o in outs]
    res = [srv.wait(t)[0] for t in ts]
    assert res[:2] == [N.GS3_ERR_OOM, N.GS3_ERR_OOM] and res[2:] == [0, 0]
    want = alone(scenes[1], cam, light)
    assert torch.equal(outs[2], want) and torch.equal(outs[3], want)
    st = srv.stats()
    assert st.failed == 2 and st.completed == 2
    srv.close()


def test_rejects_bad_requests(scenes):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    budget = 256 << 20
    srv = R.Server(hbm_budget=budget, max_inflight=1)
    sid_small = srv.add_scene(scenes[1])
    sid_big = srv.add_scene(scenes[0])
    cam, light = synth.camera_light_pair(2, 64, 64)
    out = torch.empty((64, 64, 3), device="cuda")
    with pytest.raises(N.GS3Error):
        srv.submit(sid_small + 5, cam, light, out)
    # an output buffer far too small for the image (8 floats, in a 2 MB allocator
    # segment, for a 48 MB image) is refused before any work is queued
    bc, bl = synth.camera_light_pair(2, 2048, 2048)
    with pytest.raises(N.GS3Error):
        srv.submit(sid_small, bc, bl, torch.empty((8,), device="cuda"))
    # a request whose workspace can never fit the budget fails with OOM, others proceed
    res = 2048
    est = int(scenes[0].n * (4 + 64 * res * res / 640000.0))
    assert N.gs3_workspace_size(scenes[0].n, res, res, est) > budget
    big, blight = synth.camera_light_pair(2, res, res)
    big_out = torch.empty((res, res, 3), device="cuda")
    t_big = srv.submit(sid_big, big, blight, big_out)
    t_ok = srv.submit(sid_small, cam, light, out)
    assert srv.wait(t_big)[0] == N.GS3_ERR_OOM
    assert srv.wait(t_ok)[0] == 0
    srv.close()


def test_batches_render_frames_together(scenes):
    """Requests that queue while a slot is busy are rendered as one batch (the
    shadow and camera composites of all its frames in single launches); each
    frame still equals the same frame rendered alone, bit for bit, across
    scenes, MLP precisions, resolutions and ablations within a batch."""
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    srv = R.Server(hbm_budget=8 << 30, max_inflight=1, max_batch=4)
    ids = [srv.add_scene(d) for d in scenes]
    big_cam, big_light = synth.camera_light_pair(20, 1024, 1024)
    blocker = torch.empty((1024, 1024, 3), device="cuda")
    mix = [(0, 256, 21, 0), (1, 128, 22, N.GS3_ABLATE_SHADOW_SPLAT), (2, 160, 23, 0), (0, 200, 24, N.GS3_ABLATE_PHI),
           (1, 96, 25, 0), (0, 256, 26, N.GS3_ABLATE_SPECULAR), (2, 144, 27, N.GS3_ABLATE_PSI), (0, 320, 28, 0)]
    outs = [torch.full((res, res, 3), -1.0, device="cuda") for _, res, _, _ in mix]
    torch.cuda.synchronize()
    tickets = [srv.submit(ids[0], big_cam, big_light, blocker)]  # keeps the only slot busy
    for (si, res, seed, ab), out in zip(mix, outs):
        cam, light = synth.camera_light_pair(seed, res, res)
        tickets.append(srv.submit(ids[si], cam, light, out, R.opts_struct(ablate=ab)))
    for t in tickets:
        assert srv.wait(t)[0] == 0
    st = srv.stats()
    assert st.max_batch >= 2 and st.batches < len(tickets), (st.max_batch, st.batches)
    for (si, res, seed, ab), out in zip(mix, outs):
        cam, light = synth.camera_light_pair(seed, res, res)
        rd = R.Renderer(scenes[si], res, res, 1 << 23)
        want = rd.render(cam, light, R.opts_struct(ablate=ab)).clone()
        torch.cuda.synchronize()
        rd.check()
        assert torch.equal(out, want), (si, res, seed, ab)
    srv.close()


def test_shadow_chain_bounded_wait_gives_up(scenes):
    """The shadow composite's chained segment products wait for the segment
    before them; a chain whose first segments never publish gives up after the
    poll bound, records GS3_ERR_TIMEOUT, and the context stays usable."""
    import time
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = synth.object_scene(2, n=20000)
    ds = R.DeviceScene(scene)
    cam, light = synth.camera_light_pair(7, 256, 256)
    rd = R.Renderer(ds, 256, 256, 1 << 22)
    t0 = time.perf_counter()
    status = N.gs3_selftest_shadow_wait(ds.handle, R.camera_struct(cam), R.light_struct(light), R.opts_struct(),
                                        rd.ws, rd.ws.numel(), rd.cap)
    assert status == N.GS3_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    img = rd.render(cam, light).clone()  # a normal frame on the same context afterwards
    torch.cuda.synchronize()
    assert rd.check().status == 0 and torch.isfinite(img).all()
    ds.close()

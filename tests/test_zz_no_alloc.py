"""gs3_depth_order_static, the depth sort that allocates nothing.

Some callers may not allocate device memory at all (a renderer embedded in a
host application that owns the GPU's memory budget, a real-time loop that
must not risk an allocation stall or an out-of-memory failure mid-frame).
For them the library keeps the sort's scratch in a fixed device array.  This
file checks, through the C ABI, that its order equals the one gs3_render
leaves in its workspace, on two calls in a row (the array keeps the previous
call's contents between calls).  It is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2410_11419_gb300 import synth

pytestmark = pytest.mark.gpu


def test_static_depth_order_matches_render(gs3):
    import torch
    from paper_2410_11419_gb300 import _native as N, render as R
    scene = synth.object_scene(3, n=50_000)
    cam, light = synth.camera_light_pair(3, 256, 256)
    ds = R.DeviceScene(scene)
    rd = R.Renderer(ds, 256, 256, 1 << 23)
    rd.render(cam, light)
    torch.cuda.synchronize()
    rd.check()
    stream = torch.cuda.current_stream().cuda_stream
    for splat in (0, 1):
        keys = rd.stage("key", splat).clone()
        want = rd.stage("order", splat).clone()
        out = torch.empty(scene.n, dtype=torch.int32, device="cuda")
        for _ in range(2):
            out.fill_(-1)
            N.gs3_depth_order_static(keys, scene.n, out, stream)
            torch.cuda.synchronize()
            assert torch.equal(out, want)
    ds.close()


def test_static_depth_order_limits(gs3):
    import torch
    from paper_2410_11419_gb300 import _native as N
    stream = torch.cuda.current_stream().cuda_stream
    n = N.GS3_STATIC_SORT_MAX_KEYS
    rng = np.random.default_rng(0)
    host = rng.integers(0, 1 << 20, n, dtype=np.uint32)  # many ties: stability matters
    keys = torch.from_numpy(host.view(np.int32)).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    N.gs3_depth_order_static(keys, n, out, stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), np.argsort(host, kind="stable"))
    with pytest.raises(N.GS3Error) as e:
        N.gs3_depth_order_static(keys, n + 1, out, stream)
    assert e.value.status == N.GS3_ERR_INVALID_ARG
    assert "GS3_STATIC_SORT_MAX_KEYS" in str(e.value)
    N.gs3_depth_order_static(keys, 0, out, stream)  # empty input is a no-op


def test_static_depth_order_allocates_nothing(gs3):
    """After a first call (which may load the library's device code, and with
    it the fixed array), a call at the size limit leaves the device's free
    memory exactly as it was."""
    import torch
    from paper_2410_11419_gb300 import _native as N
    stream = torch.cuda.current_stream().cuda_stream
    n = N.GS3_STATIC_SORT_MAX_KEYS
    rng = np.random.default_rng(1)
    host = rng.integers(0, 1 << 31, n, dtype=np.uint32)
    keys = torch.from_numpy(host.view(np.int32)).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    N.gs3_depth_order_static(keys, n, out, stream)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    N.gs3_depth_order_static(keys, n, out, stream)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    np.testing.assert_array_equal(out.cpu().numpy(), np.argsort(host, kind="stable"))

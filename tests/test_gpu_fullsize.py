"""Parity at the benchmark's full size: the 300,000-Gaussian object scene,
K = 8, 3x128 MLPs, 800x800, with the capacity bench.py uses, against the full
FP64 oracle frame (about a minute of host time).  Integer stages bit for bit;
shading, shadow values, T', residual and the image within
|g - o| <= 1e-4 |o| + 1e-6 + bound (the oracle's decision-ambiguity bound)."""
import pytest

from paper_2410_11419_gb300 import synth
from tests.test_gpu_parity import check_float_stages, check_integer_stages, run_both

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("pair", [0, 57])
def test_object_scene_800(gs3, oracle, pair):
    scene = synth.object_scene(0)
    cam, light = synth.camera_light_pair(pair, 800, 800)
    g, fr = run_both(gs3, oracle, scene, cam, light, cap=40_000_000)
    assert g["hdr"].pairs_cam == fr["cam_P"] and g["hdr"].pairs_light == fr["light_P"]
    assert fr["cam_P"] > 10_000_000
    check_integer_stages(g, fr)
    check_float_stages(g, fr)

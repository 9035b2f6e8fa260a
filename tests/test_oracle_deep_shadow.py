"""The shadow-ray stop on a deep stack of nearly opaque layers, CPU.

The GPU composite stops a shadow ray once its occluder product falls below
2^-40 (the product is frozen from there on).  These pins check on a stack
whose exact products fall far below the FP32 range that the stopped
definition (a sequential O(L) walk per ray in tests/bruteforce.py) moves
every shadow value of the exact definition (the oracle) by less than 2^-40,
and that frozen products stay far from the denormals.
"""
import numpy as np

from paper_2410_11419_gb300 import synth
from tests import bruteforce

STOP = 2.0 ** -40


def deep_stack(res=48, layers=32, grid=8, seed=3):
    """The layered scene lit from z = 1.2 on its axis, seen obliquely."""
    sc = synth.layered_scene(seed, layers=layers, grid=grid)
    cam = synth.look_at_camera([1.6, 0.9, 1.4], width=res, height=res)
    light = synth.Light(pos=np.array([0.0, 0.0, 1.2], dtype=np.float32), intensity=10.0)
    return sc, cam, light


def test_stack_is_deep_and_stop_moves_shadow_by_less_than_the_stop(oracle):
    sc, cam, light = deep_stack()
    opts = oracle.Opts()
    fr = oracle.render(sc, cam, light, opts)
    T_stop, log2_exact, frozen_min = bruteforce.shadow_values_stopped(fr, opts, STOP)
    # many rays' exact products are below the smallest FP32 denormal
    assert np.mean(log2_exact < -149) > 0.15, np.percentile(log2_exact, [10, 50, 90])
    # a frozen product is at least stop (1 - alpha_max): far from the denormals
    assert frozen_min.min() >= STOP * (1.0 - opts.alpha_max) * (1.0 - 1e-12)
    diff = np.abs(T_stop - fr["T"])
    assert diff.max() < STOP
    assert diff.max() > 0.0  # the stop is active on this stack
    # front layers are lit, back layers dark
    z = sc.mean_op[:, 2]
    assert fr["T"][z > z.max() - 0.01].mean() > 0.3 and fr["T"][z < z.min() + 0.01].max() < 1e-6


def test_stopped_walk_without_stop_is_the_definition(oracle):
    """stop = 0 takes every occluder: the walk equals the O(L^2) product."""
    sc, cam, light = deep_stack(res=32, layers=6, grid=5)
    opts = oracle.Opts()
    fr = oracle.render(sc, cam, light, opts)
    T0, _, _ = bruteforce.shadow_values_stopped(fr, opts, 0.0)
    np.testing.assert_allclose(T0, bruteforce.shadow_values(fr, opts), rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(T0, fr["T"], rtol=1e-11, atol=1e-300)

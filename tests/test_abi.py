"""The C-ABI library loads and exports every symbol include/gs3.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs3.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs3_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libgs3():
    import __graft_entry__ as ge
    ge.build()
    from paper_2410_11419_gb300 import _native as N
    return N


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gs3_create_scene", "gs3_destroy_scene", "gs3_render", "gs3_workspace_size"):
        assert must in names


def test_library_exports_every_declared_symbol(libgs3):
    lib = ctypes.CDLL(libgs3.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(libgs3.SIGNATURES)


def test_struct_sizes_match_header_layout(libgs3):
    N = libgs3
    # field-for-field mirrors of the C structs (natural alignment)
    assert ctypes.sizeof(N.gs3_camera) == 4 * (9 + 3 + 3 + 4 + 2)
    assert ctypes.sizeof(N.gs3_light) == 4 * (3 + 1 + 1 + 3 + 1)   # pos, intensity, type, dir, extent
    assert ctypes.sizeof(N.gs3_render_opts) == 4 * (7 + 3 + 3)
    assert ctypes.sizeof(N.gs3_ws_header) == 4 * (8 + 12 + 1)
    assert ctypes.sizeof(N.gs3_ws_layout) == 8 * (2 + 5 * 2 + 8)
    assert ctypes.sizeof(N.gs3_server_opts) == 8 + 4 * 6      # budget, 5 int32/float fields, light_cache
    assert ctypes.sizeof(N.gs3_server_counters) == 8 * 12     # 8 counters, span, batches, max_batch, reuse


def test_host_only_entry_points(libgs3):
    N = libgs3
    o = N.gs3_default_opts()
    assert abs(o.shadow_bias - 0.015) < 1e-9 and o.tile == 16
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.t_stop - 1e-4) < 1e-10
    a = N.gs3_workspace_size(1000, 128, 128, 1 << 20)
    b = N.gs3_workspace_size(1000, 128, 128, 1 << 21)
    assert 0 < a < b
    lay = N.gs3_workspace_layout(1000, 128, 128, 1 << 20)
    assert lay.total == a
    offs = [lay.header, *lay.key, *lay.order, *lay.tile_start, *lay.list, lay.shade, lay.shadow,
            lay.shadow_refined, lay.residual, lay.final_t, lay.n_contrib, lay.light_final, lay.light_stop]
    assert all(o % 256 == 0 and o < a for o in offs)
    assert N.gs3_workspace_size(0, 128, 128, 10) == 0
    with pytest.raises(N.GS3Error):
        N.gs3_workspace_layout(0, 128, 128, 10)
    # the bounded-wait self-test validates its arguments before any CUDA call
    for bad in (0, 4096, (1 << 20) + 1):
        with pytest.raises(N.GS3Error):
            N.gs3_selftest_wait_timeout(bad)
    # so does the ALU peak measurement
    for bad in (0, 101):
        with pytest.raises(N.GS3Error):
            N.gs3_measure_alu_peak(bad)

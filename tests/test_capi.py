"""CPU checks of the C ABI: the library builds, loads, and exports every
entry point include/wrf.h declares; host-side argument validation runs
without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wrf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wrf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_12787_b300 import build, _lib
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2506_12787_b300 import _lib
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS)


def test_version_and_error_string(lib):
    assert lib.wrf_version() >= 1
    assert isinstance(lib.wrf_last_error(), bytes)


def test_host_validation_rejects_bad_arguments(lib):
    """Argument errors are caught on the host before any launch."""
    from paper_2506_12787_b300 import _lib
    g = _lib.Grid(90, 360, 12, 16, 9.0)  # unsupported tile shape
    st = lib.wrf_render(None, None, None, None, 0, 0, 1, C.byref(g), None, None)
    assert st == _lib.WRF_EUNSUPPORTED
    assert b"tile" in lib.wrf_last_error()
    g = _lib.Grid(90, 360, 16, 16, -1.0)
    assert lib.wrf_render(None, None, None, None, 0, 0, 1, C.byref(g), None, None) == _lib.WRF_EINVAL
    g = _lib.Grid(90, 360, 16, 16, 9.0)
    # NULL outputs with Q > 0
    assert lib.wrf_render(None, None, None, None, 0, 0, 1, C.byref(g), None, None) == _lib.WRF_EINVAL
    s = _lib.Scene(10, 3, None, None, None, None, None)  # three channels: unsupported
    assert lib.wrf_project(C.byref(s), None, 1, C.byref(g), None, None, None) == _lib.WRF_EUNSUPPORTED
    s = _lib.Scene(10, 2, None, None, None, None, None)  # two channels, NULL arrays
    assert lib.wrf_project(C.byref(s), None, 1, C.byref(g), None, None, None) == _lib.WRF_EINVAL
    m = _lib.Mlp()
    m.n_layers = 5
    m.L_mean, m.L_tx = 6, 10
    for i, d in enumerate([89, 128, 128, 128, 100, 5]):
        m.dims[i] = d
    assert lib.wrf_deform_workspace_size(10, 2, C.byref(m)) > 0
    s = _lib.Scene(0, 1, None, None, None, None, None)
    st = lib.wrf_deform(C.byref(s), C.byref(m), C.byref(g), None, 0, None, None, 0, None)
    assert st == _lib.WRF_EUNSUPPORTED  # hidden width 100


def test_mlp_precision_validation(lib):
    """Precision codes: FP32, BF16 and BF16X3 accepted; an unknown code is
    EINVAL; the tensor-core precisions take at most three hidden 128 x 128
    layers; saved activations need FP32 or BF16X3.  Weight pointers are
    placeholders: validation never dereferences them."""
    from paper_2506_12787_b300 import _lib

    def mlp(n_layers, precision):
        m = _lib.Mlp()
        m.n_layers = n_layers
        m.L_mean, m.L_tx = 6, 10
        dims = [89] + [128] * (n_layers - 1) + [5]
        for i, d in enumerate(dims):
            m.dims[i] = d
        for i in range(n_layers):
            m.W[i] = m.b[i] = 4096
        for i in range(3):
            m.room_size[i] = 1.0
        m.precision = precision
        return m

    g = _lib.Grid(90, 360, 16, 16, 9.0)
    s = _lib.Scene(0, 1, None, None, None, None, None)
    ws = C.c_void_p(1 << 20)
    tx = C.c_void_p(4096)
    acts = C.c_void_p(1 << 16)

    def deform(m, with_acts):
        need = lib.wrf_deform_workspace_size(0, 1, C.byref(m))
        if with_acts:
            return lib.wrf_deform_acts(C.byref(s), C.byref(m), C.byref(g), tx, 1, None, acts,
                                       ws, need, None)
        return lib.wrf_deform(C.byref(s), C.byref(m), C.byref(g), tx, 1, None, ws, need, None)

    for p in (_lib.WRF_FP32, _lib.WRF_BF16, _lib.WRF_BF16X3):
        assert deform(mlp(5, p), False) == _lib.WRF_OK  # N = 0: nothing to launch
    assert deform(mlp(5, 3), False) == _lib.WRF_EINVAL
    assert b"precision" in lib.wrf_last_error()
    assert deform(mlp(6, _lib.WRF_FP32), False) == _lib.WRF_OK
    for p in (_lib.WRF_BF16, _lib.WRF_BF16X3):
        assert deform(mlp(6, p), False) == _lib.WRF_EUNSUPPORTED
    assert deform(mlp(5, _lib.WRF_BF16), True) == _lib.WRF_EUNSUPPORTED
    assert deform(mlp(5, _lib.WRF_BF16X3), True) == _lib.WRF_OK
    assert deform(mlp(5, _lib.WRF_FP32), True) == _lib.WRF_OK


def test_rasteriser_knob_validation(lib):
    """Pixels per thread 2 or 4 (4 needs tiles >= 16 wide), records per thread
    1 or 2; 0 picks the default; both renderers take every combination."""
    from paper_2506_12787_b300 import _lib, autotune
    def render(g):
        return lib.wrf_render(None, None, None, None, 0, 0, 1, C.byref(g), None, None)
    for px, bf, want in [(3, 0, _lib.WRF_EUNSUPPORTED), (0, 3, _lib.WRF_EUNSUPPORTED),
                         (1, 1, _lib.WRF_EUNSUPPORTED), (4, 2, _lib.WRF_EINVAL),
                         (0, 0, _lib.WRF_EINVAL), (2, 1, _lib.WRF_EINVAL)]:
        # WRF_EINVAL: the knobs pass and the NULL outputs are caught next
        assert render(_lib.Grid(90, 360, 16, 16, 9.0, 0, px, bf)) == want, (px, bf)
    assert render(_lib.Grid(90, 360, 8, 8, 9.0, 0, 4, 1)) == _lib.WRF_EUNSUPPORTED
    assert b"tile_w" in lib.wrf_last_error()
    g = _lib.Grid(90, 360, 16, 16, 9.0, 0, 4, 1)  # knobs pass; the NULL outputs do not
    assert lib.wrf_render_complex(None, None, None, None, 0, 0, 1, C.byref(g), None,
                                  None) == _lib.WRF_EINVAL
    assert render(_lib.Grid(90, 360, 16, 16, 9.0, 0, 2, 1, 2)) == _lib.WRF_EINVAL
    assert b"tma_staging" in lib.wrf_last_error()
    # the autotuner's search space is exactly the supported combinations
    sp = autotune.space()
    assert len(sp) == 2 * (5 * 4 - 2) and len(set(sp)) == len(sp)
    for tw, th, px, bf, tma in sp:
        # every combination passes validation (the NULL outputs are caught next)
        assert render(_lib.Grid(90, 360, tw, th, 9.0, 0, px, bf, tma)) == _lib.WRF_EINVAL
        assert b"NULL" in lib.wrf_last_error()
    assert sorted({autotune.batch_records(*c) for c in sp}) == [32, 64, 128, 256, 512]
    assert autotune.parse_config("32x8") == (32, 8, 2, 1, 0)
    assert autotune.parse_config("16x16p4b2") == (16, 16, 4, 2, 0)
    assert autotune.parse_config("16x16p4b2t") == (16, 16, 4, 2, 1)
    for name in ("32x16p2b2", "32x16p4b1t"):
        assert autotune.config_name(*autotune.parse_config(name)) == name
    k1 = autotune.workload_key(20000, 90, 360, 256, 1, 9.0)
    k2 = autotune.workload_key(20000, 90, 360, 256, 1, 9.0, candidates=sp[:3])
    assert k1 != k2  # the key names the search space


def test_paper_head_host_validation(lib):
    """The paper head's entry point checks its network shape on the host."""
    from paper_2506_12787_b300 import _lib
    g = _lib.Grid(90, 360, 16, 16, 9.0)
    s = _lib.PaperScene(10, None, None, None, None)
    assert lib.wrf_paper_deform_project(C.byref(s), None, C.byref(g), None, 1, None, None, 0,
                                        None) == _lib.WRF_EINVAL  # NULL arrays
    s = _lib.PaperScene(0, None, None, None, None)
    m = _lib.PaperMlp()
    m.n_hidden, m.width, m.L_mean, m.L_tx = 8, 161, 10, 6
    assert lib.wrf_paper_deform_project(C.byref(s), C.byref(m), C.byref(g), None, 1, None, None,
                                        0, None) == _lib.WRF_EUNSUPPORTED
    m.width, m.n_hidden = 156, 9
    assert lib.wrf_paper_deform_project(C.byref(s), C.byref(m), C.byref(g), None, 1, None, None,
                                        0, None) == _lib.WRF_EUNSUPPORTED
    m.n_hidden = 8
    assert lib.wrf_paper_deform_project(C.byref(s), C.byref(m), C.byref(g), None, 1, None, None,
                                        0, None) == _lib.WRF_EINVAL  # NULL weights
    assert lib.wrf_paper_deform_project(C.byref(s), None, C.byref(g), None, 70000, None, None,
                                        0, None) == _lib.WRF_EUNSUPPORTED  # Q > 65535
    # no Gaussians, no deformation: nothing to do
    assert lib.wrf_paper_deform_project(C.byref(s), None, C.byref(g), None, 4, None, None, 0,
                                        None) == _lib.WRF_OK
    assert 0 < lib.wrf_paper_workspace_size(100, 2) < lib.wrf_paper_workspace_size(10000, 64)


def test_workspace_sizes_are_monotone(lib):
    from paper_2506_12787_b300 import _lib
    g = _lib.Grid(90, 360, 16, 16, 9.0)
    a = lib.wrf_bin_workspace_size(20000, 16, C.byref(g))
    b = lib.wrf_bin_workspace_size(20000, 256, C.byref(g))
    assert 0 < a < b


def test_product_path_does_not_import_the_oracle():
    """The library package never references the oracle or a CPU fallback."""
    pkg = os.path.join(ROOT, "paper_2506_12787_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f


def test_pipeline_host_validation(lib):
    """wrf_pipeline_*: argument errors come back before any CUDA call (no GPU
    needed); NULL handles are rejected, and destroying NULL is a no-op."""
    from paper_2506_12787_b300 import _lib
    m = _lib.Mlp()
    m.n_layers = 5
    m.L_mean, m.L_tx = 6, 10
    for i, d in enumerate([89, 128, 128, 128, 128, 5]):
        m.dims[i] = d
    for i in range(5):
        m.W[i] = m.b[i] = 4096  # placeholders: validation never dereferences them
    for i in range(3):
        m.room_size[i] = 1.0
    m.precision = _lib.WRF_BF16
    s = _lib.Scene(0, 1, None, None, None, None, None)
    g = _lib.Grid(90, 360, 32, 16, 9.0)
    p = C.c_void_p()
    assert lib.wrf_pipeline_create(C.byref(s), C.byref(m), C.byref(g), 4, 0.0, None) == \
        _lib.WRF_EINVAL
    bad = _lib.Grid(90, 360, 12, 16, 9.0)
    assert lib.wrf_pipeline_create(C.byref(s), C.byref(m), C.byref(bad), 4, 0.0, C.byref(p)) == \
        _lib.WRF_EUNSUPPORTED
    assert p.value is None
    for Q in (0, -1, 70000):
        assert lib.wrf_pipeline_create(C.byref(s), C.byref(m), C.byref(g), Q, 0.0,
                                       C.byref(p)) == _lib.WRF_EINVAL
    for margin in (0.5, -1.0, float("nan")):
        assert lib.wrf_pipeline_create(C.byref(s), C.byref(m), C.byref(g), 4, margin,
                                       C.byref(p)) == _lib.WRF_EINVAL
        assert b"key_margin" in lib.wrf_last_error()
    assert lib.wrf_pipeline_step(None, None, None) == _lib.WRF_EINVAL
    assert lib.wrf_pipeline_wait(None) == _lib.WRF_EINVAL
    assert lib.wrf_pipeline_destroy(None) == _lib.WRF_OK

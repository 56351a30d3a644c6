"""The C ABI library builds, loads and exports every symbol include/flic.h declares.
No compute call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "flic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flic_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2003_00575_gb300 import build
    return build.build()


def test_header_declares_the_hot_path():
    names = _declared()
    for n in ("flic_create", "flic_project", "flic_label", "flic_scatter", "flic_destroy",
              "flic_label_batch", "flic_edges", "flic_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2003_00575_gb300 import flic
    assert sorted(flic.SIGNATURES) == _declared()
    assert flic.flic_abi_version() == 1


def test_invalid_arguments_rejected_without_gpu(lib_path):
    """Argument checks run before any CUDA call, so they work on a machine with no GPU."""
    from paper_2003_00575_gb300 import flic
    import numpy as np
    lib = flic._lib
    out = ctypes.c_void_p()
    elev = np.zeros(4)
    assert lib.flic_create(0, 8, elev.ctypes.data, 0.1, 0.5, 1, ctypes.byref(out)) == flic.FLIC_ERR_INVALID
    assert lib.flic_create(4, 8, None, 0.1, 0.5, 1, ctypes.byref(out)) == flic.FLIC_ERR_INVALID
    assert lib.flic_create(4, 8, elev.ctypes.data, 0.1, -0.5, 1, ctypes.byref(out)) == flic.FLIC_ERR_INVALID
    assert lib.flic_create(4, 8, elev.ctypes.data, 0.1, 0.5, 9, ctypes.byref(out)) == flic.FLIC_ERR_INVALID
    assert lib.flic_create(4, 8, elev.ctypes.data, float("nan"), 0.5, 1, ctypes.byref(out)) == flic.FLIC_ERR_INVALID
    assert b"az_step" in lib.flic_last_error()
    assert lib.flic_label(None, None, None, None) == flic.FLIC_ERR_INVALID
    assert lib.flic_batch_create(0, ctypes.byref(out)) == flic.FLIC_ERR_INVALID
    assert lib.flic_destroy(None) == flic.FLIC_OK
    assert lib.flic_batch_destroy(None) == flic.FLIC_OK
    assert lib.flic_label_batch_host(None, None, 1, None, None, 0, 0, None) == flic.FLIC_ERR_INVALID
    assert lib.flic_label_filter_batch(None, None, None, None, 1, 100, None, None) == flic.FLIC_ERR_INVALID
    assert lib.flic_filter_relabel_batch(None, None, None, 1, 100, None, None) == flic.FLIC_ERR_INVALID


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2003_00575_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "flic_oracle" not in text, fn


@pytest.mark.parametrize("seed", range(300))
def test_strip_planner_invariants(lib_path, seed):
    """Host-only planner: strips cover the columns, every strip of a multi-strip frame is at
    least S wide (so an edge crosses at most one border and lands in the first S columns of
    the next strip), widths are multiples of 4, and the padded strip fits 16-bit indices."""
    import numpy as np
    from paper_2003_00575_gb300 import flic
    g = np.random.default_rng(seed)
    R = int(g.integers(1, 513))
    C = int(g.integers(1, max(2, (1 << 21) // R + 1)))
    S = int(g.integers(1, 9))
    px = int(g.choice([64, 1024, 4096, 8192, 16384, 32768]))
    cl = int(g.integers(1, 65))
    try:
        p = flic.flic_plan_frame(R, C, S, px, cl)
    except flic.FlicError as e:
        assert e.status == flic.FLIC_ERR_UNSUPPORTED
        return
    n, W, P = p["strips"], p["strip_w"], p["pitch"]
    assert 1 <= n <= cl
    assert (n - 1) * W < C <= n * W
    last = C - (n - 1) * W
    if n > 1:
        assert W % 4 == 0 and W >= S and last >= S
    assert P >= max(W, 32) and P & (P - 1) == 0
    assert R * P <= 32768
    rp = (W + S + 3) // 4 * 4
    assert 4 * R * max(rp, P) + 4 * R * (P // 32) * (2 * S + 1) + 64 == p["smem"]
    assert p["smem"] <= 227 * 1024 - 1024


def test_diagonal_and_sparse_map_flags_are_exclusive():
    """The flags are checked before any device work, so this runs without a GPU."""
    import numpy as np
    from paper_2003_00575_gb300 import flic
    with pytest.raises(flic.FlicError) as e:
        flic.flic_create(4, 16, np.radians([3.0, 1.0, -1.0, -3.0]), 2 * np.pi / 16, 0.5, 2,
                         lattice=True, diagonal=True)
    assert e.value.status == flic.FLIC_ERR_INVALID

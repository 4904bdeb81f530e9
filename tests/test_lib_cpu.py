"""Host-side checks of the C ABI library (no GPU needed): it builds for sm_103a,
loads, and exports every entry point that include/jz.h declares."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(jz_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2003_08746_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("jz_create_grid", "jz_compute_metrics", "jz_set_state", "jz_rk_step", "jz_residual",
                     "jz_get_metrics", "jz_create", "jz_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header(lib):
    from paper_2003_08746_gb300 import jz
    assert set(jz.EXPORTS) <= set(_declared_functions())
    assert set(_declared_functions()) <= set(jz.EXPORTS) | {"jz_adjoint_step"}


def test_version_and_error_without_gpu(lib):
    lib.jz_version.restype = ctypes.c_int
    assert lib.jz_version() >= 1
    lib.jz_last_error.restype = ctypes.c_char_p
    assert lib.jz_last_error() is not None


def test_argument_errors_do_not_need_a_gpu(lib):
    """Bad sizes and NULL pointers are rejected before any CUDA call."""
    vp = ctypes.c_void_p
    lib.jz_create_grid.argtypes = [ctypes.c_int] * 3 + [vp, vp, ctypes.c_int, ctypes.POINTER(vp)]
    lib.jz_create_grid.restype = ctypes.c_int
    lib.jz_last_error.restype = ctypes.c_char_p
    h = vp()
    buf = (ctypes.c_double * 48)()
    assert lib.jz_create_grid(4, 4, 3, ctypes.cast(buf, vp), None, 2, ctypes.byref(h)) == -1   # odd nk
    assert b"even" in lib.jz_last_error()
    assert lib.jz_create_grid(4, 4, 4, None, None, 2, ctypes.byref(h)) == -1
    assert lib.jz_create_grid(4, 4, 4, ctypes.cast(buf, vp), None, 1, ctypes.byref(h)) == -1   # no period
    assert lib.jz_create_grid(4, 4, 4, ctypes.cast(buf, vp), None, 7, ctypes.byref(h)) == -1
    lib.jz_rk_step.argtypes = [vp, ctypes.c_int, vp]
    assert lib.jz_rk_step(None, 1, None) == -1
    lib.jz_destroy.argtypes = [vp]
    assert lib.jz_destroy(None) == -1
    # entry points beside the hot path
    for name, args in (("jz_grid_compact", [None]), ("jz_stats_begin", [None, 1]), ("jz_stats_sample", [None]),
                       ("jz_stats_end", [None]), ("jz_save_snapshot", [None, b"x"]), ("jz_load_snapshot", [None, b"x"]),
                       ("jz_check_math", [None, None, None]), ("jz_compute_metrics", [None]), ("jz_get_state", [None, None])):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        assert fn(*args) == -1, name
        assert lib.jz_last_error(), name


def test_product_path_has_no_oracle_import():
    """The library package never imports the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2003_08746_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "from oracle" not in src and "import oracle" not in src


def test_snapshot_reader_layout(tmp_path):
    """read_snapshot parses the documented layout: 256-byte little-endian header, then
    Q^n as [5][nk][nj][ni] float64 (file written here field by field)."""
    import struct
    from paper_2003_08746_gb300 import jz
    ni, nj, nk = 5, 4, 6
    q = np.random.default_rng(0).standard_normal((5, nk, nj, ni))
    head = b"JZSNAP01" + struct.pack("<8i", 1, 256, ni, nj, nk, 2, 1, 1) + struct.pack("<q", 17)
    head += struct.pack("<4d", 0.25, 1e-3, 3.5, 0.0) + struct.pack("<2Q", 11, 22)
    head += bytes(256 - len(head))
    assert len(head) == 256
    p = tmp_path / "s.bin"
    p.write_bytes(head + q.astype("<f8").tobytes())
    hd, qr = jz.read_snapshot(p)
    assert (hd["ni"], hd["nj"], hd["nk"], hd["topology"], hd["precision"], hd["flags"]) == (ni, nj, nk, 2, 1, 1)
    assert hd["steps"] == 17 and hd["t"] == 0.25 and hd["dt"] == 1e-3 and hd["params_hash"] == 11
    assert np.array_equal(qr, q)
    p.write_bytes(head + q.astype("<f8").tobytes()[:-8])
    with pytest.raises(ValueError, match="short"):
        jz.read_snapshot(p)


def test_station_and_core_helpers_vs_oracle():
    """The library's host-only station and potential-core helpers (no GPU) against the
    oracle's definitions on random profiles."""
    import torch
    from oracle import jz_oracle as O
    from paper_2003_08746_gb300 import jz
    rng = np.random.default_rng(4)
    x = np.cumsum(np.r_[0.0, rng.uniform(0.1, 0.5, 40)])
    f = rng.standard_normal((9, x.size))
    for x0 in (x[0], x[5], 0.3 * x[10] + 0.7 * x[11], x[-1], 2.5, 5.0):
        got = jz.jz_station_profile(f, x, x0)
        ref = O.station_profile(torch.from_numpy(f), x, float(x0)).numpy()
        assert np.abs(got - ref).max() <= 1e-15 * np.abs(f).max()
    with pytest.raises(jz.JzError):
        jz.jz_station_profile(f, x, x[-1] + 0.1)
    axis = 1.4 - 0.05 * np.maximum(x - 3.0, 0.0) + 1e-3 * rng.standard_normal(x.size) * (x > 3.0)
    got, ref = jz.jz_potential_core(axis, x, 1.4), O.potential_core_length(torch.from_numpy(axis), x, 1.4)
    assert ref is not None and abs(got - ref) <= 1e-13
    assert jz.jz_potential_core(np.full(x.size, 1.4), x, 1.4) is None

"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/dsc.h declares.  CPU only: no compute call needs a GPU here."""
import os
import re

import pytest

from paper_0908_4417_gb300 import build as B
from paper_0908_4417_gb300 import dsc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "dsc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dsc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return dsc.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(dsc.EXPORTS) == names


def test_library_metadata(lib):
    assert dsc.dsc_abi_version() == 3
    assert lib.dsc_status_str(0) == b"ok"
    assert lib.dsc_status_str(5) == b"device wait timed out"
    assert dsc.dsc_launch_count() >= 0


def test_null_arguments_are_rejected(lib):
    import ctypes as C
    out = C.c_void_p()
    assert lib.dsc_create_geometry(None, None, 0, None, None, C.byref(out)) == 1
    assert b"null" in lib.dsc_last_error()
    assert lib.dsc_compute_dij(None, None, None, C.byref(out)) == 1
    peaks = (C.c_double * 6)()
    assert lib.dsc_measure_alu_peaks(200.0, None, 6, None) == 1
    assert lib.dsc_measure_alu_peaks(200.0, peaks, 5, None) == 1
    assert lib.dsc_measure_alu_peaks(0.5, peaks, 6, None) == 1
    assert b"ms_per_loop" in lib.dsc_last_error()
    assert lib.dsc_measure_alu_peaks(float("nan"), peaks, 6, None) == 1
    link = (C.c_double * 4)()
    assert lib.dsc_measure_host_link(1 << 20, 3, None, 4, None) == 1
    assert lib.dsc_measure_host_link(1 << 20, 3, link, 3, None) == 1
    assert lib.dsc_measure_host_link(1000, 3, link, 4, None) == 1
    assert lib.dsc_measure_host_link(1 << 20, 0, link, 4, None) == 1
    assert lib.dsc_measure_host_link(1 << 20, 101, link, 4, None) == 1
    assert lib.dsc_probe_tail(3, None, 0, None, None, None) == 1
    assert lib.dsc_probe_tail(0, None, 4, None, None, None) == 1
    assert lib.dsc_probe_tail(0, None, 0, None, None, None) == 0       # nothing to do
    a, b = C.c_int64(), C.c_int64()
    assert lib.dsc_get_refine_counts(None, C.byref(a), C.byref(b), C.byref(a)) == 1
    assert lib.dsc_get_tile_counts(None, C.byref(a), C.byref(b)) == 1
    assert lib.dsc_copy_csr_to_host(None, None, None, None, None, None) == 1
    assert lib.dsc_copy_csr_to_host_async(None, None, None, None, None, None) == 1


def test_struct_layouts_match_header():
    import ctypes as C
    assert C.sizeof(dsc.GridDesc) == 3 * 4 + 4 + 6 * 8
    assert C.sizeof(dsc.BeamDesc) == 8 * 7 + 8
    assert C.sizeof(dsc.ComputeOpts) == 32
    assert C.sizeof(dsc.CsrView) == 3 * 8 + 3 * 8 + 8 + 8 + 8 + 8
    assert C.sizeof(dsc.Tuning) == 8
    assert C.sizeof(dsc.FspbModel) == 8 + 8 + 8 + 48 + 8 + 8 + 8


def test_tuning_is_validated_and_round_trips(lib):
    """Host-only entry points: the work decomposition setting."""
    before = dsc.dsc_get_tuning()
    assert before == (8192, 0)
    for bad in ((100, 0), (1 << 20, 0), (8192, -1), (8192, 1000)):
        with pytest.raises(dsc.DscError):
            dsc.dsc_set_tuning(*bad)
    assert dsc.dsc_get_tuning() == before
    dsc.dsc_set_tuning(4096, 3)
    assert dsc.dsc_get_tuning() == (4096, 3)
    dsc.dsc_set_tuning(*before)
    assert lib.dsc_set_tuning(None) == 1 and lib.dsc_get_tuning(None) == 1
    assert lib.dsc_autotune(None, 0, None, None, 1, None, None) == 1


def test_model_validation_before_any_device_work(lib):
    """Every width c3_i must be finite and > 0 and T finite; rejected on the
    host before a device is touched (CPU only)."""
    import ctypes as C
    import numpy as np
    from paper_0908_4417_gb300 import phantoms as P
    m = P.synthetic_model()
    g = dsc.grid_desc(P.centred_grid(4, 4, 4, 2.0, 2.0, 2.0))
    rho = np.ones(64, np.float32)
    out = C.c_void_p()
    for col, bad in ((2, 0.0), (3, -1.0), (1, float("nan")), (0, float("inf"))):
        lut = m.lut.copy()
        lut[7, col] = bad
        mm = dsc._ModelRef(P.Model(lut=lut, d_max=m.d_max))
        st = lib.dsc_create_geometry(C.byref(g), rho.ctypes.data, 0, C.byref(mm.s), None, C.byref(out))
        assert st == 1, (col, bad)
        assert b"finite" in lib.dsc_last_error()
    bad_profile = dsc._ModelRef(P.Model(lut=m.lut, d_max=m.d_max, profile=3))
    assert lib.dsc_create_geometry(C.byref(g), rho.ctypes.data, 0, C.byref(bad_profile.s), None, C.byref(out)) == 1

"""ctypes binding of libdsc (include/dsc.h), same entry-point names.

Argument marshalling only: every step of the D_ij path runs in the library's
sm_103a kernels.  There is no CPU fallback -- if libdsc.so is missing or no
CUDA device is present, calls raise.

Device buffers handed to the library (density_on_device=1) are torch CUDA
tensors' ``data_ptr()``; streams are ``torch.cuda.Stream.cuda_stream`` (or 0
for the legacy default stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdsc.so")

DSC_OK = 0
DSC_E_BUSY = 8
DSC_W_INEXACT = 9
DSC_CUTOFF_VOI6, DSC_CUTOFF_SIGMA, DSC_CUTOFF_NONE = 0, 1, 2
DSC_VALUE_F32, DSC_VALUE_BF16 = 0, 1
DSC_PROFILE_ERF, DSC_PROFILE_LAPLACE, DSC_PROFILE_LOGISTIC = 0, 1, 2
DSC_FLAG_TIMING = 1
DSC_FLAG_TRILINEAR_TABLE = 2
STAGES = ("setup", "siddon", "count", "eval", "beam_scale", "compact", "finish", "total")

EXPORTS = [
    "dsc_status_str", "dsc_last_error", "dsc_abi_version", "dsc_launch_count",
    "dsc_create_geometry", "dsc_upload_density", "dsc_add_beam", "dsc_clear_beams", "dsc_destroy_geometry",
    "dsc_compute_dij", "dsc_compute_dij_batch", "dsc_result_wait", "dsc_get_csr", "dsc_copy_csr_to_host",
    "dsc_copy_csr_to_host_async",
    "dsc_release_result", "dsc_get_beamlets", "dsc_get_depth_tables", "dsc_get_row_stats", "dsc_get_stage_times",
    "dsc_server_create", "dsc_server_submit", "dsc_server_poll", "dsc_server_stats", "dsc_server_destroy",
    "dsc_compute_dij_noalloc", "dsc_set_tuning", "dsc_get_tuning", "dsc_autotune", "dsc_dose", "dsc_beamlet_dot",
    "dsc_measure_alu_peaks", "dsc_probe_tail", "dsc_get_refine_counts", "dsc_get_server_timing",
    "dsc_measure_host_link", "dsc_get_tile_counts",
]


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("origin", C.c_double * 3)]


class FspbModel(C.Structure):
    _fields_ = [("n", C.c_int32), ("d_max", C.c_double), ("table4", C.c_void_p),
                ("c1", C.c_double * 3), ("c2", C.c_double * 3), ("cutoff_mode", C.c_int32), ("cutoff_k", C.c_double),
                ("profile", C.c_int32)]


class BeamDesc(C.Structure):
    _fields_ = [("gantry_deg", C.c_double), ("sad", C.c_double), ("iso", C.c_double * 3),
                ("a", C.c_double), ("b", C.c_double), ("n_u", C.c_int32), ("n_v", C.c_int32)]


class ComputeOpts(C.Structure):
    _fields_ = [("rel_threshold", C.c_double), ("value_dtype", C.c_int32), ("h_frac", C.c_double),
                ("flags", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("target_cand", C.c_int32), ("eval_blocks_per_sm", C.c_int32)]


class CsrView(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("value_dtype", C.c_int32), ("nbeams", C.c_int32), ("beam_scale", C.c_void_p),
                ("pairs", C.c_int64), ("on_device", C.c_int32)]


class DscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dsc status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libdsc.so (built by build.py).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdsc.so not built ({LIB_PATH}); run paper_0908_4417_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, V, I32, I64, U64 = C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
        sig = {
            "dsc_status_str": (C.c_char_p, [C.c_int]),
            "dsc_last_error": (C.c_char_p, []),
            "dsc_abi_version": (I32, []),
            "dsc_launch_count": (I64, []),
            "dsc_create_geometry": (C.c_int, [C.POINTER(GridDesc), P, I32, C.POINTER(FspbModel), P, C.POINTER(P)]),
            "dsc_upload_density": (C.c_int, [P, P, I32, P]),
            "dsc_add_beam": (C.c_int, [P, C.POINTER(BeamDesc), C.POINTER(I32)]),
            "dsc_clear_beams": (C.c_int, [P]),
            "dsc_destroy_geometry": (None, [P]),
            "dsc_compute_dij": (C.c_int, [P, C.POINTER(ComputeOpts), P, C.POINTER(P)]),
            "dsc_compute_dij_batch": (C.c_int, [C.POINTER(P), I32, C.POINTER(ComputeOpts), P, C.POINTER(P)]),
            "dsc_result_wait": (C.c_int, [P]),
            "dsc_get_csr": (C.c_int, [P, I32, C.POINTER(CsrView)]),
            "dsc_copy_csr_to_host": (C.c_int, [P, P, P, P, P, P]),
            "dsc_copy_csr_to_host_async": (C.c_int, [P, P, P, P, P, P]),
            "dsc_release_result": (None, [P]),
            "dsc_get_beamlets": (C.c_int, [P, P, I64]),
            "dsc_get_depth_tables": (C.c_int, [P, P, I64, C.POINTER(I32)]),
            "dsc_get_row_stats": (C.c_int, [P, P, P]),
            "dsc_get_stage_times": (C.c_int, [P, P, I32]),
            "dsc_server_create": (C.c_int, [C.c_size_t, I32, I32, C.POINTER(P)]),
            "dsc_server_submit": (C.c_int, [P, P, C.POINTER(BeamDesc), I32, C.POINTER(ComputeOpts), C.POINTER(U64)]),
            "dsc_server_poll": (C.c_int, [P, U64, I32, C.POINTER(P)]),
            "dsc_server_stats": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(I64),
                                           C.POINTER(I64)]),
            "dsc_server_destroy": (None, [P]),
            "dsc_compute_dij_noalloc": (C.c_int, [C.POINTER(GridDesc), P, C.POINTER(FspbModel), C.POINTER(BeamDesc),
                                                  I32, C.POINTER(ComputeOpts), P, P, P, I64, C.POINTER(I64), P]),
            "dsc_dose": (C.c_int, [P, P, P, P]),
            "dsc_beamlet_dot": (C.c_int, [P, P, P, P]),
            "dsc_set_tuning": (C.c_int, [C.POINTER(Tuning)]),
            "dsc_get_tuning": (C.c_int, [C.POINTER(Tuning)]),
            "dsc_autotune": (C.c_int, [C.POINTER(P), I32, C.POINTER(ComputeOpts), P, I32, C.POINTER(Tuning),
                                       C.POINTER(C.c_float)]),
            "dsc_measure_alu_peaks": (C.c_int, [C.c_double, C.POINTER(C.c_double), I32, P]),
            "dsc_measure_host_link": (C.c_int, [I64, I32, C.POINTER(C.c_double), I32, P]),
            "dsc_probe_tail": (C.c_int, [I32, P, I64, P, P, P]),
            "dsc_get_refine_counts": (C.c_int, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
            "dsc_get_tile_counts": (C.c_int, [P, C.POINTER(I64), C.POINTER(I64)]),
            "dsc_get_server_timing": (C.c_int, [P, C.POINTER(I32), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st):
    if st != DSC_OK:
        raise DscError(st, lib().dsc_last_error().decode(errors="replace"))


# ---------------------------------------------------------------------------
# descriptors from plain objects (phantom dataclasses or anything alike)
# ---------------------------------------------------------------------------
def grid_desc(g) -> GridDesc:
    return GridDesc(int(g.nx), int(g.ny), int(g.nz), float(g.dx), float(g.dy), float(g.dz),
                    (C.c_double * 3)(*[float(v) for v in g.origin]))


def beam_desc(b) -> BeamDesc:
    return BeamDesc(float(b.gantry_deg), float(b.sad), (C.c_double * 3)(*[float(v) for v in b.iso]),
                    float(b.a), float(b.b), int(b.n_u), int(b.n_v))


def compute_opts(tau=1e-3, value_dtype=DSC_VALUE_F32, h_frac=0.5, flags=0) -> ComputeOpts:
    return ComputeOpts(float(tau), int(value_dtype), float(h_frac), int(flags))


class _ModelRef:
    def __init__(self, m):
        self.table = np.ascontiguousarray(m.lut, dtype=np.float32)
        self.s = FspbModel(int(self.table.shape[0]), float(m.d_max), self.table.ctypes.data,
                           (C.c_double * 3)(*[float(v) for v in m.c1]), (C.c_double * 3)(*[float(v) for v in m.c2]),
                           int(m.cutoff_mode), float(m.cutoff_k), int(getattr(m, "profile", 0)))


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def dsc_abi_version() -> int:
    return int(lib().dsc_abi_version())


def dsc_launch_count() -> int:
    return int(lib().dsc_launch_count())


def dsc_create_geometry(grid, density, density_on_device: bool, model, stream=0):
    """density: numpy float32 [nz][ny][nx] (host) or a device pointer (int)."""
    g = grid_desc(grid)
    mr = _ModelRef(model)
    if density_on_device:
        ptr = int(density)
    else:
        density = np.ascontiguousarray(density, dtype=np.float32)
        assert density.shape == (grid.nz, grid.ny, grid.nx)
        ptr = density.ctypes.data
    out = C.c_void_p()
    _check(lib().dsc_create_geometry(C.byref(g), ptr, int(bool(density_on_device)), C.byref(mr.s), stream,
                                     C.byref(out)))
    return out.value


def dsc_upload_density(geom, density, density_on_device: bool, stream=0):
    if density_on_device:
        ptr = int(density)
    else:
        density = np.ascontiguousarray(density, dtype=np.float32)
        ptr = density.ctypes.data
    _check(lib().dsc_upload_density(geom, ptr, int(bool(density_on_device)), stream))


def dsc_add_beam(geom, beam) -> int:
    idx = C.c_int32()
    _check(lib().dsc_add_beam(geom, C.byref(beam_desc(beam)), C.byref(idx)))
    return idx.value


def dsc_clear_beams(geom):
    _check(lib().dsc_clear_beams(geom))


def dsc_destroy_geometry(geom):
    lib().dsc_destroy_geometry(geom)


def dsc_compute_dij(geom, opts: ComputeOpts, stream=0):
    out = C.c_void_p()
    _check(lib().dsc_compute_dij(geom, C.byref(opts), stream, C.byref(out)))
    return out.value


def dsc_compute_dij_batch(geoms, opts: ComputeOpts, stream=0):
    n = len(geoms)
    arr = (C.c_void_p * n)(*geoms)
    outs = (C.c_void_p * n)()
    _check(lib().dsc_compute_dij_batch(arr, n, C.byref(opts), stream, outs))
    return [outs[i] for i in range(n)]


def dsc_set_tuning(target_cand: int, eval_blocks_per_sm: int = 0):
    _check(lib().dsc_set_tuning(C.byref(Tuning(int(target_cand), int(eval_blocks_per_sm)))))


def dsc_get_tuning() -> tuple:
    t = Tuning()
    _check(lib().dsc_get_tuning(C.byref(t)))
    return int(t.target_cand), int(t.eval_blocks_per_sm)


def dsc_autotune(geoms, opts: ComputeOpts, stream=0, reps: int = 3) -> tuple:
    """Times the tile shapes on `geoms`, installs the fastest; returns
    ((target_cand, eval_blocks_per_sm), median ms)."""
    n = len(geoms)
    arr = (C.c_void_p * n)(*geoms)
    t, ms = Tuning(), C.c_float()
    _check(lib().dsc_autotune(arr, n, C.byref(opts), stream, int(reps), C.byref(t), C.byref(ms)))
    return (int(t.target_cand), int(t.eval_blocks_per_sm)), float(ms.value)


def dsc_dose(res, w_ptr: int, dose_ptr: int, stream=0):
    """Eq. 1 on the device: dose (ncols floats) = sum_j w_j D_j; pointers are device addresses."""
    _check(lib().dsc_dose(res, w_ptr, dose_ptr, stream))


def dsc_beamlet_dot(res, g_ptr: int, out_ptr: int, stream=0):
    """out (nrows floats) = D g on the device; pointers are device addresses."""
    _check(lib().dsc_beamlet_dot(res, g_ptr, out_ptr, stream))


def dsc_measure_alu_peaks(ms_per_loop: float = 200.0, stream=0) -> dict:
    """FP32 FMA and MUFU (ex2, rcp) rates of the current GPU, measured by the
    library's own loops; TFLOP/s and 10^12 operations/s, with device ms."""
    out = (C.c_double * 6)()
    _check(lib().dsc_measure_alu_peaks(float(ms_per_loop), out, 6, stream))
    return {"fp32_tflops": out[0], "ex2_tops": out[1], "rcp_tops": out[2],
            "ms": {"fma": out[3], "ex2": out[4], "rcp": out[5]}}


def dsc_measure_host_link(nbytes: int, reps: int = 3, stream=0) -> dict:
    """Host-link rates measured with pinned copies of nbytes each way (GB/s,
    10^9 bytes/s, the shortest of `reps`), with their device ms."""
    out = (C.c_double * 4)()
    _check(lib().dsc_measure_host_link(int(nbytes), int(reps), out, 4, stream))
    return {"d2h_gbs": out[0], "h2d_gbs": out[1], "ms": {"d2h": out[2], "h2d": out[3]}}


def dsc_probe_tail(profile: int, y_ptr: int, n: int, ours_ptr: int, cuda_ptr: int, stream=0):
    """T(y) as the evaluation computes it, and CUDA's erfcf / expf of the same
    tail; device pointers to n floats each."""
    _check(lib().dsc_probe_tail(int(profile), y_ptr, int(n), ours_ptr, cuda_ptr, stream))


def dsc_get_refine_counts(res) -> tuple:
    """(pairs re-evaluated in FP64 near a threshold, near a row maximum,
    near-threshold pairs past the list's capacity, decided in FP32)."""
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().dsc_get_refine_counts(res, C.byref(a), C.byref(b), C.byref(c)))
    return int(a.value), int(b.value), int(c.value)


def dsc_get_tile_counts(res) -> tuple:
    """(compaction tiles of the launch, tiles whose values the count pass
    read; the others took the evaluation's own count)."""
    a, b = C.c_int64(), C.c_int64()
    _check(lib().dsc_get_tile_counts(res, C.byref(a), C.byref(b)))
    return int(a.value), int(b.value)


def dsc_get_server_timing(res) -> tuple:
    """(slot, device start ms, device end ms) of a served result's launch,
    times after the server's creation."""
    slot, a, b = C.c_int32(), C.c_double(), C.c_double()
    _check(lib().dsc_get_server_timing(res, C.byref(slot), C.byref(a), C.byref(b)))
    return int(slot.value), float(a.value), float(b.value)


def dsc_result_wait(res):
    _check(lib().dsc_result_wait(res))


def dsc_get_csr(res, copy_to_host: bool = False) -> CsrView:
    v = CsrView()
    _check(lib().dsc_get_csr(res, int(bool(copy_to_host)), C.byref(v)))
    return v


def _host_ptr(a):
    if a is None:
        return None
    return a if isinstance(a, int) else (a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())


def dsc_copy_csr_to_host(res, row_ptr, col, val, beam_scale=None, stream=0):
    """Arguments are host buffers (numpy arrays or pinned torch tensors: pass data pointers as ints)."""
    _check(lib().dsc_copy_csr_to_host(res, _host_ptr(row_ptr), _host_ptr(col), _host_ptr(val), _host_ptr(beam_scale),
                                      stream))


def dsc_copy_csr_to_host_async(res, row_ptr, col, val, beam_scale=None, stream=0):
    """The copies queued on `stream` (returns before they run); buffers as for dsc_copy_csr_to_host."""
    _check(lib().dsc_copy_csr_to_host_async(res, _host_ptr(row_ptr), _host_ptr(col), _host_ptr(val),
                                            _host_ptr(beam_scale), stream))


def dsc_release_result(res):
    lib().dsc_release_result(res)


def dsc_get_beamlets(res, nrows: int) -> np.ndarray:
    out = np.zeros((max(nrows, 1), 16), dtype=np.float64)
    _check(lib().dsc_get_beamlets(res, out.ctypes.data, nrows))
    return out[:nrows]


def dsc_get_depth_tables(res, nrows: int) -> np.ndarray:
    n_max = C.c_int32()
    _check(lib().dsc_get_depth_tables(res, None, 0, C.byref(n_max)))
    out = np.zeros((nrows, n_max.value), dtype=np.float32)
    _check(lib().dsc_get_depth_tables(res, out.ctypes.data, out.size, C.byref(n_max)))
    return out


def dsc_get_row_stats(res, nrows: int):
    rm = np.zeros(max(nrows, 1), dtype=np.float32)
    rc = np.zeros(max(nrows, 1), dtype=np.int64)
    _check(lib().dsc_get_row_stats(res, rm.ctypes.data, rc.ctypes.data))
    return rm[:nrows], rc[:nrows]


def dsc_get_stage_times(res) -> dict:
    ms = np.zeros(8, dtype=np.float32)
    _check(lib().dsc_get_stage_times(res, ms.ctypes.data, 8))
    return dict(zip(STAGES, ms.tolist()))


def dsc_server_create(hbm_budget_bytes: int, max_inflight: int = 2, max_batch: int = 8):
    out = C.c_void_p()
    _check(lib().dsc_server_create(int(hbm_budget_bytes), int(max_inflight), int(max_batch), C.byref(out)))
    return out.value


def dsc_server_submit(srv, geom, beams, opts: ComputeOpts) -> int:
    arr = (BeamDesc * len(beams))(*[beam_desc(b) for b in beams])
    rid = C.c_uint64()
    _check(lib().dsc_server_submit(srv, geom, arr, len(beams), C.byref(opts), C.byref(rid)))
    return rid.value


def dsc_server_poll(srv, req_id: int, wait_ms: int = -1):
    """Returns the result handle, or None if not finished within wait_ms."""
    out = C.c_void_p()
    st = lib().dsc_server_poll(srv, int(req_id), int(wait_ms), C.byref(out))
    if st == DSC_E_BUSY:
        return None
    _check(st)
    return out.value


def dsc_server_stats(srv):
    p50, p99 = C.c_double(), C.c_double()
    n, pairs = C.c_int64(), C.c_int64()
    _check(lib().dsc_server_stats(srv, C.byref(p50), C.byref(p99), C.byref(n), C.byref(pairs)))
    return {"p50_ms": p50.value, "p99_ms": p99.value, "n_done": n.value, "pairs_done": pairs.value}


def dsc_server_destroy(srv):
    lib().dsc_server_destroy(srv)


def dsc_compute_dij_noalloc(grid, density_ptr: int, model, beams, opts: ComputeOpts, row_ptr_ptr: int, col_ptr: int,
                            val_ptr: int, capacity: int, stream=0, inexact: list = None) -> int:
    """D_ij into caller-allocated device buffers, no allocation by the library.
    Returns the number of kept entries.  DSC_W_INEXACT (complete, but some
    decisions near the threshold were taken in FP32) is not raised: it is
    appended to `inexact` when a list is given."""
    g = grid_desc(grid)
    mr = _ModelRef(model)
    arr = (BeamDesc * len(beams))(*[beam_desc(b) for b in beams])
    nnz = C.c_int64()
    st = lib().dsc_compute_dij_noalloc(C.byref(g), int(density_ptr), C.byref(mr.s), arr, len(beams), C.byref(opts),
                                       int(row_ptr_ptr), int(col_ptr), int(val_ptr), int(capacity), C.byref(nnz),
                                       stream)
    if st == DSC_W_INEXACT:
        if inexact is not None:
            inexact.append(lib().dsc_last_error().decode(errors="replace"))
        st = DSC_OK
    _check(st)
    return nnz.value


# ---------------------------------------------------------------------------
# conveniences on top of the entry points
# ---------------------------------------------------------------------------
class HostCSR:
    """A result's CSR copied to host numpy arrays (values as float32)."""

    def __init__(self, res):
        v = dsc_get_csr(res, False)
        self.nrows, self.ncols, self.nnz, self.pairs = int(v.nrows), int(v.ncols), int(v.nnz), int(v.pairs)
        self.value_dtype = int(v.value_dtype)
        self.row_ptr = np.zeros(self.nrows + 1, dtype=np.int64)
        self.col = np.zeros(max(self.nnz, 1), dtype=np.int32)
        raw = np.zeros(max(self.nnz, 1), dtype=np.uint16 if self.value_dtype == DSC_VALUE_BF16 else np.float32)
        self.beam_scale = np.zeros(max(int(v.nbeams), 1), dtype=np.float32)
        dsc_copy_csr_to_host(res, self.row_ptr, self.col, raw, self.beam_scale)
        self.col = self.col[:self.nnz]
        raw = raw[:self.nnz]
        if self.value_dtype == DSC_VALUE_BF16:
            self.raw = raw
            self.val = (raw.astype(np.uint32) << 16).view(np.float32)
        else:
            self.val = raw

    def row(self, r):
        a, b = self.row_ptr[r], self.row_ptr[r + 1]
        return self.col[a:b], self.val[a:b]


def geometry_from_workload(w, stream=0):
    g = dsc_create_geometry(w.grid, w.density, False, w.model, stream)
    for b in w.beams:
        dsc_add_beam(g, b)
    return g


def compute_workload(w, stream=0, flags=0, value_dtype=None):
    """One-shot: geometry, D_ij, host CSR.  Returns (HostCSR, result handle, geometry handle)."""
    g = geometry_from_workload(w, stream)
    dt = w.value_dtype if value_dtype is None else value_dtype
    if getattr(w, "table_mode", 0) == 1:
        flags |= DSC_FLAG_TRILINEAR_TABLE
    res = dsc_compute_dij(g, compute_opts(w.tau, dt, w.h_frac, flags), stream)
    return HostCSR(res), res, g

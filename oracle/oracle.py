"""ctypes front end of the FP64 C oracle (``dsc_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm use this module.  It never imports
the CUDA package; inputs arrive as plain descriptors (any object with the
attributes of the phantom dataclasses) and numpy arrays.

``build()`` compiles the oracle with gcc (-O2, no fast-math, OpenMP) into
``oracle/_build/``.  Everything the oracle computes is double precision;
the FP32 density and beam-model table are promoted, not re-rounded.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsc_oracle.c")
_OUT = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class OrBeam(C.Structure):
    _fields_ = [("gantry_deg", C.c_double), ("sad", C.c_double), ("iso", C.c_double * 3),
                ("a", C.c_double), ("b", C.c_double), ("n_u", C.c_int), ("n_v", C.c_int)]


class OrModel(C.Structure):
    _fields_ = [("n", C.c_int), ("d_max", C.c_double), ("lut", C.c_void_p),
                ("c1", C.c_double * 3), ("c2", C.c_double * 3),
                ("cutoff_mode", C.c_int), ("cutoff_k", C.c_double), ("profile", C.c_int)]


class OrResult(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double)), ("row_max", C.POINTER(C.c_double)),
                ("row_cand", C.POINTER(C.c_int64)), ("n_amb", C.c_int64),
                ("amb_row", C.POINTER(C.c_int64)), ("amb_col", C.POINTER(C.c_int32)),
                ("amb_kind", C.POINTER(C.c_int32))]


def build(force: bool = False) -> str:
    """Compile liboracle.so if it is missing or older than its source."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.or_compute.restype = C.c_int
        L.or_compute.argtypes = [C.POINTER(OrGrid), C.c_void_p, C.POINTER(OrModel), C.POINTER(OrBeam), C.c_int,
                                 C.c_double, C.c_double, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                                 C.POINTER(OrResult)]
        L.or_free_result.argtypes = [C.POINTER(OrResult)]
        L.or_beamlets.argtypes = [C.POINTER(OrGrid), C.POINTER(OrBeam), C.c_int, C.c_double, C.c_void_p]
        L.or_row_table.restype = C.c_int
        L.or_row_table.argtypes = [C.POINTER(OrGrid), C.c_void_p, C.POINTER(OrBeam), C.c_int, C.c_int,
                                   C.c_double, C.c_int, C.c_void_p, C.c_int]
        L.or_trilinear.restype = C.c_double
        L.or_trilinear.argtypes = [C.POINTER(OrGrid), C.c_void_p, C.c_void_p]
        L.or_depth_interp.restype = C.c_double
        L.or_depth_interp.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
        L.or_lut_eval.argtypes = [C.POINTER(OrModel), C.c_double, C.c_void_p]
        L.or_profile_F.restype = C.c_double
        L.or_profile_F.argtypes = [C.POINTER(OrModel), C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_point_dose.restype = C.c_double
        L.or_point_dose.argtypes = [C.POINTER(OrModel), C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_double]
        L.or_max_threads.restype = C.c_int
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling
# ---------------------------------------------------------------------------
def _grid(g) -> OrGrid:
    return OrGrid(int(g.nx), int(g.ny), int(g.nz), float(g.dx), float(g.dy), float(g.dz),
                  float(g.origin[0]), float(g.origin[1]), float(g.origin[2]))


def _beams(beams):
    arr = (OrBeam * max(1, len(beams)))()
    for i, b in enumerate(beams):
        arr[i] = OrBeam(float(b.gantry_deg), float(b.sad), (C.c_double * 3)(*[float(v) for v in b.iso]),
                        float(b.a), float(b.b), int(b.n_u), int(b.n_v))
    return arr


class _ModelRef:
    """Keeps the LUT array alive while the C struct points at it."""

    def __init__(self, m):
        self.lut = np.ascontiguousarray(m.lut, dtype=np.float32)
        self.s = OrModel(int(self.lut.shape[0]), float(m.d_max), self.lut.ctypes.data,
                         (C.c_double * 3)(*[float(v) for v in m.c1]),
                         (C.c_double * 3)(*[float(v) for v in m.c2]),
                         int(m.cutoff_mode), float(m.cutoff_k), int(getattr(m, "profile", 0)))


class OracleCSR:
    """Oracle output over the requested rows, as numpy arrays."""

    def __init__(self, r: OrResult, rows):
        n, nnz, na = int(r.nrows), int(r.nnz), int(r.n_amb)
        self.rows = rows
        self.row_ptr = np.ctypeslib.as_array(r.row_ptr, (n + 1,)).copy()
        self.col = np.ctypeslib.as_array(r.col, (max(nnz, 1),))[:nnz].copy()
        self.val = np.ctypeslib.as_array(r.val, (max(nnz, 1),))[:nnz].copy()
        self.row_max = np.ctypeslib.as_array(r.row_max, (max(n, 1),))[:n].copy()
        self.row_cand = np.ctypeslib.as_array(r.row_cand, (max(n, 1),))[:n].copy()
        self.amb_row = np.ctypeslib.as_array(r.amb_row, (max(na, 1),))[:na].copy()
        self.amb_col = np.ctypeslib.as_array(r.amb_col, (max(na, 1),))[:na].copy()
        self.amb_kind = np.ctypeslib.as_array(r.amb_kind, (max(na, 1),))[:na].copy()

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def pairs(self) -> int:
        return int(self.row_cand.sum())

    def row(self, r):
        a, b = self.row_ptr[r], self.row_ptr[r + 1]
        return self.col[a:b], self.val[a:b]

    def ambiguous(self, r):
        m = self.amb_row == r
        return set(self.amb_col[m].tolist())


def compute(grid, density, model, beams, tau=1e-3, h_frac=0.5, rows=None, nthreads=0, full_scan=False,
            table_mode=0):
    """D_ij over ``rows`` (global row indices) or every row.  table_mode 0:
    depth table = exact integral (Siddon); 1: trilinear samples, trapezoid."""
    L = lib()
    g = _grid(grid)
    mr = _ModelRef(model)
    ba = _beams(beams)
    rho = np.ascontiguousarray(density, dtype=np.float32)
    assert rho.shape == (grid.nz, grid.ny, grid.nx)
    res = OrResult()
    if rows is None:
        rp, nsel = None, 0
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        rp, nsel = rows.ctypes.data, int(rows.size)
    rc = L.or_compute(C.byref(g), rho.ctypes.data, C.byref(mr.s), ba, len(beams), float(tau), float(h_frac),
                      rp, nsel, int(nthreads), int(bool(full_scan)), int(table_mode), C.byref(res))
    if rc != 0:
        raise ValueError("oracle: bad row index")
    try:
        return OracleCSR(res, rows)
    finally:
        L.or_free_result(C.byref(res))


def compute_workload(w, rows=None, nthreads=0, full_scan=False):
    return compute(w.grid, w.density, w.model, w.beams, tau=w.tau, h_frac=w.h_frac, rows=rows,
                   nthreads=nthreads, full_scan=full_scan, table_mode=getattr(w, "table_mode", 0))


def _sparse(orc: "OracleCSR", nvox: int):
    import scipy.sparse
    return scipy.sparse.csr_matrix((orc.val, orc.col, orc.row_ptr), shape=(len(orc.row_ptr) - 1, int(nvox)))


def dose(orc: "OracleCSR", w, nvox: int) -> np.ndarray:
    """Eq. 1: the dose at every voxel, sum over the rows j of w_j D_j(voxel),
    in FP64 (a sparse matrix-vector product of the oracle's own D_ij)."""
    return _sparse(orc, nvox).T @ np.asarray(w, dtype=np.float64)


def beamlet_dot(orc: "OracleCSR", g, nvox: int) -> np.ndarray:
    """Per row j: sum over voxels of D_j(voxel) g(voxel), the product with
    the transpose of Eq. 1's operator (an optimiser's gradient), in FP64."""
    return _sparse(orc, nvox) @ np.asarray(g, dtype=np.float64)


def beamlets(grid, beams, h_frac=0.5) -> np.ndarray:
    """Per row: S[3] e[3] x[3] z[3] tA tB theta hit n_table h a b (20 doubles)."""
    n = sum(b.n_u * b.n_v for b in beams)
    out = np.zeros((max(n, 1), 20), dtype=np.float64)
    lib().or_beamlets(C.byref(_grid(grid)), _beams(beams), len(beams), float(h_frac), out.ctypes.data)
    return out[:n]


def row_table(grid, density, beam, iu, iv, h_frac=0.5, table_mode=0) -> np.ndarray:
    rho = np.ascontiguousarray(density, dtype=np.float32)
    cap = 1 << 16
    out = np.zeros(cap, dtype=np.float64)
    n = lib().or_row_table(C.byref(_grid(grid)), rho.ctypes.data, C.byref(_beams([beam])[0]), int(iu), int(iv),
                           float(h_frac), int(table_mode), out.ctypes.data, cap)
    if n < 0:
        raise ValueError("table too long")
    return out[:n].copy()


def trilinear(grid, density, p) -> float:
    """Density at point p (mm) by trilinear interpolation of the voxel centres."""
    rho = np.ascontiguousarray(density, dtype=np.float32)
    q = np.ascontiguousarray(p, dtype=np.float64)
    return float(lib().or_trilinear(C.byref(_grid(grid)), rho.ctypes.data, q.ctypes.data))


def depth_interp(table, h, s) -> float:
    t = np.ascontiguousarray(table, dtype=np.float64)
    return float(lib().or_depth_interp(t.ctypes.data, int(t.size), float(h), float(s)))


def lut_eval(model, d) -> np.ndarray:
    mr = _ModelRef(model)
    out = np.zeros(4, dtype=np.float64)
    lib().or_lut_eval(C.byref(mr.s), float(d), out.ctypes.data)
    return out


def profile_F(model, c3, xp, zp, a_t, b_t) -> float:
    mr = _ModelRef(model)
    c = np.ascontiguousarray(c3, dtype=np.float64)
    return float(lib().or_profile_F(C.byref(mr.s), c.ctypes.data, float(xp), float(zp), float(a_t), float(b_t)))


def point_dose(model, xp, zp, t, d, sad, a, b) -> float:
    mr = _ModelRef(model)
    return float(lib().or_point_dose(C.byref(mr.s), float(xp), float(zp), float(t), float(d), float(sad),
                                     float(a), float(b)))


def max_threads() -> int:
    return int(lib().or_max_threads())

"""The x-line enumeration of the candidate count and the evaluation, checked on
the CPU against the oracle.

A beamlet row's candidates (Section 2.1: the voxels inside its VOI) lie on
x-lines (iy, iz) of a voxel box around the VOI.  For each z-slice of the box
the library keeps only the lines whose centre y lies in the y-extent of the
VOI's cross-section at that height (a convex polygon: the four lateral
half-planes cut to the box's voxel-centre range), widened by a margin, and
computes the extent in FP32 from the polygon's feasible vertices.  This
replays that arithmetic in numpy's IEEE FP32 and checks, for rows of the
workloads' beams (the 3-sigma cutoff, the 6-beamlet-width VOI, gantry 0 and
oblique), that every line holding one of the oracle's candidates is
enumerated, and that the enumeration leaves out the empty lines of oblique
beams' boxes."""
import numpy as np
import pytest

from paper_0908_4417_gb300 import phantoms as P
from oracle import oracle as O

F = np.float32
MARGIN = F(0.02)      # mm, as in the kernel


def row_frames(w):
    """Per row: S, e, x, z, hit (the oracle's beamlet set-up) and its beam."""
    b = O.beamlets(w.grid, w.beams, w.h_frac)
    beam_of = np.concatenate([np.full(B.n_u * B.n_v, k) for k, B in enumerate(w.beams)])
    return b, beam_of


def voxel_box(g, S, e, x, z, kx, kz, bx, bz):
    """The voxel box of the set-up: the hull of the VOI's end rectangles at the
    smallest and largest t of the grid's corners, one voxel of slack (FP64)."""
    blo = np.array(g.origin, float)
    bhi = blo + np.array([g.nx * g.dx, g.ny * g.dy, g.nz * g.dz])
    corners = np.array([[bhi[0] if c & 1 else blo[0], bhi[1] if c & 2 else blo[1], bhi[2] if c & 4 else blo[2]]
                        for c in range(8)])
    ts = (corners - S) @ e
    tlo, thi = max(ts.min(), 0.0), ts.max()
    pts = []
    for c in range(8):
        t = thi if c & 1 else tlo
        hx, hz = kx * t + bx, kz * t + bz
        pts.append(S + t * e + (hx if c & 2 else -hx) * x + (hz if c & 4 else -hz) * z)
    lo3, hi3 = np.min(pts, 0), np.max(pts, 0)
    d = (g.dx, g.dy, g.dz)
    n = (g.nx, g.ny, g.nz)
    box = []
    for k in range(3):
        a = max(0, int(np.floor((lo3[k] - blo[k]) / d[k] - 0.5)) - 1)
        b = min(n[k] - 1, int(np.ceil((hi3[k] - blo[k]) / d[k] - 0.5)) + 1)
        box.append((a, b))
    return box


def slice_lines(g, S, e, x, z, kx, kz, bx, bz, box):
    """{iz: (iy_lo, count)} as the kernel forms them, in FP32."""
    (ix0, ix1), (iy0, iy1), (iz0, iz1) = box
    A, B, C0, Cz = [], [], [], []
    for k in range(4):
        sg = F(-1.0) if k & 1 else F(1.0)
        kk = F(kx) if k < 2 else F(kz)
        u = x if k < 2 else z
        a = [sg * F(u[i]) - kk * F(e[i]) for i in range(3)]
        A.append(a[0])
        B.append(a[1])
        C0.append(F(bx if k < 2 else bz) + a[0] * F(S[0]) + a[1] * F(S[1]) + a[2] * F(S[2]))
        Cz.append(a[2])
    xc0 = F(g.origin[0] + (ix0 + 0.5) * g.dx)
    xc1 = F(g.origin[0] + (ix1 + 0.5) * g.dx)
    yc0 = F(g.origin[1] + (iy0 + 0.5) * g.dy)
    yc1 = F(g.origin[1] + (iy1 + 0.5) * g.dy)
    A += [F(-1), F(1), F(0), F(0)]
    B += [F(0), F(0), F(-1), F(1)]
    C0 += [-xc0, xc1, -yc0, yc1]
    Cz += [F(0)] * 4
    dyi, oyh = F(1) / F(g.dy), F(g.origin[1]) + F(0.5) * F(g.dy)
    out = {}
    for iz in range(iz0, iz1 + 1):
        zc = (F(iz) + F(0.5)) * F(g.dz) + F(g.origin[2])
        C = [C0[k] - Cz[k] * zc for k in range(8)]
        ys = []
        for i in range(8):
            for j in range(i + 1, 8):
                det = A[i] * B[j] - A[j] * B[i]
                if abs(det) < F(1e-9):
                    continue
                idet = F(1) / det
                px = (C[i] * B[j] - C[j] * B[i]) * idet
                py = (A[i] * C[j] - A[j] * C[i]) * idet
                if all(A[k] * px + B[k] * py <= C[k] + MARGIN for k in range(8)):
                    ys.append(py)
        if not ys:
            out[iz] = (iy0, 0)
            continue
        a0 = int(np.ceil((min(ys) - MARGIN - oyh) * dyi))
        a1 = int(np.floor((max(ys) + MARGIN - oyh) * dyi))
        lo = max(a0, iy0)
        out[iz] = (lo, max(0, min(a1, iy1) - lo + 1))
    return out


def check_rows(w, rows):
    """Every line holding an oracle candidate is enumerated; returns the
    enumerated and the box's line counts."""
    g, m = w.grid, w.model
    b, beam_of = row_frames(w)
    orc = O.compute(g, w.density, m, w.beams, tau=0.0, h_frac=w.h_frac, rows=rows)
    c3max = float(np.max(m.lut[:, 1]))
    kept = box_lines = 0
    for k, r in enumerate(rows):
        S, e, x, z = b[r, 0:3], b[r, 3:6], b[r, 6:9], b[r, 9:12]
        B = w.beams[beam_of[r]]
        if m.cutoff_mode == P.CUTOFF_SIGMA:
            kx, kz, bx, bz = 0.5 * B.a / B.sad, 0.5 * B.b / B.sad, m.cutoff_k * c3max, m.cutoff_k * c3max
        else:
            kx, kz, bx, bz = 3.0 * B.a / B.sad, 3.0 * B.b / B.sad, 0.0, 0.0
        box = voxel_box(g, S, e, x, z, kx, kz, bx, bz)
        sl = slice_lines(g, S, e, x, z, kx, kz, bx, bz, box)
        cols = orc.row(k)[0]
        assert cols.size > 0, r
        iz, rem = np.divmod(cols, g.nx * g.ny)
        iy = rem // g.nx
        for yy, zz in set(zip(iy.tolist(), iz.tolist())):
            assert zz in sl, (r, yy, zz)
            lo, n = sl[zz]
            assert lo <= yy < lo + n, (r, yy, zz, lo, n)
        kept += sum(n for _, n in sl.values())
        box_lines += (box[1][1] - box[1][0] + 1) * (box[2][1] - box[2][0] + 1)
    return kept, box_lines


def test_lines_of_the_sigma_cutoff_at_gantry_0():
    w = P.water_32()
    check_rows(w, [0, 19, 190, 210, 399])


def test_lines_of_the_voi_on_the_slab_phantom():
    w = P.slabs_128(value_dtype=P.VALUE_F32)
    check_rows(w, [0, 39, 780, 820, 1599])


@pytest.mark.parametrize("field", [1, 2, 4])
def test_oblique_fields_drop_empty_lines(field):
    """Rows of the 40, 80 and 160 degree prostate fields: no candidate line is
    lost, and at least a third of the box's lines are left out."""
    w = P.prostate_256()
    base = sum(B.n_u * B.n_v for B in w.beams[:field])
    n = w.beams[field].n_u * w.beams[field].n_v
    kept, box_lines = check_rows(w, [base, base + n // 2, base + n - 1])
    assert kept <= 0.67 * box_lines, (kept, box_lines)

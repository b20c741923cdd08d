"""Pins of the FP64 oracle to facts fixed outside it (closed forms, invariants,
brute force, the paper's printed VOI counts).  CPU only.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a misplaced beamlet) breaks at
least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_4417_gb300 import phantoms as P

HERE = os.path.dirname(os.path.abspath(__file__))


def rows_of(beam):
    """(row, iu, iv) in the engine's row order: iv major, iu minor."""
    return [(iv * beam.n_u + iu, iu, iv) for iv in range(beam.n_v) for iu in range(beam.n_u)]


def dense(csr, nrows, nvox):
    M = np.zeros((nrows, nvox))
    for r in range(nrows):
        c, v = csr.row(r)
        M[r, c] = v
    return M


# ---------------------------------------------------------------------------
# entry / exit points (Fig. 1: A and B on the encasing prism)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gantry", [0.0, 33.0, 90.0, 137.5, 251.0])
def test_entry_exit_on_prism(gantry):
    g = P.centred_grid(24, 20, 16, 3.0, 2.5, 4.0)
    beam = P.Beam(gantry, 400.0, (3.0, -2.0, 1.0), 6.0, 5.0, 5, 4)
    bl = O.beamlets(g, [beam])
    lo = np.array(g.origin)
    hi = lo + np.array([g.nx * g.dx, g.ny * g.dy, g.nz * g.dz])
    for r in range(bl.shape[0]):
        S, e = bl[r, 0:3], bl[r, 3:6]
        assert abs(np.linalg.norm(e) - 1) < 1e-14
        assert bl[r, 15] == 1
        for t in (bl[r, 12], bl[r, 13]):
            p = S + t * e
            assert np.all(p >= lo - 1e-9) and np.all(p <= hi + 1e-9)
            assert np.min(np.minimum(np.abs(p - lo), np.abs(p - hi))) < 1e-9   # on a face
        # just outside A and B the axis is outside the prism
        for t in (bl[r, 12] - 1e-6, bl[r, 13] + 1e-6):
            p = S + t * e
            assert np.any(p < lo) or np.any(p > hi)


def test_beamlet_axes_tile_isocentre_plane():
    """Beamlet axes cross the isocentre plane on a regular a x b lattice centred at I,
    with rows ordered iv-major; x', z' are orthonormal and perpendicular to the axis."""
    g = P.centred_grid(16, 16, 16, 4.0, 4.0, 4.0)
    for gantry in (0.0, 57.0, 212.0):
        beam = P.Beam(gantry, 800.0, (1.0, 2.0, -3.0), 7.0, 3.0, 6, 5)
        bl = O.beamlets(g, [beam])
        gr = math.radians(gantry)
        E = np.array([-math.sin(gr), math.cos(gr), 0.0])   # broad-beam axis, pointing away from S
        u = np.array([math.cos(gr), math.sin(gr), 0.0])
        I = np.array(beam.iso)
        for r, iu, iv in rows_of(beam):
            S, e, x, z = bl[r, 0:3], bl[r, 3:6], bl[r, 6:9], bl[r, 9:12]
            assert np.allclose(I - S, beam.sad * E, atol=1e-9)
            t = np.dot(I - S, E) / np.dot(e, E)
            q = S + t * e - I                              # crossing of the iso plane
            assert abs(np.dot(q, E)) < 1e-9
            assert abs(np.dot(q, u) - (iu - (beam.n_u - 1) / 2) * beam.a) < 1e-9
            assert abs(q[2] - (iv - (beam.n_v - 1) / 2) * beam.b) < 1e-9
            for v in (x, z):
                assert abs(np.linalg.norm(v) - 1) < 1e-13 and abs(np.dot(v, e)) < 1e-13
            assert abs(np.dot(x, z)) < 1e-13
            assert np.dot(x, u) > 0 and z[2] > 0           # x' along +u, z' along +v
            assert abs(math.cos(bl[r, 14]) - np.dot(e, E)) < 1e-12


# ---------------------------------------------------------------------------
# radiological depth: closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gantry", [0.0, 33.0, 90.0, 137.5, 251.0])
@pytest.mark.parametrize("rho0", [1.0, 0.37])
def test_uniform_density_depth_is_scaled_geometric(gantry, rho0):
    g = P.centred_grid(24, 20, 16, 3.0, 2.5, 4.0)
    rho = np.full(g.shape, rho0, np.float32)
    beam = P.Beam(gantry, 400.0, (3.0, -2.0, 1.0), 6.0, 5.0, 5, 4)
    bl = O.beamlets(g, [beam])
    h = 0.5 * 2.5
    for r, iu, iv in rows_of(beam):
        tab = O.row_table(g, rho, beam, iu, iv)
        L = bl[r, 13] - bl[r, 12]
        assert tab.size == int(math.ceil(L / h)) + 1 == int(bl[r, 16])
        k = np.arange(tab.size)
        expect = float(np.float32(rho0)) * np.minimum(k * h, L)
        assert np.allclose(tab, expect, rtol=0, atol=1e-10)


def test_slab_phantom_depth_closed_form():
    """Lung 0.25 at [40,80) mm and bone 1.8 at [100,120) mm depth from the entry face:
    along a ray with cos(phi) = e_y entering through y_min, d(s) = G(s cos phi)/cos phi,
    G(l) = l - 0.75 |[0,l] & [40,80]| + 0.8 |[0,l] & [100,120]|."""
    w = P.slabs_128()
    g, beam = w.grid, w.beams[0]
    bl = O.beamlets(g, [beam])

    def overlap(l, a, b):
        return np.clip(np.minimum(l, b) - a, 0.0, None)

    lung, bone = float(np.float32(0.25)), float(np.float32(1.8))   # the stored FP32 densities

    def G(l):
        return l - (1 - lung) * overlap(l, 40.0, 80.0) + (bone - 1) * overlap(l, 100.0, 120.0)

    h = 0.5 * g.dx
    for r, iu, iv in rows_of(beam)[::37]:
        S, e, tA = bl[r, 0:3], bl[r, 3:6], bl[r, 12]
        assert abs((S + tA * e)[1] - g.origin[1]) < 1e-9
        tab = O.row_table(g, w.density, beam, iu, iv)
        L = bl[r, 13] - tA
        s = np.minimum(np.arange(tab.size) * h, L)
        expect = G(s * e[1]) / e[1]
        assert np.allclose(tab, expect, rtol=0, atol=1e-9), np.abs(tab - expect).max()


def test_axis_aligned_ray_sums_voxel_row():
    rho = P.random_grid_density(7, (6, 7, 5))
    g = P.Grid(5, 7, 6, 1.5, 2.0, 1.25, (-3.75, -7.0, -3.75))
    x_c = g.origin[0] + 2.5 * g.dx
    z_c = g.origin[2] + 3.5 * g.dz
    beam = P.Beam(0.0, 50.0, (x_c, 0.0, z_c), 1.0, 1.0, 1, 1)
    tab = O.row_table(g, rho, beam, 0, 0)
    assert abs(tab[-1] - g.dy * rho[3, :, 2].astype(np.float64).sum()) < 1e-12


# ---------------------------------------------------------------------------
# radiological depth: brute-force ray marching on tiny random grids
# ---------------------------------------------------------------------------
def march(g, rho, S, e, t_points, delta):
    """Midpoint-rule integral of density from the source to each t (density 0 outside)."""
    tmax = float(np.max(t_points))
    M = int(math.ceil(tmax / delta)) + 1
    u = (np.arange(M) + 0.5) * delta
    p = S[None, :] + u[:, None] * e[None, :]
    idx = np.floor((p - np.array(g.origin)) / np.array([g.dx, g.dy, g.dz])).astype(np.int64)
    inside = np.all((idx >= 0) & (idx < np.array([g.nx, g.ny, g.nz])), axis=1)
    vals = np.zeros(M)
    ii = idx[inside]
    vals[inside] = rho[ii[:, 2], ii[:, 1], ii[:, 0]]
    cum = np.concatenate([[0.0], np.cumsum(vals) * delta])
    m = np.floor(np.asarray(t_points) / delta).astype(np.int64)
    return cum[m] + (np.asarray(t_points) - m * delta) * vals[np.minimum(m, M - 1)]


def brute_cases():
    cases = []
    for seed in range(6):
        r = P._Draw(1000 + seed)
        n = [2 + r.randint(0, 6) for _ in range(3)]
        sp = [0.5 + 1.5 * r.u() for _ in range(3)]
        g = P.centred_grid(n[0], n[1], n[2], sp[0], sp[1], sp[2], centre=(r.u() - 0.5, r.u() - 0.5, r.u() - 0.5))
        iso = tuple(g.centre()[k] + (r.u() - 0.5) * 0.5 * [n[0] * sp[0], n[1] * sp[1], n[2] * sp[2]][k]
                    for k in range(3))
        diag = math.sqrt(sum((n[k] * sp[k]) ** 2 for k in range(3)))
        beam = P.Beam(360.0 * r.u(), diag + 2.0 + 10.0 * r.u(), iso, 0.5 + 4 * r.u(), 0.5 + 4 * r.u(),
                      1 + r.randint(0, 3), 1 + r.randint(0, 3))
        cases.append((g, P.random_grid_density(seed, g.shape), beam))
    # rays inside a grid plane, along a grid line (voxel edges) and through corners
    g = P.Grid(4, 5, 3, 1.0, 1.0, 1.0, (-2.0, -2.5, -1.5))
    rho = P.random_grid_density(99, g.shape)
    cases.append((g, rho, P.Beam(0.0, 20.0, (0.0, 0.0, 0.3), 1.0, 1.0, 1, 1)))      # in plane x = 0
    cases.append((g, rho, P.Beam(0.0, 20.0, (0.0, 0.0, 0.5), 1.0, 1.0, 1, 1)))      # on edge x=0, z=0.5
    cases.append((g, rho, P.Beam(45.0, 20.0, (0.0, 0.5, 0.5), 1.0, 1.0, 1, 1)))     # diagonal through corners
    cases.append((g, rho, P.Beam(90.0, 20.0, (0.3, 0.5, -0.5), 1.0, 1.0, 1, 1)))    # along x on a y-z edge
    return cases


@pytest.mark.parametrize("case", range(10))
def test_siddon_matches_brute_force_march(case):
    g, rho, beam = brute_cases()[case]
    bl = O.beamlets(g, [beam])
    delta = 2e-5
    rmax = float(rho.max())
    for r, iu, iv in rows_of(beam):
        if not bl[r, 15]:
            continue
        S, e, tA, tB, h = bl[r, 0:3], bl[r, 3:6], bl[r, 12], bl[r, 13], bl[r, 17]
        tab = O.row_table(g, rho, beam, iu, iv)
        tk = tA + np.minimum(np.arange(tab.size) * h, tB - tA)
        ref = march(g, rho.astype(np.float64), S, e, tk, delta)
        crossings = sum(abs(e[k]) * (tB - tA) / [g.dx, g.dy, g.dz][k] + 2 for k in range(3))
        bound = (crossings + 2) * delta * rmax
        assert np.abs(tab - ref).max() <= bound, (np.abs(tab - ref).max(), bound)


# ---------------------------------------------------------------------------
# interpolation (depth table and beam-model LUT)
# ---------------------------------------------------------------------------
def test_interpolation_nodes_and_midpoints():
    m = P.synthetic_model()
    n = m.lut.shape[0]
    for k in (0, 1, 7, 128, n - 2, n - 1):
        d = k * m.d_max / (n - 1)
        assert np.allclose(O.lut_eval(m, d), m.lut[k].astype(np.float64), rtol=1e-14, atol=0)
    for k in (0, 17, n - 2):
        d = (k + 0.5) * m.d_max / (n - 1)
        mid = 0.5 * (m.lut[k].astype(np.float64) + m.lut[k + 1].astype(np.float64))
        assert np.allclose(O.lut_eval(m, d), mid, rtol=1e-13)
    assert np.array_equal(O.lut_eval(m, 2 * m.d_max), m.lut[-1].astype(np.float64))
    tab = np.array([0.0, 1.0, 3.0, 3.5])
    assert O.depth_interp(tab, 2.0, 4.0) == 3.0
    assert O.depth_interp(tab, 2.0, 3.0) == 2.0
    assert O.depth_interp(tab, 2.0, -1.0) == 0.0
    assert O.depth_interp(tab, 2.0, 100.0) == 3.5


# ---------------------------------------------------------------------------
# Eq. 3: lateral integral and erf tiling (normalisation / self-consistency)
# ---------------------------------------------------------------------------
def test_profile_integral_closed_form():
    """Each erf pair integrates to 2 c2 a_t, so the double integral of F over the
    plane is sum_i c1_i c2_i^2 a_t b_t."""
    m = P.synthetic_model(c1=(0.7, 0.2, 0.1), c2=(0.9, 1.1, 1.3))
    c3 = np.array([1.7, 4.3, 9.1])
    a_t, b_t = 5.3, 3.1
    R = 12 * c3.max() + 2 * max(a_t, b_t)
    n = 401
    xs = np.linspace(-R, R, n)
    wts = np.ones(n)
    wts[1:-1:2], wts[2:-1:2] = 4.0, 2.0
    wts *= (xs[1] - xs[0]) / 3.0
    F = np.array([[O.profile_F(m, c3, x, z, a_t, b_t) for x in xs] for z in xs])
    integral = wts @ F @ wts
    expect = sum(m.c1[i] * m.c2[i] ** 2 for i in range(3)) * a_t * b_t
    assert abs(integral / expect - 1) < 1e-6, integral / expect


@pytest.mark.parametrize("profile", [P.PROFILE_ERF, P.PROFILE_LAPLACE, P.PROFILE_LOGISTIC])
def test_profile_is_the_erf_box_in_the_narrow_limit(profile):
    """sigma -> 0: each erf pair is 2 inside |x'| < c2 a_t/2 and 0 outside
    (every profile: the box convolved with a vanishing spread kernel)."""
    m = P.synthetic_model(c1=(0.5, 0.3, 0.2), c2=(1.0, 0.5, 0.25), profile=profile)
    c3 = np.array([1e-7, 1e-7, 1e-7])
    a_t, b_t = 8.0, 4.0
    for x, z, expect in [(0.1, 0.1, 1.0), (3.0, 0.5, 0.5), (1.5, 0.2, 0.8), (3.0, 1.2, 0.5),
                         (0.5, 1.5, 0.5), (0.5, 0.7, 0.8), (4.5, 0.0, 0.0), (0.0, 2.5, 0.0)]:
        assert abs(O.profile_F(m, c3, x, z, a_t, b_t) - expect) < 1e-12, (x, z)


@pytest.mark.parametrize("profile", [P.PROFILE_ERF, P.PROFILE_LAPLACE, P.PROFILE_LOGISTIC])
def test_beamlets_tile_a_broad_beam(profile):
    """Parallel limit, water, no cutoff, no threshold: the sum over a field of
    n_u x n_v beamlets equals the dose of one beamlet of the whole field (the
    self-consistency condition of Section 2.1, for every profile)."""
    g = P.centred_grid(16, 12, 10, 3.0, 3.0, 3.0)
    rho = np.ones(g.shape, np.float32)
    m = P.synthetic_model(cutoff_mode=P.CUTOFF_NONE, profile=profile)
    sad = 1e9
    small = P.Beam(0.0, sad, (0.0, 0.0, 0.0), 4.0, 6.0, 4, 3)
    broad = P.Beam(0.0, sad, (0.0, 0.0, 0.0), 16.0, 18.0, 1, 1)
    rs = O.compute(g, rho, m, [small], tau=0.0)
    rb = O.compute(g, rho, m, [broad], tau=0.0)
    S = dense(rs, 12, g.nvox).sum(axis=0)
    B = dense(rb, 1, g.nvox)[0]
    assert B.min() > 0
    assert np.abs(S / B - 1).max() < 1e-6


# ---------------------------------------------------------------------------
# Eq. 2: inverse square and the divergent VOI of 6x the beamlet side
# ---------------------------------------------------------------------------
def test_inverse_square_and_voi_in_vacuum():
    """Density 0 (d = 0), widths c3 -> 0: D = T(0) (SAD/t)^2 sum(c1) inside the
    divergent beamlet (|x'| < a t/2SAD, |z'| < b t/2SAD) and 0 outside; the
    candidate set is |x'| <= 3 a t/SAD, |z'| <= 3 b t/SAD (VOI of 6x the side)."""
    lut = P.synthetic_model().lut.copy()
    lut[:, 1:] = 1e-6
    m = P.Model(lut=lut, d_max=300.0, c1=(0.6, 0.3, 0.05), c2=(1, 1, 1), cutoff_mode=P.CUTOFF_VOI6)
    sad, a, b = 100.0, 8.0, 5.0
    g = P.centred_grid(40, 10, 36, 1.3, 1.3, 1.3, centre=(0.37, 0.0, 0.21))
    rho = np.zeros(g.shape, np.float32)
    beam = P.Beam(0.0, sad, (0.0, 0.0, 0.0), a, b, 1, 1)
    r = O.compute(g, rho, m, [beam], tau=0.0)
    x, y, z = g.voxel_centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    t = Y + sad
    inside = (np.abs(X) < a * t / (2 * sad)) & (np.abs(Z) < b * t / (2 * sad))
    cand = (np.abs(X) <= 3 * a * t / sad) & (np.abs(Z) <= 3 * b * t / sad)
    # no voxel centre sits within 1e-4 mm of an edge
    for lim, c in ((a / (2 * sad), X), (b / (2 * sad), Z), (3 * a / sad, X), (3 * b / sad, Z)):
        assert np.abs(np.abs(c) - lim * t).min() > 1e-4
    assert r.pairs == int(cand.sum())
    expect = (float(lut[0, 0]) * (sad / t) ** 2 * sum(m.c1)).ravel()
    cols, vals = r.row(0)
    assert np.array_equal(np.sort(cols), np.flatnonzero(inside.ravel()))
    assert np.allclose(vals, expect[cols], rtol=1e-12)
    assert 1.2 < expect[cols].max() / expect[cols].min()        # the factor really varies


# ---------------------------------------------------------------------------
# the sigma cutoff (the 32^3 water workload's "lateral cutoff 3 sigma"):
# half-width a_t/2 + k c3^(1)(d) on each lateral axis, inclusive
# ---------------------------------------------------------------------------
_C3_FLAT = (1.7, 4.1, 9.3)       # three distinct widths, so a term mix-up moves the edge


def _flat_model(c3=_C3_FLAT, T=0.8, cutoff_mode=P.CUTOFF_SIGMA, k=2.5):
    """A beam model whose table is the same at every depth: T and c3 do not
    depend on d, so the cutoff's half-width is a closed form of t alone."""
    lut = np.empty((256, 4), np.float32)
    lut[:, 0] = T
    lut[:, 1:] = c3
    return P.Model(lut=lut, d_max=300.0, c1=(0.6, 0.3, 0.1), c2=(1, 1, 1), cutoff_mode=cutoff_mode, cutoff_k=k)


def _central_beamlet_frame(g, gantry, sad):
    """t, x', z' of every voxel centre for the single beamlet through the
    isocentre (0, 0, 0), written out for gantry 0 (source at -y, x' = x,
    z' = z) and gantry 90 (source at +x, x' = y, z' = z)."""
    x, y, z = g.voxel_centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    if gantry == 0.0:
        return Y + sad, X, Z
    assert gantry == 90.0
    return sad - X, Y, Z


def _sigma_margin(t, xp, zp, a, b, sad, k, c3_1):
    return np.minimum(a * t / (2 * sad) + k * c3_1 - np.abs(xp), b * t / (2 * sad) + k * c3_1 - np.abs(zp))


@pytest.mark.parametrize("gantry", [0.0, 90.0])
def test_sigma_cutoff_candidate_set_closed_form(gantry):
    """Candidates are exactly the voxel centres with |x'| <= a_t/2 + k c3_1 and
    |z'| <= b_t/2 + k c3_1 (a_t = a t/SAD), whatever the density: the table is
    flat, so the half-width depends on t alone.  The test also checks that it
    would see the plausible slips: c3 of term 2 or 3 in place of term 1, a
    dropped a_t/2, k applied to a_t/2 too, and a and b exchanged."""
    sad, a, b, k = 100.0, 6.0, 3.5, 2.5
    m = _flat_model(k=k)
    if gantry == 0.0:
        g = P.centred_grid(20, 30, 16, 1.3, 1.3, 1.3, centre=(0.37, 0.0, 0.21))
    else:
        g = P.centred_grid(30, 20, 16, 1.3, 1.3, 1.3, centre=(0.0, 0.37, 0.21))
    rho = P.random_grid_density(17, g.shape, 0.2, 1.8)
    beam = P.Beam(gantry, sad, (0.0, 0.0, 0.0), a, b, 1, 1)
    r = O.compute(g, rho, m, [beam], tau=0.0)
    t, xp, zp = _central_beamlet_frame(g, gantry, sad)
    margin = _sigma_margin(t, xp, zp, a, b, sad, k, _C3_FLAT[0])
    assert np.abs(margin).min() > 1e-4                      # no centre near the edge
    expect = np.flatnonzero((margin >= 0).ravel())
    assert r.pairs == expect.size > 0
    cols, vals = r.row(0)
    assert np.array_equal(cols, expect)                     # tau = 0: every candidate has D > 0
    assert r.amb_col.size == 0                                    # nothing within 1e-3 mm of the edge
    slips = {
        "c3 of term 2": _sigma_margin(t, xp, zp, a, b, sad, k, _C3_FLAT[1]),
        "c3 of term 3": _sigma_margin(t, xp, zp, a, b, sad, k, _C3_FLAT[2]),
        "no a_t/2": np.minimum(k * _C3_FLAT[0] - np.abs(xp), k * _C3_FLAT[0] - np.abs(zp)),
        "k on a_t/2": _sigma_margin(t, xp, zp, k * a, k * b, sad, k, _C3_FLAT[0]),
        "a and b exchanged": _sigma_margin(t, xp, zp, b, a, sad, k, _C3_FLAT[0]),
    }
    for name, s in slips.items():
        assert np.count_nonzero((s >= 0) != (margin >= 0)) > 20, name


def test_sigma_cutoff_depends_on_depth_through_c3():
    """With c3_1 growing with depth the half-width follows c3_1(d): in vacuum
    d = 0, so the edge is a_t/2 + k c3_1(0); in uniform density 0.5 the depth
    at O' is 0.5 (t - t_A) and the edge is a_t/2 + k c3_1(d) with c3_1 read
    off the table by linear interpolation (written out here)."""
    sad, a, b, k = 100.0, 4.0, 4.0, 2.0
    lut = np.empty((256, 4), np.float32)
    dd = np.linspace(0.0, 300.0, 256)
    lut[:, 0] = 1.0
    lut[:, 1] = 1.0 + 0.05 * dd          # c3_1 grows 0.05 mm per mm of depth
    lut[:, 2] = 3.0
    lut[:, 3] = 8.0
    m = P.Model(lut=lut, d_max=300.0, c1=(0.9, 0.08, 0.02), c2=(1, 1, 1), cutoff_mode=P.CUTOFF_SIGMA,
                cutoff_k=k)
    g = P.centred_grid(24, 40, 6, 1.1, 1.1, 1.1, centre=(0.23, 0.0, 0.17))
    beam = P.Beam(0.0, sad, (0.0, 0.0, 0.0), a, b, 1, 1)
    t, xp, zp = _central_beamlet_frame(g, 0.0, sad)
    tA = g.origin[1] + sad
    for rho0 in (0.0, 0.5):
        rho = np.full(g.shape, rho0, np.float32)
        d = float(np.float32(rho0)) * np.clip(t - tA, 0.0, None)
        gi = d * 255 / 300.0
        kk = np.floor(gi).astype(int)
        c3_1 = lut[kk, 1].astype(np.float64) + (gi - kk) * (lut[kk + 1, 1].astype(np.float64) - lut[kk, 1])
        margin = np.minimum(a * t / (2 * sad) + k * c3_1 - np.abs(xp), b * t / (2 * sad) + k * c3_1 - np.abs(zp))
        band = np.abs(margin) <= 1e-3
        r = O.compute(g, rho, m, [beam], tau=0.0)
        keep = (margin >= 0).ravel()
        amb = r.ambiguous(0)
        assert amb == set(np.flatnonzero(band.ravel()).tolist())
        cols, _ = r.row(0)
        got = np.zeros(g.nvox, bool)
        got[cols] = True
        assert np.array_equal(got[~band.ravel()], keep[~band.ravel()])
    # the two densities give different candidate sets (the depth matters)
    assert r.pairs != O.compute(g, np.zeros(g.shape, np.float32), m, [beam], tau=0.0).pairs


def test_cutoff_band_is_classified_kind_2():
    """A voxel centre placed 4e-4 mm inside the x edge and another 4e-4 mm
    outside the z edge are both in the cutoff band (kind 2); the band is
    exactly the set of centres whose closed-form margin is within 1e-3 mm."""
    sad, a, k = 100.0, 6.0, 2.5
    g = P.centred_grid(20, 30, 16, 1.3, 1.3, 1.3, centre=(0.37, 0.0, 0.21))
    t, xp, zp = _central_beamlet_frame(g, 0.0, sad)
    # choose c3_1 so the x edge passes 4e-4 mm beyond centre (ix=15, iy=10,
    # iz=8), then b so the z edge stops 4e-4 mm short of centre (iz=12,
    # iy=20, ix=10); the other lateral coordinate is well inside at both
    X1, T1 = xp[8, 10, 15], t[8, 10, 15]
    c3_1 = (abs(X1) + 4e-4 - a * T1 / (2 * sad)) / k
    Z2, T2 = zp[12, 20, 10], t[12, 20, 10]
    b = (abs(Z2) - 4e-4 - k * c3_1) * 2 * sad / T2
    assert c3_1 > 0 and b > 0
    c3 = (c3_1, 2.0 * c3_1 + 1.0, 4.0 * c3_1 + 3.0)
    m = _flat_model(c3=c3, k=k)
    c3_1 = float(np.float32(c3_1))                       # the table stores FP32
    beam = P.Beam(0.0, sad, (0.0, 0.0, 0.0), a, b, 1, 1)
    rho = np.ones(g.shape, np.float32)
    r = O.compute(g, rho, m, [beam], tau=0.0)
    margin = _sigma_margin(t, xp, zp, a, b, sad, k, c3_1)
    assert np.all(np.abs(np.abs(margin) - 1e-3) > 1e-6)    # the band's own edge is clear
    band = np.flatnonzero((np.abs(margin) <= 1e-3).ravel())
    c_in = (8 * g.ny + 10) * g.nx + 15
    c_out = (12 * g.ny + 20) * g.nx + 10
    assert margin.ravel()[c_in] == pytest.approx(4e-4, abs=1e-6)
    assert margin.ravel()[c_out] == pytest.approx(-4e-4, abs=1e-6)
    kinds = dict(zip(r.amb_col.tolist(), r.amb_kind.tolist()))
    assert set(kinds) == set(band.tolist()) and {c_in, c_out} <= set(kinds)
    assert set(kinds.values()) == {2}
    cols, _ = r.row(0)
    assert c_in in cols and c_out not in cols


@pytest.mark.parametrize("side", [+1, -1])
def test_threshold_band_is_classified_kind_1(side):
    """Vacuum and widths -> 0: inside the beamlet D = T(0) (SAD/t)^2 sum(c1),
    so the row maximum sits at the smallest t and D/M = (t_min/t)^2.  With
    tau = (t_min/t_k)^2 (1 + side 5e-7) the voxels inside the beamlet at
    depth row k are within 1e-6 of the threshold (kind 1): dropped for side
    +1, kept for side -1; no other pair is in a band."""
    lut = P.synthetic_model().lut.copy()
    lut[:, 1:] = 1e-6
    m = P.Model(lut=lut, d_max=300.0, c1=(0.6, 0.3, 0.05), c2=(1, 1, 1), cutoff_mode=P.CUTOFF_VOI6)
    sad, a, b = 100.0, 8.0, 5.0
    g = P.centred_grid(16, 24, 12, 1.3, 1.3, 1.3, centre=(0.37, 0.0, 0.21))
    rho = np.zeros(g.shape, np.float32)
    beam = P.Beam(0.0, sad, (0.0, 0.0, 0.0), a, b, 1, 1)
    t, xp, zp = _central_beamlet_frame(g, 0.0, sad)
    inside = (np.abs(xp) < a * t / (2 * sad)) & (np.abs(zp) < b * t / (2 * sad))
    cand = (np.abs(xp) <= 3 * a * t / sad) & (np.abs(zp) <= 3 * b * t / sad)
    ty = t[0, :, 0]
    t_min, kk = ty[0], 13
    assert inside[:, 0, :].any() and inside[:, kk, :].any()
    tau = (t_min / ty[kk]) ** 2 * (1 + side * 5e-7)
    r = O.compute(g, rho, m, [beam], tau=tau)
    M = float(lut[0, 0]) * (sad / t_min) ** 2 * sum(m.c1)
    assert r.row_max[0] == pytest.approx(M, rel=1e-12)
    assert r.pairs == int(cand.sum())
    row_k = np.zeros(g.shape, bool)
    row_k[:, kk, :] = True
    band = np.flatnonzero((inside & row_k).ravel())
    kinds = dict(zip(r.amb_col.tolist(), r.amb_kind.tolist()))
    assert set(kinds) == set(band.tolist()) and set(kinds.values()) == {1}
    kept = inside & ((t < ty[kk]) | ((t == ty[kk]) & (side < 0)))
    cols, _ = r.row(0)
    assert np.array_equal(cols, np.flatnonzero(kept.ravel()))


def test_water_depth_at_projection_point():
    """Water, widths c3 -> 0: inside the divergent beamlet D (t/SAD)^2 / sum(c1) equals
    T at the geometric depth of O' (the projection of P on the axis), t - t_A, for every
    lateral offset -- the depth is taken at O', not along SP."""
    base = P.synthetic_model()
    lut = base.lut.copy()
    lut[:, 1:] = 1e-6
    m = P.Model(lut=lut, d_max=300.0, c1=(0.6, 0.3, 0.05), c2=(1, 1, 1), cutoff_mode=P.CUTOFF_VOI6)
    sad, a, b = 100.0, 40.0, 36.0
    g = P.centred_grid(32, 20, 30, 1.3, 1.3, 1.3, centre=(0.37, 0.0, 0.21))
    rho = np.ones(g.shape, np.float32)
    beam = P.Beam(0.0, sad, (0.0, 0.0, 0.0), a, b, 1, 1)
    r = O.compute(g, rho, m, [beam], tau=0.0)
    x, y, z = g.voxel_centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    t = (Y + sad).ravel()
    tA = g.origin[1] + sad
    cols, vals = r.row(0)
    assert np.unique(np.round(X.ravel()[cols], 6)).size > 20          # many lateral offsets
    got = vals * (t[cols] / sad) ** 2 / sum(m.c1)
    expect = np.array([O.lut_eval(m, tc - tA)[0] for tc in t[cols]])
    assert np.allclose(got, expect, rtol=1e-12)


# ---------------------------------------------------------------------------
# invariants: mirror symmetry and gantry rotation
# ---------------------------------------------------------------------------
def test_mirror_symmetry_of_centred_field():
    g = P.centred_grid(20, 12, 14, 2.5, 2.5, 2.5)
    rho = np.ones(g.shape, np.float32)
    m = P.synthetic_model()
    beam = P.Beam(0.0, 1000.0, (0.0, 0.0, 0.0), 5.0, 5.0, 6, 4)
    r = O.compute(g, rho, m, [beam], tau=1e-3)
    D = dense(r, 24, g.nvox).reshape(4, 6, g.nz, g.ny, g.nx)        # iv, iu, iz, iy, ix
    assert D.max() > 0
    for mirrored in (D[:, ::-1, :, :, ::-1], D[::-1, :, ::-1, :, :]):
        both = (D > 0) & (mirrored > 0)
        assert np.allclose(D[both], mirrored[both], rtol=1e-12)
        diff = np.argwhere((D > 0) != (mirrored > 0))
        for iv, iu, iz, iy, ix in diff:          # structure differs only in the bands
            row = iv * 6 + iu
            col = (iz * g.ny + iy) * g.nx + ix
            assert col in r.ambiguous(row) or np.any(
                [(cc in r.ambiguous(rr)) for rr, cc in _mirror_pairs(row, col, g)])


def _mirror_pairs(row, col, g):
    iv, iu = divmod(row, 6)
    iz, rem = divmod(col, g.ny * g.nx)
    iy, ix = divmod(rem, g.nx)
    return [(iv * 6 + (5 - iu), (iz * g.ny + iy) * g.nx + (g.nx - 1 - ix)),
            ((3 - iv) * 6 + iu, ((g.nz - 1 - iz) * g.ny + iy) * g.nx + ix)]


def test_gantry_90_rotation_permutes_voxels():
    n = 16
    g = P.centred_grid(n, n, 10, 3.0, 3.0, 3.0)
    rho = np.ones(g.shape, np.float32)
    m = P.synthetic_model()
    b0 = P.Beam(0.0, 1000.0, (0.0, 0.0, 0.0), 6.0, 4.0, 4, 3)
    b90 = P.Beam(90.0, 1000.0, (0.0, 0.0, 0.0), 6.0, 4.0, 4, 3)
    r0 = O.compute(g, rho, m, [b0], tau=1e-3)
    r90 = O.compute(g, rho, m, [b90], tau=1e-3)
    D0 = dense(r0, 12, g.nvox).reshape(12, g.nz, n, n)                 # row, iz, iy, ix
    D90 = dense(r90, 12, g.nvox).reshape(12, g.nz, n, n)
    # voxel (ix, iy) at gantry 0 sits at (n-1-iy, ix) at gantry 90
    rot = np.transpose(D0, (0, 1, 3, 2))[:, :, :, ::-1]                # [row, iz, ix, n-1-iy]
    both = (rot > 0) & (D90 > 0)
    assert both.sum() > 1000
    assert np.allclose(rot[both], D90[both], rtol=1e-9)
    for row, iz, iy, ix in np.argwhere((rot > 0) != (D90 > 0)):
        assert ((iz * n + iy) * n + ix) in r90.ambiguous(row)


# ---------------------------------------------------------------------------
# enumeration: the VOI bounding box loses nothing; threshold semantics
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode,gantry", [(P.CUTOFF_VOI6, 40.0), (P.CUTOFF_SIGMA, 0.0), (P.CUTOFF_VOI6, 300.0)])
def test_bounding_box_matches_full_scan(mode, gantry):
    g = P.centred_grid(28, 24, 20, 4.0, 4.0, 5.0, centre=(5.0, -3.0, 2.0))
    rho = P.random_grid_density(5, g.shape, 0.2, 1.8)
    m = P.synthetic_model(cutoff_mode=mode)
    beams = [P.Beam(gantry, 1000.0, (0.0, 0.0, 0.0), 5.0, 10.0, 8, 4)]
    a = O.compute(g, rho, m, beams)
    b = O.compute(g, rho, m, beams, full_scan=True)
    assert a.pairs == b.pairs > 0
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.val, b.val)


def test_threshold_keeps_relative_to_row_max():
    w = P.water_32()
    full = O.compute(w.grid, w.density, w.model, w.beams, tau=0.0)
    thr = O.compute(w.grid, w.density, w.model, w.beams, tau=1e-3)
    assert full.nnz == full.pairs == thr.pairs
    assert np.array_equal(full.row_max, thr.row_max)
    for r in range(0, 400, 13):
        c, v = full.row(r)
        keep = v >= 1e-3 * full.row_max[r]
        c2, v2 = thr.row(r)
        assert np.array_equal(c[keep], c2) and np.array_equal(v[keep], v2)
        assert np.all(np.diff(c2) > 0)            # columns ascending
        assert full.row_max[r] == v.max()


def test_row_subset_equals_full_rows():
    w = P.slabs_128()
    sel = np.array([5, 800, 1599, 0, 777])
    a = O.compute_workload(w, rows=sel)
    g, b1 = w.grid, w.beams[0]
    for i, row in enumerate(sel):
        single = O.compute(g, w.density, w.model,
                           [P.Beam(b1.gantry_deg, b1.sad, b1.iso, b1.a, b1.b, b1.n_u, b1.n_v)], rows=[row])
        ca, va = a.row(i)
        cs, vs = single.row(0)
        assert np.array_equal(ca, cs) and np.array_equal(va, vs)


# ---------------------------------------------------------------------------
# the paper's printed VOI counts (Table 1, N'_voxel)
# ---------------------------------------------------------------------------
def load_table1():
    rows = {}
    with open(os.path.join(HERE, "golden", "table1_nprime.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            c, vox, bl, nbl, npr = line.split()
            rows[int(c)] = (float(vox), float(bl), int(nbl), float(npr))
    return rows


@pytest.mark.parametrize("case", [1, 7])
def test_voi_count_against_table1(case):
    """The count of voxel centres inside all VOIs of 6x the beamlet side falls
    within [0.5, 1.0] of the paper's N'_voxel (the paper's counting rule for
    voxels straddling the VOI edge is not stated; a 5x or 7x VOI falls out)."""
    vox, bl, nbl, nprime = load_table1()[case]
    w = P.table1_water(case)
    assert w.beams[0].nbeamlets == nbl
    assert abs(w.grid.dx - vox * 10) < 0.05 * vox * 10
    r = O.compute_workload(w)
    assert 0.5 <= r.pairs / nprime <= 1.0, r.pairs / nprime


# ---------------------------------------------------------------------------
# the paper's trilinear-sampled depth table (Section 2.2; NEXT-1)
# ---------------------------------------------------------------------------
def _tri_grid():
    return P.Grid(7, 9, 6, 2.0, 1.5, 2.5, (-7.0, -6.75, -7.5))


def _centre(g, ix, iy, iz):
    return np.array([g.origin[0] + (ix + 0.5) * g.dx, g.origin[1] + (iy + 0.5) * g.dy,
                     g.origin[2] + (iz + 0.5) * g.dz])


def test_trilinear_reproduces_voxel_values_at_centres():
    g = _tri_grid()
    rho = P.random_grid_density(11, (g.nz, g.ny, g.nx))
    for ix, iy, iz in [(0, 0, 0), (3, 4, 2), (6, 8, 5), (1, 7, 3)]:
        assert O.trilinear(g, rho, _centre(g, ix, iy, iz)) == pytest.approx(float(rho[iz, iy, ix]), abs=1e-12)


def test_trilinear_is_exact_on_linear_fields_and_clamps_at_the_edge():
    """A field linear in x, y, z (stored at the voxel centres) is reproduced
    exactly between the centre planes; past the outermost centre plane the
    edge plane's value holds (clamp to edge), along each axis separately."""
    g = _tri_grid()
    a, bx, by, bz = 1.0, 0.03, -0.02, 0.05
    zc, yc, xc = np.meshgrid(*[g.origin[k] + (np.arange(n) + 0.5) * d
                               for k, n, d in ((2, g.nz, g.dz), (1, g.ny, g.dy), (0, g.nx, g.dx))], indexing="ij")
    rho = (a + bx * xc + by * yc + bz * zc).astype(np.float32)
    lin = lambda p: a + bx * p[0] + by * p[1] + bz * p[2]
    lo = _centre(g, 0, 0, 0)
    hi = _centre(g, g.nx - 1, g.ny - 1, g.nz - 1)
    rng = np.random.default_rng(5)
    for _ in range(50):
        p = lo + rng.random(3) * (hi - lo)
        assert O.trilinear(g, rho, p) == pytest.approx(lin(p), abs=2e-7)
    # outside the centre span: coordinates clamp to the outermost centre, per axis
    for p in (np.array([g.origin[0] + 0.3, 0.2, 0.1]), np.array([0.4, g.origin[1] + g.ny * g.dy, -0.2]),
              np.array([lo[0] - 0.7, hi[1] + 0.4, hi[2] + 1.0])):
        q = np.minimum(np.maximum(p, lo), hi)
        assert O.trilinear(g, rho, p) == pytest.approx(lin(q), abs=2e-7)


@pytest.mark.parametrize("gantry", [0.0, 41.0, 90.0, 222.0])
def test_trilinear_table_uniform_density(gantry):
    g = P.centred_grid(24, 20, 16, 3.0, 2.5, 4.0)
    rho = np.full(g.shape, 0.83, np.float32)
    beam = P.Beam(gantry, 400.0, (3.0, -2.0, 1.0), 6.0, 5.0, 3, 2)
    bl = O.beamlets(g, [beam])
    h = 0.5 * 2.5
    for r, iu, iv in rows_of(beam):
        tab = O.row_table(g, rho, beam, iu, iv, table_mode=1)
        L = bl[r, 13] - bl[r, 12]
        assert tab.size == int(math.ceil(L / h)) + 1
        expect = float(np.float32(0.83)) * np.minimum(np.arange(tab.size) * h, L)
        assert np.allclose(tab, expect, rtol=0, atol=1e-10)


def test_trilinear_table_linear_field_along_the_ray():
    """Ray along +y (gantry 0, one beamlet through the isocentre), density
    linear in y between the first and last centre planes and clamped beyond.
    With h = dy/2 the kinks fall on sample points, so the trapezoid rule is
    exact: d(s) = integral of the clamped line.  The isocentre sits off the
    voxel centres in x and z so the x and z weights matter (the field is
    also linear in x with zero y-x coupling)."""
    g = P.Grid(6, 10, 5, 2.0, 1.5, 2.0, (-6.0, -7.5, -5.0))
    a, by, bx = 0.9, 0.04, 0.02
    zc, yc, xc = np.meshgrid(*[g.origin[k] + (np.arange(n) + 0.5) * d
                               for k, n, d in ((2, g.nz, g.dz), (1, g.ny, g.dy), (0, g.nx, g.dx))], indexing="ij")
    rho = (a + by * yc + bx * xc).astype(np.float32)
    x0, z0 = 0.37, -0.61
    beam = P.Beam(0.0, 300.0, (x0, 0.0, z0), 1.0, 1.0, 1, 1)
    tab = O.row_table(g, rho, beam, 0, 0, h_frac=0.5, table_mode=1)
    y_first = g.origin[1] + 0.5 * g.dy
    y_last = g.origin[1] + (g.ny - 0.5) * g.dy

    def rho_y(y):
        return a + bx * x0 + by * np.clip(y, y_first, y_last)

    def integral(y1):                      # from the entry face y = origin to y1
        ys = np.linspace(g.origin[1], y1, 20001)
        return np.trapezoid(rho_y(ys), ys) if hasattr(np, "trapezoid") else np.trapz(rho_y(ys), ys)
    h = 0.5 * g.dy
    for k in range(tab.size):
        y1 = g.origin[1] + min(k * h, g.ny * g.dy)
        assert tab[k] == pytest.approx(integral(y1), abs=1e-6)


def test_trilinear_table_converges_at_second_order():
    """Halving the element length on a random field: the table's end value
    converges to the line integral of the trilinear field at rate ~4."""
    g = _tri_grid()
    rho = P.random_grid_density(3, (g.nz, g.ny, g.nx))
    beam = P.Beam(27.0, 80.0, (0.4, -0.3, 0.2), 1.0, 1.0, 1, 1)
    ends = [O.row_table(g, rho, beam, 0, 0, h_frac=f, table_mode=1)[-1] for f in (1 / 2, 1 / 4, 1 / 8, 1 / 16)]
    d1, d2, d3 = abs(ends[0] - ends[1]), abs(ends[1] - ends[2]), abs(ends[2] - ends[3])
    assert d1 > 0 and d2 / d3 > 3.0 and d1 / d2 > 3.0


# ---------------------------------------------------------------------------
# Eq. 1: dose superposition on the oracle's D_ij (NEXT-3)
# ---------------------------------------------------------------------------
def test_weighted_superposition_equals_a_half_field():
    """Parallel limit, water, no cutoff, no threshold: weights 1 on the two
    left columns of a 4 x 3 field of 4 x 6 mm beamlets and 0 elsewhere give
    the dose of one 8 x 18 mm beamlet centred on the left half (Eq. 1 with
    the erf tiling of Section 2.1); a row-order or weight slip moves it."""
    g = P.centred_grid(16, 12, 10, 3.0, 3.0, 3.0)
    rho = np.ones(g.shape, np.float32)
    m = P.synthetic_model(cutoff_mode=P.CUTOFF_NONE)
    sad = 1e9
    small = P.Beam(0.0, sad, (0.0, 0.0, 0.0), 4.0, 6.0, 4, 3)
    half = P.Beam(0.0, sad, (-4.0, 0.0, 0.0), 8.0, 18.0, 1, 1)
    rs = O.compute(g, rho, m, [small], tau=0.0)
    rh = O.compute(g, rho, m, [half], tau=0.0)
    w = np.array([1.0 if iu < 2 else 0.0 for _, iu, _ in rows_of(small)])
    d = O.dose(rs, w, g.nvox)
    ref = dense(rh, 1, g.nvox)[0]
    assert ref.min() > 0
    assert np.abs(d / ref - 1).max() < 1e-6
    # and the right half is the mirror image: weights on the right columns
    d_right = O.dose(rs, 1.0 - w, g.nvox).reshape(g.shape)
    assert np.abs(d_right[:, :, ::-1] - d.reshape(g.shape)).max() < 1e-9 * d.max()


def test_dose_and_beamlet_dot_are_adjoint():
    """<dose(w), g> = <w, beamlet_dot(g)> for random w, g (the two products
    are transposes of one operator; a transposed operand breaks it)."""
    w_ = P.water_32()
    orc = O.compute_workload(w_)
    rng = np.random.default_rng(2)
    wv = rng.random(w_.nrows)
    gv = rng.standard_normal(w_.grid.nvox)
    lhs = np.dot(O.dose(orc, wv, w_.grid.nvox), gv)
    rhs = np.dot(wv, O.beamlet_dot(orc, gv, w_.grid.nvox))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)



# ---------------------------------------------------------------------------
# other FSPB kernels (Section 2.1; NEXT-4): Laplace and logistic spread
# ---------------------------------------------------------------------------
def _one_component(profile, i, c2=1.2):
    c1 = [0.0, 0.0, 0.0]
    c1[i] = 1.0
    c2s = [1.0, 1.0, 1.0]
    c2s[i] = c2
    return P.synthetic_model(c1=tuple(c1), c2=tuple(c2s), profile=profile)


def _spread(profile, c3):
    return c3 / math.sqrt(2.0) if profile == P.PROFILE_LAPLACE else c3 * math.sqrt(3.0) / math.pi


def _P_closed(profile, x, h, s):
    """box of half-width h convolved with the kernel, written out from the
    kernel's density by hand: Laplace density exp(-|u|/s)/(2s), logistic
    density exp(-u/s)/(s (1 + exp(-u/s))^2)."""
    if profile == P.PROFILE_LAPLACE:
        x = abs(x)
        if x <= h:
            return 1.0 - math.exp(-h / s) * math.cosh(x / s)
        return math.sinh(h / s) * math.exp(-x / s)
    cdf = lambda u: 1.0 / (1.0 + math.exp(-u / s))
    return cdf(x + h) - cdf(x - h)


@pytest.mark.parametrize("profile", [P.PROFILE_LAPLACE, P.PROFILE_LOGISTIC])
def test_new_profiles_closed_form_points(profile):
    c3 = np.array([1.3, 3.7, 8.2])
    a_t, b_t = 5.0, 3.0
    for i in range(3):
        m = _one_component(profile, i)
        s = _spread(profile, c3[i])
        hx, hz = 1.2 * a_t / 2, 1.2 * b_t / 2
        for x, z in [(0.0, 0.0), (hx, 0.0), (0.4 * hx, 1.3 * hz), (2.5 * hx, 0.2), (-1.1 * hx, -2 * hz)]:
            expect = _P_closed(profile, x, hx, s) * _P_closed(profile, z, hz, s)
            assert O.profile_F(m, c3, x, z, a_t, b_t) == pytest.approx(expect, rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("profile", [P.PROFILE_LAPLACE, P.PROFILE_LOGISTIC])
def test_new_profiles_normalisation(profile):
    """Per axis the profile integrates to the beamlet side 2h (the
    normalisation condition): integral of F(x, 0) dx = 2 h_x P_z(0), with
    P_z(0) = F(0, 0) / P_x(0) and P(0) closed form."""
    c3 = np.array([1.3, 3.7, 8.2])
    a_t, b_t = 5.0, 3.0
    for i in range(3):
        m = _one_component(profile, i)
        s = _spread(profile, c3[i])
        hx = 1.2 * a_t / 2
        R = hx + 40 * s
        xs = np.linspace(-R, R, 40001)
        fx = np.array([O.profile_F(m, c3, x, 0.0, a_t, b_t) for x in xs])
        w = np.ones(xs.size)
        w[1:-1:2], w[2:-1:2] = 4.0, 2.0
        integral = (w @ fx) * (xs[1] - xs[0]) / 3.0
        pz0 = O.profile_F(m, c3, 0.0, 0.0, a_t, b_t) / _P_closed(profile, 0.0, hx, s)
        assert integral == pytest.approx(2 * hx * pz0, rel=2e-7)

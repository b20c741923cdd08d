/*
 * dsc_oracle.c -- plain FP64 CPU oracle for finite-size pencil beam (FSPB)
 * dose-deposition coefficients D_ij (Gu et al., "GPU-based ultra fast dose
 * calculation using a finite pencil beam model").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline / reference arm call this file.  It shares no code,
 * header, table or constant with the CUDA path, and it is deliberately slow
 * and direct: every step is the definition written out in double precision,
 * in the order of the paper's CPU algorithm (Fig. 2a: loop over beamlets,
 * build the radiological-depth table, loop over the voxels of the beamlet's
 * VOI and evaluate Eq. 2-3).
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes): the off-axis factor A(theta, d) is a tabulated depth-dose T(d)
 * times the inverse square (SAD/t)^2 with no extra theta dependence; beamlet
 * sides a, b are given at the isocentre plane and scale with t/SAD; the
 * evaluation point is the voxel centre; the depth table holds the exact
 * piecewise-constant integral of density (Siddon 1985) at points spaced
 * h = h_frac * min voxel side; depths before A clamp to 0 and past B to d(B);
 * depths past the LUT range clamp to the last entry; entries are kept when
 * D > 0 and D >= tau * (maximum of the beamlet's row).
 *
 * Parity pins for every function live in tests/test_oracle_pins.py: closed
 * forms (water depth, slab depth, inverse square, lateral integral),
 * invariants (mirror symmetry, 90-degree rotation, erf tiling of a broad
 * field) and brute-force ray marching on tiny random grids.  Absolute dose
 * against a measured 6 MV beam is parity unpinned: the fitted beam data the
 * paper uses is not available, so a synthetic parameter set defines truth.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

typedef struct { int nx, ny, nz; double dx, dy, dz; double ox, oy, oz; } or_grid;
typedef struct { double gantry_deg, sad, iso[3], a, b; int n_u, n_v; } or_beam;
typedef struct {
    int n;              /* LUT entries, equally spaced on [0, d_max] */
    double d_max;
    const float* lut;   /* n x 4: T(d), c3_1(d), c3_2(d), c3_3(d) */
    double c1[3], c2[3];
    int cutoff_mode;    /* 0 VOI6, 1 SIGMA, 2 NONE */
    double cutoff_k;
    int profile;        /* lateral spread kernel: 0 Gaussian (Eq. 3), 1 Laplace, 2 logistic */
} or_model;

/* one beamlet's frame (Fig. 1b): source S, unit axis e, lateral axes x, z */
typedef struct {
    double S[3], e[3], x[3], z[3];
    double sad, a, b;
    double tA, tB;      /* axis parameter of entry A and exit B (|e| = 1) */
    int hit;            /* 1 if the axis crosses the grid prism */
    double theta;       /* angle between beamlet axis and broad-beam axis */
} or_beamlet;

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void normalize3(double* v) {
    double n = sqrt(dot3(v, v));
    v[0] /= n; v[1] /= n; v[2] /= n;
}

/* ---------------------------------------------------------------------------
 * Ray / prism intersection: the parameters t of the entry point A and exit
 * point B of the line S + t e through the smallest prism that holds the CT
 * grid (Fig. 1 caption).  Slab method, one axis at a time.
 * ------------------------------------------------------------------------- */
static int ray_box(const or_grid* g, const double* S, const double* e, double* tA, double* tB) {
    double lo[3] = {g->ox, g->oy, g->oz};
    double hi[3] = {g->ox + g->nx * g->dx, g->oy + g->ny * g->dy, g->oz + g->nz * g->dz};
    double t0 = -INFINITY, t1 = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (e[k] == 0.0) {
            if (S[k] < lo[k] || S[k] > hi[k]) return 0;
            continue;
        }
        double ta = (lo[k] - S[k]) / e[k];
        double tb = (hi[k] - S[k]) / e[k];
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (t0 < 0.0) t0 = 0.0;
    if (!(t1 > t0)) return 0;
    *tA = t0;
    *tB = t1;
    return 1;
}

/* ---------------------------------------------------------------------------
 * Beam and beamlet frames (Section 2.1, Fig. 1).
 * Gantry rotates about +z: S = I + SAD (sin g, -cos g, 0), broad-beam axis
 * E = (I - S)/SAD, u = (cos g, sin g, 0), v = (0, 0, 1).  Beamlet (iu, iv)
 * is centred at C = I + uc u + vc v with uc = (iu + 1/2 - n_u/2) a and
 * vc = (iv + 1/2 - n_v/2) b.  Its axis is e = (C - S)/|C - S|, theta the
 * angle between e and E, and x', z' are the components along u and v made
 * perpendicular to e (Gram-Schmidt).
 * ------------------------------------------------------------------------- */
int or_beamlet_setup(const or_grid* g, const or_beam* bm, int iu, int iv, or_beamlet* out) {
    double gr = bm->gantry_deg * OR_PI / 180.0;
    double sg = sin(gr), cg = cos(gr);
    double S[3] = {bm->iso[0] + bm->sad * sg, bm->iso[1] - bm->sad * cg, bm->iso[2]};
    double E[3] = {-sg, cg, 0.0};
    double u[3] = {cg, sg, 0.0};
    double v[3] = {0.0, 0.0, 1.0};
    double uc = (iu + 0.5 - 0.5 * bm->n_u) * bm->a;
    double vc = (iv + 0.5 - 0.5 * bm->n_v) * bm->b;
    double C[3];
    for (int k = 0; k < 3; ++k) C[k] = bm->iso[k] + uc * u[k] + vc * v[k];
    memcpy(out->S, S, sizeof S);
    for (int k = 0; k < 3; ++k) out->e[k] = C[k] - S[k];
    normalize3(out->e);
    double pu = dot3(u, out->e);
    for (int k = 0; k < 3; ++k) out->x[k] = u[k] - pu * out->e[k];
    normalize3(out->x);
    double pv = dot3(v, out->e), px = dot3(v, out->x);
    for (int k = 0; k < 3; ++k) out->z[k] = v[k] - pv * out->e[k] - px * out->x[k];
    normalize3(out->z);
    double ce = dot3(out->e, E);
    if (ce > 1.0) ce = 1.0;
    out->theta = acos(ce);
    out->sad = bm->sad;
    out->a = bm->a;
    out->b = bm->b;
    out->hit = ray_box(g, out->S, out->e, &out->tA, &out->tB);
    if (!out->hit) { out->tA = 0.0; out->tB = 0.0; }
    return 0;
}

/* the grid voxel holding point p, clamped to the grid; points on a plane go
 * to the higher index */
static void voxel_of(const or_grid* g, const double* p, int* ix, int* iy, int* iz) {
    int i = (int)floor((p[0] - g->ox) / g->dx);
    int j = (int)floor((p[1] - g->oy) / g->dy);
    int k = (int)floor((p[2] - g->oz) / g->dz);
    *ix = i < 0 ? 0 : (i >= g->nx ? g->nx - 1 : i);
    *iy = j < 0 ? 0 : (j >= g->ny ? g->ny - 1 : j);
    *iz = k < 0 ? 0 : (k >= g->nz ? g->nz - 1 : k);
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* ---------------------------------------------------------------------------
 * Radiological-depth lookup table (Section 2.2): n equally spaced points on
 * AB at spacing h; entry k is the radiological depth from A to the point
 * A + min(k h, |AB|) e, i.e. the integral of density along the axis.  The
 * integral is exact for piecewise-constant voxels: Siddon's algorithm takes
 * every crossing of an x, y or z grid plane between A and B, sorts them, and
 * each segment between consecutive crossings lies in the voxel of its
 * midpoint.  Returns n, or -1 if cap is too small.  n = 0 when the axis
 * misses the grid.
 * ------------------------------------------------------------------------- */
int or_depth_table(const or_grid* g, const float* rho, const or_beamlet* bl, double h, double* out, int cap) {
    if (!bl->hit) return 0;
    double L = bl->tB - bl->tA;
    int n = (int)ceil(L / h) + 1;
    if (n > cap) return -1;
    const double* S = bl->S;
    const double* e = bl->e;
    int nplanes[3] = {g->nx + 1, g->ny + 1, g->nz + 1};
    double org[3] = {g->ox, g->oy, g->oz};
    double sp[3] = {g->dx, g->dy, g->dz};
    int maxc = nplanes[0] + nplanes[1] + nplanes[2] + 2;
    double* al = (double*)malloc(sizeof(double) * maxc);
    int na = 0;
    al[na++] = bl->tA;
    al[na++] = bl->tB;
    for (int k = 0; k < 3; ++k) {
        if (e[k] == 0.0) continue;
        for (int m = 0; m < nplanes[k]; ++m) {
            double t = (org[k] + m * sp[k] - S[k]) / e[k];
            if (t > bl->tA && t < bl->tB) al[na++] = t;
        }
    }
    qsort(al, na, sizeof(double), cmp_double);
    int nu = 0;
    for (int i = 0; i < na; ++i)
        if (nu == 0 || al[i] != al[nu - 1]) al[nu++] = al[i];
    /* walk segments and table points together */
    double cum = 0.0;   /* depth from A to the start of the current segment */
    int seg = 0;
    for (int k = 0; k < n; ++k) {
        double s = k * h;
        if (s > L) s = L;
        double tk = bl->tA + s;
        while (seg < nu - 1 && al[seg + 1] <= tk) {
            double t0 = al[seg], t1 = al[seg + 1];
            double mid = 0.5 * (t0 + t1);
            double p[3] = {S[0] + mid * e[0], S[1] + mid * e[1], S[2] + mid * e[2]};
            int ix, iy, iz;
            voxel_of(g, p, &ix, &iy, &iz);
            cum += (t1 - t0) * (double)rho[((size_t)iz * g->ny + iy) * g->nx + ix];
            ++seg;
        }
        double part = 0.0;
        if (seg < nu - 1 && tk > al[seg]) {
            double t0 = al[seg], t1 = al[seg + 1];
            double mid = 0.5 * (t0 + t1);
            double p[3] = {S[0] + mid * e[0], S[1] + mid * e[1], S[2] + mid * e[2]};
            int ix, iy, iz;
            voxel_of(g, p, &ix, &iy, &iz);
            part = (tk - t0) * (double)rho[((size_t)iz * g->ny + iy) * g->nx + ix];
        }
        out[k] = cum + part;
    }
    free(al);
    (void)sp;
    return n;
}

/* ---------------------------------------------------------------------------
 * Density at a point by trilinear interpolation of the voxel-centred values
 * (Section 2.2 samples the CT this way, in software).  Along each axis the
 * two voxel centres around the point are blended linearly; before the first
 * centre or past the last one the edge value is used (clamp to edge).
 * ------------------------------------------------------------------------- */
double or_trilinear(const or_grid* g, const float* rho, const double* p) {
    const int n[3] = {g->nx, g->ny, g->nz};
    const double f[3] = {(p[0] - g->ox) / g->dx - 0.5, (p[1] - g->oy) / g->dy - 0.5, (p[2] - g->oz) / g->dz - 0.5};
    int i0[3], i1[3];
    double w[3];
    for (int k = 0; k < 3; ++k) {
        if (f[k] <= 0.0) { i0[k] = i1[k] = 0; w[k] = 0.0; }
        else if (f[k] >= n[k] - 1) { i0[k] = i1[k] = n[k] - 1; w[k] = 0.0; }
        else { i0[k] = (int)floor(f[k]); i1[k] = i0[k] + 1; w[k] = f[k] - i0[k]; }
    }
    double v = 0.0;
    for (int c = 0; c < 8; ++c) {
        int ix = (c & 1) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 4) ? i1[2] : i0[2];
        double wt = ((c & 1) ? w[0] : 1.0 - w[0]) * ((c & 2) ? w[1] : 1.0 - w[1]) * ((c & 4) ? w[2] : 1.0 - w[2]);
        v += wt * (double)rho[((size_t)iz * g->ny + iy) * g->nx + ix];
    }
    return v;
}

/* ---------------------------------------------------------------------------
 * The paper's own table construction (Section 2.2): the density is sampled
 * by trilinear interpolation at the n equally spaced points of AB (the same
 * points as or_depth_table, the last one at B), and entry k is the
 * radiological depth from A to point k, accumulated over the sample
 * intervals by the trapezoid rule (the paper does not name the quadrature).
 * Returns n, or -1 if cap is too small; 0 when the axis misses the grid.
 * ------------------------------------------------------------------------- */
int or_depth_table_trilinear(const or_grid* g, const float* rho, const or_beamlet* bl, double h, double* out,
                             int cap) {
    if (!bl->hit) return 0;
    double L = bl->tB - bl->tA;
    int n = (int)ceil(L / h) + 1;
    if (n > cap) return -1;
    double s_prev = 0.0, r_prev = 0.0;
    for (int k = 0; k < n; ++k) {
        double s = k * h;
        if (s > L) s = L;
        double t = bl->tA + s;
        double p[3] = {bl->S[0] + t * bl->e[0], bl->S[1] + t * bl->e[1], bl->S[2] + t * bl->e[2]};
        double r = or_trilinear(g, rho, p);
        out[k] = k == 0 ? 0.0 : out[k - 1] + (s - s_prev) * 0.5 * (r_prev + r);
        s_prev = s;
        r_prev = r;
    }
    return n;
}

/* depth at O' (Section 2.2): linear interpolation of the two neighbouring
 * table entries; s = |AO'| along the axis, clamped to [0, |AB|] */
double or_depth_interp(const double* tab, int n, double h, double s) {
    if (n <= 0) return 0.0;
    if (s <= 0.0) return 0.0;
    double f = s / h;
    double kf = floor(f);
    if (kf >= n - 1) return tab[n - 1];
    int k = (int)kf;
    return tab[k] + (f - kf) * (tab[k + 1] - tab[k]);
}

/* beam-model table at depth d: T(d) and c3^(1..3)(d), linear between the n
 * equally spaced entries on [0, d_max], last entry beyond d_max */
void or_lut_eval(const or_model* m, double d, double* out4) {
    double g = d * (m->n - 1) / m->d_max;
    if (g < 0.0) g = 0.0;
    if (g >= m->n - 1) {
        for (int c = 0; c < 4; ++c) out4[c] = (double)m->lut[(m->n - 1) * 4 + c];
        return;
    }
    int k = (int)floor(g);
    double w = g - k;
    for (int c = 0; c < 4; ++c) {
        double a = (double)m->lut[k * 4 + c], b = (double)m->lut[(k + 1) * 4 + c];
        out4[c] = a + w * (b - a);
    }
}

/* Eq. 3: F(x', d, z', C) with the beamlet sides a_t, b_t at the depth of O' */
static double profile_erf(const or_model* m, const double* c3, double xp, double zp, double a_t, double b_t) {
    double F = 0.0;
    for (int i = 0; i < 3; ++i) {
        double s = sqrt(2.0) * c3[i];
        double hx = m->c2[i] * a_t / 2.0;
        double hz = m->c2[i] * b_t / 2.0;
        double X = erf((hx - xp) / s) + erf((hx + xp) / s);
        double Z = erf((hz - zp) / s) + erf((hz + zp) / s);
        F += m->c1[i] / 4.0 * X * Z;
    }
    return F;
}

/* Other FSPB kernels the paper admits (Section 2.1: any profile that keeps
 * the self-consistency and normalisation conditions; Jelen et al. combine
 * exponentials, Lin et al. use the Boltzmann function).  Both are written
 * like Eq. 3, as the beamlet's box convolved per axis with a spread kernel
 * of standard deviation c3(d), i.e. per axis
 *     P(x) = G(( |x| - h) / s) - G((|x| + h) / s),   h = c2 a_t / 2,
 * with G the kernel's complementary distribution function, and
 * F = sum_i c1_i P_x P_z (Eq. 3 is the Gaussian case, G = erfc(y / sqrt 2) / 2).
 *   profile 1, Laplace (exponential) kernel: s = c3 / sqrt 2,
 *              G(y) = exp(-y) / 2 for y >= 0, 1 - exp(y) / 2 for y < 0;
 *   profile 2, logistic kernel (the Boltzmann function): s = c3 sqrt 3 / pi,
 *              G(y) = 1 / (1 + exp(y)).
 * Each G(y) for y < 0 is taken as 1 - G(-y) so the tails never cancel. */
static double tail_laplace(double y) { return y >= 0.0 ? 0.5 * exp(-y) : 1.0 - 0.5 * exp(y); }
static double tail_logistic(double y) {
    if (y >= 0.0) { double e = exp(-y); return e / (1.0 + e); }
    double e = exp(y);
    return 1.0 - e / (1.0 + e);
}

static double profile_sum(const or_model* m, const double* c3, double xp, double zp, double a_t, double b_t) {
    double F = 0.0;
    for (int i = 0; i < 3; ++i) {
        double s = m->profile == 1 ? c3[i] / sqrt(2.0) : c3[i] * sqrt(3.0) / OR_PI;
        double hx = m->c2[i] * a_t / 2.0, hz = m->c2[i] * b_t / 2.0;
        double ax = fabs(xp), az = fabs(zp);
        double Px, Pz;
        if (m->profile == 1) {
            Px = tail_laplace((ax - hx) / s) - tail_laplace((ax + hx) / s);
            Pz = tail_laplace((az - hz) / s) - tail_laplace((az + hz) / s);
        } else {
            Px = tail_logistic((ax - hx) / s) - tail_logistic((ax + hx) / s);
            Pz = tail_logistic((az - hz) / s) - tail_logistic((az + hz) / s);
        }
        F += m->c1[i] * Px * Pz;
    }
    return F;
}

double or_profile_F(const or_model* m, const double* c3, double xp, double zp, double a_t, double b_t) {
    return m->profile == 0 ? profile_erf(m, c3, xp, zp, a_t, b_t) : profile_sum(m, c3, xp, zp, a_t, b_t);
}

/* signed lateral cutoff margin (mm, > 0 inside): VOI of 6x the side
 * (Section 2.1), or a_t/2 + k sigma_1(d), or no cutoff */
static double cutoff_margin(const or_model* m, double xp, double zp, double a_t, double b_t, double c3_1) {
    if (m->cutoff_mode == 0) {
        double mx = 3.0 * a_t - fabs(xp), mz = 3.0 * b_t - fabs(zp);
        return mx < mz ? mx : mz;
    }
    if (m->cutoff_mode == 1) {
        double mx = a_t / 2.0 + m->cutoff_k * c3_1 - fabs(xp);
        double mz = b_t / 2.0 + m->cutoff_k * c3_1 - fabs(zp);
        return mx < mz ? mx : mz;
    }
    return INFINITY;
}

/* ---------------------------------------------------------------------------
 * Full row evaluation
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t n, cap;
    int32_t* col;
    double* val;
} pairbuf;

static void pb_push(pairbuf* b, int32_t c, double v) {
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 1024;
        b->col = (int32_t*)realloc(b->col, sizeof(int32_t) * b->cap);
        b->val = (double*)realloc(b->val, sizeof(double) * b->cap);
    }
    b->col[b->n] = c;
    b->val[b->n] = v;
    ++b->n;
}

typedef struct {
    pairbuf cand;       /* every candidate (col ascending) with its D */
    pairbuf amb;        /* pairs in the cutoff band (val = margin) */
    double rowmax;
} rowres;

/* which beam and beamlet a global row index names (rows: beam, then iv, then iu) */
static int row_locate(const or_beam* beams, int nbeams, int64_t row, int* b, int* iu, int* iv) {
    for (int k = 0; k < nbeams; ++k) {
        int64_t nb = (int64_t)beams[k].n_u * beams[k].n_v;
        if (row < nb) {
            *b = k;
            *iv = (int)(row / beams[k].n_u);
            *iu = (int)(row % beams[k].n_u);
            return 1;
        }
        row -= nb;
    }
    return 0;
}

static void eval_row(const or_grid* g, const float* rho, const or_model* m, const or_beam* bm, int iu, int iv,
                     double h, int full_scan, int table_mode, rowres* rr) {
    or_beamlet bl;
    or_beamlet_setup(g, bm, iu, iv, &bl);
    rr->rowmax = 0.0;
    if (!bl.hit) return;
    int cap = (int)ceil((bl.tB - bl.tA) / h) + 2;
    double* tab = (double*)malloc(sizeof(double) * cap);
    int n = table_mode == 1 ? or_depth_table_trilinear(g, rho, &bl, h, tab, cap)
                            : or_depth_table(g, rho, &bl, h, tab, cap);

    /* voxel index box that holds the VOI: the VOI between the smallest and
     * largest t of the grid's corners is the convex hull of its two end
     * cross-sections, so the box of those 8 corners holds every candidate */
    int ix0 = 0, ix1 = g->nx - 1, iy0 = 0, iy1 = g->ny - 1, iz0 = 0, iz1 = g->nz - 1;
    if (!full_scan && m->cutoff_mode != 2) {
        double tlo = INFINITY, thi = -INFINITY;
        for (int c = 0; c < 8; ++c) {
            double p[3] = {g->ox + ((c & 1) ? g->nx * g->dx : 0.0), g->oy + ((c & 2) ? g->ny * g->dy : 0.0),
                           g->oz + ((c & 4) ? g->nz * g->dz : 0.0)};
            double w[3] = {p[0] - bl.S[0], p[1] - bl.S[1], p[2] - bl.S[2]};
            double t = dot3(w, bl.e);
            if (t < tlo) tlo = t;
            if (t > thi) thi = t;
        }
        if (tlo < 0.0) tlo = 0.0;
        double c3max = 0.0;
        for (int k = 0; k < m->n; ++k)
            if ((double)m->lut[k * 4 + 1] > c3max) c3max = (double)m->lut[k * 4 + 1];
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int c = 0; c < 8; ++c) {
            double t = (c & 1) ? thi : tlo;
            double hx, hz;
            if (m->cutoff_mode == 0) { hx = 3.0 * bl.a * t / bl.sad; hz = 3.0 * bl.b * t / bl.sad; }
            else { hx = bl.a * t / bl.sad / 2.0 + m->cutoff_k * c3max; hz = bl.b * t / bl.sad / 2.0 + m->cutoff_k * c3max; }
            double su = (c & 2) ? hx : -hx, sv = (c & 4) ? hz : -hz;
            for (int k = 0; k < 3; ++k) {
                double p = bl.S[k] + t * bl.e[k] + su * bl.x[k] + sv * bl.z[k];
                if (p < lo[k]) lo[k] = p;
                if (p > hi[k]) hi[k] = p;
            }
        }
        int a0 = (int)floor((lo[0] - g->ox) / g->dx - 0.5) - 1, a1 = (int)ceil((hi[0] - g->ox) / g->dx - 0.5) + 1;
        int b0 = (int)floor((lo[1] - g->oy) / g->dy - 0.5) - 1, b1 = (int)ceil((hi[1] - g->oy) / g->dy - 0.5) + 1;
        int c0 = (int)floor((lo[2] - g->oz) / g->dz - 0.5) - 1, c1 = (int)ceil((hi[2] - g->oz) / g->dz - 0.5) + 1;
        if (a0 > ix0) ix0 = a0;
        if (a1 < ix1) ix1 = a1;
        if (b0 > iy0) iy0 = b0;
        if (b1 < iy1) iy1 = b1;
        if (c0 > iz0) iz0 = c0;
        if (c1 < iz1) iz1 = c1;
    }

    for (int iz = iz0; iz <= iz1; ++iz)
        for (int iy = iy0; iy <= iy1; ++iy)
            for (int ix = ix0; ix <= ix1; ++ix) {
                double P[3] = {g->ox + (ix + 0.5) * g->dx, g->oy + (iy + 0.5) * g->dy, g->oz + (iz + 0.5) * g->dz};
                double w[3] = {P[0] - bl.S[0], P[1] - bl.S[1], P[2] - bl.S[2]};
                double t = dot3(w, bl.e);
                if (t <= 0.0) continue;
                double xp = dot3(w, bl.x), zp = dot3(w, bl.z);
                double a_t = bl.a * t / bl.sad, b_t = bl.b * t / bl.sad;
                double d = or_depth_interp(tab, n, h, t - bl.tA);
                double lut[4];
                or_lut_eval(m, d, lut);
                double margin = cutoff_margin(m, xp, zp, a_t, b_t, lut[1]);
                int32_t col = (int32_t)(((int64_t)iz * g->ny + iy) * g->nx + ix);
                if (fabs(margin) <= 1e-3) pb_push(&rr->amb, col, margin);
                if (margin < 0.0) continue;
                double F = or_profile_F(m, lut + 1, xp, zp, a_t, b_t);
                double D = lut[0] * (bl.sad / t) * (bl.sad / t) * F;   /* Eq. 2, A = T(d)(SAD/t)^2 */
                pb_push(&rr->cand, col, D);
                if (D > rr->rowmax) rr->rowmax = D;
            }
    free(tab);
}

/* result of or_compute; arrays are malloc'd, release with or_free_result */
typedef struct {
    int64_t nrows;          /* rows computed, in the order requested */
    int64_t nnz;
    int64_t* row_ptr;       /* nrows + 1 */
    int32_t* col;           /* nnz, ascending within a row */
    double* val;            /* nnz */
    double* row_max;        /* nrows: max D over the row's candidates */
    int64_t* row_cand;      /* nrows: candidate count (pairs inside the cutoff) */
    int64_t n_amb;
    int64_t* amb_row;       /* index into the requested rows */
    int32_t* amb_col;
    int32_t* amb_kind;      /* 1 threshold band, 2 cutoff band */
} or_result;

void or_free_result(or_result* r) {
    free(r->row_ptr); free(r->col); free(r->val); free(r->row_max); free(r->row_cand);
    free(r->amb_row); free(r->amb_col); free(r->amb_kind);
    memset(r, 0, sizeof *r);
}

/* D_ij for the listed rows (or every row when rows == NULL): Eq. 2-3 on each
 * candidate voxel of each beamlet's VOI, then the relative threshold and a
 * CSR with columns ascending.  Rows are processed in parallel when OpenMP is
 * available (nthreads <= 0: the runtime default). */
int or_compute(const or_grid* g, const float* rho, const or_model* m, const or_beam* beams, int nbeams,
               double tau, double h_frac, const int64_t* rows, int64_t nsel, int nthreads, int full_scan,
               int table_mode, or_result* out) {
    memset(out, 0, sizeof *out);
    int64_t total = 0;
    for (int k = 0; k < nbeams; ++k) total += (int64_t)beams[k].n_u * beams[k].n_v;
    if (!rows) nsel = total;
    double dmin = g->dx < g->dy ? g->dx : g->dy;
    if (g->dz < dmin) dmin = g->dz;
    double h = h_frac * dmin;
    rowres* rr = (rowres*)calloc(nsel > 0 ? nsel : 1, sizeof(rowres));
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int64_t r = 0; r < nsel; ++r) {
        int64_t row = rows ? rows[r] : r;
        int b, iu, iv;
        if (!row_locate(beams, nbeams, row, &b, &iu, &iv)) { bad |= 1; continue; }
        eval_row(g, rho, m, &beams[b], iu, iv, h, full_scan, table_mode, &rr[r]);
    }
    (void)nthreads;
    if (bad) { free(rr); return -1; }
    out->nrows = nsel;
    out->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (nsel + 1));
    out->row_max = (double*)malloc(sizeof(double) * (nsel > 0 ? nsel : 1));
    out->row_cand = (int64_t*)malloc(sizeof(int64_t) * (nsel > 0 ? nsel : 1));
    int64_t nnz = 0, namb = 0;
    for (int64_t r = 0; r < nsel; ++r) {
        double thr = tau * rr[r].rowmax;
        for (int64_t i = 0; i < rr[r].cand.n; ++i) {
            double D = rr[r].cand.val[i];
            if (D > 0.0 && D >= thr) ++nnz;
            if (thr > 0.0 && fabs(D / thr - 1.0) <= 1e-6) ++namb;
        }
        namb += rr[r].amb.n;
    }
    out->nnz = nnz;
    out->col = (int32_t*)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
    out->val = (double*)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
    out->n_amb = namb;
    out->amb_row = (int64_t*)malloc(sizeof(int64_t) * (namb > 0 ? namb : 1));
    out->amb_col = (int32_t*)malloc(sizeof(int32_t) * (namb > 0 ? namb : 1));
    out->amb_kind = (int32_t*)malloc(sizeof(int32_t) * (namb > 0 ? namb : 1));
    int64_t p = 0, q = 0;
    for (int64_t r = 0; r < nsel; ++r) {
        out->row_ptr[r] = p;
        out->row_max[r] = rr[r].rowmax;
        out->row_cand[r] = rr[r].cand.n;
        double thr = tau * rr[r].rowmax;
        for (int64_t i = 0; i < rr[r].cand.n; ++i) {
            double D = rr[r].cand.val[i];
            if (D > 0.0 && D >= thr) {
                out->col[p] = rr[r].cand.col[i];
                out->val[p] = D;
                ++p;
            }
            if (thr > 0.0 && fabs(D / thr - 1.0) <= 1e-6) {
                out->amb_row[q] = r; out->amb_col[q] = rr[r].cand.col[i]; out->amb_kind[q] = 1; ++q;
            }
        }
        for (int64_t i = 0; i < rr[r].amb.n; ++i) {
            out->amb_row[q] = r; out->amb_col[q] = rr[r].amb.col[i]; out->amb_kind[q] = 2; ++q;
        }
        free(rr[r].cand.col); free(rr[r].cand.val); free(rr[r].amb.col); free(rr[r].amb.val);
    }
    out->row_ptr[nsel] = p;
    free(rr);
    return 0;
}

/* frames, entry/exit and table length for every row, 20 doubles per row:
 * S[3] e[3] x[3] z[3] tA tB theta hit n_table h a b sad 0 */
int or_beamlets(const or_grid* g, const or_beam* beams, int nbeams, double h_frac, double* out) {
    double dmin = g->dx < g->dy ? g->dx : g->dy;
    if (g->dz < dmin) dmin = g->dz;
    double h = h_frac * dmin;
    int64_t r = 0;
    for (int b = 0; b < nbeams; ++b)
        for (int iv = 0; iv < beams[b].n_v; ++iv)
            for (int iu = 0; iu < beams[b].n_u; ++iu, ++r) {
                or_beamlet bl;
                or_beamlet_setup(g, &beams[b], iu, iv, &bl);
                double* o = out + 20 * r;
                memcpy(o, bl.S, 3 * sizeof(double));
                memcpy(o + 3, bl.e, 3 * sizeof(double));
                memcpy(o + 6, bl.x, 3 * sizeof(double));
                memcpy(o + 9, bl.z, 3 * sizeof(double));
                o[12] = bl.tA; o[13] = bl.tB; o[14] = bl.theta; o[15] = bl.hit;
                o[16] = bl.hit ? (double)((int)ceil((bl.tB - bl.tA) / h) + 1) : 0.0;
                o[17] = h; o[18] = bl.a; o[19] = bl.b;
            }
    return 0;
}

/* depth table of one row (b, iu, iv): table_mode 0 the exact integral
 * (Siddon), 1 trilinear samples (trapezoid); returns n or -1 */
int or_row_table(const or_grid* g, const float* rho, const or_beam* bm, int iu, int iv, double h_frac,
                 int table_mode, double* out, int cap) {
    double dmin = g->dx < g->dy ? g->dx : g->dy;
    if (g->dz < dmin) dmin = g->dz;
    or_beamlet bl;
    or_beamlet_setup(g, bm, iu, iv, &bl);
    return table_mode == 1 ? or_depth_table_trilinear(g, rho, &bl, h_frac * dmin, out, cap)
                           : or_depth_table(g, rho, &bl, h_frac * dmin, out, cap);
}

/* D at arbitrary pencil-beam coordinates with the depth given (for pins):
 * returns T(d) (SAD/t)^2 F(x', d, z') */
double or_point_dose(const or_model* m, double xp, double zp, double t, double d, double sad, double a, double b) {
    double lut[4];
    or_lut_eval(m, d, lut);
    double a_t = a * t / sad, b_t = b * t / sad;
    return lut[0] * (sad / t) * (sad / t) * or_profile_F(m, lut + 1, xp, zp, a_t, b_t);
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

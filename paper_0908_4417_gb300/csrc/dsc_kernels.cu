// dsc_kernels.cu -- sm_103a kernels of the FSPB D_ij path.
//
//   k_setup          beamlet frames, entry/exit, VOI box and work items   (Section 2.1, Fig. 1)
//   k_siddon         radiological-depth table per beamlet, warp per ray   (Section 2.2, Siddon 1985)
//   k_count          candidate pairs per work item                        (VOI, Section 2.1)
//   k_eval           D_ij = T(d) (SAD/t)^2 F(x', d, z')  (persistent)     (Eq. 2-3)
//   k_beam_scale     per-beam maximum for BF16 storage
//   k_compact_count  kept pairs per item (D >= tau * row max)
//   k_compact_write  CSR columns/values, ascending voxel index
//   k_scan_*         device-wide exclusive scans with device-side length
//
// The evaluation is FP32 with compensated (float-float) voxel coordinates:
// every x-line of voxels gets its s = t - t_A, x' and z' at ix = 0 in
// float-float, and a candidate at ix adds ix times a float-float slope with
// FMAs, so position errors stay near ulp(value) instead of ulp(SAD).  FP64 is
// used only in the per-beamlet set-up and for Siddon's plane-crossing
// parameters alpha.
#include "dsc_internal.h"
#include "dsc_erfc_coeffs.h"

#include <cuda_bf16.h>
#include <math_constants.h>

namespace dsc {

// ---------------------------------------------------------------------------
// float-float arithmetic (error-free transformations; intrinsics keep the
// compiler from contracting them into FMAs)
// ---------------------------------------------------------------------------
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, lo);
}
// a * n for an integer n (exact in FP32)
__device__ __forceinline__ ff ff_mul_i(ff a, float n) {
  float p = __fmul_rn(a.hi, n);
  float e = fmaf(a.hi, n, -p);
  e = fmaf(a.lo, n, e);
  return quick_two_sum(p, e);
}
__host__ __device__ inline ff ff_from_double(double v) {
  float hi = (float)v;
  float lo = (float)(v - (double)hi);
  return {hi, lo};
}

// ---------------------------------------------------------------------------
// k_setup: one thread per beamlet row (FP64; a few thousand rows)
// ---------------------------------------------------------------------------
__device__ inline void normalize3(double* v) {
  double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n; v[1] /= n; v[2] /= n;
}
__device__ inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

__global__ void k_setup(const DInst* __restrict__ inst, const DBeam* __restrict__ beams, int nbeams, DRow* rows,
                        int nrows, int* row_items, int target_cand) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int lo = 0, hi = nbeams - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (beams[mid].row_base <= r) lo = mid; else hi = mid - 1;
  }
  const DBeam B = beams[lo];
  const DInst G = inst[B.inst];
  DRow R;
  R.inst = B.inst;
  R.beam = lo;
  int local = r - B.row_base;
  int iv = local / B.n_u, iu = local - iv * B.n_u;

  // beam and beamlet frames (Fig. 1): S = I + SAD (sin g, -cos g, 0), u = (cos g, sin g, 0), v = z
  double sg, cg;
  sincospi(B.gantry_deg / 180.0, &sg, &cg);
  double S[3] = {B.iso[0] + B.sad * sg, B.iso[1] - B.sad * cg, B.iso[2]};
  double u[3] = {cg, sg, 0.0};
  double uc = (iu + 0.5 - 0.5 * B.n_u) * B.a;
  double vc = (iv + 0.5 - 0.5 * B.n_v) * B.b;
  double e[3] = {B.iso[0] + uc * u[0] - S[0], B.iso[1] + uc * u[1] - S[1], B.iso[2] + vc - S[2]};
  normalize3(e);
  double pu = dot3(u, e);
  double x[3] = {u[0] - pu * e[0], u[1] - pu * e[1], u[2] - pu * e[2]};
  normalize3(x);
  double z[3] = {-e[2] * e[0] - x[2] * x[0], -e[2] * e[1] - x[2] * x[1], 1.0 - e[2] * e[2] - x[2] * x[2]};
  normalize3(z);
  for (int k = 0; k < 3; ++k) {
    R.S[k] = S[k]; R.e[k] = e[k]; R.x[k] = x[k]; R.z[k] = z[k];
    R.inv_e[k] = e[k] != 0.0 ? 1.0 / e[k] : 0.0;
  }

  // entry A / exit B on the grid prism (slab method)
  double blo[3] = {G.ox, G.oy, G.oz};
  double bhi[3] = {G.ox + G.nx * G.dx, G.oy + G.ny * G.dy, G.oz + G.nz * G.dz};
  double t0 = -CUDART_INF, t1 = CUDART_INF;
  bool hit = true;
  for (int k = 0; k < 3; ++k) {
    if (e[k] == 0.0) {
      if (S[k] < blo[k] || S[k] > bhi[k]) hit = false;
      continue;
    }
    double ta = (blo[k] - S[k]) / e[k], tb = (bhi[k] - S[k]) / e[k];
    if (ta > tb) { double s = ta; ta = tb; tb = s; }
    t0 = fmax(t0, ta);
    t1 = fmin(t1, tb);
  }
  if (t0 < 0.0) t0 = 0.0;
  if (!(t1 > t0)) hit = false;
  R.hit = hit;
  R.tA = hit ? t0 : 0.0;
  R.tB = hit ? t1 : 0.0;
  R.tA_f = (float)R.tA;
  R.n_table = hit ? (int)ceil((R.tB - R.tA) / G.hd) + 1 : 0;

  // voxel-loop constants: w0 = centre of voxel (0,0,0) - S
  double w0[3] = {G.ox + 0.5 * G.dx - S[0], G.oy + 0.5 * G.dy - S[1], G.oz + 0.5 * G.dz - S[2]};
  double sp[3] = {G.dx, G.dy, G.dz};
  R.S0 = ff_from_double(dot3(w0, e) - R.tA);
  R.X0 = ff_from_double(dot3(w0, x));
  R.Z0 = ff_from_double(dot3(w0, z));
  for (int k = 0; k < 3; ++k) {
    R.Ss[k] = ff_from_double(sp[k] * e[k]);
    R.Xs[k] = ff_from_double(sp[k] * x[k]);
    R.Zs[k] = ff_from_double(sp[k] * z[k]);
  }
  R.sad = (float)B.sad;
  R.a_sad = (float)(B.a / B.sad);
  R.b_sad = (float)(B.b / B.sad);
  double kx, kz, bx, bz;
  if (G.cutoff_mode == 0) { kx = 3.0 * B.a / B.sad; kz = 3.0 * B.b / B.sad; bx = bz = 0.0; }
  else if (G.cutoff_mode == 1) {
    kx = 0.5 * B.a / B.sad; kz = 0.5 * B.b / B.sad;
    bx = bz = (double)G.cutoff_k * (double)G.c3max;
  } else { kx = kz = 0.0; bx = bz = 0.0; }
  R.kx = (float)kx; R.kz = (float)kz; R.bx = (float)bx; R.bz = (float)bz;

  // voxel box of the VOI: between the smallest and largest t of the grid
  // corners the VOI is the hull of its two end rectangles
  int ix0 = 0, ix1 = G.nx - 1, iy0 = 0, iy1 = G.ny - 1, iz0 = 0, iz1 = G.nz - 1;
  double w_mid = 0.0;
  if (hit && G.cutoff_mode != 2) {
    double tlo = CUDART_INF, thi = -CUDART_INF;
    for (int c = 0; c < 8; ++c) {
      double p[3] = {(c & 1) ? bhi[0] : blo[0], (c & 2) ? bhi[1] : blo[1], (c & 4) ? bhi[2] : blo[2]};
      double w[3] = {p[0] - S[0], p[1] - S[1], p[2] - S[2]};
      double t = dot3(w, e);
      tlo = fmin(tlo, t);
      thi = fmax(thi, t);
    }
    tlo = fmax(tlo, 0.0);
    double lo3[3] = {CUDART_INF, CUDART_INF, CUDART_INF}, hi3[3] = {-CUDART_INF, -CUDART_INF, -CUDART_INF};
    for (int c = 0; c < 8; ++c) {
      double t = (c & 1) ? thi : tlo;
      double hx = kx * t + bx, hz = kz * t + bz;
      double su = (c & 2) ? hx : -hx, sv = (c & 4) ? hz : -hz;
      for (int k = 0; k < 3; ++k) {
        double p = S[k] + t * e[k] + su * x[k] + sv * z[k];
        lo3[k] = fmin(lo3[k], p);
        hi3[k] = fmax(hi3[k], p);
      }
    }
    ix0 = max(ix0, (int)floor((lo3[0] - G.ox) / G.dx - 0.5) - 1);
    ix1 = min(ix1, (int)ceil((hi3[0] - G.ox) / G.dx - 0.5) + 1);
    iy0 = max(iy0, (int)floor((lo3[1] - G.oy) / G.dy - 0.5) - 1);
    iy1 = min(iy1, (int)ceil((hi3[1] - G.oy) / G.dy - 0.5) + 1);
    iz0 = max(iz0, (int)floor((lo3[2] - G.oz) / G.dz - 0.5) - 1);
    iz1 = min(iz1, (int)ceil((hi3[2] - G.oz) / G.dz - 0.5) + 1);
    w_mid = 2.0 * (fmax(kx, kz) * 0.5 * (tlo + thi) + fmax(bx, bz));
  }
  R.ix0 = ix0; R.ix1 = ix1; R.iy0 = iy0; R.iy1 = iy1; R.iz0 = iz0; R.iz1 = iz1;
  long long lines = 0;
  if (hit && ix1 >= ix0 && iy1 >= iy0 && iz1 >= iz0) lines = (long long)(iy1 - iy0 + 1) * (iz1 - iz0 + 1);
  // expected candidates on one x-line: the VOI width over the sine of the
  // angle between the axis and x, at most the box's x extent
  double nxb = (double)(ix1 - ix0 + 1);
  double est = nxb;
  if (G.cutoff_mode != 2) {
    double sn = sqrt(fmax(1.0 - e[0] * e[0], 1e-6));
    est = fmin(nxb, fmax(1.0, w_mid / (sn * G.dx)));
  }
  int lpc = (int)fmin((double)kMaxLinesPerItem, fmax(1.0, (double)target_cand / est));
  R.lpc = lpc;
  R.nitems = (int)((lines + lpc - 1) / lpc);
  rows[r] = R;
  row_items[r] = R.nitems;
}

// ---------------------------------------------------------------------------
// k_siddon: radiological depth table, one warp per beamlet axis.
// Lane l walks table intervals [l Q, (l+1) Q) with Siddon's incremental
// plane crossings (alpha in FP64), stores its lane-local cumulative depth,
// then adds the warp-exclusive prefix of the lane totals.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kSiddonWarps) k_siddon(const DInst* __restrict__ inst,
                                                              const DRow* __restrict__ rows, int nrows,
                                                              float* __restrict__ tables, int stride) {
  int warp = blockIdx.x * kSiddonWarps + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  const DRow& R = rows[warp];
  int n = R.n_table;
  if (n <= 0) return;
  const DInst& G = inst[R.inst];
  float* tab = tables + (size_t)warp * stride;
  if (lane == 0) tab[0] = 0.0f;
  int nint = n - 1;                                  // intervals
  int Q = (nint + 31) >> 5;
  int k0 = min(lane * Q, nint), k1 = min(k0 + Q, nint);
  const double L = R.tB - R.tA;
  const double h = G.hd;
  const double* S = R.S;
  const double* e = R.e;
  const double org[3] = {G.ox, G.oy, G.oz};
  const double sp[3] = {G.dx, G.dy, G.dz};
  const double isp[3] = {G.idx, G.idy, G.idz};
  const int nv[3] = {G.nx, G.ny, G.nz};
  double total = 0.0;
  if (k0 < k1) {
    double tcur = R.tA + fmin(k0 * h, L);
    int idx[3], step[3];
    double alpha[3], dalpha[3];
    for (int a = 0; a < 3; ++a) {
      double p = fma(tcur, e[a], S[a]);
      int i = (int)floor((p - org[a]) * isp[a]);
      idx[a] = min(max(i, 0), nv[a] - 1);
      const double ie = R.inv_e[a];
      if (e[a] > 0.0) {
        step[a] = 1;
        alpha[a] = (org[a] + (idx[a] + 1) * sp[a] - S[a]) * ie;
        dalpha[a] = sp[a] * ie;
      } else if (e[a] < 0.0) {
        step[a] = -1;
        alpha[a] = (org[a] + idx[a] * sp[a] - S[a]) * ie;
        dalpha[a] = -sp[a] * ie;
      } else {
        step[a] = 0;
        alpha[a] = CUDART_INF;
        dalpha[a] = 0.0;
      }
    }
    const float* rho = G.rho;
    const size_t sy = (size_t)G.nx, sz = (size_t)G.nx * G.ny;
    int guard = 4 * (G.nx + G.ny + G.nz) + 8 * (k1 - k0) + 16;
    for (int k = k0; k < k1; ++k) {
      double tend = (k + 1 == nint) ? R.tB : R.tA + fmin((k + 1) * h, L);
      for (;;) {
        double am = fmin(alpha[0], fmin(alpha[1], alpha[2]));
        if (am >= tend || --guard < 0) break;
        double len = fmax(am - tcur, 0.0);
        total = fma(len, (double)__ldg(rho + idx[0] + idx[1] * sy + idx[2] * sz), total);
        tcur = fmax(tcur, am);
        int a = (alpha[0] == am) ? 0 : ((alpha[1] == am) ? 1 : 2);
        idx[a] = min(max(idx[a] + step[a], 0), nv[a] - 1);
        alpha[a] += dalpha[a];
      }
      double len = fmax(tend - tcur, 0.0);
      total = fma(len, (double)__ldg(rho + idx[0] + idx[1] * sy + idx[2] * sz), total);
      tcur = fmax(tcur, tend);
      tab[k + 1] = (float)total;                     // lane-local, fixed below
    }
  }
  // exclusive prefix of the lane totals
  double incl = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  double prefix = incl - total;
  for (int k = k0; k < k1; ++k) tab[k + 1] = (float)(prefix + (double)tab[k + 1]);
}

// ---------------------------------------------------------------------------
// x-lines of a work item
// ---------------------------------------------------------------------------
struct LineSm {
  int lo[kMaxLinesPerItem];
  int colbase[kMaxLinesPerItem];      // nx (iy + ny iz) of the line
  int off[kMaxLinesPerItem + 1];
  float sh[kMaxLinesPerItem], sl[kMaxLinesPerItem];
  float xh[kMaxLinesPerItem], xl[kMaxLinesPerItem];
  float zh[kMaxLinesPerItem], zl[kMaxLinesPerItem];
  int wscan[kEvalThreads / 32];
  unsigned short map[kWindow];
  long long item;
  int row;
  int nl;
  int total;
};

// the candidate interval [lo, hi] of one x-line (iy, iz) of row R and its
// float-float s, x', z' at ix = 0
__device__ __forceinline__ int line_setup(const DRow& R, int mode, int nx, int iy, int iz, ff& s0, ff& x0, ff& z0,
                                          int& lo_out) {
  float fy = (float)iy, fz = (float)iz;
  s0 = ff_add(ff_add(R.S0, ff_mul_i(R.Ss[1], fy)), ff_mul_i(R.Ss[2], fz));
  x0 = ff_add(ff_add(R.X0, ff_mul_i(R.Xs[1], fy)), ff_mul_i(R.Xs[2], fz));
  z0 = ff_add(ff_add(R.Z0, ff_mul_i(R.Zs[1], fy)), ff_mul_i(R.Zs[2], fz));
  // t(i) = T0 + i tx, x'(i) = X0 + i xx, z'(i) = Z0 + i zx; constraints c i <= r
  float T0 = R.tA_f + s0.hi, tx = R.Ss[0].hi;
  float X0 = x0.hi, xx = R.Xs[0].hi, Z0 = z0.hi, zx = R.Zs[0].hi;
  float lo = 0.0f, hi = (float)(nx - 1);
  bool empty = false;
  auto constrain = [&](float c, float r) {
    if (c > 0.0f) hi = fminf(hi, __fdiv_rn(r, c));
    else if (c < 0.0f) lo = fmaxf(lo, __fdiv_rn(r, c));
    else if (r < 0.0f) empty = true;
  };
  if (mode != 2) {
    constrain(fmaf(-R.kx, tx, xx), fmaf(R.kx, T0, R.bx) - X0);
    constrain(fmaf(-R.kx, tx, -xx), fmaf(R.kx, T0, R.bx) + X0);
    constrain(fmaf(-R.kz, tx, zx), fmaf(R.kz, T0, R.bz) - Z0);
    constrain(fmaf(-R.kz, tx, -zx), fmaf(R.kz, T0, R.bz) + Z0);
  } else {
    // t > 0 (voxels in front of the source)
    if (tx > 0.0f) lo = fmaxf(lo, floorf(__fdiv_rn(-T0, tx)) + 1.0f);
    else if (tx < 0.0f) hi = fminf(hi, ceilf(__fdiv_rn(-T0, tx)) - 1.0f);
    else if (T0 <= 0.0f) empty = true;
  }
  int ilo = (int)ceilf(lo), ihi = (int)floorf(hi);
  lo_out = ilo;
  if (empty || ihi < ilo) return 0;
  return ihi - ilo + 1;
}

// row of an item: last r with row_item_base[r] <= item
__device__ __forceinline__ int row_of_item(const long long* __restrict__ base, int nrows, long long item) {
  int lo = 0, hi = nrows - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// block-wide exclusive scan of one int per thread (kEvalThreads threads); returns the total
__device__ __forceinline__ int block_excl_scan(int v, int& excl, int* wscan) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wscan[w] = incl;
  __syncthreads();
  int wpre = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < kEvalThreads / 32; ++i) {
    int s = wscan[i];
    if (i < w) wpre += s;
    tot += s;
  }
  __syncthreads();
  excl = wpre + incl - v;
  return tot;
}

// line (iy, iz) of line index l of row R
__device__ __forceinline__ void line_yz(const DRow& R, long long l, int& iy, int& iz) {
  int nyb = R.iy1 - R.iy0 + 1;
  iz = R.iz0 + (int)(l / nyb);
  iy = R.iy0 + (int)(l - (long long)(iz - R.iz0) * nyb);
}

// lines of a work item: [chunk * lpc, min(+lpc, lines of the row))
__device__ __forceinline__ int item_nlines(const DRow& R, long long chunk, long long& l0) {
  long long nlines = (long long)(R.iy1 - R.iy0 + 1) * (R.iz1 - R.iz0 + 1);
  l0 = chunk * R.lpc;
  return (int)min((long long)R.lpc, nlines - l0);
}

// set up all lines of an item in shared memory (each thread takes lines t and
// t + kEvalThreads); returns the candidate count
__device__ int item_lines(LineSm& sm, const DRow& R, int mode, int nx, int ny, long long chunk) {
  constexpr int per = kMaxLinesPerItem / kEvalThreads;
  long long l0;
  int nl = item_nlines(R, chunk, l0);
  int t = threadIdx.x;
  int len[per];
  int mine = 0;
#pragma unroll
  for (int q = 0; q < per; ++q) {
    int li = t * per + q;             // consecutive lines per thread keep the scan order
    len[q] = 0;
    if (li < nl) {
      int iy, iz;
      line_yz(R, l0 + li, iy, iz);
      ff s0, x0, z0;
      int lo;
      len[q] = line_setup(R, mode, nx, iy, iz, s0, x0, z0, lo);
      sm.lo[li] = lo;
      sm.colbase[li] = nx * (iy + ny * iz);
      sm.sh[li] = s0.hi; sm.sl[li] = s0.lo;
      sm.xh[li] = x0.hi; sm.xl[li] = x0.lo;
      sm.zh[li] = z0.hi; sm.zl[li] = z0.lo;
    }
    mine += len[q];
  }
  int excl;
  int tot = block_excl_scan(mine, excl, sm.wscan);
#pragma unroll
  for (int q = 0; q < per; ++q) {
    int li = t * per + q;
    if (li < nl) sm.off[li] = excl;
    excl += len[q];
  }
  if (t == 0) { sm.nl = nl; sm.off[nl] = tot; }
  __syncthreads();
  return tot;
}

// line index of every candidate in [w0, w0 + wl): mark line starts, then an
// inclusive max-scan over the window
__device__ void item_map(LineSm& sm, int w0, int wl) {
  constexpr int per = kWindow / kEvalThreads;
  int t = threadIdx.x;
  int nl = sm.nl;
  int base = t * per;
  int mk[per];
#pragma unroll
  for (int j = 0; j < per; ++j) mk[j] = -1;
  // scatter the starts into a shared buffer (the map itself as scratch)
  for (int j = t; j < kWindow; j += kEvalThreads) sm.map[j] = 0xffff;
  __syncthreads();
  for (int li = t; li < nl; li += kEvalThreads) {
    int o = sm.off[li], e = sm.off[li + 1];
    if (e > o) {
      if (o >= w0 && o < w0 + wl) sm.map[o - w0] = (unsigned short)li;
      else if (o < w0 && e > w0) sm.map[0] = (unsigned short)li;
    }
  }
  __syncthreads();
  int run = -1;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    int v = sm.map[base + j];
    if (v != 0xffff) run = v;
    mk[j] = run;
  }
  // warp inclusive max-scan of the per-thread last value, then across warps
  int lane = t & 31, w = t >> 5;
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl = max(incl, v);
  }
  if (lane == 31) sm.wscan[w] = incl;
  __syncthreads();
  int wpre = -1;
#pragma unroll
  for (int i = 0; i < kEvalThreads / 32; ++i)
    if (i < w) wpre = max(wpre, sm.wscan[i]);
  int excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = -1;
  int carry = max(wpre, excl);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < per; ++j) sm.map[base + j] = (unsigned short)max(mk[j], carry);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// k_count: candidate pairs per work item, one warp per item
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEvalThreads) k_count(const DInst* __restrict__ inst, const DRow* __restrict__ rows,
                                                        const long long* __restrict__ row_item_base, int nrows,
                                                        const long long* __restrict__ n_items, int* item_cand) {
  const long long ni = *n_items;
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (kEvalThreads / 32);
  for (long long item = blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5); item < ni; item += nw) {
    int row = row_of_item(row_item_base, nrows, item);
    const DRow& R = rows[row];
    const DInst& G = inst[R.inst];
    long long l0;
    int nl = item_nlines(R, item - row_item_base[row], l0);
    int cnt = 0;
    for (int li = lane; li < nl; li += 32) {
      int iy, iz;
      line_yz(R, l0 + li, iy, iz);
      ff s0, x0, z0;
      int lo;
      cnt += line_setup(R, G.cutoff_mode, G.nx, iy, iz, s0, x0, z0, lo);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) item_cand[item] = cnt;
  }
}

// ---------------------------------------------------------------------------
// FSPB evaluation (Eq. 2-3)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// erfc(u) for u >= 0, given v = u sqrt(log2 e):  t exp(-u^2) P(t) with
// t = 1/(1 + p u) (coefficients from fit_erfc.py) and exp(-u^2) = 2^(-v^2),
// v^2 split exactly into vh + vl so the exponent carries no rounding
__device__ __forceinline__ float erfc_v(float v) {
  constexpr float kInvSqrtL = 0.83255461115769775635f;   // 1 / sqrt(log2 e)
  constexpr float kLn2 = 0.69314718055994530942f;
  float t = rcp_approx(fmaf(kErfcP * kInvSqrtL, v, 1.0f));
  float p = kErfcC[kErfcN];
#pragma unroll
  for (int k = kErfcN - 1; k >= 0; --k) p = fmaf(p, t, kErfcC[k]);
  float vh = __fmul_rn(v, v);
  float vl = fmaf(v, v, -vh);
  float e = ex2_approx(-vh);
  e = fmaf(e, -vl * kLn2, e);
  return (t * p) * e;
}

// erf(u1) + erf(u2) for u1 = (h - |x'|)/s, u2 = (h + |x'|)/s (h >= 0), from
// the scaled arguments v = u sqrt(log2 e): inside the beamlet
// 2 - erfc(u1) - erfc(u2), outside erfc(|u1|) - erfc(u2) (no cancellation of
// 1 - erf in the tails)
__device__ __forceinline__ float erf_pair(float h, float ax, float inv_s) {
  float v1 = (h - ax) * inv_s;
  float v2 = (h + ax) * inv_s;
  float e1 = erfc_v(fabsf(v1));
  float e2 = erfc_v(v2);
  return v1 >= 0.0f ? (2.0f - e1) - e2 : e1 - e2;
}

struct RowConst {
  ff Sx;            // slope of s per ix
  float Xxh, Xxl, Zxh, Zxl;
  float tA, h, inv_h, sad, a_sad, b_sad;
  float kx, kz, bx, bz;
  int n_table;
};

// D for candidate ix of a line; returns -1 outside the SIGMA cutoff
__device__ __forceinline__ float eval_pair(const RowConst& C, const DInst& G, const float* __restrict__ tab,
                                           float fi, float sh, float sl, float xh, float xl, float zh, float zl,
                                           int mode) {
  // s = t - tA in float-float
  float ph = __fmul_rn(fi, C.Sx.hi);
  float pl = fmaf(fi, C.Sx.hi, -ph);
  ff a = two_sum(sh, ph);
  float s_lo = __fadd_rn(a.lo, __fadd_rn(pl, fmaf(fi, C.Sx.lo, sl)));
  float s_hi = a.hi;
  float xp = fmaf(fi, C.Xxh, xh) + fmaf(fi, C.Xxl, xl);
  float zp = fmaf(fi, C.Zxh, zh) + fmaf(fi, C.Zxl, zl);
  float t = s_hi + C.tA;

  // radiological depth at O' (Section 2.2): linear interpolation of the table
  float d;
  if (s_hi + s_lo <= 0.0f) {
    d = 0.0f;
  } else {
    float kf = floorf(s_hi * C.inv_h);
    float khh = __fmul_rn(kf, C.h);
    float khl = fmaf(kf, C.h, -khh);
    float r = __fadd_rn(__fsub_rn(__fsub_rn(s_hi, khh), khl), s_lo);
    if (r < 0.0f) { kf -= 1.0f; r += C.h; }
    else if (r >= C.h) { kf += 1.0f; r -= C.h; }
    int k = (int)kf;
    if (k >= C.n_table - 1) {
      d = __ldg(tab + C.n_table - 1);
    } else {
      k = max(k, 0);
      float f = r * C.inv_h;
      float d0 = __ldg(tab + k), d1 = __ldg(tab + k + 1);
      d = fmaf(f, d1 - d0, d0);
    }
  }
  // beam-model table: T(d), c3_1..3(d)
  float g = fmaxf(d * G.lut_scale, 0.0f);   // also maps a NaN depth to 0
  float4 P;
  if (g >= (float)(G.n_lut - 1)) {
    P = __ldg(G.lut + G.n_lut - 1);
  } else {
    float kl = floorf(g);
    float w = g - kl;
    int k = (int)kl;
    float4 A = __ldg(G.lut + k), B = __ldg(G.lut + k + 1);
    P.x = fmaf(w, B.x - A.x, A.x);
    P.y = fmaf(w, B.y - A.y, A.y);
    P.z = fmaf(w, B.z - A.z, A.z);
    P.w = fmaf(w, B.w - A.w, A.w);
  }
  float a_t = C.a_sad * t, b_t = C.b_sad * t;
  float ax = fabsf(xp), az = fabsf(zp);
  if (mode == 1) {
    float lim = G.cutoff_k * P.y;
    if (ax > fmaf(0.5f, a_t, lim) || az > fmaf(0.5f, b_t, lim)) return -1.0f;
  }
  // Eq. 3: three erf-pair products; arguments scaled by sqrt(log2 e):
  // 1/(sqrt(2) c3) * sqrt(log2 e) = sqrt(log2(e)/2) / c3
  constexpr float kSqrtHalfL = 0.84932180028801904272f;
  float c3[3] = {P.y, P.z, P.w};
  float F = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float inv_s = kSqrtHalfL * __frcp_rn(c3[i]);
    float X = erf_pair(G.c2h[i] * a_t, ax, inv_s);
    float Z = erf_pair(G.c2h[i] * b_t, az, inv_s);
    F = fmaf(G.c1q[i] * X, Z, F);
  }
  // Eq. 2 with A = T(d) (SAD/t)^2
  float q = __fdiv_rn(C.sad, t);
  return P.x * (q * q) * F;
}

__device__ __forceinline__ void load_row_const(RowConst& C, const DRow& R, const DInst& G) {
  C.Sx = R.Ss[0];
  C.Xxh = R.Xs[0].hi; C.Xxl = R.Xs[0].lo;
  C.Zxh = R.Zs[0].hi; C.Zxl = R.Zs[0].lo;
  C.tA = R.tA_f;
  C.h = G.h;
  C.inv_h = G.inv_h;
  C.sad = R.sad;
  C.a_sad = R.a_sad;
  C.b_sad = R.b_sad;
  C.kx = R.kx; C.kz = R.kz; C.bx = R.bx; C.bz = R.bz;
  C.n_table = R.n_table;
}

// persistent: CTAs take work items from a queue; every candidate's D goes to
// vals[item_off[item] + k] and the row maximum is kept with atomicMax on the
// float bits (D >= 0)
__global__ void __launch_bounds__(kEvalThreads) k_eval(EvalParams p) {
  __shared__ LineSm sm;
  const long long ni = *p.n_items;
  for (;;) {
    if (threadIdx.x == 0) {
      long long it = atomicAdd(p.item_counter, 1);
      sm.item = it;
      if (it < ni) sm.row = row_of_item(p.row_item_base, p.nrows, it);
    }
    __syncthreads();
    const long long item = sm.item;
    if (item >= ni) break;
    const int row = sm.row;
    const DRow& R = p.rows[row];
    const DInst& G = p.inst[R.inst];
    const int mode = G.cutoff_mode;
    const int total = item_lines(sm, R, mode, G.nx, G.ny, item - p.row_item_base[row]);
    RowConst C;
    load_row_const(C, R, G);
    const float* tab = p.tables + (size_t)row * p.table_stride;
    float* out = p.vals + p.item_off[item];
    int* outc = p.cols + p.item_off[item];
    float vmax = 0.0f;
    for (int w0 = 0; w0 < total; w0 += kWindow) {
      int wl = min(kWindow, total - w0);
      item_map(sm, w0, wl);
      for (int j = threadIdx.x; j < wl; j += kEvalThreads) {
        int li = min((int)sm.map[j], sm.nl - 1);
        int ix = sm.lo[li] + (w0 + j - sm.off[li]);
        float D = eval_pair(C, G, tab, (float)ix, sm.sh[li], sm.sl[li], sm.xh[li], sm.xl[li], sm.zh[li], sm.zl[li],
                            mode);
        out[w0 + j] = D;
        outc[w0 + j] = sm.colbase[li] + ix;
        vmax = fmaxf(vmax, D);
      }
      __syncthreads();
    }
    // block max -> row max
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0 && vmax > 0.0f) atomicMax(p.row_max + row, __float_as_uint(vmax));
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// per-beam scale for BF16 storage: s_b = max over the beam's rows
// ---------------------------------------------------------------------------
__global__ void k_beam_scale(const DBeam* __restrict__ beams, int nbeams, const unsigned* __restrict__ row_max,
                             const OutSlot* __restrict__ slot) {
  float* beam_scale = slot->beam_scale;
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbeams) return;
  const DBeam B = beams[b];
  int n = B.n_u * B.n_v;
  float m = 0.0f;
  for (int r = 0; r < n; ++r) m = fmaxf(m, __uint_as_float(row_max[B.row_base + r]));
  beam_scale[b] = m > 0.0f ? m : 1.0f;
}

// ---------------------------------------------------------------------------
// compaction: kept = D > 0 and D >= tau * row max
// ---------------------------------------------------------------------------


// kept = D > 0 and D >= tau * row max; one warp per item, 8 loads in
// flight per lane
__global__ void __launch_bounds__(kEvalThreads) k_compact_count(CompactParams p) {
  const long long ni = *p.n_items;
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (kEvalThreads / 32);
  for (long long item = blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5); item < ni; item += nw) {
    int row = row_of_item(p.row_item_base, p.nrows, item);
    float thr = p.tau * __uint_as_float(p.row_max[row]);
    long long a = p.item_off[item], b = p.item_off[item + 1];
    int kept = 0, valid = 0;
    for (long long i0 = a; i0 < b; i0 += 8 * 32) {
      float D[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        long long i = i0 + u * 32 + lane;
        D[u] = i < b ? __ldcs(p.vals + i) : -1.0f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        kept += (D[u] > 0.0f && D[u] >= thr);
        valid += (D[u] >= 0.0f);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kept += __shfl_xor_sync(0xffffffffu, kept, o);
      valid += __shfl_xor_sync(0xffffffffu, valid, o);
    }
    if (lane == 0) {
      p.item_kept[item] = kept;
      if (valid) atomicAdd((unsigned long long*)(p.row_cand + row), (unsigned long long)valid);
    }
  }
}

// CSR columns and values: each warp compacts one item in candidate order
// (ascending voxel index) with ballots; 8 x 32 candidates per round
__global__ void __launch_bounds__(kEvalThreads) k_compact_write(CompactParams p) {
  const long long ni = *p.n_items;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long nw = (long long)gridDim.x * (kEvalThreads / 32);
  int* col = p.slot->col;
  void* valp = p.slot->val;
  for (long long item = blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5); item < ni; item += nw) {
    int row = row_of_item(p.row_item_base, p.nrows, item);
    float thr = p.tau * __uint_as_float(p.row_max[row]);
    float scale = 1.0f;
    if (p.value_dtype == 1) scale = p.slot->beam_scale[p.rows[row].beam];
    long long a = p.item_off[item], b = p.item_off[item + 1];
    long long o = p.item_out[item];
    for (long long i0 = a; i0 < b; i0 += 8 * 32) {
      float D[8];
      int C[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        long long i = i0 + u * 32 + lane;
        D[u] = i < b ? __ldcs(p.vals + i) : -1.0f;
        C[u] = i < b ? __ldcs(p.cols + i) : 0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        bool keep = D[u] > 0.0f && D[u] >= thr;
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          long long q = o + __popc(m & lt);
          col[q] = C[u];
          if (p.value_dtype == 1)
            ((__nv_bfloat16*)valp)[q] = __float2bfloat16_rn(__fdiv_rn(D[u], scale));
          else
            ((float*)valp)[q] = D[u];
        }
        o += __popc(m);
      }
    }
  }
}

// CSR row pointers of one instance (rows [row_base, row_base + nrows)),
// relative to the instance's first output slot, which goes to inst_begin
__global__ void k_row_ptr(const long long* __restrict__ row_item_base, const long long* __restrict__ item_out,
                          int row_base, int nrows, long long rp_off, int inst, int last,
                          const OutSlot* __restrict__ slot) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  long long b = item_out[row_item_base[row_base]];
  if (r <= nrows) slot->row_ptr[rp_off + r] = item_out[row_item_base[row_base + r]] - b;
  if (r == 0) {
    slot->inst_begin[inst] = b;
    if (last) slot->inst_begin[inst + 1] = item_out[row_item_base[row_base + nrows]];
  }
}

// per-row statistics into the result
__global__ void k_copy_stats(const unsigned* __restrict__ row_max, const long long* __restrict__ row_cand, int nrows,
                             const OutSlot* __restrict__ slot) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrows) {
    slot->row_max[r] = row_max[r];
    slot->row_cand[r] = row_cand[r];
  }
}

// ---------------------------------------------------------------------------
// device-wide exclusive scan: out[0..n] with out[n] = total; n is read from
// device memory so the launch sequence needs no host round trip
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) k_scan_partial(const int* __restrict__ in, const long long* n_ptr,
                                                                long long n_const, long long* block_sums) {
  long long n = n_ptr ? *n_ptr : n_const;
  long long seg = (n + kScanBlocks - 1) / kScanBlocks;
  long long a = blockIdx.x * seg, b = min(a + seg, n);
  long long s = 0;
  for (long long i = a + threadIdx.x; i < b; i += kScanThreads) s += (long long)in[i];
  __shared__ long long ws[kScanThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < kScanThreads / 32; ++i) t += ws[i];
    block_sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kScanBlocks) k_scan_blocks(long long* block_sums) {
  __shared__ long long ws[kScanBlocks / 32];
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  long long v = block_sums[t];
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) ws[w] = incl;
  __syncthreads();
  if (w == 0) {
    long long s = ws[lane];
    long long si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long x = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += x;
    }
    ws[lane] = si - s;
    if (lane == 31) block_sums[kScanBlocks] = si;
  }
  __syncthreads();
  block_sums[t] = ws[w] + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const int* __restrict__ in, const long long* n_ptr,
                                                              long long n_const, const long long* block_sums,
                                                              long long* out) {
  long long n = n_ptr ? *n_ptr : n_const;
  long long seg = (n + kScanBlocks - 1) / kScanBlocks;
  long long a = blockIdx.x * seg, b = min(a + seg, n);
  __shared__ long long ws[kScanThreads / 32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = block_sums[blockIdx.x];
  __syncthreads();
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long long c = a; c < b; c += kScanThreads) {
    long long i = c + threadIdx.x;
    long long v = (i < b) ? (long long)in[i] : 0;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    long long wpre = 0, tot = 0;
    for (int k = 0; k < kScanThreads / 32; ++k) {
      if (k < w) wpre += ws[k];
      tot += ws[k];
    }
    if (i < b) out[i] = carry + wpre + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = block_sums[kScanBlocks];
}


}  // namespace dsc

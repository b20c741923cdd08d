// dsc_kernels.cu -- sm_103a kernels of the FSPB D_ij path.
//
//   k_setup          beamlet frames, entry/exit, VOI box and work items   (Section 2.1, Fig. 1)
//   k_siddon         radiological-depth table per beamlet, warp per ray   (Section 2.2, Siddon 1985)
//   k_count          candidate pairs per work item                        (VOI, Section 2.1)
//   k_eval           D_ij = T(d) (SAD/t)^2 F(x', d, z')  (persistent)     (Eq. 2-3)
//   k_beam_scale     per-beam maximum for BF16 storage
//   k_tile_count     kept entries (D >= tau * row max) per tile of candidates;
//                    lists the values too close to their threshold or row
//                    maximum for FP32 to decide (k_refine in dsc_refine.cu)
//   k_tile_write     CSR columns/values of the kept entries, tile by tile
//   k_row_ptr        CSR row pointers per instance
//   k_scan_*         device-wide exclusive scans with device-side length
//   k_tail_probe     a profile's tail as the evaluation computes it (tests)
//
// The evaluation is FP32 with compensated (float-float) voxel coordinates:
// every x-line of voxels gets its s = t - t_A, x' and z' at ix = 0 in
// float-float, and a candidate at ix adds ix times a float-float slope with
// FMAs, so position errors stay near ulp(value) instead of ulp(SAD).  FP64 is
// used only in the per-beamlet set-up, for Siddon's plane-crossing parameters
// alpha, and in the re-evaluation of the few pairs FP32 cannot decide.
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
                        int nrows, int* row_items, int target_cand, StepClear clr) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  if (clr.row_max) {
    clr.row_max[r] = 0u;
    clr.row_cand[r] = 0;
    clr.mcount[r] = 0;
    if (r == 0) {
      for (int k = 0; k < 4; ++k) { clr.counter[k] = 0; clr.rcount[k] = 0ull; }
      if (clr.ord_cnt)
        for (int k = 0; k < kOrderClasses; ++k) clr.ord_cnt[k] = 0;
    }
  }
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
  {
    // fixed-point constants of the Siddon walk: the unit 2^-q mm keeps t_B
    // (plus one plane step) below 2^60 units; q <= 48 (3.6e-15 mm)
    double tmax = R.tB + fmax(G.dx, fmax(G.dy, G.dz)) * 2.0 + 1.0;
    // ceil(log2(tmax)) from the exponent bits (tmax >= 1): the exponent, one
    // more when the mantissa has any bit set; 2^q built the same way
    const long long tb = __double_as_longlong(tmax);
    const int cl2 = (int)((tb >> 52) & 0x7ff) - 1023 + ((tb & 0xfffffffffffffll) != 0);
    int q = min(max(60 - cl2, 0), 48);
    double fx = __longlong_as_double((long long)(q + 1023) << 52);
    R.fix_q = q;
    R.fx_tA = __double2ll_rn(R.tA * fx);
    R.fx_tB = __double2ll_rn(R.tB * fx);
    R.fx_h = __double2ll_rn(G.hd * fx);
  }

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
  {
    const double u = 4294967296.0 / G.hd;          // fixed-point units per mm (2^32 / h)
    R.sfx0 = __double2ll_rn((dot3(w0, e) - R.tA) * u);
    for (int k = 0; k < 3; ++k) R.sfx_s[k] = __double2ll_rn(sp[k] * e[k] * u);
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
  // corners the VOI is the hull of its two end rectangles.  FP32: the box
  // has a voxel of slack on every side, far above this rounding, and only
  // bounds the lines that are tested.
  int ix0 = 0, ix1 = G.nx - 1, iy0 = 0, iy1 = G.ny - 1, iz0 = 0, iz1 = G.nz - 1;
  float w_mid = 0.0f;
  if (hit && G.cutoff_mode != 2) {
    const float Sf[3] = {(float)S[0], (float)S[1], (float)S[2]};
    const float ef[3] = {(float)e[0], (float)e[1], (float)e[2]};
    const float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
    const float zf[3] = {(float)z[0], (float)z[1], (float)z[2]};
    const float blf[3] = {(float)blo[0], (float)blo[1], (float)blo[2]};
    const float bhf[3] = {(float)bhi[0], (float)bhi[1], (float)bhi[2]};
    const float kxf = (float)kx, kzf = (float)kz, bxf = (float)bx, bzf = (float)bz;
    float tlo = CUDART_INF_F, thi = -CUDART_INF_F;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float p0 = (c & 1) ? bhf[0] : blf[0], p1 = (c & 2) ? bhf[1] : blf[1], p2 = (c & 4) ? bhf[2] : blf[2];
      const float t = (p0 - Sf[0]) * ef[0] + (p1 - Sf[1]) * ef[1] + (p2 - Sf[2]) * ef[2];
      tlo = fminf(tlo, t);
      thi = fmaxf(thi, t);
    }
    tlo = fmaxf(tlo, 0.0f);
    float lo3[3] = {CUDART_INF_F, CUDART_INF_F, CUDART_INF_F}, hi3[3] = {-CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float t = (c & 1) ? thi : tlo;
      const float hx = kxf * t + bxf, hz = kzf * t + bzf;
      const float su = (c & 2) ? hx : -hx, sv = (c & 4) ? hz : -hz;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float p = Sf[k] + t * ef[k] + su * xf[k] + sv * zf[k];
        lo3[k] = fminf(lo3[k], p);
        hi3[k] = fmaxf(hi3[k], p);
      }
    }
    const float dxi = __frcp_rn((float)G.dx), dyi = __frcp_rn((float)G.dy), dzi = __frcp_rn((float)G.dz);
    ix0 = max(ix0, (int)floorf((lo3[0] - blf[0]) * dxi - 0.5f) - 1);
    ix1 = min(ix1, (int)ceilf((hi3[0] - blf[0]) * dxi - 0.5f) + 1);
    iy0 = max(iy0, (int)floorf((lo3[1] - blf[1]) * dyi - 0.5f) - 1);
    iy1 = min(iy1, (int)ceilf((hi3[1] - blf[1]) * dyi - 0.5f) + 1);
    iz0 = max(iz0, (int)floorf((lo3[2] - blf[2]) * dzi - 0.5f) - 1);
    iz1 = min(iz1, (int)ceilf((hi3[2] - blf[2]) * dzi - 0.5f) + 1);
    w_mid = 2.0f * (fmaxf(kxf, kzf) * 0.5f * (tlo + thi) + fmaxf(bxf, bzf));
  }
  R.ix0 = ix0; R.ix1 = ix1; R.iy0 = iy0; R.iy1 = iy1; R.iz0 = iz0; R.iz1 = iz1;
  long long lines = 0;
  if (hit && ix1 >= ix0 && iy1 >= iy0 && iz1 >= iz0) lines = (long long)(iy1 - iy0 + 1) * (iz1 - iz0 + 1);
  // expected candidates on one x-line: the VOI width over the sine of the
  // angle between the axis and x, at most the box's x extent
  const float nxb = (float)(ix1 - ix0 + 1);
  float est = nxb;
  if (G.cutoff_mode != 2) {
    const float e0f = (float)e[0];
    const float sn = sqrtf(fmaxf(1.0f - e0f * e0f, 1e-6f));
    est = fminf(nxb, fmaxf(1.0f, w_mid / (sn * (float)G.dx)));
  }
  int lpc = (int)fminf((float)kMaxLinesPerItem, fmaxf(1.0f, (float)target_cand / est));
  R.lpc = lpc;
  // the box's lines; k_slices keeps only those that can meet the VOI
  R.nlines = (int)lines;
  R.nitems = (int)((lines + lpc - 1) / lpc);
  rows[r] = R;
  row_items[r] = R.nitems;
}

// ---------------------------------------------------------------------------
// k_slices: the x-lines of each row's voxel box that can meet its VOI, one
// warp per row, a lane per z-slice.  At the slice's voxel-centre height the
// VOI's cross-section is convex: the four lateral half-planes
// |x'| <= kx t + bx, |z'| <= kz t + bz (linear in x and y at fixed z), cut to
// the box's range of voxel centres in x and y.  The slice's lines are those
// whose centre y lies within the polygon's y-extent, found from its
// vertices.  FP32 with a margin of kSliceMargin mm: a line that the
// evaluation's own FP32 interval test could give a candidate is never left
// out (its rounding is far below the margin); a line kept by the margin may
// still have none.  Without a lateral cutoff every line of the box is kept.
// Writes the row's slice table, line count and work items (replacing the
// box's).
// ---------------------------------------------------------------------------
constexpr float kSliceMargin = 0.02f;

// y-extent at height zc of {A_k x + B_k y <= C_k, k < 8}, from the
// feasible pairwise intersections (within tol).  The pairs are expanded at
// compile time, so every index is a constant and the arrays stay in
// registers; parallel box sides (4, 5) and (6, 7) have no vertex.
struct YExtent {
  bool any = false;
  float ymin = 3.0e38f, ymax = -3.0e38f;
};
template <int I, int J>
__device__ __forceinline__ void pair_vertex(const float (&A)[8], const float (&B)[8], const float (&C)[8], float tol,
                                            YExtent& ye) {
  if ((I == 4 && J == 5) || (I == 6 && J == 7)) return;
  const float det = A[I] * B[J] - A[J] * B[I];
  if (fabsf(det) < 1e-9f) return;
  const float id = __frcp_rn(det);
  const float x = (C[I] * B[J] - C[J] * B[I]) * id;
  const float y = (A[I] * C[J] - A[J] * C[I]) * id;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 8; ++k) ok = ok && (A[k] * x + B[k] * y <= C[k] + tol);
  if (ok) {
    ye.any = true;
    ye.ymin = fminf(ye.ymin, y);
    ye.ymax = fmaxf(ye.ymax, y);
  }
}
template <int I, int J>
struct PolygonPairs {
  static __device__ __forceinline__ void run(const float (&A)[8], const float (&B)[8], const float (&C)[8], float tol,
                                             YExtent& ye) {
    pair_vertex<I, J>(A, B, C, tol, ye);
    PolygonPairs<I, J + 1>::run(A, B, C, tol, ye);
  }
};
template <int I>
struct PolygonPairs<I, 8> {
  static __device__ __forceinline__ void run(const float (&A)[8], const float (&B)[8], const float (&C)[8], float tol,
                                             YExtent& ye) {
    PolygonPairs<I + 1, I + 2>::run(A, B, C, tol, ye);
  }
};
template <>
struct PolygonPairs<7, 8> {
  static __device__ __forceinline__ void run(const float (&)[8], const float (&)[8], const float (&)[8], float,
                                             YExtent&) {}
};

__global__ void __launch_bounds__(128) k_slices(const DInst* __restrict__ inst, DRow* rows, int nrows, int* slice_pre,
                                                int* slice_lo, int stride, int* row_items) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (r >= nrows) return;                              // warp-uniform
  DRow& R = rows[r];
  const DInst& G = inst[R.inst];
  const bool box = R.hit && R.ix1 >= R.ix0 && R.iy1 >= R.iy0 && R.iz1 >= R.iz0;
  const int nzr = box ? min(R.iz1 - R.iz0 + 1, stride - 1) : 0;
  const int nyb = R.iy1 - R.iy0 + 1;
  const bool cut = G.cutoff_mode != 2;
  int* pre = slice_pre + (size_t)r * stride;
  int* lo = slice_lo + (size_t)r * stride;
  // the four lateral half-planes a.w <= b with w = p - S: a = +-x - k e,
  // +-z - k e; in x and y at height zc: A x + B y <= b - a2 (zc - S2) + A S0 + B S1
  float A[8], B[8], C0[8], Cz[8];
  {
    const float kx = R.kx, kz = R.kz;
    const float e0 = (float)R.e[0], e1 = (float)R.e[1], e2 = (float)R.e[2];
    const float x0 = (float)R.x[0], x1 = (float)R.x[1], x2 = (float)R.x[2];
    const float z0 = (float)R.z[0], z1 = (float)R.z[1], z2 = (float)R.z[2];
    const float S0 = (float)R.S[0], S1 = (float)R.S[1], S2 = (float)R.S[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float sg = (k & 1) ? -1.0f : 1.0f;             // +x', -x', +z', -z'
      const float kk = k < 2 ? kx : kz;
      const float u0 = k < 2 ? x0 : z0, u1 = k < 2 ? x1 : z1, u2 = k < 2 ? x2 : z2;
      const float a0 = sg * u0 - kk * e0, a1 = sg * u1 - kk * e1, a2 = sg * u2 - kk * e2;
      A[k] = a0;
      B[k] = a1;
      C0[k] = (k < 2 ? R.bx : R.bz) + a0 * S0 + a1 * S1 + a2 * S2;   // C = C0 - Cz zc
      Cz[k] = a2;
    }
    // the box's voxel-centre range in x and y
    const float xc0 = (float)(G.ox + (R.ix0 + 0.5) * G.dx), xc1 = (float)(G.ox + (R.ix1 + 0.5) * G.dx);
    const float yc0 = (float)(G.oy + (R.iy0 + 0.5) * G.dy), yc1 = (float)(G.oy + (R.iy1 + 0.5) * G.dy);
    A[4] = -1.0f; B[4] = 0.0f; C0[4] = -xc0; Cz[4] = 0.0f;
    A[5] = 1.0f;  B[5] = 0.0f; C0[5] = xc1;  Cz[5] = 0.0f;
    A[6] = 0.0f;  B[6] = -1.0f; C0[6] = -yc0; Cz[6] = 0.0f;
    A[7] = 0.0f;  B[7] = 1.0f;  C0[7] = yc1;  Cz[7] = 0.0f;
  }
  const float dyi = __frcp_rn((float)G.dy), oyh = (float)G.oy + 0.5f * (float)G.dy;
  const float ozf = (float)G.oz, dzf = (float)G.dz;
  int run = 0;
  for (int s0 = 0; s0 < nzr; s0 += 32) {               // warp-uniform
    const int s = s0 + lane;
    int cnt = 0, ylo = R.iy0;
    if (s < nzr) {
      if (!cut) {
        cnt = nyb;
      } else {
        const float zc = fmaf((float)(R.iz0 + s) + 0.5f, dzf, ozf);
        float C[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) C[k] = C0[k] - Cz[k] * zc;
        YExtent ye;
        PolygonPairs<0, 1>::run(A, B, C, kSliceMargin, ye);
        if (ye.any) {
          // centres y = oy + (iy + 0.5) dy within [ymin - margin, ymax + margin]
          const int a0 = (int)ceilf((ye.ymin - kSliceMargin - oyh) * dyi);
          const int a1 = (int)floorf((ye.ymax + kSliceMargin - oyh) * dyi);
          ylo = max(a0, R.iy0);
          cnt = max(0, min(a1, R.iy1) - ylo + 1);
        }
      }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (s < nzr) {
      pre[s] = run + incl - cnt;
      lo[s] = ylo;
    }
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) {
    pre[nzr] = run;
    R.nlines = run;
    R.nitems = (run + R.lpc - 1) / R.lpc;
    row_items[r] = R.nitems;
  }
}

// ---------------------------------------------------------------------------
// k_siddon: radiological depth table, one CTA of kSiddonThreads lanes per
// beamlet axis.  Lane l walks the table intervals [l Q, (l+1) Q) with
// Siddon's incremental plane crossings (alpha in FP64), stores its
// lane-local cumulative depth, then adds the CTA-exclusive prefix of the
// lane totals.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSiddonThreads) k_siddon(const DInst* __restrict__ inst,
                                                            const DRow* __restrict__ rows, int nrows,
                                                            float* __restrict__ tables, int stride) {
  __shared__ double wsum[kSiddonThreads / 32];
  const int ray = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (ray >= nrows) return;
  const DRow& R = rows[ray];
  const int n = R.n_table;
  if (n <= 0) return;                                // uniform over the CTA
  const DInst& G = inst[R.inst];
  float* tab = tables + (size_t)ray * stride;
  if (threadIdx.x == 0) tab[0] = 0.0f;
  const int nint = n - 1;                            // intervals
  const int Q = (nint + kSiddonThreads - 1) / kSiddonThreads;
  const int k0 = min((int)threadIdx.x * Q, nint), k1 = min(k0 + Q, nint);
  const double L = R.tB - R.tA;
  const double h = G.hd;
  const double* S = R.S;
  const double* e = R.e;
  const double org[3] = {G.ox, G.oy, G.oz};
  const double sp[3] = {G.dx, G.dy, G.dz};
  const double isp[3] = {G.idx, G.idy, G.idz};
  const int nv[3] = {G.nx, G.ny, G.nz};
  // The walk runs in fixed point (crossing parameters alpha as 64-bit
  // integers from the FP64 set-up in k_setup, in units finer than an FP64 ulp
  // at these distances) on the integer pipes; the density integral is a
  // compensated FP32 sum, as fine as the FP32 table that stores it.
  double total = 0.0;
  if (k0 < k1) {
    const long long kNever = 0x3fffffffffffffffll;
    const float unfix = ldexpf(1.0f, -R.fix_q);
    const long long tcur0 = R.fx_tA + min((long long)k0 * R.fx_h, R.fx_tB - R.fx_tA);
    long long tcur = tcur0;
    // starting voxel and next crossing per axis (FP64 once per lane), then
    // fixed point; a crossing past t_B never happens, and steps are capped so
    // that no sum overflows
    const double tcur_d = R.tA + fmin(k0 * h, L);
    const double fx = ldexp(1.0, R.fix_q);
    const double tlim = R.tB + 1.0;
    long long al[3], da[3];
    int i[3], st[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double p = fma(tcur_d, e[a], S[a]);
      int q = (int)floor((p - org[a]) * isp[a]);
      i[a] = min(max(q, 0), nv[a] - 1);
      const double ie = R.inv_e[a];
      double an = CUDART_INF, dn = 0.0;
      if (e[a] > 0.0) {
        st[a] = 1;
        an = (org[a] + (i[a] + 1) * sp[a] - S[a]) * ie;
        dn = sp[a] * ie;
      } else if (e[a] < 0.0) {
        st[a] = -1;
        an = (org[a] + i[a] * sp[a] - S[a]) * ie;
        dn = -sp[a] * ie;
      } else {
        st[a] = 0;
      }
      al[a] = an <= tlim ? __double2ll_rn(an * fx) : kNever;
      da[a] = dn <= tlim ? __double2ll_rn(dn * fx) : kNever;
    }
    // scalar walk state (no dynamically indexed arrays: they would live in local memory)
    int ix = i[0], iy = i[1], iz = i[2];
    const int sx = st[0], sy_ = st[1], sz_ = st[2];
    long long ax = al[0], ay = al[1], az = al[2];
    const long long dax = da[0], day = da[1], daz = da[2];
    const float* rho = G.rho;
    const long long ny_s = G.nx, nz_s = (long long)G.nx * G.ny;
    long long vox = ix + iy * ny_s + iz * nz_s;
    float rv = __ldg(rho + vox) * unfix;              // density per fixed-point unit
    float sum = 0.0f, comp = 0.0f;                     // Kahan sum of the lane
    long long tend = tcur0;
    int guard = 4 * (G.nx + G.ny + G.nz) + 8 * (k1 - k0) + 16;
    for (int k = k0; k < k1; ++k) {
      tend = (k + 1 == nint) ? R.fx_tB : min(tend + R.fx_h, R.fx_tB);
      for (;;) {
        const long long am = min(ax, min(ay, az));
        if (am >= tend || --guard < 0) break;
        {
          float y = fmaf((float)max(am - tcur, 0ll), rv, -comp);
          float tt = sum + y;
          comp = (tt - sum) - y;
          sum = tt;
        }
        tcur = max(tcur, am);
        if (ax == am) {
          int n2 = ix + sx;
          if (n2 >= 0 && n2 < G.nx) { ix = n2; vox += sx; }
          ax = ax + dax > ax ? min(ax + dax, kNever) : kNever;
        } else if (ay == am) {
          int n2 = iy + sy_;
          if (n2 >= 0 && n2 < G.ny) { iy = n2; vox += sy_ * ny_s; }
          ay = ay + day > ay ? min(ay + day, kNever) : kNever;
        } else {
          int n2 = iz + sz_;
          if (n2 >= 0 && n2 < G.nz) { iz = n2; vox += sz_ * nz_s; }
          az = az + daz > az ? min(az + daz, kNever) : kNever;
        }
        rv = __ldg(rho + vox) * unfix;
      }
      {
        float y = fmaf((float)max(tend - tcur, 0ll), rv, -comp);
        float tt = sum + y;
        comp = (tt - sum) - y;
        sum = tt;
      }
      tcur = max(tcur, tend);
      tab[k + 1] = sum - comp;                         // lane-local, fixed below
    }
    total = (double)sum - (double)comp;
  }
  // exclusive prefix of the lane totals over the CTA
  double incl = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  double prefix = incl - total;
  for (int i = 0; i < w; ++i) prefix += wsum[i];
  for (int k = k0; k < k1; ++k) tab[k + 1] = (float)(prefix + (double)tab[k + 1]);
}

// ---------------------------------------------------------------------------
// k_trilinear_table: the paper's own table construction (Section 2.2).  The
// density is sampled by software trilinear interpolation of the voxel-centred
// values (clamped to the edge) at the n points s_k = min(k h, |AB|) of AB, and
// entry k is the depth from A to point k, accumulated over the sample
// intervals by the trapezoid rule.  One CTA per beamlet axis; each lane takes
// a contiguous run of intervals (one extra sample at its start), sums its
// trapezoids with a compensated FP32 sum, and the CTA prefix of the lane
// totals is added in FP64, as in k_siddon.  Sample positions and cell
// fractions in FP64, the blend of the eight densities in FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float trilinear_at(const DInst& G, double px, double py, double pz) {
  const double f[3] = {(px - G.ox) * G.idx - 0.5, (py - G.oy) * G.idy - 0.5, (pz - G.oz) * G.idz - 0.5};
  const int n[3] = {G.nx, G.ny, G.nz};
  int i0[3], i1[3];
  float w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (f[a] <= 0.0) { i0[a] = 0; i1[a] = 0; w[a] = 0.0f; }
    else if (f[a] >= n[a] - 1) { i0[a] = n[a] - 1; i1[a] = n[a] - 1; w[a] = 0.0f; }
    else {
      const double fl = floor(f[a]);
      i0[a] = (int)fl; i1[a] = i0[a] + 1; w[a] = (float)(f[a] - fl);
    }
  }
  const float* rho = G.rho;
  const long long sy = G.nx, sz = (long long)G.nx * G.ny;
  const long long y0 = i0[1] * sy, y1 = i1[1] * sy, z0 = i0[2] * sz, z1 = i1[2] * sz;
  const float c000 = __ldg(rho + i0[0] + y0 + z0), c100 = __ldg(rho + i1[0] + y0 + z0);
  const float c010 = __ldg(rho + i0[0] + y1 + z0), c110 = __ldg(rho + i1[0] + y1 + z0);
  const float c001 = __ldg(rho + i0[0] + y0 + z1), c101 = __ldg(rho + i1[0] + y0 + z1);
  const float c011 = __ldg(rho + i0[0] + y1 + z1), c111 = __ldg(rho + i1[0] + y1 + z1);
  const float c00 = fmaf(w[0], c100 - c000, c000), c10 = fmaf(w[0], c110 - c010, c010);
  const float c01 = fmaf(w[0], c101 - c001, c001), c11 = fmaf(w[0], c111 - c011, c011);
  const float c0 = fmaf(w[1], c10 - c00, c00), c1 = fmaf(w[1], c11 - c01, c01);
  return fmaf(w[2], c1 - c0, c0);
}

__global__ void __launch_bounds__(kSiddonThreads) k_trilinear_table(const DInst* __restrict__ inst,
                                                                     const DRow* __restrict__ rows, int nrows,
                                                                     float* __restrict__ tables, int stride) {
  __shared__ double wsum[kSiddonThreads / 32];
  const int ray = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (ray >= nrows) return;
  const DRow& R = rows[ray];
  const int n = R.n_table;
  if (n <= 0) return;                                // uniform over the CTA
  const DInst& G = inst[R.inst];
  float* tab = tables + (size_t)ray * stride;
  if (threadIdx.x == 0) tab[0] = 0.0f;
  const int nint = n - 1;                            // intervals
  const int Q = (nint + kSiddonThreads - 1) / kSiddonThreads;
  const int k0 = min((int)threadIdx.x * Q, nint), k1 = min(k0 + Q, nint);
  const double L = R.tB - R.tA;
  const double h = G.hd;
  double total = 0.0;
  if (k0 < k1) {
    double s_prev = fmin(k0 * h, L);
    double t = R.tA + s_prev;
    float r_prev = trilinear_at(G, fma(t, R.e[0], R.S[0]), fma(t, R.e[1], R.S[1]), fma(t, R.e[2], R.S[2]));
    float sum = 0.0f, comp = 0.0f;                     // Kahan sum of the lane
    for (int k = k0; k < k1; ++k) {
      const double s = fmin((k + 1) * h, L);
      t = R.tA + s;
      const float r = trilinear_at(G, fma(t, R.e[0], R.S[0]), fma(t, R.e[1], R.S[1]), fma(t, R.e[2], R.S[2]));
      const float y = fmaf((float)(s - s_prev) * 0.5f, r_prev + r, -comp);
      const float tt = sum + y;
      comp = (tt - sum) - y;
      sum = tt;
      tab[k + 1] = sum - comp;                         // lane-local, fixed below
      s_prev = s;
      r_prev = r;
    }
    total = (double)sum - (double)comp;
  }
  double incl = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  double prefix = incl - total;
  for (int i = 0; i < w; ++i) prefix += wsum[i];
  for (int k = k0; k < k1; ++k) tab[k + 1] = (float)(prefix + (double)tab[k + 1]);
}

// ---------------------------------------------------------------------------
// x-lines of a work item
// ---------------------------------------------------------------------------
constexpr int kTabSmem = 1024;   // depth-table entries a work item stages in shared memory
#ifndef DSC_LUT_SMEM
#define DSC_LUT_SMEM 256
#endif
// beam-model table rows a CTA stages in shared memory (as (row, difference)
// pairs) beside the depth table; 0: read through L1
constexpr int kLutSmem = DSC_LUT_SMEM;
#if DSC_LUT_SMEM
#define SMLUT sm.lut
#else
#define SMLUT nullptr
#endif
// The x-lines of a work item, rebased on the item's candidate index jj (0 at
// the item's first candidate): candidate jj on line li has ix = ixb + jj,
// column colb + jj and depth coordinate sfb + jj * dsf, so a candidate needs
// its line index and three loads.
struct LineSm {
  float4 sx[kMaxLinesPerItem];        // t at ix = 0, colb (int bits), x' hi, z' hi at ix = 0
  float4 zc[kMaxLinesPerItem];        // x' lo, z' lo at ix = 0, ixb (int bits), unused
  long long sf[kMaxLinesPerItem];     // sfb: s of candidate jj = 0 (fixed point, units of h 2^-32)
  unsigned char map[kWindow];         // line of each candidate of the window (4-byte aligned)
  int off[kMaxLinesPerItem + 1];      // first candidate (jj) of each line
  int wscan[kEvalThreads / 32];
  float tab[kTabSmem];                // the row's depth table, when it fits
#if DSC_LUT_SMEM
  float4 lut[2 * kLutSmem];           // the instance's beam-model table, when it fits
  int lut_inst;                       // instance whose table is in lut (-1: none)
#endif
  long long item;
  int row;
  int nl;
  int total;
  float dl_ukeep, dl_bc, dl_bh, dl_mlo;   // L's kept bound, band centre and half-width, near-L bound
  unsigned* tmeta;                    // the item's first tile's entry of tile_meta
};

// float-float s, x', z' of x-line (iy, iz) of row R at ix = 0 (the
// evaluation's per-candidate values start from these)
__device__ __forceinline__ void line_base(const DRow& R, int iy, int iz, ff& s0, ff& x0, ff& z0) {
  float fy = (float)iy, fz = (float)iz;
  s0 = ff_add(ff_add(R.S0, ff_mul_i(R.Ss[1], fy)), ff_mul_i(R.Ss[2], fz));
  x0 = ff_add(ff_add(R.X0, ff_mul_i(R.Xs[1], fy)), ff_mul_i(R.Xs[2], fz));
  z0 = ff_add(ff_add(R.Z0, ff_mul_i(R.Zs[1], fy)), ff_mul_i(R.Zs[2], fz));
}

// the row constants of a line's candidate interval: the FP32 bases and
// steps of t, x', z' and the slopes c of the four lateral constraints along
// x with their reciprocals.  A loop over a row's lines loads them once.
struct LineCut {
  float tA, S0, Sy, Sz, X0, Xy, Xz, Z0, Zy, Zz;
  float kx, bx, kz, bz;
  float c[4], rc[4];
  float tx, rtx;
  int mode, nx;
  __device__ __forceinline__ LineCut(const DRow& R, int mode_, int nx_) : mode(mode_), nx(nx_) {
    tA = R.tA_f;
    S0 = R.S0.hi; Sy = R.Ss[1].hi; Sz = R.Ss[2].hi;
    X0 = R.X0.hi; Xy = R.Xs[1].hi; Xz = R.Xs[2].hi;
    Z0 = R.Z0.hi; Zy = R.Zs[1].hi; Zz = R.Zs[2].hi;
    kx = R.kx; bx = R.bx; kz = R.kz; bz = R.bz;
    tx = R.Ss[0].hi;
    const float xx = R.Xs[0].hi, zx = R.Zs[0].hi;
    c[0] = fmaf(-kx, tx, xx);
    c[1] = fmaf(-kx, tx, -xx);
    c[2] = fmaf(-kz, tx, zx);
    c[3] = fmaf(-kz, tx, -zx);
#pragma unroll
    for (int k = 0; k < 4; ++k) rc[k] = rcp_approx(c[k]);
    rtx = rcp_approx(tx);
  }
};

// candidate interval [lo, lo + len) of x-line (iy, iz)
__device__ __forceinline__ int line_interval(const LineCut& L, int iy, int iz, int& lo_out) {
  // t(i) = T0 + i tx, x'(i) = X0 + i xx, z'(i) = Z0 + i zx; constraints c i <= r.
  // T0, X0, Z0 at ix = 0 in plain FP32: their error (about 1e-4 mm) is far
  // inside the 1e-3 mm band around the cutoff that parity leaves open, and the
  // enumeration count and the evaluation both take the interval from here, so
  // they agree exactly
  const float fy = (float)iy, fz = (float)iz;
  const float T0 = L.tA + fmaf(L.Sz, fz, fmaf(L.Sy, fy, L.S0));
  const float X0 = fmaf(L.Xz, fz, fmaf(L.Xy, fy, L.X0));
  const float Z0 = fmaf(L.Zz, fz, fmaf(L.Zy, fy, L.Z0));
  float lo = 0.0f, hi = (float)(L.nx - 1);
  bool empty = false;
  auto constrain = [&](int k, float r) {
    const float q = r * L.rc[k];
    if (L.c[k] > 0.0f) hi = fminf(hi, q);
    else if (L.c[k] < 0.0f) lo = fmaxf(lo, q);
    else if (r < 0.0f) empty = true;
  };
  if (L.mode != 2) {
    const float rx = fmaf(L.kx, T0, L.bx), rz = fmaf(L.kz, T0, L.bz);
    constrain(0, rx - X0);
    constrain(1, rx + X0);
    constrain(2, rz - Z0);
    constrain(3, rz + Z0);
  } else {
    // t > 0 (voxels in front of the source)
    if (L.tx > 0.0f) lo = fmaxf(lo, floorf(-T0 * L.rtx) + 1.0f);
    else if (L.tx < 0.0f) hi = fminf(hi, ceilf(-T0 * L.rtx) - 1.0f);
    else if (T0 <= 0.0f) empty = true;
  }
  int ilo = (int)ceilf(lo), ihi = (int)floorf(hi);
  lo_out = ilo;
  if (empty || ihi < ilo) return 0;
  return ihi - ilo + 1;
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

// line (iy, iz) of line index l >= 0 of row R (a row's VOI box has fewer than
// 2^31 lines: the grid has fewer than 2^31 voxels).  inv_nyb = 1 / (lines per
// iz), correctly rounded.  Below 2^22 the FP32 quotient is within 1/2 of l /
// nyb, so its truncation is off by at most one, which the remainder corrects.
// the slice of line l of a row: the last s with pre[s] <= l (nzr slices)
__device__ __forceinline__ int line_slice(const int* __restrict__ pre, int nzr, int l) {
  int s = 0;
#pragma unroll 1
  for (int step = nzr > 1 ? 1 << (31 - __clz(nzr - 1)) : 0; step > 0; step >>= 1)
    if (s + step < nzr && pre[s + step] <= l) s += step;
  return s;
}
// walks consecutive lines of a row through its slice table
struct LineWalk {
  const int* pre;
  const int* lo;
  int nzr;
  int s = -1, first = 0, next = 0, ylo = 0;
  __device__ LineWalk(const SliceTab& T, int row, int nzr_) : pre(T.pre + (size_t)row * T.stride),
                                                             lo(T.lo + (size_t)row * T.stride), nzr(nzr_) {}
  // (iy, iz) of line l; lines are visited in increasing order
  __device__ __forceinline__ void at(const DRow& R, int l, int& iy, int& iz) {
    if (s < 0) {
      s = line_slice(pre, nzr, l);
      first = pre[s];
      next = pre[s + 1];
      ylo = lo[s];
    }
    while (l >= next && s < nzr - 1) {                // also past empty slices
      ++s;
      first = next;
      next = pre[s + 1];
      ylo = lo[s];
    }
    iz = R.iz0 + s;
    iy = ylo + (l - first);
  }
};
// nzr of a row as k_slices wrote its table
__device__ __forceinline__ int row_slices(const DRow& R, int stride) {
  const bool box = R.hit && R.ix1 >= R.ix0 && R.iy1 >= R.iy0 && R.iz1 >= R.iz0;
  return box ? min(R.iz1 - R.iz0 + 1, stride - 1) : 0;
}

// lines of a work item: [chunk * lpc, min(+lpc, lines of the row))
__device__ __forceinline__ int item_nlines(const DRow& R, long long chunk, int& l0) {
  l0 = (int)chunk * R.lpc;
  return min(R.lpc, R.nlines - l0);
}

// set up all lines of an item in shared memory (each thread takes kMaxLinesPerItem /
// kEvalThreads consecutive lines), rebased on the item's candidate index;
// returns the candidate count
__device__ int item_lines(LineSm& sm, const DRow& R, const SliceTab& T, int row, int mode, int nx, int ny,
                          long long chunk) {
  constexpr int per = kMaxLinesPerItem / kEvalThreads;
  int l0;
  int nl = item_nlines(R, chunk, l0);
  int t = threadIdx.x;
  int len[per], lo[per], cb[per];
  long long sfl[per];
  int mine = 0;
  LineWalk walk(T, row, row_slices(R, T.stride));
  const LineCut L(R, mode, nx);
#pragma unroll
  for (int q = 0; q < per; ++q) {
    int li = t * per + q;             // consecutive lines per thread keep the scan order
    len[q] = 0;
    lo[q] = 0;
    cb[q] = 0;
    sfl[q] = 0;
    if (li < nl) {
      int iy, iz;
      walk.at(R, l0 + li, iy, iz);
      len[q] = line_interval(L, iy, iz, lo[q]);
      if (len[q] > 0) {                  // an empty line's record is never read
        ff s0, x0, z0;
        line_base(R, iy, iz, s0, x0, z0);
        cb[q] = nx * (iy + ny * iz);
        sfl[q] = R.sfx0 + (long long)iy * R.sfx_s[1] + (long long)iz * R.sfx_s[2];
        sm.sx[li] = make_float4(R.tA_f + s0.hi, 0.0f, x0.hi, z0.hi);
        sm.zc[li] = make_float4(x0.lo, z0.lo, 0.0f, 0.0f);
      }
    }
    mine += len[q];
  }
  int excl;
  int tot = block_excl_scan(mine, excl, sm.wscan);
#pragma unroll
  for (int q = 0; q < per; ++q) {
    int li = t * per + q;
    if (li < nl) {
      const int ixb = lo[q] - excl;   // ix of candidate jj on this line: ixb + jj
      sm.off[li] = excl;
      reinterpret_cast<int*>(&sm.sx[li])[1] = cb[q] + ixb;
      reinterpret_cast<int*>(&sm.zc[li])[2] = ixb;
      sm.sf[li] = sfl[q] + (long long)ixb * R.sfx_s[0];
    }
    excl += len[q];
  }
  if (t == 0) { sm.nl = nl; sm.off[nl] = tot; }
  __syncthreads();
  return tot;
}

// line index of every candidate in [w0, w0 + wl), one byte each (an item
// has at most 256 lines): mark line starts, then an inclusive max-scan over
// the window.  Each thread reads its 32 consecutive entries as two 16-byte
// vectors (scalar accesses at that stride conflict 8 ways in the banks),
// scans them in registers and writes them back the same way.  One-byte
// entries let a window of 4096 candidates share the space of 2048 two-byte
// ones, which halves the barriers per candidate.
static_assert(kMaxLinesPerItem <= 256, "line indices of an item fit a byte");
__device__ void item_map(LineSm& sm, int w0, int wl) {
  constexpr int per = kWindow / kEvalThreads;
  constexpr int vecs = per / 16;                        // 16-byte vectors per thread
  static_assert(per % 16 == 0, "whole 16-byte vectors of the map per thread");
  const int t = threadIdx.x;
  const int nl = sm.nl;
  uint4* mv = reinterpret_cast<uint4*>(sm.map) + t * vecs;
  // zero-filled: line indices rise along the window and position 0 always
  // holds a start, so a running maximum over the starts gives every line
#pragma unroll
  for (int j = 0; j < vecs; ++j) mv[j] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int li = t; li < nl; li += kEvalThreads) {
    int o = sm.off[li], e = sm.off[li + 1];
    if (e > o) {
      if (o >= w0 && o < w0 + wl) sm.map[o - w0] = (unsigned char)li;
      else if (o < w0 && e > w0) sm.map[0] = (unsigned char)li;
    }
  }
  __syncthreads();
  unsigned wv[4 * vecs];
#pragma unroll
  for (int j = 0; j < vecs; ++j) {
    const uint4 q = mv[j];
    wv[4 * j] = q.x; wv[4 * j + 1] = q.y; wv[4 * j + 2] = q.z; wv[4 * j + 3] = q.w;
  }
  int run = 0;
#pragma unroll
  for (int j = 0; j < 4 * vecs; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) run = max(run, (int)((wv[j] >> (8 * k)) & 0xffu));
  int lane = t & 31, w = t >> 5;
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl = max(incl, v);
  }
  if (lane == 31) sm.wscan[w] = incl;
  __syncthreads();
  int wpre = 0;
#pragma unroll
  for (int i = 0; i < kEvalThreads / 32; ++i)
    if (i < w) wpre = max(wpre, sm.wscan[i]);
  int excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = 0;
  run = max(wpre, excl);
  // second pass: running maximum from the carry
#pragma unroll
  for (int j = 0; j < 4 * vecs; ++j) {
    const unsigned v = wv[j];
    unsigned o = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      run = max(run, (int)((v >> (8 * k)) & 0xffu));
      o |= (unsigned)run << (8 * k);
    }
    wv[j] = o;
  }
#pragma unroll
  for (int j = 0; j < vecs; ++j) mv[j] = make_uint4(wv[4 * j], wv[4 * j + 1], wv[4 * j + 2], wv[4 * j + 3]);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// k_item_rows: the row of every work item (rows own items
// [row_item_base[r], row_item_base[r+1]))
// ---------------------------------------------------------------------------
__global__ void k_item_rows(const long long* __restrict__ row_item_base, int nrows, int* item_row) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  for (long long i = row_item_base[r]; i < row_item_base[r + 1]; ++i) item_row[i] = r;
}

// ---------------------------------------------------------------------------
// k_count: candidate pairs per work item, one warp per item
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEvalThreads) k_count(const DInst* __restrict__ inst, const DRow* __restrict__ rows,
                                                        SliceTab T, const long long* __restrict__ row_item_base,
                                                        int nrows, const long long* __restrict__ n_items,
                                                        int* item_cand, const int* __restrict__ item_row,
                                                        int* ord_cnt, int* item_crank, int target_cand) {
  const long long ni = *n_items;
  const int lane = threadIdx.x & 31, half = lane >> 4, sub = lane & 15;
  // a half-warp per item, so that two items' dependent loads are in flight
  const long long nh = (long long)gridDim.x * (kEvalThreads / 16);
  for (long long base = ((long long)blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5)) * 2; base < ni;
       base += nh) {                                   // warp-uniform
    const long long item = base + half;
    int cnt = 0;
    if (item < ni) {
      const int row = item_row[item];
      const DRow& R = rows[row];
      const DInst& G = inst[R.inst];
      int l0;
      const int nl = item_nlines(R, item - row_item_base[row], l0);
      // each lane takes consecutive lines, so it walks its slices from one search
      constexpr int lpl = kMaxLinesPerItem / 16;
      LineWalk walk(T, row, row_slices(R, T.stride));
      const LineCut L(R, G.cutoff_mode, G.nx);
      for (int li = sub * lpl; li < min(nl, (sub + 1) * lpl); ++li) {
        int iy, iz;
        walk.at(R, l0 + li, iy, iz);
        int lo;
        cnt += line_interval(L, iy, iz, lo);
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);   // within the half
    // items are padded to whole compaction tiles (the evaluation writes
    // whole tiles; padding slots hold -1, never kept); each takes a rank in
    // its size class for the evaluation's queue order (k_tile_map)
    if (sub == 0 && item < ni) {
      const int n = (cnt + kTile - 1) & ~(kTile - 1);
      item_cand[item] = n;
      if (item_crank) {
        const int c = order_class(n, target_cand);
        item_crank[item] = (c << kOrderRankBits) | atomicAdd(ord_cnt + c, 1);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FSPB evaluation (Eq. 2-3)
// ---------------------------------------------------------------------------
// erfc(u) for u >= 0, given v = u sqrt(log2 e):  t exp(-u^2) P(t) with
// t = 1/(1 + p u) (coefficients from fit_erfc.py) and exp(-u^2) = 2^(-v^2).
// Rounding v^2 to FP32 costs a relative error of about 4e-8 v^2 in the
// exponential, below the fit's own 4.6e-7 where the terms matter.
// Two arguments at once in packed FP32x2 arithmetic: one instruction per
// pair of operations, each half rounded as the scalar fmaf / mul.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
constexpr float kInvSqrtL = 0.83255461115769775635f;   // 1 / sqrt(log2 e)

__device__ __forceinline__ float2 rcp2(float2 d) { return make_float2(rcp_approx(d.x), rcp_approx(d.y)); }

// the reciprocals t = 1/(1 + p |v|) of the four erfc denominators of a
// profile term (a: X and Z at y1, b: at y2), by product inversion:
//   DSC_SHARED_RCP 2: one reciprocal r = 1/(q_x q_y) of the product of all
//     four, q = da db; 1/q_x = r q_y, 1/q_y = r q_x, then 1/da = (1/q) db and
//     1/db = (1/q) da (one rcp.approx and six multiplications);
//   DSC_SHARED_RCP 1: r = 1/q per axis, 1/da = r db, 1/db = r da (two
//     rcp.approx and three packed multiplications);
//   0: four rcp.approx.
// Each result is within a few ulp.  The denominators lie in [1, 1 + p |v|];
// the host's limits on the model and the geometry keep the products finite.
#ifndef DSC_SHARED_RCP
#define DSC_SHARED_RCP 0
#endif
constexpr float kPs = kErfcP * kInvSqrtL;   // p / sqrt(log2 e)
__device__ __forceinline__ void erfc_recips(float2 a, float2 b, float2& ta, float2& tb) {
  const float2 da = make_float2(fmaf(kPs, fabsf(a.x), 1.0f), fmaf(kPs, fabsf(a.y), 1.0f));
  const float2 db = make_float2(fmaf(kPs, fabsf(b.x), 1.0f), fmaf(kPs, fabsf(b.y), 1.0f));
#if DSC_SHARED_RCP == 2
  const float2 q = __fmul2_rn(da, db);
  const float r = rcp_approx(__fmul_rn(q.x, q.y));
  const float2 rq = make_float2(__fmul_rn(r, q.y), __fmul_rn(r, q.x));
  ta = __fmul2_rn(rq, db);
  tb = __fmul2_rn(rq, da);
#elif DSC_SHARED_RCP == 1
  const float2 rq = rcp2(__fmul2_rn(da, db));
  ta = __fmul2_rn(rq, db);
  tb = __fmul2_rn(rq, da);
#else
  ta = rcp2(da);
  tb = rcp2(db);
#endif
}

// given t = 1/(1 + p |v|): tp = t P(t) (P from `c`: the
// fitted coefficients, or their negatives for -t P(t)), e = 2^(-v^2);
// erfc(|u|) = tp e, kept apart so that callers fold the product into an FMA
__device__ __forceinline__ void erfc_parts(float2 t, float2 v, const float2* __restrict__ c, float2& tp, float2& e) {
  float2 p = c[kErfcN];
#pragma unroll
  for (int k = kErfcN - 1; k >= 0; --k) p = __ffma2_rn(p, t, c[k]);
  const float2 vv = __fmul2_rn(v, v);
  e = make_float2(ex2_approx(-vv.x), ex2_approx(-vv.y));
  tp = __fmul2_rn(t, p);
}

// The X and Z factors of one profile term together.  Every profile is the
// beamlet's box convolved per axis with a spread kernel: with G the kernel's
// complementary distribution function and y1 = (|x'| - h)/s,
// y2 = (|x'| + h)/s (h = c2/2 a_t, b_t for Z),
//   X = 2 [G(y1) - G(y2)],   2 G(y1) = (1 - sgn y1) + sgn(y1) T(|y1|),
// T(y) = 2 G(y) for y >= 0 the kernel's tail; the sign bit of y1 picks the
// form, so the tails never cancel.  For Eq. 3 (Gaussian) X is the erf pair
// erf(u1) + erf(u2) = erfc(-u1) - erfc(u2), T = erfc.  Arguments arrive
// scaled (v = y in the units the tail wants: Prof<P>::K / c3); abt = (a_t,
// b_t), axz = (|x'|, |z'|), c2hn = -c2/2; |x'| -/+ h and the sums round once.
//   P = 0  Gaussian:  T = erfc(u), v = u sqrt(log2 e)
//   P = 1  Laplace:   T = exp(-y) = 2^-v,                 s = c3 / sqrt 2
//   P = 2  logistic:  T = 2 exp(-y) / (1 + exp(-y)),      s = c3 sqrt 3 / pi
template <int PROF> struct Prof;
template <> struct Prof<0> { static constexpr float K = 0.84932180028801904272f; };   // sqrt(log2(e) / 2)
template <> struct Prof<1> { static constexpr float K = 2.04027889319357896350f; };   // log2(e) sqrt 2
template <> struct Prof<2> { static constexpr float K = 2.61675934794826075443f; };   // log2(e) pi / sqrt 3

template <int PROF>
__device__ __forceinline__ float2 erf_pair2(float c2h, float c2hn, float2 abt, float2 axz, float inv_s) {
  const float2 x = __fmul2_rn(__ffma2_rn(f2(c2hn), abt, axz), f2(inv_s));   // y1, scaled
  const float2 v2 = __fmul2_rn(__ffma2_rn(f2(c2h), abt, axz), f2(inv_s));  // y2, scaled (>= 0)
  float2 tp1, e1, tp2n, e2;
  if (PROF == 0) {
    // denominators as scalar FMAs with immediate operands: no packed constant pairs to build
    float2 t1, t2;
    erfc_recips(x, v2, t1, t2);
    erfc_parts(t1, x, kErfcC2, tp1, e1);
    erfc_parts(t2, v2, kErfcC2n, tp2n, e2);
  } else {
    e1 = make_float2(ex2_approx(-fabsf(x.x)), ex2_approx(-fabsf(x.y)));
    e2 = make_float2(ex2_approx(-v2.x), ex2_approx(-v2.y));
    if (PROF == 1) {
      tp1 = f2(1.0f);
      tp2n = f2(-1.0f);
    } else {                                  // 2 / (1 + e) from the reciprocal of (1 + e) / 2
      tp1 = rcp2(__ffma2_rn(e1, f2(0.5f), f2(0.5f)));
      tp2n = rcp2(__ffma2_rn(e2, f2(-0.5f), f2(-0.5f)));
    }
  }
  // 2 G(y1) = (1 - s) + s tp e, s = +-1 the sign of y1: s tp is tp with y1's
  // sign bit (tp >= 0), and 1 - s (0 or 2) is that sign bit shifted onto
  // 2.0f's exponent bit -- integer operations, exact, off the FMA pipe
  const unsigned sbx = __float_as_uint(x.x) & 0x80000000u, sby = __float_as_uint(x.y) & 0x80000000u;
  const float2 stp1 = make_float2(__uint_as_float(__float_as_uint(tp1.x) | sbx),
                                  __uint_as_float(__float_as_uint(tp1.y) | sby));
  const float2 oms = make_float2(__uint_as_float(sbx >> 1), __uint_as_float(sby >> 1));
  const float2 erfc_x = __ffma2_rn(stp1, e1, oms);
  return __ffma2_rn(tp2n, e2, erfc_x);
}

// everything the per-pair evaluation reads, loaded once per work item
struct RowConst {
  long long dsf;         // slope of s per ix, fixed point (units of h 2^-32)
  float tx;              // slope of t per ix
  float2 XZh, XZl;       // slopes of (x', z') per ix, float-float
  float2 ab_sad;         // (a, b) / SAD
  int n_table;
  const float* tab;      // the row's depth table
  const float4* lut;     // beam-model table
  float lut_scale, lut_last;
  float c1q[3], c2h[3], c2hn[3];   // c1/4 SAD^2, c2/2, -c2/2
  float cutoff_k;
};

// FP32 value of a small non-negative integer (n < 2^23) without a conversion
// instruction: 2^23 + n is exact in FP32 and its bits are 0x4B000000 + n
__device__ __forceinline__ float small_int_to_float(int n) {
  return __fsub_rn(__int_as_float(0x4B000000 + n), 8388608.0f);
}

// D for a candidate at ix = fi of a line (A, B: the line's records, s: its
// depth coordinate); -1 outside the sigma cutoff (SIG).  TS: the row's depth
// table is staged in shared memory at stab
template <int PROF, bool TS, bool SIG>
__device__ __forceinline__ float eval_pair(const RowConst& C, float fi, float4 A, float4 B, long long s,
                                           const float* stab, const float4* slut) {
  // t, x', z' of voxel ix on the line (compensated FP32 for x', z': hi and
  // lo slopes times ix, added once)
  const float t = fmaf(fi, C.tx, A.x);
  const float2 fii = f2(fi);
  const float2 xz = __fadd2_rn(__ffma2_rn(fii, C.XZh, make_float2(A.z, A.w)),
                               __ffma2_rn(fii, C.XZl, make_float2(B.x, B.y)));

  // radiological depth at O' (Section 2.2): linear interpolation of the
  // table; s = t - tA in fixed point (units of h 2^-32): the cell is the
  // high word, the fraction the low word.  s <= 0 gives depth 0 (cell 0,
  // fraction 0: s = 0 does so on the general path, so the test is the
  // cell's sign), past the last entry the last value.
  const int cell = (int)(s >> 32);
  const bool neg = cell < 0;
  const bool past = cell >= C.n_table - 1;
  const int k = neg ? 0 : (past ? C.n_table - 2 : cell);
  const float f = neg ? 0.0f : __uint_as_float(((unsigned)s >> 9) | 0x3f800000u) - 1.0f;   // low word / 2^32
  const float d0 = TS ? stab[k] : __ldg(C.tab + k), d1 = TS ? stab[k + 1] : __ldg(C.tab + k + 1);
  const float d = past ? d1 : fmaf(f, d1 - d0, d0);

  // beam-model table: T(d), c3_1..3(d) / K (K = Prof<PROF>::K, folded in
  // when the table was built); past the end, the last row.  g is clamped to
  // [0, last] (a NaN depth maps to 0); its row is the truncation of g, a
  // conversion on the MUFU pipe (less busy than the FMA pipe and the ALU,
  // which the same floor from 2^23 + g rounding would use).  At g = last the
  // row is the last one, whose difference to the next is 0, and w = 0: the
  // last row exactly.
  const float g = fminf(fmaxf(d * C.lut_scale, 0.0f), C.lut_last);
  const int kk = __float2int_rz(g);   // g >= 0: the floor
  const float w = g - small_int_to_float(kk);   // in [0, 1), exact
#if DSC_LUT_SMEM
  const float4 L = TS ? slut[2 * kk] : __ldg(C.lut + 2 * kk);                 // row kk
  const float4 dL = TS ? slut[2 * kk + 1] : __ldg(C.lut + 2 * kk + 1);        // row kk+1 - row kk
#else
  const float4 L = __ldg(C.lut + 2 * kk), dL = __ldg(C.lut + 2 * kk + 1);   // row kk, row kk+1 - row kk
#endif
  const float2 Pxy = __ffma2_rn(f2(w), make_float2(dL.x, dL.y), make_float2(L.x, L.y));
  const float2 Pzw = __ffma2_rn(f2(w), make_float2(dL.z, dL.w), make_float2(L.z, L.w));

  const float2 abt = __fmul2_rn(C.ab_sad, f2(t));   // (a_t, b_t)
  const float2 axz = make_float2(fabsf(xz.x), fabsf(xz.y));
  constexpr float kK = Prof<PROF>::K;
  if (SIG) {
    float lim = (C.cutoff_k * kK) * Pxy.y;   // cutoff_k c3_1
    if (axz.x > fmaf(0.5f, abt.x, lim) || axz.y > fmaf(0.5f, abt.y, lim)) return -1.0f;
  }
  // Eq. 3 (or another profile): three pair products, arguments scaled by
  // K / c3 (for Eq. 3: 1/(sqrt(2) c3) * sqrt(log2 e)), the reciprocal of the
  // table's c3 / K
  const float c3k[3] = {Pxy.y, Pzw.x, Pzw.y};
  float F = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float inv_s = rcp_approx(c3k[i]);
    const float2 XZ = erf_pair2<PROF>(C.c2h[i], C.c2hn[i], abt, axz, inv_s);
    F = fmaf(C.c1q[i] * XZ.x, XZ.y, F);
  }
  // Eq. 2 with A = T(d) (SAD/t)^2, SAD^2 carried in c1q; rcp.approx is
  // within an ulp of 1/t
  const float it = rcp_approx(t);
  return Pxy.x * (it * it) * F;
}

__device__ __forceinline__ void load_row_const(RowConst& C, const DRow& R, const DInst& G, const float* tab) {
  C.dsf = R.sfx_s[0];
  C.tx = R.Ss[0].hi;
  C.XZh = make_float2(R.Xs[0].hi, R.Zs[0].hi);
  C.XZl = make_float2(R.Xs[0].lo, R.Zs[0].lo);
  C.ab_sad = make_float2(R.a_sad, R.b_sad);
  C.n_table = R.n_table;
  C.tab = tab;
  C.lut = G.lut;
  C.lut_scale = G.lut_scale;
  C.lut_last = (float)(G.n_lut - 1);
  const float sad2 = R.sad * R.sad;
  for (int i = 0; i < 3; ++i) { C.c1q[i] = G.c1q[i] * sad2; C.c2h[i] = G.c2h[i]; C.c2hn[i] = -G.c2h[i]; }
  C.cutoff_k = G.cutoff_k;
}

// The decisions a row maximum M gives, in FP32 (the evaluation's tile
// counts and the count pass form them with this one function, so that both
// compare the same numbers): kept is D >= thr1 = max(tau M, smallest
// denormal); a value in the refinement window (ulo, uhi) is decided in FP64;
// one at or above mlo is near the maximum; ukeep = uhi (1 + 2^-16) bounds the
// window of any final maximum a little above M.  All are non-decreasing in M.
struct Decide {
  float thr1, ulo, uhi, mlo, ukeep;
};
__device__ __forceinline__ Decide decide_at(float tau, float inv_tau_m, float M) {
  constexpr float kTiny = 1.40129846e-45f;
  constexpr float kLo = 1.0f - kRefineDelta, kHi = 1.0f + kRefineDelta;
  Decide d;
  d.thr1 = fmaxf(tau * M, kTiny);
  d.ulo = d.thr1 * kLo;
  d.uhi = d.thr1 * kHi;
  d.mlo = d.thr1 * inv_tau_m;
  d.ukeep = d.uhi * 1.0000152587890625f;        // 1 + 2^-16
  return d;
}

// the candidates [w0, w0 + wl) of an item's window (the item's first wl
// candidates past w0 are real; the rest of the last group of 4 is padding),
// profile PROF (block-uniform); TS: the depth table is in sm.tab; SIG: the
// sigma cutoff.
// Each thread takes groups of 4 consecutive candidates (four independent
// chains; a warp's 32 groups are one tile of 128), writes their values and
// columns with aligned 16-byte stores (the item starts on a tile), and keeps
// the maximum and, with SIG, the count inside the cutoff.
template <int PROF, bool TS, bool SIG>
__device__ __forceinline__ void eval_window(const RowConst& C, const LineSm& sm, int w0, int wl, float* out,
                                            int* outc, float& vmax, int& valid) {
  for (int g = 4 * (int)threadIdx.x; g < wl; g += 4 * kEvalThreads) {
    const int jj = w0 + g;                              // item-relative index of the group's first candidate
    const unsigned mmb = *reinterpret_cast<const unsigned*>(sm.map + g);
    const int lidx[4] = {(int)(mmb & 0xffu), (int)((mmb >> 8) & 0xffu), (int)((mmb >> 16) & 0xffu), (int)(mmb >> 24)};
    float D[4];
    int col[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // every entry holds a line of the item: position 0 of a window always
      // starts one, and the scan carries it on (past wl: the last line); a
      // byte index is in range of the 256-entry records in any case
      const int li = lidx[k];
      const float4 A = sm.sx[li], B = sm.zc[li];
      const int j = jj + k;
      const int ix = __float_as_int(B.z) + j;
      col[k] = __float_as_int(A.y) + j;
      D[k] = eval_pair<PROF, TS, SIG>(C, small_int_to_float(ix), A, B, sm.sf[li] + (long long)j * C.dsf, sm.tab,
                                      SMLUT);
    }
    if (g + 4 > wl) {                                   // the last real group's padding
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (g + k >= wl) { D[k] = -1.0f; col[k] = 0; }
    }
    *reinterpret_cast<float4*>(out + jj) = make_float4(D[0], D[1], D[2], D[3]);
    *reinterpret_cast<int4*>(outc + jj) = make_int4(col[0], col[1], col[2], col[3]);
    const float lmax = fmaxf(fmaxf(D[0], D[1]), fmaxf(D[2], D[3]));
    vmax = fmaxf(vmax, lmax);
    if (SIG) valid += (D[0] >= 0.0f) + (D[1] >= 0.0f) + (D[2] >= 0.0f) + (D[3] >= 0.0f);
    // the tile's count under the item's bound L (thresholds in shared
    // memory, read each time so that they hold no registers): the values at
    // or above L's kept bound ukeep, and the lanes with a value within bh of
    // bc (a superset of L's band (ulo, ukeep)) or at or above mlo (near L),
    // summed over the warp in one reduction (count in the low 8 bits).  The
    // warp's lanes in this iteration are a prefix of it (those whose group
    // starts before wl), all in one tile.
    const float ukeep = *(volatile const float*)&sm.dl_ukeep, bc = *(volatile const float*)&sm.dl_bc,
                bh = *(volatile const float*)&sm.dl_bh, mlo = *(volatile const float*)&sm.dl_mlo;
    const unsigned a = (D[0] >= ukeep) + (D[1] >= ukeep) + (D[2] >= ukeep) + (D[3] >= ukeep);
    const float md = fminf(fminf(fabsf(D[0] - bc), fabsf(D[1] - bc)), fminf(fabsf(D[2] - bc), fabsf(D[3] - bc)));
    unsigned v = a | (md < bh || lmax >= mlo ? 0x100u : 0u);
    const unsigned lane = threadIdx.x & 31u;
    const unsigned g0 = (unsigned)g - 4u * lane;        // the tile's first candidate in the window
    const unsigned nl = ((unsigned)wl - g0 + 3u) >> 2;  // lanes of this warp in the iteration
    v = __reduce_add_sync(nl >= 32u ? 0xffffffffu : (1u << nl) - 1u, v);
    static_assert(kTile == 128, "tile index by shift");
    if (lane == 0u) (*(unsigned* volatile const*)&sm.tmeta)[((unsigned)w0 + g0) >> 7] = v;
  }
}

template <int PROF, bool TS>
__device__ __forceinline__ void eval_window_mode(bool sig, const RowConst& C, const LineSm& sm, int w0, int wl,
                                                 float* out, int* outc, float& vmax, int& valid) {
  if (sig) eval_window<PROF, TS, true>(C, sm, w0, wl, out, outc, vmax, valid);
  else eval_window<PROF, TS, false>(C, sm, w0, wl, out, outc, vmax, valid);
}

// persistent: CTAs take work items from a queue; every candidate's D goes to
// vals[item_off[item] + k] and the row maximum is kept with atomicMax on the
// float bits (D >= 0)
#ifndef DSC_EVAL_MINBLOCKS
#define DSC_EVAL_MINBLOCKS 8
#endif
__global__ void __launch_bounds__(kEvalThreads, DSC_EVAL_MINBLOCKS) k_eval(EvalParams p) {
  __shared__ LineSm sm;
  const long long ni = *p.n_items;
#if DSC_LUT_SMEM
  if (threadIdx.x == 0) sm.lut_inst = -1;           // read after the first barrier below
#endif
  for (;;) {
    if (threadIdx.x == 0) {
      long long it = atomicAdd(p.item_counter, 1);
      if (it < ni) {
        if (p.item_ord) it = p.item_ord[it];
        sm.row = p.item_row[it];
      }
      sm.item = it;
    }
    __syncthreads();
    const long long item = sm.item;
    if (item >= ni) break;
    const int row = sm.row;
    // the running row maximum (every value of it is a lower bound of the
    // final one), read once for the whole item; the others read it after
    // item_lines' barriers
    const long long a_off = p.item_off[item];
    if (threadIdx.x == 0) {
      const unsigned lb = __ldcg(p.row_max + row);
      p.item_L[item] = lb;
      const Decide DL = decide_at(p.tau, p.inv_tau_m, __uint_as_float(lb));
      sm.dl_ukeep = DL.ukeep;
      // |D - bc| < bh holds for every D in (ulo, ukeep): ukeep - ulo is exact
      // (the two are within a factor 2), and the widening covers the rounding
      // of bc and of D - bc; an empty band (ulo = ukeep) gives bh = 0
      sm.dl_bc = 0.5f * (DL.ulo + DL.ukeep);
      sm.dl_bh = 0.5f * (DL.ukeep - DL.ulo) * 1.0625f;
      sm.dl_mlo = DL.mlo;
      sm.tmeta = p.tile_meta + a_off / kTile;
    }
    const DRow& R = p.rows[row];
    const DInst& G = p.inst[R.inst];
    const int mode = G.cutoff_mode;
    const bool sig = mode == 1;
#if DSC_LUT_SMEM
    // read before item_lines' barriers; thread 0 updates it after them
    const bool lut_stale = sm.lut_inst != R.inst;
#endif
    const int padded = (int)(p.item_off[item + 1] - a_off);   // the counted range, whole tiles
    const int total = min(item_lines(sm, R, p.slices, row, mode, G.nx, G.ny, item - p.row_item_base[row]),
                          padded);                             // never past the counted range
    // the padding past the last real group, to the end of its tile (fewer
    // than 32 groups): -1, never kept; written first, so that padded is not
    // held through the evaluation
    for (int g = ((total + 3) & ~3) + 4 * (int)threadIdx.x; g < padded; g += 4 * kEvalThreads) {
      *reinterpret_cast<float4*>(p.vals + a_off + g) = make_float4(-1.0f, -1.0f, -1.0f, -1.0f);
      *reinterpret_cast<int4*>(p.cols + a_off + g) = make_int4(0, 0, 0, 0);
    }
    RowConst C;
    load_row_const(C, R, G, p.tables + (size_t)row * p.table_stride);
    // the row's depth table into shared memory when it fits (block-uniform);
    // the previous item's readers finished at its closing barrier, and this
    // item's first reader comes after the barrier in item_map
#if DSC_LUT_SMEM
    // the depth table and the beam-model table both staged, or neither
    const bool ts = R.n_table <= kTabSmem && G.n_lut <= kLutSmem;
    if (ts && lut_stale) {
      for (int k = threadIdx.x; k < 2 * G.n_lut; k += kEvalThreads) sm.lut[k] = C.lut[k];
      if (threadIdx.x == 0) sm.lut_inst = R.inst;     // read after the next barrier (item_map)
    }
#else
    const bool ts = R.n_table <= kTabSmem;
#endif
    if (ts)
      for (int k = threadIdx.x; k < R.n_table; k += kEvalThreads) sm.tab[k] = C.tab[k];
    float* out = p.vals + a_off;
    int* outc = p.cols + a_off;
    float vmax = 0.0f;
    int valid = (!sig && threadIdx.x == 0) ? total : 0;   // outside the sigma cutoff every candidate counts
    for (int w0 = 0; w0 < total; w0 += kWindow) {
      const int wl = min(kWindow, total - w0);
      item_map(sm, w0, wl);
      if (ts) {
        switch (G.profile) {
          case 1: eval_window_mode<1, true>(sig, C, sm, w0, wl, out, outc, vmax, valid); break;
          case 2: eval_window_mode<2, true>(sig, C, sm, w0, wl, out, outc, vmax, valid); break;
          default: eval_window_mode<0, true>(sig, C, sm, w0, wl, out, outc, vmax, valid); break;
        }
      } else {
        switch (G.profile) {
          case 1: eval_window_mode<1, false>(sig, C, sm, w0, wl, out, outc, vmax, valid); break;
          case 2: eval_window_mode<2, false>(sig, C, sm, w0, wl, out, outc, vmax, valid); break;
          default: eval_window_mode<0, false>(sig, C, sm, w0, wl, out, outc, vmax, valid); break;
        }
      }
      __syncthreads();
    }
    // row max and candidates inside the cutoff (one atomic per warp)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      valid += __shfl_xor_sync(0xffffffffu, valid, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (vmax > 0.0f) atomicMax(p.row_max + row, __float_as_uint(vmax));
      if (valid) atomicAdd((unsigned long long*)(p.row_cand + row), (unsigned long long)valid);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_row_bound: a lower bound of every row's maximum before the evaluation,
// one warp per row.  Past the depth dT where the depth-dose factor T(d) of
// the beam model peaks, every factor of Eq. 2 falls along the beamlet axis,
// and laterally the dose is largest on the axis, so a row's maximum lies by
// the axis at a depth below dT.  Up to 32 points of the axis, a voxel
// apart where they fit, span the stretch where the radiological depth (the
// row's table) lies in [dT - 10 mm, dT + 2 mm]; the 8 voxels whose centres
// surround each point, those that are candidates of the row, are evaluated
// with the evaluation's own functions, (point, voxel) pairs spread over the
// lanes.  The largest value, times
// (1 - 2^-18) so that it stays below the evaluation's value of the same
// voxel under any contraction of the same formulas, seeds row_max.  The
// bound only decides which tiles the count pass takes from the evaluation's
// counts; a bound that is too low costs their values' reads.
// ---------------------------------------------------------------------------
// the first k in [0, n) with a[k] >= x (n if none); a non-decreasing, the
// warp probes 32 entries at a time
__device__ __forceinline__ int warp_lower_bound(const float* __restrict__ a, int n, float x, int lane) {
  int lo = 0, hi = n;                                  // a[lo - 1] < x, a[hi] >= x (or hi = n)
#pragma unroll 1
  while (lo < hi) {                                    // warp-uniform
    const int step = (hi - lo + 31) / 32;
    const int k = lo + lane * step;
    const unsigned b = __ballot_sync(0xffffffffu, k < hi && a[k] >= x);
    if (b == 0u) {
      lo = min(lo + 31 * step, hi - 1) + 1;            // past the last probe below hi
    } else {
      const int f = __ffs(b) - 1;
      hi = lo + f * step;
      if (f > 0) lo = lo + (f - 1) * step + 1;
    }
  }
  return lo;
}

template <int PROF, bool SIG>
__device__ float bound_voxel(const RowConst& C, const DRow& R, int ix, int iy, int iz) {
  ff s0, x0, z0;
  line_base(R, iy, iz, s0, x0, z0);
  const float4 A = make_float4(R.tA_f + s0.hi, 0.0f, x0.hi, z0.hi);
  const float4 B = make_float4(x0.lo, z0.lo, 0.0f, 0.0f);
  const long long sf = R.sfx0 + (long long)iy * R.sfx_s[1] + (long long)iz * R.sfx_s[2] + (long long)ix * C.dsf;
  return eval_pair<PROF, false, SIG>(C, small_int_to_float(ix), A, B, sf, nullptr, nullptr);
}

__global__ void __launch_bounds__(128) k_row_bound(const DInst* __restrict__ inst, const DRow* __restrict__ rows,
                                                   int nrows, const float* __restrict__ tables, int stride, SliceTab T,
                                                   unsigned* row_max) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (row >= nrows) return;                            // warp-uniform
  const DRow& R = rows[row];
  const int nzr = row_slices(R, T.stride);
  if (nzr <= 0 || R.n_table < 2) return;
  const DInst& G = inst[R.inst];
  const float* tab = tables + (size_t)row * stride;
  const int k0 = warp_lower_bound(tab, R.n_table, G.d_peak - 10.0f, lane);
  const int k1 = warp_lower_bound(tab, R.n_table, nextafterf(G.d_peak + 2.0f, CUDART_INF_F), lane) - 1;
  if (k0 > k1) return;
  const float hd = (float)G.hd;
  const float ta = R.tA_f + (float)k0 * hd, span = (float)(k1 - k0) * hd;
  const float vmin = (float)fmin(G.dx, fmin(G.dy, G.dz));
  const int np = min(32, (int)(span / vmin) + 1);
  const float dt = np > 1 ? span / (float)(np - 1) : 0.0f;
  const int* pre = T.pre + (size_t)row * T.stride;
  const int* ylo = T.lo + (size_t)row * T.stride;
  const LineCut L(R, G.cutoff_mode, G.nx);
  RowConst C;
  load_row_const(C, R, G, tab);
  const bool sig = G.cutoff_mode == 1;
  float best = 0.0f;
  // (point, voxel) pairs over the lanes
#pragma unroll 1
  for (int e = lane; e < 8 * np; e += 32) {
    const float t = ta + (float)(e >> 3) * dt;
    const int c = e & 7;
    const int ix = (int)floorf(((float)R.S[0] + t * (float)R.e[0] - (float)G.ox) / (float)G.dx - 0.5f) + (c & 1);
    const int iy = (int)floorf(((float)R.S[1] + t * (float)R.e[1] - (float)G.oy) / (float)G.dy - 0.5f) + ((c >> 1) & 1);
    const int iz = (int)floorf(((float)R.S[2] + t * (float)R.e[2] - (float)G.oz) / (float)G.dz - 0.5f) + ((c >> 2) & 1);
    const int sl = iz - R.iz0;
    if (ix < 0 || ix >= G.nx || iy < 0 || iy >= G.ny || sl < 0 || sl >= nzr) continue;
    const int y0 = ylo[sl];
    if (iy < y0 || iy >= y0 + (pre[sl + 1] - pre[sl])) continue;   // a line the row enumerates
    int lo;
    const int len = line_interval(L, iy, iz, lo);
    if (ix < lo || ix >= lo + len) continue;           // a candidate of the line
    float D;
    switch (G.profile) {
      case 1: D = sig ? bound_voxel<1, true>(C, R, ix, iy, iz) : bound_voxel<1, false>(C, R, ix, iy, iz); break;
      case 2: D = sig ? bound_voxel<2, true>(C, R, ix, iy, iz) : bound_voxel<2, false>(C, R, ix, iy, iz); break;
      default: D = sig ? bound_voxel<0, true>(C, R, ix, iy, iz) : bound_voxel<0, false>(C, R, ix, iy, iz); break;
    }
    best = fmaxf(best, D);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  best *= 0.99999618530273437500f;                     // 1 - 2^-18
  if (lane == 0 && best > 0.0f) atomicMax(row_max + row, __float_as_uint(best));
}

// ---------------------------------------------------------------------------
// the lateral-profile tail T(y), y >= 0 in units of the spread, with the
// evaluation's own primitives and constants (argument scale K, the fitted
// erfc, rcp.approx, ex2.approx), four values per thread in packed FP32x2 as
// erf_pair2 forms a term's four tails (the same shared reciprocal), beside
// CUDA's own function of the same tail
// ---------------------------------------------------------------------------
template <int PROF>
__device__ __forceinline__ void tail4(float2 ya, float2 yb, float2& ra, float2& rb) {
  const float2 va = __fmul2_rn(ya, f2(Prof<PROF>::K)), vb = __fmul2_rn(yb, f2(Prof<PROF>::K));
  float2 tpa, ea, tpb, eb;
  if (PROF == 0) {
    float2 ta, tb;
    erfc_recips(va, vb, ta, tb);                       // the evaluation's four denominators of a term
    erfc_parts(ta, va, kErfcC2, tpa, ea);
    erfc_parts(tb, vb, kErfcC2, tpb, eb);
  } else {
    ea = make_float2(ex2_approx(-va.x), ex2_approx(-va.y));
    eb = make_float2(ex2_approx(-vb.x), ex2_approx(-vb.y));
    tpa = PROF == 1 ? f2(1.0f) : rcp2(__ffma2_rn(ea, f2(0.5f), f2(0.5f)));
    tpb = PROF == 1 ? f2(1.0f) : rcp2(__ffma2_rn(eb, f2(0.5f), f2(0.5f)));
  }
  ra = __fmul2_rn(tpa, ea);
  rb = __fmul2_rn(tpb, eb);
}

__global__ void k_tail_probe(int profile, const float* __restrict__ y, long long n, float* __restrict__ ours,
                             float* __restrict__ cuda_ref) {
  const long long i = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  float yy[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) yy[h] = i + h < n ? y[i + h] : 0.0f;
  float2 ra, rb;
  const float2 ya = make_float2(yy[0], yy[1]), yb = make_float2(yy[2], yy[3]);
  if (profile == 1) tail4<1>(ya, yb, ra, rb);
  else if (profile == 2) tail4<2>(ya, yb, ra, rb);
  else tail4<0>(ya, yb, ra, rb);
  const float r[4] = {ra.x, ra.y, rb.x, rb.y};
  for (int h = 0; h < 4 && i + h < n; ++h) {
    const float a = yy[h];
    ours[i + h] = r[h];
    float c;
    if (profile == 1) c = expf(-1.41421356237309504880f * a);                     // exp(-sqrt 2 y)
    else if (profile == 2) {
      const float q = expf(-1.81379936423421785059f * a);                          // exp(-pi y / sqrt 3)
      c = 2.0f * q / (1.0f + q);
    } else c = erfcf(0.70710678118654752440f * a);                                 // erfc(y / sqrt 2)
    cuda_ref[i + h] = c;
  }
}

// ---------------------------------------------------------------------------
// beam-model table as the evaluation reads it: entry k = {row k, row k+1 -
// row k} (the FP32 difference the linear interpolation forms; zero for the
// last row), so one interpolation is one FMA per column.  The three c3
// columns are divided by the profile's argument scale K first (one rounding),
// so the evaluation's 1/s is one reciprocal.
// ---------------------------------------------------------------------------
__global__ void k_lut_pairs(const float4* __restrict__ rows, int n, int profile, float4* __restrict__ pairs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float ik = profile == 1 ? 1.0f / Prof<1>::K : (profile == 2 ? 1.0f / Prof<2>::K : 1.0f / Prof<0>::K);
  float4 a = rows[k];
  float4 b = k + 1 < n ? rows[k + 1] : a;
  a = make_float4(a.x, a.y * ik, a.z * ik, a.w * ik);
  b = make_float4(b.x, b.y * ik, b.z * ik, b.w * ik);
  pairs[2 * k] = a;
  pairs[2 * k + 1] = make_float4(__fsub_rn(b.x, a.x), __fsub_rn(b.y, a.y), __fsub_rn(b.z, a.z), __fsub_rn(b.w, a.w));
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
// compaction: kept = D > 0 and D >= tau * row max, over tiles of kTile
// candidates, one warp per tile (kTilePer consecutive candidates per lane,
// vector loads, no block barriers).  Work items are padded to whole tiles,
// so every tile lies in one item and one row:
//   k_tile_map    the row of every tile
//   k_tile_count  kept entries per tile
//   (scan)        tile output offsets; an item's output starts at its first
//                 tile's offset
//   k_tile_write  warp scan within the tile, kept entries staged in shared
//                 memory and written coalesced
// ---------------------------------------------------------------------------
constexpr int kTileWarps = kEvalThreads / 32;
static_assert(kTilePer == 4, "one 16-byte vector per lane and array");

struct TileKeep {
  float D[kTilePer];
  int C[kTilePer];
  unsigned keep;
  int cnt;            // count pass: kept entries of the lane
};

// the lane's kTilePer candidate values (and columns) from [p0, p0 + kTilePer);
// the candidate count is a whole number of tiles
template <bool kCols>
__device__ __forceinline__ void tile_load(const CompactParams& p, long long p0, TileKeep& K) {
  const float4 v = __ldcs(reinterpret_cast<const float4*>(p.vals + p0));
  K.D[0] = v.x; K.D[1] = v.y; K.D[2] = v.z; K.D[3] = v.w;
  if (kCols) {
    const int4 c = __ldcs(reinterpret_cast<const int4*>(p.cols + p0));
    K.C[0] = c.x; K.C[1] = c.y; K.C[2] = c.z; K.C[3] = c.w;
  }
}

// keep flags of the lane's loaded candidates, all of the tile's row
template <bool kCols>
__device__ __forceinline__ void tile_decide(const CompactParams& p, long long p0, long long tile, TileKeep& K) {
  const bool bf16 = kCols && p.value_dtype == 1;
  const int r = p.tile_row[tile];
  float thr, scale = 1.0f;
  if (kCols) {
    thr = p.tile_thr[tile];
    if (bf16) scale = p.tile_scale[tile];
  } else {
    // the count pass forms the tile's threshold (the row maxima are final)
    // and leaves it, and the BF16 scale, for the write pass
    thr = p.tau * __uint_as_float(p.row_max[r]);
    if ((threadIdx.x & 31) == 0) {
      p.tile_thr[tile] = thr;
      if (p.value_dtype == 1) p.tile_scale[tile] = p.slot->beam_scale[p.rows[r].beam];
    }
  }
  // kept = D > 0 and D >= thr, i.e. D >= max(thr, smallest denormal); the
  // padding holds -1
  constexpr float kTiny = 1.40129846e-45f;
  const float thr1 = fmaxf(thr, kTiny);
  if (kCols) {
    unsigned kp = 0;
#pragma unroll
    for (int i = 0; i < kTilePer; ++i)
      if (K.D[i] >= thr1) {
        kp |= 1u << i;
        if (bf16) K.D[i] = __fdiv_rn(K.D[i], scale);
      }
    K.keep = kp;
    return;
  }
  // count pass: outside the refinement window (ulo, uhi) the decision
  // D >= thr1 is D >= uhi (the window is empty when thr1 is the smallest
  // denormal: no value lies strictly between ulo and uhi); a value inside it,
  // or near the row maximum, is handled after the loop
  const Decide DM = decide_at(p.tau, p.inv_tau_m, __uint_as_float(p.row_max[r]));
  const float ulo = DM.ulo, uhi = DM.uhi, mlo = DM.mlo;
  unsigned keep = 0, special = 0;
#pragma unroll
  for (int i = 0; i < kTilePer; ++i) {
    const float D = K.D[i];
    const bool above = D >= uhi;
    if (above) keep |= 1u << i;
    if ((D > ulo && !above) || D >= mlo) special |= 1u << i;
  }
  if (special) {
    // candidates near their threshold or their row maximum (rare).  A value
    // within kRefineDelta of its threshold does not settle the decision in
    // FP32: it is listed for the FP64 re-evaluation, which adds it to the
    // count if kept, and it leaves this count.  A value within kRefineDelta
    // of the row maximum goes to the row's slots, from which the
    // re-evaluation takes the FP64 maximum; a row with more such values than
    // slots is listed once, and its FP64 maximum comes from a scan of the row
    // (k_refine_rowmax).  A full list leaves the FP32 decision in place (and
    // is counted).
    if ((unsigned)r >= (unsigned)p.nrows) {           // checked: skip and flag
      atomicOr(p.slot->status, kStatusIndex);
    } else {
#pragma unroll
      for (int i = 0; i < kTilePer; ++i) {            // static positions: K stays in registers
        if (!(special & (1u << i))) continue;
        const long long pos = p0 + i;
        const float D = K.D[i];
        if (D > ulo && D < uhi) {
          const unsigned long long e = atomicAdd(p.rcount, 1ull);
          if (e < (unsigned long long)p.cap_u) p.rlist_u[e] = refine_entry(pos, r);
          else if (D >= thr1) keep |= 1u << i;        // list full: the FP32 decision
        }
        if (D >= mlo) {
          atomicAdd(p.rcount + 1, 1ull);
          const int k = atomicAdd(p.mcount + r, 1);
          if (k < kMaxSlots) {
            p.mslot[(size_t)r * kMaxSlots + k] = pos;
          } else if (k == kMaxSlots) {                 // the row overflows its slots: list it once
            const unsigned long long e = atomicAdd(p.rcount + 2, 1ull);
            if (e < (unsigned long long)p.nrows) p.ovf_rows[e] = r;
          }
        }
      }
    }
  }
  K.keep = keep;
  K.cnt = __popc(keep);
}

// the item and row of every tile, from the work decomposition alone (it
// runs before the evaluation), and the evaluation queue's order of the items
// (item_ord: the size classes from the largest, each item at its class's
// first position plus its rank in the class, from k_count; none when null);
// one warp per item, a tile per lane
__global__ void k_tile_map(const long long* __restrict__ item_off, const long long* __restrict__ n_items_p,
                           const int* __restrict__ item_row, int* tile_item, int* tile_row,
                           const int* __restrict__ ord_cnt, const int* __restrict__ item_crank, int* item_ord) {
  const long long ni = *n_items_p;
  const int lane = threadIdx.x & 31;
  // the classes' first positions: an exclusive scan of the class counts
  int pre = 0;
  if (item_ord) {
    const int v = lane < kOrderClasses ? ord_cnt[lane] : 0;
    pre = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += x;
    }
    pre -= v;
  }
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < ni; i += nw) {
    if (item_ord) {
      const int cr = item_crank[i];
      const int first = __shfl_sync(0xffffffffu, pre, cr >> kOrderRankBits);
      if (lane == 0) item_ord[first + (cr & ((1 << kOrderRankBits) - 1))] = (int)i;
    }
    const long long a = item_off[i] / kTile, b = item_off[i + 1] / kTile;
    const int r = item_row[i];
    for (long long t = a + lane; t < b; t += 32) {
      tile_item[t] = (int)i;
      tile_row[t] = r;
    }
  }
}

#ifndef DSC_COMPACT_MINB
#define DSC_COMPACT_MINB 12
#endif
// the count pass holds no columns: 16 CTAs per SM (32 registers) keep more
// of its loads in flight
#ifndef DSC_COUNT_MINB
#define DSC_COUNT_MINB 16
#endif

// kept entries per tile.  Each lane takes one tile and forms its threshold
// from the final row maximum M.  The evaluation counted the tile against the
// bound L its item started with: when no value lay in L's band or near L
// (flag clear) and M's window lies below L's kept bound (M.uhi <= L.ukeep),
// every value is at or below L.ulo <= M.ulo (dropped) or at or above
// L.ukeep >= M.uhi (kept), none is near M, and that count is the tile's.
// The warp counts the other tiles from their values, one at a time.
__global__ void __launch_bounds__(kEvalThreads, DSC_COUNT_MINB) k_tile_count(CompactParams p, int* tile_cnt) {
  const int lane = threadIdx.x & 31;
  const long long n_tiles = p.n_cand / kTile;
  const long long t0 = ((long long)blockIdx.x * kTileWarps + (threadIdx.x >> 5)) * 32;
  if (t0 >= n_tiles) return;                           // warp-uniform
  const long long t = t0 + lane;
  bool slow = false;
  if (t < n_tiles) {
    const int r = p.tile_row[t];
    const float M = __uint_as_float(p.row_max[r]);
    p.tile_thr[t] = p.tau * M;
    if (p.value_dtype == 1) p.tile_scale[t] = p.slot->beam_scale[p.rows[r].beam];
    const unsigned meta = p.tile_meta[t];
    const Decide DM = decide_at(p.tau, p.inv_tau_m, M);
    const Decide DL = decide_at(p.tau, p.inv_tau_m, __uint_as_float(p.item_L[p.tile_item[t]]));
    if ((meta >> 8) == 0u && DM.uhi <= DL.ukeep) tile_cnt[t] = (int)(meta & 0xffu);
    else slow = true;
  }
  unsigned todo = __ballot_sync(0xffffffffu, slow);
  if (lane == 0 && todo) atomicAdd(p.rcount + 3, (unsigned long long)__popc(todo));
  while (todo) {                                       // warp-uniform
    const long long tile = t0 + (__ffs(todo) - 1);
    todo &= todo - 1u;
    const long long p0 = tile * kTile + (long long)lane * kTilePer;
    TileKeep K;
    tile_load<false>(p, p0, K);
    tile_decide<false>(p, p0, tile, K);
    int c = K.cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) tile_cnt[tile] = c;
  }
}

__global__ void __launch_bounds__(kEvalThreads, DSC_COMPACT_MINB) k_tile_write(CompactParams p,
                                                                              const long long* __restrict__ tile_off) {
  __shared__ int s_col[kTileWarps][kTile];
  __shared__ float s_val[kTileWarps][kTile];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long n_tiles = p.n_cand / kTile;
  const long long t0 = ((long long)blockIdx.x * kTileWarps + w) * kTilesPerWarp;
  if (t0 >= n_tiles) return;                           // warp-uniform
  // the tiles' output offsets first: a tile that keeps nothing is not read
  static_assert(kTilesPerWarp == 2, "three offsets");
  const long long o0 = tile_off[t0], o1 = tile_off[min(t0 + 1, n_tiles)], o2 = tile_off[min(t0 + 2, n_tiles)];
  TileKeep K[kTilesPerWarp];
#pragma unroll
  for (int u = 0; u < kTilesPerWarp; ++u) {
    if (t0 + u < n_tiles && (u == 0 ? o1 > o0 : o2 > o1))
      tile_load<true>(p, (t0 + u) * kTile + (long long)lane * kTilePer, K[u]);
    else K[u] = TileKeep{};                             // not read: defined on every path, so K stays in registers
  }
#pragma unroll
  for (int u = 0; u < kTilesPerWarp; ++u) {
    const long long tile = t0 + u;
    const long long prefix = u == 0 ? o0 : o1;
    if (tile >= n_tiles || (u == 0 ? o1 : o2) == prefix) continue;   // warp-uniform: past the end, or nothing kept
    tile_decide<true>(p, tile * kTile + (long long)lane * kTilePer, tile, K[u]);
    const int cnt = __popc(K[u].keep);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    int q = incl - cnt;
#pragma unroll
    for (int i = 0; i < kTilePer; ++i) {
      if (K[u].keep & (1u << i)) {
        s_col[w][q] = K[u].C[i];
        s_val[w][q] = K[u].D[i];
        ++q;
      }
    }
    __syncwarp();
    int* col = p.slot->col;
    if (p.value_dtype == 1) {
      __nv_bfloat16* val = (__nv_bfloat16*)p.slot->val;
      for (int k = lane; k < tot; k += 32) {
        __stcs(col + prefix + k, s_col[w][k]);
        __stcs(reinterpret_cast<unsigned short*>(val) + prefix + k,
               __bfloat16_as_ushort(__float2bfloat16_rn(s_val[w][k])));
      }
    } else {
      float* val = (float*)p.slot->val;
      for (int k = lane; k < tot; k += 32) {
        __stcs(col + prefix + k, s_col[w][k]);
        __stcs(val + prefix + k, s_val[w][k]);
      }
    }
    __syncwarp();                                      // the staging buffer is reused by the next tile
  }
}

// the kept count before work item i: the output offset of its first tile, or
// the total when it starts past the end
__device__ __forceinline__ long long kept_before_item(const long long* __restrict__ item_off,
                                                      const long long* __restrict__ tile_off, long long ni,
                                                      long long n_cand, long long total, long long i) {
  return (i >= ni || item_off[i] >= n_cand) ? total : tile_off[item_off[i] / kTile];
}

// CSR row pointers of one instance (rows [row_base, row_base + nrows)),
// relative to the instance's first output slot, which goes to inst_begin.
// Row r starts at item row_item_base[r].
__global__ void k_row_ptr(const long long* __restrict__ row_item_base, const long long* __restrict__ item_off,
                          const long long* __restrict__ tile_off, const long long* __restrict__ n_items_p,
                          long long n_cand, int row_base, int nrows, long long rp_off, int inst, int last,
                          const OutSlot* __restrict__ slot) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const long long ni = *n_items_p, total = tile_off[n_cand / kTile];
  const long long b = kept_before_item(item_off, tile_off, ni, n_cand, total, row_item_base[row_base]);
  if (r <= nrows)
    slot->row_ptr[rp_off + r] =
        kept_before_item(item_off, tile_off, ni, n_cand, total, row_item_base[row_base + r]) - b;
  if (r == 0) {
    slot->inst_begin[inst] = b;
    if (last) slot->inst_begin[inst + 1] = total;
  }
}

// the start of a computation: its output pointers into the plan's slot, the
// status and the summary cleared and, for FP32 values, the per-beam scales
// set to 1.  The pointers travel as the launch's argument, so the host
// stages nothing (a copy from pageable host memory may wait on the stream).
__global__ void k_out_init(OutSlot* __restrict__ d_slot, OutSlot q, int ninst, int nbeams, int unit_scale) {
  const int t = threadIdx.x;
  if (t == 0) *d_slot = q;
  if (q.summary) {
    for (int k = t; k < 1 + 2 * ninst; k += blockDim.x) q.summary[k] = 0;
  } else if (t == 0) {
    *q.status = 0;
  }
  if (unit_scale)
    for (int b = t; b < nbeams; b += blockDim.x) q.beam_scale[b] = 1.0f;
}

// the end of a computation, one thread per entry of the launch's row
// pointers (all instances) and per row: each instance's row pointers, as
// k_row_ptr forms them (instance k holds entries [inst_rp[k], inst_rp[k + 1]),
// nrows_k + 1 of them, and its first row is inst_rp[k] - k); the per-row
// statistics; and refine = {pairs listed near a threshold (within the list's
// capacity), near-maximum candidates, listed pairs past the capacity (their
// decision stayed FP32), tiles counted from their values}
__global__ void k_finish(const long long* __restrict__ row_item_base, const long long* __restrict__ item_off,
                         const long long* __restrict__ tile_off, const long long* __restrict__ n_items_p,
                         long long n_cand, const long long* __restrict__ inst_rp, int ninst,
                         const unsigned* __restrict__ row_max, const long long* __restrict__ row_cand, int nrows,
                         const unsigned long long* __restrict__ rcount, int cap_u, const OutSlot* __restrict__ slot) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < inst_rp[ninst]) {
    int lo = 0, hi = ninst - 1;                         // the instance: inst_rp[k] <= t < inst_rp[k + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (inst_rp[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const long long ni = *n_items_p, total = tile_off[n_cand / kTile];
    const long long r = t - inst_rp[lo];
    const long long row_base = inst_rp[lo] - lo;
    const long long b = kept_before_item(item_off, tile_off, ni, n_cand, total, row_item_base[row_base]);
    const long long v = kept_before_item(item_off, tile_off, ni, n_cand, total, row_item_base[row_base + r]) - b;
    slot->row_ptr[t] = v;
    if (r == 0) {
      slot->inst_begin[lo] = b;
      if (lo == ninst - 1) slot->inst_begin[ninst] = total;
      if (slot->summary) slot->summary[1 + 2 * lo] = b;
    }
    if (t == inst_rp[lo + 1] - 1 && slot->summary) slot->summary[2 + 2 * lo] = v;   // the last entry: the kept count
  }
  if (t < nrows) {
    slot->row_max[t] = row_max[t];
    slot->row_cand[t] = row_cand[t];
  }
  if (t == 0 && slot->refine) {
    const unsigned long long cap = (unsigned long long)cap_u, n0 = rcount[0];
    slot->refine[0] = n0 < cap ? n0 : cap;
    slot->refine[1] = rcount[1];
    slot->refine[2] = n0 > cap ? n0 - cap : 0ull;
    slot->refine[3] = rcount[3];
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

// the same scan in one block, for short inputs (one launch instead of three):
// each thread takes a contiguous run, the block scans the run totals
__global__ void __launch_bounds__(1024) k_scan_small(const int* __restrict__ in, const long long* n_ptr,
                                                     long long n_const, long long* out) {
  __shared__ long long ws[32];
  const long long n = n_ptr ? *n_ptr : n_const;
  const long long per = (n + 1023) / 1024;
  const long long a = threadIdx.x * per, b = min(a + per, n);
  long long s = 0;
  for (long long i = a; i < b; ++i) s += (long long)in[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) ws[w] = incl;
  __syncthreads();
  if (w == 0) {
    const long long v = ws[lane];
    long long vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long x = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += x;
    }
    ws[lane] = vi - v;
    if (lane == 31) out[n] = vi;                    // total
  }
  __syncthreads();
  long long run = ws[w] + incl - s;
  for (long long i = a; i < b; ++i) {
    out[i] = run;
    run += (long long)in[i];
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

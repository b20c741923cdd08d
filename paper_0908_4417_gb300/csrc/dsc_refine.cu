// dsc_refine.cu -- the decisions FP32 cannot settle, re-evaluated in FP64.
//
// The evaluation computes every D_ij in FP32 with a relative error below
// about 3e-6 (the fitted erfc, FP32 arguments, erf pairs that partly cancel
// in the lateral tails).  Two kinds of decision are closer than that:
//   * keep or drop, for a value within kRefineDelta of tau * M_j;
//   * which candidate is the row maximum M_j itself, for values within
//     kRefineDelta of the FP32 maximum.
// The count pass lists both kinds (a few thousand pairs per step).  Here each
// listed pair is evaluated again in FP64 from the same inputs: the voxel
// centre, the beamlet frame and entry point (FP64 from the set-up), the
// row's depth table (Section 2.2) and the beam model as given, Eq. 2 with the
// profile's erf pair (Eq. 3).  One kernel, a warp per listed pair: the warp
// evaluates the pair and its row's near-maximum candidates (the row maximum
// M_j in FP64), two pairs at a time in half-warps, the twelve tails of a pair
// spread over twelve lanes, and decides against tau * M_j in FP64.  The
// kernel is a single short wave: its time is a few pairs' FP64 latency.  The
// refined value is
// written back, and where its FP32 rounding falls on the other side of the
// compaction's FP32 threshold it is set to that threshold (kept) or one ulp
// below it (dropped), a change no larger than the gap between the FP32 and
// FP64 thresholds (a few 1e-6 relative); kept pairs are added to their tile's
// count.  The FP64 depth table is the FP32 one widened, which limits
// the refined value to about 3e-7 relative: decisions farther than 1e-6 from
// the threshold are exact.
#include "dsc_internal.h"

namespace dsc {
namespace {

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kSqrt3OverPi = 0.55132889542179204315;   // sqrt 3 / pi

// 2 G(u s) for u >= 0: the tail of the lateral kernel at a distance of u
// times its scale s, from the argument w = u * kTailArg[profile]
__device__ double tail2(int profile, double w) {
  if (profile == 1) return exp(-w);                      // Laplace
  if (profile == 2) {                                    // logistic
    const double e = exp(-w);
    return 2.0 * e / (1.0 + e);
  }
  return erfc(w);                                        // Gaussian: w = u / sqrt 2
}

// D for the pair (row R, voxel col) in FP64, one half-warp per pair.  The
// FP64 pipe runs two threads per cycle per SM, so each step runs on as few
// lanes as it needs: sub-lane 0 forms the geometry, the depth and the beam
// model, and the reciprocal scales of the three terms, and broadcasts them;
// sub-lanes 0..11 take one tail each (term i = sub / 4; 4i, 4i+1: X at y1,
// y2; 4i+2, 4i+3: Z); sub-lane 0 forms the sum of Eq. 3 from the tails
// shuffled within the half.  The result is valid in sub-lane 0 of each half;
// both halves must call together.
__device__ double eval_pair64_half(const DRow& R, const DInst& G, const DBeam& B, const float* tab, int col,
                                   int sub) {
  double t = 0.0, xp = 0.0, zp = 0.0, ts = 0.0, T = 0.0, is0 = 0.0, is1 = 0.0, is2 = 0.0;
  if (sub == 0) {
    // reciprocals independent of the pair, off its dependency chain
    const double ihd = 1.0 / G.hd, glut = (G.n_lut - 1) / G.d_max, isad = 1.0 / B.sad;
    const int nxy = G.nx * G.ny;
    const int iz = col / nxy;
    const int rem = col - iz * nxy;
    const int iy = rem / G.nx, ix = rem - iy * G.nx;
    // voxel centre relative to the source; t, x', z' on the beamlet frame (Fig. 1)
    const double w0 = G.ox + (ix + 0.5) * G.dx - R.S[0];
    const double w1 = G.oy + (iy + 0.5) * G.dy - R.S[1];
    const double w2 = G.oz + (iz + 0.5) * G.dz - R.S[2];
    t = w0 * R.e[0] + w1 * R.e[1] + w2 * R.e[2];
    xp = w0 * R.x[0] + w1 * R.x[1] + w2 * R.x[2];
    zp = w0 * R.z[0] + w1 * R.z[1] + w2 * R.z[2];
    ts = 0.5 * t * isad;                                 // half the field width per unit side at t
    // radiological depth at O' (Section 2.2): the table, linearly
    double d = 0.0;
    const double s = t - R.tA;
    if (R.n_table > 0 && s > 0.0) {
      const double f = s * ihd, kf = floor(f);
      if (!(kf < R.n_table - 1)) {                   // also a NaN s: the last entry
        d = tab[R.n_table - 1];
      } else {
        const int k = (int)kf;
        d = (double)tab[k] + (f - kf) * ((double)tab[k + 1] - (double)tab[k]);
      }
    }
    // beam model at d: T and c3_1..3, linearly between rows, the last row beyond
    double c3[3];
    double g = d * glut;
    if (!(g > 0.0)) g = 0.0;                          // also a NaN depth: the first row
    if (g >= G.n_lut - 1) {
      const float4 r = G.lut_rows[G.n_lut - 1];
      T = r.x; c3[0] = r.y; c3[1] = r.z; c3[2] = r.w;
    } else {
      const int k = (int)floor(g);
      const double wt = g - k;
      const float4 a = G.lut_rows[k], b = G.lut_rows[k + 1];
      T = a.x + wt * ((double)b.x - a.x);
      c3[0] = a.y + wt * ((double)b.y - a.y);
      c3[1] = a.z + wt * ((double)b.z - a.z);
      c3[2] = a.w + wt * ((double)b.w - a.w);
    }
    // the tail argument per unit distance: 1 / (s kTailArg), s the term's
    // scale (c3 for the Gaussian, c3 / sqrt 2 Laplace, c3 sqrt 3 / pi logistic)
    const double k = G.profile == 1 ? 1.0 / kSqrt2 : (G.profile == 2 ? kSqrt3OverPi : kSqrt2);
    is0 = 1.0 / (c3[0] * k);
    is1 = 1.0 / (c3[1] * k);
    is2 = 1.0 / (c3[2] * k);
  }
  t = __shfl_sync(0xffffffffu, t, 0, 16);
  xp = __shfl_sync(0xffffffffu, xp, 0, 16);
  zp = __shfl_sync(0xffffffffu, zp, 0, 16);
  ts = __shfl_sync(0xffffffffu, ts, 0, 16);
  is0 = __shfl_sync(0xffffffffu, is0, 0, 16);
  is1 = __shfl_sync(0xffffffffu, is1, 0, 16);
  is2 = __shfl_sync(0xffffffffu, is2, 0, 16);
  // this lane's tail: 2 G(y) with y1 = (|x| - h) / s, y2 = (|x| + h) / s,
  // 2 G(y) = 2 - 2 G(-y) for y < 0 (the tails never cancel)
  double v = 0.0;
  if (sub < 12) {
    const int i = sub >> 2;
    const bool zax = (sub & 2) != 0, second = (sub & 1) != 0;
    const double h = G.c2d[i] * (zax ? B.b : B.a) * ts;           // c2 a_t / 2 (b_t for Z)
    const double ax = fabs(zax ? zp : xp);
    const double w = (second ? ax + h : ax - h) * (i == 0 ? is0 : (i == 1 ? is1 : is2));
    const double g2 = tail2(G.profile, fabs(w));
    v = w >= 0.0 ? g2 : 2.0 - g2;
  }
  double F = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double x1 = __shfl_sync(0xffffffffu, v, 4 * i, 16), x2 = __shfl_sync(0xffffffffu, v, 4 * i + 1, 16);
    const double z1 = __shfl_sync(0xffffffffu, v, 4 * i + 2, 16), z2 = __shfl_sync(0xffffffffu, v, 4 * i + 3, 16);
    if (sub == 0) F += 0.25 * G.c1d[i] * (x1 - x2) * (z1 - z2);
  }
  if (sub != 0 || !(t > 0.0)) return 0.0;
  // Eq. 2: A = T(d) (SAD / t)^2
  const double q = B.sad / t;
  return T * q * q * F;
}

}  // namespace

// The FP64 maximum of every row whose near-maximum candidates overflowed its
// slots (listed by the count pass, rcount[2] of them): one CTA per listed row
// scans the row's candidates, evaluates each value within kRefineDelta of the
// row's FP32 maximum again in FP64 (the count pass's own criterion; two pairs
// per warp at a time, in half-warps) and stores the largest in row_max64.
// Runs before k_refine, which decides the row's listed pairs against it.
__global__ void __launch_bounds__(kRefineThreads) k_refine_rowmax(RefineParams P) {
  constexpr float kTiny = 1.40129846e-45f;
  __shared__ double s_max[kRefineThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, half = lane >> 4, sub = lane & 15;
  const unsigned long long n = min(P.rcount[2], (unsigned long long)P.nrows);
  const long long ni = *P.n_items;
  for (unsigned long long e = blockIdx.x; e < n; e += gridDim.x) {
    const int r = P.ovf_rows[e];
    if ((unsigned)r >= (unsigned)P.nrows) {           // checked (block-uniform): skip and flag
      if (threadIdx.x == 0) atomicOr(P.slot->status, kStatusIndex);
      continue;
    }
    const DRow& R = P.rows[r];
    const DInst& G = P.inst[R.inst];
    const DBeam& B = P.beams[R.beam];
    const float* tab = P.tables + (size_t)r * P.table_stride;
    const long long i0 = P.row_item_base[r], i1 = P.row_item_base[r + 1];
    const long long c0 = i0 < ni ? P.item_off[i0] : P.n_cand;
    const long long c1 = min(i1 < ni ? P.item_off[i1] : P.n_cand, P.n_cand);
    const float mlo = fmaxf(P.tau * __uint_as_float(P.row_max[r]), kTiny) * P.inv_tau_m;
    const long long nvox = (long long)G.nx * G.ny * G.nz;
    double M = 0.0;
    for (long long cb = c0 + 32ll * w; cb < c1; cb += 32ll * (kRefineThreads / 32)) {   // warp-uniform
      const long long c = cb + lane;
      const float v = c < c1 ? P.vals[c] : -1.0f;
      unsigned m = __ballot_sync(0xffffffffu, v >= mlo);
      while (m) {                                     // warp-uniform: two flagged candidates at a time
        const int a = __ffs(m) - 1;
        m &= m - 1u;
        const int b = m ? __ffs(m) - 1 : a;
        if (m) m &= m - 1u;
        int col = P.cols[cb + (half ? b : a)];
        if (col < 0 || (long long)col >= nvox) {      // checked: evaluate voxel 0 instead, and flag
          atomicOr(P.slot->status, kStatusIndex);
          col = 0;
        }
        const double D = eval_pair64_half(R, G, B, tab, col, sub);
        M = fmax(M, fmax(__shfl_sync(0xffffffffu, D, 0), __shfl_sync(0xffffffffu, D, 16)));
      }
    }
    if (lane == 0) s_max[w] = M;
    __syncthreads();
    if (threadIdx.x == 0) {
      double mm = 0.0;
      for (int k = 0; k < kRefineThreads / 32; ++k) mm = fmax(mm, s_max[k]);
      P.row_max64[r] = mm;
    }
    __syncthreads();
  }
}

// keep decisions of the listed pairs in FP64, a warp per pair.  The warp
// evaluates the pair and its row's near-maximum candidates, takes M_j as the
// largest of the latter, and decides D >= tau M_j; the value written back
// makes the compaction's FP32 test agree, and kept pairs join their tile's
// count.  A row whose near-maximum candidates overflowed its slots takes its
// FP64 maximum from k_refine_rowmax.
__global__ void __launch_bounds__(kRefineThreads) k_refine(RefineParams P) {
  constexpr float kTiny = 1.40129846e-45f;
  const int lane = threadIdx.x & 31, half = lane >> 4, sub = lane & 15;
  const unsigned long long n = min(P.rcount[0], (unsigned long long)P.cap_u);
  const unsigned long long warps = (unsigned long long)gridDim.x * (kRefineThreads / 32);
  for (unsigned long long e = blockIdx.x * (unsigned long long)(kRefineThreads / 32) + (threadIdx.x >> 5); e < n;
       e += warps) {
    const unsigned long long entry = P.rlist_u[e];
    const long long p = (long long)(entry & ((1ull << kRefineRowShift) - 1ull));
    const int r = (int)(entry >> kRefineRowShift);
    if (p >= P.n_cand || r >= P.nrows) {              // checked (warp-uniform): skip and flag
      if (lane == 0) atomicOr(P.slot->status, kStatusIndex);
      continue;
    }
    const DRow& R = P.rows[r];
    const DInst& G = P.inst[R.inst];
    const DBeam& B = P.beams[R.beam];
    const float* tab = P.tables + (size_t)r * P.table_stride;
    const int mc = P.mcount[r];
    // the pair, then the row's near-maximum candidates (a row that overflowed
    // its slots has its FP64 maximum from k_refine_rowmax)
    const int total = mc > kMaxSlots ? 1 : 1 + mc;
    double own = 0.0, M = 0.0;
    for (int j0 = 0; j0 < total; j0 += 2) {           // warp-uniform
      const int j = j0 + half;
      long long q = (j == 0 || j >= total) ? p : P.mslot[(size_t)r * kMaxSlots + j - 1];
      int col = 0;
      if (q >= 0 && q < P.n_cand) col = P.cols[q];
      if (q < 0 || q >= P.n_cand || col < 0 || (long long)col >= (long long)G.nx * G.ny * G.nz) {
        atomicOr(P.slot->status, kStatusIndex);     // checked: evaluate the pair itself instead
        col = P.cols[p];
      }
      const double D = eval_pair64_half(R, G, B, tab, col, sub);
      const double d0 = __shfl_sync(0xffffffffu, D, 0), d1 = __shfl_sync(0xffffffffu, D, 16);
      if (j0 == 0) own = d0; else M = fmax(M, d0);
      if (j0 + 1 < total) M = fmax(M, d1);
    }
    if (lane != 0) continue;
    if (mc > kMaxSlots) M = P.row_max64[r];
    const float thr1 = fmaxf(P.tau * __uint_as_float(P.row_max[r]), kTiny);   // the compaction's FP32 threshold
    float v;
    bool keep;
    if (mc >= 1 && M > 0.0) {
      keep = own > 0.0 && own >= P.tau_d * M;
      v = __double2float_rn(own);
      if (keep && v < thr1) v = thr1;
      if (!keep && v >= thr1) v = __uint_as_float(__float_as_uint(thr1) - 1u);   // thr1 > smallest denormal
    } else {                                                            // no FP64 maximum: FP32 decides
      v = P.vals[p];
      keep = v >= thr1;
    }
    P.vals[p] = v;
    if (keep) atomicAdd(P.tile_cnt + p / kTile, 1);
  }
}

}  // namespace dsc

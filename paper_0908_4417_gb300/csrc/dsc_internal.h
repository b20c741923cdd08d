// dsc_internal.h -- device-side data layout of libdsc (host and device code).
//
// Flat layout over all instances of a launch: instances (geometries) own rows
// (beamlets, Eq. 1 index i); rows own work items; items own candidate pairs.
// Every buffer lives in HBM for the life of a plan and is indexed by these
// flat ids, so one kernel launch covers a whole batch of re-plan instances.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dsc {

constexpr int kEvalThreads = 128;     // threads per CTA of the evaluation / compaction kernels
#ifndef DSC_LINES_PER_ITEM
#define DSC_LINES_PER_ITEM 256
#endif
constexpr int kMaxLinesPerItem = DSC_LINES_PER_ITEM;  // x-lines handled by one work item (multiple of kEvalThreads)
constexpr int kWindow = 4096;         // candidates mapped to lines per pass of an item
constexpr int kSiddonThreads = 32;    // lanes per ray (one warp, one CTA) of the depth-table kernels
constexpr int kScanBlocks = 1024;     // blocks of the device-wide scan
constexpr int kScanThreads = 256;
constexpr long long kSmallScan = 4096;   // inputs up to this length use the one-block scan

// float-float value: hi + lo with |lo| <= ulp(hi)/2 (compensated FP32)
struct ff { float hi, lo; };

// The accumulators of one computation, cleared by k_setup (one thread per
// row; thread 0 the counters) instead of separate memsets: null pointers are
// left alone.
struct StepClear {
  unsigned* row_max;               // nrows
  long long* row_cand;             // nrows
  int* mcount;                     // nrows
  int* counter;                    // 4
  unsigned long long* rcount;      // 4
  int* ord_cnt;                    // kOrderClasses
};

// One geometry of a launch.
struct DInst {
  const float* rho;        // density [nz][ny][nx]
  const float4* lut;       // n_lut entries {row k, row k+1 - row k}, rows {T, c3_1, c3_2, c3_3}
  int nx, ny, nz;
  int n_lut;
  double dx, dy, dz;
  double ox, oy, oz;       // outer corner of voxel (0,0,0)
  double idx, idy, idz;    // 1 / voxel sides
  float lut_scale;         // (n_lut - 1) / d_max
  float c3max;             // max of c3_1 over the table (SIGMA superset)
  float d_peak;            // depth of the table's largest T (the first such row), mm
  float c1q[3];            // c1 / 4
  float c2h[3];            // c2 / 2
  int cutoff_mode;
  float cutoff_k;
  int profile;             // lateral profile: 0 erf (Eq. 3), 1 Laplace, 2 logistic
  // the model as given, for the FP64 re-evaluation of decisive pairs
  const float4* lut_rows;  // n_lut rows {T, c3_1, c3_2, c3_3}
  double d_max;
  double c1d[3], c2d[3];
  int row_base, nrows;     // rows of this instance in the flat row list
  int beam_base, nbeams;
  float h;                 // depth-table spacing
  float inv_h;
  double hd;
};

// One beam of a launch (Section 2.1: broad beam from a point source).
struct DBeam {
  int inst;
  int row_base;
  int n_u, n_v;
  double gantry_deg, sad, iso[3], a, b;
};

// One beamlet row: frame, ray and the constants of its voxel loop.
struct DRow {
  // Siddon ray (FP64 crossing parameters)
  double S[3];             // source
  double e[3];             // unit beamlet axis
  double x[3], z[3];       // lateral unit axes (x', z' directions)
  double tA, tB;           // entry A and exit B along the axis
  double inv_e[3];         // 1 / e (0 where e is 0)
  // Siddon walk in fixed point (units of 2^-fix_q mm, set up in FP64)
  long long fx_tA, fx_h, fx_tB;
  int fix_q;
  // voxel loop, compensated FP32: value at voxel (0,0,0) and per-index slopes
  ff S0, X0, Z0;           // s = t - tA, x', z' at voxel (0,0,0)
  ff Ss[3], Xs[3], Zs[3];  // change of s, x', z' per step in ix, iy, iz
  // s again in 64-bit fixed point, units of h 2^-32 (the depth-table cell is
  // the high word, the fraction the low word): value at voxel (0,0,0), steps
  long long sfx0, sfx_s[3];
  float tA_f;
  float kx, kz, bx, bz;    // lateral cutoff |x'| <= kx t + bx, |z'| <= kz t + bz
  float a_sad, b_sad;      // a / SAD, b / SAD (a_t = a_sad * t)
  float sad;
  int inst, beam;
  int hit;                 // the axis crosses the grid prism
  int n_table;             // depth-table entries (0 when !hit)
  int iy0, iy1, iz0, iz1;  // voxel box of the VOI (lines to visit)
  int ix0, ix1;
  int lpc;                 // lines per work item
  int nitems;
  int nlines;              // x-lines enumerated: those of the box that can meet the VOI (k_slices)
};

// The x-lines of a row that can meet its VOI, slice by slice (k_slices):
// for slice s = iz - iz0 of row r, slice_pre[r * stride + s] lines come
// before it and its lines are iy = slice_lo[r * stride + s] + 0, 1, ...;
// slice_pre[r * stride + nzr] is the row's total (nzr = iz1 - iz0 + 1).
struct SliceTab {
  const int* pre;
  const int* lo;
  int stride;
};

struct EvalParams {
  const DInst* inst;
  const DRow* rows;
  SliceTab slices;
  const float* tables;      // [nrows][table_stride]
  int table_stride;
  const long long* row_item_base;  // nrows + 1
  int nrows;
  const long long* item_off;       // n_items + 1: first candidate of each item
  const int* item_row;             // n_items: row of each item
  const long long* n_items;        // device scalar (= row_item_base[nrows])
  float* vals;                     // candidate values (D, or -1 outside the SIGMA cutoff)
  int* cols;                       // candidate voxel indices
  unsigned* row_max;               // float bits, atomicMax
  long long* row_cand;             // candidates inside the cutoff per row (atomic add)
  int* item_counter;               // persistent-kernel work queue head
  // the queue hands out the items largest first (its tail holds the small
  // ones), in this order (k_tile_map); null: index order
  const int* item_ord;
  // the count of each tile taken during the evaluation: an item takes the
  // running row maximum at its start as a lower bound L of the final one;
  // per tile, the values at or above the kept bound L gives, and the lanes
  // with a value in L's refinement band or near L (tile_meta: count in the
  // low 8 bits, those lanes above)
  float tau, inv_tau_m;
  unsigned* tile_meta;             // n_tiles
  unsigned* item_L;                // n_items: float bits of L
};

// Output pointers of the computation in flight.  Kernels read them from this
// device-side slot so that a captured launch sequence can be replayed into
// freshly allocated result buffers.
struct OutSlot {
  long long* row_ptr;      // per instance (nrows + 1), relative to the instance's first entry
  int* col;
  void* val;               // float or bf16
  float* beam_scale;       // per beam
  unsigned* row_max;       // per row, float bits
  long long* row_cand;     // per row
  long long* inst_begin;   // per instance: first output slot; [ninst] = total
  int* status;             // nonzero: kStatusWait (a bounded device wait expired) or kStatusIndex
  long long* summary;      // null, or [0]: the status word (status points at it), then per instance k
                           // [1 + 2k] its first output entry and [2 + 2k] its kept count (k_finish), so
                           // that the host reads all it needs to size a read-back in one copy
  unsigned long long* refine;  // [4] pairs listed for the FP64 re-evaluation: near a threshold, near a row
                               // maximum; near-threshold pairs past the list's capacity (decided in FP32);
                               // compaction tiles whose values the count pass read
};

// size classes of the work items for the evaluation's queue order, the
// largest first: class 0 holds items of at least 15/8 of the target size,
// class 15 those below 1/8 of it
constexpr int kOrderClasses = 16;
constexpr int kOrderRankBits = 27;    // an item's class and rank in one int (fewer than 2^27 items)
__host__ __device__ __forceinline__ int order_class(long long n, int target_cand) {
  const long long unit = target_cand >= 8 ? target_cand / 8 : 1;
  const long long q = n / unit;
  return kOrderClasses - 1 - (int)(q < kOrderClasses - 1 ? q : kOrderClasses - 1);
}

constexpr int kTilePer = 4;                       // candidates per thread of the compaction
// candidates per compaction tile; every work item is padded to a whole
// number of tiles, so a tile lies in one item, and one warp-iteration of the
// evaluation (32 lanes x 4 candidates) writes one tile
constexpr int kTile = 32 * kTilePer;
#ifndef DSC_TPW
#define DSC_TPW 2
#endif
// tiles per warp in the count and write passes: a warp loads all its tiles'
// candidates before deciding any, so more loads are in flight
constexpr int kTilesPerWarp = DSC_TPW;
// tiles per warp in the count pass: a tile per lane
constexpr int kCountTilesPerWarp = 32;
// CTAs (of kEvalThreads) over n_tiles tiles, tpw tiles per warp
inline unsigned tile_blocks(long long n_tiles, int tpw) {
  const long long warps = (n_tiles + tpw - 1) / tpw;
  const long long b = (warps + kEvalThreads / 32 - 1) / (kEvalThreads / 32);
  return (unsigned)(b > 0 ? b : 1);
}
// CTAs of the write pass
inline unsigned compact_blocks(long long n_tiles) { return tile_blocks(n_tiles, kTilesPerWarp); }

struct CompactParams {
  const DRow* rows;
  const long long* item_off;      // n_items + 1
  const int* item_row;
  const long long* n_items;
  long long n_cand;
  const float* vals;
  const int* cols;
  const unsigned* row_max;
  float tau;
  const int* tile_row;            // per tile: the row of the item holding the tile
  const int* tile_item;           // per tile: the item holding the tile
  const unsigned* tile_meta;      // per tile: the evaluation's count and flags (EvalParams)
  const unsigned* item_L;         // per item: the lower bound of the row maximum it was counted against
  float* tile_thr;                // per tile: threshold of that row (written by the count pass)
  float* tile_scale;              // per tile: BF16 scale of that row's beam (written by the count pass)
  int value_dtype;
  const OutSlot* slot;
  // decisions FP32 cannot settle: candidates within kRefineDelta (relative)
  // of their threshold go to rlist_u and are left out of the tile counts;
  // candidates within kRefineDelta of their row maximum go to their row's
  // slots (kMaxSlots per row)
  unsigned long long* rlist_u;   // refine_entry(candidate, row)
  unsigned long long* rcount;     // [0] entries listed in rlist_u, [1] near-maximum candidates (may exceed capacities),
                                  // [2] rows with more than kMaxSlots near-maximum candidates (listed in ovf_rows),
                                  // [3] tiles counted from their values
  int* mcount;                    // per row: near-maximum candidates seen
  long long* mslot;               // per row: kMaxSlots candidate indices
  int* ovf_rows;                  // rows whose near-maximum candidates overflowed their slots (nrows entries)
  int cap_u;
  int nrows;
  float inv_tau_m;                // (1 - kRefineDelta) / tau (infinite for tau = 0)
};

// a refine-list entry: candidate index in the low 40 bits, row above (a
// launch has fewer than 2^24 rows and 2^40 candidates)
constexpr int kRefineRowShift = 40;
__host__ __device__ __forceinline__ unsigned long long refine_entry(long long p, int row) {
  return ((unsigned long long)row << kRefineRowShift) | (unsigned long long)p;
}

// result status bits: a bounded device wait expired; an index a kernel
// checks was out of range (the access was skipped)
constexpr int kStatusWait = 1;
constexpr int kStatusIndex = 2;

// near-maximum candidates kept per row for its FP64 maximum; a row with more
// is listed, and k_refine_rowmax takes its FP64 maximum from a scan of the row
constexpr int kMaxSlots = 4;

// relative window around a threshold (and below a row maximum) inside which
// the FP32 value does not settle a decision: the evaluation's FP32 error is
// below 3e-6 relative
constexpr float kRefineDelta = 1e-5f;

// the FP64 re-evaluation: one warp per listed pair, kRefineThreads per CTA,
// enough CTAs for a warp per entry up to 4096 entries (grid-stride beyond);
// the warp evaluates its pair and its row's near-maximum candidates, two
// pairs at a time in half-warps
constexpr int kRefineThreads = 128;
// CTAs of k_refine_rowmax (grid-stride over the rows that overflowed their slots)
constexpr int kRefineRowmaxBlocks = 152;
inline unsigned refine_blocks(int cap) {
  const int warps = cap < 4096 ? cap : 4096;
  return (unsigned)((warps + kRefineThreads / 32 - 1) / (kRefineThreads / 32));
}

// the FP64 re-evaluation of the pairs in the refine lists
struct RefineParams {
  const DInst* inst;
  const DRow* rows;
  const DBeam* beams;
  const float* tables;
  int table_stride;
  const long long* item_off;
  const int* item_row;
  const long long* n_items;
  float* vals;                    // refined values are written back
  const int* cols;
  const unsigned* row_max;        // FP32 row maxima (float bits), as the compaction reads them
  float tau;                      // the compaction's FP32 threshold factor
  double tau_d;                   // the threshold factor as given
  const unsigned long long* rlist_u;
  const unsigned long long* rcount;
  int cap_u;
  const int* mcount;              // per row: near-maximum candidates seen
  const long long* mslot;         // per row: kMaxSlots candidate indices
  const int* ovf_rows;            // rows with more than kMaxSlots near-maximum candidates (rcount[2] of them)
  double* row_max64;              // per row: FP64 maximum of an overflowing row (k_refine_rowmax)
  const long long* row_item_base; // nrows + 1: first work item of each row
  float inv_tau_m;                // (1 - kRefineDelta) / tau: a value >= thr * this is near its row maximum
  int* tile_cnt;                  // kept refined pairs are added to their tile's count
  int nrows;
  long long n_cand;
  const OutSlot* slot;            // status of the computation (kStatusIndex)
};

// process-wide work decomposition (dsc_set_tuning): candidates per work item
// and evaluation CTAs per SM (0 = occupancy limit)
void current_tuning(int* target_cand, int* eval_blocks_per_sm);
// sets the text dsc_last_error() returns on the calling thread
void set_error(const char* msg);
// adds n kernel launches to the process-wide count dsc_launch_count() returns
void count_launches(long long n);

}  // namespace dsc

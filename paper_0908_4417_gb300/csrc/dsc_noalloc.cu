// dsc_noalloc.cu -- dsc_compute_dij_noalloc: D_ij into caller buffers with no
// memory allocation by the library.
//
// For callers that must not allocate device memory while they run: treatment
// and re-planning loops that pre-reserve every byte up front, processes that
// share a GPU under a fixed memory quota, or code that runs where cudaMalloc
// is not permitted.  The working memory of the computation (beam model copy,
// per-beamlet set-up, depth tables, work items, candidate values, scan
// partials) lives in one fixed array that is part of this library's device
// image: it is reserved on every GPU that loads the library and stays there
// until the process exits.  The caller passes the density and the CSR output
// buffers.
//
// The launch sequence is the one of dsc_compute_dij (the same kernels), run
// eagerly on the caller's stream.
#include "dsc_internal.h"
#include "../../include/dsc.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <limits>
#include <mutex>

namespace dsc {
__global__ void k_setup(const DInst*, const DBeam*, int, DRow*, int, int*, int, StepClear);
__global__ void k_siddon(const DInst*, const DRow*, int, float*, int);
__global__ void k_trilinear_table(const DInst*, const DRow*, int, float*, int);
__global__ void k_count(const DInst*, const DRow*, SliceTab, const long long*, int, const long long*, int*, const int*,
                        int*, int*, int);
__global__ void k_slices(const DInst*, DRow*, int, int*, int*, int, int*);
__global__ void k_item_rows(const long long*, int, int*);
__global__ void k_tile_map(const long long*, const long long*, const int*, int*, int*, const int*, const int*, int*);
__global__ void k_row_bound(const DInst*, const DRow*, int, const float*, int, SliceTab, unsigned*);
__global__ void k_eval(EvalParams);
__global__ void k_tile_count(CompactParams, int*);
__global__ void k_lut_pairs(const float4*, int, int, float4*);
__global__ void k_refine(RefineParams);
__global__ void k_refine_rowmax(RefineParams);
__global__ void k_tile_write(CompactParams, const long long*);
__global__ void k_row_ptr(const long long*, const long long*, const long long*, const long long*, long long, int, int,
                          long long, int, int, const OutSlot*);
__global__ void k_scan_partial(const int*, const long long*, long long, long long*);
__global__ void k_scan_blocks(long long*);
__global__ void k_scan_final(const int*, const long long*, long long, const long long*, long long*);
__global__ void k_scan_small(const int*, const long long*, long long, long long*);
}  // namespace dsc

using namespace dsc;


// The fixed working memory: 80 MiB per device.  Every call uses it from the
// start, so calls whose device work overlaps (different streams, or
// different host threads) race on it; serialise them on one stream.
static constexpr size_t kNoAllocBytes = 80ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_na_mu;
static void* g_na_base[64];   // device address of the array, per device

static dsc_status na_fail(dsc_status s, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  dsc::set_error(buf);
  return s;
}

#define NA_CU(call)                                                                                     \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return na_fail(DSC_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
  } while (0)
#define NA_LAUNCH()                                                                                     \
  do {                                                                                                  \
    dsc::count_launches(1);                                                                             \
    cudaError_t e_ = cudaGetLastError();                                                                \
    if (e_ != cudaSuccess) return na_fail(DSC_E_CUDA, "launch: %s", cudaGetErrorString(e_));          \
  } while (0)

// Host code cannot use g_noalloc_scratch's name as a device address: it
// names a host-side shadow.  The device address comes from
// cudaGetSymbolAddress, once per device, with that device current, and is
// kept for the life of the process (the library is not used across a reset
// of a device's primary context).
static dsc_status na_base(unsigned char** base) {
  int dev = 0;
  NA_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return na_fail(DSC_E_CUDA, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(DSC_E_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch): %s", cudaGetErrorString(e));
    g_na_base[dev] = p;
  }
  *base = (unsigned char*)g_na_base[dev];
  return DSC_OK;
}

// bump carving of the fixed array, 256-byte aligned pieces
struct Carve {
  unsigned char* base;
  size_t used = 0;
  size_t need = 0;   // bytes the request would need (also past the end)
  template <typename T>
  T* take(size_t n) {
    size_t off = (need + 255) & ~size_t(255);
    need = off + (n > 0 ? n : 1) * sizeof(T);
    if (need > kNoAllocBytes) return nullptr;
    used = need;
    return (T*)(base + off);
  }
};

static dsc_status na_scan(const int* in, const long long* n_dev, long long n_const, long long* tmp, long long* out,
                          cudaStream_t s, long long n_host) {
  if (n_host <= kSmallScan) {
    k_scan_small<<<1, 1024, 0, s>>>(in, n_dev, n_const, out);
    NA_LAUNCH();
    return DSC_OK;
  }
  k_scan_partial<<<kScanBlocks, kScanThreads, 0, s>>>(in, n_dev, n_const, tmp);
  NA_LAUNCH();
  k_scan_blocks<<<1, kScanBlocks, 0, s>>>(tmp);
  NA_LAUNCH();
  k_scan_final<<<kScanBlocks, kScanThreads, 0, s>>>(in, n_dev, n_const, tmp, out);
  NA_LAUNCH();
  return DSC_OK;
}

extern "C" dsc_status dsc_compute_dij_noalloc(const dsc_grid_desc* grid, const float* density_dev,
                                              const dsc_fspb_model* model, const dsc_beam_desc* beams, int32_t nbeams,
                                              const dsc_compute_opts* opts, int64_t* row_ptr_dev, int32_t* col_dev,
                                              float* val_dev, int64_t capacity, int64_t* nnz_out, void* stream) {
  if (!grid || !density_dev || !model || !beams || nbeams < 1 || !opts || !row_ptr_dev || !col_dev || !val_dev ||
      !nnz_out)
    return na_fail(DSC_E_INVAL, "null argument");
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0 && grid->dy > 0 && grid->dz > 0) ||
      (long long)grid->nx * grid->ny * grid->nz >= (1ll << 31))
    return na_fail(DSC_E_INVAL, "grid: need dimensions >= 1, sides > 0, fewer than 2^31 voxels");
  if (model->n < 2 || model->n > 4096 || !model->table4 || !(model->d_max > 0) || model->cutoff_mode < 0 ||
      model->cutoff_mode > 2 || model->profile < 0 || model->profile > 2)
    return na_fail(DSC_E_INVAL, "model: need 2 <= n <= 4096, d_max > 0, cutoff_mode 0..2, profile 0..2");
  if (opts->value_dtype != DSC_VALUE_F32 || !(opts->rel_threshold >= 0) || !(opts->h_frac > 0 && opts->h_frac <= 1))
    return na_fail(DSC_E_INVAL, "opts: FP32 values only, rel_threshold >= 0, 0 < h_frac <= 1");
  if (capacity < 0) return na_fail(DSC_E_INVAL, "capacity < 0");
  *nnz_out = 0;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  NA_CU(cudaGetDevice(&dev));

  // host-side descriptors (no allocation: fixed-size locals and the beams array)
  DInst I{};
  I.rho = density_dev;
  I.nx = grid->nx; I.ny = grid->ny; I.nz = grid->nz;
  I.n_lut = model->n;
  I.dx = grid->dx; I.dy = grid->dy; I.dz = grid->dz;
  I.ox = grid->origin[0]; I.oy = grid->origin[1]; I.oz = grid->origin[2];
  I.idx = 1.0 / I.dx; I.idy = 1.0 / I.dy; I.idz = 1.0 / I.dz;
  I.lut_scale = (float)((model->n - 1) / model->d_max);
  float c3max = 0.f;
  int kpeak = 0;
  for (int k = 0; k < model->n; ++k) {
    for (int c = 1; c <= 3; ++c) {
      const float w = model->table4[4 * k + c];
      if (!(w > 0.f) || !std::isfinite(w)) return na_fail(DSC_E_INVAL, "model: c3 widths must be finite and > 0");
    }
    if (!std::isfinite(model->table4[4 * k])) return na_fail(DSC_E_INVAL, "model: T(d) must be finite");
    float v = model->table4[4 * k + 1];
    c3max = v > c3max ? v : c3max;
    if (model->table4[4 * k] > model->table4[4 * kpeak]) kpeak = k;
  }
  I.c3max = c3max;
  I.d_peak = (float)(kpeak * (model->d_max / (model->n - 1)));
  for (int i = 0; i < 3; ++i) { I.c1q[i] = (float)(model->c1[i] / 4.0); I.c2h[i] = (float)(model->c2[i] / 2.0); }
  I.cutoff_mode = model->cutoff_mode;
  I.cutoff_k = (float)model->cutoff_k;
  I.profile = model->profile;
  double dmin = grid->dx < grid->dy ? grid->dx : grid->dy;
  dmin = grid->dz < dmin ? grid->dz : dmin;
  I.hd = opts->h_frac * dmin;
  I.h = (float)I.hd;
  I.inv_h = (float)(1.0 / I.hd);
  I.row_base = 0;
  I.beam_base = 0;
  I.nbeams = nbeams;
  long long nrows_ll = 0;
  for (int b = 0; b < nbeams; ++b) {
    const dsc_beam_desc& B = beams[b];
    if (!(B.sad > 0) || !(B.a > 0) || !(B.b > 0) || B.n_u < 1 || B.n_v < 1)
      return na_fail(DSC_E_INVAL, "beam %d: need sad, a, b > 0 and n_u, n_v >= 1", b);
    double gr = B.gantry_deg * M_PI / 180.0;
    double S[3] = {B.iso[0] + B.sad * sin(gr), B.iso[1] - B.sad * cos(gr), B.iso[2]};
    bool inside = S[0] >= I.ox && S[0] <= I.ox + I.nx * I.dx && S[1] >= I.oy && S[1] <= I.oy + I.ny * I.dy &&
                  S[2] >= I.oz && S[2] <= I.oz + I.nz * I.dz;
    if (inside) return na_fail(DSC_E_INVAL, "beam %d: the source lies inside the grid", b);
    nrows_ll += (long long)B.n_u * B.n_v;
  }
  if (nrows_ll > (1 << 24)) return na_fail(DSC_E_INVAL, "too many beamlets");
  const int nrows = (int)nrows_ll;
  I.nrows = nrows;
  double diag = std::sqrt(std::pow(I.nx * I.dx, 2) + std::pow(I.ny * I.dy, 2) + std::pow(I.nz * I.dz, 2));
  int stride = (((int)std::ceil(diag / I.hd) + 2) + 3) & ~3;

  unsigned char* base = nullptr;
  dsc_status st = na_base(&base);
  if (st != DSC_OK) return st;
  std::lock_guard<std::mutex> lk(g_na_mu);   // one host thread at a time carves and launches
  // Declared after the lock, so it runs before the unlock: once work has been
  // queued, every return (an error included) first waits for that work, and
  // the next call cannot reuse the array while this one's kernels still run.
  struct SyncOnReturn {
    cudaStream_t s;
    bool armed;
    ~SyncOnReturn() {
      if (armed) cudaStreamSynchronize(s);
    }
  } drain{s, false};

  Carve cv{base};
  float4* d_lut_rows = cv.take<float4>(model->n);
  float4* d_lut = cv.take<float4>(2 * (size_t)model->n);
  DInst* d_inst = cv.take<DInst>(1);
  DBeam* d_beams = cv.take<DBeam>(nbeams);
  DRow* d_rows = cv.take<DRow>(nrows);
  int* d_row_items = cv.take<int>(nrows);
  const int slice_stride = std::max(2, grid->nz + 1);
  int* d_slice_pre = cv.take<int>((size_t)nrows * slice_stride);
  int* d_slice_lo = cv.take<int>((size_t)nrows * slice_stride);
  const SliceTab slices{d_slice_pre, d_slice_lo, slice_stride};
  long long* d_rib = cv.take<long long>(nrows + 1);
  float* d_tables = cv.take<float>((size_t)nrows * stride);
  long long* d_scan = cv.take<long long>(kScanBlocks + 1);
  int* d_counter = cv.take<int>(4);
  OutSlot* d_slot = cv.take<OutSlot>(1);
  unsigned* d_row_max = cv.take<unsigned>(nrows);
  long long* d_row_cand = cv.take<long long>(nrows);
  float* d_scale = cv.take<float>(1);
  int* d_status = cv.take<int>(1);
  long long* d_inst_begin = cv.take<long long>(2);
  unsigned long long* d_rcount = cv.take<unsigned long long>(4);
  int* d_mcount = cv.take<int>(nrows);
  long long* d_mslot = cv.take<long long>((size_t)nrows * kMaxSlots);
  int* d_ovf_rows = cv.take<int>(nrows);
  double* d_row_max64 = cv.take<double>(nrows);
  if (!d_row_max64)
    return na_fail(DSC_E_INVAL, "needs more than %zu bytes of working memory (the fixed maximum) for %d beamlets",
                   kNoAllocBytes, nrows);

  drain.armed = true;
  NA_CU(cudaMemcpyAsync(d_lut_rows, model->table4, sizeof(float4) * model->n, cudaMemcpyHostToDevice, s));
  k_lut_pairs<<<(model->n + 127) / 128, 128, 0, s>>>(d_lut_rows, model->n, model->profile, d_lut);
  NA_LAUNCH();
  I.lut = d_lut;
  I.lut_rows = d_lut_rows;
  I.d_max = model->d_max;
  for (int i = 0; i < 3; ++i) { I.c1d[i] = model->c1[i]; I.c2d[i] = model->c2[i]; }
  NA_CU(cudaMemcpyAsync(d_inst, &I, sizeof(DInst), cudaMemcpyHostToDevice, s));
  NA_CU(cudaMemsetAsync(d_rcount, 0, sizeof(unsigned long long) * 4, s));
  NA_CU(cudaMemsetAsync(d_mcount, 0, sizeof(int) * nrows, s));
  for (int b = 0, row = 0; b < nbeams; ++b) {
    DBeam D{};
    D.inst = 0;
    D.row_base = row;
    D.n_u = beams[b].n_u; D.n_v = beams[b].n_v;
    D.gantry_deg = beams[b].gantry_deg; D.sad = beams[b].sad;
    for (int i = 0; i < 3; ++i) D.iso[i] = beams[b].iso[i];
    D.a = beams[b].a; D.b = beams[b].b;
    NA_CU(cudaMemcpyAsync(d_beams + b, &D, sizeof(DBeam), cudaMemcpyHostToDevice, s));
    row += beams[b].n_u * beams[b].n_v;
  }
  // the array keeps the previous call's contents: clear what accumulates
  NA_CU(cudaMemsetAsync(d_row_max, 0, sizeof(unsigned) * nrows, s));
  NA_CU(cudaMemsetAsync(d_row_cand, 0, sizeof(long long) * nrows, s));
  NA_CU(cudaMemsetAsync(d_counter, 0, sizeof(int) * 4, s));
  NA_CU(cudaMemsetAsync(d_status, 0, sizeof(int), s));

  int sms = 0, nb = 0;
  NA_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  NA_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval, kEvalThreads, 0));
  int target_cand = 8192, eval_bps = 0;
  current_tuning(&target_cand, &eval_bps);
  nb = nb > 0 ? nb : 1;
  const int grid_eval = (eval_bps > 0 && eval_bps < nb ? eval_bps : nb) * sms;
  NA_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_count, kEvalThreads, 0));
  const int grid_items = (nb > 0 ? nb : 1) * sms;

  // set-up and work items
  k_setup<<<(nrows + 31) / 32, 32, 0, s>>>(d_inst, d_beams, nbeams, d_rows, nrows, d_row_items, target_cand,
                                           StepClear{});
  NA_LAUNCH();
  k_slices<<<(nrows + 3) / 4, 128, 0, s>>>(d_inst, d_rows, nrows, d_slice_pre, d_slice_lo, slice_stride, d_row_items);
  NA_LAUNCH();
  st = na_scan(d_row_items, nullptr, nrows, d_scan, d_rib, s, nrows);
  if (st != DSC_OK) return st;
  long long n_items = 0;
  NA_CU(cudaMemcpyAsync(&n_items, d_rib + nrows, sizeof(long long), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  int* d_item_cand = cv.take<int>(n_items);
  int* d_item_row = cv.take<int>(n_items);
  long long* d_item_off = cv.take<long long>(n_items + 1);
  unsigned* d_item_L = cv.take<unsigned>(n_items);
  if (!d_item_L)
    return na_fail(DSC_E_INVAL, "needs more than %zu bytes of working memory (the fixed maximum): %lld work items",
                   kNoAllocBytes, n_items);
  const long long* n_items_dev = d_rib + nrows;
  if (opts->flags & DSC_FLAG_TRILINEAR_TABLE)
    k_trilinear_table<<<nrows, kSiddonThreads, 0, s>>>(d_inst, d_rows, nrows, d_tables, stride);
  else
    k_siddon<<<nrows, kSiddonThreads, 0, s>>>(d_inst, d_rows, nrows, d_tables, stride);
  NA_LAUNCH();
  k_row_bound<<<(nrows + 3) / 4, 128, 0, s>>>(d_inst, d_rows, nrows, d_tables, stride, slices, d_row_max);
  NA_LAUNCH();
  k_item_rows<<<(nrows + 127) / 128, 128, 0, s>>>(d_rib, nrows, d_item_row);
  NA_LAUNCH();
  k_count<<<grid_items, kEvalThreads, 0, s>>>(d_inst, d_rows, slices, d_rib, nrows, n_items_dev, d_item_cand,
                                              d_item_row, nullptr, nullptr, target_cand);
  NA_LAUNCH();
  st = na_scan(d_item_cand, n_items_dev, 0, d_scan, d_item_off, s, n_items);
  if (st != DSC_OK) return st;
  long long n_cand = 0;
  NA_CU(cudaMemcpyAsync(&n_cand, d_item_off + n_items, sizeof(long long), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  const long long n_tiles = n_cand / kTile;           // items are whole tiles
  float* d_vals = cv.take<float>(n_cand + 4);
  int* d_cols = cv.take<int>(n_cand + 4);
  int* d_tile_cnt = cv.take<int>(n_tiles);
  long long* d_tile_off = cv.take<long long>(n_tiles + 1);
  float* d_tile_thr = cv.take<float>(n_tiles);
  float* d_tile_scale = cv.take<float>(n_tiles);
  int* d_tile_row = cv.take<int>(n_tiles);
  int* d_tile_item = cv.take<int>(n_tiles);
  unsigned* d_tile_meta = cv.take<unsigned>(n_tiles);
  const int cap_u = (int)std::min<long long>(std::max<long long>(1 << 16, n_cand >> 10), 1 << 28);
  unsigned long long* d_rlist_u = cv.take<unsigned long long>(cap_u);
  if (!d_rlist_u)
    return na_fail(DSC_E_INVAL, "needs %zu bytes of working memory for %lld candidate pairs; the fixed maximum is %zu",
                   cv.need, n_cand, kNoAllocBytes);

  // evaluation and compaction
  EvalParams ep{};
  ep.inst = d_inst;
  ep.rows = d_rows;
  ep.slices = slices;
  ep.tables = d_tables;
  ep.table_stride = stride;
  ep.row_item_base = d_rib;
  ep.nrows = nrows;
  ep.item_off = d_item_off;
  ep.item_row = d_item_row;
  ep.n_items = n_items_dev;
  ep.vals = d_vals;
  ep.cols = d_cols;
  ep.row_max = d_row_max;
  ep.row_cand = d_row_cand;
  ep.item_counter = d_counter;
  ep.tau = (float)opts->rel_threshold;
  ep.inv_tau_m = ep.tau > 0.0f ? (1.0f - kRefineDelta) / ep.tau : std::numeric_limits<float>::infinity();
  ep.tile_meta = d_tile_meta;
  ep.item_L = d_item_L;
  k_eval<<<grid_eval, kEvalThreads, 0, s>>>(ep);
  NA_LAUNCH();
  OutSlot q{};
  q.row_ptr = (long long*)row_ptr_dev;
  q.col = col_dev;
  q.val = val_dev;
  q.beam_scale = d_scale;
  q.row_max = d_row_max;
  q.row_cand = d_row_cand;
  q.inst_begin = d_inst_begin;
  q.status = d_status;
  NA_CU(cudaMemcpyAsync(d_slot, &q, sizeof(OutSlot), cudaMemcpyHostToDevice, s));
  CompactParams cp{};
  cp.rows = d_rows;
  cp.item_off = d_item_off;
  cp.item_row = d_item_row;
  cp.n_items = n_items_dev;
  cp.n_cand = n_cand;
  cp.vals = d_vals;
  cp.cols = d_cols;
  cp.row_max = d_row_max;
  cp.tau = (float)opts->rel_threshold;
  cp.tile_thr = d_tile_thr;
  cp.tile_scale = d_tile_scale;
  cp.tile_row = d_tile_row;
  cp.tile_item = d_tile_item;
  cp.tile_meta = d_tile_meta;
  cp.item_L = d_item_L;
  cp.value_dtype = DSC_VALUE_F32;
  cp.slot = d_slot;
  cp.rlist_u = d_rlist_u;
  cp.rcount = d_rcount;
  cp.mcount = d_mcount;
  cp.mslot = d_mslot;
  cp.ovf_rows = d_ovf_rows;
  cp.cap_u = cap_u;
  cp.nrows = nrows;
  cp.inv_tau_m = cp.tau > 0.0f ? (1.0f - kRefineDelta) / cp.tau : std::numeric_limits<float>::infinity();
  k_tile_map<<<1024, 256, 0, s>>>(d_item_off, n_items_dev, d_item_row, d_tile_item, d_tile_row, nullptr, nullptr,
                                 nullptr);
  NA_LAUNCH();
  // kept count first, so the capacity is checked before any output is touched
  const unsigned tiles = compact_blocks(n_tiles);
  k_tile_count<<<tile_blocks(n_tiles, kCountTilesPerWarp), kEvalThreads, 0, s>>>(cp, d_tile_cnt);
  NA_LAUNCH();
  RefineParams rp{};
  rp.inst = d_inst;
  rp.rows = d_rows;
  rp.beams = d_beams;
  rp.tables = d_tables;
  rp.table_stride = stride;
  rp.item_off = d_item_off;
  rp.item_row = d_item_row;
  rp.n_items = n_items_dev;
  rp.vals = d_vals;
  rp.cols = d_cols;
  rp.row_max = d_row_max;
  rp.tau = cp.tau;
  rp.tau_d = opts->rel_threshold;
  rp.rlist_u = d_rlist_u;
  rp.rcount = d_rcount;
  rp.cap_u = cap_u;
  rp.mcount = d_mcount;
  rp.mslot = d_mslot;
  rp.ovf_rows = d_ovf_rows;
  rp.row_max64 = d_row_max64;
  rp.row_item_base = d_rib;
  rp.inv_tau_m = cp.inv_tau_m;
  rp.tile_cnt = d_tile_cnt;
  rp.nrows = nrows;
  rp.n_cand = n_cand;
  rp.slot = d_slot;
  k_refine_rowmax<<<kRefineRowmaxBlocks, kRefineThreads, 0, s>>>(rp);
  NA_LAUNCH();
  k_refine<<<refine_blocks(cap_u), kRefineThreads, 0, s>>>(rp);
  NA_LAUNCH();
  st = na_scan(d_tile_cnt, nullptr, n_tiles, d_scan, d_tile_off, s, n_tiles);
  if (st != DSC_OK) return st;
  long long nnz = 0;
  int status = 0;
  unsigned long long listed = 0;
  NA_CU(cudaMemcpyAsync(&nnz, d_tile_off + n_tiles, sizeof(long long), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaMemcpyAsync(&listed, d_rcount, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  if (nnz > capacity)
    return na_fail(DSC_E_INVAL, "output capacity %lld < %lld kept entries", (long long)capacity, nnz);
  k_tile_write<<<tiles, kEvalThreads, 0, s>>>(cp, d_tile_off);
  NA_LAUNCH();
  k_row_ptr<<<(nrows + 1 + 255) / 256, 256, 0, s>>>(d_rib, d_item_off, d_tile_off, n_items_dev, n_cand, 0, nrows, 0,
                                                    0, 1, d_slot);
  NA_LAUNCH();
  NA_CU(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));   // the array is free for the next call once this returns
  if (status & kStatusIndex) return na_fail(DSC_E_CUDA, "a kernel found an index out of range (status %d)", status);
  if (status) return na_fail(DSC_E_TIMEOUT, "a bounded device wait expired (status %d)", status);
  *nnz_out = nnz;
  if (listed > (unsigned long long)cap_u)   // complete, but these decisions stayed FP32
    return na_fail(DSC_W_INEXACT, "%llu pairs within 1e-5 of their threshold past the FP64 list's %d entries "
                   "were decided in FP32", listed - (unsigned long long)cap_u, cap_u);
  return DSC_OK;
}

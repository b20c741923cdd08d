// dsc_api.cu -- host side of the libdsc C ABI (include/dsc.h).
//
// A "plan" is the device-resident working set of one launch: the flat list
// of instances (geometries) with their beams, the per-row set-up, depth
// tables, per-item candidate counts and the candidate-value scratch.  Plans
// are sized once (two stream-ordered reads of device counts) and cached by
// the identity of their geometries, beam lists and options; every later
// computation with the same key replays the whole launch sequence -- set-up,
// Siddon, enumeration, evaluation, compaction with its FP64 refinement -- as
// one CUDA graph with no host round trip.  Results own their CSR buffers (stream-ordered pool
// allocations) and stay valid after later computations.
#include "dsc_internal.h"
#include "../../include/dsc.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <limits>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace dsc {
// kernels (dsc_kernels.cu)
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
__global__ void k_beam_scale(const DBeam*, int, const unsigned*, const OutSlot*);
__global__ void k_tile_count(CompactParams, int*);
__global__ void k_lut_pairs(const float4*, int, int, float4*);
__global__ void k_out_init(OutSlot*, OutSlot, int, int, int);
__global__ void k_dose_scale(const unsigned*, const float*, int, int*);
__global__ void k_dose_scatter(const long long*, const long long*, const int*, const void*, int, const DRow*, int,
                               const float*, const float*, int, const int*, unsigned long long*);
__global__ void k_dose_finish(const unsigned long long*, long long, const int*, float*);
__global__ void k_beamlet_dot(const long long*, const long long*, const int*, const void*, int, const DRow*, int,
                              const float*, const float*, int, float*);
__global__ void k_tile_write(CompactParams, const long long*);
__global__ void k_finish(const long long*, const long long*, const long long*, const long long*, long long,
                         const long long*, int, const unsigned*, const long long*, int, const unsigned long long*, int,
                         const OutSlot*);
__global__ void k_scan_partial(const int*, const long long*, long long, long long*);
__global__ void k_scan_blocks(long long*);
__global__ void k_scan_final(const int*, const long long*, long long, const long long*, long long*);
__global__ void k_scan_small(const int*, const long long*, long long, long long*);
__global__ void k_tail_probe(int, const float*, long long, float*, float*);
__global__ void k_refine(RefineParams);
__global__ void k_refine_rowmax(RefineParams);
}  // namespace dsc

using namespace dsc;

// ---------------------------------------------------------------------------
// errors, launch accounting
// ---------------------------------------------------------------------------
static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

static dsc_status fail(dsc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CU(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail(e_ == cudaErrorMemoryAllocation ? DSC_E_NOMEM : DSC_E_CUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                   \
  } while (0)

#define CHECK_LAUNCH()                                                                           \
  do {                                                                                           \
    g_launches.fetch_add(1, std::memory_order_relaxed);                                          \
    cudaError_t e_ = cudaGetLastError();                                                         \
    if (e_ != cudaSuccess) return fail(DSC_E_CUDA, "launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define TRY(x)                       \
  do {                               \
    dsc_status s_ = (x);             \
    if (s_ != DSC_OK) return s_;     \
  } while (0)

// A library-owned stream per device for releasing memory: frees wait on the
// completion event of the work that used the memory, so they never depend on
// the caller's stream still existing.
static cudaStream_t free_stream(int dev) {
  static std::mutex mu;
  static std::map<int, cudaStream_t> m;
  std::lock_guard<std::mutex> lk(mu);
  auto it = m.find(dev);
  if (it != m.end()) return it->second;
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  m[dev] = s;
  return s;
}

static void release_after(cudaEvent_t ev, int dev, void* const* ps, int n, const std::vector<cudaEvent_t>* also = nullptr) {
  cudaStream_t fs = free_stream(dev);
  if (ev) cudaStreamWaitEvent(fs, ev, 0);
  if (also)
    for (cudaEvent_t e : *also) cudaStreamWaitEvent(fs, e, 0);
  for (int i = 0; i < n; ++i)
    if (ps[i]) cudaFreeAsync(ps[i], fs);
}

// work decomposition of new plans (dsc_set_tuning / dsc_autotune)
static std::mutex g_tuning_mu;
static dsc_tuning g_tuning = {8192, 0};

namespace dsc {
void current_tuning(int* target_cand, int* eval_blocks_per_sm) {
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  *target_cand = g_tuning.target_cand;
  *eval_blocks_per_sm = g_tuning.eval_blocks_per_sm;
}
}  // namespace dsc

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
static std::atomic<unsigned long long> g_geom_ids{1};

struct dsc_geometry {
  unsigned long long id;
  int device;
  dsc_grid_desc grid;
  int n_lut;
  double d_max;
  double c1[3], c2[3];
  int cutoff_mode;
  double cutoff_k;
  int profile = 0;                   // DSC_PROFILE_*
  float c3max;
  float d_peak;                      // depth of the model's largest T (the first such row), mm
  float* d_rho = nullptr;
  float4* d_lut = nullptr;            // evaluation table: (row, difference) pairs, c3 / K
  float4* d_lut_rows = nullptr;       // the model's rows as given (FP64 re-evaluation)
  std::vector<dsc_beam_desc> beams;
};

struct Plan;
struct OutBufs {
  int device = 0;
  cudaEvent_t done = nullptr;        // end of the computation that writes these buffers
  OutSlot slot{};                    // row_ptr, col, val, beam_scale, row_max, row_cand, inst_begin, status
  int ninst = 0;                     // instances of the launch (entries of slot.summary: 1 + 2 ninst)
  long long n_tiles = 0;             // compaction tiles of the launch
  // ends of the asynchronous read-backs queued from these buffers: they are
  // freed only after those too
  std::mutex readers_mu;
  std::vector<cudaEvent_t> readers;
  ~OutBufs() {
    // the status word lives in the summary's first entry
    void* ps[] = {slot.row_ptr, slot.col, slot.val, slot.beam_scale, slot.row_max, slot.row_cand, slot.inst_begin,
                  slot.summary, slot.refine};
    release_after(done, device, ps, (int)(sizeof(ps) / sizeof(ps[0])), &readers);
    for (cudaEvent_t e : readers) cudaEventDestroy(e);
    if (done) cudaEventDestroy(done);
  }
};

struct EventSet {
  std::vector<cudaEvent_t> ev;
  ~EventSet() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

struct dsc_result {
  std::shared_ptr<Plan> plan;
  std::shared_ptr<OutBufs> out;
  std::shared_ptr<EventSet> stage_ev;  // timing events (DSC_FLAG_TIMING)
  int inst = 0;                        // instance index in the plan
  int row_base = 0, nrows = 0, beam_base = 0, nbeams = 0;
  long long rp_off = 0;                // offset of this instance's row_ptr in the output
  long long ncols = 0;
  int value_dtype = 0;
  cudaEvent_t done = nullptr;
  bool have_counts = false, have_pairs = false;
  long long out_begin = 0, nnz = 0, pairs = 0;
  // served results: the server slot and the device interval of the launch
  // that computed it (ms after the server's creation; -1: not served)
  int srv_slot = -1;
  double srv_t0_ms = -1.0, srv_t1_ms = -1.0;
  // host copies (copy_to_host = 1)
  long long* h_row_ptr = nullptr;
  int* h_col = nullptr;
  void* h_val = nullptr;
  float* h_scale = nullptr;
  ~dsc_result() {
    void* ps[] = {h_row_ptr, h_col, h_val, h_scale};
    for (void* p : ps)
      if (p) cudaFreeHost(p);
    if (done) cudaEventDestroy(done);
  }
};

struct Plan {
  std::vector<dsc_geometry*> geoms;
  std::vector<unsigned long long> geom_ids;
  dsc_compute_opts opts;
  int device = 0;
  int ninst = 0, nrows = 0, nbeams = 0, stride = 0;
  long long n_items = 0, n_cand = 0;
  std::vector<DInst> h_inst;
  std::vector<DBeam> h_beams;
  std::vector<long long> rp_off;     // per instance offset into the row_ptr output
  long long* d_inst_rp = nullptr;    // rp_off on the device, and rp_total
  long long rp_total = 0;
  // device scratch
  DInst* d_inst = nullptr;
  DBeam* d_beams = nullptr;
  DRow* d_rows = nullptr;
  int* d_row_items = nullptr;
  int* d_slice_pre = nullptr;        // per row: lines before each z-slice of its box (k_slices)
  int* d_slice_lo = nullptr;         // per row: first iy of each z-slice's lines
  int slice_stride = 0;              // entries per row: the largest nz + 1
  long long* d_row_item_base = nullptr;
  float* d_tables = nullptr;
  int* d_item_cand = nullptr;
  int* d_item_row = nullptr;
  int* d_ord_cnt = nullptr;          // kOrderClasses: items per size class (the evaluation's queue order)
  int* d_item_crank = nullptr;       // per item: its size class and rank in it
  int* d_item_ord = nullptr;         // the evaluation queue's order of the items
  long long* d_item_off = nullptr;
  int* d_tile_cnt = nullptr;
  long long* d_tile_off = nullptr;   // n_tiles + 1
  float* d_tile_thr = nullptr;
  float* d_tile_scale = nullptr;
  int* d_tile_row = nullptr;
  int* d_tile_item = nullptr;
  unsigned* d_tile_meta = nullptr;   // per tile: the evaluation's count under its item's bound
  unsigned* d_item_L = nullptr;      // per item: the bound of its row maximum it was counted against
  long long n_tiles = 0;
  float* d_vals = nullptr;
  int* d_cols = nullptr;
  unsigned* d_row_max = nullptr;
  long long* d_row_cand = nullptr;
  long long* d_scan = nullptr;       // kScanBlocks + 1
  int* d_counter = nullptr;
  // decisions the FP32 values cannot settle (the count pass lists them)
  unsigned long long* d_rlist_u = nullptr;   // near a threshold: cap_u entries
  unsigned long long* d_rcount = nullptr;    // [4] listed counts, tiles counted from their values
  int* d_mcount = nullptr;                   // per row: near-maximum candidates seen
  long long* d_mslot = nullptr;              // per row: kMaxSlots near-maximum candidates
  int* d_ovf_rows = nullptr;                 // rows that overflowed their near-maximum slots
  double* d_row_max64 = nullptr;             // per row: FP64 maximum of an overflowing row
  int cap_u = 0;
  OutSlot* d_slot = nullptr;         // output pointers of the computation in flight
  cudaGraphExec_t graph = nullptr;   // the captured launch sequence
  cudaStream_t cap_stream = nullptr; // private stream the sequence is captured on
  cudaStream_t cap_side = nullptr;   // second branch of the captured sequence (the depth tables)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t last_done = nullptr;   // end of the latest computation
  cudaStream_t last_stream = nullptr;
  int grid_eval = 0, grid_items = 0;
  int target_cand = 8192;            // candidates per work item
  int eval_bps = 0;                  // evaluation CTAs per SM (0 = occupancy limit)
  int kernels_per_run = 0;           // kernel launches in one computation
  std::mutex mu;                     // one computation at a time per plan
  void free_scratch() {
    void* ps[] = {d_item_cand, d_item_off, d_tile_cnt, d_tile_off, d_vals, d_cols, d_item_row, d_tile_thr,
                  d_tile_scale, d_rlist_u, d_tile_row, d_tile_item, d_tile_meta, d_item_L, d_ord_cnt,
                  d_item_crank, d_item_ord};
    release_after(last_done, device, ps, (int)(sizeof(ps) / sizeof(ps[0])));
    d_item_cand = nullptr; d_item_off = nullptr; d_tile_cnt = nullptr; d_tile_off = nullptr;
    d_vals = nullptr; d_cols = nullptr; d_item_row = nullptr; d_tile_thr = nullptr; d_tile_scale = nullptr;
    d_rlist_u = nullptr; d_tile_row = nullptr; d_tile_item = nullptr; d_tile_meta = nullptr; d_item_L = nullptr;
    d_ord_cnt = nullptr; d_item_crank = nullptr; d_item_ord = nullptr;
    if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }
  }
  ~Plan() {
    free_scratch();
    void* ps[] = {d_inst, d_beams, d_rows, d_row_items, d_slice_pre, d_slice_lo, d_row_item_base, d_tables, d_row_max,
                  d_row_cand, d_scan,
                  d_counter, d_slot, d_rcount, d_mcount, d_mslot, d_ovf_rows, d_row_max64, d_inst_rp};
    release_after(last_done, device, ps, (int)(sizeof(ps) / sizeof(ps[0])));
    if (last_done) cudaEventDestroy(last_done);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (cap_side) cudaStreamDestroy(cap_side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
  }
};

static SliceTab slice_tab(const Plan* P) { return SliceTab{P->d_slice_pre, P->d_slice_lo, P->slice_stride}; }

// ---------------------------------------------------------------------------
// plan cache
// ---------------------------------------------------------------------------
static std::mutex g_cache_mu;
static std::map<std::string, std::shared_ptr<Plan>> g_cache;
static std::vector<std::string> g_cache_order;
static const size_t kCacheMax = 16;

static dsc_tuning tuning_now() {
  dsc_tuning t;
  current_tuning(&t.target_cand, &t.eval_blocks_per_sm);
  return t;
}

static std::string plan_key(dsc_geometry* const* geoms, int n, const dsc_compute_opts* o, const dsc_tuning& tu) {
  std::string k;
  char buf[128];
  snprintf(buf, sizeof buf, "%.17g/%d/%.17g/%d/%d/%d|", o->rel_threshold, o->value_dtype, o->h_frac, o->flags,
           tu.target_cand, tu.eval_blocks_per_sm);
  k += buf;
  for (int i = 0; i < n; ++i) {
    snprintf(buf, sizeof buf, "%llu:", geoms[i]->id);
    k += buf;
    for (const auto& b : geoms[i]->beams) {
      k.append((const char*)&b, sizeof b);
    }
    k += ";";
  }
  return k;
}

static void cache_purge_geometry(unsigned long long id) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (auto it = g_cache.begin(); it != g_cache.end();) {
    bool uses = false;
    for (auto g : it->second->geom_ids) uses |= (g == id);
    if (uses) {
      g_cache_order.erase(std::remove(g_cache_order.begin(), g_cache_order.end(), it->first), g_cache_order.end());
      it = g_cache.erase(it);
    } else {
      ++it;
    }
  }
}

// ---------------------------------------------------------------------------
// library
// ---------------------------------------------------------------------------
extern "C" const char* dsc_status_str(dsc_status s) {
  switch (s) {
    case DSC_OK: return "ok";
    case DSC_E_INVAL: return "invalid argument";
    case DSC_E_NOMEM: return "out of memory";
    case DSC_E_NOMEM_BUDGET: return "exceeds HBM budget";
    case DSC_E_CUDA: return "CUDA error";
    case DSC_E_TIMEOUT: return "device wait timed out";
    case DSC_E_STATE: return "invalid state";
    case DSC_E_NOTFOUND: return "not found";
    case DSC_E_BUSY: return "not ready";
    case DSC_W_INEXACT: return "complete, some decisions near the threshold in FP32";
  }
  return "unknown status";
}
extern "C" const char* dsc_last_error(void) { return g_err.c_str(); }
void dsc::set_error(const char* msg) { g_err = msg; }
void dsc::count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
extern "C" int32_t dsc_abi_version(void) { return DSC_ABI_VERSION; }
extern "C" int64_t dsc_launch_count(void) { return g_launches.load(); }

static dsc_status ensure_device(int* dev) {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0)
    return fail(DSC_E_CUDA, "no CUDA device: %s", e == cudaSuccess ? "device count is 0" : cudaGetErrorString(e));
  CU(cudaGetDevice(dev));
  static std::once_flag once[64];
  if (*dev < 64)
    std::call_once(once[*dev], [d = *dev]() {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
    });
  return DSC_OK;
}

template <typename T>
static dsc_status dalloc(T** p, size_t count, cudaStream_t s) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  void* q = nullptr;
  cudaError_t e = cudaMallocAsync(&q, bytes, s);
  if (e != cudaSuccess) return fail(DSC_E_NOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
  *p = (T*)q;
  return DSC_OK;
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
extern "C" dsc_status dsc_create_geometry(const dsc_grid_desc* grid, const float* density, int32_t density_on_device,
                                          const dsc_fspb_model* model, void* stream, dsc_geometry** out) {
  if (!grid || !density || !model || !out) return fail(DSC_E_INVAL, "null argument");
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(DSC_E_INVAL, "grid dimensions must be >= 1");
  if ((long long)grid->nx * grid->ny * grid->nz >= (1ll << 31)) return fail(DSC_E_INVAL, "grid too large (>= 2^31 voxels)");
  if (!(grid->dx > 0 && grid->dy > 0 && grid->dz > 0)) return fail(DSC_E_INVAL, "voxel sides must be > 0");
  if (model->n < 2 || model->n > 4096 || !model->table4 || !(model->d_max > 0))
    return fail(DSC_E_INVAL, "model table: need 2 <= n <= 4096, d_max > 0");
  if (model->cutoff_mode < 0 || model->cutoff_mode > 2) return fail(DSC_E_INVAL, "cutoff_mode");
  if (model->profile < 0 || model->profile > 2) return fail(DSC_E_INVAL, "profile: DSC_PROFILE_ERF, _LAPLACE or _LOGISTIC");
  float c3max = 0.f;
  int kpeak = 0;
  for (int k = 0; k < model->n; ++k) {
    for (int c = 1; c <= 3; ++c) {
      const float v = model->table4[4 * k + c];
      if (!(v > 0.f) || !std::isfinite(v)) return fail(DSC_E_INVAL, "c3 widths must be finite and > 0");
    }
    if (!std::isfinite(model->table4[4 * k])) return fail(DSC_E_INVAL, "T(d) must be finite");
    c3max = std::max(c3max, model->table4[4 * k + 1]);
    if (model->table4[4 * k] > model->table4[4 * kpeak]) kpeak = k;
  }
  int dev;
  TRY(ensure_device(&dev));
  cudaStream_t s = (cudaStream_t)stream;
  auto* g = new dsc_geometry();
  g->id = g_geom_ids.fetch_add(1);
  g->device = dev;
  g->grid = *grid;
  g->n_lut = model->n;
  g->d_max = model->d_max;
  for (int i = 0; i < 3; ++i) { g->c1[i] = model->c1[i]; g->c2[i] = model->c2[i]; }
  g->cutoff_mode = model->cutoff_mode;
  g->cutoff_k = model->cutoff_k;
  g->profile = model->profile;
  g->c3max = c3max;
  g->d_peak = (float)(kpeak * (model->d_max / (model->n - 1)));
  size_t nvox = (size_t)grid->nx * grid->ny * grid->nz;
  dsc_status st = dalloc(&g->d_rho, nvox, s);
  if (st == DSC_OK) st = dalloc(&g->d_lut, 2 * (size_t)model->n, s);
  if (st == DSC_OK) st = dalloc(&g->d_lut_rows, (size_t)model->n, s);
  if (st != DSC_OK) { dsc_destroy_geometry(g); return st; }
  cudaError_t e = cudaMemcpyAsync(g->d_lut_rows, model->table4, sizeof(float4) * model->n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_lut_pairs<<<(model->n + 127) / 128, 128, 0, s>>>(g->d_lut_rows, model->n, model->profile, g->d_lut);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_rho, density, nvox * sizeof(float),
                        density_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // model table is a caller buffer
  if (e != cudaSuccess) {
    dsc_destroy_geometry(g);
    return fail(DSC_E_CUDA, "upload: %s", cudaGetErrorString(e));
  }
  *out = g;
  return DSC_OK;
}

extern "C" dsc_status dsc_upload_density(dsc_geometry* g, const float* density, int32_t on_device, void* stream) {
  if (!g || !density) return fail(DSC_E_INVAL, "null argument");
  size_t nvox = (size_t)g->grid.nx * g->grid.ny * g->grid.nz;
  CU(cudaMemcpyAsync(g->d_rho, density, nvox * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     (cudaStream_t)stream));
  return DSC_OK;
}

static dsc_status check_beam(const dsc_geometry* g, const dsc_beam_desc* b) {
  if (!(b->sad > 0) || !(b->a > 0) || !(b->b > 0) || b->n_u < 1 || b->n_v < 1)
    return fail(DSC_E_INVAL, "beam: need sad, a, b > 0 and n_u, n_v >= 1");
  if ((long long)b->n_u * b->n_v > (1 << 24)) return fail(DSC_E_INVAL, "beam: too many beamlets");
  double gr = b->gantry_deg * M_PI / 180.0;
  double S[3] = {b->iso[0] + b->sad * sin(gr), b->iso[1] - b->sad * cos(gr), b->iso[2]};
  const dsc_grid_desc& G = g->grid;
  bool inside = S[0] >= G.origin[0] && S[0] <= G.origin[0] + G.nx * G.dx && S[1] >= G.origin[1] &&
                S[1] <= G.origin[1] + G.ny * G.dy && S[2] >= G.origin[2] && S[2] <= G.origin[2] + G.nz * G.dz;
  if (inside) return fail(DSC_E_INVAL, "beam: the source lies inside the grid");
  return DSC_OK;
}

extern "C" dsc_status dsc_add_beam(dsc_geometry* g, const dsc_beam_desc* b, int32_t* idx) {
  if (!g || !b) return fail(DSC_E_INVAL, "null argument");
  TRY(check_beam(g, b));
  g->beams.push_back(*b);
  if (idx) *idx = (int32_t)g->beams.size() - 1;
  cache_purge_geometry(g->id);
  return DSC_OK;
}

extern "C" dsc_status dsc_clear_beams(dsc_geometry* g) {
  if (!g) return fail(DSC_E_INVAL, "null argument");
  g->beams.clear();
  cache_purge_geometry(g->id);
  return DSC_OK;
}

extern "C" void dsc_destroy_geometry(dsc_geometry* g) {
  if (!g) return;
  cache_purge_geometry(g->id);
  cudaDeviceSynchronize();
  if (g->d_rho) cudaFree(g->d_rho);
  if (g->d_lut) cudaFree(g->d_lut);
  if (g->d_lut_rows) cudaFree(g->d_lut_rows);
  delete g;
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------
// n_host: the input length as the host knows it (the plan's sizes); short
// inputs take the one-block scan
static dsc_status scan_launch(const int* in, const long long* n_dev, long long n_const, long long* tmp, long long* out,
                              cudaStream_t s, long long n_host) {
  if (n_host <= kSmallScan) {
    k_scan_small<<<1, 1024, 0, s>>>(in, n_dev, n_const, out);
    CHECK_LAUNCH();
    return DSC_OK;
  }
  k_scan_partial<<<kScanBlocks, kScanThreads, 0, s>>>(in, n_dev, n_const, tmp);
  CHECK_LAUNCH();
  k_scan_blocks<<<1, kScanBlocks, 0, s>>>(tmp);
  CHECK_LAUNCH();
  k_scan_final<<<kScanBlocks, kScanThreads, 0, s>>>(in, n_dev, n_const, tmp, out);
  CHECK_LAUNCH();
  return DSC_OK;
}

static dsc_status plan_build(dsc_geometry* const* geoms, int n, const dsc_compute_opts* o, cudaStream_t s,
                             std::shared_ptr<Plan>& out, const dsc_tuning& tu) {
  auto P = std::make_shared<Plan>();
  P->opts = *o;
  P->target_cand = tu.target_cand;
  P->eval_bps = tu.eval_blocks_per_sm;
  P->last_stream = s;
  TRY(ensure_device(&P->device));
  P->ninst = n;
  int row = 0, beam = 0;
  long long rp = 0;
  for (int k = 0; k < n; ++k) {
    dsc_geometry* g = geoms[k];
    P->geoms.push_back(g);
    P->geom_ids.push_back(g->id);
    DInst I{};
    if (!g->d_rho || !g->d_lut || !g->d_lut_rows) return fail(DSC_E_STATE, "geometry %d has no device tables", k);
    I.rho = g->d_rho;
    I.lut = g->d_lut;
    I.lut_rows = g->d_lut_rows;
    I.d_max = g->d_max;
    for (int i = 0; i < 3; ++i) { I.c1d[i] = g->c1[i]; I.c2d[i] = g->c2[i]; }
    I.nx = g->grid.nx; I.ny = g->grid.ny; I.nz = g->grid.nz;
    I.n_lut = g->n_lut;
    I.dx = g->grid.dx; I.dy = g->grid.dy; I.dz = g->grid.dz;
    I.ox = g->grid.origin[0]; I.oy = g->grid.origin[1]; I.oz = g->grid.origin[2];
    I.idx = 1.0 / I.dx; I.idy = 1.0 / I.dy; I.idz = 1.0 / I.dz;
    I.lut_scale = (float)((g->n_lut - 1) / g->d_max);
    I.c3max = g->c3max;
    I.d_peak = g->d_peak;
    for (int i = 0; i < 3; ++i) { I.c1q[i] = (float)(g->c1[i] / 4.0); I.c2h[i] = (float)(g->c2[i] / 2.0); }
    I.cutoff_mode = g->cutoff_mode;
    I.cutoff_k = (float)g->cutoff_k;
    I.profile = g->profile;
    double dmin = std::min(g->grid.dx, std::min(g->grid.dy, g->grid.dz));
    I.hd = o->h_frac * dmin;
    I.h = (float)I.hd;
    I.inv_h = (float)(1.0 / I.hd);
    I.row_base = row;
    I.beam_base = beam;
    I.nbeams = (int)g->beams.size();
    double diag = std::sqrt(std::pow(g->grid.nx * g->grid.dx, 2) + std::pow(g->grid.ny * g->grid.dy, 2) +
                            std::pow(g->grid.nz * g->grid.dz, 2));
    P->stride = std::max(P->stride, (int)std::ceil(diag / I.hd) + 2);
    for (const auto& b : g->beams) {
      DBeam B{};
      B.inst = k;
      B.row_base = row;
      B.n_u = b.n_u; B.n_v = b.n_v;
      B.gantry_deg = b.gantry_deg; B.sad = b.sad;
      for (int i = 0; i < 3; ++i) B.iso[i] = b.iso[i];
      B.a = b.a; B.b = b.b;
      P->h_beams.push_back(B);
      row += b.n_u * b.n_v;
      ++beam;
    }
    I.nrows = row - I.row_base;
    P->h_inst.push_back(I);
    P->rp_off.push_back(rp);
    rp += I.nrows + 1;
  }
  P->nrows = row;
  P->nbeams = beam;
  P->rp_total = rp;
  if (P->nrows == 0) return fail(DSC_E_STATE, "no beams");
  P->stride = (P->stride + 3) & ~3;
  TRY(dalloc(&P->d_inst, n, s));
  TRY(dalloc(&P->d_inst_rp, n + 1, s));
  {
    std::vector<long long> rp(P->rp_off);
    rp.push_back(P->rp_total);
    // pageable source: staged before the call returns
    CU(cudaMemcpyAsync(P->d_inst_rp, rp.data(), sizeof(long long) * rp.size(), cudaMemcpyHostToDevice, s));
  }
  TRY(dalloc(&P->d_beams, P->nbeams, s));
  TRY(dalloc(&P->d_rows, P->nrows, s));
  TRY(dalloc(&P->d_row_items, P->nrows, s));
  P->slice_stride = 2;
  for (const DInst& I : P->h_inst) P->slice_stride = std::max(P->slice_stride, I.nz + 1);
  TRY(dalloc(&P->d_slice_pre, (size_t)P->nrows * P->slice_stride, s));
  TRY(dalloc(&P->d_slice_lo, (size_t)P->nrows * P->slice_stride, s));
  TRY(dalloc(&P->d_row_item_base, P->nrows + 1, s));
  TRY(dalloc(&P->d_tables, (size_t)P->nrows * P->stride, s));
  TRY(dalloc(&P->d_row_max, P->nrows, s));
  TRY(dalloc(&P->d_row_cand, P->nrows, s));
  TRY(dalloc(&P->d_scan, kScanBlocks + 1, s));
  TRY(dalloc(&P->d_counter, 4, s));
  if (P->nrows >= (1 << 24)) return fail(DSC_E_INVAL, "too many beamlets in one launch (%d)", P->nrows);
  TRY(dalloc(&P->d_rcount, 4, s));
  TRY(dalloc(&P->d_mcount, P->nrows, s));
  TRY(dalloc(&P->d_ovf_rows, P->nrows, s));
  TRY(dalloc(&P->d_row_max64, P->nrows, s));
  TRY(dalloc(&P->d_mslot, (size_t)P->nrows * kMaxSlots, s));
  TRY(dalloc(&P->d_slot, 1, s));
  CU(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  CU(cudaStreamCreateWithFlags(&P->cap_side, cudaStreamNonBlocking));
  CU(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&P->last_done, cudaEventDisableTiming));
  CU(cudaMemcpyAsync(P->d_inst, P->h_inst.data(), sizeof(DInst) * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(P->d_beams, P->h_beams.data(), sizeof(DBeam) * P->nbeams, cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(P->d_tables, 0, sizeof(float) * (size_t)P->nrows * P->stride, s));

  // sizes: items (from the set-up) and candidates (from the count)
  k_setup<<<(P->nrows + 31) / 32, 32, 0, s>>>(P->d_inst, P->d_beams, P->nbeams, P->d_rows, P->nrows,
                                                 P->d_row_items, P->target_cand, StepClear{});
  CHECK_LAUNCH();
  k_slices<<<(P->nrows + 3) / 4, 128, 0, s>>>(P->d_inst, P->d_rows, P->nrows, P->d_slice_pre, P->d_slice_lo,
                                              P->slice_stride, P->d_row_items);
  CHECK_LAUNCH();
  TRY(scan_launch(P->d_row_items, nullptr, P->nrows, P->d_scan, P->d_row_item_base, s, P->nrows));
  CU(cudaMemcpyAsync(&P->n_items, P->d_row_item_base + P->nrows, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  TRY(dalloc(&P->d_item_cand, P->n_items, s));
  TRY(dalloc(&P->d_item_row, P->n_items, s));
  TRY(dalloc(&P->d_item_off, P->n_items + 1, s));
  TRY(dalloc(&P->d_item_L, P->n_items, s));
  TRY(dalloc(&P->d_ord_cnt, kOrderClasses, s));
  TRY(dalloc(&P->d_item_crank, P->n_items, s));
  TRY(dalloc(&P->d_item_ord, P->n_items, s));
  if (P->n_items >= (1ll << kOrderRankBits)) return fail(DSC_E_INVAL, "too many work items (%lld)", P->n_items);
  int sms = 0, nb = 0;
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device));
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval, kEvalThreads, 0));
  nb = std::max(1, nb);
  P->grid_eval = (P->eval_bps > 0 ? std::min(P->eval_bps, nb) : nb) * sms;
  // the candidate count runs beside the depth tables (one 32-thread CTA per
  // beamlet): at most half of an SM's threads, so that both are resident
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_count, kEvalThreads, 0));
  P->grid_items = std::min(std::max(1, nb), 8) * sms;
  k_item_rows<<<(P->nrows + 127) / 128, 128, 0, s>>>(P->d_row_item_base, P->nrows, P->d_item_row);
  CHECK_LAUNCH();
  k_count<<<P->grid_items, kEvalThreads, 0, s>>>(P->d_inst, P->d_rows, slice_tab(P.get()), P->d_row_item_base,
                                                 P->nrows, P->d_row_item_base + P->nrows, P->d_item_cand,
                                                 P->d_item_row, nullptr, nullptr, P->target_cand);
  CHECK_LAUNCH();
  TRY(scan_launch(P->d_item_cand, P->d_row_item_base + P->nrows, 0, P->d_scan, P->d_item_off, s, P->n_items));
  CU(cudaMemcpyAsync(&P->n_cand, P->d_item_off + P->n_items, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  P->n_tiles = P->n_cand / kTile;                     // items are whole tiles
  TRY(dalloc(&P->d_vals, P->n_cand + 4, s));
  TRY(dalloc(&P->d_cols, P->n_cand + 4, s));
  TRY(dalloc(&P->d_tile_cnt, P->n_tiles, s));
  TRY(dalloc(&P->d_tile_off, P->n_tiles + 1, s));
  TRY(dalloc(&P->d_tile_thr, P->n_tiles, s));
  TRY(dalloc(&P->d_tile_scale, P->n_tiles, s));
  TRY(dalloc(&P->d_tile_row, P->n_tiles, s));
  TRY(dalloc(&P->d_tile_item, P->n_tiles, s));
  TRY(dalloc(&P->d_tile_meta, P->n_tiles, s));
  // about 1e-5 of the candidates fall within kRefineDelta of their threshold
  P->cap_u = (int)std::min<long long>(std::max<long long>(1 << 16, P->n_cand >> 10), 1 << 28);
  TRY(dalloc(&P->d_rlist_u, P->cap_u, s));
  out = P;
  return DSC_OK;
}

static dsc_status plan_get(dsc_geometry* const* geoms, int n, const dsc_compute_opts* o, cudaStream_t s,
                           std::shared_ptr<Plan>& out) {
  const dsc_tuning tu = tuning_now();
  std::string key = plan_key(geoms, n, o, tu);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) { out = it->second; return DSC_OK; }
  }
  TRY(plan_build(geoms, n, o, s, out, tu));
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_cache[key] = out;
  g_cache_order.push_back(key);
  while (g_cache_order.size() > kCacheMax) {
    g_cache.erase(g_cache_order.front());
    g_cache_order.erase(g_cache_order.begin());
  }
  return DSC_OK;
}


// ---------------------------------------------------------------------------
// the launch sequence of one computation (stream-ordered, graph-capturable)
// ---------------------------------------------------------------------------
enum { ST_SETUP, ST_SIDDON, ST_COUNT, ST_EVAL, ST_SCALE, ST_COMPACT, ST_FINISH, ST_N };

static dsc_status record(EventSet* ev, int i, cudaStream_t s) {
  if (ev) CU(cudaEventRecord(ev->ev[i], s));
  return DSC_OK;
}

// the FP64 re-evaluation of the listed pairs (their row maxima and keep decisions)
static dsc_status refine_launch(Plan* P, const CompactParams& cp, cudaStream_t s) {
  RefineParams rp{};
  rp.inst = P->d_inst;
  rp.rows = P->d_rows;
  rp.beams = P->d_beams;
  rp.tables = P->d_tables;
  rp.table_stride = P->stride;
  rp.item_off = P->d_item_off;
  rp.item_row = P->d_item_row;
  rp.n_items = cp.n_items;
  rp.vals = P->d_vals;
  rp.cols = P->d_cols;
  rp.row_max = P->d_row_max;
  rp.tau = cp.tau;
  rp.tau_d = P->opts.rel_threshold;
  rp.rlist_u = P->d_rlist_u;
  rp.rcount = P->d_rcount;
  rp.cap_u = P->cap_u;
  rp.mcount = P->d_mcount;
  rp.ovf_rows = P->d_ovf_rows;
  rp.row_max64 = P->d_row_max64;
  rp.row_item_base = P->d_row_item_base;
  rp.inv_tau_m = cp.inv_tau_m;
  rp.mslot = P->d_mslot;
  rp.tile_cnt = P->d_tile_cnt;
  rp.nrows = P->nrows;
  rp.n_cand = P->n_cand;
  rp.slot = P->d_slot;
  k_refine_rowmax<<<kRefineRowmaxBlocks, kRefineThreads, 0, s>>>(rp);
  CHECK_LAUNCH();
  k_refine<<<refine_blocks(P->cap_u), kRefineThreads, 0, s>>>(rp);
  CHECK_LAUNCH();
  return DSC_OK;
}

static dsc_status enqueue(Plan* P, cudaStream_t s, EventSet* ev, int* nk) {
  int k0 = (int)g_launches.load();
  const long long* n_items = P->d_row_item_base + P->nrows;
  TRY(record(ev, 0, s));
  const StepClear clr{P->d_row_max, P->d_row_cand, P->d_mcount, P->d_counter, P->d_rcount, P->d_ord_cnt};
  k_setup<<<(P->nrows + 31) / 32, 32, 0, s>>>(P->d_inst, P->d_beams, P->nbeams, P->d_rows, P->nrows,
                                                 P->d_row_items, P->target_cand, clr);
  CHECK_LAUNCH();
  k_slices<<<(P->nrows + 3) / 4, 128, 0, s>>>(P->d_inst, P->d_rows, P->nrows, P->d_slice_pre, P->d_slice_lo,
                                              P->slice_stride, P->d_row_items);
  CHECK_LAUNCH();
  TRY(scan_launch(P->d_row_items, nullptr, P->nrows, P->d_scan, P->d_row_item_base, s, P->nrows));
  TRY(record(ev, 1, s));
  // a2: radiological-depth tables.  The captured sequence (no stage events)
  // traces them on a second branch beside a3, which does not read them; the
  // branches join before the evaluation.
  const bool fork = ev == nullptr;
  cudaStream_t ts = s;
  if (fork) {
    CU(cudaEventRecord(P->ev_fork, s));
    CU(cudaStreamWaitEvent(P->cap_side, P->ev_fork, 0));
    ts = P->cap_side;
  }
  if (P->opts.flags & DSC_FLAG_TRILINEAR_TABLE)
    k_trilinear_table<<<P->nrows, kSiddonThreads, 0, ts>>>(P->d_inst, P->d_rows, P->nrows, P->d_tables, P->stride);
  else
    k_siddon<<<P->nrows, kSiddonThreads, 0, ts>>>(P->d_inst, P->d_rows, P->nrows, P->d_tables, P->stride);
  CHECK_LAUNCH();
  // a lower bound of each row maximum, from the voxels by the axis (the
  // evaluation counts the tiles against it)
  k_row_bound<<<(P->nrows + 3) / 4, 128, 0, ts>>>(P->d_inst, P->d_rows, P->nrows, P->d_tables, P->stride, slice_tab(P),
                                                  P->d_row_max);
  CHECK_LAUNCH();
  if (fork) CU(cudaEventRecord(P->ev_join, ts));
  TRY(record(ev, 2, s));
  // a3: candidate pairs per work item
  k_item_rows<<<(P->nrows + 127) / 128, 128, 0, s>>>(P->d_row_item_base, P->nrows, P->d_item_row);
  CHECK_LAUNCH();
  k_count<<<P->grid_items, kEvalThreads, 0, s>>>(P->d_inst, P->d_rows, slice_tab(P), P->d_row_item_base, P->nrows,
                                                 n_items, P->d_item_cand, P->d_item_row, P->d_ord_cnt,
                                                 P->d_item_crank, P->target_cand);
  CHECK_LAUNCH();
  TRY(scan_launch(P->d_item_cand, n_items, 0, P->d_scan, P->d_item_off, s, P->n_items));
  k_tile_map<<<1024, 256, 0, s>>>(P->d_item_off, n_items, P->d_item_row, P->d_tile_item, P->d_tile_row,
                                 P->d_ord_cnt, P->d_item_crank, P->d_item_ord);
  CHECK_LAUNCH();
  if (fork) CU(cudaStreamWaitEvent(s, P->ev_join, 0));
  TRY(record(ev, 3, s));
  // a4: FSPB evaluation
  EvalParams ep{};
  ep.inst = P->d_inst;
  ep.rows = P->d_rows;
  ep.slices = slice_tab(P);
  ep.tables = P->d_tables;
  ep.table_stride = P->stride;
  ep.row_item_base = P->d_row_item_base;
  ep.nrows = P->nrows;
  ep.item_off = P->d_item_off;
  ep.item_row = P->d_item_row;
  ep.n_items = n_items;
  ep.vals = P->d_vals;
  ep.cols = P->d_cols;
  ep.row_max = P->d_row_max;
  ep.row_cand = P->d_row_cand;
  ep.item_counter = P->d_counter;
  ep.item_ord = P->d_item_ord;
  ep.tau = (float)P->opts.rel_threshold;
  ep.inv_tau_m = ep.tau > 0.0f ? (1.0f - kRefineDelta) / ep.tau : std::numeric_limits<float>::infinity();
  ep.tile_meta = P->d_tile_meta;
  ep.item_L = P->d_item_L;
  k_eval<<<P->grid_eval, kEvalThreads, 0, s>>>(ep);
  CHECK_LAUNCH();
  TRY(record(ev, 4, s));
  // a6: per-beam scale of the BF16 values
  if (P->opts.value_dtype == DSC_VALUE_BF16) {
    k_beam_scale<<<(P->nbeams + 127) / 128, 128, 0, s>>>(P->d_beams, P->nbeams, P->d_row_max, P->d_slot);
    CHECK_LAUNCH();
  }
  TRY(record(ev, 5, s));
  // a5: threshold + CSR compaction: kept count per tile, scan, write
  CompactParams cp{};
  cp.rows = P->d_rows;
  cp.item_off = P->d_item_off;
  cp.item_row = P->d_item_row;
  cp.n_items = n_items;
  cp.n_cand = P->n_cand;
  cp.vals = P->d_vals;
  cp.cols = P->d_cols;
  cp.row_max = P->d_row_max;
  cp.tau = (float)P->opts.rel_threshold;
  cp.tile_thr = P->d_tile_thr;
  cp.tile_scale = P->d_tile_scale;
  cp.tile_row = P->d_tile_row;
  cp.tile_item = P->d_tile_item;
  cp.tile_meta = P->d_tile_meta;
  cp.item_L = P->d_item_L;
  cp.value_dtype = P->opts.value_dtype;
  cp.slot = P->d_slot;
  cp.rlist_u = P->d_rlist_u;
  cp.rcount = P->d_rcount;
  cp.mcount = P->d_mcount;
  cp.mslot = P->d_mslot;
  cp.ovf_rows = P->d_ovf_rows;
  cp.cap_u = P->cap_u;
  cp.nrows = P->nrows;
  cp.inv_tau_m = cp.tau > 0.0f ? (1.0f - kRefineDelta) / cp.tau : std::numeric_limits<float>::infinity();
  const unsigned tiles = compact_blocks(P->n_tiles);
  k_tile_count<<<tile_blocks(P->n_tiles, kCountTilesPerWarp), kEvalThreads, 0, s>>>(cp, P->d_tile_cnt);
  CHECK_LAUNCH();
  TRY(refine_launch(P, cp, s));
  TRY(scan_launch(P->d_tile_cnt, nullptr, P->n_tiles, P->d_scan, P->d_tile_off, s, P->n_tiles));
  k_tile_write<<<tiles, kEvalThreads, 0, s>>>(cp, P->d_tile_off);
  CHECK_LAUNCH();
  TRY(record(ev, 6, s));
  // row pointers of every instance, row statistics and counts, one launch
  k_finish<<<(unsigned)((P->rp_total + 255) / 256), 256, 0, s>>>(P->d_row_item_base, P->d_item_off, P->d_tile_off,
                                                                 n_items, P->n_cand, P->d_inst_rp, P->ninst,
                                                                 P->d_row_max, P->d_row_cand, P->nrows, P->d_rcount,
                                                                 P->cap_u, P->d_slot);
  CHECK_LAUNCH();
  TRY(record(ev, 7, s));
  if (nk) *nk = (int)(g_launches.load() - k0);
  return DSC_OK;
}

static dsc_status alloc_outputs(Plan* P, cudaStream_t s, std::shared_ptr<OutBufs>& O) {
  O = std::make_shared<OutBufs>();
  O->device = P->device;
  CU(cudaEventCreateWithFlags(&O->done, cudaEventDisableTiming));
  OutSlot& q = O->slot;
  TRY(dalloc(&q.row_ptr, P->rp_total, s));
  TRY(dalloc(&q.col, P->n_cand, s));
  if (P->opts.value_dtype == DSC_VALUE_BF16) {
    __nv_bfloat16* v;
    TRY(dalloc(&v, P->n_cand, s));
    q.val = v;
  } else {
    float* v;
    TRY(dalloc(&v, P->n_cand, s));
    q.val = v;
  }
  TRY(dalloc(&q.beam_scale, P->nbeams, s));
  TRY(dalloc(&q.row_max, P->nrows, s));
  TRY(dalloc(&q.row_cand, P->nrows, s));
  TRY(dalloc(&q.inst_begin, P->ninst + 1, s));
  TRY(dalloc(&q.refine, 4, s));
  O->n_tiles = P->n_tiles;
  O->ninst = P->ninst;
  TRY(dalloc(&q.summary, 1 + 2 * (size_t)P->ninst, s));
  q.status = reinterpret_cast<int*>(q.summary);
  // cleared (and, for FP32 values, which carry no scale, the beam scales set
  // to 1) by k_out_init at the head of the computation
  return DSC_OK;
}

// One computation over `n` geometries with plan P (caller holds P->mu).
static dsc_status run_plan(const std::shared_ptr<Plan>& P, cudaStream_t s, bool timing, dsc_result** outs) {
  P->last_stream = s;
  std::shared_ptr<OutBufs> O;
  TRY(alloc_outputs(P.get(), s, O));
  k_out_init<<<1, 256, 0, s>>>(P->d_slot, O->slot, P->ninst, P->nbeams, P->opts.value_dtype != DSC_VALUE_BF16);
  CHECK_LAUNCH();
  std::shared_ptr<EventSet> ev;
  if (timing) {
    ev = std::make_shared<EventSet>();
    ev->ev.resize(ST_N + 1);
    for (auto& e : ev->ev) CU(cudaEventCreate(&e));
    TRY(enqueue(P.get(), s, ev.get(), &P->kernels_per_run));
  } else {
    if (!P->graph) {
      cudaGraph_t g;
      cudaStream_t cs = P->cap_stream;
      CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      long long before = g_launches.load();
      dsc_status st = enqueue(P.get(), cs, nullptr, &P->kernels_per_run);
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      g_launches.store(before);   // captured, not launched
      if (st != DSC_OK) return st;
      if (e != cudaSuccess) return fail(DSC_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&P->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(DSC_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    CU(cudaGraphLaunch(P->graph, s));
    g_launches.fetch_add(P->kernels_per_run);
  }
  CU(cudaEventRecord(O->done, s));
  CU(cudaEventRecord(P->last_done, s));
  for (int k = 0; k < P->ninst; ++k) {
    auto* r = new dsc_result();
    r->plan = P;
    r->out = O;
    r->stage_ev = ev;
    r->inst = k;
    const DInst& I = P->h_inst[k];
    r->row_base = I.row_base;
    r->nrows = I.nrows;
    r->beam_base = I.beam_base;
    r->nbeams = I.nbeams;
    r->rp_off = P->rp_off[k];
    r->ncols = (long long)I.nx * I.ny * I.nz;
    r->value_dtype = P->opts.value_dtype;
    CU(cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming));
    CU(cudaEventRecord(r->done, s));
    outs[k] = r;
  }
  return DSC_OK;
}

static dsc_status check_opts(const dsc_compute_opts* o) {
  if (!o) return fail(DSC_E_INVAL, "null opts");
  if (!(o->rel_threshold >= 0) || !(o->h_frac > 0 && o->h_frac <= 1) ||
      (o->value_dtype != DSC_VALUE_F32 && o->value_dtype != DSC_VALUE_BF16))
    return fail(DSC_E_INVAL, "opts: need rel_threshold >= 0, 0 < h_frac <= 1, value_dtype F32 or BF16");
  return DSC_OK;
}

static dsc_status compute_common(dsc_geometry* const* geoms, int n, const dsc_compute_opts* opts, void* stream,
                                 dsc_result** outs, bool cache) {
  if (!geoms || n < 1 || !outs) return fail(DSC_E_INVAL, "null argument");
  TRY(check_opts(opts));
  for (int k = 0; k < n; ++k) {
    outs[k] = nullptr;
    if (!geoms[k]) return fail(DSC_E_INVAL, "null geometry");
    if (geoms[k]->beams.empty()) return fail(DSC_E_STATE, "geometry %d has no beams", k);
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::shared_ptr<Plan> P;
  if (cache) {
    TRY(plan_get(geoms, n, opts, s, P));
  } else {
    TRY(plan_build(geoms, n, opts, s, P, tuning_now()));
  }
  std::lock_guard<std::mutex> lk(P->mu);
  dsc_status st = run_plan(P, s, (opts->flags & DSC_FLAG_TIMING) != 0, outs);
  if (st != DSC_OK)
    for (int k = 0; k < n; ++k) { delete outs[k]; outs[k] = nullptr; }
  return st;
}

extern "C" dsc_status dsc_compute_dij(dsc_geometry* geom, const dsc_compute_opts* opts, void* stream, dsc_result** out) {
  return compute_common(&geom, 1, opts, stream, out, true);
}

extern "C" dsc_status dsc_compute_dij_batch(dsc_geometry* const* geoms, int32_t n, const dsc_compute_opts* opts,
                                            void* stream, dsc_result** outs) {
  return compute_common(geoms, n, opts, stream, outs, true);
}

// ---------------------------------------------------------------------------
// work decomposition and its autotuner
// ---------------------------------------------------------------------------
static dsc_status check_tuning(const dsc_tuning* t) {
  if (!t) return fail(DSC_E_INVAL, "null tuning");
  if (t->target_cand < 512 || t->target_cand > 65536 || t->eval_blocks_per_sm < 0 || t->eval_blocks_per_sm > 64)
    return fail(DSC_E_INVAL, "tuning: need 512 <= target_cand <= 65536 and 0 <= eval_blocks_per_sm <= 64");
  return DSC_OK;
}

extern "C" dsc_status dsc_set_tuning(const dsc_tuning* t) {
  TRY(check_tuning(t));
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  g_tuning = *t;
  return DSC_OK;
}

extern "C" dsc_status dsc_get_tuning(dsc_tuning* t) {
  if (!t) return fail(DSC_E_INVAL, "null tuning");
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  *t = g_tuning;
  return DSC_OK;
}

extern "C" dsc_status dsc_autotune(dsc_geometry* const* geoms, int32_t n, const dsc_compute_opts* opts, void* stream,
                                   int32_t reps, dsc_tuning* best, float* best_ms) {
  if (!geoms || n < 1 || !best || reps < 1 || reps > 100) return fail(DSC_E_INVAL, "autotune: bad arguments");
  TRY(check_opts(opts));
  for (int k = 0; k < n; ++k) {
    if (!geoms[k]) return fail(DSC_E_INVAL, "null geometry");
    if (geoms[k]->beams.empty()) return fail(DSC_E_STATE, "geometry %d has no beams", k);
  }
  cudaStream_t s = (cudaStream_t)stream;
  dsc_compute_opts o = *opts;
  o.flags &= ~DSC_FLAG_TIMING;   // graph replays, as production calls run
  int dev, sms = 0, nb = 0;
  TRY(ensure_device(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval, kEvalThreads, 0));
  nb = std::max(1, nb);
  std::vector<int> bps_set = {0};
  for (int b : {(3 * nb) / 4, nb / 2})
    if (b >= 1 && b < nb && std::find(bps_set.begin(), bps_set.end(), b) == bps_set.end()) bps_set.push_back(b);
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  std::vector<dsc_result*> outs(n, nullptr);
  auto release = [&]() {
    for (auto& r : outs) {
      dsc_release_result(r);
      r = nullptr;
    }
  };
  dsc_status st = DSC_OK;
  float best_t = 1e30f;
  dsc_tuning bt = tuning_now();
  for (int tc = 2048; tc <= 32768 && st == DSC_OK; tc *= 2) {
    for (int bps : bps_set) {
      const dsc_tuning tu = {tc, bps};
      std::shared_ptr<Plan> P;
      st = plan_build(geoms, n, &o, s, P, tu);
      if (st != DSC_OK) break;
      std::lock_guard<std::mutex> lk(P->mu);
      st = run_plan(P, s, false, outs.data());   // warm-up: captures the graph
      release();
      std::vector<float> t;
      for (int r = 0; r < reps && st == DSC_OK; ++r) {
        cudaEventRecord(e0, s);
        st = run_plan(P, s, false, outs.data());
        cudaEventRecord(e1, s);
        if (st == DSC_OK) {
          cudaError_t e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) st = fail(DSC_E_CUDA, "autotune timing: %s", cudaGetErrorString(e));
          t.push_back(ms);
        }
        release();
      }
      if (st != DSC_OK) break;
      std::sort(t.begin(), t.end());
      const float med = t[t.size() / 2];
      if (med < best_t) { best_t = med; bt = tu; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DSC_OK) return st;
  TRY(dsc_set_tuning(&bt));
  *best = bt;
  if (best_ms) *best_ms = best_t;
  return DSC_OK;
}

// ---------------------------------------------------------------------------
// results
// ---------------------------------------------------------------------------
static dsc_status status_error(int st) {
  if (st & kStatusIndex) return fail(DSC_E_CUDA, "a kernel found an index out of range (status %d); the result is invalid", st);
  if (st) return fail(DSC_E_TIMEOUT, "a bounded device wait expired (status %d); the result is invalid", st);
  return DSC_OK;
}

static dsc_status check_status(dsc_result* r) {
  int st = 0;
  CU(cudaEventSynchronize(r->done));
  CU(cudaMemcpy(&st, r->out->slot.status, sizeof(int), cudaMemcpyDeviceToHost));
  return status_error(st);
}

extern "C" dsc_status dsc_result_wait(dsc_result* r) {
  if (!r) return fail(DSC_E_INVAL, "null result");
  return check_status(r);
}

// the result's status, first output entry and kept count: one copy of the
// summary's head (the status word, then two entries per instance)
static dsc_status fetch_counts(dsc_result* r) {
  if (r->have_counts) return DSC_OK;
  CU(cudaEventSynchronize(r->done));
  const size_t n = 3 + 2 * (size_t)r->inst;
  long long sm[3 + 2 * 64];
  std::vector<long long> big;
  long long* h = sm;
  if (n > sizeof(sm) / sizeof(sm[0])) {
    big.resize(n);
    h = big.data();
  }
  CU(cudaMemcpy(h, r->out->slot.summary, sizeof(long long) * n, cudaMemcpyDeviceToHost));
  TRY(status_error((int)(h[0] & 0xffffffffll)));
  r->out_begin = h[1 + 2 * r->inst];
  r->nnz = h[2 + 2 * r->inst];
  r->have_counts = true;
  return DSC_OK;
}

// candidate pairs of the result's rows (read when asked for: the read-back
// does not need them)
static dsc_status fetch_pairs(dsc_result* r) {
  if (r->have_pairs) return DSC_OK;
  TRY(fetch_counts(r));
  std::vector<long long> rc(r->nrows);
  CU(cudaMemcpy(rc.data(), r->out->slot.row_cand + r->row_base, sizeof(long long) * r->nrows, cudaMemcpyDeviceToHost));
  long long p = 0;
  for (auto v : rc) p += v;
  r->pairs = p;
  r->have_pairs = true;
  return DSC_OK;
}

static size_t val_size(int dt) { return dt == DSC_VALUE_BF16 ? 2 : 4; }

extern "C" dsc_status dsc_get_csr(dsc_result* r, int32_t copy_to_host, dsc_csr_view* v) {
  if (!r || !v) return fail(DSC_E_INVAL, "null argument");
  TRY(fetch_pairs(r));
  const OutSlot& q = r->out->slot;
  v->nrows = r->nrows;
  v->ncols = r->ncols;
  v->nnz = r->nnz;
  v->value_dtype = r->value_dtype;
  v->nbeams = r->nbeams;
  v->pairs = r->pairs;
  if (!copy_to_host) {
    v->row_ptr = (const int64_t*)(q.row_ptr + r->rp_off);
    v->col = q.col + r->out_begin;
    v->val = (const char*)q.val + val_size(r->value_dtype) * r->out_begin;
    v->beam_scale = q.beam_scale + r->beam_base;
    v->on_device = 1;
    return DSC_OK;
  }
  if (!r->h_row_ptr) {
    CU(cudaMallocHost((void**)&r->h_row_ptr, sizeof(long long) * (r->nrows + 1)));
    CU(cudaMallocHost((void**)&r->h_col, sizeof(int) * std::max<long long>(r->nnz, 1)));
    CU(cudaMallocHost(&r->h_val, val_size(r->value_dtype) * std::max<long long>(r->nnz, 1)));
    CU(cudaMallocHost((void**)&r->h_scale, sizeof(float) * std::max(r->nbeams, 1)));
    TRY(dsc_copy_csr_to_host(r, (int64_t*)r->h_row_ptr, r->h_col, r->h_val, r->h_scale, nullptr));
  }
  v->row_ptr = (const int64_t*)r->h_row_ptr;
  v->col = r->h_col;
  v->val = r->h_val;
  v->beam_scale = r->h_scale;
  v->on_device = 0;
  return DSC_OK;
}

extern "C" dsc_status dsc_copy_csr_to_host_async(dsc_result* r, int64_t* row_ptr, int32_t* col, void* val,
                                                 float* beam_scale, void* stream) {
  if (!r || !row_ptr || !col || !val) return fail(DSC_E_INVAL, "null argument");
  TRY(fetch_counts(r));                                // the computation has finished: its counts size the copies
  cudaStream_t s = (cudaStream_t)stream;
  const OutSlot& q = r->out->slot;
  CU(cudaMemcpyAsync(row_ptr, q.row_ptr + r->rp_off, sizeof(long long) * (r->nrows + 1), cudaMemcpyDeviceToHost, s));
  if (r->nnz > 0) {
    CU(cudaMemcpyAsync(col, q.col + r->out_begin, sizeof(int) * r->nnz, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(val, (const char*)q.val + val_size(r->value_dtype) * r->out_begin,
                       val_size(r->value_dtype) * r->nnz, cudaMemcpyDeviceToHost, s));
  }
  if (beam_scale)
    CU(cudaMemcpyAsync(beam_scale, q.beam_scale + r->beam_base, sizeof(float) * r->nbeams, cudaMemcpyDeviceToHost, s));
  // the device buffers outlive these copies, also when the result is released first
  cudaEvent_t e = nullptr;
  CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaError_t err = cudaEventRecord(e, s);
  if (err != cudaSuccess) {
    cudaEventDestroy(e);
    return fail(DSC_E_CUDA, "cudaEventRecord: %s", cudaGetErrorString(err));
  }
  std::lock_guard<std::mutex> lk(r->out->readers_mu);
  r->out->readers.push_back(e);
  return DSC_OK;
}

extern "C" dsc_status dsc_copy_csr_to_host(dsc_result* r, int64_t* row_ptr, int32_t* col, void* val, float* beam_scale,
                                           void* stream) {
  TRY(dsc_copy_csr_to_host_async(r, row_ptr, col, val, beam_scale, stream));
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  return DSC_OK;
}

extern "C" void dsc_release_result(dsc_result* r) { delete r; }

extern "C" dsc_status dsc_get_beamlets(dsc_result* r, double* out, int64_t cap_rows) {
  if (!r || !out) return fail(DSC_E_INVAL, "null argument");
  if (cap_rows < r->nrows) return fail(DSC_E_INVAL, "cap_rows < nrows");
  if (!r->plan->d_rows) return fail(DSC_E_STATE, "stage data released");
  CU(cudaEventSynchronize(r->done));
  std::vector<DRow> rows(r->nrows);
  CU(cudaMemcpy(rows.data(), r->plan->d_rows + r->row_base, sizeof(DRow) * r->nrows, cudaMemcpyDeviceToHost));
  for (int i = 0; i < r->nrows; ++i) {
    double* o = out + 16 * (size_t)i;
    const DRow& R = rows[i];
    for (int k = 0; k < 3; ++k) { o[k] = R.S[k]; o[3 + k] = R.e[k]; o[6 + k] = R.x[k]; o[9 + k] = R.z[k]; }
    o[12] = R.tA; o[13] = R.tB; o[14] = R.hit; o[15] = R.n_table;
  }
  return DSC_OK;
}

extern "C" dsc_status dsc_get_depth_tables(dsc_result* r, float* out, int64_t cap, int32_t* n_max) {
  if (!r || !n_max) return fail(DSC_E_INVAL, "null argument");
  *n_max = r->plan->stride;
  if (!out) return DSC_OK;
  if (cap < (int64_t)r->nrows * r->plan->stride) return fail(DSC_E_INVAL, "cap < nrows * n_max");
  CU(cudaEventSynchronize(r->done));
  CU(cudaMemcpy(out, r->plan->d_tables + (size_t)r->row_base * r->plan->stride,
                sizeof(float) * (size_t)r->nrows * r->plan->stride, cudaMemcpyDeviceToHost));
  return DSC_OK;
}

// ---------------------------------------------------------------------------
// products with the resident D_ij (Eq. 1 and its transpose)
// ---------------------------------------------------------------------------
static unsigned row_blocks_grid(int nrows) {
  return (unsigned)std::max(1, std::min(nrows, 152 * 32));   // one 256-thread block per row, grid-stride beyond
}

extern "C" dsc_status dsc_dose(dsc_result* r, const float* w_dev, float* dose_dev, void* stream) {
  if (!r || !w_dev || !dose_dev) return fail(DSC_E_INVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaStreamWaitEvent(s, r->done, 0));
  const OutSlot& q = r->out->slot;
  unsigned long long* acc = nullptr;
  int* ex = nullptr;
  TRY(dalloc(&acc, (size_t)r->ncols, s));
  TRY(dalloc(&ex, 1, s));
  CU(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)r->ncols, s));
  k_dose_scale<<<1, 1024, 0, s>>>(q.row_max + r->row_base, w_dev, r->nrows, ex);
  CHECK_LAUNCH();
  k_dose_scatter<<<row_blocks_grid(r->nrows), 256, 0, s>>>(q.row_ptr + r->rp_off, q.inst_begin + r->inst, q.col, q.val,
                                                          r->value_dtype, r->plan->d_rows, r->row_base, q.beam_scale,
                                                          w_dev, r->nrows, ex, acc);
  CHECK_LAUNCH();
  const long long nb = std::min<long long>((r->ncols + 255) / 256, 152 * 32);
  k_dose_finish<<<(unsigned)std::max(1ll, nb), 256, 0, s>>>(acc, r->ncols, ex, dose_dev);
  CHECK_LAUNCH();
  CU(cudaFreeAsync(acc, s));
  CU(cudaFreeAsync(ex, s));
  return DSC_OK;
}

extern "C" dsc_status dsc_beamlet_dot(dsc_result* r, const float* g_dev, float* out_dev, void* stream) {
  if (!r || !g_dev || !out_dev) return fail(DSC_E_INVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaStreamWaitEvent(s, r->done, 0));
  const OutSlot& q = r->out->slot;
  k_beamlet_dot<<<row_blocks_grid(r->nrows), 256, 0, s>>>(q.row_ptr + r->rp_off, q.inst_begin + r->inst, q.col, q.val,
                                                         r->value_dtype, r->plan->d_rows, r->row_base, q.beam_scale,
                                                         g_dev, r->nrows, out_dev);
  CHECK_LAUNCH();
  return DSC_OK;
}

extern "C" dsc_status dsc_probe_tail(int32_t profile, const float* y_dev, int64_t n, float* ours_dev, float* cuda_dev,
                                     void* stream) {
  if (profile < 0 || profile > 2) return fail(DSC_E_INVAL, "profile: DSC_PROFILE_ERF, _LAPLACE or _LOGISTIC");
  if (n < 0 || (n > 0 && (!y_dev || !ours_dev || !cuda_dev))) return fail(DSC_E_INVAL, "null argument or n < 0");
  if (n == 0) return DSC_OK;
  const long long threads = (n + 3) / 4;
  k_tail_probe<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(profile, y_dev, n, ours_dev,
                                                                                    cuda_dev);
  CHECK_LAUNCH();
  return DSC_OK;
}

extern "C" dsc_status dsc_get_refine_counts(dsc_result* r, int64_t* near_threshold, int64_t* near_max,
                                            int64_t* fp32_decided) {
  if (!r || !near_threshold || !near_max) return fail(DSC_E_INVAL, "null argument");
  CU(cudaEventSynchronize(r->done));
  unsigned long long c[3] = {0, 0, 0};
  CU(cudaMemcpy(c, r->out->slot.refine, sizeof c, cudaMemcpyDeviceToHost));
  *near_threshold = (int64_t)c[0];
  *near_max = (int64_t)c[1];
  if (fp32_decided) *fp32_decided = (int64_t)c[2];
  return DSC_OK;
}

extern "C" dsc_status dsc_get_tile_counts(dsc_result* r, int64_t* tiles, int64_t* tiles_read) {
  if (!r || !tiles || !tiles_read) return fail(DSC_E_INVAL, "null argument");
  CU(cudaEventSynchronize(r->done));
  unsigned long long c[4] = {0, 0, 0, 0};
  CU(cudaMemcpy(c, r->out->slot.refine, sizeof c, cudaMemcpyDeviceToHost));
  *tiles = r->out->n_tiles;
  *tiles_read = (int64_t)c[3];
  return DSC_OK;
}

extern "C" dsc_status dsc_get_row_stats(dsc_result* r, float* row_max, int64_t* row_cand) {
  if (!r) return fail(DSC_E_INVAL, "null argument");
  CU(cudaEventSynchronize(r->done));
  if (row_max)
    CU(cudaMemcpy(row_max, r->out->slot.row_max + r->row_base, sizeof(float) * r->nrows, cudaMemcpyDeviceToHost));
  if (row_cand)
    CU(cudaMemcpy(row_cand, r->out->slot.row_cand + r->row_base, sizeof(long long) * r->nrows, cudaMemcpyDeviceToHost));
  return DSC_OK;
}

extern "C" dsc_status dsc_get_stage_times(dsc_result* r, float* ms, int32_t n) {
  if (!r || !ms || n < ST_N + 1) return fail(DSC_E_INVAL, "need n >= 8");
  if (!r->stage_ev) return fail(DSC_E_STATE, "computed without DSC_FLAG_TIMING");
  auto& ev = r->stage_ev->ev;
  CU(cudaEventSynchronize(ev[ST_N]));
  for (int i = 0; i < ST_N; ++i) CU(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
  CU(cudaEventElapsedTime(&ms[ST_N], ev[0], ev[ST_N]));
  return DSC_OK;
}

// ---------------------------------------------------------------------------
// serving: continuous batching with HBM-footprint admission
//
// A worker thread owns `max_inflight` device slots (streams).  Whenever a slot
// is free it admits queued requests in arrival order -- up to `max_batch`
// with identical options, while the summed footprint of admitted requests
// stays within the budget -- and launches them as one batched computation on
// that slot's stream, so requests that arrive while others run start as soon
// as a slot and memory free up, and their work overlaps on the device.  A
// request's footprint is charged from admission until its device work
// finishes; its scratch is released then, its CSR belongs to the caller.
// ---------------------------------------------------------------------------
namespace {
double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct SrvReq {
  uint64_t id = 0;
  dsc_geometry view;            // non-owning copy of the geometry with the request's beams
  dsc_compute_opts opts{};
  size_t footprint = 0;
  double t_submit = 0, t_done = 0;
  int state = 0;                // 0 queued, 1 running, 2 done, 3 failed
  dsc_status status = DSC_OK;
  std::string err;
  dsc_result* result = nullptr;
};

struct SrvSlot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;       // end of the slot's launch (timing enabled)
  cudaEvent_t ev_start = nullptr; // its start (timing enabled)
  bool busy = false;
  size_t footprint = 0;
  std::shared_ptr<Plan> plan;
  std::vector<std::shared_ptr<SrvReq>> reqs;
};

struct dsc_server {
  size_t budget = 0, used = 0;
  int max_inflight = 1, max_batch = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<SrvReq>> queue;
  std::map<uint64_t, std::shared_ptr<SrvReq>> reqs;
  std::vector<SrvSlot> slots;
  cudaEvent_t t0 = nullptr;     // the server's creation: origin of the slots' device intervals
  std::thread worker;
  bool stop = false;
  std::vector<double> lat_ms;
  long long n_done = 0, pairs_done = 0;
  uint64_t next_id = 1;
};

// Upper estimate of a request's device bytes: for every beamlet the VOI
// frustum over the grid's depth range, widened by one voxel diagonal, in
// voxels, times 12 bytes per candidate (value scratch + column + value),
// plus depth tables and per-row / per-item state.
static size_t estimate_footprint(const dsc_geometry& g, const dsc_compute_opts& o) {
  const dsc_grid_desc& G = g.grid;
  double vox = G.dx * G.dy * G.dz;
  double wd = std::sqrt(G.dx * G.dx + G.dy * G.dy + G.dz * G.dz);
  double diag = std::sqrt(std::pow(G.nx * G.dx, 2) + std::pow(G.ny * G.dy, 2) + std::pow(G.nz * G.dz, 2));
  double nvox = (double)G.nx * G.ny * G.nz;
  double h = o.h_frac * std::min(G.dx, std::min(G.dy, G.dz));
  double cx = G.origin[0] + 0.5 * G.nx * G.dx, cy = G.origin[1] + 0.5 * G.ny * G.dy, cz = G.origin[2] + 0.5 * G.nz * G.dz;
  double total = 0, rows = 0;
  for (const auto& b : g.beams) {
    double gr = b.gantry_deg * M_PI / 180.0;
    double S[3] = {b.iso[0] + b.sad * sin(gr), b.iso[1] - b.sad * cos(gr), b.iso[2]};
    double dist = std::sqrt(std::pow(cx - S[0], 2) + std::pow(cy - S[1], 2) + std::pow(cz - S[2], 2));
    double t0 = std::max(0.0, dist - 0.5 * diag), t1 = dist + 0.5 * diag;
    double kx, kz, bx, bz;
    if (g.cutoff_mode == 0) { kx = 3 * b.a / b.sad; kz = 3 * b.b / b.sad; bx = bz = 0; }
    else if (g.cutoff_mode == 1) { kx = 0.5 * b.a / b.sad; kz = 0.5 * b.b / b.sad; bx = bz = g.cutoff_k * g.c3max; }
    else { kx = kz = 0; bx = bz = 1e30; }
    // integral of (2(kx t + bx) + wd)(2(kz t + bz) + wd) dt
    double A = 2 * bx + wd, B = 2 * bz + wd;
    auto F = [&](double t) { return 4 * kx * kz * t * t * t / 3 + (2 * kx * B + 2 * kz * A) * t * t / 2 + A * B * t; };
    double per_row = std::min(nvox, (g.cutoff_mode == 2) ? nvox : (F(t1) - F(t0)) / vox);
    double n = (double)b.n_u * b.n_v;
    total += n * per_row;
    rows += n;
  }
  double bytes = total * 12.0 + rows * (diag / h + 2) * 4.0 + rows * 512.0 + (1 << 20);
  return (size_t)bytes;
}

static dsc_status fetch_pairs(dsc_result* r);

// options compared field by field (the struct has padding bytes)
static bool same_opts(const dsc_compute_opts& a, const dsc_compute_opts& b) {
  return a.rel_threshold == b.rel_threshold && a.value_dtype == b.value_dtype && a.h_frac == b.h_frac &&
         a.flags == b.flags;
}

static void srv_finish_slot(dsc_server* S, SrvSlot& sl) {
  double t = now_s();
  float ms0 = -1.0f, ms1 = -1.0f;
  if (cudaEventElapsedTime(&ms0, S->t0, sl.ev_start) != cudaSuccess ||
      cudaEventElapsedTime(&ms1, S->t0, sl.ev) != cudaSuccess)
    ms0 = ms1 = -1.0f;
  const int slot_index = (int)(&sl - S->slots.data());
  for (auto& q : sl.reqs) {
    if (q->result) {
      q->result->srv_slot = slot_index;
      q->result->srv_t0_ms = ms0;
      q->result->srv_t1_ms = ms1;
    }
    q->t_done = t;
    q->state = 2;
    S->lat_ms.push_back(1e3 * (t - q->t_submit));
    S->n_done++;
    if (q->result && fetch_pairs(q->result) == DSC_OK) S->pairs_done += q->result->pairs;
  }
  S->used -= sl.footprint;
  if (sl.plan) {
    std::lock_guard<std::mutex> lk(sl.plan->mu);
    sl.plan->free_scratch();
  }
  sl.plan.reset();
  sl.reqs.clear();
  sl.footprint = 0;
  sl.busy = false;
}

static void srv_loop(dsc_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progress = false;
    int busy = 0;
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      cudaError_t e = cudaEventQuery(sl.ev);
      if (e == cudaSuccess) {
        srv_finish_slot(S, sl);
        progress = true;
      } else if (e != cudaErrorNotReady) {
        for (auto& q : sl.reqs) { q->state = 3; q->status = DSC_E_CUDA; q->err = cudaGetErrorString(e); }
        S->used -= sl.footprint;
        sl.reqs.clear();
        sl.plan.reset();
        sl.busy = false;
        progress = true;
      } else {
        ++busy;
      }
    }
    if (S->stop && S->queue.empty() && busy == 0) break;
    // admission: fill free slots in arrival order
    for (auto& sl : S->slots) {
      if (sl.busy || S->queue.empty()) continue;
      std::vector<std::shared_ptr<SrvReq>> batch;
      size_t fp = 0;
      while (!S->queue.empty() && (int)batch.size() < S->max_batch) {
        auto& q = S->queue.front();
        if (!batch.empty() && !same_opts(q->opts, batch[0]->opts)) break;
        if (S->used + fp + q->footprint > S->budget) break;
        fp += q->footprint;
        batch.push_back(q);
        S->queue.pop_front();
      }
      if (batch.empty()) break;   // the head does not fit yet: wait for memory
      S->used += fp;
      for (auto& q : batch) q->state = 1;
      std::vector<dsc_geometry*> geoms;
      for (auto& q : batch) geoms.push_back(&q->view);
      std::vector<dsc_result*> outs(batch.size(), nullptr);
      lk.unlock();
      cudaEventRecord(sl.ev_start, sl.s);
      dsc_status st = compute_common(geoms.data(), (int)geoms.size(), &batch[0]->opts, sl.s, outs.data(), false);
      std::string err = st == DSC_OK ? "" : g_err;
      if (st == DSC_OK) cudaEventRecord(sl.ev, sl.s);
      lk.lock();
      progress = true;
      if (st != DSC_OK) {
        S->used -= fp;
        for (auto& q : batch) { q->state = 3; q->status = st; q->err = err; }
        continue;
      }
      sl.busy = true;
      sl.footprint = fp;
      sl.plan = outs[0]->plan;
      sl.reqs = batch;
      for (size_t k = 0; k < batch.size(); ++k) batch[k]->result = outs[k];
    }
    if (progress) {
      S->cv.notify_all();
      continue;
    }
    S->cv.wait_for(lk, std::chrono::microseconds(50));
  }
  S->cv.notify_all();
}

extern "C" dsc_status dsc_server_create(size_t hbm_budget_bytes, int32_t max_inflight, int32_t max_batch,
                                        dsc_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_inflight < 1 || max_batch < 1) return fail(DSC_E_INVAL, "bad argument");
  *out = nullptr;
  int dev;
  TRY(ensure_device(&dev));
  auto* S = new dsc_server();
  S->budget = hbm_budget_bytes;
  S->max_inflight = max_inflight;
  S->max_batch = max_batch;
  S->device = dev;
  S->slots.resize(max_inflight);
  for (auto& sl : S->slots) {
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.ev) != cudaSuccess || cudaEventCreate(&sl.ev_start) != cudaSuccess) {
      delete S;
      return fail(DSC_E_CUDA, "stream/event creation failed");
    }
  }
  if (cudaEventCreate(&S->t0) != cudaSuccess || cudaEventRecord(S->t0, S->slots[0].s) != cudaSuccess ||
      cudaEventSynchronize(S->t0) != cudaSuccess) {
    delete S;
    return fail(DSC_E_CUDA, "server reference event failed");
  }
  S->worker = std::thread(srv_loop, S);
  *out = S;
  return DSC_OK;
}

extern "C" dsc_status dsc_server_submit(dsc_server* S, dsc_geometry* geom, const dsc_beam_desc* beams, int32_t nbeams,
                                        const dsc_compute_opts* opts, uint64_t* req_id) {
  if (!S || !geom || !beams || nbeams < 1 || !req_id) return fail(DSC_E_INVAL, "null argument");
  TRY(check_opts(opts));
  auto q = std::make_shared<SrvReq>();
  q->view.id = g_geom_ids.fetch_add(1);
  q->view.device = geom->device;
  q->view.grid = geom->grid;
  q->view.n_lut = geom->n_lut;
  q->view.d_max = geom->d_max;
  for (int i = 0; i < 3; ++i) { q->view.c1[i] = geom->c1[i]; q->view.c2[i] = geom->c2[i]; }
  q->view.cutoff_mode = geom->cutoff_mode;
  q->view.cutoff_k = geom->cutoff_k;
  q->view.profile = geom->profile;
  q->view.c3max = geom->c3max;
  q->view.d_peak = geom->d_peak;
  q->view.d_rho = geom->d_rho;
  q->view.d_lut = geom->d_lut;
  q->view.d_lut_rows = geom->d_lut_rows;
  for (int i = 0; i < nbeams; ++i) {
    TRY(check_beam(geom, &beams[i]));
    q->view.beams.push_back(beams[i]);
  }
  q->opts = *opts;
  q->footprint = estimate_footprint(q->view, *opts);
  if (q->footprint > S->budget)
    return fail(DSC_E_NOMEM_BUDGET, "request needs ~%zu bytes, budget %zu", q->footprint, S->budget);
  q->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(DSC_E_STATE, "server stopping");
    q->id = S->next_id++;
    S->reqs[q->id] = q;
    S->queue.push_back(q);
  }
  S->cv.notify_all();
  *req_id = q->id;
  return DSC_OK;
}

extern "C" dsc_status dsc_server_poll(dsc_server* S, uint64_t id, int32_t wait_ms, dsc_result** out) {
  if (!S || !out) return fail(DSC_E_INVAL, "null argument");
  *out = nullptr;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(DSC_E_NOTFOUND, "unknown request %llu", (unsigned long long)id);
  auto q = it->second;
  auto ready = [&] { return q->state >= 2; };
  if (wait_ms < 0) S->cv.wait(lk, ready);
  else if (wait_ms > 0) S->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
  if (!ready()) return DSC_E_BUSY;
  S->reqs.erase(it);
  if (q->state == 3) return fail(q->status, "request %llu failed: %s", (unsigned long long)id, q->err.c_str());
  *out = q->result;
  q->result = nullptr;
  return DSC_OK;
}

extern "C" dsc_status dsc_server_stats(dsc_server* S, double* p50, double* p99, int64_t* n_done, int64_t* pairs_done) {
  if (!S) return fail(DSC_E_INVAL, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    size_t i = (size_t)std::ceil(p * v.size()) - 1;
    return v[std::min(i, v.size() - 1)];
  };
  if (p50) *p50 = pct(0.50);
  if (p99) *p99 = pct(0.99);
  if (n_done) *n_done = S->n_done;
  if (pairs_done) *pairs_done = S->pairs_done;
  return DSC_OK;
}

extern "C" void dsc_server_destroy(dsc_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& kv : S->reqs)
    if (kv.second->result) dsc_release_result(kv.second->result);
  for (auto& sl : S->slots) {
    if (sl.s) cudaStreamSynchronize(sl.s);
    sl.plan.reset();
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.ev_start) cudaEventDestroy(sl.ev_start);
    if (sl.s) cudaStreamDestroy(sl.s);
  }
  if (S->t0) cudaEventDestroy(S->t0);
  delete S;
}

extern "C" dsc_status dsc_get_server_timing(dsc_result* r, int32_t* slot, double* start_ms, double* end_ms) {
  if (!r || !slot || !start_ms || !end_ms) return fail(DSC_E_INVAL, "null argument");
  if (r->srv_slot < 0) return fail(DSC_E_STATE, "not a served result, or its device interval is unknown");
  *slot = r->srv_slot;
  *start_ms = r->srv_t0_ms;
  *end_ms = r->srv_t1_ms;
  return DSC_OK;
}

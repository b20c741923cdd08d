/*
 * dsc.h -- C ABI of libdsc, a GB300 (sm_103a) engine for IMRT dose-deposition
 * coefficients D_ij with a finite-size pencil beam (FSPB) model, after Gu et
 * al., "GPU-based ultra fast dose calculation using a finite pencil beam
 * model" (2009).
 *
 * The problem statement follows the paper: a CT density grid in the smallest
 * rectangular prism that holds the patient (Fig. 1), beams from point
 * sources (Section 2.2) divided into a x b beamlets (Section 2.1, Eq. 3), an
 * FSPB kernel D^p = A(theta, d) F(x', d, z', C) (Eq. 2) with the three-term
 * erf profile F (Eq. 3), and the output D_ij: the dose from beamlet i to voxel
 * j (Eq. 1).  Radiological depth d comes from a lookup table along each
 * beamlet axis built from the exact density integral (Siddon ray tracing,
 * Section 2.2) and interpolated linearly at the projection O' of the voxel
 * centre.  Only voxels inside the beamlet's volume of interest (VOI: a
 * co-axial beamlet with 6x the side, Section 2.1) are evaluated.  Entries
 * below a relative threshold of the row maximum are dropped and the rest is
 * compacted into CSR (rows = beamlets, columns = voxels).
 *
 * Conventions (units mm, angles degrees):
 *  - Density is FP32 [nz][ny][nx], x fastest.  grid.origin is the outer
 *    corner of voxel (0,0,0); voxel centres are origin + (i + 1/2) * spacing.
 *  - Beam frame: gantry g rotates about +z; source S = iso + SAD (sin g,
 *    -cos g, 0); broad-beam axis (iso - S)/SAD; u = (cos g, sin g, 0);
 *    v = (0, 0, 1).  Beamlet (iu, iv) is centred on the isocentre plane at
 *    iso + (iu + 1/2 - n_u/2) a u + (iv + 1/2 - n_v/2) b v; a, b are the
 *    beamlet sides at the isocentre plane and scale as t/SAD along the axis.
 *  - Row order: beams in dsc_add_beam order, then iv, then iu.  Column of
 *    voxel (ix, iy, iz) = ix + nx (iy + ny iz).  Columns ascend within a row.
 *  - A(theta, d) = T(d) (SAD/t)^2: T is the tabulated depth-dose, t the
 *    distance from S to O' along the beamlet axis.
 *
 * Errors: every entry point returns a dsc_status; no exception or signal
 * crosses the ABI.  dsc_last_error() returns a thread-local description of
 * the last failure on the calling thread.  Handles are not thread-safe
 * unless stated; distinct handles may be used from distinct threads.
 * Nothing in this library falls back to the CPU: with no usable CUDA device
 * every compute entry point fails with DSC_E_CUDA.
 */
#ifndef DSC_H
#define DSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSC_ABI_VERSION 3

typedef enum {
    DSC_OK = 0,
    DSC_E_INVAL = 1,         /* bad argument: null pointer, size <= 0, source inside the grid, ... */
    DSC_E_NOMEM = 2,         /* a device or pinned-host allocation failed */
    DSC_E_NOMEM_BUDGET = 3,  /* a request's HBM footprint exceeds the server budget */
    DSC_E_CUDA = 4,          /* CUDA runtime error; text in dsc_last_error() */
    DSC_E_TIMEOUT = 5,       /* a bounded device-side wait expired (status word set by a kernel) */
    DSC_E_STATE = 6,         /* call not valid in the handle's current state */
    DSC_E_NOTFOUND = 7,      /* unknown request id */
    DSC_E_BUSY = 8,          /* result not ready (non-blocking poll) */
    DSC_W_INEXACT = 9        /* completed, outputs valid, but some keep decisions within 1e-5 of the
                              * threshold were taken in FP32 (more such pairs than the FP64 list holds);
                              * only dsc_compute_dij_noalloc returns it */
} dsc_status;

typedef struct dsc_geometry dsc_geometry;   /* device-resident density + beam model + beam list */
typedef struct dsc_result dsc_result;       /* device-resident CSR D_ij and per-row statistics */
typedef struct dsc_server dsc_server;       /* continuous-batching request server */

/* CT grid (Fig. 1: the smallest prism that holds the CT). */
typedef struct {
    int32_t nx, ny, nz;      /* voxels per axis, each >= 1; nx*ny*nz < 2^31 */
    double dx, dy, dz;       /* voxel sides, > 0 */
    double origin[3];        /* outer corner of voxel (0,0,0) */
} dsc_grid_desc;

/* Lateral cutoff: which voxels of a beamlet are evaluated at all. */
enum {
    DSC_CUTOFF_VOI6 = 0,     /* |x'| <= 3 a_t and |z'| <= 3 b_t: VOI of 6x the side (Section 2.1) */
    DSC_CUTOFF_SIGMA = 1,    /* |x'| <= a_t/2 + k c3_1(d), same in z' */
    DSC_CUTOFF_NONE = 2      /* every voxel in front of the source */
};

/* Lateral profile F of Eq. 2.  Section 2.1 admits any FSPB kernel that keeps
 * the self-consistency and normalisation conditions; each profile here is the
 * beamlet's box convolved per axis with a spread kernel whose standard
 * deviation is c3_i(d):  F = sum_i c1_i P_x P_z with
 * P(x) = G((|x| - h)/s) - G((|x| + h)/s), h = c2_i a_t / 2, G the kernel's
 * complementary distribution function. */
enum {
    DSC_PROFILE_ERF = 0,      /* Gaussian kernel: Eq. 3 (Jiang's three erf terms) */
    DSC_PROFILE_LAPLACE = 1,  /* exponential (Laplace) kernel, s = c3 / sqrt 2 */
    DSC_PROFILE_LOGISTIC = 2  /* logistic kernel, G = Boltzmann function 1/(1 + e^y), s = c3 sqrt 3 / pi */
};

/* FSPB beam model (Eq. 2-3).  table4 holds n rows {T(d), c3_1(d), c3_2(d),
 * c3_3(d)} at n equally spaced depths on [0, d_max]; values are interpolated
 * linearly and clamped to the last row beyond d_max.  c1, c2 are the
 * depth-independent weights and width factors of the three terms.  The
 * table is copied; the caller keeps ownership of table4.  DSC_E_INVAL unless
 * every c3 is finite and > 0 and every T finite. */
typedef struct {
    int32_t n;               /* 2 <= n <= 4096 */
    double d_max;            /* > 0 */
    const float* table4;     /* host pointer, n*4 floats */
    double c1[3];
    double c2[3];
    int32_t cutoff_mode;     /* DSC_CUTOFF_* */
    double cutoff_k;         /* k of DSC_CUTOFF_SIGMA */
    int32_t profile;         /* DSC_PROFILE_* */
} dsc_fspb_model;

/* One broad beam from a point source, divided into n_u x n_v beamlets. */
typedef struct {
    double gantry_deg;
    double sad;              /* source-axis distance, > 0; the source must lie outside the grid */
    double iso[3];           /* isocentre */
    double a, b;             /* beamlet sides at the isocentre plane (along u and v), > 0 */
    int32_t n_u, n_v;        /* >= 1 */
} dsc_beam_desc;

enum { DSC_VALUE_F32 = 0, DSC_VALUE_BF16 = 1 };
enum {
    DSC_FLAG_TIMING = 1,     /* record CUDA events around each stage (dsc_get_stage_times) */
    /* depth table as the paper builds it (Section 2.2): density sampled by
     * trilinear interpolation of the voxel centres (clamped to the edge) at
     * the table points, accumulated by the trapezoid rule.  Default: the
     * exact integral of the piecewise-constant density (Siddon). */
    DSC_FLAG_TRILINEAR_TABLE = 2
};

typedef struct {
    double rel_threshold;    /* keep D_ij > 0 with D_ij >= rel_threshold * max_j' D_ij' (row max); >= 0.
                              * Values are FP32; a value within 1e-5 (relative) of its threshold, and the
                              * row maximum it is compared with, are evaluated again in FP64 and decided
                              * there (dsc_get_refine_counts), so every decision farther than about 1e-6
                              * from the threshold is the one exact arithmetic makes. */
    int32_t value_dtype;     /* DSC_VALUE_F32, or DSC_VALUE_BF16: value / beam_scale[beam] rounded to bf16 */
    double h_frac;           /* depth-table spacing / min voxel side, (0, 1]; the paper uses 1/2 */
    int32_t flags;           /* DSC_FLAG_* */
} dsc_compute_opts;

/* A view of a result's CSR.  On-device pointers stay valid until
 * dsc_release_result; host pointers (copy_to_host = 1) are owned by the
 * result.  val is float (DSC_VALUE_F32) or bf16 bits (uint16_t, DSC_VALUE_BF16);
 * with bf16, D_ij = bf16_to_float(val) * beam_scale[beam of the row]. */
typedef struct {
    int64_t nrows, ncols, nnz;
    const int64_t* row_ptr;  /* nrows + 1 */
    const int32_t* col;      /* nnz */
    const void* val;         /* nnz */
    int32_t value_dtype;
    int32_t nbeams;
    const float* beam_scale; /* nbeams (1.0 for DSC_VALUE_F32) */
    int64_t pairs;           /* voxel-beamlet pairs evaluated (inside the lateral cutoff) */
    int32_t on_device;
} dsc_csr_view;

/* --- library ------------------------------------------------------------ */
const char* dsc_status_str(dsc_status s);
const char* dsc_last_error(void);
int32_t dsc_abi_version(void);
/* kernels this library has launched in this process (for launch accounting) */
int64_t dsc_launch_count(void);

/* --- geometry (Fig. 1, Section 2.2) -------------------------------------- */
/* Copies the grid, density and model to the current device on `stream`
 * (a cudaStream_t, NULL = legacy default stream).  density is a host pointer
 * (density_on_device = 0) or a device pointer read stream-ordered (= 1).  The
 * geometry starts with no beams. */
dsc_status dsc_create_geometry(const dsc_grid_desc* grid, const float* density, int32_t density_on_device,
                               const dsc_fspb_model* model, void* stream, dsc_geometry** out);
/* Replaces the density (same grid) -- a new CT of the same patient set-up. */
dsc_status dsc_upload_density(dsc_geometry* geom, const float* density, int32_t density_on_device, void* stream);
/* Appends a beam; its rows follow the rows of the beams added before it. */
dsc_status dsc_add_beam(dsc_geometry* geom, const dsc_beam_desc* beam, int32_t* beam_index_out);
dsc_status dsc_clear_beams(dsc_geometry* geom);
/* Frees the geometry after all work queued on it has finished. */
void dsc_destroy_geometry(dsc_geometry* geom);

/* --- computation --------------------------------------------------------- */
/* D_ij of every beamlet of every beam of `geom` (Eq. 1-3).  All work is
 * queued on `stream`; the call returns without waiting except for one
 * stream-ordered read of the total candidate count the first time a
 * geometry/beam set is planned.  The result is usable on `stream` at once;
 * host views need dsc_get_csr, which waits. */
dsc_status dsc_compute_dij(dsc_geometry* geom, const dsc_compute_opts* opts, void* stream, dsc_result** out);
/* Many independent geometries (re-plan instances) in one launch sequence:
 * each kernel stage runs once over all instances, the evaluation is one
 * persistent kernel over a shared work queue, and the sequence is captured
 * in a CUDA graph that is replayed while the set of geometries, their beams
 * and the options stay the same.  outs[k] receives instance k's result. */
dsc_status dsc_compute_dij_batch(dsc_geometry* const* geoms, int32_t n, const dsc_compute_opts* opts,
                                 void* stream, dsc_result** outs);
/* --- work decomposition ("tile shape") and its autotuner ---------------- */
/* The evaluation walks work items of about target_cand candidate pairs (a
 * chunk of one beamlet's x-lines, at most 512 lines) taken from a queue by a
 * persistent kernel of eval_blocks_per_sm CTAs per SM.  The result does not
 * depend on either value, only the time does.  Process-wide; a plan reads the
 * setting when it is built (plans already cached keep theirs). */
typedef struct {
    int32_t target_cand;         /* 512 .. 65536; default 8192 */
    int32_t eval_blocks_per_sm;  /* 0 = the occupancy limit (default), else 1 .. that limit */
} dsc_tuning;
/* DSC_E_INVAL outside the ranges above. */
dsc_status dsc_set_tuning(const dsc_tuning* t);
dsc_status dsc_get_tuning(dsc_tuning* t);
/* Times every tile shape of a fixed set (target_cand 2048 .. 32768 by powers
 * of two x eval_blocks_per_sm {limit, 3/4 limit, 1/2 limit}) on the caller's
 * geometries: per shape a fresh plan, one warm-up, then `reps` (1 .. 100)
 * replays of the batched computation, each timed with CUDA events on
 * `stream`.  Installs the shape with the lowest median time (dsc_set_tuning),
 * and returns it and that median in milliseconds (best_ms may be NULL).
 * Blocks until done; the plans it builds are not cached and the results are
 * released.  geoms as for dsc_compute_dij_batch. */
dsc_status dsc_autotune(dsc_geometry* const* geoms, int32_t n, const dsc_compute_opts* opts, void* stream,
                        int32_t reps, dsc_tuning* best, float* best_ms);

/* Blocks until the result's device work has finished; returns DSC_E_TIMEOUT
 * if a bounded device wait expired, DSC_E_CUDA on a device error. */
dsc_status dsc_result_wait(dsc_result* res);
/* copy_to_host = 0: device view (waits only for nnz); 1: copies to
 * result-owned pinned host buffers and waits. */
dsc_status dsc_get_csr(dsc_result* res, int32_t copy_to_host, dsc_csr_view* out);
/* Copies the CSR into caller-provided host buffers (ideally pinned) on
 * `stream` and waits for the copy.  Sizes come from dsc_get_csr(res, 0, ...):
 * row_ptr nrows+1, col nnz, val nnz * (4 or 2) bytes, beam_scale nbeams (may be NULL). */
dsc_status dsc_copy_csr_to_host(dsc_result* res, int64_t* row_ptr, int32_t* col, void* val, float* beam_scale,
                                void* stream);
/* The same copies, queued on `stream` without waiting for them: the call
 * waits on the host for the computation to finish (its counts size the
 * copies), queues the copies and returns.  The host buffers hold the CSR once
 * `stream` has passed the copies (synchronise it or an event recorded after
 * the call); with pinned buffers the copies overlap other work, so the read-back
 * of one result can be queued behind another's.  The result's device buffers
 * are kept until the copies have run, also when the result is released before
 * that.  Errors as for dsc_copy_csr_to_host. */
dsc_status dsc_copy_csr_to_host_async(dsc_result* res, int64_t* row_ptr, int32_t* col, void* val, float* beam_scale,
                                      void* stream);
void dsc_release_result(dsc_result* res);

/* --- products with the resident D_ij (no copy to the host) -------------- */
/* Eq. 1 (Section 2.1): dose[v] = sum_j w[j] D_jv over the result's rows j
 * (its beamlets; one instance of a batch), for every voxel v of its grid.
 * w_dev: nrows floats, dose_dev: ncols floats (voxel order ix + nx (iy + ny
 * iz)), both device pointers, caller-owned.  Queued on `stream` after the
 * computation; the call does not wait.  Each product w_j D_jv is rounded to
 * FP32 and summed exactly in 64-bit fixed point scaled to a bound on |dose|,
 * so the result does not depend on thread order (bit-identical across
 * calls); relative error at most 2^-24 per term plus one final FP32
 * rounding.  BF16 results use D_jv = bf16 value x beam_scale.  Scratch: 8
 * bytes per voxel for the call. */
dsc_status dsc_dose(dsc_result* res, const float* w_dev, float* dose_dev, void* stream);
/* out[j] = sum_v D_jv g[v] for every row j (the product with the transpose
 * of Eq. 1's operator, which an optimiser's gradient needs).  g_dev: ncols
 * floats, out_dev: nrows floats, device pointers; FP64 sums per row in a fixed
 * order, queued on `stream`. */
dsc_status dsc_beamlet_dot(dsc_result* res, const float* g_dev, float* out_dev, void* stream);

/* --- arithmetic rates of this GPU ---------------------------------------- */
/* The denominators of the evaluation kernel's roofline, measured: every SM
 * filled with independent dependency chains of one operation, timed with CUDA
 * events on `stream` over one launch of about ms_per_loop milliseconds (1 to
 * 2000) after an untimed one, so that the clocks settle where a long run
 * holds them.  out[0] = FP32 TFLOP/s of fused multiply-adds (2 flops each),
 * out[1] = ex2.approx.ftz.f32 and out[2] = rcp.approx.ftz.f32 in 10^12
 * operations/s (the MUFU unit), out[3..5] = device ms of the three timed
 * launches; n >= 6.  Waits for the stream.  DSC_E_INVAL for a short `out` or
 * ms_per_loop out of range. */
dsc_status dsc_measure_alu_peaks(double ms_per_loop, double* out, int32_t n, void* stream);
/* The host link's rate in each direction, which bounds the end-to-end path
 * (a step's density up, its CSR down): `bytes` (1 MiB to 8 GiB) copied with
 * cudaMemcpyAsync between a device buffer and a pinned host buffer, both
 * allocated by the call and freed before it returns, on `stream`; one untimed
 * copy each way, then the shortest of `reps` (1 to 100) copies, timed with
 * CUDA events.  out[0] = device-to-host GB/s (10^9 bytes/s), out[1] =
 * host-to-device GB/s, out[2], out[3] = their ms; n >= 4.  Waits for the
 * stream.  DSC_E_INVAL for a short `out` or an argument out of range,
 * DSC_E_NOMEM when a buffer cannot be allocated.  Not part of the paper:
 * a measurement of this machine. */
dsc_status dsc_measure_host_link(int64_t bytes, int32_t reps, double* out, int32_t n, void* stream);

/* --- stage inspection (per-step parity and timing) ---------------------- */
/* The lateral-profile tail T(y) = 2 G(y) of Eq. 3 (profile DSC_PROFILE_ERF:
 * erfc(y / sqrt 2)) or of the other profiles (DSC_PROFILE_LAPLACE:
 * exp(-sqrt 2 y); DSC_PROFILE_LOGISTIC: 2 q / (1 + q), q = exp(-pi y / sqrt 3)),
 * y >= 0 in units of the spread c3, computed with the evaluation kernel's own
 * primitives and constants, and the same tail from CUDA's erfcf / expf for
 * comparison.  y_dev, ours_dev, cuda_dev: n floats each, device pointers;
 * queued on `stream`.  DSC_E_INVAL for an unknown profile or a null pointer
 * with n > 0. */
dsc_status dsc_probe_tail(int32_t profile, const float* y_dev, int64_t n, float* ours_dev, float* cuda_dev,
                          void* stream);
/* Per row 16 doubles: S[3] e[3] x'[3] z'[3] tA tB hit n_table. */
dsc_status dsc_get_beamlets(dsc_result* res, double* out, int64_t cap_rows);
/* Depth tables, row-major [nrows][n_max] floats (entries past a row's n_table are 0). */
dsc_status dsc_get_depth_tables(dsc_result* res, float* out, int64_t cap, int32_t* n_max_out);
/* Pairs of the computation (all instances of its launch) whose decision the
 * FP32 values could not settle and that were evaluated again in FP64: values
 * within 1e-5 (relative) of their row's threshold (the keep decision), and
 * within 1e-5 of their row's maximum (the maximum itself; a row with more
 * than 4 of them is scanned in full for its FP64 maximum).  fp32_decided
 * (may be NULL): pairs within 1e-5 of their threshold beyond the FP64 list's
 * capacity (at least 65536 and n_cand / 1024), whose decision stayed FP32;
 * 0 means every decision farther than about 1e-6 from the threshold is the
 * one exact arithmetic makes. */
dsc_status dsc_get_refine_counts(dsc_result* res, int64_t* near_threshold, int64_t* near_max,
                                 int64_t* fp32_decided);
/* Compaction tiles of the computation (all instances of its launch; 128
 * candidate slots each, work items padded to whole tiles), and those whose
 * values the count pass read.  The others took the count the evaluation
 * formed against a lower bound of their row maximum (the running maximum
 * when their work item started, seeded from the voxels by the beamlet axis),
 * which is the tile's exact count whenever the final threshold lies within
 * 2^-16 of that bound's and no value of the tile lies near either; a tile
 * read or not gives the same CSR. */
dsc_status dsc_get_tile_counts(dsc_result* res, int64_t* tiles, int64_t* tiles_read);
/* Per row: max D over the row's candidates and the candidate count. */
dsc_status dsc_get_row_stats(dsc_result* res, float* row_max, int64_t* row_cand);
/* Milliseconds per stage (needs DSC_FLAG_TIMING): [set-up + item scan, Siddon
 * tables, candidate count + scan, evaluation, beam scale, compaction, row
 * pointers + statistics, total]. n >= 8. */
dsc_status dsc_get_stage_times(dsc_result* res, float* ms, int32_t n);

/* --- serving: continuous batching of re-plan requests -------------------- */
/* hbm_budget_bytes: cap on the summed device footprint of admitted requests;
 * max_inflight: concurrent device slots (streams); max_batch: requests fused
 * into one batched launch. */
dsc_status dsc_server_create(size_t hbm_budget_bytes, int32_t max_inflight, int32_t max_batch, dsc_server** out);
/* Queues D_ij for `geom` with an explicit beam set (the geometry's own beam
 * list is not used).  Never blocks; DSC_E_NOMEM_BUDGET if the request could
 * never fit the budget.  The geometry (its density and model table) must
 * stay alive until the request has been polled. */
dsc_status dsc_server_submit(dsc_server* srv, dsc_geometry* geom, const dsc_beam_desc* beams, int32_t nbeams,
                             const dsc_compute_opts* opts, uint64_t* req_id);
/* Waits up to wait_ms (0 = do not wait, < 0 = forever) for request req_id;
 * on DSC_OK *out is the caller's to release.  DSC_E_BUSY if not finished. */
dsc_status dsc_server_poll(dsc_server* srv, uint64_t req_id, int32_t wait_ms, dsc_result** out);
/* Latency (submit -> device completion) statistics in ms over finished requests. */
dsc_status dsc_server_stats(dsc_server* srv, double* p50_ms, double* p99_ms, int64_t* n_done, int64_t* pairs_done);
/* Drains queued work, then frees the server. */
void dsc_server_destroy(dsc_server* srv);
/* For a result returned by dsc_server_poll: the device slot (stream) that
 * computed it and the device interval of that slot's launch (the request's
 * batch), in ms after the server's creation, from CUDA events recorded on the
 * slot's stream around the launch.  Two requests whose intervals intersect
 * had their work on the GPU at the same time.  DSC_E_STATE for a result that
 * did not come from a server. */
dsc_status dsc_get_server_timing(dsc_result* res, int32_t* slot, double* start_ms, double* end_ms);

/* --- computation without allocation -------------------------------------- */
/* dsc_compute_dij without any memory allocation by the library, for callers
 * that must not allocate device memory while they run (loops that reserve
 * every byte before treatment starts, processes held to a fixed GPU memory
 * quota, code running where cudaMalloc is not allowed).  This entry point has
 * no counterpart in the paper; it is the same computation and the same
 * kernels as dsc_compute_dij for one geometry, FP32 values only.
 *
 * Inputs: grid, density_dev (device pointer, FP32 [nz][ny][nx]), model (its
 * table4 on the host), beams[nbeams] (host), opts (value_dtype must be
 * DSC_VALUE_F32).  Outputs, caller-allocated device buffers: row_ptr_dev
 * (nrows + 1 int64), col_dev and val_dev (capacity entries each).  On
 * DSC_OK, *nnz_out holds the number of kept entries and the CSR is complete
 * (the call waits for its work on `stream`).
 *
 * Working memory is a fixed array of 80 MiB inside the library's device
 * image, present on every GPU that loads the library until the process
 * exits.  A request whose working set (set-up, depth tables, line tables,
 * work items, 8 bytes per candidate pair and 32 bytes per tile of 128
 * candidates) exceeds it fails with DSC_E_INVAL and says so in
 * dsc_last_error(); so does an output capacity below the kept count
 * (nothing is written to the outputs then).  The first call on a device
 * looks up the array's device address (kept for the life of the process: do
 * not use the library across a reset of the device's primary context); make
 * that first call before any stream capture.  The call waits for its own
 * work: it synchronises `stream` several times, and on every return, error
 * or not, no work of its own is left on the GPU.  Every call reuses the
 * array from the start: calls whose device work overlapped would race, so
 * the library runs one call at a time per process (a second host thread
 * waits for the first call to return).  The call allocates no
 * device or host memory.  DSC_W_INEXACT: the CSR is complete and valid, but
 * some keep decisions within 1e-5 of the threshold stayed FP32 (how many is
 * in dsc_last_error()). */
dsc_status dsc_compute_dij_noalloc(const dsc_grid_desc* grid, const float* density_dev, const dsc_fspb_model* model,
                                   const dsc_beam_desc* beams, int32_t nbeams, const dsc_compute_opts* opts,
                                   int64_t* row_ptr_dev, int32_t* col_dev, float* val_dev, int64_t capacity,
                                   int64_t* nnz_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DSC_H */

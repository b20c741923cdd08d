// dsc_peaks.cu -- arithmetic rates of this GPU for the evaluation kernel's
// roofline: FP32 fused multiply-adds and the two MUFU operations the FSPB
// evaluation issues (ex2.approx for the Gaussian factor of erfc, rcp.approx
// for t = 1/(1 + p x), 1/s and 1/t).
//
// Each thread runs kChains independent dependency chains, every SM is filled
// (8 CTAs of 256 threads), and one loop takes long enough that the clocks
// settle where a long run holds them.  The chains stay bounded (FMA:
// a <- 0.9999 a + 1e-4 tends to 1; ex2: a <- 2^-a stays in [0.5, 1]; rcp:
// a <- 1/a + 1/4 tends to 1.13, the FMA keeping the compiler from folding
// two reciprocals into the identity), and their sum, which is never
// negative, decides a store the compiler cannot remove.
#include "dsc.h"
#include "dsc_internal.h"

#include <algorithm>
#include <cstdio>

namespace dsc {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;
constexpr int kInner = 16;   // chain steps per loop trip, unrolled

__device__ __forceinline__ float peak_ex2(float x) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float peak_rcp(float x) {
  float r;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// OP 0: FMA, 1: ex2, 2: rcp; kChains * kInner * iters operations per thread
template <int OP>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float b, float c, float* __restrict__ sink) {
  float a[kChains];
#pragma unroll
  for (int u = 0; u < kChains; ++u) a[u] = 0.75f + 0.01f * (float)u + 1e-6f * (float)(threadIdx.x & 63);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < kInner; ++r) {
#pragma unroll
      for (int u = 0; u < kChains; ++u) {
        if (OP == 0) a[u] = fmaf(a[u], b, c);
        else if (OP == 1) a[u] = peak_ex2(-a[u]);
        else a[u] = fmaf(peak_rcp(a[u]), b, c);   // an FMA between steps: rcp(rcp(a)) may fold to a
      }
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int u = 0; u < kChains; ++u) s += a[u];
  if (s < 0.0f) sink[0] = s;   // never taken: every chain stays positive
}

namespace {

dsc_status peak_fail(dsc_status st, const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "dsc_measure_alu_peaks: %s%s%s", what, e != cudaSuccess ? ": " : "",
           e != cudaSuccess ? cudaGetErrorString(e) : "");
  set_error(buf);
  return st;
}

cudaError_t peak_launch(int op, int blocks, int iters, cudaStream_t s, float* sink) {
  count_launches(1);
  if (op == 0) k_peak<0><<<blocks, kPeakThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
  else if (op == 1) k_peak<1><<<blocks, kPeakThreads, 0, s>>>(iters, 0.0f, 0.0f, sink);
  else k_peak<2><<<blocks, kPeakThreads, 0, s>>>(iters, 1.0f, 0.25f, sink);
  return cudaGetLastError();
}

// device ms of one launch
cudaError_t peak_time(int op, int blocks, int iters, cudaStream_t s, float* sink, cudaEvent_t e0, cudaEvent_t e1,
                      float* ms) {
  cudaError_t e;
  if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
  if ((e = peak_launch(op, blocks, iters, s, sink)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
  if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
  return cudaEventElapsedTime(ms, e0, e1);
}

}  // namespace
}  // namespace dsc

extern "C" dsc_status dsc_measure_alu_peaks(double ms_per_loop, double* out, int32_t n, void* stream) {
  using namespace dsc;
  if (!out || n < 6) return peak_fail(DSC_E_INVAL, "out needs 6 entries", cudaSuccess);
  if (!(ms_per_loop >= 1.0 && ms_per_loop <= 2000.0))
    return peak_fail(DSC_E_INVAL, "ms_per_loop outside [1, 2000]", cudaSuccess);
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, tpm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&tpm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess)
    return peak_fail(DSC_E_CUDA, "device query", e);
  const int blocks = sms * std::max(1, tpm / kPeakThreads);
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaMallocAsync(&sink, sizeof(float), s)) != cudaSuccess) return peak_fail(DSC_E_NOMEM, "sink", e);
  dsc_status st = DSC_OK;
  const char* what = "";
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = DSC_E_CUDA;
    what = "event";
  }
  for (int op = 0; op < 3 && st == DSC_OK; ++op) {
    // probes grow 8x until one takes 2 ms, which sizes the long launch; the
    // long launch runs once untimed, then once timed
    int probe = 64;
    float ms = 0.0f;
    for (int k = 0; k < 8; ++k, probe *= 8) {
      if ((e = peak_time(op, blocks, probe, s, sink, e0, e1, &ms)) != cudaSuccess) break;
      if (ms >= 2.0f || probe >= (1 << 21)) break;
    }
    if (e != cudaSuccess) {
      st = DSC_E_CUDA;
      what = "probe launch";
      break;
    }
    const double scaled = probe * ms_per_loop / std::max(1e-3, (double)ms);
    const int iters = (int)std::min({std::max(scaled, 1.0), 1000.0 * probe, (double)(1 << 24)});
    if ((e = peak_launch(op, blocks, iters, s, sink)) != cudaSuccess ||
        (e = peak_time(op, blocks, iters, s, sink, e0, e1, &ms)) != cudaSuccess) {
      st = DSC_E_CUDA;
      what = "timed launch";
      break;
    }
    const double ops = (double)blocks * kPeakThreads * kChains * kInner * (double)iters * (op == 0 ? 2.0 : 1.0);
    out[op] = ops / (ms * 1e-3) / 1e12;
    out[3 + op] = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  const cudaError_t ef = cudaFreeAsync(sink, s);
  if (st != DSC_OK) return peak_fail(st, what, e);
  if (ef != cudaSuccess) return peak_fail(DSC_E_CUDA, "free", ef);
  return DSC_OK;
}

// ---------------------------------------------------------------------------
// host-link bandwidth: the end-to-end path moves each step's density up and
// its CSR down, so its bound is the link's rate in each direction
// ---------------------------------------------------------------------------
namespace {
dsc_status link_fail(dsc_status st, const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "dsc_measure_host_link: %s%s%s", what, e != cudaSuccess ? ": " : "",
           e != cudaSuccess ? cudaGetErrorString(e) : "");
  dsc::set_error(buf);
  return st;
}
}  // namespace

extern "C" dsc_status dsc_measure_host_link(int64_t bytes, int32_t reps, double* out, int32_t n, void* stream) {
  if (!out || n < 4) return link_fail(DSC_E_INVAL, "out needs 4 entries", cudaSuccess);
  if (bytes < (1 << 20) || bytes > (8ll << 30)) return link_fail(DSC_E_INVAL, "bytes outside [1 MiB, 8 GiB]", cudaSuccess);
  if (reps < 1 || reps > 100) return link_fail(DSC_E_INVAL, "reps outside [1, 100]", cudaSuccess);
  cudaStream_t s = (cudaStream_t)stream;
  void* d = nullptr;
  void* h = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMallocAsync(&d, (size_t)bytes, s);
  if (e != cudaSuccess) return link_fail(DSC_E_NOMEM, "device buffer", e);
  dsc_status st = DSC_OK;
  const char* what = "";
  if ((e = cudaHostAlloc(&h, (size_t)bytes, cudaHostAllocDefault)) != cudaSuccess) {
    st = DSC_E_NOMEM;
    what = "pinned host buffer";
  } else if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
             (e = cudaMemsetAsync(d, 0, (size_t)bytes, s)) != cudaSuccess) {
    st = DSC_E_CUDA;
    what = "set-up";
  }
  // best of `reps` copies each way, after one untimed copy each way
  float best[2] = {0.0f, 0.0f};
  for (int dir = 0; dir < 2 && st == DSC_OK; ++dir) {
    for (int r = 0; r <= reps && st == DSC_OK; ++r) {
      float ms = 0.0f;
      if ((e = cudaEventRecord(e0, s)) != cudaSuccess ||
          (e = dir == 0 ? cudaMemcpyAsync(h, d, (size_t)bytes, cudaMemcpyDeviceToHost, s)
                        : cudaMemcpyAsync(d, h, (size_t)bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
          (e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        st = DSC_E_CUDA;
        what = "timed copy";
      } else if (r > 0 && (best[dir] == 0.0f || ms < best[dir])) {
        best[dir] = ms;
      }
    }
  }
  if (st == DSC_OK) {
    for (int dir = 0; dir < 2; ++dir) {
      out[dir] = (double)bytes / (best[dir] * 1e-3) / 1e9;
      out[2 + dir] = best[dir];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  const cudaError_t ef = cudaFreeAsync(d, s);
  const cudaError_t es = cudaStreamSynchronize(s);
  if (h) cudaFreeHost(h);
  if (st != DSC_OK) return link_fail(st, what, e);
  if (ef != cudaSuccess || es != cudaSuccess) return link_fail(DSC_E_CUDA, "free", ef != cudaSuccess ? ef : es);
  return DSC_OK;
}

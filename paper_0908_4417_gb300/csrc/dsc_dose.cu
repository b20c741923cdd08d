// dsc_dose.cu -- products with the resident D_ij (Eq. 1 and its transpose).
//
//   dose(v)  = sum_j w_j D_jv       (Eq. 1: dose superposition over beamlets)
//   out(j)   = sum_v D_jv g(v)      (the transpose product an optimiser's
//                                    gradient needs)
//
// Both read one instance's CSR where the computation left it (rows = the
// instance's beamlets, columns = voxel indices).  FP64 arithmetic is slow on
// this GPU, so no per-entry step uses it.  The dose is a scatter over rows:
// every product w_j D_jv is rounded once to FP32, converted exactly (integer
// shifts of its mantissa) to 64-bit fixed point at a power-of-two scale
// chosen from a bound on |dose|, and added with integer atomics, so the sum
// does not depend on the order the atomics land in (deterministic; each term
// within 2^-24 of its exact product, the sum rounded once to FP32).  The transpose product is a gather per
// row, one warp per row, compensated FP32 sums per lane reduced in FP64 in
// a fixed order.
#include "dsc_internal.h"

#include <cuda_bf16.h>

namespace dsc {

constexpr int kRowThreads = 256;   // threads per row of the products

namespace {
// the stored D_jv as FP32 (BF16 values times the beam's scale, rounded once)
__device__ __forceinline__ float entry_value(const void* val, int dtype, long long k, float scale) {
  if (dtype == 1) return __bfloat162float(((const __nv_bfloat16*)val)[k]) * scale;
  return ((const float*)val)[k];
}

// x * 2^e rounded to a 64-bit integer (ties away from zero), from the FP32
// bits with integer operations only; |x| 2^e < 2^62 by the choice of e
__device__ __forceinline__ long long fixed_of(float x, int e) {
  const unsigned b = __float_as_uint(x);
  const int E = (int)((b >> 23) & 0xffu);
  if (E == 0 && (b & 0x7fffffu) == 0) return 0;
  const long long m = (long long)((b & 0x7fffffu) | (E ? 0x800000u : 0u));
  const int sh = (E ? E : 1) - 150 + e;           // x = m 2^((E ? E : 1) - 150)
  long long q;
  if (sh >= 0) q = m << sh;
  else if (sh > -40) q = (m + (1ll << (-sh - 1))) >> -sh;
  else q = 0;
  return (b >> 31) ? -q : q;
}
}  // namespace

// bound on |dose| (sum_j |w_j| * row max_j; stored values never exceed the row
// maximum by more than the BF16 rounding) and the fixed-point exponent e with
// bound * 2^e < 2^61; one block, fixed reduction order
__global__ void __launch_bounds__(1024) k_dose_scale(const unsigned* __restrict__ row_max, const float* __restrict__ w,
                                                     int nrows, int* exp_out) {
  __shared__ double part[1024];
  double s = 0.0;
  for (int j = threadIdx.x; j < nrows; j += blockDim.x) s += fabs((double)w[j]) * (double)__uint_as_float(row_max[j]);
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double b = part[0] * 1.01;
    *exp_out = b > 0.0 ? 60 - ilogb(b) : 0;
  }
}

// one block per row (grid-stride over rows), four entries in flight per thread
__global__ void __launch_bounds__(kRowThreads) k_dose_scatter(
    const long long* __restrict__ row_ptr, const long long* __restrict__ inst_begin, const int* __restrict__ col,
    const void* __restrict__ val, int dtype, const DRow* __restrict__ rows, int row_base,
    const float* __restrict__ beam_scale, const float* __restrict__ w, int nrows, const int* __restrict__ exp_in,
    unsigned long long* __restrict__ acc) {
  const long long base = *inst_begin;
  const int e = *exp_in;
  for (int j = blockIdx.x; j < nrows; j += gridDim.x) {
    const float wj = w[j];
    if (wj == 0.0f) continue;                         // block-uniform
    const float sc = dtype == 1 ? beam_scale[rows[row_base + j].beam] : 1.0f;
    const long long a = base + row_ptr[j], b = base + row_ptr[j + 1];
    for (long long k0 = a + threadIdx.x; k0 < b; k0 += 4 * kRowThreads) {
      int c[4];
      float D[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long k = k0 + (long long)u * kRowThreads;
        c[u] = k < b ? col[k] : -1;
        D[u] = k < b ? entry_value(val, dtype, k, sc) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (c[u] < 0) continue;
        atomicAdd(acc + c[u], (unsigned long long)fixed_of(wj * D[u], e));   // the FP32 product, exactly
      }
    }
  }
}

__global__ void k_dose_finish(const unsigned long long* __restrict__ acc, long long n, const int* __restrict__ exp_in,
                              float* __restrict__ dose) {
  const int e = *exp_in;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    dose[v] = ldexpf(__ll2float_rn((long long)acc[v]), -e);   // one rounding to FP32
}

// one block per row (grid-stride over rows), four entries in flight per
// thread, compensated FP32 sums per thread, then FP64 over the block in a
// fixed order
__global__ void __launch_bounds__(kRowThreads) k_beamlet_dot(
    const long long* __restrict__ row_ptr, const long long* __restrict__ inst_begin, const int* __restrict__ col,
    const void* __restrict__ val, int dtype, const DRow* __restrict__ rows, int row_base,
    const float* __restrict__ beam_scale, const float* __restrict__ g, int nrows, float* __restrict__ out) {
  __shared__ double part[kRowThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long base = *inst_begin;
  for (int j = blockIdx.x; j < nrows; j += gridDim.x) {
    const float sc = dtype == 1 ? beam_scale[rows[row_base + j].beam] : 1.0f;
    const long long a = base + row_ptr[j], b = base + row_ptr[j + 1];
    float sum = 0.0f, comp = 0.0f;                    // compensated FP32 sum of the thread
    for (long long k0 = a + threadIdx.x; k0 < b; k0 += 4 * kRowThreads) {
      float p[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long k = k0 + (long long)u * kRowThreads;
        p[u] = k < b ? entry_value(val, dtype, k, sc) * g[col[k]] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float y = p[u] - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
      }
    }
    double s = (double)sum - (double)comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < kRowThreads / 32; ++i) t += part[i];
      out[j] = (float)t;
    }
    __syncthreads();
  }
}

}  // namespace dsc

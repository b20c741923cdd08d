// dsc_dose.cu -- products with the resident D_ij (Eq. 1 and its transpose).
//
//   dose(v)  = sum_j w_j D_jv       (Eq. 1: dose superposition over beamlets)
//   out(j)   = sum_v D_jv g(v)      (the transpose product an optimiser's
//                                    gradient needs)
//
// Both read one instance's CSR where the computation left it (rows = the
// instance's beamlets, columns = voxel indices).  The dose is a scatter over
// rows: every product w_j D_jv is formed exactly in FP64, scaled by a power
// of two chosen from a bound on |dose|, rounded to a 64-bit integer and added
// with integer atomics, so the sum does not depend on the order the atomics
// land in (deterministic, within one FP32 rounding of the exact sum of the
// products).  The transpose product is a gather per row, one warp per row,
// FP64 sums reduced in a fixed order.
#include "dsc_internal.h"

#include <cuda_bf16.h>

namespace dsc {

namespace {
__device__ __forceinline__ double entry_value(const void* val, int dtype, long long k, float scale) {
  if (dtype == 1) return (double)__bfloat162float(((const __nv_bfloat16*)val)[k]) * (double)scale;
  return (double)((const float*)val)[k];
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

__global__ void k_dose_scatter(const long long* __restrict__ row_ptr, const long long* __restrict__ inst_begin,
                               const int* __restrict__ col, const void* __restrict__ val, int dtype,
                               const DRow* __restrict__ rows, int row_base, const float* __restrict__ beam_scale,
                               const float* __restrict__ w, int nrows, const int* __restrict__ exp_in,
                               unsigned long long* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const long long base = *inst_begin;
  const int e = *exp_in;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long j = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); j < nrows; j += nw) {
    const double wj = (double)w[j];
    if (wj == 0.0) continue;                          // warp-uniform
    const float sc = dtype == 1 ? beam_scale[rows[row_base + j].beam] : 1.0f;
    const long long a = base + row_ptr[j], b = base + row_ptr[j + 1];
    for (long long k = a + lane; k < b; k += 32) {
      const double p = wj * entry_value(val, dtype, k, sc);   // exact: FP32 x FP32 (x power of two)
      const long long q = __double2ll_rn(ldexp(p, e));
      atomicAdd(acc + col[k], (unsigned long long)q);
    }
  }
}

__global__ void k_dose_finish(const unsigned long long* __restrict__ acc, long long n, const int* __restrict__ exp_in,
                              float* __restrict__ dose) {
  const int e = *exp_in;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    dose[v] = (float)ldexp((double)(long long)acc[v], -e);
}

__global__ void k_beamlet_dot(const long long* __restrict__ row_ptr, const long long* __restrict__ inst_begin,
                              const int* __restrict__ col, const void* __restrict__ val, int dtype,
                              const DRow* __restrict__ rows, int row_base, const float* __restrict__ beam_scale,
                              const float* __restrict__ g, int nrows, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long base = *inst_begin;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long j = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); j < nrows; j += nw) {
    const float sc = dtype == 1 ? beam_scale[rows[row_base + j].beam] : 1.0f;
    const long long a = base + row_ptr[j], b = base + row_ptr[j + 1];
    double s = 0.0;
    for (long long k = a + lane; k < b; k += 32) s = fma(entry_value(val, dtype, k, sc), (double)g[col[k]], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[j] = (float)s;
  }
}

}  // namespace dsc

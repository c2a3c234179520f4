// Grid-wide sums with a deterministic last-block finish.
//
// Each block reduces its threads' partials (warp shuffles, then shared memory) in
// double and writes one value per sum to `partials`; the last block to arrive (an
// atomic ticket, no waiting) adds the per-block values in block order and hands the
// totals to thread 0, which updates the solver scalars.  Results are bitwise
// reproducible for a fixed grid size.
#pragma once

#include "bem_internal.cuh"

namespace bem {

// Per-thread accumulator.  For float data the running sum is kept as an unevaluated
// pair (hi, lo) updated with Knuth's TwoSum, so the thread partial carries about
// twice the float precision before it is widened to double.
template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = hi + x;
    const float bp = t - hi;
    const float err = (hi - (t - bp)) + (x - bp);
    hi = t;
    lo += err;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

constexpr int RED_MAX_BLOCKS = 1024;

// Returns true in thread 0 of the last block, with tot[] filled.
template <int NS>
__device__ bool grid_reduce(double (&v)[NS], double* __restrict__ partials, unsigned int* ticket,
                            double (&tot)[NS]) {
  __shared__ double sh[NS][NTHREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double acc = 0.0;
      for (int w = 0; w < NTHREADS / 32; ++w) acc += sh[s][w];
      partials[s * RED_MAX_BLOCKS + blockIdx.x] = acc;
    }
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NTHREADS) x += __ldcg(&partials[s * RED_MAX_BLOCKS + b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    __syncthreads();
    if (lane == 0) sh[s][warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = 0.0;
      for (int w = 0; w < NTHREADS / 32; ++w) acc += sh[s][w];
      tot[s] = acc;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return threadIdx.x == 0;
}

}  // namespace bem

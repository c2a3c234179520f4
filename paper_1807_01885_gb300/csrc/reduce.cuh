// Grid-wide sums with a deterministic last-block finish.
//
// Each thread accumulates its elements; the block combines its threads (warp
// shuffles, then shared memory) and writes one 8-byte partial per sum to `partials`; the
// last block to arrive (an atomic ticket, no waiting) adds the per-block values in
// block order and hands the totals to thread 0, which updates the solver scalars.
// Results are bitwise reproducible for a fixed grid size.
//
// Float data: GB300 runs double-precision arithmetic at a small fraction of the
// float rate, so the thread and block levels keep each running sum as an
// unevaluated pair (hi, lo) of floats, combined with Knuth's TwoSum (about 44 bits
// of mantissa), block partials included; only the final totals are doubles.
#pragma once

#include "bem_internal.cuh"

namespace bem {

template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_sq(double x) { s += x * x; }
  __device__ __forceinline__ void add4(const double (&x)[4]) { s += (x[0] + x[1]) + (x[2] + x[3]); }
  __device__ __forceinline__ void combine(const Acc& o) { s += o.s; }
  __device__ __forceinline__ Acc shfl_down(int o) const {
    Acc r;
    r.s = __shfl_down_sync(0xffffffffu, s, o);
    return r;
  }
  __device__ __forceinline__ double value() const { return s; }
  // a block partial in its 8-byte slot
  __device__ __forceinline__ void store(double* slot) const { *slot = s; }
  __device__ __forceinline__ static Acc load(const double* slot) {
    Acc r;
    r.s = __ldcg(slot);
    return r;
  }
};
template <> struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = hi + x;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (x - bp);
    hi = t;
  }
  // x^2 with its rounding error (TwoProduct by fma) added in: the sum of squares keeps
  // the pair's precision even when the squares are large against their spread
  __device__ __forceinline__ void add_sq(float x) {
    const float q = x * x;
    const float e = fmaf(x, x, -q);
    add(q);
    lo += e;
  }
  // four terms of one 16-byte group: summed pairwise in float (each term carries its
  // own float rounding already), then one compensated addition
  __device__ __forceinline__ void add4(const float (&x)[4]) { add((x[0] + x[1]) + (x[2] + x[3])); }
  __device__ __forceinline__ void combine(const Acc& o) {
    const float t = hi + o.hi;
    const float bp = t - hi;
    const float e = (hi - (t - bp)) + (o.hi - bp);
    const float l = lo + o.lo + e;
    hi = t + l;                    // renormalise (Fast2Sum)
    lo = l - (hi - t);
  }
  __device__ __forceinline__ Acc shfl_down(int o) const {
    Acc r;
    r.hi = __shfl_down_sync(0xffffffffu, hi, o);
    r.lo = __shfl_down_sync(0xffffffffu, lo, o);
    return r;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
  // a block partial in its 8-byte slot, kept as the float pair: the last block then
  // combines partials without double arithmetic (a small fraction of the float rate)
  __device__ __forceinline__ void store(double* slot) const { *reinterpret_cast<float2*>(slot) = make_float2(hi, lo); }
  __device__ __forceinline__ static Acc load(const double* slot) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(slot));
    Acc r;
    r.hi = v.x;
    r.lo = v.y;
    return r;
  }
};

constexpr int RED_MAX_BLOCKS = 2048;

// Returns true in thread 0 of the last block, with tot[] filled.
template <int NS, typename T>
__device__ bool grid_reduce(Acc<T> (&a)[NS], double* __restrict__ partials, unsigned int* ticket,
                            double (&tot)[NS]) {
  __shared__ Acc<T> sh[NS][NTHREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    Acc<T> x = a[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x.combine(x.shfl_down(o));
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Acc<T> acc = sh[s][0];
      for (int w = 1; w < NTHREADS / 32; ++w) acc.combine(sh[s][w]);
      acc.store(&partials[s * RED_MAX_BLOCKS + blockIdx.x]);
    }
    // one acquire-release atomic: the release publishes this block's partials, the
    // acquire (in the block that draws the last ticket) makes every block's visible;
    // the barrier below extends that to the block's other threads
    unsigned int t;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(t) : "l"(ticket) : "memory");
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  // every partial this thread adds is loaded in one unrolled pass (all loads in
  // flight at once); each sum still combines its partials in block order
  Acc<T> xs[NS];
#pragma unroll
  for (int k = 0; k < RED_MAX_BLOCKS / NTHREADS; ++k) {
    const int b = threadIdx.x + k * NTHREADS;
    if (b < (int)gridDim.x) {
#pragma unroll
      for (int s = 0; s < NS; ++s) xs[s].combine(Acc<T>::load(&partials[s * RED_MAX_BLOCKS + b]));
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    Acc<T> x = xs[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x.combine(x.shfl_down(o));
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Acc<T> acc = sh[s][0];
      for (int w = 1; w < NTHREADS / 32; ++w) acc.combine(sh[s][w]);
      tot[s] = acc.value();
    }
    *ticket = 0u;
  }
  return threadIdx.x == 0;
}

}  // namespace bem

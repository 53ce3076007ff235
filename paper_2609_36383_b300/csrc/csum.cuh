// csum.cuh -- compensated summation for the step diagnostics' reductions
// (kinetic and field energy, constraint residuals, work sums, outer residual
// norms).  A CSum carries a sum and the accumulated rounding error of its
// additions; every addition is an exact TwoSum (Knuth), so the result is the
// rounded exact sum up to O(eps^2 n) however many terms and in whatever tree
// the reduction combines them.
#pragma once

#include <cuda_runtime.h>

struct CSum {
  double s, c;
};

__host__ __device__ __forceinline__ CSum csum_zero() { return CSum{0.0, 0.0}; }

// a += x, the rounding error of the addition kept in a.c
__host__ __device__ __forceinline__ void csum_add(CSum &a, double x) {
  const double t = a.s + x;
  const double bp = t - a.s;
  a.c += (a.s - (t - bp)) + (x - bp);
  a.s = t;
}

__host__ __device__ __forceinline__ CSum csum_merge(CSum a, const CSum &b) {
  csum_add(a, b.s);
  a.c += b.c;
  return a;
}

__host__ __device__ __forceinline__ double csum_value(const CSum &a) { return a.s + a.c; }

// warp reduction of one CSum per lane (the result in lane 0)
__device__ __forceinline__ CSum csum_warp(CSum a) {
  for (int o = 16; o > 0; o >>= 1) {
    CSum b;
    b.s = __shfl_down_sync(0xffffffffu, a.s, o);
    b.c = __shfl_down_sync(0xffffffffu, a.c, o);
    a = csum_merge(a, b);
  }
  return a;
}


// dual.cuh -- forward-mode dual numbers for the tangent of the particle map.
//
// A Dual carries a value and its directional derivative (tangent); every
// arithmetic operation applies the chain rule, so running the particle map
// (map_device.cuh) on Duals evaluates the map and its tangent in the
// direction seeded into the inputs, through the inner Picard iteration, the
// knot-split orbit integrals (whose piece ends move with the orbit), the
// GM-HC push and the deposit.  Comparisons, floor and the choices of
// fmin/fmax/fabs follow the value, so the tangent is that of the branch the
// value takes (the one-sided derivative at a tie).
#pragma once

#include <cmath>

struct Dual {
  double v, d;
  Dual() = default;
  __host__ __device__ constexpr Dual(double x) : v(x), d(0.0) {}
  __host__ __device__ constexpr Dual(double x, double dx) : v(x), d(dx) {}
  __host__ __device__ explicit operator int() const { return (int)v; }
  __host__ __device__ explicit operator double() const { return v; }
  __host__ __device__ Dual &operator+=(const Dual &b) {
    v += b.v;
    d += b.d;
    return *this;
  }
  __host__ __device__ Dual &operator-=(const Dual &b) {
    v -= b.v;
    d -= b.d;
    return *this;
  }
  __host__ __device__ Dual &operator*=(const Dual &b) {
    d = d * b.v + v * b.d;
    v *= b.v;
    return *this;
  }
};

__host__ __device__ inline Dual operator+(const Dual &a, const Dual &b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(const Dual &a, const Dual &b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator-(const Dual &a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator*(const Dual &a, const Dual &b) {
  return Dual(a.v * b.v, a.d * b.v + a.v * b.d);
}
__host__ __device__ inline Dual operator/(const Dual &a, const Dual &b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__host__ __device__ inline bool operator<(const Dual &a, const Dual &b) { return a.v < b.v; }
__host__ __device__ inline bool operator>(const Dual &a, const Dual &b) { return a.v > b.v; }
__host__ __device__ inline bool operator<=(const Dual &a, const Dual &b) { return a.v <= b.v; }
__host__ __device__ inline bool operator>=(const Dual &a, const Dual &b) { return a.v >= b.v; }
__host__ __device__ inline bool operator==(const Dual &a, const Dual &b) { return a.v == b.v; }
__host__ __device__ inline bool operator!=(const Dual &a, const Dual &b) { return a.v != b.v; }

__device__ inline Dual floor(const Dual &a) { return Dual(::floor(a.v), 0.0); }
__device__ inline Dual fabs(const Dual &a) { return a.v < 0.0 ? -a : a; }
__device__ inline Dual fmin(const Dual &a, const Dual &b) { return b.v < a.v ? b : a; }
__device__ inline Dual fmax(const Dual &a, const Dual &b) { return b.v > a.v ? b : a; }
__device__ inline Dual sqrt(const Dual &a) {
  const double s = ::sqrt(a.v);
  return Dual(s, s > 0.0 ? 0.5 * a.d / s : 0.0);
}
__device__ inline Dual rsqrt(const Dual &a) {
  const double r = ::rsqrt(a.v);
  return Dual(r, -0.5 * r * r * r * a.d);
}
__device__ inline bool isfinite(const Dual &a) { return ::isfinite(a.v) && ::isfinite(a.d); }

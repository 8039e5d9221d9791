// Forward-mode dual numbers: a value and one derivative, carried through generic system
// code (the flux, the source and the manufactured-state assembly of systems.cuh).
#pragma once

#include <type_traits>

namespace lbx {

template <typename T>
struct Dual {
  T v, d;
  __host__ __device__ Dual() : v(0), d(0) {}
  __host__ __device__ Dual(T a, T b) : v(a), d(b) {}
  template <typename U, typename = typename std::enable_if<std::is_arithmetic<U>::value>::type>
  __host__ __device__ Dual(U a) : v(T(a)), d(0) {}
  __host__ __device__ Dual& operator+=(const Dual& o) { v += o.v; d += o.d; return *this; }
  __host__ __device__ Dual& operator-=(const Dual& o) { v -= o.v; d -= o.d; return *this; }
  __host__ __device__ Dual& operator*=(const Dual& o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
};
template <typename T> __host__ __device__ inline Dual<T> operator+(Dual<T> a, const Dual<T>& b) { return a += b; }
template <typename T> __host__ __device__ inline Dual<T> operator-(Dual<T> a, const Dual<T>& b) { return a -= b; }
template <typename T> __host__ __device__ inline Dual<T> operator-(const Dual<T>& a) { return Dual<T>(-a.v, -a.d); }
template <typename T> __host__ __device__ inline Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) {
  return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d);
}
template <typename T> __host__ __device__ inline Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  const T inv = T(1) / b.v;
  const T q = a.v * inv;
  return Dual<T>(q, (a.d - q * b.d) * inv);
}

// sin(pi a) and cos(pi a) of a dual number (the derivative carries the factor pi).
template <typename T>
__device__ inline void sincospi_dual(const Dual<T>& a, Dual<T>* s, Dual<T>* c) {
  T sv, cv;
  sincospi(a.v, &sv, &cv);
  const T pi = T(3.141592653589793238462643383279502884);
  *s = Dual<T>(sv, pi * cv * a.d);
  *c = Dual<T>(cv, -pi * sv * a.d);
}

// Forward mode with N tangent directions carried at once: one evaluation of the system code
// gives the value and N directional derivatives.  With seeds that are compile-time unit
// vectors, the compiler folds the tangents that stay zero through the leading operations, so
// a chunk of N directions costs far less than N single-tangent passes.
template <typename T, int N>
struct DualN {
  T v, d[N];
  __host__ __device__ DualN() : v(0) {
#pragma unroll
    for (int j = 0; j < N; ++j) d[j] = T(0);
  }
  template <typename U, typename = typename std::enable_if<std::is_arithmetic<U>::value>::type>
  __host__ __device__ DualN(U a) : v(T(a)) {
#pragma unroll
    for (int j = 0; j < N; ++j) d[j] = T(0);
  }
  __host__ __device__ DualN& operator+=(const DualN& o) {
    v += o.v;
#pragma unroll
    for (int j = 0; j < N; ++j) d[j] += o.d[j];
    return *this;
  }
  __host__ __device__ DualN& operator-=(const DualN& o) {
    v -= o.v;
#pragma unroll
    for (int j = 0; j < N; ++j) d[j] -= o.d[j];
    return *this;
  }
  __host__ __device__ DualN& operator*=(const DualN& o) {
#pragma unroll
    for (int j = 0; j < N; ++j) d[j] = d[j] * o.v + v * o.d[j];
    v *= o.v;
    return *this;
  }
};
template <typename T, int N>
__host__ __device__ inline DualN<T, N> operator+(DualN<T, N> a, const DualN<T, N>& b) { return a += b; }
template <typename T, int N>
__host__ __device__ inline DualN<T, N> operator-(DualN<T, N> a, const DualN<T, N>& b) { return a -= b; }
template <typename T, int N>
__host__ __device__ inline DualN<T, N> operator-(const DualN<T, N>& a) {
  DualN<T, N> r;
  r.v = -a.v;
#pragma unroll
  for (int j = 0; j < N; ++j) r.d[j] = -a.d[j];
  return r;
}
template <typename T, int N>
__host__ __device__ inline DualN<T, N> operator*(DualN<T, N> a, const DualN<T, N>& b) { return a *= b; }
template <typename T, int N>
__host__ __device__ inline DualN<T, N> operator/(const DualN<T, N>& a, const DualN<T, N>& b) {
  const T inv = T(1) / b.v;
  DualN<T, N> r;
  r.v = a.v * inv;
#pragma unroll
  for (int j = 0; j < N; ++j) r.d[j] = (a.d[j] - r.v * b.d[j]) * inv;
  return r;
}

}  // namespace lbx

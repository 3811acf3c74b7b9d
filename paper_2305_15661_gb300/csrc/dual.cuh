// Forward-mode dual numbers with N derivative directions, for the pointwise
// derivatives of the Roe flux (dH/dU+, dH/dU-, dH/dn) inside the element kernels.
#pragma once
#include <cuda_runtime.h>

namespace ift {

template <class T, int N>
struct Dual {
  T v;
  T d[N];
};

template <class T, int N>
__device__ __forceinline__ Dual<T, N> dconst(T a) {
  Dual<T, N> r;
  r.v = a;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = T(0);
  return r;
}

template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator*(T s, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = s * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * b.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator*(const Dual<T, N>& b, T s) {
  return s * b;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator+(const Dual<T, N>& a, T s) {
  Dual<T, N> r = a;
  r.v += s;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator+(T s, const Dual<T, N>& a) {
  return a + s;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator-(const Dual<T, N>& a, T s) {
  Dual<T, N> r = a;
  r.v -= s;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator-(T s, const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = s - a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
// 1 / b
template <class T, int N>
__device__ __forceinline__ Dual<T, N> recip(const Dual<T, N>& b) {
  Dual<T, N> r;
  T inv = T(1) / b.v;
  r.v = inv;
  T m = -inv * inv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = m * b.d[i];
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  T inv = T(1) / b.v;
  r.v = a.v * inv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
  return r;
}
template <class T, int N>
__device__ __forceinline__ Dual<T, N> dsqrt(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = sqrt(a.v);
  T h = T(0.5) / r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = h * a.d[i];
  return r;
}
// |a| with derivative sign(a), sign(0) = 0
template <class T, int N>
__device__ __forceinline__ Dual<T, N> dabs(const Dual<T, N>& a) {
  T s = (a.v > T(0)) ? T(1) : ((a.v < T(0)) ? T(-1) : T(0));
  Dual<T, N> r;
  r.v = fabs(a.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
  return r;
}

}  // namespace ift

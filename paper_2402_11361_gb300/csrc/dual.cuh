// Forward-mode dual numbers for exact pointwise Jacobians on the device.
//
// Dual<T, N> = v + sum_i d[i] eps_i with eps_i eps_j = 0.  T may itself be a Dual,
// which gives second derivatives (the SUPG strong residual contains first
// derivatives of the fluxes, and the Newton blocks of eq. C312 differentiate it
// once more).  Everything is header-only and usable on host and device.
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define HD __host__ __device__ __forceinline__
#else
#define HD inline
#endif

template <class T, int N>
struct Dual {
  T v;
  T d[N];
};

// innermost scalar type of a (possibly nested) dual; constants mixed into dual
// arithmetic are converted to it, so that FP32 duals never compute in FP64
template <class T> struct Base { typedef T type; };
template <class T, int N> struct Base<Dual<T, N>> { typedef typename Base<T>::type type; };
template <class T> HD typename Base<T>::type bcast(double c) { return static_cast<typename Base<T>::type>(c); }

// innermost value of a (possibly nested) scalar, as a double
HD double val0(double x) { return x; }
HD double val0(float x) { return x; }
template <class T, int N>
HD double val0(const Dual<T, N>& x) { return val0(x.v); }

template <class T> struct Zero { HD static T get() { return T(0.0); } };
template <class T, int N> struct Zero<Dual<T, N>> {
  HD static Dual<T, N> get() {
    Dual<T, N> r;
    r.v = Zero<T>::get();
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = Zero<T>::get();
    return r;
  }
};
template <class T> HD T zero() { return Zero<T>::get(); }

// constant of type T
template <class T> struct Cst { HD static T get(double c) { return T(c); } };
template <class T, int N> struct Cst<Dual<T, N>> {
  HD static Dual<T, N> get(double c) {
    Dual<T, N> r = Zero<Dual<T, N>>::get();
    r.v = Cst<T>::get(c);
    return r;
  }
};
template <class T> HD T cst(double c) { return Cst<T>::get(c); }

// ---------------------------------------------------------------- arithmetic
template <class T, int N>
HD Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class T, int N>
HD Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class T, int N>
HD Dual<T, N> operator-(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class T, int N>
HD Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <class T, int N>
HD Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r;
  T inv = cst<T>(1.0) / b.v;
  r.v = a.v * inv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
  return r;
}
// mixed with plain doubles
template <class T, int N>
HD Dual<T, N> operator+(const Dual<T, N>& a, double b) { Dual<T, N> r = a; r.v = a.v + bcast<T>(b); return r; }
template <class T, int N>
HD Dual<T, N> operator+(double b, const Dual<T, N>& a) { return a + b; }
template <class T, int N>
HD Dual<T, N> operator-(const Dual<T, N>& a, double b) { Dual<T, N> r = a; r.v = a.v - bcast<T>(b); return r; }
template <class T, int N>
HD Dual<T, N> operator-(double b, const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = bcast<T>(b) - a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class T, int N>
HD Dual<T, N> operator*(const Dual<T, N>& a, double b) {
  Dual<T, N> r;
  const auto c = bcast<T>(b);
  r.v = a.v * c;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * c;
  return r;
}
template <class T, int N>
HD Dual<T, N> operator*(double b, const Dual<T, N>& a) { return a * b; }
template <class T, int N>
HD Dual<T, N> operator/(const Dual<T, N>& a, double b) {
  const auto c = bcast<T>(1.0) / bcast<T>(b);
  Dual<T, N> r;
  r.v = a.v * c;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * c;
  return r;
}
template <class T, int N>
HD Dual<T, N> operator/(double b, const Dual<T, N>& a) {
  Dual<T, N> r;
  T inv = cst<T>(1.0) / a.v;
  r.v = bcast<T>(b) * inv;
  T f = -(r.v * inv);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * f;
  return r;
}
// ---------------------------------------------------------------- functions
HD double dsqrt(double x) { return sqrt(x); }
HD float dsqrt(float x) { return sqrtf(x); }
template <class T, int N>
HD Dual<T, N> dsqrt(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dsqrt(a.v);
  T f = cst<T>(0.5) / r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * f;
  return r;
}
// sqrt of a sum of squares x = v.v: the magnitude |v| is not differentiable at v = 0, and its
// derivative there is taken as 0 (as sign(0) = 0 for |x|), so a gas at rest gives finite
// Jacobians
HD double dsqrt0(double x) { return sqrt(x); }
HD float dsqrt0(float x) { return sqrtf(x); }
template <class T, int N>
HD Dual<T, N> dsqrt0(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dsqrt0(a.v);
  if (!(val0(a) > 0.0)) {
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = zero<T>();
    return r;
  }
  T f = cst<T>(0.5) / r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * f;
  return r;
}
HD double dsin(double x) { return sin(x); }
HD double dcos(double x) { return cos(x); }
HD float dsin(float x) { return sinf(x); }
HD float dcos(float x) { return cosf(x); }
template <class T, int N>
HD Dual<T, N> dsin(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dsin(a.v);
  T c = dcos(a.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * c;
  return r;
}
template <class T, int N>
HD Dual<T, N> dcos(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dcos(a.v);
  T s = -dsin(a.v);
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s;
  return r;
}
// |x| with derivative sign(x), sign(0) = 0
HD double dlog(double x) { return log(x); }
HD float dlog(float x) { return logf(x); }
template <class T, int N>
HD Dual<T, N> dlog(const Dual<T, N>& a) {
  Dual<T, N> r;
  r.v = dlog(a.v);
  T f = cst<T>(1.0) / a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * f;
  return r;
}
HD double dabs(double x) { return x > 0 ? x : (x < 0 ? -x : 0.0); }
HD float dabs(float x) { return x > 0 ? x : (x < 0 ? -x : 0.f); }
template <class T, int N>
HD Dual<T, N> dabs(const Dual<T, N>& a) {
  double s = val0(a);
  double sg = s > 0 ? 1.0 : (s < 0 ? -1.0 : 0.0);
  return a * sg;
}

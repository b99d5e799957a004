// Shared device helpers: complex arithmetic templated on the real type, launch
// checks, and the status word every kernel reports device-side failures through.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>

#include "../../include/hsweep.h"

template <typename R>
struct alignas(2 * sizeof(R)) Cx {
  R re, im;
  Cx() = default;
  __host__ __device__ constexpr Cx(R a, R b = R(0)) : re(a), im(b) {}
};

using c64 = Cx<float>;
using c128 = Cx<double>;

template <typename R> __host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return Cx<R>(a.re + b.re, a.im + b.im); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return Cx<R>(a.re - b.re, a.im - b.im); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a) { return Cx<R>(-a.re, -a.im); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return Cx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return Cx<R>(s * a.re, s * a.im); }
template <typename R> __host__ __device__ __forceinline__ Cx<R>& operator+=(Cx<R>& a, Cx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <typename R> __host__ __device__ __forceinline__ Cx<R>& operator-=(Cx<R>& a, Cx<R> b) { a.re -= b.re; a.im -= b.im; return a; }
template <typename R> __host__ __device__ __forceinline__ Cx<R> conj(Cx<R> a) { return Cx<R>(a.re, -a.im); }
template <typename R> __host__ __device__ __forceinline__ R abs2(Cx<R> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b (complex fused multiply-add)
template <typename R> __host__ __device__ __forceinline__ void cfma(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <typename R> __host__ __device__ __forceinline__ void cfma_conj(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
template <typename To, typename From> __host__ __device__ __forceinline__ Cx<To> cvt(Cx<From> a) {
  return Cx<To>(To(a.re), To(a.im));
}
// 1 / a
template <typename R> __host__ __device__ __forceinline__ Cx<R> cinv(Cx<R> a) {
  R s = R(1) / (a.re * a.re + a.im * a.im);
  return Cx<R>(a.re * s, -a.im * s);
}

// principal square root
template <typename R> __host__ __device__ __forceinline__ Cx<R> csqrt(Cx<R> a) {
  R r = sqrt(a.re * a.re + a.im * a.im);
  R x = sqrt((r + a.re) * R(0.5));
  R y = sqrt((r - a.re) * R(0.5));
  return Cx<R>(x, a.im < 0 ? -y : y);
}

template <typename R> __device__ __forceinline__ Cx<R> shfl_xor(Cx<R> v, int off) {
  return Cx<R>(__shfl_xor_sync(0xffffffffu, v.re, off), __shfl_xor_sync(0xffffffffu, v.im, off));
}

// L2-only loads/stores for data exchanged between CTAs of one sweep team.
template <typename R> __device__ __forceinline__ Cx<R> ld_cg(const Cx<R>* p);
template <> __device__ __forceinline__ Cx<float> ld_cg(const Cx<float>* p) {
  float2 v = __ldcg(reinterpret_cast<const float2*>(p)); return Cx<float>(v.x, v.y);
}
template <> __device__ __forceinline__ Cx<double> ld_cg(const Cx<double>* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p)); return Cx<double>(v.x, v.y);
}
template <typename R> __device__ __forceinline__ void st_cg(Cx<R>* p, Cx<R> v);
template <> __device__ __forceinline__ void st_cg(Cx<float>* p, Cx<float> v) {
  __stcg(reinterpret_cast<float2*>(p), make_float2(v.re, v.im));
}
template <> __device__ __forceinline__ void st_cg(Cx<double>* p, Cx<double> v) {
  __stcg(reinterpret_cast<double2*>(p), make_double2(v.re, v.im));
}

// Device status word: [0] = first error code (HSWEEP_ERR_*), [1] = layer.
__device__ __forceinline__ void report_error(int* status, int code, int layer) {
  if (status && atomicCAS(status, 0, code) == 0) status[1] = layer;
}

#define HSW_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return HSWEEP_ERR_CUDA;       \
  } while (0)

static inline unsigned div_up(long long a, long long b) { return unsigned((a + b - 1) / b); }

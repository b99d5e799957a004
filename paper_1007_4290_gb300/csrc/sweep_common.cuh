// Device helpers shared by the sweep kernels (sweep_team.cu, sweep_strong.cu): paired
// FP32 multiply-adds on complex64, tagged 8-byte words for partial sums exchanged through
// L2, complex multiply-accumulate in the storage precision, and the padded row stride of
// the shared-memory vector arrays.
#pragma once
#include <type_traits>
#include "handle.h"

namespace sweepc {

typedef unsigned long long u64;

// padded row stride (entries) of the shared vector arrays: conflict-free reads of one
// row per lane group, 16-byte aligned rows where pairs are read together
template <typename R>
__host__ __device__ constexpr int vstride(int G) {
  return sizeof(R) == 4 ? (G % 4 == 0 ? G + 2 : G) : (G % 2 == 0 ? G + 1 : G);
}

__device__ __forceinline__ u64 pk2(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(u64 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ void fma2(u64& acc, u64 a, u64 b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
// bring the 128-byte line at p into L2 (no register result, nothing waits for it)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Tagged partial sums in L2.  Naturally aligned 8-byte accesses are single-copy atomic,
// so one tag bit (bit 0, the lowest mantissa bit of the real part in complex64, of each
// part in complex128) per 8-byte word identifies the step that wrote the word.
template <typename R> struct Tagged;
template <> struct Tagged<float> {
  typedef u64 W;     // one complex64 value: (re, im) in one 8-byte word
  static __device__ __forceinline__ W pack(Cx<float> v, unsigned tag) {
    return (u64)((__float_as_uint(v.re) & ~1u) | tag) | ((u64)__float_as_uint(v.im) << 32);
  }
  static __device__ __forceinline__ bool ok(W w, unsigned tag) { return ((unsigned)w & 1u) == tag; }
  static __device__ __forceinline__ Cx<float> value(W w) {
    return Cx<float>(__uint_as_float((unsigned)w), __uint_as_float((unsigned)(w >> 32)));
  }
  static __device__ __forceinline__ void store(W* p, W w) { __stcg(reinterpret_cast<unsigned long long*>(p), w); }
  static __device__ __forceinline__ W load(const W* p) { return __ldcg(reinterpret_cast<const unsigned long long*>(p)); }
};
template <> struct Tagged<double> {
  typedef ulonglong2 W;   // one complex128 value: two 8-byte words, each tagged
  static __device__ __forceinline__ u64 tag64(double x, unsigned tag) {
    return ((u64)__double_as_longlong(x) & ~1ull) | (u64)tag;
  }
  static __device__ __forceinline__ W pack(Cx<double> v, unsigned tag) {
    W w;
    w.x = tag64(v.re, tag);
    w.y = tag64(v.im, tag);
    return w;
  }
  static __device__ __forceinline__ bool ok(W w, unsigned tag) {
    return ((unsigned)w.x & 1u) == tag && ((unsigned)w.y & 1u) == tag;
  }
  static __device__ __forceinline__ Cx<double> value(W w) {
    return Cx<double>(__longlong_as_double((long long)w.x), __longlong_as_double((long long)w.y));
  }
  static __device__ __forceinline__ void store(W* p, W w) { __stcg(p, w); }
  static __device__ __forceinline__ W load(const W* p) { return __ldcg(p); }
};

// complex multiply-accumulate in the storage precision
template <typename R> struct Mac;
template <> struct Mac<float> {
  struct A { u64 a, b; };          // a = sum Re(f) x, b = sum Im(f) x  (x as (re, im))
  struct F { u64 rr, ii; };        // (Re f, Re f), (Im f, Im f)
  typedef u64 X;
  static __device__ __forceinline__ void zero(A& s) { s.a = 0ull; s.b = 0ull; }
  static __device__ __forceinline__ F f(const Cx<float>* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    F r;
    r.rr = pk2(v.x, v.x);
    r.ii = pk2(v.y, v.y);
    return r;
  }
  static __device__ __forceinline__ void mac(A& s, const F& f, X x) { fma2(s.a, f.rr, x); fma2(s.b, f.ii, x); }
  static __device__ __forceinline__ Cx<float> get(const A& s) {
    float ar, ai, br, bi;
    upk2(s.a, ar, ai);
    upk2(s.b, br, bi);
    return Cx<float>(ar - bi, ai + br);
  }
};
template <> struct Mac<double> {
  typedef Cx<double> A, F, X;
  static __device__ __forceinline__ void zero(A& s) { s = Cx<double>(0.0, 0.0); }
  static __device__ __forceinline__ F f(const Cx<double>* p) { return *p; }
  static __device__ __forceinline__ void mac(A& s, const F& f, X x) { cfma(s, f, x); }
  static __device__ __forceinline__ Cx<double> get(const A& s) { return s; }
};

// the G entries of one vector row (16-byte pairs for complex64 rows of even length)
template <typename R, int G>
__device__ __forceinline__ void load_row(const Cx<R>* p, typename Mac<R>::X (&v)[G]) {
  if constexpr (std::is_same<R, float>::value && G % 2 == 0) {
#pragma unroll
    for (int g = 0; g < G; g += 2) {
      const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(p + g);
      v[g] = t.x;
      v[g + 1] = t.y;
    }
  } else if constexpr (std::is_same<R, float>::value) {
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = *reinterpret_cast<const u64*>(p + g);
  } else {
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = p[g];
  }
}

}  // namespace sweepc

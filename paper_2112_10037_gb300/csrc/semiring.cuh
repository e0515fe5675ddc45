// Sum and product of the numeric pass.  Row i of C is the sum over the
// nonzeros A(i,k) of A(i,k) * B(k,:) (Sec. 2.2); the same row-wise step
// computes a product over another semiring when + and * are replaced:
// min-plus (shortest paths), max-plus (longest paths) and or-and
// (reachability).  Min and max do not depend on the order of their
// operands, so those products are exact.
//
// Each policy gives the sum's identity (the cleared state of an
// accumulator word), the product, the sum, their fusion acc (+) a (*) b, and
// shared-memory updates that other lanes may race with: red_value (*p (+)=
// x), red_shared (*p (+)= a (*) b) and madd_shared (the same, returning
// whether the word still held the identity when read, i.e. whether this may
// be the column's first product).
#pragma once

#include "internal.cuh"

namespace sg {

__device__ __forceinline__ unsigned long long sr_bits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned sr_bits(float v) { return __float_as_uint(v); }

template <typename T> __device__ __forceinline__ T sr_inf();
template <> __device__ __forceinline__ double sr_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }
template <> __device__ __forceinline__ float sr_inf<float>() { return __int_as_float(0x7f800000); }

__device__ __forceinline__ unsigned long long sr_cas(double* p, unsigned long long old, unsigned long long nv) {
  return atomicCAS(reinterpret_cast<unsigned long long*>(p), old, nv);
}
__device__ __forceinline__ unsigned sr_cas(float* p, unsigned old, unsigned nv) {
  return atomicCAS(reinterpret_cast<unsigned*>(p), old, nv);
}

// *p = min(*p, x) (MIN) or max(*p, x) by compare-and-swap, written only
// when x improves the word; returns whether the word held `zero` when read.
template <bool MIN, typename T>
__device__ __forceinline__ bool minmax_shared(T* p, T x, T zero, uint32_t* err) {
  T old = *reinterpret_cast<volatile T*>(p);
  const bool first = sr_bits(old) == sr_bits(zero);
  for (int it = 0; it < CAS_RETRY_LIMIT; ++it) {
    if (MIN ? !(x < old) : !(x > old)) return first;
    const auto prev = sr_cas(p, sr_bits(old), sr_bits(x));
    if (prev == sr_bits(old)) return first;
    if (sizeof(T) == 8) old = __longlong_as_double((long long)prev);
    else old = __uint_as_float((unsigned)prev);
  }
  atomicOr(err, EB_INTERNAL);  // never expected: each failed swap is another update's improvement
  return first;
}

template <typename T, int SR> struct SrOps;

template <typename T> struct SrOps<T, SPGEMM_PLUS_TIMES> {
  __device__ static T zero() { return T(0); }
  __device__ static bool cleared(T v) { return is_cleared(v); }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T add(T x, T y) { return x + y; }
  __device__ static T madd(T a, T b, T acc) { return fma(a, b, acc); }
  __device__ static void red_value(T* p, T x, uint32_t*) { red_add_shared(p, x); }
  __device__ static void red_shared(T* p, T a, T b, uint32_t*) { red_add_shared(p, a * b); }
  __device__ static bool madd_shared(T* p, T a, T b, uint32_t* err) { return fma_shared(p, a, b, err); }
};

template <typename T> struct SrOps<T, SPGEMM_MIN_PLUS> {
  __device__ static T zero() { return sr_inf<T>(); }
  __device__ static bool cleared(T v) { return sr_bits(v) == sr_bits(zero()); }
  __device__ static T mul(T a, T b) { return a + b; }
  __device__ static T add(T x, T y) { return y < x ? y : x; }
  __device__ static T madd(T a, T b, T acc) { return add(acc, a + b); }
  __device__ static void red_value(T* p, T x, uint32_t* err) { minmax_shared<true>(p, x, zero(), err); }
  __device__ static void red_shared(T* p, T a, T b, uint32_t* err) { minmax_shared<true>(p, a + b, zero(), err); }
  __device__ static bool madd_shared(T* p, T a, T b, uint32_t* err) {
    return minmax_shared<true>(p, a + b, zero(), err);
  }
};

template <typename T> struct SrOps<T, SPGEMM_MAX_PLUS> {
  __device__ static T zero() { return -sr_inf<T>(); }
  __device__ static bool cleared(T v) { return sr_bits(v) == sr_bits(zero()); }
  __device__ static T mul(T a, T b) { return a + b; }
  __device__ static T add(T x, T y) { return y > x ? y : x; }
  __device__ static T madd(T a, T b, T acc) { return add(acc, a + b); }
  __device__ static void red_value(T* p, T x, uint32_t* err) { minmax_shared<false>(p, x, zero(), err); }
  __device__ static void red_shared(T* p, T a, T b, uint32_t* err) { minmax_shared<false>(p, a + b, zero(), err); }
  __device__ static bool madd_shared(T* p, T a, T b, uint32_t* err) {
    return minmax_shared<false>(p, a + b, zero(), err);
  }
};

template <typename T> struct SrOps<T, SPGEMM_OR_AND> {
  __device__ static T zero() { return T(0); }
  __device__ static bool cleared(T v) { return is_cleared(v); }
  __device__ static T mul(T a, T b) { return (a != T(0) && b != T(0)) ? T(1) : T(0); }
  __device__ static T add(T x, T y) { return (x != T(0) || y != T(0)) ? T(1) : T(0); }
  __device__ static T madd(T a, T b, T acc) { return add(acc, mul(a, b)); }
  // every writer stores the same 1, so racing stores need no atomics
  __device__ static void red_value(T* p, T x, uint32_t*) {
    if (x != T(0)) *reinterpret_cast<volatile T*>(p) = T(1);
  }
  __device__ static void red_shared(T* p, T a, T b, uint32_t*) {
    if (a != T(0) && b != T(0)) *reinterpret_cast<volatile T*>(p) = T(1);
  }
  __device__ static bool madd_shared(T* p, T a, T b, uint32_t*) {
    const T old = *reinterpret_cast<volatile T*>(p);
    if (a != T(0) && b != T(0) && old == T(0)) *reinterpret_cast<volatile T*>(p) = T(1);
    return is_cleared(old);
  }
};

}  // namespace sg

// Float-pair ("FP64X") arithmetic on the FP32 pipes, shared by the CUDA-core H·v kernels.
//
// A double x is carried as (hi, lo) = (fl(x), fl(x - hi)): about 48 significant bits.
// Products are exact in two floats (hi*hi by the FMA error-free transformation, cross
// terms added to the error word; lo*lo dropped, 2^-48 relative); sums use the two-sum of
// Knuth on the high words with all errors collected in the low word, renormalised when
// converted back.  Relative error of a sum of K products ~ 2^-48 sqrt(K).
#pragma once

namespace dmrg2d {

struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
// acc (sum in hi, collected errors in lo) += a * b
__device__ __forceinline__ void ff_fma(ff& acc, const ff a, const ff b) {
  // __fmul_rn / __fadd_rn: never contracted into an FMA, which would break the two-sum
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);        // exact: a.hi b.hi = p + e
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = __fadd_rn(acc.hi, p);  // two-sum of the high words
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ double ff_to_double(const ff a) { return (double)a.hi + (double)a.lo; }

// the same operations for the native types, so that one kernel template serves FP64,
// FP32 and float pairs: the compute type's zero, conversion in and out, and acc += a b
template <typename Tc>
__device__ __forceinline__ Tc c_zero() {
  return Tc(0);
}
template <>
__device__ __forceinline__ ff c_zero<ff>() {
  return {0.f, 0.f};
}
template <typename Tc, typename Tin>
__device__ __forceinline__ Tc c_in(Tin x) {
  return (Tc)x;
}
template <>
__device__ __forceinline__ ff c_in<ff, double>(double x) {
  return ff_of(x);
}
__device__ __forceinline__ double c_out(double x) { return x; }
__device__ __forceinline__ float c_out(float x) { return x; }
__device__ __forceinline__ double c_out(ff x) { return ff_to_double(x); }
__device__ __forceinline__ void c_mac(double& acc, double a, double b) { acc += a * b; }
__device__ __forceinline__ void c_mac(float& acc, float a, float b) { acc += a * b; }
__device__ __forceinline__ void c_mac(ff& acc, ff a, ff b) { ff_fma(acc, a, b); }

}  // namespace dmrg2d

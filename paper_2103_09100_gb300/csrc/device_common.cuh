// Device helpers shared by the force kernels: the transform op convention
// of mesh_upload and the point-load time functions of the paper (Sec. 5).
#pragma once
#include <math.h>
#include <stdint.h>

#include "../../include/sbx.h"

namespace sbx {

// op = 8 * perm_index + sign_bits; node by node u_master[r] =
// (-1)^{bit r} u_cell[perm[r]] (permutations of (0,1,2), lexicographic).
__device__ __forceinline__ int op_perm_of(int op, int r) {
  // permutation i (lexicographic): perm[0] = i / 2, perm[1] from a 2-bit
  // table, perm[2] = 3 - perm[0] - perm[1]
  const int i = op >> 3;
  const int p0 = i >> 1;
  const int p1 = (int)((0x489u >> (2 * i)) & 3u);   // {1, 2, 0, 2, 0, 1}[i]
  return r == 0 ? p0 : (r == 1 ? p1 : 3 - p0 - p1);
}

// 2^k as a float, k in [-126, 127].
__device__ __forceinline__ float exp2i(int k) { return __int_as_float((k + 127) << 23); }

// FP64 -> FP32 pair (hi, lo) with hi = x rounded to 24 significant bits
// (ties away from zero) and lo = (x - hi) rounded to FP32, using integer
// operations and FP32 multiplies only: GB300's FP64 pipe runs at ~1/64 of
// FP32, and a displacement field is exactly zero away from the wave front,
// so every case must stay off that pipe.
//   |x| < 2^-103 (zero, subnormal, tiny): hi = lo = 0 (signed)
//   2^-103 <= |x| < 2^-74:                 hi exact to 24 bits, lo = 0
//   |x| >= 2^126, Inf, NaN:                hi = +-Inf or NaN, lo = 0
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned int sgn = (unsigned int)(b >> 63) << 31;
  if (e < 920) {
    hi = __uint_as_float(sgn);
    lo = hi;
    return;
  }
  if (e > 1148) {
    const bool nan = e == 0x7FF && (b & 0xFFFFFFFFFFFFFull) != 0;
    hi = __uint_as_float(sgn | (nan ? 0x7FC00000u : 0x7F800000u));
    lo = 0.0f;
    return;
  }
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long hm = (mant + (1ull << 28)) >> 29;           // <= 2^24
  const int rem = (int)((long long)mant - (long long)(hm << 29));      // |rem| <= 2^28
  float h = (float)(unsigned)hm * exp2i(e - 1046);
  float l = e >= 949 ? (float)rem * exp2i(e - 1075) : 0.0f;
  hi = __uint_as_float(__float_as_uint(h) ^ sgn);
  lo = __uint_as_float(__float_as_uint(l) ^ sgn);
}

// FP32 -> FP64 by re-packing the bits (exact for normal numbers); zero and
// subnormals give a signed zero, Inf and NaN keep their kind.
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned int b = __float_as_uint(x);
  const unsigned int e = (b >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(b >> 31) << 63;
  if (e == 0u) return __longlong_as_double((long long)s);
  const unsigned long long de = e == 255u ? 0x7FFull : (unsigned long long)(e + 896u);
  const unsigned long long d = s | (de << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// L2 eviction priorities.  Per step the mixed form touches ~1.2x the L2 in
// streams that are read or written once (U_n, U_{n-1}, w, U_{n+1}) and two
// working sets that live across kernels: the FP32 force accumulator
// (reduced into by the force kernels, read and cleared by the update) and
// the (hi, lo) pairs (written by the update, gathered by the next force).
// The streams carry evict_first, the working sets evict_last, so that the
// working sets stay in L2 from one kernel to the next.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// read-only for the whole kernel (non-coherent path)
__device__ __forceinline__ double ld_nc_hint(const double *a, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_hint(const double *a, uint64_t pol) {
  double v;
  asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint(double *a, double v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ float4 ld_hint(const float4 *a, uint64_t pol) {
  float4 q;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w)
               : "l"(a), "l"(pol));
  return q;
}
__device__ __forceinline__ void st_hint(float4 *a, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x),
               "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ double2 ld_nc_hint(const double2 *a, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_hint(const double2 *a, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint(double2 *a, double2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(a), "d"(v.x), "d"(v.y),
               "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_hint(float2 *a, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y),
               "l"(pol)
               : "memory");
}

// Eqs. (Ricker), (Triangle), (Lamb).
__device__ __forceinline__ double wavelet_value(int kind, double t, double t1, double ncyc) {
  if (kind == SBX_WAVE_RICKER) {
    const double tau = (t - t1) / (t1 / 5.0);
    return (1.0 - tau * tau) * exp(-0.5 * tau * tau);
  } else if (kind == SBX_WAVE_TRIANGLE) {
    if (t < 0.0 || t > 2.0 * t1) return 0.0;
    return 1.0 - fabs(t / t1 - 1.0);
  } else {
    if (t < 0.0 || t > t1) return 0.0;
    const double s = sin(M_PI * t / t1);
    return sin(2.0 * M_PI * ncyc * t / t1) * s * s;
  }
}

}  // namespace sbx

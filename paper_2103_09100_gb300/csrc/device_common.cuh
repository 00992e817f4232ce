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
  // byte i holds permutation i with perm[r] in bits 2r..2r+1
  const uint64_t tab = 0x061209211824ull;
  return (int)((tab >> (8 * (op >> 3) + 2 * r)) & 3u);
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

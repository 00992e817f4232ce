// sbx_step_static: one explicit step on caller-owned device arrays that
// allocates nothing.  Its only working memory, the global internal-force
// accumulator, is a file-scope static device array (SBX_STATIC_MAX_DOF
// doubles, declared in include/sbx.h), which every GPU that loads this
// library holds until the process exits.
//
// Host code may not hand `g_static_force` itself to a kernel: in host code
// that name is only a host-side stand-in for the device symbol.  The device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and cached, beside the device's SM count; the first call
// on each device does this and should therefore come before any stream
// capture.  The cache assumes the device's primary context lives as long as
// the process: after a cudaDeviceReset the cached address is stale, and the
// caller must not use this entry point again in that process.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "../../include/sbx.h"

namespace {

constexpr int TC = 32;            // cells per CTA
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_static_force[SBX_STATIC_MAX_DOF];

__constant__ int8_t c_perm_s[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                      {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct PatternTable {
  int n;                           // patterns
  int32_t m[SBX_STATIC_MAX_PATTERNS];
  int64_t cstart[SBX_STATIC_MAX_PATTERNS];   // first cell of the pattern
  int64_t ccount[SBX_STATIC_MAX_PATTERNS];
  int64_t koff[SBX_STATIC_MAX_PATTERNS];     // offset of K_p in K_packed
  int64_t coff[SBX_STATIC_MAX_PATTERNS];     // offset of the pattern's conn block
  int32_t tile0[SBX_STATIC_MAX_PATTERNS + 1];  // first CTA of the pattern
};

// FP64 internal force of TC cells of one pattern, accumulated into f.
__global__ void __launch_bounds__(256) k_force_static(const PatternTable T, const double *K,
                                                      const int32_t *conn, const uint8_t *sym,
                                                      const double *scale, const double *u,
                                                      double *f) {
  int p = 0;
  while (p + 1 < T.n && (int)blockIdx.x >= T.tile0[p + 1]) ++p;
  const int m = T.m[p], n = m / 3;
  const int64_t Cp = T.ccount[p];
  const int64_t c0 = (int64_t)(blockIdx.x - T.tile0[p]) * TC;
  const int nc = (Cp - c0 < TC) ? (int)(Cp - c0) : TC;
  extern __shared__ __align__(16) unsigned char sm[];
  double *Ks = reinterpret_cast<double *>(sm);
  double *Us = Ks + m * m;
  int32_t *Ns = reinterpret_cast<int32_t *>(Us + m * TC);
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Ks[i] = K[T.koff[p] + i];
  const int32_t *cn = conn + T.coff[p];
  const int64_t g0 = T.cstart[p] + c0;
  for (int idx = threadIdx.x; idx < n * TC; idx += blockDim.x) {
    const int k = idx / TC, c = idx % TC;
    if (c < nc) {
      const int32_t node = cn[(int64_t)k * Cp + c0 + c];
      const int op = sym[g0 + c];
      for (int r = 0; r < 3; ++r) {
        const double s = ((op >> r) & 1) ? -1.0 : 1.0;
        Us[(3 * k + r) * TC + c] = s * u[3 * (int64_t)node + c_perm_s[op >> 3][r]];
      }
      Ns[k * TC + c] = node;
    }
  }
  __syncthreads();
  const int c = threadIdx.x % TC;
  if (c < nc) {
    const double s = scale[g0 + c];
    const int op = sym[g0 + c];
    for (int i = threadIdx.x / TC; i < m; i += blockDim.x / TC) {
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc = fma(Ks[i * m + j], Us[j * TC + c], acc);
      const int k = i / 3, r = i % 3;
      const double sg = ((op >> r) & 1) ? -1.0 : 1.0;
      atomicAdd(&f[3 * (int64_t)Ns[k * TC + c] + c_perm_s[op >> 3][r]], sg * s * acc);
    }
  }
}

// U_{n+1} = -dt^2 minv f + 2 U_n - U_{n-1}, written over U_{n-1}.
__global__ void k_update_static(int64_t nd, const double *minv, const double *f, const double *un,
                                double *unm1, double dt2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    unm1[i] = -dt2 * minv[i] * f[i] + 2.0 * un[i] - unm1[i];
}

std::mutex g_mu;
double *g_addr[MAX_DEVICES] = {};   // device address of g_static_force, per device
int g_sms[MAX_DEVICES] = {};        // multiprocessors of the device

int scratch_address(int dev, double **out, int *sms) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sm < 1) {
      cudaGetLastError();
      return SBX_ECUDA;
    }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_force) != cudaSuccess) {
      cudaGetLastError();
      return SBX_ECUDA;
    }
    const size_t smem = (size_t)(78 * 78 + 78 * TC) * 8 + 26 * TC * 4;
    if (cudaFuncSetAttribute(k_force_static, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return SBX_ECUDA;
    }
    g_sms[dev] = n_sm;
    g_addr[dev] = static_cast<double *>(p);
  }
  *out = g_addr[dev];
  *sms = g_sms[dev];
  return SBX_OK;
}

}  // namespace

extern "C" int sbx_step_static(void *cuda_stream, int64_t n_dof, int n_patterns,
                               const int32_t *pat_nodes, const int64_t *pat_cells,
                               const double *K_packed, const int32_t *conn, const uint8_t *sym,
                               const double *scale, const double *minv, double dt,
                               const double *u_n, double *u_nm1) {
  if (n_dof < 3 || n_dof % 3 != 0 || n_dof > SBX_STATIC_MAX_DOF) return SBX_EINVAL;
  if (n_patterns < 1 || n_patterns > SBX_STATIC_MAX_PATTERNS || !pat_nodes || !pat_cells)
    return SBX_EINVAL;
  if (!K_packed || !conn || !sym || !scale || !minv || !u_n || !u_nm1 || !(dt > 0))
    return SBX_EINVAL;
  PatternTable T;
  T.n = n_patterns;
  int64_t cells = 0, ko = 0, co = 0, tiles = 0;
  int max_m = 0;
  for (int p = 0; p < n_patterns; ++p) {
    if (pat_nodes[p] < 8 || pat_nodes[p] > 26 || pat_cells[p] < 0) return SBX_EINVAL;
    T.m[p] = 3 * pat_nodes[p];
    T.cstart[p] = cells;
    T.ccount[p] = pat_cells[p];
    T.koff[p] = ko;
    T.coff[p] = co;
    T.tile0[p] = (int32_t)tiles;
    cells += pat_cells[p];
    ko += (int64_t)T.m[p] * T.m[p];
    co += (int64_t)pat_nodes[p] * pat_cells[p];
    tiles += (pat_cells[p] + TC - 1) / TC;
    if (pat_cells[p] > 0 && T.m[p] > max_m) max_m = T.m[p];
    if (tiles > INT32_MAX / 2) return SBX_EINVAL;
  }
  T.tile0[n_patterns] = (int32_t)tiles;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return SBX_ECUDA;
  }
  double *f = nullptr;
  int n_sm = 0;
  if (int rc = scratch_address(dev, &f, &n_sm)) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(f, 0, (size_t)n_dof * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return SBX_ECUDA;
  }
  if (tiles > 0) {
    const size_t smem = (size_t)(max_m * max_m + max_m * TC) * 8 + (size_t)(max_m / 3) * TC * 4;
    k_force_static<<<(unsigned)tiles, 256, smem, s>>>(T, K_packed, conn, sym, scale, u_n, f);
  }
  int blocks = (int)((n_dof + 255) / 256);
  if (blocks > n_sm * 8) blocks = n_sm * 8;
  k_update_static<<<blocks, 256, 0, s>>>(n_dof, minv, f, u_n, u_nm1, dt * dt);
  if (cudaGetLastError() != cudaSuccess) return SBX_ECUDA;
  return SBX_OK;
}

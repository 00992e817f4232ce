// Kernels of the discrete adjoint of the undamped explicit step.
//
// Forward: U_{n+1} = 2 U_n - U_{n-1} - W (K U_n - R_ext(t_n)), W = dt^2 M^-1.
// Misfit J = 1/2 sum_{n>=1} sum_r (U_n[r] - d_n[r])^2 at receiver DOFs r.
// Adjoint: lambda_n = g_n + 2 lambda_{n+1} - K (W lambda_{n+1}) - lambda_{n+2},
// g_n = U_n[r] - d_n[r] at the receivers; K W = (W K)^T since K is symmetric.
// Gradient: dJ/dE_e = -h_e sum_{n=0}^{N-1} (W lambda_{n+1})_e^T T^T K_p T U_{n,e}.
// K (W lambda) reuses the force kernel (loads off); the kernels here are the
// element-wise parts and the per-cell sum v_e^T K_p u_e.
#include <math.h>

#include "device_common.cuh"
#include "sbx_internal.cuh"

namespace sbx {
namespace {

int grid_for(const sbx_ctx *ctx, int64_t n) {
  const int64_t g = (n + 255) / 256, cap = (int64_t)ctx->n_sm * 8;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

__global__ void k_weight(int64_t nd, const double *w, const double *lam, double *v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * lam[i];
}

// lambda_n = 2 lambda_{n+1} - f - lambda_{n+2}, written over lambda_{n+2}
__global__ void k_adj_update(int64_t nd, const double *f, const double *lam1, double *lam2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    lam2[i] = fma(2.0, lam1[i], -f[i]) - lam2[i];
}

// lambda_n[r] += U_n[r] - d_n[r];  J += 1/2 (U_n[r] - d_n[r])^2
__global__ void k_residual(int64_t n_rec, const int64_t *rec, const double *u, const double *d,
                           double *lam, double *J) {
  double part = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rec;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r = u[rec[i]] - d[i];
    atomicAdd(&lam[rec[i]], r);   // receivers may repeat a DOF
    part += 0.5 * r * r;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(J, part);
}

// acc[e] += v_e^T K_p u_e (master frame, unit K_p) for the cells of a tile
// of up to 32 cells of one pattern.  T = float: u minus its per-cell mean
// translation (FP64) and v rounded to FP32, FP32 contraction; T = double:
// FP64 throughout.  The per-cell sums are combined in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_grad(const Tile *__restrict__ tiles, MeshView M,
                                              const T *__restrict__ Kp,
                                              const double *__restrict__ u,
                                              const double *__restrict__ v,
                                              double *__restrict__ acc) {
  constexpr int TC = SIMT_TILE;
  const Tile t = tiles[blockIdx.x];
  const int p = t.pat, m = M.pat_m[p], n = m / 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *part = reinterpret_cast<double *>(smem_raw);                // [8][TC]
  double *mean = part + 8 * TC;                                      // [3][TC]
  T *Ks = reinterpret_cast<T *>(mean + 3 * TC);
  T *Us = Ks + m * m;
  T *Vs = Us + m * TC;
  const T *Kg = Kp + M.koff[p];
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Ks[i] = Kg[i];
  const int64_t Cp = M.pat_ccount[p];
  const int32_t *cn = M.conn + M.conn_off[p];
  const int64_t gbase = M.pat_cstart[p] + t.cell0;
  const int nc = t.ncell;
  for (int idx = threadIdx.x; idx < 3 * TC; idx += blockDim.x) mean[idx] = 0.0;
  __syncthreads();
  if constexpr (sizeof(T) == 4) {   // per-cell mean translation of u (master frame)
    for (int idx = threadIdx.x; idx < 3 * TC; idx += blockDim.x) {
      const int r = idx / TC, c = idx % TC;
      if (c >= nc) continue;
      const int op = M.sym[gbase + c];
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        s += u[3 * (int64_t)cn[(int64_t)k * Cp + t.cell0 + c] + op_perm_of(op, r)];
      mean[r * TC + c] = (((op >> r) & 1) ? -s : s) / n;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * TC; idx += blockDim.x) {
    const int k = idx / TC, c = idx % TC;
    if (c >= nc) continue;
    const int64_t node = cn[(int64_t)k * Cp + t.cell0 + c];
    const int op = M.sym[gbase + c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int a = op_perm_of(op, r);
      const double sg = ((op >> r) & 1) ? -1.0 : 1.0;
      Us[(3 * k + r) * TC + c] = (T)(sg * u[3 * node + a] - mean[r * TC + c]);
      Vs[(3 * k + r) * TC + c] = (T)(sg * v[3 * node + a]);
    }
  }
  __syncthreads();
  const int c = threadIdx.x % TC, g = threadIdx.x / TC, G = blockDim.x / TC;
  double dot = 0.0;
  if (c < nc) {
    for (int i = g; i < m; i += G) {
      T a = 0;
      const T *Kr = Ks + i * m;
      for (int j = 0; j < m; ++j) a = fma(Kr[j], Us[j * TC + c], a);
      dot += (double)a * (double)Vs[i * TC + c];
    }
  }
  part[g * TC + c] = dot;
  __syncthreads();
  if (g == 0 && c < nc) {
    double s = 0.0;
    for (int q = 0; q < G; ++q) s += part[q * TC + c];
    acc[gbase + c] += s;
  }
}

size_t grad_smem(int m, bool fp32) {
  const size_t T = fp32 ? 4 : 8;
  return (size_t)(8 + 3) * SIMT_TILE * 8 + (size_t)(m * m + 2 * m * SIMT_TILE) * T;
}

}  // namespace

cudaError_t launch_weight(const sbx_ctx *ctx, const double *lam, double *v, cudaStream_t s) {
  k_weight<<<grid_for(ctx, ctx->ndof), 256, 0, s>>>(ctx->ndof, ctx->d_w, lam, v);
  return cudaGetLastError();
}

cudaError_t launch_adj_update(const sbx_ctx *ctx, const double *f, const double *lam1,
                              double *lam2_to_lam, cudaStream_t s) {
  k_adj_update<<<grid_for(ctx, ctx->ndof), 256, 0, s>>>(ctx->ndof, f, lam1, lam2_to_lam);
  return cudaGetLastError();
}

cudaError_t launch_residual(const sbx_ctx *ctx, int64_t n_rec, const int64_t *rec,
                            const double *u_n, const double *data_n, double *lam, double *J,
                            cudaStream_t s) {
  if (n_rec == 0) return cudaSuccess;
  (void)ctx;
  k_residual<<<grid_for(ctx, n_rec), 256, 0, s>>>(n_rec, rec, u_n, data_n, lam, J);
  return cudaGetLastError();
}

cudaError_t launch_grad(const sbx_ctx *ctx, const double *u, const double *v, double *acc,
                        cudaStream_t s) {
  if (ctx->n_tiles_simt == 0) return cudaSuccess;
  const bool fp32 = ctx->prec == SBX_PREC_FP32;
  const size_t smem = grad_smem(ctx->max_m, fp32);
  if (fp32)
    k_grad<float><<<ctx->n_tiles_simt, 256, smem, s>>>(ctx->d_tiles_simt, ctx->view(), ctx->d_K32,
                                                       u, v, acc);
  else
    k_grad<double><<<ctx->n_tiles_simt, 256, smem, s>>>(ctx->d_tiles_simt, ctx->view(), ctx->d_K64,
                                                        u, v, acc);
  return cudaGetLastError();
}

cudaError_t prepare_adjoint_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_grad<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)grad_smem(78, true));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_grad<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)grad_smem(78, false));
}

}  // namespace sbx

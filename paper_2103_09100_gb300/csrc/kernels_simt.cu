// SIMT kernels of the explicit step: element-by-element internal force
// (gather -> K_p contraction -> signed-permutation scatter), the lumped-mass
// central-difference update and the start-up of Eq. (D0).
//
// Internal force (Eqs. Rinte, Rintep): for each cell e of pattern p,
//   u_m = T_e u_e            (node order already in master order; component
//                             permutation and signs of the cell's op)
//   f_m = s_e K_p u_m        (s_e = E_e h_e, Eq. KM_scale)
//   R_int[V_e] += T_e^T f_m  (Sec. 3.2.2: back-transform with Q^-1 = Q^T)
// One CTA handles a tile of up to SIMT_TILE cells of one pattern; K_p and
// the gathered displacements live in shared memory; every thread owns one
// cell and a strided subset of K_p's rows, so a warp reads one K_p entry as
// a broadcast and 32 distinct displacement entries.
#include <math.h>

#include <algorithm>

#include "device_common.cuh"
#include "sbx_internal.cuh"
#include "tc_ptx.cuh"

namespace sbx {

__constant__ int8_t c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                    {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

__device__ __forceinline__ int op_perm(int op, int r) { return c_perm[op >> 3][r]; }
__device__ __forceinline__ double op_sign(int op, int r) { return ((op >> r) & 1) ? -1.0 : 1.0; }

// Time functions of Sec. 5: Eqs. (Ricker), (Triangle), (Lamb).
__device__ double wavelet(int kind, double t, double t1, double ncyc) {
  if (kind == SBX_WAVE_RICKER) {
    double tau = (t - t1) / (t1 / 5.0);
    return (1.0 - tau * tau) * exp(-0.5 * tau * tau);
  } else if (kind == SBX_WAVE_TRIANGLE) {
    if (t < 0.0 || t > 2.0 * t1) return 0.0;
    return 1.0 - fabs(t / t1 - 1.0);
  } else {
    if (t < 0.0 || t > t1) return 0.0;
    double s = sin(M_PI * t / t1);
    return sin(2.0 * M_PI * ncyc * t / t1) * s * s;
  }
}

// f -= R_ext(t_n): called by one CTA of the force kernel.
__device__ void add_external(const LoadTable L, const int64_t *d_step, double dt, double *f) {
  if (L.n == 0) return;
  double t = (double)(*d_step) * dt;
  for (int l = threadIdx.x; l < L.n; l += blockDim.x)
    atomicAdd(&f[L.dof[l]], -L.amp[l] * wavelet(L.kind[l], t, L.t1[l], L.ncyc[l]));
}

// T = double: FP64 DFMA contraction.
// T = float : the gathered displacement minus its per-cell mean translation
//             (computed in FP64; K_p annihilates translations) is rounded to
//             FP32 and contracted with FP32 K_p in FFMA; the result is scaled
//             by s_e and accumulated in FP64.
template <typename T, int TC>
__global__ void __launch_bounds__(256) k_force_simt(const Tile *__restrict__ tiles, MeshView M,
                                                    const T *__restrict__ Kp,
                                                    const double *__restrict__ u,
                                                    double *__restrict__ f, LoadTable L,
                                                    const int64_t *__restrict__ d_step, double dt) {
  const Tile t = tiles[blockIdx.x];
  const int p = t.pat;
  const int m = M.pat_m[p];
  const int n = m / 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ks = reinterpret_cast<T *>(smem_raw);
  T *Us = Ks + m * m;
  int32_t *Ns = reinterpret_cast<int32_t *>(Us + m * TC);
  const T *Kg = Kp + M.koff[p];
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Ks[i] = Kg[i];

  const int64_t Cp = M.pat_ccount[p];
  const int32_t *cn = M.conn + M.conn_off[p];
  const int64_t gbase = M.pat_cstart[p] + t.cell0;
  const int nc = t.ncell;

  if constexpr (sizeof(T) == 8) {
    for (int idx = threadIdx.x; idx < n * TC; idx += blockDim.x) {
      const int k = idx / TC, c = idx % TC;
      if (c < nc) {
        const int32_t node = cn[(int64_t)k * Cp + t.cell0 + c];
        const int op = M.sym[gbase + c];
        const double *un = u + 3 * (int64_t)node;
        const double v[3] = {un[0], un[1], un[2]};
#pragma unroll
        for (int r = 0; r < 3; ++r) Us[(3 * k + r) * TC + c] = op_sign(op, r) * v[op_perm(op, r)];
        Ns[k * TC + c] = node;
      }
    }
    __syncthreads();
  } else {
    // FP32 path: gather in FP64 into a scratch area that aliases nothing
    // else (placed after Ns), take the per-cell mean, then round.
    double *Ud = reinterpret_cast<double *>(
        smem_raw + (((size_t)(m * m + m * TC) * sizeof(T) + (size_t)n * TC * 4 + 15) & ~(size_t)15));
    double *mean = Ud + m * TC;
    for (int idx = threadIdx.x; idx < n * TC; idx += blockDim.x) {
      const int k = idx / TC, c = idx % TC;
      if (c < nc) {
        const int32_t node = cn[(int64_t)k * Cp + t.cell0 + c];
        const int op = M.sym[gbase + c];
        const double *un = u + 3 * (int64_t)node;
        const double v[3] = {un[0], un[1], un[2]};
#pragma unroll
        for (int r = 0; r < 3; ++r) Ud[(3 * k + r) * TC + c] = op_sign(op, r) * v[op_perm(op, r)];
        Ns[k * TC + c] = node;
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 3 * TC; idx += blockDim.x) {
      const int r = idx / TC, c = idx % TC;
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += Ud[(3 * k + r) * TC + c];
      mean[r * TC + c] = s / n;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * TC; idx += blockDim.x) {
      const int i = idx / TC, c = idx % TC;
      Us[idx] = (T)(Ud[idx] - mean[(i % 3) * TC + c]);
    }
    __syncthreads();
  }

  const int c = threadIdx.x % TC;
  const int G = blockDim.x / TC;
  if (c < nc) {
    const double s = M.scale[gbase + c];
    const int op = M.sym[gbase + c];
    for (int i = threadIdx.x / TC; i < m; i += G) {
      T acc = 0;
      const T *Kr = Ks + i * m;
      for (int j = 0; j < m; ++j) acc = fma(Kr[j], Us[j * TC + c], acc);
      const int k = i / 3, r = i - 3 * (i / 3);
      atomicAdd(&f[3 * (int64_t)Ns[k * TC + c] + op_perm(op, r)], op_sign(op, r) * s * (double)acc);
    }
  }
  if (blockIdx.x == 0) add_external(L, d_step, dt, f);
}

// In-place Walsh-Hadamard transform of 8 values: x[p] <- sum_n (-1)^popcount(p & n) x[n].
__device__ __forceinline__ void wht8(double *x) {
#pragma unroll
  for (int h = 1; h < 8; h <<= 1)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if ((i & h) == 0) {
        const double a = x[i], b = x[i + h];
        x[i] = a + b;
        x[i + h] = a - b;
      }
}

// FP64 internal force of the 8-node cells with the identity op, one thread
// per cell: the nodal values of each component r are Walsh-transformed over
// the corners (n = a + 2 b + 4 c), block s of the transformed K_p couples
// the components' values at indices s ^ 1, s ^ 2, s ^ 4, and the result is
// transformed back (the transform is its own transpose; T T^T = 8 I).  216
// FP64 operations per cell instead of 576 FMAs, same products to rounding.
__global__ void __launch_bounds__(128) k_force_wht(MeshView M, int p, int64_t nc,
                                                   WhtBlocks Kh, const double *__restrict__ u,
                                                   double *__restrict__ f, LoadTable L,
                                                   const int64_t *__restrict__ d_step, double dt) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c < nc) {
    const int32_t *cn = M.conn + M.conn_off[p] + c;
    int32_t node[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) node[k] = cn[(int64_t)k * nc];
    double x[3][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double *un = u + 3 * (int64_t)node[k];
      x[0][k] = un[0];
      x[1][k] = un[1];
      x[2][k] = un[2];
    }
    wht8(x[0]);
    wht8(x[1]);
    wht8(x[2]);
    double y[3][8];
#pragma unroll
    for (int sb = 0; sb < 8; ++sb) {
      const double *B = Kh.blk + 9 * sb;
      const double v0 = x[0][sb ^ 1], v1 = x[1][sb ^ 2], v2 = x[2][sb ^ 4];
      y[0][sb ^ 1] = fma(B[0], v0, fma(B[1], v1, B[2] * v2));
      y[1][sb ^ 2] = fma(B[3], v0, fma(B[4], v1, B[5] * v2));
      y[2][sb ^ 4] = fma(B[6], v0, fma(B[7], v1, B[8] * v2));
    }
    wht8(y[0]);
    wht8(y[1]);
    wht8(y[2]);
    const double sc = M.scale[M.pat_cstart[p] + c] * 0.125;
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int r = 0; r < 3; ++r) atomicAdd(&f[3 * (int64_t)node[k] + r], sc * y[r][k]);
  }
  if (blockIdx.x == 0) add_external(L, d_step, dt, f);
}

static size_t simt_smem(int m, bool fp32) {
  const int n = m / 3, TC = SIMT_TILE;
  size_t T = fp32 ? 4 : 8;
  size_t b = (size_t)(m * m + m * TC) * T + (size_t)n * TC * 4;
  if (fp32) b = ((b + 15) & ~(size_t)15) + (size_t)(m * TC + 3 * TC) * 8;
  return b;
}

cudaError_t launch_force_simt(const sbx_ctx *ctx, const double *u, double *f, double dt,
                              cudaStream_t s, bool with_loads) {
  const bool fp32 = ctx->prec == SBX_PREC_FP32;
  const size_t smem = simt_smem(ctx->max_m, fp32);
  if (ctx->n_tiles_simt == 0) return cudaSuccess;
  LoadTable L = ctx->loads();
  if (!with_loads) L.n = 0;
  if (fp32) {
    auto k = k_force_simt<float, SIMT_TILE>;
    k<<<ctx->n_tiles_simt, 256, smem, s>>>(ctx->d_tiles_simt, ctx->view(), ctx->d_K32, u, f, L,
                                           ctx->d_step, dt);
  } else if (ctx->wht_pat >= 0) {
    const int grid = (int)((ctx->wht_cells + 127) / 128);
    k_force_wht<<<grid, 128, 0, s>>>(ctx->view(), ctx->wht_pat, ctx->wht_cells, ctx->wht, u, f, L,
                                     ctx->d_step, dt);
    L.n = 0;
    if (ctx->n_tiles_rest > 0) {
      auto k = k_force_simt<double, SIMT_TILE>;
      k<<<ctx->n_tiles_rest, 256, smem, s>>>(ctx->d_tiles_rest, ctx->view(), ctx->d_K64, u, f, L,
                                             ctx->d_step, dt);
    }
  } else {
    auto k = k_force_simt<double, SIMT_TILE>;
    k<<<ctx->n_tiles_simt, 256, smem, s>>>(ctx->d_tiles_simt, ctx->view(), ctx->d_K64, u, f, L,
                                           ctx->d_step, dt);
  }
  return cudaGetLastError();
}

static cudaError_t prepare_update_kernels();

cudaError_t prepare_kernels() {
  if (const cudaError_t e0 = prepare_update_kernels()) return e0;
  const int a = (int)simt_smem(78, false), b = (int)simt_smem(78, true);
  cudaError_t e = cudaFuncSetAttribute(k_force_simt<double, SIMT_TILE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, a);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_force_simt<float, SIMT_TILE>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

// ------------------------------------------------------------------ update
// Eq. (DnMdiag) with f = R_int - R_ext and w = dt^2 M^-1 / (1 + a dt/2):
//   U_{n+1} = -w f + (2 U_n - (1 - a dt/2) U_{n-1}) / (1 + a dt/2),
// written over U_{n-1}.  Undamped: two FP64 FMAs per DOF (GB300's FP64 pipe
// runs at ~1/64 of FP32, so the update is kept at the minimum FP64 work).
// f is reset to zero for the next step (unless the caller keeps it for
// read-back).  Thread 0 advances the device step index.
__device__ __forceinline__ bool nonfinite(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF;
}

template <bool DAMPED>
__device__ __forceinline__ double cdm_update(double w, double f, double uc, double up, double a,
                                             double b) {
  if (DAMPED) return fma(-w, f, fma(a, uc, -b * up));
  return fma(-w, f, fma(2.0, uc, -up));
}

template <bool DAMPED>
__global__ void __launch_bounds__(256) k_update(int64_t nd, const double *__restrict__ w,
                                                double *__restrict__ f,
                                                const double *__restrict__ uc,
                                                double *__restrict__ up, double a, double b,
                                                int zero_f, int32_t *flags, int64_t *d_step) {
  bool bad = false;
  const int64_t n2 = nd / 2;
  const double2 *f2 = reinterpret_cast<const double2 *>(f);
  const double2 *w2 = reinterpret_cast<const double2 *>(w);
  const double2 *c2 = reinterpret_cast<const double2 *>(uc);
  double2 *p2 = reinterpret_cast<double2 *>(up);
  double2 *fz = reinterpret_cast<double2 *>(f);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 fv = f2[i], wv = w2[i], cv = c2[i], pv = p2[i];
    double2 r;
    r.x = cdm_update<DAMPED>(wv.x, fv.x, cv.x, pv.x, a, b);
    r.y = cdm_update<DAMPED>(wv.y, fv.y, cv.y, pv.y, a, b);
    bad |= nonfinite(r.x) || nonfinite(r.y);
    p2[i] = r;
    if (zero_f) fz[i] = make_double2(0.0, 0.0);
  }
  if ((nd & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t d = nd - 1;
    const double r = cdm_update<DAMPED>(w[d], f[d], uc[d], up[d], a, b);
    bad |= nonfinite(r);
    up[d] = r;
    if (zero_f) f[d] = 0.0;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_step += 1;
}

static int update_grid(const sbx_ctx *ctx, int64_t nd) {
  int64_t want = (nd / 2 + 255) / 256;
  int64_t cap = (int64_t)ctx->n_sm * 8;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Mixed form: f is float [N][4]; one thread per node.  FP32 -> FP64 by bit
// re-packing, and U_{n+1} split into FP32 (hi, lo) for the next force
// evaluation, with integer operations (both off the FP64 pipe).
__device__ __forceinline__ void put_pair(float *p, double x0, double x1, double x2) {
  float h0, h1, h2, l0, l1, l2;
  split_f64(x0, h0, l0);
  split_f64(x1, h1, l1);
  split_f64(x2, h2, l2);
  float2 *q = reinterpret_cast<float2 *>(p);   // 6 floats, 8-byte aligned
  q[0] = make_float2(h0, h1);
  q[1] = make_float2(h2, l0);
  q[2] = make_float2(l1, l2);
}
// the same, written with an L2 eviction priority
__device__ __forceinline__ void put_pair(float *p, double x0, double x1, double x2, uint64_t pol) {
  float h0, h1, h2, l0, l1, l2;
  split_f64(x0, h0, l0);
  split_f64(x1, h1, l1);
  split_f64(x2, h2, l2);
  float2 *q = reinterpret_cast<float2 *>(p);
  st_hint(q, make_float2(h0, h1), pol);
  st_hint(q + 1, make_float2(h2, l0), pol);
  st_hint(q + 2, make_float2(l1, l2), pol);
}

// UPD_U nodes per thread and round, all their loads issued before any
// arithmetic (the update is bound by memory latency x parallelism).
constexpr int UPD_U = 2;
template <bool DAMPED>
__global__ void __launch_bounds__(256) k_update_f32(int64_t nn, const double *__restrict__ w,
                                                    float4 *__restrict__ f,
                                                    const double *__restrict__ uc,
                                                    double *__restrict__ up,
                                                    float *__restrict__ pairs, double a, double b,
                                                    int zero_f, int32_t *flags, int64_t *d_step) {
  bool bad = false;
  const uint64_t stream = l2_evict_first(), keep = l2_evict_last();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < nn;
       i0 += UPD_U * stride) {
    float4 fv[UPD_U];
    double wv[UPD_U][3], cv[UPD_U][3], pv[UPD_U][3];
#pragma unroll
    for (int q = 0; q < UPD_U; ++q) {
      const int64_t i = i0 + q * stride < nn ? i0 + q * stride : i0;
      fv[q] = ld_hint(f + i, keep);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        wv[q][d] = ld_nc_hint(w + 3 * i + d, stream);
        cv[q][d] = ld_nc_hint(uc + 3 * i + d, stream);
        pv[q][d] = ld_hint(up + 3 * i + d, stream);
      }
    }
#pragma unroll
    for (int q = 0; q < UPD_U; ++q) {
      const int64_t i = i0 + q * stride;
      if (i >= nn) break;
      const double r0 = cdm_update<DAMPED>(wv[q][0], f2d_bits(fv[q].x), cv[q][0], pv[q][0], a, b);
      const double r1 = cdm_update<DAMPED>(wv[q][1], f2d_bits(fv[q].y), cv[q][1], pv[q][1], a, b);
      const double r2 = cdm_update<DAMPED>(wv[q][2], f2d_bits(fv[q].z), cv[q][2], pv[q][2], a, b);
      bad |= nonfinite(r0) || nonfinite(r1) || nonfinite(r2);
      st_hint(up + 3 * i, r0, stream);
      st_hint(up + 3 * i + 1, r1, stream);
      st_hint(up + 3 * i + 2, r2, stream);
      put_pair(pairs + 6 * i, r0, r1, r2, keep);
      if (zero_f) st_hint(f + i, make_float4(0.0f, 0.0f, 0.0f, 0.0f), keep);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_step += 1;
}

// The same update with the memory-level parallelism taken off the
// registers: each CTA streams chunks of UB_NODES nodes (their w, U_n and
// U_{n-1} rows and force rows) into shared memory by 1-D bulk copies,
// UB_STAGES chunks in flight, and updates a chunk with one thread per node.
// The update is bound by the FP64 pipe (2 DFMA per DOF, ~1 TFLOP/s on this
// GPU: ~14 us of pipe time per step on 3.4M DOF) as much as by HBM; small
// chunks, two stages and eight CTAs per SM overlapped the two best in a
// sweep of shapes (27.1 us against 28.1 for k_update_f32).
// The arithmetic is k_update_f32's (bit-identical results).  Every chunk
// but the last starts 16-byte aligned (UB_NODES even, 24-byte rows); an odd
// last node is read from global memory by its thread.  A wait that gives
// up sets flag bit 2 after the copies in flight have landed (bounded).
constexpr int UB_NODES = 128;
constexpr int UB_STAGES = 2;
constexpr uint32_t UB_ROWS = 24u * UB_NODES;                   // one array's rows per chunk
constexpr uint32_t UB_STAGE = 3u * UB_ROWS + 16u * UB_NODES;   // w, U_n, U_{n-1}, f
constexpr uint32_t UB_SMEM = 64u + UB_STAGES * UB_STAGE;
constexpr int UB_CTAS_PER_SM = 8;
constexpr uint32_t UB_WAIT_POLLS = 1u << 22;

template <bool DAMPED>
__global__ void __launch_bounds__(UB_NODES) k_update_f32_bulk(
    int64_t nn, const double *__restrict__ w, float4 *__restrict__ f,
    const double *__restrict__ uc, double *__restrict__ up, float *__restrict__ pairs, double a,
    double b, int zero_f, int32_t *flags, int64_t *d_step) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint64_t stream = l2_evict_first(), keep = l2_evict_last();
  const int tid = threadIdx.x;
  const int64_t nchunks = (nn + UB_NODES - 1) / UB_NODES, G = gridDim.x;
  const uint32_t mb0 = tc::smem_addr(smem);
  auto stage = [&](int s) { return smem + 64u + (uint32_t)s * UB_STAGE; };
  auto issue = [&](int s, int64_t c) {   // thread 0
    const int64_t n0 = c * UB_NODES;
    const int n = (int)(nn - n0 < UB_NODES ? nn - n0 : UB_NODES);
    const uint32_t rb = 24u * (uint32_t)(n & ~1), fb = 16u * (uint32_t)n;
    const uint32_t mb = mb0 + 8u * (uint32_t)s, d = tc::smem_addr(stage(s));
    tc::fence_proxy_async_smem();
    tc::mbar_arrive_expect_tx(mb, 3u * rb + fb);
    if (rb) {
      tc::bulk_g2s_hint(d, w + 3 * n0, rb, mb, stream);
      tc::bulk_g2s_hint(d + UB_ROWS, uc + 3 * n0, rb, mb, stream);
      tc::bulk_g2s_hint(d + 2u * UB_ROWS, up + 3 * n0, rb, mb, stream);
    }
    tc::bulk_g2s_hint(d + 3u * UB_ROWS, f + n0, fb, mb, keep);
  };
  uint32_t pend = 0u, ph = 0u;   // thread 0: stages with copies in flight, their phases
  if (tid == 0) {
    for (int s = 0; s < UB_STAGES; ++s) tc::mbar_init(mb0 + 8u * (uint32_t)s, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < UB_STAGES; ++s)
      if (blockIdx.x + s * G < nchunks) {
        issue(s, blockIdx.x + s * G);
        pend |= 1u << s;
      }
  bool bad = false, ok = true;
  int k = 0;
  for (int64_t c = blockIdx.x; c < nchunks; c += G, ++k) {
    const int s = k % UB_STAGES;
    const bool got =
        tc::mbar_wait_bounded(mb0 + 8u * (uint32_t)s, (uint32_t)(k / UB_STAGES) & 1u, UB_WAIT_POLLS);
    const int64_t n0 = c * UB_NODES;
    const int n = (int)(nn - n0 < UB_NODES ? nn - n0 : UB_NODES);
    if (got && tid < n) {
      const int64_t i = n0 + tid;
      const double *W = reinterpret_cast<const double *>(stage(s));
      const double *C = W + 3 * UB_NODES, *Pm = C + 3 * UB_NODES;
      const float4 fv = reinterpret_cast<const float4 *>(Pm + 3 * UB_NODES)[tid];
      double wv[3], cv[3], pv[3];
      if (tid < (n & ~1)) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          wv[d] = W[3 * tid + d];
          cv[d] = C[3 * tid + d];
          pv[d] = Pm[3 * tid + d];
        }
      } else {   // the odd last node
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          wv[d] = w[3 * i + d];
          cv[d] = uc[3 * i + d];
          pv[d] = up[3 * i + d];
        }
      }
      const double r0 = cdm_update<DAMPED>(wv[0], f2d_bits(fv.x), cv[0], pv[0], a, b);
      const double r1 = cdm_update<DAMPED>(wv[1], f2d_bits(fv.y), cv[1], pv[1], a, b);
      const double r2 = cdm_update<DAMPED>(wv[2], f2d_bits(fv.z), cv[2], pv[2], a, b);
      bad |= nonfinite(r0) || nonfinite(r1) || nonfinite(r2);
      st_hint(up + 3 * i, r0, stream);
      st_hint(up + 3 * i + 1, r1, stream);
      st_hint(up + 3 * i + 2, r2, stream);
      put_pair(pairs + 6 * i, r0, r1, r2, keep);
      if (zero_f) st_hint(f + i, make_float4(0.0f, 0.0f, 0.0f, 0.0f), keep);
    }
    ok = __syncthreads_and(got);   // also: every thread is done with stage s
    if (!ok) break;
    if (tid == 0) {
      ph ^= 1u << s;
      pend &= ~(1u << s);
      if (c + UB_STAGES * G < nchunks) {
        issue(s, c + UB_STAGES * G);
        pend |= 1u << s;
      }
    }
  }
  if (!ok && tid == 0) {   // let the copies in flight land before the CTA exits
    atomicOr(flags, 2);
    for (int s = 0; s < UB_STAGES; ++s)
      if (pend & (1u << s)) tc::mbar_wait_bounded(mb0 + 8u * (uint32_t)s, (ph >> s) & 1u, UB_WAIT_POLLS);
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(flags, 1);
  if (blockIdx.x == 0 && tid == 0) *d_step += 1;
}

static cudaError_t prepare_update_kernels() {
  for (const void *k : {(const void *)k_update_f32_bulk<false>, (const void *)k_update_f32_bulk<true>}) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, UB_SMEM);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

__global__ void k_split_flat(int64_t nv, const double *u, float2 *pairs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
       i += (int64_t)gridDim.x * blockDim.x) {
    float h, l;
    split_f64(u[i], h, l);
    pairs[i] = make_float2(h, l);
  }
}

__global__ void k_widen_flat(int64_t nv, const float *f, double *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = f2d_bits(f[i]);
}

__global__ void k_split_pairs(int64_t nn, const double *u, float *pairs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x)
    put_pair(pairs + 6 * i, u[3 * i], u[3 * i + 1], u[3 * i + 2]);
}

__global__ void k_widen_f32(int64_t nn, const float4 *f, double *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = f[i];
    out[3 * i] = f2d_bits(v.x);
    out[3 * i + 1] = f2d_bits(v.y);
    out[3 * i + 2] = f2d_bits(v.z);
  }
}

// Receiver time history: row = (device step index after the update) -
// step0 - 1, i.e. the step just taken; rows past the capacity are dropped.
__global__ void k_record(const int64_t *__restrict__ d_step, int64_t step0, int64_t cap,
                         int64_t n_rec, const int64_t *__restrict__ rec,
                         const double *__restrict__ u, double *__restrict__ hist) {
  const int64_t row = *d_step - step0 - 1;
  if (row < 0 || row >= cap) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rec;
       i += (int64_t)gridDim.x * blockDim.x)
    hist[row * n_rec + i] = u[rec[i]];
}

cudaError_t launch_record(const sbx_ctx *ctx, const double *u, cudaStream_t s) {
  if (ctx->n_rec_hist == 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((ctx->n_rec_hist + 255) / 256, ctx->n_sm);
  k_record<<<grid, 256, 0, s>>>(ctx->d_step, ctx->rec_step0, ctx->rec_cap, ctx->n_rec_hist,
                                ctx->d_rec_idx, u, ctx->d_hist);
  return cudaGetLastError();
}

__global__ void k_make_w(int64_t nd, const double *minv, double *w, double c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = c * minv[i];
}

cudaError_t prepare_update(sbx_ctx *ctx, double dt, double alpha, cudaStream_t s) {
  if (ctx->w_valid && ctx->w_dt == dt && ctx->w_alpha == alpha) return cudaSuccess;
  const int64_t nd = ctx->ndof;   // w is per DOF, shared by all load cases
  const double cp = 1.0 + 0.5 * alpha * dt;
  k_make_w<<<update_grid(ctx, nd), 256, 0, s>>>(nd, ctx->d_minv, ctx->d_w, dt * dt / cp);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    ctx->w_valid = true;
    ctx->w_dt = dt;
    ctx->w_alpha = alpha;
  }
  return e;
}

cudaError_t launch_update(const sbx_ctx *ctx, const double *uc, double *up, double *f, double dt,
                          double alpha, int zero_f, cudaStream_t s) {
  const int64_t nd = ctx->ndof * ctx->B;
  const double cm = 1.0 - 0.5 * alpha * dt, cp = 1.0 + 0.5 * alpha * dt;
  if (alpha == 0.0)
    k_update<false><<<update_grid(ctx, nd), 256, 0, s>>>(nd, ctx->d_w, f, uc, up, 2.0, 1.0, zero_f,
                                                    ctx->d_flags, ctx->d_step);
  else
    k_update<true><<<update_grid(ctx, nd), 256, 0, s>>>(nd, ctx->d_w, f, uc, up, 2.0 / cp, cm / cp,
                                                   zero_f, ctx->d_flags, ctx->d_step);
  return cudaGetLastError();
}

cudaError_t launch_update_f32(const sbx_ctx *ctx, const double *uc, double *up, float *f4,
                              float *pairs_out, double dt, double alpha, int zero_f,
                              cudaStream_t s) {
  const int64_t nn = ctx->N;
  const double cm = 1.0 - 0.5 * alpha * dt, cp = 1.0 + 0.5 * alpha * dt;
  float4 *f = reinterpret_cast<float4 *>(f4);
  auto a16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (ctx->update_bulk && a16(ctx->d_w) && a16(uc) && a16(up) && a16(f)) {
    const int64_t nchunks = (nn + UB_NODES - 1) / UB_NODES;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(nchunks, (int64_t)ctx->n_sm * UB_CTAS_PER_SM));
    if (alpha == 0.0)
      k_update_f32_bulk<false><<<grid, UB_NODES, UB_SMEM, s>>>(
          nn, ctx->d_w, f, uc, up, pairs_out, 2.0, 1.0, zero_f, ctx->d_flags, ctx->d_step);
    else
      k_update_f32_bulk<true><<<grid, UB_NODES, UB_SMEM, s>>>(
          nn, ctx->d_w, f, uc, up, pairs_out, 2.0 / cp, cm / cp, zero_f, ctx->d_flags,
          ctx->d_step);
    return cudaGetLastError();
  }
  if (alpha == 0.0)
    k_update_f32<false><<<update_grid(ctx, 2 * nn), 256, 0, s>>>(
        nn, ctx->d_w, f, uc, up, pairs_out, 2.0, 1.0, zero_f, ctx->d_flags, ctx->d_step);
  else
    k_update_f32<true><<<update_grid(ctx, 2 * nn), 256, 0, s>>>(
        nn, ctx->d_w, f, uc, up, pairs_out, 2.0 / cp, cm / cp, zero_f, ctx->d_flags,
        ctx->d_step);
  return cudaGetLastError();
}

cudaError_t launch_split_pairs(const sbx_ctx *ctx, const double *u, float *pairs, cudaStream_t s) {
  if (ctx->B > 1) {
    const int64_t nv = ctx->ndof * ctx->B;
    k_split_flat<<<update_grid(ctx, nv), 256, 0, s>>>(nv, u, reinterpret_cast<float2 *>(pairs));
  } else {
    k_split_pairs<<<update_grid(ctx, 2 * ctx->N), 256, 0, s>>>(ctx->N, u, pairs);
  }
  return cudaGetLastError();
}

cudaError_t launch_widen_f32(const sbx_ctx *ctx, const float *f4, double *out, cudaStream_t s) {
  if (ctx->B > 1) {
    const int64_t nv = ctx->ndof * ctx->B;
    k_widen_flat<<<update_grid(ctx, nv), 256, 0, s>>>(nv, f4, out);
  } else {
    k_widen_f32<<<update_grid(ctx, 2 * ctx->N), 256, 0, s>>>(
        ctx->N, reinterpret_cast<const float4 *>(f4), out);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- start-up
// Eq. (D0): U_-1 = U_0 - dt V_0 + dt^2/2 A_0 with A_0 = -M^-1 f - alpha V_0,
// f = K U_0 - R_ext(0).  Fixed DOFs (minv == 0) stay zero.
// Fields hold B load cases per DOF (entry DOF * B + case); minv is per DOF.
__global__ void k_init_um1(int64_t nd, int B, const double *minv, const double *u0,
                           const double *v0, double *um1, const double *f, double dt,
                           double alpha) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = v0 ? v0[i] : 0.0;
    const double mi = minv[i / B];
    if (mi == 0.0) {
      um1[i] = 0.0;
      continue;
    }
    const double acc = -mi * f[i] - alpha * v;
    um1[i] = u0[i] - dt * v + 0.5 * dt * dt * acc;
  }
}

cudaError_t launch_init_um1(const sbx_ctx *ctx, const double *u0, const double *v0, double *um1,
                            const double *f, double dt, double alpha, cudaStream_t s) {
  const int64_t nd = ctx->ndof * ctx->B;
  k_init_um1<<<update_grid(ctx, nd), 256, 0, s>>>(nd, ctx->B, ctx->d_minv, u0, v0, um1, f, dt, alpha);
  return cudaGetLastError();
}

__global__ void k_zero_fixed(int64_t nd, int B, const double *minv, double *u) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    if (minv[i / B] == 0.0) u[i] = 0.0;
}

cudaError_t launch_zero_fixed(const sbx_ctx *ctx, double *u, cudaStream_t s) {
  const int64_t nd = ctx->ndof * ctx->B;
  k_zero_fixed<<<update_grid(ctx, nd), 256, 0, s>>>(nd, ctx->B, ctx->d_minv, u);
  return cudaGetLastError();
}

}  // namespace sbx

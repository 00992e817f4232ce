// Lanczos iteration for the free vibration problem K x = omega^2 M x of an
// uploaded mesh (the cube example of Sec. 5 computes its eigenfrequencies
// with the K and lumped M the explicit solver steps with).  The operator
// A = W^1/2 K W^1/2, W = M^-1 (0 on the fixed DOFs), is symmetric positive
// semi-definite and vanishes outside the free DOFs; its eigenvalues there
// are omega^2.  K is applied by the FP64 element-by-element force kernel of
// the explicit step (loads off); the vector work (scalings, dot products,
// two classical Gram-Schmidt passes against every earlier Lanczos vector)
// is in the kernels below.  Nothing leaves the GPU inside the iteration:
// alpha_j, beta_j and the normalisation are read from device memory.
#include <math.h>

#include <algorithm>

#include "sbx_internal.cuh"

namespace sbx {
namespace {

constexpr int EIG_THREADS = 256;

// y = a * x (a = W^1/2: also zeroes the fixed DOFs)
__global__ void k_mul(int64_t n, const double *__restrict__ a, const double *__restrict__ x,
                      double *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] * x[i];
}

// a = sqrt(w) per DOF
__global__ void k_sqrt(int64_t n, const double *__restrict__ w, double *__restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = sqrt(w[i]);
}

// y = x where a != 0, else 0 (start vector restricted to the free DOFs)
__global__ void k_mask(int64_t n, const double *__restrict__ a, const double *__restrict__ x,
                       double *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] != 0.0 ? x[i] : 0.0;
}

// part[b ncol + c] = this block's share of sum_i Q[c ld + i] w[i]; eight
// columns per pass over w, one barrier per eight columns
constexpr int DOT_COLS = 8;
__global__ void k_dots(int64_t n, const double *__restrict__ Q, int64_t ld, int ncol,
                       const double *__restrict__ w, double *__restrict__ part) {
  __shared__ double red[EIG_THREADS / 32][DOT_COLS];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < ncol; c0 += DOT_COLS) {
    const int nc = ncol - c0 < DOT_COLS ? ncol - c0 : DOT_COLS;
    double s[DOT_COLS];
#pragma unroll
    for (int q = 0; q < DOT_COLS; ++q) s[q] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int q = 0; q < DOT_COLS; ++q)
        if (q < nc) s[q] = fma(Q[(int64_t)(c0 + q) * ld + i], wi, s[q]);
    }
#pragma unroll
    for (int q = 0; q < DOT_COLS; ++q)
      for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < DOT_COLS; ++q) red[wp][q] = s[q];
    __syncthreads();
    if (threadIdx.x < nc) {
      double t = 0.0;
      for (int v = 0; v < (int)(blockDim.x >> 5); ++v) t += red[v][threadIdx.x];
      part[(int64_t)blockIdx.x * ncol + c0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// out[c] = sum_b part[b ncol + c]
__global__ void k_reduce(int nb, int ncol, const double *__restrict__ part, double *__restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * ncol + c];
    out[c] = s;
  }
}

// w -= sum_c Q[c ld + i] h[c]
__global__ void k_gemv_sub(int64_t n, const double *__restrict__ Q, int64_t ld, int ncol,
                           const double *__restrict__ h, double *__restrict__ w) {
  extern __shared__ double hs[];
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) hs[c] = h[c];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int c = 0; c < ncol; ++c) s = fma(-Q[c * ld + i], hs[c], s);
    w[i] = s;
  }
}

// q = w / sqrt(nrm2) (0 once the Krylov space is exhausted)
__global__ void k_normalize(int64_t n, const double *__restrict__ w, const double *__restrict__ nrm2,
                            double *__restrict__ q) {
  const double r = *nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    q[i] = w[i] * r;
}

// alpha_j = (q_j . A q_j) from both passes, beta_j = |residual|
__global__ void k_coeff(int j, const double *__restrict__ h1, const double *__restrict__ h2,
                        const double *__restrict__ nrm2, double *__restrict__ alpha,
                        double *__restrict__ beta) {
  alpha[j] = h1[j] + h2[j];
  beta[j] = sqrt(fmax(*nrm2, 0.0));
}

}  // namespace

int lanczos_run(sbx_ctx *ctx, int64_t k, const double *v0_dev, double *alpha_dev,
                double *beta_dev, std::string &err) {
  const int64_t n = ctx->ndof;
  cudaStream_t s = ctx->stream;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + EIG_THREADS - 1) / EIG_THREADS,
                                                               (int64_t)ctx->n_sm * 8));
  double *Q = nullptr, *a = nullptr, *t = nullptr, *f = nullptr, *w = nullptr, *part = nullptr,
         *h1 = nullptr, *h2 = nullptr, *nrm = nullptr;
  auto cleanup = [&]() {
    for (double *p : {Q, a, t, f, w, part, h1, h2, nrm})
      if (p) cudaFree(p);
  };
  const size_t nb = (size_t)n * sizeof(double);
  if (cudaMalloc(&Q, (size_t)(k + 1) * nb) != cudaSuccess || cudaMalloc(&a, nb) != cudaSuccess ||
      cudaMalloc(&t, nb) != cudaSuccess || cudaMalloc(&f, nb) != cudaSuccess ||
      cudaMalloc(&w, nb) != cudaSuccess ||
      cudaMalloc(&part, (size_t)grid * (k + 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h1, (k + 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h2, (k + 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&nrm, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    err = "cudaMalloc failed (Lanczos vectors)";
    return SBX_ENOMEM;
  }
  auto dots = [&](const double *Qc, int ncol, const double *x, double *out) {
    k_dots<<<grid, EIG_THREADS, 0, s>>>(n, Qc, n, ncol, x, part);
    k_reduce<<<(ncol + 255) / 256, 256, 0, s>>>(grid, ncol, part, out);
  };
  // W^1/2 (W = M^-1, 0 on the fixed DOFs; dt = 1 in the weight)
  k_sqrt<<<grid, EIG_THREADS, 0, s>>>(n, ctx->d_minv, a);
  k_mask<<<grid, EIG_THREADS, 0, s>>>(n, a, v0_dev, w);
  dots(w, 1, w, nrm);
  k_normalize<<<grid, EIG_THREADS, 0, s>>>(n, w, nrm, Q);
  for (int64_t j = 0; j < k; ++j) {
    const double *qj = Q + j * n;
    const int ncol = (int)(j + 1);
    k_mul<<<grid, EIG_THREADS, 0, s>>>(n, a, qj, t);
    cudaMemsetAsync(f, 0, nb, s);
    cudaError_t e = launch_force_simt(ctx, t, f, 0.0, s, false);   // f = K t
    if (e != cudaSuccess) {
      cleanup();
      err = "K apply failed";
      return SBX_ECUDA;
    }
    k_mul<<<grid, EIG_THREADS, 0, s>>>(n, a, f, w);
    dots(Q, ncol, w, h1);
    k_gemv_sub<<<grid, EIG_THREADS, ncol * sizeof(double), s>>>(n, Q, n, ncol, h1, w);
    dots(Q, ncol, w, h2);
    k_gemv_sub<<<grid, EIG_THREADS, ncol * sizeof(double), s>>>(n, Q, n, ncol, h2, w);
    dots(w, 1, w, nrm);
    k_coeff<<<1, 1, 0, s>>>((int)j, h1, h2, nrm, alpha_dev, beta_dev);
    k_normalize<<<grid, EIG_THREADS, 0, s>>>(n, w, nrm, Q + (j + 1) * n);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) {
    err = std::string("Lanczos iteration failed: ") + cudaGetErrorString(e);
    return SBX_ECUDA;
  }
  return SBX_OK;
}

}  // namespace sbx

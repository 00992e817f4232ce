// Interface sum of the node-cut partition (Sec. 4.2), neighbour by
// neighbour: the pack of the force rows a part sends to its neighbours and
// the canonical sum of each cut node's partial forces.
//
// Rows follow the force accumulator's layout: FP64 forms 3 doubles per
// node (x, y, z), the mixed form 4 floats (x, y, z, unused; one 16-byte
// vector).  The sum starts from zero and adds a cut node's contributions in
// the order of the plan (the holding parts in ascending rank), so every
// holder of the node computes the same value bit for bit.
#include "sbx_internal.cuh"

namespace sbx {
namespace {

template <typename Row>
__global__ void k_halo_pack(int64_t n, const int64_t *__restrict__ idx, const Row *__restrict__ f,
                            Row *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = f[idx[i]];
}

struct D3 {
  double x, y, z;
};

__device__ __forceinline__ void add_row(D3 &a, const D3 &b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
}
__device__ __forceinline__ void add_row(float4 &a, const float4 &b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
}
__device__ __forceinline__ void zero_row(D3 &a) { a.x = a.y = a.z = 0.0; }
__device__ __forceinline__ void zero_row(float4 &a) { a = make_float4(0.0f, 0.0f, 0.0f, 0.0f); }

template <typename Row>
__global__ void k_halo_sum(int64_t n_cut, const int64_t *__restrict__ cut,
                           const int64_t *__restrict__ ptr, const int64_t *__restrict__ src,
                           const Row *__restrict__ recv, Row *__restrict__ f) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_cut;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = cut[j];
    const Row own = f[v];
    Row acc;
    zero_row(acc);
    for (int64_t q = ptr[j]; q < ptr[j + 1]; ++q) add_row(acc, src[q] < 0 ? own : recv[src[q]]);
    f[v] = acc;
  }
}

int grid_of(const sbx_ctx *ctx, int64_t n) {
  const int64_t g = (n + 255) / 256, cap = (int64_t)ctx->n_sm * 4;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_halo_pack(const sbx_ctx *ctx, void *out, cudaStream_t s) {
  const int64_t n = ctx->halo_n_send;
  if (n == 0) return cudaSuccess;
  if (ctx->prec == SBX_PREC_MIXED)
    k_halo_pack<float4><<<grid_of(ctx, n), 256, 0, s>>>(
        n, ctx->d_halo_send, reinterpret_cast<const float4 *>(ctx->d_f),
        reinterpret_cast<float4 *>(out));
  else
    k_halo_pack<D3><<<grid_of(ctx, n), 256, 0, s>>>(n, ctx->d_halo_send,
                                                    reinterpret_cast<const D3 *>(ctx->d_f),
                                                    reinterpret_cast<D3 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_halo_sum(const sbx_ctx *ctx, const void *recv, cudaStream_t s) {
  const int64_t n = ctx->halo_n_cut;
  if (n == 0) return cudaSuccess;
  if (ctx->prec == SBX_PREC_MIXED)
    k_halo_sum<float4><<<grid_of(ctx, n), 256, 0, s>>>(
        n, ctx->d_halo_cut, ctx->d_halo_ptr, ctx->d_halo_src,
        reinterpret_cast<const float4 *>(recv), reinterpret_cast<float4 *>(ctx->d_f));
  else
    k_halo_sum<D3><<<grid_of(ctx, n), 256, 0, s>>>(n, ctx->d_halo_cut, ctx->d_halo_ptr,
                                                   ctx->d_halo_src,
                                                   reinterpret_cast<const D3 *>(recv),
                                                   reinterpret_cast<D3 *>(ctx->d_f));
  return cudaGetLastError();
}

}  // namespace sbx

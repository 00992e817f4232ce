// Mixed-precision internal force on the 5th-generation tensor cores.
//
// Per CTA: one tile of up to 128 cells of one pattern p (m = 3 n_p DOFs).
//   1. The tile's unique nodes (host-sorted list) are gathered once into
//      shared memory (FP64); each (cell, slot) refers to them through a
//      16-bit local index, which replaces the 32-bit connectivity.
//   2. A (128 x K) = transformed cell displacements, each minus the
//      displacement of the cell's first node (K_p annihilates translations,
//      so the difference is exact in FP64 and only the deformation part is
//      rounded), split into TF32 hi + lo.
//   3. D (TMEM, 128 x N, FP32) = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T with
//      B = K_p split the same way (tcgen05.mma kind::tf32, issued by one
//      thread, completion through tcgen05.commit -> mbarrier).
//   4. Epilogue: tcgen05.ld rows of D (row = cell), scale by E_e h_e in FP64,
//      back-transform (Q^T), accumulate per unique node in shared memory
//      (FP64), then one global FP64 atomic per unique node DOF.
// Operands use the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices, row groups stored one after another (stride nK * 128 B), K groups
// 128 B apart inside a row group.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "sbx_internal.cuh"
#include "tc_ptx.cuh"

namespace sbx {

namespace {

constexpr uint32_t WAIT_POLLS = 1u << 22;

struct SmemLayout {
  uint32_t B, A, ucache, fnode, lidx, cell, total;
};

__host__ __device__ inline uint32_t align128(uint32_t x) { return (x + 127u) & ~127u; }

__host__ __device__ inline SmemLayout layout(int kmax, int nmax, int max_nodes, int nmax_nodes_cell) {
  SmemLayout L;
  uint32_t off = 128;                                   // mbarrier + TMEM address
  L.B = off;      off = align128(off + 2u * nmax * kmax * 4u);
  L.A = off;      off = align128(off + 2u * 128u * kmax * 4u);
  L.ucache = off; off = align128(off + (uint32_t)max_nodes * 24u);
  L.fnode = off;  off = align128(off + (uint32_t)max_nodes * 24u);
  L.lidx = off;   off = align128(off + (uint32_t)nmax_nodes_cell * 128u * 2u);
  L.cell = off;   off = align128(off + 128u * 8u + 128u);
  L.total = off;
  return L;
}

__global__ void __launch_bounds__(256, 1)
    k_force_tc(const TcTile *__restrict__ tiles, const TcPattern *__restrict__ pats,
               const int32_t *__restrict__ tile_nodes, const uint16_t *__restrict__ lidx,
               const float *__restrict__ Kc, const uint8_t *__restrict__ sym,
               const double *__restrict__ scale, const double *__restrict__ u,
               double *__restrict__ f, LoadTable Ld, const int64_t *__restrict__ d_step,
               double dt, int32_t *flags, int kmax, int nmax, int max_nodes, int nmax_nodes_cell) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemLayout SL = layout(kmax, nmax, max_nodes, nmax_nodes_cell);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(smem + 8);
  float *Bs = reinterpret_cast<float *>(smem + SL.B);
  float *As = reinterpret_cast<float *>(smem + SL.A);
  double *ucache = reinterpret_cast<double *>(smem + SL.ucache);
  double *fnode = reinterpret_cast<double *>(smem + SL.fnode);
  uint16_t *lid = reinterpret_cast<uint16_t *>(smem + SL.lidx);
  double *scale_s = reinterpret_cast<double *>(smem + SL.cell);
  uint8_t *sym_s = smem + SL.cell + 128 * 8;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcTile T = tiles[blockIdx.x];
  const TcPattern P = pats[T.pat];
  const int m = P.m, n = m / 3, kpad = P.kpad, npad = P.npad, nK = kpad / 4;
  const int ncell = T.ncell;
  const int64_t gbase = P.cstart + T.cell0;

  if (warp == 0) {
    tc::tmem_alloc(tc::smem_addr(taddr_s), (uint32_t)P.tcols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_addr(mbar), 1);
    tc::mbar_fence_init();
  }
  // B = K_p hi | lo, stored in canonical layout in global memory
  {
    const float4 *src = reinterpret_cast<const float4 *>(Kc + P.kc_off);
    float4 *dst = reinterpret_cast<float4 *>(Bs);
    const int nv = (2 * npad * kpad) / 4;
    for (int i = tid; i < nv; i += 256) dst[i] = src[i];
  }
  for (int c = tid; c < ncell; c += 256) {
    sym_s[c] = sym[gbase + c];
    scale_s[c] = scale[gbase + c];
  }
  for (int i = tid; i < T.n_nodes; i += 256) {
    const int64_t node = tile_nodes[T.node_off + i];
    ucache[3 * i + 0] = u[3 * node + 0];
    ucache[3 * i + 1] = u[3 * node + 1];
    ucache[3 * i + 2] = u[3 * node + 2];
    fnode[3 * i + 0] = 0.0;
    fnode[3 * i + 1] = 0.0;
    fnode[3 * i + 2] = 0.0;
  }
  for (int idx = tid; idx < n * 128; idx += 256) {
    const int k = idx >> 7, c = idx & 127;
    if (c < ncell) lid[idx] = lidx[P.lidx_off + (int64_t)k * P.ccount + T.cell0 + c];
  }
  __syncthreads();

  // A: row c, column 3k + r  ->  byte (c/8)*nK*128 + (col/4)*128 + (c%8)*16 + (col%4)*4
  float *Ahi = As, *Alo = As + 128 * kpad;
  for (int idx = tid; idx < n * 128; idx += 256) {
    const int k = idx >> 7, c = idx & 127;
    if (c >= ncell) continue;
    const int op = sym_s[c];
    const int li = lid[idx], l0 = lid[c];
    const int rowoff = (c >> 3) * nK * 32 + (c & 7) * 4;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int a = op_perm_of(op, r);
      const double sg = ((op >> r) & 1) ? -1.0 : 1.0;
      const float x = (float)(sg * (ucache[3 * li + a] - ucache[3 * l0 + a]));
      const float hi = tc::to_tf32(x);
      const float lo = tc::to_tf32(x - hi);
      const int col = 3 * k + r;
      const int off = rowoff + (col >> 2) * 32 + (col & 3);
      Ahi[off] = hi;
      Alo[off] = lo;
    }
  }
  for (int idx = tid; idx < (kpad - m) * 128; idx += 256) {   // zero K padding
    const int col = m + idx / 128, c = idx % 128;
    const int off = (c >> 3) * nK * 32 + (c & 7) * 4 + (col >> 2) * 32 + (col & 3);
    Ahi[off] = 0.0f;
    Alo[off] = 0.0f;
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *taddr_s;
  const uint32_t mbar_a = tc::smem_addr(mbar);

  if (tid == 0) {
    const uint32_t idesc = tc::idesc_tf32(128, npad);
    const uint32_t a_hi = tc::smem_addr(Ahi), a_lo = tc::smem_addr(Alo);
    const uint32_t b_hi = tc::smem_addr(Bs), b_lo = tc::smem_addr(Bs + npad * kpad);
    const uint32_t sbo = (uint32_t)nK * 128u;
    for (int s = 0; s < kpad / 8; ++s) {
      const uint32_t o = (uint32_t)s * 256u;
      const uint64_t ah = tc::smem_desc(a_hi + o, 128, sbo), al = tc::smem_desc(a_lo + o, 128, sbo);
      const uint64_t bh = tc::smem_desc(b_hi + o, 128, sbo), bl = tc::smem_desc(b_lo + o, 128, sbo);
      tc::mma_tf32(taddr, ah, bh, idesc, s > 0 ? 1u : 0u);
      tc::mma_tf32(taddr, ah, bl, idesc, 1u);
      tc::mma_tf32(taddr, al, bh, idesc, 1u);
    }
    tc::mma_commit(mbar_a);
  }
  bool ok = tc::mbar_wait_bounded(mbar_a, 0, WAIT_POLLS);
  ok = __syncthreads_and(ok);
  tc::fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicOr(flags, 2);
    tc::mbar_wait_bounded(mbar_a, 0, WAIT_POLLS);   // let in-flight MMAs drain
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)P.tcols);
    return;
  }

  // epilogue: D row = cell.  Warps w and w+4 share lanes 32*(w%4).. and
  // split the columns.  F (FP32, row stride npad+1) overwrites A.
  float *F = As;
  const int half = npad / 2;
  {
    const int c = 32 * (warp & 3) + lane;
    const int col0 = (warp >> 2) * half;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    for (int cc = col0; cc < col0 + half; cc += 8) {
      float v[8];
      tc::tmem_ld8(taddr + lane_base + (uint32_t)cc, v);
      tc::tmem_ld_wait();
      if (c < ncell) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (cc + i < m) F[c * (npad + 1) + cc + i] = v[i];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)P.tcols);

  for (int idx = tid; idx < n * 128; idx += 256) {
    const int k = idx >> 7, c = idx & 127;
    if (c >= ncell) continue;
    const int op = sym_s[c];
    const int li = lid[idx];
    const double s = scale_s[c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double sg = ((op >> r) & 1) ? -s : s;
      atomicAdd(&fnode[3 * li + op_perm_of(op, r)], sg * (double)F[c * (npad + 1) + 3 * k + r]);
    }
  }
  __syncthreads();
  for (int i = tid; i < T.n_nodes; i += 256) {
    const int64_t node = tile_nodes[T.node_off + i];
    atomicAdd(&f[3 * node + 0], fnode[3 * i + 0]);
    atomicAdd(&f[3 * node + 1], fnode[3 * i + 1]);
    atomicAdd(&f[3 * node + 2], fnode[3 * i + 2]);
  }
  if (blockIdx.x == 0 && Ld.n > 0) {
    const double t = (double)(*d_step) * dt;
    for (int l = tid; l < Ld.n; l += 256)
      atomicAdd(&f[Ld.dof[l]], -Ld.amp[l] * wavelet_value(Ld.kind[l], t, Ld.t1[l], Ld.ncyc[l]));
  }
}

float tf32_round_host(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  if ((b & 0x7F800000u) == 0x7F800000u) return x;
  b += 0x1000u;
  b &= ~0x1FFFu;
  float r;
  memcpy(&r, &b, 4);
  return r;
}

}  // namespace

// Host preparation of the tile lists, local indices and canonical K_p.
int tc_setup(sbx_ctx *ctx, const std::vector<int32_t> &conn, const std::vector<int64_t> &conn_off,
             const std::vector<int64_t> &cnt, const std::vector<int64_t> &start, std::string &err) {
  const int P = ctx->n_pat;
  std::vector<TcPattern> pats(P);
  std::vector<float> Kc;
  std::vector<uint16_t> lidx(std::max<size_t>(conn.size(), 1));
  std::vector<int32_t> nodes;
  // launch classes by the tile's own shared-memory need: <= 56 KB (4 CTAs
  // per SM), <= 113 KB (2 per SM), larger (1 per SM)
  std::vector<TcTile> tiles[TC_CLASSES];
  int kmax[TC_CLASSES], nmax[TC_CLASSES], maxn[TC_CLASSES], maxnc[TC_CLASSES];
  for (int c = 0; c < TC_CLASSES; ++c) {
    kmax[c] = 8;
    nmax[c] = 16;
    maxn[c] = 1;
    maxnc[c] = 8;
  }
  const uint32_t class_limit[TC_CLASSES] = {56u * 1024u, 113u * 1024u, 227u * 1024u};
  for (int p = 0; p < P; ++p) {
    const int np = ctx->pat_nodes[p], m = 3 * np;
    TcPattern &tp = pats[p];
    tp.m = m;
    tp.kpad = (m + 7) / 8 * 8;
    tp.npad = (m + 15) / 16 * 16;
    tp.tcols = tp.npad <= 32 ? 32 : (tp.npad <= 64 ? 64 : 128);
    tp.kc_off = (int64_t)Kc.size();
    tp.lidx_off = conn_off[p];
    tp.cstart = start[p];
    tp.ccount = cnt[p];
    const int nK = tp.kpad / 4;
    std::vector<float> B(2 * (size_t)tp.npad * tp.kpad, 0.0f);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double kv = ctx->K_host[ctx->pat_koff[p] + (int64_t)i * m + j];
        const float hi = tf32_round_host((float)kv);
        const float lo = tf32_round_host((float)(kv - (double)hi));
        const size_t off = (size_t)(i >> 3) * nK * 32 + (j >> 2) * 32 + (i & 7) * 4 + (j & 3);
        B[off] = hi;
        B[(size_t)tp.npad * tp.kpad + off] = lo;
      }
    Kc.insert(Kc.end(), B.begin(), B.end());
    if (cnt[p] == 0) continue;
    const int per = m <= 36 ? 128 : 64;
    std::vector<std::pair<int32_t, int32_t>> v;   // (node, k * C_p + j)
    for (int64_t c0 = 0; c0 < cnt[p]; c0 += per) {
      const int nc = (int)std::min<int64_t>(per, cnt[p] - c0);
      v.clear();
      for (int k = 0; k < np; ++k)
        for (int c = 0; c < nc; ++c) {
          const int64_t pos = (int64_t)k * cnt[p] + c0 + c;
          v.emplace_back(conn[conn_off[p] + pos], (int32_t)pos);
        }
      std::sort(v.begin(), v.end());
      TcTile t;
      t.pat = p;
      t.ncell = nc;
      t.cell0 = c0;
      t.node_off = (int64_t)nodes.size();
      int cntu = 0;
      for (size_t i = 0; i < v.size(); ++i) {
        if (i == 0 || v[i].first != v[i - 1].first) {
          nodes.push_back(v[i].first);
          ++cntu;
        }
        if (cntu - 1 > 65535) {
          err = "tile has more than 65536 unique nodes";
          return SBX_EINVAL;
        }
        lidx[conn_off[p] + v[i].second] = (uint16_t)(cntu - 1);
      }
      t.n_nodes = cntu;
      t.pad = 0;
      const uint32_t need = layout(tp.kpad, tp.npad, cntu, np).total;
      int cls = 0;
      while (cls < TC_CLASSES - 1 && need > class_limit[cls]) ++cls;
      if (need > class_limit[TC_CLASSES - 1]) {
        err = "tensor-core tile needs more than 227 KB of shared memory";
        return SBX_EINVAL;
      }
      kmax[cls] = std::max(kmax[cls], tp.kpad);
      nmax[cls] = std::max(nmax[cls], tp.npad);
      maxnc[cls] = std::max(maxnc[cls], np);
      maxn[cls] = std::max(maxn[cls], cntu);
      tiles[cls].push_back(t);
    }
  }
  auto up = [&](auto **dst, const auto &vec) -> int {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    size_t bytes = std::max<size_t>(vec.size(), 1) * sizeof(T);
    if (cudaMalloc((void **)dst, bytes) != cudaSuccess) {
      cudaGetLastError();
      err = "cudaMalloc failed (tensor-core tables)";
      return SBX_ENOMEM;
    }
    if (!vec.empty() &&
        cudaMemcpyAsync(*dst, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess) {
      err = "copy of tensor-core tables failed";
      return SBX_ECUDA;
    }
    return SBX_OK;
  };
  if (int rc = up(&ctx->d_tc_pat, pats)) return rc;
  if (int rc = up(&ctx->d_tc_K, Kc)) return rc;
  if (int rc = up(&ctx->d_tc_lidx, lidx)) return rc;
  if (int rc = up(&ctx->d_tc_nodes, nodes)) return rc;
  for (int cls = 0; cls < TC_CLASSES; ++cls) {
    if (int rc = up(&ctx->d_tc_tiles[cls], tiles[cls])) return rc;
    ctx->n_tc_tiles[cls] = (int)tiles[cls].size();
    ctx->tc_kmax[cls] = kmax[cls];
    ctx->tc_nmax[cls] = nmax[cls];
    ctx->tc_maxnodes[cls] = maxn[cls];
    ctx->tc_maxnc[cls] = maxnc[cls];
    ctx->tc_smem[cls] = layout(kmax[cls], nmax[cls], maxn[cls], maxnc[cls]).total;
    if (ctx->n_tc_tiles[cls] && ctx->tc_smem[cls] > 227 * 1024) {
      err = "tensor-core tile needs more than 227 KB of shared memory";
      return SBX_EINVAL;
    }
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    err = "stream synchronisation failed";
    return SBX_ECUDA;
  }
  return SBX_OK;
}

cudaError_t prepare_tc_kernels() {
  return cudaFuncSetAttribute(k_force_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

cudaError_t launch_force_tc(const sbx_ctx *ctx, const double *u, double *f, double dt,
                            cudaStream_t s) {
  bool load_done = false;   // the load term is added by CTA 0 of one launch only
  for (int cls = 0; cls < TC_CLASSES; ++cls) {
    if (ctx->n_tc_tiles[cls] == 0) continue;
    LoadTable L = ctx->loads();
    if (load_done) L.n = 0;
    load_done = true;
    k_force_tc<<<ctx->n_tc_tiles[cls], 256, ctx->tc_smem[cls], s>>>(
        ctx->d_tc_tiles[cls], ctx->d_tc_pat, ctx->d_tc_nodes, ctx->d_tc_lidx, ctx->d_tc_K,
        ctx->d_sym, ctx->d_scale, u, f, L, ctx->d_step, dt, ctx->d_flags,
        ctx->tc_kmax[cls], ctx->tc_nmax[cls], ctx->tc_maxnodes[cls], ctx->tc_maxnc[cls]);
  }
  return cudaGetLastError();
}

}  // namespace sbx

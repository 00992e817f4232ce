// Mixed-precision internal force on the 5th-generation tensor cores:
// a persistent, software-pipelined kernel.
//
// Work unit: a tile of up to 128 cells of one pattern p (m = 3 n_p DOFs) and
// the tile's unique nodes.  The host packs each tile into one contiguous
// record (layout below) that replaces the connectivity.  Each CTA (256
// threads) walks its tiles with two stages:
//   * the record of tile i+2 streams in by one 1-D bulk copy (TMA engine,
//     completion on an mbarrier) and the displacements of tile i+1's nodes
//     by per-thread cp.async, while tile i is computed.  U_n arrives as FP32
//     (hi, lo) pairs per component (float [N][6], written by the update
//     kernel with integer operations), hi + lo = U_n to ~2^-48;
//   * tile i: A (128 x K) = each cell's displacements minus its slot-0
//     node's (K_p annihilates translations), transformed by its op
//     (Sec. 3.2.2), formed in FP32 as (hi - hi_ref) + (lo - lo_ref) and
//     rounded to TF32 hi + lo;  D (TMEM) = A_hi B_hi^T + A_hi B_lo^T +
//     A_lo B_hi^T with B = K_p split the same way (tcgen05.mma kind::tf32 by
//     one thread, completion by tcgen05.commit -> mbarrier);  tcgen05.ld D
//     (row = cell), times E_e h_e, into shared memory; each node sums its
//     incidences (back in the cell frame) in FP32 and adds the sum to f with
//     one 16-byte vector reduction (f is float [N][4]).  No shared-memory
//     atomics.
// No FP64 arithmetic runs per node or per incidence (GB300's FP64 pipe is
// ~1/64 of FP32).
//
// Two code paths: FAST for tiles of the 8-node cell with the identity op
// (most cells of a refined octree; every loop unrolled, each thread owns
// one cell and four of its nodes), and a general one (any pattern and op;
// work items (cell, node) over all threads).
//
// Operands use the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices, row groups nK * 128 B apart, K groups 128 B apart within a row
// group (LBO = 128 B, SBO = nK * 128 B).
//
// Record layout (every part padded to 16 bytes):
//   int32 {pat, ncell, nn, n | ident << 8 | log2(cells per tile) << 9}
//   uint8 sym[ncell]                   op of each cell
//   float scale[ncell]                 E_e h_e rounded to FP32
//   int32 nodes[nn]                    unique node ids, ascending
//   uint16 lid[ncell][lrow]            per cell, the local index (into
//                                      nodes) of each slot; lrow = n
//                                      rounded up to 8
//   uint16 off[nn + 1]                 incidences of each node:
//   uint16 inc[n * ncell]              inc[off[q] .. off[q+1]) = cell * 32 + slot
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

constexpr int TC_THREADS = 256;
constexpr int FAST_NN_CAP = 272;   // unique nodes of an 8-node-cell tile (4 CTAs per SM)
constexpr uint32_t WAIT_POLLS = 1u << 22;

__host__ __device__ inline uint32_t a16(uint32_t x) { return (x + 15u) & ~15u; }
__host__ __device__ inline uint32_t a128(uint32_t x) { return (x + 127u) & ~127u; }
__host__ __device__ inline int lid_row(int n) { return (n + 7) & ~7; }

struct RecLayout {
  uint32_t sym, scale, nodes, lid, off, inc, bytes;
};
__host__ __device__ inline RecLayout rec_layout(int ncell, int nn, int n) {
  RecLayout R;
  uint32_t o = 16;
  R.sym = o;   o += a16((uint32_t)ncell);
  R.scale = o; o += a16(4u * ncell);
  R.nodes = o; o += a16(4u * nn);
  R.lid = o;   o += a16(2u * (uint32_t)lid_row(n) * ncell);
  R.off = o;   o += a16(2u * (nn + 1));
  R.inc = o;   o += a16(2u * (uint32_t)n * ncell);
  R.bytes = o;
  return R;
}

struct SmemLayout {
  uint32_t B, A, stage[2], u_off, total;
};
// kmax, nmax: padded K and N; rec_max: largest record; nn_max: most nodes.
// A also holds F after the MMA: FAST float4 [8][128] (slot, cell), general
// FP32 rows (cell, column; stride nmax + 1).  Each stage: the record, then
// the tile's node pairs (hi xyz, lo xyz; 24 bytes per node).
__host__ __device__ inline SmemLayout smem_layout(int kmax, int nmax, int rec_max, int nn_max) {
  SmemLayout L;
  uint32_t o = 128;                                    // 3 mbarriers + TMEM address
  L.B = o;   o = a128(o + 2u * nmax * kmax * 4u);
  const uint32_t a_bytes = 2u * 128u * kmax * 4u, f_bytes = 128u * (nmax + 1) * 4u;
  L.A = o;   o = a128(o + (a_bytes > f_bytes ? a_bytes : f_bytes));
  L.u_off = a16((uint32_t)rec_max);
  const uint32_t st = a128(L.u_off + 24u * (uint32_t)nn_max);
  L.stage[0] = o; o += st;
  L.stage[1] = o; o += st;
  L.total = o;
  return L;
}

struct Stage {
  const int32_t *hdr;
  const uint8_t *sym;
  const float *scale;
  const int32_t *nodes;
  const uint16_t *lid, *off, *inc;
  const float *u;   // node pairs
};
__device__ inline Stage stage_view(const unsigned char *base, uint32_t u_off) {
  Stage S;
  S.hdr = reinterpret_cast<const int32_t *>(base);
  const RecLayout R = rec_layout(S.hdr[1], S.hdr[2], S.hdr[3] & 0xFF);
  S.sym = base + R.sym;
  S.scale = reinterpret_cast<const float *>(base + R.scale);
  S.nodes = reinterpret_cast<const int32_t *>(base + R.nodes);
  S.lid = reinterpret_cast<const uint16_t *>(base + R.lid);
  S.off = reinterpret_cast<const uint16_t *>(base + R.off);
  S.inc = reinterpret_cast<const uint16_t *>(base + R.inc);
  S.u = reinterpret_cast<const float *>(base + u_off);
  return S;
}

// Float offset of A(c, col) in the canonical K-major layout.
__device__ __forceinline__ int a_off(int c, int col, int nK) {
  return (c >> 3) * nK * 32 + (c & 7) * 4 + (col >> 2) * 32 + (col & 3);
}

__device__ __forceinline__ void red_add_v4(float *addr, float x, float y, float z) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(x), "f"(y),
               "f"(z), "f"(0.0f)
               : "memory");
}

// The op of a cell: u_master[r] = sgn[r] u_cell[perm[r]].
struct Op {
  int p0, p1, p2;
  float s0, s1, s2;
};
__device__ __forceinline__ Op op_of(int op) {
  Op o;
  o.p0 = op_perm_of(op, 0);
  o.p1 = op_perm_of(op, 1);
  o.p2 = op_perm_of(op, 2);
  o.s0 = (op & 1) ? -1.0f : 1.0f;
  o.s1 = (op & 2) ? -1.0f : 1.0f;
  o.s2 = (op & 4) ? -1.0f : 1.0f;
  return o;
}
__device__ __forceinline__ float pick3(int i, float a, float b, float c) {
  return i == 0 ? a : (i == 1 ? b : c);
}

// (hi - hi_ref) + (lo - lo_ref) for one component pair of two nodes
__device__ __forceinline__ void node_diff(const float *p, const float *r, float &d0, float &d1,
                                          float &d2) {
  const float2 a = *reinterpret_cast<const float2 *>(p);       // hx hy
  const float2 b = *reinterpret_cast<const float2 *>(p + 2);   // hz lx
  const float2 c = *reinterpret_cast<const float2 *>(p + 4);   // ly lz
  const float2 ra = *reinterpret_cast<const float2 *>(r);
  const float2 rb = *reinterpret_cast<const float2 *>(r + 2);
  const float2 rc = *reinterpret_cast<const float2 *>(r + 4);
  d0 = (a.x - ra.x) + (b.y - rb.y);
  d1 = (a.y - ra.y) + (c.x - rc.x);
  d2 = (b.x - rb.x) + (c.y - rc.y);
}

template <bool FAST>
__global__ void __launch_bounds__(TC_THREADS, FAST ? 4 : 1)
    k_force_tc(const TcTile *__restrict__ tiles, int ntiles, int chunk,
               const uint8_t *__restrict__ recs, const TcPattern *__restrict__ pats,
               const float *__restrict__ Kc, const float *__restrict__ u,
               float *__restrict__ f4, LoadTable Ld, const int64_t *__restrict__ d_step,
               double dt, int32_t *flags, int kmax, int nmax, int rec_max, int nn_max,
               int tcols) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemLayout SL = smem_layout(kmax, nmax, rec_max, nn_max);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);   // [0] MMA, [1], [2] records
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(smem + 32);
  float *Bs = reinterpret_cast<float *>(smem + SL.B);
  float *As = reinterpret_cast<float *>(smem + SL.A);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  const uint32_t mb_mma = tc::smem_addr(&mbar[0]);
  const uint32_t mb_rec0 = tc::smem_addr(&mbar[1]);   // stage s: mb_rec0 + 8 s

  if (warp == 0) {
    tc::tmem_alloc(tc::smem_addr(taddr_s), (uint32_t)tcols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(mb_mma, 1);
    tc::mbar_init(mb_rec0, 1);
    tc::mbar_init(mb_rec0 + 8u, 1);
    tc::mbar_fence_init();
  }
  if (blockIdx.x == 0 && Ld.n > 0) {   // external load of this step (Sec. 5)
    const double t = (double)(*d_step) * dt;
    for (int l = tid; l < Ld.n; l += TC_THREADS) {
      const int64_t dof = Ld.dof[l];
      const float v = (float)(-Ld.amp[l] * wavelet_value(Ld.kind[l], t, Ld.t1[l], Ld.ncyc[l]));
      atomicAdd(&f4[4 * (dof / 3) + dof % 3], v);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *taddr_s;

  // tiles of this CTA: blockIdx.x + i G (chunk == 0) or a contiguous run
  auto tile_at = [&](int i) -> int {
    if (chunk == 0) {
      const int t = blockIdx.x + i * G;
      return t < ntiles ? t : -1;
    }
    if (i >= chunk) return -1;
    const int t = blockIdx.x * chunk + i;
    return t < ntiles ? t : -1;
  };
  auto issue_record = [&](int s, int tile) {   // thread 0 only
    const TcTile T = tiles[tile];
    tc::fence_proxy_async_smem();
    const uint32_t mb = mb_rec0 + 8u * (uint32_t)s;
    tc::mbar_arrive_expect_tx(mb, (uint32_t)T.rec_bytes);
    tc::bulk_g2s(tc::smem_addr(smem + (s ? SL.stage[1] : SL.stage[0])), recs + T.rec_off, (uint32_t)T.rec_bytes, mb);
  };
  auto issue_gather = [&](int s) {            // all threads
    const Stage S = stage_view(smem + (s ? SL.stage[1] : SL.stage[0]), SL.u_off);
    const int nn = S.hdr[2];
    const uint32_t ub = tc::smem_addr(S.u);
    for (int i = tid; i < nn; i += TC_THREADS) {
      const float *src = u + 6 * (int64_t)S.nodes[i];
      tc::cp_async8(ub + 24u * i, src);
      tc::cp_async8(ub + 24u * i + 8u, src + 2);
      tc::cp_async8(ub + 24u * i + 16u, src + 4);
    }
    tc::cp_async_commit();
  };

  // bit s of ph_rec / pend: parity and "copy in flight" of stage s's record
  uint32_t ph_rec = 0u, pend = 0u, ph_mma = 0u;
  bool ok = true;
  {
    const int t0 = tile_at(0), t1 = tile_at(1);
    if (t0 >= 0) {
      if (tid == 0) {
        issue_record(0, t0);
        if (t1 >= 0) issue_record(1, t1);
      }
      pend = 1u | (t1 >= 0 ? 2u : 0u);
      ok = __syncthreads_and(tc::mbar_wait_bounded(mb_rec0, ph_rec & 1u, WAIT_POLLS));
      if (ok) {
        ph_rec ^= 1u;
        pend &= ~1u;
        issue_gather(0);
      }
    }
  }
  int cur_pat = -1, pm = 0, pkpad = 8, pnpad = 16;
  for (int i = 0; ok; ++i) {
    const int tile = tile_at(i);
    if (tile < 0) break;
    const int s = i & 1;
    const uint32_t so = (uint32_t)(s ^ 1);
    tc::cp_async_wait_all();
    __syncthreads();
    const int next = tile_at(i + 1);
    if (next >= 0) {
      ok = __syncthreads_and(
          tc::mbar_wait_bounded(mb_rec0 + 8u * so, (ph_rec >> so) & 1u, WAIT_POLLS));
      if (!ok) break;
      ph_rec ^= 1u << so;
      pend &= ~(1u << so);
      issue_gather(s ^ 1);
    }
    const Stage S = stage_view(smem + (s ? SL.stage[1] : SL.stage[0]), SL.u_off);
    const int pat = S.hdr[0], ncell = S.hdr[1], nn = S.hdr[2];
    if (pat != cur_pat) {   // B = K_p hi | lo, canonical layout
      const TcPattern P = pats[pat];
      pm = P.m;
      pkpad = P.kpad;
      pnpad = P.npad;
      const float4 *src = reinterpret_cast<const float4 *>(Kc + P.kc_off);
      float4 *dst = reinterpret_cast<float4 *>(Bs);
      const int nv = (2 * pnpad * pkpad) / 4;
      for (int q = tid; q < nv; q += TC_THREADS) dst[q] = src[q];
      cur_pat = pat;
    }
    const int m = FAST ? 24 : pm, kpad = FAST ? 24 : pkpad, npad = FAST ? 32 : pnpad;
    const int nK = kpad / 4;
    float *Ahi = As, *Alo = As + 128 * kpad;
    // FAST: thread (c, h) owns cell c and its nodes 4h .. 4h + 3
    const int fc = tid & 127, fh = tid >> 7;
    uint32_t lw0 = 0, lw1 = 0;   // FAST: local indices of the four nodes (2 x u16 each)
    if (FAST) {
      if (fc < ncell) {
        const uint4 L = *reinterpret_cast<const uint4 *>(S.lid + 8 * fc);
        lw0 = fh ? L.z : L.x;
        lw1 = fh ? L.w : L.y;
        const float *ref = S.u + 6 * (L.x & 0xFFFFu);
        float vh[12], vl[12];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t lk = ((t < 2 ? lw0 : lw1) >> (16 * (t & 1))) & 0xFFFFu;
          float d0, d1, d2;
          node_diff(S.u + 6 * lk, ref, d0, d1, d2);
          vh[3 * t] = tc::to_tf32(d0);
          vh[3 * t + 1] = tc::to_tf32(d1);
          vh[3 * t + 2] = tc::to_tf32(d2);
          vl[3 * t] = tc::to_tf32(d0 - vh[3 * t]);
          vl[3 * t + 1] = tc::to_tf32(d1 - vh[3 * t + 1]);
          vl[3 * t + 2] = tc::to_tf32(d2 - vh[3 * t + 2]);
        }
#pragma unroll
        for (int g = 0; g < 3; ++g) {
          const int o = a_off(fc, 12 * fh + 4 * g, nK);
          *reinterpret_cast<float4 *>(Ahi + o) =
              make_float4(vh[4 * g], vh[4 * g + 1], vh[4 * g + 2], vh[4 * g + 3]);
          *reinterpret_cast<float4 *>(Alo + o) =
              make_float4(vl[4 * g], vl[4 * g + 1], vl[4 * g + 2], vl[4 * g + 3]);
        }
      }
    } else {
      // items (cell, node): cell = w mod cells-per-tile, node = w / it
      const int n = m / 3, lrow = lid_row(n), cpl = (S.hdr[3] >> 9) & 7;
      const int cmask = (1 << cpl) - 1;
      const bool ident = ((S.hdr[3] >> 8) & 1) != 0;
      for (int w = tid; w < (n << cpl); w += TC_THREADS) {
        const int c = w & cmask, k = w >> cpl;
        if (c >= ncell) continue;
        const uint16_t *lr = S.lid + lrow * c;
        const int l0 = lr[0], lk = lr[k];
        float d0, d1, d2;
        node_diff(S.u + 6 * lk, S.u + 6 * l0, d0, d1, d2);
        float x0 = d0, x1 = d1, x2 = d2;
        if (!ident) {
          const Op o = op_of(S.sym[c]);
          x0 = o.s0 * pick3(o.p0, d0, d1, d2);
          x1 = o.s1 * pick3(o.p1, d0, d1, d2);
          x2 = o.s2 * pick3(o.p2, d0, d1, d2);
        }
        const float h0 = tc::to_tf32(x0), h1 = tc::to_tf32(x1), h2 = tc::to_tf32(x2);
        const int o0 = a_off(c, 3 * k, nK), o1 = a_off(c, 3 * k + 1, nK),
                  o2 = a_off(c, 3 * k + 2, nK);
        Ahi[o0] = h0;
        Ahi[o1] = h1;
        Ahi[o2] = h2;
        Alo[o0] = tc::to_tf32(x0 - h0);
        Alo[o1] = tc::to_tf32(x1 - h1);
        Alo[o2] = tc::to_tf32(x2 - h2);
      }
      // zero the K padding columns m .. kpad - 1
      for (int w = tid; w < ((kpad - m) << cpl); w += TC_THREADS) {
        const int c = w & cmask, col = m + (w >> cpl);
        if (c >= ncell) continue;
        const int o = a_off(c, col, nK);
        Ahi[o] = 0.0f;
        Alo[o] = 0.0f;
      }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, npad);
      const uint32_t a_hi = tc::smem_addr(Ahi), a_lo = tc::smem_addr(Alo);
      const uint32_t b_hi = tc::smem_addr(Bs), b_lo = tc::smem_addr(Bs + npad * kpad);
      const uint32_t sbo = (uint32_t)nK * 128u;
      for (int ks = 0; ks < kpad / 8; ++ks) {
        const uint32_t o = (uint32_t)ks * 256u;
        const uint64_t ah = tc::smem_desc(a_hi + o, 128, sbo), al = tc::smem_desc(a_lo + o, 128, sbo);
        const uint64_t bh = tc::smem_desc(b_hi + o, 128, sbo), bl = tc::smem_desc(b_lo + o, 128, sbo);
        tc::mma_tf32(taddr, ah, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32(taddr, ah, bl, idesc, 1u);
        tc::mma_tf32(taddr, al, bh, idesc, 1u);
      }
      tc::mma_commit(mb_mma);
    }
    ok = __syncthreads_and(tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_POLLS));
    tc::fence_after_sync();
    if (!ok) break;
    ph_mma ^= 1u;
    // epilogue: warps w and w + 4 read TMEM lanes 32 (w % 4) .. + 31 (cells)
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    if (FAST) {
      float v[12];
      {
        float v8[8];
        tc::tmem_ld8(taddr + lane_base + (uint32_t)(12 * fh), v8);
        uint32_t r4[4];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r4[0]), "=r"(r4[1]), "=r"(r4[2]), "=r"(r4[3])
                     : "r"(taddr + lane_base + (uint32_t)(12 * fh + 8)));
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = v8[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[8 + q] = __uint_as_float(r4[q]);
      }
      if (fc < ncell) {   // F4[slot][cell] = E h D
        const float sc = S.scale[fc];
        float4 *F4 = reinterpret_cast<float4 *>(As);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          F4[(4 * fh + t) * 128 + fc] =
              make_float4(sc * v[3 * t], sc * v[3 * t + 1], sc * v[3 * t + 2], 0.0f);
      }
      tc::fence_before_sync();
    } else {
      // D rows to shared memory (F, row stride npad + 1; A is free)
      float *F = As;
      {
        const int c = 32 * (warp & 3) + lane;
        const int half = npad / 2;   // a multiple of 8
        const int c0 = (warp >> 2) * half;
        for (int cc = c0; cc < c0 + half; cc += 8) {
          float v[8];
          tc::tmem_ld8(taddr + lane_base + (uint32_t)cc, v);
          tc::tmem_ld_wait();
          if (c < ncell) {
#pragma unroll
            for (int q = 0; q < 8; ++q) F[c * (npad + 1) + cc + q] = v[q];
          }
        }
      }
      tc::fence_before_sync();
    }
    __syncthreads();
    // node sums over the incidences (cell c, slot k), in the cell frame
    if (FAST) {
      const float4 *F4 = reinterpret_cast<const float4 *>(As);
      for (int q = tid; q < nn; q += TC_THREADS) {
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
        const int j0 = S.off[q], nj = S.off[q + 1] - j0;   // <= 8 cells share a node
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < nj) {
            const int e = S.inc[j0 + j];
            const float4 v = F4[((e & 31) << 7) | (e >> 5)];
            a0 += v.x;
            a1 += v.y;
            a2 += v.z;
          }
        }
        red_add_v4(f4 + 4 * (int64_t)S.nodes[q], a0, a1, a2);
      }
    } else {
      const float *F = As;
      const bool ident = ((S.hdr[3] >> 8) & 1) != 0;
      for (int q = tid; q < nn; q += TC_THREADS) {
        float a[3] = {0.0f, 0.0f, 0.0f};
        for (int j = S.off[q]; j < S.off[q + 1]; ++j) {
          const int e = S.inc[j], c = e >> 5, k = e & 31;
          const float *Fr = F + c * (npad + 1) + 3 * k;
          const float sc = S.scale[c];
          const float g0 = sc * Fr[0], g1 = sc * Fr[1], g2 = sc * Fr[2];
          if (ident) {
            a[0] += g0;
            a[1] += g1;
            a[2] += g2;
          } else {   // f_cell[perm r] = sgn r f_master[r]
            const Op o = op_of(S.sym[c]);
            const float w0 = o.s0 * g0, w1 = o.s1 * g1, w2 = o.s2 * g2;
            a[0] += (o.p0 == 0 ? w0 : 0.0f) + (o.p1 == 0 ? w1 : 0.0f) + (o.p2 == 0 ? w2 : 0.0f);
            a[1] += (o.p0 == 1 ? w0 : 0.0f) + (o.p1 == 1 ? w1 : 0.0f) + (o.p2 == 1 ? w2 : 0.0f);
            a[2] += (o.p0 == 2 ? w0 : 0.0f) + (o.p1 == 2 ? w1 : 0.0f) + (o.p2 == 2 ? w2 : 0.0f);
          }
        }
        red_add_v4(f4 + 4 * (int64_t)S.nodes[q], a[0], a[1], a[2]);
      }
    }
    __syncthreads();   // stage s and the sums are free
    const int after = tile_at(i + 2);
    if (after >= 0) {
      if (tid == 0) issue_record(s, after);
      pend |= 1u << s;
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(flags, 2);
    // let in-flight copies and MMAs drain before the CTA leaves
    tc::cp_async_wait_all();
    if (pend & 1u) tc::mbar_wait_bounded(mb_rec0, ph_rec & 1u, WAIT_POLLS);
    if (pend & 2u) tc::mbar_wait_bounded(mb_rec0 + 8u, (ph_rec >> 1) & 1u, WAIT_POLLS);
    tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_POLLS);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)tcols);
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

template <typename T>
void put(std::vector<uint8_t> &buf, size_t at, const T *src, size_t n) {
  memcpy(buf.data() + at, src, n * sizeof(T));
}

}  // namespace

// Host preparation of the tile records and canonical K_p.
int tc_setup(sbx_ctx *ctx, const std::vector<int32_t> &conn, const std::vector<int64_t> &conn_off,
             const std::vector<int64_t> &cnt, const std::vector<int64_t> &start,
             const std::vector<uint8_t> &sym_sorted, const std::vector<double> &scale_sorted,
             std::string &err) {
  const int P = ctx->n_pat;
  std::vector<TcPattern> pats(P);
  std::vector<float> Kc;
  std::vector<uint8_t> recs;
  // launch classes: 0 = FAST tiles (8-node cells, identity op, 128 cells);
  // general tiles by their own shared-memory need: 1 <= 113 KB, 2 larger
  std::vector<TcTile> tiles[TC_CLASSES];
  int kmax[TC_CLASSES], nmax[TC_CLASSES], recmax[TC_CLASSES], nnmax[TC_CLASSES], tcols[TC_CLASSES];
  for (int c = 0; c < TC_CLASSES; ++c) {
    kmax[c] = 8;
    nmax[c] = 16;
    recmax[c] = 16;
    nnmax[c] = 1;
    tcols[c] = 32;
  }
  const uint32_t class_limit[TC_CLASSES] = {56u * 1024u, 113u * 1024u, 227u * 1024u};
  std::vector<int64_t> mark(ctx->N, -1);   // node -> last tile that holds it
  int64_t stamp = 0;
  for (int p = 0; p < P; ++p) {
    const int np = ctx->pat_nodes[p], m = 3 * np;
    TcPattern &tp = pats[p];
    tp.m = m;
    tp.kpad = (m + 7) / 8 * 8;
    tp.npad = (m + 15) / 16 * 16;
    tp.tcols = tp.npad <= 32 ? 32 : (tp.npad <= 64 ? 64 : 128);
    tp.kc_off = (int64_t)Kc.size();
    const int nK = tp.kpad / 4;
    std::vector<float> B(2 * (size_t)tp.npad * tp.kpad, 0.0f);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double kv = ctx->K_host[ctx->pat_koff[p] + (int64_t)i * m + j];
        const float hi = tf32_round_host((float)kv);
        const float lo = tf32_round_host((float)(kv - (double)hi));
        const size_t o = (size_t)(i >> 3) * nK * 32 + (j >> 2) * 32 + (i & 7) * 4 + (j & 3);
        B[o] = hi;
        B[(size_t)tp.npad * tp.kpad + o] = lo;
      }
    Kc.insert(Kc.end(), B.begin(), B.end());
    if (cnt[p] == 0) continue;
    // dense, frequent small patterns: 128 cells per tile; the rest (rarer,
    // scattered, larger): 32, which keeps double-buffered records within
    // shared memory and spreads them over more CTAs
    // (the 8-node tiles also stop before their unique nodes exceed
    // FAST_NN_CAP, which keeps three CTAs per SM)
    const int per = (cnt[p] >= 4096 && m <= 30) ? 128 : 32;
    const int cpl = per == 128 ? 7 : 5;
    const int nn_cap = np == 8 ? FAST_NN_CAP : 1 << 30;
    const int lrow = lid_row(np);
    std::vector<std::pair<int32_t, int32_t>> v;   // (node, cell * 32 + slot)
    for (int64_t c0 = 0, nc = 0; c0 < cnt[p]; c0 += nc) {
      // greedy cut: up to `per` cells, at most nn_cap unique nodes
      ++stamp;
      int nn_new = 0;
      nc = 0;
      while (c0 + nc < cnt[p] && nc < per) {
        int add = 0;
        for (int k = 0; k < np; ++k) {
          const int32_t q = conn[conn_off[p] + (int64_t)k * cnt[p] + c0 + nc];
          if (mark[q] != stamp) ++add;
        }
        if (nc > 0 && nn_new + add > nn_cap) break;
        for (int k = 0; k < np; ++k) {
          const int32_t q = conn[conn_off[p] + (int64_t)k * cnt[p] + c0 + nc];
          if (mark[q] != stamp) {
            mark[q] = stamp;
            ++nn_new;
          }
        }
        ++nc;
      }
      v.clear();
      for (int k = 0; k < np; ++k)
        for (int c = 0; c < nc; ++c)
          v.emplace_back(conn[conn_off[p] + (int64_t)k * cnt[p] + c0 + c], c * 32 + k);
      std::sort(v.begin(), v.end());
      std::vector<int32_t> nodes;
      std::vector<uint16_t> lid((size_t)lrow * nc, 0), offs, inc;
      for (size_t i = 0; i < v.size(); ++i) {
        if (i == 0 || v[i].first != v[i - 1].first) {
          nodes.push_back(v[i].first);
          offs.push_back((uint16_t)inc.size());
        }
        lid[(size_t)(v[i].second >> 5) * lrow + (v[i].second & 31)] = (uint16_t)(nodes.size() - 1);
        inc.push_back((uint16_t)v[i].second);
      }
      offs.push_back((uint16_t)inc.size());
      const int nn = (int)nodes.size();
      const RecLayout R = rec_layout(nc, nn, np);
      const size_t at = recs.size();
      recs.resize(at + R.bytes, 0);
      std::vector<float> sc(nc);
      int ident = 1;
      for (int c = 0; c < nc; ++c) {
        recs[at + R.sym + c] = sym_sorted[start[p] + c0 + c];
        ident &= sym_sorted[start[p] + c0 + c] == 0;
        sc[c] = (float)scale_sorted[start[p] + c0 + c];
      }
      const int32_t hdr[4] = {p, (int32_t)nc, nn, np | (ident << 8) | (cpl << 9)};
      put(recs, at, hdr, 4);
      put(recs, at + R.scale, sc.data(), nc);
      put(recs, at + R.nodes, nodes.data(), nn);
      put(recs, at + R.lid, lid.data(), lid.size());
      put(recs, at + R.off, offs.data(), offs.size());
      put(recs, at + R.inc, inc.data(), inc.size());
      TcTile t;
      t.rec_off = (int64_t)at;
      t.rec_bytes = (int32_t)R.bytes;
      t.pat = p;
      const uint32_t need = smem_layout(tp.kpad, tp.npad, R.bytes, nn).total;
      int cls;
      if (np == 8 && ident && per == 128 && need <= class_limit[0]) {
        cls = 0;
      } else {
        cls = 1;
        if (need > class_limit[1]) cls = 2;
        if (need > class_limit[2]) {
          err = "tensor-core tile needs more than 227 KB of shared memory";
          return SBX_EINVAL;
        }
      }
      kmax[cls] = std::max(kmax[cls], tp.kpad);
      nmax[cls] = std::max(nmax[cls], tp.npad);
      recmax[cls] = std::max(recmax[cls], (int)R.bytes);
      nnmax[cls] = std::max(nnmax[cls], nn);
      tcols[cls] = std::max(tcols[cls], tp.tcols);
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
  if (int rc = up(&ctx->d_tc_rec, recs)) return rc;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  for (int cls = 0; cls < TC_CLASSES; ++cls) {
    if (int rc = up(&ctx->d_tc_tiles[cls], tiles[cls])) return rc;
    const int64_t nt = (int64_t)tiles[cls].size();
    ctx->n_tc_tiles[cls] = (int)nt;
    ctx->tc_kmax[cls] = kmax[cls];
    ctx->tc_nmax[cls] = nmax[cls];
    ctx->tc_rec_max[cls] = recmax[cls];
    ctx->tc_nn_max[cls] = nnmax[cls];
    ctx->tc_tcols[cls] = tcols[cls];
    const uint32_t smem = smem_layout(kmax[cls], nmax[cls], recmax[cls], nnmax[cls]).total;
    ctx->tc_smem[cls] = smem;
    // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per
    // CTA), tensor memory (512 columns) and the FAST kernel's register bound
    int per_sm = (int)((228u * 1024u) / (smem + 1024u));
    per_sm = std::max(1, std::min(per_sm, std::min(cls == 0 ? 4 : 8, 512 / tcols[cls])));
    int64_t grid = std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)nsm * per_sm));
    // FAST tiles round-robin (neighbouring tiles run together and share
    // nodes in L2); general tiles in contiguous runs (fewer K_p reloads)
    int chunk = 0;
    if (cls != 0 && nt > 0) {
      chunk = (int)((nt + grid - 1) / grid);
      grid = (nt + chunk - 1) / chunk;
    }
    ctx->tc_grid[cls] = (int)grid;
    ctx->tc_chunk[cls] = chunk;
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    err = "stream synchronisation failed";
    return SBX_ECUDA;
  }
  return SBX_OK;
}

cudaError_t prepare_tc_kernels() {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_force_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           227 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           227 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force_tc<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_force_tc<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}

cudaError_t launch_force_tc(const sbx_ctx *ctx, const float *pairs, float *f4, double dt,
                            cudaStream_t s) {
  bool load_done = false;   // the load term is added by CTA 0 of one launch only
  for (int cls = 0; cls < TC_CLASSES; ++cls) {
    if (ctx->n_tc_tiles[cls] == 0) continue;
    LoadTable L = ctx->loads();
    if (load_done) L.n = 0;
    load_done = true;
    auto k = cls == 0 ? k_force_tc<true> : k_force_tc<false>;
    k<<<ctx->tc_grid[cls], TC_THREADS, ctx->tc_smem[cls], s>>>(
        ctx->d_tc_tiles[cls], ctx->n_tc_tiles[cls], ctx->tc_chunk[cls], ctx->d_tc_rec,
        ctx->d_tc_pat, ctx->d_tc_K, pairs, f4, L, ctx->d_step, dt, ctx->d_flags, ctx->tc_kmax[cls],
        ctx->tc_nmax[cls], ctx->tc_rec_max[cls], ctx->tc_nn_max[cls], ctx->tc_tcols[cls]);
  }
  return cudaGetLastError();
}

}  // namespace sbx

// Mixed-precision internal force (SBX_PREC_MIXED, one load case).
//
// U_n enters as FP32 (hi, lo) pairs per component (float [N][6], written by
// the update kernel with integer operations; hi + lo = U_n to ~2^-48).  Each
// cell's displacements are taken relative to its slot-0 node (K_p
// annihilates translations) as (hi - hi_ref) + (lo - lo_ref) in FP32, so the
// contraction works on differences accurate to FP32 however large U_n is.
// f is float [N][4] (x, y, z, unused); every node sum is added with one
// 16-byte vector reduction.  No FP64 arithmetic runs per node or cell
// (GB300's FP64 pipe is ~1/64 of FP32).
//
// The kernels:
//   k_force_wht32 (default for) the 8-node cell with the identity op (the
//                bulk of a refined octree): the same tiles and pipeline as
//                k_force_tc below, one thread per cell, and K_p applied in
//                the Walsh basis of the cell's corners, where it is eight
//                3 x 3 blocks (FP32 SIMT; no tensor memory).
//   k_force_tc   the same cells on the 5th-generation tensor cores
//                (sbx_set_mixed_kernel): a persistent,
//                software-pipelined kernel over tiles of up to 128 cells.
//                The record of tile i+2 streams in by one 1-D bulk copy (TMA
//                engine, completion on an mbarrier) while tile i is
//                computed; tile i+1's node pairs follow by per-thread
//                cp.async, issued while tile i's MMAs run.
//                A (128 x 24) = the cells' differences rounded to TF32 hi +
//                lo, written to tensor memory by tcgen05.st (row = cell =
//                TMEM lane);  D (TMEM) = A_hi B_hi^T + A_hi B_lo^T + A_lo
//                B_hi^T with B = K_p split the same way in shared memory
//                (tcgen05.mma kind::tf32 by one thread, completion by
//                tcgen05.commit -> mbarrier);
//                tcgen05.ld D (row = cell) times E_e h_e into shared memory;
//                each node sums its incidences (per-tile list) in FP32.
//   k_force_gen_tc  every other pattern and op (hanging-node cells: a few
//                per cent of the cells, up to 78 DOFs) on the tensor cores
//                (the default): tiles of up to 128 cells of one pattern,
//                A = the cells' master-frame differences in tensor memory,
//                B = K_p TF32 hi | lo bulk-copied per pattern, TF32 x 3.
//   k_force_gen  the same cells on FP32 SIMT (SBX_HANGING_SIMT): 32 cells
//                per CTA, FP32 K_p in shared memory, F = K_p d by FFMA,
//                back to the cell frame (Sec. 3.2.2), one vector reduction
//                per (cell, node).
// and, for the batched FP32 form, k_force_batch_tc: the hanging-node
// patterns' (cell, load case) rows on the tensor cores.
//
// B uses the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices, row groups nK * 128 B apart, K groups 128 B apart within a row
// group (LBO = 128 B, SBO = nK * 128 B).  TMEM columns: D 0..31, A_hi
// 32..55, A_lo 64..87.
//
// Tile records of k_force_tc and k_force_wht32 (every part padded to 16
// bytes), two kinds:
//  brick (kind 1): 128 same-size cells forming a complete 4 x 4 x 8 block,
//   cell c at (c & 3, (c >> 2) & 3, c >> 4), nodes on the 5 x 5 x 9 lattice,
//   node (a, b, c) = index a + 5 b + 25 c; slot k = corner (k & 1, k >> 1 & 1,
//   k >> 2); every index is arithmetic.
//   int32 {pat, 128, 225, 1}           header
//   float scale[128]                   E_e h_e rounded to FP32
//   int32 nodes[225]                   lattice node ids
//  list (kind 0): any cells (up to 128):
//   int32 {pat, ncell, nn, 0}          header
//   float scale[ncell]                 E_e h_e rounded to FP32
//   int32 nodes[nn]                    unique node ids, ascending
//   uint16 lid[ncell][8]               per cell, the local index (into
//                                      nodes) of each slot
//   uint16 off[nn + 1]                 incidences of each node:
//   uint16 inc[8 * ncell]              inc[off[q] .. off[q+1]) = cell * 32 + slot
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
constexpr uint32_t WAIT_POLLS = 1u << 22;
constexpr int FAST_NN_CAP = 320;   // unique nodes per tile: keeps 4 CTAs per SM
constexpr int KM = 24, KPAD = 24, NPAD = 32, NK = KPAD / 4;   // 8-node cell
constexpr int TCOLS = 128, COL_AHI = 32, COL_ALO = 64;         // TMEM columns
constexpr int GEN_TILE = 32;       // cells per k_force_gen CTA

__host__ __device__ inline uint32_t a16(uint32_t x) { return (x + 15u) & ~15u; }
__host__ __device__ inline uint32_t a128(uint32_t x) { return (x + 127u) & ~127u; }

constexpr int BRICK_NX = 4, BRICK_NY = 4, BRICK_NZ = 8;   // cells of a brick tile
constexpr int BRICK_CELLS = BRICK_NX * BRICK_NY * BRICK_NZ;  // 128
constexpr int BRICK_NODES = 5 * 5 * 9;                      // 225

struct RecLayout {
  uint32_t scale, nodes, lid, off, inc, bytes;
};
__host__ __device__ inline RecLayout rec_layout(int ncell, int nn, int kind) {
  RecLayout R;
  uint32_t o = 16;
  R.scale = o; o += a16(4u * ncell);
  R.nodes = o; o += a16(4u * nn);
  R.lid = R.off = R.inc = o;
  if (kind == 0) {
    R.lid = o; o += a16(16u * ncell);
    R.off = o; o += a16(2u * (nn + 1));
    R.inc = o; o += a16(16u * ncell);
  }
  R.bytes = o;
  return R;
}

struct SmemLayout {
  uint32_t B, F, stage[2], u_off, total;
};
// F = E h D as float4 [8][128] (slot, cell).  Each stage: a record, then the
// tile's node pairs (24 B per node).
__host__ __device__ inline SmemLayout smem_layout(int rec_max, int nn_max) {
  SmemLayout L;
  uint32_t o = 128;                                    // 3 mbarriers + TMEM address
  L.B = o;   o = a128(o + 2u * NPAD * KPAD * 4u);
  L.F = o;   o = a128(o + 8u * 128u * 16u);
  L.u_off = a16((uint32_t)rec_max);
  const uint32_t st = a128(L.u_off + 24u * (uint32_t)nn_max);
  L.stage[0] = o; o += st;
  L.stage[1] = o; o += st;
  L.total = o;
  return L;
}

struct Stage {
  const int32_t *hdr;
  const float *scale;
  const int32_t *nodes;
  const uint16_t *lid, *off, *inc;
  const float *u;   // node pairs
};
__device__ inline Stage stage_view(const unsigned char *base, uint32_t u_off) {
  Stage S;
  S.hdr = reinterpret_cast<const int32_t *>(base);
  const RecLayout R = rec_layout(S.hdr[1], S.hdr[2], S.hdr[3]);
  S.scale = reinterpret_cast<const float *>(base + R.scale);
  S.nodes = reinterpret_cast<const int32_t *>(base + R.nodes);
  S.lid = reinterpret_cast<const uint16_t *>(base + R.lid);
  S.off = reinterpret_cast<const uint16_t *>(base + R.off);
  S.inc = reinterpret_cast<const uint16_t *>(base + R.inc);
  S.u = reinterpret_cast<const float *>(base + u_off);
  return S;
}

// the FP32 force accumulator stays in L2 (evict_last) from the force
// kernels to the update that reads and clears it
__device__ __forceinline__ void red_add_v4(float *addr, float x, float y, float z) {
  asm volatile(
      "{\n\t.reg .b64 pol;\n\t"
      "createpolicy.fractional.L2::evict_last.b64 pol, 1.0;\n\t"
      "red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, pol;\n\t}" ::"l"(addr),
      "f"(x), "f"(y), "f"(z), "f"(0.0f)
      : "memory");
}

// (hi - hi_ref) + (lo - lo_ref) per component; p, r: node pairs (hx hy hz lx ly lz)
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

// Brick tiles: node sums of one corner layer by warp shuffles.  v[3 t + r]
// holds component r of corner (t & 1, t >> 1, h) of this lane's cell, already
// scaled by E h; lane = x + 4 y + 16 zl, cell (x, y, z = 2 (w % 4) + zl).
// The node (a, b) of lattice layer z + h sums corner (dx, dy) of the cells
// (a - dx, b - dy): lane (x, y) forms node (x, y) (and (4, y), (x, 4),
// (4, 4) on the +x / +y rows) from its own corners and its -x, -y, -x-y
// neighbours' (warp shuffles), one vector reduction per node.
__device__ __forceinline__ void brick_node_sums(const Stage &S, const float *v, int warp,
                                                int lane, int h, float *f4) {
  const int x = lane & 3, y = (lane >> 2) & 3;
  float s1[6], s4[6], s5[3];   // from lane - 1: corners 1, 3; lane - 4: 2, 3; lane - 5: 3
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    s1[r] = __shfl_up_sync(0xffffffffu, v[3 + r], 1);
    s1[3 + r] = __shfl_up_sync(0xffffffffu, v[9 + r], 1);
    s4[r] = __shfl_up_sync(0xffffffffu, v[6 + r], 4);
    s4[3 + r] = __shfl_up_sync(0xffffffffu, v[9 + r], 4);
    s5[r] = __shfl_up_sync(0xffffffffu, v[9 + r], 5);
  }
#pragma unroll
  for (int r = 0; r < 6; ++r) {   // neighbours outside the layer contribute nothing
    s1[r] = x > 0 ? s1[r] : 0.0f;
    s4[r] = y > 0 ? s4[r] : 0.0f;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) s5[r] = (x > 0 && y > 0) ? s5[r] : 0.0f;
  const int base = 25 * (2 * (warp & 3) + ((lane >> 4) & 1) + h);
  red_add_v4(f4 + 4 * (int64_t)S.nodes[base + x + 5 * y], v[0] + s1[0] + s4[0] + s5[0],
             v[1] + s1[1] + s4[1] + s5[1], v[2] + s1[2] + s4[2] + s5[2]);
  if (x == 3)   // node (4, y): own corner (1, 0), cell (3, y - 1) corner (1, 1)
    red_add_v4(f4 + 4 * (int64_t)S.nodes[base + 4 + 5 * y], v[3] + s4[3], v[4] + s4[4],
               v[5] + s4[5]);
  if (y == 3)   // node (x, 4): own corner (0, 1), cell (x - 1, 3) corner (1, 1)
    red_add_v4(f4 + 4 * (int64_t)S.nodes[base + x + 20], v[6] + s1[3], v[7] + s1[4],
               v[8] + s1[5]);
  if (x == 3 && y == 3)   // node (4, 4)
    red_add_v4(f4 + 4 * (int64_t)S.nodes[base + 24], v[9], v[10], v[11]);
}

// external load of the step (Sec. 5), added into the FP32 accumulator
__device__ __forceinline__ void add_loads(const LoadTable &Ld, const int64_t *d_step, double dt,
                                          float *f4) {
  const double t = (double)(*d_step) * dt;
  for (int l = threadIdx.x; l < Ld.n; l += blockDim.x) {
    const int64_t dof = Ld.dof[l];
    const float v = (float)(-Ld.amp[l] * wavelet_value(Ld.kind[l], t, Ld.t1[l], Ld.ncyc[l]));
    atomicAdd(&f4[4 * (dof / 3) + dof % 3], v);
  }
}

__global__ void __launch_bounds__(TC_THREADS, 4)
    k_force_tc(const TcTile *__restrict__ tiles, int ntiles, const uint8_t *__restrict__ recs,
               const float *__restrict__ Bg, const float *__restrict__ u,
               float *__restrict__ f4, LoadTable Ld, const int64_t *__restrict__ d_step,
               double dt, int32_t *flags, int rec_max, int nn_max) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemLayout SL = smem_layout(rec_max, nn_max);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);   // [0] MMA, [1], [2] records
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(smem + 32);
  float *Bs = reinterpret_cast<float *>(smem + SL.B);
  float4 *F4 = reinterpret_cast<float4 *>(smem + SL.F);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int G = gridDim.x;
  const uint32_t mb_mma = tc::smem_addr(&mbar[0]);
  const uint32_t mb_rec0 = tc::smem_addr(&mbar[1]);   // stage s: mb_rec0 + 8 s

  if (warp == 0) {
    tc::tmem_alloc(tc::smem_addr(taddr_s), (uint32_t)TCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(mb_mma, 1);
    tc::mbar_init(mb_rec0, 1);
    tc::mbar_init(mb_rec0 + 8u, 1);
    tc::mbar_fence_init();
  }
  if (blockIdx.x == 0 && Ld.n > 0) add_loads(Ld, d_step, dt, f4);
  {   // B = K_p hi | lo (canonical layout), once per CTA
    const float4 *src = reinterpret_cast<const float4 *>(Bg);
    float4 *dst = reinterpret_cast<float4 *>(Bs);
    for (int q = tid; q < (2 * NPAD * KPAD) / 4; q += TC_THREADS) dst[q] = src[q];
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *taddr_s;

  auto stage_base = [&](int s) { return smem + (s ? SL.stage[1] : SL.stage[0]); };
  auto issue_record = [&](int s, const TcTile &T) {   // thread 0 only
    tc::fence_proxy_async_smem();
    const uint32_t mb = mb_rec0 + 8u * (uint32_t)s;
    tc::mbar_arrive_expect_tx(mb, (uint32_t)T.rec_bytes);
    tc::bulk_g2s(tc::smem_addr(stage_base(s)), recs + T.rec_off, (uint32_t)T.rec_bytes, mb);
  };
  auto issue_gather = [&](int s) {            // all threads
    const Stage S = stage_view(stage_base(s), SL.u_off);
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
  int tile = blockIdx.x;
  if (tile < ntiles) {
    if (tid == 0) {
      issue_record(0, tiles[tile]);
      if (tile + G < ntiles) issue_record(1, tiles[tile + G]);
    }
    pend = 1u | (tile + G < ntiles ? 2u : 0u);
    ok = __syncthreads_and(tc::mbar_wait_bounded(mb_rec0, ph_rec & 1u, WAIT_POLLS));
    if (ok) {
      ph_rec ^= 1u;
      pend &= ~1u;
      issue_gather(0);
    }
  }
  // thread (c, h): cell c (= TMEM lane) and its slots 4h .. 4h + 3
  const int fc = tid & 127, fh = tid >> 7;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  TcTile ahead;   // descriptor of the tile after next (thread 0), fetched a tile early
  for (int i = 0; ok && tile < ntiles; ++i, tile += G) {
    const int s = i & 1;
    const uint32_t so = (uint32_t)(s ^ 1);
    const int next = tile + G;
    // this tile's node pairs (own cp.async, issued during the previous tile)
    tc::cp_async_wait_all();
    __syncthreads();
    // every warp is past the previous tile: its stage takes the next record
    if (i > 0 && next < ntiles) {
      if (tid == 0) issue_record((int)so, ahead);
      pend |= 1u << so;
    }
    if (tid == 0 && next + G < ntiles) ahead = tiles[next + G];
    const Stage S = stage_view(stage_base(s), SL.u_off);
    const int ncell = S.hdr[1], nn = S.hdr[2];
    const bool brick = S.hdr[3] == 1;
    // A rows: differences to slot 0, TF32 hi + lo, into TMEM columns
    // COL_AHI / COL_ALO + 12 h .. + 11 of lane = cell (rows past ncell: 0)
    {
      float vh[12], vl[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) vh[q] = vl[q] = 0.0f;
      if (fc < ncell) {
        uint32_t lw0, lw1, l0;   // local node indices of slots 4h .. 4h + 3 (2 x u16), slot 0
        if (brick) {   // lattice: slot k = corner (k & 1, k >> 1 & 1, k >> 2)
          const int b0 = (fc & 3) + 5 * ((fc >> 2) & 3) + 25 * (fc >> 4) + 25 * fh;
          l0 = (uint32_t)(b0 - 25 * fh);
          lw0 = (uint32_t)b0 | (uint32_t)(b0 + 1) << 16;
          lw1 = (uint32_t)(b0 + 5) | (uint32_t)(b0 + 6) << 16;
        } else {
          const uint4 L = *reinterpret_cast<const uint4 *>(S.lid + 8 * fc);
          lw0 = fh ? L.z : L.x;
          lw1 = fh ? L.w : L.y;
          l0 = L.x & 0xFFFFu;
        }
        const float *ref = S.u + 6 * l0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t lk = ((t < 2 ? lw0 : lw1) >> (16 * (t & 1))) & 0xFFFFu;
          float d[3];
          node_diff(S.u + 6 * lk, ref, d[0], d[1], d[2]);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            vh[3 * t + r] = tc::to_tf32(d[r]);
            vl[3 * t + r] = tc::to_tf32(d[r] - vh[3 * t + r]);
          }
        }
      }
      const uint32_t col = (uint32_t)(12 * fh);
      const float h8[8] = {vh[0], vh[1], vh[2], vh[3], vh[4], vh[5], vh[6], vh[7]};
      const float l8[8] = {vl[0], vl[1], vl[2], vl[3], vl[4], vl[5], vl[6], vl[7]};
      tc::tmem_st8(taddr + lane_base + COL_AHI + col, h8);
      tc::tmem_st4(taddr + lane_base + COL_AHI + col + 8u, vh[8], vh[9], vh[10], vh[11]);
      tc::tmem_st8(taddr + lane_base + COL_ALO + col, l8);
      tc::tmem_st4(taddr + lane_base + COL_ALO + col + 8u, vl[8], vl[9], vl[10], vl[11]);
      tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, NPAD);
      const uint32_t b_hi = tc::smem_addr(Bs), b_lo = tc::smem_addr(Bs + NPAD * KPAD);
      const uint32_t sbo = (uint32_t)NK * 128u;
#pragma unroll
      for (int ks = 0; ks < KPAD / 8; ++ks) {
        const uint32_t o = (uint32_t)ks * 256u;
        const uint64_t bh = tc::smem_desc(b_hi + o, 128, sbo), bl = tc::smem_desc(b_lo + o, 128, sbo);
        const uint32_t ah = taddr + COL_AHI + 8u * ks, al = taddr + COL_ALO + 8u * ks;
        tc::mma_tf32_ta(taddr, ah, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ta(taddr, ah, bl, idesc, 1u);
        tc::mma_tf32_ta(taddr, al, bh, idesc, 1u);
      }
      tc::mma_commit(mb_mma);
    }
    // while the MMAs run: the next tile's record (issued a tile ago) and
    // the gather of its node pairs
    bool got = true;
    if (next < ntiles) {
      got = tc::mbar_wait_bounded(mb_rec0 + 8u * so, (ph_rec >> so) & 1u, WAIT_POLLS);
      if (got) issue_gather(s ^ 1);
    }
    got = tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_POLLS) && got;
    ok = __syncthreads_and(got);
    tc::fence_after_sync();
    if (!ok) break;
    ph_mma ^= 1u;
    if (next < ntiles) {
      ph_rec ^= 1u << so;
      pend &= ~(1u << so);
    }
    // epilogue: warps w and w + 4 read TMEM lanes 32 (w % 4) .. + 31, columns
    // 12 h .. 12 h + 11 (cell, slots 4 h .. 4 h + 3) times E h
    {
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
      tc::fence_before_sync();
      if (brick) {
        const float sc = S.scale[fc];
#pragma unroll
        for (int q = 0; q < 12; ++q) v[q] *= sc;
        brick_node_sums(S, v, warp, tid & 31, fh, f4);
      } else if (fc < ncell) {
        const float sc = S.scale[fc];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          F4[(4 * fh + t) * 128 + fc] =
              make_float4(sc * v[3 * t], sc * v[3 * t + 1], sc * v[3 * t + 2], 0.0f);
      }
    }
    __syncthreads();
    // list tiles: node sums over the incidences (cell, slot), at most 8 per node
    if (!brick) {
      for (int q = tid; q < nn; q += TC_THREADS) {
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
        const int j0 = S.off[q], nj = S.off[q + 1] - j0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < nj) {
            const int e = S.inc[j0 + j];
            const float4 w = F4[((e & 31) << 7) | (e >> 5)];
            a0 += w.x;
            a1 += w.y;
            a2 += w.z;
          }
        }
        red_add_v4(f4 + 4 * (int64_t)S.nodes[q], a0, a1, a2);
      }
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
  if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)TCOLS);
}

// ------------------------------------------------- Walsh-basis SIMT variant
// The same tiles, records and node sums as k_force_tc, one thread per cell
// (128 threads per tile) and no tensor cores: the regular cell's K_p is
// block-diagonal in the Walsh basis of its corners (eight 3 x 3 blocks;
// see mesh_upload), so the differences to slot 0 are Walsh-transformed per
// component, multiplied block by block and transformed back in FP32
// registers (~300 operations per cell against a 24 x 24 contraction).
constexpr int WT_THREADS = 128;

struct WhtF {
  float blk[72];   // blocks of T K_p T^T / 8, divided by 8 once more (T T^T = 8 I)
};

// Local order of a list tile's nodes (host side).  A half-warp of the
// force kernels' threads reads, for one corner, the node pairs of 16 cells
// at a 24-byte stride: nodes whose local indices agree mod 16 share a pair
// of shared-memory banks.  The order keeps the indices a permutation of
// 0 .. nn-1 and gives each node the residue mod 16 that clashes least with
// the residues already taken in the (half-warp, corner) sets it belongs to
// (nodes in the most sets first); lid, the incidence lists and the node
// list are renumbered to match.
inline void bank_aware_order(size_t nc, std::vector<int32_t> &nodes, std::vector<uint16_t> &lid,
                             std::vector<uint16_t> &offs, std::vector<uint16_t> &inc) {
  const int nn = (int)nodes.size();
  int cap[16] = {0};
  for (int j = 0; j < nn; ++j) cap[j & 15]++;
  std::vector<std::vector<int>> sets((size_t)nn);   // (half-warp, corner) set ids per node
  for (size_t c = 0; c < nc; ++c)
    for (int k = 0; k < 8; ++k) sets[lid[c * 8 + k]].push_back((int)(c / 16) * 8 + k);
  std::vector<uint32_t> taken(((nc + 15) / 16) * 8, 0u);   // bit r: residue r used in the set
  std::vector<int> ord((size_t)nn);
  for (int i = 0; i < nn; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int a, int b) { return sets[a].size() > sets[b].size(); });
  std::vector<int> res((size_t)nn, 0);
  for (int i : ord) {
    int best = -1, bcost = 1 << 30;
    for (int r = 0; r < 16; ++r) {
      if (!cap[r]) continue;
      int cost = 0;
      for (int sid : sets[i]) cost += (int)((taken[sid] >> r) & 1u);
      if (cost < bcost || (cost == bcost && cap[r] > cap[best])) {
        best = r;
        bcost = cost;
      }
    }
    res[i] = best;
    cap[best]--;
    for (int sid : sets[i]) taken[sid] |= 1u << best;
  }
  int next[16];
  for (int r = 0; r < 16; ++r) next[r] = r;
  std::vector<int> perm((size_t)nn), inv((size_t)nn);
  for (int i = 0; i < nn; ++i) {
    perm[i] = next[res[i]];
    next[res[i]] += 16;
    inv[perm[i]] = i;
  }
  std::vector<int32_t> nodes2((size_t)nn);
  for (int i = 0; i < nn; ++i) nodes2[perm[i]] = nodes[i];
  for (auto &l : lid) l = (uint16_t)perm[l];
  std::vector<uint16_t> offs2, inc2;
  offs2.reserve(offs.size());
  inc2.reserve(inc.size());
  for (int j = 0; j < nn; ++j) {
    offs2.push_back((uint16_t)inc2.size());
    const int o = inv[j];
    for (int q = offs[o]; q < offs[o + 1]; ++q) inc2.push_back(inc[q]);
  }
  offs2.push_back((uint16_t)inc2.size());
  nodes.swap(nodes2);
  offs.swap(offs2);
  inc.swap(inc2);
}

// Shared-memory slot of brick-lattice node q = a + 5 b + 25 c in the Walsh
// kernel: layer c at 37 c, row-major with a row pitch of 4 for a < 4 and
// the fifth column after the layer's rows.  Slot mod 16 = (a + 4 b) mod 16
// (+ the layer's offset), so the 16 nodes that a half-warp's cells read
// for one corner (a 4 x 4 window of a layer) fall on 16 different pairs of
// banks at the 24-byte node stride (lattice order puts q and q + 16 on the
// same banks).
constexpr int WT_BRICK_SLOTS = 9 * 37;
__host__ __device__ inline int wt_brick_slot(int q) {
  const int a = q % 5, b = (q / 5) % 5, c = q / 25;
  return 37 * c + (a < 4 ? a + 4 * b : 20 + 4 * b);
}

struct WtLayout {
  uint32_t stage[2], u_off, total;
};
__host__ __device__ inline WtLayout wt_layout(int rec_max, int nn_max) {
  WtLayout L;
  uint32_t o = 128;   // 2 record mbarriers
  L.u_off = a16((uint32_t)rec_max);
  const int slots = nn_max > WT_BRICK_SLOTS ? nn_max : WT_BRICK_SLOTS;
  const uint32_t st = a128(L.u_off + 24u * (uint32_t)slots);
  L.stage[0] = o; o += st;
  L.stage[1] = o; o += st;
  L.total = o;
  return L;
}

__device__ __forceinline__ void wht8f(float *x) {
#pragma unroll
  for (int h = 1; h < 8; h <<= 1)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if ((i & h) == 0) {
        const float a = x[i], b = x[i + h];
        x[i] = a + b;
        x[i + h] = a - b;
      }
}

// The same transform on (x, y) pairs of components held as float2: Blackwell's
// packed FP32 arithmetic does both lanes in one instruction.  a - b is
// b * (-1) + a (an exact product, one rounding), so the results equal the
// scalar transform's bit for bit.
__device__ __forceinline__ void wht8f2(float2 *x) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
  for (int h = 1; h < 8; h <<= 1)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if ((i & h) == 0) {
        const float2 a = x[i], b = x[i + h];
        x[i] = __fadd2_rn(a, b);
        x[i + h] = __ffma2_rn(b, m1, a);
      }
}

__global__ void __launch_bounds__(WT_THREADS, 6)
    k_force_wht32(const TcTile *__restrict__ tiles, int ntiles, const uint8_t *__restrict__ recs,
                  const WhtF Kw, const float *__restrict__ u, float *__restrict__ f4, LoadTable Ld,
                  const int64_t *__restrict__ d_step, double dt, int32_t *flags, int rec_max,
                  int nn_max) {
  extern __shared__ __align__(128) unsigned char smem[];
  const WtLayout SL = wt_layout(rec_max, nn_max);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);   // [0], [1] records of stage 0, 1
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  const uint32_t mb_rec0 = tc::smem_addr(&mbar[0]);
  if (tid == 0) {
    tc::mbar_init(mb_rec0, 1);
    tc::mbar_init(mb_rec0 + 8u, 1);
    tc::mbar_fence_init();
  }
  if (blockIdx.x == 0 && Ld.n > 0) add_loads(Ld, d_step, dt, f4);
  __syncthreads();

  auto stage_base = [&](int s) { return smem + (s ? SL.stage[1] : SL.stage[0]); };
  auto issue_record = [&](int s, const TcTile &T) {   // thread 0 only
    tc::fence_proxy_async_smem();
    const uint32_t mb = mb_rec0 + 8u * (uint32_t)s;
    tc::mbar_arrive_expect_tx(mb, (uint32_t)T.rec_bytes);
    tc::bulk_g2s(tc::smem_addr(stage_base(s)), recs + T.rec_off, (uint32_t)T.rec_bytes, mb);
  };
  auto issue_gather = [&](int s) {            // all threads
    const Stage S = stage_view(stage_base(s), SL.u_off);
    const int nn = S.hdr[2];
    const bool brick = S.hdr[3] == 1;
    const uint32_t ub = tc::smem_addr(S.u);
    for (int i = tid; i < nn; i += WT_THREADS) {
      const float *src = u + 6 * (int64_t)S.nodes[i];
      const uint32_t d = ub + 24u * (uint32_t)(brick ? wt_brick_slot(i) : i);
      tc::cp_async8(d, src);
      tc::cp_async8(d + 8u, src + 2);
      tc::cp_async8(d + 16u, src + 4);
    }
    tc::cp_async_commit();
  };

  uint32_t ph_rec = 0u, pend = 0u;
  bool ok = true;
  int tile = blockIdx.x;
  if (tile < ntiles) {
    if (tid == 0) {
      issue_record(0, tiles[tile]);
      if (tile + G < ntiles) issue_record(1, tiles[tile + G]);
    }
    pend = 1u | (tile + G < ntiles ? 2u : 0u);
    ok = __syncthreads_and(tc::mbar_wait_bounded(mb_rec0, ph_rec & 1u, WAIT_POLLS));
    if (ok) {
      ph_rec ^= 1u;
      pend &= ~1u;
      issue_gather(0);
    }
  }
  const int fc = tid;   // this thread's cell
  TcTile ahead;         // descriptor of the tile after next (thread 0), fetched a tile early
  for (int i = 0; ok && tile < ntiles; ++i, tile += G) {
    const int s = i & 1;
    const uint32_t so = (uint32_t)(s ^ 1);
    const int next = tile + G;
    tc::cp_async_wait_all();
    __syncthreads();
    if (i > 0 && next < ntiles) {   // every thread is past the previous tile: its stage is free
      if (tid == 0) issue_record((int)so, ahead);
      pend |= 1u << so;
    }
    if (tid == 0 && next + G < ntiles) ahead = tiles[next + G];
    const Stage S = stage_view(stage_base(s), SL.u_off);
    const int ncell = S.hdr[1], nn = S.hdr[2];
    const bool brick = S.hdr[3] == 1;
    // o[r][k]: component r at corner k = a + 2 b + 4 c of this cell's force
    float o[3][8];
    if (fc < ncell) {
      uint32_t lk[8];
      if (brick) {   // wt_brick_slot of lattice node (x + dx) + 5 (y + dy) + 25 (z + dz)
        const int x = fc & 3;
        const int b0 = x + 4 * ((fc >> 2) & 3) + 37 * (fc >> 4);
        const int sx = x < 3 ? 1 : 17;   // the +x corner: next column, or the layer's fifth
#pragma unroll
        for (int k = 0; k < 8; ++k)
          lk[k] = (uint32_t)(b0 + (k & 1) * sx + 4 * ((k >> 1) & 1) + 37 * (k >> 2));
      } else {
        const uint4 Lw = *reinterpret_cast<const uint4 *>(S.lid + 8 * fc);
        const uint32_t w4[4] = {Lw.x, Lw.y, Lw.z, Lw.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) lk[k] = (w4[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
      }
      // differences to slot 0: (x, y) as packed pairs, z scalar; corner 0's are 0
      float2 X[8];
      float Z[8];
      X[0] = make_float2(0.0f, 0.0f);
      Z[0] = 0.0f;
      {
        const float *ref = S.u + 6 * lk[0];
        const float2 ra = *reinterpret_cast<const float2 *>(ref);       // hx hy
        const float2 rb = *reinterpret_cast<const float2 *>(ref + 2);   // hz lx
        const float2 rc = *reinterpret_cast<const float2 *>(ref + 4);   // ly lz
        const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
        for (int k = 1; k < 8; ++k) {
          const float *p = S.u + 6 * lk[k];
          const float2 a = *reinterpret_cast<const float2 *>(p);
          const float2 b = *reinterpret_cast<const float2 *>(p + 2);
          const float2 c = *reinterpret_cast<const float2 *>(p + 4);
          X[k] = __fadd2_rn(__ffma2_rn(ra, m1, a), make_float2(b.y - rb.y, c.x - rc.x));
          Z[k] = (b.x - rb.x) + (c.y - rc.y);
        }
      }
      wht8f2(X);
      wht8f(Z);
      float2 Y[8];
      float YZ[8];
#pragma unroll
      for (int sb = 0; sb < 8; ++sb) {
        const float *B = Kw.blk + 9 * sb;
        const float v0 = X[sb ^ 1].x, v1 = X[sb ^ 2].y, v2 = Z[sb ^ 4];
        Y[sb ^ 1].x = fmaf(B[0], v0, fmaf(B[1], v1, B[2] * v2));
        Y[sb ^ 2].y = fmaf(B[3], v0, fmaf(B[4], v1, B[5] * v2));
        YZ[sb ^ 4] = fmaf(B[6], v0, fmaf(B[7], v1, B[8] * v2));
      }
      wht8f2(Y);
      wht8f(YZ);
      const float sc = S.scale[fc];
      const float2 sc2 = make_float2(sc, sc);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float2 q = __fmul2_rn(sc2, Y[k]);
        o[0][k] = q.x;
        o[1][k] = q.y;
        o[2][k] = sc * YZ[k];
      }
    }
    // the next tile's record (issued a tile ago) and the gather of its node
    // pairs, under this tile's node sums
    bool got = true;
    if (next < ntiles) {
      got = tc::mbar_wait_bounded(mb_rec0 + 8u * so, (ph_rec >> so) & 1u, WAIT_POLLS);
      if (got) issue_gather((int)so);
    }
    ok = __syncthreads_and(got);
    if (!ok) break;
    if (next < ntiles) {
      ph_rec ^= 1u << so;
      pend &= ~(1u << so);
    }
    if (brick) {
      if (fc < ncell) {   // (whole warps: a brick has 128 cells)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[12];
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int r = 0; r < 3; ++r) v[3 * t + r] = o[r][4 * h + t];
          brick_node_sums(S, v, warp, lane, h, f4);
        }
      }
    } else if (fc < ncell) {   // list tile: one vector reduction per corner
      const uint4 Lw = *reinterpret_cast<const uint4 *>(S.lid + 8 * fc);
      const uint32_t w4[4] = {Lw.x, Lw.y, Lw.z, Lw.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int lk = (int)((w4[k >> 1] >> (16 * (k & 1))) & 0xFFFFu);
        red_add_v4(f4 + 4 * (int64_t)S.nodes[lk], o[0][k], o[1][k], o[2][k]);
      }
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(flags, 2);
    tc::cp_async_wait_all();
    if (pend & 1u) tc::mbar_wait_bounded(mb_rec0, ph_rec & 1u, WAIT_POLLS);
    if (pend & 2u) tc::mbar_wait_bounded(mb_rec0 + 8u, (ph_rec >> 1) & 1u, WAIT_POLLS);
  }
}

// Cells of the other patterns: one tile (<= 32 cells of pattern p) per CTA.
// K_p and the tile's node pairs arrive by cp.async (node ids loaded first,
// all at once); D[c][j] (FP32 differences to slot 0, master frame; row
// stride ds),
// F[i][c] = E h sum_j K_p[i][j] D[c][j] with K_p rows padded to mp (a
// multiple of 4).  Warp g owns rows g, g + 8, ..., lane = cell: per four j
// one 16-byte load of D (conflict-free: ds / 4 is odd) serves up to ten
// rows, each a broadcast 16-byte load of K_p and four FFMA.
constexpr int GEN_RMAX = 10;   // rows per warp: ceil(78 / 8)
constexpr int GEN_THREADS = 256;
constexpr int GEN_Q = 4;       // (cell, slot) items per thread: 26 * 32 <= 4 * 256
__host__ __device__ inline int gen_mp(int m) { return (m + 3) & ~3; }
__host__ __device__ inline int gen_ds(int m) {
  const int mp = gen_mp(m);
  return ((mp >> 2) & 1) ? mp : mp + 4;
}
// F[i][lane] = sc sum_j K_p[i][j] D[lane][j] for the rows i = g + 8 r, r < R
// (the last group may run past m).
template <int R>
__device__ __forceinline__ void gen_contract(const float *Ks, const float *Dc, float *F, int mp,
                                             int m, int g, int lane, float sc) {
  float acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0f;
  const bool last = g + 8 * (R - 1) < m;
  for (int j = 0; j < mp; j += 4) {
    const float4 x = *reinterpret_cast<const float4 *>(Dc + j);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r == R - 1 && !last) break;
      const float4 k = *reinterpret_cast<const float4 *>(Ks + (g + 8 * r) * mp + j);
      acc[r] = fmaf(k.x, x.x, fmaf(k.y, x.y, fmaf(k.z, x.z, fmaf(k.w, x.w, acc[r]))));
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (g + 8 * r < m) F[(g + 8 * r) * GEN_TILE + lane] = sc * acc[r];
}

__global__ void __launch_bounds__(GEN_THREADS) k_force_gen(const Tile *__restrict__ tiles, MeshView M,
                                                   const float *__restrict__ Kpad,
                                                   const int64_t *__restrict__ kpoff,
                                                   const float *__restrict__ u,
                                                   float *__restrict__ f4, LoadTable Ld,
                                                   const int64_t *__restrict__ d_step,
                                                   double dt) {
  const Tile t = tiles[blockIdx.x];
  const int p = t.pat, m = M.pat_m[p], n = m / 3, nc = t.ncell;
  const int mp = gen_mp(m), ds = gen_ds(m);
  const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
  extern __shared__ __align__(16) unsigned char smem_g[];
  float *Ks = reinterpret_cast<float *>(smem_g);   // [m][mp]
  float *D = Ks + m * mp;                         // [32][ds]
  float *F = D + GEN_TILE * ds;                   // [m][32]
  float *U = F + m * GEN_TILE;                    // [n][32] node pairs (hi, lo), item k * 32 + c
  if (blockIdx.x == 0 && Ld.n > 0) add_loads(Ld, d_step, dt, f4);
  {   // K_p rows padded to mp in global memory (16-byte aligned per pattern)
    const float *src = Kpad + kpoff[p];
    const uint32_t dst = tc::smem_addr(Ks);
    for (int q = tid; q < (m * mp) >> 2; q += blockDim.x) tc::cp_async16(dst + 16u * q, src + 4 * q);
  }
  const int64_t Cp = M.pat_ccount[p];
  const int32_t *cn = M.conn + M.conn_off[p] + t.cell0;
  const int64_t gbase = M.pat_cstart[p] + t.cell0;
  // item w = k * 32 + c (slot k of cell c): node ids first (independent
  // loads), then the node pairs by cp.async; the ids stay for the scatter
  // the item's cell is c = w % 32 = lane for every q: its op and E h are
  // loaded once, beside the node ids
  const int op_c = lane < nc ? (int)M.sym[gbase + lane] : 0;
  const float sc = lane < nc ? (float)M.scale[gbase + lane] : 0.0f;
  int32_t nodeq[GEN_Q];
#pragma unroll
  for (int q = 0; q < GEN_Q; ++q) {
    const int w = tid + q * GEN_THREADS;
    nodeq[q] = (w < n * GEN_TILE && (w & 31) < nc) ? cn[(int64_t)(w >> 5) * Cp + (w & 31)] : -1;
  }
  {
    const uint32_t ub = tc::smem_addr(U);
#pragma unroll
    for (int q = 0; q < GEN_Q; ++q) {
      if (nodeq[q] < 0) continue;
      const uint32_t d = ub + 24u * (uint32_t)(tid + q * GEN_THREADS);
      const float *src = u + 6 * (int64_t)nodeq[q];
      tc::cp_async8(d, src);
      tc::cp_async8(d + 8u, src + 2);
      tc::cp_async8(d + 16u, src + 4);
    }
    tc::cp_async_commit();
  }
  if (lane < nc)   // zero the padding columns of D
    for (int j = m + g; j < mp; j += 8) D[lane * ds + j] = 0.0f;
  tc::cp_async_wait_all();
  __syncthreads();
  // D[c][3 k + r]: differences to slot 0 in the master frame
  for (int w = tid; w < n * GEN_TILE; w += blockDim.x) {
    const int k = w >> 5, c = w & 31;
    float x[3] = {0.0f, 0.0f, 0.0f};
    if (c < nc) {
      float d[3];
      node_diff(U + 6 * w, U + 6 * c, d[0], d[1], d[2]);
      const int op = op_c;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int a = op_perm_of(op, r);
        const float y = a == 0 ? d[0] : (a == 1 ? d[1] : d[2]);
        x[r] = ((op >> r) & 1) ? -y : y;
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) D[c * ds + 3 * k + r] = x[r];
  }
  __syncthreads();
  {
    const float *Dc = D + lane * ds;
    switch ((m + 7) >> 3) {   // rows per warp, so that no unrolled row is idle
      case 1: gen_contract<1>(Ks, Dc, F, mp, m, g, lane, sc); break;
      case 2: gen_contract<2>(Ks, Dc, F, mp, m, g, lane, sc); break;
      case 3: gen_contract<3>(Ks, Dc, F, mp, m, g, lane, sc); break;
      case 4: gen_contract<4>(Ks, Dc, F, mp, m, g, lane, sc); break;
      case 5: gen_contract<5>(Ks, Dc, F, mp, m, g, lane, sc); break;
      case 6: gen_contract<6>(Ks, Dc, F, mp, m, g, lane, sc); break;
      case 7: gen_contract<7>(Ks, Dc, F, mp, m, g, lane, sc); break;
      case 8: gen_contract<8>(Ks, Dc, F, mp, m, g, lane, sc); break;
      case 9: gen_contract<9>(Ks, Dc, F, mp, m, g, lane, sc); break;
      default: gen_contract<GEN_RMAX>(Ks, Dc, F, mp, m, g, lane, sc); break;
    }
  }
  __syncthreads();
  // back to the cell frame, f_cell[perm r] = sgn r f_master[r]
#pragma unroll
  for (int q = 0; q < GEN_Q; ++q) {
    const int w = tid + q * GEN_THREADS;
    if (nodeq[q] < 0) continue;
    const int k = w >> 5, c = w & 31;
    const int op = op_c;
    float y[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float v = F[(3 * k + r) * GEN_TILE + c];
      const float sv = ((op >> r) & 1) ? -v : v;
      const int a = op_perm_of(op, r);
      y[0] += a == 0 ? sv : 0.0f;
      y[1] += a == 1 ? sv : 0.0f;
      y[2] += a == 2 ? sv : 0.0f;
    }
    red_add_v4(f4 + 4 * (int64_t)nodeq[q], y[0], y[1], y[2]);
  }
}

// ------------------------------------ hanging-node patterns on the tensor cores
// k_force_gen_tc: the cells of every pattern other than the identity-op
// 8-node cell, in tiles of up to 128 cells of one pattern (any op), on the
// 5th-generation tensor cores.  Persistent: CTA b takes tiles b, b + G, ...
//  * the tile's record (one 1-D bulk copy, issued while the previous tile's
//    MMAs and epilogue run): int32 {pat, ncell, n, 0}, float scale[128]
//    (E_e h_e), uint8 sym[128], int32 ids[n][128] (node ids, master node
//    order, slot-major);
//  * B = K_p of the pattern as TF32 hi | lo, NP x KP each in the canonical
//    no-swizzle K-major layout (NP = m rounded up to 16, KP = m rounded up
//    to 8, zero padding), one bulk copy whenever the pattern changes;
//  * A (128 x KP) = each cell's differences to its slot-0 node in the
//    master frame (op applied), TF32 hi and lo, written to tensor memory by
//    the threads (lane = cell; hi and lo interleaved every 8 columns);
//  * D (tensor memory, 128 x NP) = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
//    (tcgen05.mma kind::tf32, M128 N=NP K8, issued by one thread, completion
//    by tcgen05.commit on an mbarrier);
//  * epilogue: each cell's row of D (tcgen05.ld) times E_e h_e, back to the
//    cell frame, one vector reduction per node.
// Thread c = cell c of the tile; its nodes in groups of 8.
constexpr int GT_THREADS = 128;
constexpr int GT_GROUPS = 4;        // 8-node groups: up to 32 >= 26 nodes
constexpr uint32_t GT_COLS = 256;   // TMEM: D in 0..79, A from column 80 on
constexpr uint32_t GT_COL_A = 80;   // chunk ks: hi at 80 + 16 ks, lo at 88 + 16 ks
constexpr int GT_NPMAX = 80, GT_KPMAX = 80;
constexpr uint32_t GT_B_OFF = 128;   // B at 128, the record after the largest B of the mesh

__host__ __device__ inline int gt_kp(int m) { return (m + 7) & ~7; }
__host__ __device__ inline int gt_np(int m) { return (m + 15) & ~15; }
struct GtRec {
  uint32_t scale, sym, ids, bytes;
};
__host__ __device__ inline GtRec gt_rec_layout(int n) {
  GtRec R;
  R.scale = 16;
  R.sym = R.scale + 128u * 4u;
  R.ids = R.sym + 128u;
  R.bytes = R.ids + 128u * 4u * (uint32_t)n;
  return R;
}
__host__ __device__ inline uint32_t gt_rec_off(int b_floats_max) {
  return GT_B_OFF + 4u * (uint32_t)b_floats_max;
}
__host__ __device__ inline uint32_t gt_smem_bytes(int n_max, int b_floats_max) {
  return gt_rec_off(b_floats_max) + gt_rec_layout(n_max).bytes;
}

__global__ void __launch_bounds__(GT_THREADS, 1)
    k_force_gen_tc(const TcTile *__restrict__ tiles, int ntiles, const uint8_t *__restrict__ recs,
                   const float *__restrict__ Bg, const int64_t *__restrict__ boff,
                   const float *__restrict__ u, float *__restrict__ f4, LoadTable Ld,
                   const int64_t *__restrict__ d_step, double dt, int32_t *flags,
                   uint32_t rec_off) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);   // [0] record, [1] B, [2] MMA
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(smem + 32);
  float *Bs = reinterpret_cast<float *>(smem + GT_B_OFF);
  unsigned char *rec = smem + rec_off;
  const int tid = threadIdx.x, warp = tid >> 5, c = tid;
  const int G = gridDim.x;
  const uint32_t mb_rec = tc::smem_addr(&mbar[0]), mb_b = mb_rec + 8u, mb_mma = mb_rec + 16u;
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_addr(taddr_s), GT_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(mb_rec, 1);
    tc::mbar_init(mb_b, 1);
    tc::mbar_init(mb_mma, 1);
    tc::mbar_fence_init();
  }
  if (blockIdx.x == 0 && Ld.n > 0) add_loads(Ld, d_step, dt, f4);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *taddr_s;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;

  auto issue_record = [&](const TcTile &T) {   // thread 0
    tc::fence_proxy_async_smem();
    tc::mbar_arrive_expect_tx(mb_rec, (uint32_t)T.rec_bytes);
    tc::bulk_g2s(tc::smem_addr(rec), recs + T.rec_off, (uint32_t)T.rec_bytes, mb_rec);
  };
  auto issue_b = [&](int pat) {   // thread 0
    const int64_t o = boff[pat];
    const uint32_t bytes = (uint32_t)(boff[pat + 1] - o) * 4u;
    tc::fence_proxy_async_smem();
    tc::mbar_arrive_expect_tx(mb_b, bytes);
    tc::bulk_g2s(tc::smem_addr(Bs), Bg + o, bytes, mb_b);
  };

  uint32_t ph_rec = 0u, ph_b = 0u, ph_mma = 0u;
  bool pend_rec = false, pend_b = false, pend_mma = false, ok = true;
  int tile = blockIdx.x, bpat = -1;
  if (tile < ntiles) {
    const TcTile T = tiles[tile];
    if (tid == 0) {
      issue_record(T);
      issue_b(T.pat);
    }
    pend_rec = pend_b = true;
    bpat = T.pat;
  }
  for (; ok && tile < ntiles; tile += G) {
    const int next = tile + G;
    // this tile's record and B (issued during the previous tile)
    bool got = tc::mbar_wait_bounded(mb_rec, ph_rec, WAIT_POLLS);
    if (pend_b) got = tc::mbar_wait_bounded(mb_b, ph_b, WAIT_POLLS) && got;
    ok = __syncthreads_and(got);
    if (!ok) break;
    ph_rec ^= 1u;
    pend_rec = false;
    if (pend_b) {
      ph_b ^= 1u;
      pend_b = false;
    }
    const int32_t *hdr = reinterpret_cast<const int32_t *>(rec);
    const int ncell = hdr[1], n = hdr[2], m = 3 * n;
    const int KP = gt_kp(m), NP = gt_np(m);
    const GtRec R = gt_rec_layout(n);
    const bool live = c < ncell;
    const float sc = live ? reinterpret_cast<const float *>(rec + R.scale)[c] : 0.0f;
    const int op = live ? (int)rec[R.sym + c] : 0;
    const int32_t *ids = reinterpret_cast<const int32_t *>(rec + R.ids);
    int32_t id[GT_GROUPS][8];
    const int32_t id0 = live ? ids[c] : 0;
#pragma unroll
    for (int g = 0; g < GT_GROUPS; ++g)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = 8 * g + j;
        id[g][j] = (live && k < n) ? ids[k * 128 + c] : -1;
      }
    int sg[3], pm[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      sg[r] = (op >> r) & 1;
      pm[r] = op_perm_of(op, r);
    }
    __syncthreads();   // the record is read: its stage takes the next one
    if (tid == 0 && next < ntiles) issue_record(tiles[next]);
    pend_rec = next < ntiles;
    // A: master-frame differences to slot 0, TF32 hi / lo, into TMEM
    {
      float ref[6];
      if (live) {
        const float2 a = *reinterpret_cast<const float2 *>(u + 6 * (int64_t)id0);
        const float2 b = *reinterpret_cast<const float2 *>(u + 6 * (int64_t)id0 + 2);
        const float2 d = *reinterpret_cast<const float2 *>(u + 6 * (int64_t)id0 + 4);
        ref[0] = a.x; ref[1] = a.y; ref[2] = b.x; ref[3] = b.y; ref[4] = d.x; ref[5] = d.y;
      } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) ref[q] = 0.0f;
      }
#pragma unroll
      for (int g = 0; g < GT_GROUPS; ++g) {
        if (24 * g >= KP) break;   // uniform over the CTA's tile
        float p6[8][6];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (id[g][j] >= 0) {
            const float *src = u + 6 * (int64_t)id[g][j];
            const float2 a = *reinterpret_cast<const float2 *>(src);
            const float2 b = *reinterpret_cast<const float2 *>(src + 2);
            const float2 d = *reinterpret_cast<const float2 *>(src + 4);
            p6[j][0] = a.x; p6[j][1] = a.y; p6[j][2] = b.x;
            p6[j][3] = b.y; p6[j][4] = d.x; p6[j][5] = d.y;
          } else {
#pragma unroll
            for (int q = 0; q < 6; ++q) p6[j][q] = ref[q];
          }
        }
        float hi[24], lo[24];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float d[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) d[r] = (p6[j][r] - ref[r]) + (p6[j][3 + r] - ref[3 + r]);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const float y = pm[r] == 0 ? d[0] : (pm[r] == 1 ? d[1] : d[2]);
            const float x = sg[r] ? -y : y;
            hi[3 * j + r] = tc::to_tf32(x);
            lo[3 * j + r] = tc::to_tf32(x - hi[3 * j + r]);
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int ks = 3 * g + q;
          if (8 * ks >= KP) break;
          const float h8[8] = {hi[8 * q], hi[8 * q + 1], hi[8 * q + 2], hi[8 * q + 3],
                               hi[8 * q + 4], hi[8 * q + 5], hi[8 * q + 6], hi[8 * q + 7]};
          const float l8[8] = {lo[8 * q], lo[8 * q + 1], lo[8 * q + 2], lo[8 * q + 3],
                               lo[8 * q + 4], lo[8 * q + 5], lo[8 * q + 6], lo[8 * q + 7]};
          tc::tmem_st8(taddr + lane_base + GT_COL_A + 16u * (uint32_t)ks, h8);
          tc::tmem_st8(taddr + lane_base + GT_COL_A + 16u * (uint32_t)ks + 8u, l8);
        }
      }
      tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, NP);
      const uint32_t b_hi = tc::smem_addr(Bs), b_lo = b_hi + (uint32_t)(NP * KP) * 4u;
      const uint32_t sbo = (uint32_t)(KP / 4) * 128u;
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint32_t o = (uint32_t)ks * 256u;
        const uint64_t bh = tc::smem_desc(b_hi + o, 128, sbo), bl = tc::smem_desc(b_lo + o, 128, sbo);
        const uint32_t ah = taddr + GT_COL_A + 16u * (uint32_t)ks, al = ah + 8u;
        tc::mma_tf32_ta(taddr, ah, bh, idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ta(taddr, ah, bl, idesc, 1u);
        tc::mma_tf32_ta(taddr, al, bh, idesc, 1u);
      }
      tc::mma_commit(mb_mma);
    }
    pend_mma = true;
    got = tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_POLLS);
    ok = __syncthreads_and(got);
    tc::fence_after_sync();
    if (!ok) break;
    ph_mma ^= 1u;
    pend_mma = false;
    // B of the next tile's pattern, if it differs (the MMAs reading B are done)
    if (next < ntiles) {
      const int np_ = tiles[next].pat;
      if (np_ != bpat) {
        if (tid == 0) issue_b(np_);
        pend_b = true;
        bpat = np_;
      }
    }
    // epilogue: this cell's rows of D times E h, back to the cell frame
#pragma unroll
    for (int g = 0; g < GT_GROUPS; ++g) {
      if (24 * g >= NP) break;
      float v[24];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float v8[8];
        if (24 * g + 8 * q < NP) {
          tc::tmem_ld8(taddr + lane_base + (uint32_t)(24 * g + 8 * q), v8);
        } else {
#pragma unroll
          for (int z = 0; z < 8; ++z) v8[z] = 0.0f;
        }
#pragma unroll
        for (int z = 0; z < 8; ++z) v[8 * q + z] = v8[z];
      }
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (id[g][j] < 0) continue;
        float y[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float fv = sc * v[3 * j + r];
          const float s = sg[r] ? -fv : fv;
          y[0] += pm[r] == 0 ? s : 0.0f;
          y[1] += pm[r] == 1 ? s : 0.0f;
          y[2] += pm[r] == 2 ? s : 0.0f;
        }
        red_add_v4(f4 + 4 * (int64_t)id[g][j], y[0], y[1], y[2]);
      }
    }
    tc::fence_before_sync();
    __syncthreads();   // D is read: the next tile's MMAs may overwrite it
    tc::fence_after_sync();
  }
  if (!ok) {
    if (tid == 0) atomicOr(flags, 2);
    if (pend_rec) tc::mbar_wait_bounded(mb_rec, ph_rec, WAIT_POLLS);
    if (pend_b) tc::mbar_wait_bounded(mb_b, ph_b, WAIT_POLLS);
    if (pend_mma) tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_POLLS);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, GT_COLS);
}

// ------------------------- hanging-node patterns of the batched form, tcgen05
// k_force_batch_tc: the batched FP32 form's cells of every pattern other
// than the 8-node cell, on the tensor cores.  Fields [node][3][B] (entry
// (3 node + d) B + b); U_n as (hi, lo) FP32 pairs (float2).  Work item =
// (record of up to 128 cells of one pattern -- the k_force_gen_tc records
// and B blocks --, chunk of 32 load cases, a quarter of the record's
// cells); persistent CTAs over contiguous ranges of items.
// Per item, groups of 4 cells: TMEM lane 32 w + l = (cell 4 g + w, case
// 32 chunk + l) with warp w and lane l, so A (128 x KP) holds the 128
// (cell, case) rows of master-frame differences to slot 0, and D = A B^T
// (TF32 x 3 as above) their forces; the epilogue adds each row's node
// forces to f, coalesced over the warp's 32 cases.
constexpr int BTC_THREADS = 128;

__global__ void __launch_bounds__(BTC_THREADS, 2)
    k_force_batch_tc(const TcTile *__restrict__ tiles, int ntiles, int nchunks,
                     const uint8_t *__restrict__ recs, const float *__restrict__ Bg,
                     const int64_t *__restrict__ boff, const float2 *__restrict__ u,
                     float *__restrict__ f, int B, LoadTable Ld, const int64_t *__restrict__ d_step,
                     double dt, int32_t *flags, uint32_t rec_off) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);   // [0] record, [1] B, [2] MMA
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(smem + 32);
  float *Bs = reinterpret_cast<float *>(smem + GT_B_OFF);
  unsigned char *rec = smem + rec_off;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  const uint32_t mb_rec = tc::smem_addr(&mbar[0]), mb_b = mb_rec + 8u, mb_mma = mb_rec + 16u;
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_addr(taddr_s), GT_COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(mb_rec, 1);
    tc::mbar_init(mb_b, 1);
    tc::mbar_init(mb_mma, 1);
    tc::mbar_fence_init();
  }
  if (blockIdx.x == 0 && Ld.n > 0) {
    const double t = (double)(*d_step) * dt;
    for (int l = tid; l < Ld.n; l += BTC_THREADS)
      atomicAdd(&f[Ld.dof[l]], (float)(-Ld.amp[l] * wavelet_value(Ld.kind[l], t, Ld.t1[l], Ld.ncyc[l])));
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *taddr_s;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  uint32_t ph_rec = 0u, ph_b = 0u, ph_mma = 0u;
  bool pend_rec = false, pend_b = false, pend_mma = false, ok = true;
  int cur_tile = -1, bpat = -1;
  // items = (tile, chunk, quarter: 8 groups of 4 cells); CTA b takes a
  // contiguous range of them, so that it reuses the record and B
  const int per_tile = nchunks * 4, items = ntiles * per_tile;
  const int it0 = (int)((int64_t)items * blockIdx.x / G);
  const int it1 = (int)((int64_t)items * (blockIdx.x + 1) / G);
  for (int item = it0; ok && item < it1; ++item) {
    const int tile = item / per_tile, rem = item - tile * per_tile;
    const int chunk = rem >> 2, quarter = rem & 3;
    if (tile != cur_tile) {   // this item's record (and B when the pattern changes)
      const TcTile T = tiles[tile];
      if (tid == 0) {
        tc::fence_proxy_async_smem();
        tc::mbar_arrive_expect_tx(mb_rec, (uint32_t)T.rec_bytes);
        tc::bulk_g2s(tc::smem_addr(rec), recs + T.rec_off, (uint32_t)T.rec_bytes, mb_rec);
      }
      pend_rec = true;
      if (T.pat != bpat) {
        if (tid == 0) {
          const int64_t o = boff[T.pat];
          const uint32_t bytes = (uint32_t)(boff[T.pat + 1] - o) * 4u;
          tc::fence_proxy_async_smem();
          tc::mbar_arrive_expect_tx(mb_b, bytes);
          tc::bulk_g2s(tc::smem_addr(Bs), Bg + o, bytes, mb_b);
        }
        pend_b = true;
        bpat = T.pat;
      }
      bool got = tc::mbar_wait_bounded(mb_rec, ph_rec, WAIT_POLLS);
      if (pend_b) got = tc::mbar_wait_bounded(mb_b, ph_b, WAIT_POLLS) && got;
      ok = __syncthreads_and(got);
      if (!ok) break;
      ph_rec ^= 1u;
      pend_rec = false;
      if (pend_b) {
        ph_b ^= 1u;
        pend_b = false;
      }
      cur_tile = tile;
    }
    const int32_t *hdr = reinterpret_cast<const int32_t *>(rec);
    const int ncell = hdr[1], n = hdr[2], m = 3 * n;
    const int KP = gt_kp(m), NP = gt_np(m);
    const GtRec R = gt_rec_layout(n);
    const float *scl = reinterpret_cast<const float *>(rec + R.scale);
    const int32_t *ids = reinterpret_cast<const int32_t *>(rec + R.ids);
    const int64_t b = (int64_t)chunk * 32 + lane;
    for (int g = 8 * quarter; ok && g < 8 * quarter + 8 && 4 * g < ncell; ++g) {
      const int c = 4 * g + warp;
      const bool live = c < ncell;
      const int op = live ? (int)rec[R.sym + c] : 0;
      int sg[3], pm[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        sg[r] = (op >> r) & 1;
        pm[r] = op_perm_of(op, r);
      }
      // A: this (cell, case) row's master-frame differences to slot 0
      {
        float2 ref[3];
        const int64_t n0 = live ? ids[c] : 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          ref[a] = live ? u[(3 * n0 + a) * B + b] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < GT_GROUPS; ++q) {
          if (24 * q >= KP) break;   // uniform
          float x[24];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int k = 8 * q + j;
            float d[3] = {0.0f, 0.0f, 0.0f};
            if (live && k < n) {
              const int64_t nk = ids[k * 128 + c];
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                const float2 v = u[(3 * nk + a) * B + b];
                d[a] = (v.x - ref[a].x) + (v.y - ref[a].y);
              }
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              const float y = pm[r] == 0 ? d[0] : (pm[r] == 1 ? d[1] : d[2]);
              x[3 * j + r] = sg[r] ? -y : y;
            }
          }
#pragma unroll
          for (int h = 0; h < 3; ++h) {
            const int ks = 3 * q + h;
            if (8 * ks >= KP) break;
            float h8[8], l8[8];
#pragma unroll
            for (int z = 0; z < 8; ++z) {
              h8[z] = tc::to_tf32(x[8 * h + z]);
              l8[z] = tc::to_tf32(x[8 * h + z] - h8[z]);
            }
            tc::tmem_st8(taddr + lane_base + GT_COL_A + 16u * (uint32_t)ks, h8);
            tc::tmem_st8(taddr + lane_base + GT_COL_A + 16u * (uint32_t)ks + 8u, l8);
          }
        }
        tc::tmem_st_wait();
      }
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (tid == 0) {
        const uint32_t idesc = tc::idesc_tf32(128, NP);
        const uint32_t b_hi = tc::smem_addr(Bs), b_lo = b_hi + (uint32_t)(NP * KP) * 4u;
        const uint32_t sbo = (uint32_t)(KP / 4) * 128u;
        for (int ks = 0; ks < KP / 8; ++ks) {
          const uint32_t o = (uint32_t)ks * 256u;
          const uint64_t bh = tc::smem_desc(b_hi + o, 128, sbo), bl = tc::smem_desc(b_lo + o, 128, sbo);
          const uint32_t ah = taddr + GT_COL_A + 16u * (uint32_t)ks, al = ah + 8u;
          tc::mma_tf32_ta(taddr, ah, bh, idesc, ks > 0 ? 1u : 0u);
          tc::mma_tf32_ta(taddr, ah, bl, idesc, 1u);
          tc::mma_tf32_ta(taddr, al, bh, idesc, 1u);
        }
        tc::mma_commit(mb_mma);
      }
      pend_mma = true;
      ok = __syncthreads_and(tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_POLLS));
      tc::fence_after_sync();
      if (!ok) break;
      ph_mma ^= 1u;
      pend_mma = false;
      // epilogue: the row's forces times E h, back to the cell frame
      const float sc = live ? scl[c] : 0.0f;
#pragma unroll
      for (int q = 0; q < GT_GROUPS; ++q) {
        if (24 * q >= NP) break;   // uniform
        float v[24];
#pragma unroll
        for (int h = 0; h < 3; ++h) {
          float v8[8];
          if (24 * q + 8 * h < NP) {
            tc::tmem_ld8(taddr + lane_base + (uint32_t)(24 * q + 8 * h), v8);
          } else {
#pragma unroll
            for (int z = 0; z < 8; ++z) v8[z] = 0.0f;
          }
#pragma unroll
          for (int z = 0; z < 8; ++z) v[8 * h + z] = v8[z];
        }
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = 8 * q + j;
          if (!live || k >= n) continue;
          const int64_t nk = ids[k * 128 + c];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const float fv = sc * v[3 * j + r];
            atomicAdd(&f[(3 * nk + pm[r]) * B + b], sg[r] ? -fv : fv);
          }
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(flags, 2);
    if (pend_rec) tc::mbar_wait_bounded(mb_rec, ph_rec, WAIT_POLLS);
    if (pend_b) tc::mbar_wait_bounded(mb_b, ph_b, WAIT_POLLS);
    if (pend_mma) tc::mbar_wait_bounded(mb_mma, ph_mma, WAIT_POLLS);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, GT_COLS);
}

// Self-test of the bounded completion wait every tensor-core kernel uses:
// one thread waits on a fresh mbarrier (arrived on first when `arrive`),
// giving up after `polls` polls; a give-up sets bit 2 of the flags, which
// the host reports as SBX_ETIMEOUT.
__global__ void k_wait_selftest(int32_t *flags, uint32_t polls, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t mb = tc::smem_addr(&bar);
  tc::mbar_init(mb, 1);
  tc::mbar_fence_init();
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
  if (!tc::mbar_wait_bounded(mb, 0u, polls)) atomicOr(flags, 2);
}

size_t gen_smem(int m) {
  return (size_t)(m * gen_mp(m) + GEN_TILE * gen_ds(m) + m * GEN_TILE + 2 * m * GEN_TILE) *
         sizeof(float);
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

// Tables of the tensor-core kernels for the patterns marked in `use`: per
// pattern B = K_p as TF32 hi | lo in the canonical layout (offsets in
// floats, boff[P] = end; patterns not used get an empty range) and records
// of up to 128 consecutive cells, heaviest first.
int gt_setup(sbx_ctx *ctx, const std::vector<int32_t> &conn, const std::vector<int64_t> &conn_off,
             const std::vector<int64_t> &cnt, const std::vector<int64_t> &start,
             const std::vector<uint8_t> &sym_sorted, const std::vector<double> &scale_sorted,
             const std::vector<char> &use, std::string &err) {
  const int P = ctx->n_pat;
  std::vector<float> Bgt;
  std::vector<int64_t> boff(P + 1, 0);
  std::vector<uint8_t> recs;
  std::vector<std::pair<int64_t, TcTile>> tl;   // (cost, tile)
  int nmax = 1, bmax = 0;
  for (int p = 0; p < P; ++p) {
    boff[p] = (int64_t)Bgt.size();
    if (!use[p] || cnt[p] == 0) continue;
    const int np = ctx->pat_nodes[p], m = 3 * np;
    const int KP = gt_kp(m), NP = gt_np(m), NKc = KP / 4;
    bmax = std::max(bmax, 2 * NP * KP);
    Bgt.resize(Bgt.size() + 2 * (size_t)NP * KP, 0.0f);
    float *Bh = Bgt.data() + boff[p], *Bl = Bh + (size_t)NP * KP;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double kv = ctx->K_host[ctx->pat_koff[p] + (int64_t)i * m + j];
        const float hi = tf32_round_host((float)kv);
        const float lo = tf32_round_host((float)(kv - (double)hi));
        const size_t o = (size_t)(i >> 3) * NKc * 32 + (j >> 2) * 32 + (i & 7) * 4 + (j & 3);
        Bh[o] = hi;
        Bl[o] = lo;
      }
    nmax = std::max(nmax, np);
    const GtRec R = gt_rec_layout(np);
    const int64_t Cp = cnt[p];
    for (int64_t c0 = 0; c0 < Cp; c0 += 128) {
      const int nc = (int)std::min<int64_t>(128, Cp - c0);
      const size_t at = recs.size();
      recs.resize(at + R.bytes, 0);
      const int32_t hdr[4] = {p, nc, np, 0};
      put(recs, at, hdr, 4);
      std::vector<float> sc(128, 0.0f);
      std::vector<uint8_t> sy(128, 0);
      std::vector<int32_t> ids((size_t)np * 128, 0);
      for (int c = 0; c < nc; ++c) {
        sc[c] = (float)scale_sorted[start[p] + c0 + c];
        sy[c] = sym_sorted[start[p] + c0 + c];
        for (int k = 0; k < np; ++k)
          ids[(size_t)k * 128 + c] = conn[conn_off[p] + (int64_t)k * Cp + c0 + c];
      }
      put(recs, at + R.scale, sc.data(), 128);
      put(recs, at + R.sym, sy.data(), 128);
      put(recs, at + R.ids, ids.data(), ids.size());
      TcTile t;
      t.rec_off = (int64_t)at;
      t.rec_bytes = (int32_t)R.bytes;
      t.pat = p;
      tl.emplace_back((int64_t)NP * KP * nc, t);
    }
  }
  boff[P] = (int64_t)Bgt.size();
  std::stable_sort(tl.begin(), tl.end(),
                   [](const std::pair<int64_t, TcTile> &a, const std::pair<int64_t, TcTile> &b) {
                     return a.first > b.first;
                   });
  std::vector<TcTile> tiles;
  for (auto &x : tl) tiles.push_back(x.second);
  auto up = [&](auto **dst, const auto &vec) -> int {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    if (cudaMalloc((void **)dst, std::max<size_t>(vec.size(), 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      err = "cudaMalloc failed (tensor-core pattern tables)";
      return SBX_ENOMEM;
    }
    if (!vec.empty() && cudaMemcpyAsync(*dst, vec.data(), vec.size() * sizeof(T),
                                        cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
      err = "copy of tensor-core pattern tables failed";
      return SBX_ECUDA;
    }
    return SBX_OK;
  };
  if (int rc = up(&ctx->d_gt_B, Bgt)) return rc;
  if (int rc = up(&ctx->d_gt_boff, boff)) return rc;
  if (int rc = up(&ctx->d_gt_rec, recs)) return rc;
  if (int rc = up(&ctx->d_gt_tiles, tiles)) return rc;
  ctx->n_gt_tiles = (int)tiles.size();
  ctx->gt_rec_off = gt_rec_off(bmax);
  ctx->gt_smem = gt_smem_bytes(nmax, bmax);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    err = "stream synchronisation failed";
    return SBX_ECUDA;
  }
  return SBX_OK;
}

// Host preparation: tile records of the 8-node cell (tensor-core kernel) and
// 32-cell tiles of every other pattern.
int tc_setup(sbx_ctx *ctx, const std::vector<int32_t> &conn, const std::vector<int64_t> &conn_off,
             const std::vector<int64_t> &cnt, const std::vector<int64_t> &start,
             const std::vector<uint8_t> &sym_sorted, const std::vector<double> &scale_sorted,
             std::string &err) {
  const int P = ctx->n_pat;
  std::vector<float> Bhl(2 * (size_t)NPAD * KPAD, 0.0f);
  std::vector<uint8_t> recs;
  std::vector<TcTile> tiles;
  std::vector<Tile> gen;
  int recmax = 16, nnmax = 1, gen_mmax = 3;
  std::vector<float> Kpad;                 // FP32 K_p, rows padded to gen_mp(m)
  std::vector<int64_t> kpoff(P, 0);
  std::vector<int64_t> mark(ctx->N, -1);   // node -> last tile that holds it
  int64_t stamp = 0;
  ctx->n_brick_tiles = 0;

  for (int p = 0; p < P; ++p) {
    if (cnt[p] == 0) continue;
    const int np = ctx->pat_nodes[p], m = 3 * np;
    bool ident = true;
    for (int64_t c = 0; c < cnt[p]; ++c) ident &= sym_sorted[start[p] + c] == 0;
    if (np != 8 || !ident) {
      const int mp = gen_mp(m);
      kpoff[p] = (int64_t)Kpad.size();
      Kpad.resize(Kpad.size() + (size_t)m * mp, 0.0f);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
          Kpad[kpoff[p] + (int64_t)i * mp + j] = (float)ctx->K_host[ctx->pat_koff[p] + (int64_t)i * m + j];
      for (int64_t c0 = 0; c0 < cnt[p]; c0 += GEN_TILE) {
        Tile t;
        t.pat = p;
        t.ncell = (int32_t)std::min<int64_t>(GEN_TILE, cnt[p] - c0);
        t.cell0 = c0;
        gen.push_back(t);
      }
      gen_mmax = std::max(gen_mmax, m);
      continue;
    }
    // B = K_p hi | lo in the canonical layout (rows 24 .. 31 zero)
    for (int i = 0; i < KM; ++i)
      for (int j = 0; j < KM; ++j) {
        const double kv = ctx->K_host[ctx->pat_koff[p] + (int64_t)i * KM + j];
        const float hi = tf32_round_host((float)kv);
        const float lo = tf32_round_host((float)(kv - (double)hi));
        const size_t o = (size_t)(i >> 3) * NK * 32 + (j >> 2) * 32 + (i & 7) * 4 + (j & 3);
        Bhl[o] = hi;
        Bhl[(size_t)NPAD * KPAD + o] = lo;
      }
    const int64_t Cp = cnt[p];
    auto corner = [&](int64_t j, int k) { return conn[conn_off[p] + (int64_t)k * Cp + j]; };
    // bricks: complete 4 x 4 x 8 blocks of same-size cells, found from the
    // connectivity (the +x / +y / +z neighbour of a cell is the cell whose
    // slot-0 node is its slot 1 / 2 / 4 node), greedily in Morton order
    std::vector<int64_t> c0(ctx->N, -1);
    for (int64_t j = 0; j < Cp; ++j) c0[corner(j, 0)] = j;
    auto step = [&](int64_t j, int k) -> int64_t {
      if (j < 0) return -1;
      const int64_t n = c0[corner(j, k)];
      return (n >= 0 && ctx->h_hs[start[p] + n] == ctx->h_hs[start[p] + j]) ? n : -1;
    };
    std::vector<char> used(Cp, 0);
    std::vector<std::pair<int64_t, TcTile>> ptiles;   // (first cell, tile) for ordering
    std::vector<int64_t> bc(BRICK_CELLS);
    for (int64_t j = 0; j < Cp; ++j) {
      if (used[j]) continue;
      bool ok = true;
      int64_t zc = j;
      for (int z = 0; z < BRICK_NZ && ok; ++z) {
        int64_t yc = zc;
        for (int y = 0; y < BRICK_NY && ok; ++y) {
          int64_t xc = yc;
          for (int x = 0; x < BRICK_NX && ok; ++x) {
            if (xc < 0 || used[xc]) {
              ok = false;
              break;
            }
            bc[x + BRICK_NX * y + BRICK_NX * BRICK_NY * z] = xc;
            if (x + 1 < BRICK_NX) xc = step(xc, 1);
          }
          if (y + 1 < BRICK_NY) yc = step(yc, 2);
        }
        if (z + 1 < BRICK_NZ) zc = step(zc, 4);
      }
      if (!ok) continue;
      int32_t nodes[BRICK_NODES];
      for (int q = 0; q < BRICK_NODES; ++q) {
        const int a = q % 5, b = (q / 5) % 5, c = q / 25;
        const int x = std::min(a, 3), y = std::min(b, 3), z = std::min(c, 7);
        nodes[q] = corner(bc[x + 4 * y + 16 * z], (a - x) + 2 * (b - y) + 4 * (c - z));
      }
      float sc[BRICK_CELLS];
      for (int c = 0; c < BRICK_CELLS; ++c) {
        used[bc[c]] = 1;
        sc[c] = (float)scale_sorted[start[p] + bc[c]];
      }
      const RecLayout R = rec_layout(BRICK_CELLS, BRICK_NODES, 1);
      const size_t at = recs.size();
      recs.resize(at + R.bytes, 0);
      const int32_t hdr[4] = {p, BRICK_CELLS, BRICK_NODES, 1};
      put(recs, at, hdr, 4);
      put(recs, at + R.scale, sc, BRICK_CELLS);
      put(recs, at + R.nodes, nodes, BRICK_NODES);
      TcTile t;
      t.rec_off = (int64_t)at;
      t.rec_bytes = (int32_t)R.bytes;
      t.pat = p;
      recmax = std::max(recmax, (int)R.bytes);
      nnmax = std::max(nnmax, BRICK_NODES);
      ptiles.emplace_back(j, t);
      ++ctx->n_brick_tiles;
    }
    // the other cells: list tiles, greedy cut at 128 cells or
    // FAST_NN_CAP unique nodes
    std::vector<int64_t> rest;
    for (int64_t j = 0; j < Cp; ++j)
      if (!used[j]) rest.push_back(j);
    std::vector<std::pair<int32_t, int32_t>> v;   // (node, cell * 32 + slot)
    for (size_t r0 = 0, nc = 0; r0 < rest.size(); r0 += nc) {
      ++stamp;
      int nn_new = 0;
      nc = 0;
      while (r0 + nc < rest.size() && nc < 128) {
        const int64_t j = rest[r0 + nc];
        int add = 0;
        for (int k = 0; k < 8; ++k)
          if (mark[corner(j, k)] != stamp) ++add;
        if (nc > 0 && nn_new + add > FAST_NN_CAP) break;
        for (int k = 0; k < 8; ++k) {
          const int32_t q = corner(j, k);
          if (mark[q] != stamp) {
            mark[q] = stamp;
            ++nn_new;
          }
        }
        ++nc;
      }
      v.clear();
      for (int k = 0; k < 8; ++k)
        for (size_t c = 0; c < nc; ++c) v.emplace_back(corner(rest[r0 + c], k), (int32_t)(c * 32 + k));
      std::sort(v.begin(), v.end());
      std::vector<int32_t> nodes;
      std::vector<uint16_t> lid((size_t)8 * nc, 0), offs, inc;
      for (size_t i = 0; i < v.size(); ++i) {
        if (i == 0 || v[i].first != v[i - 1].first) {
          nodes.push_back(v[i].first);
          offs.push_back((uint16_t)inc.size());
        }
        lid[(size_t)(v[i].second >> 5) * 8 + (v[i].second & 31)] = (uint16_t)(nodes.size() - 1);
        inc.push_back((uint16_t)v[i].second);
      }
      offs.push_back((uint16_t)inc.size());
      bank_aware_order(nc, nodes, lid, offs, inc);
      const int nn = (int)nodes.size();
      const RecLayout R = rec_layout((int)nc, nn, 0);
      const size_t at = recs.size();
      recs.resize(at + R.bytes, 0);
      std::vector<float> sc(nc);
      for (size_t c = 0; c < nc; ++c) sc[c] = (float)scale_sorted[start[p] + rest[r0 + c]];
      const int32_t hdr[4] = {p, (int32_t)nc, nn, 0};
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
      recmax = std::max(recmax, (int)R.bytes);
      nnmax = std::max(nnmax, nn);
      ptiles.emplace_back(rest[r0], t);
    }
    // tiles in Morton order of their first cell (neighbouring tiles run
    // together and share nodes in L2)
    std::stable_sort(ptiles.begin(), ptiles.end(),
                     [](const std::pair<int64_t, TcTile> &a, const std::pair<int64_t, TcTile> &b) {
                       return a.first < b.first;
                     });
    for (auto &pt : ptiles) tiles.push_back(pt.second);
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
  if (int rc = up(&ctx->d_tc_K, Bhl)) return rc;
  if (int rc = up(&ctx->d_tc_rec, recs)) return rc;
  if (int rc = up(&ctx->d_tc_tiles[0], tiles)) return rc;
  // largest patterns first (the CTAs are issued in order: long ones start
  // early, short ones fill the end)
  std::stable_sort(gen.begin(), gen.end(), [&](const Tile &a, const Tile &b) {
    const int na = ctx->pat_nodes[a.pat], nb = ctx->pat_nodes[b.pat];
    return na * na * a.ncell > nb * nb * b.ncell;   // ~ the tile's multiply-adds
  });
  if (int rc = up(&ctx->d_gen_tiles, gen)) return rc;
  if (int rc = up(&ctx->d_gen_K, Kpad)) return rc;
  if (int rc = up(&ctx->d_gen_koff, kpoff)) return rc;
  {   // the other patterns in the tensor-core form as well
    std::vector<char> use(P, 0);
    for (const Tile &t : gen) use[t.pat] = 1;
    if (int rc = gt_setup(ctx, conn, conn_off, cnt, start, sym_sorted, scale_sorted, use, err))
      return rc;
  }
  const int64_t nt = (int64_t)tiles.size();
  ctx->n_tc_tiles[0] = (int)nt;
  ctx->tc_rec_max[0] = recmax;
  ctx->tc_nn_max[0] = nnmax;
  ctx->tc_smem[0] = smem_layout(recmax, nnmax).total;
  ctx->n_gen_tiles = (int)gen.size();
  ctx->gen_smem = gen_smem(gen_mmax);
  const int nsm = ctx->n_sm;
  // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per
  // CTA), at most 4 (registers, tensor memory); 3 when k_force_gen runs
  // beside it
  int per_sm = (int)((228u * 1024u) / (ctx->tc_smem[0] + 1024u));
  per_sm = std::max(1, std::min(per_sm, gen.empty() ? 4 : 3));
  ctx->tc_grid[0] = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)nsm * per_sm));
  // Walsh-basis variant: 128 threads, no tensor memory, no staging of the
  // cell forces; 6 CTAs per SM (its launch bounds; 4, 5 and 7 measured
  // 1-2 % slower on the cavity cube, k_force_gen filling in as they finish)
  ctx->wt_smem = wt_layout(recmax, nnmax).total;
  int per_sm_w = (int)((228u * 1024u) / (ctx->wt_smem + 1024u));
  per_sm_w = std::max(1, std::min(per_sm_w, 8));
  ctx->wt_grid = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)nsm * per_sm_w));
  if (ctx->tc_smem[0] > 227u * 1024u) {
    err = "tensor-core tile needs more than 227 KB of shared memory";
    return SBX_EINVAL;
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    err = "stream synchronisation failed";
    return SBX_ECUDA;
  }
  return SBX_OK;
}

cudaError_t launch_wait_selftest(const sbx_ctx *ctx, uint32_t polls, int arrive, cudaStream_t s) {
  k_wait_selftest<<<1, 1, 0, s>>>(ctx->d_flags, polls, arrive);
  return cudaGetLastError();
}

cudaError_t prepare_tc_kernels() {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_force_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force_wht32, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force_gen_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)gt_smem_bytes(26, 2 * GT_NPMAX * GT_KPMAX));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_force_batch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)gt_smem_bytes(26, 2 * GT_NPMAX * GT_KPMAX));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_force_gen, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gen_smem(78));
}

cudaError_t launch_force_batch_tc(const sbx_ctx *ctx, const float *pairs, float *f, double dt,
                                  LoadTable L, cudaStream_t s) {
  const int nchunks = ctx->B / 32;
  const int items = ctx->n_gt_tiles * nchunks * 4;
  const int grid = std::max(1, std::min(items, 2 * ctx->n_sm));
  k_force_batch_tc<<<grid, BTC_THREADS, ctx->gt_smem, s>>>(
      ctx->d_gt_tiles, ctx->n_gt_tiles, nchunks, ctx->d_gt_rec, ctx->d_gt_B, ctx->d_gt_boff,
      reinterpret_cast<const float2 *>(pairs), f, ctx->B, L, ctx->d_step, dt, ctx->d_flags,
      ctx->gt_rec_off);
  return cudaGetLastError();
}

// The kernel of the regular cells and the kernel of the other patterns run
// side by side: the second one on the context's second stream (fork and
// join by events; also under capture), launched first.  Grids are sized so
// that both are resident together: with k_force_gen_tc (one CTA and 256
// TMEM columns per SM) the Walsh kernel takes 4 CTAs per SM (registers)
// and the tcgen05 kernel of the regular cells 2 (tensor memory).
cudaError_t launch_force_tc(const sbx_ctx *ctx, const float *pairs, float *f4, double dt,
                            cudaStream_t s) {
  LoadTable L = ctx->loads();   // added by CTA 0 of the first launch only
  const bool gtc = ctx->hanging_tc && ctx->n_gt_tiles > 0;
  const int n_hang = gtc ? ctx->n_gt_tiles : ctx->n_gen_tiles;
  const bool both = ctx->n_tc_tiles[0] > 0 && n_hang > 0;
  const int nsm = ctx->n_sm;
  cudaError_t e;
  if (both) {
    if ((e = cudaEventRecord(ctx->ev_fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0)) != cudaSuccess) return e;
  }
  if (n_hang > 0) {
    cudaStream_t sg = both ? ctx->side : s;
    if (gtc) {
      const int grid = std::min(ctx->n_gt_tiles, std::max(1, ctx->hanging_ctas) * nsm);
      k_force_gen_tc<<<grid, GT_THREADS, ctx->gt_smem, sg>>>(
          ctx->d_gt_tiles, ctx->n_gt_tiles, ctx->d_gt_rec, ctx->d_gt_B, ctx->d_gt_boff, pairs, f4,
          L, ctx->d_step, dt, ctx->d_flags, ctx->gt_rec_off);
    } else {
      k_force_gen<<<ctx->n_gen_tiles, GEN_THREADS, ctx->gen_smem, sg>>>(
          ctx->d_gen_tiles, ctx->view(), ctx->d_gen_K, ctx->d_gen_koff, pairs, f4, L, ctx->d_step,
          dt);
    }
    L.n = 0;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ctx->n_tc_tiles[0] > 0 && ctx->mixed_wht && ctx->wht_pat >= 0) {
    WhtF kw;
    for (int q = 0; q < 72; ++q) kw.blk[q] = (float)(ctx->wht.blk[q] * 0.125);
    const int per_sm = ctx->walsh_ctas > 0 ? ctx->walsh_ctas
                                           : (gtc ? (ctx->hanging_ctas > 1 ? 3 : 4) : 6);
    const int grid = std::max(1, std::min(ctx->wt_grid, per_sm * nsm));
    k_force_wht32<<<grid, WT_THREADS, ctx->wt_smem, s>>>(
        ctx->d_tc_tiles[0], ctx->n_tc_tiles[0], ctx->d_tc_rec, kw, pairs, f4, L, ctx->d_step, dt,
        ctx->d_flags, ctx->tc_rec_max[0], ctx->tc_nn_max[0]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else if (ctx->n_tc_tiles[0] > 0) {
    const int grid = gtc ? std::max(1, std::min(ctx->tc_grid[0], 2 * nsm)) : ctx->tc_grid[0];
    k_force_tc<<<grid, TC_THREADS, ctx->tc_smem[0], s>>>(
        ctx->d_tc_tiles[0], ctx->n_tc_tiles[0], ctx->d_tc_rec, ctx->d_tc_K, pairs, f4, L,
        ctx->d_step, dt, ctx->d_flags, ctx->tc_rec_max[0], ctx->tc_nn_max[0]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (both) {
    if ((e = cudaEventRecord(ctx->ev_join, ctx->side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, ctx->ev_join, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sbx

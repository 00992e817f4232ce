// Mixed-precision internal force on the 5th-generation tensor cores:
// a persistent, software-pipelined kernel.
//
// Work unit: a tile of up to 128 cells of one pattern p (m = 3 n_p DOFs) and
// the tile's unique nodes.  The host packs each tile into one contiguous
// record (layout below) that replaces the connectivity.  Each CTA (256
// threads) walks tiles blockIdx.x, +gridDim.x, ... with two stages:
//   * the record of tile i+2 streams in by one 1-D bulk copy (TMA engine,
//     completion on an mbarrier) and the displacements of tile i+1's nodes by
//     per-thread cp.async, while tile i is computed;
//   * tile i: A (128 x K) = each cell's displacements, transformed by its op
//     (Sec. 3.2.2) and minus its slot-0 node's displacement (K_p annihilates
//     translations), formed in FP32 from a bit-level FP64 -> (hi, lo) split,
//     rounded to TF32 hi + lo;  D (TMEM) = A_hi B_hi^T + A_hi B_lo^T +
//     A_lo B_hi^T with B = K_p split the same way (tcgen05.mma kind::tf32 by
//     one thread, completion by tcgen05.commit -> mbarrier);  tcgen05.ld D
//     (row = cell) times E_e h_e;  per node, sum Q^T F over its incidences in
//     FP32 and add it with one FP64 atomic per DOF.
// No FP64 arithmetic runs per incidence (GB300's FP64 pipe is ~1/64 of FP32).
// Operands use the canonical no-swizzle K-major layout: 8-row x 16-byte core
// matrices, row groups nK * 128 B apart, K groups 128 B apart within a row
// group (LBO = 128 B, SBO = nK * 128 B).
//
// Record layout (every part padded to 16 bytes):
//   int32 {pat, ncell, nn, n | ident << 16}  header (16 B); ident: every
//                                      cell of the tile has the identity op
//   uint8 sym[ncell]                   op of each cell
//   float scale[ncell]                 E_e h_e rounded to FP32
//   int32 nodes[nn]                    unique node ids, ascending
//   uint16 off[nn + 1]                 incidence offsets per node
//   uint16 inc[n * ncell]              incidences (cell << 5 | slot) by node
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

__host__ __device__ inline uint32_t a16(uint32_t x) { return (x + 15u) & ~15u; }
__host__ __device__ inline uint32_t a128(uint32_t x) { return (x + 127u) & ~127u; }

struct RecLayout {
  uint32_t sym, scale, nodes, off, inc, bytes;
};
__host__ __device__ inline RecLayout rec_layout(int ncell, int nn, int n) {
  RecLayout R;
  uint32_t o = 16;
  R.sym = o;   o += a16((uint32_t)ncell);
  R.scale = o; o += a16(4u * ncell);
  R.nodes = o; o += a16(4u * nn);
  R.off = o;   o += a16(2u * (nn + 1));
  R.inc = o;   o += a16(2u * n * ncell);
  R.bytes = o;
  return R;
}

struct SmemLayout {
  uint32_t B, A, ref, stage[2], u_off, total;
};
// kmax, nmax: padded K and N; rec_max: largest record; nn_max: most nodes
__host__ __device__ inline SmemLayout smem_layout(int kmax, int nmax, int rec_max, int nn_max) {
  SmemLayout L;
  uint32_t o = 128;                                    // 3 mbarriers + TMEM address
  L.B = o;   o = a128(o + 2u * nmax * kmax * 4u);
  L.A = o;   o = a128(o + 2u * 128u * kmax * 4u);
  L.ref = o; o = a128(o + 128u * ((kmax + 2) / 3) * 2u);  // lid[slot][cell], uint16
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
  const uint16_t *off, *inc;
  double *u;
};
__device__ inline Stage stage_view(unsigned char *base, uint32_t u_off) {
  Stage S;
  S.hdr = reinterpret_cast<const int32_t *>(base);
  const RecLayout R = rec_layout(S.hdr[1], S.hdr[2], S.hdr[3] & 0xFFFF);
  S.sym = base + R.sym;
  S.scale = reinterpret_cast<const float *>(base + R.scale);
  S.nodes = reinterpret_cast<const int32_t *>(base + R.nodes);
  S.off = reinterpret_cast<const uint16_t *>(base + R.off);
  S.inc = reinterpret_cast<const uint16_t *>(base + R.inc);
  S.u = reinterpret_cast<double *>(base + u_off);
  return S;
}

// One item of A: cell c, nodes 4 k4 .. 4 k4 + 3 (12 columns, three float4
// per operand).  d = (hi - hi_ref) + (lo - lo_ref) in FP32 with the cell's
// slot-0 node as reference, transformed by the op, split into TF32 hi + lo.
// A(c, col) -> float (c/8)*nK*32 + (c%8)*4 + (col/4)*32 + col%4.
template <bool IDENT>
__device__ __forceinline__ void build_a_item(int c, int k4, int op, const float *uf,
                                             const uint16_t *lid, int n, int nK, int kpad,
                                             float *Ahi, float *Alo) {
  int p0 = 0, p1 = 1, p2 = 2;
  float s0 = 1.0f, s1 = 1.0f, s2 = 1.0f;
  if (!IDENT) {
    p0 = op_perm_of(op, 0);
    p1 = op_perm_of(op, 1);
    p2 = op_perm_of(op, 2);
    s0 = (op & 1) ? -1.0f : 1.0f;
    s1 = (op & 2) ? -1.0f : 1.0f;
    s2 = (op & 4) ? -1.0f : 1.0f;
  }
  const float *rf = uf + 6 * lid[c];
  const float rh[3] = {rf[0], rf[1], rf[2]}, rl[3] = {rf[3], rf[4], rf[5]};
  const int rowoff = (c >> 3) * nK * 32 + (c & 7) * 4;
  float vh[12], vl[12];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int k = 4 * k4 + t;
    float d[3] = {0.0f, 0.0f, 0.0f};
    if (k < n) {
      const float *nf = uf + 6 * lid[k * 128 + c];
#pragma unroll
      for (int a = 0; a < 3; ++a) d[a] = (nf[a] - rh[a]) + (nf[3 + a] - rl[a]);
    }
    float x[3];
    if (IDENT) {
      x[0] = d[0];
      x[1] = d[1];
      x[2] = d[2];
    } else {
      x[0] = s0 * (p0 == 0 ? d[0] : (p0 == 1 ? d[1] : d[2]));
      x[1] = s1 * (p1 == 0 ? d[0] : (p1 == 1 ? d[1] : d[2]));
      x[2] = s2 * (p2 == 0 ? d[0] : (p2 == 1 ? d[1] : d[2]));
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      vh[3 * t + r] = tc::to_tf32(x[r]);
      vl[3 * t + r] = tc::to_tf32(x[r] - vh[3 * t + r]);
    }
  }
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const int q4 = 3 * k4 + g;   // float4 column group
    if (4 * q4 < kpad) {
      const int o = rowoff + q4 * 32;
      *reinterpret_cast<float4 *>(Ahi + o) =
          make_float4(vh[4 * g], vh[4 * g + 1], vh[4 * g + 2], vh[4 * g + 3]);
      *reinterpret_cast<float4 *>(Alo + o) =
          make_float4(vl[4 * g], vl[4 * g + 1], vl[4 * g + 2], vl[4 * g + 3]);
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 4)
    k_force_tc(const TcTile *__restrict__ tiles, int ntiles, const uint8_t *__restrict__ recs,
               const TcPattern *__restrict__ pats, const float *__restrict__ Kc,
               const double *__restrict__ u, double *__restrict__ f, LoadTable Ld,
               const int64_t *__restrict__ d_step, double dt, int32_t *flags, int kmax, int nmax,
               int rec_max, int nn_max, int tcols) {
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemLayout SL = smem_layout(kmax, nmax, rec_max, nn_max);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);   // [0] MMA, [1], [2] records
  uint32_t *taddr_s = reinterpret_cast<uint32_t *>(smem + 32);
  float *Bs = reinterpret_cast<float *>(smem + SL.B);
  float *As = reinterpret_cast<float *>(smem + SL.A);
  uint16_t *lid = reinterpret_cast<uint16_t *>(smem + SL.ref);   // [slot][cell]
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
    for (int l = tid; l < Ld.n; l += TC_THREADS)
      atomicAdd(&f[Ld.dof[l]], -Ld.amp[l] * wavelet_value(Ld.kind[l], t, Ld.t1[l], Ld.ncyc[l]));
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *taddr_s;

  auto issue_record = [&](int s, int tile) {   // thread 0 only
    const TcTile T = tiles[tile];
    tc::fence_proxy_async_smem();
    const uint32_t mb = mb_rec0 + 8u * (uint32_t)s;
    tc::mbar_arrive_expect_tx(mb, (uint32_t)T.rec_bytes);
    tc::bulk_g2s(tc::smem_addr(smem + (s ? SL.stage[1] : SL.stage[0])), recs + T.rec_off,
                 (uint32_t)T.rec_bytes, mb);
  };
  auto issue_gather = [&](int s) {            // all threads
    const Stage S = stage_view(smem + (s ? SL.stage[1] : SL.stage[0]), SL.u_off);
    const int nn = S.hdr[2];
    const uint32_t ub = tc::smem_addr(S.u);
    for (int i = tid; i < nn; i += TC_THREADS) {
      const double *src = u + 3 * (int64_t)S.nodes[i];
      tc::cp_async8(ub + 24u * i, src);
      tc::cp_async8(ub + 24u * i + 8u, src + 1);
      tc::cp_async8(ub + 24u * i + 16u, src + 2);
    }
    tc::cp_async_commit();
  };

  // bit s of ph_rec / pend: parity and "copy in flight" of stage s's record
  uint32_t ph_rec = 0u, pend = 0u, ph_mma = 0u;
  bool ok = true;
  int tile = blockIdx.x;
  if (tile < ntiles) {
    if (tid == 0) {
      issue_record(0, tile);
      if (tile + G < ntiles) issue_record(1, tile + G);
    }
    pend = 1u | (tile + G < ntiles ? 2u : 0u);
    ok = __syncthreads_and(tc::mbar_wait_bounded(mb_rec0, ph_rec & 1u, WAIT_POLLS));
    if (ok) {
      ph_rec ^= 1u;
      pend &= ~1u;
      issue_gather(0);
    }
  }
  int cur_pat = -1;
  for (int i = 0; ok && tile < ntiles; ++i, tile += G) {
    const int s = i & 1;
    const uint32_t so = (uint32_t)(s ^ 1);
    tc::cp_async_wait_all();
    __syncthreads();
    const int next = tile + G;
    if (next < ntiles) {
      ok = __syncthreads_and(
          tc::mbar_wait_bounded(mb_rec0 + 8u * so, (ph_rec >> so) & 1u, WAIT_POLLS));
      if (!ok) break;
      ph_rec ^= 1u << so;
      pend &= ~(1u << so);
      issue_gather(s ^ 1);
    }
    const Stage S = stage_view(smem + (s ? SL.stage[1] : SL.stage[0]), SL.u_off);
    const int pat = S.hdr[0], ncell = S.hdr[1], nn = S.hdr[2];
    const TcPattern P = pats[pat];
    const int m = P.m, kpad = P.kpad, npad = P.npad, nK = kpad / 4;
    if (pat != cur_pat) {   // B = K_p hi | lo, canonical layout
      const float4 *src = reinterpret_cast<const float4 *>(Kc + P.kc_off);
      float4 *dst = reinterpret_cast<float4 *>(Bs);
      const int nv = (2 * npad * kpad) / 4;
      for (int q = tid; q < nv; q += TC_THREADS) dst[q] = src[q];
      cur_pat = pat;
    }
    // phase S (per node): split U_n in place into FP32 (hi xyz, lo xyz) and
    // record the node's local index for each of its (cell, slot) incidences
    const int n = m / 3;
    {
      float *uf = reinterpret_cast<float *>(S.u);
      for (int q = tid; q < nn; q += TC_THREADS) {
        const double x0 = S.u[3 * q], x1 = S.u[3 * q + 1], x2 = S.u[3 * q + 2];
        float h0, h1, h2, l0, l1, l2;
        split_f64(x0, h0, l0);
        split_f64(x1, h1, l1);
        split_f64(x2, h2, l2);
        float *o = uf + 6 * q;
        o[0] = h0; o[1] = h1; o[2] = h2; o[3] = l0; o[4] = l1; o[5] = l2;
        for (int j = S.off[q]; j < S.off[q + 1]; ++j) {
          const int e = S.inc[j];
          lid[(e & 31) * 128 + (e >> 5)] = (uint16_t)q;
        }
      }
    }
    __syncthreads();
    // phase A (per cell, row c): d = (hi - hi_ref) + (lo - lo_ref) in FP32 with
    // the slot-0 node as reference (the hi difference of nearby values is
    // exact), transformed by the cell's op, split into TF32 hi + lo.
    // A(c, col) -> float (c/8)*nK*32 + (c%8)*4 + (col/4)*32 + col%4; four
    // nodes = 12 columns = three float4 stores per operand.
    float *Ahi = As, *Alo = As + 128 * kpad;
    const int nk4 = (kpad + 11) / 12;   // groups of four nodes (12 columns)
    const bool ident = ((S.hdr[3] >> 16) & 1) != 0;   // every cell has the identity op
    {
      const float *uf = reinterpret_cast<const float *>(S.u);
      if (ident) {
        for (int w = tid; w < ncell * nk4; w += TC_THREADS)
          build_a_item<true>(w % ncell, w / ncell, 0, uf, lid, n, nK, kpad, Ahi, Alo);
      } else {
        for (int w = tid; w < ncell * nk4; w += TC_THREADS)
          build_a_item<false>(w % ncell, w / ncell, S.sym[w % ncell], uf, lid, n, nK, kpad, Ahi,
                              Alo);
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
    // epilogue: warps w and w + 4 hold TMEM lanes 32 (w % 4) .. + 31 (cells)
    // and split the columns; F = E h D (FP32, row stride npad + 1)
    // overwrites A
    float *F = As;
    {
      const int c = 32 * (warp & 3) + lane;
      const float sc = c < ncell ? S.scale[c] : 0.0f;
      const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
      const int half = npad / 2;                // a multiple of 8
      const int c0 = (warp >> 2) * half;
      for (int cc = c0; cc < c0 + half; cc += 8) {
        float v[8];
        tc::tmem_ld8(taddr + lane_base + (uint32_t)cc, v);
        tc::tmem_ld_wait();
        if (c < ncell) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (cc + q < m) F[c * (npad + 1) + cc + q] = sc * v[q];
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    {
      const int c = tid;
      // back to the cell frame, node by node: f_cell[perm r] = sign_r f_master[r]
      if (c < ncell && !ident) {
        const int op = S.sym[c];
        const int p0 = op_perm_of(op, 0), p1 = op_perm_of(op, 1), p2 = op_perm_of(op, 2);
        float *Fr = F + c * (npad + 1);
        for (int k = 0; k < m / 3; ++k) {
          const float v0 = (op & 1) ? -Fr[3 * k] : Fr[3 * k];
          const float v1 = (op & 2) ? -Fr[3 * k + 1] : Fr[3 * k + 1];
          const float v2 = (op & 4) ? -Fr[3 * k + 2] : Fr[3 * k + 2];
          Fr[3 * k + p0] = v0;
          Fr[3 * k + p1] = v1;
          Fr[3 * k + p2] = v2;
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // node sums (FP32; below the TF32x3 contraction error) and one FP64
    // atomic per node DOF
    for (int q = tid; q < nn; q += TC_THREADS) {
      float acc[3] = {0.0f, 0.0f, 0.0f};
      for (int j = S.off[q]; j < S.off[q + 1]; ++j) {
        const int e = S.inc[j];
        const float *Fr = F + (e >> 5) * (npad + 1) + 3 * (e & 31);
        acc[0] += Fr[0];
        acc[1] += Fr[1];
        acc[2] += Fr[2];
      }
      double *fn = f + 3 * (int64_t)S.nodes[q];
      atomicAdd(fn + 0, f2d_bits(acc[0]));
      atomicAdd(fn + 1, f2d_bits(acc[1]));
      atomicAdd(fn + 2, f2d_bits(acc[2]));
    }
    __syncthreads();   // stage s and F are free
    if (next + G < ntiles) {
      if (tid == 0) issue_record(s, next + G);
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
  // launch classes by a tile's own shared-memory need (double-buffered
  // records and gathers): <= 56 KB, <= 113 KB, larger
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
  for (int p = 0; p < P; ++p) {
    const int np = ctx->pat_nodes[p], m = 3 * np;
    TcPattern &tp = pats[p];
    tp.m = m;
    tp.kpad = (m + 7) / 8 * 8;
    tp.npad = (m + 15) / 16 * 16;
    tp.tcols = tp.npad <= 32 ? 32 : (tp.npad <= 64 ? 64 : 128);
    tp.kc_off = (int64_t)Kc.size();
    tp.lidx_off = 0;
    tp.cstart = start[p];
    tp.ccount = cnt[p];
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
    // dense, frequent small patterns: 128 cells per tile; others (rarer,
    // scattered, larger): 32, which keeps double-buffered records within
    // shared memory and gives more CTAs work.  Launch class by size.
    const int per = (cnt[p] >= 4096 && m <= 30) ? 128 : 32;
    const int pcls = m <= 30 ? 0 : (m <= 48 ? 1 : 2);
    std::vector<std::pair<int32_t, int32_t>> v;   // (node, slot * 128 + cell)
    for (int64_t c0 = 0; c0 < cnt[p]; c0 += per) {
      const int nc = (int)std::min<int64_t>(per, cnt[p] - c0);
      v.clear();
      for (int k = 0; k < np; ++k)
        for (int c = 0; c < nc; ++c)
          v.emplace_back(conn[conn_off[p] + (int64_t)k * cnt[p] + c0 + c], k * 128 + c);
      std::sort(v.begin(), v.end());
      std::vector<int32_t> nodes;
      std::vector<uint16_t> offs, inc;
      for (size_t i = 0; i < v.size(); ++i) {
        if (i == 0 || v[i].first != v[i - 1].first) {
          nodes.push_back(v[i].first);
          offs.push_back((uint16_t)inc.size());
        }
        const int k = v[i].second / 128, c = v[i].second % 128;
        inc.push_back((uint16_t)((c << 5) | k));
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
      const int32_t hdr[4] = {p, nc, nn, np | (ident << 16)};   // bit 16: all ops identity
      put(recs, at, hdr, 4);
      put(recs, at + R.scale, sc.data(), nc);
      put(recs, at + R.nodes, nodes.data(), nn);
      put(recs, at + R.off, offs.data(), offs.size());
      put(recs, at + R.inc, inc.data(), inc.size());
      TcTile t;
      t.rec_off = (int64_t)at;
      t.rec_bytes = (int32_t)R.bytes;
      t.pat = p;
      const uint32_t need = smem_layout(tp.kpad, tp.npad, R.bytes, nn).total;
      int cls = pcls;
      while (cls < TC_CLASSES - 1 && need > class_limit[cls]) ++cls;
      if (need > class_limit[TC_CLASSES - 1]) {
        err = "tensor-core tile needs more than 227 KB of shared memory";
        return SBX_EINVAL;
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
    ctx->n_tc_tiles[cls] = (int)tiles[cls].size();
    ctx->tc_kmax[cls] = kmax[cls];
    ctx->tc_nmax[cls] = nmax[cls];
    ctx->tc_rec_max[cls] = recmax[cls];
    ctx->tc_nn_max[cls] = nnmax[cls];
    ctx->tc_tcols[cls] = tcols[cls];
    const uint32_t smem = smem_layout(kmax[cls], nmax[cls], recmax[cls], nnmax[cls]).total;
    ctx->tc_smem[cls] = smem;
    // resident CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per
    // CTA) and tensor memory (512 columns)
    int per_sm = (int)((228u * 1024u) / (smem + 1024u));
    per_sm = std::max(1, std::min(per_sm, std::min(8, 512 / tcols[cls])));
    ctx->tc_grid[cls] = (int)std::min<int64_t>(tiles[cls].size(), (int64_t)nsm * per_sm);
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    err = "stream synchronisation failed";
    return SBX_ECUDA;
  }
  return SBX_OK;
}

cudaError_t prepare_tc_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_force_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_force_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}

cudaError_t launch_force_tc(const sbx_ctx *ctx, const double *u, double *f, double dt,
                            cudaStream_t s) {
  bool load_done = false;   // the load term is added by CTA 0 of one launch only
  for (int cls = 0; cls < TC_CLASSES; ++cls) {
    if (ctx->n_tc_tiles[cls] == 0) continue;
    LoadTable L = ctx->loads();
    if (load_done) L.n = 0;
    load_done = true;
    k_force_tc<<<ctx->tc_grid[cls], TC_THREADS, ctx->tc_smem[cls], s>>>(
        ctx->d_tc_tiles[cls], ctx->n_tc_tiles[cls], ctx->d_tc_rec, ctx->d_tc_pat, ctx->d_tc_K, u,
        f, L, ctx->d_step, dt, ctx->d_flags, ctx->tc_kmax[cls], ctx->tc_nmax[cls],
        ctx->tc_rec_max[cls], ctx->tc_nn_max[cls], ctx->tc_tcols[cls]);
  }
  return cudaGetLastError();
}

}  // namespace sbx

// Batched explicit step: B load cases advance together (field layout
// [node][3][B], entry (3 node + d) B + b).  K_p is read once per cell and
// applied to the 32 load cases of a chunk, so the contraction is a small
// dense GEMM per cell (K_p times an m x 32 block).
//
// Force kernel, one CTA (8 warps) per (tile of cells of one pattern, chunk
// of 32 load cases); lane = load case:
//   1. gather the tile's unique nodes (the 32 cases of each DOF form one
//      coalesced row); T = float: the (hi, lo) FP32 pairs of U_n that the
//      update kernel wrote (hi + lo = U_n to ~2^-48), T = double: FP64;
//   2. warp per cell: for j = 0..m-1, d_j = U(node) - U(slot-0 node) of this
//      lane's case (K_p annihilates translations), transformed by the op
//      (Sec. 3.2.2); acc(0..MM) += K_p(j, :) d_j with K_p rows read as float4
//      broadcasts (K_p is symmetric, so row j is column j);
//   3. E_e h_e Q^T acc goes straight to f with one atomic reduction per
//      (cell, node DOF), coalesced over the warp's 32 cases (T = float: f is
//      FP32; T = double: FP64).
// T = float: FP32 contraction, on Blackwell's packed FP32 pairs (two rows of
// K_p per instruction; the regular cell's Walsh transforms on its (x, y)
// components); T = double: FP64.  The update is FP64.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "sbx_internal.cuh"

namespace sbx {
namespace {

constexpr int BT_THREADS = 256;   // 8 warps
constexpr int BT_WARPS = 8;
constexpr int BC = 32;            // load cases per chunk

__host__ __device__ inline uint32_t b16(uint32_t x) { return (x + 15u) & ~15u; }

// Record: int32 {pat, ncell, nn, n}; uint8 sym[ncell]; double scale[ncell];
// int32 nodes[nn]; uint16 lid[n][ncell] (local node of slot k of cell c)
struct BRecLayout {
  uint32_t sym, scale, nodes, lid, bytes;
};
__host__ __device__ inline BRecLayout brec_layout(int ncell, int nn, int n) {
  BRecLayout R;
  uint32_t o = 16;
  R.sym = o;   o += b16((uint32_t)ncell);
  R.scale = o; o += b16(8u * ncell);
  R.nodes = o; o += b16(4u * nn);
  R.lid = o;   o += b16(2u * n * ncell);
  R.bytes = o;
  return R;
}

struct BSmem {
  uint32_t K, u, rec, total;
};
// mm: padded row length of K_p (a multiple of 4); tsz: sizeof(T)
__host__ __device__ inline BSmem bsmem(int mm, int nn_max, int rec_max, uint32_t tsz) {
  BSmem L;
  uint32_t o = 0;
  L.K = o;   o = b16(o + (uint32_t)mm * mm * tsz);
  L.u = o;   o = b16(o + (uint32_t)nn_max * 3u * BC * 8u);          // float2 or double
  L.rec = o; o = b16(o + (uint32_t)rec_max);
  L.total = o;
  return L;
}

// d = U(node q, dir a) - U(node q0, dir a) of this lane's case; FP32: from
// the (hi, lo) pairs, (hi - hi_0) + (lo - lo_0)
template <typename T>
__device__ __forceinline__ T diff_of(const unsigned char *u, int q, int q0, int a, int lane) {
  if constexpr (sizeof(T) == 4) {
    const float2 *uu = reinterpret_cast<const float2 *>(u);
    const float2 v = uu[(q * 3 + a) * BC + lane], v0 = uu[(q0 * 3 + a) * BC + lane];
    return (v.x - v0.x) + (v.y - v0.y);
  } else {
    const double *uu = reinterpret_cast<const double *>(u);
    return uu[(q * 3 + a) * BC + lane] - uu[(q0 * 3 + a) * BC + lane];
  }
}

// Walsh transform of 8 values in place (x[p] <- sum_n (-1)^popcount(p & n) x[n]).
template <typename T>
__device__ __forceinline__ void wht8_t(T *x) {
#pragma unroll
  for (int h = 1; h < 8; h <<= 1)
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if ((i & h) == 0) {
        const T a = x[i], b = x[i + h];
        x[i] = a + b;
        x[i + h] = a - b;
      }
}

// The same transform on pairs of values held as float2 (Blackwell's packed
// FP32 arithmetic: both lanes in one instruction; a - b as b * (-1) + a, an
// exact product and one rounding, so bit-identical to the scalar form).
__device__ __forceinline__ void wht8_f2(float2 *x) {
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

// The regular 8-node cell's K_p as eight 3 x 3 blocks in the Walsh basis
// of its corners (already divided by 8), in the kernel's number type.
template <typename T>
struct WhtB {
  T blk[72];
};

// The FP32 form of one CTA's cells (steps 2 and 3 above), with the
// arithmetic on packed FP32 pairs: the differences as (hi - hi_0, lo - lo_0)
// pairs; the dense contraction two rows of K_p at a time (acc[i], acc[i + 1]
// += (K_p[j][i], K_p[j][i + 1]) d_j, the fused multiply-add of the scalar
// form per lane); the regular cell's transforms on its (x, y) components.
// Results equal the scalar FP32 arithmetic bit for bit.
template <int MM>
__device__ __forceinline__ void force_cells_f32(const unsigned char *smem, const BSmem &SL,
                                                int ncell, int n, int m, int pat,
                                                const uint8_t *sym, const double *scale,
                                                const int32_t *nodes, const uint16_t *lid,
                                                float *__restrict__ f, int B, int b0, int warp,
                                                int lane, int wht_pat, const WhtB<float> &Kw) {
  const float *Ks = reinterpret_cast<const float *>(smem + SL.K);
  const float2 *uu = reinterpret_cast<const float2 *>(smem + SL.u);
  const float2 m1 = make_float2(-1.0f, -1.0f);
  for (int c = warp; c < ncell; c += BT_WARPS) {
    const int op = sym[c];
    const int p0 = op_perm_of(op, 0), p1 = op_perm_of(op, 1), p2 = op_perm_of(op, 2);
    const int q0 = lid[c];
    const float s = (float)scale[c];
    // (hi - hi_0) + (lo - lo_0) of node q, direction a, this lane's case
    auto dif = [&](int q, int a) {
      const float2 t = __ffma2_rn(uu[(q0 * 3 + a) * BC + lane], m1, uu[(q * 3 + a) * BC + lane]);
      return t.x + t.y;
    };
    // E h Q^T of entry i (node slot i / 3) into f, one reduction per entry
    auto emit = [&](int i, float val) {
      const int k = i / 3, r = i % 3;
      const int a = r == 0 ? p0 : (r == 1 ? p1 : p2);
      const float v = ((op >> r) & 1) ? -s * val : s * val;
      atomicAdd(&f[(3 * (int64_t)nodes[lid[k * ncell + c]] + a) * B + b0 + lane], v);
    };
    float2 acc[MM / 2];   // every entry below m is set on either path
    auto put = [&](int i, float v) {
      if (i & 1) acc[i / 2].y = v;
      else acc[i / 2].x = v;
    };
    if (MM == 24 && op == 0 && pat == wht_pat) {
      // regular cell: f = T^T blockdiag(Kh) T d / 8 with the Walsh transform
      // T over the corners; (x, y) components packed, z scalar
      float2 X[8];
      float Z[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int q = lid[k * ncell + c];
        X[k] = make_float2(dif(q, 0), dif(q, 1));
        Z[k] = dif(q, 2);
      }
      wht8_f2(X);
      wht8_t(Z);
      float2 Y[8];
      float YZ[8];
#pragma unroll
      for (int sb = 0; sb < 8; ++sb) {
        const float *Bk = Kw.blk + 9 * sb;
        const float v0 = X[sb ^ 1].x, v1 = X[sb ^ 2].y, v2 = Z[sb ^ 4];
        Y[sb ^ 1].x = Bk[0] * v0 + Bk[1] * v1 + Bk[2] * v2;
        Y[sb ^ 2].y = Bk[3] * v0 + Bk[4] * v1 + Bk[5] * v2;
        YZ[sb ^ 4] = Bk[6] * v0 + Bk[7] * v1 + Bk[8] * v2;
      }
      wht8_f2(Y);
      wht8_t(YZ);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        put(3 * k, Y[k].x);
        put(3 * k + 1, Y[k].y);
        put(3 * k + 2, YZ[k]);
      }
    } else {
#pragma unroll
    for (int i = 0; i < MM / 2; ++i) acc[i] = make_float2(0.0f, 0.0f);
    // acc += K_p row j (two entries per instruction) times d_j
    auto row = [&](int j, float dj) {
      const float *kr = Ks + j * MM;
      const float2 dd = make_float2(dj, dj);
#pragma unroll
      for (int i = 0; i < MM; i += 4) {
        const float4 kv = *reinterpret_cast<const float4 *>(kr + i);
        acc[i / 2] = __ffma2_rn(make_float2(kv.x, kv.y), dd, acc[i / 2]);
        acc[i / 2 + 1] = __ffma2_rn(make_float2(kv.z, kv.w), dd, acc[i / 2 + 1]);
      }
    };
    if constexpr (MM <= 24) {
#pragma unroll
      for (int k = 0; k < MM / 3; ++k)
        if (k < n) {
          const int q = lid[k * ncell + c];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const int a = r == 0 ? p0 : (r == 1 ? p1 : p2);
            const float x = dif(q, a);
            row(3 * k + r, ((op >> r) & 1) ? -x : x);
          }
        }
    } else {
      for (int j = 0; j < m; ++j) {
        const int k = j / 3, r = j - 3 * (j / 3);
        const int a = r == 0 ? p0 : (r == 1 ? p1 : p2);
        const float x = dif(lid[k * ncell + c], a);
        row(j, ((op >> r) & 1) ? -x : x);
      }
    }
    }
#pragma unroll
    for (int i = 0; i < MM; ++i)
      if (i < m) emit(i, (i & 1) ? acc[i / 2].y : acc[i / 2].x);
  }
}

template <typename T, int MM>
__global__ void __launch_bounds__(BT_THREADS, 2)
    k_force_batch(const TcTile *__restrict__ tiles, int nchunks, const uint8_t *__restrict__ recs,
                  const T *__restrict__ Kp, const int64_t *__restrict__ koff,
                  const void *__restrict__ uv, void *__restrict__ fv, int B, LoadTable Ld,
                  const int64_t *__restrict__ d_step, double dt, int nn_max, int rec_max,
                  int wht_pat, const WhtB<T> Kw) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BSmem SL = bsmem(MM, nn_max, rec_max, sizeof(T));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x / nchunks, chunk = blockIdx.x % nchunks;
  const TcTile Tt = tiles[tile];
  {
    const int4 *src = reinterpret_cast<const int4 *>(recs + Tt.rec_off);
    int4 *dst = reinterpret_cast<int4 *>(smem + SL.rec);
    for (int q = tid; q < Tt.rec_bytes / 16; q += BT_THREADS) dst[q] = src[q];
  }
  __syncthreads();
  const int32_t *hdr = reinterpret_cast<const int32_t *>(smem + SL.rec);
  const int pat = hdr[0], ncell = hdr[1], nn = hdr[2], n = hdr[3];
  const int m = 3 * n;
  const BRecLayout R = brec_layout(ncell, nn, n);
  const uint8_t *sym = smem + SL.rec + R.sym;
  const double *scale = reinterpret_cast<const double *>(smem + SL.rec + R.scale);
  const int32_t *nodes = reinterpret_cast<const int32_t *>(smem + SL.rec + R.nodes);
  const uint16_t *lid = reinterpret_cast<const uint16_t *>(smem + SL.rec + R.lid);
  T *Ks = reinterpret_cast<T *>(smem + SL.K);

  // K_p, rows padded to MM with zeros (symmetric: row j = column j)
  for (int q = tid; q < m * MM; q += BT_THREADS) {
    const int j = q / MM, i = q % MM;
    Ks[q] = i < m ? (T)Kp[koff[pat] + (int64_t)j * m + i] : (T)0;
  }
  const int b0 = chunk * BC;
  // node rows of 32 cases: (node, dir) row t = 3 nq + a, 16-byte pieces
  for (int q = tid; q < nn * 3 * (BC / 2); q += BT_THREADS) {
    const int t = q >> 4, b = 2 * (q & 15);
    const int nq = t / 3, a = t - 3 * nq;
    const int64_t g = (3 * (int64_t)nodes[nq] + a) * B + b0 + b;
    if constexpr (sizeof(T) == 4)
      reinterpret_cast<float4 *>(smem + SL.u)[q] = *reinterpret_cast<const float4 *>(
          reinterpret_cast<const float2 *>(uv) + g);
    else
      reinterpret_cast<double2 *>(smem + SL.u)[q] = *reinterpret_cast<const double2 *>(
          reinterpret_cast<const double *>(uv) + g);
  }
  __syncthreads();

  if constexpr (sizeof(T) == 4) {
    force_cells_f32<MM>(smem, SL, ncell, n, m, pat, sym, scale, nodes, lid,
                        reinterpret_cast<float *>(fv), B, b0, warp, lane, wht_pat, Kw);
  } else
  for (int c = warp; c < ncell; c += BT_WARPS) {
    const int op = sym[c];
    const int p0 = op_perm_of(op, 0), p1 = op_perm_of(op, 1), p2 = op_perm_of(op, 2);
    const int q0 = lid[c];
    T acc[MM];
#pragma unroll
    for (int i = 0; i < MM; ++i) acc[i] = (T)0;
    if constexpr (MM <= 24) {
      // this lane's case: all differences d_j first (registers), then the
      // contraction with K_p rows as float4 broadcasts
      T d[MM];
      if (op == 0) {   // identity op (every 8-node cell): no component shuffle
#pragma unroll
        for (int k = 0; k < MM / 3; ++k) {
          const int q = k < n ? lid[k * ncell + c] : q0;
#pragma unroll
          for (int a = 0; a < 3; ++a) d[3 * k + a] = diff_of<T>(smem + SL.u, q, q0, a, lane);
        }
      } else {
#pragma unroll
        for (int k = 0; k < MM / 3; ++k) {
          const int q = k < n ? lid[k * ncell + c] : q0;
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const int a = r == 0 ? p0 : (r == 1 ? p1 : p2);
            const T x = diff_of<T>(smem + SL.u, q, q0, a, lane);
            d[3 * k + r] = ((op >> r) & 1) ? -x : x;
          }
        }
      }
      if (sizeof(T) == 4 && MM == 24 && op == 0 && pat == wht_pat) {   // (FP32: no spills)
        // regular cell: f = T^T blockdiag(Kh) T d / 8 with the Walsh transform
        // T over the corners (the translation in d drops out exactly)
        T x[3][8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int r = 0; r < 3; ++r) x[r][k] = d[3 * k + r];
        wht8_t(x[0]);
        wht8_t(x[1]);
        wht8_t(x[2]);
        T y[3][8];
#pragma unroll
        for (int sb = 0; sb < 8; ++sb) {
          const T *Bk = Kw.blk + 9 * sb;
          const T v0 = x[0][sb ^ 1], v1 = x[1][sb ^ 2], v2 = x[2][sb ^ 4];
          y[0][sb ^ 1] = Bk[0] * v0 + Bk[1] * v1 + Bk[2] * v2;
          y[1][sb ^ 2] = Bk[3] * v0 + Bk[4] * v1 + Bk[5] * v2;
          y[2][sb ^ 4] = Bk[6] * v0 + Bk[7] * v1 + Bk[8] * v2;
        }
        wht8_t(y[0]);
        wht8_t(y[1]);
        wht8_t(y[2]);
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int r = 0; r < 3; ++r) acc[3 * k + r] = y[r][k];
      } else
#pragma unroll
      for (int j = 0; j < MM; ++j) {
        if (j < m) {
          const T *kr = Ks + j * MM;
#pragma unroll
          for (int i = 0; i < MM; i += 4) {
            if constexpr (sizeof(T) == 4) {
              const float4 kv = *reinterpret_cast<const float4 *>(kr + i);
              acc[i] += kv.x * d[j];
              acc[i + 1] += kv.y * d[j];
              acc[i + 2] += kv.z * d[j];
              acc[i + 3] += kv.w * d[j];
            } else {
              acc[i] += kr[i] * d[j];
              acc[i + 1] += kr[i + 1] * d[j];
              acc[i + 2] += kr[i + 2] * d[j];
              acc[i + 3] += kr[i + 3] * d[j];
            }
          }
        }
      }
    } else {
      for (int j = 0; j < m; ++j) {
        const int k = j / 3, r = j - 3 * (j / 3);
        const int a = r == 0 ? p0 : (r == 1 ? p1 : p2);
        const int q = lid[k * ncell + c];
        T dj;
        if constexpr (sizeof(T) == 4) {
          const float2 *uu = reinterpret_cast<const float2 *>(smem + SL.u);
          const float2 v = uu[(q * 3 + a) * BC + lane], v0 = uu[(q0 * 3 + a) * BC + lane];
          dj = (v.x - v0.x) + (v.y - v0.y);
        } else {
          const double *uu = reinterpret_cast<const double *>(smem + SL.u);
          dj = uu[(q * 3 + a) * BC + lane] - uu[(q0 * 3 + a) * BC + lane];
        }
        if ((op >> r) & 1) dj = -dj;
        const T *kr = Ks + j * MM;
#pragma unroll
        for (int i = 0; i < MM; i += 4) {
          if constexpr (sizeof(T) == 4) {
            const float4 kv = *reinterpret_cast<const float4 *>(kr + i);
            acc[i] += kv.x * dj;
            acc[i + 1] += kv.y * dj;
            acc[i + 2] += kv.z * dj;
            acc[i + 3] += kv.w * dj;
          } else {
            acc[i] += kr[i] * dj;
            acc[i + 1] += kr[i + 1] * dj;
            acc[i + 2] += kr[i + 2] * dj;
            acc[i + 3] += kr[i + 3] * dj;
          }
        }
      }
    }
    const T s = (T)scale[c];
    T *f = reinterpret_cast<T *>(fv);
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      if (i < m) {
        const int k = i / 3, r = i % 3;
        const int a = r == 0 ? p0 : (r == 1 ? p1 : p2);
        const T v = ((op >> r) & 1) ? -s * acc[i] : s * acc[i];
        atomicAdd(&f[(3 * (int64_t)nodes[lid[k * ncell + c]] + a) * B + b0 + lane], v);
      }
    }
  }
  T *f = reinterpret_cast<T *>(fv);
  if (blockIdx.x == 0 && Ld.n > 0) {
    const double t = (double)(*d_step) * dt;
    for (int l = tid; l < Ld.n; l += BT_THREADS)
      atomicAdd(&f[Ld.dof[l]], (T)(-Ld.amp[l] * wavelet_value(Ld.kind[l], t, Ld.t1[l], Ld.ncyc[l])));
  }
}

// U_{n+1} = -w f + 2 U_n - U_{n-1} (undamped) or the damped form; w per DOF,
// f and U per (DOF, case); FP64.  F32: f is FP32 (widened by bit
// re-packing) and U_{n+1} is also written as its (hi, lo) FP32 pair.
template <bool DAMPED, bool F32>
__global__ void __launch_bounds__(256)
    k_update_batch(int64_t nd, int B, const double *__restrict__ w, void *__restrict__ fv,
                   const double *__restrict__ uc, double *__restrict__ up,
                   float2 *__restrict__ pairs, double a, double b, int zero_f, int32_t *flags,
                   int64_t *d_step) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wv = w[i / B];
    const double fi = F32 ? f2d_bits(reinterpret_cast<const float *>(fv)[i])
                          : reinterpret_cast<const double *>(fv)[i];
    const double r = DAMPED ? fma(-wv, fi, fma(a, uc[i], -b * up[i]))
                            : fma(-wv, fi, fma(2.0, uc[i], -up[i]));
    bad |= ((__double_as_longlong(r) >> 52) & 0x7FF) == 0x7FF;
    up[i] = r;
    if (F32) {
      float h, l;
      split_f64(r, h, l);
      pairs[i] = make_float2(h, l);
      if (zero_f) reinterpret_cast<float *>(fv)[i] = 0.0f;
    } else if (zero_f) {
      reinterpret_cast<double *>(fv)[i] = 0.0;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_step += 1;
}

int class_of(int m) { return m <= 24 ? 0 : (m <= 48 ? 1 : 2); }
constexpr int CLASS_MM[3] = {24, 48, 80};

}  // namespace

int batch_setup(sbx_ctx *ctx, const std::vector<int32_t> &conn, const std::vector<int64_t> &conn_off,
                const std::vector<int64_t> &cnt, const std::vector<uint8_t> &sym_sorted,
                const std::vector<double> &scale_sorted, const std::vector<int64_t> &start,
                std::string &err) {
  const int P = ctx->n_pat;
  const uint32_t tsz = ctx->prec == SBX_PREC_FP64 ? 8u : 4u;
  std::vector<uint8_t> recs;
  std::vector<TcTile> tiles[3];
  std::vector<int64_t> work[3];   // multiply-adds per load case of each tile
  int nnmax[3] = {1, 1, 1}, recmax[3] = {16, 16, 16};
  std::vector<std::pair<int32_t, int32_t>> v;
  for (int p = 0; p < P; ++p) {
    const int np = ctx->pat_nodes[p], m = 3 * np, cls = class_of(m);
    int64_t c0 = 0;
    const uint32_t target = (uint32_t)ctx->b_smem_kb[cls] * 1024u;
    while (c0 < cnt[p]) {
      // largest tile (b_tile_cells[cls] cells or fewer) whose staging fits
      // the class's shared-memory budget
      int nc = (int)std::min<int64_t>(ctx->b_tile_cells[cls], cnt[p] - c0);
      std::vector<int32_t> nodes;
      std::vector<uint16_t> lid;
      for (;;) {
        v.clear();
        for (int k = 0; k < np; ++k)
          for (int c = 0; c < nc; ++c)
            v.emplace_back(conn[conn_off[p] + (int64_t)k * cnt[p] + c0 + c], k * nc + c);
        std::sort(v.begin(), v.end());
        nodes.clear();
        lid.assign((size_t)np * nc, 0);
        for (size_t i = 0; i < v.size(); ++i) {
          if (i == 0 || v[i].first != v[i - 1].first) nodes.push_back(v[i].first);
          lid[v[i].second] = (uint16_t)(nodes.size() - 1);
        }
        const uint32_t need = bsmem(CLASS_MM[cls], (int)nodes.size(),
                                    (int)brec_layout(nc, (int)nodes.size(), np).bytes, tsz).total;
        if (need <= target || nc == 1) break;
        nc = std::max(1, nc / 2);
      }
      const int nn = (int)nodes.size();
      const BRecLayout R = brec_layout(nc, nn, np);
      const size_t at = recs.size();
      recs.resize(at + R.bytes, 0);
      const int32_t hdr[4] = {p, nc, nn, np};
      memcpy(recs.data() + at, hdr, 16);
      for (int c = 0; c < nc; ++c) {
        recs[at + R.sym + c] = sym_sorted[start[p] + c0 + c];
        memcpy(recs.data() + at + R.scale + 8 * c, &scale_sorted[start[p] + c0 + c], 8);
      }
      memcpy(recs.data() + at + R.nodes, nodes.data(), 4 * nn);
      memcpy(recs.data() + at + R.lid, lid.data(), 2 * lid.size());
      TcTile t;
      t.rec_off = (int64_t)at;
      t.rec_bytes = (int32_t)R.bytes;
      t.pat = p;
      tiles[cls].push_back(t);
      work[cls].push_back((int64_t)nc * m * m);
      nnmax[cls] = std::max(nnmax[cls], nn);
      recmax[cls] = std::max(recmax[cls], (int)R.bytes);
      c0 += nc;
    }
  }
  auto up = [&](auto **dst, const auto &vec) -> int {
    using TT = typename std::remove_reference<decltype(vec)>::type::value_type;
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    if (cudaMalloc((void **)dst, std::max<size_t>(vec.size(), 1) * sizeof(TT)) != cudaSuccess) {
      cudaGetLastError();
      err = "cudaMalloc failed (batched tables)";
      return SBX_ENOMEM;
    }
    if (!vec.empty() && cudaMemcpyAsync(*dst, vec.data(), vec.size() * sizeof(TT),
                                        cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
      err = "copy of batched tables failed";
      return SBX_ECUDA;
    }
    return SBX_OK;
  };
  if (int rc = up(&ctx->d_b_rec, recs)) return rc;
  // heaviest tiles first within a class (CTAs are issued in order: long ones
  // start early, short ones fill the end)
  for (int c = 0; c < 3; ++c) {
    std::vector<size_t> ord(tiles[c].size());
    for (size_t q = 0; q < ord.size(); ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](size_t a, size_t b) { return work[c][a] > work[c][b]; });
    std::vector<TcTile> sorted;
    for (size_t q : ord) sorted.push_back(tiles[c][q]);
    tiles[c].swap(sorted);
  }
  for (int c = 0; c < 3; ++c) {
    if (int rc = up(&ctx->d_b_tiles[c], tiles[c])) return rc;
    ctx->n_b_tiles[c] = (int)tiles[c].size();
    ctx->b_nnmax[c] = nnmax[c];
    ctx->b_recmax[c] = recmax[c];
    ctx->b_smem[c] = bsmem(CLASS_MM[c], nnmax[c], recmax[c], tsz).total;
    if (ctx->n_b_tiles[c] && ctx->b_smem[c] > 227u * 1024u) {
      err = "batched tile needs more than 227 KB of shared memory";
      return SBX_EINVAL;
    }
  }
  if (ctx->prec == SBX_PREC_FP32) {   // the classes beyond the 8-node cell, tensor-core form
    std::vector<char> use(P, 0);
    for (int p = 0; p < P; ++p) use[p] = class_of(3 * ctx->pat_nodes[p]) > 0;
    if (int rc = gt_setup(ctx, conn, conn_off, cnt, start, sym_sorted, scale_sorted, use, err))
      return rc;
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    err = "stream synchronisation failed";
    return SBX_ECUDA;
  }
  return SBX_OK;
}

cudaError_t prepare_batch_kernels() {
  const void *ks[6] = {(const void *)k_force_batch<float, 24>, (const void *)k_force_batch<float, 48>,
                       (const void *)k_force_batch<float, 80>, (const void *)k_force_batch<double, 24>,
                       (const void *)k_force_batch<double, 48>, (const void *)k_force_batch<double, 80>};
  for (const void *k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
static void launch_class(const sbx_ctx *ctx, int c, const T *K, const void *u, void *f,
                         LoadTable L, double dt, cudaStream_t s) {
  const int nchunks = ctx->B / BC;
  const unsigned grid = (unsigned)ctx->n_b_tiles[c] * (unsigned)nchunks;
  const size_t sm = ctx->b_smem[c];
  WhtB<T> kw;
  for (int q = 0; q < 72; ++q) kw.blk[q] = (T)(ctx->wht.blk[q] * 0.125);
#define SBX_LAUNCH(MMV)                                                                        \
  k_force_batch<T, MMV><<<grid, BT_THREADS, sm, s>>>(ctx->d_b_tiles[c], nchunks, ctx->d_b_rec, \
                                                     K, ctx->d_koff, u, f, ctx->B, L,          \
                                                     ctx->d_step, dt, ctx->b_nnmax[c],         \
                                                     ctx->b_recmax[c], ctx->wht_pat, kw)
  if (c == 0) SBX_LAUNCH(24);
  else if (c == 1) SBX_LAUNCH(48);
  else SBX_LAUNCH(80);
#undef SBX_LAUNCH
}

cudaError_t launch_force_batch(const sbx_ctx *ctx, const void *u, void *f, double dt,
                               cudaStream_t s) {
  bool load_done = false;
  // FP32 form: the hanging-node classes on the tensor cores (default)
  const bool tc = ctx->prec == SBX_PREC_FP32 && ctx->hanging_tc && ctx->n_gt_tiles > 0;
  for (int c = 0; c < 3; ++c) {
    if (ctx->n_b_tiles[c] == 0 || (tc && c > 0)) continue;
    LoadTable L = ctx->loads();
    if (load_done) L.n = 0;
    load_done = true;
    if (ctx->prec == SBX_PREC_FP64)
      launch_class<double>(ctx, c, ctx->d_K64, u, f, L, dt, s);
    else
      launch_class<float>(ctx, c, ctx->d_K32, u, f, L, dt, s);
  }
  if (tc) {
    LoadTable L = ctx->loads();
    if (load_done) L.n = 0;
    cudaError_t e = launch_force_batch_tc(ctx, reinterpret_cast<const float *>(u),
                                          reinterpret_cast<float *>(f), dt, L, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_update_batch(const sbx_ctx *ctx, const double *uc, double *up, void *f,
                                float *pairs_out, double dt, double alpha, int zero_f,
                                cudaStream_t s) {
  const int64_t nd = ctx->ndof * ctx->B;
  const double cm = 1.0 - 0.5 * alpha * dt, cp = 1.0 + 0.5 * alpha * dt;
  const int64_t want = (nd + 255) / 256;
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)ctx->n_sm * 8);
  const double a = alpha == 0.0 ? 2.0 : 2.0 / cp, b = alpha == 0.0 ? 1.0 : cm / cp;
  float2 *pr = reinterpret_cast<float2 *>(pairs_out);
#define SBX_UPD(D, F)                                                                          \
  k_update_batch<D, F><<<grid, 256, 0, s>>>(nd, ctx->B, ctx->d_w, f, uc, up, pr, a, b, zero_f, \
                                            ctx->d_flags, ctx->d_step)
  if (pairs_out) {
    if (alpha == 0.0) SBX_UPD(false, true);
    else SBX_UPD(true, true);
  } else {
    if (alpha == 0.0) SBX_UPD(false, false);
    else SBX_UPD(true, false);
  }
#undef SBX_UPD
  return cudaGetLastError();
}

}  // namespace sbx

// Set-up on the GPU (Sec. 3.2.1-3.2.2 and Alg. 1's set-up stage): pattern
// classification of every cell's 12-bit mid-edge mask, the cell's node list
// in its master's node order, the stable sort of the cells by pattern and
// the slot-major connectivity of each pattern group.  The results are the
// integers the host path computes (same rules, bit for bit):
//  * the 48 signed permutations op = 8 perm_index + sign_bits act on the
//    26 slots of the unit cell (corners, mid-edges, face centres) by
//    p -> Q (p - c) + c about the cell centre c; a mask's image under op is
//    the set of images of its mid-edges;
//  * master of a mask = the largest mask of its orbit; op = the smallest op
//    number carrying the mask onto the master;
//  * a cell's present slots: the 8 corners, its mid-edges, and the centre
//    of every face with 1, 3 or 4 of its mid-edges, or 2 that are not
//    opposite (parallel);
//  * node k of a cell in master order = the cell's node at the slot that op
//    carries onto the master's k-th present slot (slots ascending);
//  * pattern ids = ranks of the distinct masters in ascending order; cells
//    grouped by pattern, the given (Morton) order kept within a group.
#include <stdint.h>

#include "sbx_internal.cuh"

namespace sbx {
namespace {

// slot s -> doubled position (x, y, z) in {0, 1, 2}^3
__host__ __device__ inline void slot_pos(int s, int p[3]) {
  if (s < 8) {
    p[0] = 2 * (s & 1);
    p[1] = 2 * ((s >> 1) & 1);
    p[2] = 2 * ((s >> 2) & 1);
  } else if (s < 20) {
    const int e = s - 8, a = e >> 2, r = e & 3;
    const int o0 = a == 0 ? 1 : 0, o1 = a == 2 ? 1 : 2;
    p[a] = 1;
    p[o0] = 2 * (r & 1);
    p[o1] = 2 * (r >> 1);
  } else {
    const int f = s - 20;
    p[0] = p[1] = p[2] = 1;
    p[f >> 1] = 2 * (f & 1);
  }
}

// doubled position -> slot (-1: the cell centre)
__host__ __device__ inline int pos_slot(const int p[3]) {
  int n2 = (p[0] != 1) + (p[1] != 1) + (p[2] != 1);   // coordinates on the boundary
  if (n2 == 3) return (p[0] >> 1) | ((p[1] >> 1) << 1) | ((p[2] >> 1) << 2);
  if (n2 == 2) {
    const int a = p[0] == 1 ? 0 : (p[1] == 1 ? 1 : 2);
    const int o0 = a == 0 ? 1 : 0, o1 = a == 2 ? 1 : 2;
    return 8 + 4 * a + (p[o0] >> 1) + 2 * (p[o1] >> 1);
  }
  if (n2 == 1) {
    const int a = p[0] != 1 ? 0 : (p[1] != 1 ? 1 : 2);
    return 20 + 2 * a + (p[a] >> 1);
  }
  return -1;
}

__host__ __device__ inline int perm_of(int op, int r) {
  const int i = op >> 3, p0 = i >> 1, p1 = (0x489 >> (2 * i)) & 3;
  return r == 0 ? p0 : (r == 1 ? p1 : 3 - p0 - p1);
}

// the slot that op carries slot s to: p'[r] = sgn_r (p[perm r] - 1) + 1
__host__ __device__ inline int op_image(int op, int s) {
  int p[3], q[3];
  slot_pos(s, p);
  for (int r = 0; r < 3; ++r) {
    const int v = p[perm_of(op, r)] - 1;
    q[r] = ((op >> r) & 1 ? -v : v) + 1;
  }
  return pos_slot(q);
}

// the slot that op carries onto slot t (inverse image)
__host__ __device__ inline int op_preimage(int op, int t) {
  int q[3], p[3];
  slot_pos(t, q);
  for (int r = 0; r < 3; ++r) {
    const int v = q[r] - 1;
    p[perm_of(op, r)] = ((op >> r) & 1 ? -v : v) + 1;
  }
  return pos_slot(p);
}

__host__ __device__ inline int mask_image(int op, int mask) {
  int out = 0;
  for (int e = 0; e < 12; ++e)
    if ((mask >> e) & 1) out |= 1 << (op_image(op, 8 + e) - 8);
  return out;
}

// bit s of the result: slot s present in a cell of this mask
__host__ __device__ inline uint32_t present_slots(int mask) {
  uint32_t out = 0xFFu | ((uint32_t)mask << 8);
  for (int f = 0; f < 6; ++f) {
    const int a = f >> 1, side = 2 * (f & 1);
    int cnt = 0, axes = 0;
    for (int e = 0; e < 12; ++e) {
      if (!((mask >> e) & 1)) continue;
      int p[3];
      slot_pos(8 + e, p);
      if (p[a] == side) {
        ++cnt;
        axes |= 1 << (e >> 2);
      }
    }
    // two present mid-edges on one axis are opposite
    if (cnt >= 1 && !(cnt == 2 && (axes & (axes - 1)) == 0)) out |= 1u << (20 + f);
  }
  return out;
}

// table[mask] = master | op << 16
__global__ void k_mask_table(int32_t *table) {
  const int mask = blockIdx.x * blockDim.x + threadIdx.x;
  if (mask >= 4096) return;
  int best = -1, best_op = 0;
  for (int op = 0; op < 48; ++op) {
    const int img = mask_image(op, mask);
    if (img > best) {
      best = img;
      best_op = op;
    }
  }
  table[mask] = best | (best_op << 16);
}

__global__ void k_flag_masters(int64_t n, const int32_t *__restrict__ mask,
                               const int32_t *__restrict__ table, int32_t *used) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    used[table[mask[c]] & 0xFFFF] = 1;
}

// per cell: pattern id, op, node count (into cnt for the scan)
__global__ void k_classify(int64_t n, const int32_t *__restrict__ mask,
                           const int32_t *__restrict__ table, const int32_t *__restrict__ pid,
                           int32_t *pat, uint8_t *sym, int64_t *cnt) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int t = table[mask[c]], master = t & 0xFFFF;
    pat[c] = pid[master];
    sym[c] = (uint8_t)(t >> 16);
    cnt[c] = __popc(present_slots(master));
  }
}

// per cell: its nodes in master order; bad[0] counts missing nodes
__global__ void k_cell_nodes(int64_t n, const int32_t *__restrict__ slot_node,
                             const int32_t *__restrict__ mask, const int32_t *__restrict__ table,
                             const int64_t *__restrict__ ptr, int32_t *nodes, int32_t *bad) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int t = table[mask[c]], master = t & 0xFFFF, op = t >> 16;
    uint32_t pres = present_slots(master);
    int64_t o = ptr[c];
    while (pres) {
      const int ts = __ffs(pres) - 1;
      pres &= pres - 1;
      const int32_t v = slot_node[26 * c + op_preimage(op, ts)];
      if (v < 0) atomicAdd(bad, 1);
      nodes[o++] = v;
    }
  }
}

// exclusive scan of int64 values in place: per block, then the block sums
// by one block, then the offsets added
constexpr int SCAN_T = 1024;
__device__ inline int64_t block_scan_incl(int64_t v, int64_t *sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int d = 1; d < SCAN_T; d <<= 1) {
    const int64_t a = tid >= d ? sh[tid - d] : 0;
    __syncthreads();
    sh[tid] += a;
    __syncthreads();
  }
  return sh[tid];
}
__global__ void k_scan_blocks(int64_t n, int64_t *x, int64_t *bsum) {
  __shared__ int64_t sh[SCAN_T];
  const int64_t i = blockIdx.x * (int64_t)SCAN_T + threadIdx.x;
  const int64_t v = i < n ? x[i] : 0;
  const int64_t inc = block_scan_incl(v, sh);
  if (i < n) x[i] = inc - v;
  if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = inc;
}
__global__ void k_scan_sums(int64_t nb, int64_t *bsum, int64_t *total) {
  __shared__ int64_t sh[SCAN_T];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += SCAN_T) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < nb ? bsum[i] : 0;
    const int64_t inc = block_scan_incl(v, sh);
    if (i < nb) bsum[i] = carry + inc - v;
    __syncthreads();
    carry += sh[SCAN_T - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}
__global__ void k_scan_add(int64_t n, int64_t *x, const int64_t *bsum) {
  const int64_t i = blockIdx.x * (int64_t)SCAN_T + threadIdx.x;
  if (i < n) x[i] += bsum[blockIdx.x];
}

// stable counting sort by pattern: per block of SCAN_T cells the count of
// each pattern (pattern-major over blocks: cnt[p * nb + b])
__global__ void k_sort_count(int64_t n, int P, const int32_t *__restrict__ pat, int64_t *cnt,
                             int64_t nb) {
  extern __shared__ int32_t hs[];
  for (int p = threadIdx.x; p < P; p += blockDim.x) hs[p] = 0;
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)SCAN_T + threadIdx.x;
  if (i < n) atomicAdd(&hs[pat[i]], 1);
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) cnt[(int64_t)p * nb + blockIdx.x] = hs[p];
}
// ranks within the block keep the given order: per warp by match_any, the
// warps' counts per pattern scanned in warp order
__global__ void k_sort_scatter(int64_t n, int P, const int32_t *__restrict__ pat,
                               const int64_t *__restrict__ off, int64_t nb, int64_t *order) {
  extern __shared__ int32_t wc[];   // [32 warps][P]
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int q = tid; q < 32 * P; q += blockDim.x) wc[q] = 0;
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)SCAN_T + tid;
  const int p = i < n ? pat[i] : -1;
  const unsigned same = __match_any_sync(0xffffffffu, p);
  const int rank = __popc(same & ((1u << lane) - 1u));
  if (p >= 0 && rank == 0) wc[w * P + p] = __popc(same);
  __syncthreads();
  for (int q = tid; q < P; q += blockDim.x) {   // exclusive scan over the warps
    int32_t acc = 0;
    for (int v = 0; v < 32; ++v) {
      const int32_t c = wc[v * P + q];
      wc[v * P + q] = acc;
      acc += c;
    }
  }
  __syncthreads();
  if (p >= 0) order[off[(int64_t)p * nb + blockIdx.x] + wc[w * P + p] + rank] = i;
}

// slot-major connectivity: conn[conn_off[p] + k C_p + j] = node k of the
// j-th cell of pattern p
__global__ void k_conn(int64_t n, const int64_t *__restrict__ order, const int32_t *__restrict__ pat,
                       const int64_t *__restrict__ pstart, const int64_t *__restrict__ coff,
                       const int64_t *__restrict__ ptr, const int32_t *__restrict__ nodes,
                       int32_t *conn) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = order[s];
    const int p = pat[e];
    const int64_t j = s - pstart[p], Cp = pstart[p + 1] - pstart[p];
    const int np = (int)(ptr[e + 1] - ptr[e]);
    for (int k = 0; k < np; ++k) conn[coff[p] + (int64_t)k * Cp + j] = nodes[ptr[e] + k];
  }
}

}  // namespace

cudaError_t setup_mask_table(int32_t *table, cudaStream_t s) {
  k_mask_table<<<16, 256, 0, s>>>(table);
  return cudaGetLastError();
}

cudaError_t setup_flag_masters(int64_t n, const int32_t *mask, const int32_t *table, int32_t *used,
                               int grid, cudaStream_t s) {
  k_flag_masters<<<grid, 256, 0, s>>>(n, mask, table, used);
  return cudaGetLastError();
}

cudaError_t setup_classify(int64_t n, const int32_t *mask, const int32_t *table,
                           const int32_t *pid, int32_t *pat, uint8_t *sym, int64_t *cnt, int grid,
                           cudaStream_t s) {
  k_classify<<<grid, 256, 0, s>>>(n, mask, table, pid, pat, sym, cnt);
  return cudaGetLastError();
}

// exclusive scan of x[0..n) in place; *total (device) = the sum
cudaError_t setup_scan(int64_t n, int64_t *x, int64_t *work, int64_t *total, cudaStream_t s) {
  const int64_t nb = (n + SCAN_T - 1) / SCAN_T;
  if (nb > 0) k_scan_blocks<<<(unsigned)nb, SCAN_T, 0, s>>>(n, x, work);
  k_scan_sums<<<1, SCAN_T, 0, s>>>(nb, work, total);
  if (nb > 0) k_scan_add<<<(unsigned)nb, SCAN_T, 0, s>>>(n, x, work);
  return cudaGetLastError();
}

cudaError_t setup_cell_nodes(int64_t n, const int32_t *slot_node, const int32_t *mask,
                             const int32_t *table, const int64_t *ptr, int32_t *nodes, int32_t *bad,
                             int grid, cudaStream_t s) {
  k_cell_nodes<<<grid, 256, 0, s>>>(n, slot_node, mask, table, ptr, nodes, bad);
  return cudaGetLastError();
}

cudaError_t setup_sort_count(int64_t n, int P, const int32_t *pat, int64_t *cnt, cudaStream_t s) {
  const int64_t nb = (n + SCAN_T - 1) / SCAN_T;
  if (nb > 0) k_sort_count<<<(unsigned)nb, SCAN_T, P * sizeof(int32_t), s>>>(n, P, pat, cnt, nb);
  return cudaGetLastError();
}

cudaError_t setup_sort_scatter(int64_t n, int P, const int32_t *pat, const int64_t *off,
                               int64_t *order, cudaStream_t s) {
  const int64_t nb = (n + SCAN_T - 1) / SCAN_T;
  if (nb > 0)
    k_sort_scatter<<<(unsigned)nb, SCAN_T, 32 * P * sizeof(int32_t), s>>>(n, P, pat, off, nb, order);
  return cudaGetLastError();
}

cudaError_t setup_conn(int64_t n, const int64_t *order, const int32_t *pat, const int64_t *pstart,
                       const int64_t *coff, const int64_t *ptr, const int32_t *nodes,
                       int32_t *conn, int grid, cudaStream_t s) {
  k_conn<<<grid, 256, 0, s>>>(n, order, pat, pstart, coff, ptr, nodes, conn);
  return cudaGetLastError();
}

}  // namespace sbx

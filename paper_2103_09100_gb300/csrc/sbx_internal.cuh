// Internal declarations of the sbx library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <string>
#include <vector>

#include "../../include/sbx.h"

namespace sbx {

// A tile: up to `ncell` consecutive cells of one pattern.  `cell0` is the
// index of the first cell inside its pattern group.
struct Tile {
  int32_t pat;
  int32_t ncell;
  int64_t cell0;
};

// The regular 8-node cell's K_p in the Walsh basis (FP64 form): the corner
// reflections of the cube leave K_p invariant, so with the nodal values of
// each component Walsh-transformed over the 2 x 2 x 2 corners, K_p falls
// apart into eight 3 x 3 blocks (blk[9 s + 3 r + c], s = block).
struct WhtBlocks {
  double blk[72];
};

// Time function of the point loads (Sec. 5): kind, t1, peak, cycles.
struct LoadTable {
  int n;                 // number of (dof, load) entries
  const int64_t *dof;    // DOF index (batched: (3 node + d) * B + b)
  const double *amp;     // P0 * dir component
  const int32_t *kind;   // SBX_WAVE_*
  const double *t1;
  const double *ncyc;
};

// Everything a force kernel needs about the mesh; device pointers.
struct MeshView {
  int64_t n_dof;              // 3 N (per load case)
  int B;                      // load cases
  const int32_t *pat_m;       // m_p = 3 n_p
  const int64_t *koff;        // offset of K_p in the packed pattern arrays
  const int32_t *conn;        // per pattern: [n_p][C_p] node ids (slot-major)
  const int64_t *conn_off;    // offset of pattern p's block in conn
  const int64_t *pat_cstart;  // first sorted cell of pattern p
  const int64_t *pat_ccount;  // C_p
  const uint8_t *sym;         // op per sorted cell
  const double *scale;        // s_e = E_e h_e per sorted cell
};

constexpr int TC_CLASSES = 1;

// Tensor-core path: a tile of up to 128 cells of one pattern and its unique
// nodes.  A tile's record is one contiguous, 16-byte-padded block in global
// memory, fetched with one bulk copy (layout in kernels_tc.cu).
struct TcTile {
  int64_t rec_off;    // byte offset of the record
  int32_t rec_bytes;  // multiple of 16
  int32_t pat;
};

struct GraphCache {
  bool valid = false;
  double dt = 0, alpha = 0;
  int unit = 0;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  // tail[r][parity]: r full steps then the closing step (which keeps
  // R_int), for the r = (n_steps - 1) mod unit steps a call has left over
  std::map<int, std::array<cudaGraphExec_t, 2>> tail;
};

}  // namespace sbx

struct sbx_ctx {
  int device = 0;
  int n_sm = 1;                    // multiprocessors of the device (grid sizing)
  cudaStream_t stream = nullptr;
  // second stream for a force kernel that runs beside the first (forked
  // from and joined back into `stream` with the two events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool own_stream = false;
  std::string err;

  // patterns
  int n_pat = 0;
  std::vector<int32_t> pat_nodes;
  std::vector<int64_t> pat_koff;   // offsets in the packed K (m_p^2 each)
  std::vector<int64_t> pat_moff;   // offsets in the packed lumped mass
  std::vector<double> K_host, M_host;
  double *d_K64 = nullptr;         // packed K_p, FP64
  float *d_K32 = nullptr;          // packed K_p rounded to FP32
  int32_t *d_pat_m = nullptr;
  int64_t *d_koff = nullptr;

  // mesh
  bool have_mesh = false;
  int64_t N = 0, C = 0, ndof = 0;  // ndof = 3 N (one load case)
  int B = 1, prec = SBX_PREC_FP64;
  std::vector<int64_t> pat_cstart, pat_ccount;
  std::vector<int64_t> h_order;      // sorted position -> caller's cell index
  std::vector<double> h_hs;          // edge length per sorted cell
  int32_t *d_conn = nullptr;
  int64_t *d_conn_off = nullptr, *d_pat_cstart = nullptr, *d_pat_ccount = nullptr;
  uint8_t *d_sym = nullptr;
  double *d_scale = nullptr;
  double *d_minv = nullptr;        // 1 / M_diag, 0 on fixed DOFs ([3N])
  double *d_mass = nullptr;        // M_diag ([3N])
  double *d_w = nullptr;           // dt^2 M^-1 / (1 + alpha dt / 2) for (w_dt, w_alpha)
  bool w_valid = false;
  double w_dt = 0.0, w_alpha = 0.0;
  double *d_u[2] = {nullptr, nullptr};
  int cur = 0;                     // d_u[cur] = U_n, d_u[cur ^ 1] = U_{n-1}
  double *d_f = nullptr;           // R_int - R_ext accumulator; SBX_PREC_MIXED: float [N][4]
  double *d_fx = nullptr;          // SBX_PREC_MIXED: d_f widened to FP64 [3N] on demand
  // SBX_PREC_MIXED (and batched FP32): one state buffer split into FP32
  // (hi xyz, lo xyz) per node, written by the update kernel (or by
  // k_split_pairs after a host write).  One buffer serves both state
  // buffers: the update of step n writes the pairs of U_{n+1} over those of
  // U_n, which the force of step n has finished reading.  pair_of = the
  // state buffer (0, 1) whose pairs it holds, -1 for none.
  float *d_pair = nullptr;
  int pair_of = -1;
  bool f_dirty = false;
  bool f_pending = false;          // sbx_force done, sbx_update not yet
  std::vector<int64_t> h_fixed;    // Dirichlet DOFs (M^-1 = 0)
  int32_t *d_flags = nullptr;
  int64_t *d_step = nullptr;       // device copy of the step index
  int64_t step = 0;
  sbx::Tile *d_tiles_simt = nullptr;
  int n_tiles_simt = 0;
  // FP64 force: the 8-node identity-op cells by the Walsh-basis kernel
  // (pattern wht_pat, wht_cells of them), the rest by the dense tiles
  int wht_pat = -1;
  int64_t wht_cells = 0;
  sbx::WhtBlocks wht{};
  sbx::Tile *d_tiles_rest = nullptr;
  int n_tiles_rest = 0;
  int max_m = 0;

  // mixed path (SBX_PREC_MIXED): tensor-core tiles of the 8-node cell and
  // 32-cell SIMT tiles of the other patterns
  float *d_tc_K = nullptr;         // K_p of the 8-node cell, TF32 hi | lo, canonical layout
  uint8_t *d_tc_rec = nullptr;     // tile records
  sbx::TcTile *d_tc_tiles[sbx::TC_CLASSES] = {};
  int n_tc_tiles[sbx::TC_CLASSES] = {};
  int tc_rec_max[sbx::TC_CLASSES] = {}, tc_nn_max[sbx::TC_CLASSES] = {};
  int tc_grid[sbx::TC_CLASSES] = {};
  size_t tc_smem[sbx::TC_CLASSES] = {};
  int n_brick_tiles = 0;           // of n_tc_tiles[0]: complete 4 x 4 x 8 blocks
  sbx::Tile *d_gen_tiles = nullptr;
  float *d_gen_K = nullptr;        // FP32 K_p of those patterns, rows padded to a multiple of 4
  int64_t *d_gen_koff = nullptr;
  int n_gen_tiles = 0;
  size_t gen_smem = 0;
  // the other patterns on the tensor cores (k_force_gen_tc): 128-cell tile
  // records, per-pattern B = K_p TF32 hi | lo (offsets in floats, P + 1)
  uint8_t *d_gt_rec = nullptr;
  sbx::TcTile *d_gt_tiles = nullptr;
  float *d_gt_B = nullptr;
  int64_t *d_gt_boff = nullptr;
  int n_gt_tiles = 0;
  size_t gt_smem = 0;
  uint32_t gt_rec_off = 0;         // record offset in shared memory (after the largest B)
  int hanging_ctas = 1;            // k_force_gen_tc CTAs per SM
  bool hanging_tc = true;          // the other patterns on the tensor cores (mesh_upload: B == 1)
  int walsh_ctas = 0;              // Walsh-kernel CTAs per SM (0: automatic)
  bool update_bulk = true;         // mixed update: chunks by bulk copy (k_update_f32_bulk)
  // the 8-node tiles by the Walsh-basis SIMT kernel instead of the tensor
  // cores (sbx_set_mixed_kernel)
  bool mixed_wht = false;
  size_t wt_smem = 0;
  int wt_grid = 0;

  // batched path (n_rhs > 1): tile records in three classes by pattern size
  uint8_t *d_b_rec = nullptr;
  sbx::TcTile *d_b_tiles[3] = {};
  int n_b_tiles[3] = {}, b_nnmax[3] = {}, b_recmax[3] = {};
  size_t b_smem[3] = {};
  // tile shape per class (sbx_set_launch): most cells per tile and the
  // shared-memory budget per CTA in KB that bounds a tile's staging
  int b_tile_cells[3] = {32, 32, 32};
  int b_smem_kb[3] = {100, 100, 100};
  // host copies of the sorted mesh, kept to rebuild the tiles
  std::vector<int32_t> hb_conn;
  std::vector<int64_t> hb_conn_off, hb_cnt, hb_start;
  std::vector<uint8_t> hb_sym;
  std::vector<double> hb_scale;

  // receiver time history (sbx_set_receivers): hist[row][n_rec], row = step
  // index - rec_step0 - 1 of the step just taken, rows < rec_cap
  int64_t *d_rec_idx = nullptr;
  double *d_hist = nullptr;
  int64_t n_rec_hist = 0, rec_cap = 0, rec_step0 = 0;

  // loads
  int n_load = 0;
  int64_t *d_load_dof = nullptr;
  double *d_load_amp = nullptr, *d_load_t1 = nullptr, *d_load_ncyc = nullptr;
  int32_t *d_load_kind = nullptr;

  sbx::GraphCache graph;

  // node-cut interface sum with the neighbours (sbx_halo_plan)
  int64_t halo_n_send = 0, halo_n_cut = 0, halo_n_recv_rows = 0;
  int64_t *d_halo_send = nullptr, *d_halo_cut = nullptr, *d_halo_ptr = nullptr,
          *d_halo_src = nullptr;
  // sbx_share_state: this context steps nothing itself; its force kernels
  // read the owner's state and add into the owner's accumulator
  sbx_ctx *state_owner = nullptr;
  int n_guests = 0;

  sbx::MeshView view() const {
    return sbx::MeshView{ndof, B, d_pat_m, d_koff, d_conn, d_conn_off, d_pat_cstart,
                         d_pat_ccount, d_sym, d_scale};
  }
  sbx::LoadTable loads() const {
    return sbx::LoadTable{n_load, d_load_dof, d_load_amp, d_load_kind, d_load_t1, d_load_ncyc};
  }
  // FP32-contraction forms that take U_n as (hi, lo) pairs and keep f in
  // FP32: the mixed form (one load case; pairs float [N][6], f float [N][4])
  // and the batched FP32 form (pairs float2 and f float per DOF and case)
  bool uses_pairs() const {
    return (prec == SBX_PREC_MIXED && B == 1) || (prec == SBX_PREC_FP32 && B > 1);
  }
};

namespace sbx {
// kernels_simt.cu
constexpr int SIMT_TILE = 32;
cudaError_t launch_force_simt(const sbx_ctx *ctx, const double *u, double *f, double dt,
                              cudaStream_t s, bool with_loads = true);
// kernels_adjoint.cu
cudaError_t launch_weight(const sbx_ctx *ctx, const double *lam, double *v, cudaStream_t s);
cudaError_t launch_adj_update(const sbx_ctx *ctx, const double *f, const double *lam1,
                              double *lam2_to_lam, cudaStream_t s);
cudaError_t launch_residual(const sbx_ctx *ctx, int64_t n_rec, const int64_t *rec,
                            const double *u_n, const double *data_n, double *lam, double *J,
                            cudaStream_t s);
cudaError_t launch_grad(const sbx_ctx *ctx, const double *u, const double *v, double *acc,
                        cudaStream_t s);
cudaError_t prepare_adjoint_kernels();
// w = dt^2 M^-1 / (1 + alpha dt / 2) for the update; recomputed when dt or
// alpha change (outside stream capture).
cudaError_t prepare_update(sbx_ctx *ctx, double dt, double alpha, cudaStream_t s);
cudaError_t launch_update(const sbx_ctx *ctx, const double *uc, double *up, double *f, double dt,
                          double alpha, int zero_f, cudaStream_t s);
cudaError_t launch_init_um1(const sbx_ctx *ctx, const double *u0, const double *v0, double *um1,
                            const double *f, double dt, double alpha, cudaStream_t s);
cudaError_t launch_zero_fixed(const sbx_ctx *ctx, double *u, cudaStream_t s);
// receiver history: copy U at the receivers into the row of the step just
// taken (read from the device step index)
cudaError_t launch_record(const sbx_ctx *ctx, const double *u, cudaStream_t s);
// Opt every kernel into the shared-memory size it may need (call once per
// device, outside stream capture).
cudaError_t prepare_kernels();
// kernels_tc.cu
int tc_setup(sbx_ctx *ctx, const std::vector<int32_t> &conn, const std::vector<int64_t> &conn_off,
             const std::vector<int64_t> &cnt, const std::vector<int64_t> &start,
             const std::vector<uint8_t> &sym_sorted, const std::vector<double> &scale_sorted,
             std::string &err);
cudaError_t prepare_tc_kernels();
// tables of the tensor-core kernels for the other patterns (the marked ones)
int gt_setup(sbx_ctx *ctx, const std::vector<int32_t> &conn, const std::vector<int64_t> &conn_off,
             const std::vector<int64_t> &cnt, const std::vector<int64_t> &start,
             const std::vector<uint8_t> &sym_sorted, const std::vector<double> &scale_sorted,
             const std::vector<char> &use, std::string &err);
// batched FP32 form: the cells of the gt tables on the tensor cores
cudaError_t launch_force_batch_tc(const sbx_ctx *ctx, const float *pairs, float *f, double dt,
                                  LoadTable L, cudaStream_t s);
cudaError_t launch_wait_selftest(const sbx_ctx *ctx, uint32_t polls, int arrive, cudaStream_t s);
// kernels_eigen.cu: k Lanczos steps (full reorthogonalisation) of
// M^-1/2 K M^-1/2 from v0 (device, 3N); alpha, beta: device, k doubles
int lanczos_run(sbx_ctx *ctx, int64_t k, const double *v0_dev, double *alpha_dev,
                double *beta_dev, std::string &err);
// kernels_halo.cu: rows of the force accumulator to the send buffer
// (d_halo_send order) and the canonical sum of the cut nodes' partial forces
cudaError_t launch_halo_pack(const sbx_ctx *ctx, void *out, cudaStream_t s);
cudaError_t launch_halo_sum(const sbx_ctx *ctx, const void *recv, cudaStream_t s);
// kernels_setup.cu: classification, node lists, sort and connectivity on the GPU
cudaError_t setup_mask_table(int32_t *table, cudaStream_t s);
cudaError_t setup_flag_masters(int64_t n, const int32_t *mask, const int32_t *table, int32_t *used,
                               int grid, cudaStream_t s);
cudaError_t setup_classify(int64_t n, const int32_t *mask, const int32_t *table,
                           const int32_t *pid, int32_t *pat, uint8_t *sym, int64_t *cnt, int grid,
                           cudaStream_t s);
cudaError_t setup_scan(int64_t n, int64_t *x, int64_t *work, int64_t *total, cudaStream_t s);
cudaError_t setup_cell_nodes(int64_t n, const int32_t *slot_node, const int32_t *mask,
                             const int32_t *table, const int64_t *ptr, int32_t *nodes, int32_t *bad,
                             int grid, cudaStream_t s);
cudaError_t setup_sort_count(int64_t n, int P, const int32_t *pat, int64_t *cnt, cudaStream_t s);
cudaError_t setup_sort_scatter(int64_t n, int P, const int32_t *pat, const int64_t *off,
                               int64_t *order, cudaStream_t s);
cudaError_t setup_conn(int64_t n, const int64_t *order, const int32_t *pat, const int64_t *pstart,
                       const int64_t *coff, const int64_t *ptr, const int32_t *nodes,
                       int32_t *conn, int grid, cudaStream_t s);
// kernels_batch.cu
int batch_setup(sbx_ctx *ctx, const std::vector<int32_t> &conn, const std::vector<int64_t> &conn_off,
                const std::vector<int64_t> &cnt, const std::vector<uint8_t> &sym_sorted,
                const std::vector<double> &scale_sorted, const std::vector<int64_t> &start,
                std::string &err);
cudaError_t prepare_batch_kernels();
// u: FP64 state (SBX_PREC_FP64) or the (hi, lo) pairs (SBX_PREC_FP32); f:
// double or float per DOF and case
cudaError_t launch_force_batch(const sbx_ctx *ctx, const void *u, void *f, double dt,
                               cudaStream_t s);
cudaError_t launch_update_batch(const sbx_ctx *ctx, const double *uc, double *up, void *f,
                                float *pairs_out, double dt, double alpha, int zero_f,
                                cudaStream_t s);
// Mixed form: f is float [N][4] (x, y, z, unused) in the d_f allocation;
// U_n enters the force kernel as its (hi, lo) pairs, float [N][6].
cudaError_t launch_force_tc(const sbx_ctx *ctx, const float *pairs, float *f4, double dt,
                            cudaStream_t s);
cudaError_t launch_update_f32(const sbx_ctx *ctx, const double *uc, double *up, float *f4,
                              float *pairs_out, double dt, double alpha, int zero_f,
                              cudaStream_t s);
// (hi, lo) pairs of a state buffer in the layout of ctx's form
cudaError_t launch_split_pairs(const sbx_ctx *ctx, const double *u, float *pairs, cudaStream_t s);
// the FP32 force buffer as FP64 per DOF (and case): mixed out[3 i + d] =
// f4[4 i + d]; batched out[i] = f[i]
cudaError_t launch_widen_f32(const sbx_ctx *ctx, const float *f4, double *out, cudaStream_t s);
}  // namespace sbx

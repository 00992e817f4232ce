// C ABI of the explicit octree-SBFEM solver: context, validation, uploads,
// step loop.  Declarations and argument contracts: include/sbx.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "sbx_internal.cuh"

using sbx::Tile;

namespace {

int fail(sbx_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(sbx_ctx *ctx, cudaError_t e, const char *where) {
  return fail(ctx, SBX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy `bytes` from a host or device pointer into host memory.
int fetch(sbx_ctx *ctx, void *dst_host, const void *src, size_t bytes) {
  if (bytes == 0) return SBX_OK;
  if (!src) return fail(ctx, SBX_EINVAL, "null input array");
  if (is_device_ptr(src)) {
    CK(cudaMemcpyAsync(dst_host, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    memcpy(dst_host, src, bytes);
  }
  return SBX_OK;
}

template <typename T>
int fetch_vec(sbx_ctx *ctx, std::vector<T> &v, const T *src, size_t n) {
  try {
    v.resize(n);
  } catch (const std::bad_alloc &) {
    return fail(ctx, SBX_ENOMEM, "host allocation failed");
  }
  return fetch(ctx, v.data(), src, n * sizeof(T));
}

template <typename T>
int dalloc(sbx_ctx *ctx, T **p, size_t n) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, SBX_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return SBX_OK;
}

template <typename T>
int upload(sbx_ctx *ctx, T **p, const std::vector<T> &v) {
  int rc = dalloc(ctx, p, v.size());
  if (rc) return rc;
  if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return SBX_OK;
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void drop_graph(sbx_ctx *ctx) {
  for (auto &g : ctx->graph.exec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (auto &kv : ctx->graph.tail)
    for (auto &g : kv.second)
      if (g) cudaGraphExecDestroy(g);
  ctx->graph.tail.clear();
  ctx->graph.valid = false;
}

void free_mesh(sbx_ctx *ctx) {
  drop_graph(ctx);
  if (sbx_ctx *o = ctx->state_owner) {   // the state buffers are the owner's
    ctx->d_u[0] = ctx->d_u[1] = nullptr;
    ctx->d_f = nullptr;
    ctx->d_pair = nullptr;
    o->n_guests -= 1;
    ctx->state_owner = nullptr;
  }
  dfree(ctx->d_halo_send); dfree(ctx->d_halo_cut); dfree(ctx->d_halo_ptr); dfree(ctx->d_halo_src);
  ctx->halo_n_send = ctx->halo_n_cut = 0;
  dfree(ctx->d_conn); dfree(ctx->d_conn_off); dfree(ctx->d_pat_cstart); dfree(ctx->d_pat_ccount);
  dfree(ctx->d_sym); dfree(ctx->d_scale); dfree(ctx->d_minv); dfree(ctx->d_mass);
  dfree(ctx->d_w);
  ctx->w_valid = false;
  dfree(ctx->d_u[0]); dfree(ctx->d_u[1]); dfree(ctx->d_f); dfree(ctx->d_fx);
  dfree(ctx->d_pair);
  ctx->pair_of = -1;
  dfree(ctx->d_tiles_simt);
  dfree(ctx->d_tiles_rest);
  ctx->n_tiles_rest = 0;
  ctx->wht_pat = -1;
  ctx->wht_cells = 0;
  dfree(ctx->d_load_dof); dfree(ctx->d_load_amp); dfree(ctx->d_load_t1); dfree(ctx->d_load_ncyc);
  dfree(ctx->d_load_kind);
  dfree(ctx->d_tc_K); dfree(ctx->d_tc_rec); dfree(ctx->d_gen_tiles); dfree(ctx->d_gen_K);
  dfree(ctx->d_gt_rec); dfree(ctx->d_gt_tiles); dfree(ctx->d_gt_B); dfree(ctx->d_gt_boff);
  ctx->n_gt_tiles = 0;
  dfree(ctx->d_gen_koff);
  dfree(ctx->d_rec_idx); dfree(ctx->d_hist);
  ctx->n_rec_hist = ctx->rec_cap = 0;
  ctx->n_gen_tiles = 0;
  dfree(ctx->d_b_rec);
  for (int c = 0; c < 3; ++c) {
    dfree(ctx->d_b_tiles[c]);
    ctx->n_b_tiles[c] = 0;
  }
  for (int c = 0; c < sbx::TC_CLASSES; ++c) {
    dfree(ctx->d_tc_tiles[c]);
    ctx->n_tc_tiles[c] = 0;
  }
  ctx->n_load = 0;
  ctx->have_mesh = false;
}

void free_patterns(sbx_ctx *ctx) {
  dfree(ctx->d_K64); dfree(ctx->d_K32); dfree(ctx->d_pat_m); dfree(ctx->d_koff);
  ctx->n_pat = 0;
}

int set_device(sbx_ctx *ctx) {
  CK(cudaSetDevice(ctx->device));
  return SBX_OK;
}

int force(sbx_ctx *ctx, const double *u, double *f, double dt) {
  const float *pairs = nullptr;
  if (ctx->uses_pairs()) {
    const int p = u == ctx->d_u[0] ? 0 : (u == ctx->d_u[1] ? 1 : -1);
    if (p < 0) return fail(ctx, SBX_EINVAL, "this form's force runs on the state buffers only");
    if (ctx->pair_of != p) {
      CK(sbx::launch_split_pairs(ctx, u, ctx->d_pair, ctx->stream));
      ctx->pair_of = p;
    }
    pairs = ctx->d_pair;
  }
  if (ctx->B > 1) {
    CK(sbx::launch_force_batch(ctx, pairs ? (const void *)pairs : (const void *)u, f, dt,
                               ctx->stream));
  } else if (ctx->prec == SBX_PREC_MIXED) {
    CK(sbx::launch_force_tc(ctx, pairs, reinterpret_cast<float *>(f), dt, ctx->stream));
  } else {
    CK(sbx::launch_force_simt(ctx, u, f, dt, ctx->stream));
  }
  return SBX_OK;
}

int update(sbx_ctx *ctx, const double *uc, double *up, double dt, double alpha, int zero_f) {
  if (ctx->B > 1) {
    const int p = up == ctx->d_u[0] ? 0 : 1;
    float *pairs_out = ctx->uses_pairs() ? ctx->d_pair : nullptr;
    CK(sbx::launch_update_batch(ctx, uc, up, ctx->d_f, pairs_out, dt, alpha, zero_f, ctx->stream));
    if (pairs_out) ctx->pair_of = p;
  } else if (ctx->prec == SBX_PREC_MIXED) {
    const int p = up == ctx->d_u[0] ? 0 : 1;
    CK(sbx::launch_update_f32(ctx, uc, up, reinterpret_cast<float *>(ctx->d_f), ctx->d_pair, dt,
                              alpha, zero_f, ctx->stream));
    ctx->pair_of = p;
  } else {
    CK(sbx::launch_update(ctx, uc, up, ctx->d_f, dt, alpha, zero_f, ctx->stream));
  }
  return SBX_OK;
}

// Mixed form: make the (hi, lo) pairs of U_n current before replaying a
// graph (the captured steps take them from the previous update).
int ensure_pairs(sbx_ctx *ctx) {
  if (!ctx->uses_pairs() || ctx->pair_of == ctx->cur) return SBX_OK;
  CK(sbx::launch_split_pairs(ctx, ctx->d_u[ctx->cur], ctx->d_pair, ctx->stream));
  ctx->pair_of = ctx->cur;
  return SBX_OK;
}

// One CDM step from d_u[cur] (U_n) into d_u[cur ^ 1] (U_{n-1} -> U_{n+1}).
int one_step(sbx_ctx *ctx, int parity, double dt, double alpha, int zero_f) {
  double *uc = ctx->d_u[parity], *up = ctx->d_u[parity ^ 1];
  int rc = force(ctx, uc, ctx->d_f, dt);
  if (rc) return rc;
  if ((rc = update(ctx, uc, up, dt, alpha, zero_f))) return rc;
  CK(sbx::launch_record(ctx, up, ctx->stream));   // up now holds U_{n+1}
  return SBX_OK;
}

constexpr int GRAPH_UNIT = 32;  // steps per replayed graph (even)

int build_graphs(sbx_ctx *ctx, double dt, double alpha) {
  drop_graph(ctx);
  const int pair_before = ctx->pair_of;
  for (int parity = 0; parity < 2; ++parity) {
    cudaGraph_t g;
    // a graph is replayed with the pairs of its first U_n current
    // (ensure_pairs), so no split is captured into it
    ctx->pair_of = parity;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = SBX_OK;
    for (int s = 0; s < GRAPH_UNIT && rc == SBX_OK; ++s) rc = one_step(ctx, parity ^ (s & 1), dt, alpha, 1);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    ctx->pair_of = pair_before;
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->graph.exec[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
  }
  ctx->graph.valid = true;
  ctx->graph.dt = dt;
  ctx->graph.alpha = alpha;
  ctx->graph.unit = GRAPH_UNIT;
  return SBX_OK;
}

// The graphs of a call's last r + 1 steps (r < GRAPH_UNIT full steps, then
// the closing step that keeps R_int), for both parities of the state pair.
int build_tail(sbx_ctx *ctx, int r, double dt, double alpha) {
  if (!ctx->graph.valid || ctx->graph.dt != dt || ctx->graph.alpha != alpha)
    if (int rc = build_graphs(ctx, dt, alpha)) return rc;
  if (ctx->graph.tail.count(r)) return SBX_OK;
  std::array<cudaGraphExec_t, 2> ex = {nullptr, nullptr};
  const int pair_before = ctx->pair_of;
  for (int parity = 0; parity < 2; ++parity) {
    cudaGraph_t g;
    ctx->pair_of = parity;   // as in build_graphs
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = SBX_OK;
    for (int s = 0; s <= r && rc == SBX_OK; ++s)
      rc = one_step(ctx, parity ^ (s & 1), dt, alpha, s < r ? 1 : 0);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    ctx->pair_of = pair_before;
    if (rc == SBX_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaStreamEndCapture");
    if (rc == SBX_OK) {
      e = cudaGraphInstantiate(&ex[parity], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    if (rc) {
      for (auto &x : ex)
        if (x) cudaGraphExecDestroy(x);
      return rc;
    }
  }
  ctx->graph.tail[r] = ex;
  return SBX_OK;
}

int check_flags(sbx_ctx *ctx) {
  int32_t fl = 0;
  CK(cudaMemcpyAsync(&fl, ctx->d_flags, sizeof(fl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (fl & 2) return fail(ctx, SBX_ETIMEOUT, "a tensor-core completion wait gave up");
  if (fl & 1) return fail(ctx, SBX_ENONFINITE, "non-finite value in the displacement field");
  return SBX_OK;
}

}  // namespace

extern "C" {

int sbx_create(sbx_ctx **out, int device, void *cuda_stream) {
  if (!out) return SBX_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SBX_EINVAL;
  }
  sbx_ctx *ctx = new (std::nothrow) sbx_ctx();
  if (!ctx) return SBX_ENOMEM;
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      ctx->n_sm < 1) {
    cudaGetLastError();
    delete ctx;
    return SBX_ECUDA;
  }
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return SBX_ECUDA;
    }
    ctx->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    sbx_destroy(ctx);
    return SBX_ECUDA;
  }
  if (sbx::prepare_kernels() != cudaSuccess || sbx::prepare_tc_kernels() != cudaSuccess ||
      sbx::prepare_batch_kernels() != cudaSuccess || sbx::prepare_adjoint_kernels() != cudaSuccess) {
    cudaGetLastError();
    sbx_destroy(ctx);
    return SBX_ECUDA;
  }
  if (dalloc(ctx, &ctx->d_flags, 1) || dalloc(ctx, &ctx->d_step, 1)) {
    sbx_destroy(ctx);
    return SBX_ENOMEM;
  }
  cudaMemsetAsync(ctx->d_flags, 0, sizeof(int32_t), ctx->stream);
  cudaMemsetAsync(ctx->d_step, 0, sizeof(int64_t), ctx->stream);
  *out = ctx;
  return SBX_OK;
}

int sbx_destroy(sbx_ctx *ctx) {
  if (!ctx) return SBX_OK;
  if (ctx->n_guests > 0)
    return fail(ctx, SBX_ESTATE, "other contexts share this context's state: destroy them first");
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_mesh(ctx);
  free_patterns(ctx);
  dfree(ctx->d_flags);
  dfree(ctx->d_step);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return SBX_OK;
}

const char *sbx_last_error(const sbx_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int sbx_sync(sbx_ctx *ctx) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  return ctx->have_mesh ? check_flags(ctx) : SBX_OK;
}

int set_patterns(sbx_ctx *ctx, int n_patterns, const int32_t *n_nodes, const double *K_packed,
                 const double *Mlump_packed) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (n_patterns < 1 || n_patterns > 144) return fail(ctx, SBX_EINVAL, "n_patterns must be in [1, 144]");
  std::vector<int32_t> nn;
  if (int rc = fetch_vec(ctx, nn, n_nodes, n_patterns)) return rc;
  int64_t kt = 0, mt = 0;
  for (int p = 0; p < n_patterns; ++p) {
    if (nn[p] < 8 || nn[p] > 26) return fail(ctx, SBX_EINVAL, "pattern node count outside [8, 26]");
    kt += 9LL * nn[p] * nn[p];
    mt += 3LL * nn[p];
  }
  std::vector<double> K, Mv;
  if (int rc = fetch_vec(ctx, K, K_packed, kt)) return rc;
  if (int rc = fetch_vec(ctx, Mv, Mlump_packed, mt)) return rc;
  std::vector<int64_t> koff(n_patterns), moff(n_patterns);
  int64_t ko = 0, mo = 0;
  for (int p = 0; p < n_patterns; ++p) {
    const int m = 3 * nn[p];
    koff[p] = ko;
    moff[p] = mo;
    double nrm = 0;
    for (int i = 0; i < m * m; ++i) {
      if (!isfinite(K[ko + i])) return fail(ctx, SBX_EINVAL, "non-finite entry in K_p");
      nrm = fmax(nrm, fabs(K[ko + i]));
    }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < i; ++j)
        if (fabs(K[ko + i * m + j] - K[ko + j * m + i]) > 1e-12 * nrm)
          return fail(ctx, SBX_EINVAL, "K_p is not symmetric");
    for (int i = 0; i < m; ++i)
      if (!(Mv[mo + i] > 0) || !isfinite(Mv[mo + i])) return fail(ctx, SBX_EINVAL, "lumped mass must be positive");
    ko += (int64_t)m * m;
    mo += m;
  }
  free_mesh(ctx);
  free_patterns(ctx);
  std::vector<float> K32(K.begin(), K.end());
  std::vector<int32_t> pm(n_patterns);
  for (int p = 0; p < n_patterns; ++p) pm[p] = 3 * nn[p];
  if (int rc = upload(ctx, &ctx->d_K64, K)) return rc;
  if (int rc = upload(ctx, &ctx->d_K32, K32)) return rc;
  if (int rc = upload(ctx, &ctx->d_pat_m, pm)) return rc;
  if (int rc = upload(ctx, &ctx->d_koff, koff)) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->n_pat = n_patterns;
  ctx->pat_nodes = nn;
  ctx->pat_koff = koff;
  ctx->pat_moff = moff;
  ctx->K_host.swap(K);
  ctx->M_host.swap(Mv);
  return SBX_OK;
}

int mesh_upload(sbx_ctx *ctx, int64_t n_nodes, int64_t n_cells, const int32_t *cell_pattern,
                const uint8_t *cell_sym, const int64_t *cell_ptr, const int32_t *cell_nodes,
                const double *h, const double *E, const double *rho, int64_t n_fixed,
                const int64_t *fixed_dofs, int n_rhs, int precision_mode) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (ctx->n_pat == 0) return fail(ctx, SBX_ESTATE, "set_patterns must come before mesh_upload");
  if (ctx->n_guests > 0 || ctx->state_owner)
    return fail(ctx, SBX_ESTATE, "the state is shared with another context");
  if (n_nodes < 1 || n_cells < 1 || n_nodes > (int64_t)INT32_MAX)
    return fail(ctx, SBX_EINVAL, "n_nodes / n_cells out of range");
  if (n_rhs != 1 && (n_rhs < 32 || n_rhs % 32 != 0 || n_rhs > 1024))
    return fail(ctx, SBX_EINVAL, "n_rhs must be 1 or a multiple of 32 up to 1024");
  if (n_rhs > 1 && precision_mode == SBX_PREC_MIXED)
    return fail(ctx, SBX_EINVAL, "the batched form runs SBX_PREC_FP32 or SBX_PREC_FP64");
  if (precision_mode != SBX_PREC_FP64 && precision_mode != SBX_PREC_FP32 &&
      precision_mode != SBX_PREC_MIXED)
    return fail(ctx, SBX_EINVAL, "unknown precision_mode");
  std::vector<int32_t> pat;
  std::vector<uint8_t> sym;
  std::vector<int64_t> ptr, fixed;
  std::vector<int32_t> nodes;
  std::vector<double> hv, Ev, rv;
  if (int rc = fetch_vec(ctx, pat, cell_pattern, n_cells)) return rc;
  if (int rc = fetch_vec(ctx, sym, cell_sym, n_cells)) return rc;
  if (int rc = fetch_vec(ctx, ptr, cell_ptr, n_cells + 1)) return rc;
  if (ptr[0] != 0) return fail(ctx, SBX_EINVAL, "cell_ptr[0] must be 0");
  for (int64_t e = 0; e < n_cells; ++e) {
    if (pat[e] < 0 || pat[e] >= ctx->n_pat) return fail(ctx, SBX_EINVAL, "cell_pattern out of range");
    if (sym[e] >= 48) return fail(ctx, SBX_EINVAL, "cell_sym must be < 48");
    if (ptr[e + 1] - ptr[e] != ctx->pat_nodes[pat[e]])
      return fail(ctx, SBX_EINVAL, "cell node count does not match its pattern");
  }
  if (int rc = fetch_vec(ctx, nodes, cell_nodes, ptr[n_cells])) return rc;
  for (int64_t i = 0; i < ptr[n_cells]; ++i)
    if (nodes[i] < 0 || nodes[i] >= n_nodes) return fail(ctx, SBX_EINVAL, "cell node id out of range");
  if (int rc = fetch_vec(ctx, hv, h, n_cells)) return rc;
  if (int rc = fetch_vec(ctx, Ev, E, n_cells)) return rc;
  if (int rc = fetch_vec(ctx, rv, rho, n_cells)) return rc;
  for (int64_t e = 0; e < n_cells; ++e)
    if (!(hv[e] > 0) || !(Ev[e] > 0) || !(rv[e] > 0) || !isfinite(hv[e] * Ev[e] * rv[e]))
      return fail(ctx, SBX_EINVAL, "h, E and rho must be positive and finite");
  if (n_fixed < 0) return fail(ctx, SBX_EINVAL, "n_fixed < 0");
  if (int rc = fetch_vec(ctx, fixed, fixed_dofs, n_fixed)) return rc;
  const int64_t ndof = 3 * n_nodes;
  for (int64_t i = 0; i < n_fixed; ++i)
    if (fixed[i] < 0 || fixed[i] >= ndof) return fail(ctx, SBX_EINVAL, "fixed DOF out of range");

  // group cells by pattern (stable: keeps the caller's order inside a group)
  const int P = ctx->n_pat;
  std::vector<int64_t> cnt(P, 0), start(P, 0);
  for (int64_t e = 0; e < n_cells; ++e) cnt[pat[e]]++;
  for (int p = 1; p < P; ++p) start[p] = start[p - 1] + cnt[p - 1];
  std::vector<int64_t> order(n_cells), fillp(start);
  for (int64_t e = 0; e < n_cells; ++e) order[fillp[pat[e]]++] = e;
  std::vector<int64_t> conn_off(P, 0);
  int64_t co = 0;
  for (int p = 0; p < P; ++p) {
    conn_off[p] = co;
    co += cnt[p] * ctx->pat_nodes[p];
  }
  std::vector<int32_t> conn(std::max<int64_t>(co, 1));
  std::vector<uint8_t> ssym(n_cells);
  std::vector<double> scale(n_cells);
  std::vector<double> mass(ndof, 0.0);
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int max_m = 0;
  for (int p = 0; p < P; ++p) {
    const int np = ctx->pat_nodes[p];
    if (cnt[p]) max_m = std::max(max_m, 3 * np);
    for (int64_t j = 0; j < cnt[p]; ++j) {
      const int64_t s = start[p] + j, e = order[s];
      ssym[s] = sym[e];
      scale[s] = Ev[e] * hv[e];
      const double mscale = rv[e] * hv[e] * hv[e] * hv[e];
      const int op = sym[e];
      for (int k = 0; k < np; ++k) {
        const int32_t node = nodes[ptr[e] + k];
        conn[conn_off[p] + (int64_t)k * cnt[p] + j] = node;
        // master component r of this node is cell component perm[r]
        for (int r = 0; r < 3; ++r)
          mass[3 * (int64_t)node + perm[op >> 3][r]] += mscale * ctx->M_host[ctx->pat_moff[p] + 3 * k + r];
      }
    }
  }
  std::vector<double> minv(ndof);
  for (int64_t d = 0; d < ndof; ++d) {
    if (mass[d] < 0 || !isfinite(mass[d])) return fail(ctx, SBX_EINVAL, "negative or non-finite mass");
    // a node no cell touches has no mass and stays at rest until sbx_set_mass
    minv[d] = mass[d] > 0 ? 1.0 / mass[d] : 0.0;
  }
  for (int64_t i = 0; i < n_fixed; ++i) minv[fixed[i]] = 0.0;

  std::vector<Tile> tiles;
  for (int p = 0; p < P; ++p)
    for (int64_t c0 = 0; c0 < cnt[p]; c0 += sbx::SIMT_TILE)
      tiles.push_back(Tile{p, (int32_t)std::min<int64_t>(sbx::SIMT_TILE, cnt[p] - c0), c0});
  // FP64 force of the 8-node cells with the identity op in the Walsh basis
  // of the corner reflections: T[(s, r), (n, r)] = (-1)^popcount(n & (s ^
  // 2^r)) (n = corner a + 2 b + 4 c, r = component) has T T^T = 8 I and
  // T K_p T^T / 8 block-diagonal with 3 x 3 blocks (checked here; any
  // coupling between blocks beyond rounding keeps the dense path)
  int wht_pat = -1;
  sbx::WhtBlocks wht{};
  for (int p = 0; p < P && wht_pat < 0; ++p) {
    if (ctx->pat_nodes[p] != 8 || cnt[p] == 0) continue;
    bool ident = true;
    for (int64_t c = 0; c < cnt[p] && ident; ++c) ident = ssym[start[p] + c] == 0;
    if (!ident) continue;
    const double *Kp = &ctx->K_host[ctx->pat_koff[p]];
    auto Tm = [](int row, int col) -> double {   // row = 3 s + r, col = 3 n + r'
      const int s = row / 3, r = row % 3, n = col / 3, r2 = col % 3;
      if (r != r2) return 0.0;
      return (__builtin_popcount((unsigned)(n & (s ^ (1 << r)))) & 1) ? -1.0 : 1.0;
    };
    double Kh[24][24], kmax = 0.0, off = 0.0;
    for (int i = 0; i < 24; ++i)
      for (int j = 0; j < 24; ++j) {
        double acc = 0.0;
        for (int a = 0; a < 24; ++a) {
          const double ta = Tm(i, a);
          if (ta == 0.0) continue;
          for (int b = 0; b < 24; ++b) {
            const double tb = Tm(j, b);
            if (tb != 0.0) acc += ta * Kp[a * 24 + b] * tb;
          }
        }
        Kh[i][j] = acc / 8.0;
        kmax = std::max(kmax, std::fabs(Kh[i][j]));
        if (i / 3 != j / 3) off = std::max(off, std::fabs(Kh[i][j]));
      }
    if (!(off <= 1e-12 * kmax)) continue;
    for (int sb = 0; sb < 8; ++sb)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) wht.blk[9 * sb + 3 * r + c] = Kh[3 * sb + r][3 * sb + c];
    wht_pat = p;
  }
  std::vector<Tile> rest;
  for (const Tile &t : tiles)
    if (t.pat != wht_pat) rest.push_back(t);
  // heaviest first (m_p^2 per cell): the CTAs are issued in order, so long
  // ones start early and short ones fill the end
  std::stable_sort(rest.begin(), rest.end(), [&](const Tile &a, const Tile &b) {
    const int64_t na = ctx->pat_nodes[a.pat], nb = ctx->pat_nodes[b.pat];
    return na * na * a.ncell > nb * nb * b.ncell;
  });

  free_mesh(ctx);
  int rc = SBX_OK;
  if (!rc) rc = upload(ctx, &ctx->d_conn, conn);
  if (!rc) rc = upload(ctx, &ctx->d_conn_off, conn_off);
  if (!rc) rc = upload(ctx, &ctx->d_pat_cstart, start);
  if (!rc) rc = upload(ctx, &ctx->d_pat_ccount, cnt);
  if (!rc) rc = upload(ctx, &ctx->d_sym, ssym);
  if (!rc) rc = upload(ctx, &ctx->d_scale, scale);
  if (!rc) rc = upload(ctx, &ctx->d_minv, minv);
  if (!rc) rc = upload(ctx, &ctx->d_mass, mass);
  if (!rc) rc = upload(ctx, &ctx->d_tiles_simt, tiles);
  if (!rc && !rest.empty()) rc = upload(ctx, &ctx->d_tiles_rest, rest);
  const int64_t nfield = ndof * n_rhs;
  if (!rc) rc = dalloc(ctx, &ctx->d_u[0], nfield);
  if (!rc) rc = dalloc(ctx, &ctx->d_u[1], nfield);
  if (!rc) rc = dalloc(ctx, &ctx->d_f, nfield);
  if (!rc) rc = dalloc(ctx, &ctx->d_w, ndof);
  // (hi, lo) pairs and the FP64 copy of the FP32 force: 2 floats per DOF and case
  const bool pairs = (precision_mode == SBX_PREC_MIXED && n_rhs == 1) ||
                     (precision_mode == SBX_PREC_FP32 && n_rhs > 1);
  if (!rc && pairs) rc = dalloc(ctx, &ctx->d_fx, nfield);
  if (!rc && pairs) rc = dalloc(ctx, &ctx->d_pair, 2 * nfield);
  if (rc) {
    free_mesh(ctx);
    return rc;
  }
  ctx->prec = precision_mode;
  ctx->B = n_rhs;
  ctx->N = n_nodes;
  // default kernel of the hanging-node patterns: tensor cores for one load
  // case, FP32 SIMT for the batched form (measured faster there)
  ctx->hanging_tc = n_rhs == 1;
  ctx->h_order = order;
  ctx->h_hs.resize(n_cells);
  for (int64_t s = 0; s < n_cells; ++s) ctx->h_hs[s] = hv[order[s]];
  if (n_rhs > 1) {
    std::string e;
    ctx->hb_conn = conn;
    ctx->hb_conn_off = conn_off;
    ctx->hb_cnt = cnt;
    ctx->hb_start = start;
    ctx->hb_sym = ssym;
    ctx->hb_scale = scale;
    const int brc = sbx::batch_setup(ctx, conn, conn_off, cnt, ssym, scale, start, e);
    if (brc) {
      free_mesh(ctx);
      return fail(ctx, brc, e);
    }
  } else if (precision_mode == SBX_PREC_MIXED) {
    std::string e;
    const int trc = sbx::tc_setup(ctx, conn, conn_off, cnt, start, ssym, scale, e);
    if (trc) {
      free_mesh(ctx);
      return fail(ctx, trc, e);
    }
  }
  CK(cudaMemsetAsync(ctx->d_u[0], 0, nfield * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_u[1], 0, nfield * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_f, 0, nfield * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int32_t), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_step, 0, sizeof(int64_t), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->N = n_nodes;
  ctx->C = n_cells;
  ctx->ndof = ndof;
  ctx->h_fixed = fixed;
  ctx->f_pending = false;
  ctx->B = n_rhs;
  ctx->prec = precision_mode;
  ctx->pat_cstart = start;
  ctx->pat_ccount = cnt;
  ctx->n_tiles_simt = (int)tiles.size();
  ctx->n_tiles_rest = (int)rest.size();
  ctx->wht_pat = wht_pat;
  ctx->wht_cells = wht_pat >= 0 ? cnt[wht_pat] : 0;
  ctx->wht = wht;
  // mixed form: the Walsh-basis kernel for the regular cells by default
  // (faster and more accurate than the tensor-core one on these cells)
  ctx->mixed_wht = precision_mode == SBX_PREC_MIXED && n_rhs == 1 && wht_pat >= 0;
  ctx->max_m = max_m;
  ctx->cur = 0;
  ctx->step = 0;
  ctx->f_dirty = false;
  ctx->have_mesh = true;
  return SBX_OK;
}

int set_load(sbx_ctx *ctx, int n_src, const int64_t *node, const double *dir3, const int32_t *rhs,
             int wavelet, const double *t1, const double *P0, const double *ncyc) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "mesh_upload must come before set_load");
  if (n_src < 0) return fail(ctx, SBX_EINVAL, "n_src < 0");
  if (wavelet < SBX_WAVE_RICKER || wavelet > SBX_WAVE_SINE_BURST) return fail(ctx, SBX_EINVAL, "unknown wavelet");
  std::vector<int64_t> nd;
  std::vector<double> dv, tv, pv, cv;
  std::vector<int32_t> rv;
  if (int rc = fetch_vec(ctx, nd, node, n_src)) return rc;
  if (int rc = fetch_vec(ctx, dv, dir3, 3 * (size_t)n_src)) return rc;
  if (int rc = fetch_vec(ctx, tv, t1, n_src)) return rc;
  if (int rc = fetch_vec(ctx, pv, P0, n_src)) return rc;
  if (ncyc) {
    if (int rc = fetch_vec(ctx, cv, ncyc, n_src)) return rc;
  } else {
    cv.assign(n_src, 5.0);
  }
  if (rhs) {
    if (int rc = fetch_vec(ctx, rv, rhs, n_src)) return rc;
  } else {
    rv.assign(n_src, 0);
  }
  std::vector<int64_t> ldof;
  std::vector<double> lamp, lt1, lnc;
  std::vector<int32_t> lkind;
  for (int k = 0; k < n_src; ++k) {
    if (nd[k] < 0 || nd[k] >= ctx->N) return fail(ctx, SBX_EINVAL, "load node out of range");
    if (rv[k] < 0 || rv[k] >= ctx->B) return fail(ctx, SBX_EINVAL, "load rhs out of range");
    if (!(tv[k] > 0)) return fail(ctx, SBX_EINVAL, "t1 must be positive");
    for (int d = 0; d < 3; ++d) {
      if (dv[3 * k + d] == 0.0) continue;
      int64_t dof = 3 * nd[k] + d;
      if (ctx->B > 1) dof = dof * ctx->B + rv[k];
      ldof.push_back(dof);
      lamp.push_back(pv[k] * dv[3 * k + d]);
      lt1.push_back(tv[k]);
      lnc.push_back(cv[k]);
      lkind.push_back(wavelet);
    }
  }
  drop_graph(ctx);
  int rc = SBX_OK;
  if (!rc) rc = upload(ctx, &ctx->d_load_dof, ldof);
  if (!rc) rc = upload(ctx, &ctx->d_load_amp, lamp);
  if (!rc) rc = upload(ctx, &ctx->d_load_t1, lt1);
  if (!rc) rc = upload(ctx, &ctx->d_load_ncyc, lnc);
  if (!rc) rc = upload(ctx, &ctx->d_load_kind, lkind);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->n_load = (int)ldof.size();
  return SBX_OK;
}

int set_initial(sbx_ctx *ctx, const double *u0, const double *v0, double dt, double alpha) {
  if (!ctx) return SBX_EINVAL;
  if (ctx->state_owner) return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "mesh_upload must come before set_initial");
  if (!(dt > 0) || !(alpha >= 0)) return fail(ctx, SBX_EINVAL, "dt must be > 0 and alpha >= 0");
  const int64_t nd = ctx->ndof * ctx->B;
  const size_t bytes = nd * sizeof(double);
  ctx->cur = 0;
  ctx->pair_of = -1;
  double *U0 = ctx->d_u[0], *Um1 = ctx->d_u[1];
  if (u0) {
    CK(cudaMemcpyAsync(U0, u0, bytes, cudaMemcpyDefault, ctx->stream));
  } else {
    CK(cudaMemsetAsync(U0, 0, bytes, ctx->stream));
  }
  CK(sbx::launch_zero_fixed(ctx, U0, ctx->stream));
  double *V0 = nullptr;
  if (v0) {
    // staged through the (not yet used) force buffer's partner: U_-1 slot
    CK(cudaMemcpyAsync(Um1, v0, bytes, cudaMemcpyDefault, ctx->stream));
    CK(sbx::launch_zero_fixed(ctx, Um1, ctx->stream));
    V0 = Um1;
  }
  CK(cudaMemsetAsync(ctx->d_step, 0, sizeof(int64_t), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_f, 0, bytes, ctx->stream));
  if (int rc = force(ctx, U0, ctx->d_f, dt)) return rc;
  const double *F0 = ctx->d_f;
  if (ctx->uses_pairs()) {
    CK(sbx::launch_widen_f32(ctx, reinterpret_cast<const float *>(ctx->d_f), ctx->d_fx,
                             ctx->stream));
    F0 = ctx->d_fx;
  }
  // k_init_um1 reads v0[i] before writing um1[i] of the same index
  CK(sbx::launch_init_um1(ctx, U0, V0, Um1, F0, dt, alpha, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_f, 0, bytes, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int32_t), ctx->stream));
  ctx->step = 0;
  ctx->f_dirty = ctx->f_pending = false;
  return SBX_OK;
}

int step_n(sbx_ctx *ctx, int64_t n_steps, double dt, double alpha) {
  if (!ctx) return SBX_EINVAL;
  if (ctx->state_owner) return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "mesh_upload must come before step_n");
  if (n_steps < 0 || !(dt > 0) || !(alpha >= 0) || !isfinite(dt) || !isfinite(alpha))
    return fail(ctx, SBX_EINVAL, "need n_steps >= 0, dt > 0, alpha >= 0");
  if (n_steps == 0) return SBX_OK;
  const size_t bytes = ctx->ndof * ctx->B * sizeof(double);
  if (ctx->f_dirty || ctx->f_pending) {
    CK(cudaMemsetAsync(ctx->d_f, 0, bytes, ctx->stream));
    ctx->f_dirty = ctx->f_pending = false;
  }
  CK(sbx::prepare_update(ctx, dt, alpha, ctx->stream));
  if (int rc = ensure_pairs(ctx)) return rc;
  int64_t left = n_steps - 1;  // the last step keeps R_int for read-back
  if (!ctx->graph.valid || ctx->graph.dt != dt || ctx->graph.alpha != alpha)
    if (int rc = build_graphs(ctx, dt, alpha)) return rc;
  {
    while (left >= GRAPH_UNIT) {
      CK(cudaGraphLaunch(ctx->graph.exec[ctx->cur], ctx->stream));
      left -= GRAPH_UNIT;
    }
  }
  // the remaining left steps and the closing one, as one graph
  if (int rc = build_tail(ctx, (int)left, dt, alpha)) return rc;
  if (int rc = ensure_pairs(ctx)) return rc;
  CK(cudaGraphLaunch(ctx->graph.tail[(int)left][ctx->cur], ctx->stream));
  ctx->cur ^= (int)((left + 1) & 1);
  // the last update wrote the pairs of the new U_n
  if (ctx->uses_pairs()) ctx->pair_of = ctx->cur;
  ctx->f_dirty = true;
  ctx->step += n_steps;
  return SBX_OK;
}

int sbx_prepare_steps(sbx_ctx *ctx, int64_t n_steps, double dt, double alpha) {
  if (!ctx) return SBX_EINVAL;
  if (ctx->state_owner) return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "mesh_upload must come before sbx_prepare_steps");
  if (n_steps < 0 || !(dt > 0) || !(alpha >= 0) || !isfinite(dt) || !isfinite(alpha))
    return fail(ctx, SBX_EINVAL, "need n_steps >= 0, dt > 0, alpha >= 0");
  if (n_steps == 0) return SBX_OK;
  CK(sbx::prepare_update(ctx, dt, alpha, ctx->stream));
  return build_tail(ctx, (int)((n_steps - 1) % GRAPH_UNIT), dt, alpha);
}

int sbx_profile(sbx_ctx *ctx, int64_t n_steps, double dt, double alpha, double *ms_force,
                double *ms_update) {
  if (!ctx || !ms_force || !ms_update) return SBX_EINVAL;
  if (ctx->state_owner) return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "mesh_upload must come before sbx_profile");
  if (n_steps < 1 || !(dt > 0) || !(alpha >= 0)) return fail(ctx, SBX_EINVAL, "bad arguments");
  const size_t bytes = ctx->ndof * ctx->B * sizeof(double);
  if (ctx->f_dirty) {
    CK(cudaMemsetAsync(ctx->d_f, 0, bytes, ctx->stream));
    ctx->f_dirty = false;
  }
  CK(sbx::prepare_update(ctx, dt, alpha, ctx->stream));
  if (int rc = ensure_pairs(ctx)) return rc;
  std::vector<cudaEvent_t> ev(3 * n_steps, nullptr);
  int rc = SBX_OK;
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = SBX_ECUDA;
  for (int64_t s = 0; s < n_steps && rc == SBX_OK; ++s) {
    double *uc = ctx->d_u[ctx->cur], *up = ctx->d_u[ctx->cur ^ 1];
    cudaEventRecord(ev[3 * s], ctx->stream);
    rc = force(ctx, uc, ctx->d_f, dt);
    cudaEventRecord(ev[3 * s + 1], ctx->stream);
    if (rc == SBX_OK) rc = update(ctx, uc, up, dt, alpha, s + 1 < n_steps);
    cudaEventRecord(ev[3 * s + 2], ctx->stream);
    ctx->cur ^= 1;
    ctx->step += 1;
  }
  ctx->f_dirty = true;
  double tf = 0, tu = 0;
  if (rc == SBX_OK && cudaStreamSynchronize(ctx->stream) == cudaSuccess) {
    for (int64_t s = 0; s < n_steps; ++s) {
      float a = 0, b = 0;
      cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
      cudaEventElapsedTime(&b, ev[3 * s + 1], ev[3 * s + 2]);
      tf += a;
      tu += b;
    }
  } else if (rc == SBX_OK) {
    rc = fail(ctx, SBX_ECUDA, "stream synchronisation failed");
  }
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  *ms_force = tf;
  *ms_update = tu;
  if (rc) return rc;
  return check_flags(ctx);
}

int set_modulus(sbx_ctx *ctx, const double *E) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  if (ctx->B != 1 || ctx->prec == SBX_PREC_MIXED)
    return fail(ctx, SBX_EINVAL, "set_modulus needs a single-load-case FP64 or FP32 mesh");
  std::vector<double> Ev;
  if (int rc = fetch_vec(ctx, Ev, E, ctx->C)) return rc;
  std::vector<double> scale(ctx->C);
  for (int64_t s = 0; s < ctx->C; ++s) {
    const double e = Ev[ctx->h_order[s]];
    if (!(e > 0) || !isfinite(e)) return fail(ctx, SBX_EINVAL, "E must be positive and finite");
    scale[s] = e * ctx->h_hs[s];
  }
  CK(cudaMemcpyAsync(ctx->d_scale, scale.data(), scale.size() * sizeof(double),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SBX_OK;
}

int sbx_adjoint(sbx_ctx *ctx, int64_t n_steps, double dt, int64_t n_rec, const int64_t *rec_dof,
                const double *data, int64_t ckpt_every, double *misfit_out, double *grad_E_out) {
  if (!ctx) return SBX_EINVAL;
  if (ctx->state_owner) return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  if (ctx->step != 0) return fail(ctx, SBX_ESTATE, "sbx_adjoint starts from set_initial (step 0)");
  if (ctx->B != 1 || ctx->prec == SBX_PREC_MIXED)
    return fail(ctx, SBX_EINVAL, "sbx_adjoint needs a single-load-case FP64 or FP32 mesh");
  if (n_steps < 1 || !(dt > 0) || n_rec < 0 || ckpt_every < 1 || !misfit_out || !grad_E_out ||
      (n_rec > 0 && (!rec_dof || !data)))
    return fail(ctx, SBX_EINVAL, "bad adjoint arguments");
  const int64_t nd = ctx->ndof, N = n_steps, k = std::min(ckpt_every, n_steps);
  std::vector<int64_t> rec;
  std::vector<double> dat;
  if (int rc = fetch_vec(ctx, rec, rec_dof, n_rec)) return rc;
  for (int64_t r : rec)
    if (r < 0 || r >= nd) return fail(ctx, SBX_EINVAL, "receiver DOF out of range");
  if (int rc = fetch_vec(ctx, dat, data, (size_t)(N * n_rec))) return rc;
  const int64_t nseg = (N + k - 1) / k;
  int64_t *d_rec = nullptr;
  double *d_dat = nullptr, *d_ck = nullptr, *d_seg = nullptr, *d_lam = nullptr, *d_v = nullptr,
         *d_acc = nullptr, *d_J = nullptr;
  auto release = [&]() {
    dfree(d_rec); dfree(d_dat); dfree(d_ck); dfree(d_seg); dfree(d_lam); dfree(d_v);
    dfree(d_acc); dfree(d_J);
  };
  int rc = SBX_OK;
  if (!rc) rc = upload(ctx, &d_rec, rec);
  if (!rc) rc = upload(ctx, &d_dat, dat);
  if (!rc) rc = dalloc(ctx, &d_ck, (size_t)(nseg * 2 * nd));
  if (!rc) rc = dalloc(ctx, &d_seg, (size_t)((k + 1) * nd));
  if (!rc) rc = dalloc(ctx, &d_lam, (size_t)(2 * nd));
  if (!rc) rc = dalloc(ctx, &d_v, (size_t)nd);
  if (!rc) rc = dalloc(ctx, &d_acc, (size_t)ctx->C);
  if (!rc) rc = dalloc(ctx, &d_J, 1);
  if (rc) {
    release();
    return rc;
  }
  const size_t vb = nd * sizeof(double);
  cudaStream_t s = ctx->stream;
  auto go = [&]() -> int {
    CK(sbx::prepare_update(ctx, dt, 0.0, s));
    if (ctx->f_dirty) {
      CK(cudaMemsetAsync(ctx->d_f, 0, vb, s));
      ctx->f_dirty = false;
    }
    // forward with checkpoints (U_{sk}, U_{sk-1})
    for (int64_t g = 0; g < nseg; ++g) {
      CK(cudaMemcpyAsync(d_ck + (2 * g) * nd, ctx->d_u[ctx->cur], vb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(d_ck + (2 * g + 1) * nd, ctx->d_u[ctx->cur ^ 1], vb,
                         cudaMemcpyDeviceToDevice, s));
      const int64_t len = std::min(k, N - g * k);
      for (int64_t j = 0; j < len; ++j) {
        if (int r = one_step(ctx, ctx->cur, dt, 0.0, 1)) return r;
        ctx->cur ^= 1;
      }
    }
    CK(cudaMemsetAsync(d_lam, 0, 2 * vb, s));
    CK(cudaMemsetAsync(d_acc, 0, ctx->C * sizeof(double), s));
    CK(cudaMemsetAsync(d_J, 0, sizeof(double), s));
    double *lam1 = d_lam, *lam2 = d_lam + nd;   // lambda_{n+1}, lambda_{n+2}
    for (int64_t g = nseg - 1; g >= 0; --g) {
      // recompute U_{gk} .. U_{gk+len} into the segment buffer
      CK(cudaMemcpyAsync(ctx->d_u[0], d_ck + (2 * g) * nd, vb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(ctx->d_u[1], d_ck + (2 * g + 1) * nd, vb, cudaMemcpyDeviceToDevice, s));
      ctx->cur = 0;
      const int64_t n0 = g * k;
      CK(cudaMemcpyAsync(ctx->d_step, &n0, sizeof(int64_t), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(d_seg, ctx->d_u[0], vb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemsetAsync(ctx->d_f, 0, vb, s));   // holds K W lambda from the reverse sweep
      const int64_t len = std::min(k, N - n0);
      for (int64_t j = 1; j <= len; ++j) {
        if (int r = one_step(ctx, ctx->cur, dt, 0.0, 1)) return r;
        ctx->cur ^= 1;
        CK(cudaMemcpyAsync(d_seg + j * nd, ctx->d_u[ctx->cur], vb, cudaMemcpyDeviceToDevice, s));
      }
      for (int64_t n = n0 + len; n >= n0 + 1; --n) {
        // lambda_n = g_n + 2 lambda_{n+1} - K (W lambda_{n+1}) - lambda_{n+2}  (into lam2)
        CK(sbx::launch_weight(ctx, lam1, d_v, s));
        CK(cudaMemsetAsync(ctx->d_f, 0, vb, s));
        CK(sbx::launch_force_simt(ctx, d_v, ctx->d_f, dt, s, false));
        CK(sbx::launch_adj_update(ctx, ctx->d_f, lam1, lam2, s));
        CK(sbx::launch_residual(ctx, n_rec, d_rec, d_seg + (n - n0) * nd, d_dat + (n - 1) * n_rec,
                                lam2, d_J, s));
        // dJ/dE pair (lambda_n, U_{n-1})
        CK(sbx::launch_weight(ctx, lam2, d_v, s));
        CK(sbx::launch_grad(ctx, d_seg + (n - 1 - n0) * nd, d_v, d_acc, s));
        std::swap(lam1, lam2);   // lambda_{n+1} <- lambda_n, lambda_{n+2} <- old lambda_{n+1}
      }
    }
    // back to the starting state
    CK(cudaMemcpyAsync(ctx->d_u[0], d_ck, vb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_u[1], d_ck + nd, vb, cudaMemcpyDeviceToDevice, s));
    ctx->cur = 0;
    const int64_t zero = 0;
    CK(cudaMemcpyAsync(ctx->d_step, &zero, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_f, 0, vb, s));
    std::vector<double> acc(ctx->C);
    double J = 0.0;
    CK(cudaMemcpyAsync(acc.data(), d_acc, ctx->C * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&J, d_J, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> grad(ctx->C);
    for (int64_t q = 0; q < ctx->C; ++q) grad[ctx->h_order[q]] = -ctx->h_hs[q] * acc[q];
    if (is_device_ptr(grad_E_out)) {
      CK(cudaMemcpy(grad_E_out, grad.data(), ctx->C * sizeof(double), cudaMemcpyHostToDevice));
    } else {
      memcpy(grad_E_out, grad.data(), ctx->C * sizeof(double));
    }
    *misfit_out = J;
    return check_flags(ctx);
  };
  rc = go();
  ctx->step = 0;
  release();
  return rc;
}

int sbx_force(sbx_ctx *ctx, double dt) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "mesh_upload must come before sbx_force");
  if (sbx_ctx *o = ctx->state_owner) {
    // add this context's cells into the owner's accumulator, from the
    // owner's current U_n (the owner clears the accumulator in its update)
    if (!(dt > 0) || !isfinite(dt)) return fail(ctx, SBX_EINVAL, "dt must be > 0");
    if (o->f_dirty) return fail(ctx, SBX_ESTATE, "the owner's force buffer holds a finished step");
    ctx->cur = o->cur;
    ctx->pair_of = o->pair_of;
    ctx->step = o->step;
    if (int rc = ensure_pairs(ctx)) return rc;
    o->pair_of = ctx->pair_of;
    if (int rc = force(ctx, ctx->d_u[ctx->cur], ctx->d_f, dt)) return rc;
    return SBX_OK;
  }
  if (ctx->f_pending) return fail(ctx, SBX_ESTATE, "sbx_force twice without sbx_update");
  if (!(dt > 0) || !isfinite(dt)) return fail(ctx, SBX_EINVAL, "dt must be > 0");
  if (ctx->f_dirty) {
    CK(cudaMemsetAsync(ctx->d_f, 0, ctx->ndof * ctx->B * sizeof(double), ctx->stream));
    ctx->f_dirty = false;
  }
  if (int rc = ensure_pairs(ctx)) return rc;
  if (int rc = force(ctx, ctx->d_u[ctx->cur], ctx->d_f, dt)) return rc;
  ctx->f_pending = true;
  return SBX_OK;
}

int sbx_update(sbx_ctx *ctx, double dt, double alpha) {
  if (!ctx) return SBX_EINVAL;
  if (ctx->state_owner) return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "mesh_upload must come before sbx_update");
  if (!ctx->f_pending) return fail(ctx, SBX_ESTATE, "sbx_update needs a preceding sbx_force");
  if (!(dt > 0) || !(alpha >= 0) || !isfinite(dt) || !isfinite(alpha))
    return fail(ctx, SBX_EINVAL, "need dt > 0, alpha >= 0");
  CK(sbx::prepare_update(ctx, dt, alpha, ctx->stream));
  if (int rc = update(ctx, ctx->d_u[ctx->cur], ctx->d_u[ctx->cur ^ 1], dt, alpha, 1)) return rc;
  ctx->cur ^= 1;
  ctx->step += 1;
  ctx->f_pending = false;
  return SBX_OK;
}

int sbx_field_ptr(sbx_ctx *ctx, int which, void **ptr, int64_t *len, int *layout) {
  if (!ctx || !ptr || !len || !layout) return SBX_EINVAL;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  *layout = SBX_LAYOUT_F64_DOF;
  *len = ctx->ndof * ctx->B;
  switch (which) {
    case SBX_U_N: *ptr = ctx->d_u[ctx->cur]; break;
    case SBX_U_NM1: *ptr = ctx->d_u[ctx->cur ^ 1]; break;
    case SBX_F_INT:
      *ptr = ctx->d_f;
      if (ctx->prec == SBX_PREC_MIXED && ctx->B == 1) {
        *layout = SBX_LAYOUT_F32_NODE4;
        *len = 4 * ctx->N;
      } else if (ctx->uses_pairs()) {
        *layout = SBX_LAYOUT_F32_DOF;
      }
      break;
    case SBX_MASS: *ptr = ctx->d_mass; *len = ctx->ndof; break;
    default: return fail(ctx, SBX_EINVAL, "unknown field");
  }
  return SBX_OK;
}

int sbx_wait_selftest(sbx_ctx *ctx, int64_t polls, int arrive) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (polls < 1 || polls > (int64_t)1 << 30) return fail(ctx, SBX_EINVAL, "polls out of range");
  int32_t before = 0;
  CK(cudaMemcpyAsync(&before, ctx->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(sbx::launch_wait_selftest(ctx, (uint32_t)polls, arrive, ctx->stream));
  int32_t after = 0;
  CK(cudaMemcpyAsync(&after, ctx->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // leave the flags as they were
  CK(cudaMemcpyAsync(ctx->d_flags, &before, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if ((after & 2) && !(before & 2)) return fail(ctx, SBX_ETIMEOUT, "the bounded wait gave up");
  return SBX_OK;
}

int sbx_touch(sbx_ctx *ctx) {
  if (!ctx) return SBX_EINVAL;
  ctx->pair_of = -1;
  return SBX_OK;
}

int sbx_lanczos(sbx_ctx *ctx, int64_t k, const double *v0, double *alpha, double *beta) {
  if (!ctx) return SBX_EINVAL;
  if (ctx->state_owner) return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  if (k < 1 || k > 4096 || !v0 || !alpha || !beta)
    return fail(ctx, SBX_EINVAL, "need 1 <= k <= 4096 and non-NULL v0, alpha, beta");
  if (ctx->B != 1 || ctx->prec == SBX_PREC_FP32)
    return fail(ctx, SBX_EINVAL, "sbx_lanczos needs a single-load-case FP64 or mixed mesh");
  std::vector<double> hv0;
  if (int rc = fetch_vec(ctx, hv0, v0, ctx->ndof)) return rc;
  double s2 = 0.0;
  {
    std::vector<char> fixed(ctx->ndof, 0);
    for (int64_t d : ctx->h_fixed) fixed[d] = 1;
    for (int64_t d = 0; d < ctx->ndof; ++d)
      if (!fixed[d]) s2 += hv0[d] * hv0[d];
  }
  if (!(s2 > 0) || !std::isfinite(s2)) return fail(ctx, SBX_EINVAL, "v0 vanishes on the free DOFs");
  double *dv0 = nullptr, *dab = nullptr;
  if (upload(ctx, &dv0, hv0) || dalloc(ctx, &dab, 2 * k)) {
    dfree(dv0);
    return fail(ctx, SBX_ENOMEM, "Lanczos buffers");
  }
  CK(cudaMemsetAsync(dab, 0, 2 * k * sizeof(double), ctx->stream));
  std::string e;
  int rc = sbx::lanczos_run(ctx, k, dv0, dab, dab + k, e);
  if (rc == SBX_OK &&
      (cudaMemcpy(alpha, dab, k * sizeof(double), cudaMemcpyDefault) != cudaSuccess ||
       cudaMemcpy(beta, dab + k, k * sizeof(double), cudaMemcpyDefault) != cudaSuccess)) {
    rc = SBX_ECUDA;
    e = "copy of the Lanczos coefficients failed";
  }
  dfree(dv0);
  dfree(dab);
  return rc ? fail(ctx, rc, e) : SBX_OK;
}

int sbx_set_mixed_kernel(sbx_ctx *ctx, int kind) {
  if (!ctx) return SBX_EINVAL;
  if (kind != SBX_MIXED_TENSOR && kind != SBX_MIXED_WALSH)
    return fail(ctx, SBX_EINVAL, "unknown mixed kernel");
  if (ctx->have_mesh && (ctx->prec != SBX_PREC_MIXED || ctx->B != 1))
    return fail(ctx, SBX_EINVAL, "sbx_set_mixed_kernel applies to the mixed form with one load case");
  if (kind == SBX_MIXED_WALSH && ctx->wht_pat < 0)
    return fail(ctx, SBX_EINVAL, "no Walsh blocks for this mesh");
  const bool w = kind == SBX_MIXED_WALSH;
  if (ctx->mixed_wht != w) drop_graph(ctx);
  ctx->mixed_wht = w;
  return SBX_OK;
}

int sbx_halo_plan(sbx_ctx *ctx, int64_t n_send, const int64_t *send_nodes, int64_t n_cut,
                  const int64_t *cut_nodes, const int64_t *contrib_ptr,
                  const int64_t *contrib_src) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "mesh_upload must come before sbx_halo_plan");
  if (ctx->B != 1) return fail(ctx, SBX_EINVAL, "the interface sum is for one load case");
  if (n_send < 0 || n_cut < 0 || (n_send > 0 && !send_nodes) ||
      (n_cut > 0 && (!cut_nodes || !contrib_ptr)))
    return fail(ctx, SBX_EINVAL, "bad halo plan sizes or null arrays");
  std::vector<int64_t> snd, cut, ptr, src;
  if (int rc = fetch_vec(ctx, snd, send_nodes, (size_t)n_send)) return rc;
  if (int rc = fetch_vec(ctx, cut, cut_nodes, (size_t)n_cut)) return rc;
  if (n_cut > 0) {
    if (int rc = fetch_vec(ctx, ptr, contrib_ptr, (size_t)n_cut + 1)) return rc;
  } else {
    ptr.assign(1, 0);
  }
  if (ptr[0] != 0) return fail(ctx, SBX_EINVAL, "contrib_ptr must start at 0");
  for (int64_t j = 0; j < n_cut; ++j)
    if (ptr[j + 1] < ptr[j]) return fail(ctx, SBX_EINVAL, "contrib_ptr must not decrease");
  if (ptr[n_cut] > 0 && !contrib_src) return fail(ctx, SBX_EINVAL, "null contrib_src");
  if (int rc = fetch_vec(ctx, src, contrib_src, (size_t)ptr[n_cut])) return rc;
  for (int64_t v : snd)
    if (v < 0 || v >= ctx->N) return fail(ctx, SBX_EINVAL, "send node out of range");
  for (int64_t v : cut)
    if (v < 0 || v >= ctx->N) return fail(ctx, SBX_EINVAL, "cut node out of range");
  for (int64_t q : src)
    if (q < -1 || q >= n_send) return fail(ctx, SBX_EINVAL, "contribution row out of range");
  if (int rc = upload(ctx, &ctx->d_halo_send, snd)) return rc;
  if (int rc = upload(ctx, &ctx->d_halo_cut, cut)) return rc;
  if (int rc = upload(ctx, &ctx->d_halo_ptr, ptr)) return rc;
  if (int rc = upload(ctx, &ctx->d_halo_src, src)) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->halo_n_send = n_send;
  ctx->halo_n_cut = n_cut;
  return SBX_OK;
}

int sbx_halo_pack(sbx_ctx *ctx, void *send_buf) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  if (ctx->halo_n_send > 0 && !is_device_ptr(send_buf))
    return fail(ctx, SBX_EINVAL, "send_buf must be device memory");
  CK(sbx::launch_halo_pack(ctx, send_buf, ctx->stream));
  return SBX_OK;
}

int sbx_halo_sum(sbx_ctx *ctx, const void *recv_buf) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  if (ctx->halo_n_send > 0 && !is_device_ptr(recv_buf))
    return fail(ctx, SBX_EINVAL, "recv_buf must be device memory");
  CK(sbx::launch_halo_sum(ctx, recv_buf, ctx->stream));
  return SBX_OK;
}

int sbx_share_state(sbx_ctx *ctx, sbx_ctx *owner) {
  if (!ctx || !owner || ctx == owner) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh || !owner->have_mesh)
    return fail(ctx, SBX_ESTATE, "both contexts need a mesh");
  if (owner->state_owner) return fail(ctx, SBX_EINVAL, "the owner shares another context's state");
  if (ctx->state_owner || ctx->n_guests) return fail(ctx, SBX_ESTATE, "state already shared");
  if (ctx->device != owner->device || ctx->stream != owner->stream)
    return fail(ctx, SBX_EINVAL, "both contexts must use one device and one stream");
  if (ctx->N != owner->N || ctx->B != owner->B || ctx->prec != owner->prec)
    return fail(ctx, SBX_EINVAL, "node count, load cases and precision must match");
  CK(cudaStreamSynchronize(ctx->stream));
  drop_graph(ctx);
  dfree(ctx->d_u[0]); dfree(ctx->d_u[1]); dfree(ctx->d_f); dfree(ctx->d_pair);
  ctx->d_u[0] = owner->d_u[0];
  ctx->d_u[1] = owner->d_u[1];
  ctx->d_f = owner->d_f;
  ctx->d_pair = owner->d_pair;
  ctx->state_owner = owner;
  owner->n_guests += 1;
  ctx->f_dirty = ctx->f_pending = false;
  return SBX_OK;
}

int sbx_classify_cells(sbx_ctx *ctx, int64_t n_cells, const int32_t *slot_node,
                       const int32_t *mask, int32_t *masters, int32_t *n_masters,
                       int32_t *cell_pattern, uint8_t *cell_sym, int64_t *cell_ptr,
                       int32_t *cell_nodes, int64_t *order, int64_t *pat_start, int32_t *conn) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (n_cells < 1 || n_cells > ((int64_t)1 << 40))
    return fail(ctx, SBX_EINVAL, "n_cells out of range");
  if (!masters || !n_masters || !pat_start) return fail(ctx, SBX_EINVAL, "null host output");
  const void *dev[] = {slot_node, mask, cell_pattern, cell_sym, cell_ptr, cell_nodes, order, conn};
  for (const void *p : dev)
    if (!is_device_ptr(p)) return fail(ctx, SBX_EINVAL, "per-cell arrays must be device memory");
  cudaStream_t s = ctx->stream;
  const int grid = ctx->n_sm * 8;
  const int64_t nb = (n_cells + 1023) / 1024;
  int32_t *table = nullptr, *used = nullptr, *pid = nullptr, *bad = nullptr;
  int64_t *work = nullptr, *total = nullptr, *cnt = nullptr, *dstart = nullptr, *dcoff = nullptr;
  auto release = [&]() {
    dfree(table); dfree(used); dfree(pid); dfree(bad); dfree(work); dfree(total); dfree(cnt);
    dfree(dstart); dfree(dcoff);
  };
  int rc = SBX_OK;
  if (!rc) rc = dalloc(ctx, &table, 4096);
  if (!rc) rc = dalloc(ctx, &used, 4096);
  if (!rc) rc = dalloc(ctx, &pid, 4096);
  if (!rc) rc = dalloc(ctx, &bad, 1);
  if (!rc) rc = dalloc(ctx, &work, (size_t)std::max<int64_t>(nb, 1) * 145 + 2);
  if (!rc) rc = dalloc(ctx, &total, 1);
  if (rc) {
    release();
    return rc;
  }
  auto go = [&]() -> int {
    CK(cudaMemsetAsync(used, 0, 4096 * sizeof(int32_t), s));
    CK(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
    CK(sbx::setup_mask_table(table, s));
    CK(sbx::setup_flag_masters(n_cells, mask, table, used, grid, s));
    std::vector<int32_t> hu(4096), hp(4096, -1);
    CK(cudaMemcpyAsync(hu.data(), used, 4096 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int P = 0;
    for (int q = 0; q < 4096; ++q)
      if (hu[q]) {
        masters[P] = q;
        hp[q] = P++;
      }
    if (P > 144) return fail(ctx, SBX_EINVAL, "more than 144 master patterns");
    *n_masters = P;
    CK(cudaMemcpyAsync(pid, hp.data(), 4096 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(cell_ptr + n_cells, 0, sizeof(int64_t), s));
    CK(sbx::setup_classify(n_cells, mask, table, pid, cell_pattern, cell_sym, cell_ptr, grid, s));
    CK(sbx::setup_scan(n_cells + 1, cell_ptr, work, total, s));
    CK(sbx::setup_cell_nodes(n_cells, slot_node, mask, table, cell_ptr, cell_nodes, bad, grid, s));
    // stable sort by pattern: counts per (pattern, block), scanned pattern-major
    if (int r = dalloc(ctx, &cnt, (size_t)P * nb + 1)) return r;
    CK(sbx::setup_sort_count(n_cells, P, cell_pattern, cnt, s));
    CK(sbx::setup_scan((int64_t)P * nb, cnt, work, total, s));
    CK(sbx::setup_sort_scatter(n_cells, P, cell_pattern, cnt, order, s));
    std::vector<int64_t> st(P + 1);
    for (int p = 0; p < P; ++p)
      CK(cudaMemcpyAsync(&st[p], cnt + (int64_t)p * nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    int32_t nbad = 0;
    CK(cudaMemcpyAsync(&nbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nbad) return fail(ctx, SBX_EINVAL, "a cell lacks a node its pattern needs");
    st[P] = n_cells;
    std::vector<int64_t> coff(P + 1, 0);
    for (int p = 0; p <= P; ++p) pat_start[p] = st[p];
    // node counts per pattern from the scanned pointers: n_p = ptr[e + 1] - ptr[e]
    // of any cell e of the pattern (the first sorted one)
    for (int p = 0; p < P; ++p) {
      const int64_t Cp = st[p + 1] - st[p];
      int64_t e = 0, a = 0, b = 0;
      CK(cudaMemcpyAsync(&e, order + st[p], sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      CK(cudaMemcpyAsync(&a, cell_ptr + e, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&b, cell_ptr + e + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      coff[p + 1] = coff[p] + (b - a) * Cp;
    }
    if (int r = upload(ctx, &dstart, st)) return r;
    if (int r = upload(ctx, &dcoff, coff)) return r;
    CK(sbx::setup_conn(n_cells, order, cell_pattern, dstart, dcoff, cell_ptr, cell_nodes, conn,
                       grid, s));
    CK(cudaStreamSynchronize(s));
    return SBX_OK;
  };
  rc = go();
  release();
  return rc;
}

int sbx_set_launch(sbx_ctx *ctx, int what, int value) {
  if (!ctx) return SBX_EINVAL;
  ctx->err.clear();
  switch (what) {
    case SBX_LAUNCH_HANGING_KERNEL:
      if (value != SBX_HANGING_SIMT && value != SBX_HANGING_TENSOR)
        return fail(ctx, SBX_EINVAL, "unknown kernel for the hanging-node patterns");
      if (ctx->hanging_tc != (value == SBX_HANGING_TENSOR)) drop_graph(ctx);
      ctx->hanging_tc = value == SBX_HANGING_TENSOR;
      return SBX_OK;
    case SBX_LAUNCH_WALSH_CTAS_PER_SM:
      if (value < 0 || value > 8) return fail(ctx, SBX_EINVAL, "Walsh-kernel CTAs per SM: 0 .. 8");
      if (ctx->walsh_ctas != value) drop_graph(ctx);
      ctx->walsh_ctas = value;
      return SBX_OK;
    case SBX_LAUNCH_HANGING_CTAS_PER_SM:
      if (value < 1 || value > 2) return fail(ctx, SBX_EINVAL, "hanging-kernel CTAs per SM: 1 .. 2");
      if (ctx->hanging_ctas != value) drop_graph(ctx);
      ctx->hanging_ctas = value;
      return SBX_OK;
    case SBX_LAUNCH_UPDATE_KERNEL:
      if (value != SBX_UPDATE_THREAD && value != SBX_UPDATE_BULK)
        return fail(ctx, SBX_EINVAL, "unknown update kernel");
      if (ctx->update_bulk != (value == SBX_UPDATE_BULK)) drop_graph(ctx);
      ctx->update_bulk = value == SBX_UPDATE_BULK;
      return SBX_OK;
    default:
      break;
  }
  const bool cells = what >= SBX_LAUNCH_BATCH_TILE_CELLS && what < SBX_LAUNCH_BATCH_TILE_CELLS + 3;
  const bool kb = what >= SBX_LAUNCH_BATCH_SMEM_KB && what < SBX_LAUNCH_BATCH_SMEM_KB + 3;
  if (!cells && !kb) return fail(ctx, SBX_EINVAL, "unknown launch parameter");
  if (cells && (value < 1 || value > 64)) return fail(ctx, SBX_EINVAL, "cells per tile: 1 .. 64");
  if (kb && (value < 16 || value > 227)) return fail(ctx, SBX_EINVAL, "shared memory: 16 .. 227 KB");
  const int c = what - (cells ? SBX_LAUNCH_BATCH_TILE_CELLS : SBX_LAUNCH_BATCH_SMEM_KB);
  int &slot = cells ? ctx->b_tile_cells[c] : ctx->b_smem_kb[c];
  if (slot == value) return SBX_OK;
  const int old = slot;
  slot = value;
  if (!ctx->have_mesh || ctx->B == 1) return SBX_OK;
  // rebuild the batched tiles with the new shape
  if (int rc = set_device(ctx)) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  drop_graph(ctx);
  std::string e;
  const int rc = sbx::batch_setup(ctx, ctx->hb_conn, ctx->hb_conn_off, ctx->hb_cnt, ctx->hb_sym,
                                  ctx->hb_scale, ctx->hb_start, e);
  if (rc) {
    slot = old;
    std::string e2;
    sbx::batch_setup(ctx, ctx->hb_conn, ctx->hb_conn_off, ctx->hb_cnt, ctx->hb_sym, ctx->hb_scale,
                     ctx->hb_start, e2);
    return fail(ctx, rc, e);
  }
  return SBX_OK;
}

int sbx_get_launch(sbx_ctx *ctx, int what, int *value) {
  if (!ctx || !value) return SBX_EINVAL;
  switch (what) {
    case SBX_LAUNCH_HANGING_KERNEL:
      *value = ctx->hanging_tc ? SBX_HANGING_TENSOR : SBX_HANGING_SIMT;
      return SBX_OK;
    case SBX_LAUNCH_WALSH_CTAS_PER_SM:
      *value = ctx->walsh_ctas;
      return SBX_OK;
    case SBX_LAUNCH_HANGING_CTAS_PER_SM:
      *value = ctx->hanging_ctas;
      return SBX_OK;
    case SBX_LAUNCH_UPDATE_KERNEL:
      *value = ctx->update_bulk ? SBX_UPDATE_BULK : SBX_UPDATE_THREAD;
      return SBX_OK;
    default:
      break;
  }
  if (what >= SBX_LAUNCH_BATCH_TILE_CELLS && what < SBX_LAUNCH_BATCH_TILE_CELLS + 3) {
    *value = ctx->b_tile_cells[what - SBX_LAUNCH_BATCH_TILE_CELLS];
    return SBX_OK;
  }
  if (what >= SBX_LAUNCH_BATCH_SMEM_KB && what < SBX_LAUNCH_BATCH_SMEM_KB + 3) {
    *value = ctx->b_smem_kb[what - SBX_LAUNCH_BATCH_SMEM_KB];
    return SBX_OK;
  }
  return fail(ctx, SBX_EINVAL, "unknown launch parameter");
}

int sbx_set_receivers(sbx_ctx *ctx, int64_t n_rec, const int64_t *rec_idx, int64_t max_steps) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  if (n_rec < 0 || (n_rec > 0 && (!rec_idx || max_steps < 1)))
    return fail(ctx, SBX_EINVAL, "need n_rec >= 0, rec_idx and max_steps >= 1");
  std::vector<int64_t> idx;
  if (int rc = fetch_vec(ctx, idx, rec_idx, n_rec)) return rc;
  for (int64_t q : idx)
    if (q < 0 || q >= ctx->ndof * ctx->B) return fail(ctx, SBX_EINVAL, "receiver index out of range");
  drop_graph(ctx);   // the step graphs hold the recording launch (or not)
  CK(cudaStreamSynchronize(ctx->stream));
  dfree(ctx->d_rec_idx);
  dfree(ctx->d_hist);
  ctx->n_rec_hist = ctx->rec_cap = 0;
  if (n_rec == 0) return SBX_OK;
  if (upload(ctx, &ctx->d_rec_idx, idx) || dalloc(ctx, &ctx->d_hist, n_rec * max_steps))
    return fail(ctx, SBX_ENOMEM, "receiver history allocation failed");
  ctx->n_rec_hist = n_rec;
  ctx->rec_cap = max_steps;
  ctx->rec_step0 = ctx->step;
  return SBX_OK;
}

int sbx_read_history(sbx_ctx *ctx, double *out, int64_t max_rows, int64_t *n_rows) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!out || !n_rows || max_rows < 0) return fail(ctx, SBX_EINVAL, "bad arguments");
  if (ctx->n_rec_hist == 0) return fail(ctx, SBX_ESTATE, "no receivers set");
  const int64_t rows = std::min(std::min(ctx->step - ctx->rec_step0, ctx->rec_cap), max_rows);
  *n_rows = std::max<int64_t>(rows, 0);
  if (*n_rows > 0)
    CK(cudaMemcpyAsync(out, ctx->d_hist, *n_rows * ctx->n_rec_hist * sizeof(double),
                       cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_flags(ctx);
}

int sbx_set_mass(sbx_ctx *ctx, const double *mass) {
  if (!ctx) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  std::vector<double> m;
  if (int rc = fetch_vec(ctx, m, mass, (size_t)ctx->ndof)) return rc;
  std::vector<double> minv(ctx->ndof);
  for (int64_t d = 0; d < ctx->ndof; ++d) {
    if (!(m[d] > 0) || !isfinite(m[d])) return fail(ctx, SBX_EINVAL, "mass must be positive and finite");
    minv[d] = 1.0 / m[d];
  }
  for (int64_t d : ctx->h_fixed) minv[d] = 0.0;
  CK(cudaMemcpyAsync(ctx->d_mass, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_minv, minv.data(), minv.size() * sizeof(double),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->w_valid = false;
  return SBX_OK;
}

int sbx_query(sbx_ctx *ctx, int what, int64_t *out) {
  if (!ctx || !out) return SBX_EINVAL;
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  int64_t launches = 0, tiles = 0;
  if (ctx->B > 1) {
    for (int c = 0; c < 3; ++c) {
      launches += ctx->n_b_tiles[c] > 0;
      tiles += (int64_t)ctx->n_b_tiles[c] * (ctx->B / 32);
    }
  } else if (ctx->prec == SBX_PREC_MIXED) {
    launches = (ctx->n_tc_tiles[0] > 0) + (ctx->n_gen_tiles > 0);
    tiles = ctx->n_tc_tiles[0] + ctx->n_gen_tiles;
  } else {
    launches = ctx->n_tiles_simt > 0;
    tiles = ctx->n_tiles_simt;
  }
  switch (what) {
    case SBX_Q_KERNELS_PER_STEP: *out = launches + 1; break;
    case SBX_Q_FORCE_LAUNCHES: *out = launches; break;
    case SBX_Q_TILES: *out = tiles; break;
    case SBX_Q_BRICK_TILES: *out = (ctx->prec == SBX_PREC_MIXED && ctx->B == 1) ? ctx->n_brick_tiles : 0; break;
    case SBX_Q_WALSH_CELLS:
      *out = ctx->B > 1 ? (ctx->prec == SBX_PREC_FP32 ? ctx->wht_cells : 0)
             : ctx->prec == SBX_PREC_FP64 ? ctx->wht_cells
             : (ctx->prec == SBX_PREC_MIXED && ctx->mixed_wht) ? ctx->wht_cells : 0;
      break;
    default: return fail(ctx, SBX_EINVAL, "unknown query");
  }
  return SBX_OK;
}

int sbx_get_step(sbx_ctx *ctx, int64_t *n_out) {
  if (!ctx || !n_out) return SBX_EINVAL;
  *n_out = ctx->step;
  return SBX_OK;
}

int sbx_set_step(sbx_ctx *ctx, int64_t n) {
  if (!ctx || n < 0) return SBX_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  ctx->step = n;
  CK(cudaMemcpyAsync(ctx->d_step, &ctx->step, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SBX_OK;
}

int read_field(sbx_ctx *ctx, int which, double *out, int64_t len) {
  if (!ctx) return SBX_EINVAL;
  if (ctx->state_owner && which != SBX_MASS)   // its own mass stays readable
    return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  if (!out) return fail(ctx, SBX_EINVAL, "null output");
  const double *src = nullptr;
  int64_t need = ctx->ndof * ctx->B;
  switch (which) {
    case SBX_U_N: src = ctx->d_u[ctx->cur]; break;
    case SBX_U_NM1: src = ctx->d_u[ctx->cur ^ 1]; break;
    case SBX_F_INT:
      src = ctx->d_f;
      if (ctx->uses_pairs()) {   // FP32 force -> FP64 per DOF (and case)
        CK(sbx::launch_widen_f32(ctx, reinterpret_cast<const float *>(ctx->d_f), ctx->d_fx,
                                 ctx->stream));
        src = ctx->d_fx;
      }
      break;
    case SBX_MASS: src = ctx->d_mass; need = ctx->ndof; break;
    default: return fail(ctx, SBX_EINVAL, "unknown field");
  }
  if (len != need) return fail(ctx, SBX_EINVAL, "len does not match the field size");
  CK(cudaMemcpyAsync(out, src, len * sizeof(double), cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_flags(ctx);
}

int write_field(sbx_ctx *ctx, int which, const double *in, int64_t len) {
  if (!ctx) return SBX_EINVAL;
  if (ctx->state_owner) return fail(ctx, SBX_ESTATE, "this context shares another context's state: only sbx_force applies");
  if (int rc = set_device(ctx)) return rc;
  ctx->err.clear();
  if (!ctx->have_mesh) return fail(ctx, SBX_ESTATE, "no mesh");
  if (!in) return fail(ctx, SBX_EINVAL, "null input");
  if (len != ctx->ndof * ctx->B) return fail(ctx, SBX_EINVAL, "len does not match the field size");
  double *dst;
  if (which == SBX_U_N)
    dst = ctx->d_u[ctx->cur];
  else if (which == SBX_U_NM1)
    dst = ctx->d_u[ctx->cur ^ 1];
  else
    return fail(ctx, SBX_EINVAL, "only U_N and U_NM1 can be written");
  CK(cudaMemcpyAsync(dst, in, len * sizeof(double), cudaMemcpyDefault, ctx->stream));
  if (ctx->pair_of == (dst == ctx->d_u[0] ? 0 : 1)) ctx->pair_of = -1;
  return SBX_OK;
}

}  // extern "C"

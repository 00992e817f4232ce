/*
 * sbx.h -- C ABI of the GB300 explicit octree-SBFEM solver.
 *
 * One library call sequence mirrors the problem statement of the paper's
 * serial solver (Algorithm 1 and Table "Data structure of explicit solver"):
 *
 *   sbx_create        -- bind a CUDA device and stream
 *   set_patterns      -- master-cell stiffness K_p and lumped mass (Table: K_e, M_e)
 *   mesh_upload       -- cells: pattern T, transform, DOF vector V, edge length S,
 *                        modulus, density; Dirichlet DOFs Gamma_D (Alg. 1, set-up)
 *   set_load          -- point loads Gamma_N with a time function (Sec. 5, Eqs.
 *                        Ricker, Triangle, Lamb)
 *   set_initial       -- U_0, Udot_0 and the fictitious U_-1 (Eq. D0)
 *   step_n            -- n central-difference steps (Alg. 1, time loop;
 *                        Eqs. Rintep, DnMdiag)
 *   read_field / write_field -- state in and out (checkpoint / resume)
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: SBX_OK (0) or one of the
 *     SBX_E* codes below; sbx_last_error() gives a one-line message.  No
 *     C++ exception and no abort crosses this boundary.
 *   - Array arguments may point to host memory (pageable or pinned) or to
 *     device memory of the context's device; the library tells them apart
 *     with cudaPointerGetAttributes.  The library copies every input into
 *     memory it owns; the caller keeps ownership of its buffers, which may
 *     be freed as soon as the call returns.
 *   - Work is enqueued on the stream given to sbx_create.  step_n and
 *     set_initial are asynchronous with respect to the host; read_field,
 *     sbx_sync and sbx_destroy synchronise that stream.
 *   - Node ids are 0-based; DOF = 3 * node + direction (x, y, z).  With
 *     n_rhs = B > 1 load cases, a field is laid out [node][3][B]
 *     (entry (3 * node + d) * B + b).
 *   - A context is not thread-safe; use one context per host thread.
 *   - Unless stated otherwise lengths are element counts, not bytes.
 */
#ifndef SBX_H
#define SBX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbx_ctx sbx_ctx;

/* status codes */
#define SBX_OK          0
#define SBX_EINVAL      1  /* an argument is out of range or inconsistent     */
#define SBX_ENOMEM      2  /* device or host allocation failed                */
#define SBX_ECUDA       3  /* a CUDA runtime call failed                      */
#define SBX_ENONFINITE  4  /* a NaN/Inf appeared in the displacement field    */
#define SBX_ETIMEOUT    5  /* a bounded device-side wait gave up              */
#define SBX_ESTATE      6  /* call out of order (e.g. step before mesh_upload) */

/* precision modes of mesh_upload (the displacement history is FP64 in all) */
#define SBX_PREC_FP64   0  /* K_p u_e in FP64 (DFMA)                           */
#define SBX_PREC_MIXED  1  /* 8-node cells: K_p u_e in FP32 in the Walsh
                              basis of the corners (default), or as three
                              TF32 tensor-core products of split operands
                              with FP32 accumulation (tcgen05), chosen by
                              sbx_set_mixed_kernel; other patterns: FP32
                              FFMA.  All on each cell's displacements
                              relative to its slot-0 node                     */
#define SBX_PREC_FP32   2  /* K_p u_e in FP32 (FFMA), FP64 scale and update   */

/* fields of read_field / write_field */
#define SBX_U_N         0  /* U_n, displacement at the current step           */
#define SBX_U_NM1       1  /* U_{n-1}                                         */
#define SBX_F_INT       2  /* R_int of the last evaluated step (read only)    */
#define SBX_MASS        3  /* lumped global diagonal mass M_diag (read only)  */

/* wavelets of set_load */
#define SBX_WAVE_RICKER     0  /* Eq. (Ricker)                                */
#define SBX_WAVE_TRIANGLE   1  /* Eq. (Triangle)                              */
#define SBX_WAVE_SINE_BURST 2  /* Eq. (Lamb), Hann-windowed sine burst        */

/*
 * sbx_create: bind `device` and a CUDA stream.
 *   cuda_stream: a cudaStream_t of that device, or NULL for a stream the
 *   library creates (and destroys in sbx_destroy).
 *   Errors: SBX_EINVAL (out == NULL, bad device), SBX_ECUDA, SBX_ENOMEM.
 */
int sbx_create(sbx_ctx **out, int device, void *cuda_stream);

/* sbx_destroy: synchronise the stream and free everything (NULL is a no-op). */
int sbx_destroy(sbx_ctx *ctx);

/* One-line description of the last error of this context ("" if none).
 * The string lives until the next call on the context. */
const char *sbx_last_error(const sbx_ctx *ctx);

/* Block until the context's stream is idle; reports a pending
 * non-finite-field flag as SBX_ENONFINITE. */
int sbx_sync(sbx_ctx *ctx);

/*
 * set_patterns: the master cells of Sec. 3.2.2-3.2.3 (Table: K_e, M_e).
 *   n_patterns        number of master cells P (1 .. 144).
 *   n_nodes[P]        nodes n_p of master p, 8 <= n_p <= 26; m_p = 3 n_p.
 *   K_packed          the P stiffness matrices K_p for unit edge length and
 *                     E = 1 (Eq. KM_scale), each m_p x m_p row-major FP64,
 *                     concatenated in pattern order (sum m_p^2 doubles).
 *                     Must be symmetric to 1e-12 relative.
 *   Mlump_packed      the P lumped masses (Sec. 3.3) for unit edge length and
 *                     rho = 1, m_p doubles each, DOF order 3 * node + dir.
 *   Must be called before mesh_upload; calling it again invalidates the mesh.
 *   Errors: SBX_EINVAL (sizes, asymmetric K, non-positive mass), SBX_ENOMEM.
 */
int set_patterns(sbx_ctx *ctx, int n_patterns, const int32_t *n_nodes,
                 const double *K_packed, const double *Mlump_packed);

/*
 * mesh_upload: the octree mesh of Alg. 1's set-up (Table: V, T, S, M_diag,
 * Gamma_D).  Builds the lumped global mass M_diag = sum_e rho_e h_e^3 M_p(e)
 * (in cell components) and allocates the state (U_n = U_{n-1} = 0).
 *   n_nodes, n_cells  N and C.
 *   cell_pattern[C]   master index p of each cell (into set_patterns' list).
 *   cell_sym[C]       transform op in [0, 48): op = 8 * perm_index + sign_bits
 *                     with the permutations of (0,1,2) in lexicographic order;
 *                     node by node u_master[r] = (-1)^{bit r} u_cell[perm[r]]
 *                     and f_cell = Q^T f_master (Sec. 3.2.2).
 *   cell_ptr[C+1]     offsets into cell_nodes; cell_ptr[e+1]-cell_ptr[e] = n_p.
 *   cell_nodes[]      node ids of each cell in MASTER node order (the master's
 *                     present slots in increasing slot order), i.e. the DOF
 *                     vector V already arranged for the master (Sec. 3.4).
 *   h[C], E[C], rho[C] edge length, Young's modulus, density (all > 0).
 *                     K_e = E_e h_e T^T K_p T (Eq. KM_scale).
 *   n_fixed, fixed_dofs[n_fixed]  Dirichlet DOFs held at zero (Gamma_D).
 *   n_rhs             number of load cases B advanced together (1 = plain).
 *   precision_mode    SBX_PREC_*.
 *   Cells are processed grouped by pattern; within a pattern the given order
 *   is kept (pass Morton order for locality).  A node that no cell touches
 *   gets zero mass and stays at rest (M^-1 = 0) until sbx_set_mass gives it
 *   a mass (one part of a split mesh, see sbx_share_state).
 *   Errors: SBX_ESTATE (no patterns; the state is shared with another
 *   context), SBX_EINVAL (ids out of range, node count mismatch,
 *   non-positive h/E/rho), SBX_ENOMEM.
 */
int mesh_upload(sbx_ctx *ctx, int64_t n_nodes, int64_t n_cells,
                const int32_t *cell_pattern, const uint8_t *cell_sym,
                const int64_t *cell_ptr, const int32_t *cell_nodes,
                const double *h, const double *E, const double *rho,
                int64_t n_fixed, const int64_t *fixed_dofs,
                int n_rhs, int precision_mode);

/*
 * set_load: point loads (Gamma_N) R_ext(t) = sum_k P0_k P_k(t) dir_k at node_k
 * for load case rhs_k (Sec. 5 load functions).
 *   n_src             number of point loads K (0 clears the loads).
 *   node[K], dir3[3K] node id and direction vector (used as given).
 *   rhs[K]            load case in [0, n_rhs), or NULL for all 0.
 *   wavelet           SBX_WAVE_* (one kind for all loads of the call).
 *   t1[K], P0[K]      time parameter and peak of each load; ncyc[K] the
 *                     number of cycles of a sine burst (NULL otherwise).
 *   The load enters step n at t_n = n dt.
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL.
 */
int set_load(sbx_ctx *ctx, int n_src, const int64_t *node, const double *dir3,
             const int32_t *rhs, int wavelet, const double *t1,
             const double *P0, const double *ncyc);

/*
 * set_initial: U_0 and Udot_0 (NULL = zero), then the fictitious
 * U_-1 = U_0 - dt Udot_0 + dt^2/2 Uddot_0 with
 * Uddot_0 = M^-1 (R_ext(0) - K U_0) - alpha Udot_0 (Eq. D0).  Resets the step
 * index to 0.  Fixed DOFs are set to zero.  Lengths: 3 N n_rhs.
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (dt <= 0), SBX_ECUDA.
 */
int set_initial(sbx_ctx *ctx, const double *u0, const double *v0,
                double dt, double alpha);

/*
 * step_n: n_steps steps of Eq. (DnMdiag):
 *   U_{n+1} = [dt^2 M^-1 (R_ext(t_n) - R_int(U_n)) + 2 U_n
 *              - (1 - alpha dt / 2) U_{n-1}] / (1 + alpha dt / 2),
 * R_int = sum_p K_p [U_p1 ... U_pk] diag(S) assembled through V (Eq. Rintep).
 *   Asynchronous.  dt > 0, alpha >= 0.  A NaN/Inf produced in the field sets
 *   a flag that the next synchronising call reports as SBX_ENONFINITE.
 *   Errors: SBX_ESTATE, SBX_EINVAL, SBX_ECUDA.
 */
int step_n(sbx_ctx *ctx, int64_t n_steps, double dt, double alpha);

/*
 * sbx_prepare_steps: build, without running them, the CUDA graphs that a
 * later step_n(ctx, n_steps, dt, alpha) replays (Alg. 1's time loop is
 * replayed as graphs of 32 steps plus one graph for the call's remaining
 * steps), so that the first such call launches no capture.  Graphs are
 * cached per context until dt, alpha, the receivers or the kernel choice
 * change.  Enqueues nothing when the graphs exist already.
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (n_steps < 0, dt <= 0,
 *   alpha < 0), SBX_ECUDA.
 */
int sbx_prepare_steps(sbx_ctx *ctx, int64_t n_steps, double dt, double alpha);

/* Current step index n (the state holds U_n and U_{n-1}). */
int sbx_get_step(sbx_ctx *ctx, int64_t *n_out);
/* Set the step index, e.g. after write_field when resuming. */
int sbx_set_step(sbx_ctx *ctx, int64_t n);

/*
 * read_field: copy field `which` (SBX_U_N, SBX_U_NM1, SBX_F_INT, SBX_MASS)
 * into out[len]; len must equal 3 N n_rhs (3 N for SBX_MASS).  Synchronises
 * the stream.  SBX_F_INT holds R_int - R_ext of the last step.
 *   Errors: SBX_ESTATE, SBX_EINVAL (len, which), SBX_ENONFINITE, SBX_ECUDA.
 */
int read_field(sbx_ctx *ctx, int which, double *out, int64_t len);

/* write_field: overwrite SBX_U_N or SBX_U_NM1 from in[len] (resume). */
int write_field(sbx_ctx *ctx, int which, const double *in, int64_t len);

/*
 * sbx_profile: diagnostics.  Runs n_steps ordinary steps (same kernels and
 * launch shapes as step_n, without graph replay), bracketing every kernel
 * launch with CUDA events on the context stream, and returns the summed
 * device time in milliseconds of the internal-force launches (*ms_force)
 * and of the update launches (*ms_update).  Advances the state like step_n.
 *   Errors: as step_n.
 */
int sbx_profile(sbx_ctx *ctx, int64_t n_steps, double dt, double alpha,
                double *ms_force, double *ms_update);

/*
 * set_modulus: replace every cell's Young's modulus E_e (K_e = E_e h_e T^T K_p T,
 * Eq. KM_scale) without re-uploading the mesh.  E[C] in the caller's cell
 * order of mesh_upload, all > 0.  The lumped mass does not depend on E.
 * Supported for single-load-case meshes in SBX_PREC_FP64 / SBX_PREC_FP32.
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (values, mode).
 */
int set_modulus(sbx_ctx *ctx, const double *E);

/*
 * sbx_adjoint: misfit of receiver time histories and its gradient with
 * respect to every cell's modulus, by the exact discrete adjoint of the
 * undamped recurrence (alpha = 0):
 *   J = 1/2 sum_{n=1..N} sum_r (U_n[rec_r] - data[(n-1) n_rec + r])^2,
 *   lambda_n = g_n + (2 I - K W) lambda_{n+1} - lambda_{n+2},  W = dt^2 M^-1,
 *   dJ/dE_e = -h_e sum_{n=0}^{N-1} (W lambda_{n+1})_e^T T^T K_p T U_{n,e}.
 * Starts from the state set by set_initial (step index 0), which must be at
 * rest (U_0 = 0, Udot_0 = 0) so that U_-1 does not depend on the moduli.
 * The forward run stores (U_n, U_{n-1}) every ckpt_every steps; the reverse
 * sweep recomputes each segment from its checkpoint.  Device memory for
 * (N / ckpt_every + 1) checkpoints and ckpt_every + 1 states is allocated
 * for the call and freed before it returns.
 *   n_steps N >= 1, dt > 0, n_rec >= 0, rec_dof[n_rec] DOF indices,
 *   data[N * n_rec], ckpt_every >= 1.  Outputs: *misfit_out = J,
 *   grad_E_out[C] in the caller's cell order.  Afterwards the state is
 *   reset to the starting state (step 0).  Single-load-case meshes in
 *   SBX_PREC_FP64 or SBX_PREC_FP32 (the contraction runs in that precision,
 *   the recurrences and the gradient sums in FP64).
 *   Errors: SBX_ESTATE (no mesh, step index not 0), SBX_EINVAL, SBX_ENOMEM,
 *   SBX_ECUDA, SBX_ENONFINITE.
 */
int sbx_adjoint(sbx_ctx *ctx, int64_t n_steps, double dt, int64_t n_rec,
                const int64_t *rec_dof, const double *data, int64_t ckpt_every,
                double *misfit_out, double *grad_E_out);

/*
 * Split step, for a caller that must act between the internal force and the
 * update -- the interface sum of the node-cut partition (Sec. 4: each GPU
 * holds the cells of its part and the nodes they touch; the partial forces
 * of the nodes on a cut are summed over the parts before every update) or
 * any other force added from outside.  One step of step_n equals
 *   sbx_force(ctx, dt); <modify f>; sbx_update(ctx, dt, alpha);
 * sbx_force: f = R_int(U_n) - R_ext(t_n) into the force buffer (Eq. Rintep
 *   and the load term).  sbx_update: Eq. DnMdiag with that f, U_{n+1}
 *   replaces U_{n-1}, the step index advances and f is cleared.  Both are
 *   asynchronous.  Calling sbx_update without a preceding sbx_force, or
 *   sbx_force twice, is SBX_ESTATE.
 *   Errors: SBX_ESTATE, SBX_EINVAL (dt, alpha), SBX_ECUDA.
 */
int sbx_force(sbx_ctx *ctx, double dt);
int sbx_update(sbx_ctx *ctx, double dt, double alpha);

/*
 * sbx_field_ptr: device address and layout of a field the library owns, for
 * in-place access on the context's stream (e.g. a collective between
 * sbx_force and sbx_update).  which = SBX_U_N, SBX_U_NM1, SBX_F_INT or
 * SBX_MASS.  *layout:
 *   SBX_LAYOUT_F64_DOF    double per DOF (entry 3 node + d, times B load
 *                         cases as in read_field); *len = 3 N B (3 N for
 *                         SBX_MASS)
 *   SBX_LAYOUT_F32_NODE4  float [N][4] (x, y, z, unused): SBX_F_INT of
 *                         SBX_PREC_MIXED meshes; *len = 4 N
 *   SBX_LAYOUT_F32_DOF    float per DOF and case: SBX_F_INT of batched
 *                         SBX_PREC_FP32 meshes; *len = 3 N B
 * The address stays valid until the next mesh_upload or sbx_destroy; the
 * buffers behind SBX_U_N / SBX_U_NM1 swap roles every step, so ask again
 * after each step.  After writing U_n or U_{n-1} through the pointer, call
 * sbx_touch (below).
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (which, NULL outputs).
 */
#define SBX_LAYOUT_F64_DOF   0
#define SBX_LAYOUT_F32_NODE4 1
#define SBX_LAYOUT_F32_DOF   2
int sbx_field_ptr(sbx_ctx *ctx, int which, void **ptr, int64_t *len, int *layout);

/*
 * sbx_wait_selftest: diagnostics of the failure path (the paper has no
 * counterpart).  Every wait of the tensor-core kernels on an asynchronous
 * completion (bulk copy, MMA) is bounded; a wait that gives up sets a device
 * flag that the next synchronising call reports as SBX_ETIMEOUT, and the
 * kernel returns instead of hanging.  This call runs that wait on a fresh
 * barrier for at most `polls` polls (1 .. 2^30): with arrive = 1 the barrier
 * completes first (returns SBX_OK), with arrive = 0 nothing completes it
 * (returns SBX_ETIMEOUT).  The context's flags are left as they were and the
 * context stays usable.  Synchronises the stream.
 *   Errors: SBX_EINVAL (polls), SBX_ECUDA, SBX_ETIMEOUT as described.
 */
int sbx_wait_selftest(sbx_ctx *ctx, int64_t polls, int arrive);

/* sbx_touch: tell the library that U_n was changed through sbx_field_ptr
 * (the mixed form re-derives its FP32 (hi, lo) split of U_n). */
int sbx_touch(sbx_ctx *ctx);

/*
 * sbx_set_receivers: record a time history of the displacement at n_rec
 * entries of the state array (receivers, as in Sec. 5's measured
 * responses) after every step that step_n takes from now on, for at
 * most max_steps steps.  rec_idx[r] indexes the state array U_n of this
 * context: DOF 3 node + d, batched (3 node + d) B + b; host or device
 * pointer, copied.  n_rec = 0 turns recording off.  Recording costs one
 * small kernel launch per step; it is captured with the step graphs.
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (index out of range,
 *   n_rec < 0, max_steps < 1), SBX_ENOMEM.
 */
int sbx_set_receivers(sbx_ctx *ctx, int64_t n_rec, const int64_t *rec_idx, int64_t max_steps);

/*
 * sbx_read_history: the recorded rows, out[s n_rec + r] = U at receiver r
 * after the s-th step since sbx_set_receivers, for s < *n_rows =
 * min(steps taken, max_steps, max_rows).  out: host or device pointer with
 * room for max_rows n_rec doubles.  Synchronises the context's stream.
 *   Errors: SBX_ESTATE (no receivers set), SBX_EINVAL (NULL, max_rows < 0).
 */
int sbx_read_history(sbx_ctx *ctx, double *out, int64_t max_rows, int64_t *n_rows);

/*
 * sbx_lanczos: k steps of the Lanczos iteration, with full
 * reorthogonalisation (two classical Gram-Schmidt passes per step), for the
 * free vibration problem K x = omega^2 M x of the uploaded mesh -- the cube
 * example of Sec. 5 computes eigenfrequencies with the same K and lumped M
 * the explicit solver steps with.  The operator is M^-1/2 K M^-1/2 on the
 * free DOFs (M^-1 = 0 on the fixed ones); K is applied by the FP64
 * element-by-element force kernel of the explicit step.  Output: the
 * tridiagonal T_k, alpha[j] on its diagonal and beta[j] below it
 * (beta[k-1] = the norm of the last residual).  The eigenvalues of T_k
 * (Ritz values) approximate omega^2, the extreme ones first; a multiple
 * eigenvalue appears once.  Once the Krylov space is exhausted beta
 * vanishes and the later coefficients are 0.
 *   v0[3N]: start vector, host or device (fixed DOFs ignored; must not
 *   vanish on the free DOFs).  alpha, beta: host or device, k doubles each.
 *   Holds (k + 4) 3N doubles of device memory during the call; synchronises
 *   the context's stream.
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (k outside [1, 4096], NULL, a
 *   batched or FP32 mesh, v0 zero on the free DOFs), SBX_ENOMEM.
 */
int sbx_lanczos(sbx_ctx *ctx, int64_t k, const double *v0, double *alpha, double *beta);

/*
 * sbx_set_mixed_kernel: mixed form (one load case) only -- which kernel
 * applies K_p to the regular 8-node cells in the element-by-element
 * internal force (Eq. Rintep; the other patterns always run on the FP32
 * SIMT pattern kernel): SBX_MIXED_TENSOR (TF32x3 on the tensor
 * cores, tcgen05, accumulators in tensor memory) or SBX_MIXED_WALSH (FP32
 * SIMT in the Walsh basis of the cell's corners, where K_p is eight 3 x 3
 * blocks).  Both take the same tiles, differences to slot 0 and node sums;
 * the Walsh kernel is available (and the default) when the 8-node
 * pattern's K_p passed the block check at mesh_upload.
 *   Errors: SBX_EINVAL (ctx NULL, unknown kind, Walsh not available, a
 *   mesh in another form).
 */
#define SBX_MIXED_TENSOR 0
#define SBX_MIXED_WALSH  1
int sbx_set_mixed_kernel(sbx_ctx *ctx, int kind);

/*
 * sbx_set_mass: replace the lumped diagonal mass M_diag[3N] (Sec. 3.3) --
 * e.g. by the sum over all parts of a node-cut partition, whose interface
 * nodes receive mass from cells on several GPUs.  Values > 0; M^-1 stays 0
 * on the Dirichlet DOFs.
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (values, NULL).
 */
int sbx_set_mass(sbx_ctx *ctx, const double *mass);

/*
 * sbx_query: diagnostics about the uploaded mesh and the launch plan.
 *   what = SBX_Q_KERNELS_PER_STEP  kernel launches per step (force + update)
 *          SBX_Q_FORCE_LAUNCHES    force-kernel launches per step
 *          SBX_Q_TILES             CTAs of all force launches of one step
 *          SBX_Q_BRICK_TILES       mixed form: tensor-core tiles that are
 *                                  complete 4 x 4 x 8 blocks of 8-node cells
 *          SBX_Q_WALSH_CELLS       cells whose K_p is applied in the Walsh
 *                                  basis of their corners (FP64 form, batched
 *                                  FP32 form, mixed form on SBX_MIXED_WALSH)
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (unknown item, NULL out).
 */
#define SBX_Q_KERNELS_PER_STEP 0
#define SBX_Q_FORCE_LAUNCHES   1
#define SBX_Q_TILES            2
#define SBX_Q_BRICK_TILES      3
#define SBX_Q_WALSH_CELLS      5
int sbx_query(sbx_ctx *ctx, int what, int64_t *out);

/*
 * Node-cut interface sum with the neighbouring parts (Sec. 4.2: each part
 * sums the partial internal forces of the DOFs it shares with its
 * neighbours).  The caller moves the buffers between parts (e.g. NCCL
 * send / receive); the library packs and sums on the context's stream.
 * Rows follow the force accumulator (sbx_field_ptr(SBX_F_INT)): 3 doubles
 * per node in the FP64 forms, 4 floats (x, y, z, unused) in the mixed form.
 *
 * sbx_halo_plan: n_send nodes (local ids; the blocks of all neighbours in
 *   the caller's order) whose rows the pack writes, and for each of n_cut
 *   cut nodes (local ids) its contributions contrib_src[contrib_ptr[j] ..
 *   contrib_ptr[j+1]): -1 = this part's own partial force, r >= 0 = row r
 *   of the receive buffer.  The sum adds them in that order from zero, so
 *   parts that list a node's contributions in one common order (e.g. by
 *   ascending rank of the holding part) compute identical sums.  Host or
 *   device arrays (copied).  One load case only.
 *   Errors: SBX_ESTATE (no mesh), SBX_EINVAL (ids or rows out of range,
 *   contrib_ptr not starting at 0 or decreasing), SBX_ENOMEM.
 * sbx_halo_pack: send_buf[i] = row send_nodes[i] of the force accumulator
 *   (device memory, n_send rows).  Enqueued on the stream.
 * sbx_halo_sum: for every cut node, the accumulator row = the sum of its
 *   contributions (recv_buf: device memory, n_send rows, filled by the
 *   neighbours in the same block order).  Enqueued on the stream.
 */
int sbx_halo_plan(sbx_ctx *ctx, int64_t n_send, const int64_t *send_nodes, int64_t n_cut,
                  const int64_t *cut_nodes, const int64_t *contrib_ptr,
                  const int64_t *contrib_src);
int sbx_halo_pack(sbx_ctx *ctx, void *send_buf);
int sbx_halo_sum(sbx_ctx *ctx, const void *recv_buf);

/*
 * sbx_share_state: make ctx (a mesh over the same n_nodes, load cases and
 * precision, created on the same device and stream) a guest of owner: ctx
 * releases its own state and afterwards reads the owner's U_n and adds its
 * cells' internal forces into the owner's accumulator with sbx_force.  This
 * splits one part's cells in two, e.g. the cells on the interface and the
 * interior ones, so that the interface exchange can run while the interior
 * force is computed (the computation order of Sec. 4.2).  A guest's other
 * stepping calls and field reads fail with SBX_ESTATE (its own lumped mass,
 * read_field(SBX_MASS), stays readable); loads belong on the owner; the owner
 * clears the accumulator in its sbx_update and is destroyed after its
 * guests (sbx_destroy of an owner with guests: SBX_ESTATE).
 *   Errors: SBX_EINVAL (sizes, devices or streams differ), SBX_ESTATE.
 */
int sbx_share_state(sbx_ctx *ctx, sbx_ctx *owner);

/*
 * sbx_classify_cells: the set-up's integer work on the GPU (Sec. 3.2.1 -
 * 3.2.2, Alg. 1's set-up): every cell's master pattern (the largest mask of
 * its mask's orbit under the 48 signed permutations), its op (the smallest
 * op carrying it there; op convention of mesh_upload) and its node list in
 * master node order; then the cells sorted by pattern (stable: the given
 * order, e.g. Morton, is kept within a pattern) and each pattern's
 * slot-major connectivity.  These are exactly the arrays mesh_upload takes
 * and builds.
 *   slot_node[C][26]  DEVICE, node id per slot (-1: absent), mesh format of
 *                     the octree generator (corners, mid-edges, face centres).
 *   mask[C]           DEVICE, 12-bit mid-edge mask.
 *   masters, n_masters   HOST out: the distinct master masks, ascending
 *                     (pattern id = position), at most 144.
 *   cell_pattern[C], cell_sym[C], cell_ptr[C+1], cell_nodes[<= 26 C]
 *                     DEVICE out: as mesh_upload's inputs.
 *   order[C]          DEVICE out: sorted position -> cell.
 *   pat_start[P+1]    HOST out: first sorted position of each pattern.
 *   conn[<= 26 C]     DEVICE out: pattern p's block [n_p][C_p] at offset
 *                     sum_{q<p} n_q C_q.
 * Synchronises the stream.  Allocates scratch with cudaMalloc.
 *   Errors: SBX_EINVAL (sizes, host pointers where device memory is
 *   required, a cell without a node its pattern needs), SBX_ENOMEM,
 *   SBX_ECUDA.
 */
int sbx_classify_cells(sbx_ctx *ctx, int64_t n_cells, const int32_t *slot_node,
                       const int32_t *mask, int32_t *masters, int32_t *n_masters,
                       int32_t *cell_pattern, uint8_t *cell_sym, int64_t *cell_ptr,
                       int32_t *cell_nodes, int64_t *order, int64_t *pat_start, int32_t *conn);

/*
 * sbx_set_launch / sbx_get_launch: launch configuration of the force
 * kernels (no counterpart in the paper: how Eq. Rintep's contraction is
 * mapped onto the GPU).  The results do not depend on it beyond rounding;
 * the step graphs are rebuilt after a change.
 *   SBX_LAUNCH_HANGING_KERNEL      mixed and batched FP32 forms: the
 *       patterns other than the identity-op 8-node cell on the tensor cores,
 *       TF32 x 3 with FP32 accumulation in tensor memory
 *       (SBX_HANGING_TENSOR; the mixed form's default), or on FP32 SIMT
 *       (SBX_HANGING_SIMT; the batched form's default).  mesh_upload resets
 *       it to the form's default.
 *   SBX_LAUNCH_WALSH_CTAS_PER_SM   mixed form: resident CTAs per SM of the
 *       Walsh-basis kernel, 1 .. 8, or 0 for the library's choice.
 *   SBX_LAUNCH_HANGING_CTAS_PER_SM mixed form: CTAs per SM of the
 *       tensor-core kernel of the hanging-node patterns, 1 (default) or 2.
 *   SBX_LAUNCH_UPDATE_KERNEL       mixed form: Eq. DnMdiag's update with
 *       its rows streamed through shared memory in chunks of 128 nodes by
 *       1-D bulk copies, two chunks in flight per CTA (SBX_UPDATE_BULK,
 *       default), or with each thread loading its own nodes
 *       (SBX_UPDATE_THREAD).  Bit-identical results.
 *   SBX_LAUNCH_BATCH_TILE_CELLS + c   batched form, pattern class c (0: up
 *       to 8 nodes, 1: up to 16, 2: more): most cells per tile, 1 .. 64
 *       (default 32).  A change rebuilds the class's tiles.
 *   SBX_LAUNCH_BATCH_SMEM_KB + c      batched form, class c: shared memory
 *       per CTA in KB that a tile's staging may take, 16 .. 227 (default
 *       100: two CTAs per SM); tiles shrink until they fit.
 *   Errors: SBX_EINVAL (unknown parameter or value; a tile shape that does
 *   not fit leaves the previous one in place).
 */
#define SBX_LAUNCH_HANGING_KERNEL     0
#define SBX_LAUNCH_WALSH_CTAS_PER_SM  1
#define SBX_LAUNCH_HANGING_CTAS_PER_SM 2
#define SBX_LAUNCH_UPDATE_KERNEL      3
#define SBX_LAUNCH_BATCH_TILE_CELLS   16
#define SBX_LAUNCH_BATCH_SMEM_KB      20
#define SBX_HANGING_SIMT   0
#define SBX_HANGING_TENSOR 1
#define SBX_UPDATE_THREAD  0
#define SBX_UPDATE_BULK    1
int sbx_set_launch(sbx_ctx *ctx, int what, int value);
int sbx_get_launch(sbx_ctx *ctx, int what, int *value);

/*
 * sbx_step_static: one undamped explicit step with no external load that
 * allocates nothing.  The paper has no counterpart; this entry point exists
 * for callers that cannot allocate device memory: code that runs while a
 * framework's caching allocator owns the whole device, real-time or
 * embedded loops where cudaMalloc (which may synchronise the device or fail
 * under memory pressure) is not allowed, and plug-ins that may only touch
 * the buffers they are handed.  It computes
 *   f = sum_e E_e h_e T_e^T K_p T_e u_e          (same kernel arithmetic as step_n)
 *   U_{n+1} = -dt^2 minv f + 2 U_n - U_{n-1}     written over u_nm1
 * in FP64 on the CURRENT device and enqueues the work on cuda_stream
 * (NULL = legacy default stream); it neither synchronises nor allocates.
 *
 *   n_dof          3 N, at most SBX_STATIC_MAX_DOF (larger sizes: SBX_EINVAL).
 *   n_patterns     P, 1 .. SBX_STATIC_MAX_PATTERNS.
 *   pat_nodes[P], pat_cells[P]   HOST arrays: nodes of each master and the
 *                  number of cells of each pattern; cells are stored grouped
 *                  by pattern in pattern order.
 *   K_packed       DEVICE, the P master stiffnesses as in set_patterns.
 *   conn           DEVICE, per pattern p a block [n_p][C_p] of node ids in
 *                  master node order (slot-major), blocks in pattern order.
 *   sym[C], scale[C]  DEVICE, op (as in mesh_upload) and E_e h_e per cell.
 *   minv[n_dof]    DEVICE, 1 / M_diag with 0 on fixed DOFs.
 *   u_n[n_dof]     DEVICE, U_n (read).  u_nm1[n_dof]: DEVICE, U_{n-1} on
 *                  entry, U_{n+1} on return of the enqueued work.
 * Working memory: one library-owned static device array of
 * SBX_STATIC_MAX_DOF doubles (32 MiB) that every GPU loading the library
 * holds until exit.  All calls share it and it keeps the last call's
 * contents (each call clears the part it uses first), so calls whose work
 * overlaps on the GPU (different streams, or different host threads on one
 * device) race and must be ordered by the caller.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * the device's SM count, and must come before any stream capture; both stay
 * cached for the process, so the entry point must not be used again after
 * a cudaDeviceReset of that device.
 * The library trusts the device arrays' contents: the caller guarantees
 * 0 <= node id < n_dof / 3 in conn and 0 <= sym < 48; an id out of range
 * is an out-of-bounds access on the GPU.
 *   Errors: SBX_EINVAL (sizes, NULL pointers, dt <= 0), SBX_ECUDA.
 */
#define SBX_STATIC_MAX_DOF      (4 * 1024 * 1024)
#define SBX_STATIC_MAX_PATTERNS 144
int sbx_step_static(void *cuda_stream, int64_t n_dof, int n_patterns,
                    const int32_t *pat_nodes, const int64_t *pat_cells,
                    const double *K_packed, const int32_t *conn, const uint8_t *sym,
                    const double *scale, const double *minv, double dt,
                    const double *u_n, double *u_nm1);

#ifdef __cplusplus
}
#endif
#endif /* SBX_H */

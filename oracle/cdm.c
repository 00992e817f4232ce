/*
 * FP64 oracle: element-by-element explicit central-difference solver.
 * TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): nothing in the product
 * links or loads this file.
 *
 * Algorithm 1 of the paper, written plainly:
 *   for every step n:
 *     R_int = 0
 *     for every cell e (ascending): build K_e = s_e T_e^T K_p T_e entry by
 *       entry, f_e = K_e u_e (row by row, columns ascending), add f_e into
 *       R_int through the cell's DOF list                (Eqs. Rinte, Rintep)
 *     R_ext at t_n = n dt from the point loads           (Eqs. Ricker, Triangle, Lamb)
 *     U_{n+1} = [dt^2 M^-1 (R_ext - R_int) + 2 U_n - (1 - a dt/2) U_{n-1}]
 *               / (1 + a dt/2)                           (Eq. DnMdiag)
 *     U_{n-1} <- U_n, U_n <- U_{n+1}
 * dt2minv[d] = dt^2 / M_diag[d], zero on fixed DOFs (which therefore stay 0).
 *
 * K_e entry (3i+a, 3j+b) = s_e sign[a] sign[b] K_p(3 tmap[i] + comp[a],
 * 3 tmap[j] + comp[b]) is the (i,a),(j,b) entry of s_e T^T K_p T for the
 * signed permutation T that carries the cell onto its master (Sec. 3.2.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double load_amplitude(int kind, double t, double t1, double ncyc)
{
    const double pi = 3.14159265358979323846;
    if (kind == 0) {                       /* Ricker, Eq. (Ricker) */
        double tau = (t - t1) / (t1 / 5.0);
        return (1.0 - tau * tau) * exp(-0.5 * tau * tau);
    } else if (kind == 1) {                /* triangular pulse, Eq. (Triangle) */
        if (t < 0.0 || t > 2.0 * t1) return 0.0;
        return 1.0 - fabs(t / t1 - 1.0);
    } else {                               /* Hann-windowed sine burst, Eq. (Lamb) */
        if (t < 0.0 || t > t1) return 0.0;
        double s = sin(pi * t / t1);
        return sin(2.0 * pi * ncyc * t / t1) * s * s;
    }
}

typedef struct {
    int64_t n_dof, n_cells;
    const int64_t *pat_m, *pat_off; const double *kp;          /* master K_p, row-major */
    const int64_t *cell_pat; const double *scale;              /* s_e = E_e h_e */
    const int64_t *node_ptr, *dofs, *tmap, *comp, *sign;
} Mesh;

/* One internal-force evaluation into f (zeroed here); cells [c0, c1). */
static void internal_force(const Mesh *M, const double *u, double *f,
                           int64_t c0, int64_t c1, double *Ke, double *ue)
{
    for (int64_t c = c0; c < c1; ++c) {
        int64_t p = M->cell_pat[c];
        int64_t mp = M->pat_m[p];
        const double *K = M->kp + M->pat_off[p];
        int64_t n0 = M->node_ptr[c], nn = M->node_ptr[c + 1] - n0;
        int64_t m = 3 * nn;
        const int64_t *cp = M->comp + 3 * c, *sg = M->sign + 3 * c;
        const int64_t *dof = M->dofs + 3 * n0;
        for (int64_t i = 0; i < nn; ++i)
            for (int a = 0; a < 3; ++a)
                for (int64_t j = 0; j < nn; ++j)
                    for (int b = 0; b < 3; ++b) {
                        int64_t r = 3 * M->tmap[n0 + i] + cp[a];
                        int64_t q = 3 * M->tmap[n0 + j] + cp[b];
                        Ke[(3 * i + a) * m + 3 * j + b] =
                            M->scale[c] * (double)(sg[a] * sg[b]) * K[r * mp + q];
                    }
        for (int64_t k = 0; k < m; ++k) ue[k] = u[dof[k]];
        for (int64_t k = 0; k < m; ++k) {
            double acc = 0.0;
            for (int64_t l = 0; l < m; ++l) acc += Ke[k * m + l] * ue[l];
            f[dof[k]] += acc;
        }
    }
}

#define MAXM 78

/* f = sum_e K_e u_e (sequential, cell order). */
int oracle_apply_K(int64_t n_dof, int64_t n_cells,
                   const int64_t *pat_m, const int64_t *pat_off, const double *kp,
                   const int64_t *cell_pat, const double *scale,
                   const int64_t *node_ptr, const int64_t *dofs, const int64_t *tmap,
                   const int64_t *comp, const int64_t *sign,
                   const double *u, double *f)
{
    Mesh M = {n_dof, n_cells, pat_m, pat_off, kp, cell_pat, scale, node_ptr, dofs, tmap, comp, sign};
    double Ke[MAXM * MAXM], ue[MAXM];
    memset(f, 0, sizeof(double) * (size_t)n_dof);
    internal_force(&M, u, f, 0, n_cells, Ke, ue);
    return 0;
}

/*
 * The same sum with the cells split over n_threads OpenMP threads, each with
 * its own force buffer, summed afterwards in thread order.
 */
int oracle_apply_K_threads(int64_t n_dof, int64_t n_cells,
                           const int64_t *pat_m, const int64_t *pat_off, const double *kp,
                           const int64_t *cell_pat, const double *scale,
                           const int64_t *node_ptr, const int64_t *dofs, const int64_t *tmap,
                           const int64_t *comp, const int64_t *sign,
                           const double *u, double *f, int n_threads)
{
    Mesh M = {n_dof, n_cells, pat_m, pat_off, kp, cell_pat, scale, node_ptr, dofs, tmap, comp, sign};
    int nt = n_threads > 1 ? n_threads : 1;
    if (nt == 1)
        return oracle_apply_K(n_dof, n_cells, pat_m, pat_off, kp, cell_pat, scale, node_ptr,
                              dofs, tmap, comp, sign, u, f);
#ifdef _OPENMP
    double *buf = (double *)calloc((size_t)n_dof * (size_t)nt, sizeof(double));
    if (!buf) return 1;
#pragma omp parallel num_threads(nt)
    {
        int t = omp_get_thread_num();
        double Ke[MAXM * MAXM], ue[MAXM];
        int64_t c0 = n_cells * t / nt, c1 = n_cells * (t + 1) / nt;
        internal_force(&M, u, buf + (size_t)t * (size_t)n_dof, c0, c1, Ke, ue);
    }
    for (int64_t d = 0; d < n_dof; ++d) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += buf[(size_t)t * (size_t)n_dof + d];
        f[d] = s;
    }
    free(buf);
    return 0;
#else
    return 2;
#endif
}

/*
 * Per cell e: out[e] = a_e^T (h_e T_e^T K_p T_e) b_e, the cell's stiffness
 * divided by its modulus (Eq. KM_scale: K_e = E_e h_e T_e^T K_p T_e) between
 * the gathered vectors a_e and b_e.  K_e / E_e is built entry by entry as in
 * internal_force, with h in place of s_e.
 */
int oracle_cell_energy(int64_t n_dof, int64_t n_cells,
                       const int64_t *pat_m, const int64_t *pat_off, const double *kp,
                       const int64_t *cell_pat, const double *h,
                       const int64_t *node_ptr, const int64_t *dofs, const int64_t *tmap,
                       const int64_t *comp, const int64_t *sign,
                       const double *a, const double *b, double *out, int n_threads)
{
    (void)n_dof;
    int nt = n_threads > 1 ? n_threads : 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static)
#endif
    for (int64_t c = 0; c < n_cells; ++c) {
        double Ke[MAXM * MAXM];
        int64_t p = cell_pat[c];
        int64_t mp = pat_m[p];
        const double *K = kp + pat_off[p];
        int64_t n0 = node_ptr[c], nn = node_ptr[c + 1] - n0;
        int64_t m = 3 * nn;
        const int64_t *cp = comp + 3 * c, *sg = sign + 3 * c;
        const int64_t *dof = dofs + 3 * n0;
        for (int64_t i = 0; i < nn; ++i)
            for (int r = 0; r < 3; ++r)
                for (int64_t j = 0; j < nn; ++j)
                    for (int q = 0; q < 3; ++q) {
                        int64_t row = 3 * tmap[n0 + i] + cp[r];
                        int64_t col = 3 * tmap[n0 + j] + cp[q];
                        Ke[(3 * i + r) * m + 3 * j + q] =
                            h[c] * (double)(sg[r] * sg[q]) * K[row * mp + col];
                    }
        double acc = 0.0;
        for (int64_t k = 0; k < m; ++k) {
            double row = 0.0;
            for (int64_t l = 0; l < m; ++l) row += Ke[k * m + l] * b[dof[l]];
            acc += a[dof[k]] * row;
        }
        out[c] = acc;
    }
    return 0;
}

/*
 * n_steps CDM steps starting from step index n0 (time t_n = n dt).
 * u_c = U_n, u_p = U_{n-1} on entry; U_{n0+n_steps}, U_{n0+n_steps-1} on exit.
 * Loads: load_dof[k] receives load_amp[k] * P(t) of wavelet load_wave[k].
 * Receivers: rec_out[s * n_rec + r] = U_{n0+s+1}[rec_dof[r]] (if n_rec > 0).
 * n_threads > 1 splits the cells over OpenMP threads, each with its own
 * force buffer, summed afterwards in thread order (deterministic for a
 * given thread count).
 */
int oracle_cdm_run(int64_t n_dof, int64_t n_cells,
                   const int64_t *pat_m, const int64_t *pat_off, const double *kp,
                   const int64_t *cell_pat, const double *scale,
                   const int64_t *node_ptr, const int64_t *dofs, const int64_t *tmap,
                   const int64_t *comp, const int64_t *sign,
                   const double *dt2minv,
                   int64_t n_load, const int64_t *load_dof, const double *load_amp,
                   const int64_t *load_wave, const int64_t *wave_kind,
                   const double *wave_t1, const double *wave_ncyc,
                   double dt, double alpha, int64_t n0, int64_t n_steps,
                   double *u_c, double *u_p,
                   int64_t n_rec, const int64_t *rec_dof, double *rec_out,
                   double *f_last, int n_threads)
{
    Mesh M = {n_dof, n_cells, pat_m, pat_off, kp, cell_pat, scale, node_ptr, dofs, tmap, comp, sign};
    int nt = n_threads > 1 ? n_threads : 1;
    double *f = (double *)calloc((size_t)n_dof * (size_t)nt, sizeof(double));
    double *u_n = (double *)malloc(sizeof(double) * (size_t)n_dof);
    if (!f || !u_n) { free(f); free(u_n); return 1; }
    const double cm = 1.0 - 0.5 * alpha * dt, cp = 1.0 + 0.5 * alpha * dt;
    for (int64_t s = 0; s < n_steps; ++s) {
        int64_t n = n0 + s;
        if (nt == 1) {
            double Ke[MAXM * MAXM], ue[MAXM];
            memset(f, 0, sizeof(double) * (size_t)n_dof);
            internal_force(&M, u_c, f, 0, n_cells, Ke, ue);
        } else {
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
            {
                int t = omp_get_thread_num();
                double Ke[MAXM * MAXM], ue[MAXM];
                double *ft = f + (size_t)t * (size_t)n_dof;
                memset(ft, 0, sizeof(double) * (size_t)n_dof);
                int64_t c0 = n_cells * t / nt, c1 = n_cells * (t + 1) / nt;
                internal_force(&M, u_c, ft, c0, c1, Ke, ue);
            }
            for (int t = 1; t < nt; ++t)
                for (int64_t d = 0; d < n_dof; ++d) f[d] += f[(size_t)t * (size_t)n_dof + d];
#else
            free(f); free(u_n); return 2;
#endif
        }
        /* R_ext - R_int, stored in f as its negation first */
        for (int64_t d = 0; d < n_dof; ++d) f[d] = -f[d];
        double t = (double)n * dt;
        for (int64_t k = 0; k < n_load; ++k) {
            int64_t w = load_wave[k];
            f[load_dof[k]] += load_amp[k] * load_amplitude((int)wave_kind[w], t, wave_t1[w], wave_ncyc[w]);
        }
        for (int64_t d = 0; d < n_dof; ++d)
            u_n[d] = (dt2minv[d] * f[d] + 2.0 * u_c[d] - cm * u_p[d]) / cp;
        if (f_last && s == n_steps - 1)
            for (int64_t d = 0; d < n_dof; ++d) f_last[d] = f[d];
        memcpy(u_p, u_c, sizeof(double) * (size_t)n_dof);
        memcpy(u_c, u_n, sizeof(double) * (size_t)n_dof);
        for (int64_t r = 0; r < n_rec; ++r) rec_out[s * n_rec + r] = u_c[rec_dof[r]];
    }
    free(f); free(u_n);
    return 0;
}

/* P(t) of one wavelet (exported for tests). */
double oracle_load_amplitude(int kind, double t, double t1, double ncyc)
{
    return load_amplitude(kind, t, t1, ncyc);
}

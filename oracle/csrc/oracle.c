/*
 * FP64 CPU oracle for all-edge spanning centrality (AESC).
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into liboracle.so, which
 * only the tests, the smoke check and the timed CPU baseline load. It shares
 * no code, header or constant with the CUDA library.
 *
 * Two routines:
 *
 *  oracle_series  -- the truncated graph traversal of Algorithm 2 (TGT),
 *                    written plainly: for every requested source v_i a dense
 *                    FP64 vector p(., v_i) is pushed hop by hop over the
 *                    edges (Algorithm 2's hop) and the per-edge half sums
 *                    g(v_i, v_j) of Eq. (9) are accumulated (Algorithm 2's accumulation).
 *                    Truncation is per CSR entry: entry k = (i -> j) keeps
 *                    the terms with hop l <= tau[k]. The terms at
 *                    hops tau[k]+1 and tau[k]+2 are also returned (they feed
 *                    the a-posteriori tail check derived from the proof of
 *                    Theorem 3.2).
 *
 *  oracle_cg      -- the exact effective resistance r(i, j) =
 *                    (e_i - e_j)^T L^+ (e_i - e_j) (Section 2.3, the
 *                    equivalence SC = ER) by Jacobi-preconditioned conjugate
 *                    gradients on L x = e_i - e_j, one independent solve per
 *                    requested pair.
 *  oracle_cg_block -- the same solves, eight pairs side by side per thread
 *                    (bit for bit oracle_cg's values, fewer passes over the CSR).
 *
 * Both parallelise with OpenMP over independent sources / pairs only; every
 * per-source computation is sequential and in the order the paper states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/*
 * Algorithm 2 (TGT) for the sources listed in `sources`.
 *
 *   n, row_ptr, col_idx : symmetric CSR of G (rows sorted, no self loops)
 *   tau                 : per CSR entry truncation length tau_k (>= 0)
 *   extra_steps         : hops run beyond max_k tau_k of the source's row
 *                         (2 lets the caller read the hop tau+1 and tau+2 terms)
 *   g_out               : per entry k in a source row, g_tau(v_i, v_j) of Eq. (9)
 *   t1_out, t2_out      : per entry (nullable), (p_l(v_i,v_i) - p_l(v_j,v_i)) / d(v_i)
 *                         at l = tau_k + 1 and l = tau_k + 2
 * Returns 0, or -1 on a bad argument / allocation failure.
 */
int oracle_series(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                  const int32_t *tau, int32_t extra_steps, int32_t nsrc,
                  const int32_t *sources, double *g_out, double *t1_out,
                  double *t2_out, int32_t nthreads)
{
    if (n <= 0 || !row_ptr || !col_idx || !tau || !sources || !g_out || nsrc < 0 ||
        extra_steps < 0)
        return -1;
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *p_prev = (double *)malloc(sizeof(double) * (size_t)n);
        double *p_next = (double *)malloc(sizeof(double) * (size_t)n);
        if (!p_prev || !p_next) {
#pragma omp atomic write
            status = -1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int32_t si = 0; si < nsrc; ++si) {
                const int32_t i = sources[si];
                const int32_t k0 = row_ptr[i], k1 = row_ptr[i + 1];
                const double d_i = (double)(k1 - k0);
                /* initialisation: p_0(., v_i) = e_i */
                memset(p_prev, 0, sizeof(double) * (size_t)n);
                p_prev[i] = 1.0;
                /* hop 0 of Eq. (9): g(v_i, v_j) = p_0(v_i,v_i)/d(v_i) - p_0(v_j,v_i)/d(v_i) = 1/d(v_i) */
                int32_t tau_p = 0;
                for (int32_t k = k0; k < k1; ++k) {
                    g_out[k] = 1.0 / d_i;
                    if (t1_out) t1_out[k] = 0.0;
                    if (t2_out) t2_out[k] = 0.0;
                    if (tau[k] > tau_p) tau_p = tau[k]; /* the source's length: max over its edges */
                }
                const int32_t steps = tau_p + extra_steps;
                for (int32_t l = 1; l <= steps; ++l) {
                    /* hop l: p_l(., v_i) from p_{l-1}(., v_i) */
                    memset(p_next, 0, sizeof(double) * (size_t)n);
                    /* push p_{l-1}(v_j, v_i) / d(v_x) to every neighbour v_x of each v_j reached */
                    for (int32_t j = 0; j < n; ++j) {
                        const double pj = p_prev[j];
                        if (pj > 0.0) {
                            for (int32_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
                                const int32_t x = col_idx[e];
                                const double d_x = (double)(row_ptr[x + 1] - row_ptr[x]);
                                p_next[x] += pj / d_x;
                            }
                        }
                    }
                    /* Eq. (9): add hop l's term to every edge of v_i with l <= tau_ij */
                    for (int32_t k = k0; k < k1; ++k) {
                        const int32_t j = col_idx[k];
                        const double term = p_next[i] / d_i - p_next[j] / d_i;
                        if (l <= tau[k]) g_out[k] += term;
                        else if (l == tau[k] + 1) { if (t1_out) t1_out[k] = term; }
                        else if (l == tau[k] + 2) { if (t2_out) t2_out[k] = term; }
                    }
                    double *tmp = p_prev;
                    p_prev = p_next;
                    p_next = tmp;
                }
            }
        }
        free(p_prev);
        free(p_next);
    }
    return status;
}

/* y = L x for the combinatorial Laplacian L = D - A. */
static void lap_apply(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *x, double *y)
{
    for (int32_t r = 0; r < n; ++r) {
        double acc = (double)(row_ptr[r + 1] - row_ptr[r]) * x[r];
        for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
            acc -= x[col_idx[e]];
        y[r] = acc;
    }
}

/*
 * Exact effective resistance of each pair (u[q], v[q]) by Jacobi-preconditioned
 * CG on L x = e_u - e_v started from x = 0. The right-hand side is orthogonal
 * to the null space of L (the all-ones vector), so the system is consistent
 * and r = (e_u - e_v)^T x is independent of the null-space component of x.
 * Iterates until ||r_res|| <= rtol * ||b|| or max_iter.
 *   r_out[q]     : resistance
 *   iters_out[q] : iterations used (nullable); -1 if max_iter was hit
 */
int oracle_cg(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t npairs,
              const int32_t *u, const int32_t *v, double rtol, int32_t max_iter,
              double *r_out, int32_t *iters_out, int32_t nthreads)
{
    if (n <= 0 || !row_ptr || !col_idx || !u || !v || !r_out || npairs < 0)
        return -1;
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *x = (double *)malloc(sizeof(double) * (size_t)n);
        double *r = (double *)malloc(sizeof(double) * (size_t)n);
        double *z = (double *)malloc(sizeof(double) * (size_t)n);
        double *p = (double *)malloc(sizeof(double) * (size_t)n);
        double *q = (double *)malloc(sizeof(double) * (size_t)n);
        if (!x || !r || !z || !p || !q) {
#pragma omp atomic write
            status = -1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int32_t t = 0; t < npairs; ++t) {
                const int32_t a = u[t], b = v[t];
                memset(x, 0, sizeof(double) * (size_t)n);
                memset(r, 0, sizeof(double) * (size_t)n);
                r[a] += 1.0;
                r[b] -= 1.0;
                const double bnorm = sqrt(2.0);
                double rz = 0.0;
                for (int32_t i = 0; i < n; ++i) {
                    z[i] = r[i] / (double)(row_ptr[i + 1] - row_ptr[i]);
                    p[i] = z[i];
                    rz += r[i] * z[i];
                }
                int32_t it = 0;
                int converged = 0;
                for (it = 0; it < max_iter; ++it) {
                    double rn = 0.0;
                    for (int32_t i = 0; i < n; ++i) rn += r[i] * r[i];
                    if (sqrt(rn) <= rtol * bnorm) { converged = 1; break; }
                    lap_apply(n, row_ptr, col_idx, p, q);
                    double pq = 0.0;
                    for (int32_t i = 0; i < n; ++i) pq += p[i] * q[i];
                    const double alpha = rz / pq;
                    for (int32_t i = 0; i < n; ++i) {
                        x[i] += alpha * p[i];
                        r[i] -= alpha * q[i];
                    }
                    double rz_new = 0.0;
                    for (int32_t i = 0; i < n; ++i) {
                        z[i] = r[i] / (double)(row_ptr[i + 1] - row_ptr[i]);
                        rz_new += r[i] * z[i];
                    }
                    const double beta = rz_new / rz;
                    rz = rz_new;
                    for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
                }
                r_out[t] = x[a] - x[b];
                if (iters_out) iters_out[t] = converged ? it : -1;
            }
        }
        free(x); free(r); free(z); free(p); free(q);
    }
    return status;
}

/*
 * oracle_cg with CG_W pairs solved side by side per thread: the vectors are
 * n x CG_W row-major, so one pass of the Laplacian product gathers a node's
 * CG_W values from one cache line, and the vector updates of one iteration
 * share two passes. Every column runs the operations of oracle_cg: each sum
 * (over i, and over a row's entries) keeps its order; a column that meets the
 * tolerance is frozen (alpha = beta = 0 leave x and r unchanged), so each
 * resistance and iteration count equals oracle_cg's.
 */
#define CG_W 8
int oracle_cg_block(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t npairs,
                    const int32_t *u, const int32_t *v, double rtol, int32_t max_iter,
                    double *r_out, int32_t *iters_out, int32_t nthreads)
{
    if (n <= 0 || !row_ptr || !col_idx || !u || !v || !r_out || npairs < 0)
        return -1;
    int status = 0;
    const int32_t ngroups = (npairs + CG_W - 1) / CG_W;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        const size_t len = sizeof(double) * (size_t)n * CG_W;
        double *x = (double *)malloc(len), *r = (double *)malloc(len), *z = (double *)malloc(len);
        double *p = (double *)malloc(len), *q = (double *)malloc(len);
        if (!x || !r || !z || !p || !q) {
#pragma omp atomic write
            status = -1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int32_t grp = 0; grp < ngroups; ++grp) {
                const int32_t t0 = grp * CG_W;
                const int w = (npairs - t0) < CG_W ? (int)(npairs - t0) : CG_W;
                int32_t a[CG_W], b[CG_W], its[CG_W];
                int active[CG_W], conv[CG_W];
                double rz[CG_W], rn[CG_W], pq[CG_W], alpha[CG_W], rzn[CG_W], beta[CG_W];
                memset(x, 0, len);
                memset(r, 0, len);
                for (int c = 0; c < CG_W; ++c) {
                    active[c] = c < w;
                    conv[c] = 0;
                    its[c] = 0;
                    a[c] = c < w ? u[t0 + c] : 0;
                    b[c] = c < w ? v[t0 + c] : 0;
                    if (c < w) {
                        r[(size_t)a[c] * CG_W + c] += 1.0;
                        r[(size_t)b[c] * CG_W + c] -= 1.0;
                    }
                    rz[c] = 0.0;
                    rn[c] = 0.0;
                }
                const double bnorm = sqrt(2.0);
                /* z = D^-1 r, p = z, rz = r.z, rn = r.r */
                for (int32_t i = 0; i < n; ++i) {
                    const double di = (double)(row_ptr[i + 1] - row_ptr[i]);
                    double *ri = r + (size_t)i * CG_W, *zi = z + (size_t)i * CG_W, *pi = p + (size_t)i * CG_W;
                    for (int c = 0; c < CG_W; ++c) {
                        zi[c] = ri[c] / di;
                        pi[c] = zi[c];
                        rz[c] += ri[c] * zi[c];
                        rn[c] += ri[c] * ri[c];
                    }
                }
                for (int32_t it = 0; it < max_iter; ++it) {
                    int any = 0;
                    for (int c = 0; c < CG_W; ++c) {
                        if (active[c] && sqrt(rn[c]) <= rtol * bnorm) {
                            active[c] = 0;
                            conv[c] = 1;
                            its[c] = it;
                        }
                        any |= active[c];
                        pq[c] = 0.0;
                    }
                    if (!any) break;
                    /* q = L p (each column's row sum in CSR order), pq = p.q */
                    for (int32_t i = 0; i < n; ++i) {
                        const double di = (double)(row_ptr[i + 1] - row_ptr[i]);
                        const double *pi = p + (size_t)i * CG_W;
                        double acc[CG_W];
                        for (int c = 0; c < CG_W; ++c) acc[c] = di * pi[c];
                        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                            const double *pj = p + (size_t)col_idx[e] * CG_W;
                            for (int c = 0; c < CG_W; ++c) acc[c] -= pj[c];
                        }
                        double *qi = q + (size_t)i * CG_W;
                        for (int c = 0; c < CG_W; ++c) {
                            qi[c] = acc[c];
                            pq[c] += pi[c] * acc[c];
                        }
                    }
                    for (int c = 0; c < CG_W; ++c) {
                        alpha[c] = active[c] ? rz[c] / pq[c] : 0.0;
                        rzn[c] = 0.0;
                        rn[c] = 0.0;
                    }
                    /* x += alpha p, r -= alpha q, z = D^-1 r, rz_new = r.z, and the next check's r.r */
                    for (int32_t i = 0; i < n; ++i) {
                        const double di = (double)(row_ptr[i + 1] - row_ptr[i]);
                        const size_t o = (size_t)i * CG_W;
                        for (int c = 0; c < CG_W; ++c) {
                            x[o + c] += alpha[c] * p[o + c];
                            r[o + c] -= alpha[c] * q[o + c];
                            z[o + c] = r[o + c] / di;
                            rzn[c] += r[o + c] * z[o + c];
                            rn[c] += r[o + c] * r[o + c];
                        }
                    }
                    for (int c = 0; c < CG_W; ++c) {
                        beta[c] = active[c] ? rzn[c] / rz[c] : 0.0;
                        if (active[c]) rz[c] = rzn[c];
                    }
                    for (size_t o = 0; o < (size_t)n * CG_W; o += CG_W)
                        for (int c = 0; c < CG_W; ++c) p[o + c] = z[o + c] + beta[c] * p[o + c];
                }
                for (int c = 0; c < w; ++c) {
                    r_out[t0 + c] = x[(size_t)a[c] * CG_W + c] - x[(size_t)b[c] * CG_W + c];
                    if (iters_out) iters_out[t0 + c] = conv[c] ? its[c] : -1;
                }
            }
        }
        free(x); free(r); free(z); free(p); free(q);
    }
    return status;
}

/*
 * Per-hop half terms of Algorithm 2 for the sources listed: for entry k = (i -> j)
 * of a source row, out[k_local * (L + 1) + l] = (p_l(v_i,v_i) - p_l(v_j,v_i)) / d(v_i)
 * for l = 0..L, where k_local = k - row_ptr[i] + row_off[si] (row_off: prefix of the
 * sources' degrees). Used to find, per edge, the least odd length whose
 * a-posteriori tail bound meets eps.
 */
int oracle_series_terms(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t L, int32_t nsrc,
                        const int32_t *sources, const int64_t *row_off, double *out, int32_t nthreads)
{
    if (n <= 0 || !row_ptr || !col_idx || !sources || !row_off || !out || L < 0 || nsrc < 0)
        return -1;
    int status = 0;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *p_prev = (double *)malloc(sizeof(double) * (size_t)n);
        double *p_next = (double *)malloc(sizeof(double) * (size_t)n);
        if (!p_prev || !p_next) {
#pragma omp atomic write
            status = -1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int32_t si = 0; si < nsrc; ++si) {
                const int32_t i = sources[si];
                const int32_t k0 = row_ptr[i], k1 = row_ptr[i + 1];
                const double d_i = (double)(k1 - k0);
                double *o = out + row_off[si] * (int64_t)(L + 1);
                memset(p_prev, 0, sizeof(double) * (size_t)n);
                p_prev[i] = 1.0;
                for (int32_t k = k0; k < k1; ++k) o[(int64_t)(k - k0) * (L + 1)] = 1.0 / d_i;
                for (int32_t l = 1; l <= L; ++l) {
                    memset(p_next, 0, sizeof(double) * (size_t)n);
                    for (int32_t j = 0; j < n; ++j) {
                        const double pj = p_prev[j];
                        if (pj > 0.0) {
                            for (int32_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
                                const int32_t x = col_idx[e];
                                p_next[x] += pj / (double)(row_ptr[x + 1] - row_ptr[x]);
                            }
                        }
                    }
                    for (int32_t k = k0; k < k1; ++k)
                        o[(int64_t)(k - k0) * (L + 1) + l] = p_next[i] / d_i - p_next[col_idx[k]] / d_i;
                    double *tmp = p_prev;
                    p_prev = p_next;
                    p_next = tmp;
                }
            }
        }
        free(p_prev);
        free(p_next);
    }
    return status;
}

// Eigenvalue bound (step A2) and truncation lengths (step A3).
//
// A2: spectrum extremes of N = D^{-1/2} A D^{-1/2} (similar to P; Lemma 3.1)
//     by FP64 Lanczos with full (twice-applied classical Gram-Schmidt)
//     reorthogonalisation. The top eigenvector sqrt(d)/sqrt(2m) (eigenvalue
//     1) and, for a bipartite graph, the bottom one (eigenvalue -1, signs by
//     BFS level parity) are kept as locked leading basis vectors, so the
//     Krylov space never contains them. The tridiagonal Ritz problem is
//     solved on the host (Sturm bisection for the two extreme Ritz values,
//     inverse iteration for the last component of their Ritz vectors).
// A3: Eq. (6) with omega = 2, Upsilon = Delta_t = 0 (Algorithm 1's initial length), rounded
//     up to an odd integer (Eq. 5); per-source maximum (Algorithm 2's per-source length).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "philox.cuh"

namespace sc {

// ---------------------------------------------------------------------------
// A3: truncation length per CSR entry
// ---------------------------------------------------------------------------
// one warp per row (grid-stride over rows): the lanes take the row's entries
// (hub rows are long); the longest length goes through one atomic per CTA
__global__ void k_tau_entries(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                              double eps, double lam, int32_t *__restrict__ tau, int32_t *__restrict__ tau_src,
                              int32_t *ell_global) {
    __shared__ int32_t cta_best;
    if (threadIdx.x == 0) cta_best = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const double denom = __dmul_rn(eps, __dsub_rn(1.0, __dmul_rn(lam, lam)));
    const double log_inv_lam = log(__ddiv_rn(1.0, lam));
    int32_t warp_best = 0;
    for (int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += gridDim.x * (blockDim.x >> 5)) {
        const double di = static_cast<double>(row_ptr[r + 1] - row_ptr[r]);
        int32_t best = 0;
        for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
            const int32_t j = col[k];
            const double dj = static_cast<double>(row_ptr[j + 1] - row_ptr[j]);
            // X_e = 1/d_i + 1/d_j - 2/(d_i d_j), evaluated left to right without contraction
            const double xe =
                __dsub_rn(__dadd_rn(__ddiv_rn(1.0, di), __ddiv_rn(1.0, dj)), __ddiv_rn(2.0, __dmul_rn(di, dj)));
            int32_t t = 1;
            if (xe > 0.0 && lam > 0.0) {
                const double val = __dsub_rn(__ddiv_rn(log(__ddiv_rn(xe, denom)), log_inv_lam), 1.0);
                const double f = ceil(val);
                if (f > 1.0) t = f > 2.0e9 ? 2000000001 : static_cast<int32_t>(f);
            }
            if ((t & 1) == 0) t += 1;
            tau[k] = t;
            best = max(best, t);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) tau_src[r] = best;
        warp_best = max(warp_best, best);
    }
    if (lane == 0) atomicMax(&cta_best, warp_best);
    __syncthreads();
    if (threadIdx.x == 0 && cta_best > 0) atomicMax(ell_global, cta_best);
}

void tau_entries_device(sc_graph *g, double eps, double lam_star, int32_t *tau_entry, int32_t *tau_src,
                        int32_t *ell_global_host) {
    if (!(lam_star < 1.0)) SC_FAIL(SC_ERR_UNSUPPORTED, "lambda_star >= 1: the series does not converge");
    g->status.reserve(4);
    cudaStream_t s = g->stream;
    SC_CUDA(cudaMemsetAsync(g->status.get(), 0, sizeof(int32_t), s));
    const int grid = std::max(1, std::min(ceil_div(g->n, 8), (g->num_sms > 0 ? g->num_sms : 148) * 8));
    k_tau_entries<<<grid, 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), g->n, eps,
                                                       std::max(lam_star, 0.0), tau_entry, tau_src, g->status.get());
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaMemcpyAsync(ell_global_host, g->status.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// A2: Lanczos kernels (FP64, deterministic reductions)
// ---------------------------------------------------------------------------
constexpr int kDotBlocks = 256, kDotThreads = 256;

// y = D^-1/2 A D^-1/2 x, one warp per row, fixed shuffle tree
__global__ void k_spmv_norm(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                            const double *__restrict__ isd, const double *__restrict__ x, double *__restrict__ y,
                            int32_t n) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    double acc = 0.0;
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        const int32_t j = col[k];
        acc += isd[j] * x[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[r] = isd[r] * acc;
}

// partial[q * kDotBlocks + b] = block b's share of <V_q, w>, for q < nvec
__global__ void k_multidot_partial(const double *__restrict__ V, int64_t ldv, int nvec, const double *__restrict__ w,
                                   int32_t n, double *__restrict__ partial) {
    __shared__ double sh[kDotThreads];
    const int q = blockIdx.y;
    const double *v = V + q * ldv;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads)
        acc += v[i] * w[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kDotThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[q * kDotBlocks + blockIdx.x] = sh[0];
}

// out[q] = sum of the kDotBlocks partials of row q (fixed tree)
__global__ void k_multidot_final(const double *__restrict__ partial, double *__restrict__ out) {
    __shared__ double sh[kDotBlocks];
    const int q = blockIdx.x;
    sh[threadIdx.x] = partial[q * kDotBlocks + threadIdx.x];
    __syncthreads();
    for (int s = kDotBlocks / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}

// w -= sum_q c[q] V_q (q in order)
__global__ void k_sub_combination(const double *__restrict__ V, int64_t ldv, int nvec, const double *__restrict__ c,
                                  double *__restrict__ w, int32_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = w[i];
    for (int q = 0; q < nvec; ++q) acc -= c[q] * V[q * ldv + i];
    w[i] = acc;
}

// dst = src * (1 / nrm), nrm read from the device
__global__ void k_scale_into(const double *__restrict__ src, const double *__restrict__ nrm2, double *__restrict__ dst,
                             int32_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[i] = src[i] / sqrt(*nrm2);
}

// alpha of a Lanczos step: the coefficients of V_vj in the two orthogonalisation passes, summed
__global__ void k_alpha_of(const double *__restrict__ c, int nbasis, int vj, double *__restrict__ alpha) {
    *alpha = c[vj] + c[nbasis + vj];
}

// locked vectors: sqrt(d_x)/sqrt(2m), and (bipartite) the same with sign (-1)^level
__global__ void k_locked_vectors(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ level, int32_t n,
                                 double inv_sqrt_2m, int bipartite, double *__restrict__ v0, double *__restrict__ v1,
                                 double *__restrict__ isd) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = static_cast<double>(row_ptr[i + 1] - row_ptr[i]);
    const double sd = sqrt(d);
    isd[i] = 1.0 / sd;
    v0[i] = sd * inv_sqrt_2m;
    if (bipartite) v1[i] = ((level[i] & 1) ? -sd : sd) * inv_sqrt_2m;
}

// start vector: Philox4x32-10 uniform in [-1, 1), counter = node index
__global__ void k_start_vector(double *__restrict__ v, int32_t n, uint32_t k0, uint32_t k1) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Philox4 r = philox4x32_10(static_cast<uint32_t>(i), 0x4c414e43u /* stream tag */, 0u, 0u, k0, k1);
    v[i] = 2.0 * u01_53(r.v[0], r.v[1]) - 1.0;
}

// ---------------------------------------------------------------------------
// host: tridiagonal Ritz problem (alpha[0..k-1] diagonal, beta[1..k-1] off-diagonal)
// ---------------------------------------------------------------------------
// number of eigenvalues of T below x (Sturm count through the LDL^T pivots)
static int sturm_count(const std::vector<double> &a, const std::vector<double> &b, int k, double x) {
    int cnt = 0;
    double q = a[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < k; ++i) {
        if (q == 0.0) q = 1e-300;
        q = (a[i] - x) - b[i] * b[i] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// eigenvalue of index idx (0 = smallest) by bisection on [lo, hi]
static double bisect_eig(const std::vector<double> &a, const std::vector<double> &b, int k, int idx, double lo,
                         double hi) {
    for (int it = 0; it < 200 && hi - lo > 1e-17 * std::max(1.0, std::fabs(lo) + std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, k, mid) > idx) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// solve (T - theta I) y = rhs by Gaussian elimination with partial pivoting on the band
static void tridiag_solve(const std::vector<double> &a, const std::vector<double> &b, int k, double theta,
                          std::vector<double> &y) {
    // rows i: sub = b[i] (i>=1), diag = a[i]-theta, sup = b[i+1] (i < k-1)
    std::vector<double> d(k), u1(k, 0.0), u2(k, 0.0), l(k, 0.0);
    std::vector<char> swapped(k, 0);
    for (int i = 0; i < k; ++i) {
        d[i] = a[i] - theta;
        u1[i] = (i + 1 < k) ? b[i + 1] : 0.0;
    }
    // forward elimination with row interchanges (LAPACK gttrf style)
    std::vector<double> sub(k, 0.0);
    for (int i = 1; i < k; ++i) sub[i] = b[i];
    for (int i = 0; i + 1 < k; ++i) {
        if (std::fabs(d[i]) >= std::fabs(sub[i + 1])) {
            if (d[i] == 0.0) d[i] = 1e-300;
            const double f = sub[i + 1] / d[i];
            l[i] = f;
            d[i + 1] -= f * u1[i];
            y[i + 1] -= f * y[i];
            u2[i] = 0.0;
        } else {
            // swap rows i and i+1
            const double f = d[i] / sub[i + 1];
            swapped[i] = 1;
            d[i] = sub[i + 1];
            const double t_u1 = u1[i];
            u1[i] = d[i + 1];
            const double t_u2 = (i + 2 < k) ? u1[i + 1] : 0.0;
            u2[i] = t_u2;
            d[i + 1] = t_u1 - f * u1[i];
            if (i + 2 < k) u1[i + 1] = -f * t_u2;
            std::swap(y[i], y[i + 1]);
            y[i + 1] -= f * y[i];
            l[i] = f;
        }
    }
    if (d[k - 1] == 0.0) d[k - 1] = 1e-300;
    // back substitution
    y[k - 1] /= d[k - 1];
    if (k >= 2) y[k - 2] = (y[k - 2] - u1[k - 2] * y[k - 1]) / d[k - 2];
    for (int i = k - 3; i >= 0; --i) y[i] = (y[i] - u1[i] * y[i + 1] - u2[i] * y[i + 2]) / d[i];
}

// last component of the unit eigenvector of T for eigenvalue theta (inverse iteration)
static double ritz_last_component(const std::vector<double> &a, const std::vector<double> &b, int k, double theta) {
    if (k == 1) return 1.0;
    std::vector<double> y(k);
    for (int i = 0; i < k; ++i) y[i] = 1.0 / std::sqrt(static_cast<double>(k)) * (1.0 + 0.01 * ((i * 7919) % 13));
    const double shift = theta + 1e-13 * std::max(1.0, std::fabs(theta));
    for (int it = 0; it < 3; ++it) {
        tridiag_solve(a, b, k, shift, y);
        double nrm = 0.0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) return 1.0;
        for (double &v : y) v /= nrm;
    }
    return y[k - 1];
}

sc_status estimate_lambda_impl(sc_graph *g, const sc_lambda_opts *opts, sc_lambda *out) {
    return guarded([&] {
        if (!g || !out) SC_FAIL(SC_ERR_INVALID_ARG, "null argument");
        const int32_t n = g->n;
        const int nlock = g->bipartite ? 2 : 1;
        int max_iter = (opts && opts->max_iter > 0) ? opts->max_iter : 500;
        const double tol = (opts && opts->tol > 0) ? opts->tol : 1e-4;
        const uint64_t seed = opts ? opts->seed : 0x1a2b3c4dULL;
        max_iter = std::min(max_iter, n - nlock);
        if (max_iter < 1) SC_FAIL(SC_ERR_INVALID_ARG, "graph too small for Lanczos");
        cudaStream_t s = g->stream;
        const int64_t ldv = (static_cast<int64_t>(n) + 31) / 32 * 32;
        const int nbasis = nlock + max_iter + 1;
        DevBuf<double> V, w, isd, c, partial;
        V.reserve(static_cast<size_t>(nbasis) * ldv);
        w.reserve(n);
        isd.reserve(n);
        c.reserve(2 * nbasis + 8);
        partial.reserve(static_cast<size_t>(nbasis) * kDotBlocks);
        const int tb = 256;
        const int nb = ceil_div(n, tb);
        const double inv_sqrt_2m = 1.0 / std::sqrt(static_cast<double>(g->nnz));
        k_locked_vectors<<<nb, tb, 0, s>>>(g->row_ptr.get(), g->level.get(), n, inv_sqrt_2m, g->bipartite, V.get(),
                                           V.get() + ldv, isd.get());
        SC_LAUNCH_CHECK();

        // orthogonalise w against V[0..nv) twice (CGS2); the coefficients of the
        // two passes are c[0..nv) and c[nbasis..nbasis + nv)
        auto reorth = [&](int nv) {
            for (int pass = 0; pass < 2; ++pass) {
                double *cc = c.get() + (pass ? nbasis : 0);
                k_multidot_partial<<<dim3(kDotBlocks, nv), kDotThreads, 0, s>>>(V.get(), ldv, nv, w.get(), n, partial.get());
                k_multidot_final<<<nv, kDotBlocks, 0, s>>>(partial.get(), cc);
                k_sub_combination<<<nb, tb, 0, s>>>(V.get(), ldv, nv, cc, w.get(), n);
                SC_LAUNCH_CHECK();
            }
        };
        auto norm2_into = [&](double *dst) {  // dst = <w, w> on the device
            k_multidot_partial<<<dim3(kDotBlocks, 1), kDotThreads, 0, s>>>(w.get(), ldv, 1, w.get(), n, partial.get());
            k_multidot_final<<<1, kDotBlocks, 0, s>>>(partial.get(), dst);
            SC_LAUNCH_CHECK();
        };

        // start vector
        k_start_vector<<<nb, tb, 0, s>>>(w.get(), n, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
        SC_LAUNCH_CHECK();
        reorth(nlock);
        double *nrm_dev = c.get() + 2 * nbasis;
        norm2_into(nrm_dev);
        k_scale_into<<<nb, tb, 0, s>>>(w.get(), nrm_dev, V.get() + nlock * ldv, n);
        SC_LAUNCH_CHECK();

        // alpha_j and |w_j|^2 of every step stay on the device; the host reads
        // them only at the steps where it checks convergence (every 4th from
        // step 8, and the last possible one), so the steps in between run with
        // no synchronisation. A breakdown (|w_j| <= 1e-12) between two checks is
        // found at the next one and the steps after it are discarded, which
        // gives the same steps and result as stopping at the breakdown itself.
        DevBuf<double> ab;
        ab.reserve(2 * static_cast<size_t>(max_iter));
        double *d_alpha = ab.get(), *d_nrm2 = ab.get() + max_iter;
        std::vector<double> alpha, beta(1, 0.0), h_alpha, h_nrm2;
        double theta_max = 0, theta_min = 0, res_max = INFINITY, res_min = INFINITY;
        int k = 0;
        bool converged = false;
        for (int j = 0; j < max_iter; ++j) {
            const int vj = nlock + j;
            k_spmv_norm<<<ceil_div(n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), isd.get(),
                                                        V.get() + vj * ldv, w.get(), n);
            SC_LAUNCH_CHECK();
            reorth(vj + 1);
            k_alpha_of<<<1, 1, 0, s>>>(c.get(), nbasis, vj, d_alpha + j);  // both passes' coefficient of V_vj
            norm2_into(d_nrm2 + j);
            const int kk = j + 1;
            if (kk == max_iter || kk == n - nlock || (kk >= 8 && kk % 4 == 0)) {
                h_alpha.resize(kk);
                h_nrm2.resize(kk);
                SC_CUDA(cudaMemcpyAsync(h_alpha.data(), d_alpha, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
                SC_CUDA(cudaMemcpyAsync(h_nrm2.data(), d_nrm2, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
                SC_CUDA(cudaStreamSynchronize(s));
                bool exhausted = kk == n - nlock;
                int stop = kk;
                for (int q = static_cast<int>(alpha.size()); q < kk; ++q) {
                    alpha.push_back(h_alpha[q]);
                    const double b = std::sqrt(std::max(h_nrm2[q], 0.0));
                    if (!(b > 1e-12)) {  // breakdown at step q: the Krylov space is exhausted
                        stop = q + 1;
                        exhausted = true;
                        break;
                    }
                    if (q + 1 < kk) beta.push_back(b);
                }
                k = stop;
                const double bnext = std::sqrt(std::max(h_nrm2[stop - 1], 0.0));
                // extreme Ritz values and their residuals bnext * |y_k|
                theta_max = bisect_eig(alpha, beta, k, k - 1, -1.0 - 1e-9, 1.0 + 1e-9);
                theta_min = bisect_eig(alpha, beta, k, 0, -1.0 - 1e-9, 1.0 + 1e-9);
                res_max = exhausted ? 0.0 : bnext * std::fabs(ritz_last_component(alpha, beta, k, theta_max));
                res_min = exhausted ? 0.0 : bnext * std::fabs(ritz_last_component(alpha, beta, k, theta_min));
                if (res_max <= tol && res_min <= tol) {
                    converged = true;
                    break;
                }
                if (exhausted) break;
                beta.push_back(bnext);
            }
            k = kk;
            k_scale_into<<<nb, tb, 0, s>>>(w.get(), d_nrm2 + j, V.get() + (vj + 1) * ldv, n);
            SC_LAUNCH_CHECK();
        }
        out->lambda_plus = theta_max;
        out->lambda_minus = theta_min;
        out->residual_plus = res_max;
        out->residual_minus = res_min;
        out->lambda_star = std::max(std::fabs(theta_max), std::fabs(theta_min)) + std::max(res_max, res_min);
        out->iterations = k;
        out->converged = converged ? 1 : 0;
        g->lam = *out;
        g->has_lambda = true;
        if (!converged)
            SC_FAIL(SC_ERR_LAMBDA_NOT_CONVERGED, "Lanczos residuals %.3g / %.3g above %.3g after %d steps", res_max,
                    res_min, tol, k);
    });
}

}  // namespace sc

extern "C" {

sc_status sc_estimate_lambda(sc_graph *g, const sc_lambda_opts *opts, sc_lambda *out) {
    return sc::estimate_lambda_impl(g, opts, out);
}

sc_status sc_truncation_length(sc_graph *g, double eps, const sc_lambda *lam, int32_t *ell_global_out,
                               int32_t *per_source_out, int32_t *per_entry_out) {
    return sc::guarded([&] {
        if (!g) SC_FAIL(SC_ERR_INVALID_ARG, "null graph");
        if (!(eps > 0.0 && eps < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "eps must lie in (0, 1)");
        const sc_lambda *l = lam ? lam : (g->has_lambda ? &g->lam : nullptr);
        if (!l) SC_FAIL(SC_ERR_INVALID_ARG, "no eigenvalue estimate: call sc_estimate_lambda first");
        if (!(l->lambda_star < 1.0)) SC_FAIL(SC_ERR_UNSUPPORTED, "lambda_star >= 1: no finite truncation length");
        sc::DevBuf<int32_t> te, ts;
        te.reserve(g->nnz);
        ts.reserve(g->n);
        int32_t ell = 0;
        sc::tau_entries_device(g, eps, l->lambda_star, te.get(), ts.get(), &ell);
        if (ell_global_out) *ell_global_out = ell;
        if (per_source_out)
            SC_CUDA(cudaMemcpyAsync(per_source_out, ts.get(), g->n * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
        if (per_entry_out)
            SC_CUDA(cudaMemcpyAsync(per_entry_out, te.get(), g->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
        SC_CUDA(cudaStreamSynchronize(g->stream));
    });
}

}  // extern "C"

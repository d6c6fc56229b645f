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

// partial[q * kDotBlocks + b] = block b's share of <V_q, w>, for q < nvec:
// block b takes rows [b c, (b + 1) c) (c = ceil(n / kDotBlocks)), its warps
// take the vectors q = warp, warp + 8, ..., each lane a strided share of the
// rows in order, then a fixed shuffle tree. One launch of kDotBlocks blocks
// for every vector of the basis (the rows of w it reads stay in L1).
// skip (nullable): when *skip != 0 the launch does nothing (a pass the device
// decided against).
__global__ void k_multidot_partial(const double *__restrict__ V, int64_t ldv, int nvec, const double *__restrict__ w,
                                   int32_t n, double *__restrict__ partial, const int *__restrict__ skip = nullptr) {
    if (skip && *skip) return;
    const int64_t c = (static_cast<int64_t>(n) + kDotBlocks - 1) / kDotBlocks;
    const int64_t i0 = blockIdx.x * c, i1 = min(static_cast<int64_t>(n), i0 + c);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kDotThreads / 32;
    for (int q = warp; q < nvec; q += nw) {
        const double *v = V + q * ldv;
        double acc = 0.0;
        for (int64_t i = i0 + lane; i < i1; i += 32) acc += v[i] * w[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) partial[q * kDotBlocks + blockIdx.x] = acc;
    }
}

// out[q] = sum of the kDotBlocks partials of row q (fixed tree); 0 when *skip
__global__ void k_multidot_final(const double *__restrict__ partial, double *__restrict__ out,
                                 const int *__restrict__ skip = nullptr) {
    __shared__ double sh[kDotBlocks];
    const int q = blockIdx.x;
    if (skip && *skip) {
        if (threadIdx.x == 0) out[q] = 0.0;
        return;
    }
    sh[threadIdx.x] = partial[q * kDotBlocks + threadIdx.x];
    __syncthreads();
    for (int s = kDotBlocks / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
}

// w -= sum_q c[q] V_q (q in order); nothing when *skip
__global__ void k_sub_combination(const double *__restrict__ V, int64_t ldv, int nvec, const double *__restrict__ c,
                                  double *__restrict__ w, int32_t n, const int *__restrict__ skip = nullptr) {
    if (skip && *skip) return;
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

// The three-term part of a Lanczos step: w -= a V_vj + beta V_vj-1, with a =
// <w, V_vj> (from the device) and beta = sqrt(|w_prev|^2) (nrm2_prev null:
// no previous Lanczos vector, the first step)
__global__ void k_three_term(const double *__restrict__ V, int64_t ldv, int vj, const double *__restrict__ a,
                             const double *__restrict__ nrm2_prev, double *__restrict__ w, int32_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = w[i] - *a * V[vj * ldv + i];
    if (nrm2_prev) acc -= sqrt(*nrm2_prev) * V[(vj - 1) * ldv + i];
    w[i] = acc;
}

// skip the second sweep unless the first removed more than half of |w|^2
// ("twice is enough": one more sweep restores orthogonality to working
// precision when the first lost most of the vector)
__global__ void k_second_sweep_flag(const double *__restrict__ nrm2_before, const double *__restrict__ nrm2_after,
                                    int *__restrict__ skip) {
    *skip = (*nrm2_after < 0.5 * *nrm2_before) ? 0 : 1;
}

// alpha of a step with the three-term part: its coefficient plus the sweeps' coefficients of V_vj
__global__ void k_alpha_three(const double *__restrict__ a, const double *__restrict__ c, int nbasis, int vj,
                              double *__restrict__ alpha) {
    *alpha = *a + c[vj] + c[nbasis + vj];
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
                k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(V.get(), ldv, nv, w.get(), n, partial.get());
                k_multidot_final<<<nv, kDotBlocks, 0, s>>>(partial.get(), cc);
                k_sub_combination<<<nb, tb, 0, s>>>(V.get(), ldv, nv, cc, w.get(), n);
                SC_LAUNCH_CHECK();
            }
        };
        auto norm2_into = [&](double *dst) {  // dst = <w, w> on the device
            k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(w.get(), ldv, 1, w.get(), n, partial.get());
            k_multidot_final<<<1, kDotBlocks, 0, s>>>(partial.get(), dst);
            SC_LAUNCH_CHECK();
        };
        // A Lanczos step's orthogonalisation: the three-term recurrence first (w -= a V_vj +
        // beta V_vj-1), then one classical Gram-Schmidt sweep against the whole basis, and a
        // second sweep only when the first removed more than half of |w|^2 (decided on the
        // device: the skipped sweep's launches return at once and its coefficients are 0). In
        // exact arithmetic the recurrence leaves w orthogonal to the basis; the sweep removes
        // what rounding left, so the second sweep is rarely needed and a step costs about
        // half the FP64 work of two full sweeps.
        double *d_scal = nullptr;  // [0] a, [1] |w|^2 before the sweep, [2] after it
        DevBuf<double> scal;
        DevBuf<int> skip;
        scal.reserve(4);
        skip.reserve(1);
        d_scal = scal.get();
        auto step_orth = [&](int vj, const double *nrm2_prev) {
            k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(V.get() + vj * ldv, ldv, 1, w.get(), n,
                                                                          partial.get());
            k_multidot_final<<<1, kDotBlocks, 0, s>>>(partial.get(), d_scal);
            k_three_term<<<nb, tb, 0, s>>>(V.get(), ldv, vj, d_scal, nrm2_prev, w.get(), n);
            SC_LAUNCH_CHECK();
            norm2_into(d_scal + 1);
            const int nv = vj + 1;
            k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(V.get(), ldv, nv, w.get(), n, partial.get());
            k_multidot_final<<<nv, kDotBlocks, 0, s>>>(partial.get(), c.get());
            k_sub_combination<<<nb, tb, 0, s>>>(V.get(), ldv, nv, c.get(), w.get(), n);
            SC_LAUNCH_CHECK();
            norm2_into(d_scal + 2);
            k_second_sweep_flag<<<1, 1, 0, s>>>(d_scal + 1, d_scal + 2, skip.get());
            double *c2 = c.get() + nbasis;
            k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(V.get(), ldv, nv, w.get(), n, partial.get(),
                                                                           skip.get());
            k_multidot_final<<<nv, kDotBlocks, 0, s>>>(partial.get(), c2, skip.get());
            k_sub_combination<<<nb, tb, 0, s>>>(V.get(), ldv, nv, c2, w.get(), n, skip.get());
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
            step_orth(vj, j > 0 ? d_nrm2 + (j - 1) : nullptr);
            k_alpha_three<<<1, 1, 0, s>>>(d_scal, c.get(), nbasis, vj, d_alpha + j);
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

sc_status sc_graph_set_lambda(sc_graph *g, const sc_lambda *lam) {
    return sc::guarded([&] {
        if (!g || !lam) SC_FAIL(SC_ERR_INVALID_ARG, "null graph or lambda");
        const double ls = lam->lambda_star;
        if (!(ls >= 0.0 && ls <= 1.0) || !(std::fabs(lam->lambda_plus) <= ls) ||
            (!g->bipartite && !(std::fabs(lam->lambda_minus) <= ls)))
            SC_FAIL(SC_ERR_INVALID_ARG, "need 0 <= lambda_star <= 1 bounding |lambda_plus| (and |lambda_minus| "
                                        "on a graph that is not bipartite), got %g, %g, %g",
                    lam->lambda_plus, lam->lambda_minus, ls);
        g->lam = *lam;
        g->has_lambda = true;
    });
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

// ===========================================================================
// CalTau with omega eigenpairs (Algorithm 1, Eq. 6-8)
// ===========================================================================
//
// Eigenpairs: Lanczos run 1 (lambda_1's vector locked) keeps its basis; the
// tridiagonal Ritz problem is solved whole on the host (implicit symmetric QR);
// the Ritz pairs among the omega - 1 largest moduli whose residual meets the
// tolerance are the set U taken exactly. Their Ritz vectors (basis times the
// tridiagonal eigenvectors) are locked into Lanczos run 2, which starts from a
// fresh vector and so sees every mode outside U, the copies of a repeated
// eigenvalue that run 1's single Krylov sequence holds one vector of included:
// its extreme Ritz values give r, the bound on every mode left out. The proof
// of Theorem 3.2 bounds each left-out term by r^(t+1) / (1 - r^2) c_k (1 +
// lambda_k), which is what makes any such U admissible.
//
// CalTau per edge: one warp per edge (i < j), lanes over the modes of U
// (f_k node-major, so an edge reads two contiguous rows): c_k, Upsilon (Eq.
// 7), then Delta_t (Eq. 8) for t = 1, 3, 5, ... with one fixed-order warp sum
// per t until Eq. 6 with the remainder no longer reaches t.
#include <limits>
#include <numeric>

namespace sc {

constexpr int kOmegaMax = SC_OMEGA_MAX;              // pairs, lambda_1 included
constexpr int kModesPerLane = (kOmegaMax - 1 + 31) / 32;  // nontrivial modes per lane
constexpr int32_t kCalTauMaxLen = 1 << 20;

// Every eigenpair of the symmetric tridiagonal matrix with diagonal a[0..k)
// and off-diagonal e[0..k-1) (e[i] couples i and i + 1) by the implicit
// symmetric QR algorithm (Golub and Van Loan, Section 8.3): a Wilkinson shift
// from the trailing 2 x 2 block of the unreduced block [lo, hi], one Givens
// similarity on the shifted first column, then the bulge chased down by a
// rotation per row; an off-diagonal at or below machine precision times its two
// diagonal neighbours splits the matrix. Z (k x k, column-major, may be null)
// accumulates the rotations from the identity, so column q ends as the unit
// eigenvector of a[q]. Returns false when one eigenvalue takes more than 60 steps.
static bool tridiag_qr(int k, std::vector<double> &a, std::vector<double> &e, double *Z) {
    if (Z) {
        std::fill(Z, Z + static_cast<size_t>(k) * k, 0.0);
        for (int q = 0; q < k; ++q) Z[static_cast<size_t>(q) * k + q] = 1.0;
    }
    const double ulp = std::numeric_limits<double>::epsilon();
    auto negligible = [&](int i) {  // e[i] against a[i], a[i + 1]
        return std::fabs(e[i]) <= ulp * (std::fabs(a[i]) + std::fabs(a[i + 1])) || std::fabs(e[i]) < 1e-300;
    };
    int hi = k - 1, steps = 0;
    while (hi > 0) {
        if (negligible(hi - 1)) {
            e[hi - 1] = 0.0;
            --hi;
            steps = 0;
            continue;
        }
        if (++steps > 60) return false;
        int lo = hi - 1;
        while (lo > 0 && !negligible(lo - 1)) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        const double d = 0.5 * (a[hi - 1] - a[hi]);
        const double eh = e[hi - 1];
        const double mu = a[hi] - eh * eh / (d + std::copysign(std::hypot(d, eh), d));
        double x = a[lo] - mu, z = e[lo];
        for (int i = lo; i < hi; ++i) {
            const double r = std::hypot(x, z);
            const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? z / r : 0.0;
            if (i > lo) e[i - 1] = r;  // the bulge at (i - 1, i + 1) is now zero
            const double p = a[i], q = a[i + 1], b = e[i];
            a[i] = c * c * p + 2.0 * c * s * b + s * s * q;
            a[i + 1] = s * s * p - 2.0 * c * s * b + c * c * q;
            e[i] = c * s * (q - p) + (c * c - s * s) * b;
            if (i + 1 < hi) {  // the new bulge at (i, i + 2)
                x = e[i];
                z = s * e[i + 1];
                e[i + 1] *= c;
            }
            if (Z) {
                double *zi = Z + static_cast<size_t>(i) * k, *zj = zi + k;
                for (int row = 0; row < k; ++row) {
                    const double u = zi[row], v = zj[row];
                    zi[row] = c * u + s * v;
                    zj[row] = -s * u + c * v;
                }
            }
        }
    }
    return true;
}

// tridiag_qr, then the pairs in ascending order of eigenvalue
static bool tridiag_eig_sorted(int k, const double *alpha, const double *beta_off, std::vector<double> &theta,
                               std::vector<double> *Z) {
    std::vector<double> a(alpha, alpha + k), e(k > 1 ? k - 1 : 1, 0.0);
    for (int i = 0; i + 1 < k; ++i) e[i] = beta_off[i];
    std::vector<double> Zw;
    if (Z) Zw.resize(static_cast<size_t>(k) * k);
    if (!tridiag_qr(k, a, e, Z ? Zw.data() : nullptr)) return false;
    std::vector<int> ord(k);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) { return a[u] < a[v]; });
    theta.resize(k);
    for (int q = 0; q < k; ++q) theta[q] = a[ord[q]];
    if (Z) {
        Z->resize(static_cast<size_t>(k) * k);
        for (int q = 0; q < k; ++q)
            std::copy(Zw.begin() + static_cast<size_t>(ord[q]) * k, Zw.begin() + static_cast<size_t>(ord[q] + 1) * k,
                      Z->begin() + static_cast<size_t>(q) * k);
    }
    return true;
}

// Lanczos on N restricted to the complement of V[0..nlock) (orthonormal on
// entry), CGS2 against the whole basis; V[nlock..nlock + k) receives the
// basis. The host reads the step coefficients at the checks (every 4th step
// from step 8, and the last). tol > 0: stops when both extreme Ritz pairs meet
// tol; tol = 0: runs max_iter steps. A breakdown (|w| <= 1e-12) ends the run
// at that step (the Krylov space is exhausted).
struct LanczosOut {
    std::vector<double> alpha, beta;  // T: alpha[0..k), beta[1..k) (beta[0] = 0 unused)
    int k = 0;
    double bnext = 0.0;  // |w| after step k: the Ritz residual of pair q is bnext |z_q[k - 1]|
    bool exhausted = false, converged = false;
    double theta_max = 0, theta_min = 0, res_max = INFINITY, res_min = INFINITY;
};

static LanczosOut lanczos_run(sc_graph *g, double *V, int64_t ldv, int nlock, int max_iter, double tol, uint64_t seed,
                              const double *isd) {
    LanczosOut L;
    const int32_t n = g->n;
    cudaStream_t s = g->stream;
    const int nbasis = nlock + max_iter + 1;
    DevBuf<double> w, c, partial, ab;
    w.reserve(n);
    c.reserve(2 * static_cast<size_t>(nbasis) + 8);
    partial.reserve(static_cast<size_t>(nbasis) * kDotBlocks);
    ab.reserve(2 * static_cast<size_t>(max_iter));
    const int tb = 256, nb = ceil_div(n, tb);
    auto reorth = [&](int nv) {
        for (int pass = 0; pass < 2; ++pass) {
            double *cc = c.get() + (pass ? nbasis : 0);
            k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(V, ldv, nv, w.get(), n, partial.get());
            k_multidot_final<<<nv, kDotBlocks, 0, s>>>(partial.get(), cc);
            k_sub_combination<<<nb, tb, 0, s>>>(V, ldv, nv, cc, w.get(), n);
            SC_LAUNCH_CHECK();
        }
    };
    auto norm2_into = [&](double *dst) {
        k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(w.get(), ldv, 1, w.get(), n, partial.get());
        k_multidot_final<<<1, kDotBlocks, 0, s>>>(partial.get(), dst);
        SC_LAUNCH_CHECK();
    };
    k_start_vector<<<nb, tb, 0, s>>>(w.get(), n, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    SC_LAUNCH_CHECK();
    reorth(nlock);
    double *nrm_dev = c.get() + 2 * nbasis;
    norm2_into(nrm_dev);
    k_scale_into<<<nb, tb, 0, s>>>(w.get(), nrm_dev, V + nlock * ldv, n);
    SC_LAUNCH_CHECK();
    double *d_alpha = ab.get(), *d_nrm2 = ab.get() + max_iter;
    std::vector<double> h_alpha, h_nrm2;
    L.beta.assign(1, 0.0);
    int k = 0;
    for (int j = 0; j < max_iter; ++j) {
        const int vj = nlock + j;
        k_spmv_norm<<<ceil_div(n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), isd, V + vj * ldv, w.get(), n);
        SC_LAUNCH_CHECK();
        reorth(vj + 1);
        k_alpha_of<<<1, 1, 0, s>>>(c.get(), nbasis, vj, d_alpha + j);
        norm2_into(d_nrm2 + j);
        const int kk = j + 1;
        const bool last = kk == max_iter || kk == n - nlock;
        if (last || (kk >= 8 && kk % 4 == 0)) {
            h_alpha.resize(kk);
            h_nrm2.resize(kk);
            SC_CUDA(cudaMemcpyAsync(h_alpha.data(), d_alpha, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaMemcpyAsync(h_nrm2.data(), d_nrm2, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaStreamSynchronize(s));
            bool exhausted = kk == n - nlock;
            int stop = kk;
            for (int q = static_cast<int>(L.alpha.size()); q < kk; ++q) {
                L.alpha.push_back(h_alpha[q]);
                const double b = std::sqrt(std::max(h_nrm2[q], 0.0));
                if (!(b > 1e-12)) {
                    stop = q + 1;
                    exhausted = true;
                    break;
                }
                if (q + 1 < kk) L.beta.push_back(b);
            }
            k = stop;
            L.bnext = std::sqrt(std::max(h_nrm2[stop - 1], 0.0));
            L.exhausted = exhausted;
            if (tol > 0.0) {
                L.theta_max = bisect_eig(L.alpha, L.beta, k, k - 1, -1.0 - 1e-9, 1.0 + 1e-9);
                L.theta_min = bisect_eig(L.alpha, L.beta, k, 0, -1.0 - 1e-9, 1.0 + 1e-9);
                L.res_max = exhausted ? 0.0 : L.bnext * std::fabs(ritz_last_component(L.alpha, L.beta, k, L.theta_max));
                L.res_min = exhausted ? 0.0 : L.bnext * std::fabs(ritz_last_component(L.alpha, L.beta, k, L.theta_min));
                if (L.res_max <= tol && L.res_min <= tol) {
                    L.converged = true;
                    break;
                }
            }
            if (exhausted || last) break;
            L.beta.push_back(L.bnext);
        }
        k = kk;
        k_scale_into<<<nb, tb, 0, s>>>(w.get(), d_nrm2 + j, V + (vj + 1) * ldv, n);
        SC_LAUNCH_CHECK();
    }
    L.k = k;
    L.alpha.resize(k);
    L.beta.resize(k);
    return L;
}

// Y_p = sum_j V[j] Zu[j, p] for p < P (Ritz vectors), into Y + p * ldv; thread
// per row, 32 columns of Zu per grid row, j in order
constexpr int kRitzCols = 32;
__global__ void k_ritz_vectors(const double *__restrict__ V, int64_t ldv, int k, const double *__restrict__ Zu, int P,
                               int32_t n, double *__restrict__ Y) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int p0 = blockIdx.y * kRitzCols;
    if (i >= n) return;
    const int np = min(kRitzCols, P - p0);
    double acc[kRitzCols];
#pragma unroll
    for (int u = 0; u < kRitzCols; ++u) acc[u] = 0.0;
    for (int j = 0; j < k; ++j) {
        const double v = V[j * ldv + i];
        const double *z = Zu + static_cast<int64_t>(j) * P + p0;
#pragma unroll
        for (int u = 0; u < kRitzCols; ++u)
            if (u < np) acc[u] += v * z[u];
    }
#pragma unroll
    for (int u = 0; u < kRitzCols; ++u)
        if (u < np) Y[(p0 + u) * ldv + i] = acc[u];
}

// Frow[p * n + i] = sqrt(2m) isd[i] Y_p[i]: f_k = sqrt(2m) D^-1/2 phi_k
__global__ void k_f_rows(const double *__restrict__ Y, int64_t ldv, int P, const double *__restrict__ isd,
                         double sqrt_2m, int32_t n, double *__restrict__ Frow) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int p = blockIdx.y;
    if (i >= n || p >= P) return;
    Frow[static_cast<int64_t>(p) * n + i] = sqrt_2m * isd[i] * Y[p * ldv + i];
}

// Fn[i * P + p] = Frow[p * n + i] (32 x 32 tiles through shared memory)
__global__ void k_rows_to_nodes(const double *__restrict__ Frow, int32_t n, int P, double *__restrict__ Fn) {
    __shared__ double tile[32][33];
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * 32;
    const int p0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int p = p0 + r;
        const int64_t i = i0 + threadIdx.x;
        if (p < P && i < n) tile[r][threadIdx.x] = Frow[static_cast<int64_t>(p) * n + i];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r;
        const int p = p0 + threadIdx.x;
        if (p < P && i < n) Fn[i * P + p] = tile[threadIdx.x][r];
    }
}

__device__ __forceinline__ double warp_sum_fixed(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;  // every lane holds the same value (each butterfly stage adds a pair in both orders)
}

// Algorithm 1 per edge, one warp per row (grid-stride), its entries (i -> j),
// j > i, one at a time; the length goes to both directions of the edge.
__global__ void k_caltau(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                         const int32_t *__restrict__ rev, int32_t n, const double *__restrict__ Fn,
                         const double *__restrict__ lam, int P, double lam_rest, double lam_top, double eps,
                         double two_m, int32_t *__restrict__ tau, int32_t *ell_max) {
    const int lane = threadIdx.x & 31;
    const double denom0 = __dmul_rn(eps, __dsub_rn(1.0, __dmul_rn(lam_top, lam_top)));
    const double log_inv_top = log(__ddiv_rn(1.0, lam_top));
    const double rest_scale = __dsub_rn(1.0, __dmul_rn(lam_rest, lam_rest));
    const double log_inv_rest = lam_rest > 0.0 ? log(__ddiv_rn(1.0, lam_rest)) : 0.0;
    int32_t best = 0;
    for (int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += gridDim.x * (blockDim.x >> 5)) {
        const double di = static_cast<double>(row_ptr[r + 1] - row_ptr[r]);
        for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
            const int32_t j = col[k];
            if (j <= r) continue;  // warp-uniform
            const double dj = static_cast<double>(row_ptr[j + 1] - row_ptr[j]);
            const double xe =
                __dsub_rn(__dadd_rn(__ddiv_rn(1.0, di), __ddiv_rn(1.0, dj)), __ddiv_rn(2.0, __dmul_rn(di, dj)));
            // Eq. 6 with lambda_star alone: the starting length
            int32_t tau0 = 1;
            if (xe > 0.0 && lam_top > 0.0) {
                const double f = ceil(__dsub_rn(__ddiv_rn(log(__ddiv_rn(xe, denom0)), log_inv_top), 1.0));
                if (f > 1.0) tau0 = f > static_cast<double>(kCalTauMaxLen) ? kCalTauMaxLen : static_cast<int32_t>(f);
            }
            if ((tau0 & 1) == 0) tau0 += 1;
            // c_q, the Eq. 8 weights lambda^(t+1) / (1 - lambda) at t = 1, and Eq. 7
            double cq[kModesPerLane], wq[kModesPerLane], l2[kModesPerLane];
            double ups = 0.0;
#pragma unroll
            for (int u = 0; u < kModesPerLane; ++u) {
                const int q = lane + 32 * u;
                cq[u] = wq[u] = l2[u] = 0.0;
                if (q < P) {
                    const double d = __dsub_rn(Fn[static_cast<int64_t>(r) * P + q], Fn[static_cast<int64_t>(j) * P + q]);
                    const double lq = lam[q];
                    cq[u] = __dmul_rn(d, d);
                    l2[u] = __dmul_rn(lq, lq);
                    wq[u] = __ddiv_rn(l2[u], __dsub_rn(1.0, lq));
                    ups = __fma_rn(__dadd_rn(1.0, lq), cq[u], ups);
                }
            }
            ups = __ddiv_rn(warp_sum_fixed(ups), two_m);
            const double num = __dsub_rn(xe, ups);  // X_e - Upsilon: the remainder's weight
            const bool none_left = num <= 0.0 || lam_rest == 0.0;
            int32_t out = tau0;
            for (int32_t t = 1; t < tau0; t += 2) {
                double dp = 0.0;
#pragma unroll
                for (int u = 0; u < kModesPerLane; ++u) dp = __fma_rn(wq[u], cq[u], dp);
                const double budget = __dsub_rn(eps, __ddiv_rn(warp_sum_fixed(dp), two_m));
                const bool spent = budget < 0.0 || (!none_left && budget == 0.0);
                bool stop;
                if (spent) stop = false;  // Delta_t alone exceeds eps: a longer t is needed
                else if (none_left) stop = true;
                else {
                    const double f = ceil(__dsub_rn(
                        __ddiv_rn(log(__ddiv_rn(num, __dmul_rn(budget, rest_scale))), log_inv_rest), 1.0));
                    stop = static_cast<double>(t) > f;
                }
                if (stop) {
                    out = t;
                    break;
                }
#pragma unroll
                for (int u = 0; u < kModesPerLane; ++u) wq[u] = __dmul_rn(wq[u], l2[u]);
            }
            if (lane == 0) {
                tau[k] = out;
                tau[rev[k]] = out;
            }
            best = max(best, out);
        }
    }
    if (lane == 0 && best > 0) atomicMax(ell_max, best);
}

// the longest Eq. 6 length any edge can have (X_e <= 1)
static double eq6_len_bound(double eps, double lam) {
    if (!(lam > 0.0)) return 1.0;
    return std::ceil(std::log(1.0 / (eps * (1.0 - lam * lam))) / std::log(1.0 / lam) - 1.0);
}

static void caltau_device(sc_graph *g, double eps, const double *Fn_dev, const std::vector<double> &lam_used,
                          double lam_rest, int32_t *ell_out) {
    const int P = static_cast<int>(lam_used.size());
    double lam_top = lam_rest;
    for (double l : lam_used) lam_top = std::max(lam_top, std::fabs(l));
    if (!(lam_top < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "a modulus >= 1 among the pairs or the rest bound");
    if (eq6_len_bound(eps, lam_top) > kCalTauMaxLen)
        SC_FAIL(SC_ERR_UNSUPPORTED, "Eq. 6's length passes 2^20 at lambda_star %.17g", lam_top);
    cudaStream_t s = g->stream;
    DevBuf<double> lam_dev;
    lam_dev.reserve(std::max(P, 1));
    if (P > 0)
        SC_CUDA(cudaMemcpyAsync(lam_dev.get(), lam_used.data(), P * sizeof(double), cudaMemcpyHostToDevice, s));
    g->caltau_tau.reserve(g->nnz);
    g->status.reserve(4);
    SC_CUDA(cudaMemsetAsync(g->status.get(), 0, sizeof(int32_t), s));
    const int grid = std::max(1, std::min(ceil_div(g->n, 8), (g->num_sms > 0 ? g->num_sms : 148) * 8));
    k_caltau<<<grid, 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), g->rev.get(), g->n, Fn_dev, lam_dev.get(), P,
                                  lam_rest, lam_top, eps, static_cast<double>(g->nnz), g->caltau_tau.get(),
                                  g->status.get());
    SC_LAUNCH_CHECK();
    int32_t ell = 0;
    SC_CUDA(cudaMemcpyAsync(&ell, g->status.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    g->caltau_eps = eps;
    g->caltau_ready = true;
    if (ell_out) *ell_out = ell;
}

sc_status eigenpairs_impl(sc_graph *g, const sc_eig_opts *opts, double *lam_out, double *F_out, sc_eig_report *rep) {
    return guarded([&] {
        if (!g || !lam_out) SC_FAIL(SC_ERR_INVALID_ARG, "null graph or lam_out");
        const int32_t n = g->n;
        const int omega = opts ? opts->omega : 128;
        if (omega < 2 || omega > kOmegaMax || omega > n)
            SC_FAIL(SC_ERR_INVALID_ARG, "omega %d not in [2, min(%d, n)]", omega, kOmegaMax);
        if (g->bipartite) SC_FAIL(SC_ERR_UNSUPPORTED, "bipartite graph: lambda = -1 is a mode of modulus 1");
        const int max_iter = std::min(n - 1, (opts && opts->max_iter > 0) ? opts->max_iter : 3 * omega + 64);
        const double tol = (opts && opts->tol > 0) ? opts->tol : 1e-8;
        const double rest_tol = (opts && opts->rest_tol > 0) ? opts->rest_tol : 1e-6;
        const int rest_iter_opt = (opts && opts->rest_max_iter > 0) ? opts->rest_max_iter : 500;
        const uint64_t seed = opts ? opts->seed : 0x1a2b3c4dULL;
        if (max_iter < 1) SC_FAIL(SC_ERR_INVALID_ARG, "graph too small for Lanczos");
        cudaStream_t s = g->stream;
        const int64_t ldv = (static_cast<int64_t>(n) + 31) / 32 * 32;
        const int tb = 256, nb = ceil_div(n, tb);
        const double two_m = static_cast<double>(g->nnz);
        DevBuf<double> isd, V;
        isd.reserve(n);
        V.reserve(static_cast<size_t>(max_iter + 2) * ldv);
        k_locked_vectors<<<nb, tb, 0, s>>>(g->row_ptr.get(), g->level.get(), n, 1.0 / std::sqrt(two_m), 0, V.get(),
                                           V.get() + ldv, isd.get());
        SC_LAUNCH_CHECK();
        // run 1: Ritz pairs
        LanczosOut L1 = lanczos_run(g, V.get(), ldv, 1, max_iter, 0.0, seed, isd.get());
        const int k = L1.k;
        std::vector<double> theta, Z;
        std::vector<double> off(std::max(k - 1, 1), 0.0);
        for (int i = 0; i + 1 < k; ++i) off[i] = L1.beta[i + 1];
        if (!tridiag_eig_sorted(k, L1.alpha.data(), off.data(), theta, &Z))
            SC_FAIL(SC_ERR_LAMBDA_NOT_CONVERGED, "tridiagonal QR did not converge (k = %d)", k);
        std::vector<int> ord(k);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) {
            const double au = std::fabs(theta[u]), av = std::fabs(theta[v]);
            return au != av ? au > av : theta[u] > theta[v];
        });
        std::vector<int> U;
        double max_res = 0.0;
        for (int q : ord) {
            if (static_cast<int>(U.size()) == omega - 1) break;
            const double res = L1.exhausted ? 0.0 : L1.bnext * std::fabs(Z[static_cast<size_t>(q) * k + k - 1]);
            if (res <= tol) {
                U.push_back(q);
                max_res = std::max(max_res, res);
            }
        }
        const int P = static_cast<int>(U.size());
        // run 2 basis: lambda_1's vector, the Ritz vectors of U, then the new steps
        const int rest_iter = std::min(rest_iter_opt, n - 1 - P);
        DevBuf<double> V2;
        V2.reserve(static_cast<size_t>(1 + P + std::max(rest_iter, 0) + 1) * ldv);
        SC_CUDA(cudaMemcpyAsync(V2.get(), V.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (P > 0) {
            std::vector<double> Zu(static_cast<size_t>(k) * P);
            for (int j = 0; j < k; ++j)
                for (int p = 0; p < P; ++p) Zu[static_cast<size_t>(j) * P + p] = Z[static_cast<size_t>(U[p]) * k + j];
            DevBuf<double> Zu_dev;
            Zu_dev.reserve(Zu.size());
            SC_CUDA(cudaMemcpyAsync(Zu_dev.get(), Zu.data(), Zu.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            k_ritz_vectors<<<dim3(nb, ceil_div(P, kRitzCols)), tb, 0, s>>>(V.get() + ldv, ldv, k, Zu_dev.get(), P, n,
                                                                            V2.get() + ldv);
            SC_LAUNCH_CHECK();
            SC_CUDA(cudaStreamSynchronize(s));  // Zu_dev and V are released below
        }
        V.release();
        // run 2: the largest modulus outside U
        LanczosOut L2;
        double lam_rest = 0.0;
        if (rest_iter > 0) {
            L2 = lanczos_run(g, V2.get(), ldv, 1 + P, rest_iter, rest_tol, seed + 1, isd.get());
            lam_rest = std::max(std::fabs(L2.theta_max), std::fabs(L2.theta_min)) + std::max(L2.res_max, L2.res_min) +
                       max_res;
        } else {
            L2.converged = true;
            L2.res_max = L2.res_min = 0.0;
        }
        // f_k rows and the node-major copy kept for sc_caltau
        std::vector<double> lam_used(P);
        for (int p = 0; p < P; ++p) lam_used[p] = theta[U[p]];
        DevBuf<double> Frow;
        Frow.reserve(std::max<size_t>(static_cast<size_t>(P) * n, 1));
        g->eig_Fn.reserve(std::max<size_t>(static_cast<size_t>(P) * n, 1));
        if (P > 0) {
            k_f_rows<<<dim3(nb, P), tb, 0, s>>>(V2.get() + ldv, ldv, P, isd.get(), std::sqrt(two_m), n, Frow.get());
            k_rows_to_nodes<<<dim3(ceil_div(n, 32), ceil_div(P, 32)), dim3(32, 8), 0, s>>>(Frow.get(), n, P,
                                                                                          g->eig_Fn.get());
            SC_LAUNCH_CHECK();
        }
        g->eig_lam = lam_used;
        g->eig_rest = std::min(lam_rest, 1.0);
        g->eig_P = P;
        g->eig_ready = true;
        std::fill(lam_out, lam_out + omega, 0.0);
        lam_out[0] = 1.0;
        std::copy(lam_used.begin(), lam_used.end(), lam_out + 1);
        if (F_out) {
            std::fill(F_out, F_out + static_cast<size_t>(omega) * n, 0.0);
            std::fill(F_out, F_out + n, 1.0);
            if (P > 0)
                SC_CUDA(cudaMemcpyAsync(F_out + n, Frow.get(), static_cast<size_t>(P) * n * sizeof(double),
                                        cudaMemcpyDeviceToHost, s));
        }
        SC_CUDA(cudaStreamSynchronize(s));
        if (rep) {
            rep->used = 1 + P;
            rep->iterations = k;
            rep->rest_iterations = rest_iter > 0 ? L2.k : 0;
            rep->rest_converged = L2.converged ? 1 : 0;
            rep->max_residual = max_res;
            rep->rest_residual = std::max(L2.res_max, L2.res_min);
            rep->lambda_rest = lam_rest;
        }
        if (!L2.converged)
            SC_FAIL(SC_ERR_LAMBDA_NOT_CONVERGED, "second Lanczos run: residuals %.3g / %.3g above %.3g after %d steps",
                    L2.res_max, L2.res_min, rest_tol, L2.k);
    });
}

}  // namespace sc

extern "C" {

sc_status sc_eigenpairs(sc_graph *g, const sc_eig_opts *opts, double *lam_out, double *F_out, sc_eig_report *report) {
    return sc::eigenpairs_impl(g, opts, lam_out, F_out, report);
}

sc_status sc_caltau(sc_graph *g, double eps, int32_t count, const double *lam, const double *F, double lam_rest,
                    int32_t *tau_out, int32_t *ell_out) {
    return sc::guarded([&] {
        if (!g) SC_FAIL(SC_ERR_INVALID_ARG, "null graph");
        if (!(eps > 0.0 && eps < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "eps must lie in (0, 1)");
        if (g->bipartite) SC_FAIL(SC_ERR_UNSUPPORTED, "bipartite graph: lambda = -1 is a mode of modulus 1");
        cudaStream_t s = g->stream;
        const int32_t n = g->n;
        int32_t ell = 0;
        if (count == 0) {
            if (!g->eig_ready) SC_FAIL(SC_ERR_INVALID_ARG, "no eigenpairs: call sc_eigenpairs first or pass them");
            sc::caltau_device(g, eps, g->eig_Fn.get(), g->eig_lam, g->eig_rest, &ell);
        } else {
            if (count < 2 || count > sc::kOmegaMax) SC_FAIL(SC_ERR_INVALID_ARG, "count %d not in [2, %d]", count, sc::kOmegaMax);
            if (!lam || !F) SC_FAIL(SC_ERR_INVALID_ARG, "null lam or F");
            if (!(lam_rest >= 0.0 && lam_rest < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "lam_rest %g not in [0, 1)", lam_rest);
            const int P = count - 1;
            std::vector<double> lam_used(lam + 1, lam + count);
            for (double l : lam_used)
                if (!(std::fabs(l) < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "|lambda| = %g is not below 1", l);
            sc::DevBuf<double> Frow, Fn;
            Frow.reserve(static_cast<size_t>(P) * n);
            Fn.reserve(static_cast<size_t>(P) * n);
            SC_CUDA(cudaMemcpyAsync(Frow.get(), F + n, static_cast<size_t>(P) * n * sizeof(double),
                                    cudaMemcpyHostToDevice, s));
            sc::k_rows_to_nodes<<<dim3(sc::ceil_div(n, 32), sc::ceil_div(P, 32)), dim3(32, 8), 0, s>>>(Frow.get(), n, P,
                                                                                                      Fn.get());
            SC_LAUNCH_CHECK();
            sc::caltau_device(g, eps, Fn.get(), lam_used, lam_rest, &ell);
        }
        if (ell_out) *ell_out = ell;
        if (tau_out) {
            SC_CUDA(cudaMemcpyAsync(tau_out, g->caltau_tau.get(), g->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaStreamSynchronize(s));
        }
    });
}

sc_status sc_tridiag_eig(int32_t k, const double *alpha, const double *beta, double *theta, double *Z) {
    return sc::guarded([&] {
        if (k < 1 || !alpha || !theta || (k > 1 && !beta)) SC_FAIL(SC_ERR_INVALID_ARG, "k < 1 or a null array");
        std::vector<double> th, Zv;
        if (!sc::tridiag_eig_sorted(k, alpha, beta, th, Z ? &Zv : nullptr))
            SC_FAIL(SC_ERR_LAMBDA_NOT_CONVERGED, "an eigenvalue took more than 60 QR steps");
        std::copy(th.begin(), th.end(), theta);
        if (Z) std::copy(Zv.begin(), Zv.end(), Z);
    });
}

}  // extern "C"

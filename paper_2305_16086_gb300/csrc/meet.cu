// The meet-in-the-middle form of the truncated series (Eq. 2) on the device,
// the deterministic counterpart of the collision view of MonteCarlo-C
// (Section 2.3).
//
// For an edge (i, j) let u_h = r_h(i) - r_h(j), r_h(x) = e_x^T P^h, and
// c_h = D^-1 u_h^T. Reversibility gives u_{h+1}^T = A D^-1 u_h^T, so
// c_0 = e_i / d_i - e_j / d_j and c_{h+1} = P c_h: the same pull operator as
// the source traversal. The Chapman-Kolmogorov equation gives the hop-l term
// of Eq. 2 as t_l = <u_a, u_b>_{D^-1} = sum_x d_x c_a[x] c_b[x] with
// a = floor(l / 2), b = l - a, so S_tau = sum_{l <= tau} t_l needs ceil(tau / 2)
// hops of one column per edge instead of tau hops of one column per source.
//
// Layout: a block of kMeetB = 32 edges is an n x 32 FP64 block, row-major (a
// node's 32 values contiguous, one per lane). A hop is one warp per row, the
// row's neighbours in CSR order; a term is a column-wise weighted dot product,
// CTAs over row ranges, warps over rows, partials summed in a fixed order.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sc {

constexpr int kMeetB = 32;
constexpr int kMeetWarps = 8;

// c[i_b, b] = 1/d_i, c[j_b, b] = -1/d_j (c zeroed before)
__global__ void k_meet_init(const int32_t *__restrict__ ei, const int32_t *__restrict__ ej, int32_t ncols,
                            const double *__restrict__ inv_deg, double *__restrict__ c) {
    const int b = threadIdx.x;
    if (b >= ncols) return;
    c[static_cast<int64_t>(ei[b]) * kMeetB + b] = inv_deg[ei[b]];
    c[static_cast<int64_t>(ej[b]) * kMeetB + b] = -inv_deg[ej[b]];
}

// c_next = P c: one warp per row (grid-stride), lane b sums column b over N(x) in CSR order
__global__ void k_meet_hop(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                           const double *__restrict__ inv_deg, const double *__restrict__ c,
                           double *__restrict__ c_next, int32_t n) {
    const int lane = threadIdx.x & 31;
    for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); x < n;
         x += static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5)) {
        double acc = 0.0;
        for (int32_t k = row_ptr[x]; k < row_ptr[x + 1]; ++k) acc += c[static_cast<int64_t>(col[k]) * kMeetB + lane];
        c_next[x * kMeetB + lane] = acc * inv_deg[x];
    }
}

// partial[cta * 32 + b] = sum over the CTA's rows x of d_x c_a[x, b] c_b[x, b]
// (warp w takes rows base + w, base + w + 8, ...; the warps' sums in warp order)
__global__ void k_meet_dot_partial(const int32_t *__restrict__ row_ptr, const double *__restrict__ ca,
                                   const double *__restrict__ cb, int32_t n, int32_t chunk,
                                   double *__restrict__ partial) {
    __shared__ double sh[kMeetWarps][kMeetB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * chunk;
    const int64_t r1 = min(static_cast<int64_t>(n), r0 + chunk);
    double acc = 0.0;
    for (int64_t x = r0 + warp; x < r1; x += kMeetWarps) {
        const double d = static_cast<double>(row_ptr[x + 1] - row_ptr[x]);
        acc += d * ca[x * kMeetB + lane] * cb[x * kMeetB + lane];
    }
    sh[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int w = 0; w < kMeetWarps; ++w) s += sh[w][lane];
        partial[static_cast<int64_t>(blockIdx.x) * kMeetB + lane] = s;
    }
}

// S[b] += (the CTAs' partials of column b, in CTA order) when ell <= tau[b]
__global__ void k_meet_dot_final(const double *__restrict__ partial, int32_t nctas, const int32_t *__restrict__ tau,
                                 int32_t ncols, int32_t ell, double *__restrict__ S) {
    const int b = threadIdx.x;
    if (b >= ncols || ell > tau[b]) return;
    double s = 0.0;
    for (int32_t q = 0; q < nctas; ++q) s += partial[static_cast<int64_t>(q) * kMeetB + b];
    S[b] += s;
}

sc_status series_meet_impl(sc_graph *g, const int32_t *tau_host, double *s_out) {
    return guarded([&] {
        if (!g || !tau_host || !s_out) SC_FAIL(SC_ERR_INVALID_ARG, "null argument");
        const int32_t n = g->n;
        const int64_t nnz = g->nnz;
        cudaStream_t s = g->stream;
        std::vector<int32_t> col(nnz), rev(nnz);
        SC_CUDA(cudaMemcpyAsync(col.data(), g->col_idx.get(), nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaMemcpyAsync(rev.data(), g->rev.get(), nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
        // the edges (i < j) with their length; both directions must carry the same one
        std::vector<int32_t> e_i, e_j, e_tau;
        std::vector<int64_t> e_k;
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = g->h_row_ptr[i]; k < g->h_row_ptr[i + 1]; ++k) {
                if (tau_host[k] < 0 || tau_host[k] > (1 << 20))
                    SC_FAIL(SC_ERR_INVALID_ARG, "tau[%d] = %d not in [0, 2^20]", k, tau_host[k]);
                if (tau_host[rev[k]] != tau_host[k])
                    SC_FAIL(SC_ERR_INVALID_ARG, "tau differs between the two directions of entry %d", k);
                if (col[k] > i) {
                    e_i.push_back(i);
                    e_j.push_back(col[k]);
                    e_tau.push_back(tau_host[k]);
                    e_k.push_back(k);
                }
            }
        const int64_t m = static_cast<int64_t>(e_k.size());
        const size_t blk = static_cast<size_t>(n) * kMeetB;
        DevBuf<double> c0, c1, partial, S;
        DevBuf<int32_t> d_ei, d_ej, d_tau;
        c0.reserve(blk);
        c1.reserve(blk);
        const int sms = g->num_sms > 0 ? g->num_sms : 148;
        const int32_t nctas = std::max(1, std::min(ceil_div(n, 64 * kMeetWarps), 4 * sms));
        const int32_t chunk = ceil_div(n, nctas);
        partial.reserve(static_cast<size_t>(nctas) * kMeetB);
        S.reserve(kMeetB);
        d_ei.reserve(kMeetB);
        d_ej.reserve(kMeetB);
        d_tau.reserve(kMeetB);
        const int hop_grid = std::max(1, std::min(ceil_div(n, 8), 8 * sms));
        std::vector<double> h_S(kMeetB);
        auto term = [&](const double *ca, const double *cb, int ncols, int32_t ell) {
            k_meet_dot_partial<<<nctas, kMeetWarps * 32, 0, s>>>(g->row_ptr.get(), ca, cb, n, chunk, partial.get());
            k_meet_dot_final<<<1, kMeetB, 0, s>>>(partial.get(), nctas, d_tau.get(), ncols, ell, S.get());
            SC_LAUNCH_CHECK();
        };
        for (int64_t e0 = 0; e0 < m; e0 += kMeetB) {
            const int ncols = static_cast<int>(std::min<int64_t>(kMeetB, m - e0));
            int32_t tmax = 0;
            for (int b = 0; b < ncols; ++b) tmax = std::max(tmax, e_tau[e0 + b]);
            SC_CUDA(cudaMemcpyAsync(d_ei.get(), e_i.data() + e0, ncols * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            SC_CUDA(cudaMemcpyAsync(d_ej.get(), e_j.data() + e0, ncols * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            SC_CUDA(cudaMemcpyAsync(d_tau.get(), e_tau.data() + e0, ncols * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            SC_CUDA(cudaMemsetAsync(c0.get(), 0, blk * sizeof(double), s));
            SC_CUDA(cudaMemsetAsync(S.get(), 0, kMeetB * sizeof(double), s));
            k_meet_init<<<1, kMeetB, 0, s>>>(d_ei.get(), d_ej.get(), ncols, g->inv_deg_d.get(), c0.get());
            SC_LAUNCH_CHECK();
            double *ca = c0.get(), *cb = c1.get();
            const int32_t H = (tmax + 1) / 2;
            for (int32_t h = 0; h < H; ++h) {
                k_meet_hop<<<hop_grid, 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), g->inv_deg_d.get(), ca, cb, n);
                SC_LAUNCH_CHECK();
                term(ca, ca, ncols, 2 * h);      // t_2h = |u_h|^2
                term(ca, cb, ncols, 2 * h + 1);  // t_2h+1 = <u_h, u_h+1>
                std::swap(ca, cb);
            }
            if (2 * H <= tmax) term(ca, ca, ncols, 2 * H);
            SC_CUDA(cudaMemcpyAsync(h_S.data(), S.get(), kMeetB * sizeof(double), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaStreamSynchronize(s));
            for (int b = 0; b < ncols; ++b) {
                s_out[e_k[e0 + b]] = h_S[b];
                s_out[rev[e_k[e0 + b]]] = h_S[b];
            }
        }
    });
}

}  // namespace sc

extern "C" sc_status sc_series_meet(sc_graph *g, const int32_t *tau, double *s_out) {
    return sc::series_meet_impl(g, tau, s_out);
}

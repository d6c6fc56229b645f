// Host side of TGT+ (Algorithm 4): the switch test of Eq. 14 after a hop and
// the random-walk tail, dispatched over (precision, B).
#include <algorithm>
#include <cmath>

#include "tgtplus.cuh"

namespace sc {

template <typename T, int B>
static void chi_check_t(sc_graph *g, const void *x, int slices, const int32_t *src, int nsrc, int max_deg,
                        const int32_t *tau, int ell, int gamma, double eps, double log2md, bool full_scan,
                        cudaStream_t s) {
    const int ncols = slices * B;
    double *pmin = g->tp_pmin.get(), *pmax = g->tp_pmax.get();
    long long *pvol = g->tp_pvol.get();
    if (full_scan) {
        // every row of a column through a sorted list per 64-row tile, lists merged per column
        const int nct = ceil_div(g->n, kChiRowsPerCta);
        k_chi_scan<T, B><<<dim3(nct, slices), kChiScanThreads, 0, s>>>(
            g->row_ptr.get(), static_cast<const T *>(x), g->n, g->tp_pval.get(), g->tp_pid.get(), pmin, pmax, pvol);
        k_chi_merge<B><<<ncols, kChiScanThreads, 0, s>>>(nct, ncols, g->tp_pval.get(), g->tp_pid.get(), pmin, pmax,
                                                            pvol, g->tp_cval.get(), g->tp_cid.get(), g->tp_cmin.get(),
                                                            g->tp_cmax.get(), g->tp_cvol.get());
    } else {
        // tile maxima, the threshold per column, then the candidates at or above it
        const int ntiles = ceil_div(g->n, kTileRows);
        k_chi_tiles<T, B><<<dim3(ntiles, slices), kChiScanThreads, 0, s>>>(g->row_ptr.get(),
                                                                          static_cast<const T *>(x), g->n, pmax,
                                                                          pmin, pvol);
        k_chi_thresh<B><<<ncols, kChiScanThreads, 0, s>>>(ntiles, ncols, gamma, pmax, pmin, pvol, g->tp_cthr.get(),
                                                             g->tp_cmin.get(), g->tp_cmax.get(), g->tp_cvol.get());
        k_chi_select<T, B><<<ncols, kChiScanThreads, 0, s>>>(g->n, ntiles, ncols, gamma, static_cast<const T *>(x),
                                                                pmax, pmin, g->tp_cthr.get(), g->tp_cval.get(),
                                                                g->tp_cid.get());
    }
    ChiArgs a{};
    a.row_ptr = g->row_ptr.get();
    a.col = g->col_idx.get();
    a.src = src;
    a.tau = tau;
    a.n = g->n;
    a.nsrc = nsrc;
    a.ell = ell;
    a.gamma = gamma;
    a.cval = g->tp_cval.get();
    a.cmin = g->tp_cmin.get();
    a.cmax = g->tp_cmax.get();
    a.cid = g->tp_cid.get();
    a.eps = eps;
    a.log_2m_delta = log2md;
    a.walk_count = g->tp_walks.get();
    a.rhs = g->tp_counters.get();
    k_chi_source<T, B><<<nsrc, 32, 0, s>>>(static_cast<const T *>(x), a, g->tp_srcstat.get());
    const int nw = 256 / 32;
    dim3 grid(nsrc, std::min(ceil_div(std::max(max_deg, 1), nw), 65535));
    k_chi_entries<T, B><<<grid, 256, 0, s>>>(static_cast<const T *>(x), a, g->tp_srcstat.get());
}

template <typename T, int B>
static void walks_t(sc_graph *g, const void *x, const int32_t *src, int nsrc, const int32_t *tau, int tt,
                    uint64_t seed, const WalkChunkArgs &c, cudaStream_t s) {
    WalkArgs a{};
    a.row_ptr = g->row_ptr.get();
    a.col = g->col_idx.get();
    a.src = src;
    a.tau = tau;
    a.n = g->n;
    a.nsrc = nsrc;
    a.tt = tt;
    a.walk_count = g->tp_walks.get();
    a.g = nullptr;
    a.key0 = static_cast<uint32_t>(seed);
    a.key1 = static_cast<uint32_t>(seed >> 32);
    k_walk_chunks<T, B><<<ceil_div(c.nchunks, 8), 256, 0, s>>>(static_cast<const T *>(x), a, c);
}

#define SC_DISPATCH_TB(prec, B, FN, ...)                                                   \
    do {                                                                                   \
        if ((prec) == SC_PREC_FP64) {                                                      \
            if ((B) == 32) FN<double, 32>(__VA_ARGS__);                                    \
            else if ((B) == 64) FN<double, 64>(__VA_ARGS__);                               \
            else FN<double, 128>(__VA_ARGS__);                                             \
        } else if ((prec) == SC_PREC_FP32) {                                               \
            if ((B) == 32) FN<float, 32>(__VA_ARGS__);                                     \
            else if ((B) == 64) FN<float, 64>(__VA_ARGS__);                                \
            else FN<float, 128>(__VA_ARGS__);                                              \
        } else {                                                                           \
            if ((B) == 32) FN<__nv_bfloat16, 32>(__VA_ARGS__);                             \
            else if ((B) == 64) FN<__nv_bfloat16, 64>(__VA_ARGS__);                        \
            else FN<__nv_bfloat16, 128>(__VA_ARGS__);                                      \
        }                                                                                  \
    } while (0)

void tgtplus_reserve(sc_graph *g, int slices, int B) {
    const int nct = ceil_div(g->n, kChiRowsPerCta);
    const size_t cols = static_cast<size_t>(slices) * B;
    g->tp_pval.reserve(cols * nct * kGammaMax);
    g->tp_pid.reserve(cols * nct * kGammaMax);
    g->tp_pmin.reserve(cols * nct);
    g->tp_pmax.reserve(cols * nct);
    g->tp_pvol.reserve(cols * nct);
    g->tp_cval.reserve(cols * kGammaMax);
    g->tp_cid.reserve(cols * kGammaMax);
    g->tp_cmin.reserve(cols);
    g->tp_cmax.reserve(cols);
    g->tp_cthr.reserve(cols);
    g->tp_cvol.reserve(cols);
    g->tp_srcstat.reserve(3 * cols);
    g->tp_src_rhs.reserve(cols);
    g->tp_cap_list.reserve(cols);
    g->tp_walks.reserve(g->nnz);
    g->tp_counters.reserve(4);
}

// Eq. 14 after hop `ell` for the launch's sources: returns the two sides
// (frontier volume, sum of walk counts); the per-entry walk counts for
// L = tau_k - ell stay in g->tp_walks for the walk kernel. vol_src / rhs_src
// (host, nsrc each; may be null): the two sides per source.
void tgtplus_check(sc_graph *g, int prec, int B, const void *x, int slices, const int32_t *src, const int32_t *h_src,
                   int nsrc, const int32_t *tau, int ell, int gamma, double eps, double log2md, bool full_scan,
                   long long *lhs, long long *rhs, long long *steps, cudaStream_t s, long long *vol_src,
                   long long *rhs_src) {
    SC_CUDA(cudaMemsetAsync(g->tp_counters.get(), 0, 4 * sizeof(long long), s));
    int max_deg = 0;
    for (int q = 0; q < nsrc; ++q)
        if (h_src[q] >= 0) max_deg = std::max(max_deg, g->h_row_ptr[h_src[q] + 1] - g->h_row_ptr[h_src[q]]);
    SC_DISPATCH_TB(prec, B, chi_check_t, g, x, slices, src, nsrc, max_deg, tau, ell, gamma, eps, log2md, full_scan, s);
    SC_LAUNCH_CHECK();
    std::vector<long long> vol(static_cast<size_t>(slices) * B);
    long long h_cnt[3] = {0, 0, 0};
    SC_CUDA(cudaMemcpyAsync(vol.data(), g->tp_cvol.get(), vol.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaMemcpyAsync(h_cnt, g->tp_counters.get(), 3 * sizeof(long long), cudaMemcpyDeviceToHost, s));
    if (rhs_src) {
        k_walks_per_source<<<nsrc, 32, 0, s>>>(g->row_ptr.get(), src, nsrc, g->tp_walks.get(), g->tp_src_rhs.get());
        SC_LAUNCH_CHECK();
        SC_CUDA(cudaMemcpyAsync(rhs_src, g->tp_src_rhs.get(), nsrc * sizeof(long long), cudaMemcpyDeviceToHost, s));
    }
    SC_CUDA(cudaStreamSynchronize(s));
    if (vol_src)
        for (int q = 0; q < nsrc; ++q) vol_src[q] = h_src[q] >= 0 ? vol[q] : 0;
    long long h_lhs = 0;
    for (int q = 0; q < nsrc; ++q)
        if (h_src[q] >= 0) h_lhs += vol[q];
    *lhs = h_lhs;
    *rhs = h_cnt[0];
    *steps = h_cnt[2];
}

// Algorithm 4's walk phase for the launch's sources: the entries' walk pairs are cut
// into chunks of kWalkChunk (planned on the host from the packed counts), one
// warp per chunk, and each entry adds its chunk sums in chunk order.
// Returns the number of walk pairs drawn; *steps_out (nullable) receives their
// walk steps, 2 R (tau_k - tt) summed over the planned entries.
long long tgtplus_walks(sc_graph *g, int prec, int B, const void *x, const int32_t *src, const int32_t *h_src,
                        int nsrc, const int32_t *tau, int tt, uint64_t seed, double *acc_g, cudaStream_t s,
                        long long *steps_out) {
    if (steps_out) *steps_out = 0;
    std::vector<int32_t> eq, ek;
    for (int q = 0; q < nsrc; ++q) {
        const int32_t v = h_src[q];
        if (v < 0) continue;
        for (int32_t k = g->h_row_ptr[v]; k < g->h_row_ptr[v + 1]; ++k) {
            eq.push_back(q);
            ek.push_back(k);
        }
    }
    const int32_t ne = static_cast<int32_t>(ek.size());
    if (ne == 0) return 0;
    g->tp_eq.reserve(ne);
    g->tp_ek.reserve(ne);
    g->tp_packed.reserve(2 * static_cast<size_t>(ne));
    SC_CUDA(cudaMemcpyAsync(g->tp_eq.get(), eq.data(), ne * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(g->tp_ek.get(), ek.data(), ne * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_pack_counts<<<ceil_div(ne, 256), 256, 0, s>>>(g->tp_ek.get(), ne, g->tp_walks.get(), tau, tt,
                                                    g->tp_packed.get());
    SC_LAUNCH_CHECK();
    std::vector<long long> R(2 * static_cast<size_t>(ne));
    SC_CUDA(cudaMemcpyAsync(R.data(), g->tp_packed.get(), 2 * static_cast<size_t>(ne) * sizeof(long long),
                            cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    if (steps_out)
        for (int32_t e = 0; e < ne; ++e) *steps_out += R[ne + e];
    std::vector<int32_t> chunk_entry, entry_chunk0(ne + 1);
    std::vector<long long> chunk_w0;
    long long pairs = 0;
    for (int32_t e = 0; e < ne; ++e) {
        entry_chunk0[e] = static_cast<int32_t>(chunk_entry.size());
        for (long long w = 0; w < R[e]; w += kWalkChunk) {
            chunk_entry.push_back(e);
            chunk_w0.push_back(w);
        }
        pairs += R[e] > 0 ? R[e] : 0;
    }
    entry_chunk0[ne] = static_cast<int32_t>(chunk_entry.size());
    const int32_t nch = static_cast<int32_t>(chunk_entry.size());
    if (nch == 0) return 0;
    g->tp_chunk_entry.reserve(nch);
    g->tp_chunk_w0.reserve(nch);
    g->tp_chunk_sum.reserve(nch);
    g->tp_entry_chunk0.reserve(ne + 1);
    SC_CUDA(cudaMemcpyAsync(g->tp_chunk_entry.get(), chunk_entry.data(), nch * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(g->tp_chunk_w0.get(), chunk_w0.data(), nch * sizeof(long long), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(g->tp_entry_chunk0.get(), entry_chunk0.data(), (ne + 1) * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
    WalkChunkArgs c{g->tp_eq.get(), g->tp_ek.get(), g->tp_chunk_entry.get(), g->tp_chunk_w0.get(), nch,
                    g->tp_chunk_sum.get()};
    SC_DISPATCH_TB(prec, B, walks_t, g, x, src, nsrc, tau, tt, seed, c, s);
    SC_LAUNCH_CHECK();
    k_walk_finish<<<ceil_div(ne, 256), 256, 0, s>>>(g->tp_ek.get(), g->tp_entry_chunk0.get(), ne,
                                                    g->tp_chunk_sum.get(), g->tp_walks.get(), acc_g);
    SC_LAUNCH_CHECK();
    // the host buffers above are read by the async copies: finish before they go out of scope
    SC_CUDA(cudaStreamSynchronize(s));
    return pairs;
}

// Caps tau at `cap` on the rows of the listed nodes (host list of count, -1 = skip).
void tgtplus_cap_rows(sc_graph *g, const int32_t *h_list, int count, int32_t cap, int32_t *tau, cudaStream_t s) {
    SC_CUDA(cudaMemcpyAsync(g->tp_cap_list.get(), h_list, count * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_cap_rows<<<count, 128, 0, s>>>(g->row_ptr.get(), g->tp_cap_list.get(), count, cap, tau);
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaStreamSynchronize(s));  // h_list may be reused by the caller
}

}  // namespace sc

// sc_all_edges: the truncated graph traversal of Algorithm 2 (TGT) over
// blocks of sources, the per-edge combine of Algorithm 2's final combine, the
// end-corrected estimator and the a-posteriori tail bound.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>

#include <cudaTypedefs.h>

#include "hop2_mask.cuh"
#include "hop_tma.cuh"
#include "sparse_hops.cuh"
#include "tgtplus.cuh"
#include "propagate.cuh"

namespace sc {

sc_status estimate_lambda_impl(sc_graph *g, const sc_lambda_opts *opts, sc_lambda *out);
void tgtplus_reserve(sc_graph *g, int slices, int B);
void tgtplus_check(sc_graph *g, int prec, int B, const void *x, int slices, const int32_t *src, const int32_t *h_src,
                   int nsrc, const int32_t *tau, int ell, int gamma, double eps, double log2md, bool full_scan,
                   long long *lhs, long long *rhs, long long *steps, cudaStream_t s, long long *vol_src = nullptr,
                   long long *rhs_src = nullptr);
void tgtplus_cap_rows(sc_graph *g, const int32_t *h_list, int count, int32_t cap, int32_t *tau, cudaStream_t s);
long long tgtplus_walks(sc_graph *g, int prec, int B, const void *x, const int32_t *src, const int32_t *h_src,
                        int nsrc, const int32_t *tau, int tt, uint64_t seed, double *acc_g, cudaStream_t s,
                        long long *steps_out);
constexpr int kCostRuleHops = 4;  // the cost rule tests the last hops only
constexpr int kEvenDepthCap = 16;  // TGT+ at learned lengths: even hops recorded for the check (hop <= 16)
constexpr int kTuneHops = 8;       // hops of the sample block that picks the block width
// TGT+ cost rule rates measured on GB300: a hop costs about this much per
// source and CSR entry (BA-200k, FP32 blocks: 1.1 us per source over 4.0M
// entries), a walk step (three dependent random reads) about kWalkStepNs
constexpr double kHopNsPerSourceEntry = 2.75e-4;
constexpr double kWalkStepNs = 0.5;
void tau_entries_device(sc_graph *g, double eps, double lam_star, int32_t *tau_entry, int32_t *tau_src,
                        int32_t *ell_global_host);

// ---------------------------------------------------------------------------
// accumulator initialisation and combine
// ---------------------------------------------------------------------------
// s_hat(e_ij) = g(v_i,v_j) + g(v_j,v_i) (Algorithm 2's final combine) with g = unscaled / d,
// optionally + t_{tau+1}/2; tail bound from q = t_{tau+1} + t_{tau+2}.
__global__ void k_combine(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                          const int32_t *__restrict__ rev, const double *__restrict__ inv_d,
                          const double *__restrict__ g, const double *__restrict__ t1, const double *__restrict__ t2,
                          int32_t n, int end_corrected, int have_tail, double bound_scale,
                          double *__restrict__ s_out, double *__restrict__ bound_out) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const double ir = inv_d[r];
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        const int32_t j = col[k], kr = rev[k];
        const double ij = inv_d[j];
        // explicit round-to-nearest products and sums (no FMA contraction), so that
        // the entries (i,j) and (j,i) evaluate the same commutative expression
        double s = __dadd_rn(__dmul_rn(g[k], ir), __dmul_rn(g[kr], ij));
        if (have_tail) {
            const double a = __dadd_rn(__dmul_rn(t1[k], ir), __dmul_rn(t1[kr], ij));
            const double b = __dadd_rn(__dmul_rn(t2[k], ir), __dmul_rn(t2[kr], ij));
            if (end_corrected) s = __dadd_rn(s, __dmul_rn(0.5, a));
            if (bound_out) bound_out[k] = __dmul_rn(__dadd_rn(a, b), bound_scale);
        }
        s_out[k] = s;
    }
}

// deterministic reductions: fixed grid, fixed per-thread order, fixed tree
constexpr int kRedBlocks = 512, kRedThreads = 256;

template <bool MAX>
__global__ void k_reduce_partial(const double *__restrict__ x, int64_t count, double *__restrict__ partial) {
    __shared__ double sh[kRedThreads];
    double acc = MAX ? -INFINITY : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < count; i += (int64_t)kRedBlocks * kRedThreads)
        acc = MAX ? fmax(acc, x[i]) : acc + x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = MAX ? fmax(sh[threadIdx.x], sh[threadIdx.x + w]) : sh[threadIdx.x] + sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

template <bool MAX>
__global__ void k_reduce_final(const double *__restrict__ partial, double *__restrict__ out) {
    __shared__ double sh[kRedBlocks];
    for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) sh[i] = partial[i];
    __syncthreads();
    for (int w = kRedBlocks / 2; w > 0; w >>= 1) {
        for (int i = threadIdx.x; i < w; i += blockDim.x) sh[i] = MAX ? fmax(sh[i], sh[i + w]) : sh[i] + sh[i + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

double device_reduce(const double *x, int64_t count, bool max, double *scratch, cudaStream_t s) {
    double h = 0.0;
    if (max) {
        k_reduce_partial<true><<<kRedBlocks, kRedThreads, 0, s>>>(x, count, scratch);
        k_reduce_final<true><<<1, kRedThreads, 0, s>>>(scratch, scratch + kRedBlocks);
    } else {
        k_reduce_partial<false><<<kRedBlocks, kRedThreads, 0, s>>>(x, count, scratch);
        k_reduce_final<false><<<1, kRedThreads, 0, s>>>(scratch, scratch + kRedBlocks);
    }
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaMemcpyAsync(&h, scratch + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    return h;
}

// ---------------------------------------------------------------------------
// kernel dispatch over (precision, B, lane split)
// ---------------------------------------------------------------------------
static size_t elem_size(int prec) { return prec == SC_PREC_FP64 ? 8 : (prec == SC_PREC_FP32 ? 4 : 2); }

template <typename T>
static const typename AccOf<T>::type *inv_deg_of(const sc_graph *g);
template <>
const double *inv_deg_of<double>(const sc_graph *g) { return g->inv_deg_d.get(); }
template <>
const float *inv_deg_of<float>(const sc_graph *g) { return g->inv_deg_f.get(); }
template <>
const float *inv_deg_of<__nv_bfloat16>(const sc_graph *g) { return g->inv_deg_f.get(); }

// type-erased arguments of one hop launch
struct HopLaunch {
    const void *xp;
    void *xn;
    int slices;
    const int32_t *src;
    int nsrc;
    const int32_t *tau;
    int gather_ell;  // 0: no fused gather
    double *g, *t1, *t2;
    int32_t *status;  // TMA kernel: bounded-wait expiry flag
    GatherRec rec;
    // windowed launch: per slice windows, the hop computed, the bandwidth, and
    // the largest heavy-row count and window (rows) over the slices
    const SliceWin *win = nullptr;
    int32_t ell = 0, beta = 0;
    int win_heavy = 0;
    int64_t win_rows = 0;
};

// ---- TMA-gather variant (lane split value 0) --------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        SC_CUDA(cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) SC_FAIL(SC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map over `rows` rows of B elements (row pitch B * sizeof(T)), box of one
// full row: the shape tile::gather4 requires
template <typename T>
static CUtensorMap row_tensor_map(const void *base, int B, int64_t rows) {
    CUtensorMap m;
    const CUtensorMapDataType dt = std::is_same<T, double>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : std::is_same<T, float>::value  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(B), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(B) * sizeof(T)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(B), 1};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = tensor_map_encoder()(&m, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) SC_FAIL(SC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return m;
}

constexpr int kTmaPartEntries = 256;  // CSR entries per warp run

template <typename T, int B>
static void hop_tma_t(const sc_graph *g, const HopLaunch &h, cudaStream_t s) {
    using TL = TmaLayout<T, B>;
    static uint64_t attr_set = 0;  // per instantiation, one bit per device
    const uint64_t bit = 1ull << (g->device & 63);
    if (!(attr_set & bit)) {
        SC_CUDA(cudaFuncSetAttribute(k_hop_tma<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(TL::SMEM)));
        attr_set |= bit;
    }
    const CUtensorMap m = row_tensor_map<T>(h.xp, B, static_cast<int64_t>(h.slices) * g->n);
    TmaHopArgs a{};
    a.row_ptr = g->row_ptr.get();
    a.col = g->col_idx.get();
    a.inv_deg = inv_deg_of<T>(g);
    a.x_next = h.xn;
    a.n = g->n;
    a.part = g->part.get();
    a.nparts = g->nparts;
    a.part_ctas = ceil_div(g->nparts, kTmaWarps);
    a.x_prev = h.xp;
    a.src = h.src;
    a.nsrc = h.nsrc;
    a.tau = h.tau;
    a.gather_ell = h.gather_ell;
    a.g = h.g;
    a.t1 = h.t1;
    a.t2 = h.t2;
    a.rec = h.rec;
    a.status = h.status;
    if (h.win) SC_FAIL(SC_ERR_UNSUPPORTED, "the TMA-gather hop has no windowed form");
    a.gather_ctas = h.gather_ell > 0 ? B : 0;
    dim3 grid(a.gather_ctas + a.part_ctas, h.slices);
    k_hop_tma<T, B><<<grid, kTmaWarps * 32, TL::SMEM, s>>>(m, a);
}

template <typename T, int B, int VPL>
static void hop_t(const sc_graph *g, const HopLaunch &h, cudaStream_t s) {
    HopArgs<T> a{};
    a.row_ptr = g->row_ptr.get();
    a.col = g->col_idx.get();
    a.inv_deg = inv_deg_of<T>(g);
    a.x_prev = static_cast<const T *>(h.xp);
    a.x_next = static_cast<T *>(h.xn);
    a.n = g->n;
    a.row_order = g->row_order.get();
    a.n_heavy = g->n_heavy;
    a.src = h.src;
    a.nsrc = h.nsrc;
    a.tau = h.tau;
    a.gather_ell = h.gather_ell;
    a.g = h.g;
    a.t1 = h.t1;
    a.t2 = h.t2;
    a.rec = h.rec;
    a.win = h.win;
    a.ell = h.ell;
    a.beta = h.beta;
    a.heavy_ids = g->heavy_ids.get();
    a.heavy_t = g->heavy_threshold_cached;
    a.level = g->level.get();
    launch_spmm_hop<T, B, VPL>(a, h.slices, s, g->num_sms, h.win_heavy, h.win_rows);
}

// lane split 0 = the TMA-gather kernel; 1, 2, 4 = 16-byte vectors per lane of the SIMT kernel
template <typename T, int B>
static constexpr bool vpl_valid(int vpl) {
    constexpr int V = B / (16 / static_cast<int>(sizeof(T)));
    if (vpl == 0) return B * static_cast<int>(sizeof(T)) * 4 * 2 <= kTmaWarpRingBytes;
    return (vpl == 1 || vpl == 2 || vpl == 4) && V % vpl == 0 && V / vpl <= 32;
}

template <typename T, int B>
static void hop_b(const sc_graph *g, int vpl, const HopLaunch &h, cudaStream_t s) {
    if (vpl == 0) return hop_tma_t<T, B>(g, h, s);
    if (vpl == 1) {
        if constexpr (vpl_valid<T, B>(1)) return hop_t<T, B, 1>(g, h, s);
    } else if (vpl == 2) {
        if constexpr (vpl_valid<T, B>(2)) return hop_t<T, B, 2>(g, h, s);
    } else if (vpl == 4) {
        if constexpr (vpl_valid<T, B>(4)) return hop_t<T, B, 4>(g, h, s);
    }
    SC_FAIL(SC_ERR_INVALID_ARG, "unsupported lane split %d for B=%d", vpl, B);
}

template <typename T>
static void hop_p(const sc_graph *g, int B, int vpl, const HopLaunch &h, cudaStream_t s) {
    switch (B) {
    case 32: hop_b<T, 32>(g, vpl, h, s); break;
    case 64: hop_b<T, 64>(g, vpl, h, s); break;
    case 128: hop_b<T, 128>(g, vpl, h, s); break;
    default: SC_FAIL(SC_ERR_INVALID_ARG, "block width %d not in {32, 64, 128}", B);
    }
}

static bool cfg_valid(int prec, int B, int vpl) {
    switch (prec) {
    case SC_PREC_FP64:
        return B == 32 ? vpl_valid<double, 32>(vpl) : B == 64 ? vpl_valid<double, 64>(vpl) : B == 128 && vpl_valid<double, 128>(vpl);
    case SC_PREC_FP32:
        return B == 32 ? vpl_valid<float, 32>(vpl) : B == 64 ? vpl_valid<float, 64>(vpl) : B == 128 && vpl_valid<float, 128>(vpl);
    case SC_PREC_BF16:
        return B == 32 ? vpl_valid<__nv_bfloat16, 32>(vpl) : B == 64 ? vpl_valid<__nv_bfloat16, 64>(vpl)
                                                             : B == 128 && vpl_valid<__nv_bfloat16, 128>(vpl);
    }
    return false;
}

void launch_hop(const sc_graph *g, int prec, int B, int vpl, const HopLaunch &h, cudaStream_t s) {
    switch (prec) {
    case SC_PREC_FP64: hop_p<double>(g, B, vpl, h, s); break;
    case SC_PREC_FP32: hop_p<float>(g, B, vpl, h, s); break;
    case SC_PREC_BF16: hop_p<__nv_bfloat16>(g, B, vpl, h, s); break;
    default: SC_FAIL(SC_ERR_INVALID_ARG, "precision %d", prec);
    }
    SC_LAUNCH_CHECK();
}

template <typename T, int B>
static void first_gather_t(const sc_graph *g, bool first, const void *x, const int32_t *src, int nsrc,
                           const int32_t *tau, int ell, double *acc_g, double *acc_t1, double *acc_t2,
                           const GatherRec &rec, const SliceWin *win, cudaStream_t s) {
    if (nsrc <= 0) return;
    if (first)
        k_first_hop<T, B><<<nsrc, 128, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), inv_deg_of<T>(g), src, nsrc,
                                               static_cast<T *>(const_cast<void *>(x)), g->n, win);
    else
        k_gather<T, B><<<nsrc, 128, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), static_cast<const T *>(x), g->n, src,
                                            nsrc, tau, ell, acc_g, acc_t1, acc_t2, rec, win);
}

template <typename T>
static void first_gather_p(const sc_graph *g, int B, bool first, const void *x, const int32_t *src, int nsrc,
                           const int32_t *tau, int ell, double *a, double *b, double *c, const GatherRec &rec,
                           const SliceWin *win, cudaStream_t s) {
    switch (B) {
    case 32: first_gather_t<T, 32>(g, first, x, src, nsrc, tau, ell, a, b, c, rec, win, s); break;
    case 64: first_gather_t<T, 64>(g, first, x, src, nsrc, tau, ell, a, b, c, rec, win, s); break;
    case 128: first_gather_t<T, 128>(g, first, x, src, nsrc, tau, ell, a, b, c, rec, win, s); break;
    default: SC_FAIL(SC_ERR_INVALID_ARG, "block width %d", B);
    }
}

template <typename T, int B>
static void last_hop_t(sc_graph *g, const void *x, const int32_t *src, int nsrc, int max_deg, const int32_t *tau,
                       int ell, double *a, double *b, double *c, const GatherRec &rec, cudaStream_t s) {
    g->last_diag.reserve(nsrc);
    k_last_diag<T, B><<<nsrc, kSpmmWarps * 32, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), inv_deg_of<T>(g),
                                                      static_cast<const T *>(x), g->n, src, nsrc, tau, ell, a, b, c,
                                                      rec, g->last_diag.get());
    dim3 grid(nsrc, std::min(ceil_div(std::max(max_deg, 1), kSpmmWarps), 65535));
    k_last_rows<T, B><<<grid, kSpmmWarps * 32, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), inv_deg_of<T>(g),
                                                      static_cast<const T *>(x), g->n, src, nsrc, tau, ell, a, b, c,
                                                      rec, g->last_diag.get());
}

template <typename T>
static void last_hop_p(sc_graph *g, int B, const void *x, const int32_t *src, int nsrc, int max_deg,
                       const int32_t *tau, int ell, double *a, double *b, double *c, const GatherRec &rec,
                       cudaStream_t s) {
    switch (B) {
    case 32: last_hop_t<T, 32>(g, x, src, nsrc, max_deg, tau, ell, a, b, c, rec, s); break;
    case 64: last_hop_t<T, 64>(g, x, src, nsrc, max_deg, tau, ell, a, b, c, rec, s); break;
    case 128: last_hop_t<T, 128>(g, x, src, nsrc, max_deg, tau, ell, a, b, c, rec, s); break;
    default: SC_FAIL(SC_ERR_INVALID_ARG, "block width %d", B);
    }
}

template <typename T, int B>
static void hop2_mask_t(const sc_graph *g, uint32_t *mask, void *x2, int slices, const int32_t *src, int nsrc,
                        const int32_t *tau, double *a, double *b, double *c, const GatherRec &rec, uint32_t *nz,
                        cudaStream_t s) {
    k_mask_scatter<B><<<nsrc, 128, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), src, nsrc, mask, g->n);
    MaskHopArgs<T> m{};
    m.row_ptr = g->row_ptr.get();
    m.col = g->col_idx.get();
    m.inv_deg = inv_deg_of<T>(g);
    m.mask = mask;
    m.x_next = static_cast<T *>(x2);
    m.n = g->n;
    m.row_order = g->row_order.get();
    m.n_heavy = g->n_heavy;
    m.heavy_t = g->heavy_threshold_cached;
    m.light_ctas = light_ctas_for(g->n, kSpmmWarps, g->num_sms);  // one light row per warp
    m.gather_ctas = B;
    m.src = src;
    m.nsrc = nsrc;
    m.tau = tau;
    m.g = a;
    m.t1 = b;
    m.t2 = c;
    m.rec = rec;
    m.nz = nz;
    dim3 grid(m.gather_ctas + m.n_heavy + m.light_ctas, slices);
    k_hop2_mask<T, B><<<grid, kSpmmWarps * 32, 0, s>>>(m);
}

template <typename T>
static void hop2_mask_p(const sc_graph *g, int B, uint32_t *mask, void *x2, int slices, const int32_t *src, int nsrc,
                        const int32_t *tau, double *a, double *b, double *c, const GatherRec &rec, uint32_t *nz,
                        cudaStream_t s) {
    switch (B) {
    case 32: hop2_mask_t<T, 32>(g, mask, x2, slices, src, nsrc, tau, a, b, c, rec, nz, s); break;
    case 64: hop2_mask_t<T, 64>(g, mask, x2, slices, src, nsrc, tau, a, b, c, rec, nz, s); break;
    case 128: hop2_mask_t<T, 128>(g, mask, x2, slices, src, nsrc, tau, a, b, c, rec, nz, s); break;
    default: SC_FAIL(SC_ERR_INVALID_ARG, "block width %d", B);
    }
}

// hops 1 and 2 of a block from its sources alone (X_1 is never stored): marks
// N(s_b) in a bit mask (zeroed here), computes X_2 into x2 and gathers hop 1;
// with want_nz also the non-zero columns of X_2 (into g->mask_nz)
void launch_hop2_mask(sc_graph *g, int prec, int B, void *x2, int slices, const int32_t *src, int nsrc,
                      const int32_t *tau, double *a, double *b, double *cc, const GatherRec &rec, bool want_nz,
                      cudaStream_t s) {
    const size_t words = static_cast<size_t>(slices) * g->n * (B / 32);
    g->mask.reserve(words);
    uint32_t *nz = nullptr;
    if (want_nz) {
        g->mask_nz.reserve(words);
        nz = g->mask_nz.get();
    }
    SC_CUDA(cudaMemsetAsync(g->mask.get(), 0, words * sizeof(uint32_t), s));
    switch (prec) {
    case SC_PREC_FP64: hop2_mask_p<double>(g, B, g->mask.get(), x2, slices, src, nsrc, tau, a, b, cc, rec, nz, s); break;
    case SC_PREC_FP32: hop2_mask_p<float>(g, B, g->mask.get(), x2, slices, src, nsrc, tau, a, b, cc, rec, nz, s); break;
    case SC_PREC_BF16:
        hop2_mask_p<__nv_bfloat16>(g, B, g->mask.get(), x2, slices, src, nsrc, tau, a, b, cc, rec, nz, s);
        break;
    }
    SC_LAUNCH_CHECK();
}

template <typename T, int B>
static void hop_sparse_t(const sc_graph *g, bool ball, const void *xp, void *xn, int slices, const uint32_t *mask,
                         const int32_t *src, int nsrc, const int32_t *tau, int gather_ell, double *a, double *b,
                         double *c, const GatherRec &rec, cudaStream_t s) {
    SparseHopArgs<T> h{};
    h.row_ptr = g->row_ptr.get();
    h.col = g->col_idx.get();
    h.inv_deg = inv_deg_of<T>(g);
    h.x_prev = static_cast<const T *>(xp);
    h.x_next = static_cast<T *>(xn);
    h.mask = mask;
    h.n = g->n;
    h.row_order = g->row_order.get();
    h.n_heavy = g->n_heavy;
    h.heavy_t = g->heavy_threshold_cached;
    h.src = src;
    h.nsrc = nsrc;
    h.tau = tau;
    h.gather_ell = gather_ell;
    h.g = a;
    h.t1 = b;
    h.t2 = c;
    h.rec = rec;
    h.gather_ctas = gather_ell > 0 ? B : 0;
    h.heavy_ctas = g->n_heavy;
    h.light_ctas = light_ctas_for(g->n, kSpmmWarps, g->num_sms);  // one light row per warp
    dim3 grid(h.gather_ctas + g->n_heavy + h.light_ctas, slices);
    if (ball) k_hop_ball<T, B><<<grid, kSpmmWarps * 32, 0, s>>>(h);
    else k_hop_sparse<T, B><<<grid, kSpmmWarps * 32, 0, s>>>(h);
}

template <typename T>
static void hop_sparse_p(const sc_graph *g, int B, bool ball, const void *xp, void *xn, int slices,
                         const uint32_t *mask, const int32_t *src, int nsrc, const int32_t *tau, int gather_ell,
                         double *a, double *b, double *c, const GatherRec &rec, cudaStream_t s) {
    switch (B) {
    case 32: hop_sparse_t<T, 32>(g, ball, xp, xn, slices, mask, src, nsrc, tau, gather_ell, a, b, c, rec, s); break;
    case 64: hop_sparse_t<T, 64>(g, ball, xp, xn, slices, mask, src, nsrc, tau, gather_ell, a, b, c, rec, s); break;
    case 128: hop_sparse_t<T, 128>(g, ball, xp, xn, slices, mask, src, nsrc, tau, gather_ell, a, b, c, rec, s); break;
    default: SC_FAIL(SC_ERR_INVALID_ARG, "block width %d", B);
    }
}

// hop `gather_ell + 1` of a block from X_{gather_ell} (xp) into xn with the
// fused gather of X_{gather_ell}: ball = false: the full hop reading only the
// non-zero values of xp (mask = their columns, g->mask_nz); ball = true: the
// values on the sources' two-hop balls only (mask = the neighbour bits, g->mask)
void launch_hop_sparse(const sc_graph *g, int prec, int B, bool ball, const void *xp, void *xn, int slices,
                       const uint32_t *mask, const int32_t *src, int nsrc, const int32_t *tau, int gather_ell,
                       double *a, double *b, double *cc, const GatherRec &rec, cudaStream_t s) {
    switch (prec) {
    case SC_PREC_FP64:
        hop_sparse_p<double>(g, B, ball, xp, xn, slices, mask, src, nsrc, tau, gather_ell, a, b, cc, rec, s);
        break;
    case SC_PREC_FP32:
        hop_sparse_p<float>(g, B, ball, xp, xn, slices, mask, src, nsrc, tau, gather_ell, a, b, cc, rec, s);
        break;
    case SC_PREC_BF16:
        hop_sparse_p<__nv_bfloat16>(g, B, ball, xp, xn, slices, mask, src, nsrc, tau, gather_ell, a, b, cc, rec, s);
        break;
    }
    SC_LAUNCH_CHECK();
}

// hop `ell` (the block's last) computed only where its gather reads it, with
// the gathers of X_{ell-1} and X_ell; x = X_{ell-1}; max_deg = the largest
// degree of the sources
void launch_last_hop(sc_graph *g, int prec, int B, const void *x, const int32_t *src, int nsrc, int max_deg,
                     const int32_t *tau, int ell, double *a, double *b, double *cc, const GatherRec &rec,
                     cudaStream_t s) {
    if (nsrc <= 0) return;
    switch (prec) {
    case SC_PREC_FP64: last_hop_p<double>(g, B, x, src, nsrc, max_deg, tau, ell, a, b, cc, rec, s); break;
    case SC_PREC_FP32: last_hop_p<float>(g, B, x, src, nsrc, max_deg, tau, ell, a, b, cc, rec, s); break;
    case SC_PREC_BF16: last_hop_p<__nv_bfloat16>(g, B, x, src, nsrc, max_deg, tau, ell, a, b, cc, rec, s); break;
    }
    SC_LAUNCH_CHECK();
}

void launch_first_or_gather(const sc_graph *g, int prec, int B, bool first, const void *x, const int32_t *src,
                            int nsrc, const int32_t *tau, int ell, double *a, double *b, double *cc,
                            const GatherRec &rec, cudaStream_t s, const SliceWin *win = nullptr) {
    switch (prec) {
    case SC_PREC_FP64: first_gather_p<double>(g, B, first, x, src, nsrc, tau, ell, a, b, cc, rec, win, s); break;
    case SC_PREC_FP32: first_gather_p<float>(g, B, first, x, src, nsrc, tau, ell, a, b, cc, rec, win, s); break;
    case SC_PREC_BF16: first_gather_p<__nv_bfloat16>(g, B, first, x, src, nsrc, tau, ell, a, b, cc, rec, win, s); break;
    }
    SC_LAUNCH_CHECK();
}


// blocks propagated per launch: both ping-pong blocks within ~60% of L2
static int slices_for(const sc_graph *g, int B, size_t elem, int max_slices) {
    const size_t slice_bytes = static_cast<size_t>(g->n) * B * elem;
    const int64_t nblocks = (static_cast<int64_t>(g->n) + B - 1) / B;
    int slices = max_slices;
    if (slices <= 0) {
        const double budget = 0.6 * static_cast<double>(g->l2_bytes ? g->l2_bytes : (64u << 20));
        slices = static_cast<int>(std::max(1.0, std::floor(budget / (2.0 * static_cast<double>(slice_bytes)))));
    }
    return static_cast<int>(std::min<int64_t>(std::min<int64_t>(slices, nblocks), 65535));
}

// Autotuner: for every admissible (B, lane split) time what one block of
// sources costs on this graph: the zeroing of X_1, the first hop, a hop with
// the fused gather (taken L - 2 times) and a gather (standing for the last
// hop, which only computes what its gather reads), over a strided
// sample of sources (values do not change the cost). Keeps the least time per
// source; cached per graph, precision, request and length. The gathers write
// the accumulators, which the caller resets afterwards.
// per_b (nullable): the best lane split of every block width, by the same model
static TuneResult autotune(sc_graph *g, int prec, int fixB, int fixV, int max_slices, int32_t L, const GatherRec &rec,
                           bool allow_tma, cudaStream_t s, std::vector<TuneResult> *per_b = nullptr) {
    L = std::max(L, 1);
    const long long key = (static_cast<long long>(prec) << 40) ^ (static_cast<long long>(fixB) << 24) ^
                          (static_cast<long long>(fixV) << 16) ^ static_cast<long long>(max_slices & 0xffff) ^
                          (static_cast<long long>(g->n_heavy) << 44) ^ (static_cast<long long>(L) << 52) ^
                          (static_cast<long long>(allow_tma) << 62);
    auto it = g->tuned.find(key);
    if (it != g->tuned.end() && (!per_b || g->tuned_per_b.count(key))) {
        if (per_b) *per_b = g->tuned_per_b[key];
        return TuneResult{it->second.first, it->second.second, g->tuned_cost[key]};
    }
    std::vector<std::pair<int, int>> cands;
    for (int B : {32, 64, 128})
        for (int v : {0, 1, 2, 4})
            if ((fixB == 0 || fixB == B) && (fixV < 0 || fixV == v) && (v != 0 || allow_tma) && cfg_valid(prec, B, v))
                cands.push_back({B, v});
    if (cands.empty()) SC_FAIL(SC_ERR_INVALID_ARG, "no admissible kernel for B=%d split=%d", fixB, fixV);

    const size_t elem = elem_size(prec);
    size_t need = 0;
    int smax = 0;
    for (auto &c : cands) {
        const int sl = slices_for(g, c.first, elem, max_slices);
        need = std::max(need, sl * static_cast<size_t>(g->n) * c.first * elem);
        smax = std::max(smax, sl * c.first);
    }
    g->xa.reserve(need);
    g->xb.reserve(need);
    SC_CUDA(cudaMemsetAsync(g->xb.get(), 0, need, s));
    std::vector<int32_t> h_src(smax);
    for (int q = 0; q < smax; ++q) h_src[q] = static_cast<int32_t>((static_cast<int64_t>(q) * g->n) / smax);
    g->src_list.reserve(smax);
    SC_CUDA(cudaMemcpyAsync(g->src_list.get(), h_src.data(), smax * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    cudaEvent_t ev[4];
    for (auto &e : ev) SC_CUDA(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int q = 0; q < 4; ++q) cudaEventDestroy(e[q]);
        }
    } evg{ev};
    double *acc_g = g->acc_g.get(), *acc_t1 = g->acc_t1.get(), *acc_t2 = g->acc_t2.get();
    const int32_t *tau = g->tau_entry.get();
    // three interleaved rounds over the candidates (so that clock or cache drift
    // affects all of them alike), best round kept per candidate
    std::vector<double> best_block(cands.size(), INFINITY), best_hop(cands.size(), INFINITY);
    for (int round = 0; round < 3; ++round) {
        for (size_t ci = 0; ci < cands.size(); ++ci) {
            const auto &c = cands[ci];
            const int sl = slices_for(g, c.first, elem, max_slices);
            const int nsrc = sl * c.first;
            const int32_t *src = g->src_list.get();
            HopLaunch h{g->xa.get(), g->xb.get(), sl, src, nsrc, tau, 1, acc_g, acc_t1, acc_t2, g->status.get(), rec};
            if (round == 0) launch_hop(g, prec, c.first, c.second, h, s);  // warm-up
            const int reps = 4;
            SC_CUDA(cudaEventRecord(ev[0], s));
            SC_CUDA(cudaMemsetAsync(g->xa.get(), 0, static_cast<size_t>(nsrc) * g->n * elem, s));
            launch_first_or_gather(g, prec, c.first, true, g->xa.get(), src, nsrc, nullptr, 1, nullptr, nullptr,
                                   nullptr, rec, s);
            SC_CUDA(cudaEventRecord(ev[1], s));
            for (int r = 0; r < reps; ++r) launch_hop(g, prec, c.first, c.second, h, s);
            SC_CUDA(cudaEventRecord(ev[2], s));
            launch_first_or_gather(g, prec, c.first, false, g->xb.get(), src, nsrc, tau, 1, acc_g, acc_t1, acc_t2,
                                   rec, s);
            SC_CUDA(cudaEventRecord(ev[3], s));
            SC_CUDA(cudaEventSynchronize(ev[3]));
            float a = 0.f, b = 0.f, c2 = 0.f;
            SC_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
            SC_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
            SC_CUDA(cudaEventElapsedTime(&c2, ev[2], ev[3]));
            const double hop = b / reps;
            const double block = a + c2 + std::max(L - 2, 0) * hop;  // the last hop runs gather-sized
            best_block[ci] = std::min(best_block[ci], block / nsrc);
            best_hop[ci] = std::min(best_hop[ci], hop / nsrc);
        }
    }
    double best = INFINITY;
    size_t pick = 0;
    const bool log = std::getenv("SC_AUTOTUNE_LOG") != nullptr;
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        if (log)
            std::fprintf(stderr, "sc autotune: prec %d L %d B %d split %d: %.4f us per source-hop (%.4f per hop alone)\n",
                         prec, L, cands[ci].first, cands[ci].second == 0 ? -1 : cands[ci].second,
                         1e3 * best_block[ci] / L, 1e3 * best_hop[ci]);
        if (best_block[ci] < best) {
            best = best_block[ci];
            pick = ci;
        }
    }
    g->tuned[key] = cands[pick];
    g->tuned_cost[key] = best_hop[pick];
    std::vector<TuneResult> pb;
    for (int B : {32, 64, 128}) {
        int bi = -1;
        for (size_t ci = 0; ci < cands.size(); ++ci)
            if (cands[ci].first == B && (bi < 0 || best_block[ci] < best_block[bi])) bi = static_cast<int>(ci);
        if (bi >= 0) pb.push_back(TuneResult{B, cands[bi].second, best_hop[bi]});
    }
    g->tuned_per_b[key] = pb;
    if (per_b) *per_b = pb;
    return TuneResult{cands[pick].first, cands[pick].second, best_hop[pick]};
}

// ---------------------------------------------------------------------------
// accumulator reset for a set of source rows (all rows when rows == nullptr):
// the hop-0 term of Eq. (9) is 1 (unscaled); with record mode 1 the hop-0 term
// is also the "tau - 1" record of a length-1 entry, with mode 3 the first
// record slot of a length-1 entry (the second of a length-0 one)
// ---------------------------------------------------------------------------
__global__ void k_reset_rows(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ rows, int32_t nrows,
                             const int32_t *__restrict__ tau, int mode, double *__restrict__ g, double *__restrict__ t1,
                             double *__restrict__ t2, double *__restrict__ rec_all, int rec_stride) {
    const int32_t t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= nrows) return;
    const int32_t r = rows ? rows[t] : t;
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        g[k] = 1.0;
        const int32_t tk = tau[k];
        t1[k] = (mode == 1 && tk == 1) ? 1.0 : 0.0;
        t2[k] = (mode == 1 && tk == 0) ? 1.0 : 0.0;
        if (rec_all && mode == 3) {
            rec_all[static_cast<int64_t>(k) * 2] = tk == 1 ? 1.0 : 0.0;
            rec_all[static_cast<int64_t>(k) * 2 + 1] = tk == 0 ? 1.0 : 0.0;
        } else if (rec_all) {
            rec_all[static_cast<int64_t>(k) * rec_stride] = 1.0;
        }
    }
}

// tau_e = min(L_i, L_j) for every entry (one length per edge for both halves)
__global__ void k_tau_min_of_sources(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                     const int32_t *__restrict__ L, int32_t n, int32_t *__restrict__ tau) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int32_t Lr = L[r];
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) tau[k] = min(Lr, L[col[k]]);
}

// Extension step of the learned policy: an entry whose bound exceeds eps and
// whose length is below the a-priori cap gets tau <- min(2 tau + 1, cap);
// its row is marked for a rerun. Both directions of an edge carry the same
// bound, so both endpoints are marked.
// With `active` (a subset of the sources was run), only entries whose two
// endpoints were both run are checked. cap_row (nullable): a cap per row (the
// graphs of a batch; both endpoints of an edge lie in one graph), else cap.
__global__ void k_extend_failing(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                 const double *__restrict__ bound, int32_t n, double eps, int32_t cap_all,
                                 const int32_t *__restrict__ active, int32_t *__restrict__ tau,
                                 int32_t *__restrict__ row_flag, unsigned long long *count,
                                 const int32_t *__restrict__ cap_row = nullptr) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int32_t cap = cap_row ? cap_row[r] : cap_all;
    int any = 0;
    unsigned long long c = 0;
    const bool row_on = !active || active[r];
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        if (row_on && (!active || active[col[k]]) && bound[k] > eps && tau[k] < cap) {
            tau[k] = min(2 * tau[k] + 1, cap);
            any = 1;
            ++c;
        }
    }
    any = __any_sync(0xffffffffu, any);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        row_flag[r] = any;
        if (c) atomicAdd(count, c);
    }
}

// The learned length's acceptance test on a bipartite graph (lambda* = 1, no
// bound): with the end-corrected estimator the remainder past odd tau is
// sum_k c_k lambda_k^(tau+1) (1 + lambda_k) / (2 (1 - lambda_k)) >= 0 (mode
// expansion in the proof of Theorem 3.2), i.e. about the sum of the pair sums
// q(tau) = t_{tau+1} + t_{tau+2}, q(tau + 2), ... when the slow modes dominate.
// The pair sums are fitted by q(x) = C x^-p through q(tau - 2) = qp at x = tau - 1
// and q(tau) = q at x = tau + 1 (a diffusive, power-law decay), and the fitted
// pair sums are integrated past tau at half a unit of x per hop:
// C tau^(1-p) / (2 (p - 1)). An estimate, not a bound. 0 when q <= 0;
// +inf when tau < 3, qp <= 0 or p <= 1 (no decay to extrapolate).
__device__ __forceinline__ double tail_estimate(double qp, double q, int32_t tau) {
    if (q <= 0.0) return 0.0;
    if (tau < 3 || !(qp > 0.0)) return INFINITY;
    const double x = static_cast<double>(tau);
    const double p = log(qp / q) / log((x + 1.0) / (x - 1.0));
    if (!(p > 1.0)) return INFINITY;
    return q * (x + 1.0) * exp((p - 1.0) * log((x + 1.0) / x)) / (2.0 * (p - 1.0));
}

// training labels on a bipartite graph: every source ran cap + 2 hops with all
// hop terms recorded (rec[k * stride + l]); each entry takes the least odd
// tau in [3, cap] whose tail estimate is at most eps, else cap
__global__ void k_estimate_lengths(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                   const int32_t *__restrict__ rev, const double *__restrict__ inv_d,
                                   const double *__restrict__ rec, int stride, int32_t n, int32_t cap, double eps,
                                   int32_t *__restrict__ tau_out) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const double ir = inv_d[r];
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        const int32_t kr = rev[k];
        const double ij = inv_d[col[k]];
        auto full = [&](int l) {
            return __dadd_rn(__dmul_rn(rec[static_cast<int64_t>(k) * stride + l], ir),
                             __dmul_rn(rec[static_cast<int64_t>(kr) * stride + l], ij));
        };
        int32_t t = cap;
        for (int32_t c = 3; c <= cap; c += 2) {
            if (tail_estimate(__dadd_rn(full(c - 1), full(c)), __dadd_rn(full(c + 1), full(c + 2)), c) <= eps) {
                t = c;
                break;
            }
        }
        tau_out[k] = t;
    }
}

// The learned policy's test value per entry: rows whose graph has factor
// f >= 0 take the bound f (t_{tau-1} + t_tau) (R6', f = lambda*^2 / (1 -
// lambda*^2), which also bounds the end-corrected remainder, smaller than the
// plain one); rows with f < 0 (a bipartite graph) take the tail estimate of
// the end-corrected series. f = fac[r] (a batch's union of graphs) or fac_all.
// The terms of hops tau-1, tau are in t1 / t2 (record mode 1) or in pre (mode
// 3, whose t1 / t2 hold hops tau+1, tau+2). Both directions of an edge
// evaluate the same expression.
__global__ void k_learned_check(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                const int32_t *__restrict__ rev, const double *__restrict__ inv_d,
                                const double *__restrict__ pre, const double *__restrict__ t1,
                                const double *__restrict__ t2, int mode, const double *__restrict__ fac,
                                double fac_all, const int32_t *__restrict__ tau, int32_t n,
                                double *__restrict__ out) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const double ir = inv_d[r];
    const double f = fac ? fac[r] : fac_all;
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        const int32_t kr = rev[k];
        const double ij = inv_d[col[k]];
        auto full = [&](double a, double b) { return __dadd_rn(__dmul_rn(a, ir), __dmul_rn(b, ij)); };
        double qp;
        if (mode == 3)
            qp = __dadd_rn(full(pre[2 * static_cast<int64_t>(k)], pre[2 * static_cast<int64_t>(kr)]),
                           full(pre[2 * static_cast<int64_t>(k) + 1], pre[2 * static_cast<int64_t>(kr) + 1]));
        else
            qp = __dadd_rn(full(t1[k], t1[kr]), full(t2[k], t2[kr]));
        if (f >= 0.0) {
            out[k] = __dmul_rn(f, qp);
        } else {
            const double q = __dadd_rn(full(t1[k], t1[kr]), full(t2[k], t2[kr]));
            out[k] = tail_estimate(qp, q, tau[k]);
        }
    }
}

// per-source maximum of tau over its row
__global__ void k_row_max(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ tau, int32_t n,
                          int32_t *__restrict__ out) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int32_t m = 0;
    for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) m = max(m, tau[k]);
    out[r] = m;
}

void learned_lengths(sc_graph *g, int32_t cap, int32_t *L_dev, cudaStream_t s);

// lam^e / (1 - lam) * t, the power by repeated multiplication
__device__ __forceinline__ double even_hop_bound(double t, int32_t e, double lam) {
    double f = 1.0;
    for (int32_t q = 0; q < e; ++q) f = __dmul_rn(f, lam);
    return __dmul_rn(__ddiv_rn(f, __dsub_rn(1.0, lam)), t);
}

// The truncation check of TGT+ at learned lengths (Algorithm 4 keeps eps/2 for
// the truncation). For odd tau and even l <= tau + 1 the tail past tau is at
// most lam*^(tau + 1 - l) / (1 - lam*) t_l(e) (the mode expansion in the proof
// of Theorem 3.2: t_l(e) = sum_k c_k lam_k^l with every term >= 0 at even l).
// l = the largest even hop both endpoints' traversals reached (depth, capped
// at 2 (stride - 1)), at most tau + 1; t_l from the recorded half terms. An
// entry whose bound exceeds eps_half takes the least odd length the same
// bound accepts, at most cap; both directions of an edge evaluate the same
// expression, so both take the same length and mark their rows for a rerun.
// With `active` (a subset of the sources was run), only entries whose two
// endpoints were both run are checked.
__global__ void k_certify_plus(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                               const int32_t *__restrict__ rev, const double *__restrict__ inv_d,
                               const double *__restrict__ even, int32_t stride, const int32_t *__restrict__ depth,
                               const int32_t *__restrict__ active, int32_t n, double lam, double eps_half,
                               int32_t cap, int32_t *__restrict__ tau, int32_t *__restrict__ row_flag,
                               unsigned long long *count) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    int any = 0;
    unsigned long long c = 0;
    const bool row_on = !active || active[r];
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        const int32_t j = col[k], kr = rev[k], te = tau[k];
        if (!row_on || (active && !active[j]) || te >= cap) continue;
        const int32_t d = min(min(depth[r], depth[j]), min(te + 1, 2 * (stride - 1)));
        const int32_t ell = d & ~1;
        const double t = __dadd_rn(__dmul_rn(even[static_cast<int64_t>(k) * stride + (ell >> 1)], inv_d[r]),
                                   __dmul_rn(even[static_cast<int64_t>(kr) * stride + (ell >> 1)], inv_d[j]));
        if (even_hop_bound(t, te + 1 - ell, lam) > eps_half) {
            int32_t tn = te + 2;
            while (tn < cap && even_hop_bound(t, tn + 1 - ell, lam) > eps_half) tn += 2;
            tau[k] = min(tn, cap);
            any = 1;
            ++c;
        }
    }
    any = __any_sync(0xffffffffu, any);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        row_flag[r] = any;
        if (c) atomicAdd(count, c);
    }
}

// active[i] = active[j] = 1 for each listed entry k = (i -> j) (row by binary search)
__global__ void k_mark_endpoints(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                                 const int64_t *__restrict__ entries, int64_t count, int32_t *__restrict__ active) {
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t >= count) return;
    const int32_t k = static_cast<int32_t>(entries[t]);
    int32_t lo = 0, hi = n;  // the row r with row_ptr[r] <= k < row_ptr[r + 1]
    while (hi - lo > 1) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (row_ptr[mid] <= k) lo = mid;
        else hi = mid;
    }
    active[lo] = 1;
    active[col[k]] = 1;
}

__global__ void k_gather_entries(const double *__restrict__ x, const int64_t *__restrict__ entries, int64_t count,
                                 double *__restrict__ out) {
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t < count) out[t] = x[entries[t]];
}

// the listed CSR entries of sc_some_edges (host array) and where their values go
struct EdgeSubset {
    int64_t count;
    const int64_t *entries;
    double *out;
};

// ---------------------------------------------------------------------------
// the block loop: propagates the given sources in blocks, longest first
// ---------------------------------------------------------------------------
struct Run {
    sc_graph *g;
    const sc_options *o;
    cudaStream_t s;
    int prec, B, vpl, slices;
    size_t slice_bytes;
    bool plus, time_kernels;
    int gamma;
    double log2md;
    int extra;  // hops beyond the per-source length (records of tau+1, tau+2)
    GatherRec rec;
    int32_t h0 = 0x7fffffff;  // SC_PREC_BF16: first hop stored in bf16 (fp32 before)
    std::vector<int32_t> *depth = nullptr;  // TGT+: per node, the last hop its traversal reached
    bool capture = false;  // windowed loop: record into one CUDA graph
    // statistics
    int64_t launches = 0, hops = 0, source_hops = 0, hop_launches = 0, walks = 0, graph_launches = 0, walk_steps = 0;
    // per kernel class (SC_KC_*): event pairs (index into the graph's pool) and algorithmic bytes
    std::vector<std::pair<int, int64_t>> timed;
    int64_t event_pairs = 0;
    int64_t kc_launches[SC_KC_COUNT] = {};
    double kc_bytes[SC_KC_COUNT] = {};
    double walk_device_ms = 0.0;
    double alg_bytes = 0.0, switch_ms = 0.0, walk_ms = 0.0;
    int32_t ell_min_src = INT32_MAX, ell_max_src = 0, tt_min = INT32_MAX, tt_max = 0, switch_tests = 0;
};

// storage precision of X_ell
static int prec_at(const Run &R, int32_t ell) {
    return (R.prec == SC_PREC_BF16 && ell < R.h0) ? SC_PREC_FP32 : R.prec;
}

// bytes per stored value the block buffers are sized for
static size_t alloc_elem(int prec, int32_t h0) {
    return prec == SC_PREC_BF16 && h0 > 1 ? 4 : elem_size(prec);
}

static int32_t bf16_first_hop(const sc_options &o) {
    return o.precision == SC_PREC_BF16 ? (o.bf16_from_hop > 0 ? o.bf16_from_hop : 8) : 0x7fffffff;
}

// X_ell to bf16: fp32 values rounded to nearest (the rounding of the bf16 hop kernel's store)
__global__ void k_f32_to_bf16(const float4 *__restrict__ in, uint2 *__restrict__ out, int64_t count4) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= count4) return;
    const float4 v = in[i];
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    out[i] = make_uint2(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&b));
}

// one hop from X_{ell-1} (in xa) to X_ell (in xb) with the fused gather of
// X_{ell-1}; at the hop where the storage turns to bf16 the hop runs in fp32
// and its output is converted (xa / xb are swapped by the caller as usual:
// on return X_ell is in the buffer the caller will read next)
// A windowed loop also zeroes the fp32 copy after the conversion: its later
// hops write only their windows and read zeros outside them.
static void hop_mixed(const Run &R, HopLaunch h, int32_t ell, size_t elems, cudaStream_t s, void **xa, void **xb,
                      bool windowed = false) {
    const int pin = prec_at(R, ell - 1), pout = prec_at(R, ell);
    launch_hop(R.g, pin, R.B, R.vpl, h, s);
    if (pin != pout) {  // fp32 -> bf16 at hop h0: convert into the input buffer, now free
        k_f32_to_bf16<<<ceil_div(static_cast<int64_t>(elems / 4), 256), 256, 0, s>>>(
            static_cast<const float4 *>(h.xn), static_cast<uint2 *>(const_cast<void *>(h.xp)),
            static_cast<int64_t>(elems / 4));
        SC_LAUNCH_CHECK();
        if (windowed) SC_CUDA(cudaMemsetAsync(h.xn, 0, elems * sizeof(float), s));
        return;  // X_ell (bf16) is in *xa: no swap
    }
    std::swap(*xa, *xb);
}

// brackets one launch of kernel class `cls` with a pair of events from the
// graph's pool (SC_OPT_TIME_KERNELS) and books its algorithmic bytes; the
// opening call returns the pair's index (-1 when not timing)
static int64_t timer_open(Run &R, cudaStream_t s) {
    if (!R.time_kernels) return -1;
    const int64_t i = R.event_pairs++;
    while (static_cast<int64_t>(R.g->hop_events.size()) < 2 * (i + 1)) {
        cudaEvent_t e;
        SC_CUDA(cudaEventCreate(&e));
        R.g->hop_events.push_back(e);
    }
    SC_CUDA(cudaEventRecord(R.g->hop_events[2 * i], s));
    return i;
}

static void timer_close(Run &R, int64_t i, int cls, double bytes, cudaStream_t s) {
    R.kc_launches[cls] += 1;
    R.kc_bytes[cls] += bytes;
    if (i < 0) return;
    SC_CUDA(cudaEventRecord(R.g->hop_events[2 * i + 1], s));
    R.timed.push_back({cls, i});
}

static double wall_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// sources: the node ids to propagate; len[v]: hops source v needs
static void run_blocks(Run &R, std::vector<int32_t> sources, const std::vector<int32_t> &len) {
    sc_graph *g = R.g;
    cudaStream_t s = R.s;
    const int32_t n = g->n;
    const int64_t nnz = g->nnz;
    const int B = R.B;
    const int S = R.slices * B;
    if (sources.empty()) return;
    std::stable_sort(sources.begin(), sources.end(), [&](int32_t a, int32_t b) { return len[a] > len[b]; });
    const int64_t ns = static_cast<int64_t>(sources.size());
    const int64_t nsuper = (ns + S - 1) / S;
    std::vector<int32_t> h_src(nsuper * S, -1);
    std::copy(sources.begin(), sources.end(), h_src.begin());
    g->src_list.reserve(h_src.size());
    SC_CUDA(cudaMemcpyAsync(g->src_list.get(), h_src.data(), h_src.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    cudaEvent_t ev_w0, ev_w1;
    SC_CUDA(cudaEventCreate(&ev_w0));
    SC_CUDA(cudaEventCreate(&ev_w1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evg{ev_w0, ev_w1};
    // algorithmic bytes of hop ell per slice: CSR, 1/d, read X_{ell-1}, write X_ell
    const double csr_bytes = 4.0 * nnz + 4.0 * (n + 1) + (R.prec == SC_PREC_FP64 ? 8.0 : 4.0) * n;  // + 1/d
    const double mask_bytes = static_cast<double>(n) * B / 8.0;
    auto hop_bytes_per_slice = [&](int32_t ell) {
        return csr_bytes + static_cast<double>(n) * B * (elem_size(prec_at(R, ell - 1)) + elem_size(prec_at(R, ell)));
    };
    // a switch test reads the block X_ell once (the column statistics) and the degrees
    auto test_bytes_per_slice = [&](int32_t ell) {
        return static_cast<double>(n) * B * elem_size(prec_at(R, ell)) + 4.0 * n;
    };
    const bool dense_only = (R.o->flags & SC_OPT_SPARSE_HOPS) == 0;
    const bool full_scan = (R.o->flags & SC_OPT_FULL_TOPGAMMA_SCAN) != 0;
    // cost rule: the hop at which the previous block of the same length switched (-1: none
    // yet). Blocks come longest first and neighbouring blocks switch within a hop of each
    // other, so a block's tests start there instead of kCostRuleHops before its end.
    int32_t prev_tt = -1, prev_L = -1;
    for (int64_t sb = 0; sb < nsuper; ++sb) {
        const int64_t first = sb * S;
        const int nsrc = static_cast<int>(std::min<int64_t>(S, ns - first));
        const int used_slices = (nsrc + B - 1) / B;
        int32_t L = len[sources[first]];  // longest first
        for (int q = 0; q < nsrc; ++q) {
            R.ell_min_src = std::min(R.ell_min_src, len[sources[first + q]] + R.extra);
            R.ell_max_src = std::max(R.ell_max_src, len[sources[first + q]] + R.extra);
        }
        L += R.extra;
        if (L == 0) continue;
        const int32_t *src = g->src_list.get() + first;
        void *xa = g->xa.get(), *xb = g->xb.get();
        // hops 1-2 from the sources alone when X_1 is read by nothing else (no TGT+
        // switch test or walk from X_1, no sparse last hop at 2, one storage type)
        const bool test_at_1 =
            R.plus && (R.o->switch_rule != SC_SWITCH_COST || 1 >= std::max(1, L - kCostRuleHops));
        const bool from_mask = !test_at_1 && L >= 3 && prec_at(R, 1) == prec_at(R, 2);
        // hop 3 from X_2's non-zero values (a full hop: L >= 5 keeps it before hop L - 1), and
        // hop L - 1 on the sources' two-hop balls (read by the sparse last hop only: TGT, whose
        // traversal nothing else reads; no storage change around it)
        const bool hop3_sparse = from_mask && !dense_only && L >= 5 && prec_at(R, 2) == prec_at(R, 3);
        const bool ball_hop = from_mask && !dense_only && !R.plus && L >= 4 && prec_at(R, L - 2) == prec_at(R, L - 1) &&
                              prec_at(R, L - 1) == prec_at(R, L);
        int ell0 = 2;
        if (from_mask) {
            const int64_t t = timer_open(R, s);
            launch_hop2_mask(g, prec_at(R, 2), B, xb, used_slices, src, nsrc, g->tau_entry.get(), g->acc_g.get(),
                             g->acc_t1.get(), g->acc_t2.get(), R.rec, hop3_sparse, s);
            timer_close(R, t, SC_KC_MASK_HOP,
                        used_slices * (csr_bytes + (hop3_sparse ? 3.0 : 2.0) * mask_bytes +
                                       static_cast<double>(n) * B * elem_size(prec_at(R, 2))),
                        s);
            std::swap(xa, xb);
            R.launches += 2;
            ell0 = 3;
        } else {
            SC_CUDA(cudaMemsetAsync(xa, 0, used_slices * R.slice_bytes, s));
            launch_first_or_gather(g, prec_at(R, 1), B, true, xa, src, nsrc, nullptr, 1, nullptr, nullptr, nullptr,
                                   R.rec, s);
            R.launches += 1;  // the memset is not a kernel of ours
        }
        int32_t tt = L;  // hops traversed; TGT+ may switch to walks earlier
        bool last_done = false;
        // per-source switch (Algorithm 4's loop per source): each source's switch hop, -1 while traversing
        const bool per_source = R.plus && R.o->switch_rule == SC_SWITCH_PER_SOURCE;
        std::vector<int32_t> src_tt(per_source ? nsrc : 0, -1), now_list(per_source ? nsrc : 0, -1);
        std::vector<long long> vol_src(per_source ? nsrc : 0), rhs_src(per_source ? nsrc : 0);
        int n_active = 0;
        for (int q = 0; per_source && q < nsrc; ++q) n_active += h_src[first + q] >= 0 ? 1 : 0;
        for (int ell = ell0; ell <= L; ++ell) {
            const bool paper_rule = R.o->switch_rule == SC_SWITCH_PAPER;
            if (per_source) {
                // Eq. 14 per source after hop ell-1: each source whose frontier volume exceeds the sum
                // of its own walk counts walks from X_{ell-1} now, and its entries gather no hop after
                // ell-1 (their tau is capped there once the walk kernel has read it)
                long long lhs = 0, rhs = 0, steps = 0;
                const double t0 = wall_ms();
                const int64_t tc = timer_open(R, s);
                tgtplus_check(g, prec_at(R, ell - 1), B, xa, used_slices, src, h_src.data() + first, nsrc,
                              g->tau_entry.get(), ell - 1, R.gamma, R.o->eps, R.log2md, full_scan, &lhs, &rhs,
                              &steps, s, vol_src.data(), rhs_src.data());
                timer_close(R, tc, SC_KC_SWITCH_TEST, used_slices * test_bytes_per_slice(ell - 1), s);
                R.switch_ms += wall_ms() - t0;
                ++R.switch_tests;
                R.launches += 4;
                int nnow = 0;
                for (int q = 0; q < nsrc; ++q) {
                    now_list[q] = -1;
                    const int32_t v = h_src[first + q];
                    if (v >= 0 && src_tt[q] < 0 && vol_src[q] > rhs_src[q]) {
                        now_list[q] = v;
                        src_tt[q] = ell - 1;
                        ++nnow;
                    }
                }
                if (nnow > 0) {
                    const double tw = wall_ms();
                    const int64_t tw_ev = timer_open(R, s);
                    SC_CUDA(cudaEventRecord(ev_w0, s));
                    long long wsteps = 0;
                    const long long pairs = tgtplus_walks(g, prec_at(R, ell - 1), B, xa, src, now_list.data(), nsrc,
                                                          g->tau_entry.get(), ell - 1, R.o->seed, g->acc_g.get(), s,
                                                          &wsteps);
                    SC_CUDA(cudaEventRecord(ev_w1, s));
                    timer_close(R, tw_ev, SC_KC_WALKS, 0.0, s);
                    SC_CUDA(cudaEventSynchronize(ev_w1));
                    R.walk_ms += wall_ms() - tw;
                    R.launches += 3;
                    R.walks += pairs;
                    float wms = 0.f;
                    SC_CUDA(cudaEventElapsedTime(&wms, ev_w0, ev_w1));
                    R.walk_steps += wsteps;
                    R.walk_device_ms += wms;
                    tgtplus_cap_rows(g, now_list.data(), nsrc, ell - 1, g->tau_entry.get(), s);
                    R.launches += 1;
                    n_active -= nnow;
                }
                if (n_active == 0) {
                    tt = ell - 1;
                    break;
                }
            } else if (R.plus && (paper_rule || (ell - 1 >= std::max(1, L - kCostRuleHops) &&
                                                 (prev_L != L || prev_tt < 0 || ell - 1 >= prev_tt)))) {
                // switch test after hop ell-1. Paper rule (Eq. 14): frontier volume against the
                // sum of walk counts. Cost rule: predicted walk time against the time of the
                // L - (ell-1) hops the walks would replace.
                long long lhs = 0, rhs = 0, steps = 0;
                const double t0 = wall_ms();
                const int64_t tc = timer_open(R, s);
                tgtplus_check(g, prec_at(R, ell - 1), B, xa, used_slices, src, h_src.data() + first, nsrc, g->tau_entry.get(),
                              ell - 1, R.gamma, R.o->eps, R.log2md, full_scan, &lhs, &rhs, &steps, s);
                timer_close(R, tc, SC_KC_SWITCH_TEST, used_slices * test_bytes_per_slice(ell - 1), s);
                R.switch_ms += wall_ms() - t0;
                ++R.switch_tests;
                R.launches += 3;
                // cost rule with fixed GB300 rates, so that the decision (and the
                // result) depends on the graph and the seed only
                const double hop_ns = kHopNsPerSourceEntry * static_cast<double>(nnz) * used_slices * B;
                const bool go = paper_rule ? (lhs > rhs)
                                           : (static_cast<double>(steps) * kWalkStepNs <
                                              static_cast<double>(L - (ell - 1)) * hop_ns);
                if (go) {
                    tt = ell - 1;
                    break;
                }
            }
            if (ell == L && prec_at(R, ell - 1) == prec_at(R, ell)) {
                // the block's last hop: X_L only where the gather reads it, fused with
                // the gathers of X_{L-1} and X_L
                int max_deg = 0;
                for (int q = 0; q < nsrc; ++q) {
                    const int32_t v = h_src[first + q];
                    if (v >= 0) max_deg = std::max(max_deg, g->h_row_ptr[v + 1] - g->h_row_ptr[v]);
                }
                const int64_t t = timer_open(R, s);
                launch_last_hop(g, prec_at(R, ell), B, xa, src, nsrc, max_deg, g->tau_entry.get(), ell,
                                g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), R.rec, s);
                timer_close(R, t, SC_KC_LAST_HOP, 0.0, s);
                R.launches += 2;
                last_done = true;
                break;
            }
            if ((ell == 3 && hop3_sparse) || (ell == L - 1 && ball_hop)) {
                // hop ell computed where it can be non-zero (hop 3) or is read (hop L - 1), with the
                // fused gather of X_{ell-1}
                const bool ball = ell == L - 1 && ball_hop;
                const int64_t t = timer_open(R, s);
                launch_hop_sparse(g, prec_at(R, ell), B, ball, xa, xb, used_slices,
                                  ball ? g->mask.get() : g->mask_nz.get(), src, nsrc, g->tau_entry.get(), ell - 1,
                                  g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), R.rec, s);
                timer_close(R, t, ball ? SC_KC_BALL_HOP : SC_KC_SPARSE_HOP,
                            used_slices * (csr_bytes + mask_bytes +
                                           (ball ? 0.0 : static_cast<double>(n) * B * elem_size(prec_at(R, ell)))),
                            s);
                std::swap(xa, xb);
                R.launches += 1;
                continue;
            }
            // hop ell computes X_ell and, in its first CTAs, gathers X_{ell-1}
            HopLaunch h{xa, xb, used_slices, src, nsrc, g->tau_entry.get(), ell - 1,
                        g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), g->status.get(), R.rec};
            const int64_t t = timer_open(R, s);
            hop_mixed(R, h, ell, static_cast<size_t>(used_slices) * n * B, s, &xa, &xb);
            timer_close(R, t, SC_KC_DENSE_HOP, used_slices * hop_bytes_per_slice(ell), s);
            ++R.hop_launches;
            R.launches += prec_at(R, ell - 1) != prec_at(R, ell) ? 2 : 1;
            R.alg_bytes += used_slices * hop_bytes_per_slice(ell);
        }
        if (!last_done) {
            launch_first_or_gather(g, prec_at(R, tt), B, false, xa, src, nsrc, g->tau_entry.get(), tt,
                                   g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), R.rec, s);
            R.launches += 1;
        }
        R.hops += tt;
        R.source_hops += static_cast<int64_t>(tt) * nsrc;
        if (R.depth)
            for (int q = 0; q < nsrc; ++q)
                if (h_src[first + q] >= 0) (*R.depth)[h_src[first + q]] = per_source && src_tt[q] >= 0 ? src_tt[q] : tt;
        if (per_source) {
            for (int q = 0; q < nsrc; ++q) {
                if (h_src[first + q] < 0) continue;
                const int32_t t_q = src_tt[q] >= 0 ? src_tt[q] : tt;
                R.tt_min = std::min(R.tt_min, t_q);
                R.tt_max = std::max(R.tt_max, t_q);
            }
        } else if (R.plus) {
            R.tt_min = std::min(R.tt_min, tt);
            R.tt_max = std::max(R.tt_max, tt);
            prev_L = L;
            prev_tt = tt < L ? tt : -1;
            if (tt < L) {
                // Algorithm 4's walk phase: walk tails from X_tt with the counts of the last check
                const double t0 = wall_ms();
                const int64_t tw_ev = timer_open(R, s);
                SC_CUDA(cudaEventRecord(ev_w0, s));
                long long wsteps = 0;
                const long long pairs = tgtplus_walks(g, prec_at(R, tt), B, xa, src, h_src.data() + first, nsrc,
                                                      g->tau_entry.get(), tt, R.o->seed, g->acc_g.get(), s, &wsteps);
                SC_CUDA(cudaEventRecord(ev_w1, s));
                timer_close(R, tw_ev, SC_KC_WALKS, 0.0, s);
                SC_CUDA(cudaEventSynchronize(ev_w1));
                R.walk_ms += wall_ms() - t0;
                R.launches += 3;
                R.walks += pairs;
                float wms = 0.f;
                SC_CUDA(cudaEventElapsedTime(&wms, ev_w0, ev_w1));
                R.walk_steps += wsteps;
                R.walk_device_ms += wms;
            }
        }
    }
    int32_t h_status = 0;
    SC_CUDA(cudaMemcpyAsync(&h_status, g->status.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    if (h_status & 1) SC_FAIL(SC_ERR_TIMEOUT, "a bounded mbarrier wait expired in the TMA hop kernel");
}

// ---------------------------------------------------------------------------
// the windowed block loop (the frontier as an interval, K1w): blocks never
// cross a segment (one graph of a batch, or the whole graph) and hold sources
// of one length; each slice stores and computes only its window, so a slice
// costs what its window holds instead of n rows. seg_start: segment
// boundaries (nseg + 1 entries); beta: bandwidth bound of every segment (0:
// the window is the whole segment).
//
// Launches: blocks are ordered by window size class (powers of two) and by
// length, longest first; a launch (super-block) takes consecutive blocks of
// one class up to a memory budget. Hop l of a super-block runs over its
// leading blocks with L >= l - 1 (the others are done): blocks with L >= l
// compute X_l, and all of them gather X_{l-1} (Algorithm 2's accumulation of Eq. 9), which
// is the final gather of the blocks with L = l - 1. With R.capture the whole
// loop is recorded into one CUDA graph and replayed as one launch.
// ---------------------------------------------------------------------------
struct WinBlock {
    int64_t first;  // first entry in the padded source list (multiple of B)
    SliceWin w;
    int cls;        // window size class
};

struct CaptureGuard {  // ends a stream capture left open by an exception
    cudaStream_t s;
    bool open = false;
    ~CaptureGuard() {
        if (open) {
            cudaGraph_t gr = nullptr;
            cudaStreamEndCapture(s, &gr);
            if (gr) cudaGraphDestroy(gr);
        }
    }
};

static void run_blocks_win(Run &R, std::vector<int32_t> sources, const std::vector<int32_t> &len,
                           const std::vector<int32_t> &seg_start, int32_t beta,
                           const std::vector<char> &seg_bipartite = {}) {
    sc_graph *g = R.g;
    cudaStream_t s = R.s;
    const int B = R.B;
    const size_t elem = alloc_elem(R.prec, R.h0);
    if (R.plus) SC_FAIL(SC_ERR_UNSUPPORTED, "TGT+ has no windowed form");
    sources.erase(std::remove_if(sources.begin(), sources.end(), [&](int32_t v) { return len[v] + R.extra <= 0; }),
                  sources.end());
    if (sources.empty()) return;
    auto seg_of = [&](int32_t v) {
        return static_cast<int32_t>(std::upper_bound(seg_start.begin(), seg_start.end(), v) - seg_start.begin()) - 1;
    };
    // colour (BFS depth parity) of the sources of bipartite segments, -1 elsewhere: blocks of one
    // colour compute half the rows per hop (SliceWin::parity)
    const bool any_bip = std::any_of(seg_bipartite.begin(), seg_bipartite.end(), [](char c) { return c != 0; });
    std::vector<int32_t> colour(any_bip ? g->n : 0, -1);
    if (any_bip) {
        std::vector<int32_t> lev(g->n);
        SC_CUDA(cudaMemcpyAsync(lev.data(), g->level.get(), g->n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
        for (int32_t v : sources)
            if (seg_bipartite[seg_of(v)]) colour[v] = lev[v] & 1;
    }
    auto colour_of = [&](int32_t v) { return any_bip ? colour[v] : -1; };
    std::sort(sources.begin(), sources.end(), [&](int32_t a, int32_t b) {
        if (len[a] != len[b]) return len[a] > len[b];
        const int32_t sa = any_bip ? seg_of(a) : 0, sb = any_bip ? seg_of(b) : 0;
        if (sa != sb) return sa < sb;
        if (colour_of(a) != colour_of(b)) return colour_of(a) < colour_of(b);
        return a < b;
    });
    // blocks: up to B sources of one segment, one length and (bipartite segments) one colour
    std::vector<WinBlock> blocks;
    std::vector<std::vector<int32_t>> block_src;
    for (size_t i = 0; i < sources.size();) {
        const int32_t v0 = sources[i], sg = seg_of(v0), l0 = len[v0], c0 = colour_of(v0);
        size_t j = i;
        int32_t lo = v0, hi = v0;
        while (j < sources.size() && static_cast<int>(j - i) < B && len[sources[j]] == l0 && seg_of(sources[j]) == sg &&
               colour_of(sources[j]) == c0) {
            lo = std::min(lo, sources[j]);
            hi = std::max(hi, sources[j]);
            ++j;
        }
        WinBlock b{};
        SliceWin &w = b.w;
        w.parity = c0;
        w.L = l0 + R.extra;
        w.seg_lo = seg_start[sg];
        w.seg_hi = seg_start[sg + 1];
        w.src_lo = lo;
        w.src_hi = hi + 1;
        // storage: every row hop L + 1 may read (the neighbours of hop L's window)
        int32_t a, e;
        window_rows(w, beta, w.L + 1, &a, &e);
        w.base = a;
        w.rows = e - a;
        const auto &H = g->h_heavy_ids;
        w.heavy_begin = static_cast<int32_t>(std::lower_bound(H.begin(), H.end(), w.seg_lo) - H.begin());
        w.heavy_cnt = static_cast<int32_t>(std::lower_bound(H.begin(), H.end(), w.seg_hi) - H.begin()) - w.heavy_begin;
        b.cls = 0;
        while ((1 << b.cls) < w.rows && b.cls < 31) ++b.cls;
        blocks.push_back(b);
        block_src.emplace_back(sources.begin() + i, sources.begin() + j);
        i = j;
    }
    std::vector<size_t> order(blocks.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        return blocks[a].cls != blocks[b].cls ? blocks[a].cls < blocks[b].cls : blocks[a].w.L > blocks[b].w.L;
    });
    {
        std::vector<WinBlock> sorted;
        std::vector<int32_t> h;
        for (size_t q : order) {
            WinBlock b = blocks[q];
            b.first = static_cast<int64_t>(sorted.size()) * B;
            sorted.push_back(b);
        }
        blocks.swap(sorted);
    }
    std::vector<int32_t> h_src(blocks.size() * B, -1);
    for (size_t q = 0; q < order.size(); ++q)
        std::copy(block_src[order[q]].begin(), block_src[order[q]].end(), h_src.begin() + static_cast<int64_t>(q) * B);
    // super-blocks: consecutive blocks of one class within a memory budget per
    // ping-pong buffer (the windows of one launch need not share L2: a
    // launch's CTAs run slice after slice)
    size_t free_b = 0, total_b = 0;
    SC_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double budget = std::max(static_cast<double>(R.slice_bytes),
                                   std::min(4.0 * (1ull << 30), 0.125 * static_cast<double>(free_b)));
    const int max_sl = R.o->max_slices > 0 ? std::min(R.o->max_slices, 65535) : 65535;
    std::vector<size_t> sb_begin;
    size_t need = 0;
    for (size_t i = 0; i < blocks.size();) {
        sb_begin.push_back(i);
        double bytes = 0.0;
        int64_t off = 0;
        size_t j = i;
        while (j < blocks.size() && static_cast<int>(j - i) < max_sl && blocks[j].cls == blocks[i].cls) {
            const double add = static_cast<double>(blocks[j].w.rows) * B * elem;
            if (j > i && bytes + add > budget) break;
            bytes += add;
            blocks[j].w.xoff = off;
            off += static_cast<int64_t>(blocks[j].w.rows) * B;
            ++j;
        }
        need = std::max(need, static_cast<size_t>(off) * elem);
        i = j;
    }
    sb_begin.push_back(blocks.size());
    std::vector<SliceWin> h_win(blocks.size());
    for (size_t i = 0; i < blocks.size(); ++i) h_win[i] = blocks[i].w;
    g->src_list.reserve(h_src.size());
    g->win_list.reserve(h_win.size() * sizeof(SliceWin));
    g->xa.reserve(need);
    g->xb.reserve(need);
    SC_CUDA(cudaMemcpyAsync(g->src_list.get(), h_src.data(), h_src.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(g->win_list.get(), h_win.data(), h_win.size() * sizeof(SliceWin), cudaMemcpyHostToDevice, s));
    const SliceWin *d_win = reinterpret_cast<const SliceWin *>(g->win_list.get());
    const bool timed = R.time_kernels && !R.capture;
    const auto &hrp = g->h_row_ptr;
    // capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is replayed on the caller's
    struct StreamGuard {
        cudaStream_t c = nullptr;
        ~StreamGuard() {
            if (c) cudaStreamDestroy(c);
        }
    } cs;
    cudaStream_t is = s;
    if (R.capture) {
        SC_CUDA(cudaStreamSynchronize(s));
        SC_CUDA(cudaStreamCreateWithFlags(&cs.c, cudaStreamNonBlocking));
        is = cs.c;
    }
    CaptureGuard cap{is};
    if (R.capture) {
        SC_CUDA(cudaStreamBeginCapture(is, cudaStreamCaptureModeThreadLocal));
        cap.open = true;
    }
    for (size_t q = 0; q + 1 < sb_begin.size(); ++q) {
        const size_t b0 = sb_begin[q], b1 = sb_begin[q + 1];
        const int32_t Lmax = blocks[b0].w.L;
        const int32_t *src = g->src_list.get() + blocks[b0].first;
        const SliceWin *win = d_win + b0;
        size_t bytes = 0;
        for (size_t b = b0; b < b1; ++b) {
            bytes += static_cast<size_t>(blocks[b].w.rows) * B * elem;
            int32_t cnt = 0;
            for (int64_t t = blocks[b].first; t < blocks[b].first + B; ++t) cnt += h_src[t] >= 0;
            R.ell_min_src = std::min(R.ell_min_src, blocks[b].w.L);
            R.ell_max_src = std::max(R.ell_max_src, blocks[b].w.L);
            R.source_hops += static_cast<int64_t>(blocks[b].w.L) * cnt;
            R.hops += blocks[b].w.L;
        }
        void *xa = g->xa.get(), *xb = g->xb.get();
        SC_CUDA(cudaMemsetAsync(xa, 0, bytes, is));
        SC_CUDA(cudaMemsetAsync(xb, 0, bytes, is));
        launch_first_or_gather(g, prec_at(R, 1), B, true, xa, src, static_cast<int>(b1 - b0) * B, nullptr, 1, nullptr,
                               nullptr, nullptr, R.rec, is, win);
        R.launches += 1;
        size_t active = b1 - b0;
        for (int32_t ell = 2; ell <= Lmax; ++ell) {
            while (active > 0 && blocks[b0 + active - 1].w.L < ell - 1) --active;
            int heavy_max = 0;
            int64_t rows_max = 0;
            double hop_bytes = 0.0;
            for (size_t b = b0; b < b0 + active; ++b) {
                if (blocks[b].w.L < ell) continue;
                int32_t lo, hi;
                window_rows(blocks[b].w, beta, ell, &lo, &hi);
                heavy_max = std::max(heavy_max, blocks[b].w.heavy_cnt);
                rows_max = std::max<int64_t>(rows_max, hi - lo);
                hop_bytes += 4.0 * (hrp[hi] - hrp[lo]) + 4.0 * (hi - lo + 1) +
                             (R.prec == SC_PREC_FP64 ? 8.0 : 4.0) * (hi - lo) +
                             static_cast<double>(hi - lo) * B *
                                 (elem_size(prec_at(R, ell - 1)) + elem_size(prec_at(R, ell)));
            }
            const int used = static_cast<int>(active);
            HopLaunch h{xa, xb, used, src, used * B, g->tau_entry.get(), ell - 1,
                        g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), g->status.get(), R.rec};
            h.win = win;
            h.ell = ell;
            h.beta = beta;
            h.win_heavy = heavy_max;
            h.win_rows = rows_max;
            const int64_t t = timed ? timer_open(R, is) : -1;
            hop_mixed(R, h, ell, bytes / elem, is, &xa, &xb, true);
            timer_close(R, t, SC_KC_DENSE_HOP, hop_bytes, is);
            ++R.hop_launches;
            R.launches += prec_at(R, ell - 1) != prec_at(R, ell) ? 2 : 1;
            R.alg_bytes += hop_bytes;
        }
        // final gather of the blocks that run all Lmax hops (a leading run)
        size_t last = 0;
        while (b0 + last < b1 && blocks[b0 + last].w.L == Lmax) ++last;
        launch_first_or_gather(g, prec_at(R, Lmax), B, false, xa, src, static_cast<int>(last) * B, g->tau_entry.get(), Lmax,
                               g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), R.rec, is, win);
        R.launches += 1;
    }
    if (R.capture) {
        cudaGraph_t gr = nullptr;
        cap.open = false;
        SC_CUDA(cudaStreamEndCapture(is, &gr));
        cudaGraphExec_t ex = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) SC_FAIL(SC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        const cudaError_t e2 = cudaGraphLaunch(ex, s);
        cudaGraphExecDestroy(ex);  // freed once the launch completes
        if (e2 != cudaSuccess) SC_FAIL(SC_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e2));
        R.graph_launches += 1;
    }
}

// ---------------------------------------------------------------------------
// sc_all_edges
// ---------------------------------------------------------------------------
// Block width from one real block per width. autotune() models a block by its
// dense hops and leaves out the kernels that run once per block (hops 1-2 from
// the sources' masks, the last hop on the gather's rows), whose cost per source
// grows as the block narrows. Here, for the best lane split of each width, one
// launch worth of sample sources (spread over the ids; a contiguous id run for
// windowed blocks, whose cost depends on the sources' id range) runs through
// the block loop itself at min(L, kTuneHops) hops with their own lengths; a
// source's cost is that time per source plus the remaining hops at the width's
// measured hop cost. Two rounds after a warm-up, interleaved over the widths,
// the least kept; cached per request key. The traversal only (no TGT+ test or
// walk, no records). The sample's gathers write the accumulators, which the
// caller resets afterwards.
static TuneResult pick_block_width(const Run &base, const std::vector<TuneResult> &per_b,
                                   const std::vector<int32_t> &len, int32_t Lmax, bool use_win, int32_t beta,
                                   const std::vector<char> &bip, long long key) {
    sc_graph *g = base.g;
    cudaStream_t s = base.s;
    auto hit = g->tuned_block.find(key);
    if (hit != g->tuned_block.end()) return hit->second;
    const int32_t n = g->n;
    const size_t elem = alloc_elem(base.prec, base.h0);
    const int32_t Ls = std::min(Lmax, kTuneHops);
    size_t need = 0;
    for (const auto &c : per_b)
        need = std::max(need, slices_for(g, c.B, elem, base.o->max_slices) * static_cast<size_t>(n) * c.B * elem);
    g->xa.reserve(need);
    g->xb.reserve(need);
    cudaEvent_t e0, e1;
    SC_CUDA(cudaEventCreate(&e0));
    SC_CUDA(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evg{e0, e1};
    std::vector<double> best(per_b.size(), INFINITY);
    std::vector<int32_t> ls(len);
    const std::vector<int32_t> seg_whole{0, n};
    for (int round = 0; round < 3; ++round) {
        for (size_t ci = 0; ci < per_b.size(); ++ci) {
            const TuneResult &c = per_b[ci];
            Run R = base;
            R.B = c.B;
            R.vpl = c.vpl;
            R.slices = slices_for(g, c.B, elem, base.o->max_slices);
            R.slice_bytes = static_cast<size_t>(n) * c.B * elem;
            R.plus = false;
            R.time_kernels = false;
            R.depth = nullptr;
            R.capture = false;
            R.extra = 0;
            R.rec = GatherRec{base.rec.mode, nullptr, 0};
            const int32_t cnt = static_cast<int32_t>(std::min<int64_t>(static_cast<int64_t>(R.slices) * c.B, n));
            std::vector<int32_t> src(cnt);
            const int32_t lo = use_win ? (n - cnt) / 2 : 0;
            for (int32_t q = 0; q < cnt; ++q) {
                const int32_t v = use_win ? lo + q : static_cast<int32_t>((static_cast<int64_t>(q) * n) / cnt);
                src[q] = v;
                ls[v] = std::min(len[v] + base.extra, Ls);
            }
            SC_CUDA(cudaEventRecord(e0, s));
            if (use_win) run_blocks_win(R, src, ls, seg_whole, beta, bip);
            else run_blocks(R, src, ls);
            SC_CUDA(cudaEventRecord(e1, s));
            SC_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            SC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            for (int32_t q = 0; q < cnt; ++q) ls[src[q]] = len[src[q]];
            if (round == 0) continue;  // warm-up
            const double per_source = ms / cnt + std::max(Lmax - Ls, 0) * c.ms_per_source_hop;
            best[ci] = std::min(best[ci], per_source);
        }
    }
    size_t pick = 0;
    const bool log = std::getenv("SC_AUTOTUNE_LOG") != nullptr;
    for (size_t ci = 0; ci < per_b.size(); ++ci) {
        if (log)
            std::fprintf(stderr, "sc block width: B %d split %d: %.4f us per source (sample block of %d hops, L %d)\n",
                         per_b[ci].B, per_b[ci].vpl == 0 ? -1 : per_b[ci].vpl, 1e3 * best[ci], Ls, Lmax);
        if (best[ci] < best[pick]) pick = ci;
    }
    g->tuned_block[key] = per_b[pick];
    return per_b[pick];
}

static void all_edges_impl(sc_graph *g, const sc_options *o_in, double *s_hat, double *tail_bound, sc_report *rep,
                           double *rec_all = nullptr, int rec_stride = 0, const EdgeSubset *sub = nullptr) {
    if (!g || (!s_hat && !sub)) SC_FAIL(SC_ERR_INVALID_ARG, "null graph or output");
    if (sub) {
        if (sub->count < 1 || !sub->entries || !sub->out) SC_FAIL(SC_ERR_INVALID_ARG, "need count >= 1 entries and an output");
        for (int64_t t = 0; t < sub->count; ++t)
            if (sub->entries[t] < 0 || sub->entries[t] >= g->nnz)
                SC_FAIL(SC_ERR_INVALID_ARG, "entries[%lld] = %lld outside [0, nnz)", static_cast<long long>(t),
                        static_cast<long long>(sub->entries[t]));
    }
    sc_options o;
    if (o_in) o = *o_in;
    else sc_options_default(&o);
    if (!(o.eps > 0.0 && o.eps < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "eps must lie in (0, 1), got %g", o.eps);
    if (o.precision < SC_PREC_FP64 || o.precision > SC_PREC_BF16) SC_FAIL(SC_ERR_INVALID_ARG, "precision %d", o.precision);
    if (o.bf16_from_hop < 0) SC_FAIL(SC_ERR_INVALID_ARG, "bf16_from_hop %d < 0", o.bf16_from_hop);
    if (o.mode != SC_MODE_TGT && o.mode != SC_MODE_TGT_PLUS) SC_FAIL(SC_ERR_INVALID_ARG, "mode %d", o.mode);
    const bool plus = o.mode == SC_MODE_TGT_PLUS;
    if (plus && (o.estimator != SC_EST_PLAIN || (o.flags & SC_OPT_RECORD_TAIL)))
        SC_FAIL(SC_ERR_UNSUPPORTED, "TGT+ takes the plain estimator and no tail records");
    const int gamma = o.gamma < 0 ? 10 : o.gamma;
    if (plus && gamma > kGammaMax) SC_FAIL(SC_ERR_UNSUPPORTED, "gamma %d above %d", gamma, kGammaMax);
    if (o.switch_rule < SC_SWITCH_COST || o.switch_rule > SC_SWITCH_PER_SOURCE)
        SC_FAIL(SC_ERR_INVALID_ARG, "switch rule %d", o.switch_rule);
    if (o.ell_policy < SC_ELL_GLOBAL || o.ell_policy > SC_ELL_CALTAU) SC_FAIL(SC_ERR_INVALID_ARG, "length policy %d", o.ell_policy);
    const bool caltau = o.ell_policy == SC_ELL_CALTAU;
    if (caltau && plus) SC_FAIL(SC_ERR_UNSUPPORTED, "the CalTau lengths serve TGT");
    if (caltau && (!g->caltau_ready || g->caltau_eps != o.eps))
        SC_FAIL(SC_ERR_INVALID_ARG, "no CalTau lengths for eps %g: call sc_caltau with it first", o.eps);
    if (o.ell_policy == SC_ELL_FIXED && o.ell_fixed < 0) SC_FAIL(SC_ERR_INVALID_ARG, "ell_fixed < 0");
    if (o.estimator != SC_EST_PLAIN && o.estimator != SC_EST_END_CORRECTED) SC_FAIL(SC_ERR_INVALID_ARG, "estimator");
    const bool learned = o.ell_policy == SC_ELL_LEARNED;
    if (learned && !g->mlp_loaded) SC_FAIL(SC_ERR_INVALID_ARG, "no model loaded: call sc_mlp_load first");
    // a bipartite graph has no bound and no a-priori length: the learned lengths are
    // accepted by the tail estimate (end-corrected estimator) and capped by opts.ell_cap.
    // With the end-corrected estimator the learned policy records hops tau-1 .. tau+2
    // (mode 3): the bound of R6' or the tail estimate, and the end correction
    const bool est_learned = learned && g->bipartite;
    const bool learned3 = learned && !plus && o.estimator == SC_EST_END_CORRECTED;
    if (learned && plus && o.estimator != SC_EST_PLAIN)
        SC_FAIL(SC_ERR_UNSUPPORTED, "TGT+ at learned lengths certifies the plain estimator");
    if (est_learned && plus) SC_FAIL(SC_ERR_UNSUPPORTED, "TGT+ needs lambda_star < 1: the graph is bipartite");
    if (est_learned && o.estimator != SC_EST_END_CORRECTED)
        SC_FAIL(SC_ERR_UNSUPPORTED, "the learned length on a bipartite graph needs the end-corrected estimator");
    if (est_learned && (o.ell_cap < 3 || (o.ell_cap & 1) == 0))
        SC_FAIL(SC_ERR_INVALID_ARG, "the learned length on a bipartite graph needs an odd ell_cap >= 3, got %d",
                o.ell_cap);
    const bool out_dev = (o.flags & SC_OUT_DEVICE) != 0;
    const bool time_kernels = (o.flags & SC_OPT_TIME_KERNELS) != 0;
    const bool record_after = (o.flags & SC_OPT_RECORD_TAIL) || o.estimator == SC_EST_END_CORRECTED;
    const bool need_lambda = (o.ell_policy != SC_ELL_FIXED && !caltau) || record_after;
    cudaStream_t s = g->stream;
    const int32_t n = g->n;
    const int64_t nnz = g->nnz;

    cudaEvent_t ev0, ev1, ev2;
    SC_CUDA(cudaEventCreate(&ev0));
    SC_CUDA(cudaEventCreate(&ev1));
    SC_CUDA(cudaEventCreate(&ev2));
    struct EvGuard {
        cudaEvent_t a, b, c;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            cudaEventDestroy(c);
        }
    } evg{ev0, ev1, ev2};
    SC_CUDA(cudaEventRecord(ev0, s));

    if (need_lambda && !g->has_lambda) {
        sc_lambda lam;
        sc_status st = estimate_lambda_impl(g, nullptr, &lam);
        if (st != SC_OK && st != SC_ERR_LAMBDA_NOT_CONVERGED) throw Failure{st};
    }
    if (o.ell_policy != SC_ELL_FIXED && !caltau && !est_learned && (g->bipartite || g->lam.lambda_star >= 1.0))
        SC_FAIL(SC_ERR_UNSUPPORTED, "lambda_star >= 1 (bipartite graph): no finite length meets eps; use a fixed "
                                    "length or the learned one with the end-corrected estimator");
    const double lam_star = g->lam.lambda_star;

    // ---- truncation lengths --------------------------------------------------
    g->tau_entry.reserve(nnz);
    DevBuf<int32_t> tau_src;
    tau_src.reserve(n);
    std::vector<int32_t> len(n);
    int32_t ell_global = 0;
    if (o.ell_policy == SC_ELL_FIXED) {
        ell_global = o.ell_fixed;
        std::fill(len.begin(), len.end(), o.ell_fixed);
        fill_i32(g->tau_entry.get(), nnz, o.ell_fixed, s);
    } else if (caltau) {
        // Algorithm 1's per-edge lengths; each source runs the longest of its edges
        SC_CUDA(cudaMemcpyAsync(g->tau_entry.get(), g->caltau_tau.get(), nnz * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, s));
        k_row_max<<<ceil_div(n, 256), 256, 0, s>>>(g->row_ptr.get(), g->tau_entry.get(), n, tau_src.get());
        SC_LAUNCH_CHECK();
        SC_CUDA(cudaMemcpyAsync(len.data(), tau_src.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
        ell_global = *std::max_element(len.begin(), len.end());
    } else if (est_learned) {
        // per-source lengths from the model, capped by the caller's longest length
        ell_global = o.ell_cap;
        learned_lengths(g, ell_global, tau_src.get(), s);
        k_tau_min_of_sources<<<ceil_div(n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), tau_src.get(), n,
                                                              g->tau_entry.get());
        k_row_max<<<ceil_div(n, 256), 256, 0, s>>>(g->row_ptr.get(), g->tau_entry.get(), n, tau_src.get());
        SC_LAUNCH_CHECK();
        SC_CUDA(cudaMemcpyAsync(len.data(), tau_src.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
    } else {
        // TGT+ (Algorithm 4) asks for a tail of at most eps/2 and leaves eps/2 to the walks
        tau_entries_device(g, plus ? 0.5 * o.eps : o.eps, lam_star, g->tau_entry.get(), tau_src.get(), &ell_global);
        if (o.ell_policy == SC_ELL_GLOBAL) {
            std::fill(len.begin(), len.end(), ell_global);
            fill_i32(g->tau_entry.get(), nnz, ell_global, s);
        } else if (o.ell_policy == SC_ELL_LEARNED) {
            // per-source lengths from the model, capped by the a-priori length of Eq. 6
            learned_lengths(g, ell_global, tau_src.get(), s);
            k_tau_min_of_sources<<<ceil_div(n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), tau_src.get(), n,
                                                                  g->tau_entry.get());
            k_row_max<<<ceil_div(n, 256), 256, 0, s>>>(g->row_ptr.get(), g->tau_entry.get(), n, tau_src.get());
            SC_LAUNCH_CHECK();
            SC_CUDA(cudaMemcpyAsync(len.data(), tau_src.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        } else {
            SC_CUDA(cudaMemcpyAsync(len.data(), tau_src.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        }
        SC_CUDA(cudaStreamSynchronize(s));
    }

    // ---- block configuration -------------------------------------------------
    const int heavy_t = o.heavy_threshold > 0 ? o.heavy_threshold : 256;
    ensure_row_order(g, heavy_t);
    if (o.block_width != 0 && o.block_width != 32 && o.block_width != 64 && o.block_width != 128)
        SC_FAIL(SC_ERR_INVALID_ARG, "block width %d not in {32, 64, 128}", o.block_width);
    if (o.rows_split < -1 || o.rows_split == 3 || o.rows_split > 4)
        SC_FAIL(SC_ERR_INVALID_ARG, "lane split %d not in {-1 (TMA gather), 1, 2, 4}", o.rows_split);
    ensure_partition(g, kTmaPartEntries);
    g->status.reserve(4);
    SC_CUDA(cudaMemsetAsync(g->status.get(), 0, 4 * sizeof(int32_t), s));
    // rows_split: 0 = automatic, -1 = the TMA-gather kernel, 1/2/4 = SIMT lane split
    const int fixV = o.rows_split == 0 ? -1 : (o.rows_split < 0 ? 0 : o.rows_split);
    // TGT+ at learned lengths records the half terms of the even hops its traversal reaches
    // (hops <= kEvenDepthCap) for the truncation check after the run
    const bool learned_plus = learned && plus;
    DevBuf<double> even_rec;
    int even_stride = 0;
    if (learned_plus) {
        even_stride = std::min(ell_global + 1, kEvenDepthCap) / 2 + 1;
        even_rec.reserve(static_cast<size_t>(nnz) * even_stride);
        rec_all = even_rec.get();
        rec_stride = even_stride;
    }
    // mode 3 records the terms of hops tau-1, tau here (and tau+1, tau+2 in t1 / t2)
    DevBuf<double> pre_rec;
    if (learned3) {
        pre_rec.reserve(static_cast<size_t>(nnz) * 2);
        rec_all = pre_rec.get();
        rec_stride = 2;
    }
    const GatherRec rec{learned_plus ? 2 : (learned3 ? 3 : (learned ? 1 : 0)), rec_all, rec_stride};
    g->acc_g.reserve(nnz);
    g->acc_t1.reserve(nnz);
    g->acc_t2.reserve(nnz);
    // windowed blocks (the frontier as an interval) when the graph's bandwidth
    // keeps a block's last window under half the graph, or when asked for
    const int32_t beta = ensure_bandwidth(g);
    // the longest run of the first pass (a learned length's cap is reached only by extensions,
    // which rerun few sources; the windows and the launch shape are chosen for the first pass)
    const int32_t Lmax = (len.empty() ? 0 : *std::max_element(len.begin(), len.end())) + (record_after ? 2 : 0);
    const bool use_win = !plus && o.rows_split != -1 && !(o.flags & SC_OPT_WINDOWS_OFF) &&
                         ((o.flags & SC_OPT_WINDOWS_FORCE) ||
                          2.0 * (Lmax + 1.0) * static_cast<double>(beta) + 128.0 < 0.5 * static_cast<double>(n));
    // a bf16 run whose early hops are fp32 is tuned (and its buffers sized) in fp32
    const int32_t h0 = bf16_first_hop(o);
    const int tune_prec = (o.precision == SC_PREC_BF16 && h0 > 1) ? SC_PREC_FP32 : o.precision;
    std::vector<TuneResult> per_b;
    const TuneResult tr = autotune(g, tune_prec, o.block_width, fixV, o.max_slices, Lmax,
                                   GatherRec{rec.mode, nullptr, 0}, !use_win, s, &per_b);
    Run R;
    R.g = g;
    R.o = &o;
    R.s = s;
    R.prec = o.precision;
    R.h0 = h0;
    R.B = tr.B;
    R.vpl = tr.vpl;
    const size_t elem = alloc_elem(R.prec, R.h0);
    R.slice_bytes = static_cast<size_t>(n) * R.B * elem;
    R.slices = slices_for(g, R.B, elem, o.max_slices);
    R.plus = plus;
    R.time_kernels = time_kernels;
    R.gamma = gamma;
    const double delta = o.delta > 0.0 ? o.delta : 1.0 / static_cast<double>(n);  // Section 5.1: delta = 1/n
    R.log2md = std::log(2.0 * static_cast<double>(nnz / 2) / delta);
    R.extra = record_after ? 2 : 0;
    R.rec = rec;
    if (per_b.size() > 1 && Lmax >= 2) {
        // the block width from one real block of each (the request's lengths, kernels and records)
        const long long key = (static_cast<long long>(tune_prec) << 56) ^ (static_cast<long long>(fixV + 1) << 52) ^
                              (static_cast<long long>(o.max_slices & 0xfff) << 40) ^
                              (static_cast<long long>(Lmax) << 16) ^ (static_cast<long long>(use_win) << 15) ^
                              (static_cast<long long>(rec.mode) << 12) ^
                              (static_cast<long long>((o.flags & SC_OPT_SPARSE_HOPS) != 0) << 11) ^
                              (static_cast<long long>(o.ell_policy) << 8) ^ (static_cast<long long>(o.estimator) << 6) ^
                              (static_cast<long long>(plus) << 5) ^ static_cast<long long>(std::min(h0, 31));
        const TuneResult t2 = pick_block_width(R, per_b, len, Lmax, use_win, beta,
                                               std::vector<char>{static_cast<char>(g->bipartite ? 1 : 0)}, key);
        R.B = t2.B;
        R.vpl = t2.vpl;
        R.slice_bytes = static_cast<size_t>(n) * R.B * elem;
        R.slices = slices_for(g, R.B, elem, o.max_slices);
    }
    std::vector<int32_t> depth;
    if (learned_plus) {
        depth.assign(n, 0);
        R.depth = &depth;
    }
    const int64_t nblocks_total = (static_cast<int64_t>(n) + R.B - 1) / R.B;

    g->xa.reserve(R.slices * R.slice_bytes);
    g->xb.reserve(R.slices * R.slice_bytes);
    k_reset_rows<<<ceil_div(n, 8), 256, 0, s>>>(g->row_ptr.get(), nullptr, n, g->tau_entry.get(), R.rec.mode,
                                                g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), rec_all, rec_stride);
    SC_LAUNCH_CHECK();
    R.launches = 2 + (o.ell_policy == SC_ELL_FIXED ? 0 : 1) + (learned ? 4 : 0);
    if (plus) tgtplus_reserve(g, R.slices, R.B);

    // ---- propagation ----------------------------------------------------------
    SC_CUDA(cudaEventRecord(ev1, s));
    std::vector<int32_t> all;
    DevBuf<int32_t> active;   // sc_some_edges: the endpoints of the listed entries
    DevBuf<int64_t> d_entries;
    if (sub) {
        active.reserve(n);
        d_entries.reserve(sub->count);
        SC_CUDA(cudaMemsetAsync(active.get(), 0, n * sizeof(int32_t), s));
        SC_CUDA(cudaMemcpyAsync(d_entries.get(), sub->entries, sub->count * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        k_mark_endpoints<<<ceil_div(sub->count, 256), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), n,
                                                                  d_entries.get(), sub->count, active.get());
        SC_LAUNCH_CHECK();
        std::vector<int32_t> h_active(n);
        SC_CUDA(cudaMemcpyAsync(h_active.data(), active.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
        for (int32_t v = 0; v < n; ++v)
            if (h_active[v]) all.push_back(v);
        R.launches += 1;
    } else {
        all.resize(n);
        std::iota(all.begin(), all.end(), 0);
    }
    const std::vector<int32_t> seg_whole{0, n};
    auto run = [&](const std::vector<int32_t> &src, const std::vector<int32_t> &l) {
        if (use_win) run_blocks_win(R, src, l, seg_whole, beta, std::vector<char>{static_cast<char>(g->bipartite ? 1 : 0)});
        else run_blocks(R, src, l);
    };
    DevBuf<int32_t> tau_saved;
    if (learned_plus) {
        tau_saved.reserve(nnz);
        SC_CUDA(cudaMemcpyAsync(tau_saved.get(), g->tau_entry.get(), nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    run(all, len);

    // ---- combine, and for the learned lengths the check / extension loop ------
    DevBuf<double> tmp_s, tmp_b;
    double *d_s = s_hat;
    double *d_b = tail_bound;
    if (sub) {  // every entry's value in scratch; the listed ones are gathered at the end
        tmp_s.reserve(nnz);
        d_s = tmp_s.get();
        d_b = nullptr;
        if (learned && !plus) {
            tmp_b.reserve(nnz);
            d_b = tmp_b.get();
        }
    } else if (!out_dev) {
        tmp_s.reserve(nnz);
        d_s = tmp_s.get();
        if (tail_bound || (learned && !plus)) {
            tmp_b.reserve(nnz);
            d_b = tmp_b.get();
        }
    } else if (learned && !plus && !d_b) {
        tmp_b.reserve(nnz);
        d_b = tmp_b.get();
    }
    const bool have_tail = record_after || (learned && !plus);
    if (!have_tail) d_b = nullptr;
    // bound scales: after-records q = t_{tau+1} + t_{tau+2}: q / (2 (1 - lambda_plus)) (end-corrected) or
    // q / (1 - lambda*^2); learned (records of hops tau-1, tau): lambda*^2 / (1 - lambda*^2) (t_{tau-1} + t_tau).
    // lambda_plus carries its Ritz residual as a safety margin.
    double bound_scale = 0.0;
    if (learned && !plus && !learned3) {
        bound_scale = lam_star * lam_star / (1.0 - lam_star * lam_star);
    } else if (record_after) {
        const double lp = g->lam.lambda_plus + std::max(g->lam.residual_plus, 0.0);
        if (o.estimator == SC_EST_END_CORRECTED) bound_scale = lp < 1.0 ? 1.0 / (2.0 * (1.0 - lp)) : INFINITY;
        else bound_scale = lam_star < 1.0 ? 1.0 / (1.0 - lam_star * lam_star) : INFINITY;
    }
    auto combine = [&] {
        k_combine<<<ceil_div(n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), g->rev.get(), g->inv_deg_d.get(),
                                                 g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), n,
                                                 o.estimator == SC_EST_END_CORRECTED, have_tail ? 1 : 0, bound_scale,
                                                 d_s, d_b);
        SC_LAUNCH_CHECK();
        R.launches += 1;
    };
    combine();
    int64_t extended = 0;
    int32_t rounds = 0;
    if (learned_plus) {
        // certify each edge's truncation (eps/2) after the run; failing edges take a longer
        // length and both endpoints run again (their walks included), until every edge passes
        DevBuf<int32_t> row_flag, rows, d_depth, tau_target;
        row_flag.reserve(n);
        d_depth.reserve(n);
        tau_target.reserve(nnz);
        g->tp_counters.reserve(4);
        std::vector<int32_t> h_flag(n);
        // the per-source switch caps the lengths of switched rows in place: the targets are these
        SC_CUDA(cudaMemcpyAsync(tau_target.get(), tau_saved.get(), nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        while (true) {
            SC_CUDA(cudaMemcpyAsync(d_depth.get(), depth.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            SC_CUDA(cudaMemsetAsync(g->tp_counters.get(), 0, sizeof(long long), s));
            k_certify_plus<<<ceil_div(n, 8), 256, 0, s>>>(
                g->row_ptr.get(), g->col_idx.get(), g->rev.get(), g->inv_deg_d.get(), even_rec.get(), even_stride,
                d_depth.get(), sub ? active.get() : nullptr, n, lam_star, 0.5 * o.eps, ell_global, tau_target.get(),
                row_flag.get(),
                reinterpret_cast<unsigned long long *>(g->tp_counters.get()));
            SC_LAUNCH_CHECK();
            R.launches += 1;
            long long failing = 0;
            SC_CUDA(cudaMemcpyAsync(&failing, g->tp_counters.get(), sizeof(long long), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaMemcpyAsync(h_flag.data(), row_flag.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaStreamSynchronize(s));
            if (failing == 0) break;
            extended += failing / 2;
            ++rounds;
            std::vector<int32_t> redo;
            for (int32_t v = 0; v < n; ++v)
                if (h_flag[v]) redo.push_back(v);
            SC_CUDA(cudaMemcpyAsync(g->tau_entry.get(), tau_target.get(), nnz * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, s));
            k_row_max<<<ceil_div(n, 256), 256, 0, s>>>(g->row_ptr.get(), tau_target.get(), n, tau_src.get());
            SC_CUDA(cudaMemcpyAsync(len.data(), tau_src.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            rows.reserve(redo.size());
            SC_CUDA(cudaMemcpyAsync(rows.get(), redo.data(), redo.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            SC_CUDA(cudaStreamSynchronize(s));
            k_reset_rows<<<ceil_div(static_cast<int64_t>(redo.size()), 8), 256, 0, s>>>(
                g->row_ptr.get(), rows.get(), static_cast<int32_t>(redo.size()), g->tau_entry.get(), 2, g->acc_g.get(),
                g->acc_t1.get(), g->acc_t2.get(), rec_all, rec_stride);
            SC_LAUNCH_CHECK();
            R.launches += 2;
            run(redo, len);
        }
        combine();
    } else if (learned) {
        DevBuf<int32_t> row_flag, rows;
        row_flag.reserve(n);
        g->tp_counters.reserve(4);
        std::vector<int32_t> h_flag(n);
        while (true) {
            if (learned3) {  // the bound column: R6' from the recorded hops, or the tail estimate
                k_learned_check<<<ceil_div(n, 8), 256, 0, s>>>(
                    g->row_ptr.get(), g->col_idx.get(), g->rev.get(), g->inv_deg_d.get(), pre_rec.get(),
                    g->acc_t1.get(), g->acc_t2.get(), 3, nullptr,
                    est_learned ? -1.0 : lam_star * lam_star / (1.0 - lam_star * lam_star), g->tau_entry.get(), n,
                    d_b);
                SC_LAUNCH_CHECK();
                R.launches += 1;
            }
            SC_CUDA(cudaMemsetAsync(g->tp_counters.get(), 0, sizeof(long long), s));
            k_extend_failing<<<ceil_div(n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), d_b, n, o.eps,
                                                            ell_global, sub ? active.get() : nullptr,
                                                            g->tau_entry.get(), row_flag.get(),
                                                            reinterpret_cast<unsigned long long *>(g->tp_counters.get()));
            SC_LAUNCH_CHECK();
            R.launches += 1;
            long long failing = 0;
            SC_CUDA(cudaMemcpyAsync(&failing, g->tp_counters.get(), sizeof(long long), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaStreamSynchronize(s));
            if (failing == 0) break;
            extended += failing / 2;
            ++rounds;
            // rerun the marked sources with their extended lengths
            SC_CUDA(cudaMemcpyAsync(h_flag.data(), row_flag.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            k_row_max<<<ceil_div(n, 256), 256, 0, s>>>(g->row_ptr.get(), g->tau_entry.get(), n, tau_src.get());
            SC_CUDA(cudaMemcpyAsync(len.data(), tau_src.get(), n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaStreamSynchronize(s));
            std::vector<int32_t> redo;
            for (int32_t v = 0; v < n; ++v)
                if (h_flag[v]) redo.push_back(v);
            rows.reserve(redo.size());
            SC_CUDA(cudaMemcpyAsync(rows.get(), redo.data(), redo.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            k_reset_rows<<<ceil_div(static_cast<int64_t>(redo.size()), 8), 256, 0, s>>>(
                g->row_ptr.get(), rows.get(), static_cast<int32_t>(redo.size()), g->tau_entry.get(), rec.mode,
                g->acc_g.get(), g->acc_t1.get(), g->acc_t2.get(), rec_all, rec_stride);
            SC_LAUNCH_CHECK();
            R.launches += 2;
            run(redo, len);
            combine();
        }
    }
    SC_CUDA(cudaEventRecord(ev2, s));

    g->scratch_d.reserve(kRedBlocks + 8);
    DevBuf<double> sub_s, sub_b;
    int64_t red_count = nnz;
    if (sub) {  // the listed entries' values (and bounds), in the caller's order
        red_count = sub->count;
        sub_s.reserve(sub->count);
        k_gather_entries<<<ceil_div(sub->count, 256), 256, 0, s>>>(d_s, d_entries.get(), sub->count, sub_s.get());
        d_s = sub_s.get();
        if (d_b) {
            sub_b.reserve(sub->count);
            k_gather_entries<<<ceil_div(sub->count, 256), 256, 0, s>>>(d_b, d_entries.get(), sub->count, sub_b.get());
            d_b = sub_b.get();
        }
        SC_LAUNCH_CHECK();
        R.launches += d_b ? 2 : 1;
    }
    const double foster2 = device_reduce(d_s, red_count, false, g->scratch_d.get(), s);
    double max_bound = 0.0;
    if (d_b) max_bound = device_reduce(d_b, red_count, true, g->scratch_d.get(), s);
    R.launches += 2 + (d_b ? 2 : 0);
    if (sub) {
        SC_CUDA(cudaMemcpyAsync(sub->out, d_s, sub->count * sizeof(double),
                                out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    } else if (!out_dev) {
        SC_CUDA(cudaMemcpyAsync(s_hat, d_s, nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (tail_bound && d_b)
            SC_CUDA(cudaMemcpyAsync(tail_bound, d_b, nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
    } else if (tail_bound && d_b && d_b != tail_bound) {
        SC_CUDA(cudaMemcpyAsync(tail_bound, d_b, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    SC_CUDA(cudaStreamSynchronize(s));
    float prop_ms = 0.f, total_ms = 0.f;
    SC_CUDA(cudaEventElapsedTime(&prop_ms, ev1, ev2));
    SC_CUDA(cudaEventRecord(ev2, s));
    SC_CUDA(cudaEventSynchronize(ev2));
    SC_CUDA(cudaEventElapsedTime(&total_ms, ev0, ev2));
    double kc_ms[SC_KC_COUNT] = {};
    for (const auto &tk : R.timed) {
        float ms = 0.f;
        SC_CUDA(cudaEventElapsedTime(&ms, g->hop_events[2 * tk.second], g->hop_events[2 * tk.second + 1]));
        kc_ms[tk.first] += ms;
    }
    const double hop_ms = kc_ms[SC_KC_DENSE_HOP];
    double all_bytes = 0.0;
    for (int c = 0; c < SC_KC_COUNT; ++c) all_bytes += R.kc_bytes[c];
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        rep->ell_global = ell_global;
        rep->ell_min_source = R.ell_min_src == INT32_MAX ? 0 : R.ell_min_src;
        rep->ell_max_source = R.ell_max_src;
        rep->block_width = R.B;
        rep->rows_split = R.vpl == 0 ? -1 : R.vpl;
        rep->slices = R.slices;
        rep->blocks = nblocks_total;
        rep->launches = R.launches;
        rep->hops = R.hops;
        rep->source_hops = R.source_hops;
        rep->algorithmic_bytes = all_bytes;
        rep->foster_sum = sub ? foster2 : 0.5 * foster2;  // sc_some_edges: the sum of the listed entries' values
        rep->max_tail_bound = max_bound;
        rep->lambda_star = need_lambda ? lam_star : 0.0;
        rep->propagate_ms = prop_ms;
        rep->total_ms = total_ms;
        rep->hop_ms = hop_ms;
        rep->hop_launches = R.hop_launches;
        rep->hop_bytes = R.alg_bytes;
        rep->walks = R.walks;
        rep->edges_extended = static_cast<int32_t>(extended);
        rep->extension_rounds = rounds;
        rep->windowed = use_win ? 1 : 0;
        rep->uncertified = est_learned ? 1 : 0;
        rep->tt_min = plus ? (R.tt_min == INT32_MAX ? 0 : R.tt_min) : 0;
        rep->tt_max = plus ? R.tt_max : 0;
        rep->switch_tests = R.switch_tests;
        rep->switch_ms = R.switch_ms;
        rep->walk_ms = R.walk_ms;
        rep->walk_steps = R.walk_steps;
        rep->walk_device_ms = R.walk_device_ms;
        for (int c = 0; c < SC_KC_COUNT; ++c) {
            rep->kc_ms[c] = kc_ms[c];
            rep->kc_launches[c] = R.kc_launches[c];
            rep->kc_bytes[c] = R.kc_bytes[c];
        }
    }
}

// certified per-entry lengths for training labels: all sources run the
// a-priori length with every hop's half term recorded, then each edge takes
// the least odd tau whose bound lambda*^2/(1-lambda*^2) (t_{tau-1} + t_tau)
// is within eps (else the cap)
__global__ void k_certify(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                          const int32_t *__restrict__ rev, const double *__restrict__ inv_d,
                          const double *__restrict__ rec, int stride, int32_t n, int32_t cap, double factor, double eps,
                          int32_t *__restrict__ tau_out) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const double ir = inv_d[r];
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        const int32_t kr = rev[k];
        const double ij = inv_d[col[k]];
        auto full = [&](int l) {
            return __dadd_rn(__dmul_rn(rec[static_cast<int64_t>(k) * stride + l], ir),
                             __dmul_rn(rec[static_cast<int64_t>(kr) * stride + l], ij));
        };
        int32_t t = cap;
        for (int32_t c = 1; c <= cap; c += 2) {
            if (__dmul_rn(factor, __dadd_rn(full(c - 1), full(c))) <= eps) {
                t = c;
                break;
            }
        }
        tau_out[k] = t;
    }
}

void certified_lengths_impl(sc_graph *g, double eps, int precision, int32_t *per_entry_dev, int32_t *cap_out) {
    cudaStream_t s = g->stream;
    if (!g->has_lambda) {
        sc_lambda lam;
        sc_status st = estimate_lambda_impl(g, nullptr, &lam);
        if (st != SC_OK && st != SC_ERR_LAMBDA_NOT_CONVERGED) throw Failure{st};
    }
    const double lam = g->lam.lambda_star;
    if (!(lam < 1.0)) SC_FAIL(SC_ERR_UNSUPPORTED, "lambda_star >= 1: no finite length");
    int32_t cap = 0;
    {
        DevBuf<int32_t> te, ts;
        te.reserve(g->nnz);
        ts.reserve(g->n);
        tau_entries_device(g, eps, lam, te.get(), ts.get(), &cap);
    }
    DevBuf<double> rec, sh;
    const int stride = cap + 1;
    rec.reserve(static_cast<size_t>(g->nnz) * stride);
    sh.reserve(g->nnz);
    sc_options o;
    sc_options_default(&o);
    o.eps = eps;
    o.precision = precision;
    o.ell_policy = SC_ELL_FIXED;
    o.ell_fixed = cap;
    o.flags = SC_OUT_DEVICE;
    all_edges_impl(g, &o, sh.get(), nullptr, nullptr, rec.get(), stride);
    k_certify<<<ceil_div(g->n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), g->rev.get(), g->inv_deg_d.get(),
                                                rec.get(), stride, g->n, cap, lam * lam / (1.0 - lam * lam), eps,
                                                per_entry_dev);
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaStreamSynchronize(s));
    *cap_out = cap;
}

// training labels on a bipartite graph: every source runs cap + 2 hops with
// every hop's half term recorded (end-corrected estimator), then each edge
// takes the least odd tau in [3, cap] whose tail estimate is within eps
void estimated_lengths_impl(sc_graph *g, double eps, int precision, int32_t cap, int32_t *per_entry_dev) {
    cudaStream_t s = g->stream;
    if (!g->bipartite) SC_FAIL(SC_ERR_UNSUPPORTED, "the graph is not bipartite: its lengths are certified by a bound");
    if (cap < 3 || (cap & 1) == 0) SC_FAIL(SC_ERR_INVALID_ARG, "cap must be odd and >= 3, got %d", cap);
    DevBuf<double> rec, sh;
    const int stride = cap + 3;
    rec.reserve(static_cast<size_t>(g->nnz) * stride);
    sh.reserve(g->nnz);
    sc_options o;
    sc_options_default(&o);
    o.eps = eps;
    o.precision = precision;
    o.ell_policy = SC_ELL_FIXED;
    o.ell_fixed = cap;
    o.estimator = SC_EST_END_CORRECTED;
    o.flags = SC_OUT_DEVICE;
    all_edges_impl(g, &o, sh.get(), nullptr, nullptr, rec.get(), stride);
    k_estimate_lengths<<<ceil_div(g->n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), g->rev.get(),
                                                         g->inv_deg_d.get(), rec.get(), stride, g->n, cap, eps,
                                                         per_entry_dev);
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// batched traversal over many independent graphs: their disjoint union is
// propagated in windowed blocks (one graph per block, window = that graph's
// rows), recorded into one CUDA graph
// ---------------------------------------------------------------------------
__global__ void k_offset_copy(int32_t *__restrict__ dst, const int32_t *__restrict__ src, int64_t count, int32_t add) {
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < count) dst[i] = src[i] + add;
}

// per-segment sums of x over [off[i], off[i + 1]) in a fixed order (one CTA each)
__global__ void k_segment_sum(const double *__restrict__ x, const int64_t *__restrict__ off, double *__restrict__ out) {
    __shared__ double sh[256];
    const int64_t a = off[blockIdx.x], b = off[blockIdx.x + 1];
    double acc = 0.0;
    for (int64_t k = a + threadIdx.x; k < b; k += 256) acc += x[k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

static void batch_impl(sc_graph *const *graphs, int32_t count, const sc_options *o_in, const int32_t *ell_per_graph,
                       double *const *s_hat, sc_report *reports) {
    if (!graphs || count < 1 || !s_hat) SC_FAIL(SC_ERR_INVALID_ARG, "need count >= 1 graphs and outputs");
    sc_options o;
    if (o_in) o = *o_in;
    else sc_options_default(&o);
    if (!(o.eps > 0.0 && o.eps < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "eps must lie in (0, 1), got %g", o.eps);
    if (o.precision < SC_PREC_FP64 || o.precision > SC_PREC_BF16) SC_FAIL(SC_ERR_INVALID_ARG, "precision %d", o.precision);
    if (o.bf16_from_hop < 0) SC_FAIL(SC_ERR_INVALID_ARG, "bf16_from_hop %d < 0", o.bf16_from_hop);
    if (o.mode != SC_MODE_TGT) SC_FAIL(SC_ERR_UNSUPPORTED, "batches run TGT (Algorithm 2) only");
    const bool learned = o.ell_policy == SC_ELL_LEARNED;
    if (o.ell_policy != SC_ELL_GLOBAL && o.ell_policy != SC_ELL_FIXED && !learned)
        SC_FAIL(SC_ERR_UNSUPPORTED, "batches take the Eq. 6, a fixed or the learned length");
    if (o.ell_policy == SC_ELL_FIXED && o.ell_fixed < 0) SC_FAIL(SC_ERR_INVALID_ARG, "ell_fixed < 0");
    if (o.estimator != SC_EST_PLAIN && o.estimator != SC_EST_END_CORRECTED) SC_FAIL(SC_ERR_INVALID_ARG, "estimator");
    if (o.rows_split == -1) SC_FAIL(SC_ERR_UNSUPPORTED, "the TMA-gather hop has no windowed form");
    if (o.rows_split < -1 || o.rows_split == 3 || o.rows_split > 4) SC_FAIL(SC_ERR_INVALID_ARG, "lane split %d", o.rows_split);
    if (o.block_width != 0 && o.block_width != 32 && o.block_width != 64 && o.block_width != 128)
        SC_FAIL(SC_ERR_INVALID_ARG, "block width %d not in {32, 64, 128}", o.block_width);
    const bool out_dev = (o.flags & SC_OUT_DEVICE) != 0;
    const bool record_after = (o.flags & SC_OPT_RECORD_TAIL) || o.estimator == SC_EST_END_CORRECTED;
    const int extra = record_after ? 2 : 0;
    int dev = -1;
    for (int32_t i = 0; i < count; ++i) {
        if (!graphs[i] || !s_hat[i]) SC_FAIL(SC_ERR_INVALID_ARG, "graph or output %d is NULL", i);
        if (dev >= 0 && graphs[i]->device != dev) SC_FAIL(SC_ERR_INVALID_ARG, "graphs on different devices");
        dev = graphs[i]->device;
        if (ell_per_graph && ell_per_graph[i] < 0) SC_FAIL(SC_ERR_INVALID_ARG, "ell_per_graph[%d] < 0", i);
    }
    cudaStream_t s = graphs[0]->stream;
    cudaEvent_t ev0, ev1, ev2;
    SC_CUDA(cudaEventCreate(&ev0));
    SC_CUDA(cudaEventCreate(&ev1));
    SC_CUDA(cudaEventCreate(&ev2));
    struct EvGuard {
        cudaEvent_t a, b, c;
        ~EvGuard() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            cudaEventDestroy(c);
        }
    } evg{ev0, ev1, ev2};
    SC_CUDA(cudaEventRecord(ev0, s));

    // ---- per-graph lengths: an override, the fixed length, or Eq. 6 with the graph's own lambda*;
    // with the learned policy these are the caps (Eq. 6; on a bipartite graph opts.ell_cap or the
    // override) and each source takes its model's prediction
    std::vector<int32_t> ell(count);
    std::vector<double> lam(count, 0.0);
    std::vector<int64_t> n_off(count + 1, 0), k_off(count + 1, 0);
    int32_t big = 0;
    for (int32_t i = 0; i < count; ++i) {
        sc_graph *g = graphs[i];
        SC_CUDA(cudaStreamSynchronize(g->stream));
        const int32_t over = ell_per_graph ? ell_per_graph[i] : 0;
        if (learned) {
            if (!g->mlp_loaded) SC_FAIL(SC_ERR_INVALID_ARG, "graph %d: no model loaded: call sc_mlp_load first", i);
            if (!g->has_lambda) {
                sc_lambda l;
                sc_status st = estimate_lambda_impl(g, nullptr, &l);
                if (st != SC_OK && st != SC_ERR_LAMBDA_NOT_CONVERGED) throw Failure{st};
            }
            if (g->bipartite) {
                if (o.estimator != SC_EST_END_CORRECTED)
                    SC_FAIL(SC_ERR_UNSUPPORTED, "graph %d is bipartite: the learned length needs the end-corrected "
                                                "estimator", i);
                ell[i] = over > 0 ? over : o.ell_cap;
                if (ell[i] < 3 || (ell[i] & 1) == 0)
                    SC_FAIL(SC_ERR_INVALID_ARG, "graph %d is bipartite: its cap (ell_cap or the override) must be odd "
                                                "and >= 3, got %d", i, ell[i]);
            } else {
                if (g->lam.lambda_star >= 1.0) SC_FAIL(SC_ERR_UNSUPPORTED, "graph %d: lambda_star >= 1", i);
                lam[i] = g->lam.lambda_star;
                g->tau_entry.reserve(g->nnz);
                DevBuf<int32_t> ts;
                ts.reserve(g->n);
                tau_entries_device(g, o.eps, lam[i], g->tau_entry.get(), ts.get(), &ell[i]);
                if (over > 0) ell[i] = over;
            }
        } else if (over > 0) {
            ell[i] = over;
        } else if (o.ell_policy == SC_ELL_FIXED) {
            ell[i] = o.ell_fixed;
        } else {
            if (!g->has_lambda) {
                sc_lambda l;
                sc_status st = estimate_lambda_impl(g, nullptr, &l);
                if (st != SC_OK && st != SC_ERR_LAMBDA_NOT_CONVERGED) throw Failure{st};
            }
            if (g->bipartite || g->lam.lambda_star >= 1.0)
                SC_FAIL(SC_ERR_UNSUPPORTED, "graph %d: lambda_star >= 1 (bipartite): give it a length in ell_per_graph", i);
            lam[i] = g->lam.lambda_star;
            g->tau_entry.reserve(g->nnz);
            DevBuf<int32_t> ts;
            ts.reserve(g->n);
            tau_entries_device(g, o.eps, lam[i], g->tau_entry.get(), ts.get(), &ell[i]);
        }
        n_off[i + 1] = n_off[i] + g->n;
        k_off[i + 1] = k_off[i] + g->nnz;
        if (g->nnz > graphs[big]->nnz) big = i;
    }
    if (n_off[count] >= (int64_t(1) << 31) || k_off[count] >= (int64_t(1) << 31))
        SC_FAIL(SC_ERR_INVALID_ARG, "the batch holds 2^31 nodes or entries or more");
    const int32_t N = static_cast<int32_t>(n_off[count]);
    const int64_t NNZ = k_off[count];

    // ---- the disjoint union
    std::unique_ptr<sc_graph> U(new sc_graph());
    U->device = dev;
    U->stream = s;
    U->n = N;
    U->nnz = NNZ;
    U->num_sms = graphs[0]->num_sms;
    U->l2_bytes = graphs[0]->l2_bytes;
    U->row_ptr.reserve(N + 1);
    U->col_idx.reserve(NNZ);
    U->rev.reserve(NNZ);
    U->inv_deg_f.reserve(N);
    U->inv_deg_d.reserve(N);
    U->level.reserve(N);
    U->h_row_ptr.resize(N + 1);
    U->min_degree = INT32_MAX;
    for (int32_t i = 0; i < count; ++i) {
        const sc_graph *g = graphs[i];
        const int32_t a = static_cast<int32_t>(n_off[i]), ka = static_cast<int32_t>(k_off[i]);
        k_offset_copy<<<ceil_div(g->n, 256), 256, 0, s>>>(U->row_ptr.get() + a, g->row_ptr.get(), g->n, ka);
        k_offset_copy<<<ceil_div(g->nnz, 256), 256, 0, s>>>(U->col_idx.get() + ka, g->col_idx.get(), g->nnz, a);
        k_offset_copy<<<ceil_div(g->nnz, 256), 256, 0, s>>>(U->rev.get() + ka, g->rev.get(), g->nnz, ka);
        SC_LAUNCH_CHECK();
        SC_CUDA(cudaMemcpyAsync(U->level.get() + a, g->level.get(), g->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        SC_CUDA(cudaMemcpyAsync(U->inv_deg_f.get() + a, g->inv_deg_f.get(), g->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        SC_CUDA(cudaMemcpyAsync(U->inv_deg_d.get() + a, g->inv_deg_d.get(), g->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int32_t r = 0; r < g->n; ++r) U->h_row_ptr[a + r] = g->h_row_ptr[r] + ka;
        U->min_degree = std::min(U->min_degree, g->min_degree);
        U->max_degree = std::max(U->max_degree, g->max_degree);
    }
    U->h_row_ptr[N] = static_cast<int32_t>(NNZ);
    SC_CUDA(cudaMemcpyAsync(U->row_ptr.get() + N, &U->h_row_ptr[N], sizeof(int32_t), cudaMemcpyHostToDevice, s));
    U->tau_entry.reserve(NNZ);
    std::vector<int32_t> len(N);
    if (learned) {
        // per source the model's length (at most the graph's cap), per edge the shorter of its two
        for (int32_t i = 0; i < count; ++i) {
            sc_graph *g = graphs[i];
            DevBuf<int32_t> Ls;
            Ls.reserve(g->n);
            learned_lengths(g, ell[i], Ls.get(), s);
            k_tau_min_of_sources<<<ceil_div(g->n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), Ls.get(), g->n,
                                                                     U->tau_entry.get() + k_off[i]);
            SC_LAUNCH_CHECK();
        }
        DevBuf<int32_t> ts;
        ts.reserve(N);
        k_row_max<<<ceil_div(N, 256), 256, 0, s>>>(U->row_ptr.get(), U->tau_entry.get(), N, ts.get());
        SC_LAUNCH_CHECK();
        SC_CUDA(cudaMemcpyAsync(len.data(), ts.get(), N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
    } else {
        for (int32_t i = 0; i < count; ++i) {
            fill_i32(U->tau_entry.get() + k_off[i], graphs[i]->nnz, ell[i], s);
            std::fill(len.begin() + n_off[i], len.begin() + n_off[i + 1], ell[i]);
        }
    }
    const int heavy_t = o.heavy_threshold > 0 ? o.heavy_threshold : 256;
    ensure_row_order(U.get(), heavy_t);
    int32_t beta = 0;
    for (int32_t i = 0; i < count; ++i) beta = std::max(beta, ensure_bandwidth(graphs[i]));

    // ---- block width and lane split, tuned on the largest graph of the batch
    sc_graph *gb = graphs[big];
    gb->tau_entry.reserve(gb->nnz);
    fill_i32(gb->tau_entry.get(), gb->nnz, ell[big], gb->stream);
    gb->acc_g.reserve(gb->nnz);
    gb->acc_t1.reserve(gb->nnz);
    gb->acc_t2.reserve(gb->nnz);
    gb->status.reserve(4);
    SC_CUDA(cudaMemsetAsync(gb->status.get(), 0, 4 * sizeof(int32_t), gb->stream));
    ensure_row_order(gb, heavy_t);
    const int fixV = o.rows_split == 0 ? -1 : o.rows_split;
    const int32_t h0 = bf16_first_hop(o);
    const int tune_prec = (o.precision == SC_PREC_BF16 && h0 > 1) ? SC_PREC_FP32 : o.precision;
    const TuneResult tr = autotune(gb, tune_prec, o.block_width, fixV, o.max_slices, ell[big] + extra,
                                   GatherRec{0, nullptr, 0}, false, gb->stream);
    SC_CUDA(cudaStreamSynchronize(gb->stream));

    Run R;
    R.g = U.get();
    R.o = &o;
    R.s = s;
    R.prec = o.precision;
    R.B = tr.B;
    R.vpl = tr.vpl;
    int32_t nmax = 0;
    for (int32_t i = 0; i < count; ++i) nmax = std::max(nmax, graphs[i]->n);
    R.h0 = h0;
    R.slice_bytes = static_cast<size_t>(nmax) * R.B * alloc_elem(R.prec, R.h0);
    R.slices = 0;
    R.plus = false;
    R.time_kernels = false;
    R.extra = extra;
    // the learned policy's records: hops tau-1, tau (mode 1; mode 3 adds tau+1, tau+2 in t1 / t2
    // for the end-corrected estimator and the tail estimate)
    const int rec_mode = learned ? (record_after ? 3 : 1) : 0;
    DevBuf<double> pre;
    if (rec_mode == 3) pre.reserve(static_cast<size_t>(NNZ) * 2);
    R.rec = GatherRec{rec_mode, rec_mode == 3 ? pre.get() : nullptr, rec_mode == 3 ? 2 : 0};
    R.capture = true;
    U->acc_g.reserve(NNZ);
    U->acc_t1.reserve(NNZ);
    U->acc_t2.reserve(NNZ);
    U->status.reserve(4);
    SC_CUDA(cudaMemsetAsync(U->status.get(), 0, 4 * sizeof(int32_t), s));
    k_reset_rows<<<ceil_div(N, 8), 256, 0, s>>>(U->row_ptr.get(), nullptr, N, U->tau_entry.get(), rec_mode,
                                                U->acc_g.get(), U->acc_t1.get(), U->acc_t2.get(), R.rec.all,
                                                R.rec.stride);
    SC_LAUNCH_CHECK();
    std::vector<int32_t> all(N);
    std::iota(all.begin(), all.end(), 0);
    std::vector<int32_t> seg_start(count + 1);
    for (int32_t i = 0; i < count; ++i) seg_start[i] = static_cast<int32_t>(n_off[i]);
    seg_start[count] = N;
    // per graph: source-hops, shortest and longest source run
    std::vector<int64_t> g_hops(count, 0);
    std::vector<int32_t> g_lmin(count, INT32_MAX), g_lmax(count, 0);
    auto book = [&](const std::vector<int32_t> &src) {
        int32_t i = 0;
        for (int32_t v : src) {  // src is in id order: graphs in turn
            while (v >= n_off[i + 1]) ++i;
            const int32_t l = len[v] + extra;
            g_hops[i] += l;
            g_lmin[i] = std::min(g_lmin[i], l);
            g_lmax[i] = std::max(g_lmax[i], l);
        }
    };
    SC_CUDA(cudaEventRecord(ev1, s));
    std::vector<char> seg_bip(count);
    for (int32_t i = 0; i < count; ++i) seg_bip[i] = graphs[i]->bipartite ? 1 : 0;
    run_blocks_win(R, all, len, seg_start, beta, seg_bip);
    book(all);

    // ---- combine (and for the learned lengths the check / extension loop), Foster sums, outputs
    DevBuf<double> d_s, seg_sum;
    DevBuf<int64_t> d_off;
    d_s.reserve(NNZ);
    seg_sum.reserve(count);
    d_off.reserve(count + 1);
    auto combine = [&] {
        k_combine<<<ceil_div(N, 8), 256, 0, s>>>(U->row_ptr.get(), U->col_idx.get(), U->rev.get(),
                                                 U->inv_deg_d.get(), U->acc_g.get(), U->acc_t1.get(),
                                                 U->acc_t2.get(), N, o.estimator == SC_EST_END_CORRECTED,
                                                 record_after ? 1 : 0, 0.0, d_s.get(), nullptr);
        SC_LAUNCH_CHECK();
        R.launches += 1;
    };
    combine();
    int32_t rounds = 0;
    int64_t extended = 0;
    if (learned) {
        // per row: the bound factor of its graph (-1: bipartite, the tail estimate) and its cap
        std::vector<double> h_fac(N);
        std::vector<int32_t> h_cap(N);
        for (int32_t i = 0; i < count; ++i) {
            const double f = graphs[i]->bipartite ? -1.0 : lam[i] * lam[i] / (1.0 - lam[i] * lam[i]);
            std::fill(h_fac.begin() + n_off[i], h_fac.begin() + n_off[i + 1], f);
            std::fill(h_cap.begin() + n_off[i], h_cap.begin() + n_off[i + 1], ell[i]);
        }
        DevBuf<double> fac, d_b;
        DevBuf<int32_t> cap_row, row_flag, rows, ts;
        fac.reserve(N);
        cap_row.reserve(N);
        row_flag.reserve(N);
        ts.reserve(N);
        d_b.reserve(NNZ);
        U->tp_counters.reserve(4);
        SC_CUDA(cudaMemcpyAsync(fac.get(), h_fac.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
        SC_CUDA(cudaMemcpyAsync(cap_row.get(), h_cap.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        std::vector<int32_t> h_flag(N);
        while (true) {
            k_learned_check<<<ceil_div(N, 8), 256, 0, s>>>(U->row_ptr.get(), U->col_idx.get(), U->rev.get(),
                                                           U->inv_deg_d.get(), pre.get(), U->acc_t1.get(),
                                                           U->acc_t2.get(), rec_mode, fac.get(), 0.0,
                                                           U->tau_entry.get(), N, d_b.get());
            SC_CUDA(cudaMemsetAsync(U->tp_counters.get(), 0, sizeof(long long), s));
            k_extend_failing<<<ceil_div(N, 8), 256, 0, s>>>(U->row_ptr.get(), U->col_idx.get(), d_b.get(), N, o.eps, 0,
                                                            nullptr, U->tau_entry.get(), row_flag.get(),
                                                            reinterpret_cast<unsigned long long *>(
                                                                U->tp_counters.get()),
                                                            cap_row.get());
            SC_LAUNCH_CHECK();
            R.launches += 2;
            long long failing = 0;
            SC_CUDA(cudaMemcpyAsync(&failing, U->tp_counters.get(), sizeof(long long), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaStreamSynchronize(s));
            if (failing == 0) break;
            extended += failing / 2;
            ++rounds;
            SC_CUDA(cudaMemcpyAsync(h_flag.data(), row_flag.get(), N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            k_row_max<<<ceil_div(N, 256), 256, 0, s>>>(U->row_ptr.get(), U->tau_entry.get(), N, ts.get());
            SC_LAUNCH_CHECK();
            SC_CUDA(cudaMemcpyAsync(len.data(), ts.get(), N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SC_CUDA(cudaStreamSynchronize(s));
            std::vector<int32_t> redo;
            for (int32_t v = 0; v < N; ++v)
                if (h_flag[v]) redo.push_back(v);
            rows.reserve(redo.size());
            SC_CUDA(cudaMemcpyAsync(rows.get(), redo.data(), redo.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            k_reset_rows<<<ceil_div(static_cast<int64_t>(redo.size()), 8), 256, 0, s>>>(
                U->row_ptr.get(), rows.get(), static_cast<int32_t>(redo.size()), U->tau_entry.get(), rec_mode,
                U->acc_g.get(), U->acc_t1.get(), U->acc_t2.get(), R.rec.all, R.rec.stride);
            SC_LAUNCH_CHECK();
            R.launches += 2;
            run_blocks_win(R, redo, len, seg_start, beta, seg_bip);
            book(redo);
            combine();
        }
    }
    SC_CUDA(cudaMemcpyAsync(d_off.get(), k_off.data(), (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_segment_sum<<<count, 256, 0, s>>>(d_s.get(), d_off.get(), seg_sum.get());
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaEventRecord(ev2, s));
    std::vector<double> foster(count);
    SC_CUDA(cudaMemcpyAsync(foster.data(), seg_sum.get(), count * sizeof(double), cudaMemcpyDeviceToHost, s));
    for (int32_t i = 0; i < count; ++i)
        SC_CUDA(cudaMemcpyAsync(s_hat[i], d_s.get() + k_off[i], graphs[i]->nnz * sizeof(double),
                                out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    int32_t h_status = 0;
    SC_CUDA(cudaMemcpy(&h_status, U->status.get(), sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (h_status & 1) SC_FAIL(SC_ERR_TIMEOUT, "a bounded wait expired");
    float prop_ms = 0.f, total_ms = 0.f;
    SC_CUDA(cudaEventElapsedTime(&prop_ms, ev1, ev2));
    SC_CUDA(cudaEventElapsedTime(&total_ms, ev0, ev2));
    if (reports) {
        for (int32_t i = 0; i < count; ++i) {
            sc_report *rep = reports + i;
            std::memset(rep, 0, sizeof(*rep));
            rep->ell_global = ell[i];  // the length (the learned policy: the cap)
            rep->ell_min_source = g_lmin[i] == INT32_MAX ? 0 : g_lmin[i];
            rep->ell_max_source = g_lmax[i];
            rep->block_width = R.B;
            rep->rows_split = R.vpl;
            rep->slices = 0;
            rep->blocks = (graphs[i]->n + R.B - 1) / R.B;
            rep->source_hops = g_hops[i];
            rep->foster_sum = 0.5 * foster[i];
            rep->lambda_star = lam[i];
            rep->windowed = 1;
            rep->uncertified = learned && graphs[i]->bipartite ? 1 : 0;
            // batch totals
            rep->extension_rounds = rounds;
            rep->edges_extended = static_cast<int32_t>(std::min<int64_t>(extended, INT32_MAX));
            // batch totals
            rep->launches = R.launches + 4 + 3 * count;
            rep->hops = R.hops;
            rep->hop_launches = R.hop_launches;
            rep->algorithmic_bytes = R.alg_bytes;
            rep->hop_bytes = R.alg_bytes;
            rep->propagate_ms = prop_ms;
            rep->total_ms = total_ms;
        }
    }
}

}  // namespace sc

extern "C" sc_status sc_all_edges(sc_graph *g, const sc_options *opts, double *s_hat, double *tail_bound,
                                  sc_report *report) {
    return sc::guarded([&] { sc::all_edges_impl(g, opts, s_hat, tail_bound, report); });
}

extern "C" sc_status sc_some_edges(sc_graph *g, const sc_options *opts, int64_t count, const int64_t *entries,
                                   double *s_out, sc_report *report) {
    return sc::guarded([&] {
        const sc::EdgeSubset sub{count, entries, s_out};
        sc::all_edges_impl(g, opts, nullptr, nullptr, report, nullptr, 0, &sub);
    });
}

extern "C" sc_status sc_batch_all_edges(sc_graph *const *graphs, int32_t count, const sc_options *opts,
                                        const int32_t *ell_per_graph, double *const *s_hat, sc_report *reports) {
    return sc::guarded([&] { sc::batch_impl(graphs, count, opts, ell_per_graph, s_hat, reports); });
}

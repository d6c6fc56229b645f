// sc_all_edges_noalloc: the all-edges traversal for callers that cannot
// allocate device memory. The paper has no counterpart; this is plumbing
// around the same kernels as sc_all_edges.
//
// Who needs it: code that runs under a memory manager owning the whole device
// budget (an inference server's arena, a framework's caching allocator that
// has reserved the rest of memory), latency-critical paths where cudaMalloc /
// cudaFree would block or synchronise the device, and embedders that must not
// fail with out-of-memory in the middle of a run. Such callers pass only their
// CSR and output buffers; every work buffer lives in one file-scope device
// array of fixed size, so no call allocates.
//
// The array is SC_NOALLOC_SCRATCH_BYTES (64 MiB). Every GPU that loads this
// library's module holds it until the process exits. All calls share it and
// it keeps the previous call's contents, so everything that must start at
// zero is cleared by the call itself; calls that overlap on the GPU (two
// streams, two host threads, or one call still running when another is
// issued) race on it and must be serialised by the caller.
//
// Host code cannot use the array's name as a device address (it is a host
// stand-in), so the first call in each CUDA context looks the address up with
// cudaGetSymbolAddress while that context's device is current and caches it
// under the context's unique id; that first call should be made before any
// stream capture begins. A device reset creates a new context (a new id), so
// the address is looked up again instead of reusing a stale one.
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include <cuda.h>

#include "propagate.cuh"

namespace sc {

static_assert(SC_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");
static __device__ __align__(256) unsigned char g_noalloc_scratch[SC_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static std::unordered_map<unsigned long long, unsigned char *> g_noalloc_addr;

// unique id of the current context (cuCtxGetCurrent + cuCtxGetId, reached
// through the runtime's driver entry points) on `device`
static unsigned long long current_context_id(int device) {
    using CtxGetCurrent = CUresult (*)(CUcontext *);
    using CtxGetId = CUresult (*)(CUcontext, unsigned long long *);
    static CtxGetCurrent get_current = nullptr;
    static CtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        SC_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa));
        SC_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb));
        if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            SC_FAIL(SC_ERR_CUDA, "cuCtxGetCurrent / cuCtxGetId unavailable");
        get_current = reinterpret_cast<CtxGetCurrent>(a);
        get_id = reinterpret_cast<CtxGetId>(b);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) SC_FAIL(SC_ERR_CUDA, "cuCtxGetCurrent failed");
    if (!ctx) {  // no context bound to this thread yet: the runtime's primary context of the device
        SC_CUDA(cudaSetDevice(device));
        if (get_current(&ctx) != CUDA_SUCCESS || !ctx) SC_FAIL(SC_ERR_CUDA, "no CUDA context on device %d", device);
    }
    unsigned long long id = 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) SC_FAIL(SC_ERR_CUDA, "cuCtxGetId failed");
    return id;
}

static unsigned char *noalloc_scratch_address(int device) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long ctx = current_context_id(device);
    auto it = g_noalloc_addr.find(ctx);
    if (it != g_noalloc_addr.end()) return it->second;
    void *ptr = nullptr;
    SC_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    if (!ptr) SC_FAIL(SC_ERR_CUDA, "cudaGetSymbolAddress returned a null scratch address");
    g_noalloc_addr[ctx] = static_cast<unsigned char *>(ptr);
    return static_cast<unsigned char *>(ptr);
}

enum : int32_t { NA_BAD_CSR = 1, NA_SELF_LOOP = 2, NA_DUPLICATE = 4, NA_ISOLATED = 8, NA_NOT_SYMMETRIC = 16 };

// the same structural checks as graph creation; every read is bounds-guarded
__global__ void k_na_validate(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                              int64_t nnz, int32_t *status) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t b = row_ptr[r], e = row_ptr[r + 1];
    int32_t bits = 0;
    if ((r == 0 && b != 0) || (r == n - 1 && e != nnz) || b < 0 || e < b || e > nnz) {
        bits |= NA_BAD_CSR;
    } else {
        if (e == b) bits |= NA_ISOLATED;
        int32_t prev = -1;
        for (int64_t k = b; k < e; ++k) {
            const int32_t c = col[k];
            if (c < 0 || c >= n) {
                bits |= NA_BAD_CSR;
                break;
            }
            if (c == r) bits |= NA_SELF_LOOP;
            if (k > b && c == prev) bits |= NA_DUPLICATE;
            if (k > b && c < prev) bits |= NA_BAD_CSR;
            prev = c;
        }
    }
    if (bits) atomicOr(status, bits);
}

// reverse-entry map and 1/d (run only on a validated CSR)
__global__ void k_na_prepare(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                             double *__restrict__ inv_deg, int32_t *__restrict__ rev, int32_t *status) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    inv_deg[r] = 1.0 / static_cast<double>(row_ptr[r + 1] - row_ptr[r]);
    for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
        const int32_t c = col[k];
        int32_t lo = row_ptr[c], hi = row_ptr[c + 1];
        while (lo < hi) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if (col[mid] < r) lo = mid + 1;
            else hi = mid;
        }
        if (lo < row_ptr[c + 1] && col[lo] == r) {
            rev[k] = lo;
        } else {
            rev[k] = 0;
            atomicOr(status, NA_NOT_SYMMETRIC);
        }
    }
}

// hop-0 term of every half sum (1, unscaled) and one length for every entry
__global__ void k_na_init(double *__restrict__ g, int32_t *__restrict__ tau, int64_t nnz, int32_t ell) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    g[k] = 1.0;
    tau[k] = ell;
}

__global__ void k_na_sources(int32_t *__restrict__ src, int64_t count, int32_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) src[i] = i < n ? static_cast<int32_t>(i) : -1;
}

// s_hat(e_ij) = g(v_i,v_j) + g(v_j,v_i), the plain estimator of sc_all_edges
__global__ void k_na_combine(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                             const int32_t *__restrict__ rev, const double *__restrict__ inv_d,
                             const double *__restrict__ g, int32_t n, double *__restrict__ s_out) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const double ir = inv_d[r];
    for (int32_t k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) {
        const int32_t j = col[k], kr = rev[k];
        s_out[k] = __dadd_rn(__dmul_rn(g[k], ir), __dmul_rn(g[kr], inv_d[j]));
    }
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// bytes of scratch one call needs (FP64 blocks of 32 sources)
static size_t noalloc_bytes(int64_t n, int64_t nnz) {
    constexpr int64_t B = 32;
    const int64_t nsrc = (n + B - 1) / B * B;
    return align256(2 * sizeof(int32_t)) + align256(8 * n) + align256(4 * nnz) + align256(8 * nnz) +
           align256(4 * nnz) + align256(4 * nsrc) + 2 * align256(8 * B * n);
}

static void noalloc_impl(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx, int32_t ell,
                         double *s_hat, void *stream_ptr) {
    if (n < 2 || nnz < 2 || nnz >= (int64_t(1) << 31) || ell < 0 || !row_ptr || !col_idx || !s_hat)
        SC_FAIL(SC_ERR_INVALID_ARG, "need n >= 2, 2 <= nnz < 2^31, ell >= 0 and non-null device pointers");
    const size_t need = noalloc_bytes(n, nnz);
    if (need > SC_NOALLOC_SCRATCH_BYTES)
        SC_FAIL(SC_ERR_INVALID_ARG,
                "graph needs %zu bytes of scratch (about 524 n + 16 nnz), above the %zu-byte limit "
                "(n=%d nnz=%lld): use sc_all_edges",
                need, static_cast<size_t>(SC_NOALLOC_SCRATCH_BYTES), n, static_cast<long long>(nnz));
    int device = 0;
    SC_CUDA(cudaGetDevice(&device));
    unsigned char *base = noalloc_scratch_address(device);
    cudaStream_t s = static_cast<cudaStream_t>(stream_ptr);
    constexpr int B = 32;
    const int64_t nsrc = (static_cast<int64_t>(n) + B - 1) / B * B;

    unsigned char *p = base;
    auto carve = [&](size_t bytes) {
        unsigned char *q = p;
        p += align256(bytes);
        return q;
    };
    int32_t *status = reinterpret_cast<int32_t *>(carve(2 * sizeof(int32_t)));
    double *inv_deg = reinterpret_cast<double *>(carve(8 * static_cast<size_t>(n)));
    int32_t *rev = reinterpret_cast<int32_t *>(carve(4 * static_cast<size_t>(nnz)));
    double *acc = reinterpret_cast<double *>(carve(8 * static_cast<size_t>(nnz)));
    int32_t *tau = reinterpret_cast<int32_t *>(carve(4 * static_cast<size_t>(nnz)));
    int32_t *src = reinterpret_cast<int32_t *>(carve(4 * static_cast<size_t>(nsrc)));
    double *xa = reinterpret_cast<double *>(carve(8 * static_cast<size_t>(B) * n));
    double *xb = reinterpret_cast<double *>(carve(8 * static_cast<size_t>(B) * n));

    const int tb = 256;
    int32_t h_status = 0;
    SC_CUDA(cudaMemsetAsync(status, 0, 2 * sizeof(int32_t), s));
    k_na_validate<<<ceil_div(n, tb), tb, 0, s>>>(row_ptr, col_idx, n, nnz, status);
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    if (h_status & NA_BAD_CSR) SC_FAIL(SC_ERR_BAD_CSR, "malformed CSR");
    if (h_status & NA_SELF_LOOP) SC_FAIL(SC_ERR_SELF_LOOP, "self-loop");
    if (h_status & NA_DUPLICATE) SC_FAIL(SC_ERR_DUPLICATE_EDGE, "duplicate entry");
    if (h_status & NA_ISOLATED) SC_FAIL(SC_ERR_ISOLATED_NODE, "node of degree 0");
    k_na_prepare<<<ceil_div(n, tb), tb, 0, s>>>(row_ptr, col_idx, n, inv_deg, rev, status);
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    if (h_status & NA_NOT_SYMMETRIC) SC_FAIL(SC_ERR_NOT_SYMMETRIC, "an entry has no reverse");

    k_na_init<<<ceil_div(nnz, tb), tb, 0, s>>>(acc, tau, nnz, ell);
    k_na_sources<<<ceil_div(nsrc, tb), tb, 0, s>>>(src, nsrc, n);
    SC_LAUNCH_CHECK();
    int dev = 0, num_sms = 0;
    SC_CUDA(cudaGetDevice(&dev));
    SC_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    for (int64_t first = 0; first < n && ell > 0; first += B) {
        const int nb = static_cast<int>(std::min<int64_t>(B, n - first));
        const int32_t *bsrc = src + first;
        double *a = xa, *b = xb;
        SC_CUDA(cudaMemsetAsync(a, 0, 8 * static_cast<size_t>(B) * n, s));
        k_first_hop<double, B><<<nb, 128, 0, s>>>(row_ptr, col_idx, inv_deg, bsrc, nb, a, n, nullptr);
        for (int hop = 2; hop < ell; ++hop) {
            // natural row order, every row on the light path (no schedule array
            // without allocation); the first CTAs gather X_{hop-1}. hop - 1 <= ell
            // = tau[k] always, so the hop tau+1 / tau+2 records are never written.
            HopArgs<double> ha{};
            ha.row_ptr = row_ptr;
            ha.col = col_idx;
            ha.inv_deg = inv_deg;
            ha.x_prev = a;
            ha.x_next = b;
            ha.n = n;
            ha.row_order = nullptr;
            ha.n_heavy = 0;
            ha.src = bsrc;
            ha.nsrc = nb;
            ha.tau = tau;
            ha.gather_ell = hop - 1;
            ha.g = acc;
            ha.t1 = nullptr;
            ha.t2 = nullptr;
            ha.rec = GatherRec{0, nullptr, 0};
            launch_spmm_hop<double, B, 1>(ha, 1, s, num_sms);
            std::swap(a, b);
        }
        if (ell >= 2)  // the last hop only where the gather reads it, with the gathers of hops ell-1, ell
            k_last_hop<double, B><<<nb, kSpmmWarps * 32, 0, s>>>(row_ptr, col_idx, inv_deg, a, n, bsrc, nb, tau,
                                                                  ell, acc, nullptr, nullptr, GatherRec{0, nullptr, 0});
        else
            k_gather<double, B><<<nb, 128, 0, s>>>(row_ptr, col_idx, a, n, bsrc, nb, tau, ell, acc, nullptr, nullptr,
                                                   GatherRec{0, nullptr, 0}, nullptr);
        SC_LAUNCH_CHECK();
    }
    k_na_combine<<<ceil_div(n, 8), 256, 0, s>>>(row_ptr, col_idx, rev, inv_deg, acc, n, s_hat);
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace sc

extern "C" sc_status sc_all_edges_noalloc(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                                          int32_t ell, double *s_hat, void *stream) {
    return sc::guarded([&] { sc::noalloc_impl(n, nnz, row_ptr, col_idx, ell, s_hat, stream); });
}

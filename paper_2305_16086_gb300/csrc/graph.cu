// Graph ingest (step A1): CSR validation, reverse-entry map, 1/d(v),
// connectivity and the bipartite test; status strings and option defaults.
//
// Cites: Definition 2.2 (input: an undirected connected graph) and the
// notation of Section 2.1 (N(v), d(v), P = D^-1 A). Section 2.1 also assumes
// G is not bipartite; bipartiteness is detected here so that callers can
// pick the end-corrected estimator instead.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "common.cuh"

namespace sc {

static thread_local std::string t_detail;

void set_detail(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_detail = buf;
}
void clear_detail() { t_detail.clear(); }

// error bits written by the validation kernels
enum : int32_t {
    V_BAD_CSR = 1,
    V_SELF_LOOP = 2,
    V_DUPLICATE = 4,
    V_ISOLATED = 8,
    V_NOT_SYMMETRIC = 16,
    V_NOT_BIPARTITE = 32,
};

// status[0]: OR of error bits; status[1]: smallest offending row
__global__ void k_validate_rows(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                int32_t n, int64_t nnz, int32_t *status) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t b = row_ptr[r], e = row_ptr[r + 1];
    int32_t bits = 0;
    if ((r == 0 && b != 0) || (r == n - 1 && e != nnz) || b < 0 || e < b || e > nnz) {
        bits |= V_BAD_CSR;
    } else {
        if (e == b) bits |= V_ISOLATED;
        int32_t prev = -1;
        for (int64_t k = b; k < e; ++k) {
            int32_t c = col[k];
            if (c < 0 || c >= n) {
                bits |= V_BAD_CSR;
                break;
            }
            if (c == r) bits |= V_SELF_LOOP;
            if (k > b) {
                if (c == prev) bits |= V_DUPLICATE;
                else if (c < prev) bits |= V_BAD_CSR;
            }
            prev = c;
        }
    }
    if (bits) {
        atomicOr(&status[0], bits);
        atomicMin(&status[1], r);
    }
}

// rev[k] = position of (c -> r) in row c, for entry k = (r -> c)
__global__ void k_build_rev(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                            int32_t n, int32_t *__restrict__ rev, int32_t *status) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
        int32_t c = col[k];
        int32_t lo = row_ptr[c], hi = row_ptr[c + 1];  // search r in [lo, hi)
        while (lo < hi) {
            int32_t mid = lo + ((hi - lo) >> 1);
            if (col[mid] < r) lo = mid + 1;
            else hi = mid;
        }
        if (lo < row_ptr[c + 1] && col[lo] == r) {
            rev[k] = lo;
        } else {
            rev[k] = -1;
            atomicOr(&status[0], V_NOT_SYMMETRIC);
            atomicMin(&status[1], r);
        }
    }
}

__global__ void k_inv_deg(const int32_t *__restrict__ row_ptr, int32_t n, float *inv_f, double *inv_d) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double d = static_cast<double>(row_ptr[r + 1] - row_ptr[r]);
    inv_d[r] = 1.0 / d;
    inv_f[r] = static_cast<float>(1.0 / d);
}

__global__ void k_fill_i32(int32_t *p, int64_t count, int32_t v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) p[i] = v;
}

// one BFS level: expand the frontier, claiming unvisited neighbours
__global__ void k_bfs_expand(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                             const int32_t *__restrict__ frontier, int32_t fsize,
                             int32_t *__restrict__ level, int32_t next_level,
                             int32_t *__restrict__ next, int32_t *next_count) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= fsize) return;
    int32_t v = frontier[t];
    for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
        int32_t y = col[k];
        if (level[y] == -1 && atomicCAS(&level[y], -1, next_level) == -1) {
            int32_t slot = atomicAdd(next_count, 1);
            next[slot] = y;
        }
    }
}

// an edge inside one BFS level closes an odd cycle
__global__ void k_bipartite_check(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                  const int32_t *__restrict__ level, int32_t n, int32_t *status) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int32_t lr = level[r];
    for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
        if (level[col[k]] == lr) {
            atomicOr(&status[0], V_NOT_BIPARTITE);
            return;
        }
    }
}

void fill_i32(int32_t *p, int64_t count, int32_t v, cudaStream_t s) {
    if (count <= 0) return;
    k_fill_i32<<<static_cast<unsigned>((count + 255) / 256), 256, 0, s>>>(p, count, v);
    SC_LAUNCH_CHECK();
}

void ensure_row_order(sc_graph *g, int32_t heavy_threshold) {
    if (g->heavy_threshold_cached == heavy_threshold) return;
    auto deg = [&](int32_t r) { return g->h_row_ptr[r + 1] - g->h_row_ptr[r]; };
    std::vector<int32_t> heavy, order;
    order.reserve(g->n);
    for (int32_t r = 0; r < g->n; ++r)
        if (deg(r) > heavy_threshold) heavy.push_back(r);
    // heavy rows longest first (their CTAs are scheduled first), then the light
    // rows in natural order (neighbouring rows share cache lines of X on
    // locally numbered graphs)
    std::stable_sort(heavy.begin(), heavy.end(), [&](int32_t a, int32_t b) { return deg(a) > deg(b); });
    order = heavy;
    for (int32_t r = 0; r < g->n; ++r)
        if (deg(r) <= heavy_threshold) order.push_back(r);
    g->row_order.reserve(g->n);
    SC_CUDA(cudaMemcpyAsync(g->row_order.get(), order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            g->stream));
    SC_CUDA(cudaStreamSynchronize(g->stream));
    g->n_heavy = static_cast<int32_t>(heavy.size());
    g->h_heavy_ids = heavy;
    std::sort(g->h_heavy_ids.begin(), g->h_heavy_ids.end());
    g->heavy_ids.reserve(std::max<size_t>(heavy.size(), 1));
    if (!heavy.empty())
        SC_CUDA(cudaMemcpyAsync(g->heavy_ids.get(), g->h_heavy_ids.data(), heavy.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, g->stream));
    SC_CUDA(cudaStreamSynchronize(g->stream));
    g->heavy_threshold_cached = heavy_threshold;
}

// largest |i - j| over the rows' entries: threads stride over the entries of
// their rows (grid-stride), one atomic per CTA
__global__ void k_bandwidth(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                            int32_t *out) {
    __shared__ int32_t cta_m;
    if (threadIdx.x == 0) cta_m = 0;
    __syncthreads();
    int32_t m = 0;
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int32_t a = row_ptr[r], b = row_ptr[r + 1];
        if (b > a) m = max(m, max(abs(col[a] - r), abs(col[b - 1] - r)));  // rows are sorted
    }
    atomicMax(&cta_m, m);
    __syncthreads();
    if (threadIdx.x == 0 && cta_m > 0) atomicMax(out, cta_m);
}

int32_t ensure_bandwidth(sc_graph *g) {
    if (g->bandwidth >= 0) return g->bandwidth;
    DevBuf<int32_t> d;
    d.reserve(1);
    SC_CUDA(cudaMemsetAsync(d.get(), 0, sizeof(int32_t), g->stream));
    const int grid = std::max(1, std::min(ceil_div(g->n, 256), (g->num_sms > 0 ? g->num_sms : 148) * 4));
    k_bandwidth<<<grid, 256, 0, g->stream>>>(g->row_ptr.get(), g->col_idx.get(), g->n, d.get());
    SC_LAUNCH_CHECK();
    int32_t h = 0;
    SC_CUDA(cudaMemcpyAsync(&h, d.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
    SC_CUDA(cudaStreamSynchronize(g->stream));
    g->bandwidth = h;
    return h;
}

void ensure_partition(sc_graph *g, int32_t target) {
    if (g->part_target == target) return;
    // consecutive rows per warp until about `target` CSR entries (a row longer
    // than the target forms a run of its own)
    std::vector<int32_t> part;
    part.push_back(0);
    int64_t acc = 0;
    for (int32_t r = 0; r < g->n; ++r) {
        const int32_t d = g->h_row_ptr[r + 1] - g->h_row_ptr[r];
        if (acc > 0 && acc + d > target) {
            part.push_back(r);
            acc = 0;
        }
        acc += d;
    }
    part.push_back(g->n);
    g->part.reserve(part.size());
    SC_CUDA(cudaMemcpyAsync(g->part.get(), part.data(), part.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            g->stream));
    SC_CUDA(cudaStreamSynchronize(g->stream));
    g->nparts = static_cast<int32_t>(part.size()) - 1;
    g->part_target = target;
}

static void create_impl(sc_graph **out, int32_t n, int64_t nnz, const int32_t *row_ptr,
                        const int32_t *col_idx, uint32_t flags, void *stream) {
    if (!out) SC_FAIL(SC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 2 || nnz < 2 || nnz >= (int64_t(1) << 31) || !row_ptr || !col_idx)
        SC_FAIL(SC_ERR_INVALID_ARG, "need n >= 2, 2 <= nnz < 2^31 and non-null arrays (n=%d nnz=%lld)", n,
                (long long)nnz);
    if (flags & ~(SC_PTRS_DEVICE | SC_FLAG_REJECT_BIPARTITE))
        SC_FAIL(SC_ERR_INVALID_ARG, "unknown flags 0x%x", flags);

    auto *g = new sc_graph();
    struct Guard {
        sc_graph *g;
        bool keep = false;
        ~Guard() {
            if (!keep) delete g;
        }
    } guard{g};

    SC_CUDA(cudaGetDevice(&g->device));
    g->stream = static_cast<cudaStream_t>(stream);
    g->n = n;
    g->nnz = nnz;
    int l2 = 0;
    SC_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    SC_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device));
    g->l2_bytes = static_cast<size_t>(l2);

    g->row_ptr.reserve(n + 1);
    g->col_idx.reserve(nnz);
    g->rev.reserve(nnz);
    g->level.reserve(n);
    g->inv_deg_f.reserve(n);
    g->inv_deg_d.reserve(n);
    g->status.reserve(4);
    const cudaMemcpyKind kind = (flags & SC_PTRS_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t s = g->stream;
    SC_CUDA(cudaMemcpyAsync(g->row_ptr.get(), row_ptr, (n + 1) * sizeof(int32_t), kind, s));
    SC_CUDA(cudaMemcpyAsync(g->col_idx.get(), col_idx, nnz * sizeof(int32_t), kind, s));

    int32_t h_status[2] = {0, n};
    SC_CUDA(cudaMemcpyAsync(g->status.get(), h_status, sizeof(h_status), cudaMemcpyHostToDevice, s));
    const int tb = 256;
    k_validate_rows<<<ceil_div(n, tb), tb, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), n, nnz, g->status.get());
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaMemcpyAsync(h_status, g->status.get(), sizeof(h_status), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    if (h_status[0] & V_BAD_CSR) SC_FAIL(SC_ERR_BAD_CSR, "malformed CSR at row %d", h_status[1]);
    if (h_status[0] & V_SELF_LOOP) SC_FAIL(SC_ERR_SELF_LOOP, "self-loop in row %d", h_status[1]);
    if (h_status[0] & V_DUPLICATE) SC_FAIL(SC_ERR_DUPLICATE_EDGE, "duplicate entry in row %d", h_status[1]);
    if (h_status[0] & V_ISOLATED) SC_FAIL(SC_ERR_ISOLATED_NODE, "node %d has degree 0", h_status[1]);

    k_build_rev<<<ceil_div(n, tb), tb, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), n, g->rev.get(), g->status.get());
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaMemcpyAsync(h_status, g->status.get(), sizeof(h_status), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    if (h_status[0] & V_NOT_SYMMETRIC) SC_FAIL(SC_ERR_NOT_SYMMETRIC, "entry of row %d has no reverse", h_status[1]);

    k_inv_deg<<<ceil_div(n, tb), tb, 0, s>>>(g->row_ptr.get(), n, g->inv_deg_f.get(), g->inv_deg_d.get());
    SC_LAUNCH_CHECK();

    g->h_row_ptr.resize(n + 1);
    SC_CUDA(cudaMemcpyAsync(g->h_row_ptr.data(), g->row_ptr.get(), (n + 1) * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));

    // BFS from node 0: connectivity, depth and the level parity for the bipartite test
    DevBuf<int32_t> frontier, next, counter;
    frontier.reserve(n);
    next.reserve(n);
    counter.reserve(1);
    k_fill_i32<<<ceil_div(n, tb), tb, 0, s>>>(g->level.get(), n, -1);
    SC_LAUNCH_CHECK();
    const int32_t zero = 0;
    SC_CUDA(cudaMemcpyAsync(g->level.get(), &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(frontier.get(), &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    int32_t fsize = 1;
    int64_t visited = 1;
    int32_t depth = 0;
    while (fsize > 0) {
        SC_CUDA(cudaMemsetAsync(counter.get(), 0, sizeof(int32_t), s));
        k_bfs_expand<<<ceil_div(fsize, tb), tb, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), frontier.get(), fsize,
                                                         g->level.get(), depth + 1, next.get(), counter.get());
        SC_LAUNCH_CHECK();
        SC_CUDA(cudaMemcpyAsync(&fsize, counter.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
        if (fsize > 0) {
            ++depth;
            visited += fsize;
            std::swap(frontier.ptr, next.ptr);
        }
    }
    g->bfs_depth = depth;
    if (visited != n) SC_FAIL(SC_ERR_DISCONNECTED, "graph is disconnected: node 0 reaches %lld of %d nodes",
                              (long long)visited, n);

    SC_CUDA(cudaMemsetAsync(g->status.get(), 0, sizeof(int32_t), s));
    k_bipartite_check<<<ceil_div(n, tb), tb, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), g->level.get(), n,
                                                     g->status.get());
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaMemcpyAsync(h_status, g->status.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    g->bipartite = (h_status[0] & V_NOT_BIPARTITE) ? 0 : 1;
    if (g->bipartite && (flags & SC_FLAG_REJECT_BIPARTITE))
        SC_FAIL(SC_ERR_BIPARTITE, "graph is bipartite");

    int32_t dmin = INT32_MAX, dmax = 0;
    for (int32_t r = 0; r < n; ++r) {
        int32_t d = g->h_row_ptr[r + 1] - g->h_row_ptr[r];
        dmin = std::min(dmin, d);
        dmax = std::max(dmax, d);
    }
    g->min_degree = dmin;
    g->max_degree = dmax;
    guard.keep = true;
    *out = g;
}

}  // namespace sc

extern "C" {

sc_status sc_graph_create(sc_graph **out, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                          uint32_t flags, void *stream) {
    return sc::guarded([&] { sc::create_impl(out, n, nnz, row_ptr, col_idx, flags, stream); });
}

sc_status sc_graph_get_info(const sc_graph *g, sc_graph_info *out) {
    return sc::guarded([&] {
        if (!g || !out) SC_FAIL(SC_ERR_INVALID_ARG, "null argument");
        out->n = g->n;
        out->nnz = g->nnz;
        out->m = g->nnz / 2;
        out->min_degree = g->min_degree;
        out->max_degree = g->max_degree;
        out->bipartite = g->bipartite;
        out->diameter_lb = g->bfs_depth;
    });
}

void sc_graph_destroy(sc_graph *g) {
    if (!g) return;
    int cur = 0;
    const int dev = g->device;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    cudaStreamSynchronize(g->stream);
    delete g;
    if (cur != dev) cudaSetDevice(cur);
}

const char *sc_status_string(sc_status s) {
    switch (s) {
    case SC_OK: return "ok";
    case SC_ERR_INVALID_ARG: return "invalid argument";
    case SC_ERR_BAD_CSR: return "malformed CSR";
    case SC_ERR_NOT_SYMMETRIC: return "adjacency is not symmetric";
    case SC_ERR_SELF_LOOP: return "self-loop";
    case SC_ERR_DUPLICATE_EDGE: return "duplicate edge";
    case SC_ERR_ISOLATED_NODE: return "isolated node";
    case SC_ERR_DISCONNECTED: return "graph is disconnected";
    case SC_ERR_BIPARTITE: return "graph is bipartite";
    case SC_ERR_LAMBDA_NOT_CONVERGED: return "eigenvalue estimate did not converge";
    case SC_ERR_BOUND_UNMET: return "tail bound not met";
    case SC_ERR_TIMEOUT: return "device wait timed out";
    case SC_ERR_OOM: return "out of memory";
    case SC_ERR_CUDA: return "CUDA error";
    case SC_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *sc_last_error_detail(void) { return sc::t_detail.c_str(); }

int32_t sc_abi_version(void) { return SC_ABI_VERSION; }

void sc_options_default(sc_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->eps = 1e-3;
    o->mode = SC_MODE_TGT;
    o->precision = SC_PREC_FP32;
    o->ell_policy = SC_ELL_GLOBAL;
    o->ell_fixed = 0;
    o->estimator = SC_EST_PLAIN;
    o->block_width = 0;
    o->rows_split = 0;
    o->heavy_threshold = 0;
    o->max_slices = 0;
    o->flags = 0;
    o->seed = 0x5eed5eedULL;
    o->delta = 0.0;
    o->gamma = 10;
}

}  // extern "C"

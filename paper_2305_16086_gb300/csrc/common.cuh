// Internal helpers shared by the libsc translation units (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/sc.h"

namespace sc {

// ---------------------------------------------------------------------------
// Error reporting: every ABI call returns a status; the detail string is
// thread-local and describes the last failing call of the calling thread.
// ---------------------------------------------------------------------------
void set_detail(const char *fmt, ...);
void clear_detail();

struct Failure {
    sc_status status;
};

#define SC_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ::sc::set_detail("%s:%d %s: %s", __FILE__, __LINE__, #call,                   \
                             cudaGetErrorString(e_));                                     \
            throw ::sc::Failure{e_ == cudaErrorMemoryAllocation ? SC_ERR_OOM : SC_ERR_CUDA}; \
        }                                                                                 \
    } while (0)

#define SC_FAIL(status, ...)                     \
    do {                                         \
        ::sc::set_detail(__VA_ARGS__);           \
        throw ::sc::Failure{status};             \
    } while (0)

#define SC_LAUNCH_CHECK() SC_CUDA(cudaGetLastError())

// Wraps the body of an ABI function: converts Failure / std::bad_alloc into
// a status so no exception leaves the library.
template <typename F>
sc_status guarded(F &&body) {
    try {
        clear_detail();
        body();
        return SC_OK;
    } catch (const Failure &f) {
        return f.status;
    } catch (const std::bad_alloc &) {
        set_detail("host allocation failed");
        return SC_ERR_OOM;
    } catch (...) {
        set_detail("unexpected internal error");
        return SC_ERR_CUDA;
    }
}

// ---------------------------------------------------------------------------
// Device buffer with RAII ownership (plain cudaMalloc / cudaFree).
// ---------------------------------------------------------------------------
template <typename T>
struct DevBuf {
    T *ptr = nullptr;
    size_t count = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        count = 0;
    }
    // grow-only: keeps the old allocation if it is large enough
    void reserve(size_t n) {
        if (n <= count && ptr) return;
        release();
        if (n == 0) return;
        SC_CUDA(cudaMalloc(reinterpret_cast<void **>(&ptr), n * sizeof(T)));
        count = n;
    }
    T *get() const { return ptr; }
};

// ---------------------------------------------------------------------------
// Element types of the propagated block.
// ---------------------------------------------------------------------------
template <typename T>
struct AccOf {
    using type = float;
};
template <>
struct AccOf<double> {
    using type = double;
};

__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_acc(typename AccOf<T>::type v);
template <>
__device__ __forceinline__ float from_acc<float>(float v) { return v; }
template <>
__device__ __forceinline__ double from_acc<double>(double v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

inline int ceil_div(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

// a launch shape of the propagation: block width, 16-byte vectors per lane
// (0 = the TMA-gather kernel) and the measured time of one hop per source
struct TuneResult {
    int B, vpl;
    double ms_per_source_hop;
};

}  // namespace sc

// ---------------------------------------------------------------------------
// The graph object behind the opaque sc_graph handle.
// ---------------------------------------------------------------------------
struct sc_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t min_degree = 0, max_degree = 0;
    int32_t bipartite = 0;
    int32_t bfs_depth = 0;
    int num_sms = 0;
    size_t l2_bytes = 0;

    sc::DevBuf<int32_t> row_ptr, col_idx, rev, level;
    sc::DevBuf<float> inv_deg_f;
    sc::DevBuf<double> inv_deg_d;
    std::vector<int32_t> h_row_ptr;  // host copy of the row pointers (degrees, scheduling)

    // row schedule of the SIMT propagation kernel: heavy rows (degree above
    // the threshold, one CTA each, longest first) then light rows in order
    sc::DevBuf<int32_t> row_order;
    int32_t heavy_threshold_cached = -1;
    int32_t n_heavy = 0;
    // the heavy rows again, sorted by id (windowed launches), and on the host
    sc::DevBuf<int32_t> heavy_ids;
    std::vector<int32_t> h_heavy_ids;
    // bandwidth max |i - j| over the entries (i -> j); -1 until computed
    int32_t bandwidth = -1;
    // per-slice windows of windowed launches
    sc::DevBuf<unsigned char> win_list;
    // bit mask of the block's first-hop rows (hop 2 from the sources alone),
    // and the non-zero columns of X_2 (hop 3 from its non-zero values)
    sc::DevBuf<uint32_t> mask, mask_nz;
    // X_L at the sources (the last hop, computed where the gather reads it)
    sc::DevBuf<double> last_diag;
    // row runs of about equal CSR entries, one per warp, for the TMA kernel
    sc::DevBuf<int32_t> part;
    int32_t nparts = 0;
    int32_t part_target = -1;
    // autotuned (block width, lane split) per request key, and its measured ms per source-hop
    std::map<long long, std::pair<int, int>> tuned;
    std::map<long long, double> tuned_cost;
    // per request key: the best lane split of each block width, and the launch shape chosen
    // by timing one real block of each (the block loop's own kernels, see pick_block_width)
    std::map<long long, std::vector<sc::TuneResult>> tuned_per_b;
    std::map<long long, sc::TuneResult> tuned_block;

    // learned length: features (n x 6) and the loaded model
    sc::DevBuf<float> features, mlp;
    bool features_ready = false, mlp_loaded = false;

    // cached eigenvalue estimate
    bool has_lambda = false;
    sc_lambda lam{};

    // CalTau: the pairs of the last sc_eigenpairs (f_k node-major, n x eig_P,
    // their eigenvalues and the bound r on the rest) and the last sc_caltau lengths
    sc::DevBuf<double> eig_Fn;
    std::vector<double> eig_lam;
    double eig_rest = 1.0;
    int32_t eig_P = 0;
    bool eig_ready = false;
    sc::DevBuf<int32_t> caltau_tau;
    double caltau_eps = 0.0;
    bool caltau_ready = false;

    // work buffers (grow-only)
    sc::DevBuf<unsigned char> xa, xb;   // probability blocks
    sc::DevBuf<double> acc_g, acc_t1, acc_t2;
    sc::DevBuf<int32_t> tau_entry, src_list, status;
    sc::DevBuf<double> scratch_d;
    // TGT+ work buffers: CalChi partial and per-column statistics, walk counts
    sc::DevBuf<double> tp_pval, tp_pmin, tp_pmax, tp_cval, tp_cmin, tp_cmax, tp_cthr;
    sc::DevBuf<int32_t> tp_pid, tp_cid;
    sc::DevBuf<long long> tp_pvol, tp_cvol, tp_walks, tp_counters, tp_packed, tp_chunk_w0;
    sc::DevBuf<int32_t> tp_eq, tp_ek, tp_chunk_entry, tp_entry_chunk0;
    sc::DevBuf<double> tp_chunk_sum;
    sc::DevBuf<double> tp_srcstat;  // per column: rho_hat, min and max of p over N(s)
    sc::DevBuf<long long> tp_src_rhs;  // per column: Eq. 14's right side (per-source switch)
    sc::DevBuf<int32_t> tp_cap_list;   // the sources that switch at a test (per-source switch)
    std::vector<cudaEvent_t> hop_events;  // pairs bracketing timed propagation launches
    ~sc_graph() {
        for (cudaEvent_t e : hop_events) cudaEventDestroy(e);
    }
};

namespace sc {
void ensure_row_order(sc_graph *g, int32_t heavy_threshold);
int32_t ensure_bandwidth(sc_graph *g);
void ensure_partition(sc_graph *g, int32_t target);
void fill_i32(int32_t *p, int64_t count, int32_t v, cudaStream_t s);
}

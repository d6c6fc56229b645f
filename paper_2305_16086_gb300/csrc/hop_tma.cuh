// Propagation hop with TMA row gathers (sm_100a family: cp.async.bulk.tensor
// tile::gather4). Same arithmetic and summation order as k_spmm_hop
// (propagate.cuh): X_l[x, :] = (1/d_x) * sum_{j in N(x)} X_{l-1}[j, :] with
// chunks of 32 neighbours summed sequentially and chunk sums added in order,
// so both kernels give bitwise identical blocks.
//
// Each warp owns a run of consecutive rows holding about the same number of
// CSR entries (a host-built partition) and a private ring of S stages in
// shared memory; a stage holds the 4 rows X_{l-1}[j0..j3, :] fetched by one
// gather4 into consecutive rows of the stage, completing on the stage's
// mbarrier. Lane 0 keeps S stages in flight (indices read coalesced, 32 at a
// time, and broadcast by shuffles); the warp sums each landed stage into the
// running row and writes finished rows with coalesced stores. In-flight bytes
// therefore cost shared memory, not registers.
//
// Every mbarrier wait is bounded: on expiry the warp sets *status, waits
// (bounded again) for its own copies still in flight, and returns.
#pragma once

#include <cuda.h>

#include "propagate.cuh"

namespace sc {

constexpr int kTmaWarps = 8;
constexpr int kTmaWarpRingBytes = 8192;
constexpr uint64_t kStageWaitNs = 100000000ull;  // 100 ms: a stage lands within microseconds
constexpr uint64_t kDrainWaitNs = 10000000ull;   // 10 ms per in-flight copy when giving up

template <typename T, int B>
struct TmaLayout {
    using Acc = typename AccOf<T>::type;
    static constexpr int RB = B * static_cast<int>(sizeof(T));  // bytes per row
    static constexpr int STAGE = 4 * RB;                         // one gather4
    static constexpr int S = kTmaWarpRingBytes / STAGE;          // stages per warp
    static constexpr int EL = B / 32;                            // elements per lane
    static constexpr size_t SMEM = static_cast<size_t>(kTmaWarps) * kTmaWarpRingBytes + kTmaWarps * S * 8;
    static_assert(S >= 2, "ring too small");
    static_assert(B % 32 == 0, "B must be a multiple of 32");
};

struct TmaHopArgs {
    const int32_t *row_ptr;
    const int32_t *col;
    const void *inv_deg;   // Acc[n]
    void *x_next;          // slices x n x B
    int32_t n;
    const int32_t *part;   // warp w owns rows [part[w], part[w+1])
    int32_t nparts;
    int32_t part_ctas;
    int32_t gather_ctas;   // fused gather of X_{l-1} (first CTAs, one per source), as in HopArgs
    const void *x_prev;
    const int32_t *src;
    int32_t nsrc;
    const int32_t *tau;
    int32_t gather_ell;
    double *g, *t1, *t2;
    GatherRec rec;
    int32_t *status;       // bit 0: an mbarrier wait expired
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase with the given parity to complete, for at most limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// lane's EL elements of a staged row, converted to the accumulator type
template <int EL>
__device__ __forceinline__ void stage_add(const float *row, int lane, float *acc) {
    if constexpr (EL == 1) {
        acc[0] += row[lane];
    } else if constexpr (EL == 2) {
        const float2 v = reinterpret_cast<const float2 *>(row)[lane];
        acc[0] += v.x;
        acc[1] += v.y;
    } else {
        const float4 v = reinterpret_cast<const float4 *>(row)[lane];
        acc[0] += v.x;
        acc[1] += v.y;
        acc[2] += v.z;
        acc[3] += v.w;
    }
}
template <int EL>
__device__ __forceinline__ void stage_add(const double *row, int lane, double *acc) {
    if constexpr (EL == 1) {
        acc[0] += row[lane];
    } else if constexpr (EL == 2) {
        const double2 v = reinterpret_cast<const double2 *>(row)[lane];
        acc[0] += v.x;
        acc[1] += v.y;
    } else {
        const double2 v0 = reinterpret_cast<const double2 *>(row)[2 * lane];
        const double2 v1 = reinterpret_cast<const double2 *>(row)[2 * lane + 1];
        acc[0] += v0.x;
        acc[1] += v0.y;
        acc[2] += v1.x;
        acc[3] += v1.y;
    }
}
template <int EL>
__device__ __forceinline__ void stage_add(const __nv_bfloat16 *row, int lane, float *acc) {
    if constexpr (EL == 1) {
        acc[0] += __bfloat162float(row[lane]);
    } else if constexpr (EL == 2) {
        const uint32_t w = reinterpret_cast<const uint32_t *>(row)[lane];
        acc[0] += __uint_as_float(w << 16);
        acc[1] += __uint_as_float(w & 0xffff0000u);
    } else {
        const uint2 w = reinterpret_cast<const uint2 *>(row)[lane];
        acc[0] += __uint_as_float(w.x << 16);
        acc[1] += __uint_as_float(w.x & 0xffff0000u);
        acc[2] += __uint_as_float(w.y << 16);
        acc[3] += __uint_as_float(w.y & 0xffff0000u);
    }
}

template <int EL>
__device__ __forceinline__ void row_store(float *dst, int lane, const float *v) {
    if constexpr (EL == 1) dst[lane] = v[0];
    else if constexpr (EL == 2) reinterpret_cast<float2 *>(dst)[lane] = make_float2(v[0], v[1]);
    else reinterpret_cast<float4 *>(dst)[lane] = make_float4(v[0], v[1], v[2], v[3]);
}
template <int EL>
__device__ __forceinline__ void row_store(double *dst, int lane, const double *v) {
    if constexpr (EL == 1) dst[lane] = v[0];
    else if constexpr (EL == 2) reinterpret_cast<double2 *>(dst)[lane] = make_double2(v[0], v[1]);
    else {
        reinterpret_cast<double2 *>(dst)[2 * lane] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(dst)[2 * lane + 1] = make_double2(v[2], v[3]);
    }
}
template <int EL>
__device__ __forceinline__ void row_store(__nv_bfloat16 *dst, int lane, const float *v) {
    if constexpr (EL == 1) dst[lane] = __float2bfloat16_rn(v[0]);
    else if constexpr (EL == 2) reinterpret_cast<__nv_bfloat162 *>(dst)[lane] = __floats2bfloat162_rn(v[0], v[1]);
    else {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t *>(&a);
        w.y = *reinterpret_cast<uint32_t *>(&b);
        reinterpret_cast<uint2 *>(dst)[lane] = w;
    }
}

template <typename T, int B>
__global__ void __launch_bounds__(kTmaWarps * 32) k_hop_tma(const __grid_constant__ CUtensorMap tmap_prev,
                                                            const TmaHopArgs a) {
    using TL = TmaLayout<T, B>;
    using Acc = typename TL::Acc;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t cta = static_cast<int32_t>(blockIdx.x);
    const int32_t n = a.n;

    if (cta < a.gather_ctas) {  // fused gather of X_{l-1}, one CTA per source, first in the grid
        const int32_t q = static_cast<int32_t>(blockIdx.y) * B + cta;
        if (q < a.nsrc) {
            const int32_t s = a.src[q];
            if (s >= 0) {
                int32_t sb;
                const T *xs = slice_column<T, B>(static_cast<const T *>(a.x_prev), n, nullptr, q, &sb);
                gather_source<T, B>(a.row_ptr, a.col, xs, sb, s, a.tau, a.gather_ell, a.g, a.t1, a.t2, threadIdx.x,
                                    kTmaWarps * 32, a.rec);
            }
        }
        return;
    }
    const int32_t w = (cta - a.gather_ctas) * kTmaWarps + warp;
    if (w >= a.nparts) return;
    if (*reinterpret_cast<volatile int32_t *>(a.status) != 0) return;  // an earlier wait expired: stop early

    const int32_t *__restrict__ row_ptr = a.row_ptr;
    const int32_t *__restrict__ col = a.col;
    unsigned char *ring = smem + warp * kTmaWarpRingBytes;
    const uint32_t ring_u32 = smem_u32(ring);
    const uint32_t bar0 = smem_u32(smem + static_cast<size_t>(kTmaWarps) * kTmaWarpRingBytes) + warp * TL::S * 8;

    const int32_t r_begin = a.part[w], r_end = a.part[w + 1];
    const int32_t k_begin = row_ptr[r_begin], k_end = row_ptr[r_end];
    const int32_t total = k_end - k_begin;
    const int32_t nst = (total + 3) >> 2;
    const int32_t row_base = static_cast<int32_t>(blockIdx.y) * n;  // first tensor row of this slice

    if (lane == 0) {
        for (int s = 0; s < TL::S; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * s));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // issue window: lane t holds the index of stream entry 32*iw + t (padded
    // past the end with the last entry, so every gather4 reads valid rows)
    auto load_window = [&](int32_t iw) -> int32_t {
        const int32_t e = iw * 32 + lane;
        return col[k_begin + min(e, total - 1)];
    };
    int32_t cur_iw = 0;
    int32_t cur_win = load_window(0);
    int32_t nxt_win = load_window(1);
    auto issue = [&](int32_t it) {
        const int32_t e0 = it * 4;
        const int32_t iw = e0 >> 5;
        if (iw != cur_iw) {  // advances by one window at a time
            cur_win = nxt_win;
            cur_iw = iw;
            nxt_win = load_window(iw + 1);
        }
        const int o = e0 & 31;
        const int32_t j0 = __shfl_sync(0xffffffffu, cur_win, o);
        const int32_t j1 = __shfl_sync(0xffffffffu, cur_win, o + 1);
        const int32_t j2 = __shfl_sync(0xffffffffu, cur_win, o + 2);
        const int32_t j3 = __shfl_sync(0xffffffffu, cur_win, o + 3);
        if (lane == 0) {
            const int slot = it % TL::S;
            const uint32_t bar = bar0 + 8 * slot;
            const uint32_t dst = ring_u32 + slot * TL::STAGE;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(TL::STAGE) : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
                "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
                "l"(&tmap_prev), "r"(0), "r"(row_base + j0), "r"(row_base + j1), "r"(row_base + j2),
                "r"(row_base + j3), "r"(bar)
                : "memory");
        }
    };
    const int32_t first_batch = min(nst, TL::S);
    for (int32_t it = 0; it < first_batch; ++it) issue(it);

    // row bookkeeping: lane t holds row_ptr[r_begin + 32*rw + t + 1] (row ends)
    int32_t rw = 0;
    int32_t end_win = row_ptr[min(r_begin + lane + 1, r_end)];
    int32_t r = r_begin;
    int32_t row_start = k_begin;
    int32_t row_end = __shfl_sync(0xffffffffu, end_win, 0);
    Acc inv = static_cast<const Acc *>(a.inv_deg)[r];
    int32_t pos = 0;
    Acc acc[TL::EL], chunk[TL::EL];
#pragma unroll
    for (int q = 0; q < TL::EL; ++q) {
        acc[q] = Acc(0);
        chunk[q] = Acc(0);
    }
    T *xn = static_cast<T *>(a.x_next) + static_cast<int64_t>(blockIdx.y) * n * B;

    for (int32_t it = 0; it < nst; ++it) {
        const int slot = it % TL::S;
        if (!mbar_wait_bounded(bar0 + 8 * slot, static_cast<uint32_t>((it / TL::S) & 1), kStageWaitNs)) {
            if (lane == 0) atomicOr(a.status, 1);
            for (int32_t j = it + 1; j < min(nst, it + TL::S); ++j)  // copies still in flight
                mbar_wait_bounded(bar0 + 8 * (j % TL::S), static_cast<uint32_t>((j / TL::S) & 1), kDrainWaitNs);
            return;
        }
        const T *stage = reinterpret_cast<const T *>(ring + slot * TL::STAGE);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int32_t e = k_begin + it * 4 + i;
            if (e < k_end) {
                stage_add<TL::EL>(stage + i * B, lane, chunk);
                ++pos;
                if ((pos & (kChunk - 1)) == 0) {
#pragma unroll
                    for (int q = 0; q < TL::EL; ++q) {
                        acc[q] += chunk[q];
                        chunk[q] = Acc(0);
                    }
                }
                if (e + 1 == row_end) {  // row r complete
                    Acc outv[TL::EL];
#pragma unroll
                    for (int q = 0; q < TL::EL; ++q) outv[q] = (acc[q] + chunk[q]) * inv;
                    row_store<TL::EL>(xn + static_cast<int64_t>(r) * B, lane, outv);
#pragma unroll
                    for (int q = 0; q < TL::EL; ++q) {
                        acc[q] = Acc(0);
                        chunk[q] = Acc(0);
                    }
                    pos = 0;
                    ++r;
                    if (r < r_end) {
                        const int32_t t = r - r_begin - 32 * rw;
                        if (t == 32) {
                            ++rw;
                            end_win = row_ptr[min(r_begin + 32 * rw + lane + 1, r_end)];
                        }
                        row_start = row_end;
                        row_end = __shfl_sync(0xffffffffu, end_win, r - r_begin - 32 * rw);
                        inv = static_cast<const Acc *>(a.inv_deg)[r];
                    }
                }
            }
        }
        __syncwarp();
        if (it + TL::S < nst) issue(it + TL::S);
    }
    (void)row_start;
}

}  // namespace sc

// Hops of a block computed only where their values can be non-zero or are
// read (Algorithm 2 visits only the nodes its frontier reaches), for the
// single-graph block loop. Both kernels keep k_spmm_hop's summation order
// (chunks of 32 consecutive CSR entries summed in order, chunk sums added in
// chunk order, one scale by 1/d), so every value they store is bit for bit
// the one the full hop stores.
#pragma once

#include "propagate.cuh"

namespace sc {

// CPL = B/32 consecutive elements of a row: the share of one lane when a warp
// covers the B columns
template <typename T, int CPL>
struct alignas(CPL * sizeof(T)) LaneVec {
    T v[CPL];
};

template <int W>
__device__ __forceinline__ void load_words(const uint32_t *p, uint32_t *w) {
    if constexpr (W == 4) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
        w[0] = q.x, w[1] = q.y, w[2] = q.z, w[3] = q.w;
    } else if constexpr (W == 2) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
        w[0] = q.x, w[1] = q.y;
    } else {
        w[0] = __ldg(p);
    }
}

template <typename T>
struct SparseHopArgs {
    const int32_t *row_ptr, *col;
    const typename AccOf<T>::type *inv_deg;
    const T *x_prev;       // X_{l-1}, slices x n x B
    T *x_next;             // X_l
    const uint32_t *mask;  // slices x n x B/32 words: sparse hop: non-zero columns of X_{l-1};
                           // ball hop: bit b of row j marks j in N(s_b)
    int32_t n;
    const int32_t *row_order;  // heavy rows first (n_heavy of them)
    int32_t n_heavy, heavy_t, light_ctas, heavy_ctas, gather_ctas;
    // fused gather of X_{l-1} (hop gather_ell) for the slice's sources, one CTA each
    const int32_t *src;
    int32_t nsrc;
    const int32_t *tau;
    int32_t gather_ell;
    double *g, *t1, *t2;
    GatherRec rec;
};

template <typename T, int B>
__device__ __forceinline__ void fused_gather(const SparseHopArgs<T> &a) {
    const int32_t q = static_cast<int32_t>(blockIdx.y) * B + static_cast<int32_t>(blockIdx.x);
    if (q >= a.nsrc) return;
    const int32_t s = a.src[q];
    if (s < 0) return;
    int32_t sb;
    const T *xs = slice_column<T, B>(a.x_prev, a.n, nullptr, q, &sb);
    gather_source<T, B>(a.row_ptr, a.col, xs, sb, s, a.tau, a.gather_ell, a.g, a.t1, a.t2, threadIdx.x,
                        kSpmmWarps * 32, a.rec);
}

// ---------------------------------------------------------------------------
// A full hop that reads only the non-zero values of X_{l-1}. Bit b of
// mask[j] is set iff the stored X_{l-1}[j, b] != 0 (written by the hop that
// stored X_{l-1}); lane l covers the CPL columns l*CPL .. and loads a
// neighbour's CPL values only when one of their bits is set. A skipped load
// stands for CPL zeros, and adding a zero changes no sum, so X_l is the full
// hop's bit for bit while X_{l-1} is read only where it is non-zero (hop 3
// of a block: X_2 is about 1% dense on expanders).
// CTAs [0, gather_ctas): the gather of X_{l-1}; then one CTA per heavy row
// (a warp per chunk, chunk sums added in order through shared memory); then
// light rows, one warp per row, striding over the rows in natural order.
// ---------------------------------------------------------------------------
template <typename T, int B>
__global__ void __launch_bounds__(kSpmmWarps * 32) k_hop_sparse(const SparseHopArgs<T> a) {
    using Acc = typename AccOf<T>::type;
    constexpr int W = B / 32, CPL = B / 32, U = 8;
    using Vec = LaneVec<T, CPL>;
    if (static_cast<int32_t>(blockIdx.x) < a.gather_ctas) {
        fused_gather<T, B>(a);
        return;
    }
    const int32_t n = a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t soff = static_cast<int64_t>(blockIdx.y) * n * B;
    const T *__restrict__ xp = a.x_prev + soff;
    T *__restrict__ xn = a.x_next + soff;
    const uint32_t *__restrict__ nz = a.mask + static_cast<int64_t>(blockIdx.y) * n * W;
    const int32_t *__restrict__ row_ptr = a.row_ptr;
    const int32_t *__restrict__ col = a.col;
    const int lc0 = lane * CPL, lw = lc0 / 32;
    const uint32_t lmask = (CPL == 32 ? 0xffffffffu : ((1u << CPL) - 1u)) << (lc0 % 32);
    // entries [k0, k1) of a row added to chunk[] in CSR order
    auto add_range = [&](int32_t k0, int32_t k1, Acc *chunk) {
        int32_t k = k0;
        for (; k + U <= k1; k += U) {
            int32_t j[U];
            uint32_t w[U];
            Vec v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) j[u] = col[k + u];
#pragma unroll
            for (int u = 0; u < U; ++u) w[u] = __ldg(nz + static_cast<int64_t>(j[u]) * W + lw);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (w[u] & lmask) {
                    v[u] = *reinterpret_cast<const Vec *>(xp + static_cast<int64_t>(j[u]) * B + lc0);
                } else {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) v[u].v[c] = from_acc<T>(Acc(0));
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int c = 0; c < CPL; ++c) chunk[c] += to_acc(v[u].v[c]);
        }
        for (; k < k1; ++k) {
            const int32_t j = col[k];
            if (__ldg(nz + static_cast<int64_t>(j) * W + lw) & lmask) {
                const Vec v = *reinterpret_cast<const Vec *>(xp + static_cast<int64_t>(j) * B + lc0);
#pragma unroll
                for (int c = 0; c < CPL; ++c) chunk[c] += to_acc(v.v[c]);
            }
        }
    };
    const int32_t cta = static_cast<int32_t>(blockIdx.x) - a.gather_ctas;
    if (cta < a.n_heavy) {
        __shared__ Acc part[kSpmmWarps][B];
        const int32_t row = a.row_order[cta];
        const int32_t rb = row_ptr[row], re = row_ptr[row + 1];
        const int32_t nchunks = (re - rb + kChunk - 1) / kChunk;
        Acc total = Acc(0);  // thread t < B owns column t
        for (int32_t base = 0; base < nchunks; base += kSpmmWarps) {
            const int32_t c = base + warp;
            Acc chunk[CPL];
#pragma unroll
            for (int e = 0; e < CPL; ++e) chunk[e] = Acc(0);
            if (c < nchunks) add_range(rb + c * kChunk, min(rb + (c + 1) * kChunk, re), chunk);
#pragma unroll
            for (int e = 0; e < CPL; ++e) part[warp][lc0 + e] = chunk[e];
            __syncthreads();
            if (threadIdx.x < B) {
                const int cnt = min(kSpmmWarps, nchunks - base);
                for (int q = 0; q < cnt; ++q) total += part[q][threadIdx.x];
            }
            __syncthreads();
        }
        if (threadIdx.x < B) xn[static_cast<int64_t>(row) * B + threadIdx.x] = from_acc<T>(total * a.inv_deg[row]);
        return;
    }
    if (cta - a.n_heavy >= a.light_ctas) return;
    const int64_t stride = static_cast<int64_t>(a.light_ctas) * kSpmmWarps;
    const int32_t heavy_t = a.n_heavy > 0 ? a.heavy_t : 0x7fffffff;
    for (int64_t idx = static_cast<int64_t>(cta - a.n_heavy) * kSpmmWarps + warp; idx < n; idx += stride) {
        const int32_t row = static_cast<int32_t>(idx);
        const int32_t rb = row_ptr[row], re = row_ptr[row + 1];
        if (re - rb > heavy_t) continue;  // a heavy row: its own CTA computes it
        Acc acc[CPL], chunk[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = Acc(0);
        for (int32_t k0 = rb; k0 < re; k0 += kChunk) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) chunk[c] = Acc(0);
            add_range(k0, min(k0 + kChunk, re), chunk);
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[c] += chunk[c];
        }
        const Acc sc = a.inv_deg[row];
        Vec out;
#pragma unroll
        for (int c = 0; c < CPL; ++c) out.v[c] = from_acc<T>(acc[c] * sc);
        *reinterpret_cast<Vec *>(xn + static_cast<int64_t>(row) * B + lc0) = out;
    }
}

// ---------------------------------------------------------------------------
// Hop L-1 of a block whose last hop L is computed only where its gather reads
// it (k_last_diag / k_last_rows read X_{L-1} on N(s_b) and on N(N(s_b))):
// X_{L-1}[y, b] is needed only for y in the ball N(s_b) u N(N(s_b)), i.e.
// where bit b of ball(y) = mask[y] | OR_{j in N(y)} mask[j] is set (mask =
// the sources' neighbour bits of the block's hop 2). Nothing outside the
// balls is read later, so nothing else is stored. One warp per row: the lanes
// load the neighbours' mask words 32 at a time and OR them across the warp.
// A row with at most kBallSparseCols marked columns sums each of them over
// its neighbours (lane t loads neighbour t of a chunk of 32, and the chunk's
// values are added in CSR order by a shuffle fold); a row with more, or a
// heavy row (one CTA each), computes all B columns with the full hop's
// vector loads. Every value is summed in k_spmm_hop's order (chunks of 32 in
// CSR order, chunk sums in chunk order, one scale), so it is the full hop's.
// CTAs [0, gather_ctas): the gather of X_{L-2}; then one CTA per heavy row;
// then light CTAs whose warps stride over the rows.
// ---------------------------------------------------------------------------
constexpr int kBallSparseCols = 4;

template <typename T, int B>
__global__ void __launch_bounds__(kSpmmWarps * 32) k_hop_ball(const SparseHopArgs<T> a) {
    using Acc = typename AccOf<T>::type;
    constexpr int W = B / 32, CPL = B / 32, U = 8;
    using Vec = LaneVec<T, CPL>;
    if (static_cast<int32_t>(blockIdx.x) < a.gather_ctas) {
        fused_gather<T, B>(a);
        return;
    }
    const int32_t n = a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t soff = static_cast<int64_t>(blockIdx.y) * n * B;
    const T *__restrict__ xp = a.x_prev + soff;
    T *__restrict__ xn = a.x_next + soff;
    const uint32_t *__restrict__ m1 = a.mask + static_cast<int64_t>(blockIdx.y) * n * W;
    const int32_t *__restrict__ row_ptr = a.row_ptr;
    const int32_t *__restrict__ col = a.col;
    const int lc0 = lane * CPL;
    // ball bits of row y (every lane of the warp gets them)
    auto ball_of = [&](int32_t y, int32_t rb, int32_t re, uint32_t *ball) {
        load_words<W>(m1 + static_cast<int64_t>(y) * W, ball);
        for (int32_t k = rb + lane; k < re; k += 32) {
            uint32_t w[W];
            load_words<W>(m1 + static_cast<int64_t>(col[k]) * W, w);
#pragma unroll
            for (int q = 0; q < W; ++q) ball[q] |= w[q];
        }
#pragma unroll
        for (int q = 0; q < W; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ball[q] |= __shfl_xor_sync(0xffffffffu, ball[q], o);
    };
    // the lane's CPL columns of entries [k0, k1) added to chunk[] in CSR order
    auto add_range = [&](int32_t k0, int32_t k1, Acc *chunk) {
        int32_t k = k0;
        for (; k + U <= k1; k += U) {
            int32_t j[U];
            Vec v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) j[u] = col[k + u];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = *reinterpret_cast<const Vec *>(xp + static_cast<int64_t>(j[u]) * B + lc0);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int c = 0; c < CPL; ++c) chunk[c] += to_acc(v[u].v[c]);
        }
        for (; k < k1; ++k) {
            const Vec v = *reinterpret_cast<const Vec *>(xp + static_cast<int64_t>(col[k]) * B + lc0);
#pragma unroll
            for (int c = 0; c < CPL; ++c) chunk[c] += to_acc(v.v[c]);
        }
    };
    const int32_t cta = static_cast<int32_t>(blockIdx.x) - a.gather_ctas;
    if (cta < a.n_heavy) {
        // heavy row: all B columns when the row lies in any ball (chunks over the warps, sums in
        // chunk order through shared memory)
        __shared__ Acc part[kSpmmWarps][B];
        __shared__ int marked;
        const int32_t row = a.row_order[cta];
        const int32_t rb = row_ptr[row], re = row_ptr[row + 1];
        if (threadIdx.x == 0) marked = 0;
        __syncthreads();
        {
            uint32_t any = 0u;
            for (int32_t k = rb + static_cast<int32_t>(threadIdx.x); k < re; k += kSpmmWarps * 32) {
                uint32_t w[W];
                load_words<W>(m1 + static_cast<int64_t>(col[k]) * W, w);
#pragma unroll
                for (int q = 0; q < W; ++q) any |= w[q];
            }
            if (threadIdx.x < W) any |= m1[static_cast<int64_t>(row) * W + threadIdx.x];
            if (__any_sync(0xffffffffu, any != 0u) && lane == 0) atomicOr(&marked, 1);
        }
        __syncthreads();
        if (!marked) return;
        const int32_t nchunks = (re - rb + kChunk - 1) / kChunk;
        Acc total = Acc(0);  // thread t < B owns column t
        for (int32_t base = 0; base < nchunks; base += kSpmmWarps) {
            const int32_t c = base + warp;
            Acc chunk[CPL];
#pragma unroll
            for (int e = 0; e < CPL; ++e) chunk[e] = Acc(0);
            if (c < nchunks) add_range(rb + c * kChunk, min(rb + (c + 1) * kChunk, re), chunk);
#pragma unroll
            for (int e = 0; e < CPL; ++e) part[warp][lc0 + e] = chunk[e];
            __syncthreads();
            if (threadIdx.x < B) {
                const int cnt = min(kSpmmWarps, nchunks - base);
                for (int q = 0; q < cnt; ++q) total += part[q][threadIdx.x];
            }
            __syncthreads();
        }
        if (threadIdx.x < B) xn[static_cast<int64_t>(row) * B + threadIdx.x] = from_acc<T>(total * a.inv_deg[row]);
        return;
    }
    if (cta - a.n_heavy >= a.light_ctas) return;
    const int64_t stride = static_cast<int64_t>(a.light_ctas) * kSpmmWarps;
    const int32_t heavy_t = a.n_heavy > 0 ? a.heavy_t : 0x7fffffff;
    for (int64_t idx = static_cast<int64_t>(cta - a.n_heavy) * kSpmmWarps + warp; idx < n; idx += stride) {
        const int32_t y = static_cast<int32_t>(idx);
        const int32_t rb = row_ptr[y], re = row_ptr[y + 1];
        if (re - rb > heavy_t) continue;  // a heavy row: its own CTA computes it
        uint32_t ball[W];
        ball_of(y, rb, re, ball);
        int marked = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) marked += __popc(ball[q]);
        if (marked == 0) continue;
        const Acc sc = a.inv_deg[y];
        if (marked > kBallSparseCols) {
            // every column, the full hop's way
            Acc acc[CPL], chunk[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[c] = Acc(0);
            for (int32_t k0 = rb; k0 < re; k0 += kChunk) {
#pragma unroll
                for (int c = 0; c < CPL; ++c) chunk[c] = Acc(0);
                add_range(k0, min(k0 + kChunk, re), chunk);
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[c] += chunk[c];
            }
            Vec out;
#pragma unroll
            for (int c = 0; c < CPL; ++c) out.v[c] = from_acc<T>(acc[c] * sc);
            *reinterpret_cast<Vec *>(xn + static_cast<int64_t>(y) * B + lc0) = out;
            continue;
        }
        // the marked columns one by one: lane t loads neighbour t of each chunk, a shuffle fold
        // adds the chunk in CSR order
#pragma unroll
        for (int q = 0; q < W; ++q) {
            uint32_t bits = ball[q];
            while (bits) {  // warp-uniform
                const int b = q * 32 + __ffs(bits) - 1;
                bits &= bits - 1u;
                Acc acc = Acc(0);
                for (int32_t k0 = rb; k0 < re; k0 += kChunk) {
                    const int cnt = min(kChunk, re - k0);
                    const Acc x = lane < cnt ? to_acc(xp[static_cast<int64_t>(col[k0 + lane]) * B + b]) : Acc(0);
                    Acc chunk = Acc(0);
                    for (int t = 0; t < cnt; ++t) chunk += __shfl_sync(0xffffffffu, x, t);
                    acc += chunk;
                }
                if (lane == 0) xn[static_cast<int64_t>(y) * B + b] = from_acc<T>(acc * sc);
            }
        }
    }
}

}  // namespace sc

// The second hop of a block computed from its sources alone (no stored X_1
// block), for the single-graph driver.
#pragma once

#include "propagate.cuh"

namespace sc {

// ---------------------------------------------------------------------------
// Hop 2 from the sources alone. X_1[j, b] is the stored 1/d_j exactly when j
// is a neighbour of s_b (Alg. 2 line 2 and the first hop) and 0 otherwise,
// so X_2 needs no X_1 block: bit b of mask[j] marks j in N(s_b), and row r of
// X_2 sums the stored 1/d_j over its marked neighbours. Adding the zeros of
// the unmarked columns changes no sum, so every value is bit for bit the one
// of k_spmm_hop over the stored X_1 (same chunked order, same scale).
// ---------------------------------------------------------------------------
template <int B>
__global__ void k_mask_scatter(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                               const int32_t *__restrict__ src, int32_t nsrc, uint32_t *__restrict__ mask,
                               int32_t n) {
    const int32_t q = blockIdx.x;
    if (q >= nsrc) return;
    const int32_t s = src[q];
    if (s < 0) return;
    const int b = q % B;
    uint32_t *m = mask + static_cast<int64_t>(q / B) * n * (B / 32) + b / 32;
    for (int32_t k = row_ptr[s] + threadIdx.x; k < row_ptr[s + 1]; k += blockDim.x)
        atomicOr(m + static_cast<int64_t>(col[k]) * (B / 32), 1u << (b % 32));
}

template <typename T>
struct MaskHopArgs {
    const int32_t *row_ptr, *col;
    const typename AccOf<T>::type *inv_deg;
    const uint32_t *mask;  // slices x n x B/32 words
    T *x_next;             // X_2, slices x n x B
    int32_t n;
    const int32_t *row_order;  // heavy rows first (n_heavy of them)
    int32_t n_heavy, heavy_t, light_ctas, gather_ctas;
    const int32_t *src;
    int32_t nsrc;
    const int32_t *tau;
    double *g, *t1, *t2;
    GatherRec rec;
};

// four columns c0..c0+3 of X_1 at row j: the stored 1/d_j where marked
template <typename T>
__device__ __forceinline__ void mask_add(typename AccOf<T>::type *acc, uint32_t bits,
                                         typename AccOf<T>::type x) {
    using Acc = typename AccOf<T>::type;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += ((bits >> c) & 1u) ? x : Acc(0);
}

template <typename T>
__device__ __forceinline__ void store4(T *out, const typename AccOf<T>::type *v) {
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = from_acc<T>(v[c]);
}

// CTAs [0, gather_ctas): the gather of hop 1 for the slice's sources (term
// X_1[s,b] - X_1[j,b] = 0 - stored 1/d_j); the next n_heavy CTAs: one heavy
// row each; the rest: light rows, LG = B/4 lanes (four columns each) per
// row, striding over the rows in natural order and skipping heavy ones.
template <typename T, int B>
__global__ void __launch_bounds__(kSpmmWarps * 32) k_hop2_mask(const MaskHopArgs<T> a) {
    using Acc = typename AccOf<T>::type;
    constexpr int LG = B / 4, G = 32 / LG, W = B / 32, U = 8;
    const int32_t n = a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / LG, gl = lane % LG;
    const int c0 = gl * 4;
    const int shift = c0 % 32;
    const uint32_t *mask = a.mask + static_cast<int64_t>(blockIdx.y) * n * W + c0 / 32;
    T *xn = a.x_next + static_cast<int64_t>(blockIdx.y) * n * B;
    const int32_t *__restrict__ row_ptr = a.row_ptr;
    const int32_t *__restrict__ col = a.col;
    auto x1 = [&](int32_t j) { return to_acc(from_acc<T>(a.inv_deg[j])); };  // the stored X_1 value
    if (static_cast<int32_t>(blockIdx.x) < a.gather_ctas) {
        const int32_t q = static_cast<int32_t>(blockIdx.y) * B + static_cast<int32_t>(blockIdx.x);
        if (q < a.nsrc) {
            const int32_t s = a.src[q];
            if (s >= 0)
                for (int32_t k = row_ptr[s] + threadIdx.x; k < row_ptr[s + 1]; k += blockDim.x)
                    gather_term(k, 0.0 - static_cast<double>(x1(col[k])), a.tau, 1, a.g, a.t1, a.t2, a.rec);
        }
        return;
    }
    const int32_t cta = static_cast<int32_t>(blockIdx.x) - a.gather_ctas;
    if (cta < a.n_heavy) {
        constexpr int NGRP = kSpmmWarps * G;
        __shared__ Acc part[NGRP][B];
        const int32_t row = a.row_order[cta];
        const int32_t rb = row_ptr[row], re = row_ptr[row + 1];
        const int32_t nchunks = (re - rb + kChunk - 1) / kChunk;
        Acc total = Acc(0);  // thread t < B owns column t
        for (int32_t base = 0; base < nchunks; base += NGRP) {
            const int slot = warp * G + grp;
            const int32_t c = base + slot;
            Acc acc[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
            if (c < nchunks) {
                const int32_t kb = rb + c * kChunk, ke = min(kb + kChunk, re);
                for (int32_t k = kb; k < ke; ++k) {
                    const int32_t j = col[k];
                    mask_add<T>(acc, (mask[static_cast<int64_t>(j) * W] >> shift) & 0xFu, x1(j));
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) part[slot][c0 + e] = acc[e];
            __syncthreads();
            if (threadIdx.x < B) {
                const int cnt = min(NGRP, nchunks - base);
                for (int q = 0; q < cnt; ++q) total += part[q][threadIdx.x];
            }
            __syncthreads();
        }
        if (threadIdx.x < B) xn[static_cast<int64_t>(row) * B + threadIdx.x] = from_acc<T>(total * a.inv_deg[row]);
        return;
    }
    if (cta - a.n_heavy >= a.light_ctas) return;
    const int64_t stride = static_cast<int64_t>(a.light_ctas) * kSpmmWarps * G;
    const int32_t heavy_t = a.n_heavy > 0 ? a.heavy_t : 0x7fffffff;
    for (int64_t idx = (static_cast<int64_t>(cta - a.n_heavy) * kSpmmWarps + warp) * G + grp; idx < n;
         idx += stride) {
        const int32_t row = static_cast<int32_t>(idx);
        const int32_t rb = row_ptr[row], re = row_ptr[row + 1];
        if (re - rb > heavy_t) continue;  // a heavy row: its own CTA computes it
        Acc acc[4] = {Acc(0), Acc(0), Acc(0), Acc(0)}, chunk[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
        int32_t k = rb;
        for (; k + U <= re; k += U) {
            int32_t j[U];
            uint32_t m[U];
            Acc x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) j[u] = col[k + u];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                m[u] = mask[static_cast<int64_t>(j[u]) * W];
                x[u] = x1(j[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) mask_add<T>(chunk, (m[u] >> shift) & 0xFu, x[u]);
            if (((k + U - rb) % kChunk) == 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[c] += chunk[c];
                    chunk[c] = Acc(0);
                }
            }
        }
        for (; k < re; ++k) {
            const int32_t j = col[k];
            mask_add<T>(chunk, (mask[static_cast<int64_t>(j) * W] >> shift) & 0xFu, x1(j));
        }
        const Acc sc = a.inv_deg[row];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = (acc[c] + chunk[c]) * sc;
        store4<T>(xn + static_cast<int64_t>(row) * B + c0, acc);
    }
}

}  // namespace sc

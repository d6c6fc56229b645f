// The second hop of a block computed from its sources alone (no stored X_1
// block), for the single-graph block loop.
#pragma once

#include "propagate.cuh"

namespace sc {

// ---------------------------------------------------------------------------
// Hop 2 from the sources alone. X_1[j, b] is the stored 1/d_j exactly when j
// is a neighbour of s_b (Algorithm 2's initialisation and the first hop) and 0 otherwise,
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
    uint32_t *nz;  // nullable: slices x n x B/32 words, bit b of row r set iff the stored X_2[r, b] != 0
};



// CTAs [0, gather_ctas): the gather of hop 1 for the slice's sources (term
// X_1[s,b] - X_1[j,b] = 0 - stored 1/d_j); the next n_heavy CTAs: one heavy
// row each (a warp per chunk); the rest: light rows, one warp per row,
// striding over the rows in natural order and skipping heavy ones.
template <typename T, int B>
__global__ void __launch_bounds__(kSpmmWarps * 32) k_hop2_mask(const MaskHopArgs<T> a) {
    using Acc = typename AccOf<T>::type;
    constexpr int W = B / 32;  // mask words per node
    const int32_t n = a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    // one chunk of 32 entries (CSR positions k0 .. k0 + cnt) by one warp. Lane
    // l owns the CPL = W = B/32 columns l*W .., i.e. bits of mask word
    // l / GW (GW = 32 / W lanes per word). The lanes load the words in a
    // transposed order (lane l: word l / GW of neighbours r*GW + l % GW, r < W)
    // so that one shuffle per neighbour hands every lane its own word; one
    // more hands round the stored 1/d. Neighbours are taken in CSR order.
    constexpr int CPL = B / 32, GW = 32 / W;
    const int lc0 = lane * CPL, lw = lane / GW, lshift = lc0 % 32;
    const uint32_t *mrow = a.mask + static_cast<int64_t>(blockIdx.y) * n * W;
    auto chunk_sum = [&](int32_t k0, int cnt, Acc *chunk) {
        uint32_t vr[W];
#pragma unroll
        for (int r = 0; r < W; ++r) {
            const int nb = r * GW + lane % GW;
            vr[r] = nb < cnt ? mrow[static_cast<int64_t>(col[k0 + nb]) * W + lw] : 0u;
        }
        const Acc xj = lane < cnt ? x1(col[k0 + lane]) : Acc(0);
#pragma unroll
        for (int c = 0; c < CPL; ++c) chunk[c] = Acc(0);
        // X_1 is sparse: most neighbours have an all-zero mask and add only
        // zeros, so only the marked ones are handed round (still in CSR order)
#pragma unroll
        for (int r = 0; r < W; ++r) {
            const uint32_t b = __ballot_sync(0xffffffffu, vr[r] != 0u);
            uint32_t nz = 0u;  // bit uu: neighbour r * GW + uu has a marked column
#pragma unroll
            for (int w = 0; w < W; ++w) nz |= (b >> (w * GW)) & (GW == 32 ? 0xffffffffu : ((1u << GW) - 1u));
            while (nz) {
                const int uu = __ffs(nz) - 1;
                nz &= nz - 1u;
                const uint32_t m = __shfl_sync(0xffffffffu, vr[r], lw * GW + uu);
                const Acc xv = __shfl_sync(0xffffffffu, xj, r * GW + uu);
#pragma unroll
                for (int c = 0; c < CPL; ++c) chunk[c] += ((m >> (lshift + c)) & 1u) ? xv : Acc(0);
            }
        }
    };
    if (cta < a.n_heavy) {
        // heavy row: warp w sums chunks w, w + kSpmmWarps, ...; the chunk sums
        // are added in chunk order through shared memory
        __shared__ Acc part[kSpmmWarps][B];
        const int32_t row = a.row_order[cta];
        const int32_t rb = row_ptr[row], re = row_ptr[row + 1];
        const int32_t nchunks = (re - rb + kChunk - 1) / kChunk;
        Acc total = Acc(0);  // thread t < B owns column t
        for (int32_t base = 0; base < nchunks; base += kSpmmWarps) {
            const int32_t c = base + warp;
            Acc chunk[CPL];
            if (c < nchunks) {
                chunk_sum(rb + c * kChunk, min(kChunk, re - (rb + c * kChunk)), chunk);
            } else {
#pragma unroll
                for (int e = 0; e < CPL; ++e) chunk[e] = Acc(0);
            }
#pragma unroll
            for (int e = 0; e < CPL; ++e) part[warp][lc0 + e] = chunk[e];
            __syncthreads();
            if (threadIdx.x < B) {
                const int cnt = min(kSpmmWarps, nchunks - base);
                for (int q = 0; q < cnt; ++q) total += part[q][threadIdx.x];
            }
            __syncthreads();
        }
        T v = from_acc<T>(Acc(0));
        if (threadIdx.x < B) {
            v = from_acc<T>(total * a.inv_deg[row]);
            xn[static_cast<int64_t>(row) * B + threadIdx.x] = v;
        }
        if (a.nz && threadIdx.x < B) {  // B is a multiple of 32: warp w holds columns 32 w ..
            const uint32_t word = __ballot_sync(0xffffffffu, to_acc(v) != Acc(0));
            if (lane == 0) a.nz[(static_cast<int64_t>(blockIdx.y) * n + row) * W + warp] = word;
        }
        return;
    }
    // light rows: one warp per row, chunk by chunk
    if (cta - a.n_heavy >= a.light_ctas) return;
    const int64_t stride = static_cast<int64_t>(a.light_ctas) * kSpmmWarps;
    const int32_t heavy_t = a.n_heavy > 0 ? a.heavy_t : 0x7fffffff;
    // the next row's bounds are loaded while the current row's chunks are in flight
    int64_t idx = static_cast<int64_t>(cta - a.n_heavy) * kSpmmWarps + warp;
    int32_t rb_next = 0, re_next = 0;
    if (idx < n) {
        rb_next = row_ptr[idx];
        re_next = row_ptr[idx + 1];
    }
    for (; idx < n; idx += stride) {
        const int32_t row = static_cast<int32_t>(idx);
        const int32_t rb = rb_next, re = re_next;
        if (idx + stride < n) {
            rb_next = row_ptr[idx + stride];
            re_next = row_ptr[idx + stride + 1];
        }
        if (re - rb > heavy_t) continue;  // a heavy row: its own CTA computes it
        const Acc sc = a.inv_deg[row];
        Acc acc[CPL], chunk[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = Acc(0);
        for (int32_t k0 = rb; k0 < re; k0 += kChunk) {
            chunk_sum(k0, min(kChunk, re - k0), chunk);
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[c] += chunk[c];
        }
        // the lane's CPL values are contiguous: one vector store
        struct alignas(CPL * sizeof(T)) Vec {
            T v[CPL];
        } out;
#pragma unroll
        for (int c = 0; c < CPL; ++c) out.v[c] = from_acc<T>(acc[c] * sc);
        *reinterpret_cast<Vec *>(xn + static_cast<int64_t>(row) * B + lc0) = out;
        if (a.nz) {
            // the lane's CPL bits at lshift of word lw; the GW lanes of a word OR theirs together
            uint32_t bits = 0u;
#pragma unroll
            for (int c = 0; c < CPL; ++c) bits |= (to_acc(out.v[c]) != Acc(0) ? 1u : 0u) << (lshift + c);
#pragma unroll
            for (int o = GW / 2; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
            if (lane % GW == 0) a.nz[(static_cast<int64_t>(blockIdx.y) * n + row) * W + lw] = bits;
        }
    }
}

}  // namespace sc

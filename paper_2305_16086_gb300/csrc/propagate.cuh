// Kernels of the truncated graph traversal (Algorithm 2), shared by the
// single-graph entry point (propagate.cu), the allocation-free one and the
// batched one.
//
// Layout: a block of B sources is an n x B row-major matrix X (node x's B
// probabilities p_l(x, s_b) contiguous, rows 16-byte aligned); S = slices x B
// sources are propagated by one launch, slice q at X + q * n * B.
//
// Hop l: X_l[x, :] = (1/d_x) * sum_{j in N(x)} X_{l-1}[j, :]   (Algorithm 2's hop,
// pull form of the scatter p_l(v_x, v_i) += p_{l-1}(v_j, v_i) / d(v_x)).
//
// Summation order (fixed, independent of B, of the lane split, of the row
// schedule, of the light/heavy row path and of the TMA variant in hop_tma.cuh): the neighbours of a row are cut
// into chunks of 32 consecutive CSR entries; each chunk is summed
// sequentially in CSR order and the chunk sums are added in chunk order. The
// result is then scaled once by 1/d_x.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace sc {

constexpr int kChunk = 32;       // neighbours per sequential chunk
constexpr int kSpmmWarps = 4;    // warps per CTA of the propagation kernel

template <typename T, int B, int VPL>
struct Layout {
    using Acc = typename AccOf<T>::type;
    static constexpr int E = 16 / static_cast<int>(sizeof(T));  // elements per 16-byte vector
    static constexpr int V = B / E;                              // vectors per row
    static constexpr int LG = V / VPL;                           // lanes per row group
    static constexpr int G = 32 / LG;                            // row groups per warp
    static constexpr int NACC = VPL * E;                         // accumulators per lane
    static constexpr int U = (VPL >= 4) ? 2 : (VPL == 2 ? 4 : 8);  // row loads in flight per lane
    static_assert(V % VPL == 0, "bad split");
    static_assert(LG >= 1 && LG <= 32 && (32 % LG) == 0, "lanes per row must divide 32");
    static_assert(kChunk % U == 0, "unroll must divide the chunk");
};

// ---- 16-byte vector <-> accumulators ---------------------------------------
__device__ __forceinline__ void vadd(float *acc, const uint4 &v, float) {
    acc[0] += __uint_as_float(v.x);
    acc[1] += __uint_as_float(v.y);
    acc[2] += __uint_as_float(v.z);
    acc[3] += __uint_as_float(v.w);
}
__device__ __forceinline__ void vadd(double *acc, const uint4 &v, double) {
    acc[0] += __hiloint2double(static_cast<int>(v.y), static_cast<int>(v.x));
    acc[1] += __hiloint2double(static_cast<int>(v.w), static_cast<int>(v.z));
}
__device__ __forceinline__ void vadd(float *acc, const uint4 &v, __nv_bfloat16) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        acc[2 * q] += __uint_as_float(w[q] << 16);
        acc[2 * q + 1] += __uint_as_float(w[q] & 0xffff0000u);
    }
}

__device__ __forceinline__ uint4 vpack(const float *a, float) {
    return make_uint4(__float_as_uint(a[0]), __float_as_uint(a[1]), __float_as_uint(a[2]), __float_as_uint(a[3]));
}
__device__ __forceinline__ uint4 vpack(const double *a, double) {
    return make_uint4(static_cast<uint32_t>(__double2loint(a[0])), static_cast<uint32_t>(__double2hiint(a[0])),
                      static_cast<uint32_t>(__double2loint(a[1])), static_cast<uint32_t>(__double2hiint(a[1])));
}
__device__ __forceinline__ uint4 vpack(const float *a, __nv_bfloat16) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a[2 * q], a[2 * q + 1]);
        w[q] = *reinterpret_cast<uint32_t *>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint4 ld_x(const uint4 *p) { return __ldg(p); }

// What the gather records besides the half sums.
struct GatherRec {
    int mode;       // 0: t1, t2 = terms of hops tau+1, tau+2; 1: terms of hops tau-1, tau;
                    // 2: no t1 / t2; all[k * stride + ell / 2] = term of every even hop ell < 2 stride
                    // 3: as 0, and all[k * 2 + 0 / 1] = terms of hops tau-1, tau
    double *all;    // nullable: (modes 0, 1) all[k * stride + ell] = term of hop ell (every hop)
    int stride;
};

// The rows one slice of a launch covers (the frontier of Algorithm 2, which
// only visits nodes with p_{l-1} > 0, kept as an interval). The slice stores
// rows [base, base + rows) at element offset xoff of the block buffer; hop l
// computes rows [lo_l, hi_l) = [max(seg_lo, src_lo - l beta), min(seg_hi,
// src_hi + l beta)) with beta the graph's bandwidth (beta = 0: the whole
// segment). A segment is one graph of a batch (or the whole graph). The
// support of X_l lies in [lo_l, hi_l) and rows outside it stay zero, so the
// result is the one of the full hop.
struct SliceWin {
    int64_t xoff;
    int32_t base, rows;
    int32_t seg_lo, seg_hi;
    int32_t src_lo, src_hi;
    int32_t heavy_begin, heavy_cnt;  // the segment's heavy rows in the id-sorted heavy list
    int32_t L;                       // hops of the slice's block: no rows are computed past it
    // a bipartite segment whose block holds sources of one colour c (BFS depth parity): X_l is
    // zero on every row of colour c + l + 1 (mod 2), so hop l computes the rows of colour
    // c + l (mod 2) only; -1: every row
    int32_t parity;
};

__host__ __device__ __forceinline__ void window_rows(const SliceWin &w, int32_t beta, int32_t ell, int32_t *lo,
                                                     int32_t *hi) {
    int64_t a = w.seg_lo, b = w.seg_hi;
    if (beta > 0) {
        a = max(a, static_cast<int64_t>(w.src_lo) - static_cast<int64_t>(ell) * beta);
        b = min(b, static_cast<int64_t>(w.src_hi) + static_cast<int64_t>(ell) * beta);
    }
    *lo = static_cast<int32_t>(a);
    *hi = static_cast<int32_t>(b);
}

// Arguments of one hop launch.
template <typename T>
struct HopArgs {
    const int32_t *row_ptr;
    const int32_t *col;
    const typename AccOf<T>::type *inv_deg;
    const T *x_prev;   // X_{l-1}, slices x n x B
    T *x_next;         // X_l
    int32_t n;
    // row schedule: row_order[0 .. n_heavy) are the rows of degree above the
    // heavy threshold heavy_t (one CTA each, longest first); the row groups
    // take every row in natural order and skip those (n_heavy = 0: no heavy
    // rows, row_order unused)
    const int32_t *row_order;
    int32_t n_heavy;
    int32_t light_ctas;
    // fused gather of X_{l-1} for the launch's sources (gather_ell > 0), one
    // CTA per source of the slice, placed first in the grid: see gather_source
    int32_t gather_ctas;
    const int32_t *src;
    int32_t nsrc;
    const int32_t *tau;
    int32_t gather_ell;
    double *g, *t1, *t2;
    GatherRec rec;
    // windowed launch (win != nullptr): per slice (blockIdx.y) window, the hop
    // index, the bandwidth, the id-sorted heavy rows and the heavy threshold
    const SliceWin *win;
    int32_t ell, beta;
    const int32_t *heavy_ids;
    int32_t heavy_t;
    const int32_t *level;  // BFS depth per node (its parity is the colour of a bipartite graph)
};

// Algorithm 2's accumulation of Eq. 9 for hop `ell` and launch source q (slice q / B, column
// q % B): for source i = s_b and each entry k = (i -> j) the unscaled half term
// p_l(v_i,v_i) - p_l(v_j,v_i) is added to g[k] while ell <= tau[k]; t1, t2
// keep the terms of hops tau+1, tau+2 (mode 0) or tau-1, tau (mode 1). (The
// 1/d(v_i) factor of Eq. 9 is applied once in the combine.) Threads tid of
// nthr take the entries of the source's row in turn (one CTA per source, so a
// hub's row does not serialise on one warp).
// xs points at the source's column of its slice, whose first stored row is
// `base`.
// the update of entry k by its hop-ell term
__device__ __forceinline__ void gather_term(int32_t k, double term, const int32_t *__restrict__ tau, int32_t ell,
                                            double *__restrict__ g, double *__restrict__ t1, double *__restrict__ t2,
                                            const GatherRec &rec) {
    const int32_t tk = tau[k];
    if (ell <= tk) {
        g[k] += term;
        if (rec.mode == 1) {
            if (ell == tk - 1) t1[k] = term;
            else if (ell == tk) t2[k] = term;
        }
    } else if (rec.mode == 0 || rec.mode == 3) {
        if (ell == tk + 1) t1[k] = term;
        else if (ell == tk + 2) t2[k] = term;
    }
    if (rec.all) {
        if (rec.mode == 2) {
            if ((ell & 1) == 0 && (ell >> 1) < rec.stride)
                rec.all[static_cast<int64_t>(k) * rec.stride + (ell >> 1)] = term;
        } else if (rec.mode == 3) {
            if (ell == tk - 1 || ell == tk) rec.all[static_cast<int64_t>(k) * 2 + (ell - tk + 1)] = term;
        } else {
            rec.all[static_cast<int64_t>(k) * rec.stride + ell] = term;
        }
    }
}

template <typename T, int B>
__device__ __forceinline__ void gather_source(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                              const T *__restrict__ xs, int32_t base, int32_t s,
                                              const int32_t *__restrict__ tau, int32_t ell, double *__restrict__ g,
                                              double *__restrict__ t1, double *__restrict__ t2, int tid, int nthr,
                                              const GatherRec rec) {
    const double diag = static_cast<double>(to_acc(xs[static_cast<int64_t>(s - base) * B]));
    for (int32_t k = row_ptr[s] + tid; k < row_ptr[s + 1]; k += nthr) {
        const int32_t j = col[k];
        gather_term(k, diag - static_cast<double>(to_acc(xs[static_cast<int64_t>(j - base) * B])), tau, ell, g, t1,
                    t2, rec);
    }
}

// column q % B of slice q / B: pointer and first stored row
template <typename T, int B>
__device__ __forceinline__ const T *slice_column(const T *x, int32_t n, const SliceWin *win, int32_t q,
                                                 int32_t *base) {
    if (win) {
        *base = win[q / B].base;
        return x + win[q / B].xoff + (q % B);
    }
    *base = 0;
    return x + static_cast<int64_t>(q / B) * n * B + (q % B);
}

// ---------------------------------------------------------------------------
// One hop for S = gridDim.y slices. CTAs [0, gather_ctas) gather X_{l-1} for
// the slice's sources (first, so that a hub source's long row overlaps the
// hop instead of trailing it); the next n_heavy CTAs each take one heavy row
// and split its chunks over all warps; the last light_ctas CTAs give each row
// group of LG lanes one light row. A windowed launch takes its slice's
// heavy rows from the id-sorted list and its light rows in natural order over
// the window, skipping the heavy ones; rows are stored from the slice's base.
// ---------------------------------------------------------------------------
// The last entries [k, ce) of a row or chunk, fewer than U of them: loaded in
// groups of U/2, U/4, ..., 1 entries (the binary digits of their count), each
// group's loads in flight together, and added in entry order (the order of
// the one-at-a-time loop, so every sum is unchanged bit for bit).
template <typename T, int B, int VPL>
__device__ __forceinline__ void add_tail(const int32_t *__restrict__ col, const uint4 *xp, int32_t k, int32_t ce,
                                         int gl, typename Layout<T, B, VPL>::Acc *chunk) {
    using L = Layout<T, B, VPL>;
    constexpr int W = L::U / 2 > 0 ? L::U / 2 : 1;
#pragma unroll
    for (int w = W; w >= 1; w >>= 1) {
        if (k + w <= ce) {
            int32_t j[W];
#pragma unroll
            for (int u = 0; u < w; ++u) j[u] = col[k + u];
            uint4 v[W][VPL];
#pragma unroll
            for (int u = 0; u < w; ++u)
#pragma unroll
                for (int p = 0; p < VPL; ++p) v[u][p] = ld_x(xp + static_cast<int64_t>(j[u]) * L::V + gl + p * L::LG);
#pragma unroll
            for (int u = 0; u < w; ++u)
#pragma unroll
                for (int p = 0; p < VPL; ++p) vadd(chunk + p * L::E, v[u][p], T());
            k += w;
        }
    }
}

template <typename T, int B, int VPL, bool WIN>
__global__ void __launch_bounds__(kSpmmWarps * 32) k_spmm_hop(const HopArgs<T> a) {
    using L = Layout<T, B, VPL>;
    using Acc = typename L::Acc;
    const int32_t n = a.n;
    int64_t slice_off = static_cast<int64_t>(blockIdx.y) * n * B;
    int32_t base = 0, lo = 0, hi = n, n_heavy = a.n_heavy;
    int32_t want = -1;  // windowed bipartite block: the colour of the rows hop ell computes
    if constexpr (WIN) {
        const SliceWin w = a.win[blockIdx.y];
        if (w.parity >= 0) want = (w.parity + a.ell) & 1;
        slice_off = w.xoff;
        base = w.base;
        int64_t wa = w.seg_lo, wb = w.seg_hi;
        if (a.beta > 0) {
            wa = max(wa, static_cast<int64_t>(w.src_lo) - static_cast<int64_t>(a.ell) * a.beta);
            wb = min(wb, static_cast<int64_t>(w.src_hi) + static_cast<int64_t>(a.ell) * a.beta);
        }
        lo = static_cast<int32_t>(wa);
        hi = static_cast<int32_t>(wb);
        n_heavy = w.heavy_cnt;
        if (a.ell > w.L) lo = hi = 0, n_heavy = 0;  // the block is done: only its gather remains
    }
    // rows are addressed as (row - base) within the slice (base = 0 unwindowed)
    const uint4 *xp = reinterpret_cast<const uint4 *>(a.x_prev + slice_off) - static_cast<int64_t>(base) * L::V;
    uint4 *xn = reinterpret_cast<uint4 *>(a.x_next + slice_off) - static_cast<int64_t>(base) * L::V;
    const int32_t *__restrict__ row_ptr = a.row_ptr;
    const int32_t *__restrict__ col = a.col;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / L::LG, gl = lane % L::LG;
    if (static_cast<int32_t>(blockIdx.x) < a.gather_ctas) {
        // ---------------- fused gather of X_{l-1} ----------------
        const int32_t q = static_cast<int32_t>(blockIdx.y) * B + static_cast<int32_t>(blockIdx.x);
        if (q < a.nsrc) {
            const int32_t s = a.src[q];
            if (s >= 0) {
                int32_t sb;
                const T *xs = slice_column<T, B>(a.x_prev, n, WIN ? a.win : nullptr, q, &sb);
                gather_source<T, B>(row_ptr, col, xs, sb, s, a.tau, a.gather_ell, a.g, a.t1, a.t2, threadIdx.x,
                                    kSpmmWarps * 32, a.rec);
            }
        }
        return;
    }
    const int32_t cta = static_cast<int32_t>(blockIdx.x) - a.gather_ctas;

    if (cta < n_heavy) {
        // ---------------- heavy row: chunks spread over the CTA ----------------
        constexpr int NGRP = kSpmmWarps * L::G;  // chunk slots per round
        __shared__ Acc part[NGRP][B];
        int32_t row;
        if constexpr (WIN) {
            row = a.heavy_ids[a.win[blockIdx.y].heavy_begin + cta];
            if (row < lo || row >= hi) return;  // outside the window: X_l is zero there
            if (want >= 0 && (a.level[row] & 1) != want) return;  // the other colour: zero too
        } else {
            row = a.row_order[cta];
        }
        const int32_t rb = row_ptr[row], re = row_ptr[row + 1];
        const int32_t nchunks = (re - rb + kChunk - 1) / kChunk;
        Acc total = Acc(0);  // thread t < B owns column t
        for (int32_t base = 0; base < nchunks; base += NGRP) {
            const int slot = warp * L::G + grp;
            const int32_t c = base + slot;
            Acc acc[L::NACC];
#pragma unroll
            for (int q = 0; q < L::NACC; ++q) acc[q] = Acc(0);
            if (c < nchunks) {
                const int32_t kb = rb + c * kChunk;
                const int32_t ke = min(kb + kChunk, re);
                int32_t k = kb;
                for (; k + L::U <= ke; k += L::U) {
                    int32_t j[L::U];
#pragma unroll
                    for (int u = 0; u < L::U; ++u) j[u] = col[k + u];
                    uint4 v[L::U][VPL];
#pragma unroll
                    for (int u = 0; u < L::U; ++u)
#pragma unroll
                        for (int p = 0; p < VPL; ++p) v[u][p] = ld_x(xp + static_cast<int64_t>(j[u]) * L::V + gl + p * L::LG);
#pragma unroll
                    for (int u = 0; u < L::U; ++u)
#pragma unroll
                        for (int p = 0; p < VPL; ++p) vadd(acc + p * L::E, v[u][p], T());
                }
                add_tail<T, B, VPL>(col, xp, k, ke, gl, acc);
            }
#pragma unroll
            for (int p = 0; p < VPL; ++p)
#pragma unroll
                for (int e = 0; e < L::E; ++e) part[slot][(gl + p * L::LG) * L::E + e] = acc[p * L::E + e];
            __syncthreads();
            if (threadIdx.x < B) {
                const int cnt = min(NGRP, nchunks - base);
                for (int q = 0; q < cnt; ++q) total += part[q][threadIdx.x];
            }
            __syncthreads();
        }
        if (threadIdx.x < B) {
            T *out = a.x_next + slice_off + static_cast<int64_t>(row - base) * B;
            out[threadIdx.x] = from_acc<T>(total * a.inv_deg[row]);
        }
        return;
    }

    // ---------------- light rows: one row per group of LG lanes at a time ----------------
    // The light CTAs stride over the rows (a few rows per group, about 64 CTAs
    // per SM in the grid) and load the next row's bounds while the current
    // row's gathers are in flight.
    // Rows are taken in natural order; the heavy ones (their own CTAs above)
    // are skipped.
    if (cta - n_heavy >= a.light_ctas) return;
    const int64_t nlight = WIN ? static_cast<int64_t>(hi - lo) : static_cast<int64_t>(n);
    const int64_t stride = static_cast<int64_t>(a.light_ctas) * kSpmmWarps * L::G;
    const int32_t row0 = WIN ? lo : 0;
    const int32_t heavy_t = n_heavy > 0 || WIN ? a.heavy_t : 0x7fffffff;
    int64_t idx = (static_cast<int64_t>(cta - n_heavy) * kSpmmWarps + warp) * L::G + grp;
    auto row_at = [&](int64_t i) -> int32_t { return row0 + static_cast<int32_t>(i); };
    int32_t row = 0, rb = 0, re = 0, lv = 0;
    if (idx < nlight) {
        row = row_at(idx);
        rb = row_ptr[row];
        re = row_ptr[row + 1];
        if (WIN && want >= 0) lv = a.level[row];
    }
    for (; idx < nlight; idx += stride) {
        const int32_t cur = row, cb = rb, ce = re, cl = lv;
        if (idx + stride < nlight) {
            row = row_at(idx + stride);
            rb = row_ptr[row];
            re = row_ptr[row + 1];
            if (WIN && want >= 0) lv = a.level[row];
        }
        if (ce - cb > heavy_t) continue;  // a heavy row: its own CTA computes it
        if (WIN && want >= 0 && (cl & 1) != want) continue;  // the other colour: X_l is zero there
        Acc acc[L::NACC], chunk[L::NACC];
#pragma unroll
        for (int q = 0; q < L::NACC; ++q) {
            acc[q] = Acc(0);
            chunk[q] = Acc(0);
        }
        int32_t k = cb;
        for (; k + L::U <= ce; k += L::U) {
            int32_t j[L::U];
#pragma unroll
            for (int u = 0; u < L::U; ++u) j[u] = col[k + u];
            uint4 v[L::U][VPL];
#pragma unroll
            for (int u = 0; u < L::U; ++u)
#pragma unroll
                for (int p = 0; p < VPL; ++p)
                    v[u][p] = ld_x(xp + static_cast<int64_t>(j[u]) * L::V + gl + p * L::LG);
#pragma unroll
            for (int u = 0; u < L::U; ++u)
#pragma unroll
                for (int p = 0; p < VPL; ++p) vadd(chunk + p * L::E, v[u][p], T());
            if (((k + L::U - cb) % kChunk) == 0) {  // a chunk of 32 positions is complete
#pragma unroll
                for (int q = 0; q < L::NACC; ++q) {
                    acc[q] += chunk[q];
                    chunk[q] = Acc(0);
                }
            }
        }
        add_tail<T, B, VPL>(col, xp, k, ce, gl, chunk);
#pragma unroll
        for (int q = 0; q < L::NACC; ++q) acc[q] += chunk[q];
        const Acc sc = a.inv_deg[cur];
#pragma unroll
        for (int q = 0; q < L::NACC; ++q) acc[q] *= sc;
#pragma unroll
        for (int p = 0; p < VPL; ++p)
            xn[static_cast<int64_t>(cur) * L::V + gl + p * L::LG] = vpack(acc + p * L::E, T());
    }
}

// X_1 = P e_s for each source s of the launch (Algorithm 2's initialisation followed by the
// first hop): X_1[j, b] = 1/d_j for j in N(s_b). X_1 must be zero on entry.
// One CTA per source.
template <typename T, int B>
__global__ void k_first_hop(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                            const typename AccOf<T>::type *__restrict__ inv_deg, const int32_t *__restrict__ src,
                            int32_t nsrc, T *__restrict__ x1, int32_t n, const SliceWin *__restrict__ win) {
    const int32_t q = blockIdx.x;
    if (q >= nsrc) return;
    const int32_t s = src[q];
    if (s < 0) return;
    int32_t base;
    T *xs = const_cast<T *>(slice_column<T, B>(x1, n, win, q, &base));
    for (int32_t k = row_ptr[s] + threadIdx.x; k < row_ptr[s + 1]; k += blockDim.x) {
        const int32_t j = col[k];
        xs[static_cast<int64_t>(j - base) * B] = from_acc<T>(inv_deg[j]);
    }
}

// stand-alone gather (the last hop of a block, and callers without fusion):
// one CTA per source
template <typename T, int B>
__global__ void k_gather(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                         const T *__restrict__ x, int32_t n, const int32_t *__restrict__ src, int32_t nsrc,
                         const int32_t *__restrict__ tau, int32_t ell, double *__restrict__ g,
                         double *__restrict__ t1, double *__restrict__ t2, const GatherRec rec,
                         const SliceWin *__restrict__ win) {
    const int32_t q = blockIdx.x;
    if (q >= nsrc) return;
    const int32_t s = src[q];
    if (s < 0) return;
    int32_t base;
    const T *xs = slice_column<T, B>(x, n, win, q, &base);
    gather_source<T, B>(row_ptr, col, xs, base, s, tau, ell, g, t1, t2, threadIdx.x, blockDim.x, rec);
}

// X_ell[r, b] from X_{ell-1} for one row r and one column b, by one warp,
// in the summation order of k_spmm_hop (chunks of 32 consecutive entries
// summed in order, chunk sums added in chunk order, one scale by 1/d), then
// rounded to the storage type: the value a full hop would have stored.
// xs: column b of X_{ell-1}, rows addressed from `base`.
template <typename T, int B>
__device__ __forceinline__ double hop_value(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                            const typename AccOf<T>::type *__restrict__ inv_deg,
                                            const T *__restrict__ xs, int32_t base, int32_t r, int lane) {
    using Acc = typename AccOf<T>::type;
    const int32_t rb = row_ptr[r], re = row_ptr[r + 1];
    Acc acc = Acc(0);
    for (int32_t c0 = rb; c0 < re; c0 += 32 * kChunk) {  // 32 chunks per round, lane l sums chunk l
        const int32_t kb = c0 + lane * kChunk, ke = min(kb + kChunk, re);
        Acc chunk = Acc(0);
#pragma unroll 8
        for (int32_t k = kb; k < ke; ++k) chunk += to_acc(xs[static_cast<int64_t>(col[k] - base) * B]);
        const int nch = min(32, (re - c0 + kChunk - 1) / kChunk);  // chunks in this round (warp-uniform)
        for (int l = 0; l < nch; ++l) acc += __shfl_sync(0xffffffffu, chunk, l);
    }
    acc *= inv_deg[r];
    return static_cast<double>(to_acc(from_acc<T>(acc)));
}

// The last hop of a block, fused with the gathers of X_{ell-1} and X_ell
// (ell = the block's last hop, Algorithm 2's hop and accumulation): X_ell is only read at each
// source and its neighbours, so only those values are computed, one warp per
// value, instead of the whole n x B block. One CTA per source; the values are
// those of a full hop (hop_value), so the result is bit for bit the one of
// k_spmm_hop followed by k_gather.
template <typename T, int B>
__global__ void __launch_bounds__(kSpmmWarps * 32) k_last_hop(const int32_t *__restrict__ row_ptr,
                                                              const int32_t *__restrict__ col,
                                                              const typename AccOf<T>::type *__restrict__ inv_deg,
                                                              const T *__restrict__ x_prev, int32_t n,
                                                              const int32_t *__restrict__ src, int32_t nsrc,
                                                              const int32_t *__restrict__ tau, int32_t ell,
                                                              double *__restrict__ g, double *__restrict__ t1,
                                                              double *__restrict__ t2, const GatherRec rec) {
    __shared__ double diag;
    const int32_t q = blockIdx.x;
    if (q >= nsrc) return;
    const int32_t s = src[q];
    if (s < 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t base;
    const T *xs = slice_column<T, B>(x_prev, n, nullptr, q, &base);
    // hop ell - 1 (as the fused gather of a full hop-ell launch would)
    gather_source<T, B>(row_ptr, col, xs, base, s, tau, ell - 1, g, t1, t2, threadIdx.x, blockDim.x, rec);
    if (warp == 0) {
        const double v = hop_value<T, B>(row_ptr, col, inv_deg, xs, base, s, lane);
        if (lane == 0) diag = v;
    }
    __syncthreads();  // also orders the hop ell - 1 updates before the hop ell ones
    const int32_t kb = row_ptr[s], ke = row_ptr[s + 1];
    for (int32_t k = kb + warp; k < ke; k += kSpmmWarps) {
        const double xj = hop_value<T, B>(row_ptr, col, inv_deg, xs, base, col[k], lane);
        if (lane == 0) gather_term(k, diag - xj, tau, ell, g, t1, t2, rec);
    }
}

// The same last hop in two launches, so that a source with many (or heavy)
// neighbours spreads over many CTAs: k_last_diag gathers X_{ell-1} and
// computes X_ell[s, b] (one CTA per source); k_last_rows computes X_ell at
// the neighbours, one warp per neighbour, over a (source, neighbour range)
// grid, and gathers hop ell.
template <typename T, int B>
__global__ void __launch_bounds__(kSpmmWarps * 32) k_last_diag(const int32_t *__restrict__ row_ptr,
                                                               const int32_t *__restrict__ col,
                                                               const typename AccOf<T>::type *__restrict__ inv_deg,
                                                               const T *__restrict__ x_prev, int32_t n,
                                                               const int32_t *__restrict__ src, int32_t nsrc,
                                                               const int32_t *__restrict__ tau, int32_t ell,
                                                               double *__restrict__ g, double *__restrict__ t1,
                                                               double *__restrict__ t2, const GatherRec rec,
                                                               double *__restrict__ diag) {
    const int32_t q = blockIdx.x;
    if (q >= nsrc) return;
    const int32_t s = src[q];
    if (s < 0) return;
    int32_t base;
    const T *xs = slice_column<T, B>(x_prev, n, nullptr, q, &base);
    gather_source<T, B>(row_ptr, col, xs, base, s, tau, ell - 1, g, t1, t2, threadIdx.x, blockDim.x, rec);
    if (threadIdx.x < 32) {
        const double v = hop_value<T, B>(row_ptr, col, inv_deg, xs, base, s, threadIdx.x);
        if (threadIdx.x == 0) diag[q] = v;
    }
}

template <typename T, int B>
__global__ void __launch_bounds__(kSpmmWarps * 32) k_last_rows(const int32_t *__restrict__ row_ptr,
                                                               const int32_t *__restrict__ col,
                                                               const typename AccOf<T>::type *__restrict__ inv_deg,
                                                               const T *__restrict__ x_prev, int32_t n,
                                                               const int32_t *__restrict__ src, int32_t nsrc,
                                                               const int32_t *__restrict__ tau, int32_t ell,
                                                               double *__restrict__ g, double *__restrict__ t1,
                                                               double *__restrict__ t2, const GatherRec rec,
                                                               const double *__restrict__ diag) {
    const int32_t q = blockIdx.x;
    if (q >= nsrc) return;
    const int32_t s = src[q];
    if (s < 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t base;
    const T *xs = slice_column<T, B>(x_prev, n, nullptr, q, &base);
    const int32_t ke = row_ptr[s + 1];
    for (int32_t k = row_ptr[s] + static_cast<int32_t>(blockIdx.y) * kSpmmWarps + warp; k < ke;
         k += static_cast<int32_t>(gridDim.y) * kSpmmWarps) {
        const double xj = hop_value<T, B>(row_ptr, col, inv_deg, xs, base, col[k], lane);
        if (lane == 0) gather_term(k, diag[q] - xj, tau, ell, g, t1, t2, rec);
    }
}

// rows one CTA of the SIMT hop kernel computes on the light path
template <typename T, int B, int VPL>
constexpr int light_rows_per_cta() {
    return kSpmmWarps * Layout<T, B, VPL>::G;
}

// light CTAs of a launch: enough for one row per group, at most kLightCtasPerSm
// per SM (each group then takes a few rows in turn)
constexpr int kLightCtasPerSm = 64;

inline int light_ctas_for(int64_t rows, int rows_per_cta, int num_sms) {
    const int64_t need = (rows + rows_per_cta - 1) / rows_per_cta;
    const int64_t cap = static_cast<int64_t>(num_sms > 0 ? num_sms : 148) * kLightCtasPerSm;
    return static_cast<int>(std::max<int64_t>(std::min(need, cap), 1));
}

// launch helper: one hop over `slices` slices, optionally gathering X_{l-1}.
// Unwindowed: the light rows are n - n_heavy. Windowed: win_heavy is the
// largest heavy-row count and win_rows the largest window of the slices.
template <typename T, int B, int VPL>
inline void launch_spmm_hop(HopArgs<T> a, int slices, cudaStream_t s, int num_sms, int win_heavy = 0,
                            int64_t win_rows = 0) {
    using L = Layout<T, B, VPL>;
    constexpr int rpc = kSpmmWarps * L::G;
    a.light_ctas = light_ctas_for(a.win ? win_rows : a.n, rpc, num_sms);
    a.gather_ctas = a.gather_ell > 0 ? B : 0;
    dim3 grid(a.gather_ctas + (a.win ? win_heavy : a.n_heavy) + a.light_ctas, slices);
    if (a.win) k_spmm_hop<T, B, VPL, true><<<grid, kSpmmWarps * 32, 0, s>>>(a);
    else k_spmm_hop<T, B, VPL, false><<<grid, kSpmmWarps * 32, 0, s>>>(a);
}

}  // namespace sc

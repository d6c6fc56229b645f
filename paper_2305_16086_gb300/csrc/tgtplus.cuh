// TGT+ (Algorithm 4) kernels: column statistics for CalChi (Alg. 3), the
// per-entry range chi (Eq. 17 / Eq. 15) and walk count R (Eq. 13), the
// switch rule (Eq. 14) and the random-walk tail (Eq. 11).
//
// Notation: X = p_tt(., s_b) for the sources s_b of a launch (the block after
// tt hops), L = tau_k - tt the walk length of entry k = (i -> j).
#pragma once

#include "philox.cuh"
#include "propagate.cuh"

namespace sc {

constexpr int kGammaMax = 16;        // largest supported candidate count (Alg. 3)
constexpr int kChiScanThreads = 128;
constexpr int kChiRowsPerCta = 64;
constexpr uint32_t kWalkTag = 0x57414C4Bu;
constexpr long long kWalkCountCap = 1ll << 40;

// strict total order of (value, node): larger value first, then smaller id
__device__ __forceinline__ bool better(double v, int32_t x, double w, int32_t y) {
    return v > w || (v == w && x < y);
}

// a := the kGammaMax best of the two sorted (descending) lists a and b; list
// element s of a sits at av[s * as] (strided, so that the lists of the threads
// of a warp interleave across shared-memory banks)
__device__ __forceinline__ void merge_sorted(double *av, int32_t *ai, int as, const double *bv, const int32_t *bi,
                                             int bs) {
    double ov[kGammaMax];
    int32_t oi[kGammaMax];
    int x = 0, y = 0;
#pragma unroll
    for (int s = 0; s < kGammaMax; ++s) {
        const double xa = av[x * as], yb = bv[y * bs];
        const int32_t ia = ai[x * as], ib = bi[y * bs];
        const bool ta = better(xa, ia, yb, ib);
        ov[s] = ta ? xa : yb;
        oi[s] = ta ? ia : ib;
        x += ta ? 1 : 0;
        y += ta ? 0 : 1;
    }
#pragma unroll
    for (int s = 0; s < kGammaMax; ++s) {
        av[s * as] = ov[s];
        ai[s * as] = oi[s];
    }
}

// Per CTA and column: the kGammaMax largest (value, node), min, max and the
// frontier volume sum_{x: X[x,b] != 0} d_x over kChiRowsPerCta rows.
// partial layout: [slice][cta][B] entries, lists of kGammaMax.
template <typename T, int B>
__global__ void __launch_bounds__(kChiScanThreads)
    k_chi_scan(const int32_t *__restrict__ row_ptr, const T *__restrict__ x, int32_t n, double *__restrict__ pval,
               int32_t *__restrict__ pid, double *__restrict__ pmin, double *__restrict__ pmax,
               long long *__restrict__ pvol) {
    constexpr int TPC = kChiScanThreads / B;  // threads per column
    constexpr int BATCH = 8;                 // rows in flight per thread
    const int c = threadIdx.x % B, sub = threadIdx.x / B;
    const int32_t r0 = blockIdx.x * kChiRowsPerCta;
    const int32_t r1 = min(n, r0 + kChiRowsPerCta);
    const T *xs = x + static_cast<int64_t>(blockIdx.y) * n * B;
    constexpr int NT = kChiScanThreads;  // list element s of thread t at [s * NT + t]
    __shared__ double sv[kGammaMax * NT];
    __shared__ int32_t si[kGammaMax * NT];
    __shared__ double smin[NT], smax[NT];
    __shared__ long long svol[NT];
    double *val = sv + threadIdx.x;
    int32_t *id = si + threadIdx.x;
    for (int s = 0; s < kGammaMax; ++s) {
        val[s * NT] = -INFINITY;
        id[s * NT] = INT32_MAX;
    }
    // the scan compares in the block's arithmetic type V (widening to double is
    // exact and order-preserving, so every decision is the one in double; this
    // keeps the FP64 units, slow on this GPU, out of the per-element loop)
    using V = typename AccOf<T>::type;
    V vmin = V(INFINITY), vmax = V(-INFINITY), thr = V(-INFINITY);  // thr: the list's last value
    long long vol = 0;
    for (int32_t rb = r0 + sub; rb < r1; rb += TPC * BATCH) {
        V v[BATCH];
        int32_t d[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int32_t r = rb + u * TPC;
            v[u] = r < r1 ? to_acc(xs[static_cast<int64_t>(r) * B + c]) : V(-INFINITY);
            d[u] = r < r1 ? row_ptr[r + 1] - row_ptr[r] : 0;
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int32_t r = rb + u * TPC;
            if (r < r1) {
                vmin = min(vmin, v[u]);
                vmax = max(vmax, v[u]);
                if (v[u] != V(0)) vol += d[u];
                // rows arrive in increasing order: a tie never beats the last slot
                if (v[u] > thr) {
                    double cv = static_cast<double>(v[u]);
                    int32_t ci = r;
#pragma unroll 1
                    for (int s = 0; s < kGammaMax; ++s) {
                        if (better(cv, ci, val[s * NT], id[s * NT])) {
                            const double tv = val[s * NT];
                            const int32_t ti = id[s * NT];
                            val[s * NT] = cv;
                            id[s * NT] = ci;
                            cv = tv;
                            ci = ti;
                        }
                    }
                    thr = static_cast<V>(val[(kGammaMax - 1) * NT]);  // exact: list values come from V
                }
            }
        }
    }
    smin[threadIdx.x] = static_cast<double>(vmin);
    smax[threadIdx.x] = static_cast<double>(vmax);
    svol[threadIdx.x] = vol;
    __syncthreads();
    for (int half = TPC / 2; half > 0; half >>= 1) {  // tree of sorted merges over the column's threads
        if (sub < half) {
            const int o = threadIdx.x + half * B;
            merge_sorted(val, id, NT, sv + o, si + o, NT);
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[o]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[o]);
            svol[threadIdx.x] += svol[o];
        }
        __syncthreads();
    }
    if (sub == 0) {
        const int64_t base = (static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x) * B + c;
        for (int s = 0; s < kGammaMax; ++s) {
            pval[base * kGammaMax + s] = val[s * NT];
            pid[base * kGammaMax + s] = id[s * NT];
        }
        pmin[base] = smin[threadIdx.x];
        pmax[base] = smax[threadIdx.x];
        pvol[base] = svol[threadIdx.x];
    }
}

// One CTA per column (slice * B + b): threads merge strided CTA partials, then
// a tree of sorted merges in shared memory. The order is total, so the result
// does not depend on the merge order.
template <int B>
__global__ void __launch_bounds__(kChiScanThreads)
    k_chi_merge(int nct, int ncols, const double *__restrict__ pval, const int32_t *__restrict__ pid,
                const double *__restrict__ pmin, const double *__restrict__ pmax,
                const long long *__restrict__ pvol, double *__restrict__ cval, int32_t *__restrict__ cid,
                double *__restrict__ cmin, double *__restrict__ cmax, long long *__restrict__ cvol) {
    const int q = blockIdx.x;
    if (q >= ncols) return;
    const int slice = q / B, c = q % B, t = threadIdx.x;
    constexpr int NT = kChiScanThreads;
    __shared__ double sv[kGammaMax * NT];
    __shared__ int32_t si[kGammaMax * NT];
    __shared__ double smin[NT], smax[NT];
    __shared__ long long svol[NT];
    double *val = sv + t;
    int32_t *id = si + t;
    for (int s = 0; s < kGammaMax; ++s) {
        val[s * NT] = -INFINITY;
        id[s * NT] = INT32_MAX;
    }
    double vmin = INFINITY, vmax = -INFINITY;
    long long vol = 0;
    double bv[kGammaMax];
    int32_t bi[kGammaMax];
    for (int p = t; p < nct; p += kChiScanThreads) {
        const int64_t base = (static_cast<int64_t>(slice) * nct + p) * B + c;
#pragma unroll
        for (int s = 0; s < kGammaMax; ++s) {
            bv[s] = pval[base * kGammaMax + s];
            bi[s] = pid[base * kGammaMax + s];
        }
        merge_sorted(val, id, NT, bv, bi, 1);
        vmin = fmin(vmin, pmin[base]);
        vmax = fmax(vmax, pmax[base]);
        vol += pvol[base];
    }
    smin[t] = vmin;
    smax[t] = vmax;
    svol[t] = vol;
    __syncthreads();
    for (int half = kChiScanThreads / 2; half > 0; half >>= 1) {
        if (t < half) {
            merge_sorted(val, id, NT, sv + t + half, si + t + half, NT);
            smin[t] = fmin(smin[t], smin[t + half]);
            smax[t] = fmax(smax[t], smax[t + half]);
            svol[t] += svol[t + half];
        }
        __syncthreads();
    }
    if (t == 0) {
        for (int s = 0; s < kGammaMax; ++s) {
            cval[static_cast<int64_t>(q) * kGammaMax + s] = val[s * NT];
            cid[static_cast<int64_t>(q) * kGammaMax + s] = id[s * NT];
        }
        cmin[q] = smin[0];
        cmax[q] = smax[0];
        cvol[q] = svol[0];
    }
}

// ---------------------------------------------------------------------------
// Threshold form of the same column statistics (the default): the top-gamma
// list of a column needs only the entries at or above thr = the gamma-th
// largest of its tile maxima (tiles of kTileRows rows). The gamma tiles with
// the largest maxima hold gamma entries >= thr, so the gamma-th largest entry
// is >= thr, and every entry of the top-gamma list lies in a tile whose
// maximum reaches thr. Three launches: tile maxima, minima and volumes
// (k_chi_tiles); per column thr, min, max and volume (k_chi_thresh); per
// column the entries >= thr of the tiles reaching it, and the top-gamma list
// among them in the total order (k_chi_select). thr = 0 (fewer than gamma
// tiles hold a positive entry) takes the positive entries of those tiles and
// the gamma smallest-id zero rows (the ties at 0 go to smaller ids). A column
// with more than kCandMax candidates (many ties at thr) is scanned in full.
// The first gamma entries of each list equal the full scan's; entries past
// gamma are not read.
// ---------------------------------------------------------------------------
constexpr int kTileRows = 256;
constexpr int kCandMax = 2048;

// a 16-byte vector of stored values as accumulator-type elements, in memory order
__device__ __forceinline__ void unpack16(const uint4 &v, float (&a)[4]) {
    a[0] = __uint_as_float(v.x);
    a[1] = __uint_as_float(v.y);
    a[2] = __uint_as_float(v.z);
    a[3] = __uint_as_float(v.w);
}
__device__ __forceinline__ void unpack16(const uint4 &v, double (&a)[2]) {
    a[0] = __hiloint2double(static_cast<int>(v.y), static_cast<int>(v.x));
    a[1] = __hiloint2double(static_cast<int>(v.w), static_cast<int>(v.z));
}
__device__ __forceinline__ void unpack16(const uint4 &v, float (&a)[8]) {  // bf16 pairs, low half first
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        a[2 * q] = __uint_as_float(w[q] << 16);
        a[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
    }
}

// Per tile of kTileRows rows and column: maximum, minimum and frontier volume
// (sum of d_x over the rows with X[x, c] != 0). Rows are read as 16-byte
// vectors: LG lanes cover a row (VPL vectors each), a warp reads 32 / LG rows
// per load and keeps UR such loads in flight; the lanes holding the same
// columns are combined by shuffles, the warps through shared memory. Maxima,
// minima and integer sums do not depend on the order of combination.
template <typename T, int B>
__global__ void __launch_bounds__(kChiScanThreads)
    k_chi_tiles(const int32_t *__restrict__ row_ptr, const T *__restrict__ x, int32_t n, double *__restrict__ tmax,
                double *__restrict__ tmin, long long *__restrict__ tvol) {
    using V = typename AccOf<T>::type;
    constexpr int E = 16 / static_cast<int>(sizeof(T));  // elements per 16-byte vector
    constexpr int NV = B / E;                            // vectors per row
    constexpr int LG = NV < 32 ? NV : 32;                // lanes per row
    constexpr int VPL = NV / LG;                         // vectors per lane
    constexpr int RPW = 32 / LG;                         // rows per warp load
    constexpr int NW = kChiScanThreads / 32;
    constexpr int UR = 8 / VPL;                          // row loads in flight per lane
    constexpr int C = VPL * E;                           // columns per lane
    static_assert(NV % LG == 0 && 32 % LG == 0, "row layout");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % LG, rsub = lane / LG;
    const int32_t r0 = blockIdx.x * kTileRows, r1 = min(n, r0 + kTileRows);
    const uint4 *xs = reinterpret_cast<const uint4 *>(x + static_cast<int64_t>(blockIdx.y) * n * B);
    V vmax[C], vmin[C];
    long long vol[C];
#pragma unroll
    for (int e = 0; e < C; ++e) {
        vmax[e] = V(-INFINITY);
        vmin[e] = V(INFINITY);
        vol[e] = 0;
    }
    constexpr int STEP = NW * RPW;  // rows per round of the CTA's warps
    for (int32_t rb = r0 + warp * RPW + rsub; rb < r1; rb += STEP * UR) {
        uint4 v[UR][VPL];
        int32_t d[UR];
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            const int32_t r = rb + u * STEP;
            const bool in = r < r1;
            d[u] = in ? row_ptr[r + 1] - row_ptr[r] : 0;
#pragma unroll
            for (int p = 0; p < VPL; ++p)
                v[u][p] = in ? __ldg(xs + static_cast<int64_t>(r) * NV + gl + p * LG) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            if (rb + u * STEP >= r1) continue;
#pragma unroll
            for (int p = 0; p < VPL; ++p) {
                V a[E];
                unpack16(v[u][p], a);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k = p * E + e;
                    vmax[k] = max(vmax[k], a[e]);
                    vmin[k] = min(vmin[k], a[e]);
                    if (a[e] != V(0)) vol[k] += d[u];
                }
            }
        }
    }
    // lanes rsub = 0 .. RPW-1 hold the same columns: combine them
#pragma unroll
    for (int o = LG; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            vmax[k] = max(vmax[k], __shfl_xor_sync(0xffffffffu, vmax[k], o));
            vmin[k] = min(vmin[k], __shfl_xor_sync(0xffffffffu, vmin[k], o));
            vol[k] += __shfl_xor_sync(0xffffffffu, vol[k], o);
        }
    }
    __shared__ double smax[NW][B], smin[NW][B];
    __shared__ long long svol[NW][B];
    if (rsub == 0) {
#pragma unroll
        for (int p = 0; p < VPL; ++p)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int c = (gl + p * LG) * E + e;
                smax[warp][c] = static_cast<double>(vmax[p * E + e]);
                smin[warp][c] = static_cast<double>(vmin[p * E + e]);
                svol[warp][c] = vol[p * E + e];
            }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < B; c += kChiScanThreads) {
        double a = smax[0][c], b = smin[0][c];
        long long w = svol[0][c];
#pragma unroll
        for (int q = 1; q < NW; ++q) {
            a = fmax(a, smax[q][c]);
            b = fmin(b, smin[q][c]);
            w += svol[q][c];
        }
        const int64_t o = (static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x) * B + c;
        tmax[o] = a;
        tmin[o] = b;
        tvol[o] = w;
    }
}

// per column q = slice * B + b: thr, min, max and volume. One CTA per
// column; thread t takes tiles t, t + 128, ... and keeps their largest
// maximum. thr = the gamma-th largest of those 128 maxima (0 if fewer than
// gamma are positive): they are maxima of distinct tiles, so at least gamma
// tiles reach thr, every top-gamma entry is >= thr, and thr is at most the
// gamma-th largest tile maximum (a few more candidate tiles than that, no
// merge of sorted lists).
template <int B>
__global__ void __launch_bounds__(kChiScanThreads)
    k_chi_thresh(int ntiles, int ncols, int gamma, const double *__restrict__ tmax, const double *__restrict__ tmin,
                 const long long *__restrict__ tvol, double *__restrict__ cthr, double *__restrict__ cmin,
                 double *__restrict__ cmax, long long *__restrict__ cvol) {
    const int q = blockIdx.x;
    if (q >= ncols) return;
    const int slice = q / B, c = q % B, t = threadIdx.x;
    constexpr int NT = kChiScanThreads;
    __shared__ double smax[NT], smin[NT];
    __shared__ long long svol[NT];
    double vmax = -INFINITY, vmin = INFINITY;
    long long vol = 0;
    for (int p = t; p < ntiles; p += NT) {
        const int64_t o = (static_cast<int64_t>(slice) * ntiles + p) * B + c;
        vmax = fmax(vmax, tmax[o]);
        vmin = fmin(vmin, tmin[o]);
        vol += tvol[o];
    }
    smax[t] = vmax;
    smin[t] = vmin;
    svol[t] = vol;
    __syncthreads();
    // rank of each thread's maximum among the 128 (ties by thread index); rank gamma - 1 is thr
    int rank = 0;
    for (int u = 0; u < NT; ++u) rank += (smax[u] > vmax || (smax[u] == vmax && u < t)) ? 1 : 0;
    if (gamma > 0 && rank == gamma - 1) cthr[q] = vmax > 0.0 ? vmax : 0.0;
    if (rank == 0) cmax[q] = vmax;
    __syncthreads();
    for (int half = NT / 2; half > 0; half >>= 1) {
        if (t < half) {
            smin[t] = fmin(smin[t], smin[t + half]);
            svol[t] += svol[t + half];
        }
        __syncthreads();
    }
    if (t == 0) {
        cmin[q] = smin[0];
        cvol[q] = svol[0];
        if (gamma > NT || gamma <= 0) cthr[q] = 0.0;  // (gamma <= kGammaMax < NT on the product path)
    }
}

// per column: the candidates (entries >= thr in the tiles whose maximum
// reaches thr; for thr = 0 the positive entries of the tiles holding one, and
// the gamma smallest-id zero rows), then the top-kGammaMax list among them.
template <typename T, int B>
__global__ void __launch_bounds__(kChiScanThreads)
    k_chi_select(int32_t n, int ntiles, int ncols, int gamma, const T *__restrict__ x, const double *__restrict__ tmax,
                 const double *__restrict__ tmin, const double *__restrict__ cthr, double *__restrict__ cval,
                 int32_t *__restrict__ cid) {
    using V = typename AccOf<T>::type;
    const int q = blockIdx.x;
    if (q >= ncols || gamma <= 0) return;
    const int slice = q / B, c = q % B, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NT = kChiScanThreads, NW = kChiScanThreads / 32;
    const T *xs = x + static_cast<int64_t>(slice) * n * B + c;
    const double thr = cthr[q];
    const bool zero_thr = !(thr > 0.0);
    __shared__ double cand_v[kCandMax];
    __shared__ int32_t cand_i[kCandMax];
    __shared__ int ncand;
    __shared__ double sv[kGammaMax * NT];
    __shared__ int32_t si[kGammaMax * NT];
    if (t == 0) ncand = 0;
    __syncthreads();
    // candidates: each warp tests 32 tile maxima at once, then takes the tiles that reach thr
    // one by one, 32 rows at a time
    for (int pb = warp * 32; pb < ntiles; pb += NW * 32) {
        const int pl = pb + lane;
        const double tml = pl < ntiles ? tmax[(static_cast<int64_t>(slice) * ntiles + pl) * B + c] : -1.0;
        uint32_t tiles = __ballot_sync(0xffffffffu, zero_thr ? (tml > 0.0) : (tml >= thr));
        while (tiles) {  // warp-uniform
            const int p = pb + __ffs(tiles) - 1;
            tiles &= tiles - 1u;
            const int32_t r0 = p * kTileRows, r1 = min(n, r0 + kTileRows);
            constexpr int RR = kTileRows / 32;  // the tile's rows, 32 per round, loaded together
            double vals[RR];
#pragma unroll
            for (int u = 0; u < RR; ++u) {
                const int32_t r = r0 + u * 32 + lane;
                vals[u] = r < r1 ? static_cast<double>(to_acc(xs[static_cast<int64_t>(r) * B])) : -1.0;
            }
#pragma unroll
            for (int u = 0; u < RR; ++u) {
                const int32_t r = r0 + u * 32 + lane;
                const double v = vals[u];
                const bool take = zero_thr ? (v > 0.0) : (v >= thr);
                const uint32_t bal = __ballot_sync(0xffffffffu, take);
                int base = 0;
                if (lane == 0 && bal) base = atomicAdd(&ncand, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (take) {
                    const int slot = base + __popc(bal & ((1u << lane) - 1u));
                    if (slot < kCandMax) {
                        cand_v[slot] = v;
                        cand_i[slot] = r;
                    }
                }
            }
        }
    }
    __syncthreads();
    if (zero_thr && warp == 0) {
        // the gamma smallest-id zero rows, in id order
        int need = gamma;
        for (int p = 0; p < ntiles && need > 0; ++p) {
            if (tmin[(static_cast<int64_t>(slice) * ntiles + p) * B + c] > 0.0) continue;
            const int32_t r0 = p * kTileRows, r1 = min(n, r0 + kTileRows);
            for (int32_t rb = r0; rb < r1 && need > 0; rb += 32) {
                const int32_t r = rb + lane;
                const bool z = r < r1 && to_acc(xs[static_cast<int64_t>(r) * B]) == V(0);
                uint32_t bal = __ballot_sync(0xffffffffu, z);
                int base = 0;
                while (bal && need > 0) {  // warp-uniform
                    const int l = __ffs(bal) - 1;
                    bal &= bal - 1u;
                    if (lane == 0) {
                        base = ncand;
                        if (base < kCandMax) {
                            cand_v[base] = 0.0;
                            cand_i[base] = rb + l;
                        }
                        ncand = base + 1;
                    }
                    --need;
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    double *val = sv + t;
    int32_t *id = si + t;
    for (int s = 0; s < kGammaMax; ++s) {
        val[s * NT] = -INFINITY;
        id[s * NT] = INT32_MAX;
    }
    double bv[kGammaMax];
    int32_t bi[kGammaMax];
#pragma unroll
    for (int s = 1; s < kGammaMax; ++s) {
        bv[s] = -INFINITY;
        bi[s] = INT32_MAX;
    }
    const int count = ncand;
    if (count <= kCandMax) {
        for (int e = t; e < count; e += NT) {
            bv[0] = cand_v[e];
            bi[0] = cand_i[e];
            merge_sorted(val, id, NT, bv, bi, 1);
        }
    } else {
        // too many ties at thr for the buffer: every row of the column
        for (int32_t r = t; r < n; r += NT) {
            bv[0] = static_cast<double>(to_acc(xs[static_cast<int64_t>(r) * B]));
            bi[0] = r;
            merge_sorted(val, id, NT, bv, bi, 1);
        }
    }
    __syncthreads();
    for (int half = NT / 2; half > 0; half >>= 1) {
        if (t < half) merge_sorted(val, id, NT, sv + t + half, si + t + half, NT);
        __syncthreads();
    }
    if (t == 0)
        for (int s = 0; s < kGammaMax; ++s) {
            cval[static_cast<int64_t>(q) * kGammaMax + s] = sv[s * NT];
            cid[static_cast<int64_t>(q) * kGammaMax + s] = si[s * NT];
        }
}

__device__ __forceinline__ bool has_edge(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                         int32_t a, int32_t b) {
    int32_t lo = row_ptr[a], hi = row_ptr[a + 1];
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        const int32_t c = col[mid];
        if (c == b) return true;
        if (c < b) lo = mid + 1;
        else hi = mid;
    }
    return false;
}

struct ChiArgs {
    const int32_t *row_ptr, *col, *src, *tau;
    int32_t n, nsrc, ell, gamma;
    const double *cval, *cmin, *cmax;
    const int32_t *cid;
    double eps, log_2m_delta;
    long long *walk_count;   // per CSR entry (0 = no walks)
    long long *rhs;          // [0] sum of the launch's walk counts (Eq. 14 right side), [2] walk steps
};

// Per source (one warp): rho_hat (Alg. 3) and min / max of p over N(i),
// into stat[3 q .. 3 q + 2].
template <typename T, int B>
__global__ void k_chi_source(const T *__restrict__ x, const ChiArgs a, double *__restrict__ stat) {
    const int32_t q = blockIdx.x;
    const int lane = threadIdx.x & 31;
    if (q >= a.nsrc) return;
    const int32_t s = a.src[q];
    if (s < 0) return;
    const T *xs = x + static_cast<int64_t>(q / B) * a.n * B + (q % B);
    auto px = [&](int32_t v) { return static_cast<double>(to_acc(xs[static_cast<int64_t>(v) * B])); };
    const double *cv = a.cval + static_cast<int64_t>(q) * kGammaMax;
    const int32_t *ci = a.cid + static_cast<int64_t>(q) * kGammaMax;
    const int g = a.gamma;
    // rho_hat = max(max over edges inside C of p(c_a) + p(c_b), p(c_1) + p(c_gamma))
    double best = -INFINITY;
    if (g > 0) {
        for (int t = lane; t < g * g; t += 32) {
            const int u = t / g, v = t % g;
            if (u < v && has_edge(a.row_ptr, a.col, ci[u], ci[v])) best = fmax(best, __dadd_rn(cv[u], cv[v]));
        }
    }
    double nmin = INFINITY, nmax = -INFINITY;
    for (int32_t k = a.row_ptr[s] + lane; k < a.row_ptr[s + 1]; k += 32) {
        const double v = px(a.col[k]);
        nmin = fmin(nmin, v);
        nmax = fmax(nmax, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
        nmin = fmin(nmin, __shfl_xor_sync(0xffffffffu, nmin, o));
        nmax = fmax(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    }
    if (lane == 0) {
        stat[3 * q] = g > 0 ? fmax(best, __dadd_rn(cv[0], cv[g - 1])) : 0.0;
        stat[3 * q + 1] = nmin;
        stat[3 * q + 2] = nmax;
    }
}

// Per entry k = (i -> j) of source q = blockIdx.x, one warp each over a
// (source, entry range) grid so that a hub source spreads over many CTAs:
// the lanes stride over N(j) for chi (Eq. 17, or Eq. 15 for gamma = 0), then
// R (Eq. 13) for the walk length L = tau_k - ell. The floating-point
// expressions follow the oracle's evaluation order (no FMA contraction).
template <typename T, int B>
__global__ void k_chi_entries(const T *__restrict__ x, const ChiArgs a, const double *__restrict__ stat) {
    const int32_t q = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (q >= a.nsrc) return;
    const int32_t s = a.src[q];
    if (s < 0) return;
    const T *xs = x + static_cast<int64_t>(q / B) * a.n * B + (q % B);
    auto px = [&](int32_t v) { return static_cast<double>(to_acc(xs[static_cast<int64_t>(v) * B])); };
    const double vmin = a.cmin[q], vmax = a.cmax[q];
    const int g = a.gamma;
    const int32_t rb = a.row_ptr[s], re = a.row_ptr[s + 1];
    __shared__ unsigned long long sh_cnt[2];
    if (threadIdx.x == 0) {
        sh_cnt[0] = 0;
        sh_cnt[1] = 0;
    }
    __syncthreads();
    const double rho = stat[3 * q], nmin_i = stat[3 * q + 1], nmax_i = stat[3 * q + 2];
    const double d_i = static_cast<double>(re - rb);
    const double denom = __dmul_rn(__dmul_rn(__dmul_rn(d_i, d_i), a.eps), a.eps);
    unsigned long long local = 0, steps = 0;
    for (int32_t k = rb + static_cast<int32_t>(blockIdx.y) * nw + warp; k < re;
         k += static_cast<int32_t>(gridDim.y) * nw) {
        const int32_t L = a.tau[k] - a.ell;
        if (L <= 0) {
            if (lane == 0) a.walk_count[k] = 0;
            continue;
        }
        const int32_t j = a.col[k];
        double chi;
        if (g == 0) {
            chi = __dmul_rn(__dmul_rn(2.0, static_cast<double>(L)), __dsub_rn(vmax, vmin));  // Eq. 15
        } else {
            double nmin_j = INFINITY, nmax_j = -INFINITY;
            for (int32_t e = a.row_ptr[j] + lane; e < a.row_ptr[j + 1]; e += 32) {
                const double v = px(a.col[e]);
                nmin_j = fmin(nmin_j, v);
                nmax_j = fmax(nmax_j, v);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                nmin_j = fmin(nmin_j, __shfl_xor_sync(0xffffffffu, nmin_j, o));
                nmax_j = fmax(nmax_j, __shfl_xor_sync(0xffffffffu, nmax_j, o));
            }
            const double Lm1 = static_cast<double>(L - 1);
            const double lb_i = __dadd_rn(nmin_i, __dmul_rn(Lm1, vmin));
            const double lb_j = __dadd_rn(nmin_j, __dmul_rn(Lm1, vmin));
            const double tail = __ddiv_rn(__dmul_rn(Lm1, rho), 2.0);
            const double ub_i = __dadd_rn(__dadd_rn(__ddiv_rn(nmax_i, 2.0), __ddiv_rn(vmax, 2.0)), tail);
            const double ub_j = __dadd_rn(__dadd_rn(__ddiv_rn(nmax_j, 2.0), __ddiv_rn(vmax, 2.0)), tail);
            chi = __dsub_rn(__dsub_rn(__dadd_rn(ub_i, ub_j), lb_i), lb_j);  // Eq. 17
        }
        const double r = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(8.0, chi), chi), a.log_2m_delta), denom);
        const double rc = ceil(r);
        const long long R =
            rc < 1.0 ? 1 : (rc > static_cast<double>(kWalkCountCap) ? kWalkCountCap : static_cast<long long>(rc));
        if (lane == 0) {
            a.walk_count[k] = R;
            local += static_cast<unsigned long long>(R);
            steps += static_cast<unsigned long long>(R) * 2ull * static_cast<unsigned long long>(L);
        }
    }
    if (lane == 0 && local) {
        atomicAdd(&sh_cnt[0], local);
        atomicAdd(&sh_cnt[1], steps);
    }
    __syncthreads();
    if (threadIdx.x == 0 && sh_cnt[0]) {
        atomicAdd(reinterpret_cast<unsigned long long *>(a.rhs), sh_cnt[0]);
        atomicAdd(reinterpret_cast<unsigned long long *>(a.rhs + 2), sh_cnt[1]);
    }
}

struct WalkArgs {
    const int32_t *row_ptr, *col, *src, *tau;
    int32_t n, nsrc, tt;
    const long long *walk_count;
    double *g;             // unscaled half sums; the walk mean of X d_i is added
    uint32_t key0, key1;
};

// sum_{t=1..L} X[W[t]] for walk w of entry k on one side (Eq. 11)
template <typename T, int B>
__device__ __forceinline__ double walk_sum(const WalkArgs &a, const T *__restrict__ xs, int32_t start, int32_t L,
                                           uint32_t k, uint32_t w, uint32_t side) {
    int32_t cur = start;
    double sum = 0.0;
    Philox4 words{};
    for (int32_t t = 1; t <= L; ++t) {
        const int r = (t - 1) & 3;
        if (r == 0)
            words = philox4x32_10(k, w, (side << 31) | static_cast<uint32_t>((t - 1) >> 2), kWalkTag, a.key0, a.key1);
        const int32_t b = a.row_ptr[cur];
        const uint32_t d = static_cast<uint32_t>(a.row_ptr[cur + 1] - b);
        const uint32_t idx = static_cast<uint32_t>((static_cast<uint64_t>(words.v[r]) * d) >> 32);
        cur = a.col[b + idx];
        sum += static_cast<double>(to_acc(xs[static_cast<int64_t>(cur) * B]));
    }
    return sum;
}

constexpr int kWalkChunk = 128;  // walk pairs per warp-sized chunk

struct WalkChunkArgs {
    const int32_t *entry_q;     // per planned entry: launch source index q
    const int32_t *entry_k;     // per planned entry: CSR entry k
    const int32_t *chunk_entry; // per chunk: planned entry index
    const long long *chunk_w0;  // per chunk: first walk index
    int32_t nchunks;
    double *chunk_sum;          // per chunk: sum over its walks of (S_i - S_j)
};

// One warp per chunk of walk pairs of one entry; lanes take walks w0 + lane,
// w0 + lane + 32, ... in the chunk; the chunk sum is reduced by a fixed tree.
template <typename T, int B>
__global__ void k_walk_chunks(const T *__restrict__ x, const WalkArgs a, const WalkChunkArgs c) {
    const int32_t ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (ch >= c.nchunks) return;
    const int32_t e = c.chunk_entry[ch];
    const int32_t q = c.entry_q[e], k = c.entry_k[e];
    const int32_t s = a.src[q];
    const T *xs = x + static_cast<int64_t>(q / B) * a.n * B + (q % B);
    const long long R = a.walk_count[k];
    const long long w0 = c.chunk_w0[ch];
    const long long w1 = min(R, w0 + kWalkChunk);
    const int32_t L = a.tau[k] - a.tt;
    const int32_t j = a.col[k];
    double acc = 0.0;
    for (long long w = w0 + lane; w < w1; w += 32) {
        const double si = walk_sum<T, B>(a, xs, s, L, static_cast<uint32_t>(k), static_cast<uint32_t>(w), 0u);
        const double sj = walk_sum<T, B>(a, xs, j, L, static_cast<uint32_t>(k), static_cast<uint32_t>(w), 1u);
        acc += si - sj;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) c.chunk_sum[ch] = acc;
}

// g[k] += (sum of the entry's chunk sums, in chunk order) / R_k  (Algorithm 4's walk estimate)
static __global__ void k_walk_finish(const int32_t *__restrict__ entry_k, const int32_t *__restrict__ entry_chunk0,
                              int32_t nentries, const double *__restrict__ chunk_sum,
                              const long long *__restrict__ walk_count, double *__restrict__ g) {
    const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nentries) return;
    const int32_t k = entry_k[e];
    const long long R = walk_count[k];
    if (R <= 0) return;
    double t = 0.0;
    for (int32_t ch = entry_chunk0[e]; ch < entry_chunk0[e + 1]; ++ch) t += chunk_sum[ch];
    g[k] += t / static_cast<double>(R);
}

// Eq. 14's right side for one source: out[q] = the sum of the walk counts of
// source q's entries (one warp per source; 0 for an empty slot)
static __global__ void k_walks_per_source(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ src,
                                          int32_t nsrc, const long long *__restrict__ walk_count,
                                          long long *__restrict__ out) {
    const int32_t q = blockIdx.x;
    const int lane = threadIdx.x & 31;
    if (q >= nsrc) return;
    const int32_t s = src[q];
    long long acc = 0;
    if (s >= 0)
        for (int32_t k = row_ptr[s] + lane; k < row_ptr[s + 1]; k += 32) acc += walk_count[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[q] = acc;
}

// tau[k] = min(tau[k], cap) over the rows of the listed nodes (entries < 0
// skipped): a source that switched to walks at hop cap gathers no later hop
static __global__ void k_cap_rows(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ list,
                                  int32_t count, int32_t cap, int32_t *__restrict__ tau) {
    const int32_t q = blockIdx.x;
    if (q >= count) return;
    const int32_t v = list[q];
    if (v < 0) return;
    for (int32_t k = row_ptr[v] + static_cast<int32_t>(threadIdx.x); k < row_ptr[v + 1]; k += blockDim.x)
        tau[k] = min(tau[k], cap);
}

// out[e] = R of planned entry e; out[nentries + e] = its walk steps 2 R (tau_k - tt)
static __global__ void k_pack_counts(const int32_t *__restrict__ entry_k, int32_t nentries,
                                     const long long *__restrict__ walk_count, const int32_t *__restrict__ tau,
                                     int32_t tt, long long *__restrict__ out) {
    const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nentries) return;
    const int32_t k = entry_k[e];
    const long long R = walk_count[k];
    const int32_t L = tau[k] - tt;
    out[e] = R;
    out[nentries + e] = (R > 0 && L > 0) ? 2ll * R * static_cast<long long>(L) : 0ll;
}

}  // namespace sc

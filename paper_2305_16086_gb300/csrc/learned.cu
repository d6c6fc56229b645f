// Learned per-source truncation length (step A8): per-source features, a
// 6 -> 32 -> 32 -> 1 ReLU MLP trained on the GPU (forward, backward with
// deterministic reductions, Adam), and inference of the per-source lengths.
//
// The paper has no learned part. The length it predicts only sets where the
// traversal of Algorithm 2 stops; sc_all_edges then certifies every edge with
// the a-posteriori bound lambda*^2/(1-lambda*^2) (t_{tau-1} + t_tau) (from the
// mode expansion in the proof of Theorem 3.2) and extends the edges that fail,
// up to the a-priori length of Eq. (6), so the eps guarantee does not depend
// on the model. A bipartite graph (lambda* = 1) has neither: there the labels
// and the acceptance come from the power-law tail estimate of the
// end-corrected series (sc_estimated_lengths), an estimate, not a bound.
//
// Features of source i, all local and independent of the graph's size (a
// model trained on a smaller graph of a family serves a larger one): log d_i;
// log min_{j in N(i)} d_j; local clustering; log of the mean neighbour degree
// over the mean degree, log((sum_{j in N(i)} d_j / d_i) / (2m / n));
// p_2(i,i) = (1/d_i) sum_{j in N(i)} 1/d_j; p_3(i,i) = (1/d_i) sum over the
// triangles (i, j, k) of 1/(d_j d_k). Flat parameters (float): W1[32][6],
// b1[32], W2[32][32], b2[32], W3[32], b3; the model adds the features' mean
// and standard deviation used to standardise the inputs.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace sc {

void certified_lengths_impl(sc_graph *g, double eps, int precision, int32_t *per_entry_dev, int32_t *cap_out);
void estimated_lengths_impl(sc_graph *g, double eps, int precision, int32_t cap, int32_t *per_entry_dev);

constexpr int kH = SC_MLP_HIDDEN;
constexpr int kF = SC_MLP_FEATURES;
constexpr int kP = SC_MLP_PARAMS;
constexpr int oW1 = 0, oB1 = kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
static_assert(oB3 + 1 == kP, "parameter layout");
constexpr int kMlpSamples = 128;  // samples per CTA of the gradient kernel

// ---------------------------------------------------------------------------
// features (one warp per node)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool contains(const int32_t *__restrict__ col, int32_t lo, int32_t hi, int32_t v) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        const int32_t c = col[mid];
        if (c == v) return true;
        if (c < v) lo = mid + 1;
        else hi = mid;
    }
    return false;
}

__global__ void k_features(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                           double mean_deg, float *__restrict__ out) {
    const int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int32_t ib = row_ptr[i], ie = row_ptr[i + 1];
    const double d = static_cast<double>(ie - ib);
    int32_t dmin = INT32_MAX;
    long long vol = 0, tri2 = 0;
    double inv_sum = 0.0, cyc3 = 0.0;
    for (int32_t k = ib + lane; k < ie; k += 32) {
        const int32_t j = col[k];
        const int32_t jb = row_ptr[j], je = row_ptr[j + 1];
        const int32_t dj = je - jb;
        dmin = min(dmin, dj);
        vol += dj;
        inv_sum += 1.0 / static_cast<double>(dj);
        // the common neighbours x of i and j: walk the shorter list, search the longer one;
        // each closes the triangle (i, j, x), which adds 1 / (d_j d_x) to p_3(i,i) d_i
        const bool walk_j = dj <= ie - ib;
        const int32_t wb = walk_j ? jb : ib, we = walk_j ? je : ie;
        const int32_t sb = walk_j ? ib : jb, se = walk_j ? ie : je;
        for (int32_t e = wb; e < we; ++e) {
            const int32_t x = col[e];
            if (contains(col, sb, se, x)) {
                ++tri2;
                cyc3 += 1.0 / (static_cast<double>(dj) * static_cast<double>(row_ptr[x + 1] - row_ptr[x]));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
        vol += __shfl_xor_sync(0xffffffffu, vol, o);
        tri2 += __shfl_xor_sync(0xffffffffu, tri2, o);
        inv_sum += __shfl_xor_sync(0xffffffffu, inv_sum, o);
        cyc3 += __shfl_xor_sync(0xffffffffu, cyc3, o);
    }
    if (lane == 0) {
        float *f = out + static_cast<int64_t>(i) * kF;
        f[0] = static_cast<float>(log(d));
        f[1] = static_cast<float>(log(static_cast<double>(dmin)));
        f[2] = d >= 2.0 ? static_cast<float>((static_cast<double>(tri2) / 2.0) / (d * (d - 1.0) / 2.0)) : 0.0f;
        f[3] = static_cast<float>(log(static_cast<double>(vol) / d / mean_deg));
        f[4] = static_cast<float>(inv_sum / d);
        f[5] = static_cast<float>(cyc3 / d);
    }
}

// ---------------------------------------------------------------------------
// MLP
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mlp_forward(const float *__restrict__ w, const float *x, float *z1, float *h1,
                                             float *z2, float *h2) {
#pragma unroll 4
    for (int a = 0; a < kH; ++a) {
        float acc = w[oB1 + a];
#pragma unroll
        for (int f = 0; f < kF; ++f) acc = fmaf(w[oW1 + a * kF + f], x[f], acc);
        z1[a] = acc;
        h1[a] = fmaxf(acc, 0.0f);
    }
#pragma unroll 4
    for (int a = 0; a < kH; ++a) {
        float acc = w[oB2 + a];
        for (int b = 0; b < kH; ++b) acc = fmaf(w[oW2 + a * kH + b], h1[b], acc);
        z2[a] = acc;
        h2[a] = fmaxf(acc, 0.0f);
    }
    float y = w[oB3];
    for (int a = 0; a < kH; ++a) y = fmaf(w[oW3 + a], h2[a], y);
    return y;
}

// One CTA of kMlpSamples samples: per-sample forward and backward into shared
// memory, then each thread sums its parameters' gradients over the CTA's
// samples in sample order. partial[cta][p] for p < kP, partial[cta][kP] = loss sum.
__global__ void __launch_bounds__(kMlpSamples) k_mlp_grad_partial(const float *__restrict__ params,
                                                                   const float *__restrict__ X,
                                                                   const float *__restrict__ target, int32_t N,
                                                                   float *__restrict__ partial) {
    extern __shared__ float sm[];
    float *w = sm;                          // kP (padded to kP + 3)
    float *sx = w + kP + 3;                 // [kF][S]
    float *sh1 = sx + kF * kMlpSamples;     // [kH][S]
    float *sd1 = sh1 + kH * kMlpSamples;    // [kH][S]
    float *sh2 = sd1 + kH * kMlpSamples;    // [kH][S]
    float *sd2 = sh2 + kH * kMlpSamples;    // [kH][S]
    float *sdy = sd2 + kH * kMlpSamples;    // [S]
    float *sl = sdy + kMlpSamples;          // [S]
    const int t = threadIdx.x;
    for (int p = t; p < kP; p += kMlpSamples) w[p] = params[p];
    __syncthreads();
    const int64_t smp = static_cast<int64_t>(blockIdx.x) * kMlpSamples + t;
    float x[kF], z1[kH], h1[kH], z2[kH], h2[kH];
    if (smp < N) {
#pragma unroll
        for (int f = 0; f < kF; ++f) x[f] = X[smp * kF + f];
        const float y = mlp_forward(w, x, z1, h1, z2, h2);
        const float r = y - target[smp];
        const float dy = r / static_cast<float>(N);
        sl[t] = 0.5f * r * r;
        sdy[t] = dy;
        float d2[kH];
        for (int a = 0; a < kH; ++a) d2[a] = z2[a] > 0.0f ? dy * w[oW3 + a] : 0.0f;
        for (int b = 0; b < kH; ++b) {
            float acc = 0.0f;
            for (int a = 0; a < kH; ++a) acc = fmaf(d2[a], w[oW2 + a * kH + b], acc);
            sd1[b * kMlpSamples + t] = z1[b] > 0.0f ? acc : 0.0f;
            sh1[b * kMlpSamples + t] = h1[b];
        }
        for (int a = 0; a < kH; ++a) {
            sd2[a * kMlpSamples + t] = d2[a];
            sh2[a * kMlpSamples + t] = h2[a];
        }
#pragma unroll
        for (int f = 0; f < kF; ++f) sx[f * kMlpSamples + t] = x[f];
    } else {
        sl[t] = 0.0f;
        sdy[t] = 0.0f;
        for (int a = 0; a < kH; ++a) {
            sd1[a * kMlpSamples + t] = 0.0f;
            sh1[a * kMlpSamples + t] = 0.0f;
            sd2[a * kMlpSamples + t] = 0.0f;
            sh2[a * kMlpSamples + t] = 0.0f;
        }
#pragma unroll
        for (int f = 0; f < kF; ++f) sx[f * kMlpSamples + t] = 0.0f;
    }
    __syncthreads();
    float *out = partial + static_cast<int64_t>(blockIdx.x) * (kP + 1);
    for (int p = t; p <= kP; p += kMlpSamples) {
        const float *u, *v = nullptr;  // gradient = sum_s u[s] * v[s] (v null: sum_s u[s])
        if (p < oB1) {
            const int a = p / kF, f = p % kF;
            u = sd1 + a * kMlpSamples;
            v = sx + f * kMlpSamples;
        } else if (p < oW2) {
            u = sd1 + (p - oB1) * kMlpSamples;
        } else if (p < oB2) {
            const int a = (p - oW2) / kH, b = (p - oW2) % kH;
            u = sd2 + a * kMlpSamples;
            v = sh1 + b * kMlpSamples;
        } else if (p < oW3) {
            u = sd2 + (p - oB2) * kMlpSamples;
        } else if (p < oB3) {
            u = sdy;
            v = sh2 + (p - oW3) * kMlpSamples;
        } else if (p == oB3) {
            u = sdy;
        } else {
            u = sl;
        }
        float acc = 0.0f;
        if (v) {
            for (int s = 0; s < kMlpSamples; ++s) acc = fmaf(u[s], v[s], acc);
        } else {
            for (int s = 0; s < kMlpSamples; ++s) acc += u[s];
        }
        out[p] = acc;
    }
}

// grad[p] = sum over CTAs (in CTA order) of partial[cta][p]; grad[kP] = mean loss
__global__ void k_mlp_reduce(const float *__restrict__ partial, int nblk, int32_t N, float *__restrict__ grad,
                             float *__restrict__ loss_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kP) return;
    float acc = 0.0f;
    for (int b = 0; b < nblk; ++b) acc += partial[static_cast<int64_t>(b) * (kP + 1) + p];
    if (p < kP) grad[p] = acc;
    else {
        grad[kP] = acc / static_cast<float>(N);
        if (loss_out) *loss_out = acc / static_cast<float>(N);
    }
}

// Adam (Kingma and Ba) with bias correction, step t >= 1
__global__ void k_adam(float *__restrict__ params, const float *__restrict__ grad, float *__restrict__ m,
                       float *__restrict__ v, int t, float lr, float b1, float b2, float eps) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kP) return;
    const float gr = grad[p];
    const float mm = b1 * m[p] + (1.0f - b1) * gr;
    const float vv = b2 * v[p] + (1.0f - b2) * gr * gr;
    m[p] = mm;
    v[p] = vv;
    const float mhat = mm / (1.0f - powf(b1, static_cast<float>(t)));
    const float vhat = vv / (1.0f - powf(b2, static_cast<float>(t)));
    params[p] -= lr * mhat / (sqrtf(vhat) + eps);
}

// per-source length: the smallest odd integer >= exp(y) - 1/4, clipped to
// [1, cap]. Labels are odd: a prediction at most 1/4 above one takes it (a
// short prediction costs its source a rerun, a long one wasted hops)
__global__ void k_mlp_predict(const float *__restrict__ model, const float *__restrict__ F, int32_t n, int32_t cap,
                              int32_t *__restrict__ L) {
    __shared__ float w[kP + 2 * kF];
    for (int p = threadIdx.x; p < kP + 2 * kF; p += blockDim.x) w[p] = model[p];
    __syncthreads();
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[kF], z1[kH], h1[kH], z2[kH], h2[kH];
#pragma unroll
    for (int f = 0; f < kF; ++f) x[f] = (F[static_cast<int64_t>(i) * kF + f] - w[kP + f]) / w[kP + kF + f];
    const float y = mlp_forward(w, x, z1, h1, z2, h2);
    double e = ceil(exp(static_cast<double>(y)) - 0.25);
    if (!(e >= 1.0)) e = 1.0;  // also catches NaN
    if (e > static_cast<double>(cap)) e = static_cast<double>(cap);
    int32_t l = static_cast<int32_t>(e);
    if ((l & 1) == 0) l = min(l + 1, (cap & 1) ? cap : cap + 1);
    L[i] = l;
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static void ensure_features(sc_graph *g, cudaStream_t s) {
    if (g->features_ready) return;
    g->features.reserve(static_cast<size_t>(g->n) * kF);
    k_features<<<ceil_div(g->n, 8), 256, 0, s>>>(g->row_ptr.get(), g->col_idx.get(), g->n,
                                                 static_cast<double>(g->nnz) / static_cast<double>(g->n),
                                                 g->features.get());
    SC_LAUNCH_CHECK();
    SC_CUDA(cudaStreamSynchronize(s));
    g->features_ready = true;
}

void learned_lengths(sc_graph *g, int32_t cap, int32_t *L_dev, cudaStream_t s) {
    ensure_features(g, s);
    k_mlp_predict<<<ceil_div(g->n, 128), 128, 0, s>>>(g->mlp.get(), g->features.get(), g->n, cap, L_dev);
    SC_LAUNCH_CHECK();
}

static size_t grad_smem() {
    return sizeof(float) * (kP + 3 + kF * kMlpSamples + 4 * kH * kMlpSamples + 2 * kMlpSamples);
}

static void grad_launch(const float *params, const float *X, const float *y, int32_t N, float *partial, float *grad,
                        float *loss, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        SC_CUDA(cudaFuncSetAttribute(k_mlp_grad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(grad_smem())));
        attr = true;
    }
    const int nblk = ceil_div(N, kMlpSamples);
    k_mlp_grad_partial<<<nblk, kMlpSamples, grad_smem(), s>>>(params, X, y, N, partial);
    k_mlp_reduce<<<ceil_div(kP + 1, 256), 256, 0, s>>>(partial, nblk, N, grad, loss);
    SC_LAUNCH_CHECK();
}

}  // namespace sc

using namespace sc;

extern "C" {

sc_status sc_source_features(sc_graph *g, float *features) {
    return guarded([&] {
        if (!g || !features) SC_FAIL(SC_ERR_INVALID_ARG, "null argument");
        ensure_features(g, g->stream);
        SC_CUDA(cudaMemcpyAsync(features, g->features.get(), static_cast<size_t>(g->n) * kF * sizeof(float),
                                cudaMemcpyDeviceToHost, g->stream));
        SC_CUDA(cudaStreamSynchronize(g->stream));
    });
}

sc_status sc_certified_lengths(sc_graph *g, double eps, int32_t precision, int32_t *per_entry, int32_t *per_source,
                               int32_t *cap) {
    return guarded([&] {
        if (!g || !per_entry) SC_FAIL(SC_ERR_INVALID_ARG, "null argument");
        if (!(eps > 0.0 && eps < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "eps must lie in (0, 1)");
        DevBuf<int32_t> te;
        te.reserve(g->nnz);
        int32_t c = 0;
        certified_lengths_impl(g, eps, precision, te.get(), &c);
        SC_CUDA(cudaMemcpyAsync(per_entry, te.get(), g->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
        SC_CUDA(cudaStreamSynchronize(g->stream));
        if (per_source) {
            for (int32_t i = 0; i < g->n; ++i) {
                int32_t m = 0;
                for (int32_t k = g->h_row_ptr[i]; k < g->h_row_ptr[i + 1]; ++k) m = std::max(m, per_entry[k]);
                per_source[i] = m;
            }
        }
        if (cap) *cap = c;
    });
}

sc_status sc_estimated_lengths(sc_graph *g, double eps, int32_t precision, int32_t cap, int32_t *per_entry,
                               int32_t *per_source) {
    return guarded([&] {
        if (!g || !per_entry) SC_FAIL(SC_ERR_INVALID_ARG, "null argument");
        if (!(eps > 0.0 && eps < 1.0)) SC_FAIL(SC_ERR_INVALID_ARG, "eps must lie in (0, 1)");
        if (cap < 3) SC_FAIL(SC_ERR_INVALID_ARG, "cap must be >= 3, got %d", cap);
        DevBuf<int32_t> te;
        te.reserve(g->nnz);
        estimated_lengths_impl(g, eps, precision, cap, te.get());
        SC_CUDA(cudaMemcpyAsync(per_entry, te.get(), g->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
        SC_CUDA(cudaStreamSynchronize(g->stream));
        if (per_source) {
            for (int32_t i = 0; i < g->n; ++i) {
                int32_t m = 0;
                for (int32_t k = g->h_row_ptr[i]; k < g->h_row_ptr[i + 1]; ++k) m = std::max(m, per_entry[k]);
                per_source[i] = m;
            }
        }
    });
}

sc_status sc_mlp_loss_grad(const float *model, const float *features, const float *targets, int32_t count,
                           float *loss, float *grad, void *stream) {
    return guarded([&] {
        if (!model || !features || !targets || count <= 0 || !loss || !grad)
            SC_FAIL(SC_ERR_INVALID_ARG, "null argument or empty batch");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        // standardise on the host with the model's mean / std (data preparation, not the MLP)
        std::vector<float> X(static_cast<size_t>(count) * kF);
        for (int32_t i = 0; i < count; ++i)
            for (int f = 0; f < kF; ++f)
                X[static_cast<size_t>(i) * kF + f] = (features[static_cast<size_t>(i) * kF + f] - model[kP + f]) /
                                                     model[kP + kF + f];
        DevBuf<float> dp, dX, dy, part, dg;
        dp.reserve(kP);
        dX.reserve(X.size());
        dy.reserve(count);
        part.reserve(static_cast<size_t>(ceil_div(count, kMlpSamples)) * (kP + 1));
        dg.reserve(kP + 1);
        SC_CUDA(cudaMemcpyAsync(dp.get(), model, kP * sizeof(float), cudaMemcpyHostToDevice, s));
        SC_CUDA(cudaMemcpyAsync(dX.get(), X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        SC_CUDA(cudaMemcpyAsync(dy.get(), targets, count * sizeof(float), cudaMemcpyHostToDevice, s));
        grad_launch(dp.get(), dX.get(), dy.get(), count, part.get(), dg.get(), nullptr, s);
        std::vector<float> h(kP + 1);
        SC_CUDA(cudaMemcpyAsync(h.data(), dg.get(), (kP + 1) * sizeof(float), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
        std::copy(h.begin(), h.begin() + kP, grad);
        *loss = h[kP];
    });
}

sc_status sc_mlp_train(sc_graph *const *graphs, int32_t count, const sc_mlp_train_opts *opts,
                       const float *init_params, float *model_out, float *loss_curve) {
    return guarded([&] {
        if (!graphs || count <= 0 || !opts || !init_params || !model_out)
            SC_FAIL(SC_ERR_INVALID_ARG, "null argument or no graphs");
        if (opts->epochs <= 0 || !(opts->lr > 0.0f) || !(opts->eps > 0.0 && opts->eps < 1.0))
            SC_FAIL(SC_ERR_INVALID_ARG, "epochs, lr and eps must be positive (eps < 1)");
        cudaStream_t s = graphs[0]->stream;
        // training set: features and log certified (bipartite: estimated) per-source lengths of every graph
        std::vector<float> F, y;
        for (int32_t gi = 0; gi < count; ++gi) {
            sc_graph *g = graphs[gi];
            if (!g) SC_FAIL(SC_ERR_INVALID_ARG, "null graph %d", gi);
            ensure_features(g, g->stream);
            std::vector<float> f(static_cast<size_t>(g->n) * kF);
            SC_CUDA(cudaMemcpyAsync(f.data(), g->features.get(), f.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                    g->stream));
            DevBuf<int32_t> te;
            te.reserve(g->nnz);
            int32_t cap = 0;
            if (g->bipartite) {
                if (opts->ell_cap < 3 || (opts->ell_cap & 1) == 0)
                    SC_FAIL(SC_ERR_INVALID_ARG, "graph %d is bipartite: its labels need an odd ell_cap >= 3", gi);
                estimated_lengths_impl(g, opts->eps, opts->precision, opts->ell_cap, te.get());
            } else {
                certified_lengths_impl(g, opts->eps, opts->precision, te.get(), &cap);
            }
            std::vector<int32_t> tau(g->nnz);
            SC_CUDA(cudaMemcpyAsync(tau.data(), te.get(), g->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
            SC_CUDA(cudaStreamSynchronize(g->stream));
            for (int32_t i = 0; i < g->n; ++i) {
                int32_t m = 1;
                for (int32_t k = g->h_row_ptr[i]; k < g->h_row_ptr[i + 1]; ++k) m = std::max(m, tau[k]);
                y.push_back(static_cast<float>(log(static_cast<double>(m))));
            }
            F.insert(F.end(), f.begin(), f.end());
        }
        const int32_t N = static_cast<int32_t>(y.size());
        std::vector<float> model(kP + 2 * kF);
        std::copy(init_params, init_params + kP, model.begin());
        for (int f = 0; f < kF; ++f) {  // feature mean and standard deviation (population)
            double mu = 0.0, sq = 0.0;
            for (int32_t i = 0; i < N; ++i) mu += F[static_cast<size_t>(i) * kF + f];
            mu /= N;
            for (int32_t i = 0; i < N; ++i) {
                const double d = F[static_cast<size_t>(i) * kF + f] - mu;
                sq += d * d;
            }
            const double sd = std::sqrt(sq / N);
            model[kP + f] = static_cast<float>(mu);
            // a spread at rounding level marks a constant feature (scale 1); its
            // standardised input is 0 on every sample, so zero first-layer weights
            // change no step of the training and make the model ignore it elsewhere
            const bool constant = !(sd > 1e-9 * std::max(std::fabs(mu), 1.0));
            model[kP + kF + f] = constant ? 1.0f : static_cast<float>(sd);
            if (constant)
                for (int a = 0; a < kH; ++a) model[oW1 + a * kF + f] = 0.0f;
        }
        std::vector<float> X(F.size());
        for (int32_t i = 0; i < N; ++i)
            for (int f = 0; f < kF; ++f)
                X[static_cast<size_t>(i) * kF + f] = (F[static_cast<size_t>(i) * kF + f] - model[kP + f]) / model[kP + kF + f];
        DevBuf<float> dp, dm, dv, dX, dy, part, dg, curve;
        dp.reserve(kP);
        dm.reserve(kP);
        dv.reserve(kP);
        dX.reserve(X.size());
        dy.reserve(N);
        part.reserve(static_cast<size_t>(ceil_div(N, kMlpSamples)) * (kP + 1));
        dg.reserve(kP + 1);
        curve.reserve(opts->epochs);
        SC_CUDA(cudaMemcpyAsync(dp.get(), model.data(), kP * sizeof(float), cudaMemcpyHostToDevice, s));
        SC_CUDA(cudaMemsetAsync(dm.get(), 0, kP * sizeof(float), s));
        SC_CUDA(cudaMemsetAsync(dv.get(), 0, kP * sizeof(float), s));
        SC_CUDA(cudaMemcpyAsync(dX.get(), X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        SC_CUDA(cudaMemcpyAsync(dy.get(), y.data(), N * sizeof(float), cudaMemcpyHostToDevice, s));
        const float b1 = opts->beta1 > 0 ? opts->beta1 : 0.9f, b2 = opts->beta2 > 0 ? opts->beta2 : 0.999f;
        const float ae = opts->adam_eps > 0 ? opts->adam_eps : 1e-8f;
        for (int32_t e = 0; e < opts->epochs; ++e) {
            grad_launch(dp.get(), dX.get(), dy.get(), N, part.get(), dg.get(), curve.get() + e, s);
            k_adam<<<ceil_div(kP, 256), 256, 0, s>>>(dp.get(), dg.get(), dm.get(), dv.get(), e + 1, opts->lr, b1, b2, ae);
            SC_LAUNCH_CHECK();
        }
        SC_CUDA(cudaMemcpyAsync(model.data(), dp.get(), kP * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (loss_curve)
            SC_CUDA(cudaMemcpyAsync(loss_curve, curve.get(), opts->epochs * sizeof(float), cudaMemcpyDeviceToHost, s));
        SC_CUDA(cudaStreamSynchronize(s));
        std::copy(model.begin(), model.end(), model_out);
    });
}

sc_status sc_mlp_load(sc_graph *g, const float *model) {
    return guarded([&] {
        if (!g || !model) SC_FAIL(SC_ERR_INVALID_ARG, "null argument");
        for (int f = 0; f < kF; ++f)
            if (!(model[kP + kF + f] > 0.0f)) SC_FAIL(SC_ERR_INVALID_ARG, "feature scale %d must be positive", f);
        g->mlp.reserve(kP + 2 * kF);
        SC_CUDA(cudaMemcpyAsync(g->mlp.get(), model, (kP + 2 * kF) * sizeof(float), cudaMemcpyHostToDevice, g->stream));
        SC_CUDA(cudaStreamSynchronize(g->stream));
        g->mlp_loaded = true;
    });
}

sc_status sc_mlp_predict(sc_graph *g, int32_t cap, int32_t *lengths) {
    return guarded([&] {
        if (!g || !lengths || cap < 1) SC_FAIL(SC_ERR_INVALID_ARG, "null argument or cap < 1");
        if (!g->mlp_loaded) SC_FAIL(SC_ERR_INVALID_ARG, "no model loaded");
        DevBuf<int32_t> L;
        L.reserve(g->n);
        learned_lengths(g, cap, L.get(), g->stream);
        SC_CUDA(cudaMemcpyAsync(lengths, L.get(), g->n * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
        SC_CUDA(cudaStreamSynchronize(g->stream));
    });
}

}  // extern "C"

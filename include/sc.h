/*
 * sc.h -- C ABI of libsc: all-edge spanning centrality (AESC) on one GPU.
 *
 * Method: Zhang, Yang, Tang, Xiao, Tang, "Efficient Approximation Algorithms
 * for Spanning Centrality" (TGT / TGT+). The spanning centrality s(e) of an
 * edge is the fraction of spanning trees that contain it (Definition 2.1);
 * for an unweighted connected graph it equals the effective resistance, and
 * the paper computes it from the truncated random-walk series of Eq. (2),
 * accumulated per source node by a deterministic graph traversal
 * (Algorithm 2) and, for TGT+, completed by random walks (Algorithm 4).
 *
 * Conventions shared by every entry point:
 *  - Graphs are undirected, unweighted, connected and given as symmetric CSR:
 *    row_ptr int32[n+1] (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz),
 *    col_idx int32[nnz] with every row strictly increasing, no self-loops,
 *    and both (i,j) and (j,i) present. nnz = 2m < 2^31.
 *  - Per-edge outputs have one value per CSR entry, aligned with col_idx;
 *    the entries (i,j) and (j,i) carry the same value.
 *  - The caller owns every buffer it passes. A graph owns device copies of
 *    its CSR and the work buffers it allocates; sc_graph_destroy frees them.
 *  - All device work of a graph runs on the CUDA stream given to
 *    sc_graph_create (NULL = legacy default stream). Calls return after
 *    that work has completed unless stated otherwise. A graph must not be
 *    used by two host threads at once.
 *  - No C++ exception crosses this boundary. Each call returns an sc_status;
 *    sc_last_error_detail() gives a thread-local message for the last
 *    failing call of the calling thread.
 *  - Device pointers must come from the CUDA device that was current when
 *    the graph was created.
 */
#ifndef SC_H_
#define SC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SC_ABI_VERSION 1

typedef enum sc_status {
    SC_OK = 0,
    SC_ERR_INVALID_ARG = 1,        /* null pointer, negative size, bad option value */
    SC_ERR_BAD_CSR = 2,            /* row_ptr not monotone / wrong ends, column out of range, row not strictly sorted */
    SC_ERR_NOT_SYMMETRIC = 3,      /* some (i,j) has no (j,i) */
    SC_ERR_SELF_LOOP = 4,
    SC_ERR_DUPLICATE_EDGE = 5,
    SC_ERR_ISOLATED_NODE = 6,      /* a node of degree 0 */
    SC_ERR_DISCONNECTED = 7,
    SC_ERR_BIPARTITE = 8,          /* only with SC_FLAG_REJECT_BIPARTITE */
    SC_ERR_LAMBDA_NOT_CONVERGED = 9,
    SC_ERR_BOUND_UNMET = 10,       /* an edge failed its tail check after the last allowed extension */
    SC_ERR_TIMEOUT = 11,           /* a bounded device-side wait gave up */
    SC_ERR_OOM = 12,
    SC_ERR_CUDA = 13,
    SC_ERR_UNSUPPORTED = 14
} sc_status;

/* ---- flags for sc_graph_create ---------------------------------------- */
#define SC_PTRS_HOST 0u               /* row_ptr / col_idx are host pointers */
#define SC_PTRS_DEVICE 1u             /* row_ptr / col_idx are device pointers */
#define SC_FLAG_REJECT_BIPARTITE 2u   /* fail with SC_ERR_BIPARTITE on a bipartite graph */

typedef struct sc_graph sc_graph;

typedef struct sc_graph_info {
    int32_t n;
    int64_t nnz;          /* 2 m */
    int64_t m;
    int32_t min_degree;
    int32_t max_degree;
    int32_t bipartite;    /* 1 if the graph has no odd cycle */
    int32_t diameter_lb;  /* eccentricity of node 0 (BFS depth), a lower bound on the diameter */
} sc_graph_info;

/*
 * sc_graph_create -- validate a CSR graph and build its device copy.
 * Cites: the input of Definition 2.2 (an undirected connected graph) and the
 * notation of Section 2.1 (N(v), d(v), P = D^-1 A).
 *
 *   out     : receives the new graph (NULL on failure)
 *   n       : number of nodes, >= 2
 *   nnz     : number of CSR entries (2m), >= 2
 *   row_ptr : int32[n+1], host or device per flags
 *   col_idx : int32[nnz],  host or device per flags
 *   flags   : SC_PTRS_HOST | SC_PTRS_DEVICE, optionally SC_FLAG_REJECT_BIPARTITE
 *   stream  : cudaStream_t for all of this graph's work (NULL = default stream)
 *
 * Copies the arrays (the caller may free them on return), validates them on
 * the device, builds the reverse-entry map and 1/d(v), and runs a BFS from
 * node 0 for connectivity and the bipartite test. Errors: SC_ERR_BAD_CSR,
 * SC_ERR_NOT_SYMMETRIC, SC_ERR_SELF_LOOP, SC_ERR_DUPLICATE_EDGE,
 * SC_ERR_ISOLATED_NODE, SC_ERR_DISCONNECTED, SC_ERR_BIPARTITE, SC_ERR_OOM,
 * SC_ERR_CUDA, SC_ERR_INVALID_ARG.
 */
sc_status sc_graph_create(sc_graph **out, int32_t n, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, uint32_t flags, void *stream);

/* sc_graph_get_info -- sizes and structural facts found by sc_graph_create. */
sc_status sc_graph_get_info(const sc_graph *g, sc_graph_info *out);

/* sc_graph_destroy -- free the graph and its device memory (NULL is a no-op). */
void sc_graph_destroy(sc_graph *g);

/* ---- eigenvalue bound --------------------------------------------------- */

typedef struct sc_lambda {
    double lambda_plus;      /* largest eigenvalue of D^-1/2 A D^-1/2 below 1 (Ritz value) */
    double lambda_minus;     /* smallest eigenvalue; for a bipartite graph the smallest above -1 */
    double lambda_star;      /* max(|lambda_plus|, |lambda_minus|) plus the larger residual: the
                                "second largest in absolute value" of Lemma 3.1 with a safety margin */
    double residual_plus;    /* ||N y - theta y|| of the two Ritz pairs */
    double residual_minus;
    int32_t iterations;      /* Lanczos steps taken */
    int32_t converged;       /* 1 if both residuals met the tolerance */
} sc_lambda;

typedef struct sc_lambda_opts {
    int32_t max_iter;        /* Lanczos steps (0 = 500) */
    double tol;              /* residual tolerance (0 = 1e-4); the residual is added to lambda_star */
    uint64_t seed;           /* start vector (Philox4x32-10 stream) */
} sc_lambda_opts;

/*
 * sc_estimate_lambda -- spectrum extremes of N = D^{1/2} P D^{-1/2}
 * (Lemma 3.1), the lambda that sets the truncation length (Eq. 6, Algorithm 1's
 * initial length). FP64 Lanczos with full reorthogonalisation on the device, after
 * deflating the top eigenvector sqrt(d)/sqrt(2m) (and, for a bipartite graph,
 * the bottom one). opts may be NULL for defaults. The result is also cached
 * in the graph for sc_all_edges. SC_ERR_LAMBDA_NOT_CONVERGED is returned
 * (with *out filled) when a residual stays above tol after max_iter steps.
 */
sc_status sc_estimate_lambda(sc_graph *g, const sc_lambda_opts *opts, sc_lambda *out);

/*
 * sc_graph_set_lambda -- make the graph use a caller's eigenvalue bound (as
 * the paper takes lambda from an external eigensolver, Section 5.3.3) in place
 * of sc_estimate_lambda's: every later call that needs lambda (Eq. 6, the
 * learned length's checks, the end-corrected bound) reads *lam. The caller
 * vouches for it: lambda_star must bound the modulus of every eigenvalue of
 * D^-1/2 A D^-1/2 except 1 (and -1 on a bipartite graph); nothing is checked
 * beyond 0 <= lambda_star <= 1, |lambda_plus| <= lambda_star and, unless the
 * graph is bipartite, |lambda_minus| <= lambda_star. Errors: SC_ERR_INVALID_ARG.
 */
sc_status sc_graph_set_lambda(sc_graph *g, const sc_lambda *lam);

/*
 * sc_truncation_length -- tau per edge and per source from Eq. (5)-(6)
 * with omega = 2 (Algorithm 1's initial length), Upsilon = Delta_t = 0:
 *   f(e_ij, eps) = ceil( log(X_e / (eps (1 - lambda^2))) / log(1/lambda) - 1 ),
 *   X_e = 1/d_i + 1/d_j - 2/(d_i d_j), tau_ij = smallest odd integer >= max(f, 1),
 * tau_p(i) = max_j tau_ij (Algorithm 2's per-source length), ell_global = max_i tau_p(i).
 *
 *   eps            : > 0 (TGT uses eps; TGT+, Algorithm 4, passes eps/2)
 *   lam            : from sc_estimate_lambda; NULL = the graph's cached value
 *                    (SC_ERR_INVALID_ARG if none); lambda_star must be < 1
 *   ell_global_out : host int32 (may be NULL)
 *   per_source_out : host int32[n] (may be NULL)
 *   per_entry_out  : host int32[nnz] (may be NULL)
 */
sc_status sc_truncation_length(sc_graph *g, double eps, const sc_lambda *lam,
                               int32_t *ell_global_out, int32_t *per_source_out,
                               int32_t *per_entry_out);

/* ---- CalTau with omega eigenpairs (Algorithm 1, Eq. 6-8) ------------------- */

#define SC_OMEGA_MAX 257    /* eigenpairs per call, lambda_1 = 1 included */

typedef struct sc_eig_opts {
    int32_t omega;           /* eigenpairs wanted, lambda_1 = 1 included, 2..SC_OMEGA_MAX */
    int32_t max_iter;        /* Lanczos steps of the first run (0 = min(n - 1, 3 omega + 64)) */
    double tol;              /* Ritz residual a pair must meet to be taken exactly (0 = 1e-8) */
    double rest_tol;         /* residual of the second run's extreme Ritz pairs (0 = 1e-6) */
    int32_t rest_max_iter;   /* Lanczos steps of the second run (0 = 500) */
    int32_t reserved;
    uint64_t seed;           /* start vectors (Philox4x32-10 streams; the second run uses seed + 1) */
} sc_eig_opts;

typedef struct sc_eig_report {
    int32_t used;            /* pairs taken exactly, lambda_1 included (<= omega) */
    int32_t iterations;      /* steps of the first run */
    int32_t rest_iterations; /* steps of the second run (0 when every mode is taken) */
    int32_t rest_converged;  /* 1 if the second run's residuals met rest_tol */
    double max_residual;     /* largest Ritz residual among the pairs taken */
    double rest_residual;    /* larger residual of the second run's two extreme Ritz pairs */
    double lambda_rest;      /* r: bound on the modulus of every nontrivial mode not taken */
} sc_eig_report;

/*
 * sc_eigenpairs -- eigenpairs of N = D^-1/2 A D^-1/2 of largest modulus for
 * CalTau (Algorithm 1): lambda_k and f_k = sqrt(2m) D^-1/2 phi_k (Eq. 7-8's
 * vectors, the notation of Theorem 3.2's proof), and a bound r on the modulus
 * of every other nontrivial mode. Two FP64 Lanczos runs with full
 * reorthogonalisation on the device: the first, with sqrt(d)/sqrt(2m)
 * deflated, gives Ritz pairs; those of the omega - 1 largest moduli whose
 * residual meets tol are taken (U). The second runs on the complement of U
 * from a fresh start vector, so it also sees the copies of a repeated
 * eigenvalue that a single Krylov sequence cannot; r = its larger extreme
 * modulus plus its residual and the largest residual in U (the margin of
 * sc_estimate_lambda). The pairs and r are kept in the graph for sc_caltau.
 *
 *   opts     : may be NULL (omega 129 and the defaults above)
 *   lam_out  : host double[omega]; lam_out[0] = 1, then U by decreasing
 *              modulus (the larger value first on a tie), zeros past `used`
 *   F_out    : host double[omega * n] (may be NULL); row k = f_k (row 0 all
 *              ones), rows past `used` zero; the sign of a row is arbitrary
 *   report   : may be NULL
 * Errors: SC_ERR_UNSUPPORTED for a bipartite graph (lambda = -1 is a mode of
 * modulus 1: no length meets Theorem 3.2); SC_ERR_LAMBDA_NOT_CONVERGED (with
 * the outputs filled) when the second run's residual stays above rest_tol;
 * SC_ERR_INVALID_ARG for omega outside 2..SC_OMEGA_MAX or above n.
 */
sc_status sc_eigenpairs(sc_graph *g, const sc_eig_opts *opts, double *lam_out, double *F_out,
                        sc_eig_report *report);

/*
 * sc_caltau -- Algorithm 1 (CalTau) for every CSR entry: with the pairs of U
 * taken exactly and r for the rest, Upsilon = sum_U c_k (1 + lambda_k) / 2m
 * (Eq. 7) and Delta_t = sum_U c_k lambda_k^(t+1) / (1 - lambda_k) / 2m (Eq. 8),
 * c_k = (f_k[i] - f_k[j])^2; starting from tau0 = Eq. 6 with
 * lambda_star = max(max_U |lambda|, r), t = 1, 3, 5, ... until t exceeds Eq. 6
 * with X_e - Upsilon, eps - Delta_t and r in place of X_e, eps and lambda; the
 * length is min(t, tau0). The proof of Theorem 3.2 bounds each left-out term by
 * r^(t+1) / (1 - r^2) c_k (1 + lambda_k), so any U with such an r meets eps.
 * The lengths are kept in the graph for SC_ELL_CALTAU.
 *
 *   eps       : 0 < eps < 1
 *   count     : pairs in lam / F, lambda_1 = 1 included (2..SC_OMEGA_MAX);
 *               0 = the pairs of the graph's last sc_eigenpairs (lam, F and
 *               lam_rest are then ignored)
 *   lam       : host double[count], lam[0] = 1 (ignored), |lam[k]| < 1
 *   F         : host double[count * n], row k = f_k (row 0 ignored)
 *   lam_rest  : r, 0 <= r < 1
 *   tau_out   : host int32[nnz] (may be NULL); both directions of an edge equal
 *   ell_out   : host int32, the largest length (may be NULL)
 * Errors: SC_ERR_INVALID_ARG (no pairs, or a modulus >= 1); SC_ERR_UNSUPPORTED
 * for a bipartite graph or when Eq. 6's length passes 2^20 (the Delta_t loop
 * would take more than 2^19 steps per edge).
 */
sc_status sc_caltau(sc_graph *g, double eps, int32_t count, const double *lam, const double *F,
                    double lam_rest, int32_t *tau_out, int32_t *ell_out);

/*
 * sc_tridiag_eig -- every eigenpair of the symmetric tridiagonal matrix with
 * diagonal alpha[0..k) and off-diagonal beta[0..k-1) (beta[i] couples i and
 * i + 1), by the implicit symmetric QR algorithm with Wilkinson shifts: the
 * host-side step of sc_eigenpairs, exported for testing. Host only, no GPU.
 *   theta : host double[k], ascending
 *   Z     : host double[k * k] (may be NULL); column q (Z[q * k .. q * k + k))
 *           = the unit eigenvector of theta[q]
 * Errors: SC_ERR_INVALID_ARG (k < 1, NULL arrays); SC_ERR_LAMBDA_NOT_CONVERGED
 * if an eigenvalue needs more than 60 QR steps.
 */
sc_status sc_tridiag_eig(int32_t k, const double *alpha, const double *beta, double *theta, double *Z);

/*
 * sc_series_meet -- the truncated series S_tau of Eq. 2 per CSR entry by the
 * meet-in-the-middle form: for each edge (i, j) the column c_0 = e_i/d_i -
 * e_j/d_j is propagated by P for ceil(tau/2) hops, and the hop-l term is
 * t_l = sum_x d_x c_a[x] c_b[x], a = floor(l/2), b = l - a (Chapman-Kolmogorov
 * with reversibility; the deterministic form of the collision view of
 * Section 2.3). FP64, blocks of 32 edges. It gives what sc_all_edges gives with
 * the plain estimator at the same lengths, by half the hops per column but one
 * column per edge instead of per source.
 *   tau   : host int32[nnz], 0 <= tau <= 2^20, equal in both directions of an edge
 *   s_out : host double[nnz]
 * Errors: SC_ERR_INVALID_ARG (null, a length out of range or differing
 * between the two directions).
 */
sc_status sc_series_meet(sc_graph *g, const int32_t *tau, double *s_out);

/* ---- the all-edge computation --------------------------------------------- */

/* truncation policy */
#define SC_ELL_GLOBAL 0     /* one length for every edge: max of Eq. (6) over all edges */
#define SC_ELL_PER_EDGE 1   /* tau_ij of Eq. (6) per edge; sources run tau_p (Algorithm 2's per-source length) */
#define SC_ELL_FIXED 2      /* opts.ell_fixed for every edge (no eigenvalue needed) */
#define SC_ELL_LEARNED 3    /* per-source length predicted by the MLP (sc_mlp_load); every edge
                               is then certified by the bound of sc_certified_lengths and, if it
                               fails, extended (tau <- 2 tau + 1, at most Eq. 6) and recomputed;
                               the bound also covers the end-corrected estimator (whose remainder
                               is the smaller). On a bipartite graph (lambda* = 1: no bound and no
                               Eq. 6 length) with SC_EST_END_CORRECTED, an edge is accepted by the
                               tail estimate of sc_estimated_lengths instead (uncertified:
                               report.uncertified) and extended up to opts.ell_cap */
#define SC_ELL_CALTAU 4     /* the per-edge lengths of the graph's last sc_caltau (same eps; TGT only);
                               sources run the longest of their edges */

/* storage precision of the propagated probability block */
#define SC_PREC_FP64 0
#define SC_PREC_FP32 1
#define SC_PREC_BF16 2      /* bf16 storage from hop opts.bf16_from_hop on (fp32 storage before),
                               fp32 accumulation */

/* estimator */
#define SC_EST_PLAIN 0          /* S_tau of Eq. (2) */
#define SC_EST_END_CORRECTED 1  /* S_tau + t_{tau+1}/2: exact for the lambda = -1 mode of a
                                   bipartite graph, still a lower bound for odd tau */

/* algorithm */
#define SC_MODE_TGT 0           /* Algorithm 2: traversal only */
#define SC_MODE_TGT_PLUS 1      /* Algorithm 4: traversal, then random walks (Eq. 11, 13, 14) */

/* option flags */
#define SC_OUT_DEVICE 1u        /* s_hat (and aux outputs) are device pointers (else host) */
#define SC_OPT_RECORD_TAIL 2u   /* run 2 extra hops per source and report the tail bound */
#define SC_OPT_TIME_KERNELS 4u  /* bracket every propagation launch with CUDA events (report.hop_ms) */
/* Windowed blocks: Algorithm 2 visits only nodes with p_{l-1} > 0; a block of
   consecutive sources on a graph of bandwidth beta = max |i - j| reaches at
   hop l only rows within l * beta of its sources, so each block stores and
   computes that interval alone. Chosen automatically when a block's last
   window is under half the graph (grid-like numbering); the values are the
   same either way. Not with TGT+ or the TMA-gather kernel. */
#define SC_OPT_WINDOWS_OFF 8u
#define SC_OPT_WINDOWS_FORCE 16u
/* Unwindowed TGT blocks compute hop 3 from the non-zero values of X_2 only,
   and hop L-1 only on the sources' two-hop balls, where the last hop reads it
   (Algorithm 2's frontier, which visits only nodes it reaches); the values are
   those of full hops bit for bit. Off by default: on the power-law graphs
   measured the hop is bound by the latency of its dependent loads per row, not
   by the bytes it moves, and the full hop was as fast or faster. */
#define SC_OPT_SPARSE_HOPS 32u
/* TGT+ switch tests find each column's gamma largest entries (Algorithm 3's
   candidates) from the entries at or above the gamma-th largest maximum of its
   256-row tiles; this flag scans every row of the column instead (the same
   candidates; for comparison). */
#define SC_OPT_FULL_TOPGAMMA_SCAN 64u

/* kernel classes of the per-class timing in sc_report (SC_OPT_TIME_KERNELS) */
#define SC_KC_DENSE_HOP 0   /* full hops (k_spmm_hop, or the TMA-gather hop) */
#define SC_KC_MASK_HOP 1    /* hops 1-2 from the sources' neighbour bits (k_mask_scatter + k_hop2_mask) */
#define SC_KC_SPARSE_HOP 2  /* hop 3 from the non-zero values of X_2 (k_hop_sparse) */
#define SC_KC_BALL_HOP 3    /* hop L-1 on the two-hop balls (k_hop_ball) */
#define SC_KC_LAST_HOP 4    /* the last hop where its gather reads it (k_last_diag + k_last_rows) */
#define SC_KC_SWITCH_TEST 5 /* TGT+: a switch test (CalChi's column statistics, chi and R per entry, the
                               copy of the counts and the host's wait for it) */
#define SC_KC_WALKS 6       /* TGT+: a walk phase (walk counts, the host's plan, the walk kernels) */
#define SC_KC_COUNT 7

typedef struct sc_options {
    double eps;               /* absolute error target of Definition 2.2, 0 < eps < 1 */
    int32_t mode;             /* SC_MODE_* */
    int32_t precision;        /* SC_PREC_* */
    int32_t ell_policy;       /* SC_ELL_* */
    int32_t ell_fixed;        /* tau for SC_ELL_FIXED (>= 0) */
    int32_t estimator;        /* SC_EST_* */
    int32_t block_width;      /* sources per block B in {32, 64, 128}; 0 = choose automatically */
    int32_t rows_split;       /* 16-byte vectors per lane in {1, 2, 4}; -1 = the TMA-gather kernel;
                                 0 = choose automatically */
    int32_t heavy_threshold;  /* rows above this degree are split over a whole CTA (0 = 256) */
    int32_t max_slices;       /* blocks propagated together in one launch (0 = fit the L2 budget) */
    uint32_t flags;           /* SC_OUT_DEVICE | SC_OPT_* */
    uint64_t seed;            /* Philox key for TGT+ walks */
    double delta;             /* TGT+ failure probability (0 = 1/n, Section 5.1) */
    int32_t gamma;            /* CalChi candidates (Alg. 3), 0..16; default 10 when < 0 */
    int32_t switch_rule;      /* TGT+: SC_SWITCH_COST (default) or SC_SWITCH_PAPER (Eq. 14 as printed) */
    int32_t bf16_from_hop;    /* SC_PREC_BF16: X_l is stored in bf16 for l >= this hop and in fp32
                                 before it, where the probabilities are large (0 = 8; 1 = every hop) */
    int32_t ell_cap;          /* SC_ELL_LEARNED on a bipartite graph: the longest length an edge may
                                 be extended to (>= 3; required there, unused elsewhere) */
    int32_t reserved[4];
} sc_options;

/* TGT+ switch rules (when to stop the traversal and draw walks) */
#define SC_SWITCH_COST 0   /* cost: walks once their predicted time (fixed GB300 rates per walk step
                              and per source-hop entry) is below the remaining hops' */
#define SC_SWITCH_PAPER 1  /* Eq. 14: frontier volume above the sum of walk counts, both summed over
                              the sources of a launch, which switch together */
#define SC_SWITCH_PER_SOURCE 2  /* Eq. 14 per source, as Algorithm 4's loop is written: after each hop
                                   a source whose own frontier volume exceeds the sum of its own walk
                                   counts draws its walks from that hop's column and gathers no later
                                   hop; the launch continues while any source is still traversing */

/* fills *opts with defaults: eps 1e-3, TGT, FP32, global length, plain estimator, auto B */
void sc_options_default(sc_options *opts);

typedef struct sc_report {
    int32_t ell_global;        /* longest per-edge length used (the learned policy: its cap, Eq. 6
                                  or opts.ell_cap) */
    int32_t ell_min_source;    /* shortest / longest source run (hops) */
    int32_t ell_max_source;
    int32_t block_width;       /* B actually used */
    int32_t rows_split;
    int32_t slices;            /* blocks per launch */
    int64_t blocks;            /* source blocks processed */
    int64_t launches;          /* kernel launches issued */
    int64_t hops;              /* sum over blocks of hops run */
    double algorithmic_bytes;  /* bytes the propagation's hop launches must move, every kernel class */
    double foster_sum;         /* sum over edges of s_hat; Foster's theorem: n - 1 for exact values */
    double max_tail_bound;     /* with SC_OPT_RECORD_TAIL: max a-posteriori tail bound */
    double lambda_star;        /* lambda used */
    double propagate_ms;       /* device time of the traversal (events) */
    double total_ms;
    double hop_ms;             /* with SC_OPT_TIME_KERNELS: summed duration of the propagation launches */
    int64_t hop_launches;      /* propagation (SpMM hop) launches */
    double hop_bytes;          /* algorithmic bytes of those launches (part of algorithmic_bytes) */
    int64_t walks;             /* TGT+: random walk pairs drawn */
    int32_t edges_extended;    /* learned policy: edges whose length was extended */
    int32_t tt_min, tt_max;    /* TGT+: shortest / longest traversal before switching to walks */
    int32_t switch_tests;      /* TGT+: switch tests run */
    double switch_ms;          /* TGT+: wall time in switch tests (kernels, copies, host work) */
    double walk_ms;            /* TGT+: wall time drawing walks (planning, kernels) */
    int64_t source_hops;       /* sum over sources of hops traversed (the traversal's work) */
    int32_t extension_rounds;  /* learned policy: rerun rounds for edges that failed their bound */
    int32_t windowed;          /* 1 if the blocks ran windowed (SC_OPT_WINDOWS_*) */
    int64_t walk_steps;        /* TGT+: walk steps taken (both walks of every pair) */
    double walk_device_ms;     /* TGT+: device time of the walk launches (events) */
    /* with SC_OPT_TIME_KERNELS, per kernel class SC_KC_*: summed duration (events around
       each launch), launches, and the algorithmic bytes those launches must move (CSR,
       1/d, masks, block reads and writes; the dense class is hop_ms / hop_bytes) */
    double kc_ms[SC_KC_COUNT];
    int64_t kc_launches[SC_KC_COUNT];
    double kc_bytes[SC_KC_COUNT];
    int32_t uncertified;       /* 1 if the learned lengths were accepted by the tail estimate of
                                  sc_estimated_lengths (bipartite graph), not by a bound */
    int32_t reserved_r;
} sc_report;

/*
 * sc_all_edges -- estimate s(e) for every edge (Definition 2.2).
 * TGT (Algorithm 2): blocks of B sources are propagated together, X_l =
 * D^-1 A X_{l-1} (Algorithm 2's hop, in pull form), and for each source i and
 * neighbour j the half sum g(v_i, v_j) of Eq. (9) is accumulated for the
 * hops l <= tau_ij; the output is s_hat(e_ij) = g(v_i, v_j) + g(v_j, v_i)
 * (Algorithm 2's final combine), one length per edge for both halves. TGT+ (SC_MODE_TGT_PLUS, Algorithm 4): the traversal
 * of a block stops at the switch hop and the rest of each half sum is the
 * mean of Philox-driven walk pairs (Eq. 11, counts from Eq. 13 with chi from
 * Alg. 3); results are bit-identical for a given seed.
 *
 *   opts       : NULL = defaults (sc_options_default)
 *   s_hat      : double[nnz], host or device per SC_OUT_DEVICE
 *   tail_bound : nullable double[nnz]; with SC_OPT_RECORD_TAIL the
 *                a-posteriori bound on the remaining tail of each edge
 *   report     : nullable
 * The global, per-edge and learned policies need lambda: sc_estimate_lambda
 * is run first if the graph has no cached value. A bipartite graph under
 * these policies fails with SC_ERR_UNSUPPORTED (lambda_star = 1: no finite
 * length); use SC_ELL_FIXED with the end-corrected estimator. Errors:
 * SC_ERR_INVALID_ARG (NULL graph or output, bad option values),
 * SC_ERR_UNSUPPORTED (TGT+ with the learned policy, the end-corrected
 * estimator or tail records), SC_ERR_TIMEOUT (a bounded wait of the TMA hop
 * expired), SC_ERR_OOM, SC_ERR_CUDA. Outputs are unspecified on error.
 */
sc_status sc_all_edges(sc_graph *g, const sc_options *opts, double *s_hat, double *tail_bound,
                       sc_report *report);

/*
 * sc_some_edges -- s_hat for the listed CSR entries only: Definition 2.2's
 * output restricted to a set of edges. Algorithm 2's loop over sources runs
 * over the endpoints of the listed entries alone (each edge needs the half sums
 * of Eq. 9 from both of its endpoints); everything else is sc_all_edges with
 * the same options. A source's column does not depend on which sources share
 * its block, so each value equals sc_all_edges's at that entry bit for bit,
 * except under TGT+ with SC_SWITCH_COST or SC_SWITCH_PAPER, where a block's
 * switch hop depends on its sources (with SC_SWITCH_PER_SOURCE it does not).
 * The learned policy checks and extends only entries whose two endpoints ran.
 *
 *   opts    : as sc_all_edges (NULL = defaults); SC_OUT_DEVICE applies to s_out
 *   count   : number of entries, >= 1
 *   entries : host int64[count], CSR entry indices in [0, nnz) (repeats allowed)
 *   s_out   : double[count], host or device per SC_OUT_DEVICE: s_hat of entries[t]
 *   report  : nullable; as sc_all_edges, with foster_sum the sum of the count
 *             returned values and max_tail_bound the largest over the listed entries
 * Errors: those of sc_all_edges; SC_ERR_INVALID_ARG for count < 1, NULL arrays
 * or an entry outside [0, nnz).
 */
sc_status sc_some_edges(sc_graph *g, const sc_options *opts, int64_t count, const int64_t *entries, double *s_out,
                        sc_report *report);

/*
 * sc_batch_all_edges -- sc_all_edges over many independent graphs in one
 * pass (Definition 2.2 for each). The paper treats one graph at a time;
 * Algorithm 2's source loop is independent across graphs as much as across
 * sources, so the graphs' disjoint union is propagated in windowed blocks
 * (SC_OPT_WINDOWS_*): a block holds sources of one graph and one length and
 * stores and computes that graph's rows only. The launches of the whole
 * batch are recorded into one CUDA graph and replayed as one launch.
 *
 *   graphs        : count >= 1 graphs created on one device. The batch runs
 *                   on graphs[0]'s stream after waiting for every graph's
 *                   stream; each graph's lambda estimate is computed if the
 *                   Eq. 6 length needs it and none is cached.
 *   opts          : as sc_all_edges, for every graph; mode SC_MODE_TGT,
 *                   policy SC_ELL_GLOBAL (each graph its own Eq. 6 length),
 *                   SC_ELL_FIXED, or SC_ELL_LEARNED (each graph its own
 *                   loaded model; every edge checked as in sc_all_edges, by
 *                   the bound with the graph's lambda* or, on a bipartite
 *                   graph, by the tail estimate with the end-corrected
 *                   estimator; failing edges of all graphs are extended and
 *                   rerun together); no TMA-gather split.
 *   ell_per_graph : nullable; count entries; > 0 overrides graph i's length
 *                   (e.g. an empirical length for a bipartite lattice, whose
 *                   Eq. 6 length does not exist), 0 keeps the policy. With
 *                   SC_ELL_LEARNED it is graph i's cap (its longest length;
 *                   default Eq. 6, or opts.ell_cap on a bipartite graph).
 *   s_hat         : count pointers; s_hat[i] holds graphs[i]'s nnz values,
 *                   host or device per SC_OUT_DEVICE (caller-owned).
 *   reports       : nullable; count reports. Per graph: ell_global,
 *                   ell_min/max_source, blocks, source_hops, foster_sum,
 *                   lambda_star, uncertified; launches, hops, hop_launches,
 *                   bytes, times, extension_rounds and edges_extended hold
 *                   the batch totals in every report.
 * Errors: SC_ERR_UNSUPPORTED for TGT+, a bipartite graph under SC_ELL_GLOBAL
 * without an override, or under SC_ELL_LEARNED without the end-corrected
 * estimator; SC_ERR_INVALID_ARG for NULL inputs, mixed devices, negative
 * lengths, a learned batch with a graph that has no model or a bipartite
 * graph without an odd cap >= 3, or a union of 2^31 nodes or entries;
 * SC_ERR_OOM / SC_ERR_CUDA as elsewhere. Outputs are unspecified on error.
 */
sc_status sc_batch_all_edges(sc_graph *const *graphs, int32_t count, const sc_options *opts,
                             const int32_t *ell_per_graph, double *const *s_hat, sc_report *reports);

/* ---- learned per-source length (step A8; the paper has no learned part) --- */

#define SC_MLP_FEATURES 6
#define SC_MLP_HIDDEN 32
/* flat float parameters: W1[32][6], b1[32], W2[32][32], b2[32], W3[32], b3[1] */
#define SC_MLP_PARAMS 1313
/* a model = the parameters followed by the 6 feature means and 6 standard deviations */
#define SC_MLP_MODEL_FLOATS (SC_MLP_PARAMS + 2 * SC_MLP_FEATURES)

/*
 * sc_source_features -- the model's inputs for every node, host float[n * 6],
 * each local and independent of the graph's size: log d_i, log min_{j in N(i)} d_j,
 * local clustering, log((sum_{j in N(i)} d_j / d_i) / (2m / n)) (mean neighbour
 * degree over the mean degree), p_2(i,i) = (1/d_i) sum_{j in N(i)} 1/d_j, and
 * p_3(i,i) = (1/d_i) sum over the triangles (i, j, k) of 1/(d_j d_k).
 */
sc_status sc_source_features(sc_graph *g, float *features);

/*
 * sc_certified_lengths -- per entry the least odd tau whose a-posteriori bound
 * lambda*^2 / (1 - lambda*^2) * (t_{tau-1}(e) + t_tau(e)) is at most eps, where
 * t_l(e) is the hop-l term of Eq. (2) (the bound follows from the mode
 * expansion in the proof of Theorem 3.2); the a-priori length of Eq. (6) when
 * none below it passes. per_entry: host int32[nnz]; per_source (nullable):
 * host int32[n], the maximum over the row (the training label); cap
 * (nullable): the a-priori length. Traverses every source to the cap with all
 * hop terms recorded (8 (cap + 1) nnz bytes of device scratch).
 */
sc_status sc_certified_lengths(sc_graph *g, double eps, int32_t precision, int32_t *per_entry, int32_t *per_source,
                               int32_t *cap);

/*
 * sc_estimated_lengths -- the training labels and acceptance rule of the
 * learned length on a bipartite graph, where lambda* = 1 leaves neither the
 * bound above nor an a-priori length. With the end-corrected estimator the
 * remainder past odd tau is sum_k c_k lambda_k^(tau+1) (1 + lambda_k) /
 * (2 (1 - lambda_k)) >= 0 (mode expansion in the proof of Theorem 3.2, the
 * lambda = -1 mode removed exactly), and the pair sums q_e(tau) = t_{tau+1}(e)
 * + t_{tau+2}(e) >= 0 decay slowly (diffusively on a lattice). The estimate
 * fits q_e(x) = C x^-p through q_e(tau - 2) and q_e(tau) at x = tau - 1, tau + 1
 * and integrates the fitted pair sums past tau (half a unit of x per hop):
 *     p   = ln(q_e(tau - 2) / q_e(tau)) / ln((tau + 1) / (tau - 1)),
 *     est = q_e(tau) (tau + 1) ((tau + 1) / tau)^(p - 1) / (2 (p - 1)),
 * 0 when q_e(tau) <= 0, +inf when tau < 3, q_e(tau - 2) <= 0 or p <= 1. It is
 * an estimate, not a bound (no certificate exists at lambda* = 1). per_entry:
 * host int32[nnz], the least odd tau in [3, cap] whose estimate is at most
 * eps, else cap; per_source (nullable): host int32[n], the row maxima.
 * Traverses every source to cap + 2 with all hop terms recorded
 * (8 (cap + 3) nnz bytes of device scratch).
 * Errors: SC_ERR_INVALID_ARG (null, eps outside (0, 1), cap < 3),
 * SC_ERR_UNSUPPORTED (the graph is not bipartite: use sc_certified_lengths).
 */
sc_status sc_estimated_lengths(sc_graph *g, double eps, int32_t precision, int32_t cap, int32_t *per_entry,
                               int32_t *per_source);

typedef struct sc_mlp_train_opts {
    int32_t epochs;       /* full-batch Adam steps */
    float lr;             /* learning rate */
    float beta1, beta2, adam_eps;  /* 0 = 0.9, 0.999, 1e-8 */
    int32_t precision;    /* block precision used for the labels */
    double eps;           /* accuracy the labels certify */
    int32_t ell_cap;      /* bipartite training graphs: the cap of sc_estimated_lengths (>= 3) */
    int32_t reserved;
} sc_mlp_train_opts;

/*
 * sc_mlp_train -- builds the training set from `graphs` (features and log of
 * the certified per-source lengths; sc_estimated_lengths on a bipartite
 * graph), standardises the features, and trains the MLP on the device (loss:
 * mean (y - log L*)^2 / 2; full-batch Adam). A feature constant over the
 * training set (such as the clustering of a lattice) carries no information:
 * its first-layer weights are set to zero, which leaves the training
 * unchanged (its standardised input is 0) and makes the model ignore it on
 * other graphs.
 *   init_params : host float[SC_MLP_PARAMS], the starting weights (caller's choice)
 *   model_out   : host float[SC_MLP_MODEL_FLOATS]
 *   loss_curve  : host float[epochs], nullable: the loss before each step
 * Work runs on the stream of graphs[0].
 */
sc_status sc_mlp_train(sc_graph *const *graphs, int32_t count, const sc_mlp_train_opts *opts,
                       const float *init_params, float *model_out, float *loss_curve);

/* sc_mlp_load -- copies a model (host float[SC_MLP_MODEL_FLOATS]) into the graph for SC_ELL_LEARNED */
sc_status sc_mlp_load(sc_graph *g, const float *model);

/* sc_mlp_predict -- the per-source lengths the loaded model gives (host int32[n]),
 * the smallest odd integer >= exp(output) - 1/4, clipped to [1, cap] */
sc_status sc_mlp_predict(sc_graph *g, int32_t cap, int32_t *lengths);

/*
 * sc_mlp_loss_grad -- one evaluation of the training loss and its gradient on
 * host data (features host float[count * 6], targets host float[count]);
 * model as for sc_mlp_load. loss: host float; grad: host float[SC_MLP_PARAMS].
 */
sc_status sc_mlp_loss_grad(const float *model, const float *features, const float *targets, int32_t count,
                           float *loss, float *grad, void *stream);

/* ---- allocation-free variant ---------------------------------------------- */

/* size of the file-scope device array that sc_all_edges_noalloc works in */
#define SC_NOALLOC_SCRATCH_BYTES (64u << 20)

/*
 * sc_all_edges_noalloc -- the all-edges traversal without any device
 * allocation. The paper has no counterpart: this is an entry point for
 * callers that cannot call cudaMalloc -- code running under a memory manager
 * that owns the whole device budget (a serving arena, a framework's caching
 * allocator), latency-critical paths where cudaMalloc / cudaFree would block
 * or synchronise the device, and embedders that must not hit out-of-memory
 * mid-run.
 *
 * Computes what sc_all_edges computes with SC_ELL_FIXED (length `ell` for
 * every edge), SC_PREC_FP64, block width 32 and the plain estimator, with
 * every work buffer carved from one static device array of
 * SC_NOALLOC_SCRATCH_BYTES (64 MiB) that each GPU loading the library holds
 * until the process exits.
 *
 *   n, nnz           : graph size; the call needs about 524 n + 16 nnz bytes of
 *                      scratch and fails with SC_ERR_INVALID_ARG above the limit
 *                      (no partial work is done)
 *   row_ptr, col_idx : device pointers to the symmetric CSR (validated as by
 *                      sc_graph_create, except connectivity)
 *   ell              : truncation length >= 0
 *   s_hat            : device double[nnz] output
 *   stream           : cudaStream_t (NULL = default); the call returns after its work
 *
 * Calls no cudaMalloc, cudaFree or other allocating routine. All calls share
 * the one array and it keeps the previous call's contents; each call clears
 * what must start at zero itself. Calls that overlap on the GPU (two streams
 * or two host threads at once) race on the array: serialise them. The first
 * call in each CUDA context looks up the array's device address
 * (cudaGetSymbolAddress with that context's device current) and caches it
 * under the context's unique id; make that first call before any stream
 * capture. After a device reset the next call looks the address up again.
 */
sc_status sc_all_edges_noalloc(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                               int32_t ell, double *s_hat, void *stream);

/* ---- self-test -------------------------------------------------------------- */
/* sc_selftest_bounded_waits -- the library's bounded device waits giving up as
 * designed (no fault and no hang): a wait on an mbarrier phase that never
 * completes (the wait the TMA hop kernel uses for its row gathers) and a spin
 * on a device flag that is never set, each limited to limit_us microseconds
 * (1 .. 1,000,000), on the current device's default stream.
 * Returns SC_ERR_TIMEOUT when both gave up and reported it through their
 * status word (the expected outcome; the CUDA context stays usable),
 * SC_ERR_CUDA if one did not, SC_ERR_INVALID_ARG for a limit out of range. */
sc_status sc_selftest_bounded_waits(uint32_t limit_us);

/* ---- status --------------------------------------------------------------- */
const char *sc_status_string(sc_status s);
const char *sc_last_error_detail(void);
int32_t sc_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SC_H_ */

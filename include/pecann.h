/*
 * pecann.h -- C ABI of the GB300 density-peaks-clustering library.
 *
 * The library runs the data-parallel path of PECANN's density peaks
 * clustering (DPC) on one GPU: batched greedy beam search (Algorithm 1) over a
 * fixed-degree Vamana graph, used to build the graph (Sec. 3.2), to find each
 * point's k nearest neighbours and density (Algorithm 2 lines 2-4, Sec. 4.2),
 * and to find dependent points with doubling beam-width rounds (Algorithm 3);
 * then noise / center / union-find cut the dependent forest into clusters
 * (Algorithm 2 lines 5-7).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* and every array argument not marked "host" are DEVICE
 *    pointers. The caller owns all memory; the library never allocates,
 *    frees or keeps a pointer after the call returns.
 *  - `ws` is a caller-provided device workspace of `ws_bytes` bytes, 256-byte
 *    aligned, of at least pecann_workspace_size() bytes. Its contents on entry
 *    do not matter; on return they are undefined.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is
 *    queued on it. pecann_search, pecann_build_graph, pecann_build_nndescent,
 *    pecann_build_hcnng, pecann_density, pecann_density_noalloc and
 *    pecann_dependent_points return only after their work on `stream` has
 *    finished (they read back an error word or small counters); the other
 *    calls are asynchronous unless a host output is requested.
 *  - Errors are returned as pecann_status; nothing is thrown across the ABI.
 *    PECANN_EINVAL: an argument is out of range (checked on the host before
 *    any GPU work); PECANN_ENOMEM: ws_bytes is too small; PECANN_ECUDA: a
 *    CUDA call failed (the message is available from pecann_last_error());
 *    PECANN_EUNSUPPORTED: a valid combination this build has no kernel for;
 *    PECANN_EINTERNAL: a kernel detected an inconsistency (e.g. a graph entry
 *    out of range) and skipped the offending access. PECANN_ETIMEOUT: a
 *    brute-force screen (PECANN_INDEX_BRUTE_FORCE) gave up waiting on one of
 *    its own pipeline barriers after 2 s; every kernel thread stops, frees
 *    its tensor memory and returns, so the context stays usable. No other
 *    kernel waits on another (the batched form's work queue is a
 *    fetch-and-add counter).
 *  - Point rows are n x d, row-major, contiguous, 16-byte aligned. d must be
 *    a multiple of 4 (FP32), 8 (BF16) or 16 (U8, FP8). U8 supports the L2
 *    metric with d <= 256 (so that every distance is an exact integer in FP32).
 *    Speed only: U8 rows of 128 bytes on a 32-byte aligned base (as torch
 *    allocates) are scored with one 32-byte load per lane; other bases take
 *    a 16-byte layout with the same results.
 *  - Reduced-precision traversal: a BF16 or FP8 dataset must also give
 *    data_f32, the same points in FP32. Graph searches walk the BF16 / FP8
 *    rows (FP32 accumulation); every distance that leaves the library (k-NN lists,
 *    densities, dependent distances) is recomputed exactly on the FP32 rows
 *    for the candidates the traversal found: the k-NN search hands its
 *    rerank_k best points, each dependent round its first 32 points ranked
 *    above the query. Graph builds, brute-force fallbacks and the
 *    brute-force tail use the FP32 rows.
 *  - FP8 (e4m3) rows hold codes of x_j / s_j with per-dimension scales
 *    dim_scale (d floats, 16-byte aligned; e.g. s_j = max_i |x_ij| / 448, the
 *    largest e4m3 value), so the decoded point is x_j = s_j * code_j. FP8
 *    traversal supports the IP metric (the scale folds into the query: the
 *    traversal scores 1 - sum_j (q_j s_j) code_j with q from data_f32, d up
 *    to 1024); L2 on FP8 rows returns PECANN_EUNSUPPORTED.
 *  - Distances: the library orders points by the FP32 "dissimilarity" dis --
 *    the squared Euclidean distance (L2) or 1 - <x, y> (IP, unit-norm rows) --
 *    summed in one fixed order: 4-element chunk c of a row is accumulated with
 *    fmaf into partial c mod 32, chunks in ascending order, then the 32
 *    partials are combined by an xor butterfly (offsets 16, 8, 4, 2, 1).
 *    Reported distances D are sqrt(dis) for L2 and dis for IP. Ties are
 *    broken by the smaller id everywhere.
 *  - Graphs are n x R int32 out-neighbour lists, -1 padded; all ids < n.
 */
#ifndef PECANN_H
#define PECANN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PECANN_API __attribute__((visibility("default")))
#else
#define PECANN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PECANN_OK = 0,
  PECANN_EINVAL = 1,
  PECANN_ENOMEM = 2,
  PECANN_ECUDA = 3,
  PECANN_ETIMEOUT = 4,
  PECANN_EUNSUPPORTED = 5,
  PECANN_EINTERNAL = 6
} pecann_status;

typedef enum { PECANN_F32 = 0, PECANN_U8 = 1, PECANN_BF16 = 2, PECANN_FP8E4M3 = 3 } pecann_dtype;
typedef enum { PECANN_L2 = 0, PECANN_IP = 1 } pecann_metric;

/* Density functions (Sec. 4.2 and Appendix A). */
typedef enum {
  PECANN_DENS_KTH = 0,    /* rho = 1 / D(x_i, k-th neighbour)            */
  PECANN_DENS_EXPSUM = 1, /* rho = exp(-sum_j D^2 / k); ranked by exponent */
  PECANN_DENS_SUMEXP = 2, /* rho = sum_j exp(-D^2) / k                    */
  PECANN_DENS_SUM = 3     /* rho = -sum_j D                               */
} pecann_density_fn;

/* Center functions (Sec. 4.2; local: Appendix, center functions). */
typedef enum {
  PECANN_CENTER_THRESHOLD = 0, /* delta_i > delta_min                   */
  PECANN_CENTER_PRODUCT = 1,   /* the n_clusters largest delta_i * rho_i  */
  PECANN_CENTER_LOCAL = 2      /* i ranks above each of its k neighbours
                                  (pecann_cluster_sweep only)            */
} pecann_center_fn;

/* k-NN index of the density and dependent-point searches (Sec. 5.1). */
typedef enum {
  PECANN_INDEX_GRAPH = 0,      /* greedy beam search (Algorithm 1) on the given graph        */
  PECANN_INDEX_BRUTE_FORCE = 1 /* no index: exact k-NN and dependent points over all points,
                                  screened on the tensor cores (BF16 rows, FP32 accumulation)
                                  and decided exactly on the canonical distance; IP or L2,
                                  d a multiple of 8, k <= 63                               */
} pecann_index;

/* Parameters of the method. pecann_params_default() fills the paper's
   defaults; every field is read by the calls named beside it. */
typedef struct {
  int32_t k;                 /* neighbours per point (density)            density, dependent */
  int32_t R;                 /* graph degree bound                         all graph calls    */
  int32_t L_build;           /* beam width of the build searches           build              */
  int32_t L_search;          /* beam width of the k-NN searches            density            */
  int32_t L_dep;             /* initial k_dep of the doubling rounds (L_d) dependent          */
  float alpha;               /* RobustPrune slack, >= 1                    build              */
  int32_t n_start;           /* sampled start points, 1..min(n, 65536)     build              */
  float batch_frac;          /* batch size cap as a fraction of n (0.02)   build              */
  int32_t visit_cap;         /* closest visited points kept per build search (0: 2*L_build)   */
  int32_t dep_threshold;     /* doubling continues while > this many are unfinished (300)     */
  int32_t max_dep_rounds;    /* cap on doubling rounds                     dependent          */
  int32_t max_dep_beam;      /* largest k_dep searched on the graph (<= 8192) dependent       */
  int32_t density;           /* pecann_density_fn                          density            */
  int32_t normalize_density; /* rho'_i = rho_i k / sum_{j in N_i} rho_j    density            */
  int32_t center;            /* pecann_center_fn                           cluster            */
  float rho_min;             /* noise: rho_i < rho_min                     cluster            */
  float delta_min;           /* threshold center                          cluster            */
  int32_t n_clusters;        /* product center                            cluster            */
  int32_t hash_slots;        /* per-query seen-filter slots (power of 2; 0 = automatic)      */
  int32_t collect_work;      /* != 0: pecann_search / pecann_density leave the sums of
                                expansions and of distance evaluations as two int64 at
                                byte offset 80 of the workspace                          */
  int32_t build_passes;      /* 1, or 2: a first insertion pass pruning with alpha = 1,
                                then a second over all points with alpha   build              */
  int32_t rerank_k;          /* BF16 traversal: candidates per point re-scored in FP32
                                (0: min(L_search, 4k); must be >= k)         density          */
  int32_t block_warps;       /* warps per block of the search kernel (1, 2, 4 or 8; 0 =
                                automatic); with the brute-force index, the k-NN screen's
                                CTAs per cluster: 1, 2 (CTA pairs sharing one 256-row MMA)
                                or 4 (point tiles multicast); 0 = automatic (2 for
                                d >= 512, else 1). Like
                                hash_slots it changes speed, never results                 */
  int32_t index;             /* PECANN_INDEX_GRAPH (the Vamana graph given to the call) or
                                PECANN_INDEX_BRUTE_FORCE (no index, exact; the graph may be
                                NULL)                                      density, dependent */
  uint64_t seed;             /* insertion order when none is given         build              */
} pecann_params;

/* A point set. */
typedef struct {
  const void* data;       /* device, n x d row-major rows of `dtype`            */
  int64_t n;              /* number of points, 2 <= n < 2^31                     */
  int32_t d;              /* dimensions                                          */
  int32_t dtype;          /* pecann_dtype                                        */
  int32_t metric;         /* pecann_metric                                       */
  int32_t reserved0;
  const float* dim_scale; /* FP8 only: device, d per-dimension scales
                             (decoded x_j = dim_scale[j] * code_j)               */
  const float* data_f32;  /* BF16/FP8 only: device n x d FP32 rows for the exact
                             re-rank; NULL for FP32/U8 data                      */
} pecann_dataset;

/* Fills the defaults: k 16, R 32, L_build 64, L_search 64, L_dep 64,
   alpha 1.1, n_start 16, batch_frac 0.02, visit_cap 0, dep_threshold 300,
   max_dep_rounds 30, max_dep_beam 8192, kth density, no normalisation,
   product center, rho_min 0, delta_min 0, n_clusters 1, hash_slots 0,
   collect_work 0, build_passes 1, rerank_k 0, block_warps 0, seed 0. */
PECANN_API void pecann_params_default(pecann_params* p);

/* Static string for a status code. */
PECANN_API const char* pecann_status_string(int status);

/* Text of the last CUDA or validation error seen by this thread ("" if none). */
PECANN_API const char* pecann_last_error(void);

/* Library version, as major*10000 + minor*100 + patch. */
PECANN_API int32_t pecann_version(void);

/* Number of CUDA kernels this library has launched in this process (all
   threads, all devices). Lets a caller count the kernels of a call. */
PECANN_API int64_t pecann_kernel_launches(void);

/* Workspace bytes that are enough for every call below on this dataset and
   these parameters (host call; no GPU work). */
PECANN_API pecann_status pecann_workspace_size(const pecann_dataset* ds, const pecann_params* p, size_t* bytes);

/*
 * Greedy beam search, Algorithm 1, for m query points of the dataset.
 * Query q = d_queries[i] starts from the set {q} (its out-neighbours are the
 * first candidates) when d_start is NULL, else from the n_start (<= 65536)
 * ids of d_start, all of which enter the beam before the first prune keeps
 * the L closest; a query that is one of them is expanded first. The query
 * itself never occupies a beam slot and is never returned.
 * Beam width L (1 <= L <= 8192), result size k (1 <= k <= L).
 * Output per query i: d_ids[i*k .. i*k+k) and d_dis[...] -- the min(k, |beam|)
 * closest points found, ascending by (dis, id), -1 / +inf padded -- and
 * d_count[i] = number of valid entries. dis is the ordering value.
 */
PECANN_API pecann_status pecann_search(const pecann_dataset* ds, const int32_t* d_graph, int32_t R,
                            const int32_t* d_queries, int64_t m, const int32_t* d_start,
                            int32_t n_start, int32_t L, int32_t k, int32_t* d_ids, float* d_dis,
                            int32_t* d_count, const pecann_params* p, void* ws, size_t ws_bytes,
                            void* stream);

/*
 * Vamana graph construction by batched insertion (Sec. 3.2, Sec. 4.1).
 * Points are inserted in the order d_order (device, a permutation of
 * 0..n-1), or, if d_order is NULL, in a permutation drawn from p->seed. The
 * first p->n_start points of the order are the start points of every build
 * search. Batches hold 1, 2, 4, ... points, capped at ceil(batch_frac * n);
 * every search of a batch sees the graph as it stood at the batch start. Each
 * inserted point p gets RobustPrune(p, V_p u N_out(p), alpha, R) where V_p are
 * the visit_cap closest points its search visited; then each new edge p -> y
 * adds p to y, re-pruning y when its degree would exceed R.
 * Output: d_graph (n x R int32, -1 padded) and, if not NULL, d_degree (n).
 * Blocks until done.
 */
PECANN_API pecann_status pecann_build_graph(const pecann_dataset* ds, const pecann_params* p,
                                 const int32_t* d_order, int32_t* d_graph, int32_t* d_degree,
                                 void* ws, size_t ws_bytes, void* stream);

/*
 * NN-Descent graph index (Sec. 5.1, graph indices: the framework also builds
 * its graph with PyNNDescent, repeated num_repeats times). The paper prints
 * no steps for it; the library follows NN-Descent (Dong, Charikar and Li,
 * 2011) in a synchronous form, so that results do not depend on thread
 * order:
 *   for each repeat r: N(u) <- the K ids d_init[r][u] sorted by (dis, id);
 *     each round, from one snapshot of every list:
 *       R(x) <- the K smallest (dis(q, x), q) over the q with x in N(q);
 *       C(x) <- N(x) u R(x);
 *       N'(u) <- the K smallest (dis, id) of N(u) u C(u) u U_{p in C(u)} C(p),
 *                u itself left out;
 *     until no list changes or after `rounds` rounds;
 *   the repeats are merged: N(u) <- the K smallest of the union of their lists;
 *   G(u) <- RobustPrune(u, N(u), alpha, R); then every edge u -> y adds u to
 *   y as the reverse step of pecann_build_graph does for one batch holding
 *   all points (sources in id order; y re-pruned when its degree would
 *   exceed R).
 * d_init: repeats x n x K int32, each list K distinct ids in [0, n) other
 * than its point (a list that breaks this is reported as PECANN_EINTERNAL).
 * 1 <= K <= min(64, n - 1), 1 <= repeats <= 64, 0 <= rounds <= 1000; reads
 * p->R and p->alpha. FP32 (or uint8) rows: BF16 / FP8 datasets use data_f32.
 * Outputs: d_graph (n x R, -1 padded); d_degree (n, may be NULL); d_knn
 * (device n x K, may be NULL): the merged lists, ascending by (dis, id);
 * h_changes (HOST, repeats x rounds int64, may be NULL): how many lists each
 * round changed (0 for rounds not run after convergence). Blocks until done.
 */
PECANN_API pecann_status pecann_nndescent_workspace_size(const pecann_dataset* ds, const pecann_params* p,
                                                         int32_t K, int32_t repeats, size_t* bytes);
PECANN_API pecann_status pecann_build_nndescent(const pecann_dataset* ds, const pecann_params* p, int32_t K,
                                                int32_t repeats, const int32_t* d_init, int32_t rounds,
                                                int32_t* d_graph, int32_t* d_degree, int32_t* d_knn,
                                                int64_t* h_changes, void* ws, size_t ws_bytes, void* stream);

/*
 * HCNNG graph index (Sec. 5.1, graph indices: the framework also takes HCNNG
 * graphs, repeated num_repeats times and pruned with alpha; the paper prints
 * no steps). The library follows the outline of Munoz et al.'s HCNNG in a
 * deterministic form:
 *   for each repeat t: split the points hierarchically. A node [b, b + m) of
 *     the current order (initially 0..n-1) with more than leaf_size points
 *     draws two pivots p1 != p2 among its points: p1 is its (d0 mod m)-th
 *     point, p2 the (d1 mod (m - 1))-th of the others, where d_j =
 *     S(S(S(S(seed + t) + b) + m) + j) and S(x) is the SplitMix64 output for
 *     the state x (Steele, Lea and Flood 2014). Points with
 *     dis(x, p1) <= dis(x, p2) go left, the rest right, each side keeping its
 *     order; a split that leaves a side empty cuts the node at ceil(m / 2).
 *     In every leaf, a minimum spanning forest with degrees at most mst_deg:
 *     the leaf's pairs in (dis, smaller id, larger id) order, each taken when
 *     it joins two components and both ends have degree below mst_deg;
 *   C(u) = u's neighbours in the forests of all repeats;
 *   G(u) = RobustPrune(u, C(u), alpha, R) (no reverse-edge step).
 * 1 <= repeats <= 64, 2 <= leaf_size <= 200 (a leaf's pair keys are sorted
 * in shared memory), 1 <= mst_deg <= 16; reads p->R, p->alpha and p->seed.
 * FP32 (or uint8) rows: BF16 / FP8 datasets use data_f32.
 * Outputs: d_graph (n x R, -1 padded); d_degree (n, may be NULL); h_leaves
 * (HOST, repeats int64, may be NULL): the number of leaves of each repeat.
 * Blocks until done.
 */
PECANN_API pecann_status pecann_hcnng_workspace_size(const pecann_dataset* ds, const pecann_params* p,
                                                     int32_t repeats, int32_t leaf_size, int32_t mst_deg,
                                                     size_t* bytes);
PECANN_API pecann_status pecann_build_hcnng(const pecann_dataset* ds, const pecann_params* p, int32_t repeats,
                                            int32_t leaf_size, int32_t mst_deg, int32_t* d_graph,
                                            int32_t* d_degree, int64_t* h_leaves, void* ws, size_t ws_bytes,
                                            void* stream);

/*
 * k nearest neighbours and density of every point (Algorithm 2 lines 2-4).
 * N_i = the k closest points returned by Algorithm 1 for x_i with start set
 * {x_i} and beam width L_search; where the search returns fewer than k points
 * N_i is computed exactly by brute force (Sec. 4.1).
 * Outputs: d_knn_ids (n x k int32) and d_knn_dist (n x k float, reported
 * distances D), ascending by (dis, id); d_density (n, rho); d_rank_key (n):
 * the value points are ranked by -- rho, or the exponent -sum(D^2)/k for the
 * exp-sum density. Point j ranks above i iff key_j > key_i, or the keys are
 * equal and j < i (Sec. 3: ties broken by id).
 * Blocks until done: the call ends by reading the kernels' error word, and
 * returns PECANN_EINTERNAL when a search met a graph entry >= n (the entry
 * is skipped, never read through; the outputs are then unspecified).
 */
PECANN_API pecann_status pecann_density(const pecann_dataset* ds, const int32_t* d_graph,
                             const pecann_params* p, int32_t* d_knn_ids, float* d_knn_dist,
                             float* d_density, float* d_rank_key, void* ws, size_t ws_bytes,
                             void* stream);

/*
 * Dependent points, Algorithm 3 (ComputeDepPts). d_rank_key, d_knn_ids and
 * d_knn_dist are the outputs of pecann_density. Round 0: lambda_i = the
 * first point of N_i ranked above x_i. Then, while more than dep_threshold
 * points are unfinished (the maximum-rank point excluded), each unfinished
 * point runs Algorithm 1 with beam width and result size k_dep (L_dep,
 * doubling every round) and takes the closest returned point ranked above it.
 * Doubling stops after max_dep_rounds rounds or when k_dep would exceed
 * max_dep_beam; the rest is finished exactly by brute force over all points.
 * Outputs: d_dep (n, -1 for the maximum-rank point) and d_dep_dist (n, D to
 * the dependent point, +inf where there is none). If h_stats (HOST, 64
 * int64) is not NULL: [0] rounds run, [1] unfinished after round 0, [2+r]
 * unfinished after round r, [63] points finished by brute force.
 * Blocks until done.
 */
PECANN_API pecann_status pecann_dependent_points(const pecann_dataset* ds, const int32_t* d_graph,
                                      const pecann_params* p, const float* d_rank_key,
                                      const int32_t* d_knn_ids, const float* d_knn_dist,
                                      int32_t* d_dep, float* d_dep_dist, int64_t* h_stats,
                                      void* ws, size_t ws_bytes, void* stream);

/*
 * Clusters (Algorithm 2 lines 5-7). Noise: rho_i < rho_min. Centers among the
 * other points: delta_i > delta_min (threshold) or the n_clusters largest
 * delta_i * rho_i (product; ties by smaller id, 0 * inf taken as 0). Every
 * point that is neither noise nor a center and has a dependent point joins
 * its dependent point's cluster (union-find); d_labels[i] = the id of the
 * root of i's tree in the cut dependent forest, i.e. the cluster's center,
 * the noise point itself, or the maximum-rank point.
 * If h_n_clusters (HOST) is not NULL it receives the number of clusters
 * (the call then waits for the stream).
 */
PECANN_API pecann_status pecann_cluster(int64_t n, const float* d_density, const int32_t* d_dep,
                             const float* d_dep_dist, const pecann_params* p, int32_t* d_labels,
                             int64_t* h_n_clusters, void* ws, size_t ws_bytes, void* stream);

/* One clustering of a sweep: center function and its parameters. */
typedef struct {
  int32_t center;     /* pecann_center_fn                                     */
  float rho_min;      /* noise: rho_i < rho_min                               */
  float delta_min;    /* threshold center                                     */
  int32_t n_clusters; /* product center (>= 1)                                */
} pecann_cluster_setting;

/*
 * Many clusterings from one dependent forest (Sec. 1: the dependent-point
 * tree is a cluster hierarchy, and other clusterings come from re-running only
 * the last step with other pruning settings; Appendix, varying number of
 * clusters). For every setting s of the
 * HOST array h_settings[0 .. n_settings), the rules of pecann_cluster apply
 * and d_labels[s * n .. s * n + n) receives its labels. The local center
 * (PECANN_CENTER_LOCAL) marks as centers the non-noise points that rank
 * above each of their k nearest neighbours (the n x k d_knn_ids of
 * pecann_density, -1 entries ignored; rank by d_rank_key, ties to the smaller
 * id); d_knn_ids and d_rank_key may be NULL when no setting uses it.
 * n_settings in 1..4096. All settings run in the same passes: one launch
 * per radix pass of the product-center selection for every product setting,
 * one launch for every setting's parent array, and pointer-jumping sweeps
 * over all n_settings x n entries. If h_n_clusters (HOST, n_settings entries)
 * is not NULL it receives each setting's number of clusters and the call
 * waits for the stream. Workspace: pecann_cluster_workspace_size(n, n_settings),
 * which with n_settings = 1 is also enough for pecann_cluster.
 * Errors: PECANN_EINVAL for a bad setting (unknown center function,
 * n_clusters < 1 with the product center, a local center without k-NN lists)
 * -- checked on the host before any GPU work.
 */
PECANN_API pecann_status pecann_cluster_workspace_size(int64_t n, int32_t n_settings, size_t* bytes);
PECANN_API pecann_status pecann_cluster_sweep(int64_t n, const float* d_density, const int32_t* d_dep,
                                   const float* d_dep_dist, const int32_t* d_knn_ids, int32_t k,
                                   const float* d_rank_key, int32_t n_settings,
                                   const pecann_cluster_setting* h_settings, int32_t* d_labels,
                                   int64_t* h_n_clusters, void* ws, size_t ws_bytes, void* stream);

/*
 * Batched form (many independent FP32 point sets of uneven sizes): the whole
 * path -- k-NN + density, dependent points, clusters -- for every set, with
 * one launch per step for all sets. Every set follows exactly the rules of
 * the single-set calls (its own maximum-rank point, its own doubling test,
 * its own brute-force tail, its own centers).
 * Sets: `sets` (HOST array of n_sets <= 4096) of FP32 datasets with one
 * metric, d <= 1024. Global ids: set s owns ids base[s] .. base[s+1]-1 in
 * set order (base[0] = 0); every per-point array below is concatenated in
 * that order and holds set-local ids (graphs: sum(n) x R, -1 padded; k-NN:
 * sum(n) x k; density, rank key, dep, dep_dist, labels: sum(n)).
 * pecann_batch_workspace_size: bytes of workspace needed (host call).
 * pecann_batch_prepare: writes the set table (row and graph pointers, sizes,
 *   h_n_clusters[s] -- HOST, may be NULL for p->n_clusters) into the
 *   workspace; blocks until done. Call it once per batch; the workspace then
 *   belongs to that batch.
 * pecann_run_batched: one pass of the path over all sets, from the prepared
 *   workspace and the same `sets`. It issues only kernels, device-to-device
 *   copies and memsets on `stream` and reads nothing back to the host, so it
 *   can be captured into a CUDA graph and replayed. The normalised density
 *   is not offered in batched form (PECANN_EINVAL).
 */
PECANN_API pecann_status pecann_batch_workspace_size(int32_t n_sets, const pecann_dataset* sets,
                                                     const pecann_params* p, size_t* bytes);
PECANN_API pecann_status pecann_batch_prepare(int32_t n_sets, const pecann_dataset* sets,
                                              const int32_t* d_graphs, const int32_t* h_n_clusters,
                                              const pecann_params* p, void* ws, size_t ws_bytes,
                                              void* stream);
PECANN_API pecann_status pecann_run_batched(int32_t n_sets, const pecann_dataset* sets,
                                            const pecann_params* p, int32_t* d_knn_ids,
                                            float* d_knn_dist, float* d_density, float* d_rank_key,
                                            int32_t* d_dep, float* d_dep_dist, int32_t* d_labels,
                                            void* ws, size_t ws_bytes, void* stream);

/* Largest point set pecann_density_noalloc accepts. */
#define PECANN_NOALLOC_MAX_POINTS (1 << 20)

/*
 * pecann_density without a workspace, for callers that cannot allocate GPU
 * memory (for example code under an external memory manager that owns every
 * device byte, or a loop that must never take the allocator's lock, since a
 * cudaMalloc can synchronise the device). The paper has no counterpart: this
 * is a packaging of pecann_density, with the same arguments minus the
 * workspace, the same checks and the same results, element for element.
 * Its scratch (about 8 MiB: a fallback list and a density copy for up to
 * PECANN_NOALLOC_MAX_POINTS points) is one fixed device array inside the
 * library, present on every GPU that loads the library until the process
 * exits. The call allocates nothing; n > PECANN_NOALLOC_MAX_POINTS returns
 * PECANN_EINVAL, BF16 / FP8 rows PECANN_EUNSUPPORTED. Every call looks the
 * array's device address up in the current context (cudaGetSymbolAddress);
 * the first call on a device may load the library's device code there, so
 * make it before any stream capture. All calls share the array: calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller. Each call clears what must start at zero; the
 * rest keeps the previous call's contents. Like pecann_density it blocks
 * until done and returns PECANN_EINTERNAL for a graph entry >= n.
 */
PECANN_API pecann_status pecann_density_noalloc(const pecann_dataset* ds, const int32_t* d_graph,
                                                const pecann_params* p, int32_t* d_knn_ids,
                                                float* d_knn_dist, float* d_density,
                                                float* d_rank_key, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PECANN_H */

/*
 * PECANN density-peaks clustering -- CPU ORACLE (test infrastructure only).
 *
 * This file is test infrastructure. Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it. It shares no code with the
 * CUDA library: it is a plain, slow, step-by-step restatement of the paper's
 * algorithms so that the GPU results can be checked against it.
 *
 * What it computes (paper section / algorithm it follows):
 *   orc_dis               canonical FP32 dissimilarity (Sec. 2.1 defines D; the
 *                         summation order is this library's reading, below)
 *   orc_greedy_search     Algorithm 1 (greedy beam search)
 *   orc_knn_density       Algorithm 2 lines 2-4 with the density functions of
 *                         Sec. 4.2 and Appendix A
 *   orc_dependent_points  Algorithm 3 (DPBruteForce + ComputeDepPts with the
 *                         doubling rounds and the brute-force tail of Sec. 3.2)
 *   orc_cluster           Algorithm 2 lines 5-7 (noise, center, union-find)
 *   orc_cluster_local     the same with the local center function (Appendix,
 *                         center functions)
 *   orc_robust_prune      RobustPrune(alpha, R) of Vamana (Sec. 3.2 defers it
 *                         to DiskANN; the published DiskANN rule is used)
 *   orc_build_graph       Vamana batched construction (Sec. 3.2, Sec. 4.1)
 *   orc_nndescent         NN-Descent graph index (Sec. 5.1, graph indices; the
 *                         paper names it without steps: synchronous rounds of
 *                         Dong et al.'s method, see its own comment)
 *   orc_knn_density_rows  Algorithm 2 lines 2-4 for a list of points only
 *   orc_hcnng             HCNNG graph index (Sec. 5.1, graph indices; named
 *                         without steps: random hierarchical splits and
 *                         degree-bounded spanning forests, see its comment)
 *
 * Where the paper leaves a point open, this file takes the readings below:
 *  - Canonical FP32 dissimilarity. For rows a, b of d elements (d % 4 == 0) 32
 *    partial sums s[0..31] start at +0. Chunk c (elements 4c..4c+3) is owned by
 *    partial c % 32; chunks are taken in ascending c and, inside a chunk, in
 *    ascending element order, each step s = fmaf(t, t, s) with t = a - b (L2)
 *    or s = fmaf(a, b, s) (inner product). The 32 partials are then combined
 *    by a butterfly: for off = 16, 8, 4, 2, 1 every s[l] becomes s[l] + s[l^off].
 *    The ordering value "dis" is s[0] for L2 (squared distance) and 1 - s[0]
 *    for the inner-product metric. The reported distance D is sqrtf(dis) for
 *    L2 and dis for the inner product.
 *  - Order of points: (dis, id) lexicographic, smaller id first on equal dis.
 *  - Density rank: j ranks above i iff key_j > key_i or (key_j == key_i and
 *    j < i) (the worked example of Sec. 3 ranks b before c at equal density).
 *  - Algorithm 1: the query never occupies a beam slot. It is placed in the
 *    visited set first; if it belongs to the start set it is expanded first
 *    (this reproduces the worked example of Sec. 3 with k = L = 1). It is never
 *    returned.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_F32 = 0, ORC_U8 = 1 };
enum { ORC_L2 = 0, ORC_IP = 1 };
enum { DENS_KTH = 0, DENS_EXPSUM = 1, DENS_SUMEXP = 2, DENS_SUM = 3 };
enum { CENTER_THRESHOLD = 0, CENTER_PRODUCT = 1, CENTER_LOCAL = 2 };

typedef struct {
  const void* X;  /* n x d row-major */
  int64_t n;
  int32_t d;
  int32_t dtype;  /* ORC_F32 | ORC_U8 */
  int32_t metric; /* ORC_L2 | ORC_IP */
} orc_points;

typedef struct {
  float dis;
  int32_t id;
} item;

static float coord(const orc_points* P, int64_t i, int32_t j) {
  if (P->dtype == ORC_U8) return (float)((const uint8_t*)P->X)[i * P->d + j];
  return ((const float*)P->X)[i * P->d + j];
}

/* Canonical FP32 dissimilarity between rows a and b (see the header). */
float orc_dis(const orc_points* P, int64_t a, int64_t b) {
  float s[32], t[32];
  for (int l = 0; l < 32; l++) s[l] = 0.0f;
  int nchunk = P->d / 4;
  for (int c = 0; c < nchunk; c++) {
    int l = c % 32;
    for (int e = 0; e < 4; e++) {
      int j = 4 * c + e;
      float xa = coord(P, a, j), xb = coord(P, b, j);
      if (P->metric == ORC_L2) {
        float diff = xa - xb;
        s[l] = fmaf(diff, diff, s[l]);
      } else {
        s[l] = fmaf(xa, xb, s[l]);
      }
    }
  }
  for (int off = 16; off >= 1; off >>= 1) {
    for (int l = 0; l < 32; l++) t[l] = s[l] + s[l ^ off];
    for (int l = 0; l < 32; l++) s[l] = t[l];
  }
  return P->metric == ORC_L2 ? s[0] : 1.0f - s[0];
}

/* Reported distance D from the ordering value. */
float orc_out_dist(const orc_points* P, float dis) {
  return P->metric == ORC_L2 ? sqrtf(dis) : dis;
}

static int item_less(item a, item b) {
  return a.dis < b.dis || (a.dis == b.dis && a.id < b.id);
}

static int item_cmp(const void* pa, const void* pb) {
  item a = *(const item*)pa, b = *(const item*)pb;
  if (item_less(a, b)) return -1;
  if (item_less(b, a)) return 1;
  return 0;
}

/* j ranks above i under (key desc, id asc). */
static int ranks_above(const float* key, int64_t j, int64_t i) {
  return key[j] > key[i] || (key[j] == key[i] && j < i);
}

/* ---------- a tiny parallel-for over [0, n) with pthreads ---------- */
typedef void (*body_fn)(void* ctx, int64_t i, int tid);
typedef struct {
  body_fn fn;
  void* ctx;
  int64_t n;
  int64_t next;
  pthread_mutex_t mu;
  int tid;
} pfor_state;
typedef struct {
  pfor_state* st;
  int tid;
} pfor_arg;

static void* pfor_worker(void* p) {
  pfor_arg* a = (pfor_arg*)p;
  pfor_state* st = a->st;
  for (;;) {
    pthread_mutex_lock(&st->mu);
    int64_t i0 = st->next;
    st->next += 16;
    pthread_mutex_unlock(&st->mu);
    if (i0 >= st->n) break;
    int64_t i1 = i0 + 16 < st->n ? i0 + 16 : st->n;
    for (int64_t i = i0; i < i1; i++) st->fn(st->ctx, i, a->tid);
  }
  return NULL;
}

static void parallel_for(int64_t n, int nthreads, body_fn fn, void* ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads == 1 || n < 32) {
    for (int64_t i = 0; i < n; i++) fn(ctx, i, 0);
    return;
  }
  pfor_state st;
  st.fn = fn;
  st.ctx = ctx;
  st.n = n;
  st.next = 0;
  pthread_mutex_init(&st.mu, NULL);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  pfor_arg* args = (pfor_arg*)malloc(sizeof(pfor_arg) * nthreads);
  for (int t = 0; t < nthreads; t++) {
    args[t].st = &st;
    args[t].tid = t;
    pthread_create(&th[t], NULL, pfor_worker, &args[t]);
  }
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&st.mu);
  free(th);
  free(args);
}

/* ---------- Algorithm 1: greedy beam search ---------- */

/* Per-thread scratch. Membership of L and V is kept with stamps so that a
   search costs O(|L| + |V|) memory traffic instead of O(n). */
typedef struct {
  int64_t n;
  int32_t* in_beam; /* == stamp iff the point is in L */
  int32_t* in_vis;  /* == stamp iff the point is in V */
  int32_t* in_seen; /* == stamp iff D(x_q, point) was computed in this search */
  int64_t n_exp;    /* expansions of the last search (|V| without the query) */
  int64_t n_eval;   /* distinct points whose distance the last search computed */
  int32_t stamp;
  item* beam;
  int64_t beam_cap;
  item* vis;
  int64_t vis_cap;
  item* tmp;
  int64_t tmp_cap;
} search_ws;

static void ws_init(search_ws* ws, int64_t n) {
  memset(ws, 0, sizeof(*ws));
  ws->n = n;
  ws->in_beam = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  ws->in_vis = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  ws->in_seen = (int32_t*)calloc((size_t)n, sizeof(int32_t));
}

static void ws_free(search_ws* ws) {
  free(ws->in_beam);
  free(ws->in_vis);
  free(ws->in_seen);
  free(ws->beam);
  free(ws->vis);
  free(ws->tmp);
}

static void grow(item** a, int64_t* cap, int64_t need) {
  if (need <= *cap) return;
  int64_t c = *cap ? *cap : 64;
  while (c < need) c *= 2;
  *a = (item*)realloc(*a, (size_t)c * sizeof(item));
  *cap = c;
}

typedef struct {
  const orc_points* P;
  const int32_t* G;
  int32_t R;
  int64_t q;
  search_ws* ws;
  int64_t nb;
} search_state;

/* L <- L u E_out(p), the query itself excluded. */
static void add_out_neighbors(search_state* st, int64_t p) {
  search_ws* ws = st->ws;
  grow(&ws->beam, &ws->beam_cap, st->nb + st->R);
  for (int32_t r = 0; r < st->R; r++) {
    int32_t y = st->G[p * st->R + r];
    if (y < 0 || y == st->q) continue;
    if (ws->in_beam[y] == ws->stamp) continue;
    ws->beam[st->nb].dis = orc_dis(st->P, st->q, y);
    ws->beam[st->nb].id = y;
    st->nb++;
    ws->in_beam[y] = ws->stamp;
    if (ws->in_seen[y] != ws->stamp) {
      ws->in_seen[y] = ws->stamp;
      ws->n_eval++;
    }
  }
}

/* If |L| > Lw keep only the Lw closest points of L. */
static void keep_closest(search_state* st, int32_t Lw) {
  search_ws* ws = st->ws;
  if (st->nb <= Lw) return;
  qsort(ws->beam, (size_t)st->nb, sizeof(item), item_cmp);
  for (int64_t b = Lw; b < st->nb; b++) ws->in_beam[ws->beam[b].id] = 0;
  st->nb = Lw;
}

/*
 * Algorithm 1 (greedy beam search) for the query x_q over graph G (n x R,
 * -1 padded), start set S, beam width Lw.
 * Writes the min(k, |(L u V) minus q|) closest points, sorted by (dis, id), to
 * out and returns that count. If vis_out is given, V minus {q} is returned
 * there as well (unsorted, *nvis_out entries; the caller owns *vis_out).
 */
static int64_t greedy_search(const orc_points* P, const int32_t* G, int32_t R, int64_t q,
                             const int32_t* S, int64_t nS, int32_t Lw, int32_t k,
                             search_ws* ws, item* out, item** vis_out, int64_t* nvis_out) {
  search_state st = {P, G, R, q, ws, 0};
  ws->stamp++;
  ws->n_exp = 0;
  ws->n_eval = 0;
  int64_t nv = 0;
  /* V <- {q}: the query is visited first and never enters the beam. */
  ws->in_vis[q] = ws->stamp;
  /* L <- S */
  int q_in_S = 0;
  grow(&ws->beam, &ws->beam_cap, nS + R + 1);
  for (int64_t s = 0; s < nS; s++) {
    int32_t y = S[s];
    if (y == q) {
      q_in_S = 1;
      continue;
    }
    if (ws->in_beam[y] == ws->stamp) continue;
    ws->beam[st.nb].dis = orc_dis(P, q, y);
    ws->beam[st.nb].id = y;
    st.nb++;
    ws->in_beam[y] = ws->stamp;
    ws->in_seen[y] = ws->stamp;
    ws->n_eval++;
  }
  if (q_in_S) {
    /* the query is the first point popped: its out-neighbours join L */
    add_out_neighbors(&st, q);
    keep_closest(&st, Lw);
  }
  for (;;) {
    /* p* <- argmin over L \ V */
    int64_t best = -1;
    for (int64_t b = 0; b < st.nb; b++) {
      if (ws->in_vis[ws->beam[b].id] == ws->stamp) continue;
      if (best < 0 || item_less(ws->beam[b], ws->beam[best])) best = b;
    }
    if (best < 0) break; /* L \ V is empty */
    item pstar = ws->beam[best];
    add_out_neighbors(&st, pstar.id);       /* L <- L u E_out(p*) */
    ws->in_vis[pstar.id] = ws->stamp;       /* V <- V u {p*} */
    grow(&ws->vis, &ws->vis_cap, nv + 1);
    ws->vis[nv++] = pstar;
    ws->n_exp++;
    keep_closest(&st, Lw);                  /* |L| > Lw: keep the Lw closest */
  }
  /* the k closest points of (L u V) \ {q} */
  grow(&ws->tmp, &ws->tmp_cap, st.nb + nv);
  int64_t m = 0;
  for (int64_t b = 0; b < st.nb; b++) ws->tmp[m++] = ws->beam[b];
  for (int64_t v = 0; v < nv; v++)
    if (ws->in_beam[ws->vis[v].id] != ws->stamp) ws->tmp[m++] = ws->vis[v];
  qsort(ws->tmp, (size_t)m, sizeof(item), item_cmp);
  int64_t cnt = m < k ? m : k;
  if (out)
    for (int64_t t = 0; t < cnt; t++) out[t] = ws->tmp[t];
  if (vis_out) {
    *vis_out = (item*)malloc(sizeof(item) * (size_t)(nv > 0 ? nv : 1));
    memcpy(*vis_out, ws->vis, sizeof(item) * (size_t)nv);
    *nvis_out = nv;
  }
  /* leave the stamp arrays clean for the next search of this thread */
  for (int64_t b = 0; b < st.nb; b++) ws->in_beam[ws->beam[b].id] = 0;
  return cnt;
}

typedef struct {
  const orc_points* P;
  const int32_t* G;
  int32_t R, L;
  const int32_t* queries;
  int64_t* n_exp;
  int64_t* n_eval;
  search_ws* ws;
} count_ctx;

static void count_body(void* c, int64_t u, int tid) {
  count_ctx* x = (count_ctx*)c;
  int32_t q = x->queries[u];
  int32_t S[1] = {q};
  greedy_search(x->P, x->G, x->R, q, S, 1, x->L, 0, &x->ws[tid], NULL, NULL, NULL);
  x->n_exp[u] = x->ws[tid].n_exp;
  x->n_eval[u] = x->ws[tid].n_eval;
}

/* Work of Algorithm 1 per query (start set {x_q}, beam L): expansions
   (out-lists read, the query's own included) and distinct points whose
   distance was computed. These define the algorithmic bytes of a search. */
int orc_search_counts(const orc_points* P, const int32_t* G, int32_t R, int32_t L,
                      const int32_t* queries, int64_t m, int64_t* n_exp, int64_t* n_eval,
                      int nthreads) {
  if (nthreads < 1) nthreads = 1;
  search_ws* ws = (search_ws*)malloc(sizeof(search_ws) * nthreads);
  for (int t = 0; t < nthreads; t++) ws_init(&ws[t], P->n);
  count_ctx c = {P, G, R, L, queries, n_exp, n_eval, ws};
  parallel_for(m, nthreads, count_body, &c);
  for (int u = 0; u < m; u++) n_exp[u] += 1; /* the query's own out-list */
  for (int t = 0; t < nthreads; t++) ws_free(&ws[t]);
  free(ws);
  return 0;
}

/* Exact k nearest points of x_q over P \ {q} by brute force (used where a
   graph search returns fewer than k points, Sec. 4.1). */
static int64_t brute_force_knn(const orc_points* P, int64_t q, int32_t k, item* out) {
  item* all = (item*)malloc(sizeof(item) * (size_t)(P->n > 1 ? P->n - 1 : 1));
  int64_t m = 0;
  for (int64_t j = 0; j < P->n; j++) {
    if (j == q) continue;
    all[m].dis = orc_dis(P, q, j);
    all[m].id = (int32_t)j;
    m++;
  }
  qsort(all, (size_t)m, sizeof(item), item_cmp);
  int64_t cnt = m < k ? m : k;
  for (int64_t t = 0; t < cnt; t++) out[t] = all[t];
  free(all);
  return cnt;
}

/* Public single-query entry (used by the tests): Algorithm 1 with start set S. */
int64_t orc_greedy_search(const orc_points* P, const int32_t* G, int32_t R, int64_t q,
                          const int32_t* S, int64_t nS, int32_t Lw, int32_t k,
                          int32_t* out_ids, float* out_dis, int32_t* vis_ids, float* vis_dis,
                          int64_t vis_cap, int64_t* nvis) {
  search_ws ws;
  ws_init(&ws, P->n);
  item* out = (item*)malloc(sizeof(item) * (size_t)(k > 0 ? k : 1));
  item* vis = NULL;
  int64_t nv = 0;
  int64_t cnt = greedy_search(P, G, R, q, S, nS, Lw, k, &ws, out, &vis, &nv);
  for (int64_t t = 0; t < cnt; t++) {
    out_ids[t] = out[t].id;
    out_dis[t] = out[t].dis;
  }
  if (vis_ids) {
    qsort(vis, (size_t)nv, sizeof(item), item_cmp);
    for (int64_t t = 0; t < nv && t < vis_cap; t++) {
      vis_ids[t] = vis[t].id;
      vis_dis[t] = vis[t].dis;
    }
  }
  if (nvis) *nvis = nv;
  free(vis);
  free(out);
  ws_free(&ws);
  return cnt;
}

/* ---------- Algorithm 2 lines 2-4: k-NN and density ---------- */

/* Density of one point from its sorted k-NN (Sec. 4.2 and Appendix A).
   dis[t] are the ordering values, D[t] the reported distances. The rank key
   is the value points are ranked by: rho itself, except for exp-sum where it
   is the exponent -sum(D^2)/k (exp underflows to 0 long before the exponent
   loses its order). */
static void density_of(const orc_points* P, int32_t fn, int32_t k, const float* dis,
                       const float* D, float* rho, float* key) {
  if (fn == DENS_KTH) {
    /* rho = 1 / D(x_i, furthest point of N_i) */
    *rho = 1.0f / D[k - 1];
    *key = *rho;
  } else if (fn == DENS_EXPSUM) {
    /* rho = exp(-sum_j D(x_i, x_j)^2 / k) */
    float s = 0.0f;
    for (int32_t t = 0; t < k; t++) {
      float d2 = P->metric == ORC_L2 ? dis[t] : D[t] * D[t];
      s = s + d2;
    }
    *key = -s / (float)k;
    *rho = expf(*key);
  } else if (fn == DENS_SUMEXP) {
    /* rho = sum_j exp(-D(x_i, x_j)^2) / k */
    float s = 0.0f;
    for (int32_t t = 0; t < k; t++) {
      float d2 = P->metric == ORC_L2 ? dis[t] : D[t] * D[t];
      s = s + expf(-d2);
    }
    *rho = s / (float)k;
    *key = *rho;
  } else {
    /* sum: rho = -sum_j D(x_i, x_j) */
    float s = 0.0f;
    for (int32_t t = 0; t < k; t++) s = s + D[t];
    *rho = -s;
    *key = *rho;
  }
}

typedef struct {
  const orc_points* P;
  const int32_t* G;
  int32_t R, L, k, fn;
  int32_t* ids;
  float* dist;
  float* rho;
  float* key;
  int32_t* fallback;
  search_ws* ws;
  const int64_t* rows; /* NULL: row u is point u; else the point of output row u */
} knn_ctx;

static void knn_body(void* c, int64_t u, int tid) {
  knn_ctx* x = (knn_ctx*)c;
  int32_t k = x->k;
  const int64_t i = x->rows ? x->rows[u] : u;
  item* out = (item*)malloc(sizeof(item) * (size_t)k);
  int32_t S[1] = {(int32_t)i};
  int64_t cnt;
  if (x->G == NULL) {
    /* no index (Sec. 5.1, brute force): the exact k-NN over P \ {x_i} */
    cnt = brute_force_knn(x->P, i, k, out);
  } else {
    /* N_i <- G.Find-Knn(x_i, k), start set = {x_i} */
    cnt = greedy_search(x->P, x->G, x->R, i, S, 1, x->L, k, &x->ws[tid], out, NULL, NULL);
  }
  if (cnt < k) {
    /* fewer than k points returned: exact k-NN by brute force */
    cnt = brute_force_knn(x->P, i, k, out);
    x->fallback[u] = 1;
  }
  float dis[4096], D[4096];
  for (int32_t t = 0; t < k; t++) {
    x->ids[u * k + t] = out[t].id;
    dis[t] = out[t].dis;
    D[t] = orc_out_dist(x->P, out[t].dis);
    x->dist[u * k + t] = D[t];
  }
  /* rho_i <- F_density(x_i, N_i) */
  density_of(x->P, x->fn, k, dis, D, &x->rho[u], &x->key[u]);
  free(out);
}

/*
 * k-NN of every point on graph G (beam width L, start set {x_i}), followed by
 * its density. G == NULL is the brute-force index of Sec. 5.1: every k-NN is
 * the exact one over P \ {x_i} (L unused). Outputs: ids/dist n x k (sorted by (dis, id)), rho n, key n
 * (rank key), fallback n (1 where the graph search returned < k points).
 * normalize != 0 applies rho'_i = rho_i k / sum_{j in N_i} rho_j (Sec. 4.2).
 * Requires n > k and k <= 4096.
 */
int orc_knn_density(const orc_points* P, const int32_t* G, int32_t R, int32_t L, int32_t k,
                    int32_t fn, int32_t normalize, int32_t* ids, float* dist, float* rho,
                    float* key, int32_t* fallback, int nthreads) {
  if (k < 1 || k > 4096 || P->n <= k) return 1;
  if (nthreads < 1) nthreads = 1;
  search_ws* ws = (search_ws*)malloc(sizeof(search_ws) * nthreads);
  for (int t = 0; t < nthreads; t++) ws_init(&ws[t], P->n);
  memset(fallback, 0, sizeof(int32_t) * (size_t)P->n);
  knn_ctx c = {P, G, R, L, k, fn, ids, dist, rho, key, fallback, ws, NULL};
  parallel_for(P->n, nthreads, knn_body, &c);
  for (int t = 0; t < nthreads; t++) ws_free(&ws[t]);
  free(ws);
  if (normalize) {
    float* raw = (float*)malloc(sizeof(float) * (size_t)P->n);
    memcpy(raw, rho, sizeof(float) * (size_t)P->n);
    for (int64_t i = 0; i < P->n; i++) {
      float s = 0.0f;
      for (int32_t t = 0; t < k; t++) s = s + raw[ids[i * k + t]];
      rho[i] = (raw[i] * (float)k) / s;
      key[i] = rho[i];
    }
    free(raw);
  }
  return 0;
}

/*
 * The k-NN and density of the m listed points only (rows[u] for output row
 * u): the same steps as orc_knn_density (graph G, or G == NULL for the
 * brute-force index), without the normalisation, which needs every point.
 * Used to time the method on a sample of a large point set.
 */
int orc_knn_density_rows(const orc_points* P, const int32_t* G, int32_t R, int32_t L, int32_t k, int32_t fn,
                         const int64_t* rows, int64_t m, int32_t* ids, float* dist, float* rho, float* key,
                         int32_t* fallback, int nthreads) {
  if (k < 1 || k > 4096 || P->n <= k) return 1;
  if (nthreads < 1) nthreads = 1;
  search_ws* ws = (search_ws*)malloc(sizeof(search_ws) * nthreads);
  for (int t = 0; t < nthreads; t++) ws_init(&ws[t], P->n);
  memset(fallback, 0, sizeof(int32_t) * (size_t)m);
  knn_ctx c = {P, G, R, L, k, fn, ids, dist, rho, key, fallback, ws, rows};
  parallel_for(m, nthreads, knn_body, &c);
  for (int t = 0; t < nthreads; t++) ws_free(&ws[t]);
  free(ws);
  return 0;
}

/* ---------- Algorithm 3: dependent points ---------- */

/* DPBruteForce: among the candidates, the closest point ranked above x_i
   (ties by smaller id); -1 if none ranks above x_i. */
static int32_t dp_bruteforce(const orc_points* P, const float* key, int64_t i,
                             const int32_t* cand, int64_t m, float* best_dis) {
  int32_t best = -1;
  float bd = 0.0f;
  for (int64_t t = 0; t < m; t++) {
    int32_t j = cand[t];
    if (j < 0 || j == i) continue;
    if (!ranks_above(key, j, i)) continue; /* par-filter(j: rho_j > rho_i) */
    float dj = orc_dis(P, i, j);           /* par-argmin(j: D(x_i, x_j)) */
    if (best < 0 || dj < bd || (dj == bd && j < best)) {
      best = j;
      bd = dj;
    }
  }
  *best_dis = bd;
  return best;
}

typedef struct {
  const orc_points* P;
  const int32_t* G;
  int32_t R;
  const float* key;
  const int32_t* knn;
  int32_t k;
  const int32_t* U;
  int32_t kdep;
  int32_t* lam;
  float* dis;
  search_ws* ws;
} dep_ctx;

static void dep_round0_body(void* c, int64_t i, int tid) {
  (void)tid;
  dep_ctx* x = (dep_ctx*)c;
  x->lam[i] = dp_bruteforce(x->P, x->key, i, x->knn + i * x->k, x->k, &x->dis[i]);
}

static void dep_round_body(void* c, int64_t u, int tid) {
  dep_ctx* x = (dep_ctx*)c;
  int64_t i = x->U[u];
  item* out = (item*)malloc(sizeof(item) * (size_t)x->kdep);
  int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)x->kdep);
  int32_t S[1] = {(int32_t)i};
  int64_t cnt;
  if (x->G == NULL) {
    /* no index (Sec. 5.1, brute force): FindKnn is the exact k_dep-NN */
    cnt = brute_force_knn(x->P, i, x->kdep, out);
  } else {
    /* N_candidates <- G.FindKnn(i, k_dep): beam width k_dep */
    cnt = greedy_search(x->P, x->G, x->R, i, S, 1, x->kdep, x->kdep, &x->ws[tid], out, NULL, NULL);
  }
  for (int64_t t = 0; t < cnt; t++) cand[t] = out[t].id;
  x->lam[i] = dp_bruteforce(x->P, x->key, i, cand, cnt, &x->dis[i]);
  free(cand);
  free(out);
}

static int32_t* g_all_ids = NULL;

static void dep_tail_body(void* c, int64_t u, int tid) {
  (void)tid;
  dep_ctx* x = (dep_ctx*)c;
  int64_t i = x->U[u];
  /* DPBruteForce(x_i, P) */
  x->lam[i] = dp_bruteforce(x->P, x->key, i, g_all_ids, x->P->n, &x->dis[i]);
}

/*
 * ComputeDepPts (Algorithm 3). key is the rank key of every point, knn the
 * n x k neighbour lists. G == NULL is the brute-force index of Sec. 5.1:
 * FindKnn(i, k_dep) returns the exact k_dep nearest points. Round 0 searches N_i; then, while more than
 * `threshold` points are unfinished, each unfinished point (the global
 * maximum excluded) runs FindKnn with beam width and result size k_dep
 * (k_dep = Ld, doubling each round). The doubling stops early after
 * max_rounds rounds or once k_dep would exceed max_beam; whatever is left
 * is finished by DPBruteForce over all of P.
 * Outputs lam (n, -1 = none) and delta (n, reported distance, +inf = none).
 * stats (may be NULL, >= 64 entries): [0] = rounds run, [1] = |U| after
 * round 0, [2 + r] = |U| after doubling round r, stats[63] = points finished
 * by the brute-force tail.
 */
int orc_dependent_points(const orc_points* P, const int32_t* G, int32_t R, const float* key,
                         const int32_t* knn, int32_t k, int32_t Ld, int32_t threshold,
                         int32_t max_rounds, int32_t max_beam, int32_t* lam, float* delta,
                         int64_t* stats, int nthreads) {
  int64_t n = P->n;
  if (nthreads < 1) nthreads = 1;
  float* dis = (float*)malloc(sizeof(float) * (size_t)n);
  int32_t* U = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  search_ws* ws = (search_ws*)malloc(sizeof(search_ws) * nthreads);
  for (int t = 0; t < nthreads; t++) ws_init(&ws[t], n);
  if (stats) memset(stats, 0, sizeof(int64_t) * 64);

  /* the point of maximum rank has no dependent point */
  int64_t gmax = 0;
  for (int64_t i = 1; i < n; i++)
    if (ranks_above(key, i, gmax)) gmax = i;

  dep_ctx c = {P, G, R, key, knn, k, U, Ld, lam, dis, ws};
  /* lambda_i <- DPBruteForce(x_i, N_i) */
  parallel_for(n, nthreads, dep_round0_body, &c);
  /* P_unfinished <- par-filter(P, lambda_i = none), the maximum skipped */
  int64_t nu = 0;
  for (int64_t i = 0; i < n; i++)
    if (lam[i] < 0 && i != gmax) U[nu++] = (int32_t)i;
  if (stats) stats[1] = nu;
  int64_t kdep = Ld;
  int32_t rounds = 0;
  while (nu > threshold && rounds < max_rounds && kdep <= max_beam) {
    c.kdep = (int32_t)kdep;
    parallel_for(nu, nthreads, dep_round_body, &c);
    kdep *= 2;
    int64_t m = 0;
    for (int64_t u = 0; u < nu; u++)
      if (lam[U[u]] < 0) U[m++] = U[u];
    nu = m;
    if (stats && rounds < 60) stats[2 + rounds] = nu;
    rounds++;
  }
  if (stats) {
    stats[0] = rounds;
    stats[63] = nu;
  }
  /* the remaining points: DPBruteForce over all of P */
  g_all_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t j = 0; j < n; j++) g_all_ids[j] = (int32_t)j;
  parallel_for(nu, nthreads, dep_tail_body, &c);
  free(g_all_ids);
  g_all_ids = NULL;
  for (int64_t i = 0; i < n; i++)
    delta[i] = lam[i] >= 0 ? orc_out_dist(P, dis[i]) : INFINITY;
  for (int t = 0; t < nthreads; t++) ws_free(&ws[t]);
  free(ws);
  free(U);
  free(dis);
  return 0;
}

/* ---------- Algorithm 2 lines 5-7: noise, centers, union-find ---------- */

static int64_t uf_find(int32_t* parent, int64_t a) {
  while (parent[a] != a) {
    parent[a] = parent[parent[a]];
    a = parent[a];
  }
  return a;
}

typedef struct {
  float prod;
  int32_t id;
} prod_item;

static int prod_cmp(const void* pa, const void* pb) {
  prod_item a = *(const prod_item*)pa, b = *(const prod_item*)pb;
  if (a.prod > b.prod) return -1;
  if (a.prod < b.prod) return 1;
  return a.id < b.id ? -1 : (a.id > b.id ? 1 : 0);
}

/* UF.Union(i, lambda_i) for every point that is neither noise nor a center
 * nor without a dependent point; each set is named by its cut member. Frees
 * noise and center. Returns the number of sets, or -1 on an inconsistent
 * forest. */
static int64_t cluster_from_centers(int64_t n, const int32_t* lam, uint8_t* noise, uint8_t* center,
                                    int32_t* labels) {
  int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) parent[i] = (int32_t)i;
  /* UF.Union(i, lambda_i) for i not noise and not center */
  for (int64_t i = 0; i < n; i++) {
    if (noise[i] || center[i] || lam[i] < 0) continue;
    int64_t a = uf_find(parent, i), b = uf_find(parent, lam[i]);
    if (a != b) parent[a] = (int32_t)b;
  }
  /* name each set by its cut member */
  int32_t* name = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) name[i] = -1;
  int64_t roots = 0, bad = 0;
  for (int64_t i = 0; i < n; i++) {
    int cut = noise[i] || center[i] || lam[i] < 0;
    if (!cut) continue;
    int64_t r = uf_find(parent, i);
    if (name[r] >= 0) bad = 1;
    name[r] = (int32_t)i;
    roots++;
  }
  for (int64_t i = 0; i < n; i++) {
    int64_t r = uf_find(parent, i);
    labels[i] = name[r];
    if (name[r] < 0) bad = 1;
  }
  free(name);
  free(parent);
  free(noise);
  free(center);
  return bad ? -1 : roots;
}

/*
 * Noise: rho_i < rho_min (Sec. 4.2). Centers among the non-noise points:
 * threshold, delta_i > delta_min (Sec. 2.1, Sec. 4.2); or product, the
 * n_clusters largest delta_i * rho_i (ties: smaller id; 0 * inf taken as 0).
 * A point without a dependent point is a root as well. Then Union(i, lambda_i)
 * for every other point and c_i = Find(i). The label written is the root of
 * i's tree in the cut dependent forest (the one member of each set whose edge
 * was cut), which names the set independently of the union order.
 * Returns the number of clusters (roots), or -1 on inconsistent input.
 */
int64_t orc_cluster(int64_t n, const float* rho, const int32_t* lam, const float* delta,
                    int32_t center_fn, float rho_min, float delta_min, int32_t n_clusters,
                    int32_t* labels) {
  uint8_t* noise = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* center = (uint8_t*)calloc((size_t)n, 1);
  for (int64_t i = 0; i < n; i++) noise[i] = rho[i] < rho_min;
  if (center_fn == CENTER_THRESHOLD) {
    for (int64_t i = 0; i < n; i++) center[i] = !noise[i] && delta[i] > delta_min;
  } else {
    prod_item* pr = (prod_item*)malloc(sizeof(prod_item) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
      if (noise[i]) continue;
      float p = (delta[i] == 0.0f || rho[i] == 0.0f) ? 0.0f : delta[i] * rho[i];
      pr[m].prod = p;
      pr[m].id = (int32_t)i;
      m++;
    }
    qsort(pr, (size_t)m, sizeof(prod_item), prod_cmp);
    for (int64_t t = 0; t < m && t < n_clusters; t++) center[pr[t].id] = 1;
    free(pr);
  }
  return cluster_from_centers(n, lam, noise, center, labels);
}

/*
 * Local center function (Appendix, center functions): a non-noise point is a
 * center when no point of its k-NN list is denser, in the rank order above:
 * it ranks above every listed neighbour j (rank_key_i > rank_key_j, or equal
 * keys and i < j; entries < 0 are padding). Noise and union-find as in
 * orc_cluster.
 */
int64_t orc_cluster_local(int64_t n, int32_t k, const int32_t* knn_ids, const float* rank_key,
                          const float* rho, const int32_t* lam, float rho_min, int32_t* labels) {
  uint8_t* noise = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* center = (uint8_t*)calloc((size_t)n, 1);
  for (int64_t i = 0; i < n; i++) {
    noise[i] = rho[i] < rho_min;
    if (noise[i]) continue;
    int top = 1;
    for (int32_t t = 0; t < k && top; t++) {
      int32_t j = knn_ids[i * k + t];
      if (j < 0 || j == i) continue;
      if (rank_key[j] > rank_key[i] || (rank_key[j] == rank_key[i] && j < i)) top = 0;
    }
    center[i] = (uint8_t)top;
  }
  return cluster_from_centers(n, lam, noise, center, labels);
}

/* ---------- Vamana: RobustPrune and batched construction ---------- */

/*
 * RobustPrune(p, C, alpha, R), the DiskANN rule: sort C \ {p} by distance to
 * p; repeatedly move the closest remaining candidate p* to the out-list and
 * drop every remaining p' with alpha * D(p*, p') <= D(p, p'); stop at R.
 * With ordering values (squared distances for L2) the test reads
 * alpha^2 * dis(p*, p') <= dis(p, p'), alpha^2 rounded to FP32 once.
 * C[t].dis must hold dis(p, C[t].id). C is reordered. Returns |out|.
 */
static int32_t robust_prune(const orc_points* P, int64_t p, item* C, int64_t nc, float alpha,
                            int32_t R, int32_t* out) {
  int64_t m = 0;
  for (int64_t t = 0; t < nc; t++)
    if (C[t].id != p) C[m++] = C[t];
  nc = m;
  qsort(C, (size_t)nc, sizeof(item), item_cmp);
  m = 0;
  for (int64_t t = 0; t < nc; t++) /* duplicates are adjacent after the sort */
    if (m == 0 || C[m - 1].id != C[t].id) C[m++] = C[t];
  nc = m;
  float a2 = alpha * alpha;
  uint8_t* alive = (uint8_t*)malloc((size_t)(nc > 0 ? nc : 1));
  memset(alive, 1, (size_t)(nc > 0 ? nc : 1));
  int32_t deg = 0;
  for (int64_t t = 0; t < nc && deg < R; t++) {
    if (!alive[t]) continue;
    int32_t ps = C[t].id;
    out[deg++] = ps;
    if (deg == R) break;
    for (int64_t u = t + 1; u < nc; u++) {
      if (!alive[u]) continue;
      if (a2 * orc_dis(P, ps, C[u].id) <= C[u].dis) alive[u] = 0;
    }
  }
  free(alive);
  return deg;
}

/* Public single-point entry for the tests. cand_ids: candidate ids; the
   distances to p are computed here. Returns |out|. */
int32_t orc_robust_prune(const orc_points* P, int64_t p, const int32_t* cand_ids, int64_t nc,
                         float alpha, int32_t R, int32_t* out) {
  item* C = (item*)malloc(sizeof(item) * (size_t)(nc > 0 ? nc : 1));
  for (int64_t t = 0; t < nc; t++) {
    C[t].id = cand_ids[t];
    C[t].dis = orc_dis(P, p, cand_ids[t]);
  }
  int32_t m = robust_prune(P, p, C, nc, alpha, R, out);
  free(C);
  return m;
}

typedef struct {
  const orc_points* P;
  int32_t* G;
  int32_t R, L;
  float alpha;
  const int32_t* S;
  int32_t nS;
  int32_t visit_cap;
  const int32_t* batch;
  item** V;
  int64_t* nV;
  const int64_t* tgt_begin;
  const int32_t* pairs; /* (target, source) sorted */
  search_ws* ws;
} build_ctx;

static void build_search_body(void* c, int64_t t, int tid) {
  build_ctx* x = (build_ctx*)c;
  int64_t p = x->batch[t];
  /* greedy search for x_p from the start points on the frozen graph */
  greedy_search(x->P, x->G, x->R, p, x->S, x->nS, x->L, 0, &x->ws[tid], NULL, &x->V[t],
                &x->nV[t]);
  /* keep the visit_cap closest visited points */
  qsort(x->V[t], (size_t)x->nV[t], sizeof(item), item_cmp);
  if (x->nV[t] > x->visit_cap) x->nV[t] = x->visit_cap;
}

static int32_t row_degree(const int32_t* row, int32_t R) {
  int32_t d = 0;
  while (d < R && row[d] >= 0) d++;
  return d;
}

static void build_prune_body(void* c, int64_t t, int tid) {
  (void)tid;
  build_ctx* x = (build_ctx*)c;
  int64_t p = x->batch[t];
  int32_t* row = x->G + p * x->R;
  int32_t deg = row_degree(row, x->R);
  /* candidates: V_p u N_out(p) */
  int64_t nc = x->nV[t] + deg;
  item* C = (item*)malloc(sizeof(item) * (size_t)(nc > 0 ? nc : 1));
  for (int64_t u = 0; u < x->nV[t]; u++) C[u] = x->V[t][u];
  for (int32_t u = 0; u < deg; u++) {
    C[x->nV[t] + u].id = row[u];
    C[x->nV[t] + u].dis = orc_dis(x->P, p, row[u]);
  }
  int32_t* out = (int32_t*)malloc(sizeof(int32_t) * (size_t)x->R);
  int32_t m = robust_prune(x->P, p, C, nc, x->alpha, x->R, out);
  for (int32_t u = 0; u < x->R; u++) row[u] = u < m ? out[u] : -1;
  free(out);
  free(C);
}

static void build_reverse_body(void* c, int64_t g, int tid) {
  (void)tid;
  build_ctx* x = (build_ctx*)c;
  int64_t b0 = x->tgt_begin[g], b1 = x->tgt_begin[g + 1];
  int64_t y = x->pairs[2 * b0];
  int32_t* row = x->G + y * x->R;
  int32_t deg = row_degree(row, x->R);
  /* incoming sources (sorted by id, unique) not already out-neighbours of y */
  int32_t* inc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(b1 - b0));
  int64_t ni = 0;
  for (int64_t e = b0; e < b1; e++) {
    int32_t s = x->pairs[2 * e + 1];
    if (ni > 0 && inc[ni - 1] == s) continue;
    int present = 0;
    for (int32_t u = 0; u < deg; u++) present |= row[u] == s;
    if (!present) inc[ni++] = s;
  }
  if (deg + ni <= x->R) {
    for (int64_t u = 0; u < ni; u++) row[deg + u] = inc[u];
  } else {
    int64_t nc = deg + ni;
    item* C = (item*)malloc(sizeof(item) * (size_t)nc);
    for (int32_t u = 0; u < deg; u++) C[u].id = row[u];
    for (int64_t u = 0; u < ni; u++) C[deg + u].id = inc[u];
    for (int64_t u = 0; u < nc; u++) C[u].dis = orc_dis(x->P, y, C[u].id);
    int32_t* out = (int32_t*)malloc(sizeof(int32_t) * (size_t)x->R);
    int32_t m = robust_prune(x->P, y, C, nc, x->alpha, x->R, out);
    for (int32_t u = 0; u < x->R; u++) row[u] = u < m ? out[u] : -1;
    free(out);
    free(C);
  }
  free(inc);
}

static int pair_cmp(const void* pa, const void* pb) {
  const int32_t* a = (const int32_t*)pa;
  const int32_t* b = (const int32_t*)pb;
  if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
  if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
  return 0;
}

/* Number of points per insertion batch: 1, 2, 4, ... capped at
   ceil(batch_frac * n) (Sec. 4.1: batches of doubling size up to 0.02n). */
int64_t orc_batch_cap(int64_t n, float batch_frac) {
  int64_t cap = (int64_t)ceil((double)batch_frac * (double)n);
  return cap < 1 ? 1 : cap;
}

/*
 * Vamana batched construction (Sec. 3.2, Sec. 4.1). Points are inserted in
 * the order perm (a permutation of 0..n-1); the first n_start of them are the
 * randomly sampled start points of every search. For each batch, on the graph
 * as it stood at the start of the batch:
 *   1. greedy search (beam L) for each batch point from the start points,
 *      keeping the visit_cap closest visited points V_p;
 *   2. out(p) <- RobustPrune(p, V_p u N_out(p), alpha, R);
 *   3. reverse edges: every y in out(p) gains p; per y the new sources are
 *      taken in id order, appended when they fit, else
 *      N_out(y) <- RobustPrune(y, N_out(y) u new sources, alpha, R).
 * G (n x R) is written, -1 padded. Returns 0, or 1 on bad arguments.
 */
int orc_build_graph(const orc_points* P, int32_t R, int32_t L, float alpha, const int32_t* perm,
                    int32_t n_start, float batch_frac, int32_t visit_cap, int32_t passes, int32_t* G,
                    int nthreads) {
  int64_t n = P->n;
  if (R < 1 || L < 1 || n_start < 1 || n_start > n || visit_cap < 1 || passes < 1 || passes > 2) return 1;
  if (nthreads < 1) nthreads = 1;
  for (int64_t i = 0; i < n * R; i++) G[i] = -1;
  search_ws* ws = (search_ws*)malloc(sizeof(search_ws) * nthreads);
  for (int t = 0; t < nthreads; t++) ws_init(&ws[t], n);
  int64_t cap = orc_batch_cap(n, batch_frac);
  item** V = (item**)calloc((size_t)cap, sizeof(item*));
  int64_t* nV = (int64_t*)calloc((size_t)cap, sizeof(int64_t));
  int32_t* pairs = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(cap * R));
  int64_t* tgt_begin = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap * R + 1));
  build_ctx c = {P, G, R, L, alpha, perm, n_start, visit_cap, NULL, V, nV, tgt_begin, pairs, ws};
  for (int32_t pass = 0; pass < passes; pass++) {
  /* with two passes the first one prunes with alpha = 1 */
  c.alpha = (passes == 2 && pass == 0) ? 1.0f : alpha;
  int64_t pos = 0, bsz = 1;
  while (pos < n) {
    int64_t m = bsz < cap ? bsz : cap;
    if (m > n - pos) m = n - pos;
    c.batch = perm + pos;
    parallel_for(m, nthreads, build_search_body, &c);
    parallel_for(m, nthreads, build_prune_body, &c);
    /* reverse edges, grouped by target */
    int64_t np = 0;
    for (int64_t t = 0; t < m; t++) {
      int64_t p = perm[pos + t];
      for (int32_t u = 0; u < R; u++) {
        int32_t y = G[p * R + u];
        if (y < 0) break;
        pairs[2 * np] = y;
        pairs[2 * np + 1] = (int32_t)p;
        np++;
      }
    }
    qsort(pairs, (size_t)np, 2 * sizeof(int32_t), pair_cmp);
    int64_t ng = 0;
    for (int64_t e = 0; e < np; e++)
      if (e == 0 || pairs[2 * e] != pairs[2 * (e - 1)]) tgt_begin[ng++] = e;
    tgt_begin[ng] = np;
    parallel_for(ng, nthreads, build_reverse_body, &c);
    for (int64_t t = 0; t < m; t++) {
      free(V[t]);
      V[t] = NULL;
    }
    pos += m;
    if (bsz < cap) bsz *= 2; /* the doubling stops at the cap */
  }
  }
  free(tgt_begin);
  free(pairs);
  free(nV);
  free(V);
  for (int t = 0; t < nthreads; t++) ws_free(&ws[t]);
  free(ws);
  return 0;
}

/* ---------- NN-Descent graph index (Sec. 5.1, graph indices) ---------- */

/* One list per point: K (dis, id) items sorted ascending. */
static void sort_unique_top(item* a, int64_t* m, int32_t K) {
  qsort(a, (size_t)*m, sizeof(item), item_cmp);
  int64_t w = 0;
  for (int64_t t = 0; t < *m; t++) /* the same id has the same dis: adjacent */
    if (w == 0 || a[w - 1].id != a[t].id) a[w++] = a[t];
  *m = w < K ? w : K;
}

typedef struct {
  const orc_points* P;
  int32_t K;
  const int32_t* N;     /* n x K ids of the snapshot */
  const float* Nd;      /* n x K dis */
  const int32_t* Rv;    /* n x K reverse ids (-1 padded) */
  int32_t* N2;          /* n x K new ids */
  float* N2d;
  int64_t* changed;     /* per point: 1 when the list changed */
} nnd_ctx;

/* C(x) = N(x) u R(x), the valid ids */
static int32_t nnd_neigh(const nnd_ctx* x, int64_t p, int32_t* out) {
  int32_t m = 0;
  for (int32_t t = 0; t < x->K; t++) out[m++] = x->N[p * x->K + t];
  for (int32_t t = 0; t < x->K; t++)
    if (x->Rv[p * x->K + t] >= 0) out[m++] = x->Rv[p * x->K + t];
  return m;
}

static void nnd_round_body(void* c, int64_t u, int tid) {
  (void)tid;
  const nnd_ctx* x = (const nnd_ctx*)c;
  const int32_t K = x->K;
  int32_t* cu = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)K);
  int32_t* cp = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)K);
  const int32_t mu = nnd_neigh(x, u, cu);
  /* candidates: N(u), C(u), and C(p) for every p in C(u); u itself excluded */
  int64_t cap = (int64_t)K + mu + (int64_t)mu * 2 * K;
  item* a = (item*)malloc(sizeof(item) * (size_t)cap);
  int64_t m = 0;
  for (int32_t t = 0; t < K; t++) {
    a[m].id = x->N[u * K + t];
    a[m].dis = x->Nd[u * K + t];
    m++;
  }
  for (int32_t s = 0; s < mu; s++) {
    const int32_t p = cu[s];
    if (p != u) {
      a[m].id = p;
      a[m].dis = orc_dis(x->P, u, p);
      m++;
    }
    const int32_t mp = nnd_neigh(x, p, cp);
    for (int32_t t = 0; t < mp; t++) {
      const int32_t v = cp[t];
      if (v == u) continue;
      a[m].id = v;
      a[m].dis = orc_dis(x->P, u, v);
      m++;
    }
  }
  sort_unique_top(a, &m, K);
  int64_t diff = 0;
  for (int32_t t = 0; t < K; t++) {
    x->N2[u * K + t] = a[t].id;
    x->N2d[u * K + t] = a[t].dis;
    diff |= a[t].id != x->N[u * K + t];
  }
  x->changed[u] = diff;
  free(a);
  free(cp);
  free(cu);
}

/* Reverse lists of the snapshot: Rv(x) = the K smallest (dis, q) among the
   q with x in N(q); -1 padded. */
static void nnd_reverse(int64_t n, int32_t K, const int32_t* N, const float* Nd, int32_t* Rv) {
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t q = 0; q < n; q++)
    for (int32_t t = 0; t < K; t++) cnt[N[q * K + t] + 1]++;
  for (int64_t x = 0; x < n; x++) cnt[x + 1] += cnt[x];
  item* e = (item*)malloc(sizeof(item) * (size_t)(n * K > 0 ? n * K : 1));
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t x = 0; x < n; x++) pos[x] = cnt[x];
  for (int64_t q = 0; q < n; q++)
    for (int32_t t = 0; t < K; t++) {
      const int32_t x = N[q * K + t];
      e[pos[x]].id = (int32_t)q;
      e[pos[x]].dis = Nd[q * K + t];
      pos[x]++;
    }
  for (int64_t x = 0; x < n; x++) {
    item* seg = e + cnt[x];
    int64_t m = cnt[x + 1] - cnt[x];
    qsort(seg, (size_t)m, sizeof(item), item_cmp);
    for (int32_t t = 0; t < K; t++) Rv[x * K + t] = t < m ? seg[t].id : -1;
  }
  free(pos);
  free(e);
  free(cnt);
}

/*
 * NN-Descent graph index. The paper's framework offers PyNNDescent (and
 * HCNNG) graphs with a num_repeats argument (Sec. 5.1, graph indices) but
 * prints no steps; this follows NN-Descent (Dong et al., "Efficient k-nearest
 * neighbor graph construction for generic similarity measures") in a
 * synchronous form, every new list computed from the same snapshot:
 *   for each repeat r: N(u) <- the K ids init[r][u] sorted by (dis, id);
 *     repeat `rounds` times or until no list changes:
 *       R(x) <- the K smallest (D(q, x), q) among the q with x in N(q);
 *       C(x) <- N(x) u R(x);
 *       N'(u) <- the K smallest (dis, id) of N(u) u C(u) u (U_{p in C(u)} C(p)), minus u;
 *   the repeats are merged: N(u) <- the K smallest of the union of their lists;
 *   G(u) <- RobustPrune(u, N(u), alpha, R); then every edge u -> y gives y the
 *   source u, all points as one batch of the Vamana build's reverse step
 *   (sources in id order, appended when they fit, else RobustPrune(y, ...)).
 * init: repeats x n x K ids (distinct, none equal to its point). Outputs knn
 * (n x K ids, sorted by (dis, id)), G (n x R, -1 padded) and changes
 * (repeats x rounds: the lists that changed in each round, 0 after
 * convergence). Returns 0, or 1 on bad arguments.
 */
int orc_nndescent(const orc_points* P, int32_t K, int32_t repeats, const int32_t* init, int32_t rounds,
                  float alpha, int32_t R, int32_t* knn, int32_t* G, int64_t* changes, int nthreads) {
  const int64_t n = P->n;
  if (K < 1 || K >= n || repeats < 1 || rounds < 0 || R < 1) return 1;
  if (nthreads < 1) nthreads = 1;
  int32_t* N = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * K));
  float* Nd = (float*)malloc(sizeof(float) * (size_t)(n * K));
  int32_t* N2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * K));
  float* N2d = (float*)malloc(sizeof(float) * (size_t)(n * K));
  int32_t* Rv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * K));
  int64_t* changed = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  item* all = (item*)malloc(sizeof(item) * (size_t)(n * K * repeats));
  int64_t* nall = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  item* tmp = (item*)malloc(sizeof(item) * (size_t)K);
  for (int64_t i = 0; i < (int64_t)repeats * rounds; i++) changes[i] = 0;
  for (int32_t r = 0; r < repeats; r++) {
    for (int64_t u = 0; u < n; u++) {
      for (int32_t t = 0; t < K; t++) {
        tmp[t].id = init[((int64_t)r * n + u) * K + t];
        tmp[t].dis = orc_dis(P, u, tmp[t].id);
      }
      qsort(tmp, (size_t)K, sizeof(item), item_cmp);
      for (int32_t t = 0; t < K; t++) {
        N[u * K + t] = tmp[t].id;
        Nd[u * K + t] = tmp[t].dis;
      }
    }
    for (int32_t it = 0; it < rounds; it++) {
      nnd_reverse(n, K, N, Nd, Rv);
      nnd_ctx c = {P, K, N, Nd, Rv, N2, N2d, changed};
      parallel_for(n, nthreads, nnd_round_body, &c);
      int64_t ch = 0;
      for (int64_t u = 0; u < n; u++) ch += changed[u];
      changes[(int64_t)r * rounds + it] = ch;
      memcpy(N, N2, sizeof(int32_t) * (size_t)(n * K));
      memcpy(Nd, N2d, sizeof(float) * (size_t)(n * K));
      if (ch == 0) break;
    }
    for (int64_t u = 0; u < n; u++)
      for (int32_t t = 0; t < K; t++) {
        item* d = &all[(u * repeats + r) * K + t];
        d->id = N[u * K + t];
        d->dis = Nd[u * K + t];
      }
  }
  /* merge the repeats, then prune */
  for (int64_t i = 0; i < n * R; i++) G[i] = -1;
  int32_t* out = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
  for (int64_t u = 0; u < n; u++) {
    item* seg = all + u * repeats * K;
    int64_t m = (int64_t)repeats * K;
    sort_unique_top(seg, &m, K);
    for (int32_t t = 0; t < K; t++) knn[u * K + t] = seg[t].id;
    int32_t deg = robust_prune(P, u, seg, m, alpha, R, out);
    for (int32_t t = 0; t < deg; t++) G[u * R + t] = out[t];
  }
  free(out);
  /* reverse edges, all points as one batch, grouped by target */
  int64_t np = 0;
  int32_t* pairs = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(n * R > 0 ? n * R : 1));
  int64_t* tgt_begin = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * R + 1));
  for (int64_t u = 0; u < n; u++)
    for (int32_t t = 0; t < R; t++) {
      const int32_t y = G[u * R + t];
      if (y < 0) break;
      pairs[2 * np] = y;
      pairs[2 * np + 1] = (int32_t)u;
      np++;
    }
  qsort(pairs, (size_t)np, 2 * sizeof(int32_t), pair_cmp);
  int64_t ng = 0;
  for (int64_t e = 0; e < np; e++)
    if (e == 0 || pairs[2 * e] != pairs[2 * (e - 1)]) tgt_begin[ng++] = e;
  tgt_begin[ng] = np;
  build_ctx bc;
  memset(&bc, 0, sizeof(bc));
  bc.P = P;
  bc.G = G;
  bc.R = R;
  bc.alpha = alpha;
  bc.tgt_begin = tgt_begin;
  bc.pairs = pairs;
  parallel_for(ng, nthreads, build_reverse_body, &bc);
  free(tgt_begin);
  free(pairs);
  free(tmp);
  free(nall);
  free(all);
  free(changed);
  free(Rv);
  free(N2d);
  free(N2);
  free(Nd);
  free(N);
  return 0;
}

/* ---------- HCNNG graph index (Sec. 5.1, graph indices) ---------- */

/*
 * The paper's framework also offers HCNNG graphs (Munoz et al., "Hierarchical
 * clustering-based graphs for large scale approximate nearest neighbor
 * search"), repeated num_repeats times and pruned with alpha, but prints no
 * steps. This follows the method's outline in a deterministic form:
 *   for each repeat t: split the points hierarchically -- a node [b, b + m)
 *     of the current order with more than leaf_size points draws two pivots
 *     p1 != p2 from its points; every point with dis(x, p1) <= dis(x, p2)
 *     goes left, the rest right, each side keeping its order (a split that
 *     leaves a side empty cuts the node at ceil(m / 2) instead);
 *     in every leaf, a minimum spanning forest whose degrees are bounded by
 *     mst_deg: the leaf's pairs in (dis, smaller id, larger id) order, each
 *     taken when it joins two components and both ends have degree below
 *     mst_deg (Kruskal's rule with the bound);
 *   C(u) = the neighbours of u in the forests of all repeats;
 *   G(u) = RobustPrune(u, C(u), alpha, R).
 * The order starts as 0..n-1, so every node lists its points in ascending id.
 * Pivot draws use SplitMix64 (Steele, Lea and Flood 2014) as a counter-based
 * generator keyed by (seed, t, b, m, j): v = S(seed + t), v = S(v + b),
 * v = S(v + m), draw j = S(v + j), where S(x) is SplitMix64's output for the
 * state x; p1 = the (draw 0 mod m)-th point of the node, p2 = the
 * (draw 1 mod (m - 1))-th of the others.
 */
static uint64_t sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t hc_draw(uint64_t seed, int32_t t, int64_t b, int64_t m, int j) {
  uint64_t v = sm64(seed + (uint64_t)t);
  v = sm64(v + (uint64_t)b);
  v = sm64(v + (uint64_t)m);
  return sm64(v + (uint64_t)j);
}

/* For the tests: the generator's output for a state, and a node's draw. */
uint64_t orc_splitmix64(uint64_t x) { return sm64(x); }
uint64_t orc_hcnng_draw(uint64_t seed, int32_t t, int64_t b, int64_t m, int32_t j) { return hc_draw(seed, t, b, m, j); }

/* The leaves of tree t: order (n ids) and leaf_begin (n_leaves + 1 offsets,
   in the order the leaves lie in `order`). Returns the number of leaves. */
int64_t orc_hcnng_partition(const orc_points* P, int32_t t, int32_t leaf_size, uint64_t seed, int32_t* order,
                            int64_t* leaf_begin) {
  const int64_t n = P->n;
  for (int64_t i = 0; i < n; i++) order[i] = (int32_t)i;
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  uint8_t* is_leaf_start = (uint8_t*)calloc((size_t)n + 1, 1);
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * 2 * ((size_t)n + 1));
  int64_t sp = 0;
  stack[sp++] = 0;
  stack[sp++] = n;
  while (sp > 0) {
    const int64_t m = stack[--sp], b = stack[--sp];
    if (m <= leaf_size) {
      is_leaf_start[b] = 1;
      continue;
    }
    const int64_t i1 = (int64_t)(hc_draw(seed, t, b, m, 0) % (uint64_t)m);
    int64_t i2 = (int64_t)(hc_draw(seed, t, b, m, 1) % (uint64_t)(m - 1));
    if (i2 >= i1) i2++;
    const int32_t p1 = order[b + i1], p2 = order[b + i2];
    int64_t nl = 0, nr = 0;
    for (int64_t i = 0; i < m; i++) {
      const int32_t x = order[b + i];
      if (orc_dis(P, x, p1) <= orc_dis(P, x, p2))
        order[b + nl++] = x; /* in place: nl <= i, the left side never overtakes */
      else
        tmp[nr++] = x;
    }
    for (int64_t i = 0; i < nr; i++) order[b + nl + i] = tmp[i];
    if (nl == 0 || nl == m) nl = (m + 1) / 2; /* degenerate split: halves of the same order */
    stack[sp++] = b;
    stack[sp++] = nl;
    stack[sp++] = b + nl;
    stack[sp++] = m - nl;
  }
  int64_t nleaf = 0;
  for (int64_t i = 0; i < n; i++)
    if (is_leaf_start[i]) leaf_begin[nleaf++] = i;
  leaf_begin[nleaf] = n;
  free(stack);
  free(is_leaf_start);
  free(tmp);
  return nleaf;
}

typedef struct {
  float dis;
  int32_t i, j; /* local indices, i < j */
} hc_edge;

static int hc_edge_cmp(const void* pa, const void* pb) {
  const hc_edge* a = (const hc_edge*)pa;
  const hc_edge* b = (const hc_edge*)pb;
  if (a->dis != b->dis) return a->dis < b->dis ? -1 : 1;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  return a->j < b->j ? -1 : (a->j > b->j);
}

static int32_t hc_find(int32_t* parent, int32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

/* Degree-bounded minimum spanning forest of the m points ids (ascending).
   Writes its edges as id pairs (at most m - 1) and returns their number. */
int64_t orc_hcnng_leaf_mst(const orc_points* P, const int32_t* ids, int64_t m, int32_t mst_deg, int32_t* edges) {
  if (m < 2) return 0;
  const int64_t ne = m * (m - 1) / 2;
  hc_edge* E = (hc_edge*)malloc(sizeof(hc_edge) * (size_t)ne);
  int64_t e = 0;
  for (int32_t i = 0; i < m; i++)
    for (int32_t j = i + 1; j < m; j++) {
      E[e].dis = orc_dis(P, ids[i], ids[j]);
      E[e].i = i;
      E[e].j = j;
      e++;
    }
  qsort(E, (size_t)ne, sizeof(hc_edge), hc_edge_cmp);
  int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* deg = (int32_t*)calloc((size_t)m, sizeof(int32_t));
  for (int32_t i = 0; i < m; i++) parent[i] = i;
  int64_t out = 0;
  for (int64_t k = 0; k < ne && out < m - 1; k++) {
    const int32_t i = E[k].i, j = E[k].j;
    if (deg[i] >= mst_deg || deg[j] >= mst_deg) continue;
    const int32_t ri = hc_find(parent, i), rj = hc_find(parent, j);
    if (ri == rj) continue;
    parent[ri < rj ? rj : ri] = ri < rj ? ri : rj;
    deg[i]++;
    deg[j]++;
    edges[2 * out] = ids[i];
    edges[2 * out + 1] = ids[j];
    out++;
  }
  free(deg);
  free(parent);
  free(E);
  return out;
}

typedef struct {
  const orc_points* P;
  const int32_t* order;
  const int64_t* leaf_begin;
  int32_t mst_deg;
  int32_t* edges;      /* 2 (n - 1) per tree at most: leaf l writes from 2 * leaf_begin[l] */
  int64_t* leaf_ne;
} hc_leaf_ctx;

static void hc_leaf_body(void* c, int64_t l, int tid) {
  (void)tid;
  const hc_leaf_ctx* x = (const hc_leaf_ctx*)c;
  const int64_t b = x->leaf_begin[l], m = x->leaf_begin[l + 1] - b;
  x->leaf_ne[l] = orc_hcnng_leaf_mst(x->P, x->order + b, m, x->mst_deg, x->edges + 2 * b);
}

typedef struct {
  const orc_points* P;
  const int32_t* cand; /* n x cap neighbour ids */
  const int32_t* ncand;
  int32_t cap;
  float alpha;
  int32_t R;
  int32_t* G;
} hc_prune_ctx;

static void hc_prune_body(void* c, int64_t u, int tid) {
  (void)tid;
  const hc_prune_ctx* x = (const hc_prune_ctx*)c;
  const int32_t nc = x->ncand[u];
  item* C = (item*)malloc(sizeof(item) * (size_t)(nc > 0 ? nc : 1));
  int32_t* out = (int32_t*)malloc(sizeof(int32_t) * (size_t)x->R);
  for (int32_t t = 0; t < nc; t++) {
    C[t].id = x->cand[u * x->cap + t];
    C[t].dis = orc_dis(x->P, u, C[t].id);
  }
  const int32_t deg = robust_prune(x->P, u, C, nc, x->alpha, x->R, out);
  for (int32_t t = 0; t < x->R; t++) x->G[u * x->R + t] = t < deg ? out[t] : -1;
  free(out);
  free(C);
}

/* HCNNG graph (see above): G n x R, -1 padded. leaves (may be NULL): the
   number of leaves of each repeat. Returns 0, or 1 on bad arguments. */
int orc_hcnng(const orc_points* P, int32_t repeats, int32_t leaf_size, int32_t mst_deg, float alpha, int32_t R,
              uint64_t seed, int32_t* G, int64_t* leaves, int nthreads) {
  const int64_t n = P->n;
  if (repeats < 1 || leaf_size < 2 || mst_deg < 1 || R < 1 || n < 2) return 1;
  const int32_t cap = repeats * mst_deg;
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* leaf_begin = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int64_t* leaf_ne = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int32_t* edges = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)n);
  int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * (size_t)cap);
  int32_t* ncand = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  for (int32_t t = 0; t < repeats; t++) {
    const int64_t nl = orc_hcnng_partition(P, t, leaf_size, seed, order, leaf_begin);
    if (leaves) leaves[t] = nl;
    hc_leaf_ctx lc = {P, order, leaf_begin, mst_deg, edges, leaf_ne};
    parallel_for(nl, nthreads, hc_leaf_body, &lc);
    for (int64_t l = 0; l < nl; l++) {
      const int32_t* E = edges + 2 * leaf_begin[l];
      for (int64_t e = 0; e < leaf_ne[l]; e++) {
        const int32_t a = E[2 * e], b = E[2 * e + 1];
        cand[(int64_t)a * cap + ncand[a]++] = b; /* a tree gives each point at most mst_deg edges */
        cand[(int64_t)b * cap + ncand[b]++] = a;
      }
    }
  }
  hc_prune_ctx pc = {P, cand, ncand, cap, alpha, R, G};
  parallel_for(n, nthreads, hc_prune_body, &pc);
  free(ncand);
  free(cand);
  free(edges);
  free(leaf_ne);
  free(leaf_begin);
  free(order);
  return 0;
}

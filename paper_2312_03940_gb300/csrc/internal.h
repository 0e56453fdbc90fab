// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/pecann.h"

namespace pecann {

// Search modes of the beam-search kernel (epilogue selection).
enum : int { MODE_RAW = 0, MODE_KNN = 1, MODE_DEP = 2, MODE_BUILD = 3, MODE_DEPCAND = 4 };

// One point set of a batched launch (see SearchArgs::sets).
struct SetDesc {
  const uint8_t* X;   // rows of the set
  const int32_t* G;   // its graph (n x R, local ids)
  int64_t n;
  int64_t row_bytes;
  int C;
  int pad;
};

struct SearchArgs {
  const uint8_t* X;   // rows
  int64_t row_bytes;  // bytes per row
  int64_t n;
  int C;              // 16-byte chunks per row
  const int32_t* G;   // n x R
  int R;
  const int32_t* queries;  // nq query ids, or NULL for 0..nq-1
  int64_t nq;
  const int32_t* S;   // start set, or NULL for {query}
  int nS;
  int Lw;             // beam width
  int log2h;          // seen-filter size: (1 << log2h) 32-bit words
  int tag_bytes;      // set by launch_search: the filter holds (4 / tag_bytes) << log2h
                     // tags of 1, 2 or 4 (the whole id) bytes
  int stage;          // candidate staging entries per warp (>= max(R, nS))
  int vcap;           // BUILD: visited points kept
  int mode;
  int metric;
  int warp_bytes;     // shared memory per warp
  int block_warps;    // warps per block (0 = automatic)
  // RAW / KNN outputs
  int k;
  int32_t* out_ids;
  float* out_dis;
  int32_t* out_cnt;
  float* rho;
  float* rkey;
  int density_fn;
  int32_t* fb_list;   // KNN: queries whose search returned < k points
  int32_t* fb_cnt;
  // DEP
  const float* rank_key;
  int32_t* lam;
  float* delta;
  // BUILD
  int32_t* vis_ids;
  float* vis_dis;
  int32_t* vis_cnt;
  int* err;
  unsigned long long* work;  // optional: [0] expansions, [1] distance evaluations (sums)
  // batched form (sets != NULL): slots 0..nq-1 (or *nq_dev) are taken from
  // the device counter *queue; a slot's global point id (queries[slot], or
  // the slot itself) falls in set s with set_base[s] <= id < set_base[s+1];
  // outputs are concatenated over the sets and indexed by global id.
  const SetDesc* sets;
  const int64_t* set_base;
  int n_sets;
  unsigned long long* queue;
  const int32_t* nq_dev;
  const int32_t* set_active;  // batched dependent rounds: sets still doubling (NULL: all)
  int64_t id_base;           // global id of the set's point 0 (0 outside batches)
  // FP8 rows: the query is taken from its FP32 row times the per-dimension
  // scale (set by launch_search from the DataView)
  const float* qrows;        // n x d FP32 rows
  const float* scale;        // d scales: decoded x_j = scale_j * code_j
};

struct DataView {
  const uint8_t* X;
  int64_t n;
  int d;
  int dtype;
  int metric;
  int64_t row_bytes;
  int C;  // 16-byte chunks
  const float* f32_rows = nullptr;  // FP8 only: the FP32 rows (query side of the traversal)
  const float* scale = nullptr;     // FP8 only: d per-dimension scales
};

// Distance-kernel layout for a dataset: W lanes per row, CPL chunks per lane.
struct Layout {
  int W;
  int CPL;
};
bool pick_layout(int dtype, int metric, int d, Layout* out);

// Shared memory needed per warp by the search kernel.
int search_warp_bytes(int Lw, int log2h, int stage, int vcap, bool build);

// Launch the beam-search kernel. Returns a CUDA error (cudaSuccess on success).
cudaError_t launch_search(const DataView& dv, SearchArgs a, cudaStream_t st);

// Exact k-NN by brute force for the queries listed in d_list[0..*d_cnt).
cudaError_t launch_bruteforce_knn(const DataView& dv, const int32_t* d_list, const int32_t* d_cnt,
                                  int64_t max_list, int k, int32_t* knn_ids, float* knn_dist,
                                  float* rho, float* rkey, int density_fn, int* err, cudaStream_t st);

// DPBruteForce over all points for the queries in d_list[0..m).
cudaError_t launch_dep_bruteforce(const DataView& dv, const int32_t* d_list, int64_t m,
                                  const float* rank_key, unsigned long long* best, int32_t* lam,
                                  float* delta, cudaStream_t st);

// Exact FP32 re-rank of candidates found on reduced-precision rows or by
// the brute-force screen. k-NN: for each row u (0..rows), the cnt[u] <= K
// ids cand[u*K ..] of query q = list[u] (list NULL: q = u) are re-scored on
// the FP32 (or uint8) rows; the k closest (by exact (dis, id)) and the
// density are written at q; queries with 0 <= cnt[u] < k are appended to
// fb_list; rows with cnt[u] < 0 are skipped.
cudaError_t launch_rerank_knn(const DataView& f32, const int32_t* list, int64_t rows, const int32_t* cand,
                              const int32_t* cnt, int K, int k, int32_t* knn_ids, float* knn_dist, float* rho,
                              float* rkey, int density_fn, int32_t* fb_list, int32_t* fb_cnt, cudaStream_t st);
// Dependent points: for each listed query u, the exact closest of its
// cnt[u] <= K candidates cand[u*K ..] (all ranked above it) becomes lambda;
// rows with cnt[u] <= 0 are skipped.
cudaError_t launch_rerank_dep(const DataView& f32, const int32_t* list, int64_t m, const int32_t* cand,
                              const int32_t* cnt, int K, int32_t* lam, float* delta, cudaStream_t st);

// Argument checks and status helpers of the C ABI (abi.cu), shared by
// every entry point so that their rules cannot drift apart.
// check_dataset fills the view of the rows; f32 (optional) gets the FP32
// rows: the same view for FP32 / U8 data, data_f32 for BF16 / FP8.
pecann_status check_dataset(const pecann_dataset* ds, DataView* dv, DataView* f32 = nullptr);
pecann_status check_params(const pecann_params* p, int64_t n);
pecann_status check_index(const DataView& dv, const pecann_params* p);
pecann_status check_density_args(const DataView& dv, const int32_t* d_graph, const pecann_params* p,
                                 const int32_t* d_knn_ids, const float* d_knn_dist, const float* d_density,
                                 const float* d_rank_key);
pecann_status cuda_status(cudaError_t e, const char* what);
// Reads the device error word (synchronises `st`); PECANN_EINTERNAL if set.
pecann_status read_err(int* d_err, cudaStream_t st);
int log2_hash(const pecann_params* p, int Lw);
int rerank_k_of(const pecann_params* p);

// Device scratch of one k-NN + density pass. fb_list and raw hold n entries
// each; rr_* (n x rerank_k ids and distances, n counts) only for BF16 / FP8
// rows (NULL otherwise); work is optional.
struct DensityScratch {
  int32_t* fb_list = nullptr;
  float* raw = nullptr;
  int32_t* fb_cnt = nullptr;
  int* err = nullptr;
  unsigned long long* work = nullptr;
  int32_t* rr_ids = nullptr;
  float* rr_dis = nullptr;
  int32_t* rr_cnt = nullptr;
  void* bf_ws = nullptr;          // brute-force index: its scratch (bf_ws_bytes)
  int64_t* bf_counts = nullptr;   // brute-force index: host, 2 entries (see run_density_bf)
};
pecann_status run_density(const DataView& dv, const DataView& fv, const int32_t* d_graph, const pecann_params* p,
                          int32_t* d_knn_ids, float* d_knn_dist, float* d_density, float* d_rank_key,
                          const DensityScratch& sc, cudaStream_t st);

// The brute-force index on the tensor cores (bf_screen.cu). bws is a device
// scratch of bf_ws_bytes(n, d) bytes, 256-byte aligned. fv: the FP32 (or
// uint8) rows. h_counts (host, 2 entries, may be NULL): rows that took the
// collect pass, rows left to the exact SIMT kernels.
size_t bf_ws_bytes(int64_t n, int d);
pecann_status run_density_bf(const DataView& fv, const pecann_params* p, int32_t* knn_ids, float* knn_dist,
                             float* rho, float* rkey, int32_t* fb_list, int32_t* fb_cnt, int* err, void* bws,
                             int64_t* h_counts, cudaStream_t st);
// DPBruteForce over all points for the nu listed (unfinished) points U.
pecann_status run_dep_bf(const DataView& fv, const float* rank_key, const int32_t* U, int64_t nu, int32_t* lam,
                         float* delta, int* err, void* bws, int64_t* h_counts, cudaStream_t st);

// NN-Descent graph index (nnd.cu). fv: FP32 or uint8 rows; init: device
// repeats x n x K ids; h_changes (host, repeats x rounds) and knn_out (device
// n x K) may be NULL; ws: nndescent_ws_bytes(n, K, repeats, R) bytes.
size_t nndescent_ws_bytes(int64_t n, int K, int repeats, int R);
cudaError_t run_nndescent(const DataView& fv, int K, int repeats, const int32_t* init, int rounds, float alpha, int R,
                          int32_t* G, int32_t* knn_out, int64_t* h_changes, void* ws, int* d_err, cudaStream_t st);
// Out-degrees of an n x R graph (build.cu).
__global__ void k_degree(int64_t n, int R, const int32_t* G, int32_t* deg);

// HCNNG graph index (hcnng.cu). Leaves hold at most HCNNG_MAX_LEAF points
// (their pair keys fit in shared memory); degrees of the leaf forests at most
// HCNNG_MAX_DEG.
constexpr int HCNNG_MAX_LEAF = 200;
constexpr int HCNNG_MAX_DEG = 16;
size_t hcnng_ws_bytes(int64_t n, int repeats, int leaf, int mst_deg);
cudaError_t run_hcnng(const DataView& fv, int repeats, int leaf, int mst_deg, float alpha, int R, uint64_t seed,
                      int32_t* G, int64_t* h_leaves, void* ws, int* d_err, cudaStream_t st);

int num_sms();
// Counts the kernels the library launches (reported by pecann_kernel_launches).
void note_launch();
void set_last_error(const std::string& s);
// Name of the step that issued the CUDA call that failed last (for messages).
void set_where(const char* w);
const char* get_where();

}  // namespace pecann

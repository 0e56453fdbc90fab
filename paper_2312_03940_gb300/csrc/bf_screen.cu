// The brute-force index on the tensor cores (Sec. 5.1, "Brute Force": no
// index, exact k-NN by scanning every point; Sec. 6.1, the BruteForce
// instance whose result is exact DPC).
//
// Exactness comes from a screen and an exact decision:
//  1. Screen (k_bf_screen, tcgen05): approximate inner products of every
//     query row against every point row from BF16 copies of the rows, FP32
//     accumulation in TMEM. Per query the epilogue keeps the SC_KEEP best
//     approximate keys (k-NN mode: all points but the query; dependent mode:
//     only points ranked above the query).
//  2. Every approximate key is within E_q of the canonical FP32 key of the
//     pair (a bound from the BF16 rounding of both rows and the accumulation),
//     so the exact answer is among the points whose approximate key is within
//     2 E_q of the k-th (k-NN) or first (dependent) kept key. When the kept
//     list reaches past that band it holds every such point; otherwise the
//     query "overflows" and a collect pass gathers every point under its
//     threshold into a per-query list of SC_CAP; beyond that, the exact SIMT
//     kernels take the query.
//  3. Decision: the existing exact re-rank kernels re-score the candidates
//     with the canonical FP32 distance (exact integers for uint8 rows) and
//     take the k smallest (dis, id) keys, or the closest point ranked above.
// So the k-NN lists, densities and dependent points equal those of the exact
// method under the canonical distance, element for element.
//
// Screen kernel layout (one CTA per SM, persistent over 128-query tiles):
//   warp 0       TMA producer: 64-column chunks of the query tile (128 rows)
//                and of the point tile (256 rows), 128-byte swizzle, into a
//                3-stage ring of 48 KB;
//   warp 1       TMEM owner and MMA issuer (one thread): 4 x tcgen05.mma
//                (M 128, N 256, K 16) per chunk into one of two 256-column
//                TMEM accumulators;
//   warps 2..9   epilogue: two threads per query row (row = TMEM lane; the
//                warp's lane quarter), each reading one 128-column half of a
//                finished tile. A thread keeps the SC_HALF smallest keys of its
//                half in a max-heap in shared memory (slot-major, so that
//                neighbouring threads hit neighbouring banks); a 32-column
//                chunk is first reduced to its smallest key and only chunks
//                that beat the heap's largest key are taken apart. At the end
//                of a query tile the two sorted halves are merged.
// All CTAs sweep the point tiles in the same order and are kept within a few
// epochs of one another (pace_enter), so a point tile read from HBM serves
// every CTA from L2.
#include <string.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace pecann {

constexpr int SC_M = 128;          // query rows per tile (TMEM lanes)
constexpr int SC_N = 256;          // point rows per tile (TMEM columns per accumulator)
constexpr int SC_KCH = 64;         // BF16 columns per chunk (one 128-byte swizzle row)
constexpr int SC_STAGES = 3;
constexpr int SC_HALF = 40;        // heap entries per epilogue thread
constexpr int SC_KEEP = 2 * SC_HALF;  // kept candidates per query (two halves)
constexpr int SC_EPI = 256;        // epilogue threads (8 warps)
constexpr int SC_THREADS = 64 + SC_EPI;
constexpr uint32_t SC_A_BYTES = SC_M * SC_KCH * 2;   // 16 KB
constexpr uint32_t SC_B_BYTES = SC_N * SC_KCH * 2;   // 32 KB
constexpr uint64_t SC_WAIT_NS = 2000000000ull;       // 2 s per wait

constexpr int SC_CAP = 1024;       // collect pass: candidates per overflowed query

enum : int { SCR_KNN = 0, SCR_DEP = 1 };
enum : int { SCR_KEEP = 0, SCR_COLLECT = 1 };

struct ScreenArgs {
  int64_t nq;             // query rows (A operand)
  int64_t n;              // point rows (B operand)
  int kc;                 // 64-column chunks per row
  int k;                  // k-NN: the band is measured from the k-th kept key
  const int32_t* qids;    // global id of query row r (NULL: r)
  const float* pnorm2;    // squared norm of every point (L2 keys)
  const float* pnorm;     // norm of every point, rounded up (band)
  const float* maxnorm;   // the largest norm (device scalar)
  const float* rank_key;  // dependent mode: rank keys of every point
  // |approximate key - canonical key| <= E_q =
  //   dotfac (eps_rel |x_q| M + eps_abs) + eps_sq M^2, M = max norm,
  // dotfac = 2 for L2 (key |y|^2 - 2 <x, y>), 1 for IP (key -<x, y>)
  float eps_rel, eps_abs, eps_sq;
  // keep pass
  int32_t* out_ids;       // nq x SC_KEEP (collect pass: nq x cap)
  int32_t* out_cnt;       // nq; keep pass: -1 when the band overflowed the list
  float* out_thr;         // keep pass: threshold for the collect pass of an overflowed row
  int32_t* ovf_list;      // keep pass: overflowed query rows
  int32_t* ovf_cnt;
  // collect pass
  const float* in_thr;    // per query row
  int cap;
  int* err;
  // pacing (NULL: none): CTA producers count their arrivals at every epoch
  // of pace_every point tiles in pace[epoch]; before entering epoch e a
  // producer waits (bounded) until every CTA of the grid that sweeps epoch
  // e - pace_lag has entered it
  int* pace;
  int pace_every, pace_lag;
  int64_t pace_epochs;    // entries of pace[]
};

__device__ __forceinline__ bool rank_above_key(float kj, int32_t j, float ki, int32_t i) {
  return kj > ki || (kj == ki && j < i);
}

// Barrier of the SC_EPI epilogue threads that also ORs a flag over them.
__device__ __forceinline__ bool epi_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

// Max-heap of (key, id) per epilogue thread, slot-major: slot s of thread et
// at [s * SC_EPI + et]. cnt < SC_HALF: filling (sift up); full: a key below
// the root replaces it (sift down).
__device__ __forceinline__ void heap_push(float* hk, int32_t* hi, int et, int& cnt, float key, int32_t id) {
  if (cnt < SC_HALF) {
    int pos = cnt++;
    while (pos > 0) {
      const int par = (pos - 1) >> 1;
      const float pk = hk[par * SC_EPI + et];
      if (!(pk < key)) break;
      hk[pos * SC_EPI + et] = pk;
      hi[pos * SC_EPI + et] = hi[par * SC_EPI + et];
      pos = par;
    }
    hk[pos * SC_EPI + et] = key;
    hi[pos * SC_EPI + et] = id;
  } else {
    int pos = 0;
    for (;;) {
      int c = 2 * pos + 1;
      if (c >= SC_HALF) break;
      float ck = hk[c * SC_EPI + et];
      if (c + 1 < SC_HALF) {
        const float c2 = hk[(c + 1) * SC_EPI + et];
        if (c2 > ck) {
          ck = c2;
          c++;
        }
      }
      if (!(ck > key)) break;
      hk[pos * SC_EPI + et] = ck;
      hi[pos * SC_EPI + et] = hi[c * SC_EPI + et];
      pos = c;
    }
    hk[pos * SC_EPI + et] = key;
    hi[pos * SC_EPI + et] = id;
  }
}

// Sort a thread's heap ascending in place (heapsort).
__device__ __forceinline__ void heap_sort(float* hk, int32_t* hi, int et, int cnt) {
  for (int end = cnt - 1; end > 0; end--) {
    // move the root (largest) to `end`, sift the old last entry down
    const float key = hk[end * SC_EPI + et];
    const int32_t id = hi[end * SC_EPI + et];
    hk[end * SC_EPI + et] = hk[et];
    hi[end * SC_EPI + et] = hi[et];
    int pos = 0;
    for (;;) {
      int c = 2 * pos + 1;
      if (c >= end) break;
      float ck = hk[c * SC_EPI + et];
      if (c + 1 < end) {
        const float c2 = hk[(c + 1) * SC_EPI + et];
        if (c2 > ck) {
          ck = c2;
          c++;
        }
      }
      if (!(ck > key)) break;
      hk[pos * SC_EPI + et] = ck;
      hi[pos * SC_EPI + et] = hi[c * SC_EPI + et];
      pos = c;
    }
    hk[pos * SC_EPI + et] = key;
    hi[pos * SC_EPI + et] = id;
  }
}

constexpr uint64_t SC_PACE_NS = 100000000ull;  // 100 ms: then the CTA stops pacing

// Pacing of the point-tile sweep. Every CTA reads the whole point set once
// per query tile; the point rows (n x d BF16) are far larger than L2, so a
// tile read from HBM serves the other CTAs only while they sweep close to
// one another. Without a bound the CTAs drift apart over thousands of
// tiles and most tiles come from HBM again for each CTA. So the producer
// announces every epoch of pace_every tiles it enters and does not enter
// epoch e before all CTAs that sweep epoch e - pace_lag have entered that
// one. The grid is co-resident (cooperative launch) and the wait is bounded:
// after SC_PACE_NS the CTA gives up pacing for the rest of the launch, which
// changes its speed only, never its results. Returns whether to go on pacing.
__device__ __forceinline__ bool pace_enter(const ScreenArgs& a, int64_t epoch, int64_t epr, int64_t groups, int CL) {
  if (epoch >= a.pace_epochs) return false;
  atomicAdd(a.pace + epoch, 1);
  const int64_t e2 = epoch - a.pace_lag;
  if (e2 < 0) return true;
  // CTAs that sweep epoch e2: those with a query tile in its round
  const int64_t n_cl = gridDim.x / CL, round = e2 / epr;
  const int64_t left = groups - round * n_cl;
  const int need = (int)(CL * (left < n_cl ? left : n_cl));
  const volatile int* c = a.pace + e2;
  if (*c >= need) return true;
  const uint64_t t0 = tc::globaltimer_ns();
  for (;;) {
    __nanosleep(256);
    if (*c >= need) return true;
    if (tc::globaltimer_ns() - t0 > SC_PACE_NS) return false;
  }
}

// CL: CTAs per cluster. With CL > 1 the CTAs of a cluster take CL
// consecutive query tiles and sweep the point tiles in lockstep: each loads
// 1/CL of every point chunk (tb's box is SC_N / CL rows) and multicasts it to
// all of them, so a point chunk leaves L2 once per cluster; a stage is free
// again once every CTA's MMAs have read it (each MMA commit arrives on the
// stage's empty barrier in every CTA of the cluster). A CTA whose query tile
// lies past the last one still takes part, on rows that read as zeros and
// produce no output.
// Per cluster size: CL = 2 runs the pair form (one M = 256 MMA per CTA pair,
// each CTA holding its 128 query rows and half of the 256 point rows of a
// stage, so a stage is 32 KB and four fit); CL = 1 and 4 hold the whole
// point tile in each CTA.
template <int CL>
struct ScLayout {
  static constexpr bool PAIR = CL == 2;
  static constexpr int STAGES = PAIR ? 4 : SC_STAGES;
  static constexpr uint32_t B_BYTES = PAIR ? SC_B_BYTES / 2 : SC_B_BYTES;
  static constexpr uint32_t STAGE_BYTES = SC_A_BYTES + B_BYTES;
};

template <int MODE, int PASS, int METRIC, int CL>
__global__ void __launch_bounds__(SC_THREADS, 1)
    k_bf_screen(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, ScreenArgs a) {
  using L = ScLayout<CL>;
  constexpr bool PAIR = L::PAIR;
  constexpr int STAGES = L::STAGES;
  constexpr uint32_t STAGE_BYTES = L::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* ring = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* hk = reinterpret_cast<float*>(ring + STAGES * STAGE_BYTES);       // [SC_HALF][SC_EPI]
  int32_t* hi = reinterpret_cast<int32_t*>(hk + SC_HALF * SC_EPI);         // [SC_HALF][SC_EPI]
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], final_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int half_cnt[SC_EPI];   // heap sizes at the end of a query tile
  __shared__ int row_cnt[SC_M];      // collect pass: candidates per row

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_qt = (a.nq + SC_M - 1) / SC_M;
  const int64_t n_pt = (a.n + SC_N - 1) / SC_N;
  // query tiles: group g (of CL tiles) goes to cluster g mod (clusters);
  // the CTA of rank `crank` takes tile g * CL + crank
  const int64_t crank = CL > 1 ? (int64_t)tc::cluster_rank() : 0;
  const int64_t n_cl = gridDim.x / CL, cl_id = blockIdx.x / CL;
  constexpr uint16_t cl_mask = (uint16_t)((1u << CL) - 1);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; s++) {
      // pair: full_bar of the even CTA counts both CTAs' bytes; every MMA
      // commit arrives once on each CTA's empty_bar
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], PAIR ? 1 : CL);
    }
    for (int b = 0; b < 2; b++) {
      tc::mbar_init(&tfull_bar[b], 1);
      // pair: the even CTA's barrier takes the epilogue threads of both CTAs
      tc::mbar_init(&tempty_bar[b], PAIR ? 2 * SC_EPI : SC_EPI);
    }
    tc::mbar_init(&final_bar, 1);
    tc::fence_mbar_init();
  }
  if (threadIdx.x < SC_M) row_cnt[threadIdx.x] = 0;
  if (warp == 1) {
    if constexpr (PAIR) {
      tc::tmem_alloc_pair(&tmem_slot, 2 * SC_N);
      tc::tmem_relinquish_pair();
    } else {
      tc::tmem_alloc(&tmem_slot, 2 * SC_N);
      tc::tmem_relinquish();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (CL > 1) tc::cluster_sync();  // every peer's barriers exist before any multicast
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tc::prefetch_tmap(&ta);
      tc::prefetch_tmap(&tb);
      uint64_t it = 0;  // chunk loads issued
      bool ok = true;
      bool pacing = a.pace != nullptr;
      const int64_t epr = (n_pt + a.pace_every - 1) / (a.pace_every > 0 ? a.pace_every : 1);
      const int64_t groups = (n_qt + CL - 1) / CL;
      int64_t round = 0;
      for (int64_t g = cl_id; g * CL < n_qt && ok; g += n_cl, round++) {
        const int64_t qt = g * CL + crank;
        for (int64_t pt = 0; pt < n_pt && ok; pt++) {
          if (pacing && pt % a.pace_every == 0)
            pacing = pace_enter(a, round * epr + pt / a.pace_every, epr, groups, CL);
          for (int c = 0; c < a.kc; c++) {
            const int s = (int)(it % STAGES);
            const uint32_t ph = (uint32_t)((it / STAGES) & 1);
            if (!tc::mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, SC_WAIT_NS)) {
              ok = false;
              break;
            }
            uint8_t* st = ring + (size_t)s * STAGE_BYTES;
            if constexpr (PAIR) {
              // both CTAs' loads complete on the even CTA's full barrier
              const uint32_t fb = tc::mapa(tc::smem_u32(&full_bar[s]), 0);
              if (crank == 0) tc::mbar_arrive_expect_tx(&full_bar[s], 2 * STAGE_BYTES);
              tc::tma_load_2d_pair(st, &ta, c * SC_KCH, (int32_t)(qt * SC_M), fb);
              tc::tma_load_2d_pair(st + SC_A_BYTES, &tb, c * SC_KCH, (int32_t)(pt * SC_N + crank * (SC_N / 2)), fb);
            } else {
              tc::mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
              tc::tma_load_2d(st, &ta, c * SC_KCH, (int32_t)(qt * SC_M), &full_bar[s]);
              if (CL == 1)
                tc::tma_load_2d(st + SC_A_BYTES, &tb, c * SC_KCH, (int32_t)(pt * SC_N), &full_bar[s]);
              else
                tc::tma_load_2d_mc(st + SC_A_BYTES + crank * (SC_B_BYTES / CL), &tb, c * SC_KCH,
                                   (int32_t)(pt * SC_N + crank * (SC_N / CL)), &full_bar[s], cl_mask);
            }
            it++;
          }
        }
      }
      // loads still in flight land before the block exits: wait for the last
      // STAGES issued loads (bounded, whatever the abort flag says); in the
      // pair the even CTA's barriers count the odd CTA's loads too, and the
      // final cluster barrier holds the odd CTA until then
      int no_abort = 0;
      if (!PAIR || crank == 0)
        for (uint64_t j = it > STAGES ? it - STAGES : 0; j < it; j++)
          tc::mbar_wait(&full_bar[j % STAGES], (uint32_t)((j / STAGES) & 1), &no_abort, SC_WAIT_NS);
      if (!ok) set_error(a.err, ERR_TIMEOUT);
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (PAIR && crank != 0) {
      // the odd CTA of a pair issues nothing (see the end of the kernel)
    } else if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(PAIR ? 2 * SC_M : SC_M, SC_N);
      uint64_t it = 0, tile = 0;
      bool ok = true;
      for (int64_t g = cl_id; g * CL < n_qt && ok; g += n_cl) {
        for (int64_t pt = 0; pt < n_pt && ok; pt++, tile++) {
          const int b = (int)(tile & 1);
          if (!tc::mbar_wait(&tempty_bar[b], (uint32_t)(((tile >> 1) & 1) ^ 1), &abort_flag, SC_WAIT_NS)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t dacc = tmem + (uint32_t)(b * SC_N);
          for (int c = 0; c < a.kc; c++, it++) {
            const int s = (int)(it % STAGES);
            if (!tc::mbar_wait(&full_bar[s], (uint32_t)((it / STAGES) & 1), &abort_flag, SC_WAIT_NS)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_u32(ring + (size_t)s * STAGE_BYTES), sb = sa + SC_A_BYTES;
#pragma unroll
            for (int k = 0; k < SC_KCH / 16; k++) {
              if constexpr (PAIR)
                tc::mma_bf16_pair(dacc, tc::sdesc_sw128(sa + 32 * k), tc::sdesc_sw128(sb + 32 * k), idesc,
                                  (c | k) != 0);
              else
                tc::mma_bf16(dacc, tc::sdesc_sw128(sa + 32 * k), tc::sdesc_sw128(sb + 32 * k), idesc, (c | k) != 0);
            }
            if constexpr (PAIR)
              tc::mma_commit_pair(&empty_bar[s], cl_mask);
            else if (CL == 1)
              tc::mma_commit(&empty_bar[s]);
            else
              tc::mma_commit_mc(&empty_bar[s], cl_mask);
          }
          if (ok) {
            if constexpr (PAIR)
              tc::mma_commit_pair(&tfull_bar[b], cl_mask);
            else
              tc::mma_commit(&tfull_bar[b]);
          }
        }
      }
      // every MMA this thread issued completes before TMEM is released
      if constexpr (PAIR)
        tc::mma_commit_pair(&final_bar, cl_mask);
      else
        tc::mma_commit(&final_bar);
      int no_abort = 0;
      tc::mbar_wait(&final_bar, 0, &no_abort, SC_WAIT_NS);
      if (!ok) set_error(a.err, ERR_TIMEOUT);
    }
  } else {
    // ------------------------------------------------ epilogue
    const int et = threadIdx.x - 64;          // 0..255
    const int rl = 32 * (warp & 3) + lane;    // row of the tile = TMEM lane (this warp's quarter)
    const int half = (warp - 2) >> 2;         // columns [128 half, 128 half + 128) of each tile
    const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
    const float M = __ldg(a.maxnorm);
    uint64_t tile = 0;
    bool ok = true;
    for (int64_t g = cl_id; g * CL < n_qt && ok; g += n_cl) {
      const int64_t qt = g * CL + crank;
      const int64_t r = qt * SC_M + rl;
      const bool valid = r < a.nq;
      const int32_t qid = valid ? (a.qids ? __ldg(a.qids + r) : (int32_t)r) : -1;
      const float qkey = (MODE == SCR_DEP && valid) ? __ldg(a.rank_key + qid) : 0.0f;
      const float dotfac = METRIC == MET_L2 ? 2.0f : 1.0f;
      const float E = valid ? dotfac * (a.eps_rel * __ldg(a.pnorm + qid) * M + a.eps_abs) + a.eps_sq * M * M : 0.0f;
      // keep pass: a key is taken when below thr (the heap's largest once full)
      float thr = PASS == SCR_COLLECT ? (valid ? __ldg(a.in_thr + r) : -INFINITY) : (valid ? INFINITY : -INFINITY);
      int cnt = 0;
      for (int64_t pt = 0; pt < n_pt; pt++, tile++) {
        const int b = (int)(tile & 1);
        const int64_t j0 = pt * SC_N;
        if (!tc::mbar_wait(&tfull_bar[b], (uint32_t)((tile >> 1) & 1), &abort_flag, SC_WAIT_NS)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
#pragma unroll 1
        for (int c00 = 128 * half; c00 < 128 * half + 128; c00 += 64) {
          // 64 columns per TMEM load, taken as two 32-column chunks whose
          // minima are formed before either is taken apart (two independent
          // chains for the scheduler)
          float v[64];
          tc::tmem_ld64(tmem + lane_addr + (uint32_t)(b * SC_N + c00), v);
          // approximate keys, smaller = closer: -<x, y> (IP), |y|^2 - 2 <x, y>
          // (L2: the squared norms, padded past n, read four at a time
          // through L1, the same addresses for the whole warp)
          if (MODE == SCR_DEP) {
            // only points ranked above the query count: the others get the
            // worst key (rank keys padded past n with NaN, never above)
            const float4* k4 = reinterpret_cast<const float4*>(a.rank_key + j0 + c00);
            // (as a product: -inf, which gives key +inf under both metrics)
            const float worst = -INFINITY;
#pragma unroll
            for (int q = 0; q < 16; q++) {
              const float4 kk = __ldg(k4 + q);
              const float kv[4] = {kk.x, kk.y, kk.z, kk.w};
#pragma unroll
              for (int u = 0; u < 4; u++) {
                const int32_t j = (int32_t)(j0 + c00 + 4 * q + u);
                if (!rank_above_key(kv[u], j, qkey, qid)) v[4 * q + u] = worst;
              }
            }
          }
          if (METRIC == MET_L2) {
            const float4* m4 = reinterpret_cast<const float4*>(a.pnorm2 + j0 + c00);
#pragma unroll
            for (int q = 0; q < 16; q++) {
              const float4 nn = __ldg(m4 + q);
              // a masked column carries -inf as its product: its key is +inf
              v[4 * q + 0] = __fmaf_rn(-2.0f, v[4 * q + 0], nn.x);
              v[4 * q + 1] = __fmaf_rn(-2.0f, v[4 * q + 1], nn.y);
              v[4 * q + 2] = __fmaf_rn(-2.0f, v[4 * q + 2], nn.z);
              v[4 * q + 3] = __fmaf_rn(-2.0f, v[4 * q + 3], nn.w);
            }
          }
          // each chunk's best key by a tree of depth 5
          float best[2];
#pragma unroll
          for (int sub = 0; sub < 2; sub++) {
            float w[16];
#pragma unroll
            for (int t = 0; t < 16; t++)
              w[t] = METRIC == MET_L2 ? fminf(v[32 * sub + t], v[32 * sub + t + 16])
                                      : fmaxf(v[32 * sub + t], v[32 * sub + t + 16]);
#pragma unroll
            for (int h = 8; h >= 1; h >>= 1)
#pragma unroll
              for (int t = 0; t < h; t++) w[t] = METRIC == MET_L2 ? fminf(w[t], w[t + h]) : fmaxf(w[t], w[t + h]);
            best[sub] = METRIC == MET_L2 ? w[0] : -w[0];
          }
#pragma unroll
          for (int sub = 0; sub < 2; sub++) {
            if (!(PASS == SCR_COLLECT ? (best[sub] <= thr) : (best[sub] < thr))) continue;  // the common case
            // the columns that beat the threshold, then one at a time (a
            // compact loop: the key of column t is picked by selects)
            uint32_t hm = 0;
#pragma unroll
            for (int t = 0; t < 32; t++) {
              const float key = METRIC == MET_L2 ? v[32 * sub + t] : -v[32 * sub + t];
              hm |= (uint32_t)(PASS == SCR_COLLECT ? (key <= thr) : (key < thr)) << t;
            }
            const int64_t jbase = j0 + c00 + 32 * sub;
            if (jbase + 32 > a.n) hm &= jbase >= a.n ? 0u : (0xffffffffu >> (32 - (int)(a.n - jbase)));
            if (qid >= jbase && qid < jbase + 32) hm &= ~(1u << (qid - jbase));
            while (hm) {
              const int t = __ffs(hm) - 1;
              hm &= hm - 1;
              float key = v[32 * sub];
#pragma unroll
              for (int i = 1; i < 32; i++) key = t == i ? v[32 * sub + i] : key;
              if (METRIC != MET_L2) key = -key;
              const int32_t j = (int32_t)(jbase + t);
              if (PASS == SCR_COLLECT) {
                const int slot = atomicAdd(&row_cnt[rl], 1);
                if (slot < a.cap) a.out_ids[r * a.cap + slot] = j;
              } else if (key < thr) {  // thr may have dropped since the mask
                heap_push(hk, hi, et, cnt, key, j);
                if (cnt == SC_HALF) thr = hk[et];
              }
            }
          }
        }
        tc::fence_before_sync();
        if (PAIR && crank != 0)
          tc::mbar_arrive_cluster(tc::mapa(tc::smem_u32(&tempty_bar[b]), 0));
        else
          tc::mbar_arrive(&tempty_bar[b]);
      }
      // the decision to give up is made uniform over the epilogue threads
      // (a thread that left the loop early reaches this barrier too)
      if (epi_sync_or(!ok)) ok = false;
      if (!ok) break;
      // ---- the row's result: both halves of the row are complete here
      if (PASS == SCR_COLLECT) {
        epi_sync();
        if (half == 0) {
          if (valid) a.out_cnt[r] = row_cnt[rl];  // > cap: the exact SIMT kernels take this row
          row_cnt[rl] = 0;
        }
        epi_sync();
        continue;
      }
      heap_sort(hk, hi, et, cnt);
      half_cnt[et] = cnt;
      epi_sync();
      if (half == 0 && valid) {
        // merge the two sorted halves of the row (up to SC_KEEP entries)
        const int p2 = et + 128;
        const int n0 = cnt, n1 = half_cnt[p2];
        // the exact decision needs only the entries up to the reference and
        // those within the band above it (mb of them): a point whose
        // approximate key exceeds ref_key + 2E has a canonical key above
        // ref_key + E, the most the reference's canonical key can be
        int i0 = 0, i1 = 0, m = 0, mb = 0;
        const int ref = MODE == SCR_KNN ? a.k - 1 : 0;
        float ref_key = INFINITY, lim = INFINITY;
        int32_t* out = a.out_ids + r * SC_KEEP;
        while (i0 < n0 || i1 < n1) {
          const bool take0 = i1 >= n1 || (i0 < n0 && hk[i0 * SC_EPI + et] <= hk[i1 * SC_EPI + p2]);
          const float kk = take0 ? hk[i0 * SC_EPI + et] : hk[i1 * SC_EPI + p2];
          const int32_t id = take0 ? hi[i0 * SC_EPI + et] : hi[i1 * SC_EPI + p2];
          if (take0) i0++; else i1++;
          if (m == ref) {
            ref_key = kk;
            lim = ref_key + 2.0f * E;
          }
          if (m <= ref || kk <= lim) mb = m + 1;
          out[m++] = id;
        }
        // complete when each half either kept every point it saw, or its
        // largest kept key lies beyond the band around the reference key
        const bool c0ok = n0 < SC_HALF || hk[(n0 - 1) * SC_EPI + et] > lim;
        const bool c1ok = n1 < SC_HALF || hk[(n1 - 1) * SC_EPI + p2] > lim;
        if (m <= ref || (c0ok && c1ok)) {
          a.out_cnt[r] = mb;
        } else {
          a.out_cnt[r] = -1;
          a.out_thr[r] = lim;
          a.ovf_list[atomicAdd(a.ovf_cnt, 1)] = (int32_t)r;
        }
      }
      epi_sync();
    }
    if (!ok) set_error(a.err, ERR_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (PAIR && crank != 0 && threadIdx.x == 32) {
    // the odd CTA's TMEM is released only after the even CTA's last commit:
    // every MMA that writes it has completed
    int no_abort = 0;
    tc::mbar_wait(&final_bar, 0, &no_abort, SC_WAIT_NS);
  }
  // no CTA leaves while a peer may still write into its shared memory
  if (CL > 1) tc::cluster_sync();
  if (warp == 1) {
    tc::fence_after_sync();
    if constexpr (PAIR)
      tc::tmem_dealloc_pair(tmem, 2 * SC_N);
    else
      tc::tmem_dealloc(tmem, 2 * SC_N);
  }
}

// ---------------------------------------------------------------- helpers

// BF16 copy of FP32 or uint8 rows (round to nearest even; uint8 values are
// exact in BF16).
__global__ void k_rows_to_bf16(const uint8_t* X, int dtype, int64_t total, __nv_bfloat16* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = dtype == DT_F32 ? reinterpret_cast<const float*>(X)[i] : (float)X[i];
    out[i] = __float2bfloat16_rn(v);
  }
}

// Norm (rounded up) and squared norm of every row, and the largest norm.
// The sum of squares is taken in double: exact for uint8 rows (integers
// below 2^53), and within one FP32 rounding for FP32 rows.
__global__ void k_row_norms(const uint8_t* X, int dtype, int64_t n, int d, int64_t row_bytes, float* nrm,
                            float* nrm2, unsigned* maxbits) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < n; i += nw) {
    double s = 0.0;
    const uint8_t* row = X + i * row_bytes;
    for (int c = lane; c < d; c += 32) {
      const double v = dtype == DT_F32 ? (double)reinterpret_cast<const float*>(row)[c] : (double)row[c];
      s += v * v;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
    if (lane == 0) {
      const float nr = __double2float_ru(sqrt(s) * (1.0 + 1e-12));
      nrm2[i] = __double2float_rn(s);
      nrm[i] = nr;
      atomicMax(maxbits, __float_as_uint(nr));  // non-negative floats order like their bits
    }
  }
}

// Contiguous BF16 copy of the listed rows (the query operand of the
// dependent and collect passes). d is a multiple of 8: 16-byte pieces.
__global__ void k_gather_bf16(const __nv_bfloat16* rows, int d, const int32_t* list, int64_t m,
                              __nv_bfloat16* out) {
  const int64_t per = d / 8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m * per; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = i / per, c = i % per;
    reinterpret_cast<uint4*>(out)[u * per + c] =
        __ldg(reinterpret_cast<const uint4*>(rows) + (int64_t)list[u] * per + c);
  }
}

// The overflowed rows [off, off + m) of a keep pass: their query ids and
// collect thresholds, contiguous.
__global__ void k_overflow_rows(const int32_t* ovf, int64_t off, int64_t m, const int32_t* qids, const float* thr,
                                int32_t* out_ids, float* out_thr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t row = ovf[off + i];
    out_ids[i] = qids ? qids[row] : row;
    out_thr[i] = thr[row];
  }
}

// Rows of a collect pass beyond its capacity: their query ids go to the exact
// SIMT list, and their count becomes -1 so that the re-rank skips them.
__global__ void k_collect_overflow(int32_t* cnt, int64_t m, int cap, const int32_t* qids, int32_t* fb,
                                   int32_t* fb_cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    if (cnt[i] > cap) {
      fb[atomicAdd(fb_cnt, 1)] = qids[i];
      cnt[i] = -1;
    }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor map of n x d BF16 rows (row stride d * 2 bytes, a multiple of 16),
// boxes of 64 columns x box_rows rows, 128-byte swizzle; rows and columns
// beyond the matrix read as zeros. Box x coordinates are multiples of 64
// elements (128 bytes).
static cudaError_t make_map(CUtensorMap* m, const void* base, int64_t n, int d, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) {
    set_where("brute-force index: cuTensorMapEncodeTiled unavailable");
    return cudaErrorNotSupported;
  }
  cuuint64_t gdim[2] = {(cuuint64_t)d, (cuuint64_t)n};
  cuuint64_t gstride[1] = {(cuuint64_t)d * 2};
  cuuint32_t box[2] = {(cuuint32_t)SC_KCH, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim, gstride, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) set_where("brute-force index: tensor map");
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CL>
static size_t screen_smem() {
  return 1024 + (size_t)ScLayout<CL>::STAGES * ScLayout<CL>::STAGE_BYTES + 2 * (size_t)SC_HALF * SC_EPI * 4;
}

constexpr int64_t SC_PACE_MAX = 65536;  // entries of the pacing counters

template <int MODE, int PASS, int METRIC, int CL>
static cudaError_t launch_screen_t(const CUtensorMap& ta, const void* prows, int64_t n, int d, const ScreenArgs& a_in,
                                   cudaStream_t st) {
  ScreenArgs a = a_in;
  auto kern = k_bf_screen<MODE, PASS, METRIC, CL>;
  const size_t smem = screen_smem<CL>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    set_where("brute-force screen: shared-memory attribute");
    return e;
  }
  CUtensorMap tb;  // point rows: each CTA of a cluster loads SC_N / CL rows of a tile
  if ((e = make_map(&tb, prows, n, d, SC_N / CL)) != cudaSuccess) return e;
  const int64_t n_qt = (a.nq + SC_M - 1) / SC_M;
  const int64_t groups = (n_qt + CL - 1) / CL;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.blockDim = dim3(SC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CL > 1 ? 1 : 0;
  const int64_t n_pt = (n + SC_N - 1) / SC_N;
  // a persistent grid: as many clusters as can be resident at once (a
  // cluster's CTAs share one GPC, so with CL > 1 that can be fewer than
  // SMs / CL), never more than there are groups of query tiles
  int64_t resident = std::max<int64_t>(1, num_sms() / CL);
  if (CL > 1) {
    cfg.gridDim = dim3((unsigned)(CL * resident));
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) == cudaSuccess && nc > 0) resident = nc;
    cudaGetLastError();
  }
  cfg.gridDim = dim3((unsigned)(CL * std::max<int64_t>(1, std::min<int64_t>(groups, resident))));
  // pacing (see pace_enter): single-CTA clusters, point rows larger than
  // about a third of L2, a grid that is co-resident (cooperative launch);
  // the lead is bounded to about 32 MB of point rows in 4 epochs
  bool pace = false;
  if (CL == 1 && a.pace && (int64_t)n * d * 2 > ((int64_t)48 << 20) && cfg.gridDim.x > 1) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SC_THREADS, smem) == cudaSuccess && occ >= 1 &&
        (int64_t)cfg.gridDim.x <= (int64_t)occ * num_sms()) {
      const int64_t tile_bytes = (int64_t)SC_N * d * 2;
      int64_t every = std::max<int64_t>(1, std::max<int64_t>(4, ((int64_t)32 << 20) / tile_bytes) / 4);
      const int64_t rounds = (groups + cfg.gridDim.x - 1) / cfg.gridDim.x;
      while (rounds * ((n_pt + every - 1) / every) > SC_PACE_MAX) every *= 2;
      if (every <= (int64_t)1 << 30) {
        a.pace_every = (int)every;
        a.pace_lag = 4;
        a.pace_epochs = rounds * ((n_pt + every - 1) / every);
        pace = cudaMemsetAsync(a.pace, 0, (size_t)a.pace_epochs * 4, st) == cudaSuccess;
      }
    }
    cudaGetLastError();
  }
  if (!pace) a.pace = nullptr;
  if (pace) {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.numAttrs = 1;
  }
  e = cudaLaunchKernelEx(&cfg, kern, ta, tb, a);
  if (e != cudaSuccess && pace) {
    // the cooperative form was refused: the same launch without pacing
    cudaGetLastError();
    a.pace = nullptr;
    cfg.numAttrs = 0;
    e = cudaLaunchKernelEx(&cfg, kern, ta, tb, a);
  }
  note_launch();
  if (e != cudaSuccess) set_where("brute-force screen: launch");
  return e;
}

// cl: CTAs per cluster for the k-NN keep pass: 1 (single CTAs, paced
// sweep), 2 (CTA pairs, one 256-row MMA per pair) or 4 (clusters sharing
// point tiles by multicast); 0 = automatic: pairs for d >= 512, where the
// MMAs set the pace (1.28M x 1024: keep pass 2.32 -> 2.09-2.14 s, each CTA
// reading half as many operand bytes into shared memory per MMA), single
// CTAs below, where the epilogue does (1M x 128 uint8: 410 ms single, 472 ms
// in pairs). Clusters of 4 were no faster than single CTAs on either. The
// other passes run few query tiles and use 1.
static cudaError_t launch_screen(int mode, int pass, int metric, const CUtensorMap& ta, const void* prows, int64_t n,
                                 int d, const ScreenArgs& a, int cl, cudaStream_t st) {
  if (a.nq <= 0) return cudaSuccess;
  if (cl != 1 && cl != 2 && cl != 4) cl = d >= 512 ? 2 : 1;
  if (mode != SCR_KNN || pass != SCR_KEEP) cl = 1;
  if (metric == MET_IP) {
    if (mode == SCR_KNN && pass == SCR_KEEP) {
      if (cl == 4) return launch_screen_t<SCR_KNN, SCR_KEEP, MET_IP, 4>(ta, prows, n, d, a, st);
      if (cl == 2) return launch_screen_t<SCR_KNN, SCR_KEEP, MET_IP, 2>(ta, prows, n, d, a, st);
      return launch_screen_t<SCR_KNN, SCR_KEEP, MET_IP, 1>(ta, prows, n, d, a, st);
    }
    if (mode == SCR_KNN) return launch_screen_t<SCR_KNN, SCR_COLLECT, MET_IP, 1>(ta, prows, n, d, a, st);
    return pass == SCR_KEEP ? launch_screen_t<SCR_DEP, SCR_KEEP, MET_IP, 1>(ta, prows, n, d, a, st)
                            : launch_screen_t<SCR_DEP, SCR_COLLECT, MET_IP, 1>(ta, prows, n, d, a, st);
  }
  if (mode == SCR_KNN && pass == SCR_KEEP) {
    if (cl == 4) return launch_screen_t<SCR_KNN, SCR_KEEP, MET_L2, 4>(ta, prows, n, d, a, st);
    if (cl == 2) return launch_screen_t<SCR_KNN, SCR_KEEP, MET_L2, 2>(ta, prows, n, d, a, st);
    return launch_screen_t<SCR_KNN, SCR_KEEP, MET_L2, 1>(ta, prows, n, d, a, st);
  }
  if (mode == SCR_KNN) return launch_screen_t<SCR_KNN, SCR_COLLECT, MET_L2, 1>(ta, prows, n, d, a, st);
  return pass == SCR_KEEP ? launch_screen_t<SCR_DEP, SCR_KEEP, MET_L2, 1>(ta, prows, n, d, a, st)
                          : launch_screen_t<SCR_DEP, SCR_COLLECT, MET_L2, 1>(ta, prows, n, d, a, st);
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device scratch of the brute-force index (after the caller's own pieces).
struct BfWs {
  __nv_bfloat16* rows;   // n x d BF16 copy of the rows
  __nv_bfloat16* qrows;  // up to n gathered query rows
  float* nrm;            // n
  float* nrm2;           // n
  unsigned* maxbits;     // 1 (bits of the largest norm)
  int32_t* cand;         // n x SC_KEEP (a collect batch: rows x SC_CAP)
  int32_t* cnt;          // n
  float* thr;            // n
  int32_t* ovf;          // n overflowed rows
  int32_t* ovf_ids;      // n
  float* ovf_thr;        // n
  int32_t* fb;           // n query ids for the exact SIMT kernels
  int32_t* counters;     // [0] overflowed rows, [1] SIMT rows
  float* rkpad;          // dependent passes: rank keys, padded past n with NaN
  int* pace;             // SC_PACE_MAX pacing counters of the screen
};

size_t bf_ws_bytes(int64_t n, int d) {
  return 2 * al256((size_t)n * d * 2) + al256((size_t)n * SC_KEEP * 4) + 8 * al256((size_t)n * 4) +
         al256((size_t)SC_N * 4) + 256 + 256 + SC_PACE_MAX * 4 + al256((size_t)(n + SC_N) * 4);
}

static BfWs carve_bf(void* ws, int64_t n, int d) {
  BfWs w;
  uint8_t* p = (uint8_t*)ws;
  auto take = [&](size_t bytes) {
    uint8_t* q = p;
    p += al256(bytes);
    return q;
  };
  w.rows = (__nv_bfloat16*)take((size_t)n * d * 2);
  w.qrows = (__nv_bfloat16*)take((size_t)n * d * 2);
  w.cand = (int32_t*)take((size_t)n * SC_KEEP * 4);
  w.nrm = (float*)take((size_t)n * 4);
  w.nrm2 = (float*)take((size_t)(n + SC_N) * 4);  // padded: the screen reads whole 32-column chunks
  w.cnt = (int32_t*)take((size_t)n * 4);
  w.thr = (float*)take((size_t)n * 4);
  w.ovf = (int32_t*)take((size_t)n * 4);
  w.ovf_ids = (int32_t*)take((size_t)n * 4);
  w.ovf_thr = (float*)take((size_t)n * 4);
  w.fb = (int32_t*)take((size_t)n * 4);
  w.maxbits = (unsigned*)take(256);
  w.counters = (int32_t*)take(256);
  w.pace = (int*)take((size_t)SC_PACE_MAX * 4);
  w.rkpad = (float*)take((size_t)(n + SC_N) * 4);
  return w;
}

// Bounds of |approximate key - canonical key| (see ScreenArgs):
//  - FP32 rows: BF16 rounding of both rows gives (2 u + u^2) |x| |y| with
//    u = 2^-9, plus an allowance of 2^-12 |x| |y| for the FP32 accumulation
//    of the tensor cores and of the canonical sum; IP adds 2^-22 for the
//    rounding of 1 - s, L2 adds 2^-17 M^2 for the rounded squared norms and
//    the canonical sum of squared differences;
//  - uint8 rows: exact in BF16, every product and partial sum an integer
//    below 2^24, so only an allowance of one unit per 16-column MMA step.
static void eps_of(const DataView& fv, ScreenArgs* a) {
  if (fv.dtype == DT_U8) {
    a->eps_rel = 0.0f;
    a->eps_abs = (float)((fv.d + 15) / 16);
    a->eps_sq = 0.0f;
  } else {
    a->eps_rel = 1.0f / 256.0f + 1.0f / 4096.0f;
    a->eps_abs = fv.metric == MET_IP ? 1.0f / 4194304.0f : 0.0f;
    a->eps_sq = fv.metric == MET_L2 ? 1.0f / 131072.0f : 0.0f;
  }
}

static cudaError_t prepare_rows(const DataView& fv, const BfWs& w, cudaStream_t st) {
  const int64_t total = fv.n * (int64_t)fv.d;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
  k_rows_to_bf16<<<blocks, 256, 0, st>>>(fv.X, fv.dtype, total, w.rows);
  note_launch();
  cudaError_t e = cudaMemsetAsync(w.maxbits, 0, 4, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.nrm2 + fv.n, 0, (size_t)SC_N * 4, st);  // the padding
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.counters, 0, 256, st);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)std::min<int64_t>((fv.n * 32 + 255) / 256, (int64_t)num_sms() * 16);
  k_row_norms<<<nb, 256, 0, st>>>(fv.X, fv.dtype, fv.n, fv.d, fv.row_bytes, w.nrm, w.nrm2, w.maxbits);
  note_launch();
  return cudaGetLastError();
}

static ScreenArgs base_args(const DataView& fv, const BfWs& w, int* err) {
  ScreenArgs a;
  memset(&a, 0, sizeof(a));
  a.n = fv.n;
  a.kc = (fv.d + SC_KCH - 1) / SC_KCH;
  a.pnorm2 = w.nrm2;
  a.pnorm = w.nrm;
  a.maxnorm = reinterpret_cast<const float*>(w.maxbits);
  eps_of(fv, &a);
  a.err = err;
  a.pace = w.pace;
  return a;
}

static unsigned grid_for(int64_t m) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 8192)); }

static pecann_status read_count(const int32_t* d_cnt, int32_t* h, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(h, d_cnt, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_status(e, "brute-force index: readback");
}

// Collect passes over the overflowed rows of a keep pass (m on the host), in
// batches that fit the candidate buffer: each row's points under its
// threshold are gathered (up to SC_CAP) and handed to `decide`, which runs
// the exact re-rank on (query ids, candidates, counts, SC_CAP, rows); rows
// beyond the capacity go to w.fb for the exact SIMT kernels.
template <class DECIDE>
static pecann_status collect_passes(int mode, const DataView& fv, const BfWs& w,
                                    const int32_t* qids_of_rows, const float* rank_key, int k, int64_t m, int* err,
                                    cudaStream_t st, DECIDE decide) {
  const int64_t batch = std::max<int64_t>(1, (fv.n * SC_KEEP) / SC_CAP);
  pecann_status s;
  for (int64_t off = 0; off < m; off += batch) {
    const int64_t mb = std::min(batch, m - off);
    k_overflow_rows<<<grid_for(mb), 256, 0, st>>>(w.ovf, off, mb, qids_of_rows, w.thr, w.ovf_ids, w.ovf_thr);
    note_launch();
    k_gather_bf16<<<grid_for(mb * (fv.d / 8)), 256, 0, st>>>(w.rows, fv.d, w.ovf_ids, mb, w.qrows);
    note_launch();
    if ((s = cuda_status(cudaGetLastError(), "brute-force index: overflow rows"))) return s;
    CUtensorMap tq;
    if ((s = cuda_status(make_map(&tq, w.qrows, mb, fv.d, SC_M), "brute-force index"))) return s;
    ScreenArgs a = base_args(fv, w, err);
    a.nq = mb;
    a.k = k;
    a.qids = w.ovf_ids;
    a.rank_key = rank_key;
    a.in_thr = w.ovf_thr;
    a.cap = SC_CAP;
    a.out_ids = w.cand;
    a.out_cnt = w.cnt;
    if ((s = cuda_status(launch_screen(mode, SCR_COLLECT, fv.metric, tq, w.rows, fv.n, fv.d, a, 1, st), "brute-force collect pass")))
      return s;
    k_collect_overflow<<<grid_for(mb), 256, 0, st>>>(w.cnt, mb, SC_CAP, w.ovf_ids, w.fb, w.counters + 1);
    note_launch();
    if ((s = cuda_status(cudaGetLastError(), "brute-force index: collect overflow"))) return s;
    if ((s = decide(w.ovf_ids, w.cand, w.cnt, SC_CAP, mb))) return s;
  }
  return PECANN_OK;
}

pecann_status run_density_bf(const DataView& fv, const pecann_params* p, int32_t* knn_ids, float* knn_dist,
                             float* rho, float* rkey, int32_t* fb_list, int32_t* fb_cnt, int* err, void* bws,
                             int64_t* h_counts, cudaStream_t st) {
  const BfWs w = carve_bf(bws, fv.n, fv.d);
  pecann_status s;
  if ((s = cuda_status(prepare_rows(fv, w, st), "brute-force index: rows"))) return s;
  CUtensorMap tq;
  if ((s = cuda_status(make_map(&tq, w.rows, fv.n, fv.d, SC_M), "brute-force index"))) return s;
  ScreenArgs a = base_args(fv, w, err);
  a.nq = fv.n;
  a.k = p->k;
  a.out_ids = w.cand;
  a.out_cnt = w.cnt;
  a.out_thr = w.thr;
  a.ovf_list = w.ovf;
  a.ovf_cnt = w.counters + 0;
  if ((s = cuda_status(launch_screen(SCR_KNN, SCR_KEEP, fv.metric, tq, w.rows, fv.n, fv.d, a, p->block_warps, st), "brute-force screen"))) return s;
  // exact decision for the complete rows (overflowed rows carry -1: skipped)
  cudaError_t e = launch_rerank_knn(fv, nullptr, fv.n, w.cand, w.cnt, SC_KEEP, p->k, knn_ids, knn_dist, rho, rkey,
                                    p->density, fb_list, fb_cnt, st);
  if ((s = cuda_status(e, "brute-force index: exact k-NN"))) return s;
  int32_t m = 0;
  if ((s = read_count(w.counters + 0, &m, st))) return s;
  auto decide = [&](const int32_t* ids, const int32_t* cand, const int32_t* cnt, int K, int64_t rows) {
    return cuda_status(launch_rerank_knn(fv, ids, rows, cand, cnt, K, p->k, knn_ids, knn_dist, rho, rkey,
                                         p->density, fb_list, fb_cnt, st),
                       "brute-force index: exact k-NN");
  };
  if ((s = collect_passes(SCR_KNN, fv, w, nullptr, nullptr, p->k, m, err, st, decide))) return s;
  // rows beyond the collect capacity join the fallback list of the caller
  int32_t m2 = 0;
  if ((s = read_count(w.counters + 1, &m2, st))) return s;
  if (m2 > 0) {
    int32_t base = 0;
    if ((s = read_count(fb_cnt, &base, st))) return s;
    e = cudaMemcpyAsync(fb_list + base, w.fb, (size_t)m2 * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
      const int32_t total = base + m2;
      e = cudaMemcpyAsync(fb_cnt, &total, 4, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if ((s = cuda_status(e, "brute-force index: fallback list"))) return s;
  }
  if (h_counts) {
    h_counts[0] = m;
    h_counts[1] = m2;
  }
  return PECANN_OK;
}

pecann_status run_dep_bf(const DataView& fv, const float* rank_key, const int32_t* U, int64_t nu, int32_t* lam,
                         float* delta, int* err, void* bws, int64_t* h_counts, cudaStream_t st) {
  if (nu <= 0) return PECANN_OK;
  const BfWs w = carve_bf(bws, fv.n, fv.d);
  pecann_status s;
  if ((s = cuda_status(prepare_rows(fv, w, st), "brute-force index: rows"))) return s;
  // rank keys read four at a time by the screen: a copy padded with NaN
  // (never ranked above anything)
  cudaError_t e = cudaMemcpyAsync(w.rkpad, rank_key, (size_t)fv.n * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.rkpad + fv.n, 0xff, (size_t)SC_N * 4, st);
  if ((s = cuda_status(e, "brute-force index: rank keys"))) return s;
  rank_key = w.rkpad;
  k_gather_bf16<<<grid_for(nu * (fv.d / 8)), 256, 0, st>>>(w.rows, fv.d, U, nu, w.qrows);
  note_launch();
  if ((s = cuda_status(cudaGetLastError(), "brute-force index: gather"))) return s;
  CUtensorMap tq;
  if ((s = cuda_status(make_map(&tq, w.qrows, nu, fv.d, SC_M), "brute-force index"))) return s;
  ScreenArgs a = base_args(fv, w, err);
  a.nq = nu;
  a.qids = U;
  a.rank_key = rank_key;
  a.out_ids = w.cand;
  a.out_cnt = w.cnt;
  a.out_thr = w.thr;
  a.ovf_list = w.ovf;
  a.ovf_cnt = w.counters + 0;
  if ((s = cuda_status(launch_screen(SCR_DEP, SCR_KEEP, fv.metric, tq, w.rows, fv.n, fv.d, a, 1, st), "brute-force screen"))) return s;
  e = launch_rerank_dep(fv, U, nu, w.cand, w.cnt, SC_KEEP, lam, delta, st);
  if ((s = cuda_status(e, "brute-force index: exact dependent points"))) return s;
  int32_t m = 0;
  if ((s = read_count(w.counters + 0, &m, st))) return s;
  auto decide = [&](const int32_t* ids, const int32_t* cand, const int32_t* cnt, int K, int64_t rows) {
    return cuda_status(launch_rerank_dep(fv, ids, rows, cand, cnt, K, lam, delta, st),
                       "brute-force index: exact dependent points");
  };
  if ((s = collect_passes(SCR_DEP, fv, w, U, rank_key, 0, m, err, st, decide))) return s;
  int32_t m2 = 0;
  if ((s = read_count(w.counters + 1, &m2, st))) return s;
  if (m2 > 0) {
    // the exact SIMT tail; its per-query keys take the candidate buffer
    e = launch_dep_bruteforce(fv, w.fb, m2, rank_key, reinterpret_cast<unsigned long long*>(w.cand), lam, delta, st);
    if ((s = cuda_status(e, "brute-force index: exact tail"))) return s;
  }
  if (h_counts) {
    h_counts[0] = m;
    h_counts[1] = m2;
  }
  return PECANN_OK;
}

}  // namespace pecann

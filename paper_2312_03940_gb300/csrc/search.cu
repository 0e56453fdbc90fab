// Greedy beam search (Algorithm 1), one query per warp.
//
// Per warp, in shared memory:
//   beam   Lw keys, sorted ascending by (dis, id); bit 31 marks "visited".
//          This is L of Algorithm 1 with its visited part: popping the
//          closest unvisited point is a scan for the first unflagged entry.
//   ckeys  candidate keys of the current expansion (staging)
//   ss     the surviving candidates, sorted
//   vis    (build searches) the vcap closest expanded points
//   hash   a direct-mapped filter of ids already evaluated. It may forget an
//          id (two ids sharing a slot); the only cost is a repeated distance,
//          because a repeated point is either already in the beam with the
//          identical key (dropped as a duplicate by the merge) or no better
//          than the beam's current worst entry (dropped by the filter) --
//          exactly what Algorithm 1 does with a point it adds again.
//   cids   candidate ids
//
// One expansion: pop p*, read its R out-neighbours (coalesced), drop the
// query, seen ids and -1 padding, compute the canonical distances of the
// rest (W lanes per row, several rows per warp pass, loads of all rows issued
// before any arithmetic), drop candidates no better than the current L-th
// entry (they would be pruned at once), and merge the survivors into the
// sorted beam in place. Algorithm 1's k closest points of (L u V) are the
// first k beam entries: a visited point that left L was worse than all L
// points kept at that moment, and the L-th entry only improves afterwards.
#include <float.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"

namespace pecann {

struct WarpSmem {
  uint64_t* beam;
  uint64_t* ckeys;
  uint64_t* ss;
  uint64_t* vis;
  int32_t* hash;
  int32_t* cids;
};

int search_warp_bytes(int Lw, int log2h, int stage, int vcap, bool build) {
  size_t b = (size_t)Lw * 8 + (size_t)stage * 16 + (build ? (size_t)vcap * 8 : 0) +
             ((size_t)1 << log2h) * 4 + (size_t)stage * 4;
  return (int)((b + 15) & ~(size_t)15);
}

__device__ __forceinline__ WarpSmem carve(uint8_t* base, const SearchArgs& a) {
  WarpSmem w;
  w.beam = reinterpret_cast<uint64_t*>(base);
  w.ckeys = w.beam + a.Lw;
  w.ss = w.ckeys + a.stage;
  w.vis = w.ss + a.stage;
  w.hash = reinterpret_cast<int32_t*>(w.vis + (a.mode == MODE_BUILD ? a.vcap : 0));
  w.cids = w.hash + (1 << a.log2h);
  return w;
}

// Admit id y as a new candidate unless it is padding, the query or already
// evaluated (as far as the filter remembers). Collective over the warp.
__device__ __forceinline__ int admit(const SearchArgs& a, WarpSmem& w, int32_t y, int32_t q, int nc,
                                     int lane) {
  bool take = false;
  if (y >= 0) {
    if (y >= a.n) {
      set_error(a.err, ERR_BAD_ID);
    } else if (y != q) {
      uint32_t s = hash_slot(y, a.log2h);
      if (w.hash[s] != y) {
        w.hash[s] = y;
        take = true;
      }
    }
  }
  unsigned m = __ballot_sync(FULL, take);
  if (take) w.cids[nc + __popc(m & lanemask_lt())] = y;
  return nc + __popc(m);
}

// Candidate ids from the out-list of p.
__device__ __forceinline__ int gather_out(const SearchArgs& a, WarpSmem& w, int32_t p, int32_t q,
                                          int lane) {
  const int32_t* row = a.G + (int64_t)p * a.R;
  int nc = 0;
  for (int b = 0; b < a.R; b += 32) {
    int idx = b + lane;
    int32_t y = idx < a.R ? __ldg(row + idx) : -1;
    nc = admit(a, w, y, q, nc, lane);
  }
  __syncwarp();
  return nc;
}

// Candidate ids from the start points S[s0 .. s0 + stage); *q_in_s is set
// when the query itself is one of them.
__device__ __forceinline__ int gather_start(const SearchArgs& a, WarpSmem& w, int32_t q, int s0, int lane,
                                            bool* q_in_s) {
  int nc = 0;
  bool has_q = false;
  const int s1 = min(a.nS, s0 + a.stage);
  for (int b = s0; b < s1; b += 32) {
    int idx = b + lane;
    int32_t y = idx < s1 ? __ldg(a.S + idx) : -1;
    has_q |= __any_sync(FULL, y == q);
    nc = admit(a, w, y, q, nc, lane);
  }
  __syncwarp();
  *q_in_s |= has_q;
  return nc;
}

// Keys (canonical distance to the query, id) of the staged candidates.
template <int DT, int METRIC, int W, int CPL>
__device__ __forceinline__ void eval_cands(const SearchArgs& a, WarpSmem& w, int nc,
                                           const uint4 (&qv)[CPL], int lane) {
  constexpr int GR = 32 / W;
  constexpr int UNR = CPL >= 4 ? 1 : (CPL == 1 ? 4 : 2);
  const int g = lane / W, gl = lane % W;
  if (nc > GR * UNR) {
    // rows beyond the first batch: start their fetch now, so the later
    // batches find them in L2 instead of waiting a full DRAM round trip each
    for (int c = GR * UNR + lane; c < nc; c += 32) {
      const uint8_t* r = a.X + (int64_t)w.cids[c] * a.row_bytes;
      for (int64_t off = 0; off < a.row_bytes; off += 128) prefetch_l2(r + off);
    }
  }
  for (int c0 = 0; c0 < nc; c0 += GR * UNR) {
    uint4 r[UNR][CPL];
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      int c = c0 + u * GR + g;
      if (c < nc) {
        load_row<W, CPL, true>(a.X + (int64_t)w.cids[c] * a.row_bytes, gl, a.C, r[u]);
      } else {
#pragma unroll
        for (int t = 0; t < CPL; t++) r[u][t] = make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      float dv = group_dis<DT, METRIC, W, CPL>(qv, r[u]);
      int c = c0 + u * GR + g;
      if (gl == 0 && c < nc) w.ckeys[c] = make_key(dv, w.cids[c]);
    }
  }
  __syncwarp();
}

// Number of entries of the sorted clean keys s[0..m) below x.
__device__ __forceinline__ int count_below(const uint64_t* s, int m, uint64_t x) {
  int lo = 0, hi = m;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (s[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Merge the staged candidate keys into the beam (keep the Lw smallest keys,
// no duplicates). Returns the number of keys merged. Collective.
__device__ int merge_cands(WarpSmem& w, int& nb, int Lw, int nc, int& cursor, int lane) {
  // 1) drop candidates no better than the current worst entry of a full beam
  uint64_t worst = nb >= Lw ? key_clean(w.beam[Lw - 1]) : KEY_NONE;
  int m = 0;
  for (int b = 0; b < nc; b += 32) {
    int i = b + lane;
    uint64_t kk = i < nc ? w.ckeys[i] : KEY_NONE;
    bool keep = i < nc && kk < worst;
    unsigned bm = __ballot_sync(FULL, keep);
    __syncwarp();
    if (keep) w.ckeys[m + __popc(bm & lanemask_lt())] = kk;
    m += __popc(bm);
    __syncwarp();
  }
  if (m == 0) return 0;
  // 2) duplicates: of an earlier survivor, or of a beam entry
  for (int i = lane; i < m; i += 32) {
    uint64_t kk = w.ckeys[i];
    int lb = lower_bound_key(w.beam, nb, kk);
    bool dup = lb < nb && key_clean(w.beam[lb]) == kk;
    for (int j = 0; j < i && !dup; j++) dup = w.ckeys[j] == kk;
    w.cids[i] = dup ? 0 : 1;
  }
  __syncwarp();
  // 3) sort the survivors by rank counting
  int m2 = 0;
  for (int i = 0; i < m; i++) m2 += w.cids[i];
  for (int i = lane; i < m; i += 32) {
    if (!w.cids[i]) continue;
    uint64_t kk = w.ckeys[i];
    int rank = 0;
    for (int j = 0; j < m; j++) rank += (w.cids[j] && w.ckeys[j] < kk);
    w.ss[rank] = kk;
  }
  __syncwarp();
  if (m2 == 0) return 0;
  // 4) insertion points in the old beam
  for (int r = lane; r < m2; r += 32) w.cids[r] = lower_bound_key(w.beam, nb, w.ss[r]);
  __syncwarp();
  const int p0 = w.cids[0];
  // 5) shift the beam entries at or after p0, from the back, in place
  for (int hi = nb - 1; hi >= p0; hi -= 32) {
    int idx = hi - lane;
    uint64_t e = 0;
    int dst = Lw;
    if (idx >= p0) {
      e = w.beam[idx];
      dst = idx + count_below(w.ss, m2, key_clean(e));
    }
    __syncwarp();
    if (dst < Lw) w.beam[dst] = e;
    __syncwarp();
  }
  // 6) place the survivors
  for (int r = lane; r < m2; r += 32) {
    int dst = r + w.cids[r];
    if (dst < Lw) w.beam[dst] = w.ss[r];
  }
  __syncwarp();
  nb = min(Lw, nb + m2);
  if (p0 < cursor) cursor = p0;
  return m2;
}

// First unvisited beam entry at or after `from` (-1 if none); *next gets the
// second one when it lies in the same 32-entry window (else -1).
__device__ __forceinline__ int find_unvisited(const uint64_t* beam, int nb, int from, int lane, int* next) {
  for (int b = from; b < nb; b += 32) {
    int i = b + lane;
    bool u = i < nb && !(beam[i] & VFLAG);
    unsigned m = __ballot_sync(FULL, u);
    if (m) {
      unsigned rest = m & (m - 1);
      *next = rest ? b + __ffs(rest) - 1 : -1;
      return b + __ffs(m) - 1;
    }
  }
  *next = -1;
  return -1;
}

// Keep the vcap closest expanded points (build searches).
__device__ __forceinline__ void record_visit(WarpSmem& w, int& nv, int vcap, uint64_t e, int lane) {
  if (nv < vcap) {
    if (lane == 0) w.vis[nv] = e;
    nv++;
  } else {
    uint64_t mx = 0;
    int mi = -1;
    for (int i = lane; i < vcap; i += 32)
      if (w.vis[i] > mx) {
        mx = w.vis[i];
        mi = i;
      }
    uint64_t gm = mx;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      uint64_t o = __shfl_xor_sync(FULL, gm, off);
      gm = o > gm ? o : gm;
    }
    if (e < gm && mi >= 0 && mx == gm) w.vis[mi] = e;
  }
  __syncwarp();
}

// Density of a point from its first k beam entries (Sec. 4.2, Appendix A).
// Separate rounded operations, as the definition reads.
__device__ void density_from_beam(const uint64_t* beam, int k, int metric, int fn, float* rho,
                                  float* key) {
  if (fn == PECANN_DENS_KTH) {
    float D = out_dist(key_dis(key_clean(beam[k - 1])), metric);
    float r = __fdiv_rn(1.0f, D);
    *rho = r;
    *key = r;
    return;
  }
  float s = 0.0f;
  for (int t = 0; t < k; t++) {
    float dis = key_dis(key_clean(beam[t]));
    float D = out_dist(dis, metric);
    float d2 = metric == MET_L2 ? dis : __fmul_rn(D, D);
    if (fn == PECANN_DENS_EXPSUM)
      s = __fadd_rn(s, d2);
    else if (fn == PECANN_DENS_SUMEXP)
      s = __fadd_rn(s, expf(-d2));
    else
      s = __fadd_rn(s, D);
  }
  if (fn == PECANN_DENS_EXPSUM) {
    float kk = __fdiv_rn(-s, (float)k);
    *key = kk;
    *rho = expf(kk);
  } else if (fn == PECANN_DENS_SUMEXP) {
    float r = __fdiv_rn(s, (float)k);
    *rho = r;
    *key = r;
  } else {
    *rho = -s;
    *key = -s;
  }
}

template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(256, 5) k_search(SearchArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int H = 1 << a.log2h;
  const int gl = lane % W;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t qi = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; qi < a.nq; qi += nwarps) {
    const int32_t q = a.queries ? __ldg(a.queries + qi) : (int32_t)qi;
    if (q < 0 || q >= a.n) {
      if (lane == 0) set_error(a.err, ERR_BAD_ID);
      continue;
    }
    uint4 qv[CPL];
    load_row<W, CPL, false>(a.X + (int64_t)q * a.row_bytes, gl, a.C, qv);
    for (int i = lane; i < H; i += 32) w.hash[i] = -1;
    __syncwarp();
    if (lane == 0) w.hash[hash_slot(q, a.log2h)] = q;
    __syncwarp();
    int nb = 0, cursor = 0, nv = 0;
    // L <- S. A query that is itself in S (always, for the k-NN and
    // dependent searches, whose S is {x_i}) is popped first: its out-list
    // joins L and the query stays out of the beam.
    // A start set larger than the staging area goes through the merge in
    // chunks; keeping the Lw closest of each merge leaves the Lw closest
    // points of S, which is what the first prune of Algorithm 1 keeps.
    bool q_in_s = a.S == nullptr;
    int nc = 0;
    int64_t evals = 0;
    for (int s0 = 0; a.S && s0 < a.nS; s0 += a.stage) {
      nc = gather_start(a, w, q, s0, lane, &q_in_s);
      if (nc) {
        eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
        merge_cands(w, nb, a.Lw, nc, cursor, lane);
        evals += nc;
      }
    }
    int64_t iters = 0;
    if (q_in_s) {
      nc = gather_out(a, w, q, q, lane);
      iters = 1;
      if (nc) {
        eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
        merge_cands(w, nb, a.Lw, nc, cursor, lane);
        evals += nc;
      }
    }
    for (;;) {
      // p* <- argmin over L \ V
      int next;
      int pos = find_unvisited(w.beam, nb, cursor, lane, &next);
      if (pos < 0) break;
      uint64_t e = w.beam[pos];
      // the runner-up is usually the next point popped: fetch its out-list early
      if (next >= 0 && lane < (a.R * 4 + 127) / 128)
        prefetch_l2(a.G + (int64_t)key_id(w.beam[next]) * a.R + lane * 32);
      __syncwarp();
      if (lane == 0) w.beam[pos] = e | VFLAG;  // V <- V u {p*}
      __syncwarp();
      cursor = pos + 1;
      const int32_t p = key_id(e);
      if (a.mode == MODE_BUILD) record_visit(w, nv, a.vcap, key_clean(e), lane);
      // L <- L u E_out(p*), keeping the Lw closest
      nc = gather_out(a, w, p, q, lane);
      if (nc) {
        eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
        merge_cands(w, nb, a.Lw, nc, cursor, lane);
        evals += nc;
      }
      if (++iters > a.n + 1) {
        if (lane == 0) set_error(a.err, ERR_NO_PROGRESS);
        break;
      }
    }
    if (a.work && lane == 0) {
      atomicAdd(a.work, (unsigned long long)iters);
      atomicAdd(a.work + 1, (unsigned long long)evals);
    }
    // ---- epilogues
    if (a.mode == MODE_RAW || a.mode == MODE_KNN) {
      const int cnt = min(nb, a.k);
      const int64_t row = a.mode == MODE_RAW ? qi : (int64_t)q;
      for (int t = lane; t < a.k; t += 32) {
        int32_t id = -1;
        float dv = INFINITY;
        if (t < cnt) {
          uint64_t e = key_clean(w.beam[t]);
          id = key_id(e);
          dv = key_dis(e);
          if (a.mode == MODE_KNN) dv = out_dist(dv, a.metric);
        }
        a.out_ids[row * a.k + t] = id;
        a.out_dis[row * a.k + t] = dv;
      }
      if (a.mode == MODE_RAW) {
        if (lane == 0) a.out_cnt[qi] = cnt;
      } else if (lane == 0) {
        if (cnt < a.k) {
          a.fb_list[atomicAdd(a.fb_cnt, 1)] = q;
        } else {
          density_from_beam(w.beam, a.k, a.metric, a.density_fn, a.rho + q, a.rkey + q);
        }
      }
    } else if (a.mode == MODE_DEP) {
      // DPBruteForce over the returned points: the first one ranked above q
      for (int b = 0; b < nb; b += 32) {
        int t = b + lane;
        uint64_t e = 0;
        bool ok = false;
        if (t < nb) {
          e = key_clean(w.beam[t]);
          ok = ranks_above(a.rank_key, key_id(e), q);
        }
        unsigned m = __ballot_sync(FULL, ok);
        if (m) {
          if (lane == __ffs(m) - 1) {
            a.lam[q] = key_id(e);
            a.delta[q] = out_dist(key_dis(e), a.metric);
          }
          break;
        }
      }
    } else {
      const int m = min(nv, a.vcap);
      for (int t = lane; t < m; t += 32) {
        uint64_t e = w.vis[t];
        a.vis_ids[qi * a.vcap + t] = key_id(e);
        a.vis_dis[qi * a.vcap + t] = key_dis(e);
      }
      if (lane == 0) a.vis_cnt[qi] = m;
    }
    __syncwarp();
  }
}

// ----------------------------------------------------------------- layouts

bool pick_layout(int dtype, int metric, int d, Layout* out) {
  int epc = dtype == DT_F32 ? 4 : (dtype == DT_BF16 ? 8 : 16);
  if (d <= 0 || d % epc) return false;
  if (dtype == DT_U8 && (metric != MET_L2 || d > 256)) return false;
  if (dtype == DT_FP8) return false;  // FP8 traversal has no kernel in this build
  int C = d / epc;
  if (C <= 8) {
    *out = {8, 1};
  } else if (C <= 16) {
    *out = {16, 1};
  } else if (C <= 32) {
    *out = {32, 1};
  } else if (C <= 64) {
    *out = {32, 2};
  } else if (C <= 96) {
    *out = {32, 3};
  } else if (C <= 128) {
    *out = {32, 4};
  } else if (C <= 256) {
    *out = {32, 8};
  } else {
    return false;
  }
  return true;
}

template <int DT, int METRIC, int W, int CPL>
static cudaError_t launch_inst(const SearchArgs& a, cudaStream_t st) {
  auto kern = k_search<DT, METRIC, W, CPL>;
  int wpb = 8;
  while (wpb > 1 && (size_t)wpb * a.warp_bytes > 200 * 1024) wpb >>= 1;
  size_t smem = (size_t)wpb * a.warp_bytes;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    set_where("search: shared-memory attribute");
    return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
  if (e != cudaSuccess) {
    set_where("search: occupancy query");
    return e;
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t want = (a.nq + wpb - 1) / wpb;
  int64_t cap = (int64_t)num_sms() * per_sm;
  int grid = (int)(want < cap ? want : cap);
  if (grid < 1) grid = 1;
  kern<<<grid, wpb * 32, smem, st>>>(a); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_search(const DataView& dv, SearchArgs a, cudaStream_t st) {
  Layout L;
  if (!pick_layout(dv.dtype, dv.metric, dv.d, &L)) return cudaErrorNotSupported;
  if (a.nq <= 0) return cudaSuccess;
#define PECANN_INST(DT, MET)                                                  \
  if (L.W == 8) return launch_inst<DT, MET, 8, 1>(a, st);                     \
  if (L.W == 16) return launch_inst<DT, MET, 16, 1>(a, st);                   \
  if (L.CPL == 1) return launch_inst<DT, MET, 32, 1>(a, st);                  \
  if (L.CPL == 2) return launch_inst<DT, MET, 32, 2>(a, st);                  \
  if (L.CPL == 3) return launch_inst<DT, MET, 32, 3>(a, st);                  \
  if (L.CPL == 4) return launch_inst<DT, MET, 32, 4>(a, st);                  \
  return launch_inst<DT, MET, 32, 8>(a, st);
  if (dv.dtype == DT_F32 && dv.metric == MET_L2) {
    PECANN_INST(DT_F32, MET_L2)
  }
  if (dv.dtype == DT_F32 && dv.metric == MET_IP) {
    PECANN_INST(DT_F32, MET_IP)
  }
  if (dv.dtype == DT_U8) {
    if (L.W == 8) return launch_inst<DT_U8, MET_L2, 8, 1>(a, st);
    return launch_inst<DT_U8, MET_L2, 16, 1>(a, st);
  }
#undef PECANN_INST
  return cudaErrorNotSupported;
}

}  // namespace pecann

// ----------------------------------------------------------------- brute-force k-NN

namespace pecann {

struct BfKnnArgs {
  SearchArgs a;         // X, row_bytes, n, C, metric, k, outputs, density_fn, err
  const int32_t* list;  // queries
  const int32_t* cnt;   // number of queries in list (device)
  int64_t max_list;
};

// Exact k nearest points of each listed query over all other points, for the
// queries whose graph search returned fewer than k points (Sec. 4.1). The
// top-k is kept as a sorted beam of width k; every point is a candidate.
template <int DT, int METRIC, int W, int CPL>
__global__ void __launch_bounds__(128) k_bf_knn(BfKnnArgs b) {
  extern __shared__ __align__(16) uint8_t smem[];
  const SearchArgs& a = b.a;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem w = carve(smem + (size_t)wib * a.warp_bytes, a);
  const int gl = lane % W;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t m = min((int64_t)*b.cnt, b.max_list);
  for (int64_t li = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; li < m; li += nwarps) {
    const int32_t q = b.list[li];
    uint4 qv[CPL];
    load_row<W, CPL, false>(a.X + (int64_t)q * a.row_bytes, gl, a.C, qv);
    int nb = 0, cursor = 0;
    for (int64_t j0 = 0; j0 < a.n; j0 += a.stage) {
      int nc = 0;
      for (int bb = 0; bb < a.stage; bb += 32) {
        int64_t j = j0 + bb + lane;
        bool take = j < a.n && j != q;
        unsigned mm = __ballot_sync(FULL, take);
        if (take) w.cids[nc + __popc(mm & lanemask_lt())] = (int32_t)j;
        nc += __popc(mm);
      }
      __syncwarp();
      if (nc) {
        eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
        merge_cands(w, nb, a.k, nc, cursor, lane);
      }
    }
    const int cnt = min(nb, a.k);
    for (int t = lane; t < a.k; t += 32) {
      int32_t id = -1;
      float dv = INFINITY;
      if (t < cnt) {
        uint64_t e = key_clean(w.beam[t]);
        id = key_id(e);
        dv = out_dist(key_dis(e), a.metric);
      }
      a.out_ids[(int64_t)q * a.k + t] = id;
      a.out_dis[(int64_t)q * a.k + t] = dv;
    }
    __syncwarp();
    if (lane == 0 && cnt == a.k) density_from_beam(w.beam, a.k, a.metric, a.density_fn, a.rho + q, a.rkey + q);
    __syncwarp();
  }
}

template <int DT, int METRIC, int W, int CPL>
static cudaError_t launch_bf_inst(const BfKnnArgs& b, cudaStream_t st) {
  auto kern = k_bf_knn<DT, METRIC, W, CPL>;
  const int wpb = 4;
  size_t smem = (size_t)wpb * b.a.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = num_sms() * 2;
  kern<<<grid, wpb * 32, smem, st>>>(b); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bruteforce_knn(const DataView& dv, const int32_t* d_list, const int32_t* d_cnt,
                                  int64_t max_list, int k, int32_t* knn_ids, float* knn_dist,
                                  float* rho, float* rkey, int density_fn, int* err, cudaStream_t st) {
  Layout L;
  if (!pick_layout(dv.dtype, dv.metric, dv.d, &L)) return cudaErrorNotSupported;
  BfKnnArgs b;
  memset(&b, 0, sizeof(b));
  SearchArgs& a = b.a;
  a.X = dv.X;
  a.row_bytes = dv.row_bytes;
  a.n = dv.n;
  a.C = dv.C;
  a.metric = dv.metric;
  a.Lw = k;
  a.k = k;
  a.stage = 64;
  a.log2h = 0;
  a.mode = MODE_KNN;
  a.warp_bytes = search_warp_bytes(k, 0, a.stage, 0, false);
  a.out_ids = knn_ids;
  a.out_dis = knn_dist;
  a.rho = rho;
  a.rkey = rkey;
  a.density_fn = density_fn;
  a.err = err;
  b.list = d_list;
  b.cnt = d_cnt;
  b.max_list = max_list;
  if ((size_t)4 * a.warp_bytes > 227 * 1024) return cudaErrorInvalidConfiguration;
#define PECANN_BINST(DT, MET)                                                 \
  if (L.W == 8) return launch_bf_inst<DT, MET, 8, 1>(b, st);                  \
  if (L.W == 16) return launch_bf_inst<DT, MET, 16, 1>(b, st);                \
  if (L.CPL == 1) return launch_bf_inst<DT, MET, 32, 1>(b, st);               \
  if (L.CPL == 2) return launch_bf_inst<DT, MET, 32, 2>(b, st);               \
  if (L.CPL == 3) return launch_bf_inst<DT, MET, 32, 3>(b, st);               \
  if (L.CPL == 4) return launch_bf_inst<DT, MET, 32, 4>(b, st);               \
  return launch_bf_inst<DT, MET, 32, 8>(b, st);
  if (dv.dtype == DT_F32 && dv.metric == MET_L2) {
    PECANN_BINST(DT_F32, MET_L2)
  }
  if (dv.dtype == DT_F32 && dv.metric == MET_IP) {
    PECANN_BINST(DT_F32, MET_IP)
  }
  if (dv.dtype == DT_U8) {
    if (L.W == 8) return launch_bf_inst<DT_U8, MET_L2, 8, 1>(b, st);
    return launch_bf_inst<DT_U8, MET_L2, 16, 1>(b, st);
  }
#undef PECANN_BINST
  return cudaErrorNotSupported;
}

}  // namespace pecann

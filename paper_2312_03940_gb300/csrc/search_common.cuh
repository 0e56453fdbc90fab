// Device helpers of the beam-search kernels (search.cu): per-warp
// shared-memory carving, admission of candidate ids through the seen-filter,
// candidate scoring, the merge into the sorted beam, visit recording and the
// density epilogue.
#pragma once

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

inline int search_warp_bytes_impl(int Lw, int log2h, int stage, int vcap, bool build) {
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

// Admit id y as a new candidate unless it is padding (< 0), the query or
// already evaluated (as far as the filter remembers); an id >= n is skipped
// and noted in *bad. TB: tag bytes of the filter (1 or 2: slot = low id bits,
// tag = the remaining high bits, so a match still means exactly this id; 4:
// whole ids at a hashed slot). Every slot index is masked, so the table
// lookups stay in bounds for any y and need no branch. Collective.
template <int TB>
__device__ __forceinline__ int admit(const SearchArgs& a, WarpSmem& w, int32_t y, int32_t q, int nc,
                                     unsigned lt, bool* bad) {
  const bool cand = ((uint32_t)y < (uint32_t)a.n) & (y != q);
  *bad |= y >= a.n;
  bool take;
  if constexpr (TB == 1) {
    uint8_t* h = reinterpret_cast<uint8_t*>(w.hash);
    const uint32_t s = (uint32_t)y & ((4u << a.log2h) - 1);
    const uint8_t tag = (uint8_t)((uint32_t)y >> (a.log2h + 2));
    take = cand & (h[s] != tag);
    if (take) h[s] = tag;
  } else if constexpr (TB == 2) {
    uint16_t* h = reinterpret_cast<uint16_t*>(w.hash);
    const uint32_t s = (uint32_t)y & ((2u << a.log2h) - 1);
    const uint16_t tag = (uint16_t)((uint32_t)y >> (a.log2h + 1));
    take = cand & (h[s] != tag);
    if (take) h[s] = tag;
  } else {
    const uint32_t s = hash_slot(y, a.log2h);
    take = cand & (w.hash[s] != y);
    if (take) w.hash[s] = y;
  }
  const unsigned m = __ballot_sync(FULL, take);
  if (take) w.cids[nc + __popc(m & lt)] = y;
  return nc + __popc(m);
}

// Candidate ids from the out-list of p.
template <int TB>
__device__ __forceinline__ int gather_out_t(const SearchArgs& a, WarpSmem& w, int32_t p, int32_t q, int lane,
                                            unsigned lt, bool* bad) {
  const int32_t* row = a.G + wide_mul(p, a.R);
  int nc = 0;
  if ((a.R & 63) == 0 && (((uintptr_t)a.G) & 7) == 0) {
    // 8-byte aligned rows of a multiple of 64 ids: two ids per lane per load
    for (int b = 0; b < a.R; b += 64) {
      const int2 yy = __ldg(reinterpret_cast<const int2*>(row + b) + lane);
      nc = admit<TB>(a, w, yy.x, q, nc, lt, bad);
      nc = admit<TB>(a, w, yy.y, q, nc, lt, bad);
    }
  } else {
    for (int b = 0; b < a.R; b += 32) {
      const int idx = b + lane;
      const int32_t y = idx < a.R ? __ldg(row + idx) : -1;
      nc = admit<TB>(a, w, y, q, nc, lt, bad);
    }
  }
  __syncwarp();
  return nc;
}

__device__ __forceinline__ int gather_out(const SearchArgs& a, WarpSmem& w, int32_t p, int32_t q, int lane,
                                          unsigned lt, bool* bad) {
  if (a.tag_bytes == 1) return gather_out_t<1>(a, w, p, q, lane, lt, bad);
  if (a.tag_bytes == 2) return gather_out_t<2>(a, w, p, q, lane, lt, bad);
  return gather_out_t<4>(a, w, p, q, lane, lt, bad);
}

// Candidate ids from the start points S[s0 .. s0 + stage); *q_in_s is set
// when the query itself is one of them.
__device__ __forceinline__ int gather_start(const SearchArgs& a, WarpSmem& w, int32_t q, int s0, int lane,
                                            unsigned lt, bool* bad, bool* q_in_s) {
  int nc = 0;
  bool has_q = false;
  const int s1 = min(a.nS, s0 + a.stage);
  for (int b = s0; b < s1; b += 32) {
    int idx = b + lane;
    int32_t y = idx < s1 ? __ldg(a.S + idx) : -1;
    has_q |= __any_sync(FULL, y == q);
    if (a.tag_bytes == 1)
      nc = admit<1>(a, w, y, q, nc, lt, bad);
    else if (a.tag_bytes == 2)
      nc = admit<2>(a, w, y, q, nc, lt, bad);
    else
      nc = admit<4>(a, w, y, q, nc, lt, bad);
  }
  __syncwarp();
  *q_in_s |= has_q;
  return nc;
}

// Append the keys of this pass that beat `worst` (those a full beam could
// take) to the front of ckeys: `has` marks the lanes that hold a key.
__device__ __forceinline__ void keep_keys(WarpSmem& w, bool has, uint64_t key, uint64_t worst, int& m,
                                          unsigned lt) {
  const bool keep = has && key < worst;
  const unsigned mk = __ballot_sync(FULL, keep);
  if (keep) w.ckeys[m + __popc(mk & lt)] = key;
  m += __popc(mk);
}

template <bool PACK>
__device__ __forceinline__ void put_key(WarpSmem& w, bool has, uint64_t key, int c, uint64_t worst, int& m,
                                        unsigned lt) {
  if constexpr (PACK)
    keep_keys(w, has, key, worst, m, lt);
  else if (has)
    w.ckeys[c] = key;
}

// Keys (canonical distance to the query, id) of the staged candidates; the
// ones below `worst` are packed at the front of ckeys (in no particular
// order) and their number is returned. With worst = KEY_NONE every key is
// kept.
// PACK (layouts of 4 or 8 lanes per row, several keys per pass): keys are
// filtered and packed as they are made; otherwise (one or two keys per pass)
// key c goes to ckeys[c], all nc of them, and nc is returned.
template <int DT, int METRIC, int W, int CPL, int QC, bool PACK = (W <= 8)>
__device__ __forceinline__ int eval_cands(const SearchArgs& a, WarpSmem& w, int nc, const uint4 (&qv)[QC],
                                          int lane, uint64_t worst = KEY_NONE) {
  constexpr int GR = 32 / W;
  const unsigned lt = lanemask_lt();
  int m = 0;
  // rows per lane group per pass (the 4-lane uint8 layout takes 4: one L2
  // round trip covers 32 rows)
  constexpr bool U8W4 = DT == DT_U8 && W == 4 && CPL == 2;
  constexpr int UNR = CPL >= 4 ? 1 : (CPL == 1 || U8W4 ? 4 : 2);
  const int g = lane / W, gl = lane % W;
  if (nc > GR * UNR) {
    // rows beyond the first batch: start their fetch now, so the later
    // batches find them in L2 instead of waiting a full DRAM round trip each
    for (int c = GR * UNR + lane; c < nc; c += 32) {
      const uint8_t* r = a.X + wide_mul(w.cids[c], a.row_bytes);
      for (int64_t off = 0; off < a.row_bytes; off += 128) prefetch_l2(r + off);
    }
  }
  for (int c0 = 0; c0 < nc; c0 += GR * UNR) {
    if constexpr (DT == DT_U8 && W == 4 && CPL == 2) {
      if (nc - c0 <= GR) {
        // at most one row per lane group left: a pass of GR rows
        const int c = c0 + g;
        uint4 r1[2];
        ldg_nc_32b(a.X + wide_mul(w.cids[min(c, nc - 1)], a.row_bytes) + 32 * gl, r1[0], r1[1]);
        unsigned k = Partial<DT_U8, MET_L2, CPL>::run(qv, r1);
        k += __shfl_xor_sync(FULL, k, 2);
        k += __shfl_xor_sync(FULL, k, 1);
        const bool has = gl == 0 && c < nc;
        put_key<PACK>(w, has, has ? make_key_nonneg((float)k, w.cids[c]) : KEY_NONE, c, worst, m, lt);
        break;
      }
    }
    uint4 r[UNR][CPL];
#pragma unroll
    for (int u = 0; u < UNR; u++) {
      int c = c0 + u * GR + g;
      if constexpr (DT == DT_U8 && W == 4 && CPL == 2) {
        // 128-byte rows at 32-byte aligned addresses: lane gl takes bytes
        // [32 gl, 32 gl + 32) in one load, so each row line is read by one
        // instruction
        ldg_nc_32b(a.X + wide_mul(w.cids[min(c, nc - 1)], a.row_bytes) + 32 * gl, r[u][0], r[u][1]);
      } else if constexpr (DT == DT_U8) {
        // a slot past the last candidate rescores the last one (discarded)
        load_row<W, CPL, true>(a.X + wide_mul(w.cids[min(c, nc - 1)], a.row_bytes), gl, a.C, r[u]);
      } else if (c < nc) {
        load_row<W, CPL, true>(a.X + wide_mul(w.cids[c], a.row_bytes), gl, a.C, r[u]);
      } else {
#pragma unroll
        for (int t = 0; t < CPL; t++) r[u][t] = make_uint4(0, 0, 0, 0);
      }
    }
    if constexpr (DT == DT_F32 && UNR % 2 == 0) {
      // two rows per packed instruction (same bits as one row at a time)
#pragma unroll
      for (int u = 0; u < UNR; u += 2) {
        float2 s = partial_f32_pair<METRIC, CPL>(qv, r[u], r[u + 1]);
#pragma unroll
        for (int off = W / 2; off >= 1; off >>= 1) {
          s.x += __shfl_xor_sync(FULL, s.x, off);
          s.y += __shfl_xor_sync(FULL, s.y, off);
        }
        if (METRIC == MET_IP) {
          s.x = 1.0f - s.x;
          s.y = 1.0f - s.y;
        }
        const int c = c0 + u * GR + g, c1 = c + GR;
        const bool h0 = gl == 0 && c < nc, h1 = gl == 0 && c1 < nc;
        put_key<PACK>(w, h0, h0 ? make_key(s.x, w.cids[c]) : KEY_NONE, c, worst, m, lt);
        put_key<PACK>(w, h1, h1 ? make_key(s.y, w.cids[c1]) : KEY_NONE, c1, worst, m, lt);
      }
    } else if constexpr (DT == DT_U8 && UNR == 2) {
      // the same for two rows per lane group: one split step, then plain
      // butterfly steps; lane gl ends with row [gl & W/2]
      const unsigned p0 = Partial<DT_U8, MET_L2, CPL>::run(qv, r[0]);
      const unsigned p1 = Partial<DT_U8, MET_L2, CPL>::run(qv, r[1]);
      const bool b = (gl & (W / 2)) != 0;
      unsigned k = b ? p1 : p0;
      k += __shfl_xor_sync(FULL, b ? p0 : p1, W / 2);
#pragma unroll
      for (int off = W / 4; off >= 1; off >>= 1) k += __shfl_xor_sync(FULL, k, off);
      const int c = c0 + (int)b * GR + g;
      const bool has = (gl & (W / 2 - 1)) == 0 && c < nc;
      put_key<PACK>(w, has, has ? make_key_nonneg((float)k, w.cids[c]) : KEY_NONE, c, worst, m, lt);
    } else if constexpr (DT == DT_U8 && UNR == 4) {
      // integer partials, exact in any order: reduce the group's four rows
      // together. The first two steps halve the rows a lane carries (it keeps
      // row u = 2*[gl & W/2] + [gl & W/4]), plain butterfly steps finish it.
      unsigned pt[4];
#pragma unroll
      for (int u = 0; u < 4; u++) pt[u] = Partial<DT_U8, MET_L2, CPL>::run(qv, r[u]);
      const bool b2 = (gl & (W / 2)) != 0, b1 = (gl & (W / 4)) != 0;
      unsigned k0 = b2 ? pt[2] : pt[0], k1 = b2 ? pt[3] : pt[1];
      const unsigned s0 = b2 ? pt[0] : pt[2], s1 = b2 ? pt[1] : pt[3];
      k0 += __shfl_xor_sync(FULL, s0, W / 2);
      k1 += __shfl_xor_sync(FULL, s1, W / 2);
      unsigned k = b1 ? k1 : k0;
      k += __shfl_xor_sync(FULL, b1 ? k0 : k1, W / 4);
#pragma unroll
      for (int off = W / 8; off >= 1; off >>= 1) k += __shfl_xor_sync(FULL, k, off);
      const int c = c0 + (2 * (int)b2 + (int)b1) * GR + g;
      const bool has = (gl & (W / 4 - 1)) == 0 && c < nc;
      put_key<PACK>(w, has, has ? make_key_nonneg((float)k, w.cids[c]) : KEY_NONE, c, worst, m, lt);
    } else {
#pragma unroll
      for (int u = 0; u < UNR; u++) {
        float dv = group_dis<DT, METRIC, W, CPL>(qv, r[u]);
        int c = c0 + u * GR + g;
        const bool has = gl == 0 && c < nc;
        uint64_t key = KEY_NONE;
        if (has) key = METRIC == MET_L2 ? make_key_nonneg(dv, w.cids[c]) : make_key(dv, w.cids[c]);
        put_key<PACK>(w, has, key, c, worst, m, lt);
      }
    }
  }
  __syncwarp();
  return PACK ? m : nc;
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

// Rank of key x in the sorted beam (number of entries below it) and whether
// x is already there. Up to 1024 entries: one ballot over every s-th entry
// (s = ceil(nb / 32)) finds the stride that brackets x, a second ballot ranks
// it inside that stride. Collective; the result is the same on every lane.
__device__ __forceinline__ int beam_rank(const uint64_t* beam, int nb, uint64_t x, int lane, bool* dup) {
  int pos = 0;
  if (nb <= 1024) {
    const int s = (nb + 31) >> 5;
    const int j = lane * s;
    const uint64_t e = j < nb ? key_clean(beam[j]) : KEY_NONE;
    const int c1 = __popc(__ballot_sync(FULL, e < x));
    if (c1 > 0) {
      // beam[(c1 - 1) s] < x, and beam[c1 s] >= x when it exists
      const int base = (c1 - 1) * s + 1, lim = min(nb, c1 * s);
      const int t = base + lane;
      const uint64_t e2 = t < lim ? key_clean(beam[t]) : KEY_NONE;
      pos = base + __popc(__ballot_sync(FULL, e2 < x));
    }
  } else {
    for (int b = 0; b < nb; b += 32) {
      const int j = b + lane;
      const uint64_t e = j < nb ? key_clean(beam[j]) : KEY_NONE;
      pos += __popc(__ballot_sync(FULL, e < x));
    }
  }
  *dup = pos < nb && key_clean(beam[pos]) == x;
  return pos;
}

__device__ __forceinline__ int merge_filtered(WarpSmem& w, int& nb, int Lw, int m, int& cursor, int lane);

__device__ __forceinline__ uint64_t min_u64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t max_u64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// Bitonic sort (ascending) of the 32 keys x0 (position = lane) or, with TWO,
// the 64 keys x0, x1 (positions lane and 32 + lane). Collective.
template <bool TWO>
__device__ __forceinline__ void warp_sort_keys(uint64_t& x0, uint64_t& x1, int lane) {
  constexpr int NK = TWO ? 64 : 32;
#pragma unroll
  for (int k = 2; k <= NK; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {
        // k = 64: positions lane and 32 + lane, one ascending run
        const uint64_t lo = min_u64(x0, x1);
        x1 = max_u64(x0, x1);
        x0 = lo;
      } else {
        // the lower position of a pair keeps the minimum in an ascending
        // k-block ((position & k) == 0), the maximum in a descending one
        const bool lower = (lane & j) == 0;
        const uint64_t y0 = __shfl_xor_sync(FULL, x0, j);
        x0 = (lower == ((lane & k) == 0)) ? min_u64(x0, y0) : max_u64(x0, y0);
        if (TWO) {
          const uint64_t y1 = __shfl_xor_sync(FULL, x1, j);
          x1 = (lower == (((lane + 32) & k) == 0)) ? min_u64(x1, y1) : max_u64(x1, y1);
        }
      }
    }
  }
}

// Merge 4..64 candidate keys (the front of ckeys, all better than the beam's
// current Lw-th entry) into the beam: sort them in registers, drop repeats
// (adjacent once sorted) and keys already in the beam, then merge the sorted
// run into the beam in place. Returns the number merged. Collective.
__device__ __forceinline__ int merge_sorted64(WarpSmem& w, int& nb, int Lw, int m, int& cursor, int lane) {
  uint64_t x0 = lane < m ? w.ckeys[lane] : KEY_NONE;
  uint64_t x1 = lane + 32 < m ? w.ckeys[lane + 32] : KEY_NONE;
  if (m > 32)
    warp_sort_keys<true>(x0, x1, lane);
  else
    warp_sort_keys<false>(x0, x1, lane);
  const uint64_t up0 = __shfl_up_sync(FULL, x0, 1), up1 = __shfl_up_sync(FULL, x1, 1);
  const uint64_t last0 = __shfl_sync(FULL, x0, 31);
  bool ok0 = x0 != KEY_NONE && (lane == 0 || x0 != up0);
  bool ok1 = x1 != KEY_NONE && x1 != (lane == 0 ? last0 : up1);
  // insertion point in the old beam; a key already there is a repeat
  int lb0 = 0, lb1 = 0;
  if (ok0) {
    lb0 = lower_bound_key(w.beam, nb, x0);
    ok0 = !(lb0 < nb && key_clean(w.beam[lb0]) == x0);
  }
  if (ok1) {
    lb1 = lower_bound_key(w.beam, nb, x1);
    ok1 = !(lb1 < nb && key_clean(w.beam[lb1]) == x1);
  }
  const unsigned b0 = __ballot_sync(FULL, ok0), b1 = __ballot_sync(FULL, ok1);
  const int n0 = __popc(b0), m2 = n0 + __popc(b1);
  const unsigned lt = lanemask_lt();
  __syncwarp();
  if (ok0) {
    const int r = __popc(b0 & lt);
    w.ckeys[r] = x0;
    w.cids[r] = lb0;
  }
  if (ok1) {
    const int r = n0 + __popc(b1 & lt);
    w.ckeys[r] = x1;
    w.cids[r] = lb1;
  }
  __syncwarp();
  if (m2 == 0) return 0;
  const int p0 = w.cids[0];
  // beam entries at or after p0 move up by the number of new keys below
  // them, from the back, in place; then the new keys go to r + their point
  for (int hi = nb - 1; hi >= p0; hi -= 32) {
    const int idx = hi - lane;
    uint64_t e = 0;
    int dst = Lw;
    if (idx >= p0) {
      e = w.beam[idx];
      dst = idx + count_below(w.ckeys, m2, key_clean(e));
    }
    __syncwarp();
    if (dst < Lw) w.beam[dst] = e;
    __syncwarp();
  }
  for (int r = lane; r < m2; r += 32) {
    const int dst = r + w.cids[r];
    if (dst < Lw) w.beam[dst] = w.ckeys[r];
  }
  __syncwarp();
  nb = min(Lw, nb + m2);
  if (p0 < cursor) cursor = p0;
  return m2;
}

// Merge the staged candidate keys into the beam (keep the Lw smallest keys,
// no duplicates). Returns the number of keys merged. Collective.
__device__ __forceinline__ int merge_cands(WarpSmem& w, int& nb, int Lw, int nc, int& cursor, int lane) {
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
  return merge_filtered(w, nb, Lw, m, cursor, lane);
}

// Score the nc staged candidates and merge those a full beam could take.
// Returns the number of keys merged. Collective.
template <int DT, int METRIC, int W, int CPL, int QC>
__device__ __forceinline__ int eval_merge(const SearchArgs& a, WarpSmem& w, int nc, const uint4 (&qv)[QC],
                                          int lane, int& nb, int Lw, int& cursor) {
  if constexpr (W <= 8) {
    const uint64_t worst = nb >= Lw ? key_clean(w.beam[Lw - 1]) : KEY_NONE;
    const int m = eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane, worst);
    return merge_filtered(w, nb, Lw, m, cursor, lane);
  } else {
    eval_cands<DT, METRIC, W, CPL>(a, w, nc, qv, lane);
    return merge_cands(w, nb, Lw, nc, cursor, lane);
  }
}

// Merge the m candidate keys at the front of ckeys (all better than the
// beam's current Lw-th entry, or the beam is not full) into the beam.
__device__ __forceinline__ int merge_filtered(WarpSmem& w, int& nb, int Lw, int m, int& cursor, int lane) {
  if (m == 0) return 0;
  if (m <= 3) {
    // a few survivors (the usual case once the beam is full): insert them one
    // at a time -- rank in the beam, shift the tail by one
    for (int i = 0; i < m; i++) {
      const uint64_t x = w.ckeys[i];
      bool dup;
      const int pos = beam_rank(w.beam, nb, x, lane, &dup);
      if (dup || pos >= Lw) continue;
      const int top = min(nb, Lw - 1);  // entries [pos, top) move up by one
      for (int hi = top - 1; hi >= pos; hi -= 32) {
        const int idx = hi - lane;
        uint64_t e = 0;
        if (idx >= pos) e = w.beam[idx];
        __syncwarp();
        if (idx >= pos) w.beam[idx + 1] = e;
        __syncwarp();
      }
      if (lane == 0) w.beam[pos] = x;
      __syncwarp();
      nb = min(nb + 1, Lw);
      if (pos < cursor) cursor = pos;
    }
    return m;
  }
  if (m <= 64) return merge_sorted64(w, nb, Lw, m, cursor, lane);
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
__device__ __forceinline__ void density_from_beam(const uint64_t* beam, int k, int metric, int fn, float* rho,
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


}  // namespace pecann

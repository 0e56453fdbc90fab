// Device-side building blocks shared by the kernels of the library.
//
// Keys. A candidate point is carried as one 64-bit key
//   (order-preserving bits of its FP32 dissimilarity) << 32 | id
// so that comparing keys as unsigned integers orders points by (dis, id), the
// order Algorithm 1 pops and prunes by. Bit 31 of the key (never set in an id,
// ids < 2^31) marks a beam entry as visited; comparisons mask it out.
//
// Distances. A row is read as 16-byte chunks; a group of W lanes (W a power
// of two, 8..32) computes one distance, lane g of the group owning chunks
// g, g + W, g + 2W, ... With FP32 rows this is the library's canonical order
// (chunk c into partial c mod 32 via fmaf, ascending c, then an xor
// butterfly): for at most 32 chunks the partials beyond the row are exact
// zeros, so a W-lane butterfly gives the same bits as the 32-lane one.
// uint8 rows are summed exactly in integers (every partial < 2^24).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pecann {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t VFLAG = 1ull << 31;
constexpr uint64_t KEY_NONE = ~0ull;

enum : int { DT_F32 = 0, DT_U8 = 1, DT_BF16 = 2, DT_FP8 = 3 };
enum : int { MET_L2 = 0, MET_IP = 1 };

// Error codes written to the device error word (first one wins).
enum : int {
  ERR_NONE = 0,
  ERR_BAD_ID = 1,        // a graph entry or query id outside [0, n)
  ERR_NO_PROGRESS = 2,   // a search expanded more points than exist
  ERR_CAPACITY = 3,      // a staging buffer was too small
  ERR_TIMEOUT = 4        // a pipeline wait of the tensor-core screen ran past its limit
};

__device__ __forceinline__ void set_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  return __uint_as_float(b);
}
__device__ __forceinline__ uint64_t make_key(float dis, int32_t id) {
  return ((uint64_t)f2ord(dis) << 32) | (uint32_t)id;
}
// Same key for a dissimilarity known to be >= +0 (squared L2): the sign
// branch of f2ord is not needed.
__device__ __forceinline__ uint64_t make_key_nonneg(float dis, int32_t id) {
  return ((uint64_t)(__float_as_uint(dis) | 0x80000000u) << 32) | (uint32_t)id;
}
__device__ __forceinline__ uint64_t key_clean(uint64_t k) { return k & ~VFLAG; }
__device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)(k & 0x7fffffffu); }
__device__ __forceinline__ float key_dis(uint64_t k) { return ord2f((uint32_t)(k >> 32)); }

// Reported distance D from the ordering value.
__device__ __forceinline__ float out_dist(float dis, int metric) {
  return metric == MET_L2 ? sqrtf(dis) : dis;
}

// j ranks above i: key_j > key_i, or equal keys and j < i.
__device__ __forceinline__ bool ranks_above(const float* rk, int32_t j, int32_t i) {
  float a = __ldg(rk + j), b = __ldg(rk + i);
  return a > b || (a == b && j < i);
}

__device__ __forceinline__ uint4 ldg_nc(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ uint4 ldg_l1(const uint4* p) { return __ldg(p); }

// 32 bytes from a 32-byte aligned address in one load (a 256-bit load,
// sm_100 and later).
__device__ __forceinline__ void ldg_nc_32b(const void* p, uint4& a, uint4& b) {
  asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
               : "l"(p));
}

// Start moving a line into L2 without waiting for it (no register result).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ----------------------------------------------------------------- row chunks

// Load the CPL chunks of a row owned by group lane g (chunk g + W*t).
template <int W, int CPL, bool NC = true>
__device__ __forceinline__ void load_row(const uint8_t* row, int g, int C, uint4 (&r)[CPL]) {
  const uint4* p = reinterpret_cast<const uint4*>(row);
#pragma unroll
  for (int t = 0; t < CPL; t++) {
    int c = g + W * t;
    if (c < C)
      r[t] = NC ? ldg_nc(p + c) : ldg_l1(p + c);
    else
      r[t] = make_uint4(0, 0, 0, 0);
  }
}

// Partial sum of one lane over its chunks.
template <int DT, int METRIC, int CPL>
struct Partial;

template <int CPL>
struct Partial<DT_F32, MET_L2, CPL> {
  typedef float acc_t;
  __device__ __forceinline__ static float run(const uint4 (&q)[CPL], const uint4 (&r)[CPL]) {
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < CPL; t++) {
      float d0 = __uint_as_float(q[t].x) - __uint_as_float(r[t].x);
      float d1 = __uint_as_float(q[t].y) - __uint_as_float(r[t].y);
      float d2 = __uint_as_float(q[t].z) - __uint_as_float(r[t].z);
      float d3 = __uint_as_float(q[t].w) - __uint_as_float(r[t].w);
      acc = __fmaf_rn(d0, d0, acc);
      acc = __fmaf_rn(d1, d1, acc);
      acc = __fmaf_rn(d2, d2, acc);
      acc = __fmaf_rn(d3, d3, acc);
    }
    return acc;
  }
};

template <int CPL>
struct Partial<DT_F32, MET_IP, CPL> {
  typedef float acc_t;
  __device__ __forceinline__ static float run(const uint4 (&q)[CPL], const uint4 (&r)[CPL]) {
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < CPL; t++) {
      acc = __fmaf_rn(__uint_as_float(q[t].x), __uint_as_float(r[t].x), acc);
      acc = __fmaf_rn(__uint_as_float(q[t].y), __uint_as_float(r[t].y), acc);
      acc = __fmaf_rn(__uint_as_float(q[t].z), __uint_as_float(r[t].z), acc);
      acc = __fmaf_rn(__uint_as_float(q[t].w), __uint_as_float(r[t].w), acc);
    }
    return acc;
  }
};

template <int CPL>
struct Partial<DT_U8, MET_L2, CPL> {
  typedef unsigned acc_t;
  __device__ __forceinline__ static unsigned run(const uint4 (&q)[CPL], const uint4 (&r)[CPL]) {
    unsigned acc = 0;
#pragma unroll
    for (int t = 0; t < CPL; t++) {
      unsigned a0 = __vabsdiffu4(q[t].x, r[t].x), a1 = __vabsdiffu4(q[t].y, r[t].y);
      unsigned a2 = __vabsdiffu4(q[t].z, r[t].z), a3 = __vabsdiffu4(q[t].w, r[t].w);
      acc = __dp4a(a0, a0, acc);
      acc = __dp4a(a1, a1, acc);
      acc = __dp4a(a2, a2, acc);
      acc = __dp4a(a3, a3, acc);
    }
    return acc;
  }
};

// Reduced precision traversal rows: BF16 (8 per chunk) and FP8 e4m3 (16 per
// chunk, per-dimension scale applied to the difference). FP32 accumulation.
__device__ __forceinline__ float2 bf2_to_f2(unsigned v) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
  return __bfloat1622float2(h);
}

template <int CPL>
struct Partial<DT_BF16, MET_L2, CPL> {
  typedef float acc_t;
  __device__ __forceinline__ static float run(const uint4 (&q)[CPL], const uint4 (&r)[CPL]) {
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < CPL; t++) {
      unsigned qa[4] = {q[t].x, q[t].y, q[t].z, q[t].w};
      unsigned ra[4] = {r[t].x, r[t].y, r[t].z, r[t].w};
#pragma unroll
      for (int w = 0; w < 4; w++) {
        float2 a = bf2_to_f2(qa[w]), b = bf2_to_f2(ra[w]);
        float d0 = a.x - b.x, d1 = a.y - b.y;
        acc = __fmaf_rn(d0, d0, acc);
        acc = __fmaf_rn(d1, d1, acc);
      }
    }
    return acc;
  }
};

template <int CPL>
struct Partial<DT_BF16, MET_IP, CPL> {
  typedef float acc_t;
  __device__ __forceinline__ static float run(const uint4 (&q)[CPL], const uint4 (&r)[CPL]) {
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < CPL; t++) {
      unsigned qa[4] = {q[t].x, q[t].y, q[t].z, q[t].w};
      unsigned ra[4] = {r[t].x, r[t].y, r[t].z, r[t].w};
#pragma unroll
      for (int w = 0; w < 4; w++) {
        float2 a = bf2_to_f2(qa[w]), b = bf2_to_f2(ra[w]);
        acc = __fmaf_rn(a.x, b.x, acc);
        acc = __fmaf_rn(a.y, b.y, acc);
      }
    }
    return acc;
  }
};

// FP8 e4m3 rows, inner product: decoded x_j = s_j * code_j, and the query
// side carries a_j = q_j * s_j (FP32), so the dot product is sum a_j code_j
// with one decode and one FMA per element. q holds four FP32 chunks (16
// values) per 16-byte row chunk.
__device__ __forceinline__ float2 e4m3x2_to_f2(unsigned v) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(v & 0xffffu), __NV_E4M3);
  return __half22float2(*reinterpret_cast<const __half2*>(&h));
}

template <int CPL>
struct Partial<DT_FP8, MET_IP, CPL> {
  typedef float acc_t;
  __device__ __forceinline__ static float run(const uint4 (&q)[4 * CPL], const uint4 (&r)[CPL]) {
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < CPL; t++) {
      const unsigned ra[4] = {r[t].x, r[t].y, r[t].z, r[t].w};
#pragma unroll
      for (int w = 0; w < 4; w++) {
        const uint4 qq = q[4 * t + w];
        const float2 lo = e4m3x2_to_f2(ra[w]), hi = e4m3x2_to_f2(ra[w] >> 16);
        acc = __fmaf_rn(__uint_as_float(qq.x), lo.x, acc);
        acc = __fmaf_rn(__uint_as_float(qq.y), lo.y, acc);
        acc = __fmaf_rn(__uint_as_float(qq.z), hi.x, acc);
        acc = __fmaf_rn(__uint_as_float(qq.w), hi.y, acc);
      }
    }
    return acc;
  }
};

// Butterfly over a group of W lanes (every lane ends with the same value).
template <int W>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int off = W / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}
template <int W>
__device__ __forceinline__ unsigned group_sum(unsigned v) {
#pragma unroll
  for (int off = W / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

// Dissimilarity of the group's row to the query (collective over the warp;
// every lane of the group gets the value).
template <int DT, int METRIC, int W, int CPL, int QC>
__device__ __forceinline__ float group_dis(const uint4 (&q)[QC], const uint4 (&r)[CPL]) {
  auto part = Partial<DT, METRIC, CPL>::run(q, r);
  auto s = group_sum<W>(part);
  if (METRIC == MET_L2) return (float)s;
  return 1.0f - (float)s;
}

// ----------------------------------------------------------------- paired FP32 rows
// Blackwell's packed f32x2 instructions round each half exactly like the
// scalar instruction, so scoring two candidate rows with one packed register
// pair (low half: first row, high half: second row) keeps each row's
// canonical sequence of operations and gives the same bits, with half the
// arithmetic instructions.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long v) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(v));
  return f;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Canonical partial sums of one lane for two FP32 rows at once.
template <int METRIC, int CPL>
__device__ __forceinline__ float2 partial_f32_pair(const uint4 (&q)[CPL], const uint4 (&r0)[CPL],
                                                   const uint4 (&r1)[CPL]) {
  unsigned long long acc = pk2(0.0f, 0.0f);
#pragma unroll
  for (int t = 0; t < CPL; t++) {
    const unsigned qa[4] = {q[t].x, q[t].y, q[t].z, q[t].w};
    const unsigned a0[4] = {r0[t].x, r0[t].y, r0[t].z, r0[t].w};
    const unsigned a1[4] = {r1[t].x, r1[t].y, r1[t].z, r1[t].w};
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const float qf = __uint_as_float(qa[e]);
      const unsigned long long qq = pk2(qf, qf);
      const unsigned long long rr = pk2(__uint_as_float(a0[e]), __uint_as_float(a1[e]));
      if (METRIC == MET_L2) {
        const unsigned long long d = sub2(qq, rr);
        acc = fma2(d, d, acc);
      } else {
        acc = fma2(qq, rr, acc);
      }
    }
  }
  return upk2(acc);
}

// ----------------------------------------------------------------- warp helpers

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Number of entries of the sorted array a[0..n) that are < x (masked keys).
__device__ __forceinline__ int lower_bound_key(const uint64_t* a, int n, uint64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (key_clean(a[mid]) < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Offset id * stride for a non-negative id and a stride below 2^32 (a row is
// at most 4 KB, an out-list at most R ids): one 32 x 32 -> 64-bit multiply.
__device__ __forceinline__ uint64_t wide_mul(int32_t id, int64_t stride) {
  return (uint64_t)(uint32_t)id * (uint32_t)stride;
}

__device__ __forceinline__ uint32_t hash_slot(int32_t id, int log2h) {
  return ((uint32_t)id * 0x9E3779B1u) >> (32 - log2h);
}

}  // namespace pecann

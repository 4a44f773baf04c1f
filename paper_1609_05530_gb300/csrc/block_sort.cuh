// block_sort.cuh -- stable LSD radix sort of one subset inside one CTA, in
// shared memory.  Produces the permutation that orders the subset by
// (value, row index): exactly the order that defines the ordinal ranks of
// Eq. 12 with ties broken by index.
#pragma once

#include "common.cuh"

namespace cop {

// Order-preserving unsigned keys.  -0.0 is mapped to +0.0 first so the two
// compare equal (and fall back to the index order); NaN is reported.
__device__ __forceinline__ uint32_t float_key(float x, bool& nan) {
  uint32_t b = __float_as_uint(x);
  if (x == 0.0f) b = 0u;
  nan |= (x != x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint64_t double_key(double x, bool& nan) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  if (x == 0.0) b = 0ull;
  nan |= (x != x);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

template <typename KeyT>
struct KeyOf;
template <>
struct KeyOf<uint32_t> {
  using Val = float;
  static __device__ __forceinline__ uint32_t make(float x, bool& nan) { return float_key(x, nan); }
};
template <>
struct KeyOf<uint64_t> {
  using Val = double;
  static __device__ __forceinline__ uint64_t make(double x, bool& nan) { return double_key(x, nan); }
};

// Loads keys[i] = key(x[i]) for i < m.  Returns true (in every thread) if any
// value is NaN.
template <int BLOCK, typename KeyT>
__device__ __forceinline__ bool load_keys(const typename KeyOf<KeyT>::Val* __restrict__ x, int m,
                                          KeyT* keys) {
  bool nan = false;
  for (int i = threadIdx.x; i < m; i += BLOCK) keys[i] = KeyOf<KeyT>::make(x[i], nan);
  return __syncthreads_or(nan) != 0;
}

// Exclusive prefix sum of cnt[0 .. BLOCK*8) in place (every thread owns 8
// consecutive counters).  scratch: >= 33 uint32 of shared memory.
template <int BLOCK>
__device__ __forceinline__ void block_exclusive_scan8(uint32_t* cnt, uint32_t* scratch) {
  constexpr int NW = BLOCK / 32;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t v[8];
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v[j] = cnt[t * 8 + j];
    sum += v[j];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < NW ? scratch[lane] : 0u;
    uint32_t s = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NW) scratch[lane] = s - w;  // exclusive warp offsets
  }
  __syncthreads();
  uint32_t run = scratch[warp] + incl - sum;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    cnt[t * 8 + j] = run;
    run += v[j];
  }
  __syncthreads();
}

// Stable LSD radix sort by 8-bit digits.  On return idxA[pos] is the index of
// the element of rank pos+1.  idxA, idxB: m uint16 each (m <= 65535);
// cnt: 256 * (BLOCK/32) uint32 counters; scratch: >= 33 uint32.
// Warp w scans the contiguous position range [w*S, (w+1)*S); within a warp,
// elements are ranked 32 at a time with __match_any_sync, so equal digits
// keep their position order (stability).  Passes in which every element has
// the same digit are skipped.
template <int BLOCK, typename KeyT>
__device__ uint16_t* block_radix_sort_perm(const KeyT* keys, int m, uint16_t* idxA, uint16_t* idxB,
                                           uint32_t* cnt, uint32_t* scratch) {
  constexpr int NW = BLOCK / 32;
  static_assert(NW * 256 == BLOCK * 8, "counter layout assumes 8 counters per thread");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int S = (((m + NW - 1) / NW) + 31) & ~31;
  const int beg = min(m, warp * S), end = min(m, beg + S);
  for (int i = threadIdx.x; i < m; i += BLOCK) idxA[i] = (uint16_t)i;
  __syncthreads();
  constexpr int NBITS = 8 * (int)sizeof(KeyT);
  for (int shift = 0; shift < NBITS; shift += 8) {
    for (int i = threadIdx.x; i < NW * 256; i += BLOCK) cnt[i] = 0u;
    __syncthreads();
    // per-warp digit histogram, counters laid out digit-major: cnt[d*NW + w];
    // lanes sharing a digit are aggregated into one shared-memory add
    for (int base = beg; base < end; base += 32) {
      const int pos = base + lane;
      const bool valid = pos < end;
      const unsigned active = __ballot_sync(0xffffffffu, valid);
      if (valid) {
        const uint32_t d = (uint32_t)(keys[idxA[pos]] >> shift) & 255u;
        const unsigned peers = __match_any_sync(active, d);
        if ((peers & lanemask_lt()) == 0u) cnt[d * NW + warp] += (uint32_t)__popc(peers);
      }
      __syncwarp();
    }
    __syncthreads();
    // a pass where one digit holds all m elements is the identity: skip it
    bool all_same = false;
    for (int d = threadIdx.x; d < 256; d += BLOCK) {
      uint32_t tot = 0;
      for (int w = 0; w < NW; ++w) tot += cnt[d * NW + w];
      all_same |= (tot == (uint32_t)m);
    }
    if (__syncthreads_or(all_same)) continue;
    block_exclusive_scan8<BLOCK>(cnt, scratch);
    // stable scatter
    for (int base = beg; base < end; base += 32) {
      const int pos = base + lane;
      const bool valid = pos < end;
      const unsigned active = __ballot_sync(0xffffffffu, valid);
      if (valid) {
        const uint16_t idx = idxA[pos];
        const uint32_t d = (uint32_t)(keys[idx] >> shift) & 255u;
        const unsigned peers = __match_any_sync(active, d);
        const int r = __popc(peers & lanemask_lt());
        const uint32_t at = cnt[d * NW + warp];
        idxB[at + r] = idx;
        __syncwarp(active);
        if (r == 0) cnt[d * NW + warp] = at + (uint32_t)__popc(peers);
      }
      __syncwarp();
    }
    __syncthreads();
    uint16_t* t = idxA;
    idxA = idxB;
    idxB = t;
  }
  return idxA;  // the buffer holding the sorted permutation
}

}  // namespace cop

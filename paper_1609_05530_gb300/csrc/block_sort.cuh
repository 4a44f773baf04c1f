// block_sort.cuh -- stable LSD radix sort of one subset inside one CTA, in
// shared memory, with per-thread digit counters.  Produces the permutation that orders the subset by
// (value, row index): exactly the order that defines the ordinal ranks of
// Eq. 12 with ties broken by index.
#pragma once

#include "common.cuh"
#include "internal.h"

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

// Bits in which the m keys differ (OR of key ^ keys[0]); a 4-bit digit with
// no such bit is the same for every key, and its pass can be skipped.
template <int BLOCK, typename KeyT>
__device__ __forceinline__ KeyT block_varying_bits(const KeyT* keys, int m, uint32_t* scratch) {
  const KeyT k0 = keys[0];
  KeyT d = 0;
  for (int i = threadIdx.x; i < m; i += BLOCK) d |= keys[i] ^ k0;
  uint32_t lo = (uint32_t)d, hi = (uint32_t)((uint64_t)d >> 32);
  lo = __reduce_or_sync(0xffffffffu, lo);
  hi = __reduce_or_sync(0xffffffffu, hi);
  if (threadIdx.x == 0) {
    scratch[0] = 0u;
    scratch[1] = 0u;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    atomicOr(&scratch[0], lo);
    atomicOr(&scratch[1], hi);
  }
  __syncthreads();
  const KeyT r = (KeyT)(((uint64_t)scratch[1] << 32) | scratch[0]);
  __syncthreads();
  return r;
}

// Stable LSD radix sort by kRadixBits-bit digits.  Returns the buffer (idxA or idxB)
// whose entry pos is the index of the element of rank pos+1.  idxA, idxB: m
// uint16 each (m <= 65535); cnt: 2^kRadixBits * BLOCK uint16, 16-byte aligned;
// scratch: >= 33 uint32.
//
// Thread t owns the contiguous positions [t*I, (t+1)*I), I = ceil(m/BLOCK)
// rounded up to 2 mod 4,
// and private digit counters cnt[d*BLOCK + t].  A pass counts its digits
// (histogram walk), turns all 16*BLOCK counters into exclusive offsets in
// digit-major, thread-minor order (one block scan), then walks its positions
// again in order, placing each element at its digit's offset and bumping it.
// Equal digits keep position order, so every pass is stable.  Digits that
// are the same for every key are skipped.
template <int BLOCK, typename KeyT>
__device__ uint16_t* block_radix_sort_perm(const KeyT* keys, int m, uint16_t* idxA, uint16_t* idxB,
                                           SortCnt* cnt, uint32_t* scratch) {
  const int t = threadIdx.x;
  // I = 2 mod 4 (rounded up from ceil(m / BLOCK)): the 32 lanes' strided
  // uint16 reads of idxA[t*I + j] then fall in 32 distinct banks (I = 16
  // would put them in 4)
  int I = (m + BLOCK - 1) / BLOCK;
  I += (6 - (I & 3)) & 3;
  const int beg = min(m, t * I), end = min(m, beg + I);
  const KeyT vary = block_varying_bits<BLOCK, KeyT>(keys, m, scratch);
  for (int i = t; i < m; i += BLOCK) idxA[i] = (uint16_t)i;
  __syncthreads();
  constexpr int NBITS = 8 * (int)sizeof(KeyT);
  constexpr int D = kRadixDigits;
  constexpr int W = D / 2;  // 32-bit words of one thread's counters
  for (int shift = 0; shift < NBITS; shift += kRadixBits) {
    if ((((uint64_t)vary >> shift) & (uint64_t)(D - 1)) == 0u) continue;  // uniform: same for all threads
#pragma unroll
    for (int d = 0; d < D; ++d) cnt[d * BLOCK + t] = 0;
    for (int pos = beg; pos < end; ++pos) {
      const uint32_t d = (uint32_t)(keys[idxA[pos]] >> shift) & (uint32_t)(D - 1);
      cnt[d * BLOCK + t] += 1;
    }
    __syncthreads();
    // exclusive scan of the D*BLOCK counters in storage order; thread t takes
    // the D consecutive counters [D t, D t + D)
    {
      uint4* c4 = reinterpret_cast<uint4*>(cnt) + (W / 4) * t;
      uint32_t w[W];
#pragma unroll
      for (int q = 0; q < W / 4; ++q) {
        const uint4 x = c4[q];
        w[4 * q] = x.x;
        w[4 * q + 1] = x.y;
        w[4 * q + 2] = x.z;
        w[4 * q + 3] = x.w;
      }
      uint32_t sum = 0;
#pragma unroll
      for (int j = 0; j < W; ++j) sum += (w[j] & 0xffffu) + (w[j] >> 16);
      const int lane = t & 31, warp = t >> 5;
      constexpr int NW = BLOCK / 32;
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) scratch[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        const uint32_t x = lane < NW ? scratch[lane] : 0u;
        uint32_t s = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
          if (lane >= o) s += y;
        }
        if (lane < NW) scratch[lane] = s - x;
      }
      __syncthreads();
      uint32_t run = scratch[warp] + incl - sum;
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const uint32_t lo = w[j] & 0xffffu, hi = w[j] >> 16;
        w[j] = run | ((run + lo) << 16);
        run += lo + hi;
      }
#pragma unroll
      for (int q = 0; q < W / 4; ++q) c4[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    }
    __syncthreads();
    for (int pos = beg; pos < end; ++pos) {
      const uint16_t idx = idxA[pos];
      const uint32_t d = (uint32_t)(keys[idx] >> shift) & (uint32_t)(D - 1);
      const uint32_t at = cnt[d * BLOCK + t];
      cnt[d * BLOCK + t] = (SortCnt)(at + 1);
      idxB[at] = idx;
    }
    __syncthreads();
    uint16_t* tmp = idxA;
    idxA = idxB;
    idxB = tmp;
  }
  return idxA;  // the buffer holding the sorted permutation
}

}  // namespace cop

// block_sort.cuh -- the ordering of one subset inside one CTA, in shared
// memory: the permutation that orders the subset by (value, row index),
// exactly the order that defines the ordinal ranks of Eq. 12 with ties
// broken by index.  Two methods give the same permutation: ranking by value
// buckets (FP32 keys whose values spread evenly enough), and a stable LSD
// radix sort with per-thread digit counters (every other input).
#pragma once

#include <cfloat>

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

// Smallest and largest 32-bit key of a subset, when known (lets the ordering
// skip its own min/max scan).
struct KeyRange {
  bool valid = false;
  uint32_t lo = 0u, hi = 0u;
};

// Loads keys[i] = key(x[i]) for i < m.  Returns true (in every thread) if any
// value is NaN.  For 32-bit keys it also finds their range, in every thread,
// in the same pass (scratch: >= 32 uint32, free again after the next block
// barrier).
template <int BLOCK, typename KeyT>
__device__ __forceinline__ bool load_keys(const typename KeyOf<KeyT>::Val* __restrict__ x, int m,
                                          KeyT* keys, uint32_t* scratch = nullptr, KeyRange* range = nullptr) {
  bool nan = false;
  if constexpr (sizeof(KeyT) == 4) {
    if (range) {
      static_assert(BLOCK / 32 <= 16, "scratch layout");
      uint32_t lo = 0xffffffffu, hi = 0u;
      for (int i = threadIdx.x; i < m; i += BLOCK) {
        const uint32_t k = KeyOf<KeyT>::make(x[i], nan);
        keys[i] = k;
        lo = min(lo, k);
        hi = max(hi, k);
      }
      lo = __reduce_min_sync(0xffffffffu, lo);
      hi = __reduce_max_sync(0xffffffffu, hi);
      if ((threadIdx.x & 31) == 0) {
        scratch[threadIdx.x >> 5] = lo;
        scratch[16 + (threadIdx.x >> 5)] = hi;
      }
      const bool any_nan = __syncthreads_or(nan) != 0;
      lo = 0xffffffffu;
      hi = 0u;
#pragma unroll
      for (int w = 0; w < BLOCK / 32; ++w) {
        lo = min(lo, scratch[w]);
        hi = max(hi, scratch[16 + w]);
      }
      range->valid = true;
      range->lo = lo;
      range->hi = hi;
      return any_nan;
    }
  }
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

// ---------------------------------------------------------------------------
// Ranking by value buckets (32-bit keys of FP32 values).
//
// The value range [lo, hi] of the subset is cut into nb equal buckets, about
// kBucketTarget elements each, and element i goes to bucket
//   b(x_i) = min(nb - 1, trunc((x_i - lo) * (nb / (hi - lo))))
// with every operation rounded to nearest and nothing contracted.  Rounding
// is monotone, so b never decreases with x: equal values share a bucket and
// every element of a later bucket is larger than every element of an earlier
// one.  A histogram of b (shared-memory atomics) and its exclusive scan give
// each bucket's first rank; a scatter lists each bucket's elements (in any
// order); then every element counts the elements of its own bucket that
// precede it in (value, index) order.  Rank - 1 = bucket start + that count,
// the same ordinal rank a stable sort gives.  One pass of histogram, scan,
// scatter and count replaces the eight digit passes of the radix sort.
//
// It applies when the range is finite and positive and no bucket holds more
// than kBucketMaxRun elements (values spread unevenly enough to crowd one
// bucket, e.g. heavy tails, fall back to the radix sort, which returns the
// same permutation).  The decision is made by the whole block.
// ---------------------------------------------------------------------------
constexpr int kBucketTarget = 2;    // mean elements per bucket (more where the counters run out)
constexpr int kBucketMaxRun = 96;   // largest bucket the pairwise count takes

// The FP32 value of an order-preserving key (inverse of float_key).
__device__ __forceinline__ float key_value(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k ^ 0x80000000u) : ~k);
}

struct ValueBuckets {
  float lo, scale;
  int nb;
  __device__ __forceinline__ int of(uint32_t k) const {
    const float q = __fmul_rn(__fsub_rn(key_value(k), lo), scale);
    return min(nb - 1, __float2int_rz(q));
  }
};

// Smallest and largest key of the subset, in every thread.  scratch: >= 32
// uint32.
template <int BLOCK>
__device__ __forceinline__ void block_minmax_keys(const uint32_t* keys, int m, uint32_t* scratch, uint32_t& kmin,
                                                  uint32_t& kmax) {
  static_assert(BLOCK / 32 <= 16, "scratch layout");
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (int i = threadIdx.x; i < m; i += BLOCK) {
    const uint32_t k = keys[i];
    lo = min(lo, k);
    hi = max(hi, k);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    scratch[warp] = lo;
    scratch[16 + warp] = hi;
  }
  __syncthreads();
  lo = 0xffffffffu;
  hi = 0u;
#pragma unroll
  for (int w = 0; w < BLOCK / 32; ++w) {
    lo = min(lo, scratch[w]);
    hi = max(hi, scratch[16 + w]);
  }
  __syncthreads();
  kmin = lo;
  kmax = hi;
}

// Exclusive scan of the nb bucket counts in place (cnt[b] becomes bucket b's
// first position).  Returns, in every thread, whether no bucket holds more
// than kBucketMaxRun elements.  scratch: >= 32 uint32.
template <int BLOCK>
__device__ __forceinline__ bool bucket_starts(uint32_t* cnt, int nb, uint32_t* scratch) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int P = (nb + BLOCK - 1) / BLOCK;
  const int beg = min(nb, t * P), end = min(nb, beg + P);
  uint32_t sum = 0, mx = 0;
  for (int b = beg; b < end; ++b) {
    const uint32_t c = cnt[b];
    sum += c;
    mx = max(mx, c);
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 31) scratch[warp] = incl;
  if (lane == 0) scratch[16 + warp] = mx;
  __syncthreads();
  uint32_t base = 0, gmax = 0;
#pragma unroll
  for (int w = 0; w < BLOCK / 32; ++w) {
    if (w < warp) base += scratch[w];
    gmax = max(gmax, scratch[16 + w]);
  }
  uint32_t run = base + incl - sum;
  for (int b = beg; b < end; ++b) {
    const uint32_t c = cnt[b];
    cnt[b] = run;
    run += c;
  }
  __syncthreads();
  return gmax <= (uint32_t)kBucketMaxRun;
}

// The permutation that orders keys[0..m) by (key, index): returns the
// buffer (idxA or idxB) whose entry pos is the index of the element of rank
// pos + 1.  Same buffers and scratch as block_radix_sort_perm; cnt is used as
// BLOCK * kSortCntBytesPerThread / 4 uint32 bucket counters by the bucket
// method.
template <int BLOCK, typename KeyT>
__device__ uint16_t* block_rank_perm(const KeyT* keys, int m, uint16_t* idxA, uint16_t* idxB, SortCnt* cnt_raw,
                                     uint32_t* scratch, const KeyRange& range = KeyRange()) {
  if constexpr (sizeof(KeyT) == 4) {
    uint32_t* cnt = reinterpret_cast<uint32_t*>(cnt_raw);
    constexpr int kCap = BLOCK * (int)(kSortCntBytesPerThread / 4);
    const int nb = min(kCap, max(1, m / kBucketTarget));
    uint32_t kmin = range.lo, kmax = range.hi;
    if (!range.valid) block_minmax_keys<BLOCK>(keys, m, scratch, kmin, kmax);
    const float lo = key_value(kmin), hi = key_value(kmax);
    const float range = __fsub_rn(hi, lo);
    const float scale = __fdiv_rn((float)nb, range);
    if (nb >= 2 && range > 0.0f && range <= FLT_MAX && scale <= FLT_MAX) {
      const ValueBuckets B{lo, scale, nb};
      for (int b = threadIdx.x; b < nb; b += BLOCK) cnt[b] = 0u;
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += BLOCK) atomicAdd(&cnt[B.of(keys[i])], 1u);
      __syncthreads();
      if (bucket_starts<BLOCK>(cnt, nb, scratch)) {
        for (int i = threadIdx.x; i < m; i += BLOCK) {
          const uint32_t pos = atomicAdd(&cnt[B.of(keys[i])], 1u);
          idxA[pos] = (uint16_t)i;
        }
        __syncthreads();
        // cnt[b] is now the end of bucket b and the start of bucket b + 1.
        // Each element counts the elements of its bucket that precede it in
        // (value, index) order.
        for (int q = threadIdx.x; q < m; q += BLOCK) {
          const int i = idxA[q];
          const uint32_t k = keys[i];
          const int b = B.of(k);
          const int s = b ? (int)cnt[b - 1] : 0, e = (int)cnt[b];
          int c = 0;
          for (int j = s; j < e; ++j) {
            const int ii = idxA[j];
            const uint32_t kk = keys[ii];
            c += (kk < k || (kk == k && ii < i)) ? 1 : 0;
          }
          idxB[s + c] = (uint16_t)i;
        }
        __syncthreads();
        return idxB;
      }
    }
  }
  __syncthreads();  // every thread is done with scratch (the key range) before the sort reuses it
  return block_radix_sort_perm<BLOCK, KeyT>(keys, m, idxA, idxB, cnt_raw, scratch);
}

}  // namespace cop

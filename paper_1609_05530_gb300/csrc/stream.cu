// stream.cu -- fits of subsets too large for one CTA's shared memory.
//
// Ranks (Eq. 12 within the subset) by a sample sort spread over many CTAs:
//   1. splitters: per subset, 16 samples per bucket, one at a hashed row in
//      each of 16 * buckets equal strata (so rows increase with the sample
//      index), are sorted in one CTA; every 16th gives a splitter (value,
//      row), so a run of equal values is split by row like any other;
//   2. every element finds its bucket by binary search over its subset's
//      splitters; each chunk of 16,384 rows records its count of every bucket;
//   3. per subset, the counts are scanned over chunks (each chunk's base in
//      each bucket) and over buckets (bucket starts);
//   4. elements are scattered into bucket-contiguous order, stably: within
//      a bucket they keep their row order (chunk bases, then per-warp bases,
//      then the lane order of equal buckets inside a warp);
//   5. each bucket (a few thousand elements) is sorted in shared memory by
//      value alone with a stable radix sort -- equal values stay in row
//      order, the ordinal tie rule -- and each element's subset rank is its
//      bucket start plus its position.
// Then pi (v-rank in u-rank order) and sum r_u r_v, and one cooperative
// persistent kernel runs, for all large subsets at once: both margin
// transforms in u-rank order, every Newton pass of Eq. 13 (chunk partial
// sums, a grid barrier, one warp per subset summing its chunks in fixed
// order and taking the Newton step, a grid barrier), then the sandwich
// variance with segmented suffix scans, and Eq. 15 for each dataset whose
// last subset finishes here.  Chunks are handed out dynamically within each
// sweep; partial sums keep per-chunk slots, so the results are deterministic.
// Grid barriers spin with a bound and set an error flag instead of hanging.
#include <algorithm>

#include "block_sort.cuh"
#include "families.cuh"
#include "fit_common.cuh"
#include "internal.h"

namespace cop {

// ---------------------------------------------------------------------------
// 1. splitters
// ---------------------------------------------------------------------------
// integer hash (Wellons' lowbias32) choosing a row inside each stratum
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// row of sample j of s (s <= m): one per stratum [j m / s, (j+1) m / s)
__device__ __forceinline__ int64_t sample_row(int j, int s, int64_t m) {
  const int64_t a = (int64_t)j * m / s, b = (int64_t)(j + 1) * m / s;
  return a + (int64_t)(mix32((uint32_t)j) % (uint32_t)(b - a));
}

template <typename KeyT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) splitter_kernel(const void* __restrict__ x, const Seg* __restrict__ segs,
                                                            KeyT* __restrict__ spl_key, uint32_t* __restrict__ spl_idx,
                                                            SegState* state) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t scratch[40];
  using Val = typename KeyOf<KeyT>::Val;
  const Seg sg = segs[blockIdx.x];
  const int s = kSamplesPerBucket * sg.nb;
  KeyT* keys = reinterpret_cast<KeyT*>(smem);
  uint16_t* ib0 = reinterpret_cast<uint16_t*>(smem + (size_t)s * sizeof(KeyT));
  uint16_t* ib1 = ib0 + s;
  SortCnt* cnt = reinterpret_cast<SortCnt*>(smem + a16((size_t)s * sizeof(KeyT) + 4 * (size_t)s));
  const Val* col = reinterpret_cast<const Val*>(x) + sg.off;
  bool nan = false;
  for (int j = threadIdx.x; j < s; j += BLOCK) keys[j] = KeyOf<KeyT>::make(col[sample_row(j, s, sg.m)], nan);
  if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(&state[blockIdx.x].flags, 1);
  const uint16_t* perm = block_rank_perm<BLOCK, KeyT>(keys, s, ib0, ib1, cnt, scratch);
  for (int b = 1 + threadIdx.x; b < sg.nb; b += BLOCK) {
    const int j = perm[b * kSamplesPerBucket - 1];
    spl_key[sg.bucket_base + b - 1] = keys[j];
    spl_idx[sg.bucket_base + b - 1] = (uint32_t)sample_row(j, s, sg.m);
  }
}

// number of splitters (k_s, i_s) < (k, i), over sorted splitters, when
// every splitter before lo is below (k, i) and none from hi on is
template <typename KeyT>
__device__ __forceinline__ int bucket_of_elem(const KeyT* sk, const uint32_t* si, int lo, int hi, KeyT k,
                                              uint32_t i) {  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const bool less = sk[mid] < k || (sk[mid] == k && si[mid] < i);
    if (less)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// 2. bucket of every element; each chunk's count of every bucket.  With FP32
//    keys the splitters' value range is cut into kCountCells equal cells by
//    the same non-decreasing map as the value-bucket ranking (round-to-
//    nearest operations, truncation, clamping); cell[t] counts the splitters
//    whose cell is below t.  A key in cell t lies above every splitter of a
//    lower cell and below every splitter of a higher one, so its bucket is
//    found by a search among the splitters of its own cell (usually none or
//    one) instead of among all of them.
// ---------------------------------------------------------------------------
constexpr int kCountCells = 2048;

struct SplitterCells {
  float lo, scale;
  __device__ __forceinline__ int of(uint32_t k) const {
    const float q = __fmul_rn(__fsub_rn(key_value(k), lo), scale);
    return min(kCountCells - 1, max(0, __float2int_rz(q)));
  }
};

template <typename KeyT>
__global__ void __launch_bounds__(256) bucket_count_kernel(const void* __restrict__ x, StreamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Val = typename KeyOf<KeyT>::Val;
  const Chunk ch = a.chunks[blockIdx.x];
  const Seg sg = a.segs[ch.seg];
  const int nsp = sg.nb - 1;
  KeyT* sk = reinterpret_cast<KeyT*>(smem);
  uint32_t* si = reinterpret_cast<uint32_t*>(smem + (size_t)kMaxBuckets32 * sizeof(KeyT));
  uint32_t* hist = si + kMaxBuckets32;
  const KeyT* gk = reinterpret_cast<const KeyT*>(a.spl_key) + sg.bucket_base;
  for (int b = threadIdx.x; b < nsp; b += 256) {
    sk[b] = gk[b];
    si[b] = a.spl_idx[sg.bucket_base + b];
  }
  for (int b = threadIdx.x; b < sg.nb; b += 256) hist[b] = 0u;
  __syncthreads();
  uint16_t* cell = reinterpret_cast<uint16_t*>(hist + kMaxBuckets32);  // [kCountCells + 1]
  bool cells = false;
  SplitterCells C{0.0f, 0.0f};
  if constexpr (sizeof(KeyT) == 4) {
    if (nsp >= 8) {
      const float lo = key_value(sk[0]), hi = key_value(sk[nsp - 1]);
      const float range = __fsub_rn(hi, lo);
      const float scale = __fdiv_rn((float)kCountCells, range);
      cells = range > 0.0f && range <= FLT_MAX && scale <= FLT_MAX;
      if (cells) {
        C = SplitterCells{lo, scale};
        for (int t = threadIdx.x; t <= kCountCells; t += 256) {
          int l = 0, h = nsp;  // first splitter whose cell is t or above
          while (l < h) {
            const int mid = (l + h) >> 1;
            if (C.of(sk[mid]) < t)
              l = mid + 1;
            else
              h = mid;
          }
          cell[t] = (uint16_t)l;
        }
      }
    }
  }
  __syncthreads();
  const Val* col = reinterpret_cast<const Val*>(x) + sg.off;
  bool nan = false;
  constexpr int NB = 8;  // keys per thread whose loads are in flight, and searches interleaved
  for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
    Val xv[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) xv[b] = i0 + 256 * b < ch.len ? col[ch.start + i0 + 256 * b] : Val(0);
    int bb[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int64_t li = ch.start + i0 + 256 * b;
      bool nb_nan = false;
      const KeyT k = KeyOf<KeyT>::make(xv[b], nb_nan);
      if (i0 + 256 * b < ch.len) nan |= nb_nan;
      int lo = 0, hi = nsp;
      if constexpr (sizeof(KeyT) == 4) {
        if (cells) {
          const int t = C.of(k);
          lo = cell[t];
          hi = cell[t + 1];
        }
      }
      bb[b] = bucket_of_elem<KeyT>(sk, si, lo, hi, k, (uint32_t)li);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i = i0 + 256 * b;
      if (i >= ch.len) break;
      a.bucket_of[sg.c + ch.start + i] = (uint16_t)bb[b];
      atomicAdd(&hist[bb[b]], 1u);
    }
  }
  if (__syncthreads_or(nan) && threadIdx.x == 0) atomicOr(&a.state[ch.seg].flags, 1);
  uint32_t* row = a.mat + sg.mat + (int64_t)(blockIdx.x - sg.chunk_first) * sg.nb;
  for (int b = threadIdx.x; b < sg.nb; b += 256) row[b] = hist[b];
}

// ---------------------------------------------------------------------------
// 3. per subset: chunk bases within each bucket (scan over chunks), bucket
//    sizes and starts (scan over buckets)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) bucket_scan_kernel(StreamArgs a, int cap) {
  __shared__ uint32_t scratch[40];
  const Seg sg = a.segs[blockIdx.x];
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // for the bucket orderings that follow
    *a.counter = 0;
    *a.big_count = 0;
  }
  const int per = (sg.nb + 255) / 256;
  const int beg = min(sg.nb, (int)threadIdx.x * per), end = min(sg.nb, beg + per);
  uint32_t* M = a.mat + sg.mat;
  uint32_t sum = 0, mx = 0;
  for (int b = beg; b < end; ++b) {
    uint32_t run = 0;
#pragma unroll 8
    for (int k = 0; k < sg.chunk_count; ++k) {
      const uint32_t t = M[(int64_t)k * sg.nb + b];
      M[(int64_t)k * sg.nb + b] = run;
      run += t;
    }
    a.bucket_cnt[sg.bucket_base + b] = run;
    sum += run;
    mx = max(mx, run);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < 8 ? scratch[lane] : 0u;
    uint32_t t = w;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) scratch[lane] = t - w;
  }
  __syncthreads();
  uint32_t run = scratch[warp] + incl - sum;
  for (int b = beg; b < end; ++b) {
    a.bucket_start[sg.bucket_base + b] = run;
    run += a.bucket_cnt[sg.bucket_base + b];
  }
  (void)mx;
  (void)cap;
}

// ---------------------------------------------------------------------------
// 4. stable scatter into bucket order, staged through shared memory so that
//    the stores leave as runs.  Warp w of the chunk's block (16 warps) takes
//    the w-th sixteenth of its rows, in order.  A first walk counts its
//    buckets (shared-memory atomics on 16-bit counts).  The counts become
//    offsets in the chunk's bucket-ordered image (the chunk's rows of earlier
//    buckets, then this bucket's rows of earlier warps), and a second walk
//    writes each row's in-chunk index to its place, equal buckets in lane
//    order (the lanes of equal buckets found by one ballot per bit of the
//    bucket id; rank among lower lanes).  The image is copied out in order:
//    entry j of bucket b goes to slot0[b] + j of the subset's bucket arrays
//    (slot0 = the bucket's start + this chunk's base in it - the bucket's
//    first image entry), so consecutive threads store to consecutive slots
//    within a bucket.  Row order inside every bucket, as the ranking's tie
//    rule needs.
// ---------------------------------------------------------------------------
constexpr int kScatterThreads = 512, kScatterWarps = kScatterThreads / 32;

template <typename KeyT>
__global__ void __launch_bounds__(kScatterThreads) bucket_scatter_kernel(const void* __restrict__ x, StreamArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t wtot[kScatterWarps];
  using Val = typename KeyOf<KeyT>::Val;
  const Chunk ch = a.chunks[blockIdx.x];
  const Seg sg = a.segs[ch.seg];
  const int nb = sg.nb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* cnt = reinterpret_cast<uint16_t*>(smem);  // [warps][nb]
  uint32_t* slot0 = reinterpret_cast<uint32_t*>(smem + kScatterWarps * kMaxBuckets32 * sizeof(uint16_t));
  uint16_t* img = reinterpret_cast<uint16_t*>(slot0 + kMaxBuckets32);                         // [ch.len]
  uint16_t* bo = img + kChunk;  // the chunk's buckets, staged: the walks below read them in steps
  uint16_t* wc = cnt + warp * nb;
  const int per = (ch.len + kScatterWarps - 1) / kScatterWarps;
  const int w0 = min(ch.len, warp * per), w1 = min(ch.len, w0 + per);
  const unsigned lt = lanemask_lt();
  {
    const uint16_t* g = a.bucket_of + sg.c + ch.start;
    constexpr int NB = 16;  // loads in flight per thread
    for (int i0 = threadIdx.x; i0 < ch.len; i0 += kScatterThreads * NB) {
      uint16_t t[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) t[b] = i0 + kScatterThreads * b < ch.len ? g[i0 + kScatterThreads * b] : (uint16_t)0;
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (i0 + kScatterThreads * b < ch.len) bo[i0 + kScatterThreads * b] = t[b];
    }
  }
  for (int i = threadIdx.x; i < kScatterWarps * nb; i += kScatterThreads) cnt[i] = 0;
  __syncthreads();
  // 16-bit counts (at most a warp's 2,048 rows) incremented in their 32-bit
  // word, so no carry crosses into the neighbouring count
  for (int i = w0 + lane; i < w1; i += 32) {
    const int e = warp * nb + bo[i];
    atomicAdd(reinterpret_cast<uint32_t*>(cnt) + (e >> 1), 1u << ((e & 1) * 16));
  }
  __syncthreads();
  // bucket totals of the chunk, their exclusive scan over the buckets (each
  // thread a run of consecutive buckets), then the per-warp offsets
  const int pb = (nb + kScatterThreads - 1) / kScatterThreads;
  const int b0 = min(nb, (int)threadIdx.x * pb), b1 = min(nb, b0 + pb);
  uint32_t sum = 0;
  for (int b = b0; b < b1; ++b)
    for (int w = 0; w < kScatterWarps; ++w) sum += cnt[w * nb + b];
  uint32_t incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t run = incl - sum;
  for (int w = 0; w < warp; ++w) run += wtot[w];
  const uint32_t* base = a.mat + sg.mat + (int64_t)(blockIdx.x - sg.chunk_first) * nb;
  for (int b = b0; b < b1; ++b) {
    slot0[b] = a.bucket_start[sg.bucket_base + b] + base[b] - run;  // modulo 2^32
    for (int w = 0; w < kScatterWarps; ++w) {
      const uint32_t t = cnt[w * nb + b];
      cnt[w * nb + b] = (uint16_t)run;
      run += t;
    }
  }
  __syncthreads();
  for (int i0 = w0; i0 < w1; i0 += 32) {
    const int i = i0 + lane;
    const unsigned act = __ballot_sync(0xffffffffu, i < w1);
    if (i < w1) {
      const int b = bo[i];
      unsigned peers = act;  // lanes with the same bucket, bit by bit of the bucket id
#pragma unroll
      for (int bit = 0; (1 << bit) < kMaxBuckets32; ++bit) {
        const unsigned m = __ballot_sync(act, (b >> bit) & 1);
        peers &= ((b >> bit) & 1) ? m : ~m;
      }
      const int at = wc[b] + __popc(peers & lt);
      __syncwarp(act);
      if ((peers & lt) == 0u) wc[b] = (uint16_t)(wc[b] + __popc(peers));
      img[at] = (uint16_t)i;
    }
    __syncwarp();
  }
  __syncthreads();
  const Val* col = reinterpret_cast<const Val*>(x) + sg.off + ch.start;
  KeyT* bk = reinterpret_cast<KeyT*>(a.bkey) + sg.c;
  uint32_t* bi = a.bidx + sg.c;
  constexpr int NB = 8;  // image entries per thread whose loads are in flight together
  for (int j0 = threadIdx.x; j0 < ch.len; j0 += kScatterThreads * NB) {
    int ii[NB];
    uint32_t bb[NB];
    Val vv[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) ii[b] = j0 + kScatterThreads * b < ch.len ? img[j0 + kScatterThreads * b] : 0;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      bb[b] = bo[ii[b]];
      vv[b] = col[ii[b]];
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = j0 + kScatterThreads * b;
      if (j >= ch.len) break;
      const uint32_t at = slot0[bb[b]] + (uint32_t)j;
      bool nan = false;
      bk[at] = KeyOf<KeyT>::make(vv[b], nan);
      bi[at] = (uint32_t)(ch.start + ii[b]);
    }
  }
}

// ---------------------------------------------------------------------------
// 5. sort each bucket by value (stable: equal values keep row order); rank =
//    bucket start + position + 1
// ---------------------------------------------------------------------------
template <typename KeyT>
__host__ __device__ inline size_t rank_keys_bytes(int size) { return a16((size_t)size * sizeof(KeyT)); }

// The buckets of size in (floor, cap]: two launches cover them, small
// buckets by 256-thread CTAs (four per SM), the few larger ones by 512-thread
// CTAs with room for the cap.  order = false: rank_out[row] = rank (row
// order, 1-based ranks); order = true: rank_out[rank - 1] = row (the rows in
// sorted order, stored in runs).
template <typename KeyT, int BLOCK>
__global__ void __launch_bounds__(BLOCK, BLOCK == 256 ? 4 : 2)
    bucket_rank_kernel(StreamArgs a, uint32_t* __restrict__ rank_out, int floor, int cap, bool order) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t scratch[40];
  // Buckets are dealt round robin (their sizes vary by a few tens of per
  // cent around the mean, and each CTA takes ~100 of them), so a CTA knows
  // its next bucket: its bounds are read at the top of an iteration and its
  // keys and rows are moved towards L2 after the current bucket's ranking.
  for (int j = blockIdx.x; j < a.nbucket; j += gridDim.x) {
    const int nj = j + gridDim.x;
    uint32_t nsize = 0, nstart = 0;
    int nseg = 0;
    if (nj < a.nbucket) {
      nsize = a.bucket_cnt[nj];
      nstart = a.bucket_start[nj];
      nseg = a.bucket_seg[nj];
      if (nsize <= (uint32_t)floor) nsize = 0;  // not this launch's
    }
    const int size = (int)a.bucket_cnt[j];
    if (size <= floor || size > cap) continue;  // another launch's (above the cap: big_bucket_rank_kernel)
    const int sgi = a.bucket_seg[j];
    const Seg sg = a.segs[sgi];
    const uint32_t start = a.bucket_start[j];
    const KeyT* bk = reinterpret_cast<const KeyT*>(a.bkey) + sg.c + start;
    const uint32_t* bi = a.bidx + sg.c + start;
    KeyT* keys = reinterpret_cast<KeyT*>(smem);
    uint16_t* ib0 = reinterpret_cast<uint16_t*>(smem + rank_keys_bytes<KeyT>(size));
    uint16_t* ib1 = ib0 + size;
    SortCnt* cnt = reinterpret_cast<SortCnt*>(smem + a16(rank_keys_bytes<KeyT>(size) + 4 * (size_t)size));
    for (int i = threadIdx.x; i < size; i += BLOCK) keys[i] = bk[i];
    // an inner bucket's keys lie between its two splitters' keys, which then
    // bound the value buckets of the ranking (no min/max pass)
    KeyRange range;
    const int b = j - sg.bucket_base;
    if constexpr (sizeof(KeyT) == 4) {
      if (b > 0 && b < sg.nb - 1) {
        const KeyT* spl = reinterpret_cast<const KeyT*>(a.spl_key) + sg.bucket_base;
        range.valid = true;
        range.lo = spl[b - 1];
        range.hi = spl[b];
      }
    }
    __syncthreads();
    const int64_t nc = (nsize > 0 && nsize <= (uint32_t)cap) ? a.segs[nseg].c : -1;
    const uint16_t* perm = block_rank_perm<BLOCK, KeyT>(keys, size, ib0, ib1, cnt, scratch, range);
    if (nc >= 0) {
      const char* pk = reinterpret_cast<const char*>(reinterpret_cast<const KeyT*>(a.bkey) + nc + nstart);
      const char* pr = reinterpret_cast<const char*>(a.bidx + nc + nstart);
      const uint32_t kb = nsize * (uint32_t)sizeof(KeyT), rb = nsize * 4u;
      for (uint32_t o = threadIdx.x * 128u; o < kb; o += BLOCK * 128u)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pk + o));
      for (uint32_t o = threadIdx.x * 128u; o < rb; o += BLOCK * 128u)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pr + o));
    }
    // the keys are dead: their bytes take the bucket's rows (one coalesced
    // read), so that the permuted lookups below stay in shared memory
    uint32_t* rows = reinterpret_cast<uint32_t*>(smem);
    for (int i = threadIdx.x; i < size; i += BLOCK) rows[i] = bi[i];
    __syncthreads();
    if (order)
      for (int p = threadIdx.x; p < size; p += BLOCK) rank_out[sg.c + start + p] = rows[perm[p]];
    else
      for (int p = threadIdx.x; p < size; p += BLOCK) rank_out[sg.c + rows[perm[p]]] = start + (uint32_t)p + 1u;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 5b. buckets above the shared-memory cap (a sampling accident, ~1e-11 per
//     bucket for any input order, or an input built against the sampled
//     rows): listed, then ranked by direct counting -- the rank of element e
//     of such a bucket is its start plus the number of its elements below e
//     in (value, row) order, counted over the bucket's elements staged through
//     shared memory in tiles.  Exact; O(size^2) work spread over the grid.
//     The list goes to the chunk-by-bucket matrix, free once the scatter is
//     done.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) big_bucket_list_kernel(StreamArgs a, int cap) {
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= a.nbucket) return;
  if (a.bucket_cnt[j] > (uint32_t)cap) a.mat[atomicAdd(a.big_count, 1)] = (uint32_t)j;
}

constexpr int kBigTile = 256;   // elements ranked per CTA pass
constexpr int kBigStage = 2048; // elements of the bucket staged per round

template <typename KeyT>
__global__ void __launch_bounds__(kBigTile) big_bucket_rank_kernel(StreamArgs a, uint32_t* __restrict__ rank_out,
                                                                   bool order) {
  __shared__ KeyT sk[kBigStage];
  __shared__ uint32_t si[kBigStage];
  const int nbig = *(volatile int32_t*)a.big_count;
  long long tile_id = 0;  // tiles of all listed buckets, numbered in list order
  for (int b = 0; b < nbig; ++b) {
    const int j = (int)a.mat[b];
    const Seg sg = a.segs[a.bucket_seg[j]];
    const uint32_t start = a.bucket_start[j], size = a.bucket_cnt[j];
    const KeyT* bk = reinterpret_cast<const KeyT*>(a.bkey) + sg.c + start;
    const uint32_t* bi = a.bidx + sg.c + start;
    const long long ntiles = ((long long)size + kBigTile - 1) / kBigTile;
    for (long long t = 0; t < ntiles; ++t, ++tile_id) {
      if (tile_id % gridDim.x != blockIdx.x) continue;  // the same in every thread of the CTA
      const uint32_t e = (uint32_t)(t * kBigTile) + threadIdx.x;
      const bool have = e < size;
      const KeyT k = have ? bk[e] : KeyT(0);
      const uint32_t r = have ? bi[e] : 0u;
      uint32_t below = 0;
      for (uint32_t s0 = 0; s0 < size; s0 += kBigStage) {
        const uint32_t n = min((uint32_t)kBigStage, size - s0);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += kBigTile) {
          sk[i] = bk[s0 + i];
          si[i] = bi[s0 + i];
        }
        __syncthreads();
        if (have)
          for (uint32_t i = 0; i < n; ++i) below += (sk[i] < k || (sk[i] == k && si[i] < r)) ? 1u : 0u;
      }
      if (have) {
        if (order)
          rank_out[sg.c + start + below] = r;
        else
          rank_out[sg.c + r] = start + below + 1u;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// pi and sum r_u r_v (exact: 64-bit block sums, 128-bit total)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) pi_kernel(StreamArgs a) {
  __shared__ unsigned long long red[8];
  const Chunk ch = a.chunks[blockIdx.x];
  const Seg sg = a.segs[ch.seg];
  SegState& st = a.state[ch.seg];
  unsigned long long s = 0;
  bool bad = false;
  // rank_u holds the rows in u-order: pi[p] = rank_v[row of u-rank p+1],
  // a gather in place of a scatter
  constexpr int NB = 8;
  for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
    uint32_t row[NB], rv[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) row[b] = i0 + 256 * b < ch.len ? a.rank_u[sg.c + ch.start + i0 + 256 * b] : 0u;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const bool ok = i0 + 256 * b < ch.len && (int64_t)row[b] < sg.m;
      bad |= i0 + 256 * b < ch.len && !ok;
      rv[b] = ok ? a.rank_v[sg.c + row[b]] : 1u;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int i = i0 + 256 * b;
      if (i >= ch.len) break;
      const int64_t p = ch.start + i;
      if ((int64_t)rv[b] - 1 >= sg.m || rv[b] == 0u) bad = true;
      a.pi[sg.c + p] = rv[b];
      s += (unsigned long long)(p + 1) * (unsigned long long)rv[b];
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st.flags, 4);
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    const unsigned long long old = atomicAdd(&st.s_lo, t);
    if (old + t < old) atomicAdd(&st.s_hi, 1ull);
  }
}

// ---------------------------------------------------------------------------
// Kendall's tau and Spearman's rho of the large subsets.  The discordant
// pairs are the inversions of pi (pairs p < q with pi[p] > pi[q]), counted in
// two parts: inside each chunk of 16,384 u-ranks by a bottom-up merge sort in
// shared memory (every element of a pass placed by a binary search in its
// partner run, each element of a left run adding the partner elements below
// it), which leaves the chunk's pi values sorted; and across chunks, for
// every pair of chunks a < b of a subset, the elements of a above each
// element of b, from the two sorted chunks by a merge walk (each thread takes
// a run of b, finds its first element's place in a by binary search and
// walks on).  Integer counts throughout (64-bit atomics, exact), then the
// same FP64 divisions as the shared-memory kernel.
// ---------------------------------------------------------------------------
constexpr int kInvBlock = 512;

__global__ void __launch_bounds__(kInvBlock, 1) chunk_inversions_kernel(StreamArgs a, uint32_t* __restrict__ sorted) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red[kInvBlock / 32];
  const Chunk ch = a.chunks[blockIdx.x];
  const Seg sg = a.segs[ch.seg];
  SegState& st = a.state[ch.seg];
  if (*(volatile int32_t*)&st.flags) return;
  const int n = ch.len;
  uint32_t* A = reinterpret_cast<uint32_t*>(smem);
  uint32_t* B = A + kChunk;
  const uint32_t* src = a.pi + sg.c + ch.start;
  for (int i = threadIdx.x; i < n; i += kInvBlock) A[i] = src[i];
  __syncthreads();
  unsigned long long inv = 0;
  for (int lg = 0; (1 << lg) < n; ++lg) {
    const int len = 1 << lg;
    for (int i = threadIdx.x; i < n; i += kInvBlock) {
      const int r = i >> lg;
      const int rs = r << lg;
      const bool left = (r & 1) == 0;
      const int ps = left ? rs + len : rs - len;  // partner run start
      const int pl = left ? max(0, min(len, n - ps)) : len;
      const uint32_t x = A[i];
      int lo = 0, hi = pl;  // partner elements below x (pi's values are distinct)
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[ps + mid] < x)
          lo = mid + 1;
        else
          hi = mid;
      }
      B[(left ? rs : ps) + (i - rs) + lo] = x;
      if (left) inv += (unsigned long long)lo;
    }
    __syncthreads();
    uint32_t* t = A;
    A = B;
    B = t;
  }
  uint32_t* dst = sorted + sg.c + ch.start;
  for (int i = threadIdx.x; i < n; i += kInvBlock) dst[i] = A[i];
  for (int o = 16; o > 0; o >>= 1) inv += __shfl_down_sync(0xffffffffu, inv, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = inv;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kInvBlock / 32; ++w) t += red[w];
    atomicAdd(&st.inv, t);
  }
}

// chunk b = blockIdx.x against every earlier chunk a of its subset
__global__ void __launch_bounds__(256) cross_inversions_kernel(StreamArgs a, const uint32_t* __restrict__ sorted) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red[8];
  const int kb = blockIdx.x;
  const Chunk chb = a.chunks[kb];
  const Seg sg = a.segs[chb.seg];
  SegState& st = a.state[chb.seg];
  if (*(volatile int32_t*)&st.flags || kb == sg.chunk_first) return;
  uint32_t* A = reinterpret_cast<uint32_t*>(smem);
  const uint32_t* yb = sorted + sg.c + chb.start;
  // thread t takes the run [t R, t R + R) of chunk b's sorted values
  const int R = (chb.len + 255) / 256;
  const int y0 = min(chb.len, (int)threadIdx.x * R), y1 = min(chb.len, y0 + R);
  unsigned long long cnt = 0;
  for (int ka = sg.chunk_first; ka < kb; ++ka) {
    const Chunk cha = a.chunks[ka];
    const uint32_t* xa = sorted + sg.c + cha.start;
    const int na = cha.len;
    __syncthreads();
    for (int i = threadIdx.x; i < na; i += 256) A[i] = xa[i];
    __syncthreads();
    if (y0 < y1) {
      // elements of a above y = na - (elements of a below y); a and the run
      // are both increasing, so the place of each next y is found by walking
      const uint32_t y = yb[y0];
      int lo = 0, hi = na;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] < y)
          lo = mid + 1;
        else
          hi = mid;
      }
      cnt += (unsigned long long)(na - lo);
      for (int j = y0 + 1; j < y1; ++j) {
        const uint32_t yj = yb[j];
        while (lo < na && A[lo] < yj) ++lo;
        cnt += (unsigned long long)(na - lo);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(&st.inv, t);
  }
}

// tau = (P - 2 I) / (m (m - 1) / 2), P = m (m - 1) / 2 pairs, I inversions;
// rho = 1 - 6 D / (m (m^2 - 1)), D = sum d^2 = m (m + 1)(2m + 1) / 3 - 2 S
// (128-bit integers: both exceed 64 bits near the size limit)
__global__ void rank_corr_finish_kernel(StreamArgs a, double* __restrict__ tau, double* __restrict__ rho) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nseg) return;
  const Seg sg = a.segs[i];
  const SegState& st = a.state[i];
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  if (st.flags) {
    tau[sg.subset] = qnan;
    rho[sg.subset] = qnan;
    return;
  }
  const long long m = sg.m;
  const long long P = m * (m - 1) / 2;
  const double md = (double)m;
  tau[sg.subset] = (double)(P - 2 * (long long)st.inv) / (0.5 * md * (double)(m - 1));
  const unsigned __int128 S = ((unsigned __int128)st.s_hi << 64) | (unsigned __int128)st.s_lo;
  const unsigned __int128 M = (unsigned __int128)m;
  const unsigned __int128 D = M * (M + 1) * (2 * M + 1) / 3 - 2 * S;
  rho[sg.subset] = 1.0 - 6.0 * (double)D / (md * (md * md - 1.0));
}

// ---------------------------------------------------------------------------
// per-call reset: subset states, barrier, error flag, and outputs preset to
// "no result" (replaced when the fit completes)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) stream_init_kernel(StreamArgs a) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i == 0) {
    a.barrier[0] = 0u;
    a.barrier[1] = 0u;
    *a.error = 0;
  }
  if (blockIdx.x == 0 && a.phase_ctr)
    for (int j = threadIdx.x; j < a.nphase; j += 256) a.phase_ctr[j] = 0;
  if (i >= a.nseg) return;
  a.state[i] = SegState{};
  const int k = a.segs[i].subset;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  // (copula_ranks passes no outputs at all)
  if (a.theta) a.theta[k] = qnan;
  if (a.var) a.var[k] = qnan;
  if (a.info) a.info[k] = qnan;
  if (a.status) a.status[k] = ST_DEGENERATE;
  if (a.iters) a.iters[k] = 0;
  if (a.l_out) a.l_out[k] = qnan;
  if (a.g_out) a.g_out[k] = qnan;
  if (a.h_out) a.h_out[k] = qnan;
  // a dataset with a streaming subset completes in the fit kernel below, after
  // this; NaN stays if that kernel gives up
  if (a.comb) a.comb[a.segs[i].dataset] = qnan;
}

// ranks of the large subsets from compact order to their rows (copula_ranks);
// rank 0 everywhere marks a subset holding NaN
__global__ void __launch_bounds__(256) rank_copy_kernel(StreamArgs a, int32_t* __restrict__ out) {
  const Chunk ch = a.chunks[blockIdx.x];
  const Seg sg = a.segs[ch.seg];
  const bool bad = (a.state[ch.seg].flags & 3) != 0;
  for (int i = threadIdx.x; i < ch.len; i += 256)
    out[sg.off + ch.start + i] = bad ? 0 : (int32_t)a.rank_u[sg.c + ch.start + i];
}

// ---------------------------------------------------------------------------
// The cooperative persistent fit kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch: the last of gridDim.x +
// A.barrier_phantom arrivals releases it.  Each waiting block polls at most
// A.barrier_spins times, about 256 ns apart (2^24 by default: a few seconds),
// or until another block has given up.  Returns false (and leaves the error
// flag set) if it gave up waiting.
__device__ bool grid_barrier(const StreamArgs& A) {
  unsigned* bar = A.barrier;
  int* err = A.error;
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    s_ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1 + (unsigned)A.barrier_phantom) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (*(volatile int*)err) {
          s_ok = 0;
          break;
        }
        if (++spins > A.barrier_spins) {
          atomicExch(err, 1);
          s_ok = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
    if (A.stamps && blockIdx.x == 0 && s_ok && gen + 1 < (unsigned)A.nstamps) A.stamps[gen + 1] = global_ns();
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void state_to_newton(const SegState& s, Newton& n) {
  n.th = s.th;
  n.lo = s.lo;
  n.hi = s.hi;
  n.dlo = s.dlo;
  n.dhi = s.dhi;
  n.rtol = s.rtol;
  n.it = s.it;
  n.max_iter = s.max_iter;
  n.status = s.status;
  n.done = s.done != 0;
  n.probed_lo = (s.probed & 1) != 0;
  n.probed_hi = (s.probed & 2) != 0;
  n.lo_natural = s.lo_natural != 0;
}
__device__ __forceinline__ void newton_to_state(const Newton& n, SegState& s) {
  s.th = n.th;
  s.lo = n.lo;
  s.hi = n.hi;
  s.it = n.it;
  s.status = n.status;
  s.done = n.done ? 1 : 0;
  s.probed = (n.probed_lo ? 1 : 0) | (n.probed_hi ? 2 : 0);
}

// Per-theta constants of a subset, computed once by one lane per Newton step.
template <typename Real>
__device__ __forceinline__ void set_consts(SegState& st, int family) {
  const double th = st.th, at = fabs(th);
  st.cith = family == 2 ? 1.0 / th : 0.0;
  st.cE = st.ck0 = st.ck1 = st.ck2 = 0.0;
  if (family == 1 && at >= 1e-300) {
    const FrankConsts c = sizeof(Real) == 4 ? frank_consts_f32(at) : frank_consts_f64(at);
    st.cE = c.E;
    st.ck0 = c.k0;
    st.ck1 = c.k1;
    st.ck2 = c.k2;
  }
}

// per-point terms of point p (u-rank p+1) of subset sg at theta (Real)
template <typename Real>
struct PointCtx {
  const Real* tab;   // transform of u-rank p+1
  const Real* tabv;  // transform of v-rank pi[p]
  const uint32_t* pi;
  int64_t c, m;
  int family;
  Real th, ith, at, E, k0, k1, k2, inv;
  Real ec0, ec1;  // Frank: -at/(m+1) log2(e) as FP32 head + tail; FP64: -at/(m+1)
  bool flip;
};

// e^{-at r/(m+1)} for an integer rank r, as the shared-memory path tabulates
// it: in FP32 the base-2 exponent is the rounded head product plus its exact
// FMA remainder and the tail product, so the result is good to a few ulp for
// every theta up to the cap.
__device__ __forceinline__ float exp_rank(const PointCtx<float>& P, int64_t r) {
  const float rr = (float)r;
  const float p = rr * P.ec0;
  const float e = fmaf(rr, P.ec0, -p);
  const float t = fmaf(rr, P.ec1, e);
  return ex2_approx(p) * fmaf(t, 0.693147180559945309f, 1.0f);
}
__device__ __forceinline__ double exp_rank(const PointCtx<double>& P, int64_t r) { return ::exp(P.ec0 * (double)r); }

// How the v-side margin transforms (tabv, in u-rank order) are formed: in
// FP32 evaluated per point alongside the u-side table; in FP64, where one
// evaluation costs tens of FP64 operations, gathered from the finished
// u-side table after a grid barrier.
template <typename Real>
constexpr bool kGatherTabv = sizeof(Real) == 8;

// Where the mixed partials' margin factors (dx/du, a function of the rank
// alone) are applied: per point in FP32, where evaluating them costs less
// than another read and write of both scan arrays; per rank in FP64, in the
// sweep that totals the scan arrays, where each evaluation costs tens of
// FP64 operations.
template <typename Real>
constexpr bool kDeferMargin = sizeof(Real) == 8;

// Whether the variance keeps each point's score l_t from its first sweep
// (in the point's own tabv entry, no longer needed then) instead of
// evaluating it again in the xi sweep: always in FP64; in FP32 for the
// families whose terms read the tables anyway (Frank's read no table).
template <typename Real>
__device__ __forceinline__ bool keep_score(int family) {
  return sizeof(Real) == 8 || family != 1;
}

// The stored inputs of point p: its v-rank pi[p] and, but for Frank, both
// margin transforms.  The chunk sweeps load a batch of these per thread
// before any is used, so that a thread's loads are in flight together.
template <typename Real>
struct PointIn {
  uint32_t r;
  Real x, y;
};
template <typename Real>
__device__ __forceinline__ PointIn<Real> load_point(const PointCtx<Real>& P, int64_t p) {
  PointIn<Real> in;
  in.r = P.pi[P.c + p];
  if (P.family != 1) {
    in.x = P.tab[P.c + p];
    in.y = P.tabv[P.c + p];
  } else {
    in.x = in.y = Real(0);
  }
  return in;
}

// Points per thread per batch of a chunk sweep (32 bytes of each loaded array).
template <typename Real>
constexpr int kBatch = 32 / (int)sizeof(Real);

template <typename Real>
__device__ __forceinline__ Terms<Real> point_terms(const PointCtx<Real>& P, int64_t p, const PointIn<Real>& in,
                                                   bool mixed) {
  const uint32_t r = in.r;
  Terms<Real> t;
  if (P.family == 2) {
    const Real lx = in.x, ly = in.y;
    const GumbelPoint<Real> q = gumbel_point<Real, false>(P.th, P.ith, lx, ly);
    t.g = q.g;
    t.h = q.h;
    t.gu = t.gv = Real(0);
    if (mixed) {
      gumbel_mixed<Real>(P.th, lx, ly, q, t.gu, t.gv);
      if constexpr (!kDeferMargin<Real>) {
        const Real mp1 = (Real)(P.m + 1);
        t.gu *= gumbel_margin<Real>(lx, mp1, (Real)(p + 1));
        t.gv *= gumbel_margin<Real>(ly, mp1, (Real)r);
      }
    }
    return t;
  }
  if (P.family == 0) {
    const Real x = in.x, y = in.y;
    t = gaussian_terms<Real>(P.th, x, y);
    if constexpr (!kDeferMargin<Real>) {
      if (mixed) {
        t.gu *= gaussian_margin<Real>(x);
        t.gv *= gaussian_margin<Real>(y);
      }
    }
    return t;
  }
  // Frank
  const Real u = (Real)(p + 1) * P.inv;
  if (P.at < (Real)FrankSeries<Real>::cut) return frank_series_terms<Real>(P.th, u, (Real)r * P.inv, nullptr);
  const int64_t vr = P.flip ? P.m + 1 - r : r;
  const Real v = (Real)vr * P.inv;
  const Real a = exp_rank(P, p + 1), b = exp_rank(P, vr), bc = exp_rank(P, P.m + 1 - vr);
  const FrankPoint<Real> f = frank_point<Real>(u, v, a, b, bc, P.E);
  t = frank_terms<Real>(P.at, P.k1, P.k2, u, v, a, b, f);
  if (P.flip) {
    t.g = -t.g;
    t.gu = -t.gu;
  }
  return t;
}

template <typename Real>
__device__ __forceinline__ Terms<Real> stream_terms(const PointCtx<Real>& P, int64_t p, bool mixed) {
  return point_terms<Real>(P, p, load_point<Real>(P, p), mixed);
}

// Newton start of a Frank or Gumbel segment from its Spearman rho (exact
// 128-bit sum of rank products).
__device__ inline double seg_start(const StreamArgs& A, const Seg& sg, const SegState& st) {
  const double S = (double)st.s_hi * 18446744073709551616.0 + (double)st.s_lo;
  const float rs = spearman_rho(S, sg.m);
  if (sg.family == 1) {
    const double th0 = start_from_rho(A.start.frank_rho, kFrankStart0, kFrankStartStep, fabsf(rs));
    return rs < 0.0f ? -th0 : th0;
  }
  return start_from_rho(A.start.gumbel_rho, kGumbelStart0, kGumbelStartStep, rs);
}

template <typename Real>
__device__ PointCtx<Real> point_ctx(const StreamArgs& A, const Seg& sg, const SegState& st) {
  PointCtx<Real> P;
  P.tab = reinterpret_cast<const Real*>(A.tab);
  P.tabv = reinterpret_cast<const Real*>(A.tabv);
  P.pi = A.pi;
  P.c = sg.c;
  P.m = sg.m;
  P.family = sg.family;
  P.th = (Real)st.th;
  P.ith = (Real)st.cith;
  P.at = (Real)fabs(st.th);
  P.flip = st.th < 0.0;
  P.inv = Real(1) / (Real)(sg.m + 1);
  P.E = (Real)st.cE;
  P.k0 = (Real)st.ck0;
  P.k1 = (Real)st.ck1;
  P.k2 = (Real)st.ck2;
  const double c = -fabs(st.th) / (double)(sg.m + 1);
  if constexpr (sizeof(Real) == 4) {
    const double c2 = c * 1.4426950408889634074;
    P.ec0 = (float)c2;
    P.ec1 = (float)(c2 - (double)P.ec0);
  } else {
    P.ec0 = c;
    P.ec1 = 0.0;
  }
  return P;
}

// Frank log-density of point p (loglik mode)
template <typename Real>
__device__ __forceinline__ Real frank_l(const PointCtx<Real>& P, int64_t p) {
  const uint32_t r = P.pi[P.c + p];
  const Real u = (Real)(p + 1) * P.inv;
  if (P.at < (Real)FrankSeries<Real>::cut) {
    Real l = 0;
    frank_series_terms<Real>(P.th, u, (Real)r * P.inv, &l);
    return l;
  }
  const int64_t vr = P.flip ? P.m + 1 - r : r;
  const Real v = (Real)vr * P.inv;
  const Real a = exp_rank(P, p + 1), b = exp_rank(P, vr), bc = exp_rank(P, P.m + 1 - vr);
  const FrankPoint<Real> f = frank_point<Real>(u, v, a, b, bc, P.E);
  return P.k0 - P.at * (u + v) - Real(2) * Fn<Real>::log(f.D);
}

// block reduce of NV compensated sums; writes totals to part[chunk*stride + slot..]
template <typename Real, int NV>
__device__ void chunk_reduce(Acc<Real> (&acc)[NV], double* red, double* out) {
  double tot[NV];
  block_reduce<256, Real, NV>(acc, red, tot);
  if (threadIdx.x == 0)
    for (int v = 0; v < NV; ++v) out[v] = tot[v];
}

// one warp: sum slot `slot` of the partials of the subset's chunks, fixed order
__device__ double seg_sum(const StreamArgs& A, const Seg& sg, int slot) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int k = lane; k < sg.chunk_count; k += 32) s += A.part[(size_t)(sg.chunk_first + k) * kPartStride + slot];
  return warp_sum_f64(s);
}

// Elements of each scan array per shared-memory tile of the chunk suffix sums
// (16 KB per array).
template <typename Real>
constexpr int kScanTile = 16384 / (int)sizeof(Real);

__device__ __forceinline__ void acc_merge(Acc<float>& a, const Acc<float>& b) { pair_add(a.s, a.c, b.s, b.c); }
__device__ __forceinline__ void acc_merge(Acc<double>& a, const Acc<double>& b) { a.s += b.s; }

// In-place suffix sums of a chunk's two scan arrays in global memory plus
// the chunk's offsets: x[i] <- ox + sum_{i <= j < len} x[j], the same for y
// with oy.  The chunk goes through shared memory in tiles taken from its
// end, each read and written back coalesced; inside a tile every thread sums
// a run of consecutive elements (odd length: distinct banks), a block scan
// gives the runs' suffix offsets, and the sum of the tiles after it is
// carried in (compensated in FP32).  tile: 2 * kScanTile<Real> elements;
// carry: 2 accumulators in shared memory.
template <typename Real>
__device__ void chunk_suffix_sum2(Real* __restrict__ x, Real* __restrict__ y, int len, Real ox, Real oy,
                                  Real* tile, double* red, Acc<Real>* carry) {
  constexpr int T = kScanTile<Real>;
  constexpr int C = T / 256 + 1;
  Real* sx = tile;
  Real* sy = tile + T;
  Acc<Real> cx, cy;  // the tiles after the current one
  for (int t0 = ((len - 1) / T) * T; t0 >= 0; t0 -= T) {
    const int n = min(T, len - t0);
    for (int i = threadIdx.x; i < n; i += 256) {
      sx[i] = x[t0 + i];
      sy[i] = y[t0 + i];
    }
    __syncthreads();
    const int beg = min(n, (int)threadIdx.x * C), end = min(n, beg + C);
    Acc<Real> rx, ry;
    for (int i = beg; i < end; ++i) {
      rx.add(sx[i]);
      ry.add(sy[i]);
    }
    block_excl_suffix2<256>(rx, ry, red);
    acc_merge(rx, cx);
    acc_merge(ry, cy);
    for (int i = end - 1; i >= beg; --i) {
      rx.add(sx[i]);
      sx[i] = rx.value_real();
      ry.add(sy[i]);
      sy[i] = ry.value_real();
    }
    if (threadIdx.x == 0) {  // its run starts the tile: the suffix sum at the tile's first element
      carry[0] = rx;
      carry[1] = ry;
    }
    __syncthreads();
    cx = carry[0];
    cy = carry[1];
    for (int i = threadIdx.x; i < n; i += 256) {
      x[t0 + i] = sx[i] + ox;
      y[t0 + i] = sy[i] + oy;
    }
    __syncthreads();
  }
}

template <typename Real>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 3 : 2) stream_fit_kernel(StreamArgs A) {
  __shared__ double red[4 * 32 + 8];
  __shared__ __align__(16) Real scan_tile[2 * kScanTile<Real>];
  __shared__ Acc<Real> carry[2];
  // Chunk sweeps hand chunks out dynamically (one counter per sweep, the
  // sweeps numbered alike in every block), so that blocks whose chunks
  // belong to converged subsets take more; each chunk's partial sums still
  // go to its own slot, so the results do not depend on the assignment.
  __shared__ int s_chunk;
  int phase = 0;
  auto next_chunk = [&]() -> int {
    if (threadIdx.x == 0) s_chunk = phase < A.nphase ? atomicAdd(A.phase_ctr + phase, 1) : A.nchunk;
    __syncthreads();
    const int k = s_chunk;
    __syncthreads();
    return k;
  };
  const int nwarps_grid = gridDim.x * 8;
  const int gwarp = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  Real* tab = reinterpret_cast<Real*>(A.tab);
  if (A.stamps && blockIdx.x == 0 && threadIdx.x == 0 && A.nstamps > 0) A.stamps[0] = global_ns();

  // margin transforms of both coordinates of every point, in u-rank order
  // (x of u-rank p+1 and y of v-rank pi[p]), so that every later pass
  // streams them; and the Newton start per subset
  Real* tabv = reinterpret_cast<Real*>(A.tabv);
  for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
    const Chunk ch = A.chunks[k];
    const Seg sg = A.segs[ch.seg];
    if (sg.family == 1 || A.state[ch.seg].flags) continue;  // Frank needs no table; a flagged pi is not used
    constexpr int NB = kBatch<Real>;
    for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
      uint32_t rr[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int i = i0 + 256 * b;
        rr[b] = (!kGatherTabv<Real> && i < ch.len) ? A.pi[sg.c + ch.start + i] : 1u;
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
      const int i = i0 + 256 * b;
      if (i >= ch.len) break;
      const int64_t p = ch.start + i;
      const int64_t r = (int64_t)rr[b] - 1;
      if (sg.family == 0) {
        // lower half evaluated, upper half mirrored: Phi^{-1}(1-q) = -Phi^{-1}(q)
        if (2 * (p + 1) <= sg.m + 1) {
          const Real x = normal_score(p, sg.m, Real(0));
          tab[sg.c + p] = x;
          if (sg.m - 1 - p != p) tab[sg.c + sg.m - 1 - p] = -x;
        }
        if constexpr (!kGatherTabv<Real>) tabv[sg.c + p] = normal_score(r, sg.m, Real(0));
      } else {
        tab[sg.c + p] = gumbel_lx(p, sg.m, Real(0));
        if constexpr (!kGatherTabv<Real>) tabv[sg.c + p] = gumbel_lx(r, sg.m, Real(0));
      }
      }
    }
  }
  ++phase;
  for (int sgi = blockIdx.x * 256 + threadIdx.x; sgi < A.nseg; sgi += gridDim.x * 256) {
    const Seg sg = A.segs[sgi];
    SegState& st = A.state[sgi];
    const double th0 = seg_start(A, sg, st);
    Newton nt;
    if (sg.family == 1)
      nt.init(th0, -kFrankCap, kFrankCap, A.rtol, A.max_iter, false);
    else if (sg.family == 2)
      nt.init(th0, 1.0, kGumbelCap, A.rtol, A.max_iter, true);
    else
      nt.init(0.0, -kGaussCap, kGaussCap, A.rtol, A.max_iter, false);
    st.pre_it = 0;
    newton_to_state(nt, st);
    st.dlo = nt.dlo;
    st.dhi = nt.dhi;
    st.rtol = nt.rtol;
    st.max_iter = nt.max_iter;
    st.lo_natural = nt.lo_natural ? 1 : 0;
    if (st.flags) {  // NaN in the data: no fit
      st.done = 1;
      st.status = ST_DEGENERATE;
    }
    if (A.mode == MODE_LOGLIK) st.th = A.theta_in[sg.subset];
    if (sg.family == 0 && A.mode == MODE_FIT) st.done = 1;  // solved from its cubic below
    set_consts<Real>(st, sg.family);
  }
  if (!grid_barrier(A)) return;
  if constexpr (kGatherTabv<Real>) {
    // FP64: the v-side transforms gathered from the finished u-order table
    for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
      const Chunk ch = A.chunks[k];
      const Seg sg = A.segs[ch.seg];
      if (sg.family == 1 || A.state[ch.seg].flags) continue;
      constexpr int NB = kBatch<Real>;
      const uint32_t* pc = A.pi + sg.c + ch.start;
      for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
        uint32_t rr[NB];
        Real y[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) rr[b] = i0 + 256 * b < ch.len ? pc[i0 + 256 * b] : 1u;
#pragma unroll
        for (int b = 0; b < NB; ++b) y[b] = i0 + 256 * b < ch.len ? tab[sg.c + rr[b] - 1] : Real(0);
#pragma unroll
        for (int b = 0; b < NB; ++b)
          if (i0 + 256 * b < ch.len) tabv[sg.c + ch.start + i0 + 256 * b] = y[b];
      }
    }
    ++phase;
    if (!grid_barrier(A)) return;
  }

  // Gaussian: A = sum x^2 + y^2, B = sum x y, then the cubic
  for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
    const Chunk ch = A.chunks[k];
    const Seg sg = A.segs[ch.seg];
    if (sg.family != 0 || A.state[ch.seg].flags) continue;
    Acc<Real> acc[2];
    constexpr int NB = kBatch<Real>;
    const Real* tx = tab + sg.c + ch.start;
    const Real* ty = tabv + sg.c + ch.start;
    for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
      Real x[NB], y[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const bool in = i0 + 256 * b < ch.len;
        x[b] = in ? tx[i0 + 256 * b] : Real(0);
        y[b] = in ? ty[i0 + 256 * b] : Real(0);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (i0 + 256 * b < ch.len) {
          acc[0].add(x[b] * x[b] + y[b] * y[b]);
          acc[1].add(x[b] * y[b]);
        }
    }
    chunk_reduce<Real, 2>(acc, red, A.part + (size_t)k * kPartStride + 6);
  }
  ++phase;
  if (!grid_barrier(A)) return;
  for (int sgi = gwarp; sgi < A.nseg; sgi += nwarps_grid) {
    const Seg sg = A.segs[sgi];
    if (sg.family != 0) continue;
    const double As = seg_sum(A, sg, 6), Bs = seg_sum(A, sg, 7);
    if (lane == 0) {
      SegState& st = A.state[sgi];
      if (A.mode == MODE_LOGLIK) {
        const double r = st.th, om = 1.0 - r * r, md = (double)sg.m;
        if (A.l_out) A.l_out[sg.subset] = gauss_l(md, As, Bs, r);
        if (A.g_out) A.g_out[sg.subset] = md * r / om - (r * As - Bs * (1.0 + r * r)) / (om * om);
        if (A.h_out)
          A.h_out[sg.subset] = md * (1.0 + r * r) / (om * om) -
                               (As * (1.0 + 3.0 * r * r) - 2.0 * Bs * r * (3.0 + r * r)) / (om * om * om);
        st.done = 1;
      } else if (st.flags == 0) {
        int status;
        st.th = gaussian_mpl((double)sg.m, As, Bs, status);
        st.status = status;
        st.it = 0;
        set_consts<Real>(st, sg.family);
      }
    }
  }

  // FP64 path: an FP32 search first, whose root starts the FP64 passes
  if constexpr (sizeof(Real) == 8) {
    if (A.mode == MODE_FIT) {
      for (int sgi = blockIdx.x * 256 + threadIdx.x; sgi < A.nseg; sgi += gridDim.x * 256) {
        const Seg sg = A.segs[sgi];
        SegState& st = A.state[sgi];
        if (sg.family == 0 || st.done) continue;
        st.rtol = kPresolveRtol;
        set_consts<float>(st, sg.family);
      }
      if (!grid_barrier(A)) return;
      for (int it = 0; it <= A.max_iter; ++it) {
        for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
          const Chunk ch = A.chunks[k];
          const Seg sg = A.segs[ch.seg];
          const SegState& st = A.state[ch.seg];
          if (sg.family == 0 || st.done) continue;
          Acc<float> acc[3];
          constexpr int NB = kBatch<Real>;
          if (sg.family == 2) {
            // the FP64 tables, rounded to FP32 as they are read
            const float th = (float)st.th, ith = (float)st.cith;
            const Real* tx = tab + sg.c + ch.start;
            const Real* ty = tabv + sg.c + ch.start;
            for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
              float x[NB], y[NB];
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                const bool in = i0 + 256 * b < ch.len;
                x[b] = in ? (float)tx[i0 + 256 * b] : 0.5f;
                y[b] = in ? (float)ty[i0 + 256 * b] : 0.5f;
              }
#pragma unroll
              for (int b = 0; b < NB; ++b)
                if (i0 + 256 * b < ch.len) {
                  const GumbelPoint<float> q = gumbel_point<float, false>(th, ith, x[b], y[b]);
                  acc[1].add(q.g);
                  acc[2].add(q.h);
                }
            }
          } else {
            const PointCtx<float> P = point_ctx<float>(A, sg, st);  // Frank reads no table
            const uint32_t* pc = A.pi + sg.c + ch.start;
            for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
              PointIn<float> in[NB];
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                in[b].r = i0 + 256 * b < ch.len ? pc[i0 + 256 * b] : 1u;
                in[b].x = in[b].y = 0.0f;
              }
#pragma unroll
              for (int b = 0; b < NB; ++b)
                if (i0 + 256 * b < ch.len) {
                  const Terms<float> t = point_terms<float>(P, ch.start + i0 + 256 * b, in[b], false);
                  acc[1].add(t.g);
                  acc[2].add(t.h);
                }
            }
          }
          chunk_reduce<float, 3>(acc, red, A.part + (size_t)k * kPartStride);
        }
        ++phase;
        if (!grid_barrier(A)) return;
        for (int sgi = gwarp; sgi < A.nseg; sgi += nwarps_grid) {
          const Seg sg = A.segs[sgi];
          SegState& st = A.state[sgi];
          if (sg.family == 0 || st.done) continue;
          const double g = seg_sum(A, sg, 1), h = seg_sum(A, sg, 2);
          if (lane == 0) {
            Newton nt;
            state_to_newton(st, nt);
            nt.step(g, h);
            newton_to_state(nt, st);
            set_consts<float>(st, sg.family);
          }
        }
        if (!grid_barrier(A)) return;
        int active = 0;
        for (int sgi = threadIdx.x; sgi < A.nseg; sgi += 256) active |= A.state[sgi].done == 0;
        if (!__syncthreads_or(active)) break;
      }
      // every block has read the done flags of its last loop test before
      // they are set again below
      if (!grid_barrier(A)) return;
      // the FP64 search from the FP32 root, or from the rank-correlation
      // start again if the FP32 search did not end interior
      for (int sgi = blockIdx.x * 256 + threadIdx.x; sgi < A.nseg; sgi += gridDim.x * 256) {
        const Seg sg = A.segs[sgi];
        SegState& st = A.state[sgi];
        if (sg.family == 0 || st.flags) continue;
        const bool from_root = st.status == ST_OK;
        st.pre_it = st.it;
        Newton nt;
        nt.init(from_root ? st.th : seg_start(A, sg, st), st.dlo, st.dhi, A.rtol, A.max_iter, st.lo_natural != 0,
                !from_root);
        newton_to_state(nt, st);
        st.rtol = A.rtol;
        set_consts<Real>(st, sg.family);
      }
      if (!grid_barrier(A)) return;
    }
  }

  // Newton passes of Eq. 13 for Frank and Gumbel
  for (int it = 0; it <= A.max_iter; ++it) {
    for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
      const Chunk ch = A.chunks[k];
      const Seg sg = A.segs[ch.seg];
      double* out = A.part + (size_t)k * kPartStride;
      const SegState& st = A.state[ch.seg];
      if (sg.family == 0 || st.done) continue;
      const PointCtx<Real> P = point_ctx<Real>(A, sg, st);
      Acc<Real> acc[3];
      const Real* tx = tab + sg.c + ch.start;
      const Real* ty = tabv + sg.c + ch.start;
      constexpr int NB = kBatch<Real>;
      if (A.mode == MODE_FIT && sg.family == 2) {
        for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
          Real x[NB], y[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            const bool in = i0 + 256 * b < ch.len;
            x[b] = in ? tx[i0 + 256 * b] : Real(0.5);
            y[b] = in ? ty[i0 + 256 * b] : Real(0.5);
          }
#pragma unroll
          for (int b = 0; b < NB; ++b)
            if (i0 + 256 * b < ch.len) {
              const GumbelPoint<Real> q = gumbel_point<Real, false>(P.th, P.ith, x[b], y[b]);
              acc[1].add(q.g);
              acc[2].add(q.h);
            }
        }
      } else if (A.mode == MODE_FIT) {
        for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
          PointIn<Real> in[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b)
            if (i0 + 256 * b < ch.len) in[b] = load_point<Real>(P, ch.start + i0 + 256 * b);
#pragma unroll
          for (int b = 0; b < NB; ++b)
            if (i0 + 256 * b < ch.len) {
              const Terms<Real> t = point_terms<Real>(P, ch.start + i0 + 256 * b, in[b], false);
              acc[1].add(t.g);
              acc[2].add(t.h);
            }
        }
      } else if (sg.family == 2) {
        for (int i = threadIdx.x; i < ch.len; i += 256) {
          const GumbelPoint<Real> q = gumbel_point<Real, true>(P.th, P.ith, tx[i], ty[i]);
          acc[0].add(q.l);
          acc[1].add(q.g);
          acc[2].add(q.h);
        }
      } else {
        for (int i = threadIdx.x; i < ch.len; i += 256) {
          const int64_t p = ch.start + i;
          const Terms<Real> t = stream_terms<Real>(P, p, false);
          acc[0].add(frank_l<Real>(P, p));
          acc[1].add(t.g);
          acc[2].add(t.h);
        }
      }
      chunk_reduce<Real, 3>(acc, red, out);
    }
    ++phase;
    if (!grid_barrier(A)) return;
    for (int sgi = gwarp; sgi < A.nseg; sgi += nwarps_grid) {
      const Seg sg = A.segs[sgi];
      SegState& st = A.state[sgi];
      if (sg.family == 0 || st.done) continue;
      const double l = seg_sum(A, sg, 0), g = seg_sum(A, sg, 1), h = seg_sum(A, sg, 2);
      if (lane == 0) {
        if (A.mode == MODE_LOGLIK) {
          // Frank's closed form is Eq. 10's density; its subset constants are
          // in the per-point terms, so the sums are complete
          if (A.l_out) A.l_out[sg.subset] = l;
          if (A.g_out) A.g_out[sg.subset] = g;
          if (A.h_out) A.h_out[sg.subset] = h;
          st.done = 1;
        } else {
          Newton nt;
          state_to_newton(st, nt);
          nt.step(g, h);
          newton_to_state(nt, st);
          set_consts<Real>(st, sg.family);
        }
      }
    }
    if (!grid_barrier(A)) return;
    int active = 0;
    for (int sgi = threadIdx.x; sgi < A.nseg; sgi += 256) active |= A.state[sgi].done == 0;
    if (!__syncthreads_or(active)) break;
  }
  if (A.mode == MODE_LOGLIK) return;

  // sandwich variance: the scan arrays, their segmented suffix sums W1
  // (u-order) and W2 (v-order), then xi = l_t + (W1 + W2) / m and its second
  // central moment.  The mean of xi is known before xi itself: summed over
  // t, W1 gives sum_s l_tu(s) (s + 1) over u-order positions s, and W2 the
  // same over v-order positions, so the xi sweep sums (xi - mean)^2 at once.
  // Chunk partial slots: 6 sum h, 7 sum l_t (scan-array sweep); 0-3 the scan
  // arrays' totals and position-weighted totals; 4, 5 the chunk offsets;
  // 0 again the squared deviations.
  Real* wu = reinterpret_cast<Real*>(A.wu);
  Real* wv = reinterpret_cast<Real*>(A.wv);
  for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
    const Chunk ch = A.chunks[k];
    const Seg sg = A.segs[ch.seg];
    if (A.state[ch.seg].flags) continue;
    const PointCtx<Real> P = point_ctx<Real>(A, sg, A.state[ch.seg]);
    const bool keep = keep_score<Real>(sg.family);
    Acc<Real> acc[2];
    constexpr int NB = kBatch<Real>;
    for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
      PointIn<Real> in[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (i0 + 256 * b < ch.len) in[b] = load_point<Real>(P, ch.start + i0 + 256 * b);
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (i0 + 256 * b < ch.len) {
          const int64_t p = ch.start + i0 + 256 * b;
          const Terms<Real> t = point_terms<Real>(P, p, in[b], true);
          wu[sg.c + p] = t.gu;
          wv[sg.c + in[b].r - 1] = t.gv;
          if (keep) tabv[sg.c + p] = t.g;  // this point's own entry, read above
          acc[0].add(t.h);
          acc[1].add(t.g);
        }
    }
    chunk_reduce<Real, 2>(acc, red, A.part + (size_t)k * kPartStride + 6);
  }
  ++phase;
  if (!grid_barrier(A)) return;
  // chunk totals of both scan arrays, plain and weighted by position + 1; on
  // the FP64 path, for the Gaussian and Gumbel families, entry q of each
  // first takes the margin factor of rank q+1
  for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
    const Chunk ch = A.chunks[k];
    const Seg sg = A.segs[ch.seg];
    const bool margin = kDeferMargin<Real> && sg.family != 1 && A.state[ch.seg].flags == 0;
    const Real mp1 = (Real)(sg.m + 1);
    Acc<Real> acc[4];
    constexpr int NB = kBatch<Real>;
    for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
      Real wa[NB], wb[NB], wx[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const bool in = i0 + 256 * b < ch.len;
        const int64_t q = sg.c + ch.start + i0 + 256 * b;
        wa[b] = in ? wu[q] : Real(0);
        wb[b] = in ? wv[q] : Real(0);
        wx[b] = (in && margin) ? tab[q] : Real(0);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int i = i0 + 256 * b;
        if (i >= ch.len) break;
        const int64_t q = sg.c + ch.start + i;
        Real x = wa[b], y = wb[b];
        if (margin) {
          const Real f = sg.family == 0 ? gaussian_margin<Real>(wx[b])
                                        : gumbel_margin<Real>(wx[b], mp1, (Real)(ch.start + i + 1));
          x *= f;
          y *= f;
          wu[q] = x;
          wv[q] = y;
        }
        const Real w = (Real)(ch.start + i + 1);
        acc[0].add(x);
        acc[1].add(y);
        acc[2].add(x * w);
        acc[3].add(y * w);
      }
    }
    chunk_reduce<Real, 4>(acc, red, A.part + (size_t)k * kPartStride + 0);
  }
  ++phase;
  if (!grid_barrier(A)) return;
  // per subset: the mean of xi, and the sum of the chunks after each chunk
  // (suffix offsets), serially in chunk order by one lane
  for (int sgi = gwarp; sgi < A.nseg; sgi += nwarps_grid) {
    const Seg sg = A.segs[sgi];
    const double sg_l = seg_sum(A, sg, 7), s1 = seg_sum(A, sg, 2), s2 = seg_sum(A, sg, 3);
    if (lane != 0) continue;
    const double md = (double)sg.m;
    A.state[sgi].mean = (sg_l + (s1 + s2) / md) / md;
    double su = 0.0, sv = 0.0;
    for (int k = sg.chunk_count - 1; k >= 0; --k) {
      double* q = A.part + (size_t)(sg.chunk_first + k) * kPartStride;
      const double tu = q[0], tv = q[1];
      q[4] = su;
      q[5] = sv;
      su += tu;
      sv += tv;
    }
  }
  if (!grid_barrier(A)) return;
  // in-chunk suffix sums plus the chunk's offset
  for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
    const Chunk ch = A.chunks[k];
    const Seg sg = A.segs[ch.seg];
    const double* q = A.part + (size_t)k * kPartStride;
    chunk_suffix_sum2<Real>(wu + sg.c + ch.start, wv + sg.c + ch.start, ch.len, (Real)q[4], (Real)q[5], scan_tile,
                            red, carry);
  }
  ++phase;
  if (!grid_barrier(A)) return;
  // xi = l_t + (W1 + W2) / m and the sum of (xi - mean)^2 per chunk
  for (int k = next_chunk(); k < A.nchunk; k = next_chunk()) {
    const Chunk ch = A.chunks[k];
    const Seg sg = A.segs[ch.seg];
    if (A.state[ch.seg].flags) continue;
    const PointCtx<Real> P = point_ctx<Real>(A, sg, A.state[ch.seg]);
    const Real im = Real(1) / (Real)sg.m;
    const Real mean = (Real)A.state[ch.seg].mean;
    const bool keep = keep_score<Real>(sg.family);
    Acc<Real> acc[1];
    constexpr int NB = kBatch<Real>;
    for (int i0 = threadIdx.x; i0 < ch.len; i0 += 256 * NB) {
      uint32_t rr[NB];
      Real gg[NB], w1[NB], w2[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const bool in = i0 + 256 * b < ch.len;
        const int64_t q = sg.c + ch.start + i0 + 256 * b;
        rr[b] = in ? A.pi[q] : 1u;
        w1[b] = in ? wu[q] : Real(0);
        gg[b] = (in && keep) ? tabv[q] : Real(0);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) w2[b] = i0 + 256 * b < ch.len ? wv[sg.c + rr[b] - 1] : Real(0);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int i = i0 + 256 * b;
        if (i >= ch.len) break;
        PointIn<Real> in;
        in.r = rr[b];
        in.x = in.y = Real(0);  // only Frank recomputes its score here, and Frank reads no table
        const Real g = keep ? gg[b] : point_terms<Real>(P, ch.start + i, in, false).g;
        const Real d = g + (w1[b] + w2[b]) * im - mean;
        acc[0].add(d * d);
      }
    }
    chunk_reduce<Real, 1>(acc, red, A.part + (size_t)k * kPartStride + 0);
  }
  ++phase;
  if (!grid_barrier(A)) return;
  for (int sgi = gwarp; sgi < A.nseg; sgi += nwarps_grid) {
    const Seg sg = A.segs[sgi];
    const double hs = seg_sum(A, sg, 6), ds = seg_sum(A, sg, 0);
    if (lane == 0) {
      const SegState& st = A.state[sgi];
      const double md = (double)sg.m, qnan = __longlong_as_double(0x7ff8000000000000ll);
      const bool bad = st.flags != 0;
      const double beta = -hs / md;
      A.theta[sg.subset] = bad ? qnan : st.th;
      A.var[sg.subset] = bad ? qnan : ds / md / (beta * beta) / md;
      A.status[sg.subset] = bad ? ST_DEGENERATE : st.status;
      A.info[sg.subset] = bad ? qnan : -hs;
      A.iters[sg.subset] = st.pre_it + st.it;
    }
    if (A.comb) {
      const int last = __shfl_sync(0xffffffffu, lane == 0 ? (int)dataset_finished(A.ds_done, A.dss, sg.dataset) : 0, 0);
      if (last) combine_dataset(A.theta, A.var, A.info, A.status, A.dss, A.weight, sg.dataset, A.comb);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
inline size_t splitter_smem(int ks) {
  return a16((size_t)kSamplesPerBucket * kMaxBuckets32 * (ks + 4)) + 512 * kSortCntBytesPerThread;
}
inline size_t count_smem(int ks) {
  return (size_t)kMaxBuckets32 * (ks + 4 + 4) + (size_t)(kCountCells + 1) * sizeof(uint16_t);
}
inline size_t scatter_smem() {
  return (size_t)kScatterWarps * kMaxBuckets32 * sizeof(uint16_t) + (size_t)kMaxBuckets32 * 4 +
         2 * (size_t)kChunk * sizeof(uint16_t);
}
constexpr int kRankBlock = 512;
constexpr int kRankBlockSmall = 256;
// largest bucket of the 256-thread launch (four CTAs per SM)
constexpr int kSmallCap32 = 5600, kSmallCap64 = 3600;
inline size_t rank_smem(int ks, int cap, int block) {
  return a16(a16((size_t)cap * ks) + 4 * (size_t)cap) + (size_t)block * kSortCntBytesPerThread;
}
inline size_t rank_smem(int ks) { return rank_smem(ks, ks == 4 ? kBucketCap32 : kBucketCap64, kRankBlock); }
inline size_t rank_smem_small(int ks) { return rank_smem(ks, ks == 4 ? kSmallCap32 : kSmallCap64, kRankBlockSmall); }
struct Setup {
  std::atomic<bool> done{false};
  int sms = 0;
  int rank_grid32 = 0, rank_grid64 = 0;
  int rank_small_grid32 = 0, rank_small_grid64 = 0;
  int fit_per_sm32 = 0, fit_per_sm64 = 0;
};
Setup g_setup[64];

template <typename K>
cudaError_t set_smem(K k, size_t smem) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
}  // namespace

cudaError_t stream_setup(int sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  Setup& S = g_setup[dev];
  if (S.done.load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(smem_attr_mutex());  // one thread sets the attributes up
  if (S.done.load(std::memory_order_relaxed)) return cudaSuccess;
  if ((e = set_smem(splitter_kernel<uint32_t, 512>, splitter_smem(4))) != cudaSuccess) return e;
  if ((e = set_smem(splitter_kernel<uint64_t, 512>, splitter_smem(8))) != cudaSuccess) return e;
  if ((e = set_smem(bucket_count_kernel<uint32_t>, count_smem(4))) != cudaSuccess) return e;
  if ((e = set_smem(bucket_count_kernel<uint64_t>, count_smem(8))) != cudaSuccess) return e;
  if ((e = set_smem(bucket_scatter_kernel<uint32_t>, scatter_smem())) != cudaSuccess) return e;
  if ((e = set_smem(bucket_scatter_kernel<uint64_t>, scatter_smem())) != cudaSuccess) return e;
  if ((e = set_smem(bucket_rank_kernel<uint32_t, kRankBlock>, rank_smem(4))) != cudaSuccess) return e;
  if ((e = set_smem(bucket_rank_kernel<uint64_t, kRankBlock>, rank_smem(8))) != cudaSuccess) return e;
  if ((e = set_smem(bucket_rank_kernel<uint32_t, kRankBlockSmall>, rank_smem_small(4))) != cudaSuccess) return e;
  if ((e = set_smem(bucket_rank_kernel<uint64_t, kRankBlockSmall>, rank_smem_small(8))) != cudaSuccess) return e;
  if ((e = set_smem(chunk_inversions_kernel, 2 * kChunk * sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = set_smem(cross_inversions_kernel, kChunk * sizeof(uint32_t))) != cudaSuccess) return e;
  int r32 = 0, r64 = 0, f32 = 0, f64 = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r32, bucket_rank_kernel<uint32_t, kRankBlock>, kRankBlock,
                                                         rank_smem(4))) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r64, bucket_rank_kernel<uint64_t, kRankBlock>, kRankBlock,
                                                         rank_smem(8))) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f32, stream_fit_kernel<float>, 256, 0)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f64, stream_fit_kernel<double>, 256, 0)) != cudaSuccess)
    return e;
  if (f32 < 1 || f64 < 1) return cudaErrorInvalidConfiguration;
  S.sms = sms;
  int q32 = 0, q64 = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q32, bucket_rank_kernel<uint32_t, kRankBlockSmall>,
                                                         kRankBlockSmall, rank_smem_small(4))) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q64, bucket_rank_kernel<uint64_t, kRankBlockSmall>,
                                                         kRankBlockSmall, rank_smem_small(8))) != cudaSuccess)
    return e;
  S.rank_grid32 = std::max(1, r32) * sms;
  S.rank_grid64 = std::max(1, r64) * sms;
  S.rank_small_grid32 = std::max(1, q32) * sms;
  S.rank_small_grid64 = std::max(1, q64) * sms;
  S.fit_per_sm32 = std::min(f32, 4);
  S.fit_per_sm64 = std::min(f64, 4);
  S.done.store(true, std::memory_order_release);
  return cudaSuccess;
}

static const Setup* current_setup() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || !g_setup[dev].done.load(std::memory_order_acquire)) return nullptr;
  return &g_setup[dev];
}

// the five launches ranking one column of every large subset into rank_out
template <typename KeyT>
static cudaError_t rank_column(const Setup& S, const StreamArgs& a, const void* x, uint32_t* rank_out, cudaStream_t s,
                               bool order = false) {
  constexpr int ks = (int)sizeof(KeyT);
  constexpr int cap = ks == 4 ? kBucketCap32 : kBucketCap64;
  splitter_kernel<KeyT, 512><<<a.nseg, 512, splitter_smem(ks), s>>>(x, a.segs, reinterpret_cast<KeyT*>(a.spl_key),
                                                                    a.spl_idx, a.state);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bucket_count_kernel<KeyT><<<a.nchunk, 256, count_smem(ks), s>>>(x, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bucket_scan_kernel<<<a.nseg, 256, 0, s>>>(a, cap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bucket_scatter_kernel<KeyT><<<a.nchunk, kScatterThreads, scatter_smem(), s>>>(x, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  constexpr int small_cap = ks == 4 ? kSmallCap32 : kSmallCap64;
  const int grid_small = std::max(1, std::min(a.nbucket, ks == 4 ? S.rank_small_grid32 : S.rank_small_grid64));
  bucket_rank_kernel<KeyT, kRankBlockSmall><<<grid_small, kRankBlockSmall, rank_smem_small(ks), s>>>(
      a, rank_out, 0, small_cap, order);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int grid = std::max(1, std::min(a.nbucket, ks == 4 ? S.rank_grid32 : S.rank_grid64));
  bucket_rank_kernel<KeyT, kRankBlock><<<grid, kRankBlock, rank_smem(ks), s>>>(a, rank_out, small_cap, cap, order);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  big_bucket_list_kernel<<<(a.nbucket + 255) / 256, 256, 0, s>>>(a, cap);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  big_bucket_rank_kernel<KeyT><<<2 * S.sms, kBigTile, 0, s>>>(a, rank_out, order);
  return cudaGetLastError();
}

static cudaError_t init_launch(const StreamArgs& a, cudaStream_t s) {
  stream_init_kernel<<<(a.nseg + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_stream_ranks(int key_bytes, const StreamArgs& a, const void* x, int32_t* ranks_out,
                                cudaStream_t s) {
  const Setup* S = current_setup();
  if (!S) return cudaErrorNotReady;
  cudaError_t e = init_launch(a, s);
  if (e != cudaSuccess) return e;
  e = key_bytes == 4 ? rank_column<uint32_t>(*S, a, x, a.rank_u, s) : rank_column<uint64_t>(*S, a, x, a.rank_u, s);
  if (e != cudaSuccess) return e;
  rank_copy_kernel<<<a.nchunk, 256, 0, s>>>(a, ranks_out);
  return cudaGetLastError();
}

cudaError_t launch_stream_rank_corr(int key_bytes, const StreamArgs& a, double* tau, double* rho, cudaStream_t s) {
  const Setup* S = current_setup();
  if (!S) return cudaErrorNotReady;
  cudaError_t e = init_launch(a, s);
  if (e != cudaSuccess) return e;
  e = key_bytes == 4 ? rank_column<uint32_t>(*S, a, a.u, a.rank_u, s, true)
                       : rank_column<uint64_t>(*S, a, a.u, a.rank_u, s, true);
  if (e != cudaSuccess) return e;
  e = key_bytes == 4 ? rank_column<uint32_t>(*S, a, a.v, a.rank_v, s) : rank_column<uint64_t>(*S, a, a.v, a.rank_v, s);
  if (e != cudaSuccess) return e;
  pi_kernel<<<a.nchunk, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t* sorted = a.rank_u;  // free once pi is built
  chunk_inversions_kernel<<<a.nchunk, kInvBlock, 2 * kChunk * sizeof(uint32_t), s>>>(a, sorted);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cross_inversions_kernel<<<a.nchunk, 256, kChunk * sizeof(uint32_t), s>>>(a, sorted);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  rank_corr_finish_kernel<<<(a.nseg + 127) / 128, 128, 0, s>>>(a, tau, rho);
  return cudaGetLastError();
}

template <typename Real>
static cudaError_t fit_launch(const Setup& S, const StreamArgs& a, cudaStream_t s) {
  const int per_sm = sizeof(Real) == 4 ? S.fit_per_sm32 : S.fit_per_sm64;
  const int grid = std::max(1, std::min(a.nchunk, per_sm * S.sms));
  StreamArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)stream_fit_kernel<Real>, dim3(grid), dim3(256), params, 0, s);
}

cudaError_t launch_stream(int prec, int key_bytes, const StreamArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  const Setup* S = current_setup();
  if (!S) return cudaErrorNotReady;
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
  cudaError_t e = init_launch(a, s);
  if (e == cudaSuccess) e = mark(0);
  if (e != cudaSuccess) return e;
  e = key_bytes == 4 ? rank_column<uint32_t>(*S, a, a.u, a.rank_u, s, true)
                       : rank_column<uint64_t>(*S, a, a.u, a.rank_u, s, true);
  if (e == cudaSuccess) e = mark(1);
  if (e != cudaSuccess) return e;
  e = key_bytes == 4 ? rank_column<uint32_t>(*S, a, a.v, a.rank_v, s) : rank_column<uint64_t>(*S, a, a.v, a.rank_v, s);
  if (e == cudaSuccess) e = mark(2);
  if (e != cudaSuccess) return e;
  pi_kernel<<<a.nchunk, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) == cudaSuccess) e = mark(3);
  if (e != cudaSuccess) return e;
  e = prec == 1 ? fit_launch<float>(*S, a, s) : fit_launch<double>(*S, a, s);
  if (e == cudaSuccess) e = mark(4);
  return e;
}

}  // namespace cop

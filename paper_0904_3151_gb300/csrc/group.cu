// Steps A3-A4: for every kept block set K of a batch, order the n strings of
// one replicate so that strings with equal K blocks are adjacent (Sec. 2.1,
// Fig. 1; Appendix, second trick: only grouping is needed, not a total
// order).  One segment of n items per K; all segments are sorted together.
// The grouping key is computed from the strings inside the first pass and
// never stored unsorted.
//
// One point set: a most-significant-digit pass (shared-memory histograms,
// one exclusive scan, scatter ranked by shared atomics) splits every
// segment into 256 buckets by the top 8 key bits, then one CTA per bucket
// sorts it by the remaining bits in shared memory (three 8-bit LSD passes
// between registers and shared memory) and writes it back in place: one
// write and one read-modify-write of the items in HBM instead of four full
// LSD passes.  Buckets larger than shared memory are sorted by the same CTA
// in chunks through a scratch copy.  Several point sets: an LSD radix sort
// with 8-bit digits whose tiles never straddle a set.
//
// Grouping key of string s under K (kept_bits = bits in the K blocks):
//   kept_bits <= group_bits: the K blocks concatenated (exact), passed
//   through a bijection so that the top bits spread evenly;
//   otherwise: the top group_bits bits of a 64-bit mix of the masked words.
// Unequal K blocks may then share a key; the in-group check rejects such
// pairs, since it requires the K blocks to be equal.
#include <utility>

#include "msm_internal.cuh"

namespace msm {
namespace {

constexpr int kThreads = 256;
constexpr int kRadix = 256;

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  // MurmurHash3 64-bit finaliser (Appleby).
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint64_t extract_bits(const uint64_t* s, int lo,
                                                 int width) {
  int w = lo >> 6, b = lo & 63;
  uint64_t v = s[w] >> b;
  if (b + width > 64) v |= s[w + 1] << (64 - b);
  return width >= 64 ? v : (v & ((1ull << width) - 1));
}

// Per-CTA view of one mask: kept blocks (lo, width) in increasing order.
struct KeptList {
  int n;
  int exact;
  int kbits;              // bits of the K-block part of the key
  int sub_lo, sub_width;  // first gap block appended below the K part
  int lo[kMaxBlocks];
  int width[kMaxBlocks];
  uint64_t keep[kMaxWords];
};

__device__ void setup_kept(KeptList& kl, const MaskDesc& md,
                           const BlockLayout* L, int group_bits) {
  if (threadIdx.x == 0) {
    int c = 0;
    const int k = L->k;
    for (int b = 0; b < k; ++b)
      if (md.K >> b & 1u) {
        kl.lo[c] = L->lo[b];
        kl.width[c] = L->width[b];
        ++c;
      }
    kl.n = c;
    kl.exact = !md.hashed;
    kl.kbits = group_bits - md.sub_width;
    kl.sub_lo = md.sub_lo;
    kl.sub_width = md.sub_width;
    for (int w = 0; w < kMaxWords; ++w) kl.keep[w] = md.keep[w];
  }
}

// A bijection of the b-bit integers (odd multiply, xor-shift, odd multiply,
// all modulo 2^b): an exact K-block part keeps its equality classes, and its
// top bits become evenly spread, as the most-significant-digit pass of the
// grouping needs.
__device__ __forceinline__ uint64_t mix_bits(uint64_t x, int b) {
  const uint64_t mask = b >= 64 ? ~0ull : ((1ull << b) - 1ull);
  x = (x * 0x9E3779B97F4A7C15ull) & mask;
  x ^= x >> ((b + 1) / 2);
  return (x * 0xC2B2AE3D27D4EB4Full) & mask;
}

__device__ __forceinline__ uint32_t group_key(const uint64_t* str, int W,
                                              const KeptList& kl,
                                              int group_bits) {
  uint64_t s[kMaxWords];
#pragma unroll
  for (int w = 0; w < kMaxWords; ++w) s[w] = w < W ? str[w] : 0;
  uint64_t kpart;
  if (kl.exact) {
    kpart = 0;
    int off = 0;
    for (int c = 0; c < kl.n; ++c) {
      kpart |= extract_bits(s, kl.lo[c], kl.width[c]) << off;
      off += kl.width[c];
    }
    kpart = mix_bits(kpart, kl.kbits);
  } else {
    uint64_t h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int w = 0; w < kMaxWords; ++w)
      if (w < W) h = fmix64(h ^ (s[w] & kl.keep[w]));
    kpart = h >> (64 - kl.kbits);
  }
  if (kl.sub_width == 0) return (uint32_t)kpart;
  return (uint32_t)((kpart << kl.sub_width) | extract_bits(s, kl.sub_lo, kl.sub_width));
}

struct SortArgs {
  // pass source: either strings (+ masks) or keys_in/vals_in
  const uint64_t* strings;
  const MaskDesc* masks;
  int W;
  int group_bits;
  const BlockLayout* layout;
  const void* keys_in;
  const uint32_t* vals_in;
  void* keys_out;
  uint32_t* vals_out;
  int64_t n;       // items per segment
  int tiles;       // tiles per segment
  int shift;       // digit shift of this pass
  uint32_t* counts;         // [S][256][tiles] (per set: [256][set's tiles])
  const uint32_t* offsets;  // exclusive scan of counts
  // point sets (NULL tile_set: the segment is one set)
  const int* tile_set;
  const int* set_tile0;
  const int64_t* set_off;
};

// Items of radix tile `tile` of a segment: [base, base + cnt) of the
// segment, with the tile's counter index for digit 0 and the counter stride
// between digits.  Within a segment the counters are laid out set by set,
// digit-major inside a set, so one exclusive scan over all counters gives
// every (segment, set, digit, tile) its output position and every set of a
// segment stays in place.
struct TileSpan {
  int64_t base, cnt, cidx, cstride;
};

__device__ __forceinline__ TileSpan tile_span(const SortArgs& a, int seg, int tile,
                                              int tile_items) {
  int64_t lo = 0, hi = a.n, tile0 = 0, tiles_s = a.tiles;
  if (a.tile_set) {
    const int ss = a.tile_set[tile];
    lo = a.set_off[ss];
    hi = a.set_off[ss + 1];
    tile0 = a.set_tile0[ss];
    tiles_s = a.set_tile0[ss + 1] - tile0;
  }
  const int64_t t = tile - tile0;
  TileSpan sp;
  sp.base = lo + t * tile_items;
  sp.cnt = min((int64_t)tile_items, hi - sp.base);
  sp.cidx = (int64_t)seg * kRadix * a.tiles + kRadix * tile0 + t;
  sp.cstride = tiles_s;
  return sp;
}

template <typename KeyT, bool FROM_STR>
__device__ __forceinline__ KeyT load_key(const SortArgs& a, const KeptList& kl,
                                         int seg, int64_t i) {
  if constexpr (FROM_STR) {
    return (KeyT)group_key(a.strings + i * a.W, a.W, kl, a.group_bits);
  } else {
    return reinterpret_cast<const KeyT*>(a.keys_in)[(int64_t)seg * a.n + i];
  }
}

template <typename KeyT, bool FROM_STR, int IPT>
__global__ void __launch_bounds__(kThreads)
hist_kernel(SortArgs a) {
  __shared__ uint32_t h[kThreads / 32][kRadix];
  __shared__ KeptList kl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int seg = blockIdx.y, tile = blockIdx.x;
  constexpr int TILE = kThreads * IPT;
  for (int t = tid; t < (kThreads / 32) * kRadix; t += kThreads) (&h[0][0])[t] = 0;
  if constexpr (FROM_STR) setup_kept(kl, a.masks[seg], a.layout, a.group_bits);
  __syncthreads();
  const TileSpan sp = tile_span(a, seg, tile, TILE);
  const int64_t base = sp.base, cnt = sp.cnt;
#pragma unroll 4
  for (int j = 0; j < IPT; ++j) {
    int e = j * kThreads + tid;
    bool valid = e < cnt;
    uint32_t digit = 0xFFFFFFFFu;
    if (valid) digit = (uint32_t)(load_key<KeyT, FROM_STR>(a, kl, seg, base + e) >> a.shift) & 0xFFu;
    // a warp whose 32 items share one digit (runs of equal keys) counts it
    // with one add; otherwise every item adds itself (distinct bins mostly)
    const uint32_t d0 = __shfl_sync(0xffffffffu, digit, 0);
    if (__all_sync(0xffffffffu, digit == d0)) {
      if (lane == 0 && valid) h[warp][d0] += 32u;
    } else if (valid) {
      atomicAdd(&h[warp][digit], 1u);
    }
    __syncwarp();
  }
  __syncthreads();
  uint32_t sum = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) sum += h[w][tid];
  a.counts[sp.cidx + (int64_t)tid * sp.cstride] = sum;
}

// Exclusive scan of one value per thread across the CTA (256 threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v,
                                                         uint32_t* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < (int)(blockDim.x >> 5)) tmp[lane] = t;
  }
  __syncthreads();
  uint32_t excl = x - v + (warp > 0 ? tmp[warp - 1] : 0);
  __syncthreads();
  return excl;
}

template <typename KeyT, bool FROM_STR, int IPT>
__global__ void __launch_bounds__(kThreads, 4)
scatter_kernel(SortArgs a) {
  constexpr int TILE = kThreads * IPT;
  constexpr int PER_WARP = 32 * IPT;
  __shared__ KeyT ks[TILE];
  __shared__ uint32_t vs[TILE];
  __shared__ uint32_t wh[kThreads / 32][kRadix];
  __shared__ uint32_t dstart[kRadix];
  __shared__ uint32_t gofs[kRadix];
  __shared__ uint32_t tmp[32];
  __shared__ KeptList kl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int seg = blockIdx.y, tile = blockIdx.x;
  for (int t = tid; t < (kThreads / 32) * kRadix; t += kThreads) (&wh[0][0])[t] = 0;
  if constexpr (FROM_STR) setup_kept(kl, a.masks[seg], a.layout, a.group_bits);
  __syncthreads();
  const TileSpan sp = tile_span(a, seg, tile, TILE);
  const int64_t base = sp.base, cnt = sp.cnt;
  const unsigned lt_mask = (1u << lane) - 1u;

  KeyT key[IPT];
  uint32_t val[IPT], rank[IPT];
  // all loads first (independent, so they are in flight together), then
  // the ranking, whose warp-synchronous steps would serialise them
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const int e = warp * PER_WARP + r * 32 + lane;
    key[r] = 0;
    val[r] = 0;
    if (e < cnt) {
      key[r] = load_key<KeyT, FROM_STR>(a, kl, seg, base + e);
      if constexpr (FROM_STR) val[r] = (uint32_t)(base + e);
      else val[r] = a.vals_in ? a.vals_in[(int64_t)seg * a.n + base + e] : 0u;
    }
  }
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    int e = warp * PER_WARP + r * 32 + lane;
    bool valid = e < cnt;
    const KeyT k = key[r];
    const uint32_t v = val[r];
    (void)v;
    uint32_t digit = valid ? ((uint32_t)(k >> a.shift) & 0xFFu) : 0xFFFFFFFFu;
    if constexpr (FROM_STR) {
      // The first pass reads the items in point order, which nothing below
      // depends on (an LSD sort needs stable passes only after its first;
      // the one-set grouping only needs equal keys together), so an item's
      // rank within its warp and digit is the order of a shared atomic.
      rank[r] = valid ? atomicAdd(&wh[warp][digit], 1u) : 0u;
    } else {
      unsigned peers = __match_any_sync(0xffffffffu, digit);
      int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (valid && lane == leader) old = wh[warp][digit];
      old = __shfl_sync(0xffffffffu, old, leader);
      if (valid && lane == leader) wh[warp][digit] = old + __popc(peers);
      __syncwarp();
      rank[r] = old + __popc(peers & lt_mask);
    }
  }
  __syncthreads();
  // Per digit: prefix over warps, tile total, and the tile's digit start.
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) {
    uint32_t c = wh[w][tid];
    wh[w][tid] = run;
    run += c;
  }
  uint32_t start = block_exclusive_scan(run, tmp);
  dstart[tid] = start;
  gofs[tid] = a.offsets[sp.cidx + (int64_t)tid * sp.cstride];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    int e = warp * PER_WARP + r * 32 + lane;
    if (e < cnt) {
      uint32_t digit = (uint32_t)(key[r] >> a.shift) & 0xFFu;
      uint32_t pos = dstart[digit] + wh[warp][digit] + rank[r];
      ks[pos] = key[r];
      vs[pos] = val[r];
    }
  }
  __syncthreads();
  KeyT* ko = reinterpret_cast<KeyT*>(a.keys_out);
  for (int i = tid; i < cnt; i += kThreads) {
    KeyT k = ks[i];
    uint32_t digit = (uint32_t)(k >> a.shift) & 0xFFu;
    uint32_t dest = gofs[digit] + (uint32_t)(i - dstart[digit]);
    ko[dest] = k;
    if (a.vals_out) a.vals_out[dest] = vs[i];
  }
}

// ----------------------------------------------------------- bucket sort
constexpr int kBT = 512;              // threads of the bucket sort
constexpr int kBIpt = 16;             // items per thread
constexpr int kBCap = kBT * kBIpt;    // items a bucket may hold to sort in place

struct BucketArgs {
  uint32_t* keys;            // items sorted by the top digit, sorted in place
  uint32_t* vals;
  uint32_t* tkeys;           // scratch of the same size (large buckets)
  uint32_t* tvals;
  const uint32_t* offsets;   // exclusive scan of the top-digit counters
  int64_t n;                 // items per segment
  int tiles;                 // top-digit tiles per segment
  int S;                     // segments
  int passes;                // 8-bit passes below the top digit
};

struct BucketSmem {
  uint32_t ks[kBCap];
  uint32_t vs[kBCap];
  uint32_t wh[kBT / 32][kRadix];  // per-warp digit counts, then warp prefixes
  uint32_t dstart[kRadix];        // digit starts in the sorted chunk
  uint32_t run[kRadix];           // running digit offsets (chunked sort)
  uint32_t tmp[32];
};

// Items of a bucket are spread evenly over the CTA's warps in blocked order:
// warp w holds items [w pw, (w + 1) pw), pw = the smallest multiple of 32
// with kBT / 32 * pw >= m, lane l of round r item w pw + 32 r + l; the
// rounds a warp runs grow with the bucket, not with the capacity.
__device__ __forceinline__ int per_warp_items(int m) {
  const int nw = kBT / 32;
  return ((m + nw * 32 - 1) / (nw * 32)) * 32;
}

// Stable rank of the digit (key >> shift) & 0xFF of the first m items
// (held as above, pw items per warp): pos[r] gets the item's place in the
// digit-sorted order, sm.dstart the digit starts and sm.wh[w][d] the count
// of digit d in warps before w.  Ends synchronised.  Not `stable` (the first
// of the LSD passes, whose input order nothing depends on): the rank within a
// warp and digit is the order of a shared atomic instead of the item order.
template <int IPT>
__device__ __forceinline__ void bucket_rank(const uint32_t (&key)[IPT], int shift, int m,
                                            int pw, uint32_t (&pos)[IPT], BucketSmem& sm,
                                            bool stable) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int rounds = pw / 32;
  for (int t = tid; t < (kBT / 32) * kRadix; t += kBT) (&sm.wh[0][0])[t] = 0;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    if (r >= rounds || warp * pw + r * 32 >= m) break;  // warp-uniform
    const int e = warp * pw + r * 32 + lane;
    const bool valid = e < m;
    const uint32_t digit = valid ? (key[r] >> shift) & 0xFFu : 0xFFFFFFFFu;
    if (!stable) {  // warp-uniform
      pos[r] = valid ? atomicAdd(&sm.wh[warp][digit], 1u) : 0u;
      continue;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (valid && lane == leader) old = sm.wh[warp][digit];
    old = __shfl_sync(0xffffffffu, old, leader);
    if (valid && lane == leader) sm.wh[warp][digit] = old + __popc(peers);
    __syncwarp();
    pos[r] = old + __popc(peers & lt_mask);
  }
  __syncthreads();
  uint32_t run = 0;  // thread tid < kRadix owns digit tid
  if (tid < kRadix) {
#pragma unroll
    for (int w = 0; w < kBT / 32; ++w) {
      const uint32_t c = sm.wh[w][tid];
      sm.wh[w][tid] = run;
      run += c;
    }
  }
  const uint32_t ds = block_exclusive_scan(run, sm.tmp);
  if (tid < kRadix) sm.dstart[tid] = ds;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    if (r >= rounds) break;
    const int e = warp * pw + r * 32 + lane;
    if (e < m) {
      const uint32_t digit = (key[r] >> shift) & 0xFFu;
      pos[r] += sm.dstart[digit] + sm.wh[warp][digit];
    }
  }
}

// One CTA per (segment, top digit) bucket: sort its items by the bits below
// the top digit (the last two passes stable; equal keys end up together in
// no particular order).
__global__ void __launch_bounds__(kBT, 2)
bucket_sort_kernel(BucketArgs a) {
  extern __shared__ __align__(16) unsigned char bucket_smem[];
  BucketSmem& sm = *reinterpret_cast<BucketSmem*>(bucket_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int seg = blockIdx.x / kRadix, digit = blockIdx.x % kRadix;
  const int64_t cb = (int64_t)seg * kRadix * a.tiles + (int64_t)digit * a.tiles;
  const int64_t start = a.offsets[cb];
  const int64_t end = digit + 1 < kRadix ? (int64_t)a.offsets[cb + a.tiles]
                                         : (int64_t)(seg + 1) * a.n;
  const int64_t m = end - start;
  if (m <= 1) return;
  uint32_t key[kBIpt], val[kBIpt], pos[kBIpt];
  if (m <= kBCap) {
    const int pw = per_warp_items((int)m), rounds = pw / 32;
#pragma unroll
    for (int r = 0; r < kBIpt; ++r) {
      const int e = warp * pw + r * 32 + lane;
      key[r] = 0;
      val[r] = 0;
      if (r < rounds && e < m) {
        key[r] = a.keys[start + e];
        val[r] = a.vals[start + e];
      }
    }
    for (int p = 0; p < a.passes; ++p) {
      bucket_rank<kBIpt>(key, 8 * p, (int)m, pw, pos, sm, p > 0);
#pragma unroll
      for (int r = 0; r < kBIpt; ++r) {
        if (r >= rounds) break;
        const int e = warp * pw + r * 32 + lane;
        if (e < m) {
          sm.ks[pos[r]] = key[r];
          sm.vs[pos[r]] = val[r];
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kBIpt; ++r) {
        if (r >= rounds) break;
        const int e = warp * pw + r * 32 + lane;
        if (e < m) {
          key[r] = sm.ks[e];
          val[r] = sm.vs[e];
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < m; e += kBT) {  // coalesced write-back
      a.keys[start + e] = sm.ks[e];
      a.vals[start + e] = sm.vs[e];
    }
    return;
  }
  // A bucket larger than shared memory: each pass ranks it kBCap items at a
  // time and scatters them to the other buffer (digit offsets carried from
  // chunk to chunk), alternating between the items and the scratch copy.
  uint32_t *sk = a.keys + start, *sv = a.vals + start;
  uint32_t *dk = a.tkeys + start, *dv = a.tvals + start;
  for (int p = 0; p < a.passes; ++p) {
    const int shift = 8 * p;
    if (tid < kRadix) sm.run[tid] = 0;
    __syncthreads();
    for (int64_t e = tid; e < m; e += kBT) atomicAdd(&sm.run[(sk[e] >> shift) & 0xFFu], 1u);
    __syncthreads();
    const uint32_t c = tid < kRadix ? sm.run[tid] : 0u;
    __syncthreads();
    const uint32_t rs = block_exclusive_scan(c, sm.tmp);
    if (tid < kRadix) sm.run[tid] = rs;
    __syncthreads();
    for (int64_t c0 = 0; c0 < m; c0 += kBCap) {
      const int cm = (int)min((int64_t)kBCap, m - c0);
      const int pw = per_warp_items(cm), rounds = pw / 32;
#pragma unroll
      for (int r = 0; r < kBIpt; ++r) {
        const int e = warp * pw + r * 32 + lane;
        key[r] = 0;
        val[r] = 0;
        if (r < rounds && e < cm) {
          key[r] = sk[c0 + e];
          val[r] = sv[c0 + e];
        }
      }
      bucket_rank<kBIpt>(key, shift, cm, pw, pos, sm, p > 0);
#pragma unroll
      for (int r = 0; r < kBIpt; ++r) {
        if (r >= rounds) break;
        const int e = warp * pw + r * 32 + lane;
        if (e < cm) {
          const uint32_t d = (key[r] >> shift) & 0xFFu;
          const uint32_t q = sm.run[d] + pos[r] - sm.dstart[d];
          dk[q] = key[r];
          dv[q] = val[r];
        }
      }
      __syncthreads();
      // this chunk's digit counts advance the running offsets
      if (tid < kRadix) {
        const uint32_t next = tid + 1 < kRadix ? sm.dstart[tid + 1] : (uint32_t)cm;
        sm.run[tid] += next - sm.dstart[tid];
      }
      __syncthreads();
    }
    uint32_t* t;
    t = sk; sk = dk; dk = t;
    t = sv; sv = dv; dv = t;
  }
  if (sk != a.keys + start) {  // odd number of passes: copy back
    for (int64_t e = tid; e < m; e += kBT) {
      a.keys[start + e] = sk[e];
      a.vals[start + e] = sv[e];
    }
  }
}

// ------------------------------------------------------------------ scans
constexpr int kScanChunk = kThreads * 16;

template <typename T>
__global__ void scan_reduce_kernel(const T* in, int64_t len,
                                   const uint32_t* len_dev, T* partial) {
  if (len_dev) len = min(len, (int64_t)*len_dev);
  int64_t b0 = (int64_t)blockIdx.x * kScanChunk;
  if (b0 >= len) return;
  T s = 0;
  for (int64_t i = b0 + threadIdx.x; i < min(len, b0 + kScanChunk); i += kThreads) s += in[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ T ws[kThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

template <typename T>
__global__ void scan_partials_kernel(T* partial, int64_t nparts,
                                     int64_t len, const uint32_t* len_dev,
                                     T* total) {
  if (len_dev) {
    len = min(len, (int64_t)*len_dev);
    nparts = (len + kScanChunk - 1) / kScanChunk;
  }
  __shared__ T carry_s;
  __shared__ T wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t b = 0; b < nparts; b += blockDim.x) {
    int64_t i = b + threadIdx.x;
    T v = i < nparts ? partial[i] : 0;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      T t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      wsum[lane] = t;
    }
    __syncthreads();
    T excl = x - v + (warp > 0 ? wsum[warp - 1] : 0) + carry_s;
    if (i < nparts) partial[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry_s = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry_s;
}

template <typename T>
__global__ void scan_down_kernel(const T* in, T* out, int64_t len,
                                 const uint32_t* len_dev, const T* partial) {
  if (len_dev) len = min(len, (int64_t)*len_dev);
  int64_t b0 = (int64_t)blockIdx.x * kScanChunk;
  if (b0 >= len) return;
  __shared__ T wsum[kThreads / 32];
  __shared__ T carry_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // 16 consecutive items per thread
  int64_t s0 = b0 + (int64_t)threadIdx.x * 16;
  T loc[16];
  T tsum = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    int64_t i = s0 + j;
    loc[j] = i < len ? in[i] : 0;
    tsum += loc[j];
  }
  T x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  if (threadIdx.x == 0) carry_s = partial[blockIdx.x];
  __syncthreads();
  T wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += wsum[w];
  T run = x - tsum + wpre + carry_s;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    int64_t i = s0 + j;
    if (i < len) out[i] = run;
    run += loc[j];
  }
}

template <typename T>
int exclusive_scan_impl(const T* in, T* out, int64_t len,
                        const uint32_t* len_dev, void* ws, T* total,
                        cudaStream_t s) {
  if (len <= 0) {
    if (total) MSM_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
    return MSM_OK;
  }
  int64_t nparts = (len + kScanChunk - 1) / kScanChunk;
  if (nparts > 0x7fffffff) return set_error("scan too long"), MSM_E_INVAL;
  T* partial = reinterpret_cast<T*>(ws);
  kt_begin(KC_SCAN, s);
  scan_reduce_kernel<T><<<(unsigned)nparts, kThreads, 0, s>>>(in, len, len_dev, partial);
  kt_end(s);
  MSM_LAUNCH("scan_reduce_kernel");
  kt_begin(KC_SCAN, s);
  scan_partials_kernel<T><<<1, 1024, 0, s>>>(partial, nparts, len, len_dev, total);
  kt_end(s);
  MSM_LAUNCH("scan_partials_kernel");
  kt_begin(KC_SCAN, s);
  scan_down_kernel<T><<<(unsigned)nparts, kThreads, 0, s>>>(in, out, len, len_dev, partial);
  kt_end(s);
  MSM_LAUNCH("scan_down_kernel");
  return MSM_OK;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t scan_scratch_bytes(int64_t len) {
  return align256(sizeof(uint64_t) * (size_t)((len + kScanChunk - 1) / kScanChunk + 1));
}

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t len,
                       void* ws, uint32_t* total_dev, cudaStream_t s) {
  return exclusive_scan_impl<uint32_t>(in, out, len, nullptr, ws, total_dev, s);
}

int exclusive_scan_u64(const uint64_t* in, uint64_t* out, int64_t len,
                       void* ws, uint64_t* total_dev, cudaStream_t s) {
  return exclusive_scan_impl<uint64_t>(in, out, len, nullptr, ws, total_dev, s);
}

int exclusive_scan_u64_devlen(const uint64_t* in, uint64_t* out,
                              int64_t len_max, const uint32_t* len_dev,
                              void* ws, uint64_t* total_dev, cudaStream_t s) {
  return exclusive_scan_impl<uint64_t>(in, out, len_max, len_dev, ws, total_dev, s);
}

// ------------------------------------------------------------- grouping
namespace {
constexpr int kIpt32 = 16;
constexpr int kTile32 = kThreads * kIpt32;
}

int group_tile_items() { return kTile32; }

size_t group_scratch_bytes(int64_t n, int S, int nsets) {
  int64_t items = n * S;
  int64_t tiles = (n + kTile32 - 1) / kTile32 + (nsets > 1 ? nsets : 0);
  int64_t counts = (int64_t)S * kRadix * tiles;
  return 4 * align256(sizeof(uint32_t) * (size_t)items) +
         2 * align256(sizeof(uint32_t) * (size_t)counts) +
         scan_scratch_bytes(counts) + 256;
}

int run_grouping(const GroupBatch& b, void* ws, uint32_t** keys_out,
                 uint32_t** vals_out, cudaStream_t s) {
  const int64_t items = b.n * b.S;
  const int tiles = b.sets.tile_set ? b.sets.T : (int)((b.n + kTile32 - 1) / kTile32);
  const int64_t ncounts = (int64_t)b.S * kRadix * tiles;
  if (items >= (1ll << 32)) return set_error("grouping batch too large"), MSM_E_INVAL;
  char* p = reinterpret_cast<char*>(ws);
  uint32_t* kA = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)items);
  uint32_t* vA = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)items);
  uint32_t* kB = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)items);
  uint32_t* vB = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)items);
  uint32_t* counts = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)ncounts);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)ncounts);
  void* scan_ws = p;

  SortArgs a{};
  a.strings = b.strings;
  a.masks = b.masks;
  a.W = b.W;
  a.group_bits = b.group_bits;
  a.layout = b.layout;
  a.n = b.n;
  a.tiles = tiles;
  a.counts = counts;
  a.offsets = offsets;
  a.tile_set = b.sets.tile_set;
  a.set_tile0 = b.sets.set_tile0;
  a.set_off = b.sets.off;
  if (tiles == 0) return set_error("grouping: no radix tiles"), MSM_E_INVAL;
  dim3 grid(tiles, b.S);
  if (!b.sets.tile_set && b.passes >= 2) {
    // one point set: top-digit pass, then every bucket sorted in place
    a.shift = b.group_bits - 8;
    a.keys_in = nullptr;
    a.vals_in = nullptr;
    a.keys_out = kA;
    a.vals_out = vA;
    kt_begin(KC_HIST, s);
    hist_kernel<uint32_t, true, kIpt32><<<grid, kThreads, 0, s>>>(a);
    kt_end(s);
    MSM_LAUNCH("hist_kernel");
    int rc = exclusive_scan_u32(counts, offsets, ncounts, scan_ws, nullptr, s);
    if (rc) return rc;
    kt_begin(KC_SCATTER, s);
    scatter_kernel<uint32_t, true, kIpt32><<<grid, kThreads, 0, s>>>(a);
    kt_end(s);
    MSM_LAUNCH("scatter_kernel");
    BucketArgs ba;
    ba.keys = kA;
    ba.vals = vA;
    ba.tkeys = kB;
    ba.tvals = vB;
    ba.offsets = offsets;
    ba.n = b.n;
    ba.tiles = tiles;
    ba.S = b.S;
    ba.passes = (b.group_bits - 8 + 7) / 8;
    const size_t smem = sizeof(BucketSmem);
    MSM_CUDA(cudaFuncSetAttribute(bucket_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    kt_begin(KC_SCATTER, s);
    bucket_sort_kernel<<<(unsigned)(b.S * kRadix), kBT, smem, s>>>(ba);
    kt_end(s);
    MSM_LAUNCH("bucket_sort_kernel");
    *keys_out = kA;
    *vals_out = vA;
    return MSM_OK;
  }
  uint32_t *ki = nullptr, *vi = nullptr, *ko = kA, *vo = vA;
  for (int pass = 0; pass < b.passes; ++pass) {
    a.shift = 8 * pass;
    a.keys_in = ki;
    a.vals_in = vi;
    a.keys_out = ko;
    a.vals_out = vo;
    kt_begin(KC_HIST, s);
    if (pass == 0) hist_kernel<uint32_t, true, kIpt32><<<grid, kThreads, 0, s>>>(a);
    else hist_kernel<uint32_t, false, kIpt32><<<grid, kThreads, 0, s>>>(a);
    kt_end(s);
    MSM_LAUNCH("hist_kernel");
    int rc = exclusive_scan_u32(counts, offsets, ncounts, scan_ws, nullptr, s);
    if (rc) return rc;
    kt_begin(KC_SCATTER, s);
    if (pass == 0) scatter_kernel<uint32_t, true, kIpt32><<<grid, kThreads, 0, s>>>(a);
    else scatter_kernel<uint32_t, false, kIpt32><<<grid, kThreads, 0, s>>>(a);
    kt_end(s);
    MSM_LAUNCH("scatter_kernel");
    ki = ko;
    vi = vo;
    ko = (ko == kA) ? kB : kA;
    vo = (vo == vA) ? vB : vA;
  }
  *keys_out = ki;
  *vals_out = vi;
  return MSM_OK;
}

// -------------------------------------------------- 64-bit single segment
namespace {
constexpr int kIpt64 = 8;
constexpr int kTile64 = kThreads * kIpt64;
}

size_t sort64_scratch_bytes(int64_t m) {
  int64_t tiles = (m + kTile64 - 1) / kTile64;
  int64_t ncounts = (int64_t)kRadix * tiles;
  return align256(8 * (size_t)m) + align256(4 * (size_t)m) +
         2 * align256(4 * (size_t)ncounts) + scan_scratch_bytes(ncounts) + 256;
}

int sort_pairs64(uint64_t* keys, uint32_t* vals, int64_t m, int key_bits,
                 void* ws, cudaStream_t s) {
  if (m <= 1) return MSM_OK;
  if (m >= (1ll << 32)) return set_error("sort too large"), MSM_E_INVAL;
  const int tiles = (int)((m + kTile64 - 1) / kTile64);
  const int64_t ncounts = (int64_t)kRadix * tiles;
  char* p = reinterpret_cast<char*>(ws);
  uint64_t* kB = reinterpret_cast<uint64_t*>(p); p += align256(8 * (size_t)m);
  uint32_t* vB = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)m);
  uint32_t* counts = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)ncounts);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)ncounts);
  void* scan_ws = p;
  SortArgs a{};
  a.n = m;
  a.tiles = tiles;
  a.counts = counts;
  a.offsets = offsets;
  dim3 grid(tiles, 1);
  int passes = (key_bits + 7) / 8;
  uint64_t *ki = keys, *ko = kB;
  uint32_t *vi = vals, *vo = vals ? vB : nullptr;
  for (int pass = 0; pass < passes; ++pass) {
    a.shift = 8 * pass;
    a.keys_in = ki;
    a.vals_in = vi;
    a.keys_out = ko;
    a.vals_out = vo;
    kt_begin(KC_OTHER, s);
    hist_kernel<uint64_t, false, kIpt64><<<grid, kThreads, 0, s>>>(a);
    kt_end(s);
    MSM_LAUNCH("hist_kernel64");
    int rc = exclusive_scan_u32(counts, offsets, ncounts, scan_ws, nullptr, s);
    if (rc) return rc;
    kt_begin(KC_OTHER, s);
    scatter_kernel<uint64_t, false, kIpt64><<<grid, kThreads, 0, s>>>(a);
    kt_end(s);
    MSM_LAUNCH("scatter_kernel64");
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  if (ki != keys) {
    MSM_CUDA(cudaMemcpyAsync(keys, ki, 8 * (size_t)m, cudaMemcpyDeviceToDevice, s));
    if (vals) MSM_CUDA(cudaMemcpyAsync(vals, vi, 4 * (size_t)m, cudaMemcpyDeviceToDevice, s));
  }
  return MSM_OK;
}

}  // namespace msm

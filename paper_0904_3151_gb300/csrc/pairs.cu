// Steps A5-A7: split each sorted segment into runs of equal grouping keys
// (Sec. 2.1, Fig. 1: equivalence classes), then inspect every pair inside
// each run of two or more items:
//   1. Hamming distance of the two strings <= d (Sec. 2.2: blockwise masking
//      also groups non-neighbours, so the distance is checked);
//   2. the kept set K of this grouping is the set of the k-d lowest-index
//      blocks on which the two strings agree, so a pair is reported under
//      exactly one K (at least k-d blocks agree whenever Hamming <= d);
//   3. no earlier replicate g < q has Hamming <= d (Appendix, first trick).
// Survivors are appended to the candidate list E with warp-aggregated
// atomics.
//
// Work decomposition: a run of size <= 32 is one work item handled by one
// warp (its C(b,2) pairs spread over the lanes); a larger run is split into
// 32 x 32 tiles of its upper triangle, one tile per work item.  Warps take
// contiguous ranges of work items.
#include "distance.cuh"

namespace msm {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = kThreads * 16;
constexpr int kSmall = 32;

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Segment (kept-block set) of batch position x < 2^32, x / n, without the
// emulated 64-bit integer division: the float estimate carries a relative
// error below 2^-21 and the quotient is a segment index below C(16, 8) <
// 2^14, so the truncated estimate is within one of it, and one exact
// comparison fixes it.
__device__ __forceinline__ uint32_t seg_of(uint32_t x, int64_t n, float inv_n) {
  uint32_t q = __float2uint_rz(__uint2float_rz(x) * inv_n);
  const uint64_t p = (uint64_t)q * (uint64_t)n;
  if (p > x) --q;
  else if (p + (uint64_t)n <= x) ++q;
  return q;
}

struct GroupWs {
  uint32_t* cnt_start;    // [chunks]
  uint32_t* cnt_end;      // [chunks]
  uint32_t* off_start;    // [chunks]
  uint32_t* off_end;      // [chunks]
  uint32_t* starts;       // [items/2 + 1]
  uint32_t* ends;         // [items/2 + 1]
  uint64_t* work;         // [items/2 + 1]
  uint64_t* work_prefix;  // [items/2 + 1]
  uint32_t* chunk_group;  // [items/2 + 1]: group holding each chunk's first item
  uint32_t* ngroups;      // [1]
  uint64_t* total_work;   // [1]
  unsigned* grab;         // [1]: next chunk to hand out
  void* scan_ws;
};

GroupWs carve(void* ws, int64_t items) {
  int64_t chunks = (items + kChunk - 1) / kChunk;
  int64_t maxg = items / 2 + 1;
  char* p = reinterpret_cast<char*>(ws);
  GroupWs g;
  g.cnt_start = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)chunks);
  g.cnt_end = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)chunks);
  g.off_start = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)chunks);
  g.off_end = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)chunks);
  g.starts = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)maxg);
  g.ends = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)maxg);
  g.work = reinterpret_cast<uint64_t*>(p); p += align256(8 * (size_t)maxg);
  g.work_prefix = reinterpret_cast<uint64_t*>(p); p += align256(8 * (size_t)maxg);
  g.chunk_group = reinterpret_cast<uint32_t*>(p); p += align256(4 * (size_t)maxg);
  g.ngroups = reinterpret_cast<uint32_t*>(p); p += 256;
  g.total_work = reinterpret_cast<uint64_t*>(p); p += 256;
  g.grab = reinterpret_cast<unsigned*>(p); p += 256;
  g.scan_ws = p;
  return g;
}

// Work items are handed out in chunks of `chunk_size(total, cap)` items
// (at least 32, and few enough chunks to index `cap` of them).
__host__ __device__ __forceinline__ uint64_t chunk_size(uint64_t total, uint64_t cap) {
  const uint64_t c = (total + cap - 1) / cap;
  return c < 32 ? 32 : c;
}

// chunk_group[c] = the group containing work item c * chunk_size.
__global__ void chunk_index_kernel(const uint64_t* work_prefix,
                                   const uint32_t* ngroups,
                                   const uint64_t* total_work, uint64_t cap,
                                   uint32_t* chunk_group) {
  const uint64_t total = *total_work;
  const uint32_t G = *ngroups;
  if (total == 0 || G == 0) return;
  const uint64_t C = chunk_size(total, cap);
  const uint64_t nch = (total + C - 1) / C;
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < nch;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t item = c * C;
    uint32_t lo = 0, hi = G - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (work_prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    chunk_group[c] = lo;
  }
}

__device__ __forceinline__ bool bit_at(const uint32_t* bits, int64_t i) {
  return (bits[i >> 5] >> (i & 31)) & 1u;
}

// Padded shared-memory slot of chunk position e (one pad word per 16), so
// that a thread reading its 16 consecutive keys hits distinct banks.
__device__ __forceinline__ int kslot(int e) { return e + (e >> 4); }
constexpr int kStageWords = kChunk + 2 + (kChunk + 2) / 16 + 1;

// Run boundary flags of the 16 consecutive positions p0 .. p0+15 of this
// thread (bit j of *fs: a run of >= 2 starts at p0 + j; of *fe: one ends
// there).  Runs are equal K-block parts of the key (the key shifted right by
// the segment's sub-key width) inside one segment of n positions and one
// point set (sb: set starts, or NULL for a single set).  The block's keys,
// with one neighbour on each side, are first staged in shared memory by
// coalesced loads.
__device__ __forceinline__ void chunk_flags(const uint32_t* keys, int64_t items, int64_t n,
                                            float inv_n,
                                            const MaskDesc* masks, const uint32_t* sb,
                                            uint32_t* sk, uint32_t* fs_out,
                                            uint32_t* fe_out) {
  const int64_t b0 = (int64_t)blockIdx.x * kChunk;
  for (int e = threadIdx.x; e < kChunk + 2; e += kThreads) {
    const int64_t p = b0 - 1 + e;
    sk[kslot(e)] = (p >= 0 && p < items) ? keys[p] : 0u;
  }
  __syncthreads();
  const int t0 = threadIdx.x * 16;
  const int64_t p0 = b0 + t0;
  uint32_t fs = 0, fe = 0;
  int64_t seg = seg_of((uint32_t)(p0 < items ? p0 : items - 1), n, inv_n);
  int64_t local = p0 - seg * n;
  int sw = p0 < items ? masks[seg].sub_width : 0;
  uint32_t prev = sk[kslot(t0)] >> sw, cur = sk[kslot(t0 + 1)] >> sw;
  for (int j = 0; j < 16; ++j, ++local) {
    if (local >= n) {  // entering the next segment (another kept-block set)
      local -= n;
      ++seg;
      if (p0 + j < items) {
        sw = masks[seg].sub_width;
        cur = sk[kslot(t0 + j + 1)] >> sw;
      }
    }
    const int64_t p = p0 + j;
    const uint32_t next = sk[kslot(t0 + j + 2)] >> sw;
    if (p < items) {
      bool head = (local == 0) || prev != cur;
      bool tail = (local == n - 1) || next != cur;
      if (sb) {
        head = head || bit_at(sb, local);
        tail = tail || (local + 1 < n && bit_at(sb, local + 1));
      }
      fs |= (uint32_t)(head && !tail) << j;
      fe |= (uint32_t)(tail && !head) << j;
    }
    prev = cur;
    cur = next;
  }
  *fs_out = fs;
  *fe_out = fe;
}

__global__ void run_count_kernel(const uint32_t* keys, int64_t items, int64_t n, float inv_n,
                                 const MaskDesc* masks, const uint32_t* sb,
                                 uint32_t* cnt_start,
                                 uint32_t* cnt_end) {
  __shared__ uint32_t sk[kStageWords];
  uint32_t fs, fe;
  chunk_flags(keys, items, n, inv_n, masks, sb, sk, &fs, &fe);
  uint32_t cs = __popc(fs), ce = __popc(fe);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cs += __shfl_xor_sync(0xffffffffu, cs, o);
    ce += __shfl_xor_sync(0xffffffffu, ce, o);
  }
  __shared__ uint32_t ss[kThreads / 32], se[kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    ss[threadIdx.x >> 5] = cs;
    se[threadIdx.x >> 5] = ce;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0, b = 0;
    for (int w = 0; w < kThreads / 32; ++w) { a += ss[w]; b += se[w]; }
    cnt_start[blockIdx.x] = a;
    cnt_end[blockIdx.x] = b;
  }
}

__device__ __forceinline__ uint32_t block_excl(uint32_t v, uint32_t* tmp,
                                               uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  uint32_t pre = 0, tot = 0;
  for (int w = 0; w < kThreads / 32; ++w) {
    if (w < warp) pre += tmp[w];
    tot += tmp[w];
  }
  __syncthreads();
  if (total) *total = tot;
  return x - v + pre;
}

__global__ void run_write_kernel(const uint32_t* keys, int64_t items, int64_t n, float inv_n,
                                 const MaskDesc* masks, const uint32_t* sb,
                                 const uint32_t* off_start,
                                 const uint32_t* off_end, uint32_t* starts,
                                 uint32_t* ends, int64_t nchunks,
                                 const uint32_t* cnt_start, uint32_t* ngroups) {
  __shared__ uint32_t tmp[kThreads / 32];
  __shared__ uint32_t sk[kStageWords];
  const int64_t p0 = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * 16;
  uint32_t fs, fe;  // bit j: start / end at p0 + j
  chunk_flags(keys, items, n, inv_n, masks, sb, sk, &fs, &fe);
  uint32_t os = block_excl(__popc(fs), tmp, nullptr) + off_start[blockIdx.x];
  uint32_t oe = block_excl(__popc(fe), tmp, nullptr) + off_end[blockIdx.x];
  for (int j = 0; j < 16; ++j) {
    if (fs >> j & 1u) starts[os++] = (uint32_t)(p0 + j);
    if (fe >> j & 1u) ends[oe++] = (uint32_t)(p0 + j);
  }
  if (blockIdx.x == nchunks - 1 && threadIdx.x == 0)
    *ngroups = off_start[blockIdx.x] + cnt_start[blockIdx.x];
}

__host__ __device__ __forceinline__ uint64_t tiles_of(uint64_t len) {
  uint64_t t = (len + 31) / 32;
  return t * (t + 1) / 2;
}

// Work of every run (one item per run of at most 32 members, else one per
// 32 x 32 tile of its upper triangle); also adds the in-group pairs to
// *checks.
__global__ void run_work_kernel(const uint32_t* starts, const uint32_t* ends,
                                const uint32_t* ngroups, uint64_t* work,
                                unsigned long long* checks) {
  uint32_t G = *ngroups;
  unsigned long long c = 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint64_t len = (uint64_t)ends[g] - starts[g] + 1;
    work[g] = len <= (uint64_t)kSmall ? 1 : tiles_of(len);
    c += len * (len - 1) / 2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(checks, c);
}

// ------------------------------------------------------------ pair check
struct CheckArgs {
  const uint32_t* keys;     // sorted grouping keys (sub-group test)
  const uint32_t* chunk_group;
  unsigned* grab;
  uint64_t chunk_cap;
  const uint32_t* vals;
  const uint32_t* starts;
  const uint32_t* ends;
  const uint64_t* work_prefix;
  const uint64_t* total_work;
  const uint32_t* ngroups;
  const uint64_t* strings;  // [Q][n][W]
  int64_t n;
  float inv_n;  // 1 / n, for seg_of
  int W;
  int q;
  int d;
  int group_bits;
  const MaskDesc* masks;
  const BlockLayout* layout;
  uint64_t* cand;
  int64_t cap;
  unsigned long long* count;
  // fused recheck (count-only output), see PairBatch
  const void* X;
  int dtype, dim, metric;
  float eps, relS;
  const float* nrm;
  unsigned long long* kept;
  unsigned long long* set_kept;
  const int64_t* set_off;
  int nsets;
  int sw;  // bits per symbol: Hamming distances count differing symbols
  unsigned long long* evaluated;  // pairs that took the per-pair tests (or NULL)
  TileRecs recs;                  // dense-tile records (pool NULL: none)
};

// Number of differing symbols in x = a ^ b (symbols of sw = 1, 2 or 4 bits
// start at multiples of sw within every 16-bit field and every word).
__device__ __forceinline__ uint32_t sym_diff32(uint32_t x, int sw) {
  if (sw == 2) return (x | (x >> 1)) & 0x55555555u;
  if (sw == 4) return (x | (x >> 1) | (x >> 2) | (x >> 3)) & 0x11111111u;
  return x;
}
// sym_diff32 with the symbol width fixed at compile time when SW = 1 (sign
// bits: every bit is a symbol), else read at run time.
template <int SW>
__device__ __forceinline__ uint32_t symd32(uint32_t x, int sw) {
  if constexpr (SW == 1) return x;
  else return sym_diff32(x, sw);
}
__device__ __forceinline__ uint64_t sym_diff64(uint64_t x, int sw) {
  if (sw == 2) return (x | (x >> 1)) & 0x5555555555555555ull;
  if (sw == 4) return (x | (x >> 1) | (x >> 2) | (x >> 3)) & 0x1111111111111111ull;
  return x;
}

// ------------------------------------------------------- fused recheck
// In count-only mode the pairs that pass the tests of a work item are not
// appended to a candidate list: the warp queues them in shared memory (32 at
// a time) and evaluates their distances right away, 4 lanes per pair and 8
// pairs per step, with the decision rule of the stand-alone recheck.  Counts
// stay in registers (warp-uniform) until the set of the work item changes or
// the warp finishes.
struct FuseAcc {
  unsigned long long cand = 0;   // pairs that passed the tests (warp-uniform)
  unsigned long long kept = 0;   // of those, within eps (warp-uniform)
  unsigned long long nre = 0;    // double-precision decisions (per lane)
  unsigned long long mark = 0;   // kept at the start of the current set
  int set = -1;
};

// Set of point p: the largest s with off[s] <= p.
__device__ __forceinline__ int set_of(const int64_t* off, int S, int64_t p) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void fuse_flush_set(const CheckArgs& a, FuseAcc& acc, int lane) {
  if (a.set_kept && acc.set >= 0 && acc.kept > acc.mark && lane == 0)
    atomicAdd(a.set_kept + acc.set, acc.kept - acc.mark);
  acc.mark = acc.kept;
}

// Work item of group start st begins: switch the per-set counter if needed.
__device__ __forceinline__ void fuse_enter(const CheckArgs& a, FuseAcc& acc, uint32_t first_point,
                                           int lane) {
  if (!a.set_kept) return;
  const int s = set_of(a.set_off, a.nsets, first_point);
  if (s != acc.set) {
    fuse_flush_set(a, acc, lane);
    acc.set = s;
  }
}

__device__ __forceinline__ void fuse_finish(const CheckArgs& a, FuseAcc& acc, int lane) {
  fuse_flush_set(a, acc, lane);
  unsigned long long nre = acc.nre;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nre += __shfl_xor_sync(0xffffffffu, nre, o);
  if (lane == 0) {
    if (acc.cand) atomicAdd(a.count, acc.cand);
    if (acc.kept) atomicAdd(a.kept, acc.kept);
    if (nre) atomicAdd(a.kept + 1, nre);
  }
}

// Distances of the nb <= 32 queued pairs q[0..nb).
__device__ __forceinline__ void fuse_eval(const CheckArgs& a, const uint64_t* q, uint32_t nb,
                                          int lane, FuseAcc& acc) {
  const int sl = lane & 3, grp = lane >> 2;
  for (uint32_t r = 0; r < nb; r += 8) {
    const uint32_t slot = r + (uint32_t)grp;
    const bool valid = slot < nb;
    const uint64_t pr = valid ? q[slot] : 0ull;
    const int64_t i = (int64_t)(pr >> 32), j = (int64_t)(pr & 0xffffffffu);
    const float S = dist::group_sq_dist<4, false>(a.X, a.dtype, i, j, a.dim, sl);
    bool keep = false;
    if (valid && sl == 0) {
      const float ni = a.metric == MSM_COSINE ? a.nrm[i] : 0.f;
      const float nj = a.metric == MSM_COSINE ? a.nrm[j] : 0.f;
      bool exact = false;
      dist::decide(a.X, a.dtype, i, j, a.dim, a.metric, a.eps, S, ni, nj, a.relS, false,
                   &keep, &exact);
      acc.nre += exact;
    }
    acc.kept += (unsigned long long)__popc(__ballot_sync(0xffffffffu, keep));
  }
}

__device__ __forceinline__ uint64_t ordered_pair(uint32_t x, uint32_t y) {
  return x < y ? (((uint64_t)x << 32) | y) : (((uint64_t)y << 32) | x);
}

// At most one passing pair (ii, jj) per lane.
__device__ __forceinline__ void fuse_one(const CheckArgs& a, bool pass, uint32_t ii, uint32_t jj,
                                         int lane, uint64_t* q, FuseAcc& acc) {
  const unsigned bal = __ballot_sync(0xffffffffu, pass);
  if (!bal) return;
  if (pass) q[__popc(bal & ((1u << lane) - 1u))] = ordered_pair(ii, jj);
  __syncwarp();
  acc.cand += (unsigned long long)__popc(bal);
  fuse_eval(a, q, (uint32_t)__popc(bal), lane, acc);
  __syncwarp();
}

// The pairs (ia, ib[c]) for the set bits c of each lane's mask.
__device__ __forceinline__ void fuse_mask(const CheckArgs& a, uint32_t mask, uint32_t ia,
                                          const uint32_t* ib, int lane, uint64_t* q,
                                          FuseAcc& acc) {
  const uint32_t cnt = __popc(mask);
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) return;
  acc.cand += total;
  const uint32_t excl = incl - cnt;
  for (uint32_t b0 = 0; b0 < total; b0 += 32) {
    uint32_t m = mask, pos = excl;
    while (m) {
      const int c = __ffs(m) - 1;
      m &= m - 1;
      if (pos >= b0 && pos < b0 + 32) q[pos - b0] = ordered_pair(ia, ib[c]);
      ++pos;
    }
    __syncwarp();
    fuse_eval(a, q, min(32u, total - b0), lane, acc);
    __syncwarp();
  }
}

// The tests of one pair, most selective first:
//   first-mask rule, part 1: every gap block (below max K, not kept)
//   differs -- rejects almost every pair that is not reported here;
//   Hamming <= d;
//   first-mask rule, part 2: the K blocks are equal -- true for every
//   grouped pair unless two different K-block values shared a hashed key;
//   no earlier replicate within d (Appendix).
constexpr int kRegGaps = 6;  // gap masks held in registers (ngap <= d)

template <int W>
__device__ __forceinline__ bool strings_ok(const CheckArgs& a,
                                           const uint64_t (*gm)[W], int ngap,
                                           const uint64_t (&rg)[kRegGaps][W],
                                           const uint64_t* keep, bool hashed,
                                           const uint64_t* si,
                                           const uint64_t* sj) {
  uint64_t x[W];
#pragma unroll
  for (int w = 0; w < W; ++w) x[w] = si[w] ^ sj[w];
#pragma unroll
  for (int gI = 0; gI < kRegGaps; ++gI) {
    if (gI < ngap) {
      uint64_t o = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) o |= x[w] & rg[gI][w];
      if (o == 0) return false;
    }
  }
  for (int gI = kRegGaps; gI < ngap; ++gI) {
    uint64_t o = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) o |= x[w] & gm[gI][w];
    if (o == 0) return false;
  }
  int h = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) h += __popcll(sym_diff64(x[w], a.sw));
  if (h > a.d) return false;
  if (hashed) {
    uint64_t o = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) o |= x[w] & keep[w];
    if (o) return false;
  }
  return true;
}

template <int W>
__device__ __forceinline__ bool replicates_ok(const CheckArgs& a, uint32_t i,
                                              uint32_t j) {
  for (int g = 0; g < a.q; ++g) {
    const uint64_t* gi = a.strings + ((size_t)g * a.n + i) * W;
    const uint64_t* gj = a.strings + ((size_t)g * a.n + j) * W;
    int hg = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) hg += __popcll(sym_diff64(__ldg(gi + w) ^ __ldg(gj + w), a.sw));
    if (hg <= a.d) return false;
  }
  return true;
}

// Appends, for every set bit c of `mask`, the pair (ia, ib[c]): one atomic
// per warp, positions by an inclusive warp scan of the per-lane counts.
__device__ __forceinline__ void emit_mask(const CheckArgs& a, uint32_t mask,
                                          uint32_t ia, const uint32_t* ib,
                                          int lane) {
  uint32_t cnt = __popc(mask), incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane == 31) base = atomicAdd(a.count, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 31) + (incl - cnt);
  while (mask) {
    const int c = __ffs(mask) - 1;
    mask &= mask - 1;
    const uint32_t j = ib[c];
    if (base < (unsigned long long)a.cap) {
      const uint32_t lo = ia < j ? ia : j, hi = ia < j ? j : ia;
      a.cand[base] = ((uint64_t)lo << 32) | hi;
    }
    ++base;
  }
}

// MINB: resident CTAs per SM the register allocation must allow (0: no
// constraint, the compiler's choice).  The fused
// (count-only) variants hold the distance evaluation's loads in registers;
// capping them keeps the integer tests at full occupancy, at the price of
// spills on the rarely taken recheck path.
template <int W, bool FUSE, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
check_kernel(CheckArgs a) {
  __shared__ uint64_t sm_s[kThreads / 32][32][W];
  __shared__ uint32_t sm_i[kThreads / 32][32];
  __shared__ uint64_t sm_q[kThreads / 32][32];  // fused recheck queue
  __shared__ uint64_t bm[kMaxBlocks][W];
  __shared__ uint64_t sm_gm[kThreads / 32][kMaxBlocks][W];  // gap block masks
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < kMaxBlocks * W; t += kThreads)
    bm[t / W][t % W] = a.layout->mask[t / W][t % W];
  __syncthreads();
  const uint64_t total = *a.total_work;
  const uint32_t G = *a.ngroups;
  if (total == 0 || G == 0) return;
  const uint64_t C = chunk_size(total, a.chunk_cap);
  const uint64_t nch = (total + C - 1) / C;
  const uint64_t* pool = a.strings + (size_t)a.q * a.n * W;
  FuseAcc acc;
  uint32_t cur_g = 0xffffffffu;
  int cur_seg = -1, ngap = 0;
  bool hashed = false;
  uint64_t keep[W];
  uint64_t rg[kRegGaps][W];
#pragma unroll
  for (int w = 0; w < W; ++w) keep[w] = 0;
#pragma unroll
  for (int gI = 0; gI < kRegGaps; ++gI)
#pragma unroll
    for (int w = 0; w < W; ++w) rg[gI][w] = 0;
  // chunks of consecutive work items are handed out dynamically: items
  // differ ~10x in cost, so static ranges leave most warps idle at the end
  for (;;) {
  unsigned chunk = 0;
  if (lane == 0) chunk = atomicAdd(a.grab, 1u);
  chunk = __shfl_sync(0xffffffffu, chunk, 0);
  if (chunk >= nch) break;
  const uint64_t w0 = (uint64_t)chunk * C, w1 = min(total, w0 + C);
  uint32_t g = a.chunk_group[chunk];
  for (uint64_t item = w0; item < w1; ++item) {
    while (g + 1 < G && a.work_prefix[g + 1] <= item) ++g;
    const uint64_t local = item - a.work_prefix[g];
    const uint32_t st = a.starts[g];
    const uint32_t len = a.ends[g] - st + 1;
    const int seg = (int)seg_of(st, a.n, a.inv_n);
    if (FUSE && g != cur_g) {
      cur_g = g;
      fuse_enter(a, acc, a.vals[st], lane);
    }
    if (seg != cur_seg) {  // this grouping's first-mask test data
      const MaskDesc& md = a.masks[seg];
      cur_seg = seg;
      ngap = md.ngap;
      hashed = md.hashed != 0;
#pragma unroll
      for (int w = 0; w < W; ++w) keep[w] = md.keep[w];
      __syncwarp();
      if (lane < ngap) {
        const int b = md.gap[lane];
#pragma unroll
        for (int w = 0; w < W; ++w) sm_gm[warp][lane][w] = bm[b][w];
      }
      __syncwarp();
#pragma unroll
      for (int gI = 0; gI < kRegGaps; ++gI)
#pragma unroll
        for (int w = 0; w < W; ++w) rg[gI][w] = gI < ngap ? sm_gm[warp][gI][w] : 0;
    }
    if (len <= kSmall) {
      if (lane < (int)len) {
        uint32_t idx = a.vals[st + lane];
        sm_i[warp][lane] = idx;
#pragma unroll
        for (int w = 0; w < W; ++w) sm_s[warp][lane][w] = pool[(size_t)idx * W + w];
      }
      __syncwarp();
      // pairs enumerated column by column: p = b(b-1)/2 + a, a < b
      const int P = (int)(len * (len - 1) / 2);
      for (int r = 0; r < P; r += 32) {
        const int p = r + lane;
        bool pass = false;
        uint32_t ii = 0, jj = 0;
        if (p < P) {
          int b = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
          while (b * (b - 1) / 2 > p) --b;
          while ((b + 1) * b / 2 <= p) ++b;
          const int aa = p - b * (b - 1) / 2;
          if (strings_ok<W>(a, sm_gm[warp], ngap, rg, keep, hashed, sm_s[warp][aa],
                            sm_s[warp][b])) {
            ii = sm_i[warp][aa];
            jj = sm_i[warp][b];
            const uint32_t i0 = ii < jj ? ii : jj, j0 = ii < jj ? jj : ii;
            pass = replicates_ok<W>(a, i0, j0);
          }
        }
        if constexpr (FUSE) {
          fuse_one(a, pass, ii, jj, lane, sm_q[warp], acc);
          continue;
        }
        // one pair per lane: a ballot gives the positions
        const unsigned bal = __ballot_sync(0xffffffffu, pass);
        if (bal) {
          unsigned long long b0 = 0;
          if (lane == 0) b0 = atomicAdd(a.count, (unsigned long long)__popc(bal));
          b0 = __shfl_sync(0xffffffffu, b0, 0) + __popc(bal & ((1u << lane) - 1u));
          if (pass && b0 < (unsigned long long)a.cap)
            a.cand[b0] = ((uint64_t)(ii < jj ? ii : jj) << 32) | (ii < jj ? jj : ii);
        }
      }
      __syncwarp();
    } else {
      // tile (I, J), I <= J, enumerated column by column over J
      uint64_t J = (uint64_t)((sqrt(8.0 * (double)local + 1.0) - 1.0) * 0.5);
      while (J * (J + 1) / 2 > local) --J;
      while ((J + 1) * (J + 2) / 2 <= local) ++J;
      uint64_t I = local - J * (J + 1) / 2;
      uint32_t ra = (uint32_t)(I * 32 + lane);
      bool va = ra < len;
      uint64_t sa[W];
      uint32_t ia = 0;
      if (va) {
        ia = a.vals[st + ra];
#pragma unroll
        for (int w = 0; w < W; ++w) sa[w] = pool[(size_t)ia * W + w];
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w) sa[w] = 0;
      }
      uint32_t cb = (uint32_t)(J * 32 + lane);
      if (cb < len) {
        uint32_t idx = a.vals[st + cb];
        sm_i[warp][lane] = idx;
#pragma unroll
        for (int w = 0; w < W; ++w) sm_s[warp][lane][w] = pool[(size_t)idx * W + w];
      }
      __syncwarp();
      const bool diag = (I == J);
      const uint32_t ncols = min(32u, len - (uint32_t)(J * 32));
      uint32_t passm = 0;
      if (va) {
        for (uint32_t c = diag ? (uint32_t)lane + 1 : 0u; c < ncols; ++c) {
          if (strings_ok<W>(a, sm_gm[warp], ngap, rg, keep, hashed, sa, sm_s[warp][c])) {
            const uint32_t ib = sm_i[warp][c];
            const uint32_t i0 = ia < ib ? ia : ib, j0 = ia < ib ? ib : ia;
            if (replicates_ok<W>(a, i0, j0)) passm |= 1u << c;
          }
        }
      }
      if constexpr (FUSE) fuse_mask(a, passm, ia, sm_i[warp], lane, sm_q[warp], acc);
      else emit_mask(a, passm, ia, sm_i[warp], lane);
      __syncwarp();
    }
  }
  }
  if constexpr (FUSE) fuse_finish(a, acc, lane);
}

// ------------------------------------------------- field-layout variant
// Every block b of a string is re-packed into its own 16-bit field (word
// b >> 1, bits 16 (b & 1) ...), guard bits zero.  For x = f_i ^ f_j the field
// of a block is nonzero iff bit 15 of (field + 0x7FFF) is set; blocks of at
// most 15 bits cannot carry into the next field, so one add and one mask
// test two blocks per 32-bit word.  The gap test of the first-mask rule
// ("every gap block differs") then costs 3 integer operations per word and
// no branch, whatever the number of gap blocks, and Hamming distances are
// unchanged (guard bits cancel in the xor).
constexpr int kMaxFieldBlocks = 16;

struct FieldLayout {
  int k;
  int lo[kMaxFieldBlocks];
  int width[kMaxFieldBlocks];
};

template <int W>
__device__ __forceinline__ uint64_t pick_word(const uint64_t (&s)[W], int i) {
  uint64_t v = s[0];
#pragma unroll
  for (int w = 1; w < W; ++w) v = (i == w) ? s[w] : v;
  return v;
}

template <int W, int FP>
__global__ void fields_kernel(const uint64_t* strings, int64_t count,
                              FieldLayout L, uint32_t* fields) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    uint64_t s[W];
#pragma unroll
    for (int w = 0; w < W; ++w) s[w] = strings[t * W + w];
    uint32_t f[FP];
#pragma unroll
    for (int w = 0; w < FP; ++w) f[w] = 0;
#pragma unroll
    for (int b = 0; b < kMaxFieldBlocks; ++b) {
      if (b < L.k && (b >> 1) < FP) {
        const int lo = L.lo[b], wd = L.width[b];
        const int wi = lo >> 6, sh = lo & 63;
        uint64_t v = pick_word<W>(s, wi) >> sh;
        if (sh + wd > 64) v |= pick_word<W>(s, wi + 1) << (64 - sh);
        f[b >> 1] |= (uint32_t)(v & ((1ull << wd) - 1)) << ((b & 1) * 16);
      }
    }
#pragma unroll
    for (int w = 0; w < FP; w += 2)
      *reinterpret_cast<uint2*>(fields + t * FP + w) = make_uint2(f[w], f[w + 1]);
  }
}

// Gap test of one pair: true iff every gap field of x = a ^ b is nonzero.
// FU = words that hold fields (the stored FP may include one padding word).
template <int FP, int FU>
__device__ __forceinline__ bool gaps_differ(const uint32_t (&fa)[FP],
                                            const uint32_t* fb,
                                            const uint32_t (&gapf)[FP]) {
  uint32_t bad = 0;
#pragma unroll
  for (int w = 0; w < FU; ++w) {
    const uint32_t x = fa[w] ^ fb[w];
    const uint32_t nz = (x + 0x7FFF7FFFu) & 0x80008000u;
    bad |= gapf[w] & ~nz;
  }
  return bad == 0;
}

// Hamming (differing symbols) <= d and (hashed keys only) all kept fields
// equal.
template <int FP, int FU, int SW>
__device__ __forceinline__ bool fields_rest_ok(const uint32_t (&fa)[FP],
                                               const uint32_t* fb, int d, int sw,
                                               bool hashed,
                                               const uint32_t (&keepf)[FP]) {
  int h = 0;
  uint32_t bad = 0;
#pragma unroll
  for (int w = 0; w < FU; ++w) {
    const uint32_t x = fa[w] ^ fb[w];
    h += __popc(symd32<SW>(x, sw));
    bad |= keepf[w] & ((x + 0x7FFF7FFFu) & 0x80008000u);
  }
  return h <= d && (!hashed || bad == 0);
}

// No replicate g0 <= g < q has the pair within d (Appendix, first trick).
template <int FP, int SW>
__device__ __forceinline__ bool replicates_ok_fields(const CheckArgs& a,
                                                     const uint32_t* fields,
                                                     uint32_t i, uint32_t j, int g0 = 0) {
  for (int g = g0; g < a.q; ++g) {
    const uint2* fi = reinterpret_cast<const uint2*>(fields + ((size_t)g * a.n + i) * FP);
    const uint2* fj = reinterpret_cast<const uint2*>(fields + ((size_t)g * a.n + j) * FP);
    int h = 0;
#pragma unroll
    for (int w = 0; w < FP / 2; ++w) {
      const uint2 p = __ldg(fi + w), q2 = __ldg(fj + w);
      h += __popc(symd32<SW>(p.x ^ q2.x, a.sw)) + __popc(symd32<SW>(p.y ^ q2.y, a.sw));
    }
    if (h <= a.d) return false;
  }
  return true;
}

template <int FP>
__device__ __forceinline__ void load_fields(const uint32_t* pool, uint32_t idx,
                                            uint32_t (&f)[FP]) {
  const uint2* src = reinterpret_cast<const uint2*>(pool + (size_t)idx * FP);
#pragma unroll
  for (int w = 0; w < FP; w += 2) {
    const uint2 v = src[w / 2];
    f[w] = v.x;
    f[w + 1] = v.y;
  }
}

// ------------------------------------------------ pair check (field layout)
// Work items: a run of more than 32 members is split into 32 x 32 tiles
// (I, J), I <= J, of its upper triangle, enumerated column by column, so the
// tiles of one column block J (a strip) are consecutive items; a run of at
// most 32 members is the one diagonal tile (0, 0).  A warp takes chunks of
// consecutive items and reads the metadata of 32 items at once, one per
// lane (group, tile, and the sub-key skip below), so that the dependent
// loads of consecutive items overlap.
//
// Each warp keeps the column block of its last tile in shared memory: the
// members' fields, their replicate-0 fields and, for every gap block of the
// grouping, a reference value and the mask of columns that carry it.  A
// tile of the same strip only stages its rows.
//
// Reference prefilter: the reference of a gap block is its most frequent
// value among the block's 32 columns.  A row and a column that both carry
// it are equal on that gap block, which the first-mask rule rejects, so a
// row drops every column at the reference of each gap block where the row
// itself is at the reference -- one and-not per gap block per row instead
// of a gap test per pair.  Any reference value gives the same result;
// frequent ones drop the most pairs.  Where the rows are the columns (a
// diagonal tile) or a warp holds whole small runs (packed runs), the warp
// matches the values of its lanes instead (match over run and value per gap
// block), which drops exactly the pairs equal on a gap block; small runs
// hold about 40 % of the pairs that reach the exact tests otherwise.  The
// remaining pairs are queued in
// shared memory and take the exact tests 32 at a time, one pair per lane:
// every gap block differs, Hamming <= d, kept blocks equal (hashed keys
// only), and no earlier replicate within d (Appendix) -- replicate 0 from the
// staged fields, later ones from global memory.  Passing pairs are compacted
// to the front of the same queue (a round writes only entries already read)
// and collected in a per-warp buffer that is appended to E with one atomic
// when full, so the pairs of consecutive tiles lie together in E (the
// recheck then finds their rows in L1).
constexpr int kOut = 64;     // per-warp buffer of pairs for E
constexpr int kCheckCtas = 4;  // resident pair-list check CTAs per SM
constexpr int kQueue = 512;  // per-warp queue of pairs for the exact tests

// Field words are staged with an odd row stride SF (FU rounded up to odd):
// 32 lanes reading the words of 32 different columns then hit 32 different
// banks (the even stride of the padded global layout made two columns share
// a bank).
template <int FP, int SF>
struct WarpStage {
  uint32_t cf[32][SF];   // column block: fields of this replicate
  uint32_t cf0[32][SF];  // and of replicate 0
  uint32_t ci[32];       // points
  uint32_t rf[32][SF];   // rows of the current tile (off-diagonal)
  uint32_t rf0[32][SF];
  uint32_t ri[32];
  uint32_t ref[kMaxFieldBlocks];    // reference value per gap block
  uint32_t colat[kMaxFieldBlocks];  // columns at the reference
  uint64_t out[kOut];               // pairs waiting to be appended to E
  uint64_t def[32];                 // pairs waiting for the test of replicates 1 .. q-1
};

// Appends the warp's buffered pairs to E (one atomic).
template <class WS>
__device__ __forceinline__ void flush_out(const CheckArgs& a, WS& ws, uint32_t& nout, int lane) {
  if (!nout) return;
  __syncwarp();
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(a.count, (unsigned long long)nout);
  b = __shfl_sync(0xffffffffu, b, 0);
  for (uint32_t t = lane; t < nout; t += 32)
    if (b + t < (unsigned long long)a.cap) a.cand[b + t] = ws.out[t];
  __syncwarp();
  nout = 0;
}

// Lanes that share a gap-block value with this lane, for a warp whose lanes
// hold the members of runs side by side (a diagonal tile, or packed runs of
// at most 32 members): lanes of the same run `tag` that are equal on some gap
// block of Gs.  The first-mask rule rejects every such pair, so the warp
// drops them before any pair test -- exactly the pairs equal on a gap block,
// where the reference prefilter of an off-diagonal tile only catches those
// at one value per block.  Lanes that hold no member pass a tag of their own.
template <int FP, int FU>
__device__ __forceinline__ uint32_t gap_peers(const uint32_t (&f)[FP], uint32_t Gs,
                                              uint32_t tag) {
  uint32_t peers = 0;
#pragma unroll
  for (int w = 0; w < FU; ++w) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int b = 2 * w + h;
      if (!((Gs >> b) & 1u)) continue;  // warp-uniform
      peers |= __match_any_sync(0xffffffffu, ((f[w] >> (16 * h)) & 0x7FFFu) | (tag << 16));
    }
  }
  return peers;
}

// Replicate test of the deferred pairs ws.def[0 .. ndef), one per lane.  A
// pair that passed every test of this replicate and differs by more than d in
// replicate 0 still has to differ by more than d in replicates 1 .. q-1,
// whose fields are read from global memory (they do not fit in L2).  Few
// pairs get this far (about one in 30 at the scale workload), so testing
// them one batch at a time made nearly every batch of 32 wait for a DRAM
// round trip; collected 32 at a time, a warp waits once per 32 such pairs.
// Passing pairs join the E buffer.  (The count-only form tests them in
// place: its distance evaluation follows each batch.)
template <int FP, int SW, class WS>
__device__ __forceinline__ void flush_deferred(const CheckArgs& a, const uint32_t* fields,
                                               WS& ws, uint32_t& ndef,
                                               uint32_t& nout, int lane) {
  if (!ndef) return;
  __syncwarp();
  bool ok = false;
  uint64_t pr = 0;
  if ((uint32_t)lane < ndef) {
    pr = ws.def[lane];
    ok = replicates_ok_fields<FP, SW>(a, fields, (uint32_t)(pr >> 32), (uint32_t)pr, 1);
  }
  ndef = 0;
  __syncwarp();
  const unsigned bal = __ballot_sync(0xffffffffu, ok);
  if (!bal) return;
  if (nout + __popc(bal) > (uint32_t)kOut) flush_out(a, ws, nout, lane);
  if (ok) ws.out[nout + __popc(bal & ((1u << lane) - 1u))] = pr;
  nout += __popc(bal);
  __syncwarp();
}

// SW = 1: sign bits (symbol width fixed at compile time); 0: read a.sw.
template <int FP, int FU, bool FUSE, int MINB, int SW>
__global__ void __launch_bounds__(kThreads, MINB)
check_fields_kernel(CheckArgs a, const uint32_t* fields) {
  constexpr int SF = FU | 1;
  __shared__ __align__(16) WarpStage<FP, SF> stg[kThreads / 32];
  __shared__ uint64_t sm_q[FUSE ? kThreads / 32 : 1][32];  // fused recheck queue
  __shared__ uint16_t sm_qs[kThreads / 32][kQueue];       // queued pairs: row << 5 | column
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpStage<FP, SF>& ws = stg[warp];
  const uint64_t total = *a.total_work;
  const uint32_t G = *a.ngroups;
  if (total == 0 || G == 0) return;
  const uint64_t C = chunk_size(total, a.chunk_cap);
  const uint64_t nch = (total + C - 1) / C;
  const uint32_t* pool = fields + (size_t)a.q * a.n * FP;
  const uint32_t* pool0 = fields;  // replicate 0
  const bool rep0 = a.q > 0;
  FuseAcc acc;
  uint32_t cur_g = 0xffffffffu;
  int cur_seg = -1;
  uint32_t Gs = 0;  // gap blocks of the current grouping
  bool hashed = false;
  uint32_t gapf[FP], keepf[FP];
#pragma unroll
  for (int w = 0; w < FP; ++w) gapf[w] = keepf[w] = 0;
  uint32_t cache_g = 0xffffffffu, cache_J = 0;  // column block held in ws
  uint32_t nout = 0;                            // pairs in ws.out (warp-uniform)
  uint32_t ndef = 0;                            // pairs in ws.def (warp-uniform)
  unsigned long long evaluated = 0;             // queued pairs (warp-uniform)
  for (;;) {  // dynamic chunks of work items
  unsigned chunk = 0;
  if (lane == 0) chunk = atomicAdd(a.grab, 1u);
  chunk = __shfl_sync(0xffffffffu, chunk, 0);
  if (chunk >= nch) break;
  const uint64_t w0 = (uint64_t)chunk * C, w1 = min(total, w0 + C);
  uint32_t gb = a.chunk_group[chunk];  // group of item w0
  for (uint64_t base = w0; base < w1; base += 32) {
    // metadata of items base .. base + 31, one per lane; every group holds
    // at least one item, so they lie in groups gb .. gb + 31
    const uint64_t item = base + lane;
    const bool iv = item < w1;
    const uint64_t wp = gb + lane < G ? a.work_prefix[gb + lane] : ~0ull;
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) cnt += __shfl_sync(0xffffffffu, wp, i) <= item;
    const uint32_t g = gb + cnt - 1;
    const uint64_t local = item - __shfl_sync(0xffffffffu, wp, (int)((cnt - 1) & 31u));
    gb = __shfl_sync(0xffffffffu, g, 31);
    uint32_t st = 0, len = 0, I = 0, J = 0;
    bool live = false;
    if (iv) {
      st = a.starts[g];
      len = a.ends[g] - st + 1;
      if (len > kSmall) {
        uint64_t J64 = (uint64_t)((sqrtf(8.0f * (float)local + 1.0f) - 1.0f) * 0.5f);
        while (J64 * (J64 + 1) / 2 > local) --J64;
        while ((J64 + 1) * (J64 + 2) / 2 <= local) ++J64;
        J = (uint32_t)J64;
        I = (uint32_t)(local - J64 * (J64 + 1) / 2);
      }
      // every member of the tile in one run of equal full keys: all its
      // pairs are equal on the first gap block, so none is reported here
      live = true;
      if (a.masks[seg_of(st, a.n, a.inv_n)].sub_width) {
        const uint32_t last = min(len - 1, J * 32 + 31);
        live = a.keys[st + I * 32] != a.keys[st + last];
      }
    }
    unsigned lv = __ballot_sync(0xffffffffu, live);
    while (lv) {
    const int t = __ffs(lv) - 1;
    lv &= lv - 1;
    const uint32_t tg = __shfl_sync(0xffffffffu, g, t);
    const uint32_t tst = __shfl_sync(0xffffffffu, st, t);
    const uint32_t tlen = __shfl_sync(0xffffffffu, len, t);
    const uint32_t tI = __shfl_sync(0xffffffffu, I, t);
    const uint32_t tJ = __shfl_sync(0xffffffffu, J, t);
    const int seg = (int)seg_of(tst, a.n, a.inv_n);
    if (FUSE && tg != cur_g) {
      cur_g = tg;
      fuse_enter(a, acc, a.vals[tst], lane);
    }
    if (seg != cur_seg) {
      const MaskDesc& md = a.masks[seg];
      cur_seg = seg;
      hashed = md.hashed != 0;
      // gap blocks: below the highest kept block and not kept
      const uint32_t K = md.K;
      Gs = ((1u << md.maxK) - 1u) & ~K;
#pragma unroll
      for (int w = 0; w < FP; ++w) {
        gapf[w] = ((Gs >> (2 * w)) & 1u ? 0x8000u : 0u) |
                  ((Gs >> (2 * w + 1)) & 1u ? 0x80000000u : 0u);
        keepf[w] = ((K >> (2 * w)) & 1u ? 0x8000u : 0u) |
                   ((K >> (2 * w + 1)) & 1u ? 0x80000000u : 0u);
      }
    }
    // Runs of at most 32 members that follow in the batch and lie in the same
    // grouping are packed into one pass: lanes [O_r, O_r + L_r) hold the
    // members of run r, and a member pairs only with the later members of
    // its own run.
    uint32_t packmask = 1u << t;
    uint32_t ptotal = tlen;
    if (!FUSE && tlen <= (uint32_t)kSmall) {
      while (lv) {
        const int t2 = __ffs(lv) - 1;
        const uint32_t l2 = __shfl_sync(0xffffffffu, len, t2);
        const uint32_t s2 = __shfl_sync(0xffffffffu, st, t2);
        if (l2 > (uint32_t)kSmall || ptotal + l2 > 32u || (int)seg_of(s2, a.n, a.inv_n) != seg) break;
        ptotal += l2;
        packmask |= 1u << t2;
        lv &= lv - 1;
      }
    }
    bool diag;
    uint32_t cand;
    __syncwarp();  // the previous item's queue stage is done with the stage
    if (__popc(packmask) > 1) {
      diag = true;
      // offsets of the packed runs: prefix of their lengths over the batch lanes
      const uint32_t mylen = (packmask >> lane) & 1u ? len : 0u;
      uint32_t inc = mylen;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      uint32_t mst = 0, mend = 0;  // this lane's member position and run end lane
      for (uint32_t pm = packmask; pm; pm &= pm - 1) {
        const int t2 = __ffs(pm) - 1;
        const uint32_t e2 = __shfl_sync(0xffffffffu, inc, t2);
        const uint32_t l2 = __shfl_sync(0xffffffffu, len, t2);
        const uint32_t s2 = __shfl_sync(0xffffffffu, st, t2);
        const uint32_t o2 = e2 - l2;
        if ((uint32_t)lane >= o2 && (uint32_t)lane < e2) {
          mst = s2 + ((uint32_t)lane - o2);
          mend = e2;
        }
      }
      const bool vm = (uint32_t)lane < ptotal;
      uint32_t f[FP], f0[FP];
      uint32_t ic = 0;
#pragma unroll
      for (int w = 0; w < FP; ++w) f[w] = f0[w] = 0;
      if (vm) {
        ic = a.vals[mst];
        load_fields<FP>(pool, ic, f);
        if (rep0) load_fields<FP>(pool0, ic, f0);
      }
#pragma unroll
      for (int w = 0; w < FU; ++w) {
        ws.cf[lane][w] = f[w];
        ws.cf0[lane][w] = f0[w];
      }
      ws.ci[lane] = ic;
      cand = vm ? (((mend == 32u ? 0u : (1u << mend)) - 1u) & ~((2u << lane) - 1u)) : 0u;
      if (lane == 31) cand = 0u;
      cand &= ~gap_peers<FP, FU>(f, Gs, vm ? mend : 64u + (uint32_t)lane);
      cache_g = 0xffffffffu;  // the stage no longer holds a column block
      __syncwarp();
    } else {
    diag = tI == tJ;
    const uint32_t ncols = min(32u, tlen - tJ * 32);
    const bool pf = tlen > 32;  // references serve the off-diagonal tiles
    if (tg != cache_g || tJ != cache_J) {
      // stage the column block, its references and masks
      const uint32_t cb = tJ * 32 + lane;
      const bool vc = cb < tlen;
      uint32_t f[FP], f0[FP];
      uint32_t ic = 0;
#pragma unroll
      for (int w = 0; w < FP; ++w) f[w] = f0[w] = 0;
      if (vc) {
        ic = a.vals[tst + cb];
        load_fields<FP>(pool, ic, f);
        if (rep0) load_fields<FP>(pool0, ic, f0);
      }
#pragma unroll
      for (int w = 0; w < FU; ++w) {
        ws.cf[lane][w] = f[w];
        ws.cf0[lane][w] = f0[w];
      }
      ws.ci[lane] = ic;
      if (pf) {
#pragma unroll
        for (int w = 0; w < FU; ++w) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int b = 2 * w + h;
            if (!((Gs >> b) & 1u)) continue;  // warp-uniform
            // columns outside the block carry a value no field can hold
            const uint32_t v =
                vc ? (f[w] >> (16 * h)) & 0x7FFFu : (0x10000u | (uint32_t)lane);
            const uint32_t peers = __match_any_sync(0xffffffffu, v);
            const uint32_t best = __reduce_max_sync(
                0xffffffffu, ((uint32_t)__popc(peers) << 5) | (uint32_t)lane);
            const uint32_t ref = __shfl_sync(0xffffffffu, v, (int)(best & 31u));
            const uint32_t at = __ballot_sync(0xffffffffu, v == ref);
            if (lane == 0) {
              ws.ref[b] = ref;
              ws.colat[b] = at;
            }
          }
        }
      }
      cache_g = tg;
      cache_J = tJ;
      __syncwarp();
    }
    // rows: the column block itself on the diagonal, else staged here
    const uint32_t ra = tI * 32 + lane;
    const bool va = ra < tlen;
    uint32_t fa[FP];
    if (diag) {
#pragma unroll
      for (int w = 0; w < FP; ++w) fa[w] = w < FU ? ws.cf[lane][w] : 0u;
    } else {
      uint32_t f0[FP];
      uint32_t ia = 0;
#pragma unroll
      for (int w = 0; w < FP; ++w) fa[w] = f0[w] = 0;
      if (va) {
        ia = a.vals[tst + ra];
        load_fields<FP>(pool, ia, fa);
        if (rep0) load_fields<FP>(pool0, ia, f0);
      }
#pragma unroll
      for (int w = 0; w < FU; ++w) {
        ws.rf[lane][w] = fa[w];
        ws.rf0[lane][w] = f0[w];
      }
      ws.ri[lane] = ia;
    }
    cand = va ? (ncols == 32 ? 0xffffffffu : ((1u << ncols) - 1u)) : 0u;
    if (diag) {
      cand &= lane == 31 ? 0u : (0xffffffffu << (lane + 1));
      cand &= ~gap_peers<FP, FU>(fa, Gs, va ? 0u : 64u + (uint32_t)lane);
    } else if (pf) {
#pragma unroll
      for (int w = 0; w < FU; ++w) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int b = 2 * w + h;
          if (((Gs >> b) & 1u) && ((fa[w] >> (16 * h)) & 0x7FFFu) == ws.ref[b])
            cand &= ~ws.colat[b];
        }
      }
    }
    }  // tile
    const uint32_t nall = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(cand));
    if (nall == 0) continue;
    // the queue holds kQueue pairs: a tile with more is queued in two halves
    // of 16 rows (at most 512 pairs each)
    const int nparts = nall > (uint32_t)kQueue ? 2 : 1;
    for (int part = 0; part < nparts; ++part) {
    const uint32_t cpart = (nparts == 1 || (lane >> 4) == part) ? cand : 0u;
    const uint32_t cnt2 = __popc(cpart);
    uint32_t incl = cnt2;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t nq = __shfl_sync(0xffffffffu, incl, 31);
    if (nq == 0) continue;
    __syncwarp();  // the previous part's queue entries have been read
    // Queue entries row << 5 | column in row-major order.  A lane writing its
    // own row's entries one at a time takes as many steps as the fullest row;
    // the warp writing one row at a time (each lane its column) takes as
    // many as there are rows with entries.  Whichever is shorter; both give
    // the same queue.
    const uint32_t qrows = __ballot_sync(0xffffffffu, cpart != 0u);
    if (__popc(qrows) < __reduce_max_sync(0xffffffffu, cnt2)) {
      uint32_t pos = 0;
      for (uint32_t rr = qrows; rr; rr &= rr - 1) {
        const int r = __ffs(rr) - 1;
        const uint32_t cr = __shfl_sync(0xffffffffu, cpart, r);
        if ((cr >> lane) & 1u)
          sm_qs[warp][pos + __popc(cr & ((1u << lane) - 1u))] =
              (uint16_t)(((uint32_t)r << 5) | (uint32_t)lane);
        pos += __popc(cr);
      }
    } else {
      uint32_t m = cpart, pos = incl - cnt2;
      while (m) {
        const int c = __ffs(m) - 1;
        m &= m - 1;
        sm_qs[warp][pos++] = (uint16_t)(((uint32_t)lane << 5) | (uint32_t)c);
      }
    }
    __syncwarp();
    evaluated += nq;
    const uint32_t (*rowf)[SF] = diag ? ws.cf : ws.rf;
    const uint32_t (*rowf0)[SF] = diag ? ws.cf0 : ws.rf0;
    const uint32_t* rowi = diag ? ws.ci : ws.ri;
    // In a later replicate most queued pairs were already within d in
    // replicate 0 (Appendix, first trick) and are rejected there: that test
    // runs first over the whole queue, whose survivors are compacted in place
    // (a round writes only entries already read), so the other tests run on
    // a few full batches instead of on every batch.
    uint32_t nq1 = nq;
    if (rep0) {
      uint32_t n1 = 0;
      for (uint32_t b0 = 0; b0 < nq; b0 += 32) {
        __syncwarp();
        const uint32_t nb = min(32u, nq - b0);
        bool keep = false;
        uint32_t e = 0;
        if ((uint32_t)lane < nb) {
          e = sm_qs[warp][b0 + lane];
          const uint32_t r = e >> 5, c = e & 31u;
          int h = 0;
#pragma unroll
          for (int w = 0; w < FU; ++w) h += __popc(symd32<SW>(rowf0[r][w] ^ ws.cf0[c][w], a.sw));
          keep = h > a.d;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) sm_qs[warp][n1 + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)e;
        n1 += __popc(bal);
      }
      nq1 = n1;
    }
    uint32_t npass = 0;
    for (uint32_t b0 = 0; b0 < nq1; b0 += 32) {
      __syncwarp();
      const uint32_t nb = min(32u, nq1 - b0);
      bool ok = false, later = false;
      uint32_t ii = 0, jj = 0, e = 0;
      if ((uint32_t)lane < nb) {
        e = sm_qs[warp][b0 + lane];
        const uint32_t r = e >> 5, c = e & 31u;
        uint32_t fr[FP];
#pragma unroll
        for (int w = 0; w < FP; ++w) fr[w] = w < FU ? rowf[r][w] : 0u;
        // a diagonal tile or packed runs dropped every pair equal on a gap
        // block already (gap_peers): the gap test holds for all its pairs
        if ((diag || gaps_differ<FP, FU>(fr, ws.cf[c], gapf)) &&
            fields_rest_ok<FP, FU, SW>(fr, ws.cf[c], a.d, a.sw, hashed, keepf)) {
          ii = rowi[r];
          jj = ws.ci[c];
          if constexpr (FUSE) {  // replicates 1 .. q-1 in place
            ok = !rep0 || replicates_ok_fields<FP, SW>(a, fields, ii < jj ? ii : jj,
                                                   ii < jj ? jj : ii, 1);
          } else {  // replicates 1 .. q-1 are tested later, 32 pairs at a time
            later = a.q > 1;
            ok = a.q <= 1;
          }
        }
      }
      const unsigned dbal = __ballot_sync(0xffffffffu, later);
      if (!FUSE && dbal) {
        if (ndef + __popc(dbal) > 32u) flush_deferred<FP, SW>(a, fields, ws, ndef, nout, lane);
        if (later) ws.def[ndef + __popc(dbal & ((1u << lane) - 1u))] = ordered_pair(ii, jj);
        ndef += __popc(dbal);
        __syncwarp();
      }
      if constexpr (FUSE) {
        fuse_one(a, ok, ii, jj, lane, sm_q[warp], acc);
      } else {
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        __syncwarp();
        if (ok) sm_qs[warp][npass + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)e;
        npass += __popc(bal);
      }
    }
    // A tile (or packed pass) with many passing pairs becomes one record of
    // its points and entries, which the recheck reads with the tile's rows
    // staged once; if the record pool is full its pairs join E as usual.
    bool recorded = false;
    if (!FUSE && a.recs.pool && npass >= a.recs.min_pairs) {
      __syncwarp();
      const uint32_t words = (uint32_t)kRecHeader + (npass + 1) / 2;
      unsigned long long o = ~0ull, idx = 0;
      if (lane == 0) {
        idx = atomicAdd(a.recs.ctr, 1ull);
        if (idx < (unsigned long long)a.recs.cap) {
          o = atomicAdd(a.recs.ctr + 1, (unsigned long long)words);
          if (o + words <= a.recs.pool_cap) atomicAdd(a.recs.ctr + 2, (unsigned long long)npass);
          else o = ~0ull;
        }
      }
      idx = __shfl_sync(0xffffffffu, idx, 0);
      o = __shfl_sync(0xffffffffu, o, 0);
      if (o != ~0ull) {
        uint32_t* R = a.recs.pool + o;
        if (lane == 0) R[0] = npass | (diag ? 0x80000000u : 0u);
        R[1 + lane] = rowi[lane];
        R[33 + lane] = ws.ci[lane];
        for (uint32_t t2 = lane; 2 * t2 < npass; t2 += 32) {
          const uint32_t lo = sm_qs[warp][2 * t2];
          const uint32_t hi = 2 * t2 + 1 < npass ? (uint32_t)sm_qs[warp][2 * t2 + 1] : 0u;
          R[kRecHeader + t2] = lo | (hi << 16);
        }
        if (lane == 0) a.recs.offs[idx] = (uint32_t)o;
        recorded = true;
      } else if (lane == 0 && idx < (unsigned long long)a.recs.cap) {
        a.recs.offs[idx] = kNoRecord;
      }
      __syncwarp();
    }
    if (!FUSE && npass && !recorded) {
      __syncwarp();
      if (nout + npass > (uint32_t)kOut) flush_out(a, ws, nout, lane);
      if (npass > (uint32_t)kOut) {  // a tile with many pairs: its own append
        unsigned long long b1 = 0;
        if (lane == 0) b1 = atomicAdd(a.count, (unsigned long long)npass);
        b1 = __shfl_sync(0xffffffffu, b1, 0);
        for (uint32_t t2 = lane; t2 < npass; t2 += 32) {
          const uint32_t e = sm_qs[warp][t2];
          if (b1 + t2 < (unsigned long long)a.cap)
            a.cand[b1 + t2] = ordered_pair(rowi[e >> 5], ws.ci[e & 31u]);
        }
      } else {
        for (uint32_t t2 = lane; t2 < npass; t2 += 32) {
          const uint32_t e = sm_qs[warp][t2];
          ws.out[nout + t2] = ordered_pair(rowi[e >> 5], ws.ci[e & 31u]);
        }
        nout += npass;
      }
    }
    }  // parts
    }
  }
  }
  if constexpr (!FUSE) {
    flush_deferred<FP, SW>(a, fields, ws, ndef, nout, lane);
    flush_out(a, ws, nout, lane);
  } else {
    fuse_finish(a, acc, lane);
  }
  if (lane == 0 && evaluated && a.evaluated) atomicAdd(a.evaluated, evaluated);
}

// Pairs of a finished list per point set: counts[set of i] += 1 for every
// pair (i, j) (both points lie in one set).
__global__ void set_count_kernel(const uint64_t* pairs, int64_t m, const int64_t* off, int S,
                                 unsigned long long* counts) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < m; base += nwarps * 32) {
    const int64_t t = base + lane;
    const int s = t < m ? set_of(off, S, (int64_t)(pairs[t] >> 32)) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, s);
    if (s >= 0 && lane == __ffs(peers) - 1)
      atomicAdd(counts + s, (unsigned long long)__popc(peers));
  }
}

}  // namespace

int launch_set_counts(const uint64_t* pairs, int64_t m, const int64_t* off, int S,
                      unsigned long long* counts, cudaStream_t s) {
  if (m <= 0) return MSM_OK;
  int64_t grid = (m + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (grid > cap) grid = cap;
  kt_begin(KC_OTHER, s);
  set_count_kernel<<<(int)grid, kThreads, 0, s>>>(pairs, m, off, S, counts);
  kt_end(s);
  MSM_LAUNCH("set_count_kernel");
  return MSM_OK;
}

// Field layout of the strings: usable when every block fits 15 bits and the
// blocks fit 8 words.  Returns the padded word count FP (even), or 0.
int field_words(int ell_sym, int k, int sw) {
  if (k > kMaxFieldBlocks) return 0;
  for (int b = 0; b < k; ++b) {
    const int w = sw * (int)((int64_t)(b + 1) * ell_sym / k - (int64_t)b * ell_sym / k);
    if (w > 15) return 0;
  }
  const int F = (k + 1) / 2;
  return (F + 1) & ~1;
}

int launch_fields(const uint64_t* strings, int64_t count, int ell_sym, int k, int sw,
                  uint32_t* fields, cudaStream_t s) {
  const int FP = field_words(ell_sym, k, sw);
  const int ell = ell_sym * sw;
  const int W = (ell + 63) / 64;
  FieldLayout L;
  L.k = k;
  for (int b = 0; b < kMaxFieldBlocks; ++b) {
    L.lo[b] = b < k ? sw * (int)((int64_t)b * ell_sym / k) : 0;
    L.width[b] = b < k ? sw * (int)((int64_t)(b + 1) * ell_sym / k) - L.lo[b] : 0;
  }
  int64_t grid = (count + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (grid > cap) grid = cap;
  kt_begin(KC_OTHER, s);
#define MSM_FIELDS(WW, FF) \
  if (W == WW && FP == FF) fields_kernel<WW, FF><<<(int)grid, 256, 0, s>>>(strings, count, L, fields)
  MSM_FIELDS(1, 2); else MSM_FIELDS(1, 4); else MSM_FIELDS(1, 6); else MSM_FIELDS(1, 8);
  else MSM_FIELDS(2, 2); else MSM_FIELDS(2, 4); else MSM_FIELDS(2, 6); else MSM_FIELDS(2, 8);
  else MSM_FIELDS(3, 2); else MSM_FIELDS(3, 4); else MSM_FIELDS(3, 6); else MSM_FIELDS(3, 8);
  else MSM_FIELDS(4, 2); else MSM_FIELDS(4, 4); else MSM_FIELDS(4, 6); else MSM_FIELDS(4, 8);
  else {
    kt_end(s);
    return set_error("no field layout for ell=%d k=%d", ell, k), MSM_E_INVAL;
  }
#undef MSM_FIELDS
  kt_end(s);
  MSM_LAUNCH("fields_kernel");
  return MSM_OK;
}

size_t pairs_scratch_bytes(int64_t items) {
  int64_t chunks = (items + kChunk - 1) / kChunk;
  int64_t maxg = items / 2 + 1;
  return 4 * align256(4 * (size_t)chunks) + 3 * align256(4 * (size_t)maxg) +
         2 * align256(8 * (size_t)maxg) + 768 +
         scan_scratch_bytes(maxg > chunks ? maxg : chunks) + 256;
}

int find_groups(const PairBatch& b, void* ws, unsigned long long* checks_dev,
                cudaStream_t s) {
  const int64_t items = b.n * b.S;
  const int64_t chunks = (items + kChunk - 1) / kChunk;
  GroupWs g = carve(ws, items);
  kt_begin(KC_BOUNDS, s);
  run_count_kernel<<<(unsigned)chunks, kThreads, 0, s>>>(b.keys, items, b.n,
                                                        1.0f / (float)b.n, b.masks,
                                                        b.start_bits, g.cnt_start, g.cnt_end);
  kt_end(s);
  MSM_LAUNCH("run_count_kernel");
  int rc = exclusive_scan_u32(g.cnt_start, g.off_start, chunks, g.scan_ws, nullptr, s);
  if (rc) return rc;
  rc = exclusive_scan_u32(g.cnt_end, g.off_end, chunks, g.scan_ws, nullptr, s);
  if (rc) return rc;
  kt_begin(KC_BOUNDS, s);
  run_write_kernel<<<(unsigned)chunks, kThreads, 0, s>>>(
      b.keys, items, b.n, 1.0f / (float)b.n, b.masks, b.start_bits, g.off_start, g.off_end,
      g.starts, g.ends, chunks, g.cnt_start, g.ngroups);
  kt_end(s);
  MSM_LAUNCH("run_write_kernel");
  int grid = num_sms() * 4;
  kt_begin(KC_BOUNDS, s);
  run_work_kernel<<<grid, kThreads, 0, s>>>(g.starts, g.ends, g.ngroups, g.work,
                                            checks_dev);
  kt_end(s);
  MSM_LAUNCH("run_work_kernel");
  rc = exclusive_scan_u64_devlen(g.work, g.work_prefix, items / 2 + 1,
                                 g.ngroups, g.scan_ws, g.total_work, s);
  if (rc) return rc;
  kt_begin(KC_BOUNDS, s);
  chunk_index_kernel<<<grid, kThreads, 0, s>>>(g.work_prefix, g.ngroups, g.total_work,
                                               (uint64_t)(items / 2 + 1), g.chunk_group);
  kt_end(s);
  MSM_LAUNCH("chunk_index_kernel");
  return MSM_OK;
}

int check_groups(const PairBatch& b, void* ws, uint64_t* cand, int64_t cap,
                 unsigned long long* count_dev, cudaStream_t s) {
  const int64_t items = b.n * b.S;
  GroupWs g = carve(ws, items);
  CheckArgs a{};
  a.keys = b.keys;
  a.chunk_group = g.chunk_group;
  a.grab = g.grab;
  a.chunk_cap = (uint64_t)(items / 2 + 1);
  a.vals = b.vals;
  a.starts = g.starts;
  a.ends = g.ends;
  a.work_prefix = g.work_prefix;
  a.total_work = g.total_work;
  a.ngroups = g.ngroups;
  a.strings = b.strings;
  a.n = b.n;
  a.inv_n = 1.0f / (float)b.n;
  a.W = b.W;
  a.q = b.q;
  a.d = b.d;
  a.masks = b.masks;
  a.layout = b.layout;
  a.group_bits = b.group_bits;
  a.cand = cand;
  a.cap = cap;
  a.count = count_dev;
  a.X = b.X;
  a.dtype = b.dtype;
  a.dim = b.dim;
  a.metric = b.metric;
  a.eps = b.eps;
  a.relS = dist::sq_dist_rel(b.dim, 4, false);
  a.nrm = b.nrm;
  a.kept = b.kept;
  a.set_kept = b.set_kept;
  a.set_off = b.set_off;
  a.nsets = b.nsets;
  a.sw = b.sw > 0 ? b.sw : 1;
  a.evaluated = b.evaluated;
  a.recs = b.recs;
  const bool fuse = b.X != nullptr;
  if (fuse && !b.kept) return set_error("fused recheck needs counters"), MSM_E_INVAL;
  const int mb = b.min_blocks ? b.min_blocks : 4;
  const int grid = num_sms() * (b.ctas_per_sm > 0 ? b.ctas_per_sm : 6);
  MSM_CUDA(cudaMemsetAsync(g.grab, 0, sizeof(unsigned), s));
  kt_begin(KC_CHECK, s);
  if (b.fields) {
    // the kernel loops over chunks of work until none is left: one wave of
    // as many CTAs as can be resident (or as tuned)
    void (*kern)(CheckArgs, const uint32_t*) = nullptr;
    // the default launches of sign-bit strings have the symbol width
    // compiled in; tuned variants and E2LSH symbols read it at run time
    const bool sign = a.sw == 1;
#define MSM_CF(P, U, F, M, SW) kern = check_fields_kernel<P, U, F, M, SW>
#define MSM_CHECK_FIELDS(P, U)                                  \
  if (!fuse && b.min_blocks == 6) MSM_CF(P, U, false, 6, 0);     \
  else if (!fuse && b.min_blocks == 8) MSM_CF(P, U, false, 8, 0); \
  else if (!fuse && sign) MSM_CF(P, U, false, 0, 1);             \
  else if (!fuse) MSM_CF(P, U, false, 0, 0);                     \
  else if (mb == 2) MSM_CF(P, U, true, 2, 0);                    \
  else if (mb == 5) MSM_CF(P, U, true, 5, 0);                    \
  else if (sign) MSM_CF(P, U, true, 4, 1);                       \
  else MSM_CF(P, U, true, 4, 0)
    switch (b.FU) {  // words holding fields: ceil(k / 2)
      case 1: MSM_CHECK_FIELDS(2, 1); break;
      case 2: MSM_CHECK_FIELDS(2, 2); break;
      case 3: MSM_CHECK_FIELDS(4, 3); break;
      case 4: MSM_CHECK_FIELDS(4, 4); break;
      case 5: MSM_CHECK_FIELDS(6, 5); break;
      case 6: MSM_CHECK_FIELDS(6, 6); break;
      case 7: MSM_CHECK_FIELDS(8, 7); break;
      case 8: MSM_CHECK_FIELDS(8, 8); break;
      default: kt_end(s); return set_error("bad field word count"), MSM_E_INVAL;
    }
#undef MSM_CHECK_FIELDS
#undef MSM_CF
    int per_sm = b.ctas_per_sm;
    if (per_sm <= 0) {
      MSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
      if (per_sm < 1) per_sm = 1;
      // The pair list check gathers fields through L1: at most 4 CTAs per SM,
      // with shared memory sized for them, so that the rest of the SM's
      // 256 KB stays L1 (5 CTAs fit by registers, but left ~28 KB of L1 and
      // ran 27 % slower).
      if (!fuse && per_sm > kCheckCtas) {
        per_sm = kCheckCtas;
        cudaFuncAttributes fa;
        int dev = 0, smem_sm = 0;
        MSM_CUDA(cudaFuncGetAttributes(&fa, kern));
        MSM_CUDA(cudaGetDevice(&dev));
        MSM_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        const size_t need = (size_t)kCheckCtas * (fa.sharedSizeBytes + 1024);  // + per-CTA reserve
        int pct = smem_sm > 0 ? (int)((need * 100 + smem_sm - 1) / smem_sm) : 100;
        MSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      pct > 100 ? 100 : pct));
      }
    }
    kern<<<num_sms() * per_sm, kThreads, 0, s>>>(a, b.fields);
    kt_end(s);
    MSM_LAUNCH("check_fields_kernel");
    return MSM_OK;
  }
#define MSM_CHECK(WW)                                                     \
  if (fuse) check_kernel<WW, true, 4><<<grid, kThreads, 0, s>>>(a);       \
  else check_kernel<WW, false, 0><<<grid, kThreads, 0, s>>>(a)
  switch (b.W) {
    case 1: MSM_CHECK(1); break;
    case 2: MSM_CHECK(2); break;
    case 3: MSM_CHECK(3); break;
    case 4: MSM_CHECK(4); break;
    default: kt_end(s); return set_error("bad word count"), MSM_E_INVAL;
  }
#undef MSM_CHECK
  kt_end(s);
  MSM_LAUNCH("check_kernel");
  return MSM_OK;
}

}  // namespace msm

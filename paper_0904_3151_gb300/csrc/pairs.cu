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
#include "msm_internal.cuh"

namespace msm {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = kThreads * 16;
constexpr int kSmall = 32;

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct GroupWs {
  uint32_t* cnt_start;    // [chunks]
  uint32_t* cnt_end;      // [chunks]
  uint32_t* off_start;    // [chunks]
  uint32_t* off_end;      // [chunks]
  uint32_t* starts;       // [items/2 + 1]
  uint32_t* ends;         // [items/2 + 1]
  uint64_t* work;         // [items/2 + 1]
  uint64_t* work_prefix;  // [items/2 + 1]
  uint32_t* ngroups;      // [1]
  uint64_t* total_work;   // [1]
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
  g.ngroups = reinterpret_cast<uint32_t*>(p); p += 256;
  g.total_work = reinterpret_cast<uint64_t*>(p); p += 256;
  g.scan_ws = p;
  return g;
}

// Run boundary flags of flat position p whose offset in its segment (of
// length n) is `local`.
__device__ __forceinline__ void run_flags(const uint32_t* keys, int64_t n,
                                          int64_t p, int64_t local,
                                          bool& start, bool& end) {
  uint32_t k = keys[p];
  bool head = (local == 0) || keys[p - 1] != k;
  bool tail = (local == n - 1) || keys[p + 1] != k;
  start = head && !tail;
  end = tail && !head;
}

__global__ void run_count_kernel(const uint32_t* keys, int64_t items, int64_t n,
                                 uint32_t* cnt_start, uint32_t* cnt_end) {
  int64_t p0 = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * 16;
  uint32_t cs = 0, ce = 0;
  int64_t local = p0 % n;
  for (int j = 0; j < 16; ++j, ++local) {
    if (local >= n) local -= n;
    int64_t p = p0 + j;
    if (p < items) {
      bool s, e;
      run_flags(keys, n, p, local, s, e);
      cs += s;
      ce += e;
    }
  }
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

__global__ void run_write_kernel(const uint32_t* keys, int64_t items, int64_t n,
                                 const uint32_t* off_start,
                                 const uint32_t* off_end, uint32_t* starts,
                                 uint32_t* ends, int64_t nchunks,
                                 const uint32_t* cnt_start, uint32_t* ngroups) {
  __shared__ uint32_t tmp[kThreads / 32];
  int64_t p0 = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * 16;
  uint32_t fs = 0, fe = 0;  // bit j: start / end at p0 + j
  int64_t local = p0 % n;
  for (int j = 0; j < 16; ++j, ++local) {
    if (local >= n) local -= n;
    int64_t p = p0 + j;
    if (p < items) {
      bool s, e;
      run_flags(keys, n, p, local, s, e);
      fs |= (uint32_t)s << j;
      fe |= (uint32_t)e << j;
    }
  }
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
  const uint32_t* vals;
  const uint32_t* starts;
  const uint32_t* ends;
  const uint64_t* work_prefix;
  const uint64_t* total_work;
  const uint32_t* ngroups;
  const uint64_t* strings;  // [Q][n][W]
  int64_t n;
  int W;
  int q;
  int d;
  int group_bits;
  const MaskDesc* masks;
  const BlockLayout* layout;
  uint64_t* cand;
  int64_t cap;
  unsigned long long* count;
};

// The three tests of one pair, cheapest and most selective first.
//   first-mask rule: K blocks equal (only in doubt when keys were hashed)
//   and every gap block (below max K, not kept) different;
//   Hamming <= d; no earlier replicate within d (Appendix).
template <int W>
__device__ __forceinline__ bool pair_ok(const CheckArgs& a,
                                        const uint64_t (*gm)[W], int ngap,
                                        const uint64_t* keep, bool hashed,
                                        uint32_t i, uint32_t j,
                                        const uint64_t* si,
                                        const uint64_t* sj) {
  uint64_t x[W];
#pragma unroll
  for (int w = 0; w < W; ++w) x[w] = si[w] ^ sj[w];
  if (hashed) {
    uint64_t o = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) o |= x[w] & keep[w];
    if (o) return false;
  }
  for (int gI = 0; gI < ngap; ++gI) {
    uint64_t o = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) o |= x[w] & gm[gI][w];
    if (o == 0) return false;
  }
  int h = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) h += __popcll(x[w]);
  if (h > a.d) return false;
  for (int g = 0; g < a.q; ++g) {
    const uint64_t* gi = a.strings + ((size_t)g * a.n + i) * W;
    const uint64_t* gj = a.strings + ((size_t)g * a.n + j) * W;
    int hg = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) hg += __popcll(__ldg(gi + w) ^ __ldg(gj + w));
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

template <int W>
__global__ void __launch_bounds__(kThreads)
check_kernel(CheckArgs a) {
  __shared__ uint64_t sm_s[kThreads / 32][32][W];
  __shared__ uint32_t sm_i[kThreads / 32][32];
  __shared__ uint64_t bm[kMaxBlocks][W];
  __shared__ uint64_t sm_gm[kThreads / 32][kMaxBlocks][W];  // gap block masks
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < kMaxBlocks * W; t += kThreads)
    bm[t / W][t % W] = a.layout->mask[t / W][t % W];
  __syncthreads();
  const uint64_t total = *a.total_work;
  const uint32_t G = *a.ngroups;
  if (total == 0 || G == 0) return;
  const uint64_t nwarps = (uint64_t)gridDim.x * (kThreads / 32);
  const uint64_t gw = (uint64_t)blockIdx.x * (kThreads / 32) + warp;
  const uint64_t per = (total + nwarps - 1) / nwarps;
  const uint64_t w0 = gw * per;
  const uint64_t w1 = min(total, w0 + per);
  if (w0 >= w1) return;
  // group containing work item w0: last g with work_prefix[g] <= w0
  uint32_t lo = 0, hi = G - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (a.work_prefix[mid] <= w0) lo = mid; else hi = mid - 1;
  }
  uint32_t g = lo;
  const uint64_t* pool = a.strings + (size_t)a.q * a.n * W;
  int cur_seg = -1, ngap = 0;
  bool hashed = false;
  uint64_t keep[W];
#pragma unroll
  for (int w = 0; w < W; ++w) keep[w] = 0;
  for (uint64_t item = w0; item < w1; ++item) {
    while (g + 1 < G && a.work_prefix[g + 1] <= item) ++g;
    const uint64_t local = item - a.work_prefix[g];
    const uint32_t st = a.starts[g];
    const uint32_t len = a.ends[g] - st + 1;
    const int seg = (int)(st / a.n);
    if (seg != cur_seg) {  // this grouping's first-mask test data
      const MaskDesc& md = a.masks[seg];
      cur_seg = seg;
      ngap = md.ngap;
      hashed = md.kept_bits > a.group_bits;
#pragma unroll
      for (int w = 0; w < W; ++w) keep[w] = md.keep[w];
      __syncwarp();
      if (lane < ngap) {
        const int b = md.gap[lane];
#pragma unroll
        for (int w = 0; w < W; ++w) sm_gm[warp][lane][w] = bm[b][w];
      }
      __syncwarp();
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
          ii = sm_i[warp][aa];
          jj = sm_i[warp][b];
          const uint32_t i0 = ii < jj ? ii : jj, j0 = ii < jj ? jj : ii;
          pass = pair_ok<W>(a, sm_gm[warp], ngap, keep, hashed, i0, j0,
                            sm_s[warp][aa], sm_s[warp][b]);
        }
        emit_mask(a, pass ? 1u : 0u, ii, &jj, lane);
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
          const uint32_t ib = sm_i[warp][c];
          const uint32_t i0 = ia < ib ? ia : ib, j0 = ia < ib ? ib : ia;
          if (pair_ok<W>(a, sm_gm[warp], ngap, keep, hashed, i0, j0, sa, sm_s[warp][c]))
            passm |= 1u << c;
        }
      }
      emit_mask(a, passm, ia, sm_i[warp], lane);
      __syncwarp();
    }
  }
}

}  // namespace

size_t pairs_scratch_bytes(int64_t items) {
  int64_t chunks = (items + kChunk - 1) / kChunk;
  int64_t maxg = items / 2 + 1;
  return 4 * align256(4 * (size_t)chunks) + 2 * align256(4 * (size_t)maxg) +
         2 * align256(8 * (size_t)maxg) + 512 +
         scan_scratch_bytes(maxg > chunks ? maxg : chunks) + 256;
}

int find_groups(const PairBatch& b, void* ws, unsigned long long* checks_dev,
                cudaStream_t s) {
  const int64_t items = b.n * b.S;
  const int64_t chunks = (items + kChunk - 1) / kChunk;
  GroupWs g = carve(ws, items);
  kt_begin(KC_BOUNDS, s);
  run_count_kernel<<<(unsigned)chunks, kThreads, 0, s>>>(b.keys, items, b.n,
                                                        g.cnt_start, g.cnt_end);
  kt_end(s);
  MSM_LAUNCH("run_count_kernel");
  int rc = exclusive_scan_u32(g.cnt_start, g.off_start, chunks, g.scan_ws, nullptr, s);
  if (rc) return rc;
  rc = exclusive_scan_u32(g.cnt_end, g.off_end, chunks, g.scan_ws, nullptr, s);
  if (rc) return rc;
  kt_begin(KC_BOUNDS, s);
  run_write_kernel<<<(unsigned)chunks, kThreads, 0, s>>>(
      b.keys, items, b.n, g.off_start, g.off_end, g.starts, g.ends, chunks,
      g.cnt_start, g.ngroups);
  kt_end(s);
  MSM_LAUNCH("run_write_kernel");
  int grid = num_sms() * 4;
  kt_begin(KC_BOUNDS, s);
  run_work_kernel<<<grid, kThreads, 0, s>>>(g.starts, g.ends, g.ngroups, g.work,
                                            checks_dev);
  kt_end(s);
  MSM_LAUNCH("run_work_kernel");
  return exclusive_scan_u64_devlen(g.work, g.work_prefix, items / 2 + 1,
                                   g.ngroups, g.scan_ws, g.total_work, s);
}

int check_groups(const PairBatch& b, void* ws, uint64_t* cand, int64_t cap,
                 unsigned long long* count_dev, cudaStream_t s) {
  const int64_t items = b.n * b.S;
  GroupWs g = carve(ws, items);
  CheckArgs a{};
  a.vals = b.vals;
  a.starts = g.starts;
  a.ends = g.ends;
  a.work_prefix = g.work_prefix;
  a.total_work = g.total_work;
  a.ngroups = g.ngroups;
  a.strings = b.strings;
  a.n = b.n;
  a.W = b.W;
  a.q = b.q;
  a.d = b.d;
  a.masks = b.masks;
  a.layout = b.layout;
  a.group_bits = b.group_bits;
  a.cand = cand;
  a.cap = cap;
  a.count = count_dev;
  int grid = num_sms() * 6;
  kt_begin(KC_CHECK, s);
  switch (b.W) {
    case 1: check_kernel<1><<<grid, kThreads, 0, s>>>(a); break;
    case 2: check_kernel<2><<<grid, kThreads, 0, s>>>(a); break;
    case 3: check_kernel<3><<<grid, kThreads, 0, s>>>(a); break;
    case 4: check_kernel<4><<<grid, kThreads, 0, s>>>(a); break;
    default: kt_end(s); return set_error("bad word count"), MSM_E_INVAL;
  }
  kt_end(s);
  MSM_LAUNCH("check_kernel");
  return MSM_OK;
}

}  // namespace msm

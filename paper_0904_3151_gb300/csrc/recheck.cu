// Step A8 (Sec. 4.1, last step): exact distance test of each candidate pair
// in E, keeping Delta(x_i, x_j) <= eps (Def. 1.1, inclusive).
//
// The decision rule (float path with a derived error bound, double-precision
// definition inside the margin) is in distance.cuh.
#include "distance.cuh"

namespace msm {
namespace {

using namespace dist;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;  // resident CTAs of recheck_kernel per SM
constexpr int kStage = 128;    // kept pairs staged per warp before one append

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// 8 pairs per warp (4 lanes each).  Each CTA walks one contiguous range of
// E, 64 pairs at a time: the pair check appends the pairs of a tile
// together, so the rows of a tile (at most 64 points) are read from HBM or
// L2 once and then hit in L1 for the rest of its pairs.  Kept pairs are
// staged per warp in shared memory and appended kStage at a time: one
// atomic on the output counter per 8 pairs serialised the whole kernel on
// that one address.  A candidate that is not a pair i < j < n is never read:
// it is skipped and reported in *bad (when given).
__global__ void __launch_bounds__(kThreads)
recheck_kernel(const void* X, int dtype, int64_t n, int dim, int metric,
               float eps, const float* nrm, const uint64_t* cand,
               const unsigned long long* m_dev, int64_t m_max,
               uint64_t* pairs_out, float* dist_out, unsigned long long* count,
               unsigned long long* recompute, unsigned* bad, float relS) {
  constexpr int G = 4;  // lanes per pair: 8 pairs per warp in flight
  __shared__ uint64_t st_p[kThreads / 32][kStage];
  __shared__ float st_d[kThreads / 32][kStage];
  const int wb = threadIdx.x >> 5;
  uint32_t ns = 0;  // pairs staged by this warp
  auto flush = [&]() {
    __syncwarp();
    unsigned long long b0 = 0;
    if (lane_id() == 0) b0 = atomicAdd(count, (unsigned long long)ns);
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    for (uint32_t q = lane_id(); q < ns; q += 32) {
      if (pairs_out)
        __stcs(reinterpret_cast<unsigned long long*>(pairs_out) + b0 + q,
               (unsigned long long)st_p[wb][q]);
      if (dist_out) __stcs(dist_out + b0 + q, st_d[wb][q]);
    }
    __syncwarp();
    ns = 0;
  };
  int64_t m = m_max;
  if (m_dev) m = min(m, (int64_t)*m_dev);
  const int lane = threadIdx.x & 31, sl = lane & (G - 1), grp = lane / G;
  constexpr int kPerIter = kThreads / G;
  const int64_t per = ((m + gridDim.x - 1) / gridDim.x + kPerIter - 1) / kPerIter * kPerIter;
  const int64_t c0 = (int64_t)blockIdx.x * per, c1 = min(m, c0 + per);
  unsigned long long nre = 0;
  for (int64_t base = c0 + (threadIdx.x >> 5) * (32 / G); base < c1; base += kPerIter) {
    const int64_t t = base + grp;
    const bool in_range = t < c1;
    // E and the output stream through once: kept out of L2's way of the rows
    const uint64_t pr =
        in_range ? __ldcs(reinterpret_cast<const unsigned long long*>(cand) + t) : 0ull;
    const int64_t i = (int64_t)(pr >> 32), j = (int64_t)(pr & 0xffffffffu);
    const bool valid = in_range && i < j && j < n;
    if (in_range && !valid && sl == 0 && bad) atomicOr(bad, 1u);
    const float S = group_sq_dist<G>(X, dtype, valid ? i : 0, valid ? j : 0, dim, sl);
    bool keep = false, exact = false;
    double delta = 0.0;
    if (valid && sl == 0) {
      const float ni = metric == MSM_COSINE ? nrm[i] : 0.f;
      const float nj = metric == MSM_COSINE ? nrm[j] : 0.f;
      delta = decide(X, dtype, i, j, dim, metric, eps, S, ni, nj, relS, true, &keep, &exact);
      nre += exact;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const uint32_t pos = ns + __popc(bal & ((1u << lane) - 1u));
      st_p[wb][pos] = pr;
      st_d[wb][pos] = (float)delta;
    }
    ns += __popc(bal);
    if (ns > (uint32_t)(kStage - 32 / G)) flush();  // room for one more iteration
  }
  if (ns) flush();
  if (nre) atomicAdd(recompute, nre);
}

// Exhaustive count of pairs within eps: 64 x 64 tiles of the upper
// triangle, each thread 4 x 4 pairs, sequential float accumulation of the
// squared differences (error bound (dim + 5) u S), same decision rule.
constexpr int TB = 64, TK = 32;
__global__ void __launch_bounds__(256)
eps_count_kernel(const void* X, int dtype, int64_t n, int dim, int metric,
                 float eps, const float* nrm, unsigned long long* count,
                 float relS) {
  __shared__ float Xi[TB][TK + 1];
  __shared__ float Xj[TB][TK + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t nb = (n + TB - 1) / TB;
  const int64_t ntiles = nb * (nb + 1) / 2;
  unsigned long long c = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int64_t J = (int64_t)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
    while (J * (J + 1) / 2 > tile) --J;
    while ((J + 1) * (J + 2) / 2 <= tile) ++J;
    const int64_t I = tile - J * (J + 1) / 2;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int k0 = 0; k0 < dim; k0 += TK) {
      for (int e = tid; e < TB * TK; e += 256) {
        const int r = e / TK, cc = e % TK;
        const int64_t ri = I * TB + r, rj = J * TB + r;
        const int kk = k0 + cc;
        Xi[r][cc] = (ri < n && kk < dim) ? ldx(X, dtype, ri * dim + kk) : 0.f;
        Xj[r][cc] = (rj < n && kk < dim) ? ldx(X, dtype, rj * dim + kk) : 0.f;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < TK; ++kk) {
        float av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = Xi[ty * 4 + a][kk];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Xj[tx * 4 + b][kk];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const float t = av[a] - bv[b];
            acc[a][b] = fmaf(t, t, acc[a][b]);
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int64_t i = I * TB + ty * 4 + a, j = J * TB + tx * 4 + b;
        if (i < n && j < n && i < j) {
          const float ni = metric == MSM_COSINE ? nrm[i] : 0.f;
          const float nj = metric == MSM_COSINE ? nrm[j] : 0.f;
          bool keep, exact;
          decide(X, dtype, i, j, dim, metric, eps, acc[a][b], ni, nj, relS, false, &keep, &exact);
          c += keep;
        }
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((tid & 31) == 0 && c) atomicAdd(count, c);
}

// ------------------------------------------------------ dense-tile records
// One CTA of 4 warps per record: the record's 32 or 64 rows are copied whole
// into shared memory (16-byte cp.async, through L2 only), then every listed
// pair takes the decision of recheck_kernel with its sum taken from shared
// memory, one pair per lane.  The rows of a tile are thus read once for all
// its pairs instead of once per pair through L1.
constexpr int kTileThreads = 128;
constexpr int kTileStage = 64;          // kept pairs staged per warp before one append
constexpr int kTileRowBytesMax = 1024;  // rows staged whole up to 1 KB

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// S = sum (a_c - b_c)^2 of two rows held in shared memory as nch 16-byte
// chunks (nch even).  Each step takes chunk q and its partner q + nch/2; a
// lane starts at q = rot mod nch/2 and wraps around within the first half,
// so the 8 lanes of a quarter warp read 8 different chunks (32 different
// banks) whatever rows they hold, all lanes in step.  Eight fma chains over at most dim / 8
// coordinates each: with the difference's rounding (2u in its square) and
// three levels combining the chains, |S' - S| <= (dim / 8 + 8) u S.
__device__ __forceinline__ float smem_sq_dist(const unsigned char* a, const unsigned char* b,
                                              int nch, int dtype, int rot) {
  const uint4* a4 = reinterpret_cast<const uint4*>(a);
  const uint4* b4 = reinterpret_cast<const uint4*>(b);
  float c[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) c[m] = 0.f;
  const int h = nch / 2;
  int q = rot % h;
  for (int t = 0; t < h; ++t) {
    const uint4 x0 = a4[q], y0 = b4[q], x1 = a4[q + h], y1 = b4[q + h];
    if (dtype == MSM_DT_BF16) {  // 8 values per chunk: value v of a chunk feeds chain v
      const uint32_t xa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const uint32_t ya[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const float t0 = __uint_as_float(xa[w] << 16) - __uint_as_float(ya[w] << 16);
        const float t1 = __uint_as_float(xa[w] & 0xffff0000u) - __uint_as_float(ya[w] & 0xffff0000u);
        c[(2 * w) & 7] = fmaf(t0, t0, c[(2 * w) & 7]);
        c[(2 * w + 1) & 7] = fmaf(t1, t1, c[(2 * w + 1) & 7]);
      }
    } else {  // 4 floats per chunk: chunk q feeds chains 0-3, its partner 4-7
      const float d0 = __uint_as_float(x0.x) - __uint_as_float(y0.x);
      const float d1 = __uint_as_float(x0.y) - __uint_as_float(y0.y);
      const float d2 = __uint_as_float(x0.z) - __uint_as_float(y0.z);
      const float d3 = __uint_as_float(x0.w) - __uint_as_float(y0.w);
      const float d4 = __uint_as_float(x1.x) - __uint_as_float(y1.x);
      const float d5 = __uint_as_float(x1.y) - __uint_as_float(y1.y);
      const float d6 = __uint_as_float(x1.z) - __uint_as_float(y1.z);
      const float d7 = __uint_as_float(x1.w) - __uint_as_float(y1.w);
      c[0] = fmaf(d0, d0, c[0]);
      c[1] = fmaf(d1, d1, c[1]);
      c[2] = fmaf(d2, d2, c[2]);
      c[3] = fmaf(d3, d3, c[3]);
      c[4] = fmaf(d4, d4, c[4]);
      c[5] = fmaf(d5, d5, c[5]);
      c[6] = fmaf(d6, d6, c[6]);
      c[7] = fmaf(d7, d7, c[7]);
    }
    q = q + 1 == h ? 0 : q + 1;
  }
  return ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
}

__global__ void __launch_bounds__(kTileThreads)
recheck_tiles_kernel(const void* X, int dtype, int64_t n, int dim, int metric, float eps,
                     const float* nrm, const uint32_t* pool, const uint32_t* offs, uint32_t nrec,
                     uint64_t* pairs_out, float* dist_out, unsigned long long* count,
                     unsigned long long* recompute, float relS) {
  extern __shared__ __align__(16) unsigned char tsm[];
  const int rowb = dim * (dtype == MSM_DT_BF16 ? 2 : 4), nch = rowb / 16;
  unsigned char* rows = tsm;                                            // [64][rowb]
  uint32_t* pts = reinterpret_cast<uint32_t*>(tsm + 64 * (size_t)rowb);  // [64]
  uint64_t* st_p = reinterpret_cast<uint64_t*>(pts + 64);               // [4][kTileStage]
  float* st_d = reinterpret_cast<float*>(st_p + 4 * kTileStage);         // [4][kTileStage]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t* wp = st_p + warp * kTileStage;
  float* wd = st_d + warp * kTileStage;
  uint32_t ns = 0;
  unsigned long long nre = 0;
  auto flush = [&]() {
    __syncwarp();
    unsigned long long b0 = 0;
    if (lane == 0) b0 = atomicAdd(count, (unsigned long long)ns);
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    for (uint32_t t = lane; t < ns; t += 32) {
      if (pairs_out)
        __stcs(reinterpret_cast<unsigned long long*>(pairs_out) + b0 + t,
               (unsigned long long)wp[t]);
      if (dist_out) __stcs(dist_out + b0 + t, wd[t]);
    }
    __syncwarp();
    ns = 0;
  };
  for (uint32_t rec = blockIdx.x; rec < nrec; rec += gridDim.x) {
    const uint32_t o = __ldg(offs + rec);
    if (o == kNoRecord) continue;  // the same for every thread
    const uint32_t* R = pool + o;
    const uint32_t hd = __ldg(R);
    const uint32_t ne = hd & 0x7FFFFFFFu;
    const bool same = (hd >> 31) != 0u;
    const int nr = same ? 32 : 64;
    __syncthreads();  // the previous record's pairs are done with the rows
    if (tid < 64) pts[tid] = __ldg(R + 1 + tid);
    __syncthreads();
    for (int t = tid; t < nr * nch; t += kTileThreads) {
      const int sl = t / nch, ch = t - sl * nch;
      cp_async16(rows + (size_t)sl * rowb + ch * 16,
                 reinterpret_cast<const unsigned char*>(X) + (size_t)pts[sl] * rowb + ch * 16);
    }
    cp_async_wait_all();
    __syncthreads();
    for (uint32_t e0 = (uint32_t)warp * 32; e0 < ne; e0 += kTileThreads) {
      const uint32_t e = e0 + lane;
      bool keep = false;
      double delta = 0.0;
      uint64_t pr = 0;
      if (e < ne) {
        const uint32_t ent = (__ldg(R + kRecHeader + (e >> 1)) >> (16 * (e & 1u))) & 0xFFFFu;
        const int r = (int)(ent >> 5), cs = same ? (int)(ent & 31u) : 32 + (int)(ent & 31u);
        const float S = smem_sq_dist(rows + (size_t)r * rowb, rows + (size_t)cs * rowb, nch,
                                     dtype, lane);
        const uint32_t i = pts[r], j = pts[cs];
        const float ni = metric == MSM_COSINE ? nrm[i] : 0.f;
        const float nj = metric == MSM_COSINE ? nrm[j] : 0.f;
        bool exact = false;
        delta = decide(X, dtype, i, j, dim, metric, eps, S, ni, nj, relS, true, &keep, &exact);
        nre += exact;
        pr = i < j ? (((uint64_t)i << 32) | j) : (((uint64_t)j << 32) | i);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const uint32_t pos = ns + __popc(bal & ((1u << lane) - 1u));
        wp[pos] = pr;
        wd[pos] = (float)delta;
      }
      ns += __popc(bal);
      if (ns > (uint32_t)(kTileStage - 32)) flush();
    }
  }
  if (ns) flush();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nre += __shfl_xor_sync(0xffffffffu, nre, o);
  if (lane == 0 && nre) atomicAdd(recompute, nre);
}

}  // namespace

bool tile_recheck_supported(const void* X, int dtype, int dim) {
  const int rowb = dim * (dtype == MSM_DT_BF16 ? 2 : 4);
  // whole pairs of 16-byte chunks (smem_sq_dist takes two per step)
  return rowb % 32 == 0 && rowb <= kTileRowBytesMax && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
}

int launch_recheck_tiles(const void* X, int dtype, int64_t n, int dim, int metric, float eps,
                         const float* nrm32, const TileRecs& recs, uint32_t nrec,
                         uint64_t* pairs_out, float* dist_out, unsigned long long* count_dev,
                         unsigned long long* recompute_dev, cudaStream_t s) {
  if (nrec == 0) return MSM_OK;
  if (!tile_recheck_supported(X, dtype, dim))
    return set_error("dense-tile recheck: unsupported row shape"), MSM_E_INVAL;
  const int rowb = dim * (dtype == MSM_DT_BF16 ? 2 : 4);
  const size_t smem = 64 * (size_t)rowb + 64 * 4 + 4 * kTileStage * (8 + 4);
  MSM_CUDA(cudaFuncSetAttribute(recheck_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int per_sm = 0;
  MSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, recheck_tiles_kernel,
                                                         kTileThreads, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > (int64_t)nrec) grid = nrec;
  // eight chains of at most dim / 8 terms (smem_sq_dist)
  const float relS = (float)(dim / 8 + 8) * (float)kU;
  kt_begin(KC_RECHECK, s);
  recheck_tiles_kernel<<<(int)grid, kTileThreads, smem, s>>>(
      X, dtype, n, dim, metric, eps, nrm32, recs.pool, recs.offs, nrec, pairs_out, dist_out,
      count_dev, recompute_dev, relS);
  kt_end(s);
  MSM_LAUNCH("recheck_tiles_kernel");
  return MSM_OK;
}

int launch_recheck(const void* X, int dtype, int64_t n, int dim, int metric,
                   float eps, const float* nrm, const uint64_t* cand,
                   const unsigned long long* m_dev, int64_t m_max,
                   uint64_t* pairs_out, float* dist_out,
                   unsigned long long* count_dev,
                   unsigned long long* recompute_dev, unsigned* bad_dev,
                   cudaStream_t s) {
  if (m_max <= 0) return MSM_OK;
  const int64_t warps = (m_max + 7) / 8;
  int64_t grid = (warps * 32 + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms() * kCtasPerSm;
  if (grid > cap) grid = cap;
  const float relS = sq_dist_rel(dim, 4);
  kt_begin(KC_RECHECK, s);
  recheck_kernel<<<(int)grid, kThreads, 0, s>>>(X, dtype, n, dim, metric, eps, nrm, cand,
                                                m_dev, m_max, pairs_out, dist_out,
                                                count_dev, recompute_dev, bad_dev, relS);
  kt_end(s);
  MSM_LAUNCH("recheck_kernel");
  return MSM_OK;
}

int launch_eps_count(const void* X, int dtype, int64_t n, int dim, int metric,
                     float eps, const float* nrm,
                     unsigned long long* count_dev, cudaStream_t s) {
  const int64_t nb = (n + TB - 1) / TB;
  const int64_t ntiles = nb * (nb + 1) / 2;
  int64_t grid = (int64_t)num_sms() * 8;
  if (grid > ntiles) grid = ntiles;
  const float relS = (float)(dim + 6) * (float)kU;
  kt_begin(KC_OTHER, s);
  eps_count_kernel<<<(int)grid, 256, 0, s>>>(X, dtype, n, dim, metric, eps, nrm, count_dev,
                                             relS);
  kt_end(s);
  MSM_LAUNCH("eps_count_kernel");
  return MSM_OK;
}

}  // namespace msm

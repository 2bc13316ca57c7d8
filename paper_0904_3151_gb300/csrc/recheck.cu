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

}  // namespace

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

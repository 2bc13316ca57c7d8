// Step A1, Eq. 3: s_{q,i,c} = 1 iff r_{q,c}^T x_i > 0, packed 64 bits per
// word, plus the row norms used by the margin tests and by the recheck.
//
// Exactness: the float dot product t' of a row and a column differs from the
// exact t by at most gamma_D * sum_d |x_d r_d| <= gamma_D |x| |r|
// (gamma_D = D u / (1 - D u), u = 2^-24; Higham, Accuracy and Stability of
// Numerical Algorithms, Sec. 3.1).  Whenever |t'| is within twice that bound
// of zero, the sign is decided again from the double-precision dot product
// accumulated by sequential fma over the coordinates, so every bit equals the
// sign of that double-precision value.
#include <cuda_bf16.h>

#include "msm_internal.cuh"

namespace msm {
namespace {

__device__ __forceinline__ float load_x(const void* X, int dtype, int64_t idx) {
  if (dtype == MSM_DT_BF16)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[idx]);
  return reinterpret_cast<const float*>(X)[idx];
}

// One warp per row: double-precision sum of squares, flags for zero rows
// and non-finite values.
__global__ void row_norms_kernel(const void* X, int dtype, int64_t n, int dim,
                                 double* nrm64, float* nrm32,
                                 unsigned* flags) {
  int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned f = 0;
  for (int64_t i = warp; i < n; i += nwarps) {
    double acc = 0.0;
    for (int c = lane; c < dim; c += 32) {
      double v = (double)load_x(X, dtype, i * dim + c);
      acc = fma(v, v, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      double r = sqrt(acc);
      if (nrm64) nrm64[i] = r;
      if (nrm32) nrm32[i] = (float)r;
      if (acc == 0.0) f |= 1u;
      if (!isfinite(acc)) f |= 2u;
    }
  }
  if (lane == 0 && f) atomicOr(flags, f);
}

__global__ void col_norms_kernel(const float* R, int Q, int dim, int ell,
                                 float* rn) {
  int64_t total = (int64_t)Q * ell;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int q = (int)(t / ell), c = (int)(t % ell);
    const float* Rq = R + (size_t)q * dim * ell;
    double acc = 0.0;
    for (int dd = 0; dd < dim; ++dd) {
      double v = (double)Rq[(size_t)dd * ell + c];
      acc = fma(v, v, acc);
    }
    rn[t] = (float)sqrt(acc);
  }
}

constexpr int BM = 64, BN = 64, BK = 32, XPAD = 4;

// 64 x 64 tile of X R_q (rows row0.., columns col0..) in float, sequential
// fma over the coordinates; thread (ty, tx) of 256 gets rows ty*4..+3 and
// columns tx*4..+3 in acc.
__device__ __forceinline__ void simt_tile(const void* X, int dtype, int64_t n, int dim,
                                          const float* Rq, int ell, int64_t row0, int col0,
                                          float (*Xs)[BM + XPAD], float (*Rs)[BN],
                                          float (&acc)[4][4]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < dim; k0 += BK) {
#pragma unroll
    for (int j = 0; j < (BM * BK) / 256; ++j) {
      int e = tid + 256 * j;
      int r = e / BK, c = e % BK;
      int64_t row = row0 + r;
      int kk = k0 + c;
      float v = 0.f;
      if (row < n && kk < dim) v = load_x(X, dtype, row * dim + kk);
      Xs[c][r] = v;
    }
#pragma unroll
    for (int j = 0; j < (BK * BN) / 256; ++j) {
      int e = tid + 256 * j;
      int kk = e / BN, cc = e % BN;
      int col = col0 + cc;
      float v = 0.f;
      if (k0 + kk < dim && col < ell) v = Rq[(size_t)(k0 + kk) * ell + col];
      Rs[kk][cc] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      float4 a = *reinterpret_cast<const float4*>(&Xs[kk][ty * 4]);
      float4 b = *reinterpret_cast<const float4*>(&Rs[kk][tx * 4]);
      float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// Grid: x = row tiles of 64, y = Q * W column tiles (one output word per
// row).  256 threads; thread (ty, tx) owns rows ty*4..+3, columns tx*4..+3.
__global__ void __launch_bounds__(256)
project_simt_kernel(const void* X, int dtype, int64_t n, int dim,
                    const float* R, const float* rnorm, const float* xnorm,
                    int Q, int ell, int W, float mscale, float mabs,
                    uint64_t* strings, unsigned long long* recompute) {
  __shared__ __align__(16) float Xs[BK][BM + XPAD];
  __shared__ __align__(16) float Rs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int q = blockIdx.y / W, w = blockIdx.y % W;
  const int col0 = w * 64;
  const float* Rq = R + (size_t)q * dim * ell;
  float acc[4][4];
  simt_tile(X, dtype, n, dim, Rq, ell, row0, col0, Xs, Rs, acc);

  unsigned long long nre = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t row = row0 + ty * 4 + i;
    uint64_t part = 0;
    if (row < n) {
      float xn = xnorm[row];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int col = col0 + tx * 4 + j;
        if (col < ell) {
          float t = acc[i][j];
          float m = mscale * xn * rnorm[(size_t)q * ell + col] + mabs;
          bool bit;
          if (fabsf(t) <= m) {
            double t64 = 0.0;
            for (int dd = 0; dd < dim; ++dd)
              t64 = fma((double)load_x(X, dtype, row * dim + dd),
                        (double)Rq[(size_t)dd * ell + col], t64);
            bit = t64 > 0.0;
            ++nre;
          } else {
            bit = t > 0.f;
          }
          if (bit) part |= 1ull << (tx * 4 + j);
        }
      }
    }
    // OR the 16 column groups of this row (lanes of one half-warp).
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) part |= __shfl_xor_sync(0xffffffffu, part, o);
    if (tx == 0 && row < n) strings[((size_t)q * n + row) * W + w] = part;
  }
  if (nre) atomicAdd(recompute, nre);
}

// E2LSH symbols (Sec. 3.1; Datar et al. 2004): symbol c of row i is the low
// sw bits of h = floor(t / width + u_c), t = r_c^T x_i.  The float value of
// t / width + u_c is used when it lies farther than its error bound from an
// integer; otherwise t is recomputed in double by sequential fma and h taken
// from the double evaluation of the same expression, which is the definition.
// Grid: x = row tiles of 64, y = Q * ceil(ell / 64) symbol tiles; a tile's 64
// symbols fill sw words of the row's string.
__global__ void __launch_bounds__(256)
project_e2lsh_kernel(const void* X, int dtype, int64_t n, int dim, const float* R,
                     const float* rnorm, const float* xnorm, const float* u, int Q, int ell,
                     int W, int sw, float width, float mscale, float mabs, uint64_t* strings,
                     unsigned long long* recompute) {
  __shared__ __align__(16) float Xs[BK][BM + XPAD];
  __shared__ __align__(16) float Rs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int tiles = (ell + 63) / 64;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int q = blockIdx.y / tiles, tile = blockIdx.y % tiles;
  const int col0 = tile * 64;
  const float* Rq = R + (size_t)q * dim * ell;
  float acc[4][4];
  simt_tile(X, dtype, n, dim, Rq, ell, row0, col0, Xs, Rs, acc);

  const uint64_t smask = (1ull << sw) - 1;
  const int per_word = 16 / sw;  // threads (4 symbols each) sharing a word
  unsigned long long nre = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = row0 + ty * 4 + i;
    uint64_t part = 0;
    if (row < n) {
      const float xn = xnorm[row];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int col = col0 + tx * 4 + j;
        if (col < ell) {
          const float t = acc[i][j];
          const float uc = u[(size_t)q * ell + col];
          const float z = __fadd_rn(__fdiv_rn(t, width), uc);
          const float m = mscale * xn * rnorm[(size_t)q * ell + col] + mabs;
          // |z - z64| <= |t - t64| / width + rounding of the division, the
          // addition and the double reference
          const float e = m / width + 0x1.0p-22f * (fabsf(t) / width + fabsf(z) + 1.f);
          const float fl = floorf(z);
          int64_t h;
          if (z - fl > e && fl + 1.f - z > e && fabsf(z) < 0x1.0p22f) {
            h = (int64_t)fl;
          } else {
            double t64 = 0.0;
            for (int dd = 0; dd < dim; ++dd)
              t64 = fma((double)load_x(X, dtype, row * dim + dd),
                        (double)Rq[(size_t)dd * ell + col], t64);
            h = (int64_t)floor(t64 / (double)width + (double)uc);
            ++nre;
          }
          part |= ((uint64_t)h & smask) << (((tx * 4 + j) * sw) & 63);
        }
      }
    }
    // OR the threads whose symbols share a word
    for (int o = 1; o < per_word; o <<= 1) part |= __shfl_xor_sync(0xffffffffu, part, o);
    const int word = (col0 * sw + tx * 4 * sw) >> 6;
    if (tx % per_word == 0 && row < n && word < W) strings[((size_t)q * n + row) * W + word] = part;
  }
  if (nre) atomicAdd(recompute, nre);
}

}  // namespace

int launch_row_norms(const void* X, int dtype, int64_t n, int dim,
                     double* nrm64, float* nrm32, unsigned* flags,
                     cudaStream_t s) {
  int64_t warps = n;
  int64_t grid = (warps * 32 + 255) / 256;
  int64_t cap = (int64_t)num_sms() * 16;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kt_begin(KC_OTHER, s);
  row_norms_kernel<<<(int)grid, 256, 0, s>>>(X, dtype, n, dim, nrm64, nrm32, flags);
  kt_end(s);
  MSM_LAUNCH("row_norms_kernel");
  return MSM_OK;
}

int launch_col_norms(const float* R, int Q, int dim, int ell, float* rn,
                     cudaStream_t s) {
  int64_t total = (int64_t)Q * ell;
  int grid = (int)((total + 255) / 256);
  if (grid < 1) grid = 1;
  kt_begin(KC_OTHER, s);
  col_norms_kernel<<<grid, 256, 0, s>>>(R, Q, dim, ell, rn);
  kt_end(s);
  MSM_LAUNCH("col_norms_kernel");
  return MSM_OK;
}

int launch_project(const void* X, int dtype, int64_t n, int dim,
                   const float* R, const float* rnorm, const float* xnorm,
                   int Q, int ell, uint64_t* strings,
                   unsigned long long* recompute, cudaStream_t s) {
  int W = (ell + 63) / 64;
  // Twice gamma_D plus slack for the rounding of the two norms; the
  // absolute term covers products that underflow.
  float mscale = (float)(dim + 4) * 0x1.0p-23f;
  float mabs = (float)dim * 0x1.0p-120f;
  dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)(Q * W));
  if (grid.y > 65535) return set_error("Q * W too large"), MSM_E_INVAL;
  kt_begin(KC_PROJECT, s);
  project_simt_kernel<<<grid, 256, 0, s>>>(X, dtype, n, dim, R, rnorm, xnorm,
                                           Q, ell, W, mscale, mabs, strings,
                                           recompute);
  kt_end(s);
  MSM_LAUNCH("project_simt_kernel");
  return MSM_OK;
}

}  // namespace msm

namespace msm {

int launch_project_e2lsh(const void* X, int dtype, int64_t n, int dim, const float* R,
                         const float* rnorm, const float* xnorm, const float* u, int Q,
                         int ell, int sw, float width, uint64_t* strings,
                         unsigned long long* recompute, cudaStream_t s) {
  if (sw != 1 && sw != 2 && sw != 4) return set_error("symbol bits must be 1, 2 or 4"), MSM_E_INVAL;
  if (!(width > 0.f)) return set_error("E2LSH bucket width must be > 0"), MSM_E_INVAL;
  const int W = (ell * sw + 63) / 64;
  const float mscale = (float)(dim + 4) * 0x1.0p-23f;
  const float mabs = (float)dim * 0x1.0p-120f;
  dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)(Q * ((ell + 63) / 64)));
  if (grid.y > 65535) return set_error("Q * symbol tiles too large"), MSM_E_INVAL;
  kt_begin(KC_PROJECT, s);
  project_e2lsh_kernel<<<grid, 256, 0, s>>>(X, dtype, n, dim, R, rnorm, xnorm, u, Q, ell, W, sw,
                                            width, mscale, mabs, strings, recompute);
  kt_end(s);
  MSM_LAUNCH("project_e2lsh_kernel");
  return MSM_OK;
}

}  // namespace msm

// Step A0': the Gaussian projection matrix R of Eq. 3 (i.i.d. N(0, 1)
// entries, Sec. 3.2), drawn on the device from a counter-based generator so
// that any element can be produced independently of the others.
//
// Generator: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011).  Element
// e uses block e/4 (counter {e/4,0,0,0}, key {seed,0}); words (w0,w1) and
// (w2,w3) each feed one Box-Muller pair in double precision.
#include "msm_internal.cuh"

namespace msm {
namespace {

struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1,
                                               uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  U64x4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

__global__ void gaussian_kernel(uint64_t seed, int64_t count, float* out) {
  const double two_pi = 2.0 * 3.14159265358979323846;
  int64_t blocks = (count + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < blocks;
       b += (int64_t)gridDim.x * blockDim.x) {
    U64x4 w = philox4x64_10((uint64_t)b, 0, 0, 0, seed, 0);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      double u1 = (double)((w.v[2 * p] >> 11) + 1) * 0x1.0p-53;
      double u2 = (double)(w.v[2 * p + 1] >> 11) * 0x1.0p-53;
      double rad = sqrt(-2.0 * log(u1));
      double ang = two_pi * u2;
      double z0 = rad * cos(ang), z1 = rad * sin(ang);
      int64_t e = 4 * b + 2 * p;
      if (e < count) out[e] = (float)z0;
      if (e + 1 < count) out[e + 1] = (float)z1;
    }
  }
}

// Uniform random pairs (i, j), i != j, of n points, stored (min << 32) |
// max: pair t comes from block t of the same generator under key {seed, 1}
// (words w0, w1); i = w0 mod n, j = w1 mod (n - 1), shifted past i.
__global__ void random_pairs_kernel(uint64_t seed, int64_t m, int64_t n, uint64_t* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const U64x4 w = philox4x64_10((uint64_t)t, 0, 0, 0, seed, 1);
    const uint64_t i = w.v[0] % (uint64_t)n;
    uint64_t j = w.v[1] % (uint64_t)(n - 1);
    if (j >= i) ++j;
    out[t] = i < j ? ((i << 32) | j) : ((j << 32) | i);
  }
}

// E2LSH bucket offsets: element e is the top 24 bits of word 0 of block e
// under key {seed, 2}, times 2^-24 (uniform on [0, 1), exact in float).
__global__ void e2lsh_offsets_kernel(uint64_t seed, int64_t count, float* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const U64x4 w = philox4x64_10((uint64_t)e, 0, 0, 0, seed, 2);
    out[e] = (float)((double)(w.v[0] >> 40) * 0x1.0p-24);
  }
}

}  // namespace

int launch_e2lsh_offsets(uint64_t seed, int64_t count, float* out, cudaStream_t s) {
  if (count <= 0) return MSM_OK;
  int64_t grid = (count + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (grid > cap) grid = cap;
  kt_begin(KC_OTHER, s);
  e2lsh_offsets_kernel<<<(int)grid, 256, 0, s>>>(seed, count, out);
  kt_end(s);
  MSM_LAUNCH("e2lsh_offsets_kernel");
  return MSM_OK;
}

int launch_random_pairs(uint64_t seed, int64_t m, int64_t n, uint64_t* out, cudaStream_t s) {
  if (m <= 0) return MSM_OK;
  if (n < 2) return set_error("random pairs need n >= 2"), MSM_E_INVAL;
  int64_t grid = (m + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (grid > cap) grid = cap;
  kt_begin(KC_OTHER, s);
  random_pairs_kernel<<<(int)grid, 256, 0, s>>>(seed, m, n, out);
  kt_end(s);
  MSM_LAUNCH("random_pairs_kernel");
  return MSM_OK;
}

int launch_gaussian(uint64_t seed, int64_t count, float* out, cudaStream_t s) {
  if (count <= 0) return MSM_OK;
  int64_t blocks = (count + 3) / 4;
  int grid = (int)((blocks + 255) / 256);
  int cap = num_sms() * 8;
  if (grid > cap) grid = cap;
  kt_begin(KC_OTHER, s);
  gaussian_kernel<<<grid, 256, 0, s>>>(seed, count, out);
  kt_end(s);
  MSM_LAUNCH("gaussian_kernel");
  return MSM_OK;
}

}  // namespace msm

// Distance decision of the epsilon recheck (Sec. 4.1, last step; Def. 1.1,
// Eq. 2), shared by the stand-alone recheck kernel and the pair check's
// fused count/recheck path.
//
// Fast path (float): S = sum_c (x_ic - x_jc)^2, each lane of a 4-lane group
// summing its share of coordinates, then a 2-level shuffle tree.  Rows of at
// most 256 coordinates: each lane keeps four independent fma chains (at most
// m = 16 terms each), so with u = 2^-24 a term carries the difference's
// rounding (2u in its square), its chain's m roundings, two to combine the
// chains and two in the tree: |S' - S| <= (m + 8) u S (sq_dist_rel).  Longer
// rows: compensated (Kahan) summation per lane, |S' - S| <= 10u S.
//   Euclidean: Delta = sqrt(S).
//   Cosine (Eq. 2): from |x_i - x_j|^2 = |x_i|^2 + |x_j|^2 - 2 x_i.x_j,
//     Delta = (S - (|x_i| - |x_j|)^2) / (2 |x_i| |x_j|), norms in double;
//     used only when (|x_i| - |x_j|)^2 <= S / 2, so the subtraction at most
//     doubles the relative error.
// A comparison whose float-path distance lies within its error bound (plus
// the rounding error of the double-precision reference) of eps is decided
// again on the double-precision distance evaluated exactly as Eq. 2 (or the
// Euclidean norm) with sequential fma over the coordinates.
#pragma once

#include <cuda_bf16.h>

#include "msm_internal.cuh"

namespace msm {
namespace dist {

constexpr double kU = 0x1.0p-24;

__device__ __forceinline__ float ldx(const void* X, int dtype, int64_t idx) {
  if (dtype == MSM_DT_BF16)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[idx]);
  return reinterpret_cast<const float*>(X)[idx];
}

// Distance in double precision, same operation order as the definition:
// cosine 1 - dot / (sqrt(|x_i|^2) * sqrt(|x_j|^2)), Euclidean sqrt(sum t^2).
__device__ inline double exact_distance(const void* X, int dtype, int64_t i,
                                 int64_t j, int dim, int metric) {
  const int64_t bi = i * dim, bj = j * dim;
  if (metric == MSM_COSINE) {
    double dot = 0.0, ni = 0.0, nj = 0.0;
    for (int c = 0; c < dim; ++c)
      dot = fma((double)ldx(X, dtype, bi + c), (double)ldx(X, dtype, bj + c), dot);
    for (int c = 0; c < dim; ++c) {
      double v = (double)ldx(X, dtype, bi + c);
      ni = fma(v, v, ni);
    }
    for (int c = 0; c < dim; ++c) {
      double v = (double)ldx(X, dtype, bj + c);
      nj = fma(v, v, nj);
    }
    return 1.0 - dot / (sqrt(ni) * sqrt(nj));
  }
  double s = 0.0;
  for (int c = 0; c < dim; ++c) {
    double t = (double)ldx(X, dtype, bi + c) - (double)ldx(X, dtype, bj + c);
    s = fma(t, t, s);
  }
  return sqrt(s);
}

// Float-path decision from S' (relative error <= relS) and the float row
// norms (each within u of the true norm).  Everything here is float: the
// FP64 pipe of this GPU is narrow, and a per-pair double evaluation made the
// recheck FP64-bound.  Error of the cosine value (S' - T') / (2 n_i n_j):
//   S' contributes <= 2 relS (S - T) because T <= S/2 is required;
//   T' = (n_i' - n_j')^2 is off by <= 4 u |n_i' - n_j'| (n_i + n_j)
//        + 8 u^2 (n_i + n_j)^2 + 2 u T' (rounded norms, square);
//   the subtraction, product and division add <= 5 u more.
// The double-precision reference itself is within (dim + 8) 2^-51 of the
// true value.  Returns false when the float path cannot settle the
// comparison (too close to eps) or cannot guarantee 4e-6 relative accuracy
// of the reported distance (need_accuracy); the caller then evaluates the
// distance by its definition in double precision.
__device__ __forceinline__ bool decide_fast(float S, float ni, float nj,
                                            int metric, int dim, float eps,
                                            float relS, bool need_accuracy,
                                            float* delta_out, bool* keep) {
  const float u = 0x1.0p-24f;
  float delta, rel, abs_err;
  if (metric == MSM_COSINE) {
    const float dn = ni - nj;
    const float T = dn * dn;
    if (T > 0.5f * S) return false;
    const float num = S - T;
    if (!(num > 0.f)) return false;
    const float sn = ni + nj;
    const float errT = 4.f * u * fabsf(dn) * sn + 8.f * u * u * sn * sn + 2.f * u * T;
    delta = num / (2.f * ni * nj);
    // S' is off by relS S <= 2 relS num (T <= S / 2); the factor 1.25 covers
    // the rounding of S / num and second-order terms
    rel = 1.25f * relS * (S / num) + 8.f * u + errT / num;
    abs_err = (float)(dim + 8) * 0x1.0p-51f;
  } else {
    delta = sqrtf(S);
    rel = 0.5f * relS + 2.f * u + (float)(dim + 4) * 0x1.0p-52f;
    abs_err = 0.f;
  }
  if (need_accuracy && rel > 4e-6f) return false;
  const float margin = rel * delta + abs_err + 1e-30f;
  if (fabsf(delta - eps) <= margin) return false;
  *delta_out = delta;
  *keep = delta <= eps;
  return true;
}

// Decision for one pair: float path, else the double-precision definition.
__device__ __forceinline__ double decide(const void* X, int dtype, int64_t i,
                                         int64_t j, int dim, int metric,
                                         float eps, float S, float ni, float nj,
                                         float relS, bool need_accuracy,
                                         bool* keep, bool* exact) {
  float d32;
  if (decide_fast(S, ni, nj, metric, dim, eps, relS, need_accuracy, &d32, keep)) {
    *exact = false;
    return (double)d32;
  }
  const double delta = exact_distance(X, dtype, i, j, dim, metric);
  *exact = true;
  *keep = delta <= (double)eps;
  return delta;
}

// Coordinates up to which group_sq_dist sums with plain fma chains.
constexpr int kChainDim = 256;

// Relative error bound of group_sq_dist<G, CHAINS>'s S' for rows of dim
// coordinates (G <= 4: at most two tree levels).
__host__ __device__ inline float sq_dist_rel(int dim, int G, bool chains = true) {
  if (chains && dim <= kChainDim) {
    const int per_chain = ((dim + G - 1) / G + 3) / 4;
    return (float)(per_chain + 8) * 0x1.0p-24f;
  }
  return 10.f * 0x1.0p-24f;
}

// Compensated (Kahan) addition of v to acc; comp carries the lost low part.
__device__ __forceinline__ void kahan_add(float v, float& acc, float& comp) {
  const float y = v - comp;
  const float s = acc + y;
  comp = (s - acc) - y;
  acc = s;
}

__device__ __forceinline__ void sq_diff_bf16x2(uint32_t a, uint32_t b, float& acc, float& comp) {
  // two bf16 values per word: a bf16 is the high half of a float
  const float t0 = __uint_as_float(a << 16) - __uint_as_float(b << 16);
  const float t1 = __uint_as_float(a & 0xffff0000u) - __uint_as_float(b & 0xffff0000u);
  kahan_add(__fmul_rn(t0, t0), acc, comp);
  kahan_add(__fmul_rn(t1, t1), acc, comp);
}

// group_sq_dist for rows of at most kChainDim coordinates: four independent
// fma chains per lane, combined pairwise, then the shuffle tree.
template <int G>
__device__ __forceinline__ float group_sq_dist_chains(const void* X, int dtype, int64_t i,
                                                      int64_t j, int dim, int sl) {
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
  const int64_t bi = i * dim, bj = j * dim;
  const bool al16 = (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
  if (dtype == MSM_DT_BF16 && (dim & 7) == 0 && al16) {
    const uint4* xi = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(X) + bi);
    const uint4* xj = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(X) + bj);
    const int n8 = dim / 8;
    for (int b0 = sl; b0 < n8; b0 += 4 * G) {
      uint4 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c8 = b0 + u * G;
        a[u] = c8 < n8 ? __ldg(xi + c8) : make_uint4(0u, 0u, 0u, 0u);
        b[u] = c8 < n8 ? __ldg(xj + c8) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t wa[4] = {a[u].x, a[u].y, a[u].z, a[u].w};
        const uint32_t wb[4] = {b[u].x, b[u].y, b[u].z, b[u].w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {  // a bf16 is the high half of a float
          const float t0 = __uint_as_float(wa[w] << 16) - __uint_as_float(wb[w] << 16);
          const float t1 = __uint_as_float(wa[w] & 0xffff0000u) -
                           __uint_as_float(wb[w] & 0xffff0000u);
          if (w & 1) {
            c2 = fmaf(t0, t0, c2);
            c3 = fmaf(t1, t1, c3);
          } else {
            c0 = fmaf(t0, t0, c0);
            c1 = fmaf(t1, t1, c1);
          }
        }
      }
    }
  } else if (dtype == MSM_DT_F32 && (dim & 3) == 0 && al16) {
    const float4* xi = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(X) + bi);
    const float4* xj = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(X) + bj);
    const int n4 = dim / 4;
    for (int b0 = sl; b0 < n4; b0 += 4 * G) {
      float4 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c4 = b0 + u * G;
        a[u] = c4 < n4 ? __ldg(xi + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
        b[u] = c4 < n4 ? __ldg(xj + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float t0 = a[u].x - b[u].x, t1 = a[u].y - b[u].y;
        const float t2 = a[u].z - b[u].z, t3 = a[u].w - b[u].w;
        c0 = fmaf(t0, t0, c0);
        c1 = fmaf(t1, t1, c1);
        c2 = fmaf(t2, t2, c2);
        c3 = fmaf(t3, t3, c3);
      }
    }
  } else {
    int k = 0;
    for (int c = sl; c < dim; c += G, ++k) {
      const float t = ldx(X, dtype, bi + c) - ldx(X, dtype, bj + c);
      switch (k & 3) {
        case 0: c0 = fmaf(t, t, c0); break;
        case 1: c1 = fmaf(t, t, c1); break;
        case 2: c2 = fmaf(t, t, c2); break;
        default: c3 = fmaf(t, t, c3); break;
      }
    }
  }
  float acc = (c0 + c1) + (c2 + c3);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// Sum of squared differences of rows i and j by the G lanes of a group.
// Each lane first issues 4 16-byte loads per row (float4, or 8 bf16 values),
// then adds, so 8 independent loads per lane are in flight (the kernel is
// bound by gather latency).  Rows that are not 16-byte aligned are read one
// element at a time.  With CHAINS, up to kChainDim coordinates, four fma
// chains per lane (two operations per coordinate, and independent chains);
// otherwise the compensated sum (five), whose bound does not grow with the
// row and which holds fewer registers (the pair check's fused recheck).
template <int G, bool CHAINS = true>
__device__ __forceinline__ float group_sq_dist(const void* X, int dtype,
                                               int64_t i, int64_t j, int dim,
                                               int sl) {
  if (CHAINS && dim <= kChainDim) return group_sq_dist_chains<G>(X, dtype, i, j, dim, sl);
  float acc = 0.f, comp = 0.f;
  const int64_t bi = i * dim, bj = j * dim;
  const bool al16 = (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
  if (dtype == MSM_DT_BF16 && (dim & 7) == 0 && al16) {
    const uint4* xi = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(X) + bi);
    const uint4* xj = reinterpret_cast<const uint4*>(reinterpret_cast<const __nv_bfloat16*>(X) + bj);
    const int n8 = dim / 8;
    for (int c0 = sl; c0 < n8; c0 += 4 * G) {
      uint4 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c8 = c0 + u * G;
        a[u] = c8 < n8 ? __ldg(xi + c8) : make_uint4(0u, 0u, 0u, 0u);
        b[u] = c8 < n8 ? __ldg(xj + c8) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sq_diff_bf16x2(a[u].x, b[u].x, acc, comp);
        sq_diff_bf16x2(a[u].y, b[u].y, acc, comp);
        sq_diff_bf16x2(a[u].z, b[u].z, acc, comp);
        sq_diff_bf16x2(a[u].w, b[u].w, acc, comp);
      }
    }
  } else if (dtype == MSM_DT_F32 && (dim & 3) == 0 && al16) {
    const float4* xi = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(X) + bi);
    const float4* xj = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(X) + bj);
    const int n4 = dim / 4;
    for (int c0 = sl; c0 < n4; c0 += 4 * G) {
      float4 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c4 = c0 + u * G;
        a[u] = c4 < n4 ? __ldg(xi + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
        b[u] = c4 < n4 ? __ldg(xj + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float t0 = a[u].x - b[u].x, t1 = a[u].y - b[u].y;
        const float t2 = a[u].z - b[u].z, t3 = a[u].w - b[u].w;
        kahan_add(__fmul_rn(t0, t0), acc, comp);
        kahan_add(__fmul_rn(t1, t1), acc, comp);
        kahan_add(__fmul_rn(t2, t2), acc, comp);
        kahan_add(__fmul_rn(t3, t3), acc, comp);
      }
    }
  } else {
    for (int c = sl; c < dim; c += G) {
      const float t = ldx(X, dtype, bi + c) - ldx(X, dtype, bj + c);
      kahan_add(__fmul_rn(t, t), acc, comp);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

}  // namespace dist
}  // namespace msm

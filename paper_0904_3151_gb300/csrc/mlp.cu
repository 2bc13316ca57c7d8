// Learned projection (the paper's Sec. 6 suggestion of non-random hashing):
// a two-layer network y = W2 gelu(W1 x + b1) + b2 replaces x as the input of
// the sign projection (Eq. 3); the exact recheck still uses x.  Training
// pulls epsilon-neighbour pairs together and pushes other pairs apart:
//   loss = mean over pairs of max(0, m_pos - cos(y_i, y_j))  (neighbours)
//                            max(0, cos(y_i, y_j) - m_neg)  (others).
// Weights are bf16 (float master copies for the optimiser), every product
// accumulates in float.  Kernels: a 64x64 register-tiled GEMM with
// transposition flags and a bias / gelu epilogue, the pair loss with its
// gradient, column sums, and an Adam step that refreshes the bf16 copies.
#include <cuda_bf16.h>

#include "msm_internal.cuh"

namespace msm {
namespace {

constexpr int GT = 64, GK = 16;

template <typename T>
__device__ __forceinline__ float tof(T v);
template <>
__device__ __forceinline__ float tof<float>(float v) { return v; }
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float gelu(float h) {
  return 0.5f * h * (1.f + erff(h * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float h) {
  const float cdf = 0.5f * (1.f + erff(h * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * h * h);
  return cdf + h * pdf;
}

// C[M][N] = op(A) op(B) (+ bias[n]); op(A) is A [M][K] or, with TA_T, A
// stored [K][M]; op(B) is B [K][N] or, with TB_T, B stored [N][K].  With
// C2 != NULL, C2 = gelu(C) as well.  Rows of A may be gathered through
// rowmap (A row m = A[rowmap[m]]), for the training batch.
template <typename TA, typename TB, bool TA_T, bool TB_T>
__global__ void __launch_bounds__(256)
gemm_kernel(const TA* A, const TB* B, float* C, float* C2, const float* bias,
            int M, int N, int K, const uint32_t* rowmap) {
  __shared__ __align__(16) float As[GK][GT + 4];
  __shared__ __align__(16) float Bs[GK][GT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int t = tid + 256 * e;  // 0..1023 over the 64 x 16 tile
      if (!TA_T) {
        const int m = t / GK, k = t % GK;
        const int gm = m0 + m, gk = k0 + k;
        float v = 0.f;
        if (gm < M && gk < K) {
          const int64_t row = rowmap ? (int64_t)rowmap[gm] : (int64_t)gm;
          v = tof<TA>(A[row * K + gk]);
        }
        As[k][m] = v;
      } else {
        const int k = t / GT, m = t % GT;
        const int gm = m0 + m, gk = k0 + k;
        As[k][m] = (gm < M && gk < K) ? tof<TA>(A[(int64_t)gk * M + gm]) : 0.f;
      }
      if (!TB_T) {
        const int k = t / GT, n = t % GT;
        const int gn = n0 + n, gk = k0 + k;
        Bs[k][n] = (gn < N && gk < K) ? tof<TB>(B[(int64_t)gk * N + gn]) : 0.f;
      } else {
        const int n = t / GK, k = t % GK;
        const int gn = n0 + n, gk = k0 + k;
        Bs[k][n] = (gn < N && gk < K) ? tof<TB>(B[(int64_t)gn * K + gk]) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = n0 + tx * 4 + j;
      if (nn >= N) continue;
      const float v = acc[i][j] + (bias ? bias[nn] : 0.f);
      C[(int64_t)m * N + nn] = v;
      if (C2) C2[(int64_t)m * N + nn] = gelu(v);
    }
  }
}

template <typename TA, typename TB, bool TA_T, bool TB_T>
int gemm(const TA* A, const TB* B, float* C, float* C2, const float* bias, int M,
         int N, int K, const uint32_t* rowmap, cudaStream_t s) {
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  if (grid.y > 65535) return set_error("GEMM too tall"), MSM_E_INVAL;
  kt_begin(KC_OTHER, s);
  gemm_kernel<TA, TB, TA_T, TB_T><<<grid, 256, 0, s>>>(A, B, C, C2, bias, M, N, K, rowmap);
  kt_end(s);
  MSM_LAUNCH("gemm_kernel");
  return MSM_OK;
}

// One warp per pair: cos of rows a and b of Y (rows 0..B-1 are the first
// points of the pairs, B..2B-1 the second), the hinge loss, and dL/dY rows.
__global__ void pair_loss_kernel(const float* Y, int B, int dy, const uint8_t* label,
                                 float m_pos, float m_neg, float* dY, float* loss_sum) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float lsum = 0.f;
  for (int64_t p = warp; p < B; p += nwarps) {
    const float* ya = Y + p * dy;
    const float* yb = Y + (p + B) * dy;
    float dot = 0.f, na = 0.f, nb = 0.f;
    for (int c = lane; c < dy; c += 32) {
      dot = fmaf(ya[c], yb[c], dot);
      na = fmaf(ya[c], ya[c], na);
      nb = fmaf(yb[c], yb[c], nb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dot += __shfl_xor_sync(0xffffffffu, dot, o);
      na += __shfl_xor_sync(0xffffffffu, na, o);
      nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    const float sa = sqrtf(na), sb = sqrtf(nb);
    const float cs = dot / (sa * sb);
    const bool pos = label[p] != 0;
    const float viol = pos ? (m_pos - cs) : (cs - m_neg);
    const float dcos = viol > 0.f ? (pos ? -1.f : 1.f) / (float)B : 0.f;
    if (lane == 0 && viol > 0.f) lsum += viol;
    for (int c = lane; c < dy; c += 32) {
      dY[p * dy + c] = dcos * (yb[c] / (sa * sb) - cs * ya[c] / (sa * sa));
      dY[(p + B) * dy + c] = dcos * (ya[c] / (sa * sb) - cs * yb[c] / (sb * sb));
    }
  }
  if (lane == 0 && lsum != 0.f) atomicAdd(loss_sum, lsum / (float)B);
}

// dH = dA * gelu'(H), elementwise
__global__ void gelu_back_kernel(const float* H, float* dA, int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    dA[t] *= gelu_grad(H[t]);
}

// out[c] = sum over rows of M[r][c] (one thread per column, sequential)
__global__ void colsum_kernel(const float* Mx, int rows, int cols, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += Mx[(int64_t)r * cols + c];
  out[c] = s;
}

// Adam (Kingma & Ba 2015) on the float master parameters; then the bf16
// copies of the two weight matrices are refreshed.
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, int64_t count,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* src, __nv_bfloat16* dst, int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = __float2bfloat16_rn(src[t]);
}

// Xb[r][c] = X[rows[r]][c] as float
__global__ void gather_rows_kernel(const void* X, int dtype, int dim, const uint32_t* rows,
                                   int64_t P, float* Xb) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < P * dim;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / dim, c = t % dim;
    const int64_t src = (int64_t)rows[r] * dim + c;
    Xb[t] = dtype == MSM_DT_BF16
                ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[src])
                : reinterpret_cast<const float*>(X)[src];
  }
}

int grid_for(int64_t count) {
  int64_t g = (count + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

// Forward pass in row chunks; Hbuf holds chunk rows x hidden floats.
template <typename TX>
static int mlp_forward_impl(const TX* X, int64_t n, int dim, const __nv_bfloat16* W1,
                            const float* b1, const __nv_bfloat16* W2, const float* b2,
                            int hidden, int dim_out, float* Y, float* Hbuf, float* Abuf,
                            int64_t chunk, const uint32_t* rowmap, cudaStream_t s) {
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int rows = (int)((n - r0) < chunk ? (n - r0) : chunk);
    const TX* Xc = rowmap ? X : X + r0 * dim;
    const uint32_t* rm = rowmap ? rowmap + r0 : nullptr;
    int rc = gemm<TX, __nv_bfloat16, false, true>(Xc, W1, Hbuf, Abuf, b1, rows, hidden, dim, rm, s);
    if (rc) return rc;
    rc = gemm<float, __nv_bfloat16, false, true>(Abuf, W2, Y + r0 * dim_out, nullptr, b2, rows,
                                                 dim_out, hidden, nullptr, s);
    if (rc) return rc;
  }
  return MSM_OK;
}

int mlp_forward(const void* X, int dtype, int64_t n, int dim, const void* W1,
                const float* b1, const void* W2, const float* b2, int hidden,
                int dim_out, float* Y, float* Hbuf, float* Abuf, int64_t chunk,
                const uint32_t* rowmap, cudaStream_t s) {
  const __nv_bfloat16* w1 = (const __nv_bfloat16*)W1;
  const __nv_bfloat16* w2 = (const __nv_bfloat16*)W2;
  if (dtype == MSM_DT_BF16)
    return mlp_forward_impl((const __nv_bfloat16*)X, n, dim, w1, b1, w2, b2, hidden, dim_out, Y,
                            Hbuf, Abuf, chunk, rowmap, s);
  return mlp_forward_impl((const float*)X, n, dim, w1, b1, w2, b2, hidden, dim_out, Y, Hbuf,
                          Abuf, chunk, rowmap, s);
}

// Loss and gradients for one batch of B pairs.  ws must hold
// 2B * (2 hidden + 2 dim_out) floats + 2B indices + 1 float.
int mlp_grad(const void* X, int dtype, int64_t n, int dim, const void* W1,
             const float* b1, const void* W2, const float* b2, int hidden, int dim_out,
             const uint32_t* pi, const uint32_t* pj, const uint8_t* label, int64_t B,
             float m_pos, float m_neg, float* grads, float* loss_dev, void* ws,
             cudaStream_t s) {
  (void)n;
  const int64_t P = 2 * B;
  float* H = (float*)ws;
  float* A = H + P * hidden;
  float* Y = A + P * hidden;
  float* dY = Y + P * dim_out;
  uint32_t* rows = (uint32_t*)(dY + P * dim_out);
  MSM_CUDA(cudaMemcpyAsync(rows, pi, 4 * (size_t)B, cudaMemcpyDeviceToDevice, s));
  MSM_CUDA(cudaMemcpyAsync(rows + B, pj, 4 * (size_t)B, cudaMemcpyDeviceToDevice, s));
  MSM_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(float), s));
  int rc = mlp_forward(X, dtype, P, dim, W1, b1, W2, b2, hidden, dim_out, Y, H, A, P, rows, s);
  if (rc) return rc;
  kt_begin(KC_OTHER, s);
  pair_loss_kernel<<<grid_for(P * 32), 256, 0, s>>>(Y, (int)B, dim_out, label, m_pos, m_neg, dY,
                                                    loss_dev);
  kt_end(s);
  MSM_LAUNCH("pair_loss_kernel");
  float* gW1 = grads;
  float* gb1 = gW1 + (int64_t)hidden * dim;
  float* gW2 = gb1 + hidden;
  float* gb2 = gW2 + (int64_t)dim_out * hidden;
  // dW2 = dY^T A  (dim_out x hidden), db2 = column sums of dY
  rc = gemm<float, float, true, false>(dY, A, gW2, nullptr, nullptr, dim_out, hidden, (int)P,
                                       nullptr, s);
  if (rc) return rc;
  colsum_kernel<<<(dim_out + 255) / 256, 256, 0, s>>>(dY, (int)P, dim_out, gb2);
  MSM_LAUNCH("colsum_kernel");
  // dA = dY W2 (P x hidden), written over A's buffer is not allowed (A is
  // consumed above), so into H's companion: reuse A after dW2 is done
  rc = gemm<float, __nv_bfloat16, false, false>(dY, (const __nv_bfloat16*)W2, A, nullptr,
                                                nullptr, (int)P, hidden, dim_out, nullptr, s);
  if (rc) return rc;
  gelu_back_kernel<<<grid_for(P * hidden), 256, 0, s>>>(H, A, P * hidden);
  MSM_LAUNCH("gelu_back_kernel");
  // db1 = column sums of dH; dW1 = dH^T X_batch (hidden x dim), with the
  // batch rows of X gathered (as float) into H's buffer, free by now
  colsum_kernel<<<(hidden + 255) / 256, 256, 0, s>>>(A, (int)P, hidden, gb1);
  MSM_LAUNCH("colsum_kernel");
  float* Xb = H;
  gather_rows_kernel<<<grid_for(P * dim), 256, 0, s>>>(X, dtype, dim, rows, P, Xb);
  MSM_LAUNCH("gather_rows_kernel");
  return gemm<float, float, true, false>(A, Xb, gW1, nullptr, nullptr, hidden, dim, (int)P,
                                         nullptr, s);
}

// Adam step on the float master parameters [W1 | b1 | W2 | b2] and
// refresh of the bf16 weight copies [W1 | W2].
int mlp_adam(float* params, const float* grads, float* m, float* v, int64_t count,
             int step, float lr, float beta1, float beta2, float eps, void* w1h, void* w2h,
             int hidden, int dim, int dim_out, cudaStream_t s) {
  const float c1 = 1.f - powf(beta1, (float)step);
  const float c2 = 1.f - powf(beta2, (float)step);
  kt_begin(KC_OTHER, s);
  adam_kernel<<<grid_for(count), 256, 0, s>>>(params, grads, m, v, count, lr, beta1, beta2,
                                              eps, c1, c2);
  kt_end(s);
  MSM_LAUNCH("adam_kernel");
  const int64_t n1 = (int64_t)hidden * dim, n2 = (int64_t)dim_out * hidden;
  to_bf16_kernel<<<grid_for(n1), 256, 0, s>>>(params, (__nv_bfloat16*)w1h, n1);
  MSM_LAUNCH("to_bf16_kernel");
  to_bf16_kernel<<<grid_for(n2), 256, 0, s>>>(params + n1 + hidden, (__nv_bfloat16*)w2h, n2);
  MSM_LAUNCH("to_bf16_kernel");
  return MSM_OK;
}

}  // namespace msm

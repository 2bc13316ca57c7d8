// The learned projection's feature map y = W2 gelu(W1 x + b1) + b2 (the
// paper's Sec. 6 suggestion of non-random hashing) on the tcgen05 tensor
// cores, both layers fused per block of 128 rows:
//   layer 1: H_c = X W1_c^T for hidden chunks c of 64 units, into one of two
//            TMEM accumulators (TMA-fed X and W1 tiles, 128-byte swizzle);
//   epilogue: a = gelu(H_c + b1) (exact erf form), split into bf16 parts
//            a_h = bf16(a), a_l = bf16(a - a_h), written by the epilogue
//            warps into a shared-memory tile in the K-major swizzled layout
//            the MMA reads;
//   layer 2: Y += a_h W2_c^T + a_l W2_c^T into a third TMEM accumulator,
//            issued one chunk behind layer 1 so the epilogue of chunk c
//            overlaps the MMAs of chunk c + 1;
//   output:  y = Y + b2 as float.
// Float X is split the same way (X = X_h + X_l, two layer-1 products); bf16
// X and the bf16 weights are exact.  Every product accumulates in float.
// Compared with the float CUDA-core path the operands carry 16 instead of 24
// significant bits (the low parts' rounding, at most 2^-16 relative), which
// the forward test's error bound covers.
//
// Warps: 0-7 epilogue (warp w owns rows 32 (w % 4) .. and the half w / 4 of
// each chunk's columns), 8 the TMA producer, 9 the MMA issuer.  Every wait is
// bounded (poll limit and 2 s of %globaltimer); a thread that gives up raises
// a CTA flag and the status word, the others stop at their next wait, and the
// producer and MMA threads wait (bounded, ignoring the flag) for the copies
// and MMAs they issued before the CTA releases shared memory and TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include "msm_internal.cuh"
#include "readback.cuh"
#include "tcgen05.cuh"

namespace msm {
namespace {

using namespace tc;

constexpr int kM = 128;          // rows per CTA (M of both MMAs)
constexpr int kHC = 64;          // hidden units per chunk (N of layer 1, K of layer 2)
constexpr int kEpi = 8;          // epilogue warps
constexpr int kThreadsMlp = (kEpi + 2) * 32;
constexpr int kXBoxM = kM * kChunkBytes;    // 128 rows x 128 B of X (16 KB)
constexpr int kWBox = kHC * kChunkBytes;    // 64 rows x 128 B of W1 (8 KB)
constexpr int kATile = kM * kChunkBytes;    // 128 rows x 64 bf16 of a part of a (16 KB)
constexpr uint32_t kDrain = 1u << 24;
constexpr int kBars = 1 + 2 * 9 + 1;        // barX, 9 pairs, yfull

struct MlpArgs {
  int64_t n;
  int dim, hidden, dim_out;
  int xch;               // K chunks of 128 B of X (2 dim / 128)
  uint32_t idesc1;       // M = 128, N = 64
  uint32_t idesc2;       // M = 128, N = dim_out
  uint32_t polls;
  const float* b1;
  const float* b2;
  float* Y;              // [n][dim_out]
  unsigned* status;      // bit 0: a bounded wait gave up
};

__device__ __forceinline__ float gelu_exact(float h) {
  return 0.5f * h * (1.f + erff(h * 0.70710678118654752f));
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Barrier pairs (one per double-buffered resource, index s = chunk & 1).
enum { B_W1F = 0, B_W1E, B_W2F, B_W2E, B_HF, B_HE, B_AF, B_AE, B_PAIRS };

__device__ __forceinline__ uint64_t* barp(uint64_t* bars, int kind, int s) {
  return bars + 1 + 2 * kind + s;
}

__device__ __forceinline__ uint32_t pack_bf16(float x0, float x1) {
  const __nv_bfloat16 a = __float2bfloat16_rn(x0), b = __float2bfloat16_rn(x1);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Epilogue warp: rows 32 (warp % 4) + lane of the tile, columns
// 32 (warp / 4) .. of every hidden chunk and dim_out / 2 (warp / 4) .. of y.
__device__ __forceinline__ void mlp_epilogue(const MlpArgs& a, uint32_t tmem, uint8_t* sA,
                                             uint64_t* bars, uint64_t* yfull, uint32_t* abortf,
                                             int64_t row0, int warp, int lane) {
  const int quarter = warp & 3, half = warp >> 2;
  const int r = quarter * 32 + lane;  // row within the tile
  const int64_t row = row0 + r;
  const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
  const int nch = a.hidden / kHC;
  // byte offset of this row in a 128-byte swizzled K-major tile: 8-row atoms
  // of 1024 B; the 16-byte chunk q of row r sits at chunk q ^ (r mod 8)
  const uint32_t rowoff = (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u;
  bool ok = true;
  for (int c = 0; c < nch; ++c) {
    const int s = c & 1;
    const uint32_t par = (uint32_t)((c >> 1) & 1);
    ok = __all_sync(0xffffffffu, mbar_wait(barp(bars, B_HF, s), par, a.polls, abortf));
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t v[32];
    tmem_ld32(tl + (uint32_t)(s * kHC + half * 32), v);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(barp(bars, B_HE, s));
    const float* b1 = a.b1 + c * kHC + half * 32;
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const float g0 = gelu_exact(__uint_as_float(v[j]) + b1[j]);
      const float g1 = gelu_exact(__uint_as_float(v[j + 1]) + b1[j + 1]);
      const float h0 = __bfloat162float(__float2bfloat16_rn(g0));
      const float h1 = __bfloat162float(__float2bfloat16_rn(g1));
      hi[j / 2] = pack_bf16(h0, h1);
      lo[j / 2] = pack_bf16(g0 - h0, g1 - h1);
    }
    if (c >= 2) {  // layer 2 of chunk c - 2 is done with this buffer
      ok = __all_sync(0xffffffffu, mbar_wait(barp(bars, B_AE, s), par ^ 1u, a.polls, abortf));
      if (!ok) break;
    }
    uint8_t* th = sA + (2 * s) * kATile;
    uint8_t* tlo = th + kATile;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const uint32_t q = (uint32_t)(4 * half + m);
      const uint32_t pos = rowoff + ((q ^ (uint32_t)(r & 7)) * 16u);
      *reinterpret_cast<uint4*>(th + pos) =
          make_uint4(hi[4 * m], hi[4 * m + 1], hi[4 * m + 2], hi[4 * m + 3]);
      *reinterpret_cast<uint4*>(tlo + pos) =
          make_uint4(lo[4 * m], lo[4 * m + 1], lo[4 * m + 2], lo[4 * m + 3]);
    }
    fence_async_smem();  // generic-proxy writes become visible to the MMA
    __syncwarp();
    if (lane == 0) mbar_arrive(barp(bars, B_AF, s));
  }
  if (ok) ok = __all_sync(0xffffffffu, mbar_wait(yfull, 0, a.polls, abortf));
  if (!ok) {
    if (lane == 0) {
      atomicOr(a.status, 1u);
      *(volatile uint32_t*)abortf = 1u;
    }
    return;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int ycols = a.dim_out / 2;
  for (int c0 = 0; c0 < ycols; c0 += 32) {
    uint32_t v[32];
    tmem_ld32(tl + 128u + (uint32_t)(half * ycols + c0), v);
    if (row < a.n) {
      const int col = half * ycols + c0;
      float4* dst = reinterpret_cast<float4*>(a.Y + row * a.dim_out + col);
#pragma unroll
      for (int j = 0; j < 32; j += 4)
        dst[j / 4] = make_float4(__uint_as_float(v[j]) + a.b2[col + j],
                                 __uint_as_float(v[j + 1]) + a.b2[col + j + 1],
                                 __uint_as_float(v[j + 2]) + a.b2[col + j + 2],
                                 __uint_as_float(v[j + 3]) + a.b2[col + j + 3]);
    }
  }
}

template <bool XLO>
__global__ void __launch_bounds__(kThreadsMlp, 1)
mlp_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmXl,
              const __grid_constant__ CUtensorMap tmW1, const __grid_constant__ CUtensorMap tmW2,
              MlpArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int xbytes = a.xch * kXBoxM;
  const int w1bytes = a.xch * kWBox;
  const int w2bytes = a.dim_out * kChunkBytes;
  uint8_t* sX = base;
  uint8_t* sXl = base + xbytes;
  uint8_t* sW1 = base + (XLO ? 2 : 1) * xbytes;   // 2 stages
  uint8_t* sW2 = sW1 + 2 * w1bytes;               // 2 stages
  uint8_t* sA = sW2 + 2 * w2bytes;                // 2 buffers x (high, low)
  uint64_t* bars = (uint64_t*)(sA + 4 * kATile);
  uint64_t* barX = bars;
  auto bar = [bars](int kind, int s) { return barp(bars, kind, s); };
  uint64_t* yfull = bars + 1 + 2 * B_PAIRS;
  uint32_t* tslot = (uint32_t*)(bars + kBars);
  uint32_t* abortf = tslot + 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kM;
  const int nch = a.hidden / kHC;
  if (tid == 0) {
    mbar_init(barX, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(bar(B_W1F, s), 1);
      mbar_init(bar(B_W1E, s), 1);
      mbar_init(bar(B_W2F, s), 1);
      mbar_init(bar(B_W2E, s), 1);
      mbar_init(bar(B_HF, s), 1);
      mbar_init(bar(B_HE, s), kEpi);
      mbar_init(bar(B_AF, s), kEpi);
      mbar_init(bar(B_AE, s), 1);
    }
    mbar_init(yfull, 1);
    *abortf = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tslot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;  // H buffers at columns 0 and 64, Y at 128
  const int ksteps = kChunkBytes / 32;

  if (warp == kEpi) {
    // TMA producer: X once; then W1 and W2 chunks into their two stages
    if (lane == 0) {
      int last1[2] = {-1, -1}, last2[2] = {-1, -1};
      mbar_expect_tx(barX, (uint32_t)((XLO ? 2 : 1) * xbytes));
      for (int c = 0; c < a.xch; ++c) {
        tma_load_2d(sX + c * kXBoxM, &tmX, barX, c * (kChunkBytes / 2), (int)row0);
        if (XLO) tma_load_2d(sXl + c * kXBoxM, &tmXl, barX, c * (kChunkBytes / 2), (int)row0);
      }
      bool ok = true;
      for (int c = 0; ok && c < nch; ++c) {
        const int s = c & 1;
        if (c >= 2) ok = mbar_wait(bar(B_W1E, s), (uint32_t)(((c - 2) >> 1) & 1), a.polls, abortf);
        if (!ok) break;
        mbar_expect_tx(bar(B_W1F, s), (uint32_t)w1bytes);
        for (int d = 0; d < a.xch; ++d)
          tma_load_2d(sW1 + s * w1bytes + d * kWBox, &tmW1, bar(B_W1F, s), d * (kChunkBytes / 2),
                      c * kHC);
        last1[s] = c;
        if (c >= 2) ok = mbar_wait(bar(B_W2E, s), (uint32_t)(((c - 2) >> 1) & 1), a.polls, abortf);
        if (!ok) break;
        mbar_expect_tx(bar(B_W2F, s), (uint32_t)w2bytes);
        tma_load_2d(sW2 + s * w2bytes, &tmW2, bar(B_W2F, s), c * kHC, 0);
        last2[s] = c;
      }
      if (!ok) {
        atomicOr(a.status, 1u);
        *(volatile uint32_t*)abortf = 1u;
      }
      mbar_wait(barX, 0, kDrain, nullptr);
      for (int s = 0; s < 2; ++s) {
        if (last1[s] >= 0) mbar_wait(bar(B_W1F, s), (uint32_t)((last1[s] >> 1) & 1), kDrain, nullptr);
        if (last2[s] >= 0) mbar_wait(bar(B_W2F, s), (uint32_t)((last2[s] >> 1) & 1), kDrain, nullptr);
      }
    }
  } else if (warp == kEpi + 1) {
    // MMA issuer: layer 1 of chunk c, then layer 2 of chunk c - 1
    if (lane == 0) {
      int lastc[B_PAIRS][2];  // last chunk committed to each barrier (-1: none)
      for (int k = 0; k < B_PAIRS; ++k) lastc[k][0] = lastc[k][1] = -1;
      bool ycommit = false;
      bool ok = mbar_wait(barX, 0, a.polls, abortf);
      uint32_t yacc = 0;
      auto layer2 = [&](int c) -> bool {
        const int s = c & 1;
        const uint32_t par = (uint32_t)((c >> 1) & 1);
        if (!mbar_wait(bar(B_AF, s), par, a.polls, abortf)) return false;
        if (!mbar_wait(bar(B_W2F, s), par, a.polls, abortf)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint8_t* ah = sA + (2 * s) * kATile;
        const uint8_t* al = ah + kATile;
        const uint8_t* w2 = sW2 + s * w2bytes;
        for (int ks = 0; ks < ksteps; ++ks) {
          const uint64_t bd = sw128_desc(saddr(w2) + ks * 32);
          mma<true>(tmem + 128u, sw128_desc(saddr(ah) + ks * 32), bd, a.idesc2, yacc);
          yacc = 1;
          mma<true>(tmem + 128u, sw128_desc(saddr(al) + ks * 32), bd, a.idesc2, 1);
        }
        mma_commit(bar(B_AE, s));
        mma_commit(bar(B_W2E, s));
        lastc[B_AE][s] = c;
        lastc[B_W2E][s] = c;
        return true;
      };
      for (int c = 0; ok && c < nch; ++c) {
        const int s = c & 1;
        const uint32_t par = (uint32_t)((c >> 1) & 1);
        ok = mbar_wait(bar(B_W1F, s), par, a.polls, abortf);
        if (ok && c >= 2) ok = mbar_wait(bar(B_HE, s), par ^ 1u, a.polls, abortf);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(s * kHC);
        const uint8_t* w1 = sW1 + s * w1bytes;
        uint32_t acc = 0;
        for (int xc = 0; xc < a.xch; ++xc)
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t bd = sw128_desc(saddr(w1 + xc * kWBox) + ks * 32);
            mma<true>(d, sw128_desc(saddr(sX + xc * kXBoxM) + ks * 32), bd, a.idesc1, acc);
            acc = 1;
            if (XLO) mma<true>(d, sw128_desc(saddr(sXl + xc * kXBoxM) + ks * 32), bd, a.idesc1, 1);
          }
        mma_commit(bar(B_HF, s));
        mma_commit(bar(B_W1E, s));
        lastc[B_HF][s] = c;
        lastc[B_W1E][s] = c;
        if (c >= 1) ok = layer2(c - 1);
      }
      if (ok) ok = layer2(nch - 1);
      if (ok) {
        mma_commit(yfull);
        ycommit = true;
      }
      if (!ok) {
        atomicOr(a.status, 1u);
        *(volatile uint32_t*)abortf = 1u;
      }
      // drain: every commit issued has arrived
      const int kinds[4] = {B_HF, B_W1E, B_AE, B_W2E};
      for (int k = 0; k < 4; ++k)
        for (int s = 0; s < 2; ++s)
          if (lastc[kinds[k]][s] >= 0)
            mbar_wait(bar(kinds[k], s), (uint32_t)((lastc[kinds[k]][s] >> 1) & 1), kDrain, nullptr);
      if (ycommit) mbar_wait(yfull, 0, kDrain, nullptr);
    }
  } else {
    mlp_epilogue(a, tmem, sA, bars, yfull, abortf, row0, warp, lane);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                 : "memory");
}

// Xh = bf16(x), Xl = bf16(x - Xh)
__global__ void mlp_split_kernel(const float* X, int64_t count, __nv_bfloat16* Xh,
                                 __nv_bfloat16* Xl) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float v = X[e];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Xh[e] = h;
    Xl[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

inline size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t mlp_smem(int dim, int dim_out, bool xlo) {
  const int xch = (2 * dim + kChunkBytes - 1) / kChunkBytes;
  return 1024 + (size_t)(xlo ? 2 : 1) * xch * kXBoxM + 2 * (size_t)xch * kWBox +
         2 * (size_t)dim_out * kChunkBytes + 4 * (size_t)kATile + 8 * kBars + 16;
}

}  // namespace

// Shapes the fused kernel takes: rows of X of at most 256 bytes as bf16
// (128 coordinates for float X, whose two parts must fit), a hidden width
// that is a multiple of 64, and 64 or 128 outputs.
bool mlp_tc_supported(int dtype, int dim, int hidden, int dim_out, uintptr_t xaddr) {
  if (dim < 8 || dim % 8 != 0 || hidden < kHC || hidden % kHC != 0) return false;
  if (dim_out != 64 && dim_out != 128) return false;
  if (dtype == MSM_DT_BF16 ? (dim > 128 || xaddr % 16 != 0) : dim > 128) return false;
  return mlp_smem(dim, dim_out, dtype != MSM_DT_BF16) <= 227 * 1024;
}

size_t mlp_tc_scratch_bytes(int64_t n, int dim, int dtype) {
  return (dtype == MSM_DT_BF16 ? 0 : 2 * up256(2 * (size_t)n * dim)) + 256;
}

int launch_mlp_tc(const void* X, int dtype, int64_t n, int dim, const void* W1,
                  const float* b1, const void* W2, const float* b2, int hidden, int dim_out,
                  float* Y, void* ws, cudaStream_t s) {
  const bool xlo = dtype != MSM_DT_BF16;
  char* p = (char*)ws;
  __nv_bfloat16* Xh = nullptr;
  __nv_bfloat16* Xl = nullptr;
  if (xlo) {
    Xh = (__nv_bfloat16*)p; p += up256(2 * (size_t)n * dim);
    Xl = (__nv_bfloat16*)p; p += up256(2 * (size_t)n * dim);
    int64_t grid = ((int64_t)n * dim + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (grid > cap) grid = cap;
    kt_begin(KC_OTHER, s);
    mlp_split_kernel<<<(int)grid, 256, 0, s>>>((const float*)X, (int64_t)n * dim, Xh, Xl);
    kt_end(s);
    MSM_LAUNCH("mlp_split_kernel");
  }
  unsigned* status = (unsigned*)p;
  MSM_CUDA(cudaMemsetAsync(status, 0, 4, s));
  CUtensorMap mX, mXl, mW1, mW2;
  int rc = make_map(&mX, xlo ? (const void*)Xh : X, dim, n, kM);
  if (!rc) rc = make_map(&mXl, xlo ? (const void*)Xl : X, dim, n, kM);
  if (!rc) rc = make_map(&mW1, W1, dim, hidden, kHC);
  if (!rc) rc = make_map(&mW2, W2, hidden, dim_out, dim_out);
  if (rc) return rc;
  MlpArgs a;
  a.n = n;
  a.dim = dim;
  a.hidden = hidden;
  a.dim_out = dim_out;
  a.xch = (2 * dim + kChunkBytes - 1) / kChunkBytes;
  // instruction descriptors: D f32, A/B BF16, both K-major, M = 128
  a.idesc1 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHC >> 3) << 17) |
             ((uint32_t)(kM >> 4) << 24);
  a.idesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(dim_out >> 3) << 17) |
             ((uint32_t)(kM >> 4) << 24);
  a.polls = wait_polls();
  a.b1 = b1;
  a.b2 = b2;
  a.Y = Y;
  a.status = status;
  const size_t smem = mlp_smem(dim, dim_out, xlo);
  auto kern = xlo ? mlp_tc_kernel<true> : mlp_tc_kernel<false>;
  MSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)((n + kM - 1) / kM);
  kt_begin(KC_OTHER, s);
  kern<<<grid, kThreadsMlp, smem, s>>>(mX, mXl, mW1, mW2, a);
  kt_end(s);
  MSM_LAUNCH("mlp_tc_kernel");
  unsigned st = 0;
  rc = read_to_host(&st, status, 4, s);
  if (rc) return rc;
  if (st & 1u) return set_error("tensor-core feature map: a bounded wait timed out"), MSM_E_TIMEOUT;
  return MSM_OK;
}

}  // namespace msm

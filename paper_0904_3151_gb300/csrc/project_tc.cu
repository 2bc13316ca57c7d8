// Step A1 on the 5th-generation tensor cores: t = X R_q for all replicates
// as one GEMM (n x D) * (D x Q*W*64), operands staged in shared memory by
// TMA (128-byte swizzle), accumulators in TMEM, and the sign / pack of
// Eq. 3 fused into the TMEM read-out.  Each CTA owns 128 rows and walks all
// column tiles of 128 columns; each epilogue thread owns one row, so a
// 64-column half of the tile becomes one packed word without shuffles.
//
// Exactness: operands are read as TF32 (X, R float: each operand within
// 2^-10 relative) or as BF16 (X stored bf16 exactly; R split into a bf16
// high part and a bf16 low part, two MMAs, so R is represented to 2^-16).
// The accumulated float value t' then satisfies
//   |t' - t| <= (e_op + 4 D 2^-24) |x| |r|,
// with e_op = 2^-9 (TF32) or 2^-16 (BF16 split); 4 D 2^-24 is four times the
// classical bound of the float accumulation.  Bits with |t'| within that
// margin are written as 0 and queued; project_fix_kernel recomputes each in
// float with its own bound and, if still undecided, in double precision by
// sequential fma (the definition of the bit), then sets it.
#include <cuda.h>
#include <cuda_bf16.h>

#include "msm_internal.cuh"

namespace msm {
namespace {

constexpr int kRows = 128;      // M of the MMA, rows per CTA
constexpr int kCols = 64;       // N of the MMA, columns per tile (one word)
constexpr int kChunkBytes = 128;  // K bytes per swizzle atom row
constexpr int kMaxChunks = 4;   // K chunks kept resident (D*esize <= 512 B)
constexpr int kTileBytes = kRows * kChunkBytes;  // one 128 x 128 B box of X
constexpr int kBTileBytes = kCols * kChunkBytes; // one 64 x 128 B box of R
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: gives up (returns false) after
// kWaitLimit polls, after 2 s of wall-clock time, or as soon as another CTA
// has reported a failure in *status.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          const unsigned* status) {
  const uint32_t a = saddr(bar);
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 255u) == 255u) {
      if (globaltimer_ns() - t0 > 2000000000ull) return false;
      if (status && *(volatile const unsigned*)status) return false;
    }
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map,
                                            uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzled
// layout written by TMA (8-row atoms of 1024 B stacked along M/N).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)1u << 16;                       // leading offset (unused)
  d |= (uint64_t)(1024u >> 4) << 32;             // stride offset: 1024 B
  d |= (uint64_t)1u << 46;                       // descriptor version
  d |= (uint64_t)2u << 61;                       // 128-byte swizzle
  return d;
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b,
                                    uint32_t idesc, uint32_t acc) {
  if constexpr (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
      "%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31},"
      " [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
        "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
  int64_t n;
  int dim;
  int ell, W, Q;
  int ctiles;          // column tiles of 128 over the padded Q*W*64 columns
  int chunks;          // K chunks of 128 B
  uint32_t idesc;
  float mscale, mabs;  // margin = mscale * |x| * |r| + mabs
  const float* xnorm;  // [n]
  const float* rnorm;  // [Q * W * 64] (padded columns have norm 0)
  uint64_t* strings;   // [Q][n][W]
  uint64_t* fix;       // queued (row << 32 | q * ell + c)
  int64_t fix_cap;
  unsigned long long* fix_count;
  unsigned* status;    // bit 0: a bounded wait gave up
};

// 128 threads: warp 0 also allocates TMEM; thread 0 issues TMA and MMA; all
// four warps read TMEM (warp w owns lanes 32w..32w+31 = rows).
template <bool BF16>
__global__ void __launch_bounds__(128, 2)
project_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                  const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ CUtensorMap tmB2, TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int kNB = BF16 ? 2 : 1;  // B operands (R high, R low)
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + a.chunks * kTileBytes;  // then kNB * chunks boxes of R
  uint64_t* bars = (uint64_t*)(sB + kNB * a.chunks * kBTileBytes);
  uint32_t* tslot = (uint32_t*)(bars + 4);
  uint64_t* barA = bars;
  uint64_t* barB = bars + 1;
  uint64_t* barM = bars + 2;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  if (tid == 0) {
    mbar_init(barA, 1);
    mbar_init(barB, 1);
    mbar_init(barM, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tslot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  bool failed = false;

  if (tid == 0) {
    mbar_expect_tx(barA, (uint32_t)(a.chunks * kTileBytes));
    for (int c = 0; c < a.chunks; ++c)
      tma_load_2d(sA + c * kTileBytes, &tmX, barA, c * (kChunkBytes / (BF16 ? 2 : 4)),
                  (int)row0);
  }
  const int64_t row = row0 + warp * 32 + lane;
  const float xn = row < a.n ? a.xnorm[row] : 0.f;
  const int colsPerRep = a.W * 64;
  const int ksteps = kChunkBytes / 32;  // MMA K is 32 bytes for both kinds

  for (int ct = 0; ct < a.ctiles && !failed; ++ct) {
    const uint32_t par = ct & 1;
    if (tid == 0) {
      mbar_expect_tx(barB, (uint32_t)(kNB * a.chunks * kBTileBytes));
      for (int c = 0; c < a.chunks; ++c) {
        const int kx = c * (kChunkBytes / (BF16 ? 2 : 4));
        tma_load_2d(sB + c * kBTileBytes, &tmB, barB, kx, ct * kCols);
        if (BF16)
          tma_load_2d(sB + (a.chunks + c) * kBTileBytes, &tmB2, barB, kx, ct * kCols);
      }
      bool ok = (ct > 0 || mbar_wait(barA, 0, a.status)) && mbar_wait(barB, par, a.status);
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t acc = 0;
        for (int c = 0; c < a.chunks; ++c)
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t ad = sw128_desc(saddr(sA + c * kTileBytes) + ks * 32);
            const uint64_t bd = sw128_desc(saddr(sB + c * kBTileBytes) + ks * 32);
            mma<BF16>(tmem, ad, bd, a.idesc, acc);
            acc = 1;
            if (BF16) {
              const uint64_t bd2 = sw128_desc(saddr(sB + (a.chunks + c) * kBTileBytes) + ks * 32);
              mma<BF16>(tmem, ad, bd2, a.idesc, 1);
            }
          }
        mma_commit(barM);
      } else {
        atomicOr(a.status, 1u);
      }
    }
    // Every thread waits for the accumulators (a failed issue never
    // commits, so this wait also runs out); the CTA agrees on the outcome
    // so that all threads leave the loop together.
    const bool ok = mbar_wait(barM, par, a.status);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(a.status, 1u);
      failed = true;
      // let this tile's copies land before the CTA's memory is released
      if (tid == 0) {
        mbar_wait(barB, par, nullptr);
        if (ct == 0) mbar_wait(barA, 0, nullptr);
      }
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
    const bool live_row = row < a.n;
    for (int half = 0; half < kCols / 64; ++half) {
      const int gcol0 = ct * kCols + half * 64;  // first column of this word
      const int q = gcol0 / colsPerRep;
      const int cw = gcol0 % colsPerRep;         // column of the word in R_q
      const bool live = live_row && q < a.Q;
      uint64_t word = 0;
      for (int part = 0; part < 2; ++part) {
        uint32_t r[32];
        tmem_ld32(tbase + half * 64 + part * 32, r);
        uint32_t flagged = 0;
        if (live) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int c = cw + part * 32 + j;
            if (c >= a.ell) continue;
            const float t = __uint_as_float(r[j]);
            const float m = a.mscale * xn * a.rnorm[q * colsPerRep + c] + a.mabs;
            if (fabsf(t) <= m) flagged |= 1u << j;
            else if (t > 0.f) word |= 1ull << (part * 32 + j);
          }
        }
        // queue the undecided bits: one atomic per warp
        uint32_t cnt = __popc(flagged), incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
          unsigned long long b0 = 0;
          if (lane == 31) b0 = atomicAdd(a.fix_count, (unsigned long long)total);
          b0 = __shfl_sync(0xffffffffu, b0, 31) + (incl - cnt);
          while (flagged) {
            const int j = __ffs(flagged) - 1;
            flagged &= flagged - 1;
            if ((int64_t)b0 < a.fix_cap)
              a.fix[b0] = ((uint64_t)row << 32) | (uint32_t)(q * a.ell + cw + part * 32 + j);
            ++b0;
          }
        }
      }
      if (live) a.strings[((size_t)q * a.n + row) * a.W + cw / 64] = word;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                 : "memory");
}

// Rt[q * W * 64 + c][k] = R[q][k][c] for c < ell, 0 otherwise; rows padded
// to a multiple of 128.  BF16: hi = bf16(R), lo = bf16(R - hi).
template <bool BF16>
__global__ void transpose_R_kernel(const float* R, int Q, int dim, int ell,
                                   int W, int64_t rows, void* hi, void* lo,
                                   float* rnorm) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int colsPerRep = W * 64;
    const int q = (int)(t / colsPerRep), c = (int)(t % colsPerRep);
    const bool live = q < Q && c < ell;
    double nrm = 0.0;
    for (int k = 0; k < dim; ++k) {
      const float v = live ? R[((size_t)q * dim + k) * ell + c] : 0.f;
      nrm = fma((double)v, (double)v, nrm);
      if constexpr (BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        reinterpret_cast<__nv_bfloat16*>(hi)[t * dim + k] = h;
        reinterpret_cast<__nv_bfloat16*>(lo)[t * dim + k] = l;
      } else {
        reinterpret_cast<float*>(hi)[t * dim + k] = v;
      }
    }
    if (t < (int64_t)Q * colsPerRep) rnorm[t] = (float)sqrt(nrm);
  }
}

__device__ __forceinline__ float ldx(const void* X, int dtype, int64_t i) {
  if (dtype == MSM_DT_BF16)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[i]);
  return reinterpret_cast<const float*>(X)[i];
}

// One warp per queued bit: float dot with its own bound, then the
// double-precision sequential-fma value when still undecided.
// Rt: optional transposed float copy of R (row q * W * 64 + c holds column c
// of R_q, contiguous over the coordinates); the values are R's, only the
// loads of a column become coalesced.
__global__ void project_fix_kernel(const void* X, int dtype, int64_t n, int dim,
                                   const float* R, const float* Rt, int ell, int W,
                                   const float* xnorm, const float* rnorm_pad,
                                   const uint64_t* fix,
                                   const unsigned long long* fix_count,
                                   int64_t fix_cap, uint64_t* strings,
                                   unsigned long long* recompute, unsigned* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t m = (int64_t)*fix_count;
  if (m > fix_cap) {
    // the queue overflowed: the strings are incomplete and the caller must
    // project again on the CUDA-core path (status bit 1)
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 2u);
    return;
  }
  const float m2 = (float)(2 * dim + 8) * 0x1.0p-24f;
  // four queued signs per warp, eight lanes each (more loads in flight)
  const int sub = lane & 7, grp = lane >> 3;
  for (int64_t base = warp * 4; base < m; base += nwarps * 4) {
    const int64_t it = base + grp;
    const bool valid = it < m;
    const uint64_t e = valid ? fix[it] : 0ull;
    const int64_t row = (int64_t)(e >> 32);
    const int qc = (int)(e & 0xffffffffu);
    const int q = qc / ell, c = qc % ell;
    const float* Rq = R + (size_t)q * dim * ell;
    const float* rc = Rt ? Rt + (size_t)(q * W * 64 + c) * dim : nullptr;
    float acc = 0.f;
    if (valid)
      for (int k = sub; k < dim; k += 8)
        acc = fmaf(ldx(X, dtype, row * dim + k), rc ? rc[k] : Rq[(size_t)k * ell + c], acc);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (valid && sub == 0) {
      bool bit;
      const float marg = m2 * xnorm[row] * rnorm_pad[q * W * 64 + c] + (float)dim * 0x1.0p-120f;
      if (fabsf(acc) <= marg) {
        double t = 0.0;
        for (int k = 0; k < dim; ++k)
          t = fma((double)ldx(X, dtype, row * dim + k),
                  (double)(rc ? rc[k] : Rq[(size_t)k * ell + c]), t);
        bit = t > 0.0;
        atomicAdd(recompute, 1ull);
      } else {
        bit = acc > 0.f;
      }
      if (bit)
        atomicOr(reinterpret_cast<unsigned long long*>(strings) + ((size_t)q * n + row) * W + c / 64,
                 1ull << (c & 63));
    }
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D map over a row-major [rows][inner] matrix, box = 128 B x 128 rows.
int make_map(CUtensorMap* m, const void* ptr, bool bf16, int64_t inner,
             int64_t rows, int box_rows) {
  EncodeFn enc = get_encode();
  if (!enc) return set_error("cuTensorMapEncodeTiled unavailable"), MSM_E_CUDA;
  const int es = bf16 ? 2 : 4;
  cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(inner * es)};
  cuuint32_t box[2] = {(cuuint32_t)(kChunkBytes / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   2, const_cast<void*>(ptr), gdim, gstride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error("cuTensorMapEncodeTiled failed (%d)", (int)r), MSM_E_CUDA;
  return MSM_OK;
}

}  // namespace

bool tc_project_supported(int dtype, int dim, uintptr_t xaddr) {
  const int es = dtype == MSM_DT_BF16 ? 2 : 4;
  const int64_t rowbytes = (int64_t)dim * es;
  return rowbytes % kChunkBytes == 0 && rowbytes <= kMaxChunks * kChunkBytes &&
         (xaddr % 16) == 0;
}

size_t tc_project_scratch_bytes(int64_t n, int dim, int Q, int ell, int dtype) {
  const int W = (ell + 63) / 64;
  const int64_t rows = (((int64_t)Q * W * 64 + kCols - 1) / kCols) * kCols;
  const int es = dtype == MSM_DT_BF16 ? 2 : 4;
  const int64_t fix_cap = ((int64_t)n * Q * ell) / 16 + (1 << 20);
  return 2 * (size_t)rows * dim * es + 4 * (size_t)rows + 8 * (size_t)fix_cap + 4096;
}

int launch_project_tc(const void* X, int dtype, int64_t n, int dim,
                      const float* R, const float* xnorm, int Q, int ell,
                      uint64_t* strings, unsigned long long* recompute,
                      void* ws, unsigned* status, bool* fell_back,
                      cudaStream_t s) {
  const bool bf16 = dtype == MSM_DT_BF16;
  const int es = bf16 ? 2 : 4;
  const int W = (ell + 63) / 64;
  const int64_t rows = (((int64_t)Q * W * 64 + kCols - 1) / kCols) * kCols;
  const int64_t fix_cap = ((int64_t)n * Q * ell) / 16 + (1 << 20);
  char* p = (char*)ws;
  void* Bhi = p; p += (size_t)rows * dim * es;
  void* Blo = p; p += (size_t)rows * dim * es;
  float* rnorm = (float*)p; p += 4 * (size_t)rows;
  p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
  uint64_t* fix = (uint64_t*)p; p += 8 * (size_t)fix_cap;
  unsigned long long* fix_count = (unsigned long long*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
  if (fell_back) *fell_back = false;

  MSM_CUDA(cudaMemsetAsync(fix_count, 0, 8, s));
  MSM_CUDA(cudaMemsetAsync(rnorm, 0, 4 * (size_t)rows, s));
  {
    int grid = (int)((rows + 255) / 256);
    kt_begin(KC_OTHER, s);
    if (bf16) transpose_R_kernel<true><<<grid, 256, 0, s>>>(R, Q, dim, ell, W, rows, Bhi, Blo, rnorm);
    else transpose_R_kernel<false><<<grid, 256, 0, s>>>(R, Q, dim, ell, W, rows, Bhi, Blo, rnorm);
    kt_end(s);
    MSM_LAUNCH("transpose_R_kernel");
  }
  CUtensorMap mX, mB, mB2;
  int rc = make_map(&mX, X, bf16, dim, n, kRows);
  if (!rc) rc = make_map(&mB, Bhi, bf16, dim, rows, kCols);
  if (!rc) rc = make_map(&mB2, bf16 ? Blo : Bhi, bf16, dim, rows, kCols);
  if (rc) return rc;

  TcArgs a;
  a.n = n;
  a.dim = dim;
  a.ell = ell;
  a.W = W;
  a.Q = Q;
  a.ctiles = (int)(rows / kCols);
  a.chunks = (dim * es) / kChunkBytes;
  // instruction descriptor: D f32, A/B = TF32 (2) or BF16 (1), both
  // K-major, N = 128, M = 128
  const uint32_t fmt = bf16 ? 1u : 2u;
  a.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kCols >> 3) << 17) |
            ((uint32_t)(kRows >> 4) << 24);
  const float eop = bf16 ? 0x1.0p-16f : 0x1.0p-9f;
  a.mscale = eop + (float)(4 * dim) * 0x1.0p-24f;
  a.mabs = (float)dim * 0x1.0p-120f;
  a.xnorm = xnorm;
  a.rnorm = rnorm;
  a.strings = strings;
  a.fix = fix;
  a.fix_cap = fix_cap;
  a.fix_count = fix_count;
  a.status = status;

  const int kNB = bf16 ? 2 : 1;
  // X tile (chunks boxes of 128 rows) + R tile (kNB * chunks boxes of 64
  // rows) + barriers: 97 KB for float rows of 512 B, so two CTAs share an
  // SM and one's epilogue overlaps the other's copies and MMAs
  const size_t smem = 1024 + (size_t)a.chunks * (kTileBytes + kNB * kBTileBytes) + 64;
  auto kern = bf16 ? project_tc_kernel<true> : project_tc_kernel<false>;
  MSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)((n + kRows - 1) / kRows);
  kt_begin(KC_PROJECT, s);
  kern<<<grid, 128, smem, s>>>(mX, mB, mB2, a);
  kt_end(s);
  MSM_LAUNCH("project_tc_kernel");

  if (!fell_back) {
    // no host round trip: the fix-up reads the queue length on the device
    // and reports an overflow in *status (bit 1) for the caller to act on
    kt_begin(KC_PROJECT, s);
    project_fix_kernel<<<num_sms() * 16, 256, 0, s>>>(X, dtype, n, dim, R,
                                                      bf16 ? nullptr : (const float*)Bhi, ell,
                                                      W, xnorm, rnorm, fix, fix_count, fix_cap,
                                                      strings, recompute, status);
    kt_end(s);
    MSM_LAUNCH("project_fix_kernel");
    return MSM_OK;
  }
  // queued bits; an overflowing queue means the tensor-core pass cannot be
  // completed from it, so the caller reruns the projection on the SIMT path
  unsigned long long cnt = 0;
  MSM_CUDA(cudaMemcpyAsync(&cnt, fix_count, 8, cudaMemcpyDeviceToHost, s));
  MSM_CUDA(cudaStreamSynchronize(s));
  unsigned st = 0;
  MSM_CUDA(cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost));
  if (st & 1u) return set_error("tensor-core projection: a bounded wait timed out"), MSM_E_TIMEOUT;
  if ((int64_t)cnt > fix_cap) {
    *fell_back = true;
    return MSM_OK;
  }
  if (cnt > 0) {
    int64_t warps = (int64_t)cnt;
    int grid2 = (int)((warps * 32 + 255) / 256);
    const int cap = num_sms() * 16;
    if (grid2 > cap) grid2 = cap;
    kt_begin(KC_PROJECT, s);
    project_fix_kernel<<<grid2, 256, 0, s>>>(X, dtype, n, dim, R,
                                              bf16 ? nullptr : (const float*)Bhi, ell, W, xnorm,
                                              rnorm, fix, fix_count, fix_cap, strings, recompute,
                                              status);
    kt_end(s);
    MSM_LAUNCH("project_fix_kernel");
  }
  return MSM_OK;
}

}  // namespace msm

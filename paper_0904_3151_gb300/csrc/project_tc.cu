// Step A1 on the 5th-generation tensor cores: t = X R_q for all replicates
// as one GEMM (n x D) * (D x Q*W*64).  Each CTA owns 128 rows of X, staged
// once in shared memory by TMA (128-byte swizzle), and walks the column
// tiles of 64 columns (one packed output word per row): a producer warp
// keeps a ring of R tiles filled by TMA, an MMA warp issues the MMAs of
// tile t into one of two TMEM accumulators, and eight epilogue warps read
// the other accumulator (tcgen05.ld; a thread owns one row and 32 of the 64
// columns) and turn tile t - 1 into signs and packed half-words (Eq. 3), so
// copies, MMAs and the epilogue overlap.
//
// Exactness.  Both operands are split into bf16 parts: x = xh + xl + ex with
// xh = bf16(x), xl = bf16(x - xh), |ex| <= 2^-16 |x| (bf16 keeps 8
// significant bits), and likewise r = rh + rl + er (bf16 X is exact: xl = 0).
// The three MMAs xh rh + xh rl + xl rh (kind::f16, float accumulation)
// leave out xl rl + (xh + xl) er + ex (rh + rl), at most 3.1 2^-16 |x_c r_c|
// per coordinate, so with sum_c |x_c r_c| <= |x| |r| the accumulated t'
// satisfies
//   |t' - t| <= (3.125 2^-16 + 4 m 2^-24) |x| |r| + tiny,
// m = the number of accumulated products (3 D, or 2 D for bf16 X); 4 m 2^-24
// is four times the classical bound of the float accumulation.  Bits with
// |t'| within that margin are written as 0 and queued; project_fix_kernel
// recomputes each in float with its own bound and, if still undecided, in
// double precision by sequential fma (the definition of the bit), then sets
// it.
//
// Every wait is bounded (a poll limit and 2 s of %globaltimer); a thread that
// gives up raises a CTA flag and the status word, the others stop at their
// next wait, and the producer and MMA threads wait (bounded, ignoring the
// flag) for every copy and MMA they issued before the CTA releases its
// shared memory and TMEM.
#include <atomic>

#include <cuda.h>
#include <cuda_bf16.h>

#include "msm_internal.cuh"
#include "readback.cuh"
#include "tcgen05.cuh"

namespace msm {

// Poll limit of the projection's bounded waits (a testing knob).
static std::atomic<uint32_t> g_wait_polls{1u << 22};

namespace {

using namespace tc;

constexpr int kRows = 128;          // M of the MMA, rows per CTA
constexpr int kCols = 64;           // N of the MMA, columns per tile (one word)
constexpr int kMaxChunks = 4;       // bf16 rows of at most 512 B (dim <= 256)
constexpr int kXBox = kRows * kChunkBytes;  // one 128 x 128 B box of X
constexpr int kRBox = kCols * kChunkBytes;  // one 64 x 128 B box of R
constexpr int kMaxStages = 4;       // R tiles in flight
constexpr int kEpiWarps = 8;        // warp w: TMEM lanes (rows) 32 (w % 4) ..,
                                    // columns 32 (w / 4) .. of each tile
constexpr int kTcThreads = (kEpiWarps + 2) * 32;  // + TMA warp + MMA warp
constexpr uint32_t kDrainPolls = 1u << 24;
constexpr int kFixBuf = 64;         // undecided bits buffered per epilogue warp
constexpr size_t kSmemBudget = 200 * 1024 - 8 * kEpiWarps * kFixBuf;

struct TcArgs {
  int64_t n;
  int dim;
  int ell, W, Q;
  int ctiles;          // column tiles of 64 over the padded Q*W*64 columns
  int chunks;          // K chunks of 128 B of the bf16 operands
  int stages;          // R tiles in the ring
  uint32_t idesc;
  uint32_t polls;      // poll limit of the bounded waits
  float mscale, mabs;  // margin = mscale * |x| * |r| + mabs
  const float* xnorm;  // [n]
  const float* rnorm;  // [Q * W * 64] (padded columns have norm 0)
  uint64_t* strings;   // [Q][n][W]
  uint64_t* fix;       // queued (row << 32 | q * ell + c)
  int64_t fix_cap;
  unsigned long long* fix_count;
  unsigned* status;    // bit 0: a bounded wait gave up
};

// Appends a warp's buffered undecided bits to the fix-up queue (one atomic).
__device__ __forceinline__ void flush_fix(const TcArgs& a, const uint64_t* qbuf, uint32_t& nq,
                                          int lane) {
  if (!nq) return;
  __syncwarp();
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(a.fix_count, (unsigned long long)nq);
  b = __shfl_sync(0xffffffffu, b, 0);
  for (uint32_t t = lane; t < nq; t += 32)
    if ((int64_t)(b + t) < a.fix_cap) a.fix[b + t] = qbuf[t];
  __syncwarp();
  nq = 0;
}

// 320 threads: warps 0-7 epilogue (warp 0 also allocates TMEM), warp 8 lane
// 0 issues the TMA copies, warp 9 lane 0 the MMAs.
template <bool XLO>
__global__ void __launch_bounds__(kTcThreads, 1)
project_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                  const __grid_constant__ CUtensorMap tmXl,
                  const __grid_constant__ CUtensorMap tmR,
                  const __grid_constant__ CUtensorMap tmRl, TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int xbytes = a.chunks * kXBox;
  const int rbytes = a.chunks * kRBox;  // one part (high or low) of an R tile
  uint8_t* sX = base;
  uint8_t* sXl = base + xbytes;
  uint8_t* sR = base + (XLO ? 2 : 1) * xbytes;  // stage s: high, then low
  uint64_t* bars = (uint64_t*)(sR + a.stages * 2 * rbytes);
  uint64_t* barX = bars;
  uint64_t* full = bars + 1;
  uint64_t* empty = full + a.stages;
  uint64_t* tfull = empty + a.stages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tslot = (uint32_t*)(tempty + 2);
  uint32_t* abortf = tslot + 1;
  uint64_t* fixbuf = (uint64_t*)(tslot + 4);  // [kEpiWarps][kFixBuf]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * kRows;
  if (tid == 0) {
    mbar_init(barX, 1);
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, kEpiWarps);
    }
    *abortf = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tslot)),
                 "r"(2 * kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int ksteps = kChunkBytes / 32;  // MMA K is 32 bytes (16 bf16)

  if (warp == kEpiWarps) {
    // TMA producer: X once, then R tiles into the ring as stages free up
    if (lane == 0) {
      int last_t[kMaxStages];  // last tile loaded into each stage (-1: none)
      for (int s = 0; s < kMaxStages; ++s) last_t[s] = -1;
      mbar_expect_tx(barX, (uint32_t)((XLO ? 2 : 1) * xbytes));
      for (int c = 0; c < a.chunks; ++c) {
        tma_load_2d(sX + c * kXBox, &tmX, barX, c * (kChunkBytes / 2), (int)row0);
        if (XLO) tma_load_2d(sXl + c * kXBox, &tmXl, barX, c * (kChunkBytes / 2), (int)row0);
      }
      bool ok = true;
      for (int t = 0; t < a.ctiles; ++t) {
        const int s = t % a.stages, k = t / a.stages;
        if (k > 0) {  // the MMAs of tile t - stages are done with this stage
          ok = mbar_wait(empty + s, (uint32_t)((k - 1) & 1), a.polls, abortf);
          if (!ok) break;
        }
        mbar_expect_tx(full + s, (uint32_t)(2 * rbytes));
        uint8_t* dst = sR + s * 2 * rbytes;
        for (int c = 0; c < a.chunks; ++c) {
          tma_load_2d(dst + c * kRBox, &tmR, full + s, c * (kChunkBytes / 2), t * kCols);
          tma_load_2d(dst + rbytes + c * kRBox, &tmRl, full + s, c * (kChunkBytes / 2),
                      t * kCols);
        }
        last_t[s] = t;
      }
      if (!ok) {
        atomicOr(a.status, 1u);
        *(volatile uint32_t*)abortf = 1u;
      }
      // drain: every copy issued lands before the CTA releases its memory
      // (the loads of one stage complete in order, so the last one suffices)
      mbar_wait(barX, 0, kDrainPolls, nullptr);
      for (int s = 0; s < a.stages; ++s)
        if (last_t[s] >= 0)
          mbar_wait(full + s, (uint32_t)((last_t[s] / a.stages) & 1), kDrainPolls, nullptr);
    }
  } else if (warp == kEpiWarps + 1) {
    // MMA issuer: tile t into accumulator t & 1 once its R tile has landed
    // and the epilogue has read that accumulator's previous tile
    if (lane == 0) {
      int last_tb = -1, last_es = -1;
      uint32_t last_tpar = 0, last_epar = 0;
      bool ok = mbar_wait(barX, 0, a.polls, abortf);
      for (int t = 0; ok && t < a.ctiles; ++t) {
        const int s = t % a.stages, b = t & 1;
        const uint32_t sp = (uint32_t)((t / a.stages) & 1), bp = (uint32_t)((t >> 1) & 1);
        ok = mbar_wait(full + s, sp, a.polls, abortf);
        if (!ok) break;
        if (t >= 2) {
          ok = mbar_wait(tempty + b, bp ^ 1u, a.polls, abortf);
          if (!ok) break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * kCols);
        const uint8_t* rs = sR + s * 2 * rbytes;
        uint32_t acc = 0;
        for (int c = 0; c < a.chunks; ++c)
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t ah = sw128_desc(saddr(sX + c * kXBox) + ks * 32);
            const uint64_t bh = sw128_desc(saddr(rs + c * kRBox) + ks * 32);
            const uint64_t bl = sw128_desc(saddr(rs + rbytes + c * kRBox) + ks * 32);
            mma<true>(d, ah, bh, a.idesc, acc);
            acc = 1;
            mma<true>(d, ah, bl, a.idesc, 1);
            if (XLO) {
              const uint64_t al = sw128_desc(saddr(sXl + c * kXBox) + ks * 32);
              mma<true>(d, al, bh, a.idesc, 1);
            }
          }
        mma_commit(tfull + b);
        mma_commit(empty + s);
        last_tb = b;
        last_tpar = bp;
        last_es = s;
        last_epar = sp;
      }
      if (!ok) {
        atomicOr(a.status, 1u);
        *(volatile uint32_t*)abortf = 1u;
      }
      // drain: every MMA issued (and its commits) completes before the CTA
      // releases its tensor memory
      if (last_tb >= 0) mbar_wait(tfull + last_tb, last_tpar, kDrainPolls, nullptr);
      if (last_es >= 0) mbar_wait(empty + last_es, last_epar, kDrainPolls, nullptr);
    }
  } else if (warp < kEpiWarps) {
    // epilogue: rows 32 (warp % 4) + lane, columns 32 (warp / 4) .. + 31 of
    // every tile (a warp may read only its quarter of the TMEM lanes)
    const int quarter = warp & 3, half = warp >> 2;
    const int64_t row = row0 + quarter * 32 + lane;
    const bool live_row = row < a.n;
    const float xn = live_row ? a.xnorm[row] : 0.f;
    const int colsPerRep = a.W * 64;
    const uint32_t tlane = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
    uint32_t* strings32 = reinterpret_cast<uint32_t*>(a.strings);
    uint64_t* qbuf = fixbuf + warp * kFixBuf;  // this warp's undecided bits
    uint32_t nq = 0;                           // entries in qbuf (warp-uniform)
    for (int t = 0; t < a.ctiles; ++t) {
      const int b = t & 1;
      const uint32_t bp = (uint32_t)((t >> 1) & 1);
      const bool ok = mbar_wait(tfull + b, bp, a.polls, abortf);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) {
          atomicOr(a.status, 1u);
          *(volatile uint32_t*)abortf = 1u;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t r[32];
      tmem_ld32(tlane + (uint32_t)(b * kCols), r);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + b);
      const int gcol0 = t * kCols;             // first column of this word
      const int q = gcol0 / colsPerRep;
      const int cw = gcol0 % colsPerRep + half * 32;  // first column of this half in R_q
      const bool live = live_row && q < a.Q;
      uint32_t bits = 0, flagged = 0;
      if (live) {
        const float* rn = a.rnorm + q * colsPerRep + cw;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (cw + j >= a.ell) continue;
          const float tv = __uint_as_float(r[j]);
          const float m = a.mscale * xn * rn[j] + a.mabs;
          if (fabsf(tv) <= m) flagged |= 1u << j;
          else if (tv > 0.f) bits |= 1u << j;
        }
      }
      // collect the undecided bits in the warp's buffer
      uint32_t cnt = __popc(flagged), incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      if (total) {
        if (nq + total > (uint32_t)kFixBuf) flush_fix(a, qbuf, nq, lane);
        uint32_t pos = nq + incl - cnt;
        while (flagged) {
          const int j = __ffs(flagged) - 1;
          flagged &= flagged - 1;
          const uint64_t e = ((uint64_t)row << 32) | (uint32_t)(q * a.ell + cw + j);
          if (pos < (uint32_t)kFixBuf) {
            qbuf[pos] = e;
          } else {  // more than a buffer's worth in one tile: append directly
            const unsigned long long b0 = atomicAdd(a.fix_count, 1ull);
            if ((int64_t)b0 < a.fix_cap) a.fix[b0] = e;
          }
          ++pos;
        }
        nq = min(nq + total, (uint32_t)kFixBuf);
        __syncwarp();
      }
      // the low (half 0) or high (half 1) 32 bits of the word, little-endian
      if (live) strings32[(((size_t)q * a.n + row) * a.W + cw / 64) * 2 + half] = bits;
    }
    flush_fix(a, qbuf, nq, lane);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * kCols)
                 : "memory");
}

// Xh = bf16(x), Xl = bf16(x - Xh) for float X (8 elements per step).
__global__ void split_x_kernel(const float* X, int64_t count, __nv_bfloat16* Xh,
                               __nv_bfloat16* Xl) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float v = X[e];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Xh[e] = h;
    Xl[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// Rows of the transposed R: row q * W * 64 + c holds column c of R_q (zero
// for c >= ell; rows padded to a multiple of 64), as bf16 high and low parts
// (hi = bf16(R), lo = bf16(R - hi)) for the MMAs and as float for the
// fix-up's coalesced reads; rnorm = the column norms.
__global__ void transpose_R_kernel(const float* R, int Q, int dim, int ell, int W,
                                   int64_t rows, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                   float* Rt, float* rnorm) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int colsPerRep = W * 64;
    const int q = (int)(t / colsPerRep), c = (int)(t % colsPerRep);
    const bool live = q < Q && c < ell;
    double nrm = 0.0;
    for (int k = 0; k < dim; ++k) {
      const float v = live ? R[((size_t)q * dim + k) * ell + c] : 0.f;
      nrm = fma((double)v, (double)v, nrm);
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hi[t * dim + k] = h;
      lo[t * dim + k] = __float2bfloat16_rn(v - __bfloat162float(h));
      Rt[t * dim + k] = v;
    }
    if (t < (int64_t)Q * colsPerRep) rnorm[t] = (float)sqrt(nrm);
  }
}

__device__ __forceinline__ float ldx(const void* X, int dtype, int64_t i) {
  if (dtype == MSM_DT_BF16)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[i]);
  return reinterpret_cast<const float*>(X)[i];
}

// Four queued bits per warp, eight lanes each: the float dot product with
// its own bound decides the bit where it can; the rest go to a second queue
// for project_fix64_kernel.  Rt: the transposed float copy of R (row
// q * W * 64 + c holds column c of R_q, contiguous over the coordinates).
__global__ void project_fix_kernel(const void* X, int dtype, int64_t n, int dim,
                                   const float* Rt, int ell, int W,
                                   const float* xnorm, const float* rnorm_pad,
                                   const uint64_t* fix,
                                   const unsigned long long* fix_count,
                                   int64_t fix_cap, uint64_t* dq,
                                   unsigned long long* dq_count, int64_t dq_cap,
                                   uint64_t* strings, unsigned* status) {
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
  const int sub = lane & 7, grp = lane >> 3;
  for (int64_t base = warp * 4; base < m; base += nwarps * 4) {
    const int64_t it = base + grp;
    const bool valid = it < m;
    const uint64_t e = valid ? fix[it] : 0ull;
    const int64_t row = (int64_t)(e >> 32);
    const int qc = (int)(e & 0xffffffffu);
    const int q = qc / ell, c = qc % ell;
    const float* rc = Rt + (size_t)(q * W * 64 + c) * dim;
    float acc = 0.f;
    if (valid) {
#pragma unroll 4
      for (int k = sub; k < dim; k += 8) acc = fmaf(ldx(X, dtype, row * dim + k), rc[k], acc);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (valid && sub == 0) {
      const float marg = m2 * xnorm[row] * rnorm_pad[q * W * 64 + c] + (float)dim * 0x1.0p-120f;
      if (fabsf(acc) <= marg) {
        const unsigned long long slot = atomicAdd(dq_count, 1ull);
        if ((int64_t)slot < dq_cap) dq[slot] = e;
        else atomicOr(status, 2u);
      } else if (acc > 0.f) {
        atomicOr(reinterpret_cast<unsigned long long*>(strings) + ((size_t)q * n + row) * W + c / 64,
                 1ull << (c & 63));
      }
    }
  }
}

// One queued bit per thread: the double-precision dot product accumulated
// by sequential fma over the coordinates -- the definition of the bit.
__global__ void project_fix64_kernel(const void* X, int dtype, int64_t n, int dim,
                                     const float* Rt, int ell, int W, const uint64_t* dq,
                                     const unsigned long long* dq_count, int64_t dq_cap,
                                     uint64_t* strings, unsigned long long* recompute) {
  int64_t m = (int64_t)*dq_count;
  if (m > dq_cap) m = dq_cap;  // an overflow is reported in the status word
  unsigned long long cnt = 0;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < m;
       it += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t e = dq[it];
    const int64_t row = (int64_t)(e >> 32);
    const int qc = (int)(e & 0xffffffffu);
    const int q = qc / ell, c = qc % ell;
    const float* rc = Rt + (size_t)(q * W * 64 + c) * dim;
    double t = 0.0;
    for (int k = 0; k < dim; ++k) t = fma((double)ldx(X, dtype, row * dim + k), (double)rc[k], t);
    if (t > 0.0)
      atomicOr(reinterpret_cast<unsigned long long*>(strings) + ((size_t)q * n + row) * W + c / 64,
               1ull << (c & 63));
    ++cnt;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(recompute, cnt);
}

inline size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

int chunks_of(int dim) { return (2 * dim + kChunkBytes - 1) / kChunkBytes; }

int stages_for(int dim, bool xlo) {
  const size_t x = (size_t)(xlo ? 2 : 1) * chunks_of(dim) * kXBox;
  const size_t st = (size_t)2 * chunks_of(dim) * kRBox;
  if (x + st > kSmemBudget) return 0;
  size_t n = (kSmemBudget - x) / st;
  return (int)(n > (size_t)kMaxStages ? kMaxStages : n);
}

}  // namespace

uint32_t wait_polls() { return g_wait_polls.load(); }

int set_wait_polls(uint32_t polls) {
  const uint32_t old = g_wait_polls.exchange(polls ? polls : (1u << 22));
  return (int)old;
}

// Rows of X as bf16 whose row stride is a multiple of 16 bytes, at most 512
// bytes (dim <= 256), from a 16-byte-aligned address.
bool tc_project_supported(int dtype, int dim, uintptr_t xaddr) {
  if (dim < 8 || dim % 8 != 0 || chunks_of(dim) > kMaxChunks) return false;
  if (dtype == MSM_DT_BF16 && (xaddr % 16) != 0) return false;
  return stages_for(dim, dtype != MSM_DT_BF16) >= 1;
}

size_t tc_project_scratch_bytes(int64_t n, int dim, int Q, int ell, int dtype) {
  const int W = (ell + 63) / 64;
  const int64_t rows = (((int64_t)Q * W * 64 + kCols - 1) / kCols) * kCols;
  const int64_t fix_cap = ((int64_t)n * Q * ell) / 64 + (1 << 20);
  const size_t xs = dtype == MSM_DT_BF16 ? 0 : 2 * up256(2 * (size_t)n * dim);
  return xs + 2 * up256(2 * (size_t)rows * dim) + up256(4 * (size_t)rows * dim) +
         up256(4 * (size_t)rows) + up256(8 * (size_t)fix_cap) + up256(2 * (size_t)fix_cap) +
         4096;
}

int launch_project_tc(const void* X, int dtype, int64_t n, int dim,
                      const float* R, const float* xnorm, int Q, int ell,
                      uint64_t* strings, unsigned long long* recompute,
                      void* ws, unsigned* status, bool* fell_back,
                      cudaStream_t s) {
  const bool xlo = dtype != MSM_DT_BF16;
  const int W = (ell + 63) / 64;
  const int64_t rows = (((int64_t)Q * W * 64 + kCols - 1) / kCols) * kCols;
  const int64_t fix_cap = ((int64_t)n * Q * ell) / 64 + (1 << 20);
  char* p = (char*)ws;
  __nv_bfloat16* Xh = nullptr;
  __nv_bfloat16* Xl = nullptr;
  if (xlo) {
    Xh = (__nv_bfloat16*)p; p += up256(2 * (size_t)n * dim);
    Xl = (__nv_bfloat16*)p; p += up256(2 * (size_t)n * dim);
  }
  __nv_bfloat16* Rh = (__nv_bfloat16*)p; p += up256(2 * (size_t)rows * dim);
  __nv_bfloat16* Rl = (__nv_bfloat16*)p; p += up256(2 * (size_t)rows * dim);
  float* Rt = (float*)p; p += up256(4 * (size_t)rows * dim);
  float* rnorm = (float*)p; p += up256(4 * (size_t)rows);
  uint64_t* fix = (uint64_t*)p; p += up256(8 * (size_t)fix_cap);
  const int64_t dq_cap = fix_cap / 4;  // bits left undecided by the float pass
  uint64_t* dq = (uint64_t*)p; p += up256(2 * (size_t)fix_cap);
  unsigned long long* fix_count = (unsigned long long*)p;
  unsigned long long* dq_count = fix_count + 1;
  if (fell_back) *fell_back = false;

  MSM_CUDA(cudaMemsetAsync(fix_count, 0, 16, s));
  MSM_CUDA(cudaMemsetAsync(rnorm, 0, 4 * (size_t)rows, s));
  {
    int grid = (int)((rows + 255) / 256);
    kt_begin(KC_OTHER, s);
    transpose_R_kernel<<<grid, 256, 0, s>>>(R, Q, dim, ell, W, rows, Rh, Rl, Rt, rnorm);
    kt_end(s);
    MSM_LAUNCH("transpose_R_kernel");
  }
  if (xlo) {
    int64_t grid = ((int64_t)n * dim + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (grid > cap) grid = cap;
    kt_begin(KC_PROJECT, s);
    split_x_kernel<<<(int)grid, 256, 0, s>>>((const float*)X, (int64_t)n * dim, Xh, Xl);
    kt_end(s);
    MSM_LAUNCH("split_x_kernel");
  }
  CUtensorMap mX, mXl, mR, mRl;
  int rc = make_map(&mX, xlo ? (const void*)Xh : X, dim, n, kRows);
  if (!rc) rc = make_map(&mXl, xlo ? (const void*)Xl : X, dim, n, kRows);
  if (!rc) rc = make_map(&mR, Rh, dim, rows, kCols);
  if (!rc) rc = make_map(&mRl, Rl, dim, rows, kCols);
  if (rc) return rc;

  TcArgs a;
  a.n = n;
  a.dim = dim;
  a.ell = ell;
  a.W = W;
  a.Q = Q;
  a.ctiles = (int)(rows / kCols);
  a.chunks = chunks_of(dim);
  a.stages = stages_for(dim, xlo);
  if (a.stages < 1) return set_error("no tensor-core projection for dim %d", dim), MSM_E_INVAL;
  // instruction descriptor: D f32, A/B = BF16, both K-major, N = 64, M = 128
  a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kCols >> 3) << 17) |
            ((uint32_t)(kRows >> 4) << 24);
  a.polls = g_wait_polls.load();
  const int terms = (xlo ? 3 : 2) * dim;
  a.mscale = 0x1.9p-15f + (float)(4 * terms + 8) * 0x1.0p-24f;
  a.mabs = (float)dim * 0x1.0p-120f;
  a.xnorm = xnorm;
  a.rnorm = rnorm;
  a.strings = strings;
  a.fix = fix;
  a.fix_cap = fix_cap;
  a.fix_count = fix_count;
  a.status = status;

  // X tile (high [+ low]) + the ring of R tiles (high + low) + barriers +
  // the epilogue warps' buffers of undecided bits
  const size_t smem = 1024 + (size_t)(xlo ? 2 : 1) * a.chunks * kXBox +
                      (size_t)a.stages * 2 * a.chunks * kRBox + 8 * (1 + 2 * kMaxStages + 4) + 16 +
                      8 * (size_t)kEpiWarps * kFixBuf;
  auto kern = xlo ? project_tc_kernel<true> : project_tc_kernel<false>;
  MSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)((n + kRows - 1) / kRows);
  kt_begin(KC_PROJECT, s);
  kern<<<grid, kTcThreads, smem, s>>>(mX, mXl, mR, mRl, a);
  kt_end(s);
  MSM_LAUNCH("project_tc_kernel");

  if (!fell_back) {
    // no host round trip: the fix-up reads the queue lengths on the device
    // and reports an overflow in *status (bit 1) for the caller to act on
    kt_begin(KC_PROJECT, s);
    project_fix_kernel<<<num_sms() * 16, 256, 0, s>>>(X, dtype, n, dim, Rt, ell, W, xnorm, rnorm,
                                                      fix, fix_count, fix_cap, dq, dq_count,
                                                      dq_cap, strings, status);
    kt_end(s);
    MSM_LAUNCH("project_fix_kernel");
    kt_begin(KC_PROJECT, s);
    project_fix64_kernel<<<num_sms() * 4, 256, 0, s>>>(X, dtype, n, dim, Rt, ell, W, dq, dq_count,
                                                       dq_cap, strings, recompute);
    kt_end(s);
    MSM_LAUNCH("project_fix64_kernel");
    return MSM_OK;
  }
  // queued bits; an overflowing queue means the tensor-core pass cannot be
  // completed from it, so the caller reruns the projection on the SIMT path
  unsigned long long cnt = 0;
  rc = read_to_host(&cnt, fix_count, 8, s);
  if (rc) return rc;
  unsigned st = 0;
  rc = read_to_host(&st, status, 4, s);
  if (rc) return rc;
  if (st & 1u) return set_error("tensor-core projection: a bounded wait timed out"), MSM_E_TIMEOUT;
  if ((int64_t)cnt > fix_cap) {
    *fell_back = true;
    return MSM_OK;
  }
  if (cnt > 0) {
    int64_t warps = ((int64_t)cnt + 3) / 4;
    int grid2 = (int)((warps * 32 + 255) / 256);
    const int cap = num_sms() * 16;
    if (grid2 > cap) grid2 = cap;
    kt_begin(KC_PROJECT, s);
    project_fix_kernel<<<grid2, 256, 0, s>>>(X, dtype, n, dim, Rt, ell, W, xnorm, rnorm, fix,
                                              fix_count, fix_cap, dq, dq_count, dq_cap, strings,
                                              status);
    kt_end(s);
    MSM_LAUNCH("project_fix_kernel");
    unsigned long long dcnt = 0;
    rc = read_to_host(&dcnt, dq_count, 8, s);
    if (rc) return rc;
    if ((int64_t)dcnt > dq_cap) {
      *fell_back = true;
      return MSM_OK;
    }
    if (dcnt > 0) {
      int grid3 = (int)((dcnt + 255) / 256);
      if (grid3 > cap) grid3 = cap;
      kt_begin(KC_PROJECT, s);
      project_fix64_kernel<<<grid3, 256, 0, s>>>(X, dtype, n, dim, Rt, ell, W, dq, dq_count,
                                                 dq_cap, strings, recompute);
      kt_end(s);
      MSM_LAUNCH("project_fix64_kernel");
    }
  }
  return MSM_OK;
}

}  // namespace msm

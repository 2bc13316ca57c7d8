// Measurement aid, not part of the method: the throughput ceiling of the
// pair check's integer work on this GPU.
//
// The pair check's gap test spends, per 32-bit word of 16-bit block fields,
// one xor (x = a ^ b), one add (bit 15 of a field of x + 0x7FFF is set iff
// the field is nonzero) and one and-not-or (bad |= gap_mask & ~sum).  This
// kernel issues exactly that mix from registers -- no memory traffic -- over
// 8 independent chains per thread at full occupancy, so its rate is what the
// SM's integer pipes sustain for the mix.  The chains feed each round's sum
// back as the next round's `a`, which keeps the compiler from hoisting or
// folding any of the three operations.
//
// Built as its own library (libmsm_probe.so, declared in msm_probe.h) for
// the benchmark: the method's library does not carry it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/msm_probe.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads)
int_mix_kernel(uint32_t* out, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * kProbeThreads + threadIdx.x;
  uint32_t a[kChains], b[kChains], g[kChains], bad[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    const uint32_t e = tid * kChains + j;
    a[j] = e * 0x9E3779B1u + seed;
    b[j] = (e * 0x85EBCA6Bu) ^ seed;
    g[j] = (j & 1) ? 0x80008000u : 0x00008000u;
    bad[j] = 0;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      const uint32_t t = (a[j] ^ b[j]) + 0x7FFF7FFFu;
      bad[j] |= g[j] & ~t;
      a[j] = t;
    }
  }
#pragma unroll
  for (int j = 0; j < kChains; ++j) out[(size_t)tid * kChains + j] = bad[j] ^ a[j];
}

}  // namespace

extern "C" int msm_int_mix_probe(uint32_t* out, int blocks, int iters, uint32_t seed,
                                 void* stream) {
  if (!out || blocks < 1 || iters < 0) return -1;
  int_mix_kernel<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(out, iters, seed);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

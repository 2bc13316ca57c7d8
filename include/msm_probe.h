/*
 * msm_probe.h -- C ABI of libmsm_probe.so, a measurement aid built beside
 * the method's library (libmsm.so) for the benchmark.  It is not part of the
 * method: it supplies the integer-throughput ceiling against which the pair
 * check's roofline is reported.
 */
#ifndef MSM_PROBE_H
#define MSM_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Measurement aid, not part of the method: the rate at which this GPU
 * sustains the pair check's integer work.  The paper counts the cost of the
 * in-group checks (Sec. 2.2) but gives no hardware ceiling; this probe
 * supplies one.  `blocks` CTAs of 256 threads each run `iters` rounds over 8
 * independent register chains of the gap-test word operation
 *     t = (a ^ b) + 0x7FFF7FFF;  bad |= g & ~t;  a = t
 * (xor, add, and-not-or: 3 integer operations), from the starting values
 *     e = thread * 8 + chain,  a = e * 0x9E3779B1 + seed,
 *     b = (e * 0x85EBCA6B) ^ seed,  g = chain odd ? 0x80008000 : 0x8000,
 *     bad = 0   (all arithmetic modulo 2^32),
 * and writes bad ^ a of every chain to out[thread * 8 + chain]
 * (device, caller-owned, blocks * 256 * 8 words).  Timing the call with
 * events on `stream` gives integer operations per second =
 * blocks * 256 * iters * 8 * 3 / seconds.  Asynchronous; returns 0, -1 (MSM_E_INVAL) on a NULL `out`,
 * blocks < 1 or iters < 0, or -4 (MSM_E_CUDA) when the launch fails. */
int msm_int_mix_probe(uint32_t* out, int blocks, int iters, uint32_t seed,
                      void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MSM_PROBE_H */

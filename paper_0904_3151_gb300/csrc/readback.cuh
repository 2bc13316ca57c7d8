// Small device-to-host reads of counters and status words.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace msm {

// Copies `bytes` (whole, aligned 4-byte words, at most kReadBackBytes) from
// device memory to `host` after the work queued on s before it: a one-warp
// kernel stores them into host-mapped pinned memory and s is synchronised.
// No copy engine takes part, so such a read never waits behind a large
// device-to-host copy that the caller runs on another stream meanwhile.
constexpr size_t kReadBackBytes = 1024;
int read_to_host(void* host, const void* dev, size_t bytes, cudaStream_t s);

}  // namespace msm

// msm_recheck_noalloc: the epsilon recheck for callers that may not allocate
// device memory.  Its scratch (row norms and counters) lives in one
// file-scope device array instead of memory obtained per call.
//
// Who needs this: code embedded in a host application that owns every byte
// of the GPU -- for example a serving process whose caching allocator has
// reserved the device, or a component with a fixed memory budget -- where a
// cudaMalloc from inside the library would fail or break the host's
// accounting.  Such callers pass inputs and outputs they already own.
#include <mutex>

#include "msm_internal.cuh"

namespace msm {
namespace {

// Largest number of rows of X this entry point accepts, and the size of the
// static scratch it implies: 8 + 4 bytes of norms per row plus 256 bytes of
// counters (about 3 MB, held by every GPU that loads the library).
constexpr int64_t kNoAllocMaxRows = 1 << 18;
constexpr size_t kCounterBytes = 256;
constexpr size_t kNoAllocBytes = kCounterBytes + (size_t)kNoAllocMaxRows * (8 + 4);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host code may not pass g_noalloc_scratch to a kernel (the name is a host
// stand-in); the device address is looked up once per device.
std::mutex g_mu;
unsigned char* g_addr[64] = {nullptr};

int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  MSM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error("device index out of range"), MSM_E_INVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_addr[dev] = (unsigned char*)p;
  }
  *out = g_addr[dev];
  return MSM_OK;
}

}  // namespace
}  // namespace msm

using namespace msm;

extern "C" int msm_recheck_noalloc(const void* X, int64_t n, int dim, int dtype,
                                   int metric, float eps, const uint64_t* cand,
                                   int64_t m, uint64_t* pairs_out,
                                   float* dist_out, int64_t* count,
                                   int64_t* recomputed, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!X || !count || n < 2 || dim < 1 || dim > kMaxDim || m < 0 ||
      (m > 0 && (!cand || !pairs_out)) || !(eps >= 0.f) ||
      (metric != MSM_COSINE && metric != MSM_EUCLIDEAN) ||
      (dtype != MSM_DT_F32 && dtype != MSM_DT_BF16))
    return set_error("invalid msm_recheck_noalloc arguments"), MSM_E_INVAL;
  if (n > kNoAllocMaxRows)
    return set_error("msm_recheck_noalloc accepts at most %lld rows (got %lld); "
                     "use msm_recheck for larger inputs",
                     (long long)kNoAllocMaxRows, (long long)n),
           MSM_E_INVAL;
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  // layout: [flags + counters: 256 B][norms double: n][norms float: n]
  unsigned* flags = (unsigned*)base;
  unsigned long long* ctr = (unsigned long long*)(base + 64);
  double* n64 = (double*)(base + kCounterBytes);
  float* n32 = (float*)(base + kCounterBytes + 8 * (size_t)kNoAllocMaxRows);
  // the array keeps the previous call's contents: clear what must start at 0
  MSM_CUDA(cudaMemsetAsync(base, 0, kCounterBytes, s));
  rc = launch_row_norms(X, dtype, n, dim, n64, n32, flags, s);
  if (rc) return rc;
  unsigned f = 0;
  MSM_CUDA(cudaMemcpyAsync(&f, flags, sizeof(f), cudaMemcpyDeviceToHost, s));
  MSM_CUDA(cudaStreamSynchronize(s));
  if (f & 2u) return set_error("input contains NaN or Inf"), MSM_E_NONFINITE;
  if ((f & 1u) && metric == MSM_COSINE)
    return set_error("cosine distance is undefined for an all-zero row"), MSM_E_ZERO_NORM;
  rc = launch_recheck(X, dtype, n, dim, metric, eps, n32, cand, nullptr, m,
                      pairs_out, dist_out, ctr, ctr + 1, (unsigned*)(ctr + 2), s);
  if (rc) return rc;
  unsigned long long h[3] = {0, 0, 0};
  MSM_CUDA(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
  MSM_CUDA(cudaStreamSynchronize(s));
  if (h[2]) return set_error("a candidate is not a pair i < j < n"), MSM_E_INVAL;
  *count = (int64_t)h[0];
  if (recomputed) *recomputed = (int64_t)h[1];
  return MSM_OK;
}

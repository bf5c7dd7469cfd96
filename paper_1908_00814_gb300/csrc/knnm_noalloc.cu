// knnm_noalloc.cu -- knnm_step_sample_noalloc: the round sampler for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns
// every device allocation, and processes that must not grow their device
// footprint after start-up (cudaMalloc/cudaFree can synchronize the device and
// stall other streams on a request path).  This entry point runs the same
// sampler kernels as knnm_step_sample, but its scratch (the packed list keys,
// the two reverse slot arrays and the counters) lives in one file-scope
// __device__ array of fixed size instead of memory taken from an allocator.
// That array belongs to the loaded library: every GPU that loads the library
// holds it until the process exits.  The caller still provides every input and
// output array.  Each call waits for its stream at the end, so no call may be
// made while a stream capture is active.

#include "../../include/knnm.h"
#include "knnm_internal.cuh"

using namespace knnm;

// The fixed scratch.  In host code this name is only a host-side stand-in for
// the device array, not a device address: it is never passed to a kernel.
static __device__ __align__(256) unsigned char g_sample_scratch[KNNM_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_sample_scratch on the current device.  Looked up on
// every call (cheap, allocates nothing once the library's device code is
// loaded), so an address never outlives a reset of the device's context.  The
// first lookup on a device loads the library's device code there, array
// included.
cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_sample_scratch);
  if (e != cudaSuccess) return e;
  *out = (unsigned char*)p;
  return cudaSuccess;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int knnm_step_sample_noalloc(void* cuda_stream, int64_t N, int K, const int32_t* ids,
                                        const float* dists, uint8_t* flags, uint64_t seed, int t,
                                        int s, int cap_new, int cap_old, int32_t* new_ids,
                                        int32_t* new_cnt, int32_t* old_ids, int32_t* old_cnt) {
  if (N < 1 || N > 0x7FFFFFFFLL || K < 1 || K > 32 || s < 1 || s > K || cap_new < 2 * s ||
      cap_old < K + s || !ids || !dists || !flags || !new_ids || !new_cnt || !old_ids || !old_cnt)
    return KNNM_ERR_INVALID;
  // N < 2^31 and K + 2s <= 96: the products below cannot overflow.
  const size_t keys_b = align256((size_t)N * K * 8);
  const size_t slots_b = align256((size_t)N * s * 8);
  const size_t need = keys_b + 2 * slots_b + align256(sizeof(DevCounters));
  if (need > (size_t)KNNM_NOALLOC_SCRATCH_BYTES) return KNNM_ERR_INVALID;  // too large

  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return KNNM_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  uint64_t* keys = (uint64_t*)base;
  uint64_t* rev_new = (uint64_t*)(base + keys_b);
  uint64_t* rev_old = (uint64_t*)(base + keys_b + slots_b);
  DevCounters* ctr = (DevCounters*)(base + keys_b + 2 * slots_b);

  // The array keeps the previous call's contents: reset what must start empty.
  if (cudaMemsetAsync(rev_new, 0xFF, (size_t)N * s * 8, st) != cudaSuccess) return KNNM_ERR_CUDA;
  if (cudaMemsetAsync(rev_old, 0xFF, (size_t)N * s * 8, st) != cudaSuccess) return KNNM_ERR_CUDA;
  if (cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st) != cudaSuccess) return KNNM_ERR_CUDA;
  if (launch_pack((int64_t)N * K, ids, dists, keys, st) != cudaSuccess) return KNNM_ERR_CUDA;
  SampleArgs sa;
  sa.N = N;
  sa.K = K;
  sa.s = s;
  sa.seed = seed;
  sa.t = t;
  sa.keys = keys;
  sa.flags = flags;
  sa.prev_keys = nullptr;
  sa.rev_new = rev_new;
  sa.rev_old = rev_old;
  sa.cap_new = cap_new;
  sa.cap_old = cap_old;
  sa.new_ids = new_ids;
  sa.new_cnt = new_cnt;
  sa.old_ids = old_ids;
  sa.old_cnt = old_cnt;
  sa.ctr = ctr;
  if (launch_sample(sa, st) != cudaSuccess) return KNNM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return KNNM_ERR_CUDA;
  return KNNM_OK;
}

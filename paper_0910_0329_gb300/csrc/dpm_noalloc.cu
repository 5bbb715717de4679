// dpm_noalloc.cu -- dpm_run_noalloc(): the persistent queue transport for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: a host program
// whose device memory is owned by a pool or arena that forbids further device
// allocation, a process working inside a fixed device-memory budget set at
// start-up, or a pipeline that must not add allocation latency or failure
// points to a dose request.  This entry point serves them: it runs the same
// queue kernel as dpm_run() with the same physics and random numbers, but its
// scratch (particle queues, run counters, error word) is a fixed file-scope
// device array, and the integer tally goes straight into a device buffer the
// caller owns.  It calls no cudaMalloc, cudaFree or other allocating routine.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dpm_ctx.h"
#include "dpm_internal.h"
#include "dpm_queue.h"

namespace dpm {
namespace {

// Scratch of dpm_run_noalloc(): particle queues plus a 256-byte header
// (run counters and the error word).  Every GPU that loads the library holds
// this array until the process exits.
constexpr size_t kNoAllocBytes = size_t(DPM_NOALLOC_SCRATCH_BYTES);
constexpr size_t kHeader = 256;
constexpr int kNoAllocLog2Slots = 9;  // 512 slots per queue shard

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// In host code g_noalloc_scratch is only a host-side stand-in; the device
// address is looked up once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

int scratch_address(int dev, void **out, std::string &err) {
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device index out of range";
    return DPM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return DPM_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return DPM_OK;
}

}  // namespace
}  // namespace dpm

using namespace dpm;

extern "C" int dpm_run_noalloc(dpm_ctx *c, int phantom_id, const dpm_source *src, uint64_t first_history,
                               uint64_t n_histories, uint64_t seed, int64_t *d_tally) {
  if (!c) return DPM_EINVAL;
  PhantomState *p = ctx_phantom(c, phantom_id);
  if (!p) return ctx_fail(c, DPM_EINVAL, "bad phantom id");
  if (!d_tally) return ctx_fail(c, DPM_EINVAL, "null tally");
  if (n_histories > 0x7fffffffull) return ctx_fail(c, DPM_EINVAL, "at most 2^31-1 histories per call");
  RunParams R{};
  int rc = ctx_run_params(c, p, src, first_history, n_histories, seed, 0, R);
  if (rc) return rc;
  if (n_histories == 0) return DPM_OK;
  if (cudaSetDevice(c->device) != cudaSuccess) return ctx_fail(c, DPM_ECUDA, "cudaSetDevice failed");

  // first call on this device: resolve the scratch array's device address
  void *base = nullptr;
  std::string err;
  if ((rc = scratch_address(c->device, &base, err))) return ctx_fail(c, rc, err);

  // shards that fit in the scratch, at most one per resident block
  const int per_sm = queue_blocks_per_sm();
  if (per_sm < 1) return ctx_fail(c, DPM_ECUDA, "occupancy query failed");
  int K = c->sm_count * per_sm;
  while (K > 1 && kHeader + queue_bytes(K, kNoAllocLog2Slots) > kNoAllocBytes) --K;
  if (kHeader + queue_bytes(K, kNoAllocLog2Slots) > kNoAllocBytes)
    return ctx_fail(c, DPM_ENOMEM, "scratch too small for one queue shard");

  // the header holds the run counters and the error word; both start at zero
  unsigned char *hdr = static_cast<unsigned char *>(base);
  if (cudaMemsetAsync(hdr, 0, kHeader, c->stream) != cudaSuccess) return ctx_fail(c, DPM_ECUDA, "memset failed");
  R.n_batches = 1;
  R.slabs = reinterpret_cast<unsigned long long *>(d_tally);  // one batch: the caller's tally
  R.counters = reinterpret_cast<unsigned long long *>(hdr);
  R.err = reinterpret_cast<int *>(hdr + 128);
  dpm_run_opts o{};
  if ((rc = queue_launch(hdr + kHeader, K, kNoAllocLog2Slots, R, n_histories, o, c->sm_count, c->stream, nullptr,
                         err)))
    return ctx_fail(c, rc, err);

  // wait, then report the device-side status of this call
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return ctx_fail(c, DPM_ECUDA, std::string("transport failed: ") + cudaGetErrorString(e));
  }
  int dev_err = 0;
  if (cudaMemcpy(&dev_err, hdr + 128, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return ctx_fail(c, DPM_ECUDA, "status read failed");
  if (dev_err & ERR_OVERFLOW) return ctx_fail(c, DPM_EQUEUE_OVERFLOW, "particle queue overflow in the fixed scratch");
  if (dev_err) return ctx_fail(c, DPM_ETIMEOUT, "a bounded device wait timed out");
  return DPM_OK;
}

// dpm_queue.h -- persistent transport kernel with device-wide particle queues.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "dpm_internal.h"

namespace dpm {

struct QueueState {
  void *mem = nullptr;     // one device allocation holding queues and control words
  size_t bytes = 0;
  int log2_cap = 0;
  uint64_t budget = 0;          // the owning context's device-memory budget (0 = none)
  uint64_t *in_use = nullptr;   // the owning context's bytes in use (the queues' included)
};

// Launch the persistent kernel for one run; returns a dpm_status code.
// `start` (may be NULL) is recorded on the stream just before the transport kernel.
int queue_run(QueueState &q, const RunParams &R, uint64_t batch_size, const dpm_run_opts &o, int sm_count,
              cudaStream_t st, cudaEvent_t start, std::string &err);
void queue_free(QueueState &q);

// Launch shape (K shards = blocks, 2^log2cs slots per shard) for the options,
// and the context's queue memory allocated for it.
int queue_prepare(QueueState &q, const dpm_run_opts &o, int sm_count, int &K, int &log2cs, std::string &err);

// Jobs one shared (batch) launch of the queue kernel takes: their step
// records are kept in shared memory.
constexpr int kSharedJobs = 64;

// A launch pauses refills that found nothing (dpm_run_opts.refill_pause = 0)
// when its work is at most kPauseMaxHistories 6 MV photon histories, an
// electron-beam history counting kElectronHistoryWeight (20 MeV electrons run
// at about an eighth of the 6 MV beam's histories/s).  The pause shortens the
// end of a launch by about 0.3 ms and costs about 1.5 % in between, so it
// pays below about 2x10^7 photon histories.
constexpr double kPauseMaxHistories = 1.6e7;
constexpr double kElectronHistoryWeight = 8.0;
// ... and only with shards of at least 2^kPauseMinLog2 slots: small queues
// (the no-allocation entry point's, or a small queue_log2) need every refill
// to keep the producers' shards from overflowing.
constexpr int kPauseMinLog2 = 13;

// Resident blocks per SM of the queue kernel (occupancy query), or 0 on error.
int queue_blocks_per_sm();
// Load the queue kernels on the current device now (they are otherwise
// loaded at their first launch under lazy module loading); returns
// queue_blocks_per_sm(), or 0 on error.
int queue_preload();
// Device bytes the queues of K shards of 2^log2cs slots occupy.
size_t queue_bytes(int K, int log2cs);
// Lay the queues out in caller-provided device memory `mem` (at least
// queue_bytes(K, log2cs) bytes, any alignment) and launch: allocates nothing.
int queue_launch(void *mem, int K, int log2cs, const RunParams &R, uint64_t batch_size, const dpm_run_opts &o,
                 int sm_count, cudaStream_t st, cudaEvent_t start, std::string &err);

}  // namespace dpm

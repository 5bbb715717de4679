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
};

// Launch the persistent kernel for one run; returns a dpm_status code.
// `start` is recorded on the stream just before the transport kernel.
int queue_run(QueueState &q, const RunParams &R, uint64_t batch_size, const dpm_run_opts &o, int sm_count,
              cudaStream_t st, cudaEvent_t start, std::string &err);
void queue_free(QueueState &q);

}  // namespace dpm

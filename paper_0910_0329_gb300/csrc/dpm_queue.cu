// dpm_queue.cu -- persistent transport kernel with particle queues.
#include "dpm_queue.h"

namespace dpm {

int queue_run(QueueState &q, const RunParams &R, uint64_t batch_size, const dpm_run_opts &o, int sm_count,
              cudaStream_t st, std::string &err) {
  (void)q; (void)R; (void)batch_size; (void)o; (void)sm_count; (void)st;
  err = "queue kernel not built yet";
  return DPM_EINVAL;
}

void queue_free(QueueState &q) {
  if (q.mem) cudaFree(q.mem);
  q.mem = nullptr;
  q.bytes = 0;
}

}  // namespace dpm

// k_mixed.cu -- mixed-precision path (placeholder until the kernels land).
#include <cuda_runtime.h>

#include "pcv_internal.h"

namespace pcv {
int64_t slot_bytes_mixed(int32_t ld, int64_t mmax) { return slot_bytes_fp64(ld, mmax); }
int mixed_prepare(int) { return 0; }
int launch_task_mixed(const TaskArgs&, int, void*) { return (int)cudaErrorNotSupported; }
}  // namespace pcv

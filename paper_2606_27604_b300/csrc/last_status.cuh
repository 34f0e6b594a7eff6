// last_status.cuh -- which workspace the last call on a stream used, so
// sss_last_device_status(stream) can read that call's status word.
#pragma once
#include <cuda_runtime.h>

namespace sss {

// Records that the latest status-writing call enqueued on `stream` keeps its
// status word at the start of `workspace` (thread-safe).
void note_last_workspace(cudaStream_t stream, const void* workspace);

// The workspace recorded for `stream`, or nullptr.
const void* last_workspace(cudaStream_t stream);

}  // namespace sss

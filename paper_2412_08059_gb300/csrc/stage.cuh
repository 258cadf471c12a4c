// Host-built tables to device memory without a host synchronisation.
//
// A copy from pageable host memory may wait for earlier work on the stream,
// and a pinned staging buffer would have to outlive the copy.  Here each
// launch of k_stage carries up to kStageChunk bytes of the table in its own
// parameter block: CUDA copies that block when the launch is enqueued, so the
// host buffer is free again when stage_to_device returns and the copy runs in
// stream order behind earlier work.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace mpcg {

// A kernel's parameters may take 32764 bytes; the chunk stays below that.
constexpr int kStageChunk = 32 * 1024 - 128;

struct StageChunk {
  char* dst;  // 16-byte aligned
  int bytes;  // 0 < bytes <= kStageChunk
  int pad;
  alignas(16) unsigned char data[kStageChunk];
};

// __grid_constant__ reads the parameter block in place (no local copy).
__global__ void k_stage(const __grid_constant__ StageChunk c);

// Copies `bytes` from host `src` to device `dst` (16-byte aligned) on `st`.
// Returns the first launch error, or cudaErrorInvalidValue for a misaligned
// destination.
cudaError_t stage_to_device(void* dst, const void* src, size_t bytes, cudaStream_t st);

}  // namespace mpcg

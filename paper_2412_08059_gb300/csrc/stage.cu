// Kernel-parameter staging of host-built tables (stage.cuh).
#include "stage.cuh"

namespace mpcg {

__global__ void k_stage(const __grid_constant__ StageChunk c) {
  const uint4* s = reinterpret_cast<const uint4*>(c.data);
  uint4* d = reinterpret_cast<uint4*>(c.dst);
  const int nv = c.bytes >> 4;
  const int stride = gridDim.x * blockDim.x;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = t; i < nv; i += stride) d[i] = s[i];
  for (int i = (nv << 4) + t; i < c.bytes; i += stride) c.dst[i] = (char)c.data[i];
}

cudaError_t stage_to_device(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if ((uintptr_t)dst & 15u) return cudaErrorInvalidValue;
  StageChunk c;  // 32 KB on the host stack; the launch copies it
  for (size_t off = 0; off < bytes; off += (size_t)kStageChunk) {
    const size_t n = bytes - off < (size_t)kStageChunk ? bytes - off : (size_t)kStageChunk;
    c.dst = (char*)dst + off;
    c.bytes = (int)n;
    c.pad = 0;
    memcpy(c.data, (const char*)src + off, n);
    const int blocks = (int)((n + 16 * 256 - 1) / (16 * 256));
    k_stage<<<blocks, 256, 0, st>>>(c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace mpcg

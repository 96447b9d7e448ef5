// Persistent ragged-batch kernel, FP32 storage.
#include "ragged.cuh"

namespace giga {
cudaError_t rag_launch_f32(const RagParams& p, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = set_smem_once<rag_kernel<float>>(rag_max_smem<float>());
  if (e != cudaSuccess) return e;
  rag_kernel<float><<<grid, kRagThreads, smem, st>>>(p);
  note_launch();
  return cudaGetLastError();
}
}  // namespace giga

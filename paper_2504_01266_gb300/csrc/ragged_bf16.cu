// Persistent ragged-batch kernel, BF16 storage (FP32 arithmetic).
#include "ragged.cuh"

namespace giga {
cudaError_t rag_launch_bf16(const RagParams& p, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = set_smem_once<rag_kernel<__nv_bfloat16>>(rag_max_smem<__nv_bfloat16>());
  if (e != cudaSuccess) return e;
  rag_kernel<__nv_bfloat16><<<grid, kRagThreads, smem, st>>>(p);
  note_launch();
  return cudaGetLastError();
}
}  // namespace giga

// Instantiates the fused strip kernels and the two-pass row kernels for bf16 input (one translation unit per
// input type so the variants compile in parallel).
#include "twopass_kernel.cuh"

namespace gb {
template gf_status launch_strip<__nv_bfloat16, float>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_strip<__nv_bfloat16, __nv_bfloat16>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_strip<__nv_bfloat16, __half>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_batch<__nv_bfloat16, float>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_batch<__nv_bfloat16, __nv_bfloat16>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_batch<__nv_bfloat16, __half>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_row_pass<__nv_bfloat16>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_row_pass_batch<__nv_bfloat16>(const TPRows&, int, int, size_t, cudaStream_t);
}  // namespace gb

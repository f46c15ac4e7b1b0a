// Instantiates the fused strip kernels and the two-pass row kernels for f32 input (one translation unit per
// input type so the variants compile in parallel).
#include "twopass_kernel.cuh"

namespace gb {
template gf_status launch_strip<float, float>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_strip<float, __nv_bfloat16>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_strip<float, __half>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_batch<float, float>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_batch<float, __nv_bfloat16>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_batch<float, __half>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_row_pass<float>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_row_pass_batch<float>(const TPRows&, int, int, size_t, cudaStream_t);
}  // namespace gb

// Instantiates the fused strip kernels and the two-pass row kernels for f16 input (one translation unit per
// input type so the variants compile in parallel).
#include "twopass_kernel.cuh"

namespace gb {
template gf_status launch_strip<__half, float>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_strip<__half, __nv_bfloat16>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_strip<__half, __half>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_batch<__half, float>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_batch<__half, __nv_bfloat16>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_batch<__half, __half>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_row_pass<__half>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_row_pass_batch<__half>(const TPRows&, int, int, size_t, cudaStream_t);
}  // namespace gb

// Instantiates the two-pass column kernels (one per output type).
#include "twopass_kernel.cuh"

namespace gb {
template gf_status launch_col_pass<float>(const CParams&, const CUtensorMap*, int, dim3, size_t, cudaStream_t, int);
template gf_status launch_col_pass_batch<float>(const TPCols&, int, int, int, size_t, cudaStream_t);
template gf_status launch_col_pass<__nv_bfloat16>(const CParams&, const CUtensorMap*, int, dim3, size_t, cudaStream_t, int);
template gf_status launch_col_pass_batch<__nv_bfloat16>(const TPCols&, int, int, int, size_t, cudaStream_t);
template gf_status launch_col_pass<__half>(const CParams&, const CUtensorMap*, int, dim3, size_t, cudaStream_t, int);
template gf_status launch_col_pass_batch<__half>(const TPCols&, int, int, int, size_t, cudaStream_t);
}  // namespace gb

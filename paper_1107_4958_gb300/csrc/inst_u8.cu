// Instantiates the fused strip kernels and the two-pass row kernels for u8 input (one translation unit per
// input type so the variants compile in parallel).
#include "twopass_kernel.cuh"

namespace gb {
template gf_status launch_strip<uint8_t, float>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_box_sums<uint8_t>(const unsigned char*, long long, int32_t*, long long, long long, int, int,
                                         int, int, int4, int, int, int, int, int, int, int, dim3, size_t, cudaStream_t);
template gf_status launch_batch<uint8_t, float>(const BatchArgs&, int, int, int, size_t, cudaStream_t);
template gf_status launch_row_pass<uint8_t>(const KParams&, const CUtensorMap*, dim3, size_t, cudaStream_t, int);
template gf_status launch_row_pass_batch<uint8_t>(const TPRows&, int, int, size_t, cudaStream_t);
}  // namespace gb

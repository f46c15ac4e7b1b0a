// Host-side device limits and layout helpers shared by the launch code of the
// fused and the two-pass filter.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstddef>

namespace gb {

struct DeviceInfo {
    int max_smem = 0;   // opt-in shared memory per CTA
    int sm_smem = 0;    // shared memory per SM
    int reserved = 0;   // shared memory the runtime reserves per CTA
    int sms = 0;
    int* status = nullptr;   // device status word
};
// Limits of the device current at the first call (queried once).
const DeviceInfo& device_info();

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();   // null if the driver lacks it
CUtensorMapDataType tma_dtype(int dt);
int round_up(int a, int b);
int chunk_for(int need);
int ctas_per_sm(size_t smem, int tmem_cols);
size_t pad_for_tmem(size_t smem, int tmem_cols);

}  // namespace gb

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
    int* status = nullptr;   // the library's status word on this device (null: no usable device)
    int device = -1;
};
// Limits of the current device (queried the first time the library works on
// it, then cached per device ordinal).
const DeviceInfo& device_info();

// Where the kernels a host thread launches report an expired wait, and how
// long they wait.  Calls made through a gf_handle set the handle's own status
// word and wait bound for their duration (HandleScope); the handle-less calls
// use the library's word on the current device and the default bound.
struct LaunchCtx {
    int* status = nullptr;    // null: the library's word on the current device
    long long wait = 0;       // SM clock cycles per pipeline wait; 0: the default
};
LaunchCtx& launch_ctx();      // this host thread's context
int* launch_status_word();
long long launch_wait_limit();
class HandleScope {
  public:
    HandleScope(int* status, long long wait) : saved_(launch_ctx()) { launch_ctx() = LaunchCtx{status, wait}; }
    ~HandleScope() { launch_ctx() = saved_; }
    HandleScope(const HandleScope&) = delete;
    HandleScope& operator=(const HandleScope&) = delete;

  private:
    LaunchCtx saved_;
};

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();   // null if the driver lacks it
CUtensorMapDataType tma_dtype(int dt);
int round_up(int a, int b);
int chunk_for(int need);
int ctas_per_sm(size_t smem, int tmem_cols);

// Staging geometry of a row piece of `span` elements whose scan needs a row
// stride of at least `min_row` elements: TMA boxes per row (nbox x boxw),
// the staged row stride SROW (a multiple of `srow_mult` elements), and, with
// `wide`, 8-byte TMA elements (xshift) and one box per band when a row is one
// box (rows8).  Fields of struct KParams (strip_kernel.cuh).
struct KParams;
void staging_geometry(KParams& kp, int span, int min_row, int srow_mult, int isz, bool wide);
// Encodes the row map and, when kp.rows8, the 8-row map of an image for the
// geometry in kp; false if the driver refuses either.
bool encode_row_maps(const KParams& kp, const void* base, size_t pitch, int rowlen, int H, int in_dt,
                     CUtensorMap* maps);
size_t pad_for_tmem(size_t smem, int tmem_cols);

}  // namespace gb

// 3D separable filtering of a stack of slices (Sec. 3.4: the running sums of
// Eq. alg1 and differences of Eq. indep applied along a third axis; 2 d k
// additions and d k multiplications per voxel for d = 3).
//
// The in-plane filter takes the path the plan of the whole stack (one image of
// D H rows) selects: the register walk, as one launch whose blockIdx.z is the
// slice; fused, as one persistent batch launch over the slices
// (graph-replayed when the same call repeats); or two-pass, as a row launch
// over all D H rows and a column launch over the slices (blockIdx.z).  Each
// writes an FP32 intermediate held by the handle.  The depth pass filters each
// (y, element column) line across the slices: for integer stacks with small
// depth radii one depth-walk launch (a thread per line, the running sums in
// registers), otherwise one column launch whose blockIdx.z walks the image
// rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "walker.h"

using namespace gb;

extern "C" {

gf_status gauss_filter_volume(gf_handle h, const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch, int D,
                              int H, int W, int C, int in_dtype, int out_dtype, const int32_t* radii,
                              const double* weights, int K, const int32_t* radii_z, const double* weights_z, int K_z,
                              int boundary, void* stream) {
    if (!h || D < 1 || H < 1 || W < 1) return GF_EINVAL;
    if ((long long)D * H > (long long)INT32_MAX / 4) return GF_EINVAL;
    if (H > 65535) return GF_EUNSUPPORTED;   // image rows are the depth launch's grid z
    if ((radii_z == nullptr) != (weights_z == nullptr)) return GF_EINVAL;
    // the whole stack as one image of D H rows: pitches, types, overlap
    Image whole;
    whole.in = d_in;
    whole.in_pitch = in_pitch;
    whole.out = d_out;
    whole.out_pitch = out_pitch;
    whole.H = D * H;
    whole.W = W;
    whole.C = C;
    whole.in_dt = in_dtype;
    whole.out_dt = out_dtype;
    whole.boundary = boundary;
    gf_status st = validate_image(whole);
    if (st != GF_OK) return st;
    BoxKernel bk, bz;
    st = make_box_kernel(radii, weights, K, &bk);
    if (st != GF_OK) return st;
    st = radii_z ? make_box_kernel(radii_z, weights_z, K_z, &bz) : make_box_kernel(radii, weights, K, &bz);
    if (st != GF_OK) return st;
    if (cudaSetDevice(h->device) != cudaSuccess) return GF_ECUDA;
    HandleScope scope(h->status_word, h->wait_cycles);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The plan of the stack seen as one image of D H rows: its tiles are sized
    // for the whole stack (a slice alone would get short row tiles, whose
    // vertical halo costs more), and its path decides the in-plane route.
    Image tall = whole;
    tall.out_dt = GF_F32;
    apply_tuned(h, tall, bk);
    FilterPlan fp;
    st = resolve_plan(tall, bk, &tall.plan, fp);
    if (st != GF_OK) return st;
    if (fp.path == GF_PATH_HBM) return GF_EUNSUPPORTED;   // radii beyond the shared-memory ring
    if (fp.path == GF_PATH_WALK && D > 65535) {   // slices are the walk's grid z
        if (tall.plan.path == GF_PATH_WALK) return GF_EUNSUPPORTED;
        fp.path = GF_PATH_FUSED;
    }
    const bool two = fp.path == GF_PATH_TWO_PASS;
    // in-plane result R: D H rows of r_pitch bytes (128-byte aligned rows);
    // the two-pass route also holds its row-pass intermediate
    const size_t r_pitch = ((size_t)W * C * 4 + 127) / 128 * 128;
    const size_t r_bytes = r_pitch * (size_t)D * (size_t)H;
    // a larger intermediate replaces the old one once earlier work is done
    // (cudaFree waits for the device)
    st = scratch_reserve(h->vol, two ? 2 * r_bytes : r_bytes, 0);
    if (st != GF_OK) return st;
    unsigned char* R = static_cast<unsigned char*>(h->vol.dev);
    if (fp.path == GF_PATH_WALK) {
        Image slice = whole;
        slice.H = H;
        slice.out = R;
        slice.out_pitch = r_pitch;
        slice.out_dt = GF_F32;
        st = launch_walker(slice, bk, s, 0, -1, D);
        if (st != GF_OK) return st;
        h->last_launches = 1;
    } else if (two) {
        st = launch_slices_twopass(tall, D, H, bk, fp.two, R + r_bytes, R, r_pitch, s);
        if (st != GF_OK) return st;
        h->last_launches = 2;
    } else {
        const gf_plan slice_plan = {GF_PATH_FUSED, fp.strip.TWp, std::min(fp.strip.TH, H), 0, 0, 0};
        std::vector<Image> ims(D);
        std::vector<BoxKernel> bks(D, bk);
        const size_t isl = (size_t)H * in_pitch;
        for (int z = 0; z < D; ++z) {
            Image& im = ims[z];
            im.in = static_cast<const unsigned char*>(d_in) + (size_t)z * isl;
            im.in_pitch = in_pitch;
            im.out = R + (size_t)z * H * r_pitch;
            im.out_pitch = r_pitch;
            im.H = H;
            im.W = W;
            im.C = C;
            im.in_dt = in_dtype;
            im.out_dt = GF_F32;
            im.boundary = boundary;
            im.plan = slice_plan;
        }
        st = launch_filter_batch(h, ims.data(), bks.data(), D, stream);
        if (st != GF_OK) return st;
    }
    // integer stacks bound |R| by the largest pixel times (sum_i |w_i| (2 r_i + 1))^2,
    // which fixes the depth walk's quantum; other stacks, and depth radii
    // beyond its register ring, take the column-pass kernel
    st = GF_EUNSUPPORTED;
    if ((in_dtype == GF_U8 || in_dtype == GF_U16) && out_dtype == GF_F32) {
        double S = 0.0;
        for (int i = 0; i < bk.K; ++i) S += std::fabs((double)bk.w[i]) * (2.0 * bk.r[i] + 1.0);
        const double maxpix = in_dtype == GF_U8 ? 255.0 : 65535.0;
        st = launch_depth_walk(reinterpret_cast<const float*>(R), r_pitch, D, H, W, C, d_out, out_pitch, boundary, bz,
                               maxpix * S * S, s);
    }
    if (st == GF_EUNSUPPORTED)
        st = launch_depth_pass(reinterpret_cast<const float*>(R), r_pitch, D, H, W, C, d_out, out_pitch, out_dtype,
                               boundary, bz, s);
    if (st != GF_OK) return st;
    h->last_launches += 1;
    return GF_OK;
}

}  // extern "C"

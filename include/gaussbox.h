/*
 * gaussbox.h - C ABI of the GB300 box-sum Gaussian filter.
 *
 * Method: Elboher & Werman, "Efficient and Accurate Gaussian Image Filtering
 * Using Running Sums".  Each 1D Gaussian is replaced by K centred boxes
 * ("weighted slices", Sec. 3.2) whose inclusive radii r_i and weights w_i come
 * from an exhaustive fit under a natural-image quadratic-form error (Sec. 4).
 * A row is filtered by a running sum I (Eq. alg1) and, per pixel,
 *     sum_i w_i (I(x + r_i) - I(x - r_i - 1))               (Eq. indep),
 * and the columns of that result the same way (Sec. 3.4).
 *
 * Conventions for every call:
 *  - Images are interleaved H x W x C (C channels per pixel, filtered
 *    independently), row-major, with a row pitch in BYTES (>= W*C*elem_size).
 *  - "d_" pointers are device pointers (cudaMalloc'd or equivalent) owned by
 *    the caller; "h_" pointers are host pointers owned by the caller.  The
 *    library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is enqueued asynchronously on it unless stated otherwise.
 *  - Every call returns a gf_status and never aborts the process.  Argument
 *    errors are detected on the host before anything is launched.
 *  - Kernels that contain bounded waits report an expired wait through a
 *    sticky device status word (gf_get_device_status), not by trapping.
 */
#ifndef GAUSSBOX_H
#define GAUSSBOX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GF_OK = 0,
    GF_EINVAL = 1,        /* bad argument (sizes, pitches, sigma, aliasing)       */
    GF_ENOMEM = 2,        /* a library-owned allocation failed                     */
    GF_ECUDA = 3,         /* a CUDA runtime/driver call failed                     */
    GF_ETIMEOUT = 4,      /* a bounded device wait expired (see device status)     */
    GF_EUNSUPPORTED = 5,  /* K outside 1..5, dtype pair not offered, no device     */
    GF_EADMIT = 6,        /* request larger than the server's HBM budget           */
    GF_EBUSY = 7,         /* server queue full / ticket not finished yet           */
    GF_ELIMIT = 8         /* request exceeds a fixed capacity of the call          */
} gf_status;

typedef enum { GF_U8 = 0, GF_U16 = 1, GF_F32 = 2, GF_BF16 = 3, GF_F16 = 4 } gf_dtype;

/* Pixels outside the image (the paper does not fix this):
 * REPLICATE repeats the edge pixel, ZERO reads 0, REFLECT mirrors about the
 * edge pixel without repeating it (folded again when the radius exceeds the
 * image). */
typedef enum { GF_REPLICATE = 0, GF_ZERO = 1, GF_REFLECT = 2 } gf_boundary;

/* Kernel-approximation error of the fit: the quadratic form of Sec. 4.1
 * (natural-image prior, the paper's proposal) or plain l2 (A = identity, the
 * paper's "second set of parameters", Sec. 5). */
typedef enum { GF_ERR_QF = 0, GF_ERR_L2 = 1 } gf_err_kind;

#define GF_KMAX 5

/* ------------------------------------------------------------------------ */
/* Fit (host only, never touches the GPU)                                    */
/* ------------------------------------------------------------------------ */

/*
 * gauss_fit_boxes - radii and weights of the K-box approximation at `sigma`.
 *
 * Sec. 4.2 + Eq. scale1 / Eq. scale2: an exhaustive search at sigma0 = 100/pi
 * over all inclusive radii 0 <= p_1 < ... < p_K <= 99 of the sampled Gaussian
 * (integer t = -100..99) under the chosen error, weights by closed-form
 * generalised least squares; then r_i = floor(sigma*pi*p_i/100) and
 * w_i(sigma) = p_i/(2 r_i + 1) * w_i, divided by sum_i w_i(sigma)(2 r_i + 1)
 * so that a constant image is preserved.  The search runs once per (K, err)
 * per process (a fraction of a second for K = 5) and is cached.
 *
 *   sigma        > 0 and finite
 *   K            1..5 (GF_EUNSUPPORTED otherwise)
 *   err_kind     gf_err_kind
 *   radii_out    caller array of K int32: inclusive radii, non-decreasing
 *                (equal radii and 0 are legal for small sigma)
 *   weights_out  caller array of K doubles: normalised slice weights
 * Thread-safe.
 */
gf_status gauss_fit_boxes(double sigma, int K, int err_kind, int32_t* radii_out,
                          double* weights_out);

/*
 * gauss_fit_sigma0 - the unscaled fit itself (Table 1): inclusive radii p_i
 * and segment constants c_i = sum_{j>=i} w_j at sigma0, plus the residual
 * error.  Any output pointer may be NULL.
 */
gf_status gauss_fit_sigma0(int K, int err_kind, int32_t* p_out, double* c_out,
                           double* w_out, double* err_out);

/*
 * gauss_fit_kernel - K weighted slices approximating an arbitrary symmetric
 * kernel (Sec. 3.2: a symmetric kernel is approximated on [0, r] and mirrored;
 * Sec. 4: the same exhaustive search and error as the Gaussian fit).
 *
 *   half         host array of n samples: the kernel at t = 0, 1, ..., n - 1
 *                (g(-t) = g(t); zero for |t| >= n on the search grid t = -100..99)
 *   n            1..101
 *   K            1..5 (GF_EUNSUPPORTED otherwise)
 *   err_kind     GF_ERR_QF (natural-image quadratic form) or GF_ERR_L2
 *   radii_out    caller array of K int32: increasing inclusive radii in 0..99
 *   weights_out  caller array of K doubles: the optimal slice weights, not
 *                normalised (a kernel summing to 1 gives sum w_i (2 r_i + 1)
 *                close to 1; the filter calls use the weights as given)
 *   err_out      residual error of the fit, or NULL
 * Host only, thread-safe; every call runs the search (well under a second for
 * K = 5 on a few cores).  GF_EINVAL for a non-finite sample.
 */
gf_status gauss_fit_kernel(const double* half, int n, int K, int err_kind, int32_t* radii_out,
                           double* weights_out, double* err_out);

/* ------------------------------------------------------------------------ */
/* Filtering                                                                 */
/* ------------------------------------------------------------------------ */

/*
 * gauss_filter - separable box-sum Gaussian filter of one image (Sec. 3.3-3.4).
 *
 *   d_in, in_pitch     input image, in_dtype elements, H x W x C, pitch in bytes
 *   d_out, out_pitch   output image, out_dtype elements, same H x W x C
 *   H, W, C            H >= 1, W >= 1, C in 1..4
 *   in_dtype           GF_U8, GF_U16 (exact integer running sums),
 *                      GF_F32, GF_BF16, GF_F16 (FP32 arithmetic)
 *   out_dtype          GF_F32 for any input; GF_BF16 / GF_F16 for float inputs
 *   sigma, K           as gauss_fit_boxes with GF_ERR_QF
 *   boundary           gf_boundary
 *   stream             cudaStream_t
 *
 * Rows then columns.  Every box sum is accurate to its own magnitude,
 * whatever the values elsewhere in the row or column: uint8 rows are summed
 * exactly in FP32 (every partial sum is an integer below 2^24), uint16 rows
 * exactly in int32; a float value f is split into f_h, the nearest multiple of
 * a power of two q chosen per staged row, and the exact residue f - f_h, the
 * f_h / q summed exactly in int32 and the residues (at most q / 2) in FP32.
 * Each column running sum is carried as an FP32 sum plus the exact rounding
 * errors of its additions (TwoSum), so a difference of two running sums is
 * the difference of the sums plus that of the error terms, each rounded to
 * its own size.  Single-channel integer images with radii up to 22 take the
 * register walk (GF_PATH_WALK), whose column sums are an exact part on a
 * power-of-two grid plus FP32 residues.
 * Inputs must be finite: a NaN or infinity makes the outputs whose windows
 * reach it unspecified (they need not be NaN).
 * d_in and d_out must not overlap (GF_EINVAL).  Asynchronous on `stream`.
 *
 * Two execution paths compute the same sums (gf_plan): the fused strip
 * kernel, which allocates nothing, and the two-pass form (a row launch that
 * writes an H x W x C FP32 intermediate, then a column launch), chosen for
 * large radii; its intermediate comes from a stream-ordered memory pool of
 * the library (cudaMallocFromPoolAsync / cudaFreeAsync on `stream`; the pool
 * keeps freed memory for reuse).
 */
gf_status gauss_filter(const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch,
                       int H, int W, int C, int in_dtype, int out_dtype, double sigma, int K,
                       int boundary, void* stream);

/*
 * gauss_filter_boxes - as gauss_filter with explicit inclusive radii (each
 * 0..4096) and slice weights (Eq. indep with caller-chosen w_i, r_i; the
 * weights are used as given, rounded to FP32).
 *
 * Large radii: the column pass keeps the running sums (high and low parts) of
 * 2 r_K + 1 rows of a 32-column strip in shared memory, which holds r_K up to
 * about 400 on GB300 (227 KB per CTA; sigma up to ~150 with the fitted
 * kernels).  Beyond that the
 * single-image calls on their default plan (this one, gauss_filter,
 * gauss_filter_sampled, gauss_filter_host) keep the running sums in HBM
 * instead (GF_PATH_HBM: int64 prefixes of each boundary-extended line, any
 * radius up to 4096, about 4x slower than the two-pass form); explicit
 * two-pass plans, batches, the server and volumes return GF_EUNSUPPORTED
 * before launching anything.
 */
gf_status gauss_filter_boxes(const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch,
                             int H, int W, int C, int in_dtype, int out_dtype,
                             const int32_t* radii, const double* weights, int K, int boundary,
                             void* stream);

/*
 * gauss_row_box_sums - the integer part of the row pass alone: for every pixel
 * and channel the K box sums B_i = I(x + r_i) - I(x - r_i - 1) along the row
 * (Eq. alg1 and the differences of Eq. indep, without the weights), computed
 * by the same tile-local int32 running sums the filter uses.
 *
 *   d_in, in_pitch   GF_U8 or GF_U16 image, H x W x C
 *   d_out            int32 output, K planes; plane i starts at
 *                    d_out + i * plane_stride_elems, rows of W*C int32 with a
 *                    pitch of out_pitch bytes inside each plane
 *   radii            host array of K inclusive radii (0..4096)
 * Exact (bit-for-bit the integer box sums) for any image width.
 */
gf_status gauss_row_box_sums(const void* d_in, size_t in_pitch, int32_t* d_out, size_t out_pitch,
                             size_t plane_stride_elems, int H, int W, int C, int in_dtype,
                             const int32_t* radii, int K, int boundary, void* stream);

/*
 * Execution plan of one image.  Both paths compute the same running sums and
 * differences (Sec. 3.3-3.4); they differ in how the work is tiled.
 *   GF_PATH_FUSED     one launch; a CTA owns a strip of tile_w pixels by tile_h
 *                     output rows and redoes the row pass on a halo of rk
 *                     pixels left/right and rk rows above/below.
 *   GF_PATH_TWO_PASS  a row launch (segments of tile_w pixels, tile_h rows per
 *                     CTA) writes an FP32 intermediate; a column launch (col_w
 *                     element columns by col_h output rows per CTA) filters
 *                     its columns.  Halo work only along each pass's own axis,
 *                     for 8 extra bytes of HBM traffic per element.
 *   GF_PATH_HBM       running sums of whole boundary-extended lines kept in HBM
 *                     as int64 (row prefix, row gather, column prefix in
 *                     chunks, column gather): any radius, several times the
 *                     traffic of the two-pass form.  GF_PATH_AUTO takes it when
 *                     the two-pass working set does not fit shared memory (the
 *                     largest radius beyond ~400 on GB300).  Tile fields are
 *                     ignored; single-image calls only (batches, the server and
 *                     volumes return GF_EUNSUPPORTED for it).
 *   GF_PATH_WALK      single-channel uint8 / uint16 images with FP32 output and
 *                     a largest radius of at most 22: one launch of a kernel
 *                     compiled at run time (NVRTC) for the image's radii, in
 *                     which each thread walks a row, then a column, of a
 *                     128-column strip keeping the running sums of its line in
 *                     registers; the column running sums are carried as an
 *                     exact part plus a residue.  The first call for a radius
 *                     set compiles the kernel (about a second) and caches it for
 *                     the process.  GF_PATH_AUTO takes it for every image it
 *                     accepts; tile fields are ignored.  Single-image calls
 *                     only: batches, the server and volumes run such images on
 *                     the fused kernel (an explicit GF_PATH_WALK there is
 *                     GF_EUNSUPPORTED).
 * A zero field means "the library's default for this field".
 */
typedef enum { GF_PATH_AUTO = 0, GF_PATH_FUSED = 1, GF_PATH_TWO_PASS = 2, GF_PATH_HBM = 3,
               GF_PATH_WALK = 4 } gf_path;
/* Accumulation of float inputs (integer inputs are always exact):
 *   GF_ACCUM_COMPENSATED  the default: rows as exact int32 sums of values
 *                         rounded to a power-of-two grid plus FP32 sums of the
 *                         residues; columns as FP32 sums plus the exact
 *                         rounding errors of their additions
 *   GF_ACCUM_OFFSET       FP32 rows and columns: per-tile offsets, plain FP32 carries
 *   GF_ACCUM_PLAIN        plain FP32 running sums from the tile start
 * The last two exist for the precision study and run on the two-pass path
 * only (GF_PATH_AUTO then means two-pass; GF_PATH_FUSED is GF_EUNSUPPORTED). */
typedef enum { GF_ACCUM_COMPENSATED = 0, GF_ACCUM_OFFSET = 1, GF_ACCUM_PLAIN = 2 } gf_accum;
typedef struct {
    int path;     /* gf_path                                                        */
    int tile_w;   /* fused: strip width (pixels; <= 256 / C); two-pass: row segment */
    int tile_h;   /* fused: output rows per CTA; two-pass: rows per row-pass CTA     */
    int col_w;    /* two-pass: element columns per column CTA: 32, 64, 128 or 256    */
    int col_h;    /* two-pass: output rows per column CTA                           */
    int accum;    /* gf_accum                                                       */
} gf_plan;

/*
 * gauss_plan_default - the plan gauss_filter would use for this image (every
 * field filled in).  radii: host array of K inclusive radii.  Host only.
 */
gf_status gauss_plan_default(int H, int W, int C, int in_dtype, int out_dtype, const int32_t* radii, int K,
                             gf_plan* out);

/*
 * gauss_filter_planned - gauss_filter_boxes with an explicit plan (NULL = the
 * default).  GF_EINVAL for a plan field out of range or a plan with more than
 * 65535 row tiles in one launch, GF_EUNSUPPORTED for a plan whose working set
 * does not fit the device.
 */
gf_status gauss_filter_planned(const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch,
                               int H, int W, int C, int in_dtype, int out_dtype,
                               const int32_t* radii, const double* weights, int K, int boundary,
                               const gf_plan* plan, void* stream);

/*
 * gauss_walker_compile - compiles (or finds in the process cache) the kernels
 * GF_PATH_WALK runs for an image, or a volume's slices, of `in_dtype` (GF_U8
 * or GF_U16) filtered with the inclusive radii `radii[0..K-1]` (largest at
 * most 22), without launching
 * anything and without needing a device: a warm-up before timing, or a check
 * that the run-time compiler works.  GF_EUNSUPPORTED for inputs the path does
 * not take, GF_ECUDA if the compiler fails; the compiler's log is copied to
 * `log` (NUL-terminated, truncated to log_len bytes) when log is non-NULL.
 * Thread-safe.
 */
gf_status gauss_walker_compile(int in_dtype, const int32_t* radii, int K, char* log, size_t log_len);

/*
 * gauss_depth_walker_compile - compiles (or finds in the process cache) the
 * depth walk that gauss_filter_volume runs along the slices of a u8/u16 stack
 * whose depth radii `radii[0..K-1]` are at most 10 (Sec. 3.4: the running sums
 * of Eq. alg1 and the differences of Eq. indep along the third axis), without
 * launching anything and without needing a device.  GF_EUNSUPPORTED for radii
 * the walk does not take, GF_ECUDA if the compiler fails; the log as for
 * gauss_walker_compile.  Thread-safe.
 */
gf_status gauss_depth_walker_compile(const int32_t* radii, int K, char* log, size_t log_len);

/*
 * gauss_filter_sampled - the filter evaluated on a regular grid of pixels
 * only, e.g. for downscaling (Sec. 3.4: Eq. indep needs nothing but the
 * running sum at x + r_i and x - r_i - 1, so any subset of the responses can
 * be taken from one running sum per row and column):
 *
 *   out(i, j, c) = Y(off_y + i step_y, off_x + j step_x, c),
 *   i < Ho = ceil((H - off_y) / step_y),  j < Wo = ceil((W - off_x) / step_x),
 *
 * Y being the output of gauss_filter_boxes on the same arguments.
 *   step_y, step_x    >= 1
 *   off_y, off_x      0 <= off_y < min(step_y, H), 0 <= off_x < min(step_x, W)
 *   d_out, out_pitch  Ho x Wo x C out_dtype elements; pitch >= Wo C element bytes
 *   plan              NULL (default) or a GF_PATH_AUTO / GF_PATH_TWO_PASS plan
 * Runs on the two-pass path: the row launch takes running sums over every
 * pixel and differences at the sampled columns only, into an H x Wo x C FP32
 * intermediate (the library's stream-ordered pool); the column launch stores
 * the sampled rows only.  With the two-pass plan the full filter would use
 * (the same gf_plan), every output equals that filter's pixel bit for bit.
 * GF_EUNSUPPORTED for a GF_PATH_FUSED plan, GF_EINVAL for bad steps/offsets.
 */
gf_status gauss_filter_sampled(const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch,
                               int H, int W, int C, int in_dtype, int out_dtype,
                               const int32_t* radii, const double* weights, int K, int boundary,
                               int step_y, int step_x, int off_y, int off_x, const gf_plan* plan,
                               void* stream);

/* ------------------------------------------------------------------------ */
/* Handles, batches                                                          */
/* ------------------------------------------------------------------------ */

/* Library context: device scratch for batches (work lists, per-image
 * parameters and TMA descriptors), a CUDA-graph cache, the tile-plan tuner
 * cache and the serving state.  Not thread-safe: one host thread per handle. */
typedef struct gf_handle_s* gf_handle;

typedef struct {
    int device;                 /* CUDA device ordinal the handle works on          */
    size_t hbm_budget_bytes;    /* serving admission budget (0 = 50 % of free HBM)   */
    int use_graphs;             /* batches replay captured CUDA graphs (1) or launch */
    const char* tune_cache;     /* tile-plan cache file (JSON) or NULL               */
    long long wait_cycles;      /* bound of every pipeline wait of the handle's      */
                                /* kernels, in SM clock cycles (0 = the default,     */
                                /* about 2 s; a few cycles make the waits expire,    */
                                /* for testing the GF_ETIMEOUT path); >= 0           */
} gf_config;

/* Creates a handle on cfg->device (cfg == NULL: current device, defaults).
 * With cfg->tune_cache set, plans tuned earlier on the same kind of device
 * are loaded from that file (a missing file is not an error).  The handle
 * owns a device status word of its own (gf_handle_status): every kernel
 * launched through the handle (batches, volumes, host-buffer calls, the
 * tuner, the server) reports an expired wait there and nowhere else. */
gf_status gf_create(gf_handle* h, const gf_config* cfg);
/* Frees the handle's device memory, graphs and server state.  NULL is a no-op. */
gf_status gf_destroy(gf_handle h);

/* One image of a batch; buffers as for gauss_filter.  If radii and weights are
 * both non-NULL they are the K explicit boxes (sigma ignored), else the boxes
 * are fitted from sigma and K (quadratic-form error).  plan: NULL (or an
 * all-zero gf_plan) = the default plan of gauss_filter; read during the call. */
typedef struct {
    const void* d_in;
    size_t in_pitch;
    void* d_out;
    size_t out_pitch;
    int H, W, C;
    int in_dtype, out_dtype;
    double sigma;
    int K;
    int boundary;
    const int32_t* radii;
    const double* weights;
    const gf_plan* plan;
} gf_image_desc;

/*
 * gauss_filter_batch - filters n independent images in one persistent launch
 * per type class (input dtype, output dtype, channels, strip width).
 *
 * Every image keeps the plan it would get from gauss_filter (a function of its
 * own size, channels, dtypes and radii only) or the one its descriptor names,
 * so each output is bit-identical to filtering that image alone with that
 * plan.  Fused images are grouped into classes (kernel instantiation and
 * on-chip footprint), one persistent launch per class whose CTAs take tiles
 * from an atomic ticket.  Two-pass images of the default accumulation are
 * grouped the same way, by row kernel and column kernel, at most 32 images a
 * class: one row launch and one column launch per class, one CTA per tile,
 * intermediates in the handle's scratch; an image in a study accumulation
 * mode gets its own two launches, a register-walk image its own launch.  The
 * launches of different classes and images run concurrently on side streams
 * of the handle, joined back into `stream`.  With cfg->use_graphs the launch sequence is captured
 * once per batch signature (plans, sizes, two-pass buffers) and replayed.
 *   images  host array of n descriptors (copied during the call)
 * Asynchronous on `stream`; uses the handle's scratch (grown on demand:
 * GF_ENOMEM if that fails).  Output buffers must not overlap any input.
 */
gf_status gauss_filter_batch(gf_handle h, const gf_image_desc* images, int n, void* stream);

/*
 * gauss_filter_volume - 3D separable filter of a stack of D slices (Sec. 3.4:
 * the running sums and differences of Eq. alg1 / Eq. indep along a third
 * axis).  Each slice is filtered in-plane with (radii, weights, K) as an
 * image of its own (rows fold within the slice), then every line of D voxels
 * at a fixed (y, x, c) with (radii_z, weights_z, K_z) (both NULL: the
 * in-plane kernel; anisotropic voxels take their own depth kernel).
 *
 *   d_in, in_pitch     slice z, row y starts at d_in + (z H + y) in_pitch
 *   d_out, out_pitch   the same layout, out_dtype elements
 *   D, H, W, C         D >= 1, 1 <= H <= 65535, W >= 1, C in 1..4
 *   in/out dtypes, boundary   as gauss_filter (the boundary rule applies on all axes)
 *
 * The in-plane results go to an FP32 intermediate of D H rows held by the
 * handle (grown on demand; growing it waits for the device).  The plan of the
 * stack seen as one image of D H rows picks the in-plane route: one register
 * walk launch over all slices (single-channel u8/u16, radii up to 22), the
 * batch launcher of gauss_filter_batch (plans, graph replay), or one row and
 * one column launch.  The depth pass is one launch: a walk along the slices
 * for u8/u16 stacks with depth radii up to 10, else a column launch over all
 * image rows.  Asynchronous on
 * `stream`; the handle's batch rules apply (one host thread per handle; the
 * next batch or volume call waits until this one's staging is consumed).
 */
gf_status gauss_filter_volume(gf_handle h, const void* d_in, size_t in_pitch, void* d_out, size_t out_pitch,
                              int D, int H, int W, int C, int in_dtype, int out_dtype,
                              const int32_t* radii, const double* weights, int K,
                              const int32_t* radii_z, const double* weights_z, int K_z,
                              int boundary, void* stream);
/* Kernel launches the handle's last gauss_filter_batch enqueued (one per fused
 * class, two per two-pass image); -1 for a NULL handle. */
int gf_batch_launches(gf_handle h);

/*
 * gauss_filter_host - gauss_filter on HOST images: copies h_in to device
 * buffers owned by the handle (grown on demand), filters, copies the result to
 * h_out and waits for it.  Pinned host memory (cudaMallocHost) gives full
 * host-device bandwidth; pageable memory works too.  Pitches as gauss_filter.
 * Returns when h_out holds the result.
 */
gf_status gauss_filter_host(gf_handle h, const void* h_in, size_t in_pitch, void* h_out, size_t out_pitch,
                            int H, int W, int C, int in_dtype, int out_dtype, double sigma, int K,
                            int boundary, void* stream);

/*
 * gauss_filter_batch_noalloc - gauss_filter_batch for callers that cannot
 * allocate device memory.  The paper has no counterpart: this is an interface
 * choice of the library.
 *
 * Who needs it: code that owns no allocator or may not use one while it runs
 * - a plug-in whose host application hands out all device buffers, a server
 * that carves up HBM once at start-up and forbids later cudaMalloc calls, or
 * a latency-critical path where an allocation (and the implicit device
 * synchronisation cudaFree brings) is not acceptable.  Such callers pass in
 * the input and output images as usual; the call itself allocates nothing:
 * no cudaMalloc, cudaFree or pinned host memory.
 *
 * Its scratch (per-image kernel parameters, TMA descriptors, tile prefix sums,
 * ticket counters) is a fixed array of GF_NOALLOC_SCRATCH_BYTES compiled into
 * the library; every device that loads the library holds one copy until the
 * process exits.
 *   - At most GF_NOALLOC_MAX_IMAGES images per call, and the planned scratch
 *     must fit the array: larger requests return GF_ELIMIT and launch nothing.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current).  Make that first call before any
 *     stream capture.
 *   - Every call shares the one array and leaves its contents behind; each
 *     call rewrites what it uses and resets its ticket counters to zero.
 *     Calls whose GPU work overlaps (e.g. on two streams at once) race on the
 *     array: issue them on one stream, or wait for one before starting the
 *     next.
 *   - sigma-based descriptors run the one-time host fit of each K on first use;
 *     descriptors with explicit radii/weights avoid it.
 *   - The call returns GF_EUNSUPPORTED, and enqueues nothing, while `stream`
 *     is being captured into a CUDA graph: its parameters reach the device by
 *     a copy from library-owned host storage that the next call rewrites.
 * Every image runs on the fused path (the two-pass path needs an
 * intermediate buffer): a descriptor whose plan asks for GF_PATH_TWO_PASS, or
 * for an accumulation mode other than GF_ACCUM_COMPENSATED (those exist on
 * the two-pass path only), is GF_EUNSUPPORTED; one with no plan or
 * GF_PATH_AUTO gets the default fused tile plan.  Results are bit-identical
 * to gauss_filter_batch and to gauss_filter_planned given the same fused
 * plans.
 */
#define GF_NOALLOC_MAX_IMAGES 64
#define GF_NOALLOC_SCRATCH_BYTES (64 * 1024)
gf_status gauss_filter_batch_noalloc(const gf_image_desc* images, int n, void* stream);

/*
 * gf_tune - the plan autotuner.  Times the default plan and variants of both
 * paths (fused: strip width, rows per CTA; two-pass: row segment width, rows
 * per row CTA, column strip width, column rows per CTA; coordinate descent
 * from each path's default) on the image `img` describes, with CUDA events on
 * `stream` (the call is synchronous; img->d_out is overwritten), and records
 * the fastest plan for the image's shape class: input/output dtype, C, K and
 * half-octave buckets of H, W and the largest radius.  With a tune_cache file
 * the table is rewritten after every call.
 *   best   out: the chosen plan (may be NULL)
 * From then on gauss_filter_batch, gauss_filter_host and the server use the
 * tuned plan for every image of that class whose descriptor names no plan;
 * each result is then bit-identical to gauss_filter_planned with that plan.
 * gf_tuned_plan reports the plan recorded for an image's class (GF_EINVAL if
 * none).
 */
gf_status gf_tune(gf_handle h, const gf_image_desc* img, void* stream, gf_plan* best);
gf_status gf_tuned_plan(gf_handle h, const gf_image_desc* img, gf_plan* out);

/* ------------------------------------------------------------------------ */
/* Serving                                                                   */
/* ------------------------------------------------------------------------ */

/*
 * Continuous-batching server on a handle.  Requests are device-resident
 * images (d_in/in_pitch of a gf_image_desc; its d_out/out_pitch are ignored):
 * the server gives each one an output buffer from an HBM arena of
 * hbm_budget_bytes (the admission budget), so a request is admitted only when
 * it has been released (its release time has passed) and its output fits.
 * Admitted requests are packed into steps of at most max_batch images (one
 * persistent launch per type class, as gauss_filter_batch) issued round-robin
 * on max_inflight streams, so steps overlap on the device while later
 * requests keep arriving.  Completion is observed through CUDA events.  Each
 * result is bit-identical to gauss_filter on the same image.  In plain mode
 * every request is its own gauss_filter launch on one stream instead (the
 * per-image baseline).  The server runs a host thread; all calls below are
 * thread-safe with respect to it.
 */
typedef struct {
    size_t hbm_budget_bytes;   /* arena for outputs (0 = the handle's budget, else half the free HBM) */
    int max_batch;             /* requests per step (0 = 64)                    */
    int max_inflight;          /* steps in flight = streams (0 = 4)             */
    int plain;                 /* 1 = one gauss_filter launch per request        */
} gf_server_config;

typedef struct {
    void* d_out;               /* output buffer in the arena (valid until released) */
    size_t out_pitch;
    double t_release, t_admit, t_done;   /* gf_clock_now() seconds               */
    int status;                /* GF_OK, or the launch error                    */
} gf_completion;

typedef struct {
    long long submitted, completed, rejected, steps;
    double sum_batch;          /* sum of step sizes (mean batch = sum_batch / steps) */
    size_t arena_bytes, arena_peak;
    double busy_first_release, busy_last_done;
    long long launches;        /* kernel launches of all steps                   */
} gf_server_stats;

/* Host monotonic clock in seconds (the clock of release and completion times). */
double gf_clock_now(void);

gf_status gf_server_start(gf_handle h, const gf_server_config* cfg);
/* Queues one request, released at release_time (<= 0: now).  If auto_release
 * is non-zero the output buffer returns to the arena as soon as the request
 * completes (timing-only clients).  GF_EADMIT if the output alone exceeds the
 * arena.  *ticket identifies the request. */
gf_status gf_server_submit(gf_handle h, const gf_image_desc* req, double release_time, int auto_release,
                           long long* ticket);
/* GF_OK and *out filled once the request completed, GF_EBUSY before. */
gf_status gf_server_poll(gf_handle h, long long ticket, gf_completion* out);
/* Blocks until the request completed (or timeout_s elapsed: GF_ETIMEOUT). */
gf_status gf_server_wait(gf_handle h, long long ticket, double timeout_s, gf_completion* out);
/* Returns a completed request's output buffer to the arena and forgets it. */
gf_status gf_server_release(gf_handle h, long long ticket);
/* Blocks until every submitted request completed (or timeout: GF_ETIMEOUT). */
gf_status gf_server_drain(gf_handle h, double timeout_s);
gf_status gf_server_stats_get(gf_handle h, gf_server_stats* out);
/* Drains and stops the server thread; frees the arena. */
gf_status gf_server_stop(gf_handle h);

/* ------------------------------------------------------------------------ */
/* Device status                                                             */
/* ------------------------------------------------------------------------ */

/* Reads (and, if clear != 0, resets) the sticky status word that the
 * handle-less calls (gauss_filter, gauss_filter_boxes, gauss_filter_planned,
 * gauss_filter_sampled, gauss_row_box_sums, gauss_filter_batch_noalloc) set
 * on the current device when a bounded wait of their kernels expires: GF_OK
 * or GF_ETIMEOUT.  Each device has its own word; handles have their own
 * (gf_handle_status), which this call neither reads nor clears.  Waits for
 * the device to finish its work first. */
gf_status gf_get_device_status(int clear);

/* The same for the status word of handle h (the kernels launched through
 * it): GF_OK or GF_ETIMEOUT, reset to GF_OK if clear != 0; GF_EINVAL for a
 * NULL handle.  Waits for the handle's device to finish its work first. */
gf_status gf_handle_status(gf_handle h, int clear);

/* Human-readable name of a status code (static string). */
const char* gf_status_string(int status);

/* Library version string (static). */
const char* gf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GAUSSBOX_H */

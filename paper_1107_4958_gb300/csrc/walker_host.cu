// Host side of the register-walk fused filter (walker_kernel.cuh): which images
// it takes, the compilation of the kernel for a radius set at run time (NVRTC,
// cached per process), the tile plan, the column quantum and the launch.
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "walker.h"

// The text of walker_kernel.cuh and depth_walker.cuh, embedded into the
// library when it is built.
extern "C" const char gb_walker_source[];
extern "C" const char gb_depth_walker_source[];

namespace gb {

static_assert(sizeof(WalkMap) == sizeof(CUtensorMap) && alignof(WalkMap) >= 64, "tensor map size");

namespace {

int in_bytes(int in_dt) { return in_dt == GF_U8 ? 1 : 2; }

// A compiled kernel for one (input type, radii) set.
struct WalkerEntry {
    std::vector<char> cubin;
    std::string log;
    gf_status st = GF_OK;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    unsigned long long smem_set = 0;   // devices whose shared-memory limit was raised (bit per ordinal < 64)
};

std::mutex g_mu;
std::map<std::string, std::unique_ptr<WalkerEntry>> g_cache;

std::string key_of(int in_dt, const BoxKernel& bk, bool stack) {
    char buf[96];
    std::snprintf(buf, sizeof(buf), "%d:%d:%d,%d,%d,%d,%d:%d", in_dt, bk.K, bk.r[0], bk.r[1], bk.r[2], bk.r[3], bk.r[4],
                  stack ? 1 : 0);
    return buf;
}

// NVRTC compilation of walker_kernel.cuh with the radii as constants (stack:
// the variant whose blockIdx.z is the slice of a stack).
gf_status compile(int in_dt, const BoxKernel& bk, const WalkerGeom& g, bool stack, WalkerEntry& e) {
    std::string src;
    char line[320];
    std::snprintf(line, sizeof(line), "#define WK_IN %d\n#define WK_K %d\n#define WK_Z %d\n", in_dt == GF_U8 ? 0 : 1,
                  bk.K, stack ? 1 : 0);
    src += line;
    for (int i = 0; i < GF_KMAX; ++i) {
        std::snprintf(line, sizeof(line), "#define WK_R%d %d\n", i, i < bk.K ? bk.r[i] : 0);
        src += line;
    }
    std::snprintf(line, sizeof(line),
                  "#define WK_RK %d\n#define WK_TW %d\n#define WK_LC %d\n#define WK_P %d\n#define WK_RP %d\n"
                  "#define WK_CS %d\n#define WK_STAGE_OFF %d\n#define WK_WIN %d\n#define WK_WIN_OFF %d\n",
                  bk.rk, kWalkerTW, g.LC, g.P, g.RP, g.CS, g.stage_off, g.win, g.win_off);
    src += line;
    src += gb_walker_source;
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "walker_kernel.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return GF_ECUDA;
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo"};
    const nvrtcResult cr = nvrtcCompileProgram(prog, 3, opts);
    size_t ls = 0;
    if (nvrtcGetProgramLogSize(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
        e.log.resize(ls);
        nvrtcGetProgramLog(prog, &e.log[0]);
    }
    gf_status st = GF_OK;
    if (cr != NVRTC_SUCCESS) {
        st = GF_ECUDA;
    } else {
        size_t n = 0;
        if (nvrtcGetCUBINSize(prog, &n) != NVRTC_SUCCESS || n == 0) {
            st = GF_ECUDA;
        } else {
            e.cubin.resize(n);
            if (nvrtcGetCUBIN(prog, e.cubin.data()) != NVRTC_SUCCESS) st = GF_ECUDA;
        }
    }
    nvrtcDestroyProgram(&prog);
    return st;
}

// The cache entry for (in_dt, radii, stack variant), compiled on first use.
WalkerEntry* entry_for(int in_dt, const BoxKernel& bk, const WalkerGeom& g, bool stack = false) {
    const std::string k = key_of(in_dt, bk, stack);
    auto it = g_cache.find(k);
    if (it != g_cache.end()) return it->second.get();
    std::unique_ptr<WalkerEntry> e(new WalkerEntry());
    e->st = compile(in_dt, bk, g, stack, *e);
    WalkerEntry* raw = e.get();
    g_cache[k] = std::move(e);
    return raw;
}

}  // namespace

namespace {

bool walker_geom_uncached(int in_dt, int rk, WalkerGeom& g);

}  // namespace

// Geometries depend only on the input type and the largest radius: each is
// searched once per process.
bool walker_geom(int in_dt, int rk, WalkerGeom& g) {
    if (rk < 0 || rk > kWalkerMaxRk || (in_dt != GF_U8 && in_dt != GF_U16)) return false;
    static std::mutex mu;
    static WalkerGeom table[2][kWalkerMaxRk + 1];
    static signed char state[2][kWalkerMaxRk + 1] = {};   // 0 unknown, 1 valid, -1 none
    const int ti = in_dt == GF_U8 ? 0 : 1;
    std::lock_guard<std::mutex> lk(mu);
    if (state[ti][rk] == 0) state[ti][rk] = walker_geom_uncached(in_dt, rk, table[ti][rk]) ? 1 : -1;
    g = table[ti][rk];
    return state[ti][rk] > 0;
}

namespace {

bool walker_geom_uncached(int in_dt, int rk, WalkerGeom& g) {
    const int eb = in_bytes(in_dt);
    g.LC = 2 * rk + 2;
    g.P = g.LC * (kWalkerTW / g.LC);
    const int steps = kWalkerTW + 2 * rk + 1;
    const int shb = ((-(rk + 1) * eb) % 16 + 16) % 16;
    const int nch = (shb + steps * eb + 15) / 16;
    // Band rows of RP floats: RP / 4 odd, so that eight consecutive rows read
    // 16 bytes at the same offset in distinct banks; room for the TW outputs
    // and, at the tail, the folded input copy of edge strips, which the row's
    // outputs (written in groups of four as the walk goes) may overwrite only
    // once the walk has fetched those chunks into registers (chunks 0..2 up
    // front, chunk c + 2 on entering chunk c).
    for (int RP = kWalkerTW + 4; RP <= kWalkerTW + 4 + 8 * 64; RP += 8) {
        const int stage_off = RP * 4 - nch * 16;
        if (stage_off < 0) continue;
        bool ok = true;
        for (int j = 2 * rk + 1; j < steps && ok; ++j) {
            const int o = j - (2 * rk + 1);
            if ((o & 3) != 3) continue;
            const int written_end = 4 * o + 4;
            const int c = (shb + j * eb) / 16;
            const int fetched = std::min(nch, std::max(3, c + 3));
            if (fetched < nch && written_end > stage_off + 16 * fetched) ok = false;
        }
        if (ok) {
            g.RP = RP;
            g.CS = (g.LC * RP + 31) / 32 * 32;
            g.stage_off = stage_off;
            g.smem = (size_t)(g.P / g.LC) * g.CS * 4;
            // Edge window: the pixels an edge strip folds from lie within
            // (rk + 2) pixels plus one 16-byte chunk of the row's end; a
            // 16-byte aligned window one chunk wider covers them.  It is
            // kept only where it costs no CTA per SM (sm_103: 228 KiB of
            // shared memory per SM, 1 KiB reserved per CTA).
            const int reach = (rk + 2) * eb + 16;
            const int win = (reach + 15) / 16 * 16 + 16;
            constexpr size_t kSmemPerSm = 233472, kReserved = 1024;
            const size_t with = g.smem + (size_t)g.P * win;
            if (kSmemPerSm / (with + kReserved) >= kSmemPerSm / (g.smem + kReserved)) {
                g.win = win;
                g.win_off = (int)g.smem;
                g.smem = with;
            }
            return true;
        }
    }
    return false;
}

}  // namespace

bool walker_eligible(const Image& im, const BoxKernel& bk) {
    if (im.C != 1 || is_sampled(im) || im.out_dt != GF_F32) return false;
    if (im.in_dt != GF_U8 && im.in_dt != GF_U16) return false;
    WalkerGeom g;
    if (!walker_geom(im.in_dt, bk.rk, g)) return false;
    return g.smem <= (size_t)device_info().max_smem || device_info().max_smem == 0;
}

gf_status walker_compile_check(int in_dt, const BoxKernel& bk, std::string* log) {
    WalkerGeom g;
    if ((in_dt != GF_U8 && in_dt != GF_U16) || !walker_geom(in_dt, bk.rk, g)) return GF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    // the single-image kernel and the variant for stacks of slices
    WalkerEntry* e = entry_for(in_dt, bk, g);
    if (e->st == GF_OK) e = entry_for(in_dt, bk, g, true);
    if (log) *log = e->log;
    return e->st;
}

WalkerPlan walker_plan(const Image& im, const BoxKernel& bk, int nz) {
    WalkerPlan pl;
    WalkerGeom g;
    if (!walker_geom(im.in_dt, bk.rk, g)) return pl;
    const DeviceInfo& di = device_info();
    const int per_sm = std::max(1, std::min(3, (int)((size_t)di.sm_smem / (g.smem + (size_t)di.reserved))));
    const long long slots = (long long)per_sm * std::max(1, di.sms);
    const int nx = (im.W + kWalkerTW - 1) / kWalkerTW;
    // row chunks (of LC rows) per tile: the fewest rows walked by the busiest
    // SM, i.e. waves x CTAs per SM in the last wave x rows per tile
    const int per_sm_slots = std::max(1, per_sm);
    auto busiest = [&](long long tiles) {
        const long long waves = (tiles + slots - 1) / slots;
        const long long last = tiles - (waves - 1) * slots;   // CTAs of the last wave
        return (waves - 1) * per_sm_slots + (last + std::max(1, di.sms) - 1) / std::max(1, di.sms);
    };
    long long best = -1;
    for (int nch = 1; nch <= 4096; ++nch) {
        const int th = nch * g.LC - 2 * bk.rk;
        if (th < 1) continue;
        const long long ny = (im.H + th - 1) / th;
        if (ny > 65535) continue;
        const long long cost = busiest((long long)nx * ny * std::max(1, nz)) * nch;
        if (best < 0 || cost < best) {
            best = cost;
            pl.nb = nch;
            pl.th = th;
        }
        if (th >= im.H) break;
    }
    pl.geom = g;
    pl.grid_x = nx;
    pl.grid_y = pl.th > 0 ? (im.H + pl.th - 1) / pl.th : 0;
    return pl;
}

gf_status walker_prepare(const Image& im, const BoxKernel& bk) {
    cudaKernel_t kern = nullptr;
    WalkerPlan pl;
    return walker_load(im, bk, &kern, &pl);
}

gf_status walker_load(const Image& im, const BoxKernel& bk, cudaKernel_t* out, WalkerPlan* plan, int nz) {
    if (!walker_eligible(im, bk) || nz < 1 || nz > 65535) return GF_EUNSUPPORTED;
    const WalkerPlan pl = walker_plan(im, bk, nz);
    if (pl.nb <= 0 || pl.grid_y <= 0) return GF_EUNSUPPORTED;
    const DeviceInfo& di = device_info();
    if (!di.status) return GF_EUNSUPPORTED;
    cudaKernel_t kern = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        WalkerEntry* e = entry_for(im.in_dt, bk, pl.geom, nz > 1);
        if (e->st != GF_OK) return e->st;
        if (!e->lib) {
            if (cudaLibraryLoadData(&e->lib, e->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
                cudaSuccess)
                return GF_ECUDA;
            if (cudaLibraryGetKernel(&e->kern, e->lib, "walker_kernel") != cudaSuccess) return GF_ECUDA;
        }
        const int dev = di.device;
        if (dev >= 0 && dev < 64 && !((e->smem_set >> dev) & 1ull)) {
            if (cudaKernelSetAttributeForDevice(e->kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)pl.geom.smem, dev) != cudaSuccess)
                return GF_ECUDA;
            e->smem_set |= 1ull << dev;
        }
        kern = e->kern;
    }
    *out = kern;
    *plan = pl;
    return GF_OK;
}

gf_status launch_walker(const Image& im, const BoxKernel& bk, cudaStream_t s, int ty0, int ty1, int nz) {
    cudaKernel_t kern = nullptr;
    WalkerPlan pl;
    gf_status st = walker_load(im, bk, &kern, &pl, nz);
    if (st != GF_OK) return st;
    if (ty1 < 0) ty1 = pl.grid_y;
    if (ty0 < 0 || ty1 <= ty0 || ty1 > pl.grid_y) return GF_EINVAL;
    WalkParams p{};
    p.in = static_cast<const unsigned char*>(im.in);
    p.in_pitch = (long long)im.in_pitch;
    p.out = static_cast<unsigned char*>(im.out);
    p.out_pitch = (long long)im.out_pitch;
    p.H = im.H;
    p.W = im.W;
    p.boundary = im.boundary;
    p.aligned = (reinterpret_cast<uintptr_t>(im.in) % 16 == 0 && im.in_pitch % 16 == 0) ? 1 : 0;
    p.nch = pl.nb;
    p.th = pl.th;
    p.ty0 = ty0;
    p.in_z = (long long)im.H * (long long)im.in_pitch;
    p.out_z = (long long)im.H * (long long)im.out_pitch;
    double sumw = 0.0;
    for (int i = 0; i < GF_KMAX; ++i) {
        p.w[i] = i < bk.K ? bk.w[i] : 0.f;
        if (i < bk.K) sumw += std::fabs((double)bk.w[i]) * (2.0 * bk.r[i] + 1.0);
    }
    // Column quantum q: a power of two with every partial column sum of values
    // rounded to multiples of q below 2^24 q (so those sums are exact in FP32),
    // from the largest row result |R| <= max pixel * sum_i |w_i| (2 r_i + 1)
    // over the nb * P rows one tile walks.
    const double maxpix = im.in_dt == GF_U8 ? 255.0 : 65535.0;
    const double bound = (double)pl.nb * pl.geom.LC * maxpix * sumw * (1.0 + 1e-6);
    int e2 = 0;
    std::frexp(std::max(bound, 1e-30) / 16777216.0, &e2);   // bound / 2^24 < 2^e2
    e2 = std::max(-120, std::min(100, e2));
    p.q = std::ldexp(1.0f, e2);
    p.magic = std::ldexp(1.5f, e2 + 23);
    // Output tiles by TMA: a 3D view (column within strip, strip, row) of the
    // whole strips, box = one chunk's rows in shared memory (RP x 1 x LC; the
    // columns past the strip fall outside the view and are not written); a
    // stack adds the slice as a fourth dimension.
    // (the last map of this thread is reused when the output and geometry repeat)
    struct MapEntry {
        const void* out = nullptr;
        size_t pitch = 0;
        int H = 0, W = 0, RP = 0, LC = 0, nz = 0, ok = 0;
        WalkMap map;
    };
    thread_local MapEntry last;
    if (!(last.out == im.out && last.pitch == im.out_pitch && last.H == im.H && last.W == im.W &&
          last.RP == pl.geom.RP && last.LC == pl.geom.LC && last.nz == nz)) {
        WalkMap omap;
        std::memset(&omap, 0, sizeof(omap));
        int ok = 0;
        const int nfull = im.W / kWalkerTW;
        const auto enc = tensor_map_encoder();
        if (enc && nfull > 0 && reinterpret_cast<uintptr_t>(im.out) % 16 == 0 && im.out_pitch % 16 == 0 &&
            im.out_pitch < (1ull << 40) && pl.geom.RP <= 256 && pl.geom.LC <= 256) {
            const cuuint64_t gdim[4] = {(cuuint64_t)kWalkerTW, (cuuint64_t)nfull, (cuuint64_t)im.H, (cuuint64_t)nz};
            const cuuint64_t gstride[3] = {(cuuint64_t)kWalkerTW * 4, (cuuint64_t)im.out_pitch,
                                           (cuuint64_t)im.H * (cuuint64_t)im.out_pitch};
            const cuuint32_t box[4] = {(cuuint32_t)pl.geom.RP, 1, (cuuint32_t)pl.geom.LC, 1};
            const cuuint32_t estr[4] = {1, 1, 1, 1};
            ok = enc(reinterpret_cast<CUtensorMap*>(&omap), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, nz > 1 ? 4 : 3, im.out,
                     gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        }
        last.out = im.out;
        last.pitch = im.out_pitch;
        last.H = im.H;
        last.W = im.W;
        last.RP = pl.geom.RP;
        last.LC = pl.geom.LC;
        last.nz = nz;
        last.ok = ok;
        last.map = omap;
    }
    WalkMap omap = last.map;
    p.tma_out = last.ok;
    void* args[] = {&omap, &p};
    const dim3 grid(pl.grid_x, ty1 - ty0, nz), block(kWalkerTW);
    if (cudaLaunchKernel(reinterpret_cast<const void*>(kern), grid, block, args, pl.geom.smem, s) != cudaSuccess)
        return GF_ECUDA;
    return GF_OK;
}

// ------------------------------------------------------------------ depth walk
namespace {

constexpr int kDepthTW = 128;   // threads (lines) per CTA

// NVRTC compilation of depth_walker.cuh with the depth radii as constants.
gf_status compile_depth(const BoxKernel& bz, WalkerEntry& e) {
    std::string src;
    char line[320];
    std::snprintf(line, sizeof(line), "#define DW_K %d\n#define DW_RK %d\n#define DW_LC %d\n#define DW_TW %d\n",
                  bz.K, bz.rk, 2 * bz.rk + 2, kDepthTW);
    src += line;
    for (int i = 0; i < GF_KMAX; ++i) {
        std::snprintf(line, sizeof(line), "#define DW_R%d %d\n", i, i < bz.K ? bz.r[i] : 0);
        src += line;
    }
    src += gb_depth_walker_source;
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "depth_walker.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return GF_ECUDA;
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo"};
    const nvrtcResult cr = nvrtcCompileProgram(prog, 3, opts);
    size_t ls = 0;
    if (nvrtcGetProgramLogSize(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
        e.log.resize(ls);
        nvrtcGetProgramLog(prog, &e.log[0]);
    }
    gf_status st = GF_OK;
    size_t n = 0;
    if (cr != NVRTC_SUCCESS || nvrtcGetCUBINSize(prog, &n) != NVRTC_SUCCESS || n == 0) {
        st = GF_ECUDA;
    } else {
        e.cubin.resize(n);
        if (nvrtcGetCUBIN(prog, e.cubin.data()) != NVRTC_SUCCESS) st = GF_ECUDA;
    }
    nvrtcDestroyProgram(&prog);
    return st;
}

// The cache entry of the depth walk for the radii of bz (g_mu held).
WalkerEntry* depth_entry_for(const BoxKernel& bz) {
    char key[96];
    std::snprintf(key, sizeof(key), "depth:%d:%d,%d,%d,%d,%d", bz.K, bz.r[0], bz.r[1], bz.r[2], bz.r[3], bz.r[4]);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) return it->second.get();
    std::unique_ptr<WalkerEntry> e(new WalkerEntry());
    e->st = compile_depth(bz, *e);
    WalkerEntry* raw = e.get();
    g_cache[key] = std::move(e);
    return raw;
}

}  // namespace

gf_status depth_walk_compile_check(const BoxKernel& bz, std::string* log) {
    if (bz.rk < 0 || bz.rk > kDepthWalkMaxRk) return GF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    WalkerEntry* e = depth_entry_for(bz);
    if (log) *log = e->log;
    return e->st;
}

gf_status launch_depth_walk(const float* R, size_t r_pitch, int D, int H, int W, int C, void* out, size_t out_pitch,
                            int boundary, const BoxKernel& bz, double max_abs_r, cudaStream_t s) {
    if (bz.rk < 0 || bz.rk > kDepthWalkMaxRk || D < 1 || H < 1 || W < 1 || C < 1) return GF_EUNSUPPORTED;
    if (!(max_abs_r >= 0.0) || !std::isfinite(max_abs_r)) return GF_EUNSUPPORTED;
    const DeviceInfo& di = device_info();
    if (di.sms <= 0) return GF_EUNSUPPORTED;
    cudaKernel_t kern = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        WalkerEntry* e = depth_entry_for(bz);
        if (e->st != GF_OK) return GF_EUNSUPPORTED;
        if (!e->lib) {
            if (cudaLibraryLoadData(&e->lib, e->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
                    cudaSuccess ||
                cudaLibraryGetKernel(&e->kern, e->lib, "depth_walker_kernel") != cudaSuccess) {
                e->st = GF_ECUDA;
                return GF_EUNSUPPORTED;
            }
        }
        kern = e->kern;
    }
    const int LC = 2 * bz.rk + 2;
    const long long lines = (long long)H * W * C;
    const long long nx = (lines + kDepthTW - 1) / kDepthTW;
    if (nx > 0x7fffffffLL) return GF_EUNSUPPORTED;
    // tile of th = nch LC - 2 rk output slices: the fewest slices walked by the
    // busiest SM (4 CTAs per SM)
    const long long slots = 4LL * di.sms;
    auto busiest = [&](long long tiles) {
        const long long waves = (tiles + slots - 1) / slots;
        const long long last = tiles - (waves - 1) * slots;
        return (waves - 1) * 4 + (last + di.sms - 1) / di.sms;
    };
    int nch = 0, th = 0;
    long long best = -1;
    for (int n = 1; n <= 65535; ++n) {
        const int t = n * LC - 2 * bz.rk;
        if (t < 1) continue;
        const long long ny = (D + t - 1) / t;
        if (ny <= 65535) {
            const long long cost = busiest(nx * ny) * n;
            if (best < 0 || cost < best) {
                best = cost;
                nch = n;
                th = t;
            }
        }
        if (t >= D) break;
    }
    if (nch == 0) return GF_EUNSUPPORTED;
    DepthParams p{};
    p.in = reinterpret_cast<const unsigned char*>(R);
    p.in_pitch = (long long)r_pitch;
    p.in_z = (long long)H * (long long)r_pitch;
    p.out = static_cast<unsigned char*>(out);
    p.out_pitch = (long long)out_pitch;
    p.out_z = (long long)H * (long long)out_pitch;
    p.D = D;
    p.H = H;
    p.rowlen = W * C;
    p.boundary = boundary;
    p.nch = nch;
    p.th = th;
    for (int i = 0; i < GF_KMAX; ++i) p.w[i] = i < bz.K ? bz.w[i] : 0.f;
    // quantum q: a power of two with every partial sum of values rounded to
    // multiples of q, over the nch LC slices one tile walks, below 2^24 q
    const double bound = (double)nch * LC * (max_abs_r + 1.0) * (1.0 + 1e-6);
    int e2 = 0;
    std::frexp(std::max(bound, 1e-30) / 16777216.0, &e2);   // bound / 2^24 < 2^e2
    e2 = std::max(-120, std::min(100, e2));
    p.q = std::ldexp(1.0f, e2);
    p.magic = std::ldexp(1.5f, e2 + 23);
    void* args[] = {&p};
    const dim3 grid((unsigned)nx, (unsigned)((D + th - 1) / th)), block(kDepthTW);
    if (cudaLaunchKernel(reinterpret_cast<const void*>(kern), grid, block, args, 0, s) != cudaSuccess)
        return GF_ECUDA;
    return GF_OK;
}

}  // namespace gb

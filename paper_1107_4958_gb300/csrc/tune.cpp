// Plan autotuner: times candidate plans of both paths on a caller's image and
// keeps the fastest per shape class in the handle (and in its cache file).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace gb {

namespace {

int half_octave(long v) { return v <= 0 ? 0 : (int)std::lround(2.0 * std::log2((double)v)); }

bool plan_is_default(const gf_plan& p) {
    return p.path == GF_PATH_AUTO && !p.tile_w && !p.tile_h && !p.col_w && !p.col_h && !p.accum;
}

std::string device_tag(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    char buf[320];
    std::snprintf(buf, sizeof(buf), "%s/sm%d%d/%d", prop.name, prop.major, prop.minor, prop.multiProcessorCount);
    for (char* c = buf; *c; ++c)
        if (*c == '"' || *c == '\\') *c = '_';
    return buf;
}

void tune_save(const gf_handle_s* h) {
    if (h->tune_cache.empty()) return;
    const std::string tmp = h->tune_cache + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\"gaussbox_tune_cache\": 1, \"device\": \"%s\", \"entries\": {\n",
                 device_tag(h->device).c_str());
    size_t k = 0;
    for (const auto& e : h->tuned) {
        const gf_plan& p = e.second;
        std::fprintf(f, "  \"%s\": [%d, %d, %d, %d, %d]%s\n", e.first.c_str(), p.path, p.tile_w, p.tile_h, p.col_w,
                     p.col_h, ++k < h->tuned.size() ? "," : "");
    }
    std::fprintf(f, "}}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), h->tune_cache.c_str());
}

// Mean time in ms of `reps` launches of `im` on plan `p` after `warm` untimed ones.
float time_plan(const Image& im, const BoxKernel& bk, const gf_plan& p, cudaStream_t s, cudaEvent_t a,
                cudaEvent_t b, int warm, int reps) {
    for (int i = 0; i < warm; ++i)
        if (launch_filter(im, bk, &p, s) != GF_OK) return -1.f;
    if (cudaEventRecord(a, s) != cudaSuccess) return -1.f;
    for (int i = 0; i < reps; ++i)
        if (launch_filter(im, bk, &p, s) != GF_OK) return -1.f;
    if (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms / reps;
}

}  // namespace

std::string tune_key(const Image& im, const BoxKernel& bk) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "i%d_o%d_c%d_k%d_h%d_w%d_r%d", im.in_dt, im.out_dt, im.C, bk.K, half_octave(im.H),
                  half_octave(im.W), half_octave(bk.rk + 1));
    return buf;
}

void apply_tuned(const gf_handle_s* h, Image& im, const BoxKernel& bk) {
    if (!h || h->tuned.empty() || !plan_is_default(im.plan)) return;
    auto it = h->tuned.find(tune_key(im, bk));
    if (it != h->tuned.end()) im.plan = it->second;
}

void tune_load(gf_handle_s* h) {
    if (h->tune_cache.empty()) return;
    FILE* f = std::fopen(h->tune_cache.c_str(), "r");
    if (!f) return;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    std::fclose(f);
    // plans are only reused on the same kind of device
    const std::string want = "\"device\": \"" + device_tag(h->device) + "\"";
    if (text.find(want) == std::string::npos) return;
    size_t pos = text.find("\"entries\"");
    if (pos == std::string::npos) return;
    pos = text.find('{', pos);
    while (pos != std::string::npos) {
        const size_t q0 = text.find('"', pos + 1);
        if (q0 == std::string::npos) break;
        const size_t q1 = text.find('"', q0 + 1);
        if (q1 == std::string::npos) break;
        const std::string key = text.substr(q0 + 1, q1 - q0 - 1);
        gf_plan p{};
        if (std::sscanf(text.c_str() + q1 + 1, " : [%d , %d , %d , %d , %d ]", &p.path, &p.tile_w, &p.tile_h,
                        &p.col_w, &p.col_h) == 5 &&
            p.path >= GF_PATH_AUTO && p.path <= GF_PATH_HBM)
            h->tuned[key] = p;
        pos = text.find(']', q1);
    }
}

}  // namespace gb

using namespace gb;

extern "C" {

gf_status gf_tuned_plan(gf_handle h, const gf_image_desc* img, gf_plan* out) {
    if (!h || !img || !out) return GF_EINVAL;
    Image im;
    BoxKernel bk;
    BatchSpan spans[2];
    gf_status st = collect_batch(img, 1, &im, &bk, spans);
    if (st != GF_OK) return st;
    auto it = h->tuned.find(tune_key(im, bk));
    if (it == h->tuned.end()) return GF_EINVAL;
    *out = it->second;
    return GF_OK;
}

gf_status gf_tune(gf_handle h, const gf_image_desc* img, void* stream, gf_plan* best) {
    if (!h || !img) return GF_EINVAL;
    Image im;
    BoxKernel bk;
    BatchSpan spans[2];
    gf_status st = collect_batch(img, 1, &im, &bk, spans);
    if (st != GF_OK) return st;
    if (cudaSetDevice(h->device) != cudaSuccess) return GF_ECUDA;
    HandleScope scope(h->status_word, h->wait_cycles);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return GF_ECUDA;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return GF_ECUDA;
    }
    // a few launches per candidate, more for small images
    const double px = (double)im.H * im.W * im.C;
    const int reps = px > 8e6 ? 4 : (px > 5e5 ? 8 : 16);
    gf_plan best_p{};
    float best_t = -1.f;
    auto consider = [&](const gf_plan& p) {
        FilterPlan fp;
        if (resolve_plan(im, bk, &p, fp) != GF_OK) return;
        gf_plan full;
        plan_to_abi(fp, &full);
        const float t = time_plan(im, bk, full, s, a, b, 2, reps);
        if (t > 0.f && (best_t < 0.f || t < best_t)) {
            best_t = t;
            best_p = full;
        }
    };
    FilterPlan def;
    st = resolve_plan(im, bk, nullptr, def);
    if (st != GF_OK) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return st;
    }
    // fused: strip width and rows per CTA around the default
    if (fused_fits(im, bk, def.strip.TWp)) {
        const StripPlan d = def.strip;
        gf_plan base{GF_PATH_FUSED, d.TWp, d.TH, 0, 0, 0};
        consider(base);
        gf_plan cur = best_p.path == GF_PATH_FUSED ? best_p : base;
        // taller tiles only within the precision bound of the column sums
        for (int th : {d.TH / 2, d.TH * 2, d.TH * 4}) {
            if (th < 8 || th > im.H || th > std::max(d.TH, column_tile_cap(bk))) continue;
            gf_plan p = cur;
            p.tile_h = th;
            consider(p);
        }
        cur = best_p.path == GF_PATH_FUSED ? best_p : base;
        for (int tw : {d.TWp / 2, d.TWp / 4}) {
            if (tw < std::max(1, 16 / im.C)) continue;
            gf_plan p = cur;
            p.tile_w = tw;
            consider(p);
        }
    }
    // two-pass: one coordinate at a time from its default
    {
        const TwoPassPlan d = default_twopass_plan(im, bk);
        gf_plan base{GF_PATH_TWO_PASS, d.seg_px, d.row_th, d.CW, d.col_th, 0};
        consider(base);
        gf_plan cur = best_p.path == GF_PATH_TWO_PASS ? best_p : base;
        for (int seg : {256 / im.C, 1024 / im.C, 2048 / im.C}) {
            if (seg < 1 || seg > im.W || seg == cur.tile_w) continue;
            gf_plan p = cur;
            p.tile_w = seg;
            consider(p);
        }
        if (best_p.path == GF_PATH_TWO_PASS) cur = best_p;
        for (int cw : {32, 64, 128, 256}) {
            if (cw == cur.col_w) continue;
            gf_plan p = cur;
            p.col_w = cw;
            consider(p);
        }
        if (best_p.path == GF_PATH_TWO_PASS) cur = best_p;
        for (int ch : {cur.col_h / 2, cur.col_h * 2}) {
            if (ch < 8 || ch > im.H || ch > std::max(d.col_th, column_tile_cap(bk))) continue;
            gf_plan p = cur;
            p.col_h = ch;
            consider(p);
        }
        if (best_p.path == GF_PATH_TWO_PASS) cur = best_p;
        for (int rh : {cur.tile_h / 2, cur.tile_h * 2}) {
            if (rh < 8 || rh > im.H) continue;
            gf_plan p = cur;
            p.tile_h = rh;
            consider(p);
        }
    }
    // nothing fits shared memory: the running sums in HBM
    if (best_t < 0.f) consider(gf_plan{GF_PATH_HBM, 0, 0, 0, 0, 0});
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (best_t < 0.f) return GF_ECUDA;
    h->tuned[tune_key(im, bk)] = best_p;
    tune_save(h);
    if (best) *best = best_p;
    return GF_OK;
}

}  // extern "C"

"""Host code under the compiler's sanitizers (no GPU): the library's fitter
(the exhaustive search of Sec. 4.2 on several threads, Eq. scale1/scale2, the
general-kernel fit of Sec. 3.2) under AddressSanitizer + UndefinedBehavior
Sanitizer and under ThreadSanitizer, and the oracle's C (the direct
convolution on OpenMP threads, the running-sum method on the CPU, the
partition search) under AddressSanitizer + UndefinedBehaviorSanitizer.  Each
driver exercises the code on valid and invalid inputs, and the test passes
when the driver exits cleanly with no sanitizer report.  The radii the
sanitized fitter prints at sigma0 are checked against Table 1."""
import os
import shutil
import subprocess

import pytest

from golden_tables import read_param_table

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1107_4958_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

FIT_DRIVER = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include "internal.h"
namespace gb {
gf_status fit_boxes(double sigma, int K, int err_kind, int32_t* radii, double* weights);
gf_status fit_kernel(const double* half, int n, int K, int err_kind, int32_t* radii, double* weights, double* err);
gf_status fit_sigma0(int K, int err_kind, int32_t* p, double* c, double* w, double* err);
}
int main(int argc, char** argv) {
    const bool quick = argc > 1 && std::strcmp(argv[1], "quick") == 0;
    int32_t r[5];
    double w[5], c[5], e;
    for (int kind = 0; kind < (quick ? 1 : 2); ++kind)
        for (int K = quick ? 4 : 1; K <= 5; ++K) {
            if (gb::fit_sigma0(K, kind, r, c, w, &e) != GF_OK) return 1;
            std::printf("sigma0 %d %d", kind, K);
            for (int i = 0; i < K; ++i) std::printf(" %d", r[i]);
            std::printf("\n");
            for (double s : {0.5, 3.0, 8.0, 100.0, 1000.0})
                if (gb::fit_boxes(s, K, kind, r, w) != GF_OK) return 2;
        }
    if (gb::fit_boxes(std::nan(""), 3, 0, r, w) == GF_OK) return 3;
    if (gb::fit_boxes(2.0, 6, 0, r, w) == GF_OK) return 4;
    double tent[40];
    for (int i = 0; i < 40; ++i) tent[i] = 40.0 - i;
    if (gb::fit_kernel(tent, 40, 4, 0, r, w, &e) != GF_OK) return 5;
    (void)gb::fit_kernel(tent, 1, 4, 0, r, w, &e);
    (void)gb::fit_kernel(tent, 3, 5, 1, r, w, &e);
    std::printf("ok\n");
    return 0;
}
"""

ORACLE_DRIVER = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
int oracle_conv_separable(const double*, int, int, int, const int*, const double*, int, int, double*);
int oracle_boxsum_u8_f32(const uint8_t*, long long, int, int, const int*, const float*, int, int, float*);
int oracle_partition_search(const double*, const double*, double, int, int, int*, double*, double*);
int main(void) {
    const int sizes[][2] = {{1, 1}, {1, 9}, {9, 1}, {7, 13}, {33, 20}};
    const int radii[] = {0, 2, 5, 11, 40};
    const double w[] = {0.3, 0.1, 0.05, 0.01, 0.001};
    const float wf[] = {0.3f, 0.1f, 0.05f, 0.01f, 0.001f};
    for (int s = 0; s < 5; ++s) {
        const int H = sizes[s][0], W = sizes[s][1];
        for (int C = 1; C <= 4; ++C)
            for (int K = 1; K <= 5; ++K)
                for (int b = 0; b < 3; ++b) {
                    double* in = malloc(sizeof(double) * H * W * C);
                    double* out = malloc(sizeof(double) * H * W * C);
                    for (int i = 0; i < H * W * C; ++i) in[i] = (i * 37) % 101;
                    if (oracle_conv_separable(in, H, W, C, radii, w, K, b, out) != 0) return 1;
                    free(in);
                    free(out);
                }
        for (int K = 1; K <= 5; ++K)
            for (int b = 0; b < 3; ++b) {
                const long long pitch = W + 3;
                uint8_t* in = malloc((size_t)pitch * H);
                float* out = malloc(sizeof(float) * H * W);
                for (long long i = 0; i < pitch * H; ++i) in[i] = (uint8_t)((i * 53) % 256);
                if (oracle_boxsum_u8_f32(in, pitch, H, W, radii, wf, K, b, out) != 0) return 2;
                free(in);
                free(out);
            }
    }
    enum { N = 14 };
    double M[N * N], h[N];
    for (int i = 0; i < N; ++i) {
        h[i] = i + 1.0;
        for (int j = 0; j < N; ++j) M[i * N + j] = (i < j ? i : j) + 1.0;
    }
    for (int k = 1; k <= 5; ++k) {
        int q[5];
        double qw[5], err;
        if (oracle_partition_search(M, h, 1000.0, N, k, q, qw, &err) != 0) return 3;
    }
    printf("ok\n");
    return 0;
}
"""


def _compile(cmd, cwd):
    r = subprocess.run(cmd, cwd=cwd, capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        if "sanitize" in r.stderr and ("cannot find" in r.stderr or "not supported" in r.stderr):
            pytest.skip("sanitizer runtime unavailable: " + r.stderr.strip().splitlines()[-1])
        raise AssertionError("compile failed:\n" + r.stderr)


def _run(exe, *args):
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1",
               TSAN_OPTIONS="halt_on_error=1")
    r = subprocess.run([exe, *args], capture_output=True, text=True, timeout=600, env=env)
    report = r.stdout + r.stderr
    assert r.returncode == 0, report[-4000:]
    assert "ERROR: AddressSanitizer" not in report and "runtime error" not in report, report[-4000:]
    assert "WARNING: ThreadSanitizer" not in report, report[-4000:]
    assert r.stdout.strip().endswith("ok"), report[-2000:]
    return r.stdout


def _need(tool):
    if shutil.which(tool) is None:
        pytest.skip(tool + " not available")


def _fit_exe(tmp_path, flags):
    _need("g++")
    src = tmp_path / "fit_driver.cpp"
    src.write_text(FIT_DRIVER)
    exe = str(tmp_path / "fit_driver")
    _compile(["g++", "-std=c++17", "-O1", "-g", *flags, "-I" + CSRC, "-I" + os.path.join(ROOT, "include"),
              "-I" + CUDA_INC, str(src), os.path.join(CSRC, "fit.cpp"), "-o", exe, "-lpthread"], tmp_path)
    return exe


def test_fitter_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    exe = _fit_exe(tmp_path, ["-fsanitize=address,undefined", "-fno-sanitize-recover=all"])
    out = _run(exe)
    table = read_param_table("table1_quadratic_form.txt")
    for K in (3, 4, 5):
        line = [ln for ln in out.splitlines() if ln.startswith("sigma0 0 %d " % K)][0]
        assert [int(v) for v in line.split()[3:]] == table[K][0], line


def test_fitter_search_threads_under_thread_sanitizer(tmp_path):
    exe = _fit_exe(tmp_path, ["-fsanitize=thread"])
    _run(exe, "quick")


def test_oracle_c_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    _need("gcc")
    src = tmp_path / "oracle_driver.c"
    src.write_text(ORACLE_DRIVER)
    exe = str(tmp_path / "oracle_driver")
    oracle = os.path.join(ROOT, "oracle")
    _compile(["gcc", "-std=c11", "-O1", "-g", "-fopenmp", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
              str(src), os.path.join(oracle, "conv.c"), os.path.join(oracle, "search.c"), "-o", exe, "-lm"], tmp_path)
    _run(exe)

"""The compile-time FFT plans of the plane kernels against the host's plan
builder (CPU only).  The kernels index their twiddle tables with offsets
computed at compile time (plan_radix_f, plan_ns_f, plan_off_f, plan_tan_off
in csrc/tc_fft_impl.cuh), while the host builds and uploads those tables from
its own run-time plan (make_plan, tangent_twiddles in csrc/tc_api.cu).  The
two must describe the same stages for every length with a compile-time plan
and every plan family, or a kernel would read the wrong twiddles (or past the
end of a table).  This compiles a small host program against both and
compares them stage by stage."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_0711_1429_gb300")
LIB = os.path.join(PKG, "libtc.so")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "tc_fft_impl.cuh"
bool tc_build_fft_plan(int M, FftPlan& p, std::vector<long double>& re, std::vector<long double>& im, int family);

template <int M, int F> int check() {
    int bad = 0;
    if (!tc_fft_fixed_length(M)) { printf("length %d has no compile-time plan\n", M); return 1; }
    FftPlan p;
    std::vector<long double> re, im;
    if (!tc_build_fft_plan(M, p, re, im, F)) { printf("host plan failed M=%d F=%d\n", M, F); return 1; }
    constexpr int n = plan_nst_f(M, F);
    if (p.nst != n) { printf("M=%d F=%d stages host %d device %d\n", M, F, p.nst, n); return 1; }
    int tan = 0;
    for (int s = 0; s < n; ++s) {
        const int R = plan_radix_f(M, s, F), Ns = plan_ns_f(M, s, F), off = plan_off_f(M, s, F);
        if (p.R[s] != R || p.Ns[s] != Ns || p.twoff[s] != off) {
            printf("M=%d F=%d stage %d host (%d,%d,%d) device (%d,%d,%d)\n", M, F, s, p.R[s], p.Ns[s],
                   p.twoff[s], R, Ns, off);
            ++bad;
        }
        if (F == 0 || F == 3) {
            if (plan_tan_off(M, s, F) != tan) { printf("M=%d F=%d stage %d tangent offset\n", M, F, s); ++bad; }
            tan += Ns * (R == 2 ? 2 : 6);
        }
    }
    if (p.ntw != plan_off_f(M, n, F) || (int)re.size() != p.ntw || (int)im.size() != p.ntw) {
        printf("M=%d F=%d table size host %d (%zu) device %d\n", M, F, p.ntw, re.size(), plan_off_f(M, n, F));
        ++bad;
    }
    if ((F == 0 || F == 3) && plan_tan_off(M, n, F) != tan) { printf("M=%d F=%d tangent table size\n", M, F); ++bad; }
    if (F == 3 && plan_radix_f(M, n - 1, F) != 3) { printf("M=%d family 3 does not end in radix 3\n", M); ++bad; }
    return bad;
}
template <int M> int check_all() { return check<M, 0>() + check<M, 1>() + check<M, 3>(); }

int main() {
    int bad = check_all<12>() + check_all<18>() + check_all<24>() + check_all<36>() + check_all<48>() +
              check_all<72>() + check_all<96>() + check_all<144>() + check_all<192>() + check_all<288>() +
              check_all<384>() + check_all<576>() + check_all<768>() + check_all<1152>() + check_all<1536>();
    // lengths without a compile-time plan take the run-time plan
    for (int M : {6, 9, 30, 60, 255, 3072}) if (tc_fft_fixed_length(M)) { printf("%d claims a plan\n", M); ++bad; }
    printf(bad ? "FAIL %d\n" : "OK\n", bad);
    return bad ? 1 : 0;
}
"""


def test_compile_time_plans_match_host_plans(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    if not os.path.exists(LIB):
        pytest.skip("libtc.so not built")
    src = tmp_path / "plans.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "plans"
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(PKG, "csrc"), "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", PKG, "-ltc", f"-Xlinker=-rpath,{PKG}"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:] + r.stderr[-2000:]


TWIDDLES = r"""
#include <cmath>
#include <cstdio>
#include <vector>
#include "tc_internal.h"
bool tc_build_fft_plan(int M, FftPlan& p, std::vector<long double>& re, std::vector<long double>& im, int family);

int main() {
    int bad = 0, lengths = 0;
    for (int M = 6; M <= 6561; ++M) {
        for (int F : {0, 1}) {
            FftPlan p;
            std::vector<long double> re, im;
            if (!tc_build_fft_plan(M, p, re, im, F)) continue;
            ++lengths;
            int total = 0;
            for (int s = 0; s < p.nst; ++s) {
                long long num, den;
                const int count = fft_twiddle_fraction(p, s, 0, num, den);
                if (p.twoff[s] != total) { printf("M=%d F=%d stage %d offset\n", M, F, s); ++bad; }
                for (int i = 0; i < count; ++i) {
                    fft_twiddle_fraction(p, s, i, num, den);
                    const long double a = -2.0L * 3.141592653589793238462643383279503L * (long double)num / (long double)den;
                    const int k = p.twoff[s] + i;
                    if (num < 0 || num >= den || k >= (int)re.size() ||
                        fabsl(cosl(a) - re[k]) > 1e-17L || fabsl(sinl(a) - im[k]) > 1e-17L) {
                        if (bad < 10) printf("M=%d F=%d stage %d entry %d\n", M, F, s, i);
                        ++bad;
                    }
                }
                total += count;
            }
            if (total != p.ntw || (int)re.size() != p.ntw) { printf("M=%d F=%d table size\n", M, F); ++bad; }
        }
    }
    printf("%d plans\n", lengths);
    printf(bad ? "FAIL %d\n" : "OK\n", bad);
    return bad ? 1 : 0;
}
"""


def test_device_twiddle_layout_matches_host_tables(tmp_path):
    """The allocation-free transform computes its twiddle tables on the
    device from (num, den) fractions of a turn (fft_twiddle_fraction in
    csrc/tc_internal.h); every entry of every plan of both families, for all
    lengths 6..6561 that have a plan, must be the entry the host plan builder
    writes."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    if not os.path.exists(LIB):
        pytest.skip("libtc.so not built")
    src = tmp_path / "tw.cu"
    src.write_text(TWIDDLES)
    exe = tmp_path / "tw"
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(PKG, "csrc"), "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", PKG, "-ltc", f"-Xlinker=-rpath,{PKG}"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:] + r.stderr[-2000:]

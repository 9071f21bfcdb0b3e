// Spectral -> physical transform of one field for callers that cannot
// allocate device memory.
//
// Some callers of this library run where a device allocation is not allowed
// or not possible: code that must stay within a memory budget fixed before it
// starts, plug-ins whose host application owns every device buffer, or
// latency-critical loops in which cudaMalloc (which may synchronise the
// device) is forbidden.  tc_to_physical_noalloc serves them: the caller
// passes the input and output device buffers, and the intermediates the
// transform needs (the z-transformed planes and the twiddle tables) live in
// the fixed array below, which is part of the library image.
//
// The array is a host-side stand-in in host code: its device address is
// fetched with cudaGetSymbolAddress once per device, with that device
// current, the first time the entry point runs there.
//
// Nothing crosses from host memory during a call: the twiddle tables are
// computed on the device from the transform plans (cached on the host per
// pair of lengths), and as many radial planes as the array holds go through
// each pair of launches.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "tc_internal.h"
#include "../../include/tc.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[TC_NOALLOC_SCRATCH_BYTES];

bool tc_build_fft_plan(int M, FftPlan& p, std::vector<long double>& re, std::vector<long double>& im, int family);
void tc_set_error_message(const std::string& s);

namespace {

const int kMaxDevices = 64;
// shared memory the transform kernels may opt into (the library's own limit)
const size_t kSmemLimit = 200 * 1024;
unsigned char* g_scratch_dev[kMaxDevices];
std::mutex g_setup_mutex;
std::mutex g_plan_mutex;
std::map<std::pair<int, int>, std::pair<FftPlan, FftPlan>> g_plans;   // (Mz, Mt) -> (z plan, theta plan)

bool is_2a3b(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

bool is_smooth(int n) {
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7, 11, 13, 17})
        while (n % p == 0) n /= p;
    return n == 1;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// The z plan (radix 3, 16, then 8/4/2, plus the paired prime stages) and the
// theta plan (radix 3, 4, 2) of the transform, built once per pair of lengths.
bool plans_for(int Mz, int Mt, FftPlan& pz, FftPlan& pt) {
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    auto it = g_plans.find({Mz, Mt});
    if (it == g_plans.end()) {
        FftPlan a, b;
        std::vector<long double> re, im;
        if (!tc_build_fft_plan(Mz, a, re, im, 1)) return false;
        re.clear(); im.clear();
        if (!tc_build_fft_plan(Mt, b, re, im, 0)) return false;
        it = g_plans.emplace(std::make_pair(Mz, Mt), std::make_pair(a, b)).first;
    }
    pz = it->second.first;
    pt = it->second.second;
    return true;
}

// Device address of the scratch array for the current device (set-up on the
// first call per device: symbol address and the shared-memory opt-in of the
// transform kernels).
int scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        tc_set_error_message(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return TC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            tc_set_error_message(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return TC_ERR_CUDA;
        }
        e = tc_set_kernel_attributes();
        if (e != cudaSuccess) {
            tc_set_error_message(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
            return TC_ERR_CUDA;
        }
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return TC_OK;
}

}  // namespace

// Twiddle table of one plan, in the layout the transform kernels read
// (FftPlan): per stage s of radix R after Ns points, exp(-2 pi i r jm/(Ns R))
// for jm < Ns, r = 1..R-1, and for a stage of odd prime radix R the R-th roots
// exp(-2 pi i e/R), e < R, after them (fft_twiddle_fraction).  One block per
// stage; the angle is an exact fraction of a turn, reduced below one turn,
// before sincospi.
__global__ void k_noalloc_twiddles(FftPlan p, double2* tw) {
    const int s = blockIdx.x;
    if (s >= p.nst) return;
    long long num, den;
    const int count = fft_twiddle_fraction(p, s, 0, num, den);
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        fft_twiddle_fraction(p, s, i, num, den);
        double sn, cs;
        sincospi(2.0 * (double)num / (double)den, &sn, &cs);
        tw[p.twoff[s] + i] = make_double2(cs, -sn);
    }
}

extern "C" int tc_to_physical_noalloc(int Nr, int Ntheta, int Nz, const void* spectral_dev,
                                      void* physical_dev, void* cuda_stream) {
    if (Nr < 1 || Ntheta < 4 || Nz < 4 || Ntheta % 4 || Nz % 2 || !is_2a3b(Ntheta) || !is_smooth(Nz)) {
        tc_set_error_message("tc_to_physical_noalloc: Nr >= 1; Ntheta a multiple of 4 of the form 2^a 3^b; "
                             "Nz even >= 4 with prime factors in {2, 3, 5, 7, 11, 13, 17}");
        return TC_ERR_ARG;
    }
    if (!spectral_dev || !physical_dev) {
        tc_set_error_message("tc_to_physical_noalloc: null buffer");
        return TC_ERR_ARG;
    }
    TcDev d;
    memset(&d, 0, sizeof(d));
    d.Nz = Nz;
    d.Nh = Ntheta / 2;
    d.Mt = 3 * Ntheta / 2;
    d.Mz = 3 * Nz / 2;
    d.npairs = d.Nz * d.Nh;
    // Shared memory per block: 2 ztile Mz complex values in the z transform,
    // 2 Mt in the theta transform.  The z tile is the widest of 8, 4, 2, 1
    // columns that divides Ntheta/2 and fits.
    d.ztile = 0;
    for (int t : {8, 4, 2, 1})
        if (d.Nh % t == 0 && 2 * (size_t)t * d.Mz * sizeof(double2) <= kSmemLimit) { d.ztile = t; break; }
    if (d.ztile == 0 || 2 * (size_t)d.Mt * sizeof(double2) > kSmemLimit) {
        tc_set_error_message("tc_to_physical_noalloc: a padded transform length (3 Nz/2 = " + std::to_string(d.Mz) +
                             ", 3 Ntheta/2 = " + std::to_string(d.Mt) + ") needs more than the " +
                             std::to_string(kSmemLimit) + " bytes of shared memory a transform block may use");
        return TC_ERR_SIZE;
    }
    if (!plans_for(d.Mz, d.Mt, d.pz, d.pt)) {
        tc_set_error_message("tc_to_physical_noalloc: no transform plan for the padded lengths 3 Nz/2 = " +
                             std::to_string(d.Mz) + " and 3 Ntheta/2 = " + std::to_string(d.Mt) +
                             " (at most 16 stages of radix 2, 3, 4, 8, 16 and primes up to 17)");
        return TC_ERR_ARG;
    }
    const size_t nz = d.pz.ntw ? d.pz.ntw : 1, nt = d.pt.ntw ? d.pt.ntw : 1;
    const size_t tw_bytes = align256((nz + nt) * sizeof(double2));
    const size_t plane_bytes = (size_t)d.Mz * d.Nh * sizeof(double2);
    if (tw_bytes + plane_bytes > (size_t)TC_NOALLOC_SCRATCH_BYTES) {
        tc_set_error_message("tc_to_physical_noalloc: one (3 Nz/2) x (Ntheta/2) complex plane plus twiddles needs " +
                             std::to_string(tw_bytes + plane_bytes) + " bytes, more than the " +
                             std::to_string((size_t)TC_NOALLOC_SCRATCH_BYTES) + "-byte scratch");
        return TC_ERR_SIZE;
    }
    unsigned char* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // Every call rewrites the twiddles, and the z transform fully writes each
    // plane before the theta transform reads it, so nothing in the array has
    // to start at zero.
    double2* twz = reinterpret_cast<double2*>(scratch);
    double2* twt = twz + nz;
    k_noalloc_twiddles<<<d.pz.nst > 0 ? d.pz.nst : 1, 128, 0, s>>>(d.pz, twz);
    k_noalloc_twiddles<<<d.pt.nst > 0 ? d.pt.nst : 1, 128, 0, s>>>(d.pt, twt);
    d.twz_d = twz;
    d.twt_d = twt;
    d.zbuf = scratch + tw_bytes;
    const int chunk = (int)std::min<size_t>((size_t)Nr, ((size_t)TC_NOALLOC_SCRATCH_BYTES - tw_bytes) / plane_bytes);
    const double2* spec = static_cast<const double2*>(spectral_dev);
    double* phys = static_cast<double*>(physical_dev);
    for (int r0 = 0; r0 < Nr; r0 += chunk) {
        d.Nr = std::min(chunk, Nr - r0);
        d.phys = phys + (size_t)r0 * d.Mz * d.Mt;
        tc_launch_to_physical(d, spec + (size_t)r0 * d.Nz * d.Nh, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tc_set_error_message(std::string("kernel launch: ") + cudaGetErrorString(e));
        return TC_ERR_CUDA;
    }
    return TC_OK;
}

// Spectral -> physical transform of one field for callers that cannot
// allocate device memory.
//
// Some callers of this library run where a device allocation is not allowed
// or not possible: code that must stay within a memory budget fixed before it
// starts, plug-ins whose host application owns every device buffer, or
// latency-critical loops in which cudaMalloc (which may synchronise the
// device) is forbidden.  tc_to_physical_noalloc serves them: the caller
// passes the input and output device buffers, and the one intermediate the
// transform needs (the z-transformed plane, plus the twiddle tables) lives in
// the fixed array below, which is part of the library image.
//
// The array is a host-side stand-in in host code: its device address is
// fetched with cudaGetSymbolAddress once per device, with that device
// current, the first time the entry point runs there.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tc_internal.h"
#include "../../include/tc.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[TC_NOALLOC_SCRATCH_BYTES];

bool tc_build_fft_plan(int M, FftPlan& p, std::vector<long double>& re, std::vector<long double>& im, int family);
void tc_set_error_message(const std::string& s);

namespace {

const int kMaxDevices = 64;
unsigned char* g_scratch_dev[kMaxDevices];
std::mutex g_setup_mutex;

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
    d.Nr = 1;
    d.Nz = Nz;
    d.Nh = Ntheta / 2;
    d.Mt = 3 * Ntheta / 2;
    d.Mz = 3 * Nz / 2;
    d.npairs = d.Nz * d.Nh;
    d.ztile = d.Nh % 8 == 0 ? 8 : (d.Nh % 4 == 0 ? 4 : (d.Nh % 2 == 0 ? 2 : 1));
    std::vector<long double> zr, zi, tr, ti;
    if (!tc_build_fft_plan(d.Mz, d.pz, zr, zi, 1) || !tc_build_fft_plan(d.Mt, d.pt, tr, ti, 0)) {
        tc_set_error_message("tc_to_physical_noalloc: FFT length is not of the form 2^a 3^b");
        return TC_ERR_ARG;
    }
    std::vector<double2> tw(zr.size() + tr.size() + 2);
    size_t nz = zr.size() ? zr.size() : 1, nt = tr.size() ? tr.size() : 1;
    for (size_t i = 0; i < zr.size(); ++i) tw[i] = make_double2((double)zr[i], (double)zi[i]);
    if (zr.empty()) tw[0] = make_double2(1.0, 0.0);
    for (size_t i = 0; i < tr.size(); ++i) tw[nz + i] = make_double2((double)tr[i], (double)ti[i]);
    if (tr.empty()) tw[nz] = make_double2(1.0, 0.0);
    const size_t tw_bytes = align256((nz + nt) * sizeof(double2));
    const size_t plane_bytes = (size_t)d.Mz * d.Nh * sizeof(double2);
    if (tw_bytes + plane_bytes > (size_t)TC_NOALLOC_SCRATCH_BYTES) {
        tc_set_error_message("tc_to_physical_noalloc: (3 Nz/2) x (Ntheta/2) complex plane plus twiddles needs " +
                             std::to_string(tw_bytes + plane_bytes) + " bytes, more than the " +
                             std::to_string((size_t)TC_NOALLOC_SCRATCH_BYTES) + "-byte scratch");
        return TC_ERR_SIZE;
    }
    unsigned char* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // The twiddles are rewritten on every call; the plane buffer is fully
    // written by the z transform before the row transform reads it, so nothing
    // has to start at zero.
    cudaError_t e = cudaMemcpyAsync(scratch, tw.data(), (nz + nt) * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        tc_set_error_message(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
        return TC_ERR_CUDA;
    }
    d.twz_d = reinterpret_cast<const double2*>(scratch);
    d.twt_d = reinterpret_cast<const double2*>(scratch) + nz;
    d.zbuf = scratch + tw_bytes;
    const double2* spec = static_cast<const double2*>(spectral_dev);
    double* phys = static_cast<double*>(physical_dev);
    for (int r = 0; r < Nr; ++r) {
        d.phys = phys + (size_t)r * d.Mz * d.Mt;
        tc_launch_to_physical(d, spec + (size_t)r * d.Nz * d.Nh, s);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        tc_set_error_message(std::string("kernel launch: ") + cudaGetErrorString(e));
        return TC_ERR_CUDA;
    }
    return TC_OK;
}

// Plane phase: dispatch to the per-type kernels (tc_fft_f64.cu, tc_fft_f32.cu,
// tc_fft_df.cu; templates and the description of the transforms in
// tc_fft_impl.cuh), the transform-length table and the energy reduction.
#include "tc_internal.h"

void tc_plane_kernel_f64(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles);
void tc_plane_kernel_f32(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles);
void tc_plane_kernel_df(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles);
void tc_plane_kernel_batch_f64(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which, cudaStream_t s);
void tc_plane_kernel_batch_f32(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which, cudaStream_t s);
void tc_plane_kernel_batch_df(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which, cudaStream_t s);
cudaError_t tc_plane_attributes_f64();
cudaError_t tc_plane_attributes_f32();
cudaError_t tc_plane_attributes_df();
cudaError_t tc_rows_phys_attributes();

bool tc_fft_fixed_length(int M) {
    for (int m : {12, 18, 24, 36, 48, 72, 96, 144, 192, 288, 384, 576, 768, 1152, 1536})
        if (M == m) return true;
    return false;
}

// ---- kinetic-energy profile: sum over pairs of weight |u|^2+|v|^2+|w|^2 ------
__global__ void __launch_bounds__(256) k_energy(TcDev d) {
    const int r = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < d.npairs; i += blockDim.x) {
        const int j = i % d.Nh;
        const size_t o = (size_t)r * d.npairs + i;
        const double2 a = d.u[o], b = d.v[o], c = d.w[o];
        const double wgt = j == 0 ? 1.0 : 2.0;
        acc += wgt * (a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y + c.x * c.x + c.y * c.y);
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) d.eprof[r] = red[0];
}

void tc_launch_plane_kernel_tiles(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles) {
    if (d.prec == 1) tc_plane_kernel_f32(d, which, s, tile0, ntiles);
    else if (d.prec == 2) tc_plane_kernel_df(d, which, s, tile0, ntiles);
    else tc_plane_kernel_f64(d, which, s, tile0, ntiles);
}

void tc_launch_plane_kernel_batch(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which,
                                  cudaStream_t s) {
    if (d0.prec == 1) tc_plane_kernel_batch_f32(d0, ds, ymap, nplanes, which, s);
    else if (d0.prec == 2) tc_plane_kernel_batch_df(d0, ds, ymap, nplanes, which, s);
    else tc_plane_kernel_batch_f64(d0, ds, ymap, nplanes, which, s);
}

void tc_launch_plane_kernel(const TcDev& d, int which, cudaStream_t s) {
    tc_launch_plane_kernel_tiles(d, which, s, 0, d.Nh / d.ztile);
}

void tc_launch_plane_phase(const TcDev& d, cudaStream_t s) {
    for (int w = 0; w < 3; ++w) tc_launch_plane_kernel(d, w, s);
}

// Shared-memory opt-in of the FFT kernels (called once per device, before any
// stream capture).
cudaError_t tc_set_kernel_attributes() {
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {tc_plane_attributes_f64(), tc_plane_attributes_f32(), tc_plane_attributes_df(),
                          tc_rows_phys_attributes()})
        if (r != cudaSuccess) e = r;
    return e;
}

void tc_launch_energy(const TcDev& d, cudaStream_t s) {
    k_energy<<<d.Nr, 256, 0, s>>>(d);
}

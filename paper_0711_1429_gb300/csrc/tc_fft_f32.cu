// Plane-phase kernels of the f32 arithmetic (templates in tc_fft_impl.cuh).
#include "tc_fft_impl.cuh"

void tc_plane_kernel_f32(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles) {
    plane_kernel_t<float>(d, which, s, tile0, ntiles);
}

cudaError_t tc_plane_attributes_f32() { return plane_attributes_t<float>(); }

void tc_plane_kernel_batch_f32(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which,
                             cudaStream_t s) {
    plane_kernel_batch_t<float>(d0, ds, ymap, nplanes, which, s);
}

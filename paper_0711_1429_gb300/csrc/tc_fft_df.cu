// Plane-phase kernels of the df arithmetic (templates in tc_fft_impl.cuh).
#include "tc_fft_impl.cuh"

void tc_plane_kernel_df(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles) {
    plane_kernel_t<dfloat>(d, which, s, tile0, ntiles);
}

cudaError_t tc_plane_attributes_df() { return plane_attributes_t<dfloat>(); }

void tc_plane_kernel_batch_df(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which,
                             cudaStream_t s) {
    plane_kernel_batch_t<dfloat>(d0, ds, ymap, nplanes, which, s);
}

// Plane-phase kernels of the f64 arithmetic (templates in tc_fft_impl.cuh).
#include "tc_fft_impl.cuh"

void tc_plane_kernel_f64(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles) {
    plane_kernel_t<double>(d, which, s, tile0, ntiles);
}

cudaError_t tc_plane_attributes_f64() { return plane_attributes_t<double>(); }

void tc_plane_kernel_batch_f64(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which,
                             cudaStream_t s) {
    plane_kernel_batch_t<double>(d0, ds, ymap, nplanes, which, s);
}

// ---- physical output of one field (float64) ---------------------------------
__global__ void __launch_bounds__(256) k_rows_phys(TcDev d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Mt = d.Mt, Nh = d.Nh, Mz = d.Mz;
    double2* bufA = reinterpret_cast<double2*>(smem_raw);
    double2* bufB = bufA + Mt;
    const int q = blockIdx.x, r = blockIdx.y;
    const double2* fr = reinterpret_cast<const double2*>(d.zbuf) + ((size_t)r * Mz + q) * Nh;
    for (int p = threadIdx.x; p < Mt; p += blockDim.x) {
        double2 a = make_double2(0.0, 0.0);
        if (p == 0) a.x = fr[0].x;
        else if (p < Nh) a = fr[p];
        else if (p > Mt - Nh) { a = fr[Mt - p]; a.y = -a.y; }
        bufA[p] = a;
    }
    __syncthreads();
    double2* res = fft_stockham<double, +1, 0>(tg_block(), bufA, bufB, 1, d.pt, d.twt_d);
    for (int p = threadIdx.x; p < Mt; p += blockDim.x)
        d.phys[((size_t)r * Mz + q) * Mt + p] = res[p].x;
}

void tc_launch_to_physical(const TcDev& d, const double2* field, cudaStream_t s) {
    const int ct = d.ztile;
    const size_t smz = 2 * (size_t)ct * d.Mz * sizeof(double2);
    TcDev dd = d;
    // one field through slot 0 of zbuf (always float64 here)
    if (z_has_odd_primes(d)) k_zinv<double, 2><<<dim3(d.Nh / ct, d.Nr, 1), 256, smz, s>>>(dd, field, field, field, 0);
    else if (d.zfam0) k_zinv<double, 0><<<dim3(d.Nh / ct, d.Nr, 1), 256, smz, s>>>(dd, field, field, field, 0);
    else k_zinv<double, 1><<<dim3(d.Nh / ct, d.Nr, 1), 256, smz, s>>>(dd, field, field, field, 0);
    k_rows_phys<<<dim3(d.Mz, d.Nr), 256, 2 * (size_t)d.Mt * sizeof(double2), s>>>(dd);
}

cudaError_t tc_rows_phys_attributes() {
    return cudaFuncSetAttribute((const void*)k_rows_phys, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

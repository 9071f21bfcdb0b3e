// Internal declarations shared by the translation units of libtc.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#define TC_MAX_STAGES 16
#define TC_NPROD 5   // transformed products: uu-vv, uv, uw, vw, ww-vv

// Mixed-radix (2, 3, 4) Stockham plan of one transform length M.
// Stage s has radix R[s]; Ns[s] = product of the radices before it.
// Forward twiddles exp(-2 pi i r jm/(Ns R)) for jm < Ns, r = 1..R-1 sit at
// tw[twoff[s] + jm*(R-1) + r-1]; the inverse uses their conjugates.
struct FftPlan {
    int M;
    int nst;
    int R[TC_MAX_STAGES];
    int Ns[TC_MAX_STAGES];
    int twoff[TC_MAX_STAGES];
    int ntw;
};

// Entry i of stage s of the twiddle table of plan p as the fraction num/den
// of a full turn: the entry is exp(-2 pi i num/den).  Entries i < Ns (R-1)
// are the stage twiddles (jm = i / (R-1), r = i % (R-1) + 1: num = r jm,
// den = Ns R); a stage of odd prime radix R > 3 stores its R-th roots
// (num = e, den = R) after them.  Returns the number of entries of the stage
// (i is ignored when it is out of range).
__host__ __device__ inline int fft_twiddle_fraction(const FftPlan& p, int s, int i, long long& num, long long& den) {
    const int R = p.R[s], Ns = p.Ns[s];
    const bool roots = !(R == 2 || R == 3 || R == 4 || R == 8 || R == 16);
    const int nstage = Ns * (R - 1);
    if (i < nstage) { num = (long long)(i % (R - 1) + 1) * (i / (R - 1)); den = (long long)Ns * R; }
    else { num = i - nstage; den = R; }
    num %= den;
    return nstage + (roots ? R : 0);
}

// Everything a kernel needs, passed by value.
struct TcDev {
    int Nr, Nz, Nh, Mt, Mz;
    int npairs;                 // Nz * Nh
    int mixed;                  // 1: float32 FFT/products (precision == TC_PREC_MIXED)
    int prec;                   // TC_PREC_FP64, TC_PREC_MIXED or TC_PREC_DF64
    int ztile;                  // azimuthal columns per CTA of the z kernels (divides Nh)
    int line_block;             // line-kernel variant: 64/128/256 threads, or 1003/1004 =
                                // 128 threads with registers for 3/4 resident blocks per SM
    double dt, nu, m0, alpha0, W_outer;
    double fscale;              // 1/(Mt Mz), the forward-transform factor
    float fscale_f;
    float fscale_lo;            // fscale - (double)fscale_f: double-float low part
    // RK coefficients of substep k and of the substep after it
    double rk_alpha[3], rk_beta[3], rk_gamma[3], rk_zeta[3];

    // spectral fields, complex, [Nr][Nz][Nh]
    double2 *v, *eta, *u, *w, *Hv, *He;
    // spectral products [TC_NPROD][Nr][Nz][Nh] (double2, or float2 in the mixed
    // form): uu - vv, uv, uw, vw, ww - vv.  The isotropic part vv of the
    // momentum flux is a pressure gradient, which the v and eta rows
    // annihilate, so five transforms replace six.
    void* prod;
    // plane-phase intermediates: zbuf [3][Nr][Mz][Nh], pbuf [TC_NPROD][Nr][Mz][Nh]
    void* zbuf;
    void* pbuf;
    // mean flow
    double *U, *W, *HU, *HW;

    // radial tables
    const double* r;            // [Nr]
    const double* rinv;         // [Nr]
    const int* start;           // [Nr]
    const double* d0;           // [Nr][5]
    const double* l1;
    const double* l2;
    const double* l4;
    const double* dwall;        // [2][5]
    const double* dsol;         // [Nr][5] reversed factorisation of the d0 system
    const float* d0f;           // float copies of d0, l1, l2 and 1/r (mixed form)
    const float* l1f;
    const float* l2f;
    const float* rinvf;
    const float2* d0x;          // double-float (hi, lo) copies of d0, l1, l2, 1/r
    const float2* l1x;
    const float2* l2x;
    const float2* rinvx;
    const double* mean_lu;      // [2 profiles][3 substeps][Nr][5] + precombination
    const double* mean_L;       // [2][Nr][5] implicit bands of U and W rows
    // per-pair tables, structure of arrays [..][Nr][5][npairs]
    double* tab_luv;            // [3][Nr][5][npairs]
    double* tab_lue;            // [3][Nr][5][npairs]
    double* tab_lv;             // [Nr][5][npairs]
    double* tab_c;              // [Nr][npairs] c = 1/k^2
    double* tab_c1;             // [Nr][npairs] c1 = dc/dr
    float2* tab_cx;             // double-float copies of c, c1 (TC_PREC_DF64 only)
    float2* tab_c1x;

    // FFT plans and twiddles (double and float copies): pz (length Mz), pt
    // (Mt), ph (Mt/2, the real transforms of one signal) and twr[k] =
    // exp(-2 pi i k/Mt), k < Mt/2, for their pre/post-processing.
    FftPlan pz, pt, ph;
    // float64 z transforms with the theta-row plan family (radix 3, 4, 2 in
    // tangent form) when Mz has a compile-time plan: zfam0 = 1, plan pz0
    int zfam0;
    FftPlan pz0;
    const double* twz_tan;
    const double* twz3_tan;     // tangent twiddles of the family-3 plan (float64 forward z)
    const double* twt3_tan;     // tangent twiddles of the family-3 plan of Mt (float64 forward theta)
    // twiddles of the plan pz0 in the plain (cos, sin) form for the float32
    // and double-float z transforms, which use that plan too
    const float2* twz0_f;
    const float4* twz0_x;
    const double2* twz_d;
    const double2* twt_d;
    const double2* twh_d;
    // theta-row twiddles in tangent form for the float64 radix-2/3/4 stages
    // (per stage and jm: tau_r = sin/cos, the cosines and their ratios)
    const double* twt_tan;
    const double* twh_tan;
    const double2* twr_d;
    const float2* twz_f;
    const float2* twt_f;
    const float2* twh_f;
    const float2* twr_f;
    // double-float copies (hi, lo float pairs) for TC_PREC_DF64, layout
    // {re.hi, re.lo, im.hi, im.lo}
    const float4* twz_x;
    const float4* twt_x;
    const float4* twh_x;
    const float4* twr_x;

    // physical output buffer for tc_get_field (float64 [Nr][Mz][Mt])
    double* phys;
    // energy and strain-rate reduction outputs [Nr]
    double* eprof;
    double* dprof;

    int* flag;                  // device status flags: [0] non-finite, [1] pivot
};

// kernels launched from the host side (defined in the .cu files)
void tc_launch_plane_phase(const TcDev& d, cudaStream_t s);
// one kernel of the plane phase: 0 = z inverse, 1 = theta rows + products, 2 = z forward
void tc_launch_plane_kernel(const TcDev& d, int which, cudaStream_t s);
// z kernels (which = 0 or 2) on the z tiles tile0 .. tile0 + ntiles - 1 only
void tc_launch_plane_kernel_tiles(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles);
// one plane kernel (which as above) for all cases of a shape class: d0 the
// class's representative descriptor, ds / ymap on the device (descriptor per
// case; (case, radial plane) per grid row, nplanes rows)
void tc_launch_plane_kernel_batch(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which,
                                  cudaStream_t s);
cudaError_t tc_probe_fma(double* fp64_tflops, double* fp32_tflops);
void tc_launch_line_phase(const TcDev& d, int k, cudaStream_t s);
// line phase of the pairs with azimuthal index j0 <= j < j0 + nj (all axial slots)
void tc_launch_line_chunk(const TcDev& d, int k, cudaStream_t s, int j0, int nj);
// the same without the implicit part of the next RK memory (double-float and
// mixed forms; float64 launches the full kernel), which tc_launch_rk_memory
// then adds for the same pairs before the next substep's line kernel
void tc_launch_line_chunk_deferred(const TcDev& d, int k, cudaStream_t s, int j0, int nj);
// (background: in four blocks per SM, for a launch beside other kernels)
void tc_launch_rk_memory(const TcDev& d, int k, cudaStream_t s, int j0, int nj, bool background);
const void* tc_rk_memory_kernel();   // its kernel, to find its nodes in a captured graph
void tc_launch_mean_phase(const TcDev& d, int k, cudaStream_t s);
// line phase and mean flow of substep k for many cases of one precision form
// (descriptors ds on the device): the line kernel in nblocks blocks of
// tc_line_batch_block() threads, bmap[block] = (case, block within the case);
// the mean flow one block per case, maxNr the largest Nr among them
void tc_launch_line_batch(int prec, const TcDev* ds, const int2* bmap, int nblocks, int k, cudaStream_t s);
void tc_launch_mean_batch(int prec, const TcDev* ds, int ncases, int maxNr, int k, cudaStream_t s);
int tc_line_batch_block();
void tc_launch_setup_tables(const TcDev& d, cudaStream_t s);
void tc_launch_init_state(const TcDev& d, cudaStream_t s);
// zero the (0,0) and Nyquist slots and make the m = 0 column Hermitian
void tc_launch_realify(const TcDev& d, double2* field, cudaStream_t s);
void tc_launch_to_physical(const TcDev& d, const double2* field, cudaStream_t s);
void tc_launch_energy(const TcDev& d, cudaStream_t s);
// transform lengths with a compile-time plan in the FFT kernels
bool tc_fft_fixed_length(int M);
// sum over Fourier slots of 2 S:S at every radial point -> d.dprof
// (scratch: pbuf for the radial derivatives, zbuf for the densities)
void tc_launch_strain(const TcDev& d, cudaStream_t s);
cudaError_t tc_set_kernel_attributes();
cudaError_t tc_set_line_kernel_attributes();

/*
 * tc.h -- C ABI of libtc: one GPU (sm_103a) implementation of the time step
 * of the v-eta DNS method for Taylor-Couette flow of Pirro & Quadrio,
 * "Direct Numerical Simulation of turbulent Taylor-Couette flow".
 *
 * Physical problem (Sec. 2): fluid between coaxial cylinders of radii R_i and
 * R_o, radius ratio zeta = R_i/R_o, gap R_o - R_i = 2h.  Lengths are in h,
 * velocities in W_i (inner-wall speed), time in h/W_i.  Re = W_i 2h / nu, so
 * the viscous coefficient of the non-dimensional equations is 2/Re.
 *
 * Unknowns (Appendix): per Fourier pair (m, alpha), the radial velocity v and
 * the radial vorticity eta as functions of r, plus the mean profiles U(r)
 * (axial) and W(r) (azimuthal).  One call of tc_step advances them by the
 * 3-substep implicit/explicit Runge-Kutta scheme (Sec. 2.1), each substep
 * being: rebuild u, w from continuity, pseudo-spectral products with the 3/2
 * rule, the radial rows of Eqs. 6 and 7 with 5-point compact explicit
 * finite differences, and one banded radial solve per pair and variable.
 *
 * Conventions shared by every call:
 *  - Spectral arrays are complex128 (re, im interleaved), shaped
 *    [Nr][Nz][Ntheta/2], the last index fastest.  Azimuthal index j = 0 ..
 *    Ntheta/2-1 with m = j*m0; axial slots in FFT order n = 0..Nz/2-1,
 *    [Nz/2: Nyquist, always zero], -Nz/2+1..-1 with alpha = n*alpha0.
 *    Slot (j=0, n<0) holds the conjugate of (0, -n).  Slot (0, 0) of U and W
 *    holds the mean profiles; of v and eta it is zero.
 *  - Physical arrays are float64 shaped [Nr][Mz][Mt] with Mt = 3 Ntheta/2,
 *    Mz = 3 Nz/2, points theta_p = p Theta/Mt, z_q = q Lz/Mz.
 *  - Host buffers are owned by the caller; every call that takes one is
 *    synchronous with respect to that buffer.  Device memory is owned by the
 *    handle and freed by tc_destroy.
 *  - Return codes: 0 on success, a negative TC_ERR_* value on failure;
 *    tc_last_error() then returns a message (thread-local).
 *  - A handle may be used by one host thread at a time.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_handle tc_handle;

enum {
    TC_OK = 0,
    TC_ERR_ARG = -1,        /* invalid argument */
    TC_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    TC_ERR_NONFINITE = -3,  /* a NaN or Inf appeared in the state */
    TC_ERR_SIZE = -4,       /* buffer size does not match the field */
    TC_ERR_TIMEOUT = -5,    /* a bounded device wait ran out */
    TC_ERR_STATE = -6       /* a table could not be built (zero pivot) */
};

enum {                      /* field selector of tc_get_field / tc_set_field */
    TC_FIELD_U = 0,         /* axial velocity u (spectral: (0,0) slot = U(r)) */
    TC_FIELD_V = 1,         /* radial velocity v */
    TC_FIELD_W = 2,         /* azimuthal velocity w (spectral: (0,0) slot = W(r)) */
    TC_FIELD_ETA = 3,       /* radial vorticity eta = (i m/r) u - i alpha w */
    TC_FIELD_MEAN_U = 4,    /* mean axial profile U(r), float64 [Nr] */
    TC_FIELD_MEAN_W = 5     /* mean azimuthal profile W(r), float64 [Nr] */
};

enum { TC_SPECTRAL = 0, TC_PHYSICAL = 1 };

enum {
    TC_PREC_FP64 = 0,       /* every step in float64 */
    TC_PREC_MIXED = 1,      /* FFTs, products and explicit radial rows in
                               float32, their continuity term in double-float;
                               banded solves, RK memory, reconstruction and
                               the mean mode in float64 */
    TC_PREC_DF64 = 2        /* FFTs, products and explicit radial rows in
                               double-float arithmetic (pairs of float32, ~48
                               significand bits) on the float32 pipe; solves,
                               RK memory, reconstruction and the mean mode in
                               float64 */
};

typedef struct {
    int Nr, Ntheta, Nz;     /* radial points; Fourier modes in theta and z   */
    double radius_ratio;    /* zeta = R_i/R_o, 0 < zeta < 1                    */
    double Re_inner;        /* Re = W_i 2h/nu > 0                              */
    double Re_outer;        /* outer-wall Reynolds number (0: outer at rest)   */
    double dt;              /* time step in h/W_i, > 0                         */
    double Theta;           /* azimuthal box (radians); <= 0: L_theta = 10 pi h
                               at the centreline (Sec. 4)                      */
    double Lz;              /* axial box in h; <= 0: 5 h (Sec. 4)              */
    int precision;          /* TC_PREC_FP64, TC_PREC_MIXED or TC_PREC_DF64     */
    int device;             /* CUDA device ordinal; < 0: current device        */
    int autotune;           /* 1: time the candidate tile shapes of the z
                               transforms and the line-kernel variants at
                               creation, and the column groups of the step
                               graph (1 or 2) on the first tc_step of three or
                               more steps, keeping the fastest (cached per
                               shape class); results do not depend on the
                               choices                                         */
    double stretch;         /* radial grid: 0 uniform; a > 0 the tanh map
                               r_j = (R_i + 1) + tanh(a s_j)/tanh(a),
                               s_j = -1 + 2j/(Nr-1), denser at both walls (the
                               paper's grid is "smoothly stretched", Sec. 2.1) */
} tc_params;

typedef struct {
    double t;               /* time (h/W_i) */
    long long step;         /* completed steps */
    double G_inner;         /* torque T/(mu W_i L R_i) at the inner wall: Eq. 2
                               read as 2 pi R_i |W' - W/r| (Table 2) */
    double G_outer;         /* same at the outer wall: 2 pi R_o^2/R_i |W' - W/r| */
    double Re_tau_inner;    /* u_tau h/nu with u_tau^2 = nu |W' - W/r| (Sec. 5) */
    double Re_tau_outer;
    double energy;          /* (1/2) <|u|^2> over the volume */
    double dissipation;     /* nu <2 S:S>: viscous dissipation per unit volume,
                               S the strain rate, radial derivatives by the
                               compact first derivative (walls one-sided) */
    double power_in;        /* work of the wall shear stress on the moving
                               walls per unit volume:
                               nu [R_o W_o (W'-W/r)(R_o) - R_i W_i (W'-W/r)(R_i)]
                               / ((R_o^2 - R_i^2)/2); dE/dt = power_in -
                               dissipation */
} tc_stats;

/* Create a case with the default box of Sec. 4, float64 precision and the
 * tile autotuner on.
 * Nr >= 9; Ntheta a multiple of 4 of the form 2^a 3^b; Nz even >= 4 with prime
 * factors in {2, 3, 5, 7, 11, 13, 17} (the paper's 170 included);
 * 0 < zeta < 1; Re > 0;
 * dt > 0.  The state starts as circular Couette flow (Eq. 1, W(R_o) =
 * Re_outer/Re_inner) with zero perturbation.  Returns NULL on error. */
tc_handle* tc_create(int Nr, int Ntheta, int Nz, double radius_ratio,
                     double Re_inner, double Re_outer, double dt);

/* Same with every parameter explicit. */
tc_handle* tc_create_ex(const tc_params* params);

/* Advance nsteps full Runge-Kutta steps (3 substeps each, Sec. 2.1).
 * Launches on the handle's stream and waits for it.  Returns TC_ERR_NONFINITE
 * if a NaN or Inf appeared in v or eta. */
int tc_step(tc_handle* h, int nsteps);

/* Advance nsub Runge-Kutta substeps (a step is 3 substeps; Sec. 2.1), without
 * the captured graph.  Time and the step counter advance when a step is
 * completed.  tc_step may only be called at a step boundary (it returns
 * TC_ERR_ARG otherwise). */
int tc_advance_substeps(tc_handle* h, int nsub);

/* Copy one field into host_buf.  bytes must equal tc_field_bytes(h, which,
 * space).  Spectral: complex128 [Nr][Nz][Ntheta/2]; physical: float64
 * [Nr][Mz][Mt]; MEAN_U/MEAN_W: float64 [Nr] (space ignored). */
int tc_get_field(tc_handle* h, int which, int space, void* host_buf, size_t bytes);

/* Replace v (TC_FIELD_V), eta (TC_FIELD_ETA) or a mean profile (MEAN_U,
 * MEAN_W) from a host buffer (spectral layout / float64 [Nr]).  The m = 0
 * column is made Hermitian from its n > 0 slots, the Nyquist slot and (0,0)
 * are zeroed.  The Runge-Kutta memory restarts from this state. */
int tc_set_field(tc_handle* h, int which, const void* host_buf, size_t bytes);

/* The same without waiting (spectral space and mean profiles only), for
 * callers that overlap their copies with other work; buf must stay valid,
 * and host memory should be page-locked, until the copy has run.  buf may
 * also be device memory of the handle's GPU (the copy direction follows
 * from the address): a caller that moves the next input from the host into
 * a device staging buffer while a step runs, and reads results back through
 * one, overlaps the host link with the steps.
 *   tc_set_field_async: queued on the handle's stream (so ordered before the
 *     next step, which also runs there); the RK memory restarts as above.
 *   tc_get_field_async: the copy is ordered after everything queued so far on
 *     the handle's stream and runs on `cuda_stream` (NULL: the handle's
 *     stream); the caller waits for that stream before reading buf.
 * A pageable host buffer makes the copy synchronous. */
int tc_set_field_async(tc_handle* h, int which, const void* buf, size_t bytes);
int tc_get_field_async(tc_handle* h, int which, void* buf, size_t bytes, void* cuda_stream);

/* Bytes of one field in the given space. */
size_t tc_field_bytes(const tc_handle* h, int which, int space);

/* Checkpoint / resume (the paper saves fields every 10 time units, Sec. 4;
 * here the whole time-stepping state is saved, so that a resumed run is bit
 * for bit the run that was not interrupted):
 *   tc_state_bytes: size of a state image of this case;
 *   tc_save_state:  writes the image into the caller's host buffer: a header
 *                   (shape, time, step count, RK phase) and, as float64, v,
 *                   eta, u, w and the RK memories H_v, H_eta ([Nr][Nz][Ntheta/2]
 *                   complex128 each), then U, W and their RK memories ([Nr]);
 *   tc_load_state:  restores an image saved from a case of the same Nr,
 *                   Ntheta and Nz (any precision form and tiles); TC_ERR_SIZE
 *                   for a wrong size, TC_ERR_ARG for another shape or a
 *                   damaged header.
 * Both are synchronous and must not overlap a step in flight. */
size_t tc_state_bytes(const tc_handle* h);
int tc_save_state(tc_handle* h, void* host_buf, size_t bytes);
int tc_load_state(tc_handle* h, const void* host_buf, size_t bytes);

/* Torque, friction Reynolds numbers, kinetic energy, viscous dissipation
 * and wall power of the current state (synchronous on the handle's stream;
 * uses the handle's transform scratch, so not while a step is in flight). */
int tc_torque_stats(tc_handle* h, tc_stats* out);

/* Launch stream (a cudaStream_t, or NULL for the legacy default stream). */
int tc_set_stream(tc_handle* h, void* cuda_stream);

/* Override the launch shapes the autotuner would choose (for tuning studies
 * and tests; no counterpart in the paper; the arithmetic is the same for
 * every choice):
 *   ztile: azimuthal columns per block of the z transforms, 1, 2, 4 or 8,
 *          dividing Ntheta/2 (0 keeps the current value);
 *   line_variant: line-kernel launch shape, 64, 128 or 256 threads per
 *          block, 1003 / 1004 (128 threads, budget for 3 / 4 blocks per
 *          SM), 2007 (64 threads, 144 registers) or 3001 (64 threads per 32
 *          pairs: one warp advances v, the other eta, for short line phases
 *          of few pairs); 0 keeps the current;
 *   chunks: column groups of the step graph, in which the z transforms of
 *          one group overlap the line kernel of another: 1 (no overlap), 2,
 *          4 or 8, used when it divides the number of z tiles (0 keeps the
 *          current choice, initially made from the shape).
 * Returns TC_ERR_ARG for other values; a captured step graph is rebuilt. */
int tc_set_tiles(tc_handle* h, int ztile, int line_variant, int chunks);

/* The launch shapes in use (after the autotuner): z tile, line-kernel
 * variant and column groups of the step graph (1: no overlap).  Any pointer
 * may be NULL.  A step graph launches 15 kernels without groups and
 * 7 + 8 * chunks with them, 3 more with the deferred RK memory below. */
int tc_get_tiles(const tc_handle* h, int* ztile, int* line_variant, int* chunks);

/* Deferred RK memory (double-float and mixed forms; no counterpart in the
 * paper, same bits either way).  The implicit part of the next substep's
 * low-storage RK memory, H += (beta_k + alpha_k+1) dt L x^(k+1) (Sec. 2.3;
 * L the implicit band of Eq. 6 or 7), needs only the new v and eta.  With
 * the deferral on, the line kernel leaves it out and a kernel of its own
 * adds it beside the next substep's theta rows, whose float32 or
 * double-float work leaves the float64 pipe idle; within one tc_step call
 * the last substep's term of a step runs beside the next step's first
 * theta rows, and the last one is completed before tc_step returns.
 *   mode: -1 chosen by timing with the autotuner (the default; off without
 *         it), 0 off, 1 on.  No effect in the float64 form.
 * tc_get_rk_deferral reports whether it is on (1) or off (0).  TC_ERR_ARG
 * for a null handle or another mode; a captured step graph is rebuilt. */
int tc_set_rk_deferral(tc_handle* h, int mode);
int tc_get_rk_deferral(const tc_handle* h, int* on);

/* Device bytes held by the handle. */
size_t tc_device_bytes(const tc_handle* h);

void tc_destroy(tc_handle* h);

/* Measurement helpers (no counterpart in the paper). */

#define TC_NPHASES 5
/* Run nsteps steps kernel by kernel (no graph) with CUDA events between the
 * kernels on the handle's stream; ms[i] receives the average duration of one
 * launch of kernel i: 0 inverse z FFT, 1 theta transforms + products,
 * 2 forward z FFT, 3 line phase (Eqs. 6-7 rows and solves), 4 mean flow.
 * nphases must be >= TC_NPHASES.  The state advances by nsteps. */
int tc_phase_times(tc_handle* h, int nsteps, double* ms, int nphases);

/* Fused multiply-add throughput of the device (TFLOP/s, 2 flops per FMA) in
 * float64 and float32, from a short probe kernel; device < 0: current. */
int tc_fma_peak(int device, double* fp64_tflops, double* fp32_tflops);

/* Message of the last failed call on this host thread ("" if none). */
const char* tc_last_error(void);

/* ---- many cases on one GPU (the paper runs one case; no counterpart) ---- */

/* Device bytes tc_create_ex would allocate for these parameters (0 if they
 * are invalid); used for admission against a device-memory budget. */
size_t tc_estimate_device_bytes(const tc_params* params);

/* Batch: ncases independent cases (params[i] each, any shapes and
 * precisions), each with its own resident state; tc_batch_step advances all
 * of them by nsteps steps with one CUDA-graph launch per step.  Cases of the
 * same precision form, Ntheta and Nz make one shape class (any Nr, radius
 * ratio, Re and box).  Per substep, each of the three plane-phase kernels is
 * one launch per class covering all of its cases (the classes run as
 * concurrent graph branches), then the line kernel and the mean flow are one
 * launch each per precision form, covering all of its cases.  Cases are
 * reached with tc_batch_case for tc_set_field / tc_get_field /
 * tc_torque_stats; the handle stays owned by the batch.  Results equal those
 * of the same case stepped alone, bit for bit.
 * tc_batch_set_stream: the caller keeps ownership of the stream.
 * tc_batch_launches_per_step: kernels one step launches,
 * 3 x (3 x classes + 2 x forms). */
typedef struct tc_batch tc_batch;
tc_batch* tc_batch_create(int ncases, const tc_params* params);
tc_handle* tc_batch_case(tc_batch* b, int i);
int tc_batch_step(tc_batch* b, int nsteps);
int tc_batch_set_stream(tc_batch* b, void* cuda_stream);
int tc_batch_launches_per_step(const tc_batch* b);
size_t tc_batch_device_bytes(const tc_batch* b);
void tc_batch_destroy(tc_batch* b);

/* Server: continuous batching of independent cases.  tc_server_submit queues
 * a request (parameters, optional initial v and eta in the spectral layout,
 * copied at submission, number of steps, optional caller-owned host buffers
 * that receive the final v and eta); a worker thread admits queued requests
 * while the estimated device bytes of the admitted cases stay within
 * budget_bytes and at most max_active run, steps the admitted cases, and on
 * completion writes the outputs, frees the case and admits more.  Modes:
 *   TC_SERVE_PER_CASE (tc_server_create): every case on its own stream with
 *     its own step graph and one step in flight, relaunched as soon as it
 *     completes, so each case's step latency is its own.
 *   TC_SERVE_GROUPED: all admitted cases advance together, one step per
 *     graph launch of the batch's grouped kernels (one launch per plane
 *     kernel and shape class, one line-kernel and one mean-flow launch per
 *     precision form); the graph is captured again whenever the set of cases
 *     changes, which happens between steps only.  Every case's per-step
 *     latency is that of the group step.
 * Results equal those of the same case stepped alone in either mode.
 * Requests that alone exceed the budget are refused with TC_ERR_SIZE.
 * Thread-safe: submit / poll / drain / stats may be called from any host
 * thread.  tc_server_destroy drops queued requests and stops running ones
 * after their current step. */
enum { TC_SERVE_PER_CASE = 0, TC_SERVE_GROUPED = 1 };
typedef struct tc_server tc_server;
typedef struct {
    long long id;           /* from tc_server_submit */
    int status;             /* TC_OK or a TC_ERR_* code */
    long long steps;        /* steps completed */
    tc_stats stats;         /* final torque, Re_tau, energy */
    double queue_ms;        /* submission to admission */
    double run_ms;          /* admission to completion */
    double step_ms_p50;     /* per-step device latency (CUDA events) */
    double step_ms_p99;
} tc_result;
typedef struct {
    long long submitted, finished, queued, active, peak_active, steps;
    size_t budget_bytes, used_bytes, peak_used_bytes;
    double gridpoint_steps; /* sum over finished cases of Nr Ntheta Nz steps */
    double busy_ms;         /* first admission to last completion */
    double step_ms_p50, step_ms_p99;   /* over every step of finished cases */
} tc_server_stats_t;
tc_server* tc_server_create(size_t budget_bytes, int max_active, int device);
tc_server* tc_server_create_ex(size_t budget_bytes, int max_active, int device, int mode);
int tc_server_submit(tc_server* s, const tc_params* params, const void* v0, const void* eta0,
                     int nsteps, void* out_v, void* out_eta, long long* id);
int tc_server_poll(tc_server* s, tc_result* out, int max_results, int* count);
int tc_server_drain(tc_server* s, double timeout_s);
int tc_server_stats(tc_server* s, tc_server_stats_t* out);
void tc_server_destroy(tc_server* s);

/* ---- one case split across ranks (a transpose form of the paper's
 * distributed solver, Sec. 3.1; the paper pipelines radial slabs instead) ----
 *
 * Each rank holds a handle of the whole case (every array full-size) and is
 * given a share: radial planes [r0, r1) for the plane phase (transforms and
 * products, which are independent per plane) and azimuthal columns
 * [j0, j1) -- every axial slot of those columns -- for the line phase
 * (Eqs. 6-7 rows and solves, which couple all planes of one pair); the rank
 * with j0 = 0 also advances the mean flow.  One substep is
 *   1. exchange: every rank receives u, v, w of the other ranks' columns on
 *      its planes (written into its own u, v, w arrays there);
 *   2. tc_split_planes: the plane phase of its planes -> the slab products,
 *      TC_ARRAY_PROD_SLAB [5][r1-r0][Nz][Ntheta/2];
 *   3. exchange: every rank receives the slab products of all ranks for its
 *      columns (written into TC_ARRAY_PROD [5][Nr][Nz][Ntheta/2] there);
 *   4. tc_split_pairs: the line phase of its columns (and the mean flow).
 * The exchanges are the caller's (an all-to-all of each rank's collective
 * library), on the arrays tc_device_array returns; the results equal those
 * of tc_step bit for bit.  Products are complex128 in the float64 form,
 * complex64 in the mixed form and pairs of (hi, lo) float pairs in the
 * double-float form (16 bytes).  The products 0..4 are uu - vv, uv, uw, vw,
 * ww - vv.  tc_split_planes / tc_split_pairs queue work on the handle's
 * stream and return without waiting; tc_split_finish waits and reports a
 * non-finite state (TC_ERR_NONFINITE).  tc_split_set allocates the slab
 * buffer and may be called between steps only. */
enum { TC_ARRAY_U = 0, TC_ARRAY_V = 1, TC_ARRAY_W = 2, TC_ARRAY_ETA = 3,
       TC_ARRAY_PROD = 4, TC_ARRAY_PROD_SLAB = 5 };
int tc_split_set(tc_handle* h, int r0, int r1, int j0, int j1);
int tc_split_planes(tc_handle* h);
int tc_split_pairs(tc_handle* h);
int tc_split_finish(tc_handle* h);
/* Device address of one of the handle's resident arrays (NULL for an
 * unknown selector or a slab buffer not yet allocated); owned by the
 * handle.  u, v, w, eta: complex128 [Nr][Nz][Ntheta/2]. */
void* tc_device_array(tc_handle* h, int which);

/* Spectral -> physical transform that allocates nothing (no counterpart in
 * the paper).
 *
 * For callers that are not allowed to allocate device memory -- code held to
 * a device-memory budget fixed in advance, plug-ins whose host application
 * owns every buffer, loops where cudaMalloc and its implicit synchronisation
 * are forbidden.  It computes the same physical field as tc_get_field(h,
 * which, TC_PHYSICAL, ...) but needs no handle: spectral_dev is a device
 * array complex128 [Nr][Nz][Ntheta/2] (layout above), physical_dev a device
 * array float64 [Nr][3Nz/2][3Ntheta/2]; both are owned by the caller.  The
 * work is queued on cuda_stream (NULL: legacy default stream) and the call
 * returns without waiting.
 *
 * Its intermediates (the z-transformed (3Nz/2) x (Ntheta/2) complex planes,
 * as many radial planes per pass as fit) and the twiddle tables, computed on
 * the device at every call, live in a static device array of
 * TC_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  Sizes for which one plane plus the tables exceeds it, or
 * whose padded lengths need more than 200 KB of shared memory per transform
 * block (2 x 16 bytes per point of 3Nz/2 or 3Ntheta/2, times the 1-8 columns
 * of a z block), are rejected with TC_ERR_SIZE before anything is queued.
 * The first
 * call on a device does a one-time set-up with that device current (it
 * fetches the array's device address and opts the kernels into large shared
 * memory); make that first call before any stream capture.  All calls share
 * the array and each call overwrites it (nothing in it needs to start at
 * zero), so calls that overlap on the GPU -- on different streams, or from
 * different host threads -- race and must be serialised by the caller. */
#define TC_NOALLOC_SCRATCH_BYTES (16u << 20)
int tc_to_physical_noalloc(int Nr, int Ntheta, int Nz, const void* spectral_dev,
                           void* physical_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */

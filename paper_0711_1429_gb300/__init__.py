"""Python binding of libtc (include/tc.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of libtc.so; this module
converts numpy arrays to host pointers and return codes to exceptions.  It
loads the in-tree library on first use and raises if it has not been built
(there is no fallback path).
"""
import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")
HEADER = os.path.join(_HERE, "..", "include", "tc.h")

TC_OK, TC_ERR_ARG, TC_ERR_CUDA, TC_ERR_NONFINITE, TC_ERR_SIZE, TC_ERR_TIMEOUT, TC_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
TC_FIELD_U, TC_FIELD_V, TC_FIELD_W, TC_FIELD_ETA, TC_FIELD_MEAN_U, TC_FIELD_MEAN_W = range(6)
TC_SPECTRAL, TC_PHYSICAL = 0, 1
TC_PREC_FP64, TC_PREC_MIXED, TC_PREC_DF64 = 0, 1, 2
TC_ARRAY_U, TC_ARRAY_V, TC_ARRAY_W, TC_ARRAY_ETA, TC_ARRAY_PROD, TC_ARRAY_PROD_SLAB = range(6)
TC_SERVE_PER_CASE, TC_SERVE_GROUPED = 0, 1
TC_NOALLOC_SCRATCH_BYTES = 16 << 20     # size of the fixed array of tc_to_physical_noalloc


class TcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtc error {code}: {msg}")
        self.code = code


class tc_params(ctypes.Structure):
    _fields_ = [("Nr", ctypes.c_int), ("Ntheta", ctypes.c_int), ("Nz", ctypes.c_int),
                ("radius_ratio", ctypes.c_double), ("Re_inner", ctypes.c_double),
                ("Re_outer", ctypes.c_double), ("dt", ctypes.c_double),
                ("Theta", ctypes.c_double), ("Lz", ctypes.c_double),
                ("precision", ctypes.c_int), ("device", ctypes.c_int), ("autotune", ctypes.c_int),
                ("stretch", ctypes.c_double)]


class tc_stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("step", ctypes.c_longlong),
                ("G_inner", ctypes.c_double), ("G_outer", ctypes.c_double),
                ("Re_tau_inner", ctypes.c_double), ("Re_tau_outer", ctypes.c_double),
                ("energy", ctypes.c_double), ("dissipation", ctypes.c_double),
                ("power_in", ctypes.c_double)]


class tc_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("steps", ctypes.c_longlong),
                ("stats", tc_stats), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("step_ms_p50", ctypes.c_double), ("step_ms_p99", ctypes.c_double)]


class tc_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("finished", ctypes.c_longlong),
                ("queued", ctypes.c_longlong), ("active", ctypes.c_longlong),
                ("peak_active", ctypes.c_longlong), ("steps", ctypes.c_longlong),
                ("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
                ("peak_used_bytes", ctypes.c_size_t), ("gridpoint_steps", ctypes.c_double),
                ("busy_ms", ctypes.c_double), ("step_ms_p50", ctypes.c_double),
                ("step_ms_p99", ctypes.c_double)]


_lib = None


def lib():
    """The loaded libtc.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_0711_1429_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    L.tc_create.restype = vp
    L.tc_create.argtypes = [i, i, i, d, d, d, d]
    L.tc_create_ex.restype = vp
    L.tc_create_ex.argtypes = [ctypes.POINTER(tc_params)]
    L.tc_step.restype = i
    L.tc_step.argtypes = [vp, i]
    L.tc_advance_substeps.restype = i
    L.tc_advance_substeps.argtypes = [vp, i]
    L.tc_get_field.restype = i
    L.tc_get_field.argtypes = [vp, i, i, vp, sz]
    L.tc_set_field.restype = i
    L.tc_set_field.argtypes = [vp, i, vp, sz]
    L.tc_field_bytes.restype = sz
    L.tc_field_bytes.argtypes = [vp, i, i]
    L.tc_torque_stats.restype = i
    L.tc_torque_stats.argtypes = [vp, ctypes.POINTER(tc_stats)]
    L.tc_set_stream.restype = i
    L.tc_set_stream.argtypes = [vp, vp]
    L.tc_state_bytes.restype = sz
    L.tc_state_bytes.argtypes = [vp]
    L.tc_save_state.restype = i
    L.tc_save_state.argtypes = [vp, vp, sz]
    L.tc_load_state.restype = i
    L.tc_load_state.argtypes = [vp, vp, sz]
    L.tc_set_tiles.restype = i
    L.tc_set_tiles.argtypes = [vp, i, i, i]
    L.tc_set_rk_deferral.restype = i
    L.tc_set_rk_deferral.argtypes = [vp, i]
    L.tc_get_rk_deferral.restype = i
    L.tc_get_rk_deferral.argtypes = [vp, ctypes.POINTER(i)]
    L.tc_get_tiles.restype = i
    L.tc_get_tiles.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    L.tc_device_bytes.restype = sz
    L.tc_device_bytes.argtypes = [vp]
    L.tc_destroy.restype = None
    L.tc_destroy.argtypes = [vp]
    L.tc_phase_times.restype = i
    L.tc_phase_times.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double), i]
    L.tc_fma_peak.restype = i
    L.tc_fma_peak.argtypes = [i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.tc_to_physical_noalloc.restype = i
    L.tc_to_physical_noalloc.argtypes = [i, i, i, vp, vp, vp]
    L.tc_estimate_device_bytes.restype = sz
    L.tc_estimate_device_bytes.argtypes = [ctypes.POINTER(tc_params)]
    L.tc_batch_create.restype = vp
    L.tc_batch_create.argtypes = [i, ctypes.POINTER(tc_params)]
    L.tc_batch_case.restype = vp
    L.tc_batch_case.argtypes = [vp, i]
    L.tc_batch_step.restype = i
    L.tc_batch_step.argtypes = [vp, i]
    L.tc_batch_set_stream.restype = i
    L.tc_batch_set_stream.argtypes = [vp, vp]
    for nm in ("tc_split_planes", "tc_split_pairs", "tc_split_finish"):
        getattr(L, nm).restype = i
        getattr(L, nm).argtypes = [vp]
    L.tc_split_set.restype = i
    L.tc_split_set.argtypes = [vp, i, i, i, i]
    L.tc_device_array.restype = vp
    L.tc_device_array.argtypes = [vp, i]
    L.tc_set_field_async.restype = i
    L.tc_set_field_async.argtypes = [vp, i, vp, sz]
    L.tc_get_field_async.restype = i
    L.tc_get_field_async.argtypes = [vp, i, vp, sz, vp]
    L.tc_batch_launches_per_step.restype = i
    L.tc_batch_launches_per_step.argtypes = [vp]
    L.tc_batch_device_bytes.restype = sz
    L.tc_batch_device_bytes.argtypes = [vp]
    L.tc_batch_destroy.restype = None
    L.tc_batch_destroy.argtypes = [vp]
    L.tc_server_create.restype = vp
    L.tc_server_create.argtypes = [sz, i, i]
    L.tc_server_create_ex.restype = vp
    L.tc_server_create_ex.argtypes = [sz, i, i, i]
    L.tc_server_submit.restype = i
    L.tc_server_submit.argtypes = [vp, ctypes.POINTER(tc_params), vp, vp, i, vp, vp,
                                   ctypes.POINTER(ctypes.c_longlong)]
    L.tc_server_poll.restype = i
    L.tc_server_poll.argtypes = [vp, ctypes.POINTER(tc_result), i, ctypes.POINTER(ctypes.c_int)]
    L.tc_server_drain.restype = i
    L.tc_server_drain.argtypes = [vp, d]
    L.tc_server_stats.restype = i
    L.tc_server_stats.argtypes = [vp, ctypes.POINTER(tc_server_stats_t)]
    L.tc_server_destroy.restype = None
    L.tc_server_destroy.argtypes = [vp]
    L.tc_last_error.restype = ctypes.c_char_p
    L.tc_last_error.argtypes = []
    _lib = L
    return L


def declared_functions():
    """Names of the functions declared in include/tc.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z_]+)\s*\(", src)))


def _check(rc):
    if rc != TC_OK:
        raise TcError(rc, lib().tc_last_error().decode())
    return rc


def tc_create(Nr, Ntheta, Nz, radius_ratio, Re_inner, Re_outer, dt):
    """New FP64 case on the current device: Nr radial points, Ntheta x Nz
    Fourier modes, radius ratio R_i/R_o, Reynolds numbers of the inner and
    outer cylinder on the gap, time step in h/W_i.  Laminar Couette start."""
    h = lib().tc_create(Nr, Ntheta, Nz, radius_ratio, Re_inner, Re_outer, dt)
    if not h:
        raise TcError(TC_ERR_ARG, lib().tc_last_error().decode())
    return h


def make_params(Nr, Ntheta, Nz, radius_ratio, Re_inner, Re_outer, dt, Theta=0.0, Lz=0.0,
                precision=TC_PREC_FP64, device=-1, autotune=0, stretch=0.0):
    return tc_params(Nr, Ntheta, Nz, radius_ratio, Re_inner, Re_outer, dt, Theta, Lz, precision, device,
                     autotune, stretch)


def tc_create_ex(Nr, Ntheta, Nz, radius_ratio, Re_inner, Re_outer, dt, Theta=0.0, Lz=0.0,
                 precision=TC_PREC_FP64, device=-1, autotune=0, stretch=0.0):
    """New case with the full parameter set: box (Theta in radians, Lz in h;
    0 for the default box), arithmetic form (TC_PREC_*), device, tile autotuning and
    tanh stretching of the radial grid."""
    p = make_params(Nr, Ntheta, Nz, radius_ratio, Re_inner, Re_outer, dt, Theta, Lz, precision, device,
                    autotune, stretch)
    h = lib().tc_create_ex(ctypes.byref(p))
    if not h:
        raise TcError(TC_ERR_ARG, lib().tc_last_error().decode())
    return h


def tc_step(h, nsteps=1):
    """Advance by `nsteps` full three-substep Runge-Kutta steps; raises
    TcError (e.g. TC_ERR_NONFINITE) on failure."""
    return _check(lib().tc_step(h, nsteps))


def tc_advance_substeps(h, nsub=1):
    """Advance by `nsub` single Runge-Kutta substeps (phase kept across calls)."""
    return _check(lib().tc_advance_substeps(h, nsub))


def tc_field_bytes(h, which, space=TC_SPECTRAL):
    return lib().tc_field_bytes(h, which, space)


def _field_shape(h, which, space):
    nbytes = tc_field_bytes(h, which, space)
    if which in (TC_FIELD_MEAN_U, TC_FIELD_MEAN_W):
        return (nbytes // 8,), np.float64
    if space == TC_PHYSICAL:
        return (nbytes // 8,), np.float64
    return (nbytes // 16,), np.complex128


def tc_get_field(h, which, space=TC_SPECTRAL, out=None):
    """Copy a field into `out` (a C-contiguous numpy array of the right byte
    size) or a new flat array; reshape with the case's dimensions."""
    if out is None:
        shape, dt = _field_shape(h, which, space)
        out = np.empty(shape, dtype=dt)
    if not out.flags.c_contiguous:
        raise ValueError("output array must be C-contiguous")
    _check(lib().tc_get_field(h, which, space, out.ctypes.data, out.nbytes))
    return out


def tc_set_field(h, which, arr):
    """Set v or eta (complex128 [Nr][Nz][Ntheta/2]) or the mean profile U or
    W (float64 [Nr]); setting v or eta restarts the Runge-Kutta memory."""
    arr = np.ascontiguousarray(arr)
    if which in (TC_FIELD_MEAN_U, TC_FIELD_MEAN_W):
        arr = np.ascontiguousarray(arr, dtype=np.float64)
    else:
        arr = np.ascontiguousarray(arr, dtype=np.complex128)
    return _check(lib().tc_set_field(h, which, arr.ctypes.data, arr.nbytes))


def tc_set_field_ptr(h, which, host_ptr, nbytes):
    """Same as tc_set_field from a raw host pointer (e.g. pinned memory)."""
    return _check(lib().tc_set_field(h, which, host_ptr, nbytes))


def tc_get_field_ptr(h, which, space, host_ptr, nbytes):
    return _check(lib().tc_get_field(h, which, space, host_ptr, nbytes))


def tc_torque_stats(h):
    """Diagnostics of the current state as a dict: time, step, inner and
    outer torque, Re_tau at both walls, kinetic energy, dissipation and wall
    power."""
    s = tc_stats()
    _check(lib().tc_torque_stats(h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in tc_stats._fields_}


def tc_set_stream(h, stream_ptr):
    """Launch this case's work on the given CUDA stream (a cudaStream_t as
    an integer, e.g. torch.cuda.Stream().cuda_stream)."""
    return _check(lib().tc_set_stream(h, stream_ptr))


def tc_save_state(h):
    """The whole time-stepping state as a bytes object (see tc.h)."""
    n = lib().tc_state_bytes(h)
    buf = ctypes.create_string_buffer(n)
    _check(lib().tc_save_state(h, buf, n))
    return buf.raw


def tc_load_state(h, image):
    """Restore a state image from tc_save_state of a case of the same shape;
    the next step continues bit for bit."""
    buf = ctypes.create_string_buffer(image, len(image))
    return _check(lib().tc_load_state(h, buf, len(image)))


LINE_VARIANTS = (64, 128, 256, 1003, 1004, 2007, 3001)


def tc_set_tiles(h, ztile=0, line_variant=0, chunks=0):
    """Pin the z tile, the line-kernel variant (LINE_VARIANTS) and the column
    groups of the overlapped step; 0 keeps the current choice.  No launch
    shape changes the results."""
    return _check(lib().tc_set_tiles(h, ztile, line_variant, chunks))


def tc_get_tiles(h):
    """(ztile, line_variant, chunks) in use."""
    z, l, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().tc_get_tiles(h, ctypes.byref(z), ctypes.byref(l), ctypes.byref(c)))
    return z.value, l.value, c.value


def step_kernels(chunks, rk_deferred=False):
    """Kernels one step launches: the step graph, plus the three RK-memory
    kernels with the deferred RK memory."""
    return (15 if chunks <= 1 else 7 + 8 * chunks) + (3 if rk_deferred else 0)


def tc_set_rk_deferral(h, mode):
    """Deferred RK memory of the double-float and mixed forms: -1 chosen by
    timing (the default), 0 off, 1 on (no effect in the float64 form; same
    bits either way)."""
    return _check(lib().tc_set_rk_deferral(h, int(mode)))


def tc_get_rk_deferral(h):
    """Whether the deferred RK memory is on (True) for the captured steps."""
    on = ctypes.c_int()
    _check(lib().tc_get_rk_deferral(h, ctypes.byref(on)))
    return bool(on.value)


def tc_device_bytes(h):
    return lib().tc_device_bytes(h)


def tc_destroy(h):
    """Free the case and all of its device memory (None is ignored)."""
    if h:
        lib().tc_destroy(h)


PHASES = ("z_inverse", "theta_rows_products", "z_forward", "line", "mean")


def tc_phase_times(h, nsteps=1):
    """Average ms per launch of each kernel of the step (dict)."""
    ms = (ctypes.c_double * len(PHASES))()
    _check(lib().tc_phase_times(h, nsteps, ms, len(PHASES)))
    return dict(zip(PHASES, list(ms)))


def tc_fma_peak(device=-1):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().tc_fma_peak(device, ctypes.byref(a), ctypes.byref(b)))
    return {"fp64_tflops": a.value, "fp32_tflops": b.value}


def tc_to_physical_noalloc(Nr, Ntheta, Nz, spectral_dev_ptr, physical_dev_ptr, stream_ptr=None):
    """Allocation-free spectral -> physical transform on caller-owned device
    buffers (see include/tc.h); asynchronous on the given stream."""
    return _check(lib().tc_to_physical_noalloc(Nr, Ntheta, Nz, spectral_dev_ptr, physical_dev_ptr, stream_ptr))


def tc_estimate_device_bytes(params):
    return lib().tc_estimate_device_bytes(ctypes.byref(params))


def tc_set_field_async(h, which, ptr, nbytes):
    """tc_set_field from a caller-owned address, without waiting: page-locked
    host memory, or device memory of the handle's GPU."""
    return _check(lib().tc_set_field_async(h, which, ptr, nbytes))


def tc_get_field_async(h, which, ptr, nbytes, stream_ptr=None):
    """Spectral field into a caller-owned address (page-locked host memory, or
    device memory of the handle's GPU), ordered after the handle's queued
    work and run on stream_ptr (None: the handle's stream)."""
    return _check(lib().tc_get_field_async(h, which, ptr, nbytes, stream_ptr))


def tc_split_set(h, r0, r1, j0, j1):
    """This rank's share of a case split across ranks: radial planes [r0, r1)
    for the plane phase, azimuthal columns [j0, j1) for the line phase."""
    return _check(lib().tc_split_set(h, r0, r1, j0, j1))


def tc_split_planes(h):
    return _check(lib().tc_split_planes(h))


def tc_split_pairs(h):
    return _check(lib().tc_split_pairs(h))


def tc_split_finish(h):
    return _check(lib().tc_split_finish(h))


def tc_device_array(h, which):
    """Device address (an integer) of one of the handle's resident arrays."""
    p = lib().tc_device_array(h, which)
    if not p:
        raise TcError(TC_ERR_ARG, lib().tc_last_error().decode())
    return p


def tc_batch_create(params_list):
    arr = (tc_params * len(params_list))(*params_list)
    b = lib().tc_batch_create(len(params_list), arr)
    if not b:
        raise TcError(TC_ERR_ARG, lib().tc_last_error().decode())
    return b


def tc_batch_case(b, i):
    h = lib().tc_batch_case(b, i)
    if not h:
        raise TcError(TC_ERR_ARG, lib().tc_last_error().decode())
    return h


def tc_batch_step(b, nsteps=1):
    return _check(lib().tc_batch_step(b, nsteps))


def tc_batch_set_stream(b, stream_ptr):
    return _check(lib().tc_batch_set_stream(b, stream_ptr))


def tc_batch_launches_per_step(b):
    """Kernels one batch step launches: 3 x (3 x shape classes + 2 x precision forms)."""
    n = lib().tc_batch_launches_per_step(b)
    if n < 0:
        _check(n)
    return n


def tc_batch_device_bytes(b):
    return lib().tc_batch_device_bytes(b)


def tc_batch_destroy(b):
    if b:
        lib().tc_batch_destroy(b)


def tc_server_create(budget_bytes, max_active=64, device=-1, mode=None):
    """Server of independent cases within a device budget; mode
    TC_SERVE_PER_CASE (default: each case on its own stream) or
    TC_SERVE_GROUPED (all admitted cases step together in grouped launches)."""
    s = lib().tc_server_create_ex(budget_bytes, max_active, device, TC_SERVE_PER_CASE if mode is None else mode)
    if not s:
        raise TcError(TC_ERR_ARG, lib().tc_last_error().decode())
    return s


def tc_server_submit(s, params, v0=None, eta0=None, nsteps=1, out_v=None, out_eta=None):
    """Queue a case; v0/eta0 (complex128 spectral arrays) are copied now;
    out_v/out_eta (C-contiguous complex128 arrays) receive the final fields and
    must stay alive until the request finishes.  Returns the request id."""
    ptr = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.complex128).ctypes.data
    for o in (out_v, out_eta):
        if o is not None and (o.dtype != np.complex128 or not o.flags.c_contiguous):
            raise ValueError("output arrays must be C-contiguous complex128")
    keep = [None if a is None else np.ascontiguousarray(a, dtype=np.complex128) for a in (v0, eta0)]
    rid = ctypes.c_longlong()
    _check(lib().tc_server_submit(s, ctypes.byref(params),
                                  None if keep[0] is None else keep[0].ctypes.data,
                                  None if keep[1] is None else keep[1].ctypes.data,
                                  nsteps, None if out_v is None else out_v.ctypes.data,
                                  None if out_eta is None else out_eta.ctypes.data, ctypes.byref(rid)))
    return rid.value


def tc_server_poll(s, max_results=64):
    out = (tc_result * max_results)()
    n = ctypes.c_int()
    _check(lib().tc_server_poll(s, out, max_results, ctypes.byref(n)))
    res = []
    for r in out[:n.value]:
        d = {k: getattr(r, k) for k, _ in tc_result._fields_ if k != "stats"}
        d["stats"] = {k: getattr(r.stats, k) for k, _ in tc_stats._fields_}
        res.append(d)
    return res


def tc_server_drain(s, timeout_s=600.0):
    return _check(lib().tc_server_drain(s, timeout_s))


def tc_server_stats(s):
    st = tc_server_stats_t()
    _check(lib().tc_server_stats(s, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in tc_server_stats_t._fields_}


def tc_server_destroy(s):
    if s:
        lib().tc_server_destroy(s)


def tc_last_error():
    return lib().tc_last_error().decode()

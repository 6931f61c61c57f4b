"""ctypes binding of libmclbm (the C ABI declared in include/mclbm.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Functions keep the C names; a non-zero status raises MclbmError with
the library's message.  Device buffers are raw device addresses (ints), e.g.
``tensor.data_ptr()`` of a CUDA torch tensor.  There is no CPU fallback: if the
library is missing this module raises on first use.
"""
import ctypes
import os
import threading

from . import build as _build

MCLBM_OK = 0
STATUS = {
    -1: "INVALID_ARG", -2: "UNSTABLE_TAU", -3: "OOM", -4: "CUDA", -5: "NONFINITE", -6: "TIMEOUT", -7: "SHAPE", -8: "IO",
}
FP64, FP32, FP16 = 0, 1, 2
PULL, AA = 0, 1
OPT_LERAY = 1
OPT_EXACT_GAMMA = 2
Q = 19


class MclbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mclbm error {code} ({STATUS.get(code, '?')}): {msg}")
        self.code = code
        self.status = STATUS.get(code, "?")


class Config(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("M", ctypes.c_int32), ("precision", ctypes.c_int32), ("pattern", ctypes.c_int32),
        ("nu", ctypes.c_double), ("Ma", ctypes.c_double), ("dt", ctypes.c_double), ("U_c", ctypes.c_double),
        ("width", ctypes.c_double), ("seed", ctypes.c_uint64), ("init_density", ctypes.c_int32),
        ("options", ctypes.c_int32),
    ]


class Units(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("dx", "U_lat", "dt", "nu_lat", "tau", "omega")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_c = ctypes
_vp = _c.c_void_p
_dp = _c.POINTER(_c.c_double)
_i32p = _c.POINTER(_c.c_int32)
_size_p = _c.POINTER(_c.c_size_t)
_ctx_p = _c.c_void_p

_SIGNATURES = {
    "mclbm_version": (_c.c_char_p, []),
    "mclbm_last_error": (_c.c_char_p, []),
    "mclbm_lattice": (_c.c_int, [_i32p, _dp]),
    "mclbm_compute_units": (_c.c_int, [_c.POINTER(Config), _c.POINTER(Units)]),
    "mclbm_required_bytes": (_c.c_int, [_c.POINTER(Config), _size_p, _size_p]),
    "mclbm_create": (_c.c_int, [_c.POINTER(Config), _vp, _c.c_size_t, _vp, _c.c_size_t, _vp, _c.POINTER(_ctx_p)]),
    "mclbm_destroy": (None, [_ctx_p]),
    "mclbm_get_units": (_c.c_int, [_ctx_p, _c.POINTER(Units)]),
    "mclbm_init_ensemble": (_c.c_int, [_ctx_p, _dp]),
    "mclbm_draw_params": (_c.c_int, [_c.c_uint64, _c.c_int32, _c.c_int32, _c.c_double, _dp]),
    "mclbm_init_tgv": (_c.c_int, [_ctx_p]),
    "mclbm_get_params": (_c.c_int, [_ctx_p, _dp]),
    "mclbm_step": (_c.c_int, [_ctx_p, _c.c_int64]),
    "mclbm_steps_taken": (_c.c_int64, [_ctx_p]),
    "mclbm_get_populations": (_c.c_int, [_ctx_p, _c.c_int32, _vp]),
    "mclbm_set_populations": (_c.c_int, [_ctx_p, _c.c_int32, _vp]),
    "mclbm_moments": (_c.c_int, [_ctx_p, _c.c_int32, _vp, _vp]),
    "mclbm_energy": (_c.c_int, [_ctx_p, _dp, _dp]),
    "mclbm_mean_var": (_c.c_int, [_ctx_p, _vp, _vp]),
    "mclbm_energy_mean_var": (_c.c_int, [_ctx_p, _dp, _vp, _vp]),
    "mclbm_spectrum": (_c.c_int, [_ctx_p, _dp]),
    "mclbm_sf_trace": (_c.c_int, [_ctx_p, _dp]),
    "mclbm_sf_axes": (_c.c_int, [_ctx_p, _c.c_int32, _dp]),
    "mclbm_restrict": (_c.c_int, [_ctx_p, _c.c_int32, _vp]),
    "mclbm_w1_1pt": (_c.c_int, [_ctx_p, _ctx_p, _c.c_int32, _dp, _dp]),
    "mclbm_w1_work_bytes": (_c.c_size_t, [_c.c_int32, _c.c_int32, _c.c_int32]),
    "mclbm_w1_restricted": (_c.c_int, [_vp, _c.c_int32, _vp, _c.c_int32, _c.c_int32, _vp, _c.c_size_t, _vp, _dp, _dp]),
    "mclbm_w1_2pt_work_bytes": (_c.c_size_t, [_c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32]),
    "mclbm_sample_error_work_bytes": (_c.c_size_t, [_c.c_int32]),
    "mclbm_leray_params": (_c.c_int, [_dp, _c.c_int32, _c.c_int32, _dp]),
    "mclbm_sample_error": (_c.c_int, [_vp, _vp, _c.c_int32, _c.c_int32, _vp, _c.c_size_t, _vp, _dp]),
    "mclbm_w1_2pt": (_c.c_int, [_vp, _c.c_int32, _vp, _c.c_int32, _c.c_int32, _c.c_int32, _vp, _c.c_size_t, _vp, _dp,
                                _vp]),
    "mclbm_check_finite": (_c.c_int, [_ctx_p]),
    "mclbm_alu_rate": (_c.c_int, [_c.c_int32, _c.c_int32, _vp, _vp, _dp, _dp]),
    "mclbm_w1_restricted_noalloc": (_c.c_int, [_vp, _c.c_int32, _vp, _c.c_int32, _c.c_int32, _vp, _dp, _dp]),
    "mclbm_set_launch": (_c.c_int, [_ctx_p, _c.c_int32, _c.c_int32, _c.c_int32]),
    "mclbm_get_launch": (_c.c_int, [_ctx_p, _i32p, _i32p, _i32p]),
    "mclbm_set_launch_parity": (_c.c_int, [_ctx_p, _c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32]),
    "mclbm_get_launch_parity": (_c.c_int, [_ctx_p, _c.c_int32, _i32p, _i32p, _i32p]),
    "mclbm_autotune": (_c.c_int, [_ctx_p, _c.c_int32, _i32p, _i32p, _i32p, _dp]),
    "mclbm_device_status": (_c.c_int, [_ctx_p]),
    "mclbm_grad_required_bytes": (_c.c_int, [_ctx_p, _c.c_int64, _c.c_int32, _size_p]),
    "mclbm_grad": (_c.c_int, [_ctx_p, _c.c_int32, _c.c_int64, _c.c_int32, _vp, _c.c_size_t, _dp, _dp]),
    "mclbm_adjoint_step": (_c.c_int, [_ctx_p, _vp, _vp, _vp]),
    "mclbm_grad_timing": (_c.c_int, [_ctx_p, _dp]),
    "mclbm_selftest_timeout": (_c.c_int, [_ctx_p]),
    "mclbm_save": (_c.c_int, [_ctx_p, _c.c_char_p]),
    "mclbm_load": (_c.c_int, [_ctx_p, _c.c_char_p]),
    "mclbm_batch_create": (_c.c_int, [_c.POINTER(_ctx_p), _c.c_int32, _i32p, _c.POINTER(_vp)]),
    "mclbm_batch_destroy": (None, [_vp]),
    "mclbm_batch_set_graph": (_c.c_int, [_vp, _c.c_int32]),
    "mclbm_batch_set_launch": (_c.c_int, [_vp, _c.c_int32, _c.c_int32, _c.c_int32]),
    "mclbm_batch_set_launch_parity": (_c.c_int, [_vp, _c.c_int32, _c.c_int32, _c.c_int32, _c.c_int32]),
    "mclbm_batch_get_launch_parity": (_c.c_int, [_vp, _c.c_int32, _i32p, _i32p, _i32p]),
    "mclbm_batch_step": (_c.c_int, [_vp, _c.c_int64]),
    "mclbm_batch_macro_steps": (_c.c_int64, [_vp]),
    "mclbm_batch_autotune": (_c.c_int, [_vp, _c.c_int32, _i32p, _i32p, _i32p, _dp]),
}

_libs = {}  # lattice (19 or 27) -> loaded library
_owner = {}  # context / batch handle value -> lattice of the library that created it
_tls = threading.local()  # library of the calling thread's last call (for mclbm_last_error)


def library_path(lattice=19):
    return _build.LATTICE_LIBS[lattice]


def load(build_if_missing=False, lattice=19):
    """Load the in-tree library for the velocity set: libmclbm.so (D3Q19, default) or
    libmclbm_d3q27.so (D3Q27).  Raises if it is missing (there is no CPU fallback)."""
    if lattice not in _build.LATTICE_LIBS:
        raise ValueError("lattice must be 19 or 27")
    lib = _libs.get(lattice)
    if lib is None:
        path = library_path(lattice)
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(
                    f"{os.path.basename(path)} not found at {path}; build it with "
                    "paper_2608_23786_gb300.build.build() (the CUDA library is required: there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _libs[lattice] = lib
    _tls.lib = lib
    return lib


def _value(h):
    return h.value if isinstance(h, _c.c_void_p) else h


def lattice_of(h):
    """Velocity set (19 or 27) of the library that created a context or batch handle."""
    return _owner.get(_value(h), 19)


def _L(h):
    """Library that owns handle h (a context or a batch)."""
    return load(lattice=lattice_of(h))


def declared_symbols():
    """Names the binding expects the library to export (one per C-ABI entry point)."""
    return list(_SIGNATURES)


def _check(code):
    if code != MCLBM_OK:
        lib = getattr(_tls, "lib", None) or load()
        raise MclbmError(code, lib.mclbm_last_error().decode())
    return code


def _darr(a):
    """ctypes double* of a C-contiguous float64 numpy array (or None)."""
    if a is None:
        return None
    import numpy as np
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _stream(stream):
    """cudaStream_t handle for the C calls: an explicit handle (an int, 0 = the legacy default
    stream) is passed as given; None takes torch's current stream on the current device, so
    that work torch queued there (filling the inputs) is ordered before the call."""
    if stream is not None:
        return stream or None
    import torch
    if not torch.cuda.is_available():
        return None
    return torch.cuda.current_stream().cuda_stream or None


# ---- same-named wrappers ------------------------------------------------------

def mclbm_version(lattice=19):
    return load(lattice=lattice).mclbm_version().decode()


def mclbm_last_error():
    lib = getattr(_tls, "lib", None) or load()
    return lib.mclbm_last_error().decode()


def mclbm_lattice(lattice=19):
    """(c [Q][3], w [Q]) of the library for the velocity set (Q = lattice)."""
    import numpy as np
    c = np.zeros((lattice, 3), dtype=np.int32)
    w = np.zeros(lattice)
    _check(load(lattice=lattice).mclbm_lattice(c.ctypes.data_as(_i32p), _darr(w)))
    return c, w


def mclbm_compute_units(cfg):
    u = Units()
    _check(load().mclbm_compute_units(ctypes.byref(cfg), ctypes.byref(u)))
    return u


def mclbm_required_bytes(cfg, lattice=19):
    pop = ctypes.c_size_t()
    work = ctypes.c_size_t()
    _check(load(lattice=lattice).mclbm_required_bytes(ctypes.byref(cfg), ctypes.byref(pop), ctypes.byref(work)))
    return pop.value, work.value


def mclbm_create(cfg, d_pop, pop_bytes, d_work, work_bytes, stream=None, lattice=19):
    ctx = _ctx_p()
    _check(load(lattice=lattice).mclbm_create(ctypes.byref(cfg), d_pop, pop_bytes, d_work, work_bytes,
                                              _stream(stream), ctypes.byref(ctx)))
    _owner[ctx.value] = lattice
    return ctx


def mclbm_destroy(ctx):
    _L(ctx).mclbm_destroy(ctx)
    _owner.pop(_value(ctx), None)


def mclbm_get_units(ctx):
    u = Units()
    _check(_L(ctx).mclbm_get_units(ctx, ctypes.byref(u)))
    return u


def mclbm_init_ensemble(ctx, params=None):
    _check(_L(ctx).mclbm_init_ensemble(ctx, _darr(params)))


def mclbm_draw_params(seed, first_sample, M, width=0.025):
    import numpy as np
    out = np.zeros((M, 24))
    _check(load().mclbm_draw_params(int(seed), int(first_sample), int(M), float(width), _darr(out)))
    return out


def mclbm_init_tgv(ctx):
    _check(_L(ctx).mclbm_init_tgv(ctx))


def mclbm_leray_params(X, transpose=False):
    """Coefficients L X (or L^T X) of the Leray-projected perturbation, X [M][24] (host)."""
    import numpy as np
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 24)
    Y = np.zeros_like(X)
    _check(load().mclbm_leray_params(_darr(X), X.shape[0], int(bool(transpose)), _darr(Y)))
    return Y


def mclbm_get_params(ctx, out):
    _check(_L(ctx).mclbm_get_params(ctx, _darr(out)))
    return out


def mclbm_step(ctx, nsteps):
    _check(_L(ctx).mclbm_step(ctx, int(nsteps)))


def mclbm_steps_taken(ctx):
    return _L(ctx).mclbm_steps_taken(ctx)


def mclbm_get_populations(ctx, sample, d_out):
    _check(_L(ctx).mclbm_get_populations(ctx, int(sample), d_out))


def mclbm_set_populations(ctx, sample, d_in):
    _check(_L(ctx).mclbm_set_populations(ctx, int(sample), d_in))


def mclbm_moments(ctx, sample, d_rho, d_u):
    _check(_L(ctx).mclbm_moments(ctx, int(sample), d_rho, d_u))


def mclbm_energy(ctx, E, Z=None):
    _check(_L(ctx).mclbm_energy(ctx, _darr(E), _darr(Z)))


def mclbm_mean_var(ctx, d_mean, d_var):
    _check(_L(ctx).mclbm_mean_var(ctx, d_mean, d_var))


def mclbm_energy_mean_var(ctx, E, d_mean, d_var):
    _check(_L(ctx).mclbm_energy_mean_var(ctx, _darr(E), d_mean, d_var))


def mclbm_spectrum(ctx, E):
    _check(_L(ctx).mclbm_spectrum(ctx, _darr(E)))


def mclbm_sf_trace(ctx, S2):
    _check(_L(ctx).mclbm_sf_trace(ctx, _darr(S2)))


def mclbm_sf_axes(ctx, pmax, S):
    _check(_L(ctx).mclbm_sf_axes(ctx, int(pmax), _darr(S)))


def mclbm_restrict(ctx, Qd, d_out):
    _check(_L(ctx).mclbm_restrict(ctx, int(Qd), d_out))


def mclbm_w1_1pt(ctxA, ctxB, Qd, per_point=None):
    W = ctypes.c_double()
    _check(_L(ctxA).mclbm_w1_1pt(ctxA, ctxB, int(Qd), ctypes.byref(W), _darr(per_point)))
    return W.value


def mclbm_w1_work_bytes(MA, MB, G):
    return load().mclbm_w1_work_bytes(int(MA), int(MB), int(G))


def mclbm_w1_restricted(d_a, MA, d_b, MB, G, d_work, work_bytes, stream=None, per_point=None):
    W = ctypes.c_double()
    _check(load().mclbm_w1_restricted(d_a, int(MA), d_b, int(MB), int(G), d_work, work_bytes, _stream(stream),
                                      ctypes.byref(W), _darr(per_point)))
    return W.value


def mclbm_w1_2pt_work_bytes(MA, MB, G, vector):
    return load().mclbm_w1_2pt_work_bytes(int(MA), int(MB), int(G), int(vector))


def mclbm_w1_2pt(d_a, MA, d_b, MB, G, vector, d_work, work_bytes, stream=None, d_per_pair=None):
    """Two-point W1 (vector or component-wise) on restricted device fields; returns W."""
    W = ctypes.c_double()
    _check(load().mclbm_w1_2pt(d_a, int(MA), d_b, int(MB), int(G), int(vector), d_work, work_bytes, _stream(stream),
                               ctypes.byref(W), d_per_pair or None))
    return W.value


def mclbm_sample_error_work_bytes(M):
    return load().mclbm_sample_error_work_bytes(int(M))


def mclbm_sample_error(d_u, d_ref, M, G, d_work, work_bytes, stream=None):
    """Eq. (sample_error) on restricted device fields; returns [4] (x, y, z, vector)."""
    import numpy as np
    out = np.zeros(4)
    _check(load().mclbm_sample_error(d_u, d_ref, int(M), int(G), d_work, work_bytes, _stream(stream), _darr(out)))
    return out


def mclbm_w1_restricted_noalloc(d_a, MA, d_b, MB, G, stream=None, per_point=None):
    """W_{1,1} on device restricted fields without any device allocation (scratch is a fixed
    array inside the library, G <= 4096 points)."""
    W = ctypes.c_double()
    _check(load().mclbm_w1_restricted_noalloc(d_a, int(MA), d_b, int(MB), int(G), _stream(stream), ctypes.byref(W),
                                              _darr(per_point)))
    return W.value


ALU_KINDS = {"fp64_fma": 0, "fp32_fma": 1, "fp32x2_fma": 2, "half2_fma": 3, "fp32_rcp": 4}


def mclbm_alu_rate(kind, iters, d_sink, stream=None):
    """(results per second, ms) of the arithmetic-throughput kernel of `kind` (a name of
    ALU_KINDS or its number) on the current device."""
    k = ALU_KINDS.get(kind, kind)
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().mclbm_alu_rate(int(k), int(iters), d_sink, _stream(stream), ctypes.byref(r), ctypes.byref(ms)))
    return r.value, ms.value


def mclbm_check_finite(ctx):
    _check(_L(ctx).mclbm_check_finite(ctx))


def mclbm_set_launch(ctx, vec, block=256, kind=0):
    _check(_L(ctx).mclbm_set_launch(ctx, int(kind), int(vec), int(block)))


def mclbm_get_launch(ctx):
    """(kind, vec, block) of the context's stepper launch (pull steps, AA even steps)."""
    k, v, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_L(ctx).mclbm_get_launch(ctx, ctypes.byref(k), ctypes.byref(v), ctypes.byref(b)))
    return k.value, v.value, b.value


def mclbm_set_launch_parity(ctx, parity, vec, block=128, kind=0):
    _check(_L(ctx).mclbm_set_launch_parity(ctx, int(parity), int(kind), int(vec), int(block)))


def mclbm_get_launch_parity(ctx, parity):
    """(kind, vec, block) of the context's AA steps of that parity (0 even, 1 odd)."""
    k, v, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_L(ctx).mclbm_get_launch_parity(ctx, int(parity), ctypes.byref(k), ctypes.byref(v), ctypes.byref(b)))
    return k.value, v.value, b.value


def mclbm_autotune(ctx, trial_steps=5):
    """Returns (kind, vec, block, ms per step) of the fastest shape."""
    k, v, b, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(_L(ctx).mclbm_autotune(ctx, int(trial_steps), ctypes.byref(k), ctypes.byref(v), ctypes.byref(b),
                                 ctypes.byref(ms)))
    return k.value, v.value, b.value, ms.value


def mclbm_device_status(ctx):
    _check(_L(ctx).mclbm_device_status(ctx))


def mclbm_batch_create(ctxs, substeps):
    n = len(ctxs)
    lat = {lattice_of(c) for c in ctxs}
    if len(lat) != 1:
        raise ValueError("a batch takes contexts of one velocity set")
    arr = (_ctx_p * n)(*[c.value if isinstance(c, _ctx_p) else c for c in ctxs])
    sub = (ctypes.c_int32 * n)(*[int(s) for s in substeps])
    out = _vp()
    lattice = lat.pop()
    _check(load(lattice=lattice).mclbm_batch_create(arr, n, sub, ctypes.byref(out)))
    _owner[out.value] = lattice
    return out


def mclbm_batch_destroy(b):
    _L(b).mclbm_batch_destroy(b)
    _owner.pop(_value(b), None)


def mclbm_batch_set_graph(b, enable):
    _check(_L(b).mclbm_batch_set_graph(b, int(bool(enable))))


def mclbm_batch_set_launch(b, vec, block=256, kind=0):
    _check(_L(b).mclbm_batch_set_launch(b, int(kind), int(vec), int(block)))


def mclbm_batch_set_launch_parity(b, parity, vec, block=128, kind=0):
    _check(_L(b).mclbm_batch_set_launch_parity(b, int(parity), int(kind), int(vec), int(block)))


def mclbm_batch_get_launch_parity(b, parity):
    k, v, bl = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_L(b).mclbm_batch_get_launch_parity(b, int(parity), ctypes.byref(k), ctypes.byref(v), ctypes.byref(bl)))
    return k.value, v.value, bl.value


def mclbm_batch_step(b, macro_steps):
    _check(_L(b).mclbm_batch_step(b, int(macro_steps)))


def mclbm_batch_macro_steps(b):
    return _L(b).mclbm_batch_macro_steps(b)


def mclbm_batch_autotune(b, trials=2):
    """Returns (kind, vec, block, ms per macro step) of the fastest shape."""
    k, v, blk, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(_L(b).mclbm_batch_autotune(b, int(trials), ctypes.byref(k), ctypes.byref(v), ctypes.byref(blk),
                                       ctypes.byref(ms)))
    return k.value, v.value, blk.value, ms.value


def mclbm_grad_required_bytes(ctx, nsteps, ckpt_every):
    b = ctypes.c_size_t()
    _check(_L(ctx).mclbm_grad_required_bytes(ctx, int(nsteps), int(ckpt_every), ctypes.byref(b)))
    return b.value


def mclbm_grad(ctx, objective, nsteps, ckpt_every, d_buf, buf_bytes, M):
    """Returns (J [M], dJ/dX [M][24]) as numpy arrays."""
    import numpy as np
    J = np.zeros(M)
    G = np.zeros((M, 24))
    _check(_L(ctx).mclbm_grad(ctx, int(objective), int(nsteps), int(ckpt_every), d_buf, buf_bytes, _darr(J), _darr(G)))
    return J, G


def mclbm_adjoint_step(ctx, d_f, d_lambda_next, d_lambda):
    _check(_L(ctx).mclbm_adjoint_step(ctx, d_f, d_lambda_next, d_lambda))


def mclbm_grad_timing(ctx):
    """ms of the phases of the last mclbm_grad: forward, recompute, reverse, parameter reduction."""
    import numpy as np
    out = np.zeros(4)
    _check(_L(ctx).mclbm_grad_timing(ctx, _darr(out)))
    return out


def mclbm_selftest_timeout(ctx):
    _check(_L(ctx).mclbm_selftest_timeout(ctx))


def mclbm_save(ctx, path):
    _check(_L(ctx).mclbm_save(ctx, os.fsencode(path)))


def mclbm_load(ctx, path):
    _check(_L(ctx).mclbm_load(ctx, os.fsencode(path)))

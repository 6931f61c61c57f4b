"""Ensemble: one Monte Carlo KBC LBM ensemble on the GPU.

PyTorch provides the device memory (two caller-owned uint8 buffers) and the CUDA
stream; every computation runs in libmclbm's kernels through the C ABI.
"""
import numpy as np
import torch

from . import mclbm as _m


class Ensemble:
    """M RTGV samples on an N^3 periodic lattice at viscosity nu = 1/Re.

    precision: "fp64" | "fp32" | "fp16"; pattern: "pull" | "aa"; lattice: 19 (D3Q19, the
    paper's velocity set, libmclbm.so) or 27 (D3Q27, libmclbm_d3q27.so); leray: initialise
    with the Leray-projected perturbation (the paper's runs omit the projection); exact_gamma:
    the exact entropic gamma of Eq. (kbc_entropy) instead of the closed form.
    """

    PREC = {"fp64": _m.FP64, "fp32": _m.FP32, "fp16": _m.FP16}
    PAT = {"pull": _m.PULL, "aa": _m.AA}

    def __init__(self, N, M, Re=None, nu=None, Ma=None, dt=0.0, precision="fp32", pattern="pull", seed=1,
                 width=0.025, U_c=1.0, init_density=0, device=None, stream=None, lattice=19, leray=False,
                 exact_gamma=False):
        if not torch.cuda.is_available():
            raise RuntimeError("Ensemble needs a CUDA device (there is no CPU path)")
        if nu is None:
            nu = 1.0 / Re
        self.device = torch.device(device if device is not None else "cuda")
        options = (_m.OPT_LERAY if leray else 0) | (_m.OPT_EXACT_GAMMA if exact_gamma else 0)
        self.cfg = _m.Config(N=N, M=M, precision=self.PREC[precision], pattern=self.PAT[pattern], nu=nu,
                             Ma=Ma if Ma is not None else 0.0, dt=dt, U_c=U_c, width=width, seed=seed,
                             init_density=init_density, options=options)
        self.N, self.M = N, M
        self.precision, self.pattern = precision, pattern
        self.Q = self.lattice = lattice
        pop_bytes, work_bytes = _m.mclbm_required_bytes(self.cfg, lattice=lattice)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.pop = torch.empty(pop_bytes + 256, dtype=torch.uint8, device=self.device)
            self.work = torch.empty(work_bytes + 256, dtype=torch.uint8, device=self.device)
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:  # buffers are allocated on the current stream, used on self.stream
            self.stream.wait_stream(cur)
            self.pop.record_stream(self.stream)
            self.work.record_stream(self.stream)
        self._pop_ptr = (self.pop.data_ptr() + 255) // 256 * 256
        self._work_ptr = (self.work.data_ptr() + 255) // 256 * 256
        with torch.cuda.device(self.device):
            self.ctx = _m.mclbm_create(self.cfg, self._pop_ptr, pop_bytes, self._work_ptr, work_bytes,
                                       self.stream.cuda_stream, lattice=lattice)
        self.units = _m.mclbm_get_units(self.ctx).as_dict()

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            _m.mclbm_destroy(ctx)
            self.ctx = None

    @property
    def n(self):
        return self.N**3

    # ---- stream ordering between torch's current stream and the ensemble's stream ----
    def _enter(self, *tensors):
        """Make the ensemble's stream wait for work queued on torch's current stream (e.g. the
        allocation or filling of `tensors`) and mark the tensors as used on that stream."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
            for t in tensors:
                t.record_stream(self.stream)

    def _exit(self):
        """Make torch's current stream wait for the ensemble's queued work."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    # ---- evolution -------------------------------------------------------------
    def init(self, params=None):
        """Equilibrium RTGV initialisation; params [M][24] (host) or None for the Philox draw."""
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float64).reshape(self.M, 24)
        _m.mclbm_init_ensemble(self.ctx, p)
        return self

    def init_tgv(self):
        _m.mclbm_init_tgv(self.ctx)
        return self

    def params(self):
        out = np.zeros((self.M, 24))
        return _m.mclbm_get_params(self.ctx, out)

    def step(self, nsteps=1):
        _m.mclbm_step(self.ctx, nsteps)
        return self

    @property
    def steps_taken(self):
        return _m.mclbm_steps_taken(self.ctx)

    # ---- fields ----------------------------------------------------------------
    def populations(self, sample=0):
        """Pre-collision f [Q][N][N][N] (FP64, library velocity order) as a CUDA tensor."""
        out = torch.empty((self.Q, self.N, self.N, self.N), dtype=torch.float64, device=self.device)
        self._enter(out)
        _m.mclbm_get_populations(self.ctx, sample, out.data_ptr())
        self._exit()
        return out

    def set_populations(self, f, sample=0):
        f = f.to(device=self.device, dtype=torch.float64).contiguous()
        self._enter(f)
        _m.mclbm_set_populations(self.ctx, sample, f.data_ptr())
        self._exit()
        return self

    def moments(self, sample=0):
        """(rho [N][N][N], u [3][N][N][N] physical) FP64 CUDA tensors."""
        rho = torch.empty((self.N,) * 3, dtype=torch.float64, device=self.device)
        u = torch.empty((3,) + (self.N,) * 3, dtype=torch.float64, device=self.device)
        self._enter(rho, u)
        _m.mclbm_moments(self.ctx, sample, rho.data_ptr(), u.data_ptr())
        self._exit()
        return rho, u

    def energy(self, enstrophy=False):
        E = np.zeros(self.M)
        Z = np.zeros(self.M) if enstrophy else None
        _m.mclbm_energy(self.ctx, E, Z)
        return (E, Z) if enstrophy else E

    def mean_var(self):
        mean = torch.empty((3,) + (self.N,) * 3, dtype=torch.float64, device=self.device)
        var = torch.empty_like(mean)
        self._enter(mean, var)
        _m.mclbm_mean_var(self.ctx, mean.data_ptr(), var.data_ptr())
        self._exit()
        return mean, var

    def energy_mean_var(self):
        """(E [M] numpy, mean, var [3][N][N][N] FP64 CUDA tensors) in one pass over the populations."""
        E = np.zeros(self.M)
        mean = torch.empty((3,) + (self.N,) * 3, dtype=torch.float64, device=self.device)
        var = torch.empty_like(mean)
        self._enter(mean, var)
        _m.mclbm_energy_mean_var(self.ctx, E, mean.data_ptr(), var.data_ptr())
        self._exit()
        return E, mean, var

    def spectrum(self):
        E = np.zeros((self.M, self.N // 2 + 1))
        _m.mclbm_spectrum(self.ctx, E)
        return E

    def sf_trace(self):
        S = np.zeros((self.M, self.N // 2 + 1))
        _m.mclbm_sf_trace(self.ctx, S)
        return S

    def sf_axes(self, pmax=6):
        S = np.zeros((self.M, pmax - 1, self.N // 2))
        _m.mclbm_sf_axes(self.ctx, pmax, S)
        return S

    def restrict(self, Q=8):
        out = torch.empty((self.M, Q**3, 3), dtype=torch.float64, device=self.device)
        self._enter(out)
        _m.mclbm_restrict(self.ctx, Q, out.data_ptr())
        self._exit()
        return out

    def w1(self, other, Q=8, per_point=False):
        pp = np.zeros((Q**3, 3)) if per_point else None
        W = _m.mclbm_w1_1pt(self.ctx, other.ctx, Q, pp)
        return (W, pp) if per_point else W

    def w1_2pt(self, other, Q=8, vector=True):
        """Two-point W1 (W_{1,2}^v if vector, else the component-wise W_{1,2}) between the laws of
        this ensemble and `other` on the common Q^3 restriction grid (mclbm_w1_2pt)."""
        ua, ub = self.restrict(Q), other.restrict(Q)
        G = Q**3
        nb = _m.mclbm_w1_2pt_work_bytes(self.M, other.M, G, int(vector))
        work = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self._enter(work, ua, ub)
        W = _m.mclbm_w1_2pt(ua.data_ptr(), self.M, ub.data_ptr(), other.M, G, int(vector), work.data_ptr(), nb,
                            self.stream.cuda_stream)
        self._exit()
        return W

    def sample_error(self, ref, Q=8):
        """Eq. (sample_error) between this ensemble and `ref` (the same samples at another
        resolution) on the common Q^3 grid: [4] for x, y, z and the vector (mclbm_sample_error)."""
        u, ur = self.restrict(Q), ref.restrict(Q)
        nb = _m.mclbm_sample_error_work_bytes(self.M)
        work = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self._enter(work, u, ur)
        out = _m.mclbm_sample_error(u.data_ptr(), ur.data_ptr(), self.M, Q**3, work.data_ptr(), nb,
                                    self.stream.cuda_stream)
        self._exit()
        return out

    def check_finite(self):
        _m.mclbm_check_finite(self.ctx)

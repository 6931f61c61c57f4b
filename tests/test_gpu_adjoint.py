"""GPU adjoint: the hand-written transposed step against the oracle's complex-step
directional derivative (dot-product test), and dJ/dX against the oracle's complex-step
gradient and central differences."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
import oracle
from gpu_helpers import lib_to_oracle_perm
from paper_2608_23786_gb300 import Ensemble, mclbm
from paper_2608_23786_gb300.autograd import ensemble_objective

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def _to_lib(a_orc):
    """[M][19][...] oracle order -> library order."""
    return a_orc[:, lib_to_oracle_perm()]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_transposed_step_dot_product_against_complex_step(precision, tol):
    """<J v, w> with J v = Im(step(f + i h v)) / h from the oracle's complex twin equals
    <v, J^T w> from the library's adjoint step (16^3 x 2 RTGV state after 15 steps, random
    v and w)."""
    N, M, Re, Ma = 16, 2, 300.0, 0.1
    X = gen.draw_params(41, M)
    un = oracle.units(N, Re, Ma)
    f = oracle.init_ensemble(N, X, un["ulat"])
    oracle.run(f, un["omega"], 15)
    _, w_, _ = oracle.lattice()
    v = w_[None, :, None, None, None] * gen.uniform(42, f.shape)
    wv = gen.uniform(43, f.shape)
    fc = f.astype(np.complex128) + 1e-30j * v
    oracle.step(fc, un["omega"])
    Jv = fc.imag / 1e-30
    lhs = float(np.sum(Jv * wv))
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision=precision).init(X)
    d_f = torch.as_tensor(_to_lib(f), device="cuda").contiguous()
    d_w = torch.as_tensor(_to_lib(wv), device="cuda").contiguous()
    d_l = torch.empty_like(d_f)
    mclbm.mclbm_adjoint_step(ens.ctx, d_f.data_ptr(), d_w.data_ptr(), d_l.data_ptr())
    torch.cuda.synchronize()
    rhs = float(np.sum(_to_lib(v) * d_l.cpu().numpy()))
    assert abs(lhs - rhs) <= tol * abs(lhs), (lhs, rhs)


def _gpu_grad(N, M, X, Re, Ma, nsteps, K, objective, precision):
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision=precision).init(X)
    need = mclbm.mclbm_grad_required_bytes(ens.ctx, nsteps, K)
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    ptr = (buf.data_ptr() + 255) // 256 * 256
    J, G = mclbm.mclbm_grad(ens.ctx, objective, nsteps, K, ptr, need, M)
    assert ens.steps_taken == nsteps
    return J, G


@pytest.mark.parametrize("objective", [0, 1])
def test_fp64_gradient_matches_oracle_complex_step(objective):
    """FP64 adjoint gradient at 16^3 within 1e-8 of the oracle's complex-step gradient
    (20 steps, checkpoints every 7 steps: two full segments and a remainder)."""
    N, M, Re, Ma, T = 16, 2, 200.0, 0.1, 20
    X = gen.draw_params(4, M)
    un = oracle.units(N, Re, Ma)
    J, G = _gpu_grad(N, M, X, Re, Ma, T, 7, objective, "fp64")
    ref = oracle.complex_step_grad(N, X, un["ulat"], un["omega"], T, "energy" if objective == 0 else "enstrophy")
    scale = np.abs(ref).max()
    assert np.max(np.abs(G - ref)) <= 1e-8 * scale, np.max(np.abs(G - ref)) / scale
    f = oracle.init_ensemble(N, X, un["ulat"])
    oracle.run(f, un["omega"], T)
    _, u = oracle.moments(f)
    E, Z = oracle.energy(u, un["ulat"])
    np.testing.assert_allclose(J, E if objective == 0 else Z, rtol=1e-12)


def test_checkpoint_interval_does_not_change_the_gradient():
    N, M, Re, Ma, T = 16, 2, 200.0, 0.1, 12
    X = gen.draw_params(6, M)
    _, G1 = _gpu_grad(N, M, X, Re, Ma, T, 1, 0, "fp32")
    _, G5 = _gpu_grad(N, M, X, Re, Ma, T, 5, 0, "fp32")
    _, G12 = _gpu_grad(N, M, X, Re, Ma, T, 12, 0, "fp32")
    np.testing.assert_array_equal(G1, G5)
    np.testing.assert_array_equal(G1, G12)


@pytest.mark.parametrize("objective,tol", [(0, 1e-3), (1, 5e-3)])
def test_fp32_gradient_matches_oracle(objective, tol):
    """FP32 adjoint per component against the FP64 oracle (components >= 1e-3 of the largest):
    1e-3 for the kinetic energy; 5e-3 for the enstrophy, whose gradient weights the small scales
    where the FP32 state resolves Dh, and with it gamma, least (measured 3.9e-3)."""
    N, M, Re, Ma, T = 16, 2, 200.0, 0.1, 20
    X = gen.draw_params(4, M)
    un = oracle.units(N, Re, Ma)
    _, G = _gpu_grad(N, M, X, Re, Ma, T, 8, objective, "fp32")
    ref = oracle.complex_step_grad(N, X, un["ulat"], un["omega"], T, "energy" if objective == 0 else "enstrophy")
    big = np.abs(ref) >= 1e-3 * np.abs(ref).max()
    rel = np.abs(G - ref)[big] / np.abs(ref)[big]
    assert rel.max() <= tol, rel.max()


def test_fp64_gradient_at_500_steps_matches_central_differences():
    """FP64 adjoint of the full adjoint horizon (64^3, 500 steps, checkpoints every 50) against
    central differences (h = 1e-5) of the FP64 forward, on the largest components."""
    N, M, Re, Ma, T = 64, 2, 800.0, 0.025, 500
    X = gen.draw_params(1, M)
    _, G = _gpu_grad(N, M, X, Re, Ma, T, 50, 0, "fp64")
    h = 1e-5
    for k in np.argsort(-np.abs(G[0]))[:3]:
        vals = []
        for s in (1, -1):
            P = X.copy()
            P[0, k] += s * h
            vals.append(Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64").init(P).step(T).energy()[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - G[0, k]) <= 1e-5 * np.abs(G).max()


def test_fp64_gradient_matches_central_differences():
    """dJ/dX of the GPU adjoint against central differences (h = 1e-4) of the GPU FP64 forward."""
    N, M, Re, Ma, T = 16, 1, 200.0, 0.1, 10
    X = gen.draw_params(9, M)
    _, G = _gpu_grad(N, M, X, Re, Ma, T, 4, 0, "fp64")
    h = 1e-4
    for k in (0, 7, 13, 22):
        vals = []
        for s in (1, -1):
            P = X.copy()
            P[0, k] += s * h
            vals.append(Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64").init(P).step(T).energy()[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - G[0, k]) <= 1e-6 * np.abs(G).max()


def test_autograd_function():
    """torch.autograd: J.sum().backward() deposits dJ/dX in params.grad."""
    N, M, Re, Ma, T = 16, 3, 200.0, 0.1, 6
    X = gen.draw_params(12, M)
    p = torch.tensor(X, requires_grad=True)
    J = ensemble_objective(p, N=N, Ma=Ma, Re=Re, nsteps=T, precision="fp64", ckpt_every=4)
    weights = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    (J * weights).sum().backward()
    _, G = _gpu_grad(N, M, X, Re, Ma, T, 4, 0, "fp64")
    np.testing.assert_allclose(p.grad.numpy(), G * weights.numpy()[:, None], rtol=1e-13, atol=0)


def test_autograd_forward_without_backward_runs_no_adjoint(monkeypatch):
    """The forward pass is a plain run: it never enters mclbm_grad (the only caller of the
    adjoint kernels), and no k_adjoint kernel appears among the kernels it launches.  J equals
    the adjoint's J to the bit, and backward still gives the adjoint's gradient."""
    N, M, Re, Ma, T = 16, 2, 200.0, 0.1, 6
    X = gen.draw_params(13, M)
    J_ref, G_ref = _gpu_grad(N, M, X, Re, Ma, T, 4, 0, "fp32")
    calls = []
    real_grad = mclbm.mclbm_grad
    monkeypatch.setattr(mclbm, "mclbm_grad", lambda *a, **k: calls.append(1) or real_grad(*a, **k))
    p = torch.tensor(X, requires_grad=True)
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        J = ensemble_objective(p, N=N, Ma=Ma, Re=Re, nsteps=T, precision="fp32", ckpt_every=4)
        torch.cuda.synchronize()
    assert calls == []
    names = [e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA]
    assert not any("k_adjoint" in n for n in names)
    np.testing.assert_array_equal(J.detach().numpy(), J_ref)
    J.sum().backward()
    assert calls == [1]
    np.testing.assert_array_equal(p.grad.numpy(), G_ref)
    with torch.no_grad():
        J2 = ensemble_objective(p, N=N, Ma=Ma, Re=Re, nsteps=T, precision="fp32", objective="enstrophy")
    assert calls == [1] and np.all(np.isfinite(J2.numpy()))


def test_full_size_adjoint_fp32_vs_fp64():
    """The adjoint workload: 64^3 x 16 samples, 500 steps, checkpoint every 50, E(T).  J of the
    FP32 run agrees with FP64 to 2e-5.  The FP32 gradient agrees with the FP64 gradient (which is
    checked against central differences and the oracle) to 1.5e-2 in relative L2 norm and 6e-2
    of the largest component at most (measured 7.3e-3 and 3.4e-2): where Dh is small the FP32
    state does not resolve it, so gamma differs from the FP64 run there, which leaves J unchanged
    but not dJ/dX.  Over 100 steps the same comparison gives 4e-4 (bound 1e-3)."""
    N, M, Re, Ma, K = 64, 16, 800.0, 0.025, 50
    X = gen.draw_params(1, M)
    for T, l2_tol, max_tol in ((100, 1e-3, 3e-3), (500, 1.5e-2, 6e-2)):
        J32, G32 = _gpu_grad(N, M, X, Re, Ma, T, K, 0, "fp32")
        J64, G64 = _gpu_grad(N, M, X, Re, Ma, T, K, 0, "fp64")
        assert np.all(np.isfinite(G32)) and np.all(np.isfinite(G64))
        np.testing.assert_allclose(J32, J64, rtol=2e-5)
        assert np.linalg.norm(G32 - G64) <= l2_tol * np.linalg.norm(G64), T
        assert np.abs(G32 - G64).max() <= max_tol * np.abs(G64).max(), T


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("N", [8, 32, 128])
def test_reduced_precision_reverse_sweep_against_fp64_across_row_widths(lattice, N):
    """The FP32/FP16 reverse sweep fetches the periodic x-neighbours of a run in two ways: by a
    shuffle inside the row's lanes when a whole x-row lies within one warp (N <= 64; rows of 4
    and 16 lanes here), by separately copied edge words otherwise (N = 128).  Both agree with the
    FP64 adjoint (itself checked against the oracle) over 8 steps with the same omega at every N:
    FP32 to 1e-4 in relative L2 (measured 2.3e-5 at most), FP16 storage to 4e-2 (measured 1.7e-2
    at N = 8, where the state's half-precision rounding is largest against its gradients)."""
    mclbm.load(lattice=lattice)
    M, Ma, T, K = 2, 0.1, 8, 3
    Re = 100.0 * N / 16
    X = gen.draw_params(17, M)

    def grad(precision):
        ens = Ensemble(N, M, Re=Re, Ma=Ma, precision=precision, lattice=lattice).init(X)
        need = mclbm.mclbm_grad_required_bytes(ens.ctx, T, K)
        buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        return mclbm.mclbm_grad(ens.ctx, 0, T, K, (buf.data_ptr() + 255) // 256 * 256, need, M)[1]

    G64 = grad("fp64")
    for precision, tol in (("fp32", 1e-4), ("fp16", 4e-2)):
        G = grad(precision)
        assert np.all(np.isfinite(G))
        rel = np.linalg.norm(G - G64) / np.linalg.norm(G64)
        assert rel <= tol, (precision, rel)

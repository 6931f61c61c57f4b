"""The D3Q27 library (libmclbm_d3q27.so, the same kernels built for the 27-velocity set)
against the D3Q27 oracle: FP64 per population <= 1e-12, FP32 / FP16 velocity error after 100
steps, AA = pull and every launch shape bitwise, batch = per-level stepping, conservation, and
the adjoint (FP64 gradient against the oracle's complex step; FP32 transposed step by the
dot-product test)."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
import oracle
from gpu_helpers import lib_populations, lib_to_oracle_perm, rel_l2
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu
Q = 27


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True, lattice=Q)


def _oracle_run(N, X, Re, Ma, steps):
    un = oracle.units(N, Re, Ma)
    f = oracle.init_ensemble(N, X, un["ulat"], lattice=Q)
    oracle.run(f, un["omega"], steps)
    return f, un


def test_library_reports_d3q27():
    c, w = mclbm.mclbm_lattice(Q)
    co, wo, _ = oracle.lattice(Q)
    perm = lib_to_oracle_perm(Q)
    np.testing.assert_array_equal(c, co[perm])
    np.testing.assert_array_equal(w, wo[perm])
    assert "D3Q27" in mclbm.mclbm_version(Q)


@pytest.mark.parametrize("pattern", ["pull", "aa"])
@pytest.mark.parametrize("steps", [1, 7, 40])
def test_fp64_rtgv_ensemble_parity(pattern, steps):
    N, M, Re, Ma = 16, 3, 400.0, 0.1
    X = gen.draw_params(11, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64", pattern=pattern, lattice=Q).init(X).step(steps)
    f, _ = _oracle_run(N, X, Re, Ma, steps)
    assert np.max(np.abs(lib_populations(ens) - f) / np.abs(f)) <= 1e-12


def _velocity(ens):
    return np.stack([ens.moments(m)[1].cpu().numpy() for m in range(ens.M)])


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp16", 1e-3)])
def test_shifted_velocity_error_after_100_steps(precision, tol):
    N, M, Re, Ma, steps = 32, 4, 800.0, 0.025, 100
    X = gen.draw_params(2, M)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision=precision, pattern="aa" if precision == "fp16" else "pull",
                   lattice=Q).init(X).step(steps)
    f, un = _oracle_run(N, X, Re, Ma, steps)
    _, u = oracle.moments(f)
    err = rel_l2(_velocity(ens), u / un["ulat"])
    assert err <= tol, err


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_every_launch_shape_and_aa_equal_pull(precision):
    X = gen.draw_params(31, 2)
    vecs = {"fp64": [1], "fp32": [2], "fp16": [4]}[precision]
    shapes = [(k, v, b) for k in (0, 2) for v in vecs for b in (128, 256)]
    if precision != "fp64":
        shapes += [(3, v, b) for v in vecs for b in (128, 256)]
        shapes += [(k, v, 128) for k in (4, 5) for v in vecs]  # shared-memory prefetch rings
    shapes += [(1, 1, 0)]
    ref = None
    for pattern in ("pull", "aa"):
        for kind, vec, block in shapes:
            ens = Ensemble(16, 2, Re=300.0, Ma=0.1, precision=precision, pattern=pattern, lattice=Q).init(X)
            mclbm.mclbm_set_launch(ens.ctx, vec, block, kind)
            ens.step(5)
            mclbm.mclbm_device_status(ens.ctx)
            got = [ens.populations(m) for m in range(2)]
            if ref is None:
                ref = got
            else:
                for a, b in zip(ref, got):
                    assert torch.equal(a, b), (pattern, kind, vec, block)


def test_batch_equals_separate_and_conserves():
    stream = torch.cuda.Stream()
    spec = [(16, 3, 400.0, 0.1, 1), (32, 2, 1600.0, 0.05, 4)]
    X = [gen.draw_params(s + 1, M) for s, (_, M, _, _, _) in enumerate(spec)]
    lv = [Ensemble(N, M, Re=Re, Ma=Ma, precision="fp32", seed=s + 1, stream=stream, lattice=Q).init(X[s])
          for s, (N, M, Re, Ma, _) in enumerate(spec)]
    c, _ = mclbm.mclbm_lattice(Q)
    ct = torch.as_tensor(c, dtype=torch.float64, device="cuda")
    mass0 = [e.populations(0).sum().item() for e in lv]
    mom0 = [[(e.populations(0) * ct[:, a][:, None, None, None]).sum().item() for a in range(3)] for e in lv]
    b = mclbm.mclbm_batch_create([e.ctx for e in lv], [sp[4] for sp in spec])
    try:
        mclbm.mclbm_batch_step(b, 2)
        stream.synchronize()
    finally:
        mclbm.mclbm_batch_destroy(b)
    for s, ((N, M, Re, Ma, sub), e) in enumerate(zip(spec, lv)):
        sep = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp32", seed=s + 1, lattice=Q).init(X[s]).step(2 * sub)
        for m in range(M):
            assert torch.equal(e.populations(m), sep.populations(m))
        f = e.populations(0)
        assert abs(f.sum().item() - mass0[s]) <= 2e-6 * mass0[s]
        for a in range(3):
            assert abs((f * ct[:, a][:, None, None, None]).sum().item() - mom0[s][a]) <= 2e-6 * mass0[s]


def _to_lib(a_orc):
    return a_orc[:, lib_to_oracle_perm(Q)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_transposed_step_dot_product_against_complex_step(precision, tol):
    N, M, Re, Ma = 16, 2, 300.0, 0.1
    X = gen.draw_params(41, M)
    un = oracle.units(N, Re, Ma)
    f = oracle.init_ensemble(N, X, un["ulat"], lattice=Q)
    oracle.run(f, un["omega"], 15)
    _, w_, _ = oracle.lattice(Q)
    v = w_[None, :, None, None, None] * gen.uniform(42, f.shape)
    wv = gen.uniform(43, f.shape)
    fc = f.astype(np.complex128) + 1e-30j * v
    oracle.step(fc, un["omega"])
    lhs = float(np.sum(fc.imag / 1e-30 * wv))
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision=precision, lattice=Q).init(X)
    d_f = torch.as_tensor(_to_lib(f), device="cuda").contiguous()
    d_w = torch.as_tensor(_to_lib(wv), device="cuda").contiguous()
    d_l = torch.empty_like(d_f)
    mclbm.mclbm_adjoint_step(ens.ctx, d_f.data_ptr(), d_w.data_ptr(), d_l.data_ptr())
    torch.cuda.synchronize()
    rhs = float(np.sum(_to_lib(v) * d_l.cpu().numpy()))
    assert abs(lhs - rhs) <= tol * abs(lhs), (lhs, rhs)


def test_fp64_gradient_matches_oracle_complex_step():
    N, M, Re, Ma, T, K = 16, 2, 200.0, 0.1, 12, 5
    X = gen.draw_params(4, M)
    un = oracle.units(N, Re, Ma)
    ens = Ensemble(N, M, Re=Re, Ma=Ma, precision="fp64", lattice=Q).init(X)
    need = mclbm.mclbm_grad_required_bytes(ens.ctx, T, K)
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    J, G = mclbm.mclbm_grad(ens.ctx, 0, T, K, (buf.data_ptr() + 255) // 256 * 256, need, M)
    ref = oracle.complex_step_grad(N, X, un["ulat"], un["omega"], T, "energy", lattice=Q)
    assert np.max(np.abs(G - ref)) <= 1e-8 * np.abs(ref).max()

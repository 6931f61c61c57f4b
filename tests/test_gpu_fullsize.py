"""Full-size checks of the large and batched workloads: one-step parity on sampled nodes
of the 512^3 x 4 FP16 AA ensemble (the oracle collides each sampled node's upstream
neighbours, taken from the GPU's own pre-step state), and conservation in every level of
the 64^3 x 64 / 128^3 x 32 / 256^3 x 8 batch after a macro step."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
import oracle
from gpu_helpers import lib_to_oracle_perm
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def _sampled_step_parity(ens, sample, nodes, tol_over_w):
    """Compare one GPU step at `nodes` ([k, 3] x, y, z) with the oracle's collision of the
    upstream neighbours x - c_i of each node (pull view of Eq. (lbIteration))."""
    N = ens.N
    c_lib, w_lib = mclbm.mclbm_lattice()
    perm = lib_to_oracle_perm()  # oracle index of library velocity i
    inv = np.argsort(perm)       # library index of oracle velocity j
    un = ens.units
    f = ens.populations(sample)  # [19][N][N][N] FP64, library order
    k = len(nodes)
    x = torch.as_tensor(nodes[:, 0], device=f.device)
    y = torch.as_tensor(nodes[:, 1], device=f.device)
    z = torch.as_tensor(nodes[:, 2], device=f.device)
    up = np.zeros((k, 19, 19))  # [node][i: direction][j: populations of x - c_i, library order]
    for i in range(19):
        xs, ys, zs = (x - int(c_lib[i, 0])) % N, (y - int(c_lib[i, 1])) % N, (z - int(c_lib[i, 2])) % N
        up[:, i, :] = f[:, zs, ys, xs].T.cpu().numpy()
    del f
    ens.step(1)
    g = ens.populations(sample)
    got = g[:, z, y, x].T.cpu().numpy()  # [node][i]
    del g
    _, w_orc, _ = oracle.lattice()
    for n in range(k):
        for i in range(19):
            fs, *_ = oracle.collide(up[n, i][inv], un["omega"])
            expect = fs[perm[i]]
            assert abs(got[n, i] - expect) <= tol_over_w * w_lib[i], (n, i, got[n, i], expect)


def test_large_512_fp16_aa_sampled_step_parity():
    """512^3 x 4 samples, Re = 6400, Ma = 0.003125, FP16 shifted storage, in-place AA streaming:
    the step after 3 steps (odd parity) at 64 sampled nodes of sample 2.  Tolerance: FP16 rounding
    of h = f/w - 1 (|h| < 0.01 here, 2^-11 relative) plus FP32 arithmetic."""
    ens = Ensemble(512, 4, Re=6400.0, Ma=0.003125, precision="fp16", pattern="aa", seed=5).init().step(3)
    nodes = (gen.uniform(77, (64, 3), 0, 512)).astype(np.int64)
    nodes[:4] = [[0, 0, 0], [511, 511, 511], [0, 511, 255], [511, 0, 1]]  # periodic corners
    _sampled_step_parity(ens, 2, nodes, tol_over_w=2e-5)
    ens.check_finite()


def test_levels_batch_full_size_conservation():
    """The three-level batch (FP32, pull) for one macro step (1 : 4 : 16 sub-steps): per level
    the global mass and momentum of two samples are unchanged to FP32 rounding."""
    stream = torch.cuda.Stream()
    spec = [(64, 64, 400.0, 0.025, 1), (128, 32, 1600.0, 0.0125, 4), (256, 8, 3200.0, 0.00625, 16)]
    lv = [Ensemble(N, M, Re=Re, Ma=Ma, precision="fp32", pattern="pull", seed=s + 1, stream=stream).init()
          for s, (N, M, Re, Ma, _) in enumerate(spec)]
    c, _ = mclbm.mclbm_lattice()
    ct = torch.as_tensor(c, dtype=torch.float64, device="cuda")

    def totals(e, m):
        f = e.populations(m)
        return f.sum().item(), [(f * ct[:, a][:, None, None, None]).sum().item() for a in range(3)]

    before = [[totals(e, m) for m in (0, e.M - 1)] for e in lv]
    b = mclbm.mclbm_batch_create([e.ctx for e in lv], [sp[4] for sp in spec])
    try:
        mclbm.mclbm_batch_step(b, 1)
        stream.synchronize()
    finally:
        mclbm.mclbm_batch_destroy(b)
    for e, bt, sp in zip(lv, before, spec):
        assert e.steps_taken == sp[4]
        mclbm.mclbm_device_status(e.ctx)
        e.check_finite()
        for (m0, mom0), m in zip(bt, (0, e.M - 1)):
            mass, mom = totals(e, m)
            assert abs(mass - m0) <= 2e-6 * m0
            for a in range(3):
                assert abs(mom[a] - mom0[a]) <= 2e-6 * m0

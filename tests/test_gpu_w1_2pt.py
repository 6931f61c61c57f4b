"""Two-point W1 on the GPU (exact assignment per point pair) against the oracle's transport
LP / assignment (Eq. (W1_vector), Algorithms "WassersteinDistance2" and
"WassersteinDistance2_vector").  Tolerance: the GPU matching is optimal for costs computed from
FP32 atoms (relative error ~1e-7 per cost), summed in FP64, so each pair's value is within
2e-6 relative of the exact optimum."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
from oracle import stats
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu
pytest.importorskip("scipy")

RTOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def _gpu(ua, ub, vector):
    G = ua.shape[1]
    da = torch.as_tensor(ua, device="cuda").contiguous()
    db = torch.as_tensor(ub, device="cuda").contiguous()
    nb = mclbm.mclbm_w1_2pt_work_bytes(ua.shape[0], ub.shape[0], G, vector)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    per = torch.empty(G * (G + 1) // 2 * (1 if vector else 3), dtype=torch.float64, device="cuda")
    W = mclbm.mclbm_w1_2pt(da.data_ptr(), ua.shape[0], db.data_ptr(), ub.shape[0], G, vector, work.data_ptr(), nb,
                           torch.cuda.current_stream().cuda_stream, per.data_ptr())
    per = per.cpu().numpy()
    return W, per if vector else per.reshape(-1, 3)


def _check(W, per, Wref, Dref):
    scale = np.abs(Dref).max()
    assert np.all(np.abs(per - Dref) <= RTOL * np.abs(Dref) + 1e-14 * scale), np.max(np.abs(per - Dref) / scale)
    assert abs(W - Wref) <= RTOL * Wref


@pytest.mark.parametrize("MA,MB", [(6, 6), (8, 4), (6, 4), (1, 3)])
@pytest.mark.parametrize("vector", [1, 0])
def test_random_fields_against_oracle(MA, MB, vector):
    """G = 8 points (a 2^3 grid): every pair, equal and unequal sample counts (L = lcm up to 12)."""
    ua = gen.uniform(100 + MA, (MA, 8, 3))
    ub = gen.uniform(200 + MB, (MB, 8, 3)) * 1.2 + 0.05
    W, per = _gpu(ua, ub, vector)
    Wref, Dref = stats.w1_two_point(ua, ub, vector=bool(vector), per_pair=True)
    _check(W, per, Wref, Dref)


@pytest.mark.parametrize("vector", [1, 0])
def test_consecutive_levels_of_rtgv_ensembles(vector):
    """Restrictions (Q = 4, G = 64, 2080 pairs) of a 16^3 x 8 and a 32^3 x 4 RTGV ensemble after a
    few steps (L = 8)."""
    a = Ensemble(16, 8, Re=400.0, Ma=0.1, precision="fp32", seed=3).init().step(6)
    b = Ensemble(32, 4, Re=1600.0, Ma=0.05, precision="fp32", seed=4).init().step(24)
    ua, ub = a.restrict(4).cpu().numpy(), b.restrict(4).cpu().numpy()
    W, per = _gpu(ua, ub, vector)
    Wref, Dref = stats.w1_two_point(ua, ub, vector=bool(vector), per_pair=True)
    _check(W, per, Wref, Dref)
    assert abs(a.w1_2pt(b, Q=4, vector=bool(vector)) - W) <= 1e-15 * W  # the Ensemble method


def test_full_grid_64_samples_sampled_pairs():
    """G = 512 (the 8^3 grid), M = 64 against M = 32 (L = 64): 40 sampled pairs of the vector and
    component-wise problems against the oracle, and the aggregate equals the weighted pair sum."""
    M1, M2, G = 64, 32, 512
    ua = gen.normal(7, (M1, G, 3), 0.3)
    ub = gen.normal(8, (M2, G, 3), 0.3) + 0.01
    rng = np.random.default_rng(9)
    pairs = [(0, 0), (0, G - 1), (G - 1, G - 1)] + [tuple(sorted(rng.integers(0, G, 2))) for _ in range(37)]
    for vector in (1, 0):
        W, per = _gpu(ua, ub, vector)
        w = np.array([1.0 if i == j else 2.0 for i in range(G) for j in range(i, G)])
        pv = per if vector else per.sum(axis=1)
        assert abs(W - (w * pv).sum() / G**2) <= 1e-12 * W
        for i, j in pairs:
            k = stats.pair_index(i, j, G)
            if vector:
                ref = stats.ot_w1(np.concatenate([ua[:, i], ua[:, j]], axis=1),
                                  np.concatenate([ub[:, i], ub[:, j]], axis=1))
                assert abs(per[k] - ref) <= RTOL * ref
            else:
                for c in range(3):
                    ref = stats.ot_w1(np.stack([ua[:, i, c], ua[:, j, c]], axis=1),
                                      np.stack([ub[:, i, c], ub[:, j, c]], axis=1))
                    assert abs(per[k, c] - ref) <= RTOL * ref


def test_identical_laws_and_shape_errors():
    ua = gen.uniform(41, (16, 8, 3))
    for vector in (1, 0):
        W, per = _gpu(ua, ua, vector)
        assert W == 0.0 and np.all(per == 0.0)
    da = torch.zeros((1025, 8, 3), dtype=torch.float64, device="cuda")
    nb = mclbm.mclbm_w1_2pt_work_bytes(64, 64, 8, 1)
    work = torch.empty(nb, dtype=torch.uint8, device="cuda")
    assert mclbm.mclbm_w1_2pt_work_bytes(1025, 64, 8, 1) == 0
    with pytest.raises(mclbm.MclbmError) as e:  # more than 1024 samples on one side
        mclbm.mclbm_w1_2pt(da.data_ptr(), 1025, da.data_ptr(), 64, 8, 1, work.data_ptr(), nb)
    assert e.value.status == "SHAPE"
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_w1_2pt(da.data_ptr(), 64, da.data_ptr(), 64, 8, 1, work.data_ptr(), nb - 8)
    assert e.value.status == "OOM"


@pytest.mark.parametrize("vector", [1, 0])
def test_paper_sample_count_100_every_pair(vector):
    """M = 100 on both sides (the paper's smaller EOWC ensembles; one block per transport
    problem), G = 27 points: every one of the 378 pairs against the oracle's assignment, and the
    aggregate; a second call gives the same bits (fixed tie-breaking and reduction order)."""
    M, G = 100, 27
    ua = gen.normal(300, (M, G, 3), 0.3)
    ub = gen.normal(301, (M, G, 3), 0.3) + 0.02
    W, per = _gpu(ua, ub, vector)
    Wref, Dref = stats.w1_two_point(ua, ub, vector=bool(vector), per_pair=True)
    _check(W, per, Wref, Dref)
    W2, per2 = _gpu(ua, ub, vector)
    assert W2 == W and np.array_equal(per2, per)


@pytest.mark.parametrize("vector", [1, 0])
def test_paper_sample_count_1000_sampled_pairs(vector):
    """M = 1000 on both sides (the paper's larger EOWC ensembles): G = 2 points, all three pairs
    against the oracle's assignment."""
    M, G = 1000, 2
    ua = gen.normal(310, (M, G, 3), 0.3)
    ub = gen.normal(311, (M, G, 3), 0.3) + 0.01
    W, per = _gpu(ua, ub, vector)
    Wref, Dref = stats.w1_two_point(ua, ub, vector=bool(vector), per_pair=True)
    _check(W, per, Wref, Dref)


@pytest.mark.parametrize("MA,MB,G", [(120, 90, 4), (250, 240, 2), (100, 50, 4), (64, 48, 4), (7, 100, 4)])
@pytest.mark.parametrize("vector", [1, 0])
def test_unequal_sample_counts_transportation(MA, MB, G, vector):
    """Unequal sample counts beyond the replicated assignment (lcm > 64): the transportation
    problem with supply MB/g and demand MA/g per atom (g = gcd), flows in the work buffer,
    against the oracle's transport linear program on every pair."""
    ua = gen.normal(320 + MA, (MA, G, 3), 0.3)
    ub = gen.normal(321 + MB, (MB, G, 3), 0.3) + 0.03
    W, per = _gpu(ua, ub, vector)
    Wref, Dref = stats.w1_two_point(ua, ub, vector=bool(vector), per_pair=True)
    _check(W, per, Wref, Dref)


def test_coprime_sample_counts_1000_999():
    """1000 against 999 samples (coprime: lcm 999000, no replicated assignment exists): one point
    pair of the vector problem against the oracle's transport linear program."""
    ua = gen.normal(330, (1000, 1, 3), 0.3)
    ub = gen.normal(331, (999, 1, 3), 0.3) + 0.01
    W, per = _gpu(ua, ub, 1)
    Wref, Dref = stats.w1_two_point(ua, ub, vector=True, per_pair=True)
    _check(W, per, Wref, Dref)


def test_identical_laws_at_100_samples():
    ua = gen.normal(340, (100, 8, 3), 0.3)
    for vector in (1, 0):
        W, per = _gpu(ua, ua, vector)
        assert W == 0.0 and np.all(per == 0.0)

"""Launch-shape variants, the autotuner, and the batched multi-level launch with CUDA-graph
replay: all must give bit-identical states to the plain single-level path (every variant
does the same per-node arithmetic), which the oracle parity tests pin."""
import numpy as np
import pytest
import torch

import ensemble_inputs as gen
from paper_2608_23786_gb300 import Ensemble, mclbm

pytestmark = pytest.mark.gpu

VARIANTS = {"fp64": [1, 2], "fp32": [1, 2, 4], "fp16": [2, 4, 8]}
STAGED = [1, 2]


def _shapes(precision, N):
    """(kind, vec, block) of every launch shape that applies to a lattice of side N."""
    out = [(k, v, b) for k in (0, 2) for v in VARIANTS[precision] if N % v == 0 for b in (128, 256)]
    if precision != "fp64":  # packed FP32 collision of node pairs; shared-memory prefetch rings
        out += [(3, v, b) for v in VARIANTS[precision] if v % 2 == 0 and N % v == 0 for b in (128, 256)]
        out += [(k, v, 128) for k in (4, 5) for v in VARIANTS[precision] if N % v == 0]
    out += [(1, v, 0) for v in STAGED if N % v == 0]
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def _states(ens):
    return [ens.populations(m) for m in range(ens.M)]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("pattern", ["pull", "aa"])
@pytest.mark.parametrize("N,steps", [(8, 3), (32, 5), (64, 2)])
def test_every_launch_shape_gives_identical_states(precision, pattern, N, steps):
    """N = 8 (a row is one or a few threads: every lane is a row start), 32 and 64 (rows
    span part of a warp, a full warp, or several)."""
    X = gen.draw_params(31, 2)
    ref = None
    for kind, vec, block in _shapes(precision, N):
        ens = Ensemble(N, 2, Re=300.0, Ma=0.1, precision=precision, pattern=pattern).init(X)
        mclbm.mclbm_set_launch(ens.ctx, vec, block, kind)
        ens.step(steps)
        mclbm.mclbm_device_status(ens.ctx)
        got = _states(ens)
        if ref is None:
            ref = got
        else:
            for a, b in zip(ref, got):
                assert torch.equal(a, b), (kind, vec, block)
    # and AA equals pull for the default shape
    other = Ensemble(N, 2, Re=300.0, Ma=0.1, precision=precision,
                     pattern="pull" if pattern == "aa" else "aa").init(X).step(steps)
    for a, b in zip(ref, _states(other)):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_aa_parities_with_their_own_shapes_give_identical_states(precision):
    """An AA context whose odd steps take another shape (row offsets, ring kernels) than its
    even steps reaches the same state, bit for bit, as one shape for both; the shape rules:
    parity 1 only under AA, the staged kind set for one parity serves both."""
    N, steps = 32, 5
    X = gen.draw_params(32, 2)
    ref = Ensemble(N, 2, Re=300.0, Ma=0.1, precision=precision, pattern="aa").init(X)
    mclbm.mclbm_set_launch(ref.ctx, 2, 128, 0)
    ref.step(steps)
    odd_shapes = [s for s in _shapes(precision, N) if s[0] != 1]
    for even in [(3, 2, 128), (0, 4, 256)]:
        for odd in odd_shapes[:: max(1, len(odd_shapes) // 6)]:
            ens = Ensemble(N, 2, Re=300.0, Ma=0.1, precision=precision, pattern="aa").init(X)
            mclbm.mclbm_set_launch_parity(ens.ctx, 0, even[1], even[2], even[0])
            mclbm.mclbm_set_launch_parity(ens.ctx, 1, odd[1], odd[2], odd[0])
            assert mclbm.mclbm_get_launch_parity(ens.ctx, 0) == even
            assert mclbm.mclbm_get_launch_parity(ens.ctx, 1) == odd
            ens.step(steps)
            mclbm.mclbm_device_status(ens.ctx)
            for a, b in zip(_states(ref), _states(ens)):
                assert torch.equal(a, b), (even, odd)
    ens = Ensemble(N, 2, Re=300.0, Ma=0.1, precision=precision, pattern="aa").init(X)
    mclbm.mclbm_set_launch_parity(ens.ctx, 1, 2, 0, 1)  # staged: both parities
    assert mclbm.mclbm_get_launch_parity(ens.ctx, 0) == (1, 2, 0)
    mclbm.mclbm_set_launch_parity(ens.ctx, 0, 2, 128, 3)  # another kind on one parity replaces both
    assert mclbm.mclbm_get_launch_parity(ens.ctx, 1) == (3, 2, 128)
    pull = Ensemble(N, 2, Re=300.0, Ma=0.1, precision=precision, pattern="pull").init(X)
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_set_launch_parity(pull.ctx, 1, 2, 128, 3)
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_set_launch_parity(ens.ctx, 2, 2, 128, 3)


def test_aa_autotune_tunes_each_parity_and_restores_the_initial_state():
    ens = Ensemble(32, 4, Re=400.0, Ma=0.05, precision="fp16", pattern="aa", seed=9).init()
    before = _states(ens)
    kind, vec, block, ms = mclbm.mclbm_autotune(ens.ctx, 2)
    odd = mclbm.mclbm_get_launch_parity(ens.ctx, 1)
    assert (kind, vec, block) in _shapes("fp16", 32) and odd in _shapes("fp16", 32) and ms > 0
    assert (kind == 1) == (odd[0] == 1)
    assert ens.steps_taken == 0
    for a, b in zip(before, _states(ens)):
        assert torch.equal(a, b)


def test_autotune_picks_a_supported_shape_and_restores_the_initial_state():
    ens = Ensemble(32, 4, Re=400.0, Ma=0.05, precision="fp32", seed=9).init()
    before = _states(ens)
    kind, vec, block, ms = mclbm.mclbm_autotune(ens.ctx, 2)
    assert (kind, vec, block) in _shapes("fp32", 32) and ms > 0
    assert mclbm.mclbm_get_launch(ens.ctx) == (kind, vec, block)
    assert ens.steps_taken == 0
    for a, b in zip(before, _states(ens)):
        assert torch.equal(a, b)
    ens.step(1)
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_autotune(ens.ctx, 1)


def _levels(precision, pattern, stream, sizes=((16, 3), (32, 2), (64, 1)), seeds=(1, 2, 3)):
    res = (400.0, 1600.0, 3200.0)
    mas = (0.1, 0.05, 0.025)
    out = []
    for (N, M), Re, Ma, s in zip(sizes, res, mas, seeds):
        out.append(Ensemble(N, M, Re=Re, Ma=Ma, precision=precision, pattern=pattern, seed=s,
                            stream=stream).init())
    return out


@pytest.mark.parametrize("precision,pattern", [("fp32", "pull"), ("fp32", "aa"), ("fp16", "aa"), ("fp64", "pull")])
@pytest.mark.parametrize("substeps,graph,macro", [((1, 4, 16), True, 3), ((1, 4, 16), False, 2), ((2, 4, 8), True, 4),
                                                   ((1, 2, 4), True, 5)])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_batch_equals_separate_levels(precision, pattern, substeps, graph, macro, kind):
    """One persistent launch per sub-step over all levels (and its graph replay) equals
    stepping each level on its own by macro * substeps[l] steps, bit for bit; includes odd
    per-level step counts (graph period of two macro steps) and a macro count that is not a
    multiple of the period."""
    stream = torch.cuda.Stream()
    lv = _levels(precision, pattern, stream)
    ref = _levels(precision, pattern, stream)
    b = mclbm.mclbm_batch_create([e.ctx for e in lv], substeps)
    try:
        mclbm.mclbm_batch_set_graph(b, graph)
        if kind == 1:
            mclbm.mclbm_batch_set_launch(b, 1, 0, kind=1)
        elif kind == 2:
            mclbm.mclbm_batch_set_launch(b, 2, 128, kind=2)
        mclbm.mclbm_batch_step(b, macro)
        assert mclbm.mclbm_batch_macro_steps(b) == macro
        stream.synchronize()
        for e, r, s in zip(lv, ref, substeps):
            r.step(macro * s)
            assert e.steps_taken == macro * s
            mclbm.mclbm_device_status(e.ctx)
            for a, c in zip(_states(e), _states(r)):
                assert torch.equal(a, c)
    finally:
        mclbm.mclbm_batch_destroy(b)


@pytest.mark.parametrize("precision,even,odd", [("fp32", (3, 2, 128), (5, 4, 128)), ("fp16", (4, 8, 128), (3, 4, 128)),
                                                ("fp16", (0, 2, 256), (2, 4, 128))])
def test_aa_batch_with_a_shape_per_parity_equals_separate_levels(precision, even, odd):
    """An AA batch whose odd steps take another launch shape (the levels' parities differ within
    a sub-step, so each sub-step splits into one launch per parity), replayed from its graph,
    equals stepping each level on its own, bit for bit; the shapes read back per parity."""
    stream = torch.cuda.Stream()
    lv = _levels(precision, "aa", stream)
    ref = _levels(precision, "aa", stream)
    substeps, macro = (1, 4, 16), 3
    b = mclbm.mclbm_batch_create([e.ctx for e in lv], substeps)
    try:
        mclbm.mclbm_batch_set_launch_parity(b, 0, even[1], even[2], even[0])
        mclbm.mclbm_batch_set_launch_parity(b, 1, odd[1], odd[2], odd[0])
        assert mclbm.mclbm_batch_get_launch_parity(b, 0) == even
        assert mclbm.mclbm_batch_get_launch_parity(b, 1) == odd
        mclbm.mclbm_batch_step(b, macro)
        stream.synchronize()
        for e, r, sub in zip(lv, ref, substeps):
            r.step(macro * sub)
            mclbm.mclbm_device_status(e.ctx)
            for a_, c in zip(_states(e), _states(r)):
                assert torch.equal(a_, c)
    finally:
        mclbm.mclbm_batch_destroy(b)


def test_batch_autotune_and_validation():
    stream = torch.cuda.Stream()
    lv = _levels("fp32", "pull", stream)
    b = mclbm.mclbm_batch_create([e.ctx for e in lv], (1, 4, 16))
    try:
        kind, vec, block, ms = mclbm.mclbm_batch_autotune(b, 1)
        assert (kind, vec, block) in _shapes("fp32", 16) and ms > 0
        assert all(e.steps_taken == 0 for e in lv)
    finally:
        mclbm.mclbm_batch_destroy(b)
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_batch_create([e.ctx for e in lv], (1, 3, 16))  # 3 does not divide 16
    other = Ensemble(16, 1, Re=100.0, Ma=0.1, precision="fp16", stream=stream).init()
    with pytest.raises(mclbm.MclbmError):
        mclbm.mclbm_batch_create([lv[0].ctx, other.ctx], (1, 4))  # mixed precision


def test_batch_odd_step_default_follows_the_largest_level():
    """An FP16 AA batch whose odd-step shape is still the default takes the default of its largest
    level: 8 nodes per thread in the two-stage ring where the largest rows have up to 256 nodes
    (rows within one warp rotate), 4 in the packed prefetching kernel beyond; the stepped states
    equal those of per-level stepping to the bit."""
    stream = torch.cuda.Stream()
    small = [Ensemble(N, 1, Re=400.0, Ma=0.05, precision="fp16", pattern="aa", seed=N, stream=stream).init()
             for N in (32, 64)]
    b = mclbm.mclbm_batch_create([e.ctx for e in small], [1, 2])
    assert mclbm.mclbm_batch_get_launch_parity(b, 1) == (4, 8, 128)
    mclbm.mclbm_batch_destroy(b)
    big = Ensemble(512, 1, Re=400.0, Ma=0.05, precision="fp16", pattern="aa", seed=5, stream=stream)
    assert mclbm.mclbm_get_launch_parity(big.ctx, 1) == (3, 4, 128)
    del big
    spec = [(64, 2, 1), (256, 1, 2)]
    lv = [Ensemble(N, M, Re=400.0, Ma=0.05, precision="fp16", pattern="aa", seed=N, stream=stream).init()
          for N, M, _ in spec]
    b = mclbm.mclbm_batch_create([e.ctx for e in lv], [s for _, _, s in spec])
    assert mclbm.mclbm_batch_get_launch_parity(b, 1) == (4, 8, 128)
    mclbm.mclbm_batch_step(b, 3)
    stream.synchronize()
    mclbm.mclbm_batch_destroy(b)
    for (N, M, s), e in zip(spec, lv):
        ref = Ensemble(N, M, Re=400.0, Ma=0.05, precision="fp16", pattern="aa", seed=N, stream=stream).init()
        ref.step(3 * s)
        assert e.steps_taken == 3 * s
        for m in range(M):
            assert torch.equal(e.populations(m), ref.populations(m))


@pytest.mark.parametrize("precision,shapes", [("fp16", [(3, 4, 128), (3, 4, 256), (2, 4, 128)]),
                                              ("fp32", [(3, 2, 128), (2, 1, 128), (3, 4, 128)])])
def test_aa_odd_steps_with_rows_across_warps_equal_pull(precision, shapes):
    """N = 256 with 1 to 4 nodes per thread: a row spans 2 to 8 warps, so the odd step's end
    elements cross warp boundaries (loaded and stored apart); AA reaches pull's state to the bit."""
    X = gen.draw_params(33, 1)
    pull = Ensemble(256, 1, Re=800.0, Ma=0.05, precision=precision, pattern="pull").init(X).step(3)
    for kind, vec, block in shapes:
        ens = Ensemble(256, 1, Re=800.0, Ma=0.05, precision=precision, pattern="aa").init(X)
        mclbm.mclbm_set_launch_parity(ens.ctx, 1, vec, block, kind)
        ens.step(3)
        mclbm.mclbm_device_status(ens.ctx)
        assert torch.equal(ens.populations(0), pull.populations(0)), (kind, vec, block)

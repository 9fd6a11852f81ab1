"""Host logic of the batch scheduler (no GPU): the longest-processing-time-first
lane rule behind pce_apply_batch / pce_batch_create, and the uneven task mix.

LPT is checked against brute force on tiny instances: its makespan is within
Graham's bound (4/3 - 1/(3 lanes)) of the optimum, it is deterministic, and
it reduces to the obvious answers in special cases.
"""
import itertools

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lib():
    from paper_1604_04374_gb300 import build
    build.build()
    from paper_1604_04374_gb300 import pce
    pce.load_library()
    return pce


def optimum(cost, lanes):
    best = float("inf")
    for assign in itertools.product(range(lanes), repeat=len(cost)):
        load = [0.0] * lanes
        for c, l in zip(cost, assign):
            load[l] += c
        best = min(best, max(load))
    return best


@pytest.mark.parametrize("seed", range(12))
def test_lpt_within_graham_bound_of_brute_force(lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 8))
    lanes = int(rng.integers(1, 4))
    cost = [float(c) for c in rng.integers(1, 20, n)]
    lane_of, makespan = lib.pce_schedule_lpt(cost, lanes)
    load = [0.0] * lanes
    for c, l in zip(cost, lane_of):
        assert 0 <= l < lanes
        load[l] += c
    assert makespan == max(load)
    assert makespan <= (4.0 / 3.0 - 1.0 / (3 * lanes)) * optimum(cost, lanes) + 1e-12
    assert lib.pce_schedule_lpt(cost, lanes) == (lane_of, makespan)


def test_lpt_special_cases(lib):
    # one lane: everything on it
    lane_of, ms = lib.pce_schedule_lpt([3.0, 1.0, 2.0], 1)
    assert lane_of == [0, 0, 0] and ms == 6.0
    # at least as many lanes as tasks: one task per lane, makespan = largest task
    lane_of, ms = lib.pce_schedule_lpt([3.0, 1.0, 2.0], 5)
    assert len(set(lane_of)) == 3 and ms == 3.0
    # equal costs: round robin in index order
    lane_of, ms = lib.pce_schedule_lpt([1.0] * 6, 3)
    assert lane_of == [0, 1, 2, 0, 1, 2] and ms == 2.0
    # the classic LPT example: largest first keeps the two big tasks apart
    lane_of, ms = lib.pce_schedule_lpt([5.0, 5.0, 4.0, 4.0, 3.0, 3.0, 3.0], 3)
    assert ms == 11.0
    assert lib.pce_schedule_lpt([], 2) == ([], 0.0)


def test_lpt_argument_errors(lib):
    with pytest.raises(lib.PceError) as e:
        lib.pce_schedule_lpt([1.0], 0)
    assert e.value.status == lib.PCE_ERR_INVALID
    with pytest.raises(lib.PceError) as e:
        lib.pce_schedule_lpt([1.0, -2.0], 2)
    assert e.value.status == lib.PCE_ERR_INVALID


def test_batch_entry_points_reject_bad_arguments_without_a_gpu(lib):
    import ctypes
    L = lib.load_library()
    out = ctypes.c_void_p()
    assert L.pce_batch_create(None, None, 0, 4) == lib.PCE_ERR_INVALID
    assert L.pce_batch_create(ctypes.byref(out), None, 0, 0) == lib.PCE_ERR_INVALID
    assert L.pce_batch_create(ctypes.byref(out), None, 0, 65) == lib.PCE_ERR_INVALID
    assert L.pce_batch_run(None, None) == lib.PCE_ERR_INVALID
    assert L.pce_batch_launch(None, None) == lib.PCE_ERR_INVALID
    assert L.pce_batch_destroy(None) == lib.PCE_OK
    assert L.pce_plan_autotune(None, 4, None, None) == lib.PCE_ERR_INVALID
    assert L.pce_plan_tuning(None, None, None, None, None) == lib.PCE_ERR_INVALID
    assert L.pce_plan_tuning_log(None, 0, None, None, None, None) == 0


def test_batch_mix_is_seeded_and_uneven():
    a = synth.batch_mix(256, 4)
    b = synth.batch_mix(256, 4)
    assert a.op_of == b.op_of and a.adjoint == b.adjoint
    assert all(np.array_equal(x, y) for x, y in zip(a.inputs, b.inputs))
    kinds = {(a.ops[i][0], a.ops[i][1]) for i in a.op_of}
    assert {s for s, _ in kinds} == set(synth.BATCH_SHAPES)
    assert {m for _, m in kinds} == set(synth.BATCH_M)
    assert 0.35 < np.mean(a.adjoint) < 0.65
    for shape, m, w, h in a.ops:
        assert w.shape == (m,) + shape and h.shape == (m,) + shape
        assert w.dtype == np.float32 and h.dtype == np.float32
        np.testing.assert_allclose(w.sum(axis=0), 1.0, atol=1e-5)    # partition of unity
    for i, x in enumerate(a.inputs):
        assert x.shape == (1,) + a.ops[a.op_of[i]][0] and x.dtype == np.float32

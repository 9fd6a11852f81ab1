"""GPU: batches of uneven applies, CUDA-graph replay and the autotuner.

A batch runs the same kernels as single applies, on other streams and other
scratch, so its outputs must equal pce_apply / pce_apply_adjoint bit for bit
(same right-hand sides per launch); a few tasks are also checked against the
FP64 oracle (rel l2 <= 1e-5).  The autotuner's choices (column variant,
right-hand sides per launch) change rounding order only: tuned plans are
checked against the oracle, and its cache file is read back.
"""
import json

import numpy as np
import pytest

import synth
from oracle import expansion as E

pytestmark = pytest.mark.gpu

TOL = 1e-5
SMALL_SHAPES = ((256,), (4096,), (16384,), (64, 64), (128, 128), (32, 1024))
SMALL_M = (4, 8, 16)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_1604_04374_gb300 import build
    build.build()
    torch.cuda.init()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(got, ref):
    got = got.reshape(got.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))


@pytest.fixture(scope="module")
def mix(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    mx = synth.batch_mix(40, 11, SMALL_SHAPES, SMALL_M)
    plans = [Plan(dev(torch, w), h=dev(torch, h)) for _, _, w, h in mx.ops]
    ins = [dev(torch, u) for u in mx.inputs]
    return mx, plans, ins


def singles(torch, mx, plans, ins):
    outs = []
    for i, x in enumerate(ins):
        p = plans[mx.op_of[i]]
        outs.append(p.apply_adjoint(x) if mx.adjoint[i] else p.apply(x))
    torch.cuda.synchronize()
    return [host(o) for o in outs]


def tasks_of(torch, mx, plans, ins):
    outs = [torch.full_like(x, float("nan")) for x in ins]
    return [(plans[mx.op_of[i]], ins[i], outs[i], mx.adjoint[i]) for i in range(len(ins))], outs


def test_one_shot_batch_equals_single_applies(torch_cuda, mix):
    torch = torch_cuda
    from paper_1604_04374_gb300 import apply_batch
    mx, plans, ins = mix
    ref = singles(torch, mx, plans, ins)
    tasks, outs = tasks_of(torch, mx, plans, ins)
    apply_batch(tasks)
    torch.cuda.synchronize()
    for i in range(len(ins)):
        assert np.array_equal(host(outs[i]), ref[i]), i


@pytest.mark.parametrize("lanes", [1, 5, 16])
def test_batch_object_run_and_graph_launch(torch_cuda, mix, lanes):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch
    mx, plans, ins = mix
    ref = singles(torch, mx, plans, ins)
    tasks, outs = tasks_of(torch, mx, plans, ins)
    b = Batch(tasks, lanes=lanes)
    nl, scratch, launches, makespan, lane_of = b.info()
    assert nl == lanes and len(lane_of) == len(ins) and set(lane_of) <= set(range(lanes))
    assert launches == sum(plans[mx.op_of[i]].launch_count(mx.adjoint[i], 1) for i in range(len(ins)))
    b.run()
    torch.cuda.synchronize()
    for i in range(len(ins)):
        assert np.array_equal(host(outs[i]), ref[i]), i
    for o in outs:
        o.fill_(float("nan"))
    b.launch()
    b.launch()   # replay of the instantiated graph
    torch.cuda.synchronize()
    for i in range(len(ins)):
        assert np.array_equal(host(outs[i]), ref[i]), i
    b.close()


def test_batch_autotune_keeps_results(torch_cuda, mix):
    """Every policy runs the same operators: after tuning the outputs still equal the
    single applies up to rounding (column variants round differently)."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch
    mx, plans, ins = mix
    ref = singles(torch, mx, plans, ins)
    tasks, outs = tasks_of(torch, mx, plans, ins)
    b = Batch(tasks, lanes=6)
    (cp, rp), log = b.autotune()
    pols = (-1, 0, 1, 2)
    assert len(log) == 16 and {(c, r) for c, r, _ in log} == {(c, r) for c in pols for r in pols}
    assert all(ms > 0 for _, _, ms in log)
    assert (cp, rp, min(ms for _, _, ms in log)) in {(c, r, ms) for c, r, ms in log}
    for o in outs:
        o.fill_(float("nan"))
    b.launch()
    torch.cuda.synchronize()
    for i in range(len(ins)):
        assert rel(host(outs[i])[None], ref[i][None]) < 1e-6, i
    # a second batch over the same plans given the same policies by hand computes the same bits
    tasks2, outs2 = tasks_of(torch, mx, plans, ins)
    b2 = Batch(tasks2, lanes=6)
    b2.set_tuning(cp, rp)
    b2.launch()
    torch.cuda.synchronize()
    for i in range(len(ins)):
        assert np.array_equal(host(outs2[i]), host(outs[i])), i
    b2.close()
    b.close()


def test_batch_tasks_match_oracle(torch_cuda, mix):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch
    mx, plans, ins = mix
    tasks, outs = tasks_of(torch, mx, plans, ins)
    b = Batch(tasks, lanes=8)
    b.launch()
    torch.cuda.synchronize()
    checked = 0
    for i in range(len(ins)):
        shape, m, w, h = mx.ops[mx.op_of[i]]
        if int(np.prod(shape)) > 16384 or (len(shape) == 1 and shape[0] > 4096):
            continue
        fn = E.apply_adjoint if mx.adjoint[i] else E.apply
        assert rel(host(outs[i]), fn(mx.inputs[i], w, h)) < TOL, i
        checked += 1
    assert checked >= 10
    b.close()


def test_batch_rejects_dependent_or_bad_tasks(torch_cuda, mix):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan, apply_batch, pce
    from paper_1604_04374_gb300.pce import PceError
    mx, plans, ins = mix
    p = plans[mx.op_of[0]]
    x = ins[0]
    y = torch.empty_like(x)
    with pytest.raises(PceError) as e:       # two tasks write the same output
        apply_batch([(p, x, y, False), (p, x.clone(), y, True)])
    assert e.value.status == pce.PCE_ERR_INVALID
    with pytest.raises(PceError) as e:       # a task reads what another writes
        Batch([(p, x, y, False), (p, y, torch.empty_like(x), False)], lanes=2)
    assert e.value.status == pce.PCE_ERR_INVALID
    shape, m, w, h = mx.ops[mx.op_of[0]]
    if len(shape) == 2:
        up = Plan(dev(torch, w), h=dev(torch, h), flags=pce.PCE_FLAG_UNFUSED)
        with pytest.raises(PceError) as e:
            apply_batch([(up, x, y, False)])
        assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    with pytest.raises(PceError) as e:
        Batch([(p, x, y, False)], lanes=0)
    assert e.value.status == pce.PCE_ERR_INVALID
    apply_batch([])                          # empty batch is a no-op


def test_autotune_variants_and_cache(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    pr = synth.problem_2d(1024, 32, 4, 3, 61, "normal")
    cache = str(tmp_path / "tune.jsonl")
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    chunk, variant, rvariant, ms = plan.autotune(3, cache)
    assert 1 <= chunk <= 3 and variant in (0, 1) and rvariant in (0, 1, 2) and ms > 0
    # chunks 1..3 x column variants 0, 1 x row variants 0, 1, 2 (the row-pair windowed R2C
    # serves rows of any length)
    assert len(plan.tuning_log()) == 3 * 2 * 3
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["chunk"] == chunk and rec["variant"] == variant and rec["row_variant"] == rvariant
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL
    # a second plan of the same operator reads the cache; force the other variant through it
    other_r = 1 if rvariant != 1 else 0
    rec2 = dict(rec, variant=1 - variant, row_variant=other_r, chunk=1)
    with open(cache, "a") as f:
        f.write(json.dumps(rec2) + "\n")
    p2 = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    c2, v2, r2, _ = p2.autotune(3, cache)
    assert (c2, v2, r2) == (1, 1 - variant, other_r)
    assert p2.tuning_log() == []
    assert len(open(cache).read().splitlines()) == 2      # nothing appended
    assert rel(host(p2.apply(u)), E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(p2.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


@pytest.mark.parametrize("shape,m", [((256,), 4), ((16384,), 3), ((64, 128), 4)])
def test_autotune_other_plans(torch_cuda, shape, m):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    if len(shape) == 1:
        pr = synth.problem_1d(shape[0], m, 4, 62)
    else:
        pr = synth.problem_2d(shape[0], shape[1], m, 4, 62, "normal")
    plan = Plan(dev(torch, pr.w), h=dev(torch, pr.h))
    chunk, variant, rvariant, ms = plan.autotune(4)
    assert variant == 0 and ms > 0 and chunk >= 1
    assert rvariant in ((0, 1, 2) if len(shape) == 2 else (0,))
    u = dev(torch, pr.u)
    assert rel(host(plan.apply(u)), E.apply(pr.u, pr.w, pr.h)) < TOL
    assert rel(host(plan.apply_adjoint(u)), E.apply_adjoint(pr.u, pr.w, pr.h)) < TOL


def test_full_uneven_batch_as_benchmarked(torch_cuda):
    """The 256-task mix (1D 4096/16384/65536, 2D 256^2/512^2/1024^2, m 4..32, both
    directions) as one graph launch after batch-level tuning: every task equals its
    single apply up to rounding order, and sampled outputs of 1D tasks match the oracle."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan
    mx = synth.batch_mix(256, 4)
    plans = [Plan(dev(torch, w), h=dev(torch, h)) for _, _, w, h in mx.ops]
    ins = [dev(torch, u) for u in mx.inputs]
    ref = singles(torch, mx, plans, ins)
    tasks, outs = tasks_of(torch, mx, plans, ins)
    b = Batch(tasks, lanes=16)
    b.autotune()
    b.launch()
    torch.cuda.synchronize()
    for i in range(len(ins)):
        assert rel(host(outs[i])[None], ref[i][None]) < 1e-6, i
    rng = np.random.default_rng(2)
    checked = 0
    for i in range(len(ins)):
        shape, m, w, h = mx.ops[mx.op_of[i]]
        if len(shape) != 1 or checked >= 12:
            continue
        pts = rng.integers(0, shape[0], 32)[:, None]
        fn = E.apply_adjoint_at if mx.adjoint[i] else E.apply_at
        assert rel(host(outs[i]).reshape(1, -1)[:, pts[:, 0]], fn(mx.inputs[i], w, h, pts)) < TOL, i
        checked += 1
    b.close()


def test_full_mix_with_separable_plans(torch_cuda):
    """The 256-task mix with its 2D node-grid hats as separable plans (as the benchmark
    builds them): every task of the batch graph equals the dense plan's single apply to
    1e-5 (the two forms round differently), and sampled outputs of 2D separable tasks
    match the oracle."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan
    mx = synth.batch_mix(256, 4)
    dense = [Plan(dev(torch, w), h=dev(torch, h)) for _, _, w, h in mx.ops]
    plans, separable = [], []
    for (shape, m, w, h), pd in zip(mx.ops, dense):
        sep = False
        if len(shape) == 2:
            wy, wx = synth.hat_factors_2d(shape[0], shape[1], *synth.node_grid(m))
            sep = bool(np.array_equal(np.einsum("kr,kc->krc", wy, wx), w))
        plans.append(Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h)) if sep else pd)
        separable.append(sep)
    assert sum(separable) > 0
    ins = [dev(torch, u) for u in mx.inputs]
    ref = singles(torch, mx, dense, ins)
    tasks, outs = tasks_of(torch, mx, plans, ins)
    b = Batch(tasks, lanes=16)
    b.launch()
    torch.cuda.synchronize()
    for i in range(len(ins)):
        assert rel(host(outs[i])[None], ref[i][None]) < 1e-5, i
    rng = np.random.default_rng(3)
    checked = 0
    for i in range(len(ins)):
        o = mx.op_of[i]
        shape, m, w, h = mx.ops[o]
        if not separable[o] or checked >= 6:
            continue
        pts = np.stack([rng.integers(0, n, 48) for n in shape], axis=-1)
        fn = E.apply_adjoint_at if mx.adjoint[i] else E.apply_at
        got = host(outs[i])[0][tuple(pts.T)][None]
        assert rel(got, fn(mx.inputs[i], w, h, pts)) < TOL, i
        checked += 1
    b.close()

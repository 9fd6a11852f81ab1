"""GPU: plans with tensor-product windows w_k = wy_k (x) wx_k (pce_plan_create_separable).

For Ny = 1024 or 512 (FP32 storage) the applies take the separable fast path (one
row-transform slot per distinct column factor); its outputs are checked
against the FP64 oracle on the dense windows outer(wy_k, wx_k), and against
the general path of pce_plan_create on the same dense windows.  Other sizes
and storage modes fall back to the general path, which must give the same
operator.
"""
import numpy as np
import pytest

import synth
from oracle import direct as C
from oracle import expansion as E

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def sep_problem(ny, nx, gy, gx, batch, seed, random_h=False):
    wy, wx = synth.hat_factors_2d(ny, nx, gy, gx)
    pr = synth.problem_2d(ny, nx, gy * gx, batch, seed, "normal", (gy, gx))
    assert np.array_equal(pr.w, np.einsum("kr,kc->krc", wy, wx))
    h = pr.h
    if random_h:
        rng = np.random.default_rng(seed)
        h = np.zeros_like(pr.h)
        h[:, np.r_[0:6, ny - 5:ny][:, None], np.r_[0:6, nx - 5:nx][None, :]] = rng.standard_normal(
            (gy * gx, 11, 11)).astype(np.float32)
    return wy, wx, pr.w, h, pr.u


@pytest.mark.parametrize("ny,nx,gy,gx,batch", [(1024, 64, 2, 2, 2), (1024, 128, 4, 2, 1), (1024, 32, 8, 4, 3),
                                                (512, 64, 4, 4, 2), (512, 32, 2, 2, 3), (512, 128, 8, 2, 1)])
def test_separable_fast_path_matches_oracle(torch_cuda, ny, nx, gy, gx, batch):
    """Ny = 1024 and 512 (one-warp column FFTs of 1024 or 512 points)."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    wy, wx, w, h, u = sep_problem(ny, nx, gy, gx, batch, 80 + gy + gx, random_h=True)
    plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    assert plan.slots() == gx
    ud = dev(torch, u)
    assert rel(host(plan.apply(ud)), E.apply(u, w, h)) < TOL
    assert rel(host(plan.apply_adjoint(ud)), E.apply_adjoint(u, w, h)) < TOL
    if ny == 512:
        # the pruned and slot-by-slot tensor-memory variants need 1024 rows
        for cv in (3, 4):
            with pytest.raises(Exception):
                plan.set_tuning(batch, cv, 0)
        # variant 2: the tensor-memory column kernels at 512 points; variant 1 runs the
        # general block kernels on the dense windows: the same operator
        for cv, rv in ((2, 0), (2, 1), (2, 2), (1, 1)):
            plan.set_tuning(batch, cv, rv)
            assert rel(host(plan.apply(ud)), E.apply(u, w, h)) < TOL
            assert rel(host(plan.apply_adjoint(ud)), E.apply_adjoint(u, w, h)) < TOL


def test_separable_equals_general_path_on_the_bench_workload_shape(torch_cuda):
    """1024 x 1024, m = 16 hats on 4 x 4 nodes, anisotropic PSFs, B = 3."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    wy, wx, w, h, u = sep_problem(1024, 1024, 4, 4, 3, 85)
    sep = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    gen = Plan(dev(torch, w), h=dev(torch, h))
    assert sep.slots() == 4 and gen.slots() == 0
    ud = dev(torch, u)
    for fn in ("apply", "apply_adjoint"):
        a = host(getattr(sep, fn)(ud))
        b = host(getattr(gen, fn)(ud))
        assert rel(a, b) < 2e-6, fn
    # sampled outputs against the oracle (gather form)
    rng = np.random.default_rng(3)
    pts = np.stack([rng.integers(0, 1024, 96), rng.integers(0, 1024, 96)], axis=-1)
    y = host(sep.apply(ud)).reshape(3, -1)[:, pts[:, 0] * 1024 + pts[:, 1]]
    x = host(sep.apply_adjoint(ud)).reshape(3, -1)[:, pts[:, 0] * 1024 + pts[:, 1]]
    assert rel(y, E.apply_at(u, w, h, pts)) < TOL
    assert rel(x, E.apply_adjoint_at(u, w, h, pts)) < TOL


def test_separable_fallbacks_and_flags(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, pce
    # other column length: general path, same operator
    wy, wx, w, h, u = sep_problem(128, 256, 2, 4, 2, 86, random_h=True)
    p = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    assert p.slots() == 0
    ud = dev(torch, u)
    assert rel(host(p.apply(ud)), E.apply(u, w, h)) < TOL
    # Ny = 1024 with reduced storage: general path
    wy, wx, w, h, u = sep_problem(1024, 64, 2, 2, 1, 87, random_h=True)
    ud = dev(torch, u)
    q = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h), flags=pce.PCE_FLAG_LOWP_STORAGE)
    assert q.slots() == 0
    assert rel(host(q.apply(ud)), E.apply(u, w, h)) < 3e-3
    # product-convolution form on the fast path
    r = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h), flags=pce.PCE_FLAG_PRODUCT_CONVOLUTION)
    assert r.slots() == 2
    assert rel(host(r.apply(ud)), E.product_convolution(u, w, h)) < TOL
    assert rel(host(r.apply_adjoint(ud)), E.product_convolution_adjoint(u, w, h)) < TOL
    # from spectra
    hhat = np.stack([np.fft.rfft2(h[k].astype(np.float64)) for k in range(4)]).astype(np.complex64)
    s = Plan(wy=dev(torch, wy), wx=dev(torch, wx), hhat=dev(torch, hhat))
    assert s.slots() == 2
    assert rel(host(s.apply(ud)), E.apply(u, w, h)) < TOL
    # gradients run on the general structures of a separable plan
    rr = np.random.default_rng(5).standard_normal(u.shape).astype(np.float32)
    du, dw, dh = s.backward(ud, dev(torch, rr))
    gdu, gdw, _, gdh = E.grad(u, w, h.astype(np.float64), rr)
    assert rel(host(du), gdu) < TOL and rel(host(dw)[None], gdw[None]) < TOL


def test_separable_with_stockham_columns_and_in_batches(torch_cuda, tmp_path):
    """Column variant 1 (block Stockham) has no separable form: the plan uses the
    general path then; the batch scheduler runs separable plans on lane scratch."""
    torch = torch_cuda
    import json
    from paper_1604_04374_gb300 import Batch, Plan
    wy, wx, w, h, u = sep_problem(1024, 64, 2, 2, 2, 88, random_h=True)
    ud = dev(torch, u)
    p = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    ref_y, ref_x = host(p.apply(ud)), host(p.apply_adjoint(ud))
    cache = str(tmp_path / "t.jsonl")
    p.autotune(2, cache)
    rec = json.loads(open(cache).read().splitlines()[0])
    with open(cache, "a") as f:
        f.write(json.dumps(dict(rec, variant=1, chunk=2)) + "\n")
    p2 = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    assert p2.autotune(2, cache)[1] == 1
    assert rel(host(p2.apply(ud)), ref_y) < 2e-6
    assert rel(host(p2.apply_adjoint(ud)), ref_x) < 2e-6
    outs = [torch.empty_like(ud) for _ in range(4)]
    b = Batch([(p, ud, outs[0], False), (p, ud, outs[1], True), (p2, ud, outs[2], False), (p2, ud, outs[3], True)],
              lanes=4)
    b.launch()
    torch.cuda.synchronize()
    for o, r in zip(outs, (ref_y, ref_x, ref_y, ref_x)):
        assert rel(host(o), r) < 2e-6
    b.close()


def test_bench_launch_configuration_full_size(torch_cuda):
    """The headline step exactly as timed: 1024 x 1024, m = 16, B = 8, separable plan,
    forward and adjoint as one graph launch of a two-lane batch.  Outputs equal the
    plain applies bit for bit and match the oracle at sampled outputs of every
    right-hand side."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan
    pr = synth.workload("2d_1024_m16_b8")
    wy, wx = synth.hat_factors_2d(1024, 1024, 4, 4)
    assert np.array_equal(np.einsum("kr,kc->krc", wy, wx), pr.w)
    plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, pr.h))
    plan.autotune(pr.batch)
    u = dev(torch, pr.u)
    y0, x0 = host(plan.apply(u)), host(plan.apply_adjoint(u))
    y, x = torch.empty_like(u), torch.empty_like(u)
    b = Batch([(plan, u, y, False), (plan, u, x, True)], lanes=2)
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    assert np.array_equal(host(y), y0) and np.array_equal(host(x), x0)
    b.close()
    rng = np.random.default_rng(11)
    pts = np.stack([rng.integers(0, 1024, 64), rng.integers(0, 1024, 64)], axis=-1)
    flat = pts[:, 0] * 1024 + pts[:, 1]
    ys = E.apply_at(pr.u, pr.w, pr.h, pts)
    xs = E.apply_adjoint_at(pr.u, pr.w, pr.h, pts)
    assert rel(y0.reshape(8, -1)[:, flat], ys) < TOL
    assert rel(x0.reshape(8, -1)[:, flat], xs) < TOL


def banded_factors(ny, nx, bands, seed):
    """Separable windows with chosen row supports: term k has the row factor
    nonzero (random, positive) on rows bands[k] = (r0, n) taken mod ny and a
    column factor from two column hats, so slots hold one or more terms and
    slot boxes can be partial or wrap the seam."""
    rng = np.random.default_rng(seed)
    m = len(bands)
    wy = np.zeros((m, ny), dtype=np.float32)
    for k, (r0, n) in enumerate(bands):
        rows = (r0 + np.arange(n)) % ny
        wy[k, rows] = rng.uniform(0.1, 1.0, n).astype(np.float32)
    wx = np.stack([synth.hat_1d(nx, 4, k % 2) for k in range(m)]).astype(np.float32)
    return wy, wx


@pytest.mark.parametrize("case", ["hats_2x2", "hats_8x4", "partial", "wrapped"])
def test_tensor_memory_columns_match_oracle(torch_cuda, case):
    """Column variant 2 (per-warp column and accumulator in tensor memory)
    against the FP64 oracle, forward and adjoint, on full, partial and
    seam-wrapping slot boxes and several right-hand sides."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    nx = 64
    if case.startswith("hats"):
        gy, gx = (2, 2) if case == "hats_2x2" else (8, 4)
        wy, wx, w, h, u = sep_problem(1024, nx, gy, gx, 3, 90 + gy, random_h=True)
    else:
        # slots of terms {0, 2} and {1, 3}; the slot boxes (550 and 800 rows, or 294 and
        # 150 rows across the seam) fit the general scratch of 4 x the largest term box
        bands = ([(0, 300), (150, 400), (250, 300), (600, 350)] if case == "partial"
                 else [(900, 200), (1000, 100), (120, 50), (950, 150)])
        wy, wx = banded_factors(1024, nx, bands, 91)
        w = np.einsum("kr,kc->krc", wy, wx)
        pr = synth.problem_2d(1024, nx, 4, 3, 92, "normal")
        h, u = pr.h, pr.u
    plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    assert plan.slots() == gx if case.startswith("hats") else plan.slots() == 2
    ud = dev(torch, u)
    yo, xo = E.apply(u, w, h), E.apply_adjoint(u, w, h)
    # variant 3 (pruned) needs every row factor inside 512 rows: not the 2 x 2 hats (1023 rows);
    # variant 4 (slot by slot) needs two or more slots
    variants = (2, 4) if case == "hats_2x2" else (2, 3, 4)
    if case == "hats_2x2":
        from paper_1604_04374_gb300 import PceError, pce
        with pytest.raises(PceError) as e:
            plan.set_tuning(0, 3, 0)
        assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    outs = {}
    for cv in variants:
        plan.set_tuning(0, cv, 0)
        assert plan.tuning()[1] == cv
        outs[cv] = (host(plan.apply(ud)), host(plan.apply_adjoint(ud)))
        assert rel(outs[cv][0], yo) < TOL, cv
        assert rel(outs[cv][1], xo) < TOL, cv
    # the same plan on the register variant: same operator up to rounding
    plan.set_tuning(0, 0, 0)
    for cv in variants:
        assert rel(host(plan.apply(ud)), outs[cv][0]) < 2e-6
        assert rel(host(plan.apply_adjoint(ud)), outs[cv][1]) < 2e-6
    plan.close()


def test_tensor_memory_columns_on_the_bench_workload(torch_cuda):
    """1024 x 1024, m = 16 hats, B = 8 in one launch: variant 2 equals variant 0
    to rounding on every output and matches the oracle at sampled outputs of
    every right-hand side; a graph of the two-lane batch replays it bit for bit."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan
    pr = synth.workload("2d_1024_m16_b8")
    wy, wx = synth.hat_factors_2d(1024, 1024, 4, 4)
    plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, pr.h))
    u = dev(torch, pr.u)
    plan.set_tuning(8, 0, 1)
    ya, xa = host(plan.apply(u)), host(plan.apply_adjoint(u))
    plan.set_tuning(8, 3, 1)
    y3, x3 = host(plan.apply(u)), host(plan.apply_adjoint(u))
    assert rel(y3, ya) < 2e-6 and rel(x3, xa) < 2e-6
    plan.set_tuning(8, 2, 1)
    yb, xb = host(plan.apply(u)), host(plan.apply_adjoint(u))
    assert rel(yb, ya) < 2e-6 and rel(xb, xa) < 2e-6
    y, x = torch.empty_like(u), torch.empty_like(u)
    b = Batch([(plan, u, y, False), (plan, u, x, True)], lanes=2)
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    assert np.array_equal(host(y), yb) and np.array_equal(host(x), xb)
    b.close()
    rng = np.random.default_rng(12)
    pts = np.stack([rng.integers(0, 1024, 64), rng.integers(0, 1024, 64)], axis=-1)
    flat = pts[:, 0] * 1024 + pts[:, 1]
    assert rel(yb.reshape(8, -1)[:, flat], E.apply_at(pr.u, pr.w, pr.h, pts)) < TOL
    assert rel(xb.reshape(8, -1)[:, flat], E.apply_adjoint_at(pr.u, pr.w, pr.h, pts)) < TOL
    plan.close()


def test_set_tuning_rejects_missing_variants(torch_cuda):
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan, PceError, pce
    wy, wx, w, h, u = sep_problem(128, 64, 2, 2, 1, 93, random_h=True)
    p = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))   # 128 rows: general structures
    for cv in (1, 2, 3, 4):
        with pytest.raises(PceError) as e:
            p.set_tuning(0, cv, 0)
        assert e.value.status == pce.PCE_ERR_UNSUPPORTED
    with pytest.raises(PceError) as e:
        p.set_tuning(0, 5, 0)
    assert e.value.status == pce.PCE_ERR_INVALID
    # row variant 2 on rows of 64 points: the row-pair windowed R2C, block plain transforms
    p.set_tuning(0, 0, 2)
    ud = dev(torch, u)
    assert rel(host(p.apply(ud)), E.apply(u, w, h)) < TOL
    assert rel(host(p.apply_adjoint(ud)), E.apply_adjoint(u, w, h)) < TOL
    with pytest.raises(PceError) as e:
        p.set_tuning(0, 0, 3)
    assert e.value.status == pce.PCE_ERR_INVALID
    p.close()


@pytest.mark.parametrize("col_variant", [0, 2, 3, 4])
def test_bench_configuration_every_output_against_oracle(torch_cuda, col_variant):
    """The headline step as timed (1024 x 1024, m = 16, B = 8, separable plan, forward and
    adjoint as one graph launch of a two-lane batch), both one-warp column variants:
    every output of right-hand sides 0 and 7 against the compiled FP64 oracle, so every
    column CTA (128 per right-hand side) and every row-pair CTA is covered."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan
    pr = synth.workload("2d_1024_m16_b8")
    wy, wx = synth.hat_factors_2d(1024, 1024, 4, 4)
    plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, pr.h))
    plan.set_tuning(8, col_variant, 1)
    u = dev(torch, pr.u)
    y, x = torch.empty_like(u), torch.empty_like(u)
    b = Batch([(plan, u, y, False), (plan, u, x, True)], lanes=2)
    b.launch()
    torch.cuda.synchronize()
    yh, xh = host(y), host(x)
    b.close()
    plan.close()
    for k in (0, 7):
        yo = C.apply(pr.u[k:k + 1], pr.w, pr.h)
        xo = C.apply_adjoint(pr.u[k:k + 1], pr.w, pr.h)
        for got, ref in ((yh[k:k + 1], yo), (xh[k:k + 1], xo)):
            assert rel(got, ref) < TOL
            assert np.max(np.abs(got - ref)) < TOL * np.max(np.abs(ref))


def test_tuning_cache_round_trip_of_the_tensor_memory_variant(torch_cuda, tmp_path):
    """A cached choice of column variant 2 is read back by a later plan of the same
    operator (and ignored by a plan without the separable structures)."""
    torch = torch_cuda
    import json
    from paper_1604_04374_gb300 import Plan
    wy, wx, w, h, u = sep_problem(1024, 64, 4, 2, 2, 94, random_h=True)
    cache = str(tmp_path / "t.jsonl")
    p = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    p.autotune(2, cache)
    rec = json.loads(open(cache).read().splitlines()[0])
    with open(cache, "a") as f:
        f.write(json.dumps(dict(rec, variant=2, chunk=1, row_variant=0)) + "\n")
    p2 = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    assert p2.autotune(2, cache)[:3] == (1, 2, 0)
    ud = dev(torch, u)
    assert rel(host(p2.apply(ud)), E.apply(u, w, h)) < TOL
    p.close()
    p2.close()


@pytest.mark.parametrize("case", ["separable_hats", "dense_hats", "dense_ragged", "rows_2048",
                                  "separable_hats_512", "dense_ragged_512"])
def test_one_warp_row_kernels_match_oracle(torch_cuda, case):
    """Row variant 2 (the plain row transforms by one-warp kernels for rows of 1024 or
    512 points, the forward windowed pass by row pairs) against the FP64 oracle, forward
    and adjoint, with separable and dense plans, windows whose column boxes wrap the
    seam or are ragged, an odd batch, and 2048-row plans; equal to the block row
    kernels (variant 1) up to rounding."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Plan
    rng = np.random.default_rng(95)
    if case == "separable_hats":
        wy, wx, w, h, u = sep_problem(1024, 1024, 4, 4, 3, 96, random_h=True)
        plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    elif case == "separable_hats_512":
        wy, wx, w, h, u = sep_problem(512, 512, 4, 4, 3, 94, random_h=True)
        plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    elif case == "dense_hats":
        pr = synth.problem_2d(128, 1024, 8, 3, 97, "normal")
        w, h, u = pr.w, pr.h, pr.u
        plan = Plan(dev(torch, w), h=dev(torch, h))
    elif case in ("dense_ragged", "dense_ragged_512"):
        # random windows on boxes of odd sizes, one wrapping both axes
        ny, nx, m = 64, (1024 if case == "dense_ragged" else 512), 3
        w = np.zeros((m, ny, nx), dtype=np.float32)
        boxes = [(5, 17, 1000, 77), (40, 31, 3, 511), (60, 9, 700, 1)] if nx == 1024 else \
            [(5, 17, 480, 77), (40, 31, 3, 255), (60, 9, 300, 1)]
        for k, (r0, nr, c0, nc) in enumerate(boxes):
            rr = (r0 + np.arange(nr)) % ny
            cc = (c0 + np.arange(nc)) % nx
            w[k][np.ix_(rr, cc)] = rng.uniform(0.2, 1.0, (nr, nc)).astype(np.float32)
        pr = synth.problem_2d(ny, nx, 4, 5, 98, "normal")
        h, u = pr.h[:m], pr.u
        plan = Plan(dev(torch, w), h=dev(torch, h))
    else:
        pr = synth.problem_2d(2048, 1024, 4, 1, 99, "normal")
        w, h, u = pr.w, pr.h, pr.u
        plan = Plan(dev(torch, w), h=dev(torch, h))
    ud = dev(torch, u)
    cv = plan.tuning()[1]
    plan.set_tuning(0, cv, 2)
    y2, x2 = host(plan.apply(ud)), host(plan.apply_adjoint(ud))
    assert rel(y2, C.apply(u, w, h)) < TOL
    assert rel(x2, C.apply_adjoint(u, w, h)) < TOL
    plan.set_tuning(0, cv, 1)
    assert rel(host(plan.apply(ud)), y2) < 2e-6
    assert rel(host(plan.apply_adjoint(ud)), x2) < 2e-6
    plan.close()


def test_slot_by_slot_schedule_in_batches_and_graphs(torch_cuda):
    """Column variant 4 (row and column pass per slot) inside a two-lane batch replayed
    as a graph, with a batch that needs two launches per direction: equal to the
    single-pass variant 2 up to rounding, and to the oracle."""
    torch = torch_cuda
    from paper_1604_04374_gb300 import Batch, Plan
    wy, wx, w, h, u = sep_problem(1024, 256, 4, 4, 5, 100, random_h=True)
    plan = Plan(wy=dev(torch, wy), wx=dev(torch, wx), h=dev(torch, h))
    ud = dev(torch, u)
    plan.set_tuning(3, 2, 1)
    y2, x2 = host(plan.apply(ud)), host(plan.apply_adjoint(ud))
    plan.set_tuning(3, 4, 1)
    y4, x4 = host(plan.apply(ud)), host(plan.apply_adjoint(ud))
    assert rel(y4, y2) < 2e-6 and rel(x4, x2) < 2e-6
    assert rel(y4, C.apply(u, w, h)) < TOL and rel(x4, C.apply_adjoint(u, w, h)) < TOL
    y, x = torch.empty_like(ud), torch.empty_like(ud)
    b = Batch([(plan, ud, y, False), (plan, ud, x, True)], lanes=2)
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    assert np.array_equal(host(y), y4) and np.array_equal(host(x), x4)
    b.close()
    plan.close()

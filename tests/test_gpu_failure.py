"""Failure detection without a GPU fault: a bounded wait that runs out.

The one-warp column kernels (columns of length 1024 and 512, whole-grid,
separable and sectioned) wait on an mbarrier for a bulk copy of a spectrum column.  With the copies suppressed
(pce_plan_inject_wait_timeout), every wait gives up after a short bounded
time, the kernels skip the dependent work, and the plan's status word turns
the event into PCE_ERR_TIMEOUT on the host.  Nothing hangs and the context
stays usable: after restoring normal operation the results are correct again.
"""
import numpy as np
import pytest

import synth
from oracle import expansion as E

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["whole_grid", "sectioned", "separable_tmem", "separable_tmem_pruned",
                                  "whole_grid_512", "separable_tmem_512"])
def test_bounded_wait_times_out_and_recovers(kind):
    """The whole-grid column kernels, the sectioned column kernel
    (PCE_FLAG_SECTIONED, whose spectrum columns also arrive by bulk copy) and
    the separable column kernels with tensor-memory state (column variants 2 and 3),
    at 1024 and 512 rows."""
    import torch
    from paper_1604_04374_gb300 import Plan, PceError, build, pce
    build.build()
    sectioned = kind == "sectioned"
    # 4 x 4 hats (m = 16): boxes of 511 rows, which a 1024-row section holds
    pruned = kind == "separable_tmem_pruned"
    m = 16 if (sectioned or pruned) else 4
    grid = (4, 4) if m == 16 else (2, 2)
    ny = 512 if kind.endswith("_512") else 1024
    pr = synth.problem_2d(ny, 64, m, 1, 41, "normal", grid)
    dev = torch.device("cuda", 0)
    if kind.startswith("separable_tmem"):
        wy, wx = synth.hat_factors_2d(ny, 64, *grid)
        plan = Plan(wy=torch.from_numpy(wy).to(dev), wx=torch.from_numpy(wx).to(dev),
                    h=torch.from_numpy(pr.h).to(dev))
        plan.set_tuning(0, 3 if pruned else 2, 0)
    else:
        plan = Plan(torch.from_numpy(pr.w).to(dev), h=torch.from_numpy(pr.h).to(dev),
                    flags=pce.PCE_FLAG_SECTIONED if sectioned else 0)
    u = torch.from_numpy(pr.u).to(dev)
    pce.pce_plan_status(plan.handle)                       # clean start
    pce.pce_plan_inject_wait_timeout(plan.handle, 200000)  # about 0.1 ms per wait
    plan.apply(u)
    plan.apply_adjoint(u)
    with pytest.raises(PceError) as e:
        pce.pce_plan_status(plan.handle)
    assert e.value.status == pce.PCE_ERR_TIMEOUT
    pce.pce_plan_status(plan.handle)                       # cleared by the previous read
    pce.pce_plan_inject_wait_timeout(plan.handle, 0)
    y = plan.apply(u).cpu().numpy().astype(np.float64)
    x = plan.apply_adjoint(u).cpu().numpy().astype(np.float64)
    pce.pce_plan_status(plan.handle)
    pts = np.stack([np.random.default_rng(1).integers(0, n, 200) for n in pr.shape], axis=-1)
    sel = (slice(None),) + tuple(pts.T)
    yr = E.apply_at(pr.u, pr.w, pr.h, pts)
    xr = E.apply_adjoint_at(pr.u, pr.w, pr.h, pts)
    assert np.linalg.norm(y[sel] - yr) / np.linalg.norm(yr) < 1e-5
    assert np.linalg.norm(x[sel] - xr) / np.linalg.norm(xr) < 1e-5
    plan.close()

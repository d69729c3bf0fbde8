"""The allocation-free single-box level-step against the regular one.

claw_level_step_noalloc keeps its scratch in a fixed device array instead of allocating, for
callers that cannot allocate device memory where they step.  Two calls in a row (the second
on another box size, so the shared scratch is rewritten) must match claw_level_step on the
same input within the one-step tolerance of the parity tests.  This file is collected last."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs

from gpu_helpers import lib_ready, rel_err, single_grid

pytestmark = pytest.mark.gpu
TOL1 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib_ready()


def _reference_and_noalloc(n, cellwise):
    import torch

    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run, q = single_grid(n)
    lev = run.levels[0]
    if cellwise:
        _, r2, k2 = inputs.config3(n)
        H = Hierarchy([run], [[q]], [[inputs.coef_pool(lev, r2, 1)]], [[inputs.coef_pool(lev, k2, 1)]])
    else:
        H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    qa = H.pool(0)
    claw.claw_fill_ghost(H.ctx, 0, qa)
    want = torch.zeros_like(qa)
    sm_ref = torch.zeros(1, dtype=torch.float64, device=qa.device)
    claw.claw_level_step(H.ctx, 0, qa, want, H.aux[0], H.dt, sm_ref)
    got = torch.zeros_like(qa)
    sm = torch.zeros(1, dtype=torch.float64, device=qa.device)
    claw.claw_level_step_noalloc(n, n, lev.dx, lev.dy, run.limiter, run.order, run.transverse, 1.0, 4.0, qa, got,
                                 H.aux[0], H.dt, sm)
    torch.cuda.synchronize()
    sl = slice(0, 3 * (n + 4) * (n + 4))
    a = got[sl].view(3, n + 4, n + 4)[:, 2:-2, 2:-2].cpu().numpy()
    b = want[sl].view(3, n + 4, n + 4)[:, 2:-2, 2:-2].cpu().numpy()
    H.close()
    return a, b, float(sm[0]), float(sm_ref[0])


def test_noalloc_step_matches_regular_step_two_calls_in_a_row():
    for n, cellwise in ((100, False), (64, True)):
        a, b, s, sref = _reference_and_noalloc(n, cellwise)
        assert rel_err(a, b) <= TOL1
        assert s == sref > 0.0


def test_noalloc_step_rejects_boxes_beyond_its_scratch():
    import torch

    from paper_1808_02638_gb300 import claw
    q = torch.zeros(8, dtype=torch.float64, device="cuda")
    dt = torch.ones(1, dtype=torch.float64, device="cuda")
    for nx, ny in ((4096, 4096), (4200, 64)):   # 16384 tiles > 16367; nx above 4096
        with pytest.raises(claw.ClawError) as e:
            claw.claw_level_step_noalloc(nx, ny, 1e-3, 1e-3, 4, 2, 2, 1.0, 4.0, q, q.clone(), None, dt, dt.clone())
        assert e.value.status == claw.CLAW_EINVAL

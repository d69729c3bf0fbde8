"""Failure detection on the GPU without a fault: a bounded device wait that is made to run out.

The staged level-step kernels wait on a shared-memory barrier for the bulk copy of each tile.
claw_set_wait_limit(ctx, 0) lets that first wait poll zero times, so every CTA gives up at its
first tile: it records CLAW_ETIMEOUT, waits (with the normal bound) for the copies it has issued,
and returns without writing.  The copies do land, so no wait runs without a limit and nothing is
left in flight.  The tests check the reported status, that no tile was written, that the fused
Eq. cfl epilogue kept its counter consistent, and that the next step with the normal bound matches
the oracle (one step: 1e-12 max|q|)."""
import numpy as np
import pytest
import torch

from paper_1808_02638_gb300 import inputs

from gpu_helpers import M, lib_ready, oracle_single, rel_err, single_grid

pytestmark = pytest.mark.gpu

TOL1 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib_ready()


def _step(H, polls, fused):
    """one level-step of level 0 from the current pool into the other (filled with NaN first)
    with the given first-wait bound; returns (status, destination pool)"""
    from paper_1808_02638_gb300 import claw
    src, dst = H.q[0][H.cur[0]], H.q[0][1 - H.cur[0]]
    claw.claw_set_wait_limit(H.ctx, polls)
    dst.fill_(float("nan"))
    if fused:   # the bench's launch: ghosts pulled from their sources, Eq. cfl on the last CTA
        claw.claw_level_advance(H.ctx, 0, src, dst, H.aux[0], H.dt, H.smax,
                                claw.CLAW_ADVANCE_PULL_GHOSTS | claw.CLAW_ADVANCE_UPDATE_DT)
    else:
        claw.claw_fill_ghost(H.ctx, 0, src)
        claw.claw_level_step(H.ctx, 0, src, dst, H.aux[0], H.dt, H.smax)
    return claw.claw_sync_status(H.ctx), dst


def _interiors(H, pool):
    lev = H.runs[0].levels[0]
    return [H.interior(0, 0, n, pool=pool) for n in range(len(lev.boxes))]


@pytest.mark.parametrize("medium", ["uniform", "cellwise"])
@pytest.mark.parametrize("tiling,fused", [((32, 16, 1), False), ((32, 16, 2), True), ((32, 16, 2), False),
                                          ((16, 16, 1), True)])
def test_expired_copy_wait_reports_timeout_and_next_step_matches_oracle(orc, medium, tiling, fused):
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 64
    boxes = [(0, 0, 32, 64), (32, 0, 32, 32), (32, 32, 32, 32)]
    run, q = single_grid(n, pulse=False, seed=41, boxes=boxes)
    lev = run.levels[0]
    if medium == "uniform":
        H = Hierarchy([run], [[q]], rho0=1.3, K0=2.7, tiling=tiling)
        rho = np.full((n + 4, n + 4), 1.3)
        K = np.full((n + 4, n + 4), 2.7)
    else:
        _, rho2, K2 = inputs.config3(n)
        H = Hierarchy([run], [[q]], [[inputs.coef_pool(lev, rho2, 1)]], [[inputs.coef_pool(lev, K2, 1)]],
                      tiling=tiling)
        rho = np.pad(rho2, M, mode="edge")
        K = np.pad(K2, M, mode="edge")
    dt = 0.25 * (2.0 / n) / float(np.sqrt(K / rho).max())
    H.dt.fill_(dt)
    H.smax.zero_()

    status, dst = _step(H, 0, fused)
    assert status == claw.CLAW_ETIMEOUT
    for got in _interiors(H, dst):
        assert np.isnan(got).all()            # every CTA stopped at its first tile
    assert float(H.dt[0]) == dt               # no speed was published, dt kept
    assert float(H.smax[0]) == 0.0

    status, dst = _step(H, 1 << 22, fused)
    assert status == claw.CLAW_OK
    single = np.zeros((3, n + 4, n + 4))
    for k, (i0, j0, bx, by) in enumerate(boxes):
        single[:, M + j0:M + j0 + by, M + i0:M + i0 + bx] = \
            inputs.box_view(q, lev.qoff[k], bx, by, 3)[:, M:-M, M:-M]
    srun, sq = single_grid(n, pulse=False, seed=41)
    inputs.box_view(sq, 0, n, n, 3)[:] = single
    want, _ = oracle_single(orc, srun, sq, rho, K, 1, dt=dt)
    got = _interiors(H, dst)
    err = max(np.abs(got[k] - want[:, j0:j0 + by, i0:i0 + bx]).max() for k, (i0, j0, bx, by) in enumerate(boxes))
    assert err <= TOL1 * np.abs(want).max()
    if fused:   # the epilogue ran on both launches: the second set dt from the step's speeds
        assert float(H.dt[0]) == pytest.approx(0.9 * (2.0 / n) / float(np.sqrt(K / rho)[1:-1, 1:-1].max()),
                                               rel=1e-15)
    torch.cuda.synchronize()


def test_expired_copy_wait_shallow_water(orc):
    # the shallow-water kernel shares the staging skeleton and its bounded waits
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    from oracle.amr import OracleHierarchy
    n = 64
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = [inputs.Level(n, n, 2.0 / n, 2.0 / n, [(0, 0, n, n)])]
    lev = run.levels[0]
    q = np.zeros(lev.qsize)
    v = inputs.box_view(q, 0, n, n, 3)
    u = inputs.uniform(77, v.size).reshape(v.shape)
    v[0], v[1], v[2] = 0.5 + u[0], u[1] - 0.5, u[2] - 0.5
    H = Hierarchy([run], [[q]], tiling=(16, 16, 1), system="shallow_water", grav=1.0)
    H.dt.fill_(0.005)
    status, dst = _step(H, 0, False)
    assert status == claw.CLAW_ETIMEOUT
    assert np.isnan(H.interior(0, 0, 0, pool=dst)).all()
    status, dst = _step(H, 1 << 22, False)
    assert status == claw.CLAW_OK
    O = OracleHierarchy(run, [q], system="shallow_water", grav=1.0)
    O.coarse_step(dt=0.005)
    want = O.interior(0, 0)
    assert rel_err(H.interior(0, 0, 0, pool=dst), want) <= TOL1

"""Host logic of the subcycling (Sec. 2.2; no GPU): the order of a coarse step's launches, and
where each fine substep's interpolated ghosts come from.  The hierarchy's library calls are
recorded by a stand-in; a model of the pools follows what each call writes, so that every fine
substep is checked to find, in the pool it reads, interpolated ghosts written once for it: at its
own time fraction k / r, from the coarser level's states at the start and end of the coarser step
it belongs to."""
import types

import pytest

from paper_1808_02638_gb300 import solver
from paper_1808_02638_gb300.solver import Hierarchy


class Pool:
    def __init__(self, level, index):
        self.level, self.index = level, index
        self.state = (level, 0)   # (level, substeps taken into this pool so far)
        self.ghosts = None        # what the pool's interpolated ghost cells were filled from

    def __repr__(self):
        return f"Pool(L{self.level}.{self.index})"


class Recorder:
    """the library calls of solver.advance, recorded against the pool model"""

    def __init__(self):
        self.calls = []
        self.steps = 0
        self.CLAW_ADVANCE_PULL_GHOSTS = 4

    def _fill(self, level, q, cold, cnew, tau):
        assert q.level == level
        q.ghosts = (cold.state, cnew.state, tau)

    def claw_fill_ghost_interp(self, ctx, level, q, cold, cnew, tau, stream=None):
        if level == 0:   # no coarser level: nothing to fill (the library returns at once)
            assert cold is None and cnew is None
            return
        self.calls.append(("fill", level, tau))
        self._fill(level, q, cold, cnew, tau)

    def claw_level_advance_fill(self, ctx, level, q_old, q_new, aux, dt, smax, flags, jobs=(), stream=None):
        self.calls.append(("step", level, tuple((j[0], j[4]) for j in jobs)))
        assert flags == self.CLAW_ADVANCE_PULL_GHOSTS
        self.seen.append((level, q_old.state, q_old.ghosts))
        # the step's reads come first (the jobs write only cells no tile reads)
        for lev, q, cold, cnew, tau in jobs:
            assert q is not q_old and cold is not q_new and cnew is not q_new
        q_new.state = (level, q_old.state[1] + 1)
        q_new.ghosts = None   # a step writes interiors only; stale ghosts are not this substep's
        for lev, q, cold, cnew, tau in jobs:
            self._fill(lev, q, cold, cnew, tau)

    def claw_average_down(self, ctx, fine_level, qf, qc, stream=None):
        self.calls.append(("average", fine_level))


def _hierarchy(nlev, ratio, fill_ahead):
    H = Hierarchy.__new__(Hierarchy)
    H.nlev = nlev
    H.q = [[Pool(L, 0), Pool(L, 1)] for L in range(nlev)]
    H.cur = [0] * nlev
    H.aux = [None] * nlev
    H.ctx = H.dt = H.smax = None
    H.sections = None
    H.pull, H.reflux, H.patchwise = True, False, False
    H.pull_levels = [True] * nlev
    H.fuse_interp = [False] * nlev
    H.fill_ahead = fill_ahead
    H.runs = [types.SimpleNamespace(levels=[types.SimpleNamespace(ratio=1 if L == 0 else ratio)
                                            for L in range(nlev)])]
    return H


@pytest.mark.parametrize("fill_ahead", [True, False])
@pytest.mark.parametrize("nlev,ratio", [(2, 2), (3, 4), (4, 2)])
def test_every_fine_substep_reads_ghosts_filled_for_its_own_time(monkeypatch, fill_ahead, nlev, ratio):
    rec = Recorder()
    rec.seen = []
    monkeypatch.setattr(solver, "claw", rec)
    H = _hierarchy(nlev, ratio, fill_ahead)
    for coarse in range(2):
        rec.seen = []
        H.advance(0)
        # level L takes ratio^L substeps; substep k of a level L >= 1 reads its pool after k of
        # its steps in this coarser step, and finds the coarser level's states around the
        # coarser step it belongs to at time fraction (k mod r) / r
        per_level = {L: [s for s in rec.seen if s[0] == L] for L in range(nlev)}
        for L in range(nlev):
            assert len(per_level[L]) == ratio ** L
        for L in range(1, nlev):
            for n, (_, state, ghosts) in enumerate(per_level[L]):
                parent_step = n // ratio          # the coarser level's substep this one belongs to
                k = n % ratio
                base = coarse * ratio ** (L - 1)  # coarser-level steps before this coarse step
                old = (L - 1, (base + parent_step) if L > 1 else coarse)
                new = (L - 1, old[1] + 1)
                assert ghosts is not None, (L, n)
                c_old, c_new, tau = ghosts
                assert tau == k / ratio
                assert c_old == old
                # at tau = 0 the one-launch-ahead fill reads only the coarse old state
                assert c_new == (old if (fill_ahead and k == 0) else new)
    nsteps = sum(ratio ** L for L in range(nlev))
    fills = [c for c in rec.calls if c[0] == "fill"]
    steps = [c for c in rec.calls if c[0] == "step"]
    assert len(steps) == 2 * nsteps
    assert len(fills) == (0 if fill_ahead else 2 * (nsteps - 1))
    assert len([c for c in rec.calls if c[0] == "average"]) == 2 * sum(ratio ** L for L in range(nlev - 1))
    if fill_ahead:   # every fine substep's fill rides on exactly one step launch
        jobs = [j for c in steps for j in c[2]]
        assert len(jobs) == 2 * (nsteps - 1)
        assert all(len(c[2]) <= 2 for c in steps)


def test_a_level_with_its_own_evaluation_gets_no_fill_ahead(monkeypatch):
    # a level whose step evaluates its interpolated ghosts itself (pull+interp) takes no job from
    # the coarser level, and the coarser level's launch carries none for it
    rec = Recorder()
    rec.seen = []
    calls = []
    rec.claw_level_advance_interp = lambda ctx, L, *a, **k: calls.append(L)
    monkeypatch.setattr(solver, "claw", rec)
    H = _hierarchy(3, 2, True)
    H.fuse_interp = [False, False, True]
    H.q[2][0].state = H.q[2][1].state = (2, 0)
    H.advance(0)
    assert calls == [2] * 4
    for c in rec.calls:
        if c[0] == "step":
            assert all(lev != 2 for lev, _ in c[2]), c

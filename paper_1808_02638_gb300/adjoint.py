"""Differentiable rollouts: gradients of a functional of the final state with respect to the
initial state and the medium (rho, K), through the hand-written adjoint kernels.

`LevelStep.apply(H, L, dt, q_old, rho, K)` is one level-step of level L as a differentiable map.
`rollout(H, q0, rho, K, ncoarse, every)` is a torch.autograd.Function over `ncoarse` coarse
steps of hierarchy H (any number of levels and runs).  The forward keeps a checkpoint of every
level's state every `every` coarse steps; the backward recomputes one segment at a time from its
checkpoint (recording each level-step's input state and the pre-average coarse state, or, for a
cell-wise medium, each level-step's tape of intermediates); the last segment, the first to be
reversed, is recorded by the forward itself when the steps can record.  With
`every=None` the forward records that tape for the whole rollout instead (memory: every
level-step's input pool and every pre-average coarse pool, kept in HBM) and the backward
recomputes nothing.  Either way the backward runs the reverse of the AMR time step of Sec. 2.2
on the device:

  average (Sec. 2.3)        -> claw_average_down_adjoint
  fine substeps, last first -> claw_level_advance_adjoint + claw_fill_ghost_interp_adjoint (the
                               interpolation adjoint feeds the coarse old / new states)
  coarse level-step         -> claw_level_advance_adjoint + claw_fill_ghost_interp_adjoint

with the time steps frozen at their forward values.  The step adjoint routes the adjoint of
every same-level and boundary ghost to its source cell itself (H.pull, the default; with
H.pull = False: claw_level_step_adjoint + claw_fill_ghost_adjoint, the same map).  The medium
gradients leave through claw_medium_aux_adjoint and claw_fill_ghost_coef_adjoint.  This module
only sequences calls: every arithmetic operation of the gradient runs in libclaw.so.
"""
from __future__ import annotations

import torch

from . import claw


class _Node:
    __slots__ = ("L", "q_in", "cold", "cnew", "tau", "pre_avg", "fine")

    def __init__(self, L, q_in, cold, cnew, tau):
        self.L, self.q_in, self.cold, self.cnew, self.tau = L, q_in, cold, cnew, tau
        self.pre_avg = None
        self.fine = []


def _advance_record(H, L, cold, cnew, tau):
    """one level-step of level L (and its finer substeps), recording what the reverse needs"""
    q = H.q[L][H.cur[L]]
    claw.claw_fill_ghost(H.ctx, L, q, cold, cnew, tau)
    node = _Node(L, q.clone(), cold, cnew, tau)
    H.step_level(L)
    new = H.q[L][1 - H.cur[L]]
    if L + 1 < H.nlev:
        node.pre_avg = new.clone()
        r = H.ratio(L + 1)
        for k in range(r):
            node.fine.append(_advance_record(H, L + 1, node.q_in, node.pre_avg, k / r))
        claw.claw_average_down(H.ctx, L + 1, H.q[L + 1][H.cur[L + 1]], new)
    H.cur[L] ^= 1
    return node


def _reverse(H, node, lam, g_aux, lam_cold=None, lam_cnew=None):
    """adjoint of `node` (one level-step of level node.L with its substeps).  lam[L] holds the
    adjoint of each level's state after the node and is replaced by the adjoint of the state
    before it; the interpolation adjoints of node.L's ghost fill go to lam_cold / lam_cnew (the
    coarser level's old and pre-average new states)."""
    L = node.L
    lam_pre = lam[L]
    lam_in = torch.zeros_like(lam_pre)
    if node.fine:
        # averaging: covered coarse adjoints move to the fine state and are zeroed
        claw.claw_average_down_adjoint(H.ctx, L + 1, lam[L + 1], lam_pre)
        for fnode in reversed(node.fine):
            _reverse(H, fnode, lam, g_aux, lam_cold=lam_in, lam_cnew=lam_pre)
    if H.pull:   # the ghost-copy adjoint fused into the step adjoint; the interpolation's apart
        claw.claw_level_advance_adjoint(H.ctx, L, node.q_in, lam_pre, lam_in, H.aux[L], g_aux[L], H.dt,
                                        claw.CLAW_ADVANCE_PULL_GHOSTS)
        claw.claw_fill_ghost_interp_adjoint(H.ctx, L, lam_in, lam_cold, lam_cnew, node.cold, node.cnew, node.tau)
    else:
        claw.claw_level_step_adjoint(H.ctx, L, node.q_in, lam_pre, lam_in, H.aux[L], g_aux[L], H.dt)
        claw.claw_fill_ghost_adjoint(H.ctx, L, lam_in, lam_cold, lam_cnew, node.cold, node.cnew, node.tau)
    lam[L] = lam_in


def _records_ok(H):
    """whether the reverse can run from recorded step tapes (claw_level_advance_record): a
    cell-wise medium and second order"""
    return H.medium == 1 and all(r.order == 2 for r in H.runs)


class _Tape:
    """Device buffers of the level-steps of `ncoarse` coarse steps, kept per level in time
    order: state(L, i) is the input of the i-th step of level L in the segment and
    state(L, N_L) the level's state after the last one; pre[L][i] is what the i-th step of a
    level with a finer one wrote before the finer level's average went into it (the coarse
    "new" state of the space-time interpolation); dt[k] is the time step of coarse step k.
    With `record`, rec[L][i] receives the i-th step's intermediates (claw_level_advance_record),
    the reverse reads those instead of the states, and the finest level's states (which only
    its own next step reads) live in two buffers.  The recording steps use the tape's own dtw and
    smaxw; the reverse sweep reads the tape and sets the hierarchy's dt.  A segment's recompute
    and its reverse only ever touch these buffers (and the medium planes and the adjoint
    buffers), so one CUDA graph replays any segment."""

    def __init__(self, H, ncoarse, record=False):
        self.n = ncoarse
        self.record = record
        counts = [ncoarse]
        for L in range(1, H.nlev):
            counts.append(counts[-1] * H.ratio(L))
        self.counts = counts
        nstate = [2 if record and L + 1 == H.nlev else counts[L] + 1 for L in range(H.nlev)]
        self.states = [[torch.zeros_like(H.q[L][0]) for _ in range(nstate[L])] for L in range(H.nlev)]
        self.pre = [[torch.zeros_like(H.q[L][0]) for _ in range(counts[L])] if L + 1 < H.nlev else []
                    for L in range(H.nlev)]
        self.rec = [[torch.empty_like(H.aux[L]) for _ in range(counts[L])] if record else []
                    for L in range(H.nlev)]
        self.dt = torch.zeros((ncoarse, H.nruns), dtype=torch.float64, device=H.dev)
        # the recording steps' own time step and speed maximum, so that a recompute can run
        # beside a reverse sweep (which sets the hierarchy's dt) on another stream
        self.dtw = torch.zeros(H.nruns, dtype=torch.float64, device=H.dev)
        self.smaxw = torch.zeros(H.nruns, dtype=torch.float64, device=H.dev)

    def state(self, L, i):
        return self.states[L][i % len(self.states[L])]


def _record(H, T, L, i, cold=None, cnew=None, tau=0.0):
    """the i-th step of level L of the tape (and its finer substeps), with the launches of
    Hierarchy.advance: the interpolated ghosts filled, the others pulled by the step (or, on a
    level the autotuner keeps on the copy launch, all filled); time step T.dtw, speeds into
    T.smaxw"""
    q = T.state(L, i)
    dt, smax = T.dtw, T.smaxw
    fine = L + 1 < H.nlev
    dst = T.pre[L][i] if fine else T.state(L, i + 1)
    if T.record:   # the level's own ghost launch choice, as in the forward
        if H.pull_levels[L]:
            if L:
                claw.claw_fill_ghost_interp(H.ctx, L, q, cold, cnew, tau)
            claw.claw_level_advance_record(H.ctx, L, q, dst, H.aux[L], dt, smax, claw.CLAW_ADVANCE_PULL_GHOSTS,
                                           T.rec[L][i])
        else:
            claw.claw_fill_ghost(H.ctx, L, q, cold, cnew, tau)
            claw.claw_level_advance_record(H.ctx, L, q, dst, H.aux[L], dt, smax, 0, T.rec[L][i])
    elif H.pull_levels[L]:
        if L:
            claw.claw_fill_ghost_interp(H.ctx, L, q, cold, cnew, tau)
        claw.claw_level_advance(H.ctx, L, q, dst, H.aux[L], dt, smax, claw.CLAW_ADVANCE_PULL_GHOSTS)
    else:
        claw.claw_fill_ghost(H.ctx, L, q, cold, cnew, tau)
        claw.claw_level_step(H.ctx, L, q, dst, H.aux[L], dt, smax)
    if fine:
        r = H.ratio(L + 1)
        for k in range(r):
            _record(H, T, L + 1, i * r + k, q, dst, k / r)
        nxt = T.state(L, i + 1)
        nxt.copy_(dst)
        claw.claw_average_down(H.ctx, L + 1, T.state(L + 1, (i + 1) * r), nxt)


def _record_coarse(H, T, k, frozen):
    T.dt[k].copy_(T.dtw)
    _record(H, T, 0, k)
    if frozen:
        T.smaxw.zero_()
    else:
        claw.claw_dt_update(H.ctx, 0, T.smaxw, T.dtw)


def _reverse_tape(H, T, L, i, lam, lbuf, g_aux, lam_cold=None, lam_cnew=None, tau=0.0, cold=None, cnew=None):
    """adjoint of the i-th step of level L of the tape (and its substeps): lam[L] holds the
    adjoint of the level's state after the step and becomes that of the state before it, in the
    other buffer of lbuf[L]; the interpolation adjoint of the step's ghosts goes to lam_cold /
    lam_cnew (the coarser level's old and pre-average new states)."""
    lam_pre = lam[L]
    lam_in = lbuf[L][1] if lam_pre is lbuf[L][0] else lbuf[L][0]
    lam_in.zero_()
    q = T.state(L, i)
    if L + 1 < H.nlev:
        r = H.ratio(L + 1)
        # averaging: covered coarse adjoints move to the fine state and are zeroed
        claw.claw_average_down_adjoint(H.ctx, L + 1, lam[L + 1], lam_pre)
        for k in reversed(range(r)):
            _reverse_tape(H, T, L + 1, i * r + k, lam, lbuf, g_aux, lam_in, lam_pre, k / r, q, T.pre[L][i])
    if T.record:
        claw.claw_level_advance_adjoint_tape(H.ctx, L, T.rec[L][i], lam_pre, lam_in, H.aux[L], g_aux[L], H.dt,
                                             claw.CLAW_ADVANCE_PULL_GHOSTS)
    else:
        claw.claw_level_advance_adjoint(H.ctx, L, q, lam_pre, lam_in, H.aux[L], g_aux[L], H.dt,
                                        claw.CLAW_ADVANCE_PULL_GHOSTS)
    if L:
        claw.claw_fill_ghost_interp_adjoint(H.ctx, L, lam_in, lam_cold, lam_cnew, cold, cnew, tau)
    lam[L] = lam_in


def _reverse_coarse(H, T, k, lam, lbuf, g_aux):
    H.dt.copy_(T.dt[k])   # frozen forward time step
    _reverse_tape(H, T, 0, k, lam, lbuf, g_aux)


def _replayable(H, key, body):
    """a CUDA graph of body() cached on the hierarchy under `key` (the hierarchy drops its graphs
    when its levels or tilings change); body runs once eagerly before the capture (first-use
    tables and kernel attributes)"""
    cache = H.__dict__.setdefault("_graphs", {})
    if key not in cache:
        body()
        s = torch.cuda.Stream(device=H.dev)
        s.wait_stream(torch.cuda.current_stream(H.dev))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            body()
        torch.cuda.current_stream(H.dev).wait_stream(s)
        cache[key] = g
    return cache[key]


def _buffers(H, key, make):
    cache = H.__dict__.setdefault("_graph_buffers", {})
    if key not in cache:
        cache[key] = make()
    return cache[key]


def _segment_tape(H, n, rec, s):
    """the tape of checkpoint segment s (n coarse steps): two per length, by segment parity, so
    that one segment can be recomputed while the next is reversed"""
    return _buffers(H, ("tape", n, rec, s % 2), lambda: _Tape(H, n, record=rec))


def _load_segment(H, T, states, dt0):
    """a segment's starting states and recording time step into its tape (which then holds no
    rollout's recorded segment: T.owner is set by the forward that records one)"""
    T.owner = None
    for L in range(H.nlev):
        T.state(L, 0).copy_(states[L])
    T.dtw.copy_(dt0)
    T.smaxw.zero_()


def _record_segment(H, T, n, frozen, s, graphs, reload):
    """the recording steps of a segment into its tape (the cached graph of the segment's length,
    parity and dt mode); reload() puts the starting state back after the graph's eager first run"""
    def body():
        for k in range(n):
            _record_coarse(H, T, k, frozen)
    _run(H, ("bwd-first", n, frozen, True, s % 2), body, graphs, lambda: reload)


def _forward_segment(H, n, graphs):
    """n coarse steps of the hierarchy (a CUDA graph when `graphs`); every level's state ends in
    the buffer it started in"""
    cur0 = list(H.cur)

    def body():
        for _ in range(n):
            H.coarse_step()
        for L in range(H.nlev):
            if H.cur[L] != cur0[L]:
                H.q[L][cur0[L]].copy_(H.q[L][H.cur[L]])
                H.cur[L] = cur0[L]

    if not graphs:
        body()
        return
    key = ("fwd", n, H.freeze_dt, tuple(cur0))
    if key in H.__dict__.get("_graphs", {}):
        H._graphs[key].replay()
        return
    state = [[a.clone() for a in p] for p in H.q], H.dt.clone(), H.smax.clone()
    g = _replayable(H, key, body)   # ran the body twice (eager and captured): put the state back
    for L in range(H.nlev):
        for b in range(2):
            H.q[L][b].copy_(state[0][L][b])
    H.dt.copy_(state[1])
    H.smax.copy_(state[2])
    g.replay()


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, ncoarse, every, nlev, dt, graphs, records, *tensors):
        q0 = tensors[:nlev]
        rho = tensors[nlev:2 * nlev] if H.medium else [None] * nlev
        K = tensors[2 * nlev:3 * nlev] if H.medium else [None] * nlev
        with torch.no_grad():
            for L in range(nlev):
                H.cur[L] = 0
                H.q[L][0].copy_(q0[L])
                if H.medium:
                    H.rho[L].copy_(rho[L])
                    H.K[L].copy_(K[L])
                    claw.claw_fill_ghost_coef(H.ctx, L, H.rho[L])
                    claw.claw_fill_ghost_coef(H.ctx, L, H.K[L])
                    claw.claw_medium_aux(H.ctx, L, H.rho[L], H.K[L], H.aux[L])
            if dt is None:
                H.freeze_dt = False
                H.init_dt()
            else:   # time steps frozen at the caller's values (e.g. for finite differences)
                H.freeze_dt = True
                H.dt.copy_(dt)
            frozen = H.freeze_dt
            checkpoints, tapes, tape = [], None, None
            if every is None and not H.pull:   # the whole tape, recorded as the rollout runs
                tapes = []
                for n in range(ncoarse):
                    dt_n = H.dt.clone()
                    tapes.append((_advance_record(H, 0, None, None, 0.0), dt_n))
                    if H.freeze_dt:
                        H.smax.zero_()
                    else:
                        claw.claw_dt_update(H.ctx, 0, H.smax, H.dt)
            elif every is None:   # the whole rollout as one tape, recorded as it runs
                tape = _Tape(H, ncoarse)
                for L in range(nlev):
                    tape.state(L, 0).copy_(H.q[L][H.cur[L]])
                tape.dtw.copy_(H.dt)
                tape.smaxw.copy_(H.smax)
                for k in range(ncoarse):
                    _record_coarse(H, tape, k, frozen)
                for L in range(nlev):
                    H.q[L][H.cur[L]].copy_(tape.state(L, tape.counts[L]))
                H.dt.copy_(tape.dtw)
                H.smax.copy_(tape.smaxw)
            else:
                # the last segment is the first one the backward reverses: with recording steps
                # it is recorded into its tape now (a recording step costs about as much as a
                # plain one), instead of being recomputed there before anything else can run
                rec_last = H.pull and records and _records_ok(H)
                nseg = (ncoarse + every - 1) // every
                for s, s0 in enumerate(range(0, ncoarse, every)):
                    n = min(every, ncoarse - s0)
                    checkpoints.append(([H.q[L][H.cur[L]].clone() for L in range(nlev)], H.dt.clone()))
                    if rec_last and s == nseg - 1:
                        T = _segment_tape(H, n, True, s)
                        start = checkpoints[-1]
                        _load_segment(H, T, *start)
                        _record_segment(H, T, n, frozen, s, graphs, lambda: _load_segment(H, T, *start))
                        for L in range(nlev):
                            H.q[L][H.cur[L]].copy_(T.state(L, T.counts[L]))
                        H.dt.copy_(T.dtw)
                        H.smax.copy_(T.smaxw)
                        T.owner = ctx
                    elif H.pull:
                        _forward_segment(H, n, graphs)
                    else:
                        for _ in range(n):
                            H.coarse_step()
            out = [H.q[L][H.cur[L]].clone() for L in range(nlev)]
        ctx.H, ctx.ncoarse, ctx.every, ctx.nlev = H, ncoarse, every, nlev
        ctx.checkpoints = checkpoints
        ctx.tapes = tapes
        ctx.tape = tape
        ctx.frozen = frozen
        ctx.graphs = graphs
        ctx.records = records
        H.freeze_dt = False
        return tuple(out)

    @staticmethod
    def backward(ctx, *grads):
        H, nlev, every, ncoarse = ctx.H, ctx.nlev, ctx.every, ctx.ncoarse
        if not H.pull:
            g_aux = [torch.zeros_like(H.aux[L]) if H.medium else None for L in range(nlev)]
            lam = [g.clone() if g is not None else torch.zeros_like(H.q[L][0]) for L, g in enumerate(grads)]
            _backward_filled(ctx, H, lam, g_aux)
        else:
            # the adjoint and medium-adjoint buffers are the hierarchy's, so that the graphs of
            # the reverse sweep can be replayed by later gradients
            g_aux = _buffers(H, "g_aux", lambda: [torch.zeros_like(H.aux[L]) if H.medium else None
                                                  for L in range(nlev)])
            for g in g_aux:
                if g is not None:
                    g.zero_()
            lbuf = _buffers(H, "lam", lambda: [(torch.zeros_like(H.q[L][0]), torch.zeros_like(H.q[L][0]))
                                                for L in range(nlev)])
            for L, g in enumerate(grads):
                if g is None:
                    lbuf[L][0].zero_()
                else:
                    lbuf[L][0].copy_(g)
            if ctx.tape is not None:   # the recorded tape: reverse only
                T = ctx.tape
                lam = [lbuf[L][0] for L in range(nlev)]
                for k in reversed(range(T.n)):
                    _reverse_coarse(H, T, k, lam, lbuf, g_aux)
                ctx.tape = None
            else:
                lam = _backward_segments(ctx, H, lbuf, g_aux)
        grads_out = [None, None, None, None, None, None, None] + [l.clone() for l in lam]
        if H.medium:
            g_rho, g_K = [], []
            for L in range(nlev):
                gr = torch.zeros_like(H.rho[L])
                gk = torch.zeros_like(H.K[L])
                claw.claw_medium_aux_adjoint(H.ctx, L, H.rho[L], H.K[L], g_aux[L], gr, gk)
                claw.claw_fill_ghost_coef_adjoint(H.ctx, L, gr)
                claw.claw_fill_ghost_coef_adjoint(H.ctx, L, gk)
                g_rho.append(gr)
                g_K.append(gk)
            grads_out += g_rho + g_K
        return tuple(grads_out)


def _run(H, key, body, graphs, undo_first):
    """body() as a cached CUDA graph (or eagerly): on first use it runs eagerly once and is
    captured, and undo_first() then puts back the inputs that eager run changed"""
    if not graphs:
        body()
        return
    if key not in H.__dict__.get("_graphs", {}):
        undo = undo_first()
        _replayable(H, key, body)
        undo()
    H._graphs[key].replay()


def _backward_segments(ctx, H, lbuf, g_aux):
    """reverse sweep over the checkpoint segments, last first.  Segment s is reversed from its
    tape while segment s-1 is recomputed from its checkpoint into the other tape on a second
    stream (the two touch disjoint buffers: the recompute has its own dt and speed maximum), so
    the recompute of all but the last segment overlaps with the reverse sweep.  With ctx.graphs
    each such pair is one cached CUDA graph per (segment lengths, tape slot)."""
    nlev, every, ncoarse = ctx.nlev, ctx.every, ctx.ncoarse
    rec = ctx.records and _records_ok(H)
    nseg = len(ctx.checkpoints)
    lens = [min(every, ncoarse - s * every) for s in range(nseg)]
    side = _buffers(H, "side_stream", lambda: torch.cuda.Stream(device=H.dev))

    def tape(s):
        return _segment_tape(H, lens[s], rec, s)

    def load(s):   # eager: checkpoint s into its tape's first states and recording time step
        _load_segment(H, tape(s), *ctx.checkpoints[s])

    def recompute(s):
        T = tape(s)
        for k in range(lens[s]):
            _record_coarse(H, T, k, ctx.frozen)

    def reverse(s):
        T = tape(s)
        lam = [lbuf[L][0] for L in range(nlev)]
        for k in reversed(range(lens[s])):
            _reverse_coarse(H, T, k, lam, lbuf, g_aux)
        for L in range(nlev):   # the adjoint leaves in the buffer it came in
            if lam[L] is not lbuf[L][0]:
                lbuf[L][0].copy_(lam[L])

    last = nseg - 1
    if getattr(tape(last), "owner", None) is not ctx:   # not recorded by this rollout's forward
        load(last)
        _run(H, ("bwd-first", lens[last], ctx.frozen, rec, last % 2), lambda: recompute(last), ctx.graphs,
             lambda: (lambda: load(last)))
    tape(last).owner = None
    for s in reversed(range(nseg)):
        if s:
            load(s - 1)

        def body(s=s):
            main = torch.cuda.current_stream(H.dev)
            if s:
                side.wait_stream(main)
                with torch.cuda.stream(side):
                    recompute(s - 1)
            reverse(s)
            if s:
                main.wait_stream(side)

        def undo_first(s=s):
            saved = [l[0].clone() for l in lbuf], [g.clone() if g is not None else None for g in g_aux]

            def undo():
                for L in range(nlev):
                    lbuf[L][0].copy_(saved[0][L])
                    if g_aux[L] is not None:
                        g_aux[L].copy_(saved[1][L])
                if s:
                    load(s - 1)
            return undo

        key = ("bwd", lens[s], lens[s - 1] if s else 0, ctx.frozen, rec, s % 2)
        _run(H, key, body, ctx.graphs, undo_first)
    return [lbuf[L][0] for L in range(nlev)]


def _backward_filled(ctx, H, lam, g_aux):
    """the reverse sweep with every ghost filled before each step (H.pull = False)"""
    nlev, every, ncoarse = ctx.nlev, ctx.every, ctx.ncoarse
    if ctx.tapes is not None:
        for node, dt in reversed(ctx.tapes):
            H.dt.copy_(dt)   # frozen forward time step
            _reverse(H, node, lam, g_aux)
        ctx.tapes = None
    nseg = len(ctx.checkpoints)
    for s in reversed(range(nseg)):
        states, dt0 = ctx.checkpoints[s]
        n0, n1 = s * every, min((s + 1) * every, ncoarse)
        # recompute the segment, recording each coarse step
        for L in range(nlev):
            H.cur[L] = 0
            H.q[L][0].copy_(states[L])
        H.dt.copy_(dt0)
        tapes = []
        for _ in range(n0, n1):
            dt = H.dt.clone()
            tapes.append((_advance_record(H, 0, None, None, 0.0), dt))
            if ctx.frozen:
                H.smax.zero_()
            else:
                claw.claw_dt_update(H.ctx, 0, H.smax, H.dt)
        for node, dt in reversed(tapes):
            H.dt.copy_(dt)   # frozen forward time step
            _reverse(H, node, lam, g_aux)
    return lam


def _ghost_mask(H, L):
    """1.0 on the ghost cells of every box of level L (all planes), 0.0 on interiors and padding"""
    cache = H.__dict__.setdefault("_ghost_masks", {})
    if L not in cache:
        import numpy as np
        m = np.zeros(H.q[L][0].numel())
        for (ri, qb, _) in H.layout[L]:
            lev = H.runs[ri].levels[L]
            for n, b in enumerate(lev.boxes):
                nx, ny = int(b[2]), int(b[3])
                off = qb + int(lev.qoff[n])
                v = m[off:off + 3 * (nx + 4) * (ny + 4)].reshape(3, ny + 4, nx + 4)
                v[...] = 1.0
                v[:, 2:2 + ny, 2:2 + nx] = 0.0
        cache[L] = torch.from_numpy(m).to(H.q[L][0].device)
    return cache[L]


class LevelStep(torch.autograd.Function):
    """One level-step of level L of hierarchy H (Eq. wave_form_2d_2nd_order on every box) as a
    differentiable map (q_old, rho, K) -> q_new with the time step frozen.

    q_old: a q pool of level L with its ghosts filled by the caller; q_new equals q_old on the
    ghost cells and the stepped values on the interiors.  rho, K (cell-wise medium only): the
    level's coefficient pools, ghosts included (treated as independent inputs).  dt: device
    tensor of per-run level-0 time steps.  The backward runs claw_level_step_adjoint (and
    claw_medium_aux_adjoint for rho, K); ghost cells of q_new pass their adjoint straight back."""

    @staticmethod
    def forward(ctx, H, L, dt, q_old, rho=None, K=None):
        aux = None
        if H.medium:
            aux = torch.zeros_like(H.aux[L])
            claw.claw_medium_aux(H.ctx, L, rho, K, aux)
        q_new = q_old.detach().clone()
        smax = torch.zeros_like(H.smax)
        claw.claw_level_step(H.ctx, L, q_old.detach(), q_new, aux, dt, smax)
        ctx.H, ctx.L = H, L
        ctx.save_for_backward(q_old.detach(), dt, aux if aux is not None else torch.empty(0),
                              rho.detach() if rho is not None else torch.empty(0),
                              K.detach() if K is not None else torch.empty(0))
        return q_new

    @staticmethod
    def backward(ctx, lam_new):
        H, L = ctx.H, ctx.L
        q_old, dt, aux, rho, K = ctx.saved_tensors
        lam_new = lam_new.contiguous()
        lam_old = lam_new * _ghost_mask(H, L)
        g_rho = g_K = None
        if H.medium:
            g_aux = torch.zeros_like(aux)
            claw.claw_level_step_adjoint(H.ctx, L, q_old, lam_new, lam_old, aux, g_aux, dt)
            g_rho, g_K = torch.zeros_like(rho), torch.zeros_like(K)
            claw.claw_medium_aux_adjoint(H.ctx, L, rho, K, g_aux, g_rho, g_K)
        else:
            claw.claw_level_step_adjoint(H.ctx, L, q_old, lam_new, lam_old, None, None, dt)
        return None, None, None, lam_old, g_rho, g_K


def rollout(H, q0, rho=None, K=None, ncoarse=1, every=20, dt=None, graphs=True, records=True):
    """final states (one pool per level) after `ncoarse` coarse steps from q0 (pools per level),
    differentiable with respect to q0 and, for a cell-wise medium, the rho and K pools.
    every: checkpoint interval of the recomputing backward, or None for the recorded tape.
    dt: None for Eq. cfl time steps, else a device tensor of per-run level-0 time steps used
    unchanged for every coarse step.  The gradient holds the time steps fixed either way.
    graphs: the checkpointed forward segments and each segment's recompute-and-reverse run as
    CUDA graphs cached on H (replayed by later rollouts of the same shape).
    records: in the checkpointed backward, the recompute records every level-step's
    intermediates (claw_level_advance_record) and the reverse reads them
    (claw_level_advance_adjoint_tape) instead of re-running the forward inside the adjoint
    kernel; cell-wise medium, second order.  Memory: an aux-sized tape per level-step of a
    segment."""
    nlev = H.nlev
    tensors = list(q0) + (list(rho) + list(K) if H.medium else [])
    return _Rollout.apply(H, ncoarse, every, nlev, dt, bool(graphs), bool(records), *tensors)

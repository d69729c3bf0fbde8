"""Differentiable rollouts: gradients of a functional of the final state with respect to the
initial state and the medium (rho, K), through the hand-written adjoint kernels.

`LevelStep.apply(H, L, dt, q_old, rho, K)` is one level-step of level L as a differentiable map.
`rollout(H, q0, rho, K, ncoarse, every)` is a torch.autograd.Function over `ncoarse` coarse
steps of hierarchy H (any number of levels and runs).  The forward keeps a checkpoint of every
level's state every `every` coarse steps; the backward recomputes one segment at a time from its
checkpoint (recording each level-step's input state and the pre-average coarse state).  With
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


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, ncoarse, every, nlev, dt, *tensors):
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
            checkpoints, tapes = [], None
            if every is None:   # the whole tape, recorded as the rollout runs
                tapes = []
                for n in range(ncoarse):
                    dt_n = H.dt.clone()
                    tapes.append((_advance_record(H, 0, None, None, 0.0), dt_n))
                    if H.freeze_dt:
                        H.smax.zero_()
                    else:
                        claw.claw_dt_update(H.ctx, 0, H.smax, H.dt)
            else:
                for n in range(ncoarse):
                    if n % every == 0:
                        checkpoints.append(([H.q[L][H.cur[L]].clone() for L in range(nlev)], H.dt.clone()))
                    H.coarse_step()
            out = [H.q[L][H.cur[L]].clone() for L in range(nlev)]
        ctx.H, ctx.ncoarse, ctx.every, ctx.nlev = H, ncoarse, every, nlev
        ctx.checkpoints = checkpoints
        ctx.tapes = tapes
        ctx.frozen = dt is not None
        H.freeze_dt = False
        return tuple(out)

    @staticmethod
    def backward(ctx, *grads):
        H, nlev, every, ncoarse = ctx.H, ctx.nlev, ctx.every, ctx.ncoarse
        lam = [g.clone() if g is not None else torch.zeros_like(H.q[L][0]) for L, g in enumerate(grads)]
        g_aux = [torch.zeros_like(H.aux[L]) if H.medium else None for L in range(nlev)]
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
        grads_out = [None, None, None, None, None] + lam
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


def rollout(H, q0, rho=None, K=None, ncoarse=1, every=20, dt=None):
    """final states (one pool per level) after `ncoarse` coarse steps from q0 (pools per level),
    differentiable with respect to q0 and, for a cell-wise medium, the rho and K pools.
    every: checkpoint interval of the recomputing backward, or None for the recorded tape.
    dt: None for Eq. cfl time steps, else a device tensor of per-run level-0 time steps used
    unchanged for every coarse step.  The gradient holds the time steps fixed either way."""
    nlev = H.nlev
    tensors = list(q0) + (list(rho) + list(K) if H.medium else [])
    return _Rollout.apply(H, ncoarse, every, nlev, dt, *tensors)

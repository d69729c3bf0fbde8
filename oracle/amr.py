"""Oracle drivers: single-grid time stepping and the recursive AMR subcycling of Sec. 2.2.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

advance(L): fill the ghosts of level L, step every box of L from Q^n to Q^{n+1}; if a finer
level exists, take r substeps of it (its ghosts interpolated in space and time from
Q^n_L, Q^{n+1}_L at fraction k/r) and then overwrite the covered cells of Q^{n+1}_L with
the average of the fine cells ("updating", Sec. 2.2-2.3).  dt on level 0 follows the CFL
rule dt = nu_desired * min(dx, dy) / s (Eq. cfl) with s the largest speed seen on any level
in the previous coarse step (or by cfl_max before the first), and dt_{L+1} = dt_L / r_L.
No conservation fix is applied (Sec. 4.3: it does not apply to non-conservative
heterogeneous acoustics).
"""
from __future__ import annotations

import numpy as np

from . import (MBC, average_down, average_down_adjoint, cfl_max, level_fill_ghost,
               level_fill_ghost_adjoint, step, step_adjoint)


def _view(pool, off, nx, ny, ncomp):
    n = ncomp * (nx + 2 * MBC) * (ny + 2 * MBC)
    return pool[off:off + n].reshape(ncomp, ny + 2 * MBC, nx + 2 * MBC)


def _boxes(lev, off):
    return [(int(b[0]), int(b[1]), int(b[2]), int(b[3]), int(o)) for b, o in zip(lev.boxes, off)]


class OracleHierarchy:
    """State of one run on the oracle: per level a q pool and coefficient pools."""

    def __init__(self, run, q, rho, K):
        self.run = run
        self.levels = run.levels
        self.q = [np.array(a, dtype=np.float64, copy=True) for a in q]
        self.rho = [np.asarray(a, dtype=np.float64) for a in rho]
        self.K = [np.asarray(a, dtype=np.float64) for a in K]
        self.smax = max(self.level_cfl_max(L) for L in range(len(self.levels)))
        self.dt_history = []
        self.smax_history = []

    def level_cfl_max(self, L):
        lev = self.levels[L]
        s = 0.0
        for n, b in enumerate(lev.boxes):
            nx, ny = int(b[2]), int(b[3])
            r = _view(self.rho[L], lev.coff[n], nx, ny, 1)[0]
            k = _view(self.K[L], lev.coff[n], nx, ny, 1)[0]
            s = max(s, cfl_max(r, k))
        return s

    def fill(self, L, qpool, cold=None, cnew=None, tau=0.0):
        run, lev = self.run, self.levels[L]
        if L == 0:
            level_fill_ghost(_boxes(lev, lev.qoff), qpool, 3, lev.NX, lev.NY, run.bc)
        else:
            c = self.levels[L - 1]
            level_fill_ghost(_boxes(lev, lev.qoff), qpool, 3, lev.NX, lev.NY, run.bc,
                             _boxes(c, c.qoff), cold, cnew, tau, lev.ratio)

    def step_level(self, L, qold, dt):
        """Q^{n+1} of every box of level L from qold (ghosts filled); returns (qnew, smax)."""
        run, lev = self.run, self.levels[L]
        qnew = qold.copy()
        sm = 0.0
        for n, b in enumerate(lev.boxes):
            nx, ny = int(b[2]), int(b[3])
            qb = _view(qold, lev.qoff[n], nx, ny, 3)
            r = _view(self.rho[L], lev.coff[n], nx, ny, 1)[0]
            k = _view(self.K[L], lev.coff[n], nx, ny, 1)[0]
            out, s = step(qb, r, k, lev.dx, lev.dy, dt, run.order, run.transverse, run.limiter)
            _view(qnew, lev.qoff[n], nx, ny, 3)[:, MBC:MBC + ny, MBC:MBC + nx] = \
                out[:, MBC:MBC + ny, MBC:MBC + nx]
            sm = max(sm, s)
        return qnew, sm

    def advance(self, L, dt, cold=None, cnew=None, tau=0.0, smax_acc=None):
        self.fill(L, self.q[L], cold, cnew, tau)
        qold = self.q[L]
        qnew, sm = self.step_level(L, qold, dt)
        smax_acc[0] = max(smax_acc[0], sm)
        if L + 1 < len(self.levels):
            fine = self.levels[L + 1]
            r = fine.ratio
            for k in range(r):
                self.advance(L + 1, dt / r, qold, qnew, k / r, smax_acc)
            c = self.levels[L]
            average_down(_boxes(fine, fine.qoff), self.q[L + 1], _boxes(c, c.qoff), qnew, 3, r)
        self.q[L] = qnew

    def coarse_step(self, dt=None):
        lev0 = self.levels[0]
        if dt is None:
            dt = self.run.cfl * min(lev0.dx, lev0.dy) / self.smax
        acc = [0.0]
        self.advance(0, dt, smax_acc=acc)
        self.smax = acc[0]
        self.dt_history.append(dt)
        self.smax_history.append(acc[0])
        return dt

    # ------------------------------------------------------------ reverse mode
    def _advance_record(self, L, dt, cold, cnew, tau, acc):
        self.fill(L, self.q[L], cold, cnew, tau)
        node = {"L": L, "q_in": self.q[L].copy(), "cold": cold, "cnew": cnew, "tau": tau, "dt": dt,
                "fine": [], "pre_avg": None}
        qnew, sm = self.step_level(L, node["q_in"], dt)
        acc[0] = max(acc[0], sm)
        if L + 1 < len(self.levels):
            node["pre_avg"] = qnew.copy()
            fine = self.levels[L + 1]
            r = fine.ratio
            for k in range(r):
                node["fine"].append(self._advance_record(L + 1, dt / r, node["q_in"], node["pre_avg"], k / r, acc))
            c = self.levels[L]
            average_down(_boxes(fine, fine.qoff), self.q[L + 1], _boxes(c, c.qoff), qnew, 3, r)
        self.q[L] = qnew
        return node

    def _reverse(self, node, lam, g_rho, g_K, lam_cold=None, lam_cnew=None):
        run = self.run
        L = node["L"]
        lev = self.levels[L]
        lam_pre = lam[L]
        lam_in = np.zeros_like(lam_pre)
        if node["fine"]:
            fine = self.levels[L + 1]
            average_down_adjoint(_boxes(fine, fine.qoff), lam[L + 1], _boxes(lev, lev.qoff), lam_pre, 3,
                                 fine.ratio)
            for f in reversed(node["fine"]):
                self._reverse(f, lam, g_rho, g_K, lam_in, lam_pre)
        for n, b in enumerate(lev.boxes):
            nx, ny = int(b[2]), int(b[3])
            qb = _view(node["q_in"], lev.qoff[n], nx, ny, 3)
            lb = _view(lam_pre, lev.qoff[n], nx, ny, 3)
            r = _view(self.rho[L], lev.coff[n], nx, ny, 1)[0]
            k = _view(self.K[L], lev.coff[n], nx, ny, 1)[0]
            lq, gr, gk = step_adjoint(qb, r, k, lb, lev.dx, lev.dy, node["dt"], run.order, run.transverse,
                                      run.limiter)
            _view(lam_in, lev.qoff[n], nx, ny, 3)[...] += lq
            _view(g_rho[L], lev.coff[n], nx, ny, 1)[0] += gr
            _view(g_K[L], lev.coff[n], nx, ny, 1)[0] += gk
        if L == 0:
            level_fill_ghost_adjoint(_boxes(lev, lev.qoff), lam_in, 3, lev.NX, lev.NY, run.bc)
        else:
            c = self.levels[L - 1]
            level_fill_ghost_adjoint(_boxes(lev, lev.qoff), lam_in, 3, lev.NX, lev.NY, run.bc,
                                     _boxes(c, c.qoff), lam_cold, lam_cnew, node["cold"], node["cnew"],
                                     node["tau"], lev.ratio)
        lam[L] = lam_in

    def gradient(self, ncoarse, final_adjoint):
        """Runs ncoarse coarse steps (recording them) and the reverse sweep.  final_adjoint(q)
        returns, per level, the adjoint of a functional of the final pools.  Returns (J-adjoint of
        the initial q pools, of the rho pools, of the K pools), the coefficient adjoints moved from
        same-level / boundary ghosts to their source cells."""
        tapes = []
        for _ in range(ncoarse):
            lev0 = self.levels[0]
            dt = self.run.cfl * min(lev0.dx, lev0.dy) / self.smax
            acc = [0.0]
            tapes.append(self._advance_record(0, dt, None, None, 0.0, acc))
            self.smax = acc[0]
            self.dt_history.append(dt)
        lam = [np.array(a, dtype=np.float64) for a in final_adjoint(self.q)]
        g_rho = [np.zeros_like(r) for r in self.rho]
        g_K = [np.zeros_like(k) for k in self.K]
        for node in reversed(tapes):
            self._reverse(node, lam, g_rho, g_K)
        for L, lev in enumerate(self.levels):
            for g in (g_rho[L], g_K[L]):
                level_fill_ghost_adjoint(_boxes(lev, lev.coff), g, 1, lev.NX, lev.NY, self.run.bc, copy_only=True)
        return lam, g_rho, g_K

    def interior(self, L, n):
        lev = self.levels[L]
        nx, ny = int(lev.boxes[n][2]), int(lev.boxes[n][3])
        return _view(self.q[L], lev.qoff[n], nx, ny, 3)[:, MBC:MBC + ny, MBC:MBC + nx]


def run_single_grid(q, rho, K, dx, dy, nsteps, bc=(0, 0, 0, 0), cfl=0.9, dt=None,
                    order=2, transverse=2, limiter=4):
    """Steps one padded patch (3, H, W) nsteps times with physical-boundary ghosts."""
    from . import fill_bc
    q = np.array(q, dtype=np.float64, copy=True)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    smax = cfl_max(rho, K)
    dts = []
    for _ in range(nsteps):
        fill_bc(q, bc)
        d = cfl * min(dx, dy) / smax if dt is None else dt
        q, smax = step(q, rho, K, dx, dy, d, order, transverse, limiter)
        dts.append(d)
    fill_bc(q, bc)
    return q, dts

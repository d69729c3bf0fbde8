"""Oracle drivers: single-grid time stepping and the recursive AMR subcycling of Sec. 2.2.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

advance(L): fill the ghosts of level L, step every box of L from Q^n to Q^{n+1}; if a finer
level exists, take r substeps of it (its ghosts interpolated in space and time from
Q^n_L, Q^{n+1}_L at fraction k/r) and then overwrite the covered cells of Q^{n+1}_L with
the average of the fine cells ("updating", Sec. 2.2-2.3).  dt on level 0 follows the CFL
rule dt = nu_desired * min(dx, dy) / s (Eq. cfl) with s the largest speed seen on any level
in the previous coarse step (or by cfl_max before the first), and dt_{L+1} = dt_L / r_L.
The conservation fix of Sec. 2.3 ("refluxing", `reflux=True`; meaningful for a uniform
medium, where acoustics is in conservation form, and for shallow water, whose Roe solver is
conservative: A-dQ + A+dQ = f(Q_R) - f(Q_L)) corrects, after the average, every coarse
cell C that is not covered by the finer level but shares an edge e with it: the flux C's update
used through e is replaced by the average of the fine fluxes through the r fine edges over the r
substeps.  In flux form (f(Q) = A Q, A- / A+ the fluctuations, F~ the correction-plus-transverse
flux), with C left of e and the fine cells F_b right of their edges e_b:
    F_e   = f(Q_C^n) + A-dQ_e + F~_e                              (coarse step)
    F_b^k = f(Q_F^k) - A+dQ_b^k + F~_b^k                          (fine substep k)
    Q_C  += -(dt/dx) [ (1/r^2) sum_{k,b} (F_b^k - f(Q_C^n)) - (F_e - f(Q_C^n)) ]
where F_b^k - f(Q_C^n) = A (Q_F^k - Q_C^n) - A+dQ_b^k + F~_b^k is the paper's C1 + C2 + C3 (for
shallow water f(Q_F^k) - f(Q_C^n) - A+dQ_b^k + F~_b^k with the equations' flux f) and
F_e - f(Q_C^n) = A-dQ_e + F~_e its coarse part; mirrored for C right of e and in y.
"""
from __future__ import annotations

import numpy as np

from . import (MBC, average_down, average_down_adjoint, cfl_max, level_fill_ghost,
               level_fill_ghost_adjoint, step, step_adjoint, step_edges, swe_cfl_max, swe_step,
               swe_step_edges)


def _view(pool, off, nx, ny, ncomp):
    n = ncomp * (nx + 2 * MBC) * (ny + 2 * MBC)
    return pool[off:off + n].reshape(ncomp, ny + 2 * MBC, nx + 2 * MBC)


def _boxes(lev, off):
    return [(int(b[0]), int(b[1]), int(b[2]), int(b[3]), int(o)) for b, o in zip(lev.boxes, off)]


def _map(k, n, lo, hi):
    """index k on [0, n) through the physical boundary: periodic wraps, otherwise None outside"""
    if 0 <= k < n:
        return k
    if (k < 0 and lo == 1) or (k >= n and hi == 1):
        return k % n
    return None


def _find(lev, gi, gj):
    for n, b in enumerate(lev.boxes):
        if b[0] <= gi < b[0] + b[2] and b[1] <= gj < b[1] + b[3]:
            return n
    return -1


def interface(levels, Lf, bc):
    """Coarse-fine interface of level Lf: records (n_c, ci, cj, dir, side, n_f, cells) with C =
    (ci, cj) local to coarse box n_c, dir 0 for an x-edge / 1 for a y-edge, side +1 when C is
    left of / below the edge (the fine region right / above), -1 otherwise, and the r fine
    cells adjacent to the edge, local to fine box n_f."""
    fine, coarse = levels[Lf], levels[Lf - 1]
    r = fine.ratio
    NXc, NYc = coarse.NX, coarse.NY
    out = []
    for n_f, b in enumerate(fine.boxes):
        ilo, jlo, nx, ny = (int(v) for v in b)
        I0, I1, J0, J1 = ilo // r, (ilo + nx) // r, jlo // r, (jlo + ny) // r
        sides = []
        for J in range(J0, J1):
            sides.append((I1, J, 0, -1, [(nx - 1, J * r + k - jlo) for k in range(r)]))
            sides.append((I0 - 1, J, 0, +1, [(0, J * r + k - jlo) for k in range(r)]))
        for I in range(I0, I1):
            sides.append((I, J1, 1, -1, [(I * r + k - ilo, ny - 1) for k in range(r)]))
            sides.append((I, J0 - 1, 1, +1, [(I * r + k - ilo, 0) for k in range(r)]))
        for I, J, d, side, cells in sides:
            Im, Jm = _map(I, NXc, bc[0], bc[1]), _map(J, NYc, bc[2], bc[3])
            if Im is None or Jm is None:
                continue
            if _find(fine, Im * r, Jm * r) >= 0:      # covered: a fine-fine edge
                continue
            n_c = _find(coarse, Im, Jm)
            if n_c < 0:
                raise ValueError("coarse cell next to a fine box is missing (nesting)")
            cb = coarse.boxes[n_c]
            out.append((n_c, Im - int(cb[0]), Jm - int(cb[1]), d, side, n_f, cells))
    return out


class OracleHierarchy:
    """State of one run on the oracle: per level a q pool and coefficient pools."""

    def __init__(self, run, q, rho=None, K=None, reflux=False, system="acoustics", grav=1.0):
        """system="shallow_water": q = (h, hu, hv) stepped by the shallow-water oracle with
        gravity grav (rho, K unused)."""
        self.run = run
        self.reflux = reflux
        self.swe = system == "shallow_water"
        self.grav = grav
        self.levels = run.levels
        self.q = [np.array(a, dtype=np.float64, copy=True) for a in q]
        self.rho = [np.asarray(a, dtype=np.float64) for a in rho] if not self.swe else None
        self.K = [np.asarray(a, dtype=np.float64) for a in K] if not self.swe else None
        self.smax = max(self.level_cfl_max(L) for L in range(len(self.levels)))
        self._iface = {Lf: interface(self.levels, Lf, run.bc) for Lf in range(1, len(self.levels))} if reflux else {}
        self.dt_history = []
        self.smax_history = []

    def level_cfl_max(self, L):
        lev = self.levels[L]
        s = 0.0
        if self.swe:   # speeds of the state: ghosts first (level L from level L-1 at the same time)
            qc = self.q[L - 1] if L else None
            self.fill(L, self.q[L], qc, qc, 0.0)
            for n, b in enumerate(lev.boxes):
                s = max(s, swe_cfl_max(_view(self.q[L], lev.qoff[n], int(b[2]), int(b[3]), 3), self.grav))
            return s
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

    def step_level(self, L, qold, dt, edges=None):
        """Q^{n+1} of every box of level L from qold (ghosts filled); returns (qnew, smax).
        With `edges` a list, it receives each box's per-edge quantities (oracle.step_edges)."""
        run, lev = self.run, self.levels[L]
        qnew = qold.copy()
        sm = 0.0
        for n, b in enumerate(lev.boxes):
            nx, ny = int(b[2]), int(b[3])
            qb = _view(qold, lev.qoff[n], nx, ny, 3)
            if self.swe:
                if edges is None:
                    out, s = swe_step(qb, lev.dx, lev.dy, dt, self.grav, run.order, run.transverse, run.limiter)
                else:
                    out, s, e = swe_step_edges(qb, lev.dx, lev.dy, dt, self.grav, run.order, run.transverse,
                                               run.limiter)
                    edges.append(e)
                _view(qnew, lev.qoff[n], nx, ny, 3)[:, MBC:MBC + ny, MBC:MBC + nx] = \
                    out[:, MBC:MBC + ny, MBC:MBC + nx]
                sm = max(sm, s)
                continue
            r = _view(self.rho[L], lev.coff[n], nx, ny, 1)[0]
            k = _view(self.K[L], lev.coff[n], nx, ny, 1)[0]
            if edges is None:
                out, s = step(qb, r, k, lev.dx, lev.dy, dt, run.order, run.transverse, run.limiter)
            else:
                out, s, e = step_edges(qb, r, k, lev.dx, lev.dy, dt, run.order, run.transverse, run.limiter)
                edges.append(e)
            _view(qnew, lev.qoff[n], nx, ny, 3)[:, MBC:MBC + ny, MBC:MBC + nx] = \
                out[:, MBC:MBC + ny, MBC:MBC + nx]
            sm = max(sm, s)
        return qnew, sm

    # ---------------------------------------------------------- conservation fix (Sec. 2.3)
    def _flux_diff(self, L, n, i, j, d, qf, qc):
        """f(qf) - f(qc) (d = 0) or g(qf) - g(qc) (d = 1): for acoustics A (qf - qc) or
        B (qf - qc) with the medium of cell (i, j) of box n of level L; for shallow water the
        nonlinear fluxes of the equations themselves"""
        if self.swe:
            def flux(q):
                h, hu, hv = q
                g2 = 0.5 * self.grav * h * h
                return np.array([hu, hu * hu / h + g2, hu * hv / h]) if d == 0 else \
                    np.array([hv, hu * hv / h, hv * hv / h + g2])
            return flux(qf) - flux(qc)
        dq = qf - qc
        lev = self.levels[L]
        b = lev.boxes[n]
        nx, ny = int(b[2]), int(b[3])
        rho = _view(self.rho[L], lev.coff[n], nx, ny, 1)[0][MBC + j, MBC + i]
        K = _view(self.K[L], lev.coff[n], nx, ny, 1)[0][MBC + j, MBC + i]
        if d == 0:
            return np.array([K * dq[1], dq[0] / rho, 0.0])
        return np.array([K * dq[2], 0.0, dq[0] / rho])

    def _reflux_coarse(self, Lf, edges_c):
        """per interface record: minus the coarse part (F_e - f(Q_C^n)) of the level Lf-1 step"""
        buf = []
        for (n_c, ci, cj, d, side, n_f, cells) in self._iface[Lf]:
            e = edges_c[n_c]
            i, j = MBC + ci, MBC + cj
            if d == 0:
                t = e["amx"][:, j, i + 1] + e["F"][:, j, i + 1] if side > 0 else -e["apx"][:, j, i] + e["F"][:, j, i]
            else:
                t = e["amy"][:, j + 1, i] + e["G"][:, j + 1, i] if side > 0 else -e["apy"][:, j, i] + e["G"][:, j, i]
            buf.append(-t)
        return buf

    def _reflux_fine(self, Lf, edges_f, qc_old, buf):
        """adds (1/r^2) sum_b (F_b^k - f(Q_C^n)) of one fine substep to every record"""
        fine, coarse = self.levels[Lf], self.levels[Lf - 1]
        r = fine.ratio
        for rec_i, (n_c, ci, cj, d, side, n_f, cells) in enumerate(self._iface[Lf]):
            cb = coarse.boxes[n_c]
            qc = _view(qc_old, coarse.qoff[n_c], int(cb[2]), int(cb[3]), 3)[:, MBC + cj, MBC + ci]
            fb = fine.boxes[n_f]
            qf = _view(self.q[Lf], fine.qoff[n_f], int(fb[2]), int(fb[3]), 3)
            e = edges_f[n_f]
            acc = np.zeros(3)
            for (fi, fj) in cells:
                i, j = MBC + fi, MBC + fj
                t = self._flux_diff(Lf, n_f, fi, fj, d, qf[:, j, i], qc)
                if d == 0:
                    t = t + (-e["apx"][:, j, i] + e["F"][:, j, i] if side > 0 else e["amx"][:, j, i + 1] + e["F"][:, j, i + 1])
                else:
                    t = t + (-e["apy"][:, j, i] + e["G"][:, j, i] if side > 0 else e["amy"][:, j + 1, i] + e["G"][:, j + 1, i])
                acc += t
            buf[rec_i] = buf[rec_i] + acc / (r * r)

    def _reflux_apply(self, Lf, qc_new, buf, dt):
        coarse = self.levels[Lf - 1]
        for rec_i, (n_c, ci, cj, d, side, n_f, cells) in enumerate(self._iface[Lf]):
            cb = coarse.boxes[n_c]
            v = _view(qc_new, coarse.qoff[n_c], int(cb[2]), int(cb[3]), 3)
            h = coarse.dx if d == 0 else coarse.dy
            v[:, MBC + cj, MBC + ci] += -side * (dt / h) * buf[rec_i]

    def advance(self, L, dt, cold=None, cnew=None, tau=0.0, smax_acc=None, buf=None):
        self.fill(L, self.q[L], cold, cnew, tau)
        qold = self.q[L]
        refl = self.reflux and (L + 1 < len(self.levels) or (L > 0 and buf is not None))
        edges = [] if refl else None
        qnew, sm = self.step_level(L, qold, dt, edges)
        smax_acc[0] = max(smax_acc[0], sm)
        if self.reflux and L > 0 and buf is not None:
            self._reflux_fine(L, edges, cold, buf)    # this substep's fine fluxes (level L's interface)
        if L + 1 < len(self.levels):
            fine = self.levels[L + 1]
            r = fine.ratio
            fbuf = self._reflux_coarse(L + 1, edges) if self.reflux else None
            for k in range(r):
                self.advance(L + 1, dt / r, qold, qnew, k / r, smax_acc, fbuf)
            c = self.levels[L]
            average_down(_boxes(fine, fine.qoff), self.q[L + 1], _boxes(c, c.qoff), qnew, 3, r)
            if self.reflux:
                self._reflux_apply(L + 1, qnew, fbuf, dt)
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

    # ------------------------------------------------------------ regridding (Sec. 2.2)
    def regrid(self, tol, buffer, cutoff, max_size, nest=2):
        """Rebuilds levels 1.. top-down from the current state (all levels at the same time):
        flags of level L-1 (oracle.regrid.flag_level, ghosts filled first), grown by `buffer`,
        kept `nest` cells inside level L-1, clustered with `cutoff` and `max_size` (fine cells);
        the new level L takes old level-L values where it had them, else the coarse interpolation.
        Uniform medium (constant coefficient pools) or shallow water."""
        from .regrid import new_boxes, transfer
        run = self.run
        for Lf in range(1, len(self.levels)):
            coarse = self.levels[Lf - 1]
            if Lf - 1 == 0:
                self.fill(0, self.q[0])
            else:
                self.fill(Lf - 1, self.q[Lf - 1], self.q[Lf - 2], self.q[Lf - 2], 0.0)
            old = self.levels[Lf]
            boxes = new_boxes(coarse, self.q[Lf - 1], tol, buffer, cutoff, max_size, nest, old.ratio)
            new = type(old)(old.NX, old.NY, old.dx, old.dy, boxes, old.ratio)   # the caller's level type
            self.q[Lf] = transfer(old, self.q[Lf], new, coarse, self.q[Lf - 1], run.bc)
            if not self.swe:   # uniform medium: the value of level 0's first cell (level 0 keeps its boxes)
                c0 = int(self.levels[0].coff[0])
                self.rho[Lf] = np.full(new.csize, float(self.rho[0][c0]))
                self.K[Lf] = np.full(new.csize, float(self.K[0][c0]))
            self.levels[Lf] = new
        self._iface = {Lf: interface(self.levels, Lf, run.bc) for Lf in range(1, len(self.levels))} \
            if self.reflux else {}

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

"""Host orchestration of the level-steps of one or many runs on libclaw.so.

It owns the device pools (torch tensors) and sequences C-ABI calls in the order of the AMR
time step of Sec. 2.2: fill the ghosts of level L, take one level-step, then R_L substeps of
level L+1 whose ghosts are interpolated in space and time from level L, then overwrite the
covered cells of level L with the fine average ("updating").  The level-0 time step follows
Eq. cfl from the largest wave speed the previous coarse step saw, computed on the device, so
a coarse step is a fixed launch sequence that a CUDA graph replays.  With `reflux=True` (uniform
medium) the conservation fix of Sec. 2.3 corrects the coarse cells next to each finer level
after the average.  No arithmetic of the method happens here.
"""
from __future__ import annotations

import numpy as np
import torch

from . import claw, inputs

MBC = claw.CLAW_MBC


def _align(n, a=inputs.ALIGN):
    return (n + a - 1) // a * a


def band_plan(boxes, nbands, NX, NY, bc):
    """Pieces of a level for stepping it in parts: `boxes` = [(ilo, jlo, nx, ny, qoff)] of one
    run in pool order.  Returns (pieces, ranges, needs): contiguous box ranges of about equal
    cells, their element ranges in the pool (q planes of the first box to the end of the last),
    and for every piece the pieces whose boxes its ghosts read: the boxes that meet it grown by
    two cells, with the periodic images of the domain [0, NX) x [0, NY) where bc says periodic."""
    cells = np.cumsum([nx * ny for (_, _, nx, ny, _) in boxes])
    total = int(cells[-1])
    cut = [0] + [int(np.searchsorted(cells, total * k / nbands, side="right")) for k in range(1, nbands)] + \
        [len(boxes)]
    cut = sorted(set(cut))
    pieces = [(cut[k], cut[k + 1]) for k in range(len(cut) - 1) if cut[k + 1] > cut[k]]
    owner = np.zeros(len(boxes), dtype=np.int64)
    for k, (b0, b1) in enumerate(pieces):
        owner[b0:b1] = k
    shx = [0] + ([-NX, NX] if bc[0] == 1 else [])
    shy = [0] + ([-NY, NY] if bc[2] == 1 else [])
    lo = np.array([[i0, j0, i0 + nx, j0 + ny] for (i0, j0, nx, ny, _) in boxes], dtype=np.int64)
    needs = []
    for (b0, b1) in pieces:
        need = set()
        for n in range(b0, b1):
            i0, j0, i1, j1 = lo[n]
            for sx in shx:
                for sy in shy:
                    hit = (lo[:, 0] + sx < i1 + 2) & (lo[:, 2] + sx > i0 - 2) & \
                          (lo[:, 1] + sy < j1 + 2) & (lo[:, 3] + sy > j0 - 2)
                    need.update(int(v) for v in np.unique(owner[hit]))
        needs.append(sorted(need))
    ranges = []
    for (b0, b1) in pieces:
        _, _, nx, ny, qoff = boxes[b1 - 1]
        ranges.append((int(boxes[b0][4]), int(qoff) + 3 * (nx + 4) * (ny + 4)))
    return pieces, ranges, needs


class Hierarchy:
    """Device state of `runs` (a list of inputs.Run) on one context.

    q0[r][L], rho[r][L], K[r][L]: numpy pools of run r, level L in the inputs layout (rho, K
    only for a cell-wise medium; a uniform medium passes rho0, K0).  All runs' pools of a level
    are concatenated into one device pool per level.  system="shallow_water" steps q = (h, hu, hv)
    of the shallow water equations with gravity `grav` instead (no medium)."""

    def __init__(self, runs, q0, rho=None, K=None, rho0=1.0, K0=4.0, device=0, tiling=None, reflux=False,
                 system="acoustics", grav=1.0, walk=None):
        self.runs = runs
        self.nruns = len(runs)
        self.nlev = max(len(r.levels) for r in runs)
        self.medium = 0 if rho is None else 1
        self.system = claw.SYSTEMS[system]
        if self.system == claw.CLAW_SYS_SHALLOW_WATER and self.medium:
            raise ValueError("shallow water has no medium")
        self.dev = torch.device("cuda", device)
        probs = []
        for r in runs:
            p = claw.claw_problem()
            p.xlo, p.ylo, p.xhi, p.yhi = r.xlo, r.ylo, r.xhi, r.yhi
            p.nx0, p.ny0 = r.levels[0].NX, r.levels[0].NY
            p.nlev = len(r.levels)
            for L, lev in enumerate(r.levels):
                p.ratio[L] = lev.ratio if L else 1
            p.cfl = r.cfl
            p.limiter, p.order, p.transverse = r.limiter, r.order, r.transverse
            for s in range(4):
                p.bc[s] = r.bc[s]
            p.medium = self.medium
            p.rho0, p.K0 = rho0, K0
            p.system = self.system
            p.grav = grav
            probs.append(p)
        self.ctx = claw.claw_create(probs, device)
        self.q = []        # per level [A, B]
        self.cur = []
        self.aux = []
        self.rho = []
        self.K = []
        self.boxes = []    # per level list of claw_box
        self.layout = []   # per level list of (run, qbase, cbase)
        self.tiling = tiling
        # how the level-step's CTAs share the tiles (claw_set_tile_walk): None keeps the
        # library's default, 0 strides, 1 column walks
        self.walk = walk
        for L in range(self.nlev):
            boxes, lay, qb, cb = self._layout(L)
            self.boxes.append(boxes)
            self.layout.append(lay)
            claw.claw_set_level(self.ctx, L, boxes)
            self._install_tiling(L)
            qh = np.zeros(max(qb, inputs.ALIGN))
            for (ri, qbase, _) in lay:
                a = np.asarray(q0[ri][L], dtype=np.float64)
                qh[qbase:qbase + a.size] = a
            A = torch.from_numpy(qh).to(self.dev)
            self.q.append([A, torch.zeros_like(A)])
            self.cur.append(0)
            if self.medium:
                rh = np.ones(max(cb, inputs.ALIGN))
                kh = np.ones(max(cb, inputs.ALIGN))
                for (ri, _, cbase) in lay:
                    a = np.asarray(rho[ri][L], dtype=np.float64)
                    k = np.asarray(K[ri][L], dtype=np.float64)
                    rh[cbase:cbase + a.size] = a
                    kh[cbase:cbase + k.size] = k
                self.rho.append(torch.from_numpy(rh).to(self.dev))
                self.K.append(torch.from_numpy(kh).to(self.dev))
                aux = torch.zeros(claw.CLAW_NAUX * rh.size, dtype=torch.float64, device=self.dev)
                claw.claw_medium_aux(self.ctx, L, self.rho[L], self.K[L], aux)
                self.aux.append(aux)
            else:
                self.rho.append(None)
                self.K.append(None)
                self.aux.append(None)
        self.dt = torch.zeros(self.nruns, dtype=torch.float64, device=self.dev)
        self.smax = torch.zeros(self.nruns, dtype=torch.float64, device=self.dev)
        self.patchwise = False
        self.reflux = bool(reflux)
        if self.reflux and self.medium:
            raise ValueError("the conservation fix needs the uniform medium (conservation form)")
        # per fine level: the conservation fix's coarse and fine parts of every interface record
        self.rbuf = [None] + [torch.zeros(max(1, claw.claw_reflux_buffer_size(self.ctx, L)), dtype=torch.float64,
                                          device=self.dev) if self.reflux else None
                              for L in range(1, self.nlev)]
        self.freeze_dt = False   # keep dt as set (no Eq. cfl update after a coarse step)
        self.fused = False       # one-level hierarchies: one launch per step (pulled ghosts, Eq. cfl on the device)
        self.pull = True         # coarse steps pull same-level / boundary ghosts (fill only interpolated ones)
        self.pull_levels = [True] * self.nlev   # per level (the autotuner may prefer the copy launch)
        # per pulling level: the step evaluates the interpolated ghosts too (one launch) instead of
        # the interpolation launch filling them first (the autotuner decides)
        self.fuse_interp = [False] * self.nlev
        # levels whose interpolated ghosts are filled by the launch before their substep (spare CTAs
        # of the previous substep's step, or of the coarser level's step for the first one)
        # instead of by a launch of their own
        self.fill_ahead = True
        # a list while sections of eager coarse steps are timed: (name, start event, end event)
        self.sections = None

    def _install_tiling(self, L):
        if self.level_tiling(L) is not None:
            claw.claw_set_tiling(self.ctx, L, *self.level_tiling(L))
        if self.walk is not None:
            claw.claw_set_tile_walk(self.ctx, L, self.walk)

    def level_tiling(self, L):
        """(tx, ty, staging, threads) installed on level L: `tiling` is one such tuple for every
        level or a sequence of them per level (the last one for the levels beyond), or None for
        the library's default"""
        t = self.tiling
        if t is None:
            return None
        if isinstance(t[0], (tuple, list)):
            return tuple(t[min(L, len(t) - 1)])
        return tuple(t)

    def _layout(self, L):
        """(claw boxes as a claw.box_array, [(run, q base, coefficient base)], q size, coefficient
        size) of level L"""
        parts, qb, cb = [], 0, 0
        lay = []
        for ri, r in enumerate(self.runs):
            if L >= len(r.levels):
                continue
            lev = r.levels[L]
            lay.append((ri, qb, cb))
            a = claw.box_array(len(lev.boxes))
            a.run = ri
            a.ilo, a.jlo, a.nx, a.ny = lev.boxes[:, 0], lev.boxes[:, 1], lev.boxes[:, 2], lev.boxes[:, 3]
            a.qoff = qb + lev.qoff
            a.coff = cb + lev.coff
            parts.append(a)
            qb += _align(lev.qsize)
            cb += _align(lev.csize)
        boxes = np.concatenate(parts).view(np.recarray) if parts else claw.box_array(0)
        return boxes, lay, qb, cb

    # -------------------------------------------------------------- regridding (Sec. 2.2)
    def regrid(self, tol, buffer, cutoff, max_size, nest=2):
        """Rebuilds levels 1.. top-down from the current state (every level at the same time, as
        after a coarse step): the flags of level L-1 (claw_flag_cells: some component differs
        from a face neighbour by more than tol), grown by `buffer` cells and kept `nest` cells
        inside level L-1, are clustered into the new boxes of level L (claw_regrid_boxes: cutoff,
        max_size in level-L cells); the new level takes the old level's values where it had them
        and the conservative interpolation from level L-1 elsewhere (claw_regrid_transfer).
        Uniform medium.  Captured graphs and autotuned tilings of the rebuilt levels are stale."""
        if self.medium:
            raise ValueError("regridding is built for the uniform medium")
        for Lf in range(1, self.nlev):
            Lc = Lf - 1
            qc = self.q[Lc][self.cur[Lc]]
            if Lc == 0:
                claw.claw_fill_ghost(self.ctx, 0, qc)
            else:
                qcc = self.q[Lc - 1][self.cur[Lc - 1]]
                claw.claw_fill_ghost(self.ctx, Lc, qc, qcc, qcc, 0.0)
            flags = torch.zeros(max(1, claw.claw_flag_grid_size(self.ctx, Lc)), dtype=torch.uint8, device=self.dev)
            claw.claw_flag_cells(self.ctx, Lc, qc, tol, flags)
            fh = flags.cpu().numpy()
            off = 0
            for ri, run in enumerate(self.runs):
                if Lc >= len(run.levels):
                    continue
                lc = run.levels[Lc]
                grid = fh[off:off + lc.NX * lc.NY].reshape(lc.NY, lc.NX)
                off += lc.NX * lc.NY
                if Lf >= len(run.levels):
                    continue
                nb = claw.claw_regrid_boxes(self.ctx, Lc, ri, grid, buffer, nest, cutoff, max_size)
                old = run.levels[Lf]
                run.levels[Lf] = inputs.Level(old.NX, old.NY, old.dx, old.dy,
                                              np.array(nb, dtype=np.int32).reshape(-1, 4), old.ratio)
            old_boxes, old_pool = self.boxes[Lf], self.q[Lf][self.cur[Lf]]
            boxes, lay, qb, _ = self._layout(Lf)
            claw.claw_set_level(self.ctx, Lf, boxes)   # also clears the finer levels' tables
            self._install_tiling(Lf)
            new = torch.zeros(max(qb, inputs.ALIGN), dtype=torch.float64, device=self.dev)
            claw.claw_regrid_transfer(self.ctx, Lf, old_boxes, old_pool, new, qc)
            self.boxes[Lf], self.layout[Lf] = boxes, lay
            self.q[Lf] = [new, torch.zeros_like(new)]
            self.cur[Lf] = 0
            if self.reflux:
                self.rbuf[Lf] = torch.zeros(max(1, claw.claw_reflux_buffer_size(self.ctx, Lf)),
                                            dtype=torch.float64, device=self.dev)
            self.__dict__.pop("_ghost_masks", None)
            self.drop_graphs(buffers=True)

    # -------------------------------------------------------------- stepping
    def ratio(self, L):
        return self.runs[0].levels[L].ratio

    def init_dt(self):
        """dt from Eq. cfl with the largest cell speed on any level (before the first step).
        Shallow water: the speeds come from the state, so the ghosts are filled first (level L
        from level L-1 at the same time)."""
        self.smax.zero_()
        for L in range(self.nlev):
            if self.system == claw.CLAW_SYS_SHALLOW_WATER:
                qc = self.q[L - 1][self.cur[L - 1]] if L else None
                claw.claw_fill_ghost(self.ctx, L, self.q[L][self.cur[L]], qc, qc, 0.0)
                claw.claw_cfl_max_state(self.ctx, L, self.q[L][self.cur[L]], self.smax)
            else:
                claw.claw_cfl_max(self.ctx, L, self.aux[L], self.smax)
        claw.claw_dt_update(self.ctx, 0, self.smax, self.dt)

    def step_level(self, L, stream=None):
        src, dst = self.q[L][self.cur[L]], self.q[L][1 - self.cur[L]]
        fn = claw.claw_level_step_patchwise if self.patchwise else claw.claw_level_step
        fn(self.ctx, L, src, dst, self.aux[L], self.dt, self.smax, stream)

    def _section(self, name, stream):
        """Starts a timed section of an eager coarse step on the current stream; returns its end
        event (to record when the section's launches are enqueued), or None when not timing."""
        if self.sections is None or stream is not None or torch.cuda.is_current_stream_capturing():
            return None
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        self.sections.append((name, s, e))
        return e

    def section_ms(self):
        """{section: ms} summed over the sections timed since the last call (synchronises)"""
        torch.cuda.synchronize()
        out = {}
        for name, s, e in self.sections or []:
            out[name] = out.get(name, 0.0) + s.elapsed_time(e)
        if self.sections is not None:
            self.sections = []
        return out

    def _plain_pull(self, L):
        """level L's substeps pull their same-level and boundary ghosts and read the interpolated
        ones from their pool (filled by a launch before)"""
        return self.pull and self.pull_levels[L] and not self.reflux and not self.patchwise and not self.fuse_interp[L]

    def advance(self, L, cold=None, cnew=None, tau=0.0, stream=None, filled=False, tau_next=None):
        """One substep of level L (at time fraction tau of the coarser level's step, whose states
        are cold, cnew) followed by the finer levels' substeps.  filled: the interpolated ghosts of
        this substep are in its pool already; tau_next: the time fraction of level L's next substep
        in the same coarser step (None after the last).  Returns whether the launch also filled
        the next substep's interpolated ghosts."""
        q = self.q[L][self.cur[L]]
        dst = self.q[L][1 - self.cur[L]]
        filled_next = False
        child_filled = False
        if self.pull and self.pull_levels[L] and not self.reflux and not self.patchwise and self.fuse_interp[L]:
            # one launch: the step pulls the same-level and boundary ghosts from their sources and
            # evaluates the ones interpolated from the coarser level itself
            e = self._section("advance", stream)
            claw.claw_level_advance_interp(self.ctx, L, q, dst, self.aux[L], self.dt,
                                           self.smax, claw.CLAW_ADVANCE_PULL_GHOSTS, cold, cnew, tau, stream)
            if e is not None:
                e.record()
        elif self._plain_pull(L):
            # only the interpolated ghosts are filled (by the launch before when filling ahead);
            # the step pulls the others from their sources
            if not (filled and self.fill_ahead):
                e = self._section("fill", stream)
                claw.claw_fill_ghost_interp(self.ctx, L, q, cold, cnew, tau, stream)
                if e is not None:
                    e.record()
            jobs = []
            if self.fill_ahead:
                if L > 0 and tau_next is not None:   # this level's next substep, into dst
                    jobs.append((L, dst, cold, cnew, tau_next))
                    filled_next = True
                if L + 1 < self.nlev and self._plain_pull(L + 1):   # the finer level's first substep
                    jobs.append((L + 1, self.q[L + 1][self.cur[L + 1]], q, q, 0.0))
                    child_filled = True
            e = self._section("advance", stream)
            claw.claw_level_advance_fill(self.ctx, L, q, dst, self.aux[L], self.dt, self.smax,
                                         claw.CLAW_ADVANCE_PULL_GHOSTS, jobs, stream)
            if e is not None:
                e.record()
        else:
            e = self._section("fill", stream)
            claw.claw_fill_ghost(self.ctx, L, q, cold, cnew, tau, stream)
            if e is not None:
                e.record()
            e = self._section("advance", stream)
            if self.reflux and L > 0:             # this substep's fine fluxes at level L's interface
                claw.claw_reflux_fine(self.ctx, L, q, cold, self.dt, self.rbuf[L], stream)
            if self.reflux and L + 1 < self.nlev:  # the coarse fluxes at the finer level's interface
                claw.claw_reflux_coarse(self.ctx, L + 1, q, self.dt, self.rbuf[L + 1], stream)
            self.step_level(L, stream)
            if e is not None:
                e.record()
        old, new = self.q[L][self.cur[L]], self.q[L][1 - self.cur[L]]
        if L + 1 < self.nlev:
            r = self.ratio(L + 1)
            filled = child_filled
            for k in range(r):
                filled = self.advance(L + 1, old, new, k / r, stream, filled=filled,
                                      tau_next=(k + 1) / r if k + 1 < r else None)
            e = self._section("update", stream)
            claw.claw_average_down(self.ctx, L + 1, self.q[L + 1][self.cur[L + 1]], new, stream)
            if self.reflux:
                claw.claw_reflux_apply(self.ctx, L + 1, self.rbuf[L + 1], self.dt, new, stream)
            if e is not None:
                e.record()
        self.cur[L] ^= 1
        return filled_next

    def coarse_step(self, stream=None):
        if self.fused and self.nlev == 1 and not self.patchwise and not self.freeze_dt:
            # one launch: the step takes the ghosts from their source cells and applies Eq. cfl
            # on its last CTA (the ghost cells of the pools are neither read nor written)
            src, dst = self.q[0][self.cur[0]], self.q[0][1 - self.cur[0]]
            claw.claw_level_advance(self.ctx, 0, src, dst, self.aux[0], self.dt, self.smax,
                                    claw.CLAW_ADVANCE_PULL_GHOSTS | claw.CLAW_ADVANCE_UPDATE_DT, stream)
            self.cur[0] ^= 1
            return
        self.advance(0, stream=stream)
        if self.freeze_dt:
            self.smax.zero_()
        else:
            claw.claw_dt_update(self.ctx, 0, self.smax, self.dt, stream)

    def _bands(self, nbands):
        """the piece plan of level 0 for host-resident stepping (see band_plan)"""
        run0 = self.runs[0]
        lev = run0.levels[0]
        b = self.boxes[0]
        boxes = list(zip(b.ilo.tolist(), b.jlo.tolist(), b.nx.tolist(), b.ny.tolist(), b.qoff.tolist()))
        return band_plan(boxes, nbands, lev.NX, lev.NY, run0.bc)

    def packed_size(self, L=0):
        """doubles of level L's packed interiors (every box's three nx x ny planes, box order)"""
        return claw.claw_packed_size(self.ctx, L)

    def pack(self, L=0, out=None):
        """level L's interiors in packed form (a device tensor)"""
        out = torch.empty(self.packed_size(L), dtype=torch.float64, device=self.dev) if out is None else out
        claw.claw_pack_interiors(self.ctx, L, 0, len(self.boxes[L]), self.q[L][self.cur[L]], out)
        return out

    def steps_from_host(self, host_a, host_b, nsteps, bands=None):
        """One-level hierarchies of one run: `nsteps` coarse steps with the state resident in
        pinned host memory, either as the level's pool (with ghost cells) or in packed form
        (interiors only, see `pack`; chosen by the buffers' length).  Every step copies the state
        from the host, advances it, and copies the new state back into the other host buffer;
        the next step reads that one.  The level is taken in `bands` pieces of boxes
        (claw_level_advance_boxes with pulled ghosts): a piece is stepped as soon as it and the
        pieces its ghosts come from have arrived, and copied back as soon as it is stepped, so
        that the copies in both directions overlap each other and the steps.  Packed pieces are
        unpacked into the pool and packed out of it on the copy streams.  Eq. cfl follows the
        last piece of a step.  Measured on the 2048^2 workload: packed state in eight pieces
        0.71 ms per step (the default), pool state in four pieces 0.80 ms.  Returns the host
        buffer holding the final state."""
        if self.nlev != 1 or self.nruns != 1:
            raise ValueError("host-resident stepping is for one-level hierarchies of one run")
        packed = host_a.numel() == self.packed_size(0)
        if bands is None:
            bands = 8 if packed else 4
        if not hasattr(self, "_band_cache") or self._band_cache[0] != bands:
            self._band_cache = (bands, self._bands(bands))
        parts, ranges, needs = self._band_cache[1]
        if packed:
            b = self.boxes[0]
            offs = np.concatenate([[0], np.cumsum(3 * b.nx.astype(np.int64) * b.ny)])
            ranges = [(int(offs[b0]), int(offs[b1])) for (b0, b1) in parts]
            if getattr(self, "_stage", None) is None or self._stage[0].numel() != host_a.numel():
                self._stage = (torch.empty(host_a.numel(), dtype=torch.float64, device=self.dev),
                               torch.empty(host_a.numel(), dtype=torch.float64, device=self.dev))
            st_in, st_out = self._stage
        elif host_a.numel() != self.q[0][0].numel():
            raise ValueError("host buffers must hold the level's pool or its packed interiors")
        comp = torch.cuda.current_stream(self.dev)
        s_in, s_out = torch.cuda.Stream(device=self.dev), torch.cuda.Stream(device=self.dev)
        # packed form: the unpack and pack kernels run on their own streams, so that the copy
        # streams carry copies only
        s_un, s_pk = torch.cuda.Stream(device=self.dev), torch.cuda.Stream(device=self.dev)
        arrived = [torch.cuda.Event() for _ in parts]
        stepped = [torch.cuda.Event() for _ in parts]
        landed = [torch.cuda.Event() for _ in parts]      # a packed piece is in the staging buffer
        unpacked = [None] * len(parts)                    # ... and has been unpacked from it
        packed_ev = [torch.cuda.Event() for _ in parts]   # a piece is packed into the out staging
        left = [None] * len(parts)
        src, dst = host_a, host_b
        for st in (s_in, s_out, s_un, s_pk):
            st.wait_stream(comp)
        flags = claw.CLAW_ADVANCE_PULL_GHOSTS
        for _ in range(nsteps):
            q, qn = self.q[0][self.cur[0]], self.q[0][1 - self.cur[0]]
            for k, (a, b) in enumerate(ranges):
                if left[k] is not None:
                    s_in.wait_event(left[k])   # this piece of the previous step is back on the host
                if packed:
                    if unpacked[k] is not None:
                        s_in.wait_event(unpacked[k])   # its staging slot has been read
                    with torch.cuda.stream(s_in):
                        st_in[a:b].copy_(src[a:b], non_blocking=True)
                    landed[k].record(s_in)
                    s_un.wait_event(landed[k])
                    claw.claw_unpack_interiors(self.ctx, 0, parts[k][0], parts[k][1], st_in, q, s_un)
                    ev = torch.cuda.Event()
                    ev.record(s_un)
                    unpacked[k] = ev
                    arrived[k] = ev
                else:
                    with torch.cuda.stream(s_in):
                        q[a:b].copy_(src[a:b], non_blocking=True)
                    arrived[k].record(s_in)
            for k, (b0, b1) in enumerate(parts):
                for m in needs[k]:
                    comp.wait_event(arrived[m])
                claw.claw_level_advance_boxes(self.ctx, 0, b0, b1, q, qn, self.aux[0], self.dt, self.smax, flags,
                                              comp)
                stepped[k].record(comp)
            claw.claw_dt_update(self.ctx, 0, self.smax, self.dt, comp)
            for k, (a, b) in enumerate(ranges):
                if packed:
                    s_pk.wait_event(stepped[k])
                    if left[k] is not None:
                        s_pk.wait_event(left[k])   # its out staging slot has been copied out
                    claw.claw_pack_interiors(self.ctx, 0, parts[k][0], parts[k][1], qn, st_out, s_pk)
                    packed_ev[k].record(s_pk)
                    s_out.wait_event(packed_ev[k])
                    with torch.cuda.stream(s_out):
                        dst[a:b].copy_(st_out[a:b], non_blocking=True)
                else:
                    s_out.wait_event(stepped[k])
                    with torch.cuda.stream(s_out):
                        dst[a:b].copy_(qn[a:b], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_out)
                left[k] = ev
            self.cur[0] ^= 1
            src, dst = dst, src
        for st in (s_out, s_in, s_un, s_pk):
            comp.wait_stream(st)
        return src

    def launches_per_coarse_step(self):
        """kernels one coarse step enqueues (counted from the library's own counter)."""
        before = claw.claw_launch_count(self.ctx)
        state = (list(self.cur), self.dt.clone(), self.smax.clone(), [ [a.clone() for a in p] for p in self.q])
        self.coarse_step()
        n = claw.claw_launch_count(self.ctx) - before
        self.cur, dt, sm, qs = state
        self.dt.copy_(dt)
        self.smax.copy_(sm)
        for L in range(self.nlev):
            for k in range(2):
                self.q[L][k].copy_(qs[L][k])
        return n

    def capture(self, ncoarse: int = 2):
        """CUDA graph of `ncoarse` coarse steps (an even count returns every level to the same
        buffer parity, so the graph can be replayed)."""
        s = torch.cuda.Stream(device=self.dev)
        s.wait_stream(torch.cuda.current_stream(self.dev))
        g = torch.cuda.CUDAGraph()
        cur0 = list(self.cur)
        with torch.cuda.graph(g, stream=s):
            for _ in range(ncoarse):
                self.coarse_step(stream=s)
        torch.cuda.current_stream(self.dev).wait_stream(s)
        if self.cur != cur0:
            raise ValueError("capture an even number of coarse steps")
        return g

    def fused_stepper(self):
        """One-level hierarchies: a stepper whose step() replays, for the current buffer parity,
        a CUDA graph of the one launch of a step: the persistent level-step that takes its ghosts
        from their source cells and applies Eq. cfl on its last CTA."""
        return FusedStepper(self)

    def sync_status(self):
        return claw.claw_sync_status(self.ctx)

    def drop_graphs(self, buffers=False):
        """forgets the CUDA graphs the differentiable rollouts cached on this hierarchy (needed
        after a tiling or a ghost-launch choice changes; Hierarchy.regrid and the autotuner call
        it), and with `buffers` their tape and adjoint buffers too (the pools changed size)"""
        self.__dict__.pop("_graphs", None)
        if buffers:
            self.__dict__.pop("_graph_buffers", None)

    # -------------------------------------------------------------- readback
    def pool(self, L):
        return self.q[L][self.cur[L]]

    def interior(self, run, L, n, pool=None):
        """(3, ny, nx) numpy interior of box n of run `run` on level L."""
        lev = self.runs[run].levels[L]
        qbase = [qb for (ri, qb, _) in self.layout[L] if ri == run][0]
        b = lev.boxes[n]
        nx, ny = int(b[2]), int(b[3])
        off = qbase + int(lev.qoff[n])
        P = (self.pool(L) if pool is None else pool)
        v = P[off:off + 3 * (nx + 4) * (ny + 4)].view(3, ny + 4, nx + 4)
        return v[:, MBC:MBC + ny, MBC:MBC + nx].cpu().numpy()

    def level_numpy(self, run, L):
        lev = self.runs[run].levels[L]
        qbase = [qb for (ri, qb, _) in self.layout[L] if ri == run][0]
        return self.pool(L)[qbase:qbase + lev.qsize].cpu().numpy()

    def close(self):
        if self.ctx:
            claw.claw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FusedStepper:
    """Graphs of one level-step of a one-level hierarchy, one per buffer parity.

    step(events) replays the graph of the current parity and flips the parity; `events` (two
    CUDA events, optional) are recorded before and after it on the current stream."""

    def __init__(self, H: Hierarchy):
        if H.nlev != 1 or H.patchwise:
            raise ValueError("the fused stepper is for one-level hierarchies on the tiled path")
        self.H = H
        ctx = H.ctx
        flags = claw.CLAW_ADVANCE_UPDATE_DT | claw.CLAW_ADVANCE_PULL_GHOSTS

        def capture(fn):
            s = torch.cuda.Stream(device=H.dev)
            s.wait_stream(torch.cuda.current_stream(H.dev))
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                fn(s)
            torch.cuda.current_stream(H.dev).wait_stream(s)
            return g

        self.c0 = H.cur[0]
        self.graphs = []   # graphs[i] reads buffer c0 ^ i and writes the other
        for _ in range(2):
            c = H.cur[0]
            qa, qb = H.q[0][c], H.q[0][1 - c]
            # one eager launch first (tensor-map cache, kernel attributes), then capture
            claw.claw_level_advance(ctx, 0, qa, qb, H.aux[0], H.dt, H.smax, flags)
            self.graphs.append(capture(lambda s, qa=qa, qb=qb: claw.claw_level_advance(
                ctx, 0, qa, qb, H.aux[0], H.dt, H.smax, flags, s)))
            H.cur[0] ^= 1
        torch.cuda.synchronize(H.dev)
        # launches of one step, counted by the library
        before = claw.claw_launch_count(ctx)
        claw.claw_level_advance(ctx, 0, H.q[0][H.cur[0]], H.q[0][1 - H.cur[0]], H.aux[0], H.dt, H.smax, flags)
        self.launches_per_step = claw.claw_launch_count(ctx) - before
        H.cur[0] ^= 1

    def step(self, events=None):
        H = self.H
        g = self.graphs[H.cur[0] ^ self.c0]
        if events is not None:
            events[0].record()
        g.replay()
        if events is not None:
            events[1].record()
        H.cur[0] ^= 1

"""GPU adjoint (claw_level_step_adjoint and the reverse AMR transfers behind
paper_1808_02638_gb300.adjoint.rollout) against the oracle's reverse mode and against central
finite differences of a receiver functional in smooth directions."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs

from gpu_helpers import lib_ready

pytestmark = pytest.mark.gpu
M = 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib_ready()


def _tensors(H, pools, kind):
    import torch
    out = []
    for L in range(H.nlev):
        ref = {"q": H.q[L][0], "c": H.rho[L]}[kind]
        a = np.zeros(ref.numel())
        for (ri, qb, cb) in H.layout[L]:
            base = qb if kind == "q" else cb
            a[base:base + pools[ri][L].size] = pools[ri][L]
        out.append(torch.from_numpy(a).to(ref.device).requires_grad_(True))
    return out


def _receiver_J(H, outs, lev0, box):
    i0, j0, n = box
    nx, ny = int(lev0.boxes[0][2]), int(lev0.boxes[0][3])
    v = outs[0][:3 * (nx + 4) * (ny + 4)].view(3, ny + 4, nx + 4)
    return (v[0, M + j0:M + j0 + n, M + i0:M + i0 + n] ** 2).sum()


def _compare(got, want, tol):
    scale = max(np.abs(w).max() for w in want)
    err = max(np.abs(g[:w.size] - w).max() for g, w in zip(got, want)) / scale
    assert err <= tol, err
    return err


@pytest.mark.parametrize("nlev", [1, 2])
def test_recorded_tape_equals_recomputed_segments(nlev):
    # every=None records the tape during the forward instead of recomputing segments in the
    # backward: the same states enter the same reverse kernels, so the functional is identical and
    # the gradients agree to the rounding of the reverse kernels' FP64 atomics (their summation
    # order is not fixed)
    import torch
    from paper_1808_02638_gb300.adjoint import rollout
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 32
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    if nlev == 1:
        run.levels = [inputs.Level(n, n, 2 / n, 2 / n, [(0, 0, n, n)])]
    else:
        run.levels = inputs.amr_levels(run, n, 4, [(0.2, 0.45)], [31])
    r2 = inputs.smooth_field(21, n, n, 0.5, 2.0, sigma=3.0)
    k2 = inputs.smooth_field(22, n, n, 1.0, 8.0, sigma=3.0)
    q = [inputs.init_q(run, lev) for lev in run.levels]
    rho = [inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(run.levels)]
    K = [inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(run.levels)]
    H = Hierarchy([run], [q], [rho], [K])
    grads = []
    for every in (3, None):
        tq, tr, tk = _tensors(H, [q], "q"), _tensors(H, [rho], "c"), _tensors(H, [K], "c")
        outs = rollout(H, tq, tr, tk, ncoarse=7, every=every)
        J = _receiver_J(H, outs, run.levels[0], (18, 10, 6))
        J.backward()
        torch.cuda.synchronize()
        grads.append([t.grad.clone() for t in tq + tr + tk] + [J.detach().clone()])
    assert torch.equal(grads[0][-1], grads[1][-1])
    for a, b in zip(grads[0][:-1], grads[1][:-1]):
        assert float((a - b).abs().max()) <= 1e-12 * max(float(b.abs().max()), 1e-300)


@pytest.mark.parametrize("limiter", [4, 3, 2, 1, 0])
def test_recorded_step_adjoint_equals_the_recomputing_adjoint(limiter):
    # the checkpointed backward with recorded level-step tapes (claw_level_advance_record +
    # claw_level_advance_adjoint_tape, no forward phase in the adjoint kernel) against the adjoint
    # kernel that re-runs the forward from q, with and without CUDA graphs: the same map summed in
    # another order, so the gradients agree to the rounding of the FP64 reductions
    import torch
    from paper_1808_02638_gb300.adjoint import rollout
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 32
    run = inputs.Run(*inputs.PULSE_DOMAIN, limiter=limiter, bc=(1, 1, 2, 0))
    run.levels = inputs.amr_levels(run, n, 4, [(0.2, 0.45)], [31])
    run.levels[0] = inputs.Level(n, n, 2 / n, 2 / n, inputs.uniform_tiling(n, n, 16, 16))
    r2 = inputs.smooth_field(25, n, n, 0.5, 2.0, sigma=3.0)
    k2 = inputs.smooth_field(26, n, n, 1.0, 8.0, sigma=3.0)
    q = [inputs.init_q(run, lev) for lev in run.levels]
    rho = [inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(run.levels)]
    K = [inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(run.levels)]
    H = Hierarchy([run], [q], [rho], [K])
    grads = []
    for graphs, records in ((True, True), (False, True), (True, False), (False, False)):
        tq, tr, tk = _tensors(H, [q], "q"), _tensors(H, [rho], "c"), _tensors(H, [K], "c")
        outs = rollout(H, tq, tr, tk, ncoarse=5, every=3, graphs=graphs, records=records)
        v = outs[0][:3 * 20 * 20].view(3, 20, 20)
        J = (v[0, M + 3:M + 12, M + 4:M + 13] ** 2).sum()
        J.backward()
        torch.cuda.synchronize()
        grads.append([t.grad.clone() for t in tq + tr + tk] + [J.detach().clone()])
    assert H.sync_status() == 0
    for other in grads[1:]:
        assert torch.equal(grads[0][-1], other[-1])
        for a, b in zip(grads[0][:-1], other[:-1]):
            assert float((a - b).abs().max()) <= 1e-12 * max(float(b.abs().max()), 1e-300)
    assert min(float(g.abs().max()) for g in grads[0][:-1]) > 0.0


def test_rollouts_whose_backwards_interleave_keep_their_own_last_segment():
    # the forward records its last checkpoint segment into a tape the hierarchy keeps for the
    # backward; a second rollout of the same length in between overwrites that tape, so the first
    # rollout's backward must recompute its last segment: every gradient equals the one its
    # rollout gets alone
    import torch
    from paper_1808_02638_gb300.adjoint import rollout
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 32
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = inputs.amr_levels(run, n, 4, [(0.2, 0.45)], [31])
    r2 = inputs.smooth_field(27, n, n, 0.5, 2.0, sigma=3.0)
    k2 = inputs.smooth_field(28, n, n, 1.0, 8.0, sigma=3.0)
    qa = [inputs.init_q(run, lev) for lev in run.levels]
    qb = [0.5 * a for a in qa]
    rho = [inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(run.levels)]
    K = [inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(run.levels)]
    H = Hierarchy([run], [qa], [rho], [K])

    def start(q):
        tq, tr, tk = _tensors(H, [q], "q"), _tensors(H, [rho], "c"), _tensors(H, [K], "c")
        outs = rollout(H, tq, tr, tk, ncoarse=5, every=2)
        return tq + tr + tk, _receiver_J(H, outs, run.levels[0], (18, 10, 6))

    def grads(ts):
        torch.cuda.synchronize()
        return [t.grad.clone() for t in ts]

    alone = []
    for q in (qa, qb):
        ts, J = start(q)
        J.backward()
        alone.append(grads(ts))
    ta, Ja = start(qa)
    tb, Jb = start(qb)   # overwrites the tape of a's last segment
    Jb.backward()
    Ja.backward()
    for got, want in ((grads(ta), alone[0]), (grads(tb), alone[1])):
        for a, b in zip(got, want):
            assert float((a - b).abs().max()) <= 1e-12 * max(float(b.abs().max()), 1e-300)
    assert H.sync_status() == 0


@pytest.mark.parametrize("tiling", [(32, 32, 1, 256), (32, 32, 0, 512), (32, 16, 1, 256), (32, 16, 2, 256),
                                    (16, 16, 1, 128)])
def test_recorded_adjoint_matches_oracle_for_every_tiling(tiling):
    # the recording step runs with the level's installed tiling (each tile writes the tape
    # entries of the cells it owns), the tape adjoint with its own 16 x 16 tiles: for every
    # tiling the autotuner can install, the gradient of a 64^2 two-level cell-wise rollout
    # (checkpoints every 2 of 3 coarse steps) equals the oracle's reverse mode
    import torch
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.adjoint import rollout
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 64
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = inputs.amr_levels(run, n, 4, [(0.2, 0.45)], [77])
    r2 = inputs.smooth_field(27, n, n, 0.5, 2.0, sigma=5.0)
    k2 = inputs.smooth_field(28, n, n, 1.0, 8.0, sigma=5.0)
    q = [inputs.init_q(run, lev) for lev in run.levels]
    rho = [inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(run.levels)]
    K = [inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(run.levels)]
    H = Hierarchy([run], [q], [rho], [K], tiling=tiling)
    tq, tr, tk = _tensors(H, [q], "q"), _tensors(H, [rho], "c"), _tensors(H, [K], "c")
    box = (40, 24, 8)
    outs = rollout(H, tq, tr, tk, ncoarse=3, every=2)
    J = _receiver_J(H, outs, run.levels[0], box)
    J.backward()
    torch.cuda.synchronize()

    def final_adjoint(qs):
        lam = [np.zeros_like(a) for a in qs]
        i0, j0, nn = box
        v = inputs.box_view(qs[0], 0, n, n, 3)
        inputs.box_view(lam[0], 0, n, n, 3)[0, M + j0:M + j0 + nn, M + i0:M + i0 + nn] = \
            2 * v[0, M + j0:M + j0 + nn, M + i0:M + i0 + nn]
        return lam

    O = OracleHierarchy(run, q, rho, K)
    gq, gr, gk = O.gradient(3, final_adjoint)
    _compare([t.grad.cpu().numpy() for t in tq], gq, 1e-10)
    _compare([t.grad.cpu().numpy() for t in tr], gr, 1e-10)
    _compare([t.grad.cpu().numpy() for t in tk], gk, 1e-10)
    assert H.sync_status() == 0


@pytest.mark.parametrize("nlev", [1, 2])
def test_adjoint_matches_oracle_reverse_mode(nlev):
    import torch
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.adjoint import rollout
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 32
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    if nlev == 1:
        run.levels = [inputs.Level(n, n, 2 / n, 2 / n, [(0, 0, n, n)])]
    else:
        run.levels = inputs.amr_levels(run, n, 4, [(0.2, 0.45)], [31])
    r2 = inputs.smooth_field(21, n, n, 0.5, 2.0, sigma=3.0)
    k2 = inputs.smooth_field(22, n, n, 1.0, 8.0, sigma=3.0)
    q = [inputs.init_q(run, lev) for lev in run.levels]
    rho = [inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(run.levels)]
    K = [inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(run.levels)]
    nsteps = 6 if nlev == 1 else 2
    box = (18, 10, 6)
    H = Hierarchy([run], [q], [rho], [K])
    tq, tr, tk = _tensors(H, [q], "q"), _tensors(H, [rho], "c"), _tensors(H, [K], "c")
    outs = rollout(H, tq, tr, tk, ncoarse=nsteps, every=4)
    J = _receiver_J(H, outs, run.levels[0], box)
    J.backward()
    torch.cuda.synchronize()

    def final_adjoint(qs):
        lam = [np.zeros_like(a) for a in qs]
        i0, j0, nn = box
        v = inputs.box_view(qs[0], 0, n, n, 3)
        inputs.box_view(lam[0], 0, n, n, 3)[0, M + j0:M + j0 + nn, M + i0:M + i0 + nn] = \
            2 * v[0, M + j0:M + j0 + nn, M + i0:M + i0 + nn]
        return lam

    O = OracleHierarchy(run, q, rho, K)
    gq, gr, gk = O.gradient(nsteps, final_adjoint)
    assert float(J) == pytest.approx(float((inputs.box_view(O.q[0], 0, n, n, 3)
                                            [0, M + 10:M + 16, M + 18:M + 24] ** 2).sum()), rel=1e-11)
    _compare([t.grad.cpu().numpy() for t in tq], gq, 1e-10)
    _compare([t.grad.cpu().numpy() for t in tr], gr, 1e-10)
    _compare([t.grad.cpu().numpy() for t in tk], gk, 1e-10)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 2, 2), (2, 0, 2, 2)])
def test_fused_ghost_adjoint_equals_the_separate_fill_adjoint(bc):
    # the step adjoint that sends each same-level / boundary ghost's adjoint to its source cell
    # (H.pull) against the step adjoint followed by the ghost-fill adjoint: the same map, summed
    # in another order; level 0 in four boxes so that it has same-level ghosts too
    import torch
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.adjoint import rollout
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 32
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=bc)
    run.levels = inputs.amr_levels(run, n, 4, [(0.2, 0.45)], [31])
    run.levels[0] = inputs.Level(n, n, 2 / n, 2 / n, inputs.uniform_tiling(n, n, 16, 16))
    r2 = inputs.smooth_field(23, n, n, 0.5, 2.0, sigma=3.0)
    k2 = inputs.smooth_field(24, n, n, 1.0, 8.0, sigma=3.0)
    q = [inputs.init_q(run, lev) for lev in run.levels]
    rho = [inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(run.levels)]
    K = [inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(run.levels)]
    H = Hierarchy([run], [q], [rho], [K])
    grads = []
    for pull in (True, False):
        H.pull = pull
        tq, tr, tk = _tensors(H, [q], "q"), _tensors(H, [rho], "c"), _tensors(H, [K], "c")
        outs = rollout(H, tq, tr, tk, ncoarse=4, every=2)
        # receiver on the first box of level 0 (cells 2..9 of its 16 x 16 interior)
        v = outs[0][:3 * 20 * 20].view(3, 20, 20)
        J = (v[0, M + 2:M + 10, M + 2:M + 10] ** 2).sum()
        J.backward()
        torch.cuda.synchronize()
        grads.append([t.grad.clone() for t in tq + tr + tk] + [J.detach().clone()])
    assert torch.equal(grads[0][-1], grads[1][-1])
    for a, b in zip(grads[0][:-1], grads[1][:-1]):
        assert float((a - b).abs().max()) <= 1e-12 * max(float(b.abs().max()), 1e-300)
    assert max(float(g.abs().max()) for g in grads[0][:-1]) > 0.0
    lam = torch.zeros_like(H.q[0][0])
    with pytest.raises(claw.ClawError):
        claw.claw_level_advance_adjoint(H.ctx, 0, H.q[0][0], lam, lam, H.aux[0], torch.zeros_like(H.aux[0]), H.dt, 8)


@pytest.mark.parametrize("medium", ["uniform", "cellwise"])
def test_level_step_function_matches_oracle_step_adjoint(medium):
    # one level-step as a torch.autograd.Function: the gradient of <w, q_new> (w on interiors)
    # with respect to q_old (all cells), rho and K equals the oracle's reverse mode of its step
    import torch
    import oracle
    from paper_1808_02638_gb300.adjoint import LevelStep
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 40
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = [inputs.Level(n, n, 2 / n, 2 / n, [(0, 0, n, n)])]
    lev = run.levels[0]
    q = inputs.init_q(run, lev) + 0.05 * inputs.uniform(41, inputs.init_q(run, lev).size)
    r2 = inputs.smooth_field(42, n, n, 0.5, 2.0, sigma=3.0)
    k2 = inputs.smooth_field(43, n, n, 1.0, 8.0, sigma=3.0)
    rho_p, K_p = inputs.coef_pool(lev, r2, 1), inputs.coef_pool(lev, k2, 1)
    if medium == "uniform":
        H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
        rho_p = inputs.const_pool(lev, 1.0)
        K_p = inputs.const_pool(lev, 4.0)
    else:
        H = Hierarchy([run], [[q]], [[rho_p]], [[K_p]])
    H.init_dt()
    dt = H.dt.clone()
    dev = H.q[0][0].device
    tq = torch.zeros_like(H.q[0][0])
    tq[:q.size] = torch.from_numpy(q)
    tq.requires_grad_(True)
    w = np.zeros_like(q)
    inputs.box_view(w, 0, n, n, 3)[:, M:-M, M:-M] = inputs.uniform(44, 3 * n * n).reshape(3, n, n) - 0.5
    tw = torch.zeros_like(tq.detach())
    tw[:w.size] = torch.from_numpy(w)
    if medium == "uniform":
        out = LevelStep.apply(H, 0, dt, tq)
    else:
        tr = torch.ones_like(H.rho[0]); tr[:rho_p.size] = torch.from_numpy(rho_p); tr.requires_grad_(True)
        tk = torch.ones_like(H.K[0]); tk[:K_p.size] = torch.from_numpy(K_p); tk.requires_grad_(True)
        out = LevelStep.apply(H, 0, dt, tq, tr, tk)
    (out * tw).sum().backward()
    qb = inputs.box_view(q, 0, n, n, 3)
    rb = inputs.box_view(rho_p, 0, n, n, 1)[0]
    kb = inputs.box_view(K_p, 0, n, n, 1)[0]
    lb = inputs.box_view(w, 0, n, n, 3)
    lq, gr, gk = oracle.step_adjoint(qb, rb, kb, lb, lev.dx, lev.dy, float(dt[0]), run.order, run.transverse,
                                     run.limiter)
    got = inputs.box_view(tq.grad.cpu().numpy()[:q.size], 0, n, n, 3)
    assert np.abs(got - lq).max() <= 1e-11 * np.abs(lq).max()
    if medium == "cellwise":
        gotr = inputs.box_view(tr.grad.cpu().numpy()[:rho_p.size], 0, n, n, 1)[0]
        gotk = inputs.box_view(tk.grad.cpu().numpy()[:K_p.size], 0, n, n, 1)[0]
        assert np.abs(gotr - gr).max() <= 1e-10 * np.abs(gr).max()
        assert np.abs(gotk - gk).max() <= 1e-10 * np.abs(gk).max()


def test_heterogeneous_receiver_gradient_matches_finite_differences(record_property):
    # 256^2, rho ~ U[0.5,2], K ~ U[1,8] smoothed (sigma 8 cells), radial pulse, J = sum p^2 over
    # the 16 x 16 receiver box after 400 steps, checkpoints every 20; central differences
    # (h = 1e-6, time steps frozen) along 8 seeded smooth directions for each of q0, rho, K.
    # The directions have amplitude 0.1 of the fields' unit scale (q0: windowed to the ring and
    # even in x, y; rho: 0.025; K: 0.1): the limited scheme is piecewise smooth and a central
    # difference that straddles a limiter branch point errs in proportion to the perturbation,
    # about 2e-6 relative at an amplitude of 1e-6 and 2e-7 at 1e-7 over 400 steps.
    # Error measure: || adjoint . d - FD ||_2 / || FD ||_2 over the 8 directions.
    import torch
    from paper_1808_02638_gb300.adjoint import rollout
    from paper_1808_02638_gb300.solver import Hierarchy
    n, nsteps = 256, 400
    run, r2, k2 = inputs.config3(n)
    lev = run.levels[0]
    q = inputs.init_q(run, lev)
    rho, K = inputs.coef_pool(lev, r2, 1), inputs.coef_pool(lev, k2, 1)
    box = inputs.receiver_box(n)
    H = Hierarchy([run], [[q]], [[rho]], [[K]])
    tq, tr, tk = _tensors(H, [[q]], "q"), _tensors(H, [[rho]], "c"), _tensors(H, [[K]], "c")
    outs = rollout(H, tq, tr, tk, ncoarse=nsteps, every=20)
    J = _receiver_J(H, outs, lev, box)
    J.backward()
    H.init_dt()
    dt = H.dt.clone()
    g = {"q": tq[0].grad, "rho": tr[0].grad, "K": tk[0].grad}
    win = inputs.annulus_window(n, n)

    def pad(f, ref, ncomp):
        a = np.zeros(ref.numel())
        inputs.box_view(a, 0, n, n, ncomp)[0, M:-M, M:-M] = f
        return torch.from_numpy(a).to(ref.device)

    def Jof(d, h):
        with torch.no_grad():
            x = {k: v + h * d[k] if k in d else v for k, v in (("q", tq[0]), ("rho", tr[0]), ("K", tk[0]))}
            o = rollout(H, [x["q"]], [x["rho"]], [x["K"]], ncoarse=nsteps, every=nsteps, dt=dt)
            return float(_receiver_J(H, o, lev, box))

    h = 1e-6
    report, per_direction = {}, {}
    for name in ("q", "rho", "K"):
        ad, fd = [], []
        for seed in range(3100, 3108):
            if name == "q":
                d = {"q": pad(0.1 * win * inputs.fourier_field(seed, n, n, even=True), tq[0], 3)}
            elif name == "rho":
                d = {"rho": pad(0.025 * inputs.fourier_field(seed + 1000, n, n), tr[0], 1)}
            else:
                d = {"K": pad(0.1 * inputs.fourier_field(seed + 2000, n, n), tr[0], 1)}
            fd.append((Jof(d, h) - Jof(d, -h)) / (2 * h))
            ad.append(float((g[name] * d[name]).sum()))
        ad, fd = np.array(ad), np.array(fd)
        report[name] = float(np.linalg.norm(ad - fd) / np.linalg.norm(fd))
        per_direction[name] = [float(v) for v in np.abs(ad - fd) / np.abs(fd)]
    record_property("fd_relative_error", report)
    record_property("fd_relative_error_per_direction", per_direction)
    print("FD aggregate", report, "per direction", per_direction)
    assert all(v <= 1e-6 for v in report.values()), report
    assert all(max(v) <= 1e-5 for v in per_direction.values()), per_direction

// claw_api.cu -- the C ABI of libclaw.so (include/claw.h): context, host-side validation of
// the box sets of Sec. 2.2 and the launches of the level-step, ghost fill, averaging, conservation
// fix, adjoint and packing kernels.  The level tables are built in claw_tables.cu and the regrid's
// clustering in claw_clustering.cu.
#include "claw_host.h"

using namespace claw_host;

namespace {

StepArgs make_args(claw_ctx* ctx, int L, const double* q_old, double* q_new, const double* aux,
                   const double* dt, double* smax)
{
    const LevelDev& d = ctx->lev[L];
    StepArgs a;
    a.patches = d.patches;
    a.tiles = d.tiles;
    a.tmaps = nullptr;
    a.ntiles = d.ntiles;
    a.tcum = d.tcum;   // set for walking levels only (not a cell-wise medium)
    a.qold = q_old;
    a.qnew = q_new;
    a.aux = aux;
    a.dt = dt;
    a.smax = smax;
    a.err = ctx->err;
    a.order = ctx->order;
    a.transverse = ctx->transverse;
    a.rho0 = ctx->rho0;
    a.K0 = ctx->K0;
    a.grav = ctx->grav;
    a.swe = ctx->kind() == KIND_SWE;
    a.wait_polls = ctx->wait_polls;
    return a;
}

int check_step_args(claw_ctx* ctx, int L, const double* q_old, const double* q_new, const double* aux,
                    const double* dt, const double* smax)
{
    if (!ctx) return CLAW_EINVAL;
    if (L < 0 || L >= CLAW_MAXLEV) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    if (!q_old || !q_new || !dt || !smax || q_old == q_new) return CLAW_EINVAL;
    if (ctx->kind() == KIND_CELLWISE && !aux) return CLAW_EINVAL;
    return CLAW_OK;
}

}  // namespace

extern "C" {


int claw_create(claw_ctx** out, const claw_problem* runs, int32_t nruns, int32_t device)
{
    if (!out || !runs || nruns <= 0) return CLAW_EINVAL;
    *out = nullptr;
    for (int r = 0; r < nruns; ++r) {
        const claw_problem& p = runs[r];
        if (p.nlev < 1 || p.nlev > CLAW_MAXLEV || p.nx0 < 1 || p.ny0 < 1 || !(p.xhi > p.xlo) ||
            !(p.yhi > p.ylo) || !(p.cfl > 0) || p.limiter < 0 || p.limiter > 4 || p.order < 1 ||
            p.order > 2 || p.transverse < 0 || p.transverse > 2 || p.medium < 0 || p.medium > 1)
            return CLAW_EINVAL;
        for (int s = 0; s < 4; ++s)
            if (p.bc[s] < 0 || p.bc[s] > 2) return CLAW_EINVAL;
        if ((p.bc[0] == CLAW_BC_PERIODIC) != (p.bc[1] == CLAW_BC_PERIODIC) ||
            (p.bc[2] == CLAW_BC_PERIODIC) != (p.bc[3] == CLAW_BC_PERIODIC))
            return CLAW_EINVAL;
        for (int l = 1; l < p.nlev; ++l)
            if (p.ratio[l] < 2 || p.ratio[l] > 16) return CLAW_EINVAL;
        if (p.system != CLAW_SYS_ACOUSTICS && p.system != CLAW_SYS_SHALLOW_WATER) return CLAW_EINVAL;
        if (p.system == CLAW_SYS_SHALLOW_WATER && (p.medium != 0 || !(p.grav > 0) || !std::isfinite(p.grav)))
            return CLAW_EINVAL;
        if (p.system == CLAW_SYS_ACOUSTICS && p.medium == 0 && !(p.rho0 > 0 && p.K0 > 0)) return CLAW_EINVAL;
        if (p.limiter != runs[0].limiter || p.order != runs[0].order || p.transverse != runs[0].transverse ||
            p.medium != runs[0].medium || p.system != runs[0].system ||
            (p.system == CLAW_SYS_SHALLOW_WATER && p.grav != runs[0].grav) ||
            (p.system == CLAW_SYS_ACOUSTICS && p.medium == 0 && (p.rho0 != runs[0].rho0 || p.K0 != runs[0].K0)))
            return CLAW_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return CLAW_ECUDA;
    claw_ctx* c = new (std::nothrow) claw_ctx;
    if (!c) return CLAW_ENOMEM;
    DevGuard g(device);
    c->device = device;
    c->nruns = nruns;
    c->runs.assign(runs, runs + nruns);
    c->limiter = runs[0].limiter;
    c->order = runs[0].order;
    c->transverse = runs[0].transverse;
    c->medium = runs[0].medium;
    c->rho0 = runs[0].rho0;
    c->K0 = runs[0].K0;
    c->system = runs[0].system;
    c->grav = runs[0].system == CLAW_SYS_SHALLOW_WATER ? runs[0].grav : 0.0;
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
    std::vector<double> minh(CLAW_MAXLEV * nruns, 0.0), cfl(nruns);
    for (int r = 0; r < nruns; ++r) {
        cfl[r] = runs[r].cfl;
        for (int L = 0; L < runs[r].nlev; ++L)
            minh[L * nruns + r] = std::min(level_dx(runs[r], L), level_dy(runs[r], L));
    }
    if (cudaMalloc(&c->err, sizeof(int)) != cudaSuccess || cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->done, sizeof(unsigned)) != cudaSuccess || cudaMemset(c->done, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&c->minh, minh.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->cflv, cfl.size() * sizeof(double)) != cudaSuccess ||
        cudaMemcpy(c->minh, minh.data(), minh.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->cflv, cfl.data(), cfl.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        claw_destroy(c);
        return CLAW_ENOMEM;
    }
    *out = c;
    return CLAW_OK;
}

void claw_destroy(claw_ctx* ctx)
{
    if (!ctx) return;
    {
        DevGuard g(ctx->device);
        cudaDeviceSynchronize();
        for (int L = 0; L < CLAW_MAXLEV; ++L) {
            free_level(ctx, L);
            free_arena(ctx->lev[L].tables);
            free_arena(ctx->lev[L].tiletab);
            free_arena(ctx->lev[L].coeftab);
        }
        free_arena(ctx->scratch);
        cudaFree(ctx->xgrid);
        cudaFree(ctx->err);
        cudaFree(ctx->done);
        cudaFree(ctx->minh);
        cudaFree(ctx->cflv);
    }
    delete ctx;
}

int claw_set_level(claw_ctx* ctx, int32_t L, const claw_box* boxes, int32_t nboxes)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || nboxes < 0 || (nboxes > 0 && !boxes)) return CLAW_EINVAL;
    if (L > 0 && !ctx->set[L - 1]) return CLAW_ESTATE;
    DevGuard g(ctx->device);
    for (int l = L; l < CLAW_MAXLEV; ++l)
        if (ctx->set[l]) free_level(ctx, l);
    LevelDev& d = ctx->lev[L];
    d.boxes.assign(boxes, boxes + nboxes);
    d.nboxes = nboxes;
    d.ratio = 1;
    bool even = true;
    // validation: inside the domain, aligned to the coarser level, sizes, offsets
    for (int n = 0; n < nboxes; ++n) {
        const claw_box& b = boxes[n];
        if (b.run < 0 || b.run >= ctx->nruns) return CLAW_EINVAL;
        const claw_problem& p = ctx->runs[b.run];
        if (L >= p.nlev) return CLAW_EINVAL;
        if (L > 0) {
            if (d.ratio != 1 && d.ratio != p.ratio[L]) return CLAW_EINVAL;   // one ratio per level
            d.ratio = p.ratio[L];
        }
        const int NX = level_nx(p, L), NY = level_ny(p, L);
        if (b.nx < 1 || b.ny < 1 || b.nx > 4096 || b.ny > 4096 || b.ilo < 0 || b.jlo < 0 ||
            b.ilo + b.nx > NX || b.jlo + b.ny > NY || b.qoff < 0 || b.coff < 0)
            return CLAW_EINVAL;
        if (L > 0) {
            const int r = p.ratio[L];
            if (b.ilo % r || b.jlo % r || b.nx % r || b.ny % r) return CLAW_EINVAL;
        }
        if ((b.nx & 1) || (b.qoff & 1)) even = false;
    }
    // the boxes of each run bucketed (kept for the table builds of this level and the next),
    // and disjoint: boxes that overlap share a bucket
    {
        std::vector<std::vector<int>> sel(ctx->nruns);
        for (int n = 0; n < nboxes; ++n) sel[boxes[n].run].push_back(n);
        std::vector<Locator>& loc = ctx->loc[L];
        loc.assign(ctx->nruns, Locator{});
        for (int q = 0; q < ctx->nruns; ++q)
            if (L < ctx->runs[q].nlev)
                loc[q].build(&d.boxes, sel[q], level_nx(ctx->runs[q], L), level_ny(ctx->runs[q], L));
        for (int q = 0; q < ctx->nruns; ++q) {
            const Locator& lq = loc[q];
            for (size_t k = 0; k + 1 < lq.start.size(); ++k)
                for (int t = lq.start[k]; t < lq.start[k + 1]; ++t)
                    for (int u = t + 1; u < lq.start[k + 1]; ++u) {
                        const claw_box& b = boxes[lq.items[t]];
                        const claw_box& o = boxes[lq.items[u]];
                        if (b.ilo < o.ilo + o.nx && o.ilo < b.ilo + b.nx && b.jlo < o.jlo + o.ny &&
                            o.jlo < b.jlo + b.ny) {
                            loc.clear();
                            return CLAW_EINVAL;
                        }
                    }
        }
    }
    // patch table
    d.hpatches.resize(nboxes);
    for (int n = 0; n < nboxes; ++n) {
        const claw_box& b = boxes[n];
        const claw_problem& p = ctx->runs[b.run];
        PatchDev P;
        P.qoff = b.qoff;
        P.aoff = (long long)CLAW_NAUX * b.coff;
        P.nx = b.nx;
        P.ny = b.ny;
        P.run = b.run;
        P.ring = -1;
        P.interp = 0;
        P.dxinv = 1.0 / level_dx(p, L);
        P.dyinv = 1.0 / level_dy(p, L);
        P.dtscale = 1.0;
        for (int l = 1; l <= L; ++l) P.dtscale /= p.ratio[l];
        d.hpatches[n] = P;
    }
    ctx->tma_ok[L] = even;
    if (!d.tiling_set) {   // a level's first boxes; later calls keep the tiling chosen for it
        d.tx = ctx->kind() == KIND_SWE ? 16 : 32;
        d.ty = ctx->kind() == KIND_SWE ? 16 : 32;
        d.nt = 0;
        d.staging = even ? 1 : 0;
    } else if (!even) {
        d.staging = 0;
    }
    GhostTables gt;
    std::vector<AvgRect> avg;
    int rc = build_ghost_tables(ctx, L, gt, true);
    if (rc) return rc;
    d.ring_ok = gt.ring_ok;
    for (auto& P : d.hpatches)
        if (!d.ring_ok) P.ring = -1;
    {   // each box's first interpolated cell in the concatenated table (box order)
        long long c = 0;
        for (int n = 0; n < d.nboxes; ++n) {
            d.hpatches[n].interp = (int)c;
            c += (long long)gt.per[n].cells.size();
        }
    }
    // every table stays alive until pack.commit reads it
    ArenaPack pack;
    if (d.ring_ok)
        pack.add_parts(&d.ring, d.nboxes, [&](int n) -> const std::vector<longlong2>& { return gt.per[n].ring; });
    pack.add(&d.copy_start, gt.start);
    d.ncopy_blocks = gt.start.empty() ? 0 : (int)gt.start.size() - 1;
    d.max_rows = 0;
    for (const claw_box& b : d.boxes) d.max_rows = std::max(d.max_rows, b.ny + 4);
    // packed interiors: box order, 3 planes of nx x ny each
    std::vector<long long> poff(d.nboxes);
    long long o = 0;
    for (int n = 0; n < d.nboxes; ++n) {
        poff[n] = o;
        o += 3LL * d.boxes[n].nx * d.boxes[n].ny;
    }
    d.packed = o;
    pack.add(&d.poff, poff);
    // the boxes as writers into the level's flag grid
    std::vector<FlagBox> fb(d.nboxes);
    for (int n = 0; n < d.nboxes; ++n) {
        const claw_box& b = d.boxes[n];
        const int NX = level_nx(ctx->runs[b.run], L);
        fb[n].qoff = b.qoff;
        fb[n].goff = flag_grid_offset(ctx, L, b.run) + (long long)b.jlo * NX + b.ilo;
        fb[n].nx = b.nx;
        fb[n].ny = b.ny;
        fb[n].pitch = NX;
        fb[n].pad = 0;
    }
    pack.add(&d.flagboxes, fb);
    std::vector<RefluxRec> rrec;
    std::vector<int> rgroup;
    if (L > 0) {
        build_avg_tables(ctx, L, avg);
        build_reflux_tables(ctx, L, rrec, rgroup);
        pack.add(&d.reflux, rrec);
        pack.add(&d.reflux_group, rgroup);
        d.nreflux = (int)rrec.size();
        d.nreflux_groups = rgroup.empty() ? 0 : (int)rgroup.size() - 1;
    }
    pack.add(&d.patches, d.hpatches);
    pack.add_parts(&d.copies, d.nboxes, [&](int n) -> const std::vector<CopyRect>& { return gt.per[n].rects; });
    pack.add_parts(&d.interps, d.nboxes, [&](int n) -> const std::vector<InterpCell>& { return gt.per[n].cells; });
    pack.add(&d.avgs, avg);
    if ((rc = pack.commit(d.tables))) return rc;
    d.ncopy = (int)gt.nrects;
    d.ninterp = (int)gt.ncells;
    d.navg = (int)avg.size();
    // a cell-wise medium fills its coefficient pools' ghosts: those tables are built now, a
    // uniform medium builds them on first use
    if (ctx->medium && (rc = build_coef_tables(ctx, L))) return rc;
    ctx->set[L] = true;
    rc = build_tiles(ctx, L);
    if (rc) {
        ctx->set[L] = false;
        return rc;
    }
    return CLAW_OK;
}

int claw_limiter_eval(int32_t limiter, int64_t n, const double* a, const double* b, double* out, void* stream)
{
    if (limiter < CLAW_LIM_NONE || limiter > CLAW_LIM_MC || n < 0 || (n > 0 && (!a || !b || !out)))
        return CLAW_EINVAL;
    return cuda_rc(launch_limiter_eval(limiter, n, a, b, out, (cudaStream_t)stream));
}

int claw_set_wait_limit(claw_ctx* ctx, uint32_t polls)
{
    if (!ctx) return CLAW_EINVAL;
    ctx->wait_polls = polls;
    return CLAW_OK;
}

int claw_set_tiling(claw_ctx* ctx, int32_t L, int32_t tx, int32_t ty, int32_t staging, int32_t threads)
{
    if (!valid_level(ctx, L)) return CLAW_EINVAL;
    const bool shape_ok =
        ctx->kind() == KIND_SWE
            ? (tx == 16 && ty == 16 && (threads == 0 || threads == 256)) ||
                  (tx == 32 && ty == 16 && (threads == 0 || threads == 512))
            : (tx == 32 && ty == 32 && (threads == 0 || threads == 256 || threads == 512)) ||
                  (tx == 32 && ty == 16 && (threads == 0 || threads == 256)) ||
                  (tx == 16 && ty == 16 && (threads == 0 || threads == 128));
    // staging 2 (one bulk-copy buffer, three CTAs per SM) exists for the acoustics 32x16 tiles
    const bool staging2_ok = ctx->kind() != KIND_SWE && tx == 32 && ty == 16 && (threads == 0 || threads == 256);
    if (!shape_ok || staging < 0 || staging > 2 || (staging == 2 && !staging2_ok) ||
        (staging >= 1 && !ctx->tma_ok[L]))
        return CLAW_EINVAL;
    DevGuard g(ctx->device);
    LevelDev& d = ctx->lev[L];
    d.staging = staging;
    d.nt = threads;
    d.tiling_set = true;
    if (d.tx == tx && d.ty == ty) return CLAW_OK;
    d.tx = tx;
    d.ty = ty;
    return build_tiles(ctx, L);
}

int claw_set_tile_walk(claw_ctx* ctx, int32_t L, int32_t walk)
{
    if (!valid_level(ctx, L) || walk < -1 || walk > 1 || (walk > 0 && ctx->kind() == KIND_CELLWISE)) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    LevelDev& d = ctx->lev[L];
    if (d.walk == walk) return CLAW_OK;
    d.walk = walk;
    return build_tiles(ctx, L);
}

int claw_medium_aux(claw_ctx* ctx, int32_t L, const double* rho, const double* K, double* aux, void* stream)
{
    if (!valid_level(ctx, L) || !rho || !K || !aux) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[L];
    ctx->launches += d.nboxes > 0;
    return cuda_rc(launch_medium_aux(d.patches, d.nboxes, d.max_rows, rho, K, aux, (cudaStream_t)stream));
}

int claw_medium_aux_adjoint(claw_ctx* ctx, int32_t L, const double* rho, const double* K, const double* g_aux,
                            double* g_rho, double* g_K, void* stream)
{
    if (!valid_level(ctx, L) || !rho || !K || !g_aux || !g_rho || !g_K) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[L];
    ctx->launches += d.nboxes > 0;
    return cuda_rc(launch_medium_aux_adjoint(d.patches, d.nboxes, d.max_rows, rho, K, g_aux, g_rho, g_K, (cudaStream_t)stream));
}

int claw_fill_ghost(claw_ctx* ctx, int32_t L, double* q, const double* qc_old, const double* qc_new, double tau,
                    void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !q) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    const LevelDev& d = ctx->lev[L];
    if (d.ninterp > 0 && (!qc_old || !qc_new || !(tau >= 0.0 && tau <= 1.0))) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = d.ncopy ? launch_fill_copy(d.copies, d.copy_start, d.ncopy_blocks, q, s) : cudaSuccess;
    ctx->launches += d.ncopy > 0;
    if (e == cudaSuccess) {
        e = launch_fill_interp(d.interps, d.ninterp, q, qc_old, qc_new, tau, s);
        ctx->launches += d.ninterp > 0;
    }
    return cuda_rc(e);
}

int claw_fill_ghost_interp(claw_ctx* ctx, int32_t L, double* q, const double* qc_old, const double* qc_new,
                           double tau, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !q) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    const LevelDev& d = ctx->lev[L];
    if (d.ninterp == 0) return CLAW_OK;
    if (!qc_old || !qc_new || !(tau >= 0.0 && tau <= 1.0)) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    ctx->launches += 1;
    return cuda_rc(launch_fill_interp(d.interps, d.ninterp, q, qc_old, qc_new, tau, (cudaStream_t)stream));
}

int claw_fill_ghost_coef(claw_ctx* ctx, int32_t L, double* a, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !a) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    DevGuard g(ctx->device);
    int rc = ensure_coef_tables(ctx, L, stream);
    if (rc) return rc;
    const LevelDev& d = ctx->lev[L];
    ctx->launches += d.nccopy > 0;
    return cuda_rc(d.nccopy ? launch_fill_copy(d.ccopies, d.ccopy_start, d.nccopy_blocks, a, (cudaStream_t)stream, 1)
                            : cudaSuccess);
}

int claw_fill_ghost_coef_adjoint(claw_ctx* ctx, int32_t L, double* g, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !g) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    DevGuard gd(ctx->device);
    int rc = ensure_coef_tables(ctx, L, stream);
    if (rc) return rc;
    const LevelDev& d = ctx->lev[L];
    ctx->launches += d.nccopy > 0;
    return cuda_rc(d.nccopy ? launch_fill_copy_adjoint(d.ccopies, d.ccopy_start, d.nccopy_blocks, g, (cudaStream_t)stream, 1)
                            : cudaSuccess);
}

int claw_fill_ghost_interp_adjoint(claw_ctx* ctx, int32_t L, double* lam, double* lco, double* lcn,
                                   const double* qc_old, const double* qc_new, double tau, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !lam) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    const LevelDev& d = ctx->lev[L];
    if (d.ninterp > 0 && (!qc_old || !qc_new)) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    ctx->launches += d.ninterp > 0;
    return cuda_rc(launch_fill_interp_adjoint(d.interps, d.ninterp, lam, lco, lcn, qc_old, qc_new, tau,
                                              (cudaStream_t)stream));
}

int claw_fill_ghost_adjoint(claw_ctx* ctx, int32_t L, double* lam, double* lco, double* lcn, const double* qc_old,
                            const double* qc_new, double tau, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !lam) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    const LevelDev& d = ctx->lev[L];
    if (d.ninterp > 0 && (!qc_old || !qc_new)) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // interpolated ghosts first (they read coarse cells only), then the copies
    cudaError_t e = launch_fill_interp_adjoint(d.interps, d.ninterp, lam, lco, lcn, qc_old, qc_new, tau, s);
    ctx->launches += d.ninterp > 0;
    if (e == cudaSuccess && d.ncopy) {
        e = launch_fill_copy_adjoint(d.copies, d.copy_start, d.ncopy_blocks, lam, s);
        ctx->launches += 1;
    }
    return cuda_rc(e);
}

int claw_cfl_max(claw_ctx* ctx, int32_t L, const double* aux, double* smax, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !smax) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    if (ctx->kind() == KIND_SWE || (ctx->medium == 1 && !aux)) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_cfl_max(ctx->lev[L].patches, ctx->lev[L].nboxes, ctx->lev[L].max_rows, ctx->medium,
                                   std::sqrt(ctx->K0 / ctx->rho0), aux, smax, s);
    ctx->launches += ctx->lev[L].nboxes > 0;
    return cuda_rc(e);
}

int claw_cfl_max_state(claw_ctx* ctx, int32_t L, const double* q, double* smax, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !q || !smax) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    if (ctx->kind() != KIND_SWE) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[L];
    cudaError_t e = launch_cfl_max_state(d.patches, d.nboxes, d.max_rows, ctx->grav, q, smax, (cudaStream_t)stream);
    ctx->launches += d.nboxes > 0;
    return cuda_rc(e);
}

int claw_dt_update(claw_ctx* ctx, int32_t L, double* smax, double* dt, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !smax || !dt) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    ctx->launches += 1;
    if (L >= CLAW_MAXLEV) return CLAW_EINVAL;
    return cuda_rc(launch_dt_update(ctx->minh + (size_t)L * ctx->nruns, ctx->cflv, ctx->nruns, smax, dt, ctx->err,
                                    (cudaStream_t)stream));
}

int claw_level_step(claw_ctx* ctx, int32_t L, const double* q_old, double* q_new, const double* aux,
                    const double* dt, double* smax, void* stream)
{
    int rc = check_step_args(ctx, L, q_old, q_new, aux, dt, smax);
    if (rc) return rc;
    DevGuard g(ctx->device);
    LevelDev& d = ctx->lev[L];
    if (d.ntiles == 0) return CLAW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    StepArgs a = make_args(ctx, L, q_old, q_new, aux, dt, smax);
    int staging = d.staging;
    if (staging >= 1) {
        a.tmaps = get_tmaps(ctx, L, q_old, s);
        if (!a.tmaps) staging = 0;   // no descriptor (e.g. first use inside a graph capture)
    }
    const int per_sm = step_max_ctas_per_sm(ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, false, false, false,
                                            a.tcum != nullptr);
    if (per_sm <= 0) return CLAW_ECUDA;
    const int grid = std::min(d.ntiles, per_sm * ctx->nsm);
    ctx->launches += 1;
    return cuda_rc(launch_step(a, ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, grid, s));
}

static int level_advance(claw_ctx* ctx, int32_t L, const double* q_old, double* q_new, const double* aux, double* dt,
                         double* smax, int32_t flags, const double* qc_old, const double* qc_new, double tau,
                         bool interp, void* stream, const claw_fill_job* jobs = nullptr, int njobs = 0)
{
    int rc = check_step_args(ctx, L, q_old, q_new, aux, dt, smax);
    if (rc) return rc;
    if (njobs < 0 || njobs > 2 || (njobs > 0 && !jobs)) return CLAW_EINVAL;
    for (int j = 0; j < njobs; ++j) {
        // a job fills level L's or level L+1's interpolated ghosts: never those of q_old (which
        // the step reads), from coarse states the step does not write
        const claw_fill_job& J = jobs[j];
        if ((J.level != L && J.level != L + 1) || J.level < 1 || J.level >= CLAW_MAXLEV || !ctx->set[J.level])
            return CLAW_EINVAL;
        if (!J.q || !J.qc_old || !J.qc_new || !(J.tau >= 0.0 && J.tau <= 1.0)) return CLAW_EINVAL;
        if (J.q == q_old || J.qc_old == q_new || J.qc_new == q_new || (J.level != L && J.q == q_new))
            return CLAW_EINVAL;
    }
    if (flags & ~(CLAW_ADVANCE_PUSH_GHOSTS | CLAW_ADVANCE_UPDATE_DT | CLAW_ADVANCE_PULL_GHOSTS)) return CLAW_EINVAL;
    if ((flags & CLAW_ADVANCE_PULL_GHOSTS) && !ctx->lev[L].ring_ok) return CLAW_EINVAL;
    LevelDev& d = ctx->lev[L];
    if (interp && d.ninterp > 0 &&
        (!(flags & CLAW_ADVANCE_PULL_GHOSTS) || !qc_old || !qc_new || !(tau >= 0.0 && tau <= 1.0)))
        return CLAW_EINVAL;
    DevGuard g(ctx->device);
    if (d.ntiles == 0) return CLAW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    StepArgs a = make_args(ctx, L, q_old, q_new, aux, dt, smax);
    if (interp && d.ninterp > 0) {
        if (ctx->kind() == KIND_SWE) {   // no fused kernel: the interpolation launch fills them first
            cudaError_t e = launch_fill_interp(d.interps, d.ninterp, const_cast<double*>(q_old), qc_old, qc_new, tau, s);
            ctx->launches += 1;
            if (e != cudaSuccess) return CLAW_ECUDA;
        } else {
            a.interp = d.interps;
            a.cold = qc_old;
            a.cnew = qc_new;
            a.tau = tau;
        }
    }
    if (flags & CLAW_ADVANCE_UPDATE_DT) {
        a.dtupd = 1;
        a.dt_out = dt;
        a.minh = ctx->minh;   // level-0 row
        a.cflv = ctx->cflv;
        a.done = ctx->done;
        a.nruns = ctx->nruns;
    }
    if (flags & CLAW_ADVANCE_PULL_GHOSTS) a.ring = d.ring;
    int staging = d.staging;
    if (staging >= 1) {
        a.tmaps = get_tmaps(ctx, L, q_old, s);
        if (!a.tmaps) staging = 0;
    }
    const int per_sm = step_max_ctas_per_sm(ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, a.ring != nullptr,
                                            false, a.interp != nullptr, a.tcum != nullptr);
    if (per_sm <= 0) return CLAW_ECUDA;
    const int grid = std::min(d.ntiles, per_sm * ctx->nsm);
    for (int j = 0; j < njobs; ++j) {
        const LevelDev& f = ctx->lev[jobs[j].level];
        if (f.ninterp == 0) continue;
        FillJob& F = a.fills[a.nfill++];
        F.cells = f.interps;
        F.n = f.ninterp;
        F.q = jobs[j].q;
        F.cold = jobs[j].qc_old;
        F.cnew = jobs[j].qc_new;
        F.tau = jobs[j].tau;
    }
    ctx->launches += 1;
    // fill CTAs: the slots the tiles leave free, at least one per SM (those run as the step's
    // CTAs retire)
    cudaError_t e = launch_step(a, ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, grid, s,
                                std::max(per_sm * ctx->nsm - grid, ctx->nsm));
    if (e == cudaSuccess && (flags & CLAW_ADVANCE_PUSH_GHOSTS) && d.ncopy) {
        e = launch_fill_copy(d.copies, d.copy_start, d.ncopy_blocks, q_new, s);
        ctx->launches += 1;
    }
    return cuda_rc(e);
}

int claw_level_advance(claw_ctx* ctx, int32_t L, const double* q_old, double* q_new, const double* aux, double* dt,
                       double* smax, int32_t flags, void* stream)
{
    return level_advance(ctx, L, q_old, q_new, aux, dt, smax, flags, nullptr, nullptr, 0.0, false, stream);
}

int claw_level_advance_interp(claw_ctx* ctx, int32_t L, const double* q_old, double* q_new, const double* aux,
                              double* dt, double* smax, int32_t flags, const double* qc_old, const double* qc_new,
                              double tau, void* stream)
{
    return level_advance(ctx, L, q_old, q_new, aux, dt, smax, flags, qc_old, qc_new, tau, true, stream);
}

int claw_level_advance_fill(claw_ctx* ctx, int32_t L, const double* q_old, double* q_new, const double* aux,
                            double* dt, double* smax, int32_t flags, const claw_fill_job* jobs, int32_t njobs,
                            void* stream)
{
    return level_advance(ctx, L, q_old, q_new, aux, dt, smax, flags, nullptr, nullptr, 0.0, false, stream, jobs, njobs);
}

int claw_level_advance_boxes(claw_ctx* ctx, int32_t L, int32_t box_begin, int32_t box_end, const double* q_old,
                             double* q_new, const double* aux, const double* dt, double* smax, int32_t flags,
                             void* stream)
{
    int rc = check_step_args(ctx, L, q_old, q_new, aux, dt, smax);
    if (rc) return rc;
    if (flags & ~CLAW_ADVANCE_PULL_GHOSTS) return CLAW_EINVAL;
    if ((flags & CLAW_ADVANCE_PULL_GHOSTS) && !ctx->lev[L].ring_ok) return CLAW_EINVAL;
    LevelDev& d = ctx->lev[L];
    if (box_begin < 0 || box_end > d.nboxes || box_begin > box_end) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    const auto& st = ctx->ptile_start[L];
    if (box_begin == box_end || st[box_end] == st[box_begin]) return CLAW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    StepArgs a = make_args(ctx, L, q_old, q_new, aux, dt, smax);
    a.tiles = ctx->ptiles[L] + st[box_begin];
    a.ntiles = st[box_end] - st[box_begin];
    a.tcum = nullptr;
    if (flags & CLAW_ADVANCE_PULL_GHOSTS) a.ring = d.ring;
    int staging = d.staging;
    if (staging >= 1) {
        a.tmaps = get_tmaps(ctx, L, q_old, s);
        if (!a.tmaps) staging = 0;
    }
    const int per_sm = step_max_ctas_per_sm(ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, a.ring != nullptr);
    if (per_sm <= 0) return CLAW_ECUDA;
    const int grid = std::min(a.ntiles, per_sm * ctx->nsm);
    ctx->launches += 1;
    return cuda_rc(launch_step(a, ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, grid, s));
}

long long claw_packed_size(claw_ctx* ctx, int32_t L)
{
    if (!valid_level(ctx, L)) return -CLAW_EINVAL;
    return ctx->lev[L].packed;
}

static int pack_call(claw_ctx* ctx, int L, int b0, int b1, double* q, double* packed, int unpack, void* stream)
{
    if (!valid_level(ctx, L) || !q || !packed) return CLAW_EINVAL;
    const LevelDev& d = ctx->lev[L];
    if (b0 < 0 || b1 > d.nboxes || b0 > b1) return CLAW_EINVAL;
    if (b0 == b1) return CLAW_OK;
    DevGuard g(ctx->device);
    ctx->launches += 1;
    return cuda_rc(launch_pack(d.patches, d.poff, b0, b1, d.max_rows - 4, q, packed, unpack, (cudaStream_t)stream));
}

int claw_pack_interiors(claw_ctx* ctx, int32_t L, int32_t box_begin, int32_t box_end, const double* q,
                        double* packed, void* stream)
{
    return pack_call(ctx, L, box_begin, box_end, const_cast<double*>(q), packed, 0, stream);
}

int claw_unpack_interiors(claw_ctx* ctx, int32_t L, int32_t box_begin, int32_t box_end, const double* packed,
                          double* q, void* stream)
{
    return pack_call(ctx, L, box_begin, box_end, q, const_cast<double*>(packed), 1, stream);
}

int claw_level_step_patchwise(claw_ctx* ctx, int32_t L, const double* q_old, double* q_new, const double* aux,
                              const double* dt, double* smax, void* stream)
{
    int rc = check_step_args(ctx, L, q_old, q_new, aux, dt, smax);
    if (rc) return rc;
    DevGuard g(ctx->device);
    LevelDev& d = ctx->lev[L];
    cudaStream_t s = (cudaStream_t)stream;
    StepArgs a = make_args(ctx, L, q_old, q_new, aux, dt, smax);
    const auto& st = ctx->ptile_start[L];
    for (int n = 0; n < d.nboxes; ++n) {
        a.tiles = ctx->ptiles[L] + st[n];
        a.ntiles = st[n + 1] - st[n];
        a.tcum = nullptr;
        ctx->launches += 1;
        cudaError_t e = launch_step(a, ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, 0, a.ntiles, s);
        if (e != cudaSuccess) return CLAW_ECUDA;
    }
    return CLAW_OK;
}

int claw_average_down(claw_ctx* ctx, int32_t fl, const double* qf, double* qc, void* stream)
{
    if (!ctx || fl < 1 || fl >= CLAW_MAXLEV || !qf || !qc) return CLAW_EINVAL;
    if (!ctx->set[fl]) return CLAW_ESTATE;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[fl];
    ctx->launches += d.navg > 0;
    return cuda_rc(launch_average(d.avgs, d.navg, d.ratio, qf, qc, (cudaStream_t)stream));
}

int claw_average_down_adjoint(claw_ctx* ctx, int32_t fl, double* lf, double* lc, void* stream)
{
    if (!ctx || fl < 1 || fl >= CLAW_MAXLEV || !lf || !lc) return CLAW_EINVAL;
    if (!ctx->set[fl]) return CLAW_ESTATE;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[fl];
    ctx->launches += d.navg > 0;
    return cuda_rc(launch_average_adjoint(d.avgs, d.navg, d.ratio, lf, lc, (cudaStream_t)stream));
}

int claw_level_advance_adjoint(claw_ctx* ctx, int32_t L, const double* q_old, const double* lam_new,
                               double* lam_old, const double* aux, double* g_aux, const double* dt, int32_t flags,
                               void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !q_old || !lam_new || !lam_old || !dt) return CLAW_EINVAL;
    if (flags & ~CLAW_ADVANCE_PULL_GHOSTS) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    if (ctx->kind() == KIND_SWE) return CLAW_EINVAL;   // the adjoint is written for acoustics
    if (ctx->medium == 1 && (!aux || !g_aux)) return CLAW_EINVAL;
    LevelDev& d = ctx->lev[L];
    if ((flags & CLAW_ADVANCE_PULL_GHOSTS) && !d.ring_ok) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    if (d.ntiles == 0) return CLAW_OK;
    StepArgs a = make_args(ctx, L, q_old, nullptr, aux, dt, nullptr);
    a.tiles = ctx->atiles[L];
    a.ntiles = ctx->natiles[L];
    a.tcum = nullptr;
    if (flags & CLAW_ADVANCE_PULL_GHOSTS) a.ring = d.ring;
    ctx->launches += 1;
    return cuda_rc(launch_step_adjoint(a, lam_new, lam_old, g_aux, ctx->medium, ctx->limiter, ctx->nsm,
                                       (cudaStream_t)stream));
}

int claw_level_advance_record(claw_ctx* ctx, int32_t L, const double* q_old, double* q_new, const double* aux,
                              double* dt, double* smax, int32_t flags, double* tape, void* stream)
{
    int rc = check_step_args(ctx, L, q_old, q_new, aux, dt, smax);
    if (rc) return rc;
    if (!tape || ctx->kind() != KIND_CELLWISE || ctx->order != 2) return CLAW_EINVAL;
    if (flags & ~(CLAW_ADVANCE_PULL_GHOSTS | CLAW_ADVANCE_UPDATE_DT)) return CLAW_EINVAL;
    const bool pull = (flags & CLAW_ADVANCE_PULL_GHOSTS) != 0;
    if (pull && !ctx->lev[L].ring_ok) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    LevelDev& d = ctx->lev[L];
    if (d.ntiles == 0) return CLAW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    StepArgs a = make_args(ctx, L, q_old, q_new, aux, dt, smax);
    if (flags & CLAW_ADVANCE_UPDATE_DT) {
        a.dtupd = 1;
        a.dt_out = dt;
        a.minh = ctx->minh;
        a.cflv = ctx->cflv;
        a.done = ctx->done;
        a.nruns = ctx->nruns;
    }
    if (pull) a.ring = d.ring;
    a.tape = tape;
    int staging = d.staging;
    if (staging >= 1) {
        a.tmaps = get_tmaps(ctx, L, q_old, s);
        if (!a.tmaps) staging = 0;
    }
    const int per_sm = step_max_ctas_per_sm(ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, pull, true);
    if (per_sm <= 0) return CLAW_ECUDA;
    const int grid = std::min(d.ntiles, per_sm * ctx->nsm);
    ctx->launches += 1;
    return cuda_rc(launch_step(a, ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, grid, s));
}

int claw_level_advance_adjoint_tape(claw_ctx* ctx, int32_t L, const double* tape, const double* lam_new,
                                    double* lam_old, const double* aux, double* g_aux, const double* dt,
                                    int32_t flags, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !tape || !lam_new || !lam_old || !aux || !g_aux || !dt)
        return CLAW_EINVAL;
    if (flags & ~CLAW_ADVANCE_PULL_GHOSTS) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    if (ctx->kind() != KIND_CELLWISE || ctx->order != 2) return CLAW_EINVAL;
    LevelDev& d = ctx->lev[L];
    if ((flags & CLAW_ADVANCE_PULL_GHOSTS) && !d.ring_ok) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    if (d.ntiles == 0) return CLAW_OK;
    StepArgs a = make_args(ctx, L, nullptr, nullptr, aux, dt, nullptr);
    a.tiles = ctx->atiles[L];
    a.ntiles = ctx->natiles[L];
    a.tcum = nullptr;
    a.tape = const_cast<double*>(tape);
    if (flags & CLAW_ADVANCE_PULL_GHOSTS) a.ring = d.ring;
    ctx->launches += 1;
    return cuda_rc(launch_step_adjoint_tape(a, lam_new, lam_old, g_aux, ctx->limiter, ctx->nsm,
                                            (cudaStream_t)stream));
}

int claw_level_step_adjoint(claw_ctx* ctx, int32_t L, const double* q_old, const double* lam_new, double* lam_old,
                            const double* aux, double* g_aux, const double* dt, void* stream)
{
    return claw_level_advance_adjoint(ctx, L, q_old, lam_new, lam_old, aux, g_aux, dt, 0, stream);
}

static int reflux_check(claw_ctx* ctx, int L)
{
    if (!ctx || L < 1 || L >= CLAW_MAXLEV) return CLAW_EINVAL;
    if (!ctx->set[L] || !ctx->set[L - 1]) return CLAW_ESTATE;
    // the fix needs conservation form: acoustics in a uniform medium, or shallow water
    if (ctx->medium != 0) return CLAW_EINVAL;
    return CLAW_OK;
}

int claw_reflux_count(claw_ctx* ctx, int32_t L)
{
    int rc = reflux_check(ctx, L);
    return rc ? -rc : ctx->lev[L].nreflux;
}

int claw_reflux_buffer_size(claw_ctx* ctx, int32_t L)
{
    int rc = reflux_check(ctx, L);
    return rc ? -rc : 3 * ctx->lev[L].nreflux * (1 + ctx->lev[L].ratio);
}

int claw_reflux_coarse(claw_ctx* ctx, int32_t L, const double* q_c_old, const double* dt, double* buf, void* stream)
{
    int rc = reflux_check(ctx, L);
    if (rc) return rc;
    if (!q_c_old || !dt || !buf) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[L];
    const StepArgs k = make_args(ctx, L - 1, nullptr, nullptr, nullptr, dt, nullptr);
    ctx->launches += d.nreflux > 0;
    return cuda_rc(launch_reflux_coarse(d.reflux, d.nreflux, ctx->lev[L - 1].patches, q_c_old, dt, buf, d.ratio, k,
                                        ctx->limiter, (cudaStream_t)stream));
}

int claw_reflux_fine(claw_ctx* ctx, int32_t L, const double* q_f, const double* q_c_old, const double* dt, double* buf,
                     void* stream)
{
    int rc = reflux_check(ctx, L);
    if (rc) return rc;
    if (!q_f || !q_c_old || !dt || !buf) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[L];
    const StepArgs k = make_args(ctx, L, nullptr, nullptr, nullptr, dt, nullptr);
    ctx->launches += d.nreflux > 0;
    return cuda_rc(launch_reflux_fine(d.reflux, d.nreflux, ctx->lev[L - 1].patches, d.patches, q_f, q_c_old, dt, buf,
                                      d.ratio, k, ctx->limiter, (cudaStream_t)stream));
}

int claw_reflux_apply(claw_ctx* ctx, int32_t L, const double* buf, const double* dt, double* q_c_new, void* stream)
{
    int rc = reflux_check(ctx, L);
    if (rc) return rc;
    if (!buf || !dt || !q_c_new) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[L];
    ctx->launches += d.nreflux_groups > 0;
    return cuda_rc(launch_reflux_apply(d.reflux, d.nreflux, d.reflux_group, d.nreflux_groups, d.ratio,
                                       ctx->lev[L - 1].patches, dt, buf, q_c_new, (cudaStream_t)stream));
}

int claw_sync_status(claw_ctx* ctx)
{
    if (!ctx) return CLAW_EINVAL;
    DevGuard g(ctx->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return CLAW_ECUDA;
    int f = 0;
    if (cudaMemcpy(&f, ctx->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CLAW_ECUDA;
    if (f && cudaMemset(ctx->err, 0, sizeof(int)) != cudaSuccess) return CLAW_ECUDA;
    if (f & ERR_NAN) return CLAW_ENAN;
    if (f & ERR_CFL) return CLAW_ECFL;
    if (f & ERR_TIMEOUT) return CLAW_ETIMEOUT;
    return CLAW_OK;
}

int64_t claw_launch_count(claw_ctx* ctx) { return ctx ? (int64_t)ctx->launches.load() : 0; }

const char* claw_strerror(int32_t s)
{
    switch (s) {
    case CLAW_OK: return "ok";
    case CLAW_EINVAL: return "invalid argument or box set";
    case CLAW_ECUDA: return "CUDA runtime error";
    case CLAW_ENOMEM: return "out of memory";
    case CLAW_ECFL: return "CFL number above 1";
    case CLAW_ENAN: return "NaN or Inf in the state";
    case CLAW_ETIMEOUT: return "bounded device wait expired";
    case CLAW_ESTATE: return "call out of order";
    }
    return "unknown status";
}

}  // extern "C"

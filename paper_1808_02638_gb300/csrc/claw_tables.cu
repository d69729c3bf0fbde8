// claw_tables.cu -- the device task tables of a level, built on the host from its boxes when the
// level is set (Sec. 2.2, 2.3): the step's tiles, the ghost fill (copy rectangles, interpolated
// cells, per-box ghost rings for pulled ghosts), the conservation fix's interface records, the
// averaging rectangles, the coefficient-pool copies, and the tensor-map descriptors of staged
// tiles.
#include "claw_host.h"

#include <array>

namespace claw_host {

void free_arena(DevArena& a)
{
    cudaFree(a.dev);
    cudaFreeHost(a.host);
    a.dev = nullptr;
    a.host = nullptr;
    a.cap = a.host_cap = 0;
}

// Forgets a level's boxes and tables; the arenas stay allocated for the next rebuild
// (claw_destroy frees them).
void free_level(claw_ctx* ctx, int L)
{
    LevelDev& d = ctx->lev[L];
    d.ccopies = nullptr;
    d.nccopy = 0;
    d.coef_built = false;
    d.flagboxes = nullptr;
    d.ring = nullptr;
    d.poff = nullptr;
    d.packed = 0;
    d.ring_ok = false;
    d.reflux = nullptr;
    d.reflux_group = nullptr;
    d.nreflux = d.nreflux_groups = 0;
    d.copy_start = d.ccopy_start = nullptr;
    d.ncopy_blocks = d.nccopy_blocks = 0;
    ctx->atiles[L] = nullptr;
    ctx->natiles[L] = 0;
    for (auto& t : ctx->tmaps[L]) cudaFree(t.dev);
    ctx->tmaps[L].clear();
    ctx->ptiles[L] = nullptr;
    d.patches = nullptr;
    d.tiles = nullptr;
    d.copies = nullptr;
    d.interps = nullptr;
    d.avgs = nullptr;
    d.nboxes = d.ntiles = d.ncopy = d.ninterp = d.navg = 0;
    d.boxes.clear();
    d.hpatches.clear();
    d.htiles.clear();
    d.htcum.clear();
    ctx->loc[L].clear();
    d.tcum = nullptr;
    ctx->set[L] = false;
}

// The step's tiles as column walks (uniform medium, shallow water): every column of tiles of a
// box bottom to top, continued into the column of the same-level box directly above when that
// box has the same run, ilo and nx (the columns then coincide), cut into pieces of `piece`
// tiles; every tile but the first of a piece is flagged TILE_CARRY.  Crossing into the box above
// needs the shared rows to be the same in both boxes, which the ghost states are: they come from
// the box below, or from the same boundary image or coarse interpolation.  (A cell-wise
// medium's ghost coefficients are the caller's and need not match, one reason walks are not
// built for it; the other is that the cell-wise kernels keep their registers without the
// carrying code.)  cum[i] is the cost of tiles [0, i): the cells of the tile and of the halo
// rows and columns it computes edges on, plus a fixed per-tile share.
static void column_walks(const LevelDev& d, int piece, std::vector<TileDev>& out, std::vector<long long>& cum)
{
    const int nb = d.nboxes;
    std::map<std::array<int, 4>, int> by_base;   // (run, ilo, nx, jlo) -> box
    for (int n = 0; n < nb; ++n) {
        const claw_box& b = d.boxes[n];
        by_base[{b.run, b.ilo, b.nx, b.jlo}] = n;
    }
    std::vector<int> above(nb, -1), has_below(nb, 0);
    for (int n = 0; n < nb; ++n) {
        const claw_box& b = d.boxes[n];
        auto it = by_base.find({b.run, b.ilo, b.nx, b.jlo + b.ny});
        if (it != by_base.end()) {
            above[n] = it->second;
            has_below[it->second] = 1;
        }
    }
    // every column chain, then cut into pieces of `piece` tiles; the pieces are laid out band by
    // band (the first piece of every chain, then the second, ...), so that the CTAs that run at
    // the same time work side by side and share their ghost columns in L2
    std::vector<std::vector<TileDev>> chains;
    for (int n0 = 0; n0 < nb; ++n0) {
        if (has_below[n0]) continue;   // chains start at boxes with nothing aligned below
        const claw_box& b0 = d.boxes[n0];
        for (int x = 0; x < b0.nx; x += d.tx) {
            std::vector<TileDev> ch;
            for (int n = n0; n >= 0; n = above[n]) {
                const claw_box& b = d.boxes[n];
                for (int y = 0; y < b.ny; y += d.ty) {
                    TileDev T;
                    T.patch = n;
                    T.x0 = (short)x;
                    T.y0 = (short)y;
                    T.tx = (short)std::min(d.tx, b.nx - x);
                    T.ty = (short)std::min(d.ty, b.ny - y);
                    T.flags = ch.size() % piece ? TILE_CARRY : 0;
                    ch.push_back(T);
                }
            }
            chains.push_back(std::move(ch));
        }
    }
    out.clear();
    cum.assign(1, 0);
    for (size_t band = 0;; ++band) {
        bool any = false;
        for (const auto& ch : chains) {
            const size_t k0 = band * piece;
            if (k0 >= ch.size()) continue;
            any = true;
            for (size_t k = k0; k < std::min(ch.size(), k0 + piece); ++k) {
                const TileDev& T = ch[k];
                out.push_back(T);
                const long long c = (long long)(T.tx + 3) * (T.ty + (T.flags ? 0 : 3)) + 64;
                cum.push_back(cum.back() + c);
            }
        }
        if (!any) break;
    }
}

// tiles of a level for its tiling: sorted by area (largest first) for the persistent CTAs, or
// as column walks (d.walk; automatic: acoustics levels with at least kWalkTilesPerSM tiles per
// SM, where each CTA has several tiles to walk; with about one tile per CTA the area-sorted
// stride balances better), and grouped by box for the per-box launches
constexpr int kWalkTilesPerSM = 8;

int build_tiles(claw_ctx* ctx, int L)
{
    LevelDev& d = ctx->lev[L];
    std::vector<TileDev> t;
    std::vector<int> start;
    for (int n = 0; n < d.nboxes; ++n) {
        const claw_box& b = d.boxes[n];
        start.push_back((int)t.size());
        for (int y = 0; y < b.ny; y += d.ty)
            for (int x = 0; x < b.nx; x += d.tx) {
                TileDev T;
                T.patch = n;
                T.x0 = (short)x;
                T.y0 = (short)y;
                T.tx = (short)std::min(d.tx, b.nx - x);
                T.ty = (short)std::min(d.ty, b.ny - y);
                T.flags = 0;
                t.push_back(T);
            }
    }
    start.push_back((int)t.size());
    // (the pieces are read by pack.commit: t keeps the box order, d.htiles the sorted copy)
    ArenaPack pack;
    pack.add(&ctx->ptiles[L], t);
    ctx->ptile_start[L] = start;
    d.htcum.clear();
    // automatic: uniform-medium acoustics only (the shallow-water step issues 6 % fewer FP64
    // instructions with walks but ran 1.5 % slower on the 2048^2 workload, with two CTAs per SM)
    d.walking = ctx->kind() != KIND_CELLWISE &&
                (d.walk > 0 || (d.walk < 0 && ctx->kind() == KIND_UNIFORM &&
                                (long long)t.size() >= (long long)kWalkTilesPerSM * std::max(ctx->nsm, 1)));
    if (d.walking) {
        // pieces of about the tiles one CTA takes (three CTAs per SM, a guess: the launch picks
        // its grid later), at least 4 and at most 64
        const int piece = (int)std::min<long long>(64, std::max<long long>(4, ((long long)t.size() + 3LL * ctx->nsm - 1) /
                                                                                 std::max(1, 3 * ctx->nsm)));
        column_walks(d, piece, d.htiles, d.htcum);
    } else {
        d.htiles = t;
        std::stable_sort(d.htiles.begin(), d.htiles.end(), [](const TileDev& a, const TileDev& b) {
            return (int)a.tx * a.ty > (int)b.tx * b.ty;
        });
    }
    d.ntiles = (int)d.htiles.size();
    for (auto& tm : ctx->tmaps[L]) cudaFree(tm.dev);
    ctx->tmaps[L].clear();
    pack.add(&d.tiles, d.htiles);
    d.tcum = nullptr;
    if (d.walking) pack.add(&d.tcum, d.htcum);
    // adjoint tiles
    std::vector<TileDev> at;
    const int e = adjoint_tile();
    for (int n = 0; n < d.nboxes; ++n) {
        const claw_box& b = d.boxes[n];
        for (int y = 0; y < b.ny; y += e)
            for (int x = 0; x < b.nx; x += e) {
                TileDev T;
                T.patch = n;
                T.x0 = (short)x;
                T.y0 = (short)y;
                T.tx = (short)std::min(e, b.nx - x);
                T.ty = (short)std::min(e, b.ny - y);
                T.flags = 0;
                at.push_back(T);
            }
    }
    // largest first, like the step's tiles: the persistent CTAs end on small tiles
    std::stable_sort(at.begin(), at.end(),
                     [](const TileDev& a, const TileDev& b) { return (int)a.tx * a.ty > (int)b.tx * b.ty; });
    ctx->natiles[L] = (int)at.size();
    pack.add(&ctx->atiles[L], at);
    return pack.commit(d.tiletab);
}

int make_interp(claw_ctx* ctx, int L, const claw_problem& pr, const Locator& cl, long long dst, long long dplane,
                int si, int sj, int flags, InterpCell& c)
{
    const int rr = ctx->lev[L].ratio;
    const int cNX = level_nx(pr, L - 1), cNY = level_ny(pr, L - 1);
    const int I = floordiv(si, rr), J = floordiv(sj, rr);
    const int di[5] = {0, -1, 1, 0, 0}, dj[5] = {0, 0, 0, -1, 1};
    std::memset(&c, 0, sizeof(c));
    c.dst = dst;
    c.dplane = dplane;
    for (int s = 0; s < 5; ++s) {
        int cfx, cfy;
        const int ci = bc_map(I + di[s], cNX, pr.bc[0], pr.bc[1], &cfx);
        const int cj = bc_map(J + dj[s], cNY, pr.bc[2], pr.bc[3], &cfy);
        const int m = cl.find(ci, cj);
        if (m < 0) return CLAW_EINVAL;
        const claw_box& cb = ctx->lev[L - 1].boxes[m];
        c.src[s] = cell_off(cb, ci, cj);
        c.splane[s] = plane_of(cb);
        c.sflags[s] = cfx | (cfy << 1);
    }
    c.xi = ((double)(si - I * rr) + 0.5) / rr - 0.5;
    c.eta = ((double)(sj - J * rr) + 0.5) / rr - 0.5;
    c.flags = flags;
    return CLAW_OK;
}

constexpr int kRectRows = 32;          // copy rectangles are split into pieces of at most this many rows
constexpr long long kBlockCells = 256;   // cells per block of the copy kernel (about): one batch per thread


int build_ghost_tables(claw_ctx* ctx, int L, GhostTables& gt, bool want_ring)
{
    LevelDev& d = ctx->lev[L];
    const std::vector<Locator>& loc = ctx->loc[L];
    static const std::vector<Locator> none;
    const std::vector<Locator>& cloc = L > 0 ? ctx->loc[L - 1] : none;

    // per box, independently (threads): its copy rectangles, interpolated cells and ghost ring
    std::vector<BoxGhosts>& per = gt.per;
    per.assign(d.nboxes, BoxGhosts{});
    auto one_box = [&](int n, BoxGhosts& out) -> int {
        const claw_box& b = d.boxes[n];
        const claw_problem& pr = ctx->runs[b.run];
        const int NX = level_nx(pr, L), NY = level_ny(pr, L);
        const int W = b.nx + 4;
        std::vector<GhostEntry> ent;
        for (int gj = b.jlo - 2; gj < b.jlo + b.ny + 2; ++gj) {
            // the ghost cells of row gj in row order: the whole padded row above and below the
            // interior, else two cells on each side
            const bool side_only = gj >= b.jlo && gj < b.jlo + b.ny;
            for (int gi = b.ilo - 2; gi < b.ilo + b.nx + 2; gi += (side_only && gi == b.ilo - 1) ? b.nx + 1 : 1) {
                int fx, fy;
                const int si = bc_map(gi, NX, pr.bc[0], pr.bc[1], &fx);
                const int sj = bc_map(gj, NY, pr.bc[2], pr.bc[3], &fy);
                int src = (si >= b.ilo && si < b.ilo + b.nx && sj >= b.jlo && sj < b.jlo + b.ny)
                              ? n : loc[b.run].find(si, sj);
                GhostEntry e{gi, gj, src, 0, fx | (fy << 1)};
                if (src >= 0) {
                    e.soff = cell_off(d.boxes[src], si, sj);
                    ent.push_back(e);
                    if (out.want_ring) {   // ring order = this loop's order
                        const long long pl = plane_of(d.boxes[src]);
                        if (pl >= (1LL << kRingFlagShift)) out.ring_ok = false;
                        out.ring.push_back(make_longlong2(e.soff, pl | ((long long)e.flags << kRingFlagShift)));
                    }
                    continue;
                }
                if (out.want_ring) out.ring.push_back(make_longlong2(-1 - (long long)out.cells.size(), 0));
                // space-time interpolation from level L-1 at the fine cell (si, sj)
                if (L == 0) return CLAW_EINVAL;
                InterpCell c;
                if (make_interp(ctx, L, pr, cloc[b.run], cell_off(b, gi, gj), plane_of(b), si, sj, fx | (fy << 1), c))
                    return CLAW_EINVAL;   // not properly nested
                out.cells.push_back(c);
            }
        }
        // row runs of copies (consecutive ghosts of a row with one source box, one sign and a
        // constant source step), then stacked into rectangles
        struct RowRun {
            int gj, gi0, w, src, flags, sx;
            long long soff;
        };
        std::vector<RowRun> runs;
        for (size_t k = 0; k < ent.size();) {
            RowRun R{ent[k].gj, ent[k].gi, 1, ent[k].src, ent[k].flags, 0, ent[k].soff};
            size_t k2 = k + 1;
            while (k2 < ent.size() && ent[k2].gj == R.gj && ent[k2].gi == R.gi0 + R.w &&
                   ent[k2].src == R.src && ent[k2].flags == R.flags) {
                const long long step = ent[k2].soff - ent[k2 - 1].soff;
                if (R.w == 1) {
                    if (step < -1 || step > 1) break;
                    R.sx = (int)step;
                } else if (step != R.sx) {
                    break;
                }
                ++R.w;
                ++k2;
            }
            runs.push_back(R);
            k = k2;
        }
        struct Open {
            RowRun first;
            int h;
            long long sy, last_soff;
            int last_gj;
        };
        std::vector<Open> open;
        auto emit = [&](const Open& o) {
            const claw_box& sb = d.boxes[o.first.src];
            CopyRect c;
            c.dst = cell_off(b, o.first.gi0, o.first.gj);
            c.src = o.first.soff;
            c.dplane = plane_of(b);
            c.splane = plane_of(sb);
            c.w = o.first.w;
            c.h = o.h;
            c.dpitch = W;
            c.sy = (int)o.sy;
            c.sx = o.first.sx;
            c.flags = o.first.flags;
            // at most kRectRows rows per rectangle, so that long strips spread over blocks
            for (int k0 = 0; k0 < o.h; k0 += kRectRows) {
                CopyRect piece = c;
                piece.h = std::min(kRectRows, o.h - k0);
                piece.dst = c.dst + (long long)k0 * c.dpitch;
                piece.src = c.src + (long long)k0 * c.sy;
                out.rects.push_back(piece);
            }
        };
        for (const RowRun& R : runs) {
            bool merged = false;
            for (Open& o : open) {
                if (o.last_gj != R.gj - 1 || o.first.gi0 != R.gi0 || o.first.w != R.w ||
                    o.first.src != R.src || o.first.flags != R.flags || o.first.sx != R.sx)
                    continue;
                const long long step = R.soff - o.last_soff;
                const long long pitch = d.boxes[R.src].nx + 4;
                if (o.h == 1) {
                    if (step != 0 && step != pitch && step != -pitch) continue;
                    o.sy = step;
                } else if (step != o.sy) {
                    continue;
                }
                ++o.h;
                o.last_soff = R.soff;
                o.last_gj = R.gj;
                merged = true;
                break;
            }
            if (!merged) open.push_back(Open{R, 1, 0, R.soff, R.gj});
            // retire rectangles that can no longer grow
            for (size_t q = 0; q < open.size();) {
                if (open[q].last_gj < R.gj - 1) {
                    emit(open[q]);
                    open.erase(open.begin() + q);
                } else {
                    ++q;
                }
            }
        }
        for (const Open& o : open) emit(o);
            return CLAW_OK;
    };
    parallel_for(d.nboxes, [&](int n0, int n1) {
        for (int n = n0; n < n1; ++n) {
            per[n].want_ring = want_ring;
            per[n].rc = one_box(n, per[n]);
        }
    }, 4);
    gt.nrects = gt.ncells = gt.nring = 0;
    gt.ring_ok = true;
    for (int n = 0; n < d.nboxes; ++n) {
        const BoxGhosts& g = per[n];
        if (g.rc) return g.rc;
        if (want_ring) {
            d.hpatches[n].ring = gt.nring < (size_t)(1LL << 31) ? (int)gt.nring : -1;
            if (!g.ring_ok) gt.ring_ok = false;
        }
        gt.nrects += g.rects.size();
        gt.ncells += g.cells.size();
        gt.nring += g.ring.size();
    }
    if (gt.nring >= (size_t)(1LL << 31)) gt.ring_ok = false;
    // blocks of the copy kernel: consecutive rectangles up to about kBlockCells cells (and at
    // most 32 rectangles, the kernel's staging chunk)
    std::vector<int>& start = gt.start;
    start.assign(1, 0);
    long long cells_in = 0;
    int i = 0;
    for (const BoxGhosts& g : per)
        for (const CopyRect& rc : g.rects) {
            const long long c = (long long)rc.w * rc.h;
            const int nin = i - start.back();
            if (nin > 0 && (cells_in + c > kBlockCells || nin >= 32)) {
                start.push_back(i);
                cells_in = 0;
            }
            cells_in += c;
            ++i;
        }
    if (gt.nrects) start.push_back((int)gt.nrects);
    return CLAW_OK;
}

// coarse-fine interface of level L for the conservation fix: every coarse cell of level L-1
// that no box of level L covers but that shares an edge with one, per fine box side; periodic
// boundaries wrap, other boundaries end the interface.  Records are grouped by coarse cell.
void build_reflux_tables(claw_ctx* ctx, int L, std::vector<RefluxRec>& recs, std::vector<int>& group)
{
    const LevelDev& f = ctx->lev[L];
    const LevelDev& c = ctx->lev[L - 1];
    const int r = f.ratio;
    const std::vector<Locator>& floc = ctx->loc[L];
    const std::vector<Locator>& cloc = ctx->loc[L - 1];
    auto wrap = [](int k, int n, int lo, int hi, bool& ok) {
        ok = true;
        if (k >= 0 && k < n) return k;
        if ((k < 0 && lo == CLAW_BC_PERIODIC) || (k >= n && hi == CLAW_BC_PERIODIC)) return ((k % n) + n) % n;
        ok = false;
        return k;
    };
    // the records of each fine box on its own (host threads), then concatenated in box order
    std::vector<std::vector<RefluxRec>> per(f.nboxes);
    parallel_for(f.nboxes, [&](int n0, int n1) {
        for (int nf = n0; nf < n1; ++nf) {
            std::vector<RefluxRec>& out = per[nf];
            const claw_box& b = f.boxes[nf];
            const claw_problem& p = ctx->runs[b.run];
            const int NXc = level_nx(p, L - 1), NYc = level_ny(p, L - 1);
            const int I0 = b.ilo / r, I1 = (b.ilo + b.nx) / r, J0 = b.jlo / r, J1 = (b.jlo + b.ny) / r;
            auto add = [&](int I, int J, int dir, int side, int fi, int fj) {
                bool okx, oky;
                const int Im = wrap(I, NXc, p.bc[0], p.bc[1], okx), Jm = wrap(J, NYc, p.bc[2], p.bc[3], oky);
                if (!okx || !oky) return;
                if (floc[b.run].find(Im * r, Jm * r) >= 0) return;   // covered: a fine-fine edge
                const int nc = cloc[b.run].find(Im, Jm);
                if (nc < 0) return;                                 // excluded by proper nesting
                RefluxRec R;
                R.cbox = nc;
                R.fbox = nf;
                R.ci = (short)(Im - c.boxes[nc].ilo);
                R.cj = (short)(Jm - c.boxes[nc].jlo);
                R.fi = (short)fi;
                R.fj = (short)fj;
                R.dir = (short)dir;
                R.side = (short)side;
                out.push_back(R);
            };
            for (int J = J0; J < J1; ++J) {
                add(I1, J, 0, -1, b.nx - 1, J * r - b.jlo);
                add(I0 - 1, J, 0, +1, 0, J * r - b.jlo);
            }
            for (int I = I0; I < I1; ++I) {
                add(I, J1, 1, -1, I * r - b.ilo, b.ny - 1);
                add(I, J0 - 1, 1, +1, I * r - b.ilo, 0);
            }
        }
    }, 8);
    recs.clear();
    for (const auto& v : per) recs.insert(recs.end(), v.begin(), v.end());
    std::stable_sort(recs.begin(), recs.end(), [](const RefluxRec& x, const RefluxRec& y) {
        if (x.cbox != y.cbox) return x.cbox < y.cbox;
        if (x.cj != y.cj) return x.cj < y.cj;
        return x.ci < y.ci;
    });
    group.clear();
    for (size_t i = 0; i < recs.size(); ++i)
        if (i == 0 || recs[i].cbox != recs[i - 1].cbox || recs[i].ci != recs[i - 1].ci || recs[i].cj != recs[i - 1].cj)
            group.push_back((int)i);
    if (!recs.empty()) group.push_back((int)recs.size());
}

// coarse cells of level L-1 covered by each box of level L: per fine box (host threads), the
// coarse boxes its footprint meets, found through the coarse level's buckets, in box order
void build_avg_tables(claw_ctx* ctx, int L, std::vector<AvgRect>& out)
{
    const LevelDev& f = ctx->lev[L];
    const LevelDev& c = ctx->lev[L - 1];
    const int r = f.ratio;
    const std::vector<Locator>& cloc = ctx->loc[L - 1];
    std::vector<std::vector<AvgRect>> per(f.nboxes);
    parallel_for(f.nboxes, [&](int n0, int n1) {
        std::vector<int> cand;
        for (int nf = n0; nf < n1; ++nf) {
            const claw_box& F = f.boxes[nf];
            const int I0 = F.ilo / r, I1 = (F.ilo + F.nx) / r, J0 = F.jlo / r, J1 = (F.jlo + F.ny) / r;
            cand.clear();
            cloc[F.run].each(I0, J0, I1, J1, [&](int nc) { cand.push_back(nc); });
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            for (int nc : cand) {
                const claw_box& C = c.boxes[nc];
                const int i0 = std::max(I0, C.ilo), i1 = std::min(I1, C.ilo + C.nx);
                const int j0 = std::max(J0, C.jlo), j1 = std::min(J1, C.jlo + C.ny);
                if (i0 >= i1 || j0 >= j1) continue;
                AvgRect a;
                a.cdst = cell_off(C, i0, j0);
                a.fsrc = cell_off(F, i0 * r, j0 * r);
                a.cplane = plane_of(C);
                a.fplane = plane_of(F);
                a.w = i1 - i0;
                a.h = j1 - j0;
                a.cpitch = C.nx + 4;
                a.fpitch = F.nx + 4;
                per[nf].push_back(a);
            }
        }
    }, 8);
    for (const auto& v : per) out.insert(out.end(), v.begin(), v.end());
}

// tensor-map descriptors of one level for a given q pool and tiling (cached per pool)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

const void* get_tmaps(claw_ctx* ctx, int L, const double* q, cudaStream_t s)
{
    LevelDev& d = ctx->lev[L];
    auto& cache = ctx->tmaps[L];
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return nullptr;
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    for (auto& t : cache)
        if (t.q == q && t.tx == d.tx && t.ty == d.ty) {
            t.stamp = ++ctx->stamp;
            // a captured launch keeps this device pointer: the entry must outlive the graph, so
            // it is never evicted (only a rebuild of the level's tables frees it)
            if (capturing) t.pinned = true;
            return t.dev;
        }
    if (capturing) return nullptr;   // no descriptor is built inside a capture
    auto enc = encode_fn();
    if (!enc) return nullptr;
    // the copied box must fit inside every box's padded planes (else cooperative loads)
    for (const claw_box& b : d.boxes)
        if (d.tx + 4 > b.nx + 4 || d.ty + 4 > b.ny + 4) return nullptr;
    std::vector<CUtensorMap> maps(d.nboxes);
    for (int n = 0; n < d.nboxes; ++n) {
        const claw_box& b = d.boxes[n];
        const cuuint64_t W = b.nx + 4, H = b.ny + 4;
        cuuint64_t dims[3] = {W, H, 3};
        cuuint64_t strides[2] = {W * 8, W * H * 8};
        cuuint32_t box[3] = {(cuuint32_t)(d.tx + 4), (cuuint32_t)(d.ty + 4), 3};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&maps[n], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)(q + b.qoff), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return nullptr;
    }
    TmapCache t;
    t.q = q;
    t.tx = d.tx;
    t.ty = d.ty;
    if (cudaMalloc(&t.dev, maps.size() * sizeof(CUtensorMap)) != cudaSuccess) return nullptr;
    if (cudaMemcpyAsync(t.dev, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(t.dev);
        return nullptr;
    }
    t.stamp = ++ctx->stamp;
    // keep at most four entries that no capture has seen: evict the least recently used of those
    // (pinned entries stay, however many)
    size_t unpinned = 0;
    for (const auto& c : cache) unpinned += !c.pinned;
    if (unpinned >= 4) {
        auto old = cache.end();
        for (auto it = cache.begin(); it != cache.end(); ++it)
            if (!it->pinned && (old == cache.end() || it->stamp < old->stamp)) old = it;
        cudaStreamSynchronize(s);
        cudaFree(old->dev);
        cache.erase(old);
    }
    cache.push_back(t);
    return t.dev;
}

long long flag_grid_offset(const claw_ctx* ctx, int L, int run)
{
    long long off = 0;
    for (int r = 0; r < run; ++r)
        if (L < ctx->runs[r].nlev) off += (long long)level_nx(ctx->runs[r], L) * level_ny(ctx->runs[r], L);
    return off;
}

// ghost copies of one-plane coefficient pools: the same copies with offsets from coff and no
// wall sign flips
int build_coef_tables(claw_ctx* ctx, int L)
{
    LevelDev& d = ctx->lev[L];
    GhostTables gt;
    const std::vector<claw_box> saved = d.boxes;
    for (auto& b : d.boxes) b.qoff = b.coff;
    int rc = build_ghost_tables(ctx, L, gt, false);
    d.boxes = saved;
    if (rc) return rc;
    for (auto& g : gt.per)
        for (auto& r : g.rects) r.flags = 0;
    ArenaPack pack;
    pack.add(&d.ccopy_start, gt.start);
    pack.add_parts(&d.ccopies, d.nboxes, [&](int n) -> const std::vector<CopyRect>& { return gt.per[n].rects; });
    if ((rc = pack.commit(d.coeftab))) return rc;
    d.nccopy_blocks = gt.start.empty() ? 0 : (int)gt.start.size() - 1;
    d.nccopy = (int)gt.nrects;
    d.coef_built = true;
    return CLAW_OK;
}

// coefficient tables of a uniform-medium level on first use (outside stream capture)
int ensure_coef_tables(claw_ctx* ctx, int L, void* stream)
{
    if (ctx->lev[L].coef_built) return CLAW_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return CLAW_ESTATE;
    return build_coef_tables(ctx, L);
}

}  // namespace claw_host

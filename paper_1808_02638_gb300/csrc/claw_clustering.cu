// claw_clustering.cu -- regridding on the host (Sec. 2.2, 4.3): Berger-Rigoutsos clustering of a
// level's flags (grown by a buffer, kept inside the coverage), and the C ABI entry points of the
// regrid (the flag and transfer kernels are in claw_regrid.cu).
#include "claw_host.h"

using namespace claw_host;

namespace {

// ------------------------------------------------------------------ regridding (host)
// Berger-Rigoutsos clustering of a flag grid (row-major NY x NX): a box is accepted when its
// flags fill at least `cutoff` of it, it fits max_size and every cell of it is allowed (the
// nesting mask, which holds all flags); otherwise it is cut at a hole of a
// signature (the hole nearest the middle), else at the strongest sign change of a signature's
// second difference, else at the middle of its longer side, and both parts are processed again.
struct IBox {
    int i0, j0, nx, ny;
};

int hole_cut(const std::vector<long long>& sig)
{
    const int n = (int)sig.size();
    int best = -1;
    for (int k = 1; k < n - 1; ++k) {
        if (sig[k] != 0) continue;
        if (best < 0 || std::abs(2 * k + 1 - n) < std::abs(2 * best + 1 - n)) best = k;
    }
    if (best < 0) return -1;
    return (2 * best + 1 >= n) ? best : best + 1;
}

// (strength, cut) of the strongest sign change of the second difference, cut -1 when none
std::pair<long long, int> inflection_cut(const std::vector<long long>& sig)
{
    const int n = (int)sig.size();
    std::pair<long long, int> best(-1, -1);
    if (n < 4) return best;
    std::vector<long long> lap(n - 2);
    for (int t = 0; t < n - 2; ++t) lap[t] = sig[t] - 2 * sig[t + 1] + sig[t + 2];
    for (int t = 0; t + 1 < n - 2; ++t) {
        const long long a = lap[t], b = lap[t + 1];
        if ((a < 0 && b > 0) || (a > 0 && b < 0)) {
            const long long st = a > b ? a - b : b - a;
            if (best.second < 0 || st > best.first) best = {st, t + 2};
        }
    }
    return best;
}

// 2D prefix sum of a 0/1 grid: S(i, j) = sum over [0, i) x [0, j)
// (32-bit counts: grids below 2^31 cells; the table lives in a caller's buffer that is reused
// from call to call, so that a regrid does not page in fresh memory for every grid)
struct Prefix {
    int NX = 0, NY = 0;
    std::vector<int>& P;
    // g: nx x ny cells in rows of `pitch` bytes
    Prefix(const unsigned char* g, size_t pitch, int nx, int ny, bool invert, std::vector<int>& buf)
        : NX(nx), NY(ny), P(buf)
    {
        P.resize((size_t)(nx + 1) * (ny + 1));
        std::fill(P.begin(), P.begin() + (NX + 1), 0);   // row 0
        parallel_for(NY, [&](int j0, int j1) {   // prefix along each row
            for (int j = j0; j < j1; ++j) {
                int* row = &P[(size_t)(j + 1) * (NX + 1)];
                const unsigned char* src = g + (size_t)j * pitch;
                row[0] = 0;
                for (int i = 0; i < NX; ++i) row[i + 1] = row[i] + (((src[i] != 0) != invert) ? 1 : 0);
            }
        });
        parallel_for(NX + 1, [&](int i0, int i1) {   // then down each column
            for (int j = 1; j <= NY; ++j)
                for (int i = i0; i < i1; ++i) P[(size_t)j * (NX + 1) + i] += P[(size_t)(j - 1) * (NX + 1) + i];
        });
    }
    long long sum(int i0, int j0, int i1, int j1) const   // over [i0, i1) x [j0, j1)
    {
        return (long long)P[(size_t)j1 * (NX + 1) + i1] - P[(size_t)j0 * (NX + 1) + i1] -
               P[(size_t)j1 * (NX + 1) + i0] + P[(size_t)j0 * (NX + 1) + i0];
    }
};

// out[j * nx + i] = 1 when some cell of g within `rad` cells (square neighbourhood clipped to the
// grid) is set (g != 0, or g == 0 with `invert`); g is nx x ny cells in rows of `pitch` bytes.
// Separable: a running count along each row into `rows`, then one down each column.
void dilate(const unsigned char* g, size_t pitch, int nx, int ny, int rad, bool invert,
            std::vector<unsigned char>& rows, std::vector<unsigned char>& out)
{
    rows.resize((size_t)nx * ny);
    out.resize((size_t)nx * ny);
    rad = std::min(rad, std::max(nx, ny));
    parallel_for(ny, [&](int j0, int j1) {
        for (int j = j0; j < j1; ++j) {
            const unsigned char* src = g + (size_t)j * pitch;
            unsigned char* dst = &rows[(size_t)j * nx];
            auto set = [&](int i) { return ((src[i] != 0) != invert) ? 1 : 0; };
            int cnt = 0;
            for (int i = 0; i <= std::min(rad, nx - 1); ++i) cnt += set(i);
            for (int i = 0; i < nx; ++i) {
                dst[i] = cnt > 0;
                if (i + 1 + rad < nx) cnt += set(i + 1 + rad);
                if (i - rad >= 0) cnt -= set(i - rad);
            }
        }
    });
    parallel_for(nx, [&](int i0, int i1) {
        std::vector<int> cnt(i1 - i0, 0);
        for (int j = 0; j <= std::min(rad, ny - 1); ++j)
            for (int i = i0; i < i1; ++i) cnt[i - i0] += rows[(size_t)j * nx + i];
        for (int j = 0; j < ny; ++j) {
            unsigned char* dst = &out[(size_t)j * nx];
            const unsigned char* add = j + 1 + rad < ny ? &rows[(size_t)(j + 1 + rad) * nx] : nullptr;
            const unsigned char* sub = j - rad >= 0 ? &rows[(size_t)(j - rad) * nx] : nullptr;
            for (int i = i0; i < i1; ++i) {
                dst[i] = cnt[i - i0] > 0;
                if (add) cnt[i - i0] += add[i];
                if (sub) cnt[i - i0] -= sub[i];
            }
        }
    });
}

std::vector<IBox> cluster_flags(const std::vector<unsigned char>& f, int NX, int NY, double cutoff, int max_size,
                                const std::vector<unsigned char>& allowed)
{
    static thread_local std::vector<int> tl_bf, tl_bb;   // see claw_regrid_boxes
    const Prefix F(f.data(), NX, NX, NY, false, tl_bf), BAD(allowed.data(), NX, NX, NY, true, tl_bb);
    std::vector<IBox> out, stack{IBox{0, 0, NX, NY}};
    while (!stack.empty()) {
        IBox b = stack.back();
        stack.pop_back();
        // trim to the flags' bounding box, from column and row counts
        int ci0 = b.i0, ci1 = b.i0 + b.nx - 1, cj0 = b.j0, cj1 = b.j0 + b.ny - 1;
        if (F.sum(b.i0, b.j0, b.i0 + b.nx, b.j0 + b.ny) == 0) continue;
        while (F.sum(ci0, b.j0, ci0 + 1, b.j0 + b.ny) == 0) ++ci0;
        while (F.sum(ci1, b.j0, ci1 + 1, b.j0 + b.ny) == 0) --ci1;
        while (F.sum(ci0, cj0, ci1 + 1, cj0 + 1) == 0) ++cj0;
        while (F.sum(ci0, cj1, ci1 + 1, cj1 + 1) == 0) --cj1;
        b = IBox{ci0, cj0, ci1 - ci0 + 1, cj1 - cj0 + 1};
        const long long count = F.sum(b.i0, b.j0, b.i0 + b.nx, b.j0 + b.ny);
        const double eff = (double)count / (double)((long long)b.nx * b.ny);
        const bool inside = BAD.sum(b.i0, b.j0, b.i0 + b.nx, b.j0 + b.ny) == 0;
        if (eff >= cutoff && b.nx <= max_size && b.ny <= max_size && inside) {
            out.push_back(b);
            continue;
        }
        int dir = -1, k = -1;
        if (eff < cutoff) {
            std::vector<long long> sx(b.nx), sy(b.ny);
            for (int i = 0; i < b.nx; ++i) sx[i] = F.sum(b.i0 + i, b.j0, b.i0 + i + 1, b.j0 + b.ny);
            for (int j = 0; j < b.ny; ++j) sy[j] = F.sum(b.i0, b.j0 + j, b.i0 + b.nx, b.j0 + j + 1);
            const int kx = hole_cut(sx), ky = hole_cut(sy);
            if (kx >= 0) {
                dir = 0;
                k = kx;
            } else if (ky >= 0) {
                dir = 1;
                k = ky;
            } else {
                const auto ix = inflection_cut(sx), iy = inflection_cut(sy);
                if (ix.second >= 0 && (iy.second < 0 || ix.first >= iy.first)) {
                    dir = 0;
                    k = ix.second;
                } else if (iy.second >= 0) {
                    dir = 1;
                    k = iy.second;
                }
            }
        }
        if (dir < 0) {
            if (b.nx >= b.ny) {
                dir = 0;
                k = b.nx / 2;
            } else {
                dir = 1;
                k = b.ny / 2;
            }
        }
        if (dir == 0) {
            stack.push_back(IBox{b.i0 + k, b.j0, b.nx - k, b.ny});
            stack.push_back(IBox{b.i0, b.j0, k, b.ny});
        } else {
            stack.push_back(IBox{b.i0, b.j0 + k, b.nx, b.ny - k});
            stack.push_back(IBox{b.i0, b.j0, b.nx, k});
        }
    }
    return out;
}

}  // namespace

extern "C" {

long long claw_flag_grid_size(claw_ctx* ctx, int32_t L)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV) return -CLAW_EINVAL;
    return flag_grid_offset(ctx, L, ctx->nruns);
}

int claw_flag_cells(claw_ctx* ctx, int32_t L, const double* q, double tol, uint8_t* flags, void* stream)
{
    if (!ctx || L < 0 || L >= CLAW_MAXLEV || !q || !flags || !(tol >= 0.0)) return CLAW_EINVAL;
    if (!ctx->set[L]) return CLAW_ESTATE;
    DevGuard g(ctx->device);
    LevelDev& d = ctx->lev[L];
    if (d.nboxes == 0) return CLAW_OK;
    ctx->launches += 1;
    return cuda_rc(launch_flags(d.flagboxes, d.nboxes, d.max_rows, q, tol, flags, (cudaStream_t)stream));
}

int claw_regrid_boxes(claw_ctx* ctx, int32_t L, int32_t run, const uint8_t* flags, int32_t buffer, int32_t nest,
                      double cutoff, int32_t max_size, int32_t* boxes, int32_t max_boxes)
{
    if (!ctx || L < 0 || L + 1 >= CLAW_MAXLEV || run < 0 || run >= ctx->nruns) return -CLAW_EINVAL;
    if (!ctx->set[L]) return -CLAW_ESTATE;
    const claw_problem& p = ctx->runs[run];
    if (L + 1 >= p.nlev) return -CLAW_EINVAL;
    std::vector<claw_box> cover;
    for (const claw_box& b : ctx->lev[L].boxes)
        if (b.run == run) cover.push_back(b);
    return claw_cluster_flags(level_nx(p, L), level_ny(p, L), p.ratio[L + 1], cover.data(), (int32_t)cover.size(),
                              flags, buffer, nest, cutoff, max_size, boxes, max_boxes);
}

int claw_cluster_flags(int32_t NX, int32_t NY, int32_t r, const claw_box* cover, int32_t ncover, const uint8_t* flags,
                       int32_t buffer, int32_t nest, double cutoff, int32_t max_size, int32_t* boxes,
                       int32_t max_boxes)
{
    if (NX < 1 || NY < 1 || r < 1 || ncover < 0 || (ncover > 0 && !cover) || !flags || buffer < 0 || nest < 0 ||
        !(cutoff > 0.0 && cutoff <= 1.0) || max_size < 1 || max_boxes < 0 || (max_boxes > 0 && !boxes))
        return -CLAW_EINVAL;
    if ((long long)(NX + 1) * (NY + 1) >= (1LL << 31)) return -CLAW_EINVAL;
    buffer = std::min(buffer, std::max(NX, NY));   // wider reaches change nothing
    nest = std::min(nest, std::max(NX, NY));
    // scratch grids reused from call to call (no fresh pages per regrid); named through local
    // references, which the worker threads' lambdas capture (a thread_local named inside a
    // lambda would be the worker's own, empty instance)
    static thread_local std::vector<unsigned char> tl_f, tl_cov, tl_allowed, tl_rows, tl_near;
    static thread_local std::vector<int> tl_rlo, tl_rhi;
    std::vector<unsigned char>& f = tl_f;
    std::vector<unsigned char>& cov = tl_cov;
    std::vector<unsigned char>& allowed = tl_allowed;
    std::vector<unsigned char>& rows = tl_rows;
    std::vector<unsigned char>& near = tl_near;
    std::vector<int>& rlo = tl_rlo;
    std::vector<int>& rhi = tl_rhi;
    // bounding box of the flags: the grids below cover only the window of it grown by `buffer`
    // (clustering starts by trimming to the flags' bounding box, so the boxes are the same as
    // over the whole level)
    rlo.assign(NY, NX);
    rhi.assign(NY, -1);
    parallel_for(NY, [&](int ja, int jb) {
        for (int j = ja; j < jb; ++j) {
            const uint8_t* row = flags + (size_t)j * NX;
            int lo = 0;
            while (lo < NX && !row[lo]) ++lo;
            if (lo == NX) continue;
            int hi = NX - 1;
            while (!row[hi]) --hi;
            rlo[j] = lo;
            rhi[j] = hi;
        }
    });
    int bi0 = NX, bi1 = -1, bj0 = -1, bj1 = -1;
    for (int j = 0; j < NY; ++j)
        if (rhi[j] >= 0) {
            bi0 = std::min(bi0, rlo[j]);
            bi1 = std::max(bi1, rhi[j]);
            if (bj0 < 0) bj0 = j;
            bj1 = j;
        }
    if (bi1 < 0) return 0;
    const int wi0 = std::max(0, bi0 - buffer), wi1 = std::min(NX, bi1 + 1 + buffer);
    const int wj0 = std::max(0, bj0 - buffer), wj1 = std::min(NY, bj1 + 1 + buffer);
    const int WX = wi1 - wi0, WY = wj1 - wj0;
    // flags grown by `buffer` cells (square neighbourhood, clipped to the domain; no flag lies
    // outside the window)
    dilate(flags + (size_t)wj0 * NX + wi0, NX, WX, WY, buffer, false, rows, f);
    // keep cells `nest` cells inside the level's coverage: no uncovered cell in the square of
    // radius `nest` around the cell, the square clipped to the domain (the domain outside counts
    // as covered); the coverage grid spans the window grown by `nest`, so the square of a window
    // cell clipped to that grid is the square clipped to the domain
    const int ci0 = std::max(0, wi0 - nest), ci1 = std::min(NX, wi1 + nest);
    const int cj0 = std::max(0, wj0 - nest), cj1 = std::min(NY, wj1 + nest);
    const int CX = ci1 - ci0, CY = cj1 - cj0;
    cov.assign((size_t)CX * CY, 0);
    for (int k = 0; k < ncover; ++k) {
        const claw_box& b = cover[k];
        const int x0 = std::max(ci0, b.ilo), x1 = std::min(ci1, b.ilo + b.nx);
        const int y0 = std::max(cj0, b.jlo), y1 = std::min(cj1, b.jlo + b.ny);
        for (int j = y0; j < y1; ++j) std::memset(&cov[(size_t)(j - cj0) * CX + (x0 - ci0)], 1, std::max(0, x1 - x0));
    }
    dilate(cov.data(), CX, CX, CY, nest, true, rows, near);
    allowed.resize((size_t)WX * WY);
    parallel_for(WY, [&](int ja, int jb) {
        for (int j = ja; j < jb; ++j) {
            const unsigned char* nr = &near[(size_t)(j + wj0 - cj0) * CX + (wi0 - ci0)];
            for (int i = 0; i < WX; ++i) {
                const bool ok = !nr[i];
                allowed[(size_t)j * WX + i] = ok;
                if (!ok) f[(size_t)j * WX + i] = 0;
            }
        }
    });
    std::vector<IBox> out = cluster_flags(f, WX, WY, cutoff, std::max(1, max_size / r), allowed);
    for (IBox& b : out) {
        b.i0 += wi0;
        b.j0 += wj0;
    }
    if ((long long)out.size() > max_boxes) return -CLAW_ENOMEM;
    for (size_t k = 0; k < out.size(); ++k) {
        boxes[4 * k] = out[k].i0 * r;
        boxes[4 * k + 1] = out[k].j0 * r;
        boxes[4 * k + 2] = out[k].nx * r;
        boxes[4 * k + 3] = out[k].ny * r;
    }
    return (int)out.size();
}

int claw_regrid_transfer(claw_ctx* ctx, int32_t L, const claw_box* old_boxes, int32_t n_old, const double* q_old,
                         double* q_new, const double* q_coarse, void* stream)
{
    if (!ctx || L < 1 || L >= CLAW_MAXLEV || n_old < 0 || (n_old > 0 && (!old_boxes || !q_old)) || !q_new ||
        !q_coarse)
        return CLAW_EINVAL;
    if (!ctx->set[L] || !ctx->set[L - 1]) return CLAW_ESTATE;
    DevGuard g(ctx->device);
    const LevelDev& d = ctx->lev[L];
    const LevelDev& c = ctx->lev[L - 1];
    // the old boxes must lie in their run's level (they index the level-wide grid)
    for (int n = 0; n < n_old; ++n) {
        const claw_box& b = old_boxes[n];
        if (b.run < 0 || b.run >= ctx->nruns || L >= ctx->runs[b.run].nlev) return CLAW_EINVAL;
        const int NX = level_nx(ctx->runs[b.run], L), NY = level_ny(ctx->runs[b.run], L);
        if (b.nx < 1 || b.ny < 1 || b.ilo < 0 || b.jlo < 0 || b.ilo + b.nx > NX || b.jlo + b.ny > NY || b.qoff < 0)
            return CLAW_EINVAL;
    }
    auto xfer = [](const claw_box& b) { return XferBox{b.qoff, b.run, b.ilo, b.jlo, b.nx, b.ny, 0}; };
    std::vector<XferBox> nb(d.nboxes), ob(n_old), cb(c.boxes.size());
    int max_rows = 0;
    for (int n = 0; n < d.nboxes; ++n) nb[n] = xfer(d.boxes[n]), max_rows = std::max(max_rows, d.boxes[n].ny);
    for (int n = 0; n < n_old; ++n) ob[n] = xfer(old_boxes[n]), max_rows = std::max(max_rows, old_boxes[n].ny);
    for (size_t n = 0; n < c.boxes.size(); ++n) cb[n] = xfer(c.boxes[n]), max_rows = std::max(max_rows, c.boxes[n].ny);
    // per run: where its level grids start and their pitch
    std::vector<long long> fgoff(ctx->nruns), cgoff(ctx->nruns);
    std::vector<int> fpitch(ctx->nruns), cpitch(ctx->nruns);
    long long fcells = 0, ccells = 0;
    for (int q = 0; q < ctx->nruns; ++q) {
        const claw_problem& p = ctx->runs[q];
        fgoff[q] = fcells;
        cgoff[q] = ccells;
        fpitch[q] = L < p.nlev ? level_nx(p, L) : 0;
        cpitch[q] = L - 1 < p.nlev ? level_nx(p, L - 1) : 0;
        if (L < p.nlev) fcells += (long long)level_nx(p, L) * level_ny(p, L);
        if (L - 1 < p.nlev) ccells += (long long)level_nx(p, L - 1) * level_ny(p, L - 1);
    }
    const size_t need = (size_t)(fcells + ccells);
    if (need > ctx->xgrid_cap) {
        cudaFree(ctx->xgrid);
        ctx->xgrid = nullptr;
        ctx->xgrid_cap = 0;
        if (cudaMalloc((void**)&ctx->xgrid, need * sizeof(int)) != cudaSuccess) return CLAW_ENOMEM;
        ctx->xgrid_cap = need;
    }
    XferBox *dnb = nullptr, *dob = nullptr, *dcb = nullptr;
    long long *dfgoff = nullptr, *dcgoff = nullptr;
    int *dfpitch = nullptr, *dcpitch = nullptr, *derr = nullptr;
    const std::vector<int> zero(1, 0);
    ArenaPack pack;
    pack.add(&dnb, nb);
    pack.add(&dob, ob);
    pack.add(&dcb, cb);
    pack.add(&dfgoff, fgoff);
    pack.add(&dcgoff, cgoff);
    pack.add(&dfpitch, fpitch);
    pack.add(&dcpitch, cpitch);
    pack.add(&derr, zero);
    int rc = pack.commit(ctx->scratch);
    if (rc) return rc;
    XferGrids gr{dfgoff, dfpitch, dcgoff, dcpitch, ctx->xgrid, ctx->xgrid + fcells};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_regrid_transfer(dnb, d.nboxes, dob, n_old, dcb, (int)cb.size(), max_rows, d.ratio, gr,
                                           fcells, ccells, q_old, q_coarse, q_new, derr, s);
    ctx->launches += 3;
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the scratch tables are reused by the next call
    if (e != cudaSuccess) return CLAW_ECUDA;
    return herr ? CLAW_EINVAL : CLAW_OK;   // a new box not nested in the coarse level
}

}  // extern "C"

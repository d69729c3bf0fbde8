// claw_api.cu -- the C ABI of libclaw.so (include/claw.h): context, host-side validation of
// the box sets of Sec. 2.2, the task tables of the ghost fill (Sec. 2.2 items 1-3) and of the
// averaging (Sec. 2.3), tensor-map descriptors for the staged tiles, and the launches.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <exception>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unistd.h>
#include <utility>
#include <vector>

#include "claw_internal.h"

using namespace claw;

struct TmapCache {
    const double* q = nullptr;
    int tx = 0, ty = 0;
    void* dev = nullptr;   // CUtensorMap[nboxes]
    unsigned long long stamp = 0;
    bool pinned = false;   // handed to a stream capture: a graph may read it until the level is rebuilt
};

struct claw_ctx {
    int device = 0;
    int nsm = 0;
    int nruns = 0;
    std::vector<claw_problem> runs;
    int limiter = 4, order = 2, transverse = 2, medium = 0;
    double rho0 = 1, K0 = 1;
    int system = CLAW_SYS_ACOUSTICS;
    double grav = 0;
    int kind() const { return system == CLAW_SYS_SHALLOW_WATER ? KIND_SWE : medium; }
    LevelDev lev[CLAW_MAXLEV];
    bool set[CLAW_MAXLEV] = {};
    // device scalars
    int* err = nullptr;
    double* minh = nullptr;    // [CLAW_MAXLEV][nruns] min(dx, dy) of each level
    double* cflv = nullptr;    // [nruns] desired CFL
    unsigned int* done = nullptr;   // CTA completion counter of the fused dt update
    // per-level tiles ordered by box for the per-box launches
    std::vector<int> ptile_start[CLAW_MAXLEV];
    TileDev* ptiles[CLAW_MAXLEV] = {};
    // per-level tiles of the adjoint kernel (its own fixed tile edge)
    TileDev* atiles[CLAW_MAXLEV] = {};
    int natiles[CLAW_MAXLEV] = {};
    std::vector<TmapCache> tmaps[CLAW_MAXLEV];
    unsigned long long stamp = 0;
    std::atomic<long long> launches{0};
    bool tma_ok[CLAW_MAXLEV] = {};
    DevArena scratch;   // the transfer tables of a regrid
    unsigned wait_polls = kWaitPolls;   // first-wait bound of the staged step kernels
};

namespace {

struct DevGuard {   // makes the context's device current for the scope of a call
    int prev = -1;
    explicit DevGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int level_nx(const claw_problem& p, int L)
{
    long long n = p.nx0;
    for (int l = 1; l <= L; ++l) n *= p.ratio[l];
    return (int)n;
}
int level_ny(const claw_problem& p, int L)
{
    long long n = p.ny0;
    for (int l = 1; l <= L; ++l) n *= p.ratio[l];
    return (int)n;
}
double level_dx(const claw_problem& p, int L) { return (p.xhi - p.xlo) / level_nx(p, L); }
double level_dy(const claw_problem& p, int L) { return (p.yhi - p.ylo) / level_ny(p, L); }

// physical-boundary image of index k on [0, n): clamp (extrapolation), wrap (periodic),
// mirror with the normal velocity negated (wall)
int bc_map(int k, int n, int bclo, int bchi, int* flip)
{
    *flip = 0;
    if (k < 0) {
        if (bclo == CLAW_BC_PERIODIC) return ((k % n) + n) % n;
        if (bclo == CLAW_BC_WALL) { *flip = 1; return -1 - k; }
        return 0;
    }
    if (k >= n) {
        if (bchi == CLAW_BC_PERIODIC) return k % n;
        if (bchi == CLAW_BC_WALL) { *flip = 1; return 2 * n - 1 - k; }
        return n - 1;
    }
    return k;
}

int floordiv(int a, int r) { return a >= 0 ? a / r : -((-a + r - 1) / r); }

// boxes of one (run, level), bucketed for point lookups
struct Locator {
    static constexpr int B = 16;
    std::unordered_map<long long, std::vector<int>> buckets;
    const std::vector<claw_box>* boxes = nullptr;
    std::vector<int> idx;   // global box index of each entry

    static long long key(int bi, int bj) { return ((long long)bi << 32) ^ (unsigned)bj; }

    void add(const claw_box& b, int n)
    {
        for (int bj = floordiv(b.jlo, B); bj <= floordiv(b.jlo + b.ny - 1, B); ++bj)
            for (int bi = floordiv(b.ilo, B); bi <= floordiv(b.ilo + b.nx - 1, B); ++bi)
                buckets[key(bi, bj)].push_back(n);
    }
    int find(int i, int j) const
    {
        auto it = buckets.find(key(floordiv(i, B), floordiv(j, B)));
        if (it == buckets.end()) return -1;
        for (int n : it->second) {
            const claw_box& b = (*boxes)[n];
            if (i >= b.ilo && i < b.ilo + b.nx && j >= b.jlo && j < b.jlo + b.ny) return n;
        }
        return -1;
    }
};

long long cell_off(const claw_box& b, int i, int j)   // plane-0 element of level cell (i, j)
{
    return b.qoff + (long long)(j - b.jlo + CLAW_MBC) * (b.nx + 2 * CLAW_MBC) + (i - b.ilo + CLAW_MBC);
}
long long plane_of(const claw_box& b) { return (long long)(b.nx + 4) * (b.ny + 4); }

// fn(lo, hi) over [0, n) in contiguous chunks on up to 16 host threads (ghost tables, regrid
// grids), at least `grain` items a thread
// The host threads behind parallel_for: started once and kept, since starting 16 threads for
// every pass of a regrid cost milliseconds.  run(n, fn) calls fn(0..n-1) on the workers and the
// caller and returns when all are done; one run at a time.  A run from inside a worker (nested),
// or in a process forked from the one that started the workers, goes serially.  The pool is
// never destroyed: its idle workers end with the process.
class HostPool {
public:
    static HostPool& get()
    {
        static HostPool* pool = new HostPool;
        return *pool;
    }
    int threads() const { return getpid() == pid_ ? (int)workers_.size() + 1 : 1; }
    void run(int n, const std::function<void(int)>& fn)
    {
        if (n <= 1 || in_worker() || threads() == 1) {
            for (int k = 0; k < n; ++k) fn(k);
            return;
        }
        std::lock_guard<std::mutex> one_run(run_m_);
        Run r(fn, n);
        {
            std::lock_guard<std::mutex> lk(m_);
            cur_ = &r;
            ++gen_;
        }
        cv_.notify_all();
        std::exception_ptr err;
        in_worker() = true;   // a parallel_for inside an item of this run goes serially
        try {
            work(r);
        } catch (...) {   // stop handing out items, let the workers finish theirs, then rethrow
            err = std::current_exception();
            std::lock_guard<std::mutex> lk(m_);
            r.left -= std::max(0, r.n - r.next.exchange(r.n)) + 1;
        }
        in_worker() = false;
        // r lives on this frame: return only when every item is done and no worker holds r
        {
            std::unique_lock<std::mutex> lk(m_);
            done_.wait(lk, [&] { return r.left <= 0 && r.users == 0; });
            cur_ = nullptr;
        }
        if (err) std::rethrow_exception(err);
    }

private:
    struct Run {
        Run(const std::function<void(int)>& f, int count) : fn(f), n(count), left(count) {}
        const std::function<void(int)>& fn;
        const int n;
        std::atomic<int> next{0};
        int left;        // items not yet done (under m_)
        int users = 0;   // workers holding this run (under m_)
    };
    HostPool() : pid_(getpid())
    {
        const int hw = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        for (int t = 1; t < hw; ++t) workers_.emplace_back([this] { loop(); });
    }
    static bool& in_worker()
    {
        static thread_local bool w = false;
        return w;
    }
    void work(Run& r)   // take items of r until none are left
    {
        for (int k; (k = r.next.fetch_add(1)) < r.n;) {
            r.fn(k);
            std::lock_guard<std::mutex> lk(m_);
            if (--r.left == 0) done_.notify_all();
        }
    }
    void loop()
    {
        in_worker() = true;
        unsigned long seen = 0;
        for (;;) {
            Run* r;
            {
                std::unique_lock<std::mutex> lk(m_);
                cv_.wait(lk, [&] { return gen_ != seen && cur_ != nullptr; });
                seen = gen_;
                r = cur_;
                ++r->users;
            }
            work(*r);
            std::lock_guard<std::mutex> lk(m_);
            if (--r->users == 0 && r->left == 0) done_.notify_all();
        }
    }
    const pid_t pid_;
    std::vector<std::thread> workers_;
    std::mutex run_m_, m_;
    std::condition_variable cv_, done_;
    Run* cur_ = nullptr;
    unsigned long gen_ = 0;
};

template <typename F>
void parallel_for(int n, F fn, int grain = 64)
{
    HostPool& pool = HostPool::get();
    const int nt = std::max(1, std::min(pool.threads(), n / std::max(1, grain)));
    if (nt <= 1) {
        fn(0, n);
        return;
    }
    pool.run(nt, [&](int t) { fn((int)((long long)n * t / nt), (int)((long long)n * (t + 1) / nt)); });
}

// The tables of one rebuild: each table is one or more host pieces laid out back to back from a
// 256-byte aligned offset.  commit() gathers the pieces into the arena's pinned staging buffer on
// host threads, copies it to the device in one call and sets the table pointers.  The pieces are
// read by commit(), so they must live until then.
struct ArenaPack {
    struct Piece {
        const void* src;
        size_t bytes, off;
    };
    std::vector<Piece> pieces;
    std::vector<std::function<void(char*)>> place;
    size_t size = 0;
    // a table from nparts vectors, part(k) being the k-th
    template <class T, class Part>
    void add_parts(T** dst, int nparts, Part part)
    {
        *dst = nullptr;
        const size_t base = (size + 255) / 256 * 256;
        size_t off = base;
        for (int k = 0; k < nparts; ++k) {
            const std::vector<T>& v = part(k);
            if (v.empty()) continue;
            pieces.push_back(Piece{v.data(), v.size() * sizeof(T), off});
            off += v.size() * sizeof(T);
        }
        if (off == base) return;
        size = off;
        place.push_back([dst, base](char* b) { *dst = reinterpret_cast<T*>(b + base); });
    }
    template <class T>
    void add(T** dst, const std::vector<T>& v)
    {
        add_parts(dst, 1, [&](int) -> const std::vector<T>& { return v; });
    }
    // the tables laid out in h (size bytes)
    void gather(char* h) const
    {
        parallel_for((int)pieces.size(), [&](int k0, int k1) {
            for (int k = k0; k < k1; ++k) std::memcpy(h + pieces[k].off, pieces[k].src, pieces[k].bytes);
        }, 256);
    }
    // The arena may still be read by kernels in flight from before the rebuild: the device is
    // synchronised before it is overwritten.
    int commit(DevArena& a)
    {
        if (size == 0) return CLAW_OK;
        if (a.dev && cudaDeviceSynchronize() != cudaSuccess) return CLAW_ECUDA;
        if (size > a.host_cap) {
            cudaFreeHost(a.host);
            a.host = nullptr;
            a.host_cap = 0;
            if (cudaMallocHost((void**)&a.host, size + size / 4) != cudaSuccess) return CLAW_ENOMEM;
            a.host_cap = size + size / 4;
        }
        gather(a.host);
        if (size > a.cap) {
            cudaFree(a.dev);
            a.dev = nullptr;
            a.cap = 0;
            if (cudaMalloc((void**)&a.dev, size + size / 4) != cudaSuccess) return CLAW_ENOMEM;
            a.cap = size + size / 4;
        }
        if (cudaMemcpy(a.dev, a.host, size, cudaMemcpyHostToDevice) != cudaSuccess) return CLAW_ECUDA;
        for (auto& f : place) f(a.dev);
        return CLAW_OK;
    }
};

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
    ctx->set[L] = false;
}

// tiles of a level for its tiling: sorted by area (largest first) for the persistent walk,
// and grouped by box for the per-box launches
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
                T.pad = 0;
                t.push_back(T);
            }
    }
    start.push_back((int)t.size());
    // (the pieces are read by pack.commit: t keeps the box order, d.htiles the sorted copy)
    ArenaPack pack;
    pack.add(&ctx->ptiles[L], t);
    ctx->ptile_start[L] = start;
    d.htiles = t;
    std::stable_sort(d.htiles.begin(), d.htiles.end(), [](const TileDev& a, const TileDev& b) {
        return (int)a.tx * a.ty > (int)b.tx * b.ty;
    });
    d.ntiles = (int)d.htiles.size();
    for (auto& tm : ctx->tmaps[L]) cudaFree(tm.dev);
    ctx->tmaps[L].clear();
    pack.add(&d.tiles, d.htiles);
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
                T.pad = 0;
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

struct GhostEntry {
    int gi, gj;         // ghost cell (level index)
    int src;            // source box or -1 (interpolation)
    long long soff;     // source plane-0 element
    int flags;
};

// ghost tasks of one level: copy rectangles and interpolated cells
// interpolation of the fine cell (si, sj) of level L (inside the domain) from level L-1 into
// the element dst of plane stride dplane; flags: sign flips of the destination (walls)
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


// ghost tasks of one box: copy rectangles, interpolated cells and (for pulled ghosts) its ring
struct BoxGhosts {
    std::vector<CopyRect> rects;
    std::vector<InterpCell> cells;
    std::vector<longlong2> ring;
    bool want_ring = false, ring_ok = true;
    int rc = CLAW_OK;
};

// ghost tables of a level, kept per box (the device tables are their concatenation in box order)
struct GhostTables {
    std::vector<BoxGhosts> per;
    size_t nrects = 0, ncells = 0, nring = 0;
    std::vector<int> start;   // blocks of the copy kernel over the concatenated rectangles
    bool ring_ok = true;
};

int build_ghost_tables(claw_ctx* ctx, int L, GhostTables& gt, bool want_ring)
{
    LevelDev& d = ctx->lev[L];
    std::vector<Locator> loc(ctx->nruns), cloc(ctx->nruns);
    for (int r = 0; r < ctx->nruns; ++r) {
        loc[r].boxes = &d.boxes;
        if (L > 0) cloc[r].boxes = &ctx->lev[L - 1].boxes;
    }
    for (int n = 0; n < d.nboxes; ++n) loc[d.boxes[n].run].add(d.boxes[n], n);
    if (L > 0)
        for (int n = 0; n < (int)ctx->lev[L - 1].boxes.size(); ++n)
            cloc[ctx->lev[L - 1].boxes[n].run].add(ctx->lev[L - 1].boxes[n], n);

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
    std::vector<Locator> floc(ctx->nruns), cloc(ctx->nruns);
    for (int q = 0; q < ctx->nruns; ++q) {
        floc[q].boxes = &f.boxes;
        cloc[q].boxes = &c.boxes;
    }
    for (int n = 0; n < f.nboxes; ++n) floc[f.boxes[n].run].add(f.boxes[n], n);
    for (int n = 0; n < (int)c.boxes.size(); ++n) cloc[c.boxes[n].run].add(c.boxes[n], n);
    auto wrap = [](int k, int n, int lo, int hi, bool& ok) {
        ok = true;
        if (k >= 0 && k < n) return k;
        if ((k < 0 && lo == CLAW_BC_PERIODIC) || (k >= n && hi == CLAW_BC_PERIODIC)) return ((k % n) + n) % n;
        ok = false;
        return k;
    };
    recs.clear();
    for (int nf = 0; nf < f.nboxes; ++nf) {
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
            recs.push_back(R);
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

// coarse cells of level L-1 covered by each box of level L
void build_avg_tables(claw_ctx* ctx, int L, std::vector<AvgRect>& out)
{
    const LevelDev& f = ctx->lev[L];
    const LevelDev& c = ctx->lev[L - 1];
    const int r = f.ratio;
    for (const claw_box& F : f.boxes)
        for (const claw_box& C : c.boxes) {
            if (C.run != F.run) continue;
            const int i0 = std::max(F.ilo / r, C.ilo), i1 = std::min((F.ilo + F.nx) / r, C.ilo + C.nx);
            const int j0 = std::max(F.jlo / r, C.jlo), j1 = std::min((F.jlo + F.ny) / r, C.jlo + C.ny);
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
            out.push_back(a);
        }
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

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? CLAW_OK : CLAW_ECUDA; }

bool valid_level(claw_ctx* ctx, int L) { return ctx && L >= 0 && L < CLAW_MAXLEV && ctx->set[L]; }

StepArgs make_args(claw_ctx* ctx, int L, const double* q_old, double* q_new, const double* aux,
                   const double* dt, double* smax)
{
    const LevelDev& d = ctx->lev[L];
    StepArgs a;
    a.patches = d.patches;
    a.tiles = d.tiles;
    a.tmaps = nullptr;
    a.ntiles = d.ntiles;
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
    // disjointness within each run (bucketed)
    {
        std::vector<Locator> loc(ctx->nruns);
        for (int r = 0; r < ctx->nruns; ++r) loc[r].boxes = &d.boxes;
        for (int n = 0; n < nboxes; ++n) {
            const claw_box& b = boxes[n];
            // compare with boxes already added that share a bucket
            for (int bj = floordiv(b.jlo, Locator::B); bj <= floordiv(b.jlo + b.ny - 1, Locator::B); ++bj)
                for (int bi = floordiv(b.ilo, Locator::B); bi <= floordiv(b.ilo + b.nx - 1, Locator::B); ++bi) {
                    auto it = loc[b.run].buckets.find(Locator::key(bi, bj));
                    if (it == loc[b.run].buckets.end()) continue;
                    for (int m : it->second) {
                        const claw_box& o = boxes[m];
                        if (b.ilo < o.ilo + o.nx && o.ilo < b.ilo + b.nx && b.jlo < o.jlo + o.ny &&
                            o.jlo < b.jlo + b.ny)
                            return CLAW_EINVAL;
                    }
                }
            loc[b.run].add(b, n);
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
    d.tx = ctx->kind() == KIND_SWE ? 16 : 32;
    d.ty = ctx->kind() == KIND_SWE ? 16 : 32;
    d.staging = even ? 1 : 0;
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
    if (d.tx == tx && d.ty == ty) return CLAW_OK;
    d.tx = tx;
    d.ty = ty;
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
    const int per_sm = step_max_ctas_per_sm(ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging);
    if (per_sm <= 0) return CLAW_ECUDA;
    const int grid = std::min(d.ntiles, per_sm * ctx->nsm);
    ctx->launches += 1;
    return cuda_rc(launch_step(a, ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, grid, s));
}

static int level_advance(claw_ctx* ctx, int32_t L, const double* q_old, double* q_new, const double* aux, double* dt,
                         double* smax, int32_t flags, const double* qc_old, const double* qc_new, double tau,
                         bool interp, void* stream)
{
    int rc = check_step_args(ctx, L, q_old, q_new, aux, dt, smax);
    if (rc) return rc;
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
                                            false, a.interp != nullptr);
    if (per_sm <= 0) return CLAW_ECUDA;
    const int grid = std::min(d.ntiles, per_sm * ctx->nsm);
    ctx->launches += 1;
    cudaError_t e = launch_step(a, ctx->kind(), ctx->limiter, d.tx, d.ty, d.nt, staging, grid, s);
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
    std::vector<claw_box> olds(old_boxes, old_boxes + n_old);
    std::vector<Locator> oloc(ctx->nruns), cloc(ctx->nruns);
    for (int q = 0; q < ctx->nruns; ++q) {
        oloc[q].boxes = &olds;
        cloc[q].boxes = &ctx->lev[L - 1].boxes;
    }
    for (int n = 0; n < n_old; ++n) {
        if (olds[n].run < 0 || olds[n].run >= ctx->nruns) return CLAW_EINVAL;
        oloc[olds[n].run].add(olds[n], n);
    }
    for (int n = 0; n < (int)ctx->lev[L - 1].boxes.size(); ++n)
        cloc[ctx->lev[L - 1].boxes[n].run].add(ctx->lev[L - 1].boxes[n], n);
    const int r = d.ratio;
    // per new box, independently (threads): rectangles copied from old boxes, and row runs
    // interpolated from the coarse level where no old box covers it
    struct BoxTransfer {
        std::vector<RectCopy> copies;
        std::vector<InterpRun> runs;
        int rc = CLAW_OK;
    };
    std::vector<BoxTransfer> per(d.nboxes);
    auto one_box = [&](const claw_box& b, BoxTransfer& out) -> int {
        std::vector<RectCopy>& copies = out.copies;
        std::vector<InterpRun>& runs = out.runs;
        std::vector<unsigned char> mask;
        // old boxes overlapping b: copied rectangles
        mask.assign((size_t)b.nx * b.ny, 0);
        std::vector<int> seen;
        for (int bj = floordiv(b.jlo, Locator::B); bj <= floordiv(b.jlo + b.ny - 1, Locator::B); ++bj)
            for (int bi = floordiv(b.ilo, Locator::B); bi <= floordiv(b.ilo + b.nx - 1, Locator::B); ++bi) {
                auto it = oloc[b.run].buckets.find(Locator::key(bi, bj));
                if (it == oloc[b.run].buckets.end()) continue;
                for (int m : it->second) {
                    if (std::find(seen.begin(), seen.end(), m) != seen.end()) continue;
                    seen.push_back(m);
                    const claw_box& o = olds[m];
                    const int i0 = std::max(b.ilo, o.ilo), i1 = std::min(b.ilo + b.nx, o.ilo + o.nx);
                    const int j0 = std::max(b.jlo, o.jlo), j1 = std::min(b.jlo + b.ny, o.jlo + o.ny);
                    if (i0 >= i1 || j0 >= j1) continue;
                    copies.push_back(RectCopy{cell_off(b, i0, j0), cell_off(o, i0, j0), plane_of(b), plane_of(o), i1 - i0,
                                              j1 - j0, b.nx + 4, o.nx + 4});
                    for (int j = j0; j < j1; ++j)
                        std::memset(&mask[(size_t)(j - b.jlo) * b.nx + (i0 - b.ilo)], 1, (size_t)(i1 - i0));
                }
            }
        // the rest: row runs of cells over one coarse box each
        for (int j = 0; j < b.ny; ++j) {
            int i = 0;
            while (i < b.nx) {
                if (mask[(size_t)j * b.nx + i]) {
                    ++i;
                    continue;
                }
                const int gj = b.jlo + j, gi = b.ilo + i;
                const int cm = cloc[b.run].find(floordiv(gi, r), floordiv(gj, r));
                if (cm < 0) return CLAW_EINVAL;   // the new box is not nested in the coarse level
                const claw_box& cb = ctx->lev[L - 1].boxes[cm];
                int e = i + 1;
                while (e < b.nx && !mask[(size_t)j * b.nx + e] && floordiv(b.ilo + e, r) < cb.ilo + cb.nx) ++e;
                InterpRun R;
                R.dst = cell_off(b, gi, gj);
                R.dplane = plane_of(b);
                R.cbase = cb.qoff;
                R.cplane = plane_of(cb);
                R.n = e - i;
                R.gi0 = gi;
                R.gj = gj;
                R.cilo = cb.ilo;
                R.cjlo = cb.jlo;
                R.cpitch = cb.nx + 4;
                R.r = r;
                R.pad = 0;
                runs.push_back(R);
                i = e;
            }
        }
        return CLAW_OK;
    };
    parallel_for(d.nboxes, [&](int n0, int n1) {
        for (int n = n0; n < n1; ++n) per[n].rc = one_box(d.boxes[n], per[n]);
    });
    size_t ncopies = 0, nruns = 0;
    for (const BoxTransfer& t : per) {
        if (t.rc) return t.rc;
        ncopies += t.copies.size();
        nruns += t.runs.size();
    }
    RectCopy* dc = nullptr;
    InterpRun* di = nullptr;
    ArenaPack pack;
    pack.add_parts(&dc, d.nboxes, [&](int n) -> const std::vector<RectCopy>& { return per[n].copies; });
    pack.add_parts(&di, d.nboxes, [&](int n) -> const std::vector<InterpRun>& { return per[n].runs; });
    int rc = pack.commit(ctx->scratch);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = launch_rect_copy(dc, (int)ncopies, q_old, q_new, s);
        if (e == cudaSuccess) e = launch_interp_runs(di, (int)nruns, q_coarse, q_new, s);
        ctx->launches += (ncopies > 0) + (nruns > 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the scratch tables are reused by the next call
    }
    return rc ? rc : cuda_rc(e);
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

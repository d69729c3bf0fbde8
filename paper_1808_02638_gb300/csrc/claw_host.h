// claw_host.h -- host side of libclaw.so shared by its translation units (claw_api.cu: the C
// ABI entry points; claw_tables.cu: the device task tables of a level; claw_clustering.cu: flagging
// and Berger-Rigoutsos clustering of the regrid): the context, level geometry, box lookup, the
// host thread pool and the packing of tables into device arenas.  Not part of the public ABI.
#pragma once

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

inline int floordiv(int a, int r) { return a >= 0 ? a / r : -((-a + r - 1) / r); }

// The boxes of one run on one level, bucketed by B x B cells of the level (compressed rows:
// bucket k lists its boxes in items[start[k] .. start[k+1]), in box order).
struct Locator {
    static constexpr int B = 16;
    const std::vector<claw_box>* boxes = nullptr;
    int nx = 0, ny = 0, nbx = 0, nby = 0;
    std::vector<int> start, items;

    // boxes: the level's boxes; sel: the indices of the run's boxes; the level is nx x ny
    void build(const std::vector<claw_box>* bx, const std::vector<int>& sel, int nx_, int ny_)
    {
        boxes = bx;
        nx = nx_;
        ny = ny_;
        nbx = (nx + B - 1) / B;
        nby = (ny + B - 1) / B;
        start.assign((size_t)nbx * nby + 1, 0);
        auto span = [&](const claw_box& b, int& bi0, int& bi1, int& bj0, int& bj1) {
            bi0 = std::max(0, b.ilo / B);
            bj0 = std::max(0, b.jlo / B);
            bi1 = std::min(nbx - 1, (b.ilo + b.nx - 1) / B);
            bj1 = std::min(nby - 1, (b.jlo + b.ny - 1) / B);
        };
        for (int n : sel) {
            int bi0, bi1, bj0, bj1;
            span((*bx)[n], bi0, bi1, bj0, bj1);
            for (int bj = bj0; bj <= bj1; ++bj)
                for (int bi = bi0; bi <= bi1; ++bi) ++start[(size_t)bj * nbx + bi + 1];
        }
        for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
        items.assign(start.back(), 0);
        std::vector<int> fill(start.begin(), start.end() - 1);
        for (int n : sel) {
            int bi0, bi1, bj0, bj1;
            span((*bx)[n], bi0, bi1, bj0, bj1);
            for (int bj = bj0; bj <= bj1; ++bj)
                for (int bi = bi0; bi <= bi1; ++bi) items[fill[(size_t)bj * nbx + bi]++] = n;
        }
    }
    // the box holding level cell (i, j), or -1
    int find(int i, int j) const
    {
        if (i < 0 || j < 0 || i >= nx || j >= ny) return -1;
        const size_t k = (size_t)(j / B) * nbx + i / B;
        for (int t = start[k]; t < start[k + 1]; ++t) {
            const claw_box& b = (*boxes)[items[t]];
            if (i >= b.ilo && i < b.ilo + b.nx && j >= b.jlo && j < b.jlo + b.ny) return items[t];
        }
        return -1;
    }
    // f(n) for the boxes listed in the buckets meeting cells [i0, i1) x [j0, j1) (a box can come
    // more than once)
    template <class F>
    void each(int i0, int j0, int i1, int j1, F f) const
    {
        const int bi0 = std::max(0, floordiv(i0, B)), bj0 = std::max(0, floordiv(j0, B));
        const int bi1 = std::min(nbx - 1, floordiv(i1 - 1, B)), bj1 = std::min(nby - 1, floordiv(j1 - 1, B));
        for (int bj = bj0; bj <= bj1; ++bj)
            for (int bi = bi0; bi <= bi1; ++bi)
                for (int t = start[(size_t)bj * nbx + bi]; t < start[(size_t)bj * nbx + bi + 1]; ++t) f(items[t]);
    }
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
    std::vector<Locator> loc[CLAW_MAXLEV];   // per level and run: the boxes bucketed (built by claw_set_level)
    int* xgrid = nullptr;      // the index grids of a regrid transfer (fine then coarse), grown on use
    size_t xgrid_cap = 0;      // ints
    unsigned wait_polls = kWaitPolls;   // first-wait bound of the staged step kernels
};

namespace claw_host {

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

inline int level_nx(const claw_problem& p, int L)
{
    long long n = p.nx0;
    for (int l = 1; l <= L; ++l) n *= p.ratio[l];
    return (int)n;
}
inline int level_ny(const claw_problem& p, int L)
{
    long long n = p.ny0;
    for (int l = 1; l <= L; ++l) n *= p.ratio[l];
    return (int)n;
}
inline double level_dx(const claw_problem& p, int L) { return (p.xhi - p.xlo) / level_nx(p, L); }
inline double level_dy(const claw_problem& p, int L) { return (p.yhi - p.ylo) / level_ny(p, L); }

// physical-boundary image of index k on [0, n): clamp (extrapolation), wrap (periodic),
// mirror with the normal velocity negated (wall)
inline int bc_map(int k, int n, int bclo, int bchi, int* flip)
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


// boxes of one (run, level), bucketed for point lookups
inline long long cell_off(const claw_box& b, int i, int j)   // plane-0 element of level cell (i, j)
{
    return b.qoff + (long long)(j - b.jlo + CLAW_MBC) * (b.nx + 2 * CLAW_MBC) + (i - b.ilo + CLAW_MBC);
}
inline long long plane_of(const claw_box& b) { return (long long)(b.nx + 4) * (b.ny + 4); }

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

inline int cuda_rc(cudaError_t e) { return e == cudaSuccess ? CLAW_OK : CLAW_ECUDA; }

inline bool valid_level(claw_ctx* ctx, int L) { return ctx && L >= 0 && L < CLAW_MAXLEV && ctx->set[L]; }

struct GhostEntry {
    int gi, gj;         // ghost cell (level index)
    int src;            // source box or -1 (interpolation)
    long long soff;     // source plane-0 element
    int flags;
};

// ghost tasks of one level: copy rectangles and interpolated cells
// interpolation of the fine cell (si, sj) of level L (inside the domain) from level L-1 into
// the element dst of plane stride dplane; flags: sign flips of the destination (walls)

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

// claw_tables.cu
void free_arena(DevArena& a);
void free_level(claw_ctx* ctx, int L);
int build_tiles(claw_ctx* ctx, int L);
int build_ghost_tables(claw_ctx* ctx, int L, GhostTables& gt, bool want_ring);
void build_reflux_tables(claw_ctx* ctx, int L, std::vector<RefluxRec>& recs, std::vector<int>& group);
void build_avg_tables(claw_ctx* ctx, int L, std::vector<AvgRect>& out);
const void* get_tmaps(claw_ctx* ctx, int L, const double* q, cudaStream_t s);
long long flag_grid_offset(const claw_ctx* ctx, int L, int run);
int build_coef_tables(claw_ctx* ctx, int L);
int ensure_coef_tables(claw_ctx* ctx, int L, void* stream);

}  // namespace claw_host

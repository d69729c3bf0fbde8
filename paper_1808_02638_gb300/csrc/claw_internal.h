// claw_internal.h -- device table layouts and launch entry points shared by the .cu files of
// libclaw.so.  Not part of the public ABI (include/claw.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/claw.h"

namespace claw {

// aux planes of a cell (medium = 1); edge quantities belong to the edge west / south of the cell
enum AuxPlane : int {
    AUX_Z = 0,    // impedance Z = sqrt(K rho)
    AUX_C = 1,    // sound speed c = sqrt(K / rho)
    AUX_K = 2,    // bulk modulus K (= c Z)
    AUX_C2 = 3,   // c^2
    AUX_IXS = 4,  // 1 / (Z_{i-1,j} + Z_{i,j})
    AUX_FX1 = 5,  // (Z_{i-1} Z_i + 1) / (Z_{i-1}^2 + 1): limiter projection, left-going wave
    AUX_FX2 = 6,  // (Z_{i-1} Z_i + 1) / (Z_i^2 + 1): limiter projection, right-going wave
    AUX_IYS = 7,  // 1 / (Z_{i,j-1} + Z_{i,j})
    AUX_FY1 = 8,
    AUX_FY2 = 9,
};
static_assert(CLAW_NAUX == 10, "aux plane count");

// planes of a level-step's tape (claw_level_advance_record), laid out like the aux planes: the
// intermediates of the cell-wise step at the edge west / south of each padded cell, and the
// transverse fluctuation pressures of the cell.  The limited strengths carry the limiter's
// branch (LimCode) in their three lowest mantissa bits.
enum TapePlane : int {
    TAPE_A1 = 0, TAPE_A2 = 1,   // wave strengths of the x-edge (left-, right-going)
    TAPE_B1 = 2, TAPE_B2 = 3,   // of the y-edge
    TAPE_M1 = 4, TAPE_M2 = 5,   // limited strengths of the x-edge
    TAPE_N1 = 6, TAPE_N2 = 7,   // of the y-edge
    TAPE_D = 8,                 // x-fluctuation pressure into the cell
    TAPE_E = 9,                 // y-fluctuation pressure into the cell
};
constexpr int kTapePlanes = 10;
static_assert(kTapePlanes == CLAW_NAUX, "a tape has the aux pool's size");

// branch of a limited strength phi(b/a) a: its partial derivatives (d/da, d/db)
enum LimCode : int {
    LIMC_ZERO = 0,      // (0, 0)
    LIMC_A = 1,         // (1, 0)
    LIMC_B = 2,         // (0, 1)
    LIMC_2A = 3,        // (2, 0)
    LIMC_2B = 4,        // (0, 2)
    LIMC_HALF = 5,      // (1/2, 1/2)
    LIMC_SMOOTH = 6,    // van Leer: derivatives from the values
};

// One box of a level, as the kernels see it.
struct PatchDev {
    long long qoff;   // element offset of the p plane in the q pool
    long long aoff;   // element offset of the first aux plane in the aux pool (CLAW_NAUX * coff)
    int nx, ny;       // interior size
    int run;          // index into the per-run dt / smax arrays
    int ring;         // first entry of the box's ghost ring in the level's ring table (-1: none)
    int interp;       // first of the box's interpolated ghost cells in the level's InterpCell table
    double dxinv, dyinv;
    double dtscale;   // this level's dt / level-0 dt = 1 / (ratio_1 ... ratio_L)
};

// One tile of the fused step: interior cells [x0, x0+tx) x [y0, y0+ty) of box `patch`.
// TILE_CARRY (column-walk tile lists; not a cell-wise medium): the previous tile of the list is the
// tile directly below this one, with the same columns: in the same box, or in the same-level box
// whose top side this box's bottom side covers exactly.
enum : int { TILE_CARRY = 1 };
struct TileDev {
    int patch;
    short x0, y0, tx, ty;
    int flags;
};

// Rectangle of ghost cells copied from interior cells of the same level (same-level copy and
// physical boundaries).  Element (x, y) of the rectangle, plane m:
//   dst + m*dplane + y*dpitch + x   <-   sign_m * src[m*splane + y*sy + x*sx]
struct CopyRect {
    long long dst, src;
    long long dplane, splane;
    int w, h;
    int dpitch, sy, sx;
    int flags;   // bit0: negate u, bit1: negate v
};

// One coarse-fine interface edge of the conservation fix (Sec. 2.3): coarse cell C = (ci, cj)
// of coarse box cbox, not covered by the fine level, shares an edge with the fine region; the r
// fine cells next to that edge start at (fi, fj) of fine box fbox and run along the edge.
// dir 0: x-edge, 1: y-edge; side +1: C is left of / below the edge, -1: right of / above.
struct RefluxRec {
    int cbox, fbox;
    short ci, cj, fi, fj;
    short dir, side;
};

// Regridding: a box of the level being flagged (interior rows of the flag grid start at goff,
// rows pitch bytes apart) and a cell copied from an old fine pool into a new one.
struct FlagBox {
    long long qoff, goff;
    int nx, ny, pitch, pad;
};
// A box in a level's index space with its pool offset, as the regrid transfer reads it.
struct XferBox {
    long long qoff;
    int run, ilo, jlo, nx, ny, pad;
};
// The level-wide index grids of a regrid transfer: per run, the box covering each cell of the
// fine level (old boxes) and of the coarse level, or -1.  Run q's grid starts at goff[q] with
// row pitch pitch[q] (the level's NX).
struct XferGrids {
    const long long* fgoff;
    const int* fpitch;
    const long long* cgoff;
    const int* cpitch;
    int* fgrid;
    int* cgrid;
};

// One fine ghost cell filled by space-time interpolation from the coarser level.
struct InterpCell {
    long long dst;        // plane-0 element of the fine ghost cell
    long long src[5];     // plane-0 element of the coarse cells: centre, west, east, south, north
    long long dplane;     // fine plane stride
    long long splane[5];  // coarse plane strides
    double xi, eta;       // offsets of the fine centre from the coarse centre, in coarse cells
    int sflags[5];        // wall sign flips of each coarse source (bit0 u, bit1 v)
    int flags;            // wall sign flips of the fine ghost itself
};

// A fill of a fine level's interpolated ghost cells (cells, n) in pool q from the coarse states
// cold, cnew at time fraction tau, run by spare CTAs of a level-step launch.
struct FillJob {
    const InterpCell* cells = nullptr;
    int n = 0;
    double* q = nullptr;
    const double* cold = nullptr;
    const double* cnew = nullptr;
    double tau = 0.0;
};

// Coarse cells [0,w) x [0,h) at cdst, each the mean of r x r fine cells at fsrc.
struct AvgRect {
    long long cdst, fsrc;
    long long cplane, fplane;
    int w, h, cpitch, fpitch;
};

// Per (level) device tables.
// Device tables kept in one allocation that is reused (and grown when too small) from one
// rebuild of a level to the next, so that a rebuild costs one host-to-device copy instead of
// a cudaMalloc, a copy and a cudaFree per table.
struct DevArena {
    char* dev = nullptr;
    size_t cap = 0;
    char* host = nullptr;   // pinned staging buffer of the copy
    size_t host_cap = 0;
};

struct LevelDev {
    int nboxes = 0;
    int ntiles = 0;
    int ncopy = 0;
    int ninterp = 0;
    int navg = 0;          // averaging rects into the coarser level
    int ratio = 1;
    int tx = 32, ty = 32, staging = 1, nt = 0;   // tile, staging, threads per CTA (0: default)
    bool tiling_set = false;   // claw_set_tiling chose tx, ty, staging, nt (kept by claw_set_level)
    int walk = -1;         // column walks (tiles ordered up each column, tcum): 1 on, 0 off, -1 automatic
    bool walking = false;  // the tile lists in place are column walks
    PatchDev* patches = nullptr;
    TileDev* tiles = nullptr;
    long long* tcum = nullptr;     // column walk: cumulative tile costs [ntiles + 1] (null otherwise)
    CopyRect* copies = nullptr;
    CopyRect* ccopies = nullptr;   // the same copies for one-plane coefficient pools (coff offsets)
    int nccopy = 0;
    InterpCell* interps = nullptr;
    AvgRect* avgs = nullptr;
    void* tmaps = nullptr;   // CUtensorMap per box (128 B each), built for the current tiling
    int tmap_tx = 0, tmap_ty = 0;
    int* copy_start = nullptr;    // [ncopy_blocks + 1]: block k copies rectangles [start[k], start[k+1])
    int* ccopy_start = nullptr;
    int ncopy_blocks = 0, nccopy_blocks = 0;
    int max_rows = 0;             // largest (ny + 4) of the level's boxes
    RefluxRec* reflux = nullptr;  // interface with the coarser level, grouped by coarse cell
    int nreflux = 0;
    int* reflux_group = nullptr;  // [ngroups + 1]: records of coarse cell g are [group[g], group[g+1])
    int nreflux_groups = 0;
    FlagBox* flagboxes = nullptr; // the boxes as flag-grid writers (built on first use)
    longlong2* ring = nullptr;    // ghost sources of every box's ring (pulled ghosts), see ring_index
    long long* poff = nullptr;    // packed-interior offset of every box (3 nx ny doubles each)
    long long packed = 0;         // doubles of the packed interiors of the level
    bool ring_ok = false;
    bool coef_built = false;      // ccopies / ccopy_start built for the current boxes
    DevArena tables;              // patches, copies, interps, avgs, reflux, ring, poff, copy_start
    DevArena tiletab;             // the tile lists (rebuilt with the tiling)
    DevArena coeftab;             // ccopies, ccopy_start
    // host copies
    std::vector<claw_box> boxes;
    std::vector<PatchDev> hpatches;
    std::vector<TileDev> htiles;
    std::vector<long long> htcum;
};

// Ghost ring of a box: its (nx+4)(ny+4) - nx ny ghost cells in row order of the padded box.
// Entry {source, plane | sign flags << 48}: the ghost takes the pool's plane-0 element `source`
// and the elements one and two planes (`plane` elements) further, u negated if bit 0 of the
// flags, v if bit 1; a source of -1 - j marks the box's j-th ghost interpolated from the coarser
// level (entry PatchDev::interp + j of the level's InterpCell table), which the step either reads
// from the pool (filled by claw_fill_ghost_interp) or evaluates itself (claw_level_advance_interp).
constexpr int kRingFlagShift = 48;
__host__ __device__ inline int ring_index(int xp, int yp, int nx, int ny)   // -1: interior
{
    const int W = nx + 4;
    if (yp < 2) return yp * W + xp;
    if (yp >= ny + 2) return 2 * W + 4 * ny + (yp - ny - 2) * W + xp;
    if (xp < 2) return 2 * W + (yp - 2) * 4 + xp;
    if (xp >= nx + 2) return 2 * W + (yp - 2) * 4 + (xp - nx);
    return -1;
}

// default bound of a bounded mbarrier wait (polls; far beyond a normal copy)
constexpr unsigned kWaitPolls = 1u << 22;

struct StepArgs {
    const PatchDev* patches = nullptr;
    const TileDev* tiles = nullptr;
    const void* tmaps = nullptr;
    int ntiles = 0;
    // column walk: cumulative tile costs [ntiles + 1]; CTA b of the grid takes the tiles whose
    // costs start in [b, b + 1) / grid of the total.  Null: CTAs stride over the tiles by the grid.
    const long long* tcum = nullptr;
    const double* qold = nullptr;
    double* qnew = nullptr;
    const double* aux = nullptr;
    const double* dt = nullptr;
    double* smax = nullptr;
    int* err = nullptr;
    // scheme
    int order = 2, transverse = 2;
    double rho0 = 1.0, K0 = 1.0;   // uniform medium
    double grav = 0.0;             // shallow water
    int swe = 0;                   // 1: the shallow water system (the conservation fix reads it)
    const longlong2* ring = nullptr;   // not null: same-level and boundary ghosts are pulled from sources
                                   // (launch_step then picks the kernels that pull)
    // fused epilogue (0 = off)
    int dtupd = 0;                      // the last CTA applies Eq. cfl to dt and resets smax
    double* dt_out = nullptr;
    const double* minh = nullptr;       // level-0 min(dx, dy) per run
    const double* cflv = nullptr;       // desired CFL per run
    unsigned int* done = nullptr;       // CTA completion counter (0 between launches)
    int nruns = 0;
    // polls of a tile's first wait for its bulk copy before the CTA reports ERR_TIMEOUT; the
    // copies still in flight are then awaited with the full bound kWaitPolls before it exits
    unsigned wait_polls = kWaitPolls;
    double* tape = nullptr;   // recording step (cell-wise medium): the level-step's tape, aux layout
    // pulled ghosts interpolated from the coarser level inside the step (not null: the ring's
    // interpolated entries point into this table, evaluated from cold / cnew at tau)
    const InterpCell* interp = nullptr;
    const double* cold = nullptr;
    const double* cnew = nullptr;
    double tau = 0.0;
    // CTAs [step_grid, gridDim.x) of the launch fill interpolated ghosts (fills[0, nfill)) instead
    // of stepping tiles; step_grid 0: every CTA steps tiles
    int step_grid = 0;
    int nfill = 0;
    FillJob fills[2];
};

// error flag bits written by kernels
enum : int { ERR_NAN = 1, ERR_CFL = 2, ERR_TIMEOUT = 4 };

// kernel family of a level-step: acoustics in a uniform / cell-wise medium, shallow water
enum : int { KIND_UNIFORM = 0, KIND_CELLWISE = 1, KIND_SWE = 2 };

// launchers (claw_step.cu; kind: KIND_*)
// a.nfill > 0: the launch adds up to max(spare, 1) CTAs for the fill jobs
// (CTAs from index grid on)
cudaError_t launch_step(const StepArgs& a, int kind, int limiter, int tx, int ty, int nt, int staging,
                        int grid, cudaStream_t s, int spare = 0);
int step_max_ctas_per_sm(int kind, int limiter, int tx, int ty, int nt, int staging, bool pull = false,
                         bool rec = false, bool interp = false, bool walk = false);
cudaError_t launch_step_adjoint(const StepArgs& a, const double* lam_new, double* lam_old, double* g_aux,
                                int medium, int limiter, int nsm, cudaStream_t s);   // grid: resident CTAs x nsm
int adjoint_tile();   // the adjoint kernel's square tile edge
// the tape-driven adjoint of the cell-wise second-order step (claw_adjoint_tape.cu), on the tiles of
// adjoint_tape_tile() (the same edge as adjoint_tile())
cudaError_t launch_step_adjoint_tape(const StepArgs& a, const double* lam_new, double* lam_old, double* g_aux,
                                     int limiter, int nsm, cudaStream_t s);
int adjoint_tape_tile();
// the step's wave limiter elementwise (claw_step.cu)
cudaError_t launch_limiter_eval(int limiter, long long n, const double* a, const double* b, double* out,
                                cudaStream_t s);

// launchers (claw_ghost.cu)
cudaError_t launch_fill_copy(const CopyRect* r, const int* start, int nblocks, double* q, cudaStream_t s,
                             int ncomp = 3);
cudaError_t launch_fill_interp(const InterpCell* c, int n, double* q, const double* cold,
                               const double* cnew, double tau, cudaStream_t s);
cudaError_t launch_fill_copy_adjoint(const CopyRect* r, const int* start, int nblocks, double* lam, cudaStream_t s,
                                     int ncomp = 3);
cudaError_t launch_fill_interp_adjoint(const InterpCell* c, int n, double* lam, double* lco,
                                       double* lcn, const double* cold, const double* cnew,
                                       double tau, cudaStream_t s);
cudaError_t launch_average(const AvgRect* r, int n, int ratio, const double* qf, double* qc,
                           cudaStream_t s);
cudaError_t launch_average_adjoint(const AvgRect* r, int n, int ratio, double* lf, double* lc,
                                   cudaStream_t s);
// box-wise kernels: blockIdx.x = box, blockIdx.y = a chunk of kBoxRows rows (max_rows: the
// largest padded height of the boxes, so every row of every box has a block)
constexpr int kBoxRows = 16;
cudaError_t launch_medium_aux(const PatchDev* p, int n, int max_rows, const double* rho, const double* K,
                              double* aux, cudaStream_t s);
cudaError_t launch_medium_aux_adjoint(const PatchDev* p, int n, int max_rows, const double* rho,
                                      const double* K, const double* g_aux, double* g_rho,
                                      double* g_K, cudaStream_t s);
// regridding
cudaError_t launch_flags(const FlagBox* boxes, int nb, int max_rows, const double* q, double tol,
                         unsigned char* flags, cudaStream_t s);
// regrid transfer (claw_regrid.cu): index grids painted with the old fine boxes and the coarse
// boxes, then every cell of every new box copied from the old box covering it or interpolated
// from the coarse level; *err |= 1 where a new cell has no coarse cell (not nested)
cudaError_t launch_regrid_transfer(const XferBox* nb, int n_new, const XferBox* ob, int n_old, const XferBox* cb,
                                   int n_coarse, int max_rows, int ratio, const XferGrids& g, long long fcells,
                                   long long ccells, const double* q_old, const double* q_coarse, double* q_new,
                                   int* err, cudaStream_t s);

// conservation fix (uniform medium): buf holds 3 doubles per interface record (the coarse
// parts) followed by 3 per record and fine edge (the fine parts, summed over the substeps)
// (k: the scheme's order, transverse mode and uniform medium rho0, K0)
cudaError_t launch_reflux_coarse(const RefluxRec* rec, int n, const PatchDev* cp, const double* qc, const double* dt,
                                 double* buf, int ratio, const StepArgs& k, int limiter, cudaStream_t s);
cudaError_t launch_reflux_fine(const RefluxRec* rec, int n, const PatchDev* cp, const PatchDev* fp, const double* qf,
                               const double* qc, const double* dt, double* buf, int ratio, const StepArgs& k,
                               int limiter, cudaStream_t s);
cudaError_t launch_reflux_apply(const RefluxRec* rec, int n, const int* group, int ngroups, int ratio,
                                const PatchDev* cp, const double* dt, const double* buf, double* qc, cudaStream_t s);
cudaError_t launch_cfl_max(const PatchDev* p, int n, int max_rows, int medium, double c0, const double* aux,
                           double* smax, cudaStream_t s);
cudaError_t launch_pack(const PatchDev* p, const long long* poff, int b0, int b1, int max_rows, double* q,
                        double* packed, int unpack, cudaStream_t s);
cudaError_t launch_cfl_max_state(const PatchDev* p, int n, int max_rows, double grav, const double* q,
                                 double* smax, cudaStream_t s);
cudaError_t launch_dt_update(const double* minh, const double* cfl, int nruns, double* smax,
                             double* dt, int* err, cudaStream_t s);

}  // namespace claw

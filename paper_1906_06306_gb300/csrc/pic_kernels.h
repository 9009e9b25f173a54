// Host-side launchers of the PIC kernels (internal to libpic).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "pic_dev.cuh"

namespace pic {

constexpr int kMaxSpecies = 4;
#ifndef PIC_PUSH_THREADS
#define PIC_PUSH_THREADS 256
#endif
#ifndef PIC_SPILL_EVERY
#define PIC_SPILL_EVERY 16
#endif
#ifndef PIC_PUSH_MIN_BLOCKS
#define PIC_PUSH_MIN_BLOCKS 5
#endif
#ifndef PIC_PUSH_MIN_BLOCKS_TMA
#define PIC_PUSH_MIN_BLOCKS_TMA 5
#endif
// 3D: 4 blocks per SM hold the kernel to 64 registers (no spills) and, with
// the current folded into global J (PIC_FOLD_GLOBAL_3D), a block to 55 KB of
// shared memory: measured on the 1024x128x128 shock (two runs each) the
// particle kernel 5.00 -> 4.75 ms a step against 80 registers, a float window
// and 3 blocks per SM (4.83 ms with the global fold at 3 blocks).
#ifndef PIC_PUSH_MIN_BLOCKS_3D
#define PIC_PUSH_MIN_BLOCKS_3D 4
#endif
// Blocks whose tile window lies inside the lattice skip the periodic-wrap
// arithmetic (window-local indices and the new cell index).
#ifndef PIC_INTERIOR
#define PIC_INTERIOR 1
#endif
// 2D window layout with x-adjacent points paired: (Ex, By, Ex+, By+) and
// (Ey, Bx, Ey+, Bx+) as float4, (Ez, Ez+) and (Bz, Bz+) as float2, so a
// stencil row is one shared load per component pair.
#ifndef PIC_XPAIR
#define PIC_XPAIR 0
#endif
// 2D current window of 64-bit pairs of fixed-point words (SmemJ64): half the
// shared atomics of the int32 window.
#ifndef PIC_J64
#define PIC_J64 0
#endif
template <int D>
constexpr bool kJ64 = D == 2 && PIC_J64 != 0;
// The 1D/2D fused kernels stream each batch's particle records into shared
// memory with bulk copies when every record row is 16-byte aligned.
#ifndef PIC_TMA_RECORDS
#define PIC_TMA_RECORDS 0
#endif
// 3D window with x-adjacent points paired per component (one 8-byte shared
// load per stencil corner pair); the 3D fixed-point current then folds into
// the global J planes instead of a float window, which keeps the shared
// memory of a block at the size of three blocks per SM.
#ifndef PIC_X3PAIR
#define PIC_X3PAIR 0
#endif
// The 3D fixed-point current folds into the global J planes at every fold
// instead of into a float window flushed once (a smaller block: 55 KB for the
// 8x8x4-tile window, four blocks per SM); also without the x-paired window.
#ifndef PIC_FOLD_GLOBAL_3D
#define PIC_FOLD_GLOBAL_3D 1
#endif
template <int D>
constexpr bool kFoldGlobal = D == 3 && (PIC_X3PAIR != 0 || PIC_FOLD_GLOBAL_3D != 0);
// The 2D particle kernel stages the field window of a tile inside the lattice
// by one tensor copy (TMA) instead of per-thread loads.
#ifndef PIC_TMA_WINDOW
#define PIC_TMA_WINDOW 1
#endif
// The 2D/3D filter passes stage their rows by bulk copies (cp.async.bulk)
// where the rows allow it and a status word can report a wait that ran out.
#ifndef PIC_BULK_FILTER
#define PIC_BULK_FILTER 1
#endif
// Resident blocks per SM the 1D/2D adjoint tile pass is compiled for (4: 64
// registers without spills, 4 x 45 KB of shared memory for a 16x16-tile
// window; measured 0.38 -> 0.27 ms per adjoint step of the 256^2 box against 2
// blocks).  The 3D window's 128 KB allow one block, so 3D keeps 2.
#ifndef PIC_ADJ_MIN_BLOCKS
#define PIC_ADJ_MIN_BLOCKS 4
#endif
// Small periodic FDTD2 lattices take the second B half step and the E update
// of a step in one launch.
#ifndef PIC_SMALL_FIELDS
#define PIC_SMALL_FIELDS 1
#endif
// pic_step(n) replays whole sort cycles from a captured CUDA graph.
#ifndef PIC_STEP_GRAPHS
#define PIC_STEP_GRAPHS 1
#endif
#ifndef PIC_PREFETCH
#define PIC_PREFETCH 0
#endif
// Sub-tile extents of the sort key (0: the whole tile), for 2D and for 3D (1D
// tiles are not subdivided).  The tile sort orders a tile's particles by
// sub-tile, so the lanes of a warp gather from and deposit into a part of the
// tile window: fewer shared-memory bank conflicts (coinciding stencil words
// are broadcasts), more sort bins.  Measured with every other setting fixed
// (two runs each, 1024^2 turbulence with 16x8 tiles; 1024x128x128 shock with
// 8x8x4 tiles): in 2D 8x4 took the particle kernel from 0.567 to 0.553 ms
// (the sort 0.055 -> 0.063 ms, the step 0.634 -> 0.629 ms; 8x8 0.629, 4x8
// 0.631, 16x4 0.631, 4x4 slower); in 3D 2x4x2 from 5.11 to 5.04 ms (the step
// 6.59 -> 6.55 ms; 4x4x2 6.59, 4x4x4 6.66, 8x4x2 and 4x8x2 6.65, 4x4x1 6.68).
#ifndef PIC_SUBTILE_X
#define PIC_SUBTILE_X 8
#endif
#ifndef PIC_SUBTILE_Y
#define PIC_SUBTILE_Y 4
#endif
#ifndef PIC_SUBTILE3_X
#define PIC_SUBTILE3_X 2
#endif
#ifndef PIC_SUBTILE3_Y
#define PIC_SUBTILE3_Y 4
#endif
#ifndef PIC_SUBTILE3_Z
#define PIC_SUBTILE3_Z 2
#endif
constexpr int kSubTile2[3] = {PIC_SUBTILE_X, PIC_SUBTILE_Y, 0};
constexpr int kSubTile3[3] = {PIC_SUBTILE3_X, PIC_SUBTILE3_Y, PIC_SUBTILE3_Z};
// Sort bins of a tiling: sub-tiles of every tile, tile-major.
inline long long sort_bins(const TileDev& t) { return (long long)t.ntiles * t.nsub; }
constexpr int kPushThreads = PIC_PUSH_THREADS;
constexpr int kSpillEvery = PIC_SPILL_EVERY;  // batches of kPushThreads particles between spills
// Shared-memory queue of the 1D/2D tile kernels for particles outside the tile
// window (about 0.5 % of the particles between sorts).  It is drained at the
// end of each species and at a spill point where it is more than half full; a
// stray that finds it full is processed at once by its own lane.
constexpr int kQueueCap = 512;
// Particle records of a batch streamed into shared memory by bulk copies
// (1D/2D fused kernels): a ring of this many stages of kPushThreads records.
constexpr int kRecStages = 2;

// Lattice kernels run on a (x blocks, y, z) launch grid: a thread owns point x
// of the rows (y, z) of its block, stepping over rows beyond the launch grid's
// 65535 limit, so no lattice index is ever divided out of a linear one.  The
// kernel body names the extents n1, n2.
#define FOR_ROWS(j, k)                             \
  for (int k = blockIdx.z; k < n2; k += gridDim.z) \
    for (int j = blockIdx.y; j < n1; j += gridDim.y)

struct RowLaunch {
  dim3 grid;
  unsigned threads;
};
inline RowLaunch row_launch(const GridDev& g) {
  const int n0 = g.n[0];
  const unsigned t = n0 >= 256 ? 256 : n0 >= 128 ? 128 : n0 >= 64 ? 64 : 32;
  const unsigned gy = (unsigned)(g.n[1] < 65535 ? g.n[1] : 65535);
  const unsigned gz = (unsigned)(g.n[2] < 65535 ? g.n[2] : 65535);
  return {dim3((unsigned)((n0 + t - 1) / t), gy, gz), t};
}

struct PushParams {
  GridDev g;
  TileDev t;
  float* F;
  int nspecies;
  SpeciesDev sp[kMaxSpecies];
  int splits;   // thread blocks per tile
  int* status;
  float inv_c, inv_c2;
  FastDiv div0, div1;  // by n0 and n1: cell -> (i, j, k)
  int wrap_fast;       // every axis has n >= window extent: one conditional wrap suffices
  float jq;            // quantum of the int32 shared-memory current (a power of 2)
  float jq_inv;        // 1 / jq
  unsigned long long* strays;  // running count of particles that took the global path
  int pusher;                  // 0 Boris (Appendix C), 1 Higuera-Cary
  int wall;                    // conducting wall on the node plane x = wall (0: none)
  int tail_blocks;             // extra blocks for the unsorted tails [tail, n)
  int* dcount;                 // [nspecies] entries of the deferred lists (zeroed per launch)
  int rec_aligned;             // every record row read by the push starts 16-byte aligned
  // 2D field window by one tensor copy (TMA): a 3D map over the E, B planes
  // (x, y, component) with a box of win_box[0] x W1 x 6 whose x origin is the
  // window's rounded down to a multiple of 4 floats (win_shift below it);
  // used by blocks whose window lies inside the lattice
  int win_tma;
  int win_box[2];   // box extents x (a multiple of 4), y
  int win_shift;    // window x origin - box x origin
  CUtensorMap win_map;  // (the type carries the alignment a tensor map needs)
};

// Quantum of the fixed-point shared-memory current (a power of 2) for charges
// up to max_abs_q, Courant number c and `batch` particles between spills.  In
// one step a particle adds to any current word at most |q| times the sum of
// its two segments' displacements along that component (|dx| < c) times a
// transverse weight (<= 1, or 1 + c^2/12 in 3D), i.e. less than 1.02 c |q|;
// a bound of 1.25 c * batch * max|q| < 2^31 quanta can never overflow.
float current_quantum(float max_abs_q, float c, int batch);
FastDiv make_fastdiv(int d);

// message returned by pic_last_error(NULL) in the calling thread
void set_global_error(const char* msg);

// mode 0: fused gather + push + move + deposit; 1: gather + push + move and
// pre-move snapshot; 2: deposit from the snapshot and the stored new u.  Mode
// 0 with P.wall > 0 runs the fused kernel's wall variant (mode 3), which also
// reflects at the conducting wall; then the unsorted tail and the wall
// crossers are processed by two small kernels after it.
cudaError_t launch_particles(int dim, int mode, const PushParams& P, cudaStream_t st);
cudaError_t set_particle_smem_limit(int bytes);
size_t particle_smem_bytes(int dim, const TileDev& t);
// floats of a block's shared memory past the staged field window, from the
// first 128-byte boundary on: room for the 2D window's tensor copy
long long window_landing_floats(int dim, const TileDev& t);

cudaError_t launch_b_half(const GridDev& g, float* F, int zero_j, cudaStream_t st);
cudaError_t launch_e_update(const GridDev& g, float* F, cudaStream_t st);
// FDTD2 lattices of at most kSmallFieldCells points: the second B half step
// and the E update in one single-block launch (the same bits as the two);
// with chain != 0 also the next step's first B half step (clearing J)
constexpr long long kSmallFieldCells = 4096;
bool fields_small_ok(const GridDev& g);
cudaError_t launch_fields_small(const GridDev& g, float* F, cudaStream_t st, int chain = 0);
// one Binomial2 sub-pass along gridded axis `axis` over ncomp consecutive planes,
// src -> dst (a full pass is one sub-pass per gridded axis, x first)
cudaError_t launch_filter_f32(const GridDev& g, const float* src, float* dst, int ncomp, int axis,
                              cudaStream_t st);
cudaError_t launch_filter_f64(const GridDev& g, const double* src, double* dst, int ncomp,
                              int axis, cudaStream_t st);
// one full Binomial2 pass (every gridded axis, x first) over ncomp consecutive
// planes, src -> dst, the sub-passes fused through shared memory; with a
// status word (2D/3D, aligned rows) the rows are staged by bulk copies whose
// bounded waits report there, without one (nullptr) by per-thread copies
cudaError_t launch_filter_pass_f32(const GridDev& g, const float* src, float* dst, int ncomp,
                                   cudaStream_t st, int* status);

struct SortParams {
  GridDev g;
  TileDev t;
  int* status;
  FastDiv dn0, dn1;          // by the grid extents n0, n1: cell -> (i, j, k)
  FastDiv dt0, dt1, dt2;     // by the tile extents: lattice point -> tile
  FastDiv ds0, ds1, ds2;     // by the sub-tile extents: tile-local point -> sub-tile
};
SortParams make_sort_params(const GridDev& g, const TileDev& t, int* status);
cudaError_t launch_tile_count(const SortParams& P, const int* cell, long long n, int* count,
                              cudaStream_t st);
// exclusive scan of count[0..n) into start[0..n] and cursor; n above 4096 uses
// scratch (scan_scratch(n) ints)
cudaError_t launch_tile_scan(const int* count, int ntiles, int* start, int* cursor, int* scratch,
                             cudaStream_t st);
inline long long scan_scratch(long long n) { return 3 * ((n + 4095) / 4096 + 1); }
// arrays with rows of ld elements, the first n of which are particles
// perm (or null): perm[new slot] = old slot
cudaError_t launch_tile_scatter(const SortParams& P, const int* cell, const float* off,
                                const float* u, long long n, long long ld, int* cursor,
                                int* cell_out, float* off_out, float* u_out, cudaStream_t st,
                                int* perm = nullptr);
// bucket starts t[0..nb] from outside: unless they are a partition of [0, n)
// they become one bucket, and ST_BAD_BUCKETS is set
// out[i] = tstart[i] clamped to [lo, hi) for i < nb1 (one slot range's buckets)
cudaError_t launch_clip_starts(const int* tstart, long long nb1, int lo, int hi, int* out,
                               cudaStream_t st);
cudaError_t launch_check_buckets(int* tstart, long long nb, long long n, int* status,
                                 cudaStream_t st);
// out[r * ld + perm[i]] = in[r * ld + i] for i < n, r < rows (entries of perm
// outside [0, n) skipped, ST_BAD_BUCKETS set)
cudaError_t launch_unpermute(const int* perm, const float* in, float* out, long long n,
                             long long ld, int rows, int* status, cudaStream_t st);

// diagnostics: acc[0] += 0.5 sum E^2, acc[1] += 0.5 sum B^2
cudaError_t launch_field_energy(const GridDev& g, const float* F, double* acc, cudaStream_t st);
cudaError_t launch_kinetic(const float* u, long long n, long long ld, double mc2, double* acc,
                           cudaStream_t st);
cudaError_t launch_rho(const GridDev& g, const int* cell, const float* off, long long n,
                       long long ld, double q, double* rho, cudaStream_t st);
// over the nodes with i_lo <= i < i_hi: acc_max (as the bit pattern of a
// non-negative double), acc_sq += sum res^2
// one warp whose bounded barrier wait runs out (sets ST_TIMEOUT)
cudaError_t launch_wait_probe(int* status, cudaStream_t st);
cudaError_t launch_gauss(const GridDev& g, const float* F, const double* rho, int i_lo, int i_hi,
                         unsigned long long* acc_max, double* acc_sq, cudaStream_t st);

// Shock boundaries (Sect. 4.2): the conducting wall's field boundary (zero
// tangential E on the node plane x = wall, mirror image behind it) and zero E
// and B at i >= i_zero, applied after each field update.
cudaError_t launch_wall_fields(const GridDev& g, float* F, int wall, int i_zero, cudaStream_t st);

// One contiguous run of injected particles: template indices [k0, k1) of copy
// m of species s, written from output index `out` on, x = x_t + shift.
struct InjectRun {
  int s;
  long long k0, k1;
  long long out;
  double shift;
};
constexpr int kMaxInjectRuns = 3 * kMaxSpecies;
struct InjectParams {
  GridDev g;
  int lt;                      // template block length along x
  int nruns;
  long long first[kMaxInjectRuns + 1];  // prefix of run lengths (first[nruns] = total)
  InjectRun run[kMaxInjectRuns];
  const int* tcell[kMaxSpecies];  // template arrays of each species, rows of tn[s]
  const float* toff[kMaxSpecies];
  const float* tu[kMaxSpecies];
  long long tn[kMaxSpecies];
  int* cell[kMaxSpecies];         // species arrays, rows of ld[s]
  float* off[kMaxSpecies];
  float* u[kMaxSpecies];
  long long ld[kMaxSpecies];
};
cudaError_t launch_inject(const InjectParams& P, cudaStream_t st);

// Discrete adjoint of the step (FDTD2, Boris, periodic; pic_adjoint.cu).
struct AdjSpecies {
  float q, qm;
  long long n, ld;        // particles, row length of the arrays
  const int* cell;        // forward particles at the start of the step
  const float* off;       // [D][ld]
  const float* u;         // [3][ld]
  float* xbar;            // [D][ld] gradient of the position (in: after, out: before)
  float* ubar;            // [3][ld] gradient of u
  const int* tstart;      // sort-bin starts of the tile grouping, or null (global pass only)
  int* dlist;             // particles the tile pass deferred to the global pass
};
struct AdjParams {
  GridDev g;
  TileDev t;        // the tiling the particles were grouped by
  int splits;       // blocks per tile
  const float* F1;  // forward E and the B of the first half step (9-plane layout)
  float* A;         // adjoint planes: Ebar, Bbar, Jbar
  FastDiv div0, div1;  // by n0 and n1: cell -> (i, j, k)
  int nspecies;
  int* dcount;      // [nspecies] entries of the deferred lists
  AdjSpecies sp[kMaxSpecies];
};
// Bbar += c curl+ Ebar, Jbar = -Ebar (adjoint of the E update with -J)
cudaError_t launch_adj_e(const GridDev& g, float* A, cudaStream_t st);
// Ebar -= (c/2) curl- Bbar (adjoint of a B half step)
cudaError_t launch_adj_b_half(const GridDev& g, float* A, cudaStream_t st);
// adjoint of gather + Boris + move + ZigZag for every particle: the tile pass
// where every species gives its tile grouping (then the deferred ones through
// global memory), else all through global memory
cudaError_t launch_adj_particles(const AdjParams& P, cudaStream_t st);

}  // namespace pic

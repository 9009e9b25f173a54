/* pic.h - C ABI of a single-GPU relativistic particle-in-cell time step for
 * NVIDIA GB300 (sm_103a): the hot path of the PIC method of the Runko paper
 * (Nattila, arXiv:1906.06306, Sect. 2.3, Table 1, Appendices B-D).
 *
 * Units and lattice (Sect. 2.3, Appendix A): dx = dt = 1; the Courant number c
 * is the only constant of the field equations.  All boundaries are periodic,
 * unless pic_set_shock adds the conducting wall and receding injector of the
 * paper's shock set-up along x (Sect. 4.2).
 *
 * Fields: ONE caller-owned device buffer of 9 float planes, each
 * nz*ny*nx floats, x fastest: Ex Ey Ez Bx By Bz Jx Jy Jz.  Element [i,j,k] of
 * each plane lives at its Yee point (Sect. 2.3.1):
 *   Ex (i+1/2,j,k)  Ey (i,j+1/2,k)  Ez (i,j,k+1/2)
 *   Bx (i,j+1/2,k+1/2)  By (i+1/2,j,k+1/2)  Bz (i+1/2,j+1/2,k)
 *   J at the E points; charge density (diagnostics) on the nodes (i,j,k).
 * Time levels: on entry to a step E is at t^n and B at t^(n-1/2); particles
 * hold x^n and u^(n-1/2).
 *
 * Particles, per species, caller-owned device buffers (structure of arrays,
 * rows of cap elements, of which the first n are particles):
 *   cell  int32[cap]       linear cell index i + nx*(j + ny*k)
 *   off   float[dim][cap]  in-cell offset of each gridded coordinate, in [0,1)
 *   u     float[3][cap]    spatial four-velocity in units of c
 * The library keeps particles sorted by spatial tile and may reorder them
 * (pic_sort, pic_step; particles injected since the last sort follow the
 * sorted ones); after every call returns (on the stream) the caller's
 * buffers hold the current particles, whose count pic_particle_counts gives.
 *
 * Ownership: the caller owns the field and particle buffers and the stream;
 * the library owns the context, its scratch (sort buffers, tile tables,
 * pre-move snapshot, filter buffer, diagnostics, status word, injector
 * templates, deferred-particle lists) and frees them in pic_destroy.  All calls enqueue
 * work on the context's stream and return without synchronising, except
 * pic_energies, pic_check, pic_step_host, pic_stats, pic_autotune,
 * pic_kernel_times and pic_set_shock (which copies the templates), which
 * synchronise the stream.  No exception crosses the
 * ABI: every call returns a pic_status; pic_last_error gives the message of
 * the last failure on a context.  A context is not thread-safe.
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
  PIC_OK = 0,
  PIC_ERR_ARG = 1,     /* invalid argument: null pointer, bad size or layout */
  PIC_ERR_CUDA = 2,    /* a CUDA runtime call failed (message in pic_last_error) */
  PIC_ERR_OOM = 3,     /* the library could not allocate its device scratch */
  PIC_ERR_TIMEOUT = 4, /* a bounded device-side wait gave up */
  PIC_ERR_STATE = 5    /* a kernel met invalid particle data (cell index out of
                          range, offset outside [0,1), non-finite u) */
} pic_status;

#define PIC_MAX_SPECIES 4

/* Periodic box: dim = 1, 2 or 3 gridded dimensions; extents of non-gridded
 * dimensions must be 1.  nx*ny*nz must fit in int32, ny <= 65535 and
 * nz <= 21845 (launch-grid limits of the filter). */
typedef struct {
  int dim;
  int nx, ny, nz;
} pic_grid;

/* One species.  q is the charge of a macro-particle (signed, code units; the
 * ZigZag current of Appendix D is proportional to it) and m its mass, so that
 * q/m is the s-hat of the Boris scheme (Appendix C).  n is the particle count
 * and cap (>= n; 0 means n) the row length of the arrays: the room the
 * injector of pic_set_shock may fill.  Pointers are device pointers with the
 * layout above; the caller keeps them alive until pic_destroy. */
typedef struct {
  float q;
  float m;
  int64_t n;
  int32_t* cell;
  float* off;
  float* u;
  int64_t cap;
} pic_species;

/* Host-side particles of one species for pic_step_host (same layout as
 * pic_species, rows of cap elements, host pointers; pinned memory gives full
 * copy bandwidth). */
typedef struct {
  int32_t* cell;
  float* off;
  float* u;
} pic_host_species;

/* Launch and layout parameters (not physics).  Zero fields keep their current
 * value.  tile: cells per tile per gridded dimension; halo: extra cells staged
 * on each side of a tile (>= 1; a particle that has drifted further than
 * halo-1 cells from its tile since the last sort takes the global-memory
 * path); sort_every: steps between tile sorts inside pic_step; filter_passes:
 * Binomial2 passes applied to J inside pic_step (Sect. 4.2 uses 8, the
 * 3D shock-shaped workload 4); chunk: target particles per thread block (a box
 * with fewer tiles than 4 per SM splits them further, down to 256 particles
 * per block, until the particle launch has 4 blocks per SM). */
typedef struct {
  int tile[3];
  int halo;
  int sort_every;
  int filter_passes;
  int chunk;
} pic_tuning;

/* Which field update pic_field_update performs. */
#define PIC_FIELD_B_HALF 0 /* Eq. (fdB) over half a step: B -= (c/2) curl E */
#define PIC_FIELD_E 1      /* Eq. (fdE) with add_cur (Table 1): E += c curl B - J */

/* Kernel kinds reported by pic_kernel_times. */
#define PIC_KERNEL_PUSH 0   /* gather + push + move + deposit (fused) */
#define PIC_KERNEL_BHALF 1  /* B half step */
#define PIC_KERNEL_EUPD 2   /* E update with -J (on a periodic FDTD2 lattice of
                               at most 4096 points: with the second B half step,
                               and inside a multi-step pic_step call with the
                               next step's first B half step, in one launch) */
#define PIC_KERNEL_FILTER 3 /* one Binomial2 pass */
#define PIC_KERNEL_SORT 4   /* tile sort: count + scan + scatter + copy back */
#define PIC_KERNEL_BOUNDARY 5 /* wall fields and injection (pic_set_shock) */
#define PIC_KERNEL_ADJOINT 6  /* pic_adjoint_step */
#define PIC_KERNEL_KINDS 7

/* Create a context for `grid`, `nspecies` (1..PIC_MAX_SPECIES) species, Courant
 * number c (0 < c < 1 for the explicit scheme, Sect. 2.3) and time step dt,
 * which must be 1 (code units of Sect. 2.3).  `fields` is the caller's device
 * buffer of 9 planes; `stream` a cudaStream_t (NULL = legacy default stream).
 * Validates every argument, allocates the scratch, sorts the particles by
 * tile (on the stream) and stores the new context in *out.  On failure *out
 * is NULL and nothing stays allocated. */
pic_status pic_init(pic_ctx** out, const pic_grid* grid, const pic_species* species,
                    int nspecies, float c, float dt, float* fields, void* stream);

/* Read or change the launch parameters.  Changing tile re-sorts the particles. */
pic_status pic_get_tuning(pic_ctx* ctx, pic_tuning* out);
pic_status pic_set_tuning(pic_ctx* ctx, const pic_tuning* t);

/* Field solver of the context: PIC_FDTD2 (Eqs. fdE/fdB, second-order Yee; the
 * default) or PIC_FDTD4 (Table 2; read as the fourth-order staggered
 * differences (9/8)[f(i+1/2)-f(i-1/2)] - (1/24)[f(i+3/2)-f(i-3/2)] in both
 * curls, second order in time).  FDTD4 needs c sqrt(dim) 7/6 < 1, else
 * PIC_ERR_ARG.  The Gauss residual of pic_energies is the second-order one
 * that the ZigZag deposit conserves; with FDTD4 it is no longer constant. */
#define PIC_FDTD2 2
#define PIC_FDTD4 4
pic_status pic_set_field_solver(pic_ctx* ctx, int order);

/* Particle pusher of the context: PIC_PUSHER_BORIS (Appendix C; the default)
 * or PIC_PUSHER_HIGUERA_CARY (Table 2, the pusher of the paper's shock run,
 * Higuera and Cary 2017: the Boris steps with the rotation's Lorentz factor
 * solved so that the E x B drift is exact at any speed).  Takes effect from
 * the next push; PIC_ERR_ARG for other values. */
#define PIC_PUSHER_BORIS 0
#define PIC_PUSHER_HIGUERA_CARY 1
pic_status pic_set_pusher(pic_ctx* ctx, int pusher);

/* Counting sort by tile of every species (replaces the particle migration
 * routines of Table 1, check_outg_prtcls ... del_vir_prtcls, on one GPU).
 * Particles are grouped by tile; the order inside a tile is not specified. */
pic_status pic_sort(pic_ctx* ctx);

/* Number of sort bins of the current tiling (tiles, times sub-tiles where
 * the tiles are sorted by sub-tile): the length, minus one, of the bucket
 * starts that pic_sort_record writes.  *nbins is set; PIC_ERR_ARG on NULL. */
pic_status pic_sort_bins(pic_ctx* ctx, int64_t* nbins);

/* pic_sort, recorded, for the adjoint of a run that sorts (the paper has no
 * counterpart).  The particles are sorted in place (their own rows hold the
 * sorted order on return) and for every species s with particles:
 * perm[s] (int32[n_s], device) receives, for each slot i, the slot that the
 * particle now in slot i held before the sort; tstart[s] (int32[nbins + 1],
 * device, nbins from pic_sort_bins) the first slot of each sort bin, the
 * last entry n_s.  pic_adjoint_step runs its tile pass on particles grouped
 * this way, and pic_adjoint_unsort carries gradients back through perm.
 * Entries for species without particles may be NULL.  PIC_ERR_ARG on NULL
 * arguments; enqueued on the context's stream. */
pic_status pic_sort_record(pic_ctx* ctx, int32_t* const* perm, int32_t* const* tstart);

/* interp_em + push of Table 1 for every species: linear gather of E and B at
 * x^n (Sect. 2.3.2), relativistic Boris push u^(n-1/2) -> u^(n+1/2)
 * (Appendix C), position update x^(n+1) = x^n + c u / gamma (Eq. fdX) with
 * periodic wrap.  The pre-move positions are kept in library scratch for
 * pic_deposit.  PIC_ERR_STATE on a context with shock boundaries (the split
 * path does not model the wall; pic_step does). */
pic_status pic_gather_push(pic_ctx* ctx);

/* comp_curr of Table 1: adds the ZigZag current (Appendix D) of every particle's
 * move since the last pic_gather_push into the J planes (J is not cleared).
 * PIC_ERR_STATE if no pic_gather_push preceded it. */
pic_status pic_deposit(pic_ctx* ctx);

/* `passes` (>= 0) passes of the Binomial2 (1/4,1/2,1/4) filter along every
 * gridded dimension on Jx, Jy, Jz (Table 2).  The result is left in the J
 * planes. */
pic_status pic_filter_current(pic_ctx* ctx, int passes);

/* One field update, `which` = PIC_FIELD_B_HALF or PIC_FIELD_E. */
pic_status pic_field_update(pic_ctx* ctx, int which);

/* `nsteps` full time steps in the order of Table 1: B half step, gather +
 * push + deposit (fused; J cleared first), B half step, filter_passes
 * Binomial2 passes on J, E update with -J.  Every sort_every steps (counted
 * over the life of the context) the particles are re-sorted by tile before
 * the push.  On return the J planes hold the filtered current of the last
 * step.  With shock boundaries (pic_set_shock) the wall's field boundary
 * follows each field update and the injector adds particles at the end of
 * each step; PIC_ERR_ARG (before any work of that step) if a species would
 * exceed its cap. */
pic_status pic_step(pic_ctx* ctx, int nsteps);

/* Shock boundaries along x (Sect. 4.2; the paper states them in words, the
 * readings below make them precise).
 *
 * Conducting wall on the node plane x = wall (1 <= wall, 2 wall < i_zero): a
 * particle whose move ends below x = wall is reflected specularly
 * (x -> 2 wall - x, u_x -> -u_x) and its current is deposited along the true
 * path, a straight ZigZag segment to the wall plane and the mirrored
 * remainder, so charge is conserved on every node.  After each field update
 * the tangential E on the wall plane (Ey, Ez at i = wall) is set to zero and
 * the cells behind it (i < wall) to the mirror image of the plasma side that a
 * perfect conductor implies (tangential E and normal B odd, normal E and
 * tangential B even about x = wall: integer-x components at i take the value
 * at 2 wall - i, half-integer ones, stored at i for x = i + 1/2, the value at
 * 2 wall - 1 - i).  The Gauss residual of pic_energies then holds on the
 * nodes i > wall; the wall node carries the conductor's surface charge.
 *
 * Receding injector: it starts at x0 and moves at v_inj cells per step (the
 * paper: the speed of light, c) up to x_max, X(s) = min(x0 + v_inj s, x_max)
 * with s the steps since this call.  An upstream template per species (host
 * arrays in the layout of pic_host_species with rows of nt[s] elements; cells
 * index an lt x ny x nz block, sorted by x = i + off_x; q and m are those of
 * the species) is repeated along x and moves at -v_up cells per step.  In
 * template coordinates the injector is at A(s) = (X(s) - x0) + v_up s; during
 * step s every particle of copy m with A(s) - m lt <= x_t < A(s+1) - m lt is
 * appended to its species at x = x_t + ((m lt + x0) - v_up (s + 1)) (double
 * precision; the offset is rounded to float and an offset that rounds to 1
 * moves to the next cell), in the order m, then template index.  E and B at
 * i >= i_zero = floor(x_max) + 2 are set to zero after each field update.
 * The library copies the templates; the species' device arrays must have
 * room (cap) for what is injected.  Requires x0 > wall, x0 <= x_max <= nx - 3,
 * v_inj >= 0, v_up >= 0, v_inj + v_up < lt, and every particle at x >= wall
 * (particles behind the wall are flagged as invalid data by pic_check).
 * Contexts with shock boundaries cannot join a batch, and pic_gather_push /
 * pic_deposit refuse them.  PIC_ERR_ARG on invalid arguments. */
typedef struct {
  int wall;
  int lt;
  double x0, x_max, v_inj, v_up;
  int64_t nt[PIC_MAX_SPECIES];
  pic_host_species tmpl[PIC_MAX_SPECIES];
} pic_shock;
pic_status pic_set_shock(pic_ctx* ctx, const pic_shock* shock);

/* Discrete adjoint (reverse mode) of one pic_step, for gradients of a loss
 * of the state after many steps with respect to an earlier state (the
 * paper's method has no adjoint; this differentiates its time step).  The
 * step is read as the composition
 *   B1 = B - (c/2) curl+ E;  e, b = gather(E, B1; x);  u' = Boris(u, e, b);
 *   x' = x + c u'/gamma(u');  J = sum ZigZag(x, x');  B2 = B1 - (c/2) curl+ E;
 *   E' = E + c curl- B2 - F^p J      (Eqs. fdB, fdX, fdE; Apps. C, D; Table 1)
 * and reversed exactly: (curl+)^T = curl- on the periodic lattice, the
 * Binomial2 filter F is symmetric, and each particle goes back through the
 * chain rule of ZigZag, move, Boris and gather (its cell and the branch of
 * the ZigZag relay point are those of the forward step, where the step is
 * differentiable).
 *
 * fwd_fields: the caller's device copy of the 9 field planes at the start of
 * the step (E^n, B^(n-1/2)); sp[s].cell/off/u: the species' particles at the
 * start of the step, in the slots the adjoint arrays use (rows of the
 * species' cap, count from pic_particle_counts); sp[s].xbar (float[dim][cap])
 * and sp[s].ubar (float[3][cap]): on entry the gradient with respect to the
 * particles after the step, on exit before it.  adj_fields (9 planes): on
 * entry the gradient with respect to E and B after the step (the J planes
 * are scratch), on exit with respect to E and B before it (J planes zero).
 * Uses the context's grid, Courant number, species q/m and filter passes;
 * PIC_ERR_STATE unless the field solver is FDTD2, the pusher Boris and there
 * are no shock boundaries.  Enqueued on the context's stream. */
typedef struct {
  const int32_t* cell;
  const float* off;
  const float* u;
  float* xbar;
  float* ubar;
  const int32_t* tstart;
} pic_adjoint_species;
pic_status pic_adjoint_step(pic_ctx* ctx, const float* fwd_fields, const pic_adjoint_species* sp,
                            float* adj_fields);

/* The particles' rows were put back (by the caller) into an order that
 * pic_sort_record produced: the context takes its bucket starts tstart[s]
 * (int32[nbins + 1], device) as the grouping of every species, so the next
 * steps run their tile kernels on it, and sorts nothing itself.  For
 * restoring a checkpoint taken after pic_sort_record (the paper has no
 * counterpart).  Starts that do not run from 0 to n_s without decreasing
 * are replaced by one bucket (correct, but every particle then takes the
 * stray path) and the next pic_check reports PIC_ERR_STATE.  PIC_ERR_ARG on
 * NULL arguments; enqueued on the context's stream. */
pic_status pic_sort_assume(pic_ctx* ctx, const int32_t* const* tstart);

/* sp[s].tstart of pic_adjoint_step: NULL, or the bucket starts written by the
 * pic_sort_record that grouped cell/off/u (since then the particles may have
 * moved, as pic_step moves them, but not been reordered; the context's
 * tiling unchanged).  When every species with particles gives one (and the
 * tile window's 15 planes fit in 200 KB of shared memory), a tile
 * pass stages E, B and the current adjoint of each tile's window in shared
 * memory and sums the E and B adjoints there; particles whose stencil left
 * the window go through global memory, as all particles do otherwise.  The
 * result is the same up to the order of floating-point sums.  Starts that are
 * not a partition of the species' particles are replaced, for this step, by
 * one bucket, and the next pic_check reports PIC_ERR_STATE. */

/* The gradients of pic_adjoint_step carried back through a recorded sort:
 * for every species with particles, sp[s].xbar and sp[s].ubar (rows of the
 * species' cap) are permuted in place from the order after the sort to the
 * order before it (row entry i moves to slot perm[s][i]), perm[s] as written
 * by pic_sort_record (entries outside [0, n_s) are skipped and reported by
 * the next pic_check).  The other fields of sp are not used.  PIC_ERR_ARG on
 * NULL arguments, PIC_ERR_STATE while a sorted copy of the particles awaits
 * its push (the library's sort buffer is the scratch); enqueued on the
 * context's stream. */
pic_status pic_adjoint_unsort(pic_ctx* ctx, const int32_t* const* perm,
                              const pic_adjoint_species* sp);

/* Current particle count of each species (grows with injection): writes
 * nout >= nspecies values.  No synchronisation: the counts are host state. */
pic_status pic_particle_counts(pic_ctx* ctx, int64_t* n, int nout);

/* Diagnostics (synchronising).  out[0] = 0.5 sum E^2, out[1] = 0.5 sum B^2,
 * out[2+s] = sum m c^2 (gamma - 1) of species s, out[2+ns] = max |div E -
 * F^p(rho)|, out[3+ns] = rms of the same over the nodes, where rho is the
 * first-order charge on the nodes and F^p the filter_passes-fold Binomial2
 * filter (Appendix B: this residual is conserved).  Sums are accumulated in
 * double precision on the GPU.  nout must be >= 4 + nspecies. */
pic_status pic_energies(pic_ctx* ctx, double* out, int nout);

/* Synchronise the stream and read the device status word: PIC_ERR_TIMEOUT if
 * a kernel since the last check gave up a bounded wait on one of its own
 * shared-memory copies (that step's results are not valid), else
 * PIC_ERR_STATE if one met invalid particle data, otherwise PIC_OK.  The word
 * is cleared when it was set. */
pic_status pic_check(pic_ctx* ctx);

/* Failure-path check of the bounded device waits (the paper has no
 * counterpart): enqueues on the context's stream one warp that waits on a
 * shared-memory barrier that nothing completes.  Its wait gives up after about
 * a second of SM clock and sets the timeout bit of the context's status word,
 * exactly as a particle block's wait on a tensor copy that did not land would;
 * the next pic_check returns PIC_ERR_TIMEOUT and clears the word, and the
 * context stays usable.  No copy is in flight and no GPU fault is raised.
 * PIC_ERR_ARG for a NULL context, PIC_ERR_CUDA if the launch fails. */
pic_status pic_wait_probe(pic_ctx* ctx);

/* Particles per chunk of a species in pic_step_host's overlapped copies
 * (default 2^21; at most 8 chunks per species).  PIC_ERR_ARG outside
 * [1, 2^30]. */
pic_status pic_set_host_chunk(pic_ctx* ctx, int64_t particles);

/* End-to-end step from host memory: copies every species' particles from
 * `hs` and the 9 field planes from `host_fields` into the context's device
 * buffers, runs pic_step(nsteps), copies particles and fields back into the
 * same host buffers and synchronises.  Host rows have the species' cap
 * elements; the counts before the steps are copied in and those after them
 * (pic_particle_counts) copied out.  Host buffers should be pinned (page-
 * locked) for the copies to overlap.  On boxes without shock boundaries, with
 * the event timers off and nsteps >= 1, the copies overlap: each species is
 * cut into chunks of slots (pic_set_host_chunk), copied in on one stream of
 * the library's (fields first, then chunk after chunk) and out on another;
 * the last step runs the particle kernel chunk by chunk, each as soon as its
 * chunk is in (a sort due at that step waits for the whole species), and each
 * chunk is copied out as soon as its launch is done while later chunks are
 * still coming in.  The result equals pic_step's up to the float rounding of
 * J's sum (each launch adds its own window sums to J). */
pic_status pic_step_host(pic_ctx* ctx, const pic_host_species* hs, float* host_fields,
                         int nsteps);

/* Autotuner of the launch parameters (tile size, halo, sort cadence; the
 * filter passes are physics and are kept).  Runs real time steps, which
 * advance the simulation exactly as pic_step does.  Two passes over the
 * candidates, the second in reverse order: for each candidate it re-sorts if
 * the tiles change, takes 2*sort_every untimed steps (which also capture its
 * step graph), then times max(steps, 2*sort_every) steps (rounded up to whole
 * sort cycles) with CUDA events; the candidate with the smallest sum of its
 * two per-step times is kept.  candidates == NULL selects a built-in set of
 * 18 for the grid's dimension (three tile shapes around the default, halos 3
 * and 4 in 1D/2D or 2 and 3 in 3D, three cadences).  *best_index (may be
 * NULL) receives the chosen candidate's index.  Synchronises.  Candidates
 * that pic_set_tuning rejects are skipped; PIC_ERR_ARG if none is valid. */
pic_status pic_autotune(pic_ctx* ctx, const pic_tuning* candidates, int ncandidates, int steps,
                        int* best_index);

/* Synchronise and report, in *strays, how many particle updates since the
 * last call found the particle outside its tile's shared-memory window and
 * went through global memory instead (then reset the count).  The fraction
 * strays / (particles * steps) is what the sort cadence trades against. */
pic_status pic_stats(pic_ctx* ctx, int64_t* strays);

/* Per-kernel timing with CUDA events on the context stream.  While enabled,
 * every launch of the kinds above is bracketed by events.  pic_kernel_times
 * synchronises, adds the elapsed milliseconds and launch counts of each kind
 * since the last reset into ms[PIC_KERNEL_KINDS] and launches[...], and
 * resets the counters. */
pic_status pic_timing(pic_ctx* ctx, int enable);
pic_status pic_kernel_times(pic_ctx* ctx, double* ms, int64_t* launches);

/* Allocation-free variant of pic_filter_current.  The paper has no
 * counterpart; this entry point exists for callers that cannot let a library
 * allocate device memory: applications whose memory manager (for instance a
 * framework's caching allocator) owns the device and forbids raw cudaMalloc,
 * code that must stay inside a fixed memory budget, and latency-critical loops
 * where the device-wide synchronisation that cudaFree implies would stall
 * other streams.  It needs no context and calls no allocator: its scratch is
 * a fixed array of PIC_FILTER_STATIC_MAX_FLOATS floats (16 MiB) compiled into
 * the library, which every GPU that loads the library holds until the process
 * exits.
 *
 * grid: as for pic_init.  J: device pointer to the caller's three current
 * planes Jx, Jy, Jz, contiguous, nx*ny*nz floats each (the layout of planes
 * 6-8 of the field buffer), filtered in place by `passes` (>= 0) Binomial2
 * passes, enqueued on `stream` (a cudaStream_t, NULL = legacy default) without
 * synchronising.  3*nx*ny*nz larger than PIC_FILTER_STATIC_MAX_FLOATS is
 * rejected with PIC_ERR_ARG; CUDA failures give PIC_ERR_CUDA; the message is
 * in pic_last_error(NULL).
 *
 * The first call on a device looks up the device address of the scratch array
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  The address is kept per device ordinal for the life of
 * the process: after cudaDeviceReset (or when a caller makes a different
 * driver-API context current on the same device) it is stale, and calls on
 * that device must not be made again.  Every call uses the same array, which keeps the last
 * call's contents; each pass writes the whole part it later reads, so nothing
 * needs clearing.  Calls whose GPU work overlaps (on different streams or from
 * different host threads, on the same device) race on the array: the caller
 * must order them. */
#define PIC_FILTER_STATIC_MAX_FLOATS 4194304
pic_status pic_filter_current_static(const pic_grid* grid, float* J, int passes, void* stream);

/* Ensemble stepping (many independent boxes; the paper steps one box).  A
 * batch groups existing contexts (independent boxes, any mix of sizes and
 * dimensions, all on one device and one stream).  pic_batch_step advances
 * every context by nsteps: the steps of all boxes for one cycle of L steps,
 * L = lcm of the contexts' sort_every (at most 240), are captured once into a
 * single CUDA graph in which each box is an independent branch, and that graph
 * is launched nsteps / L times on `stream`; the remaining steps run through
 * pic_step.  The graph is rebuilt when a context's tuning or its position in
 * its sort cycle changed since the capture.  Results are those of pic_step
 * on each context.  Contexts must not be destroyed before the batch, and a
 * context with shock boundaries cannot join one.  Errors: PIC_ERR_ARG
 * (message in pic_last_error(NULL)), PIC_ERR_CUDA. */
typedef struct pic_batch pic_batch;
pic_status pic_batch_create(pic_batch** out, pic_ctx* const* ctxs, int nctx);
pic_status pic_batch_step(pic_batch* batch, int nsteps, void* stream);
pic_status pic_batch_destroy(pic_batch* batch);

/* Release the context and its scratch (the caller's buffers are untouched). */
pic_status pic_destroy(pic_ctx* ctx);

/* Message of the last failure on ctx ("" if none); for ctx == NULL, the last
 * failure of pic_init or pic_filter_current_static in the calling thread. */
const char* pic_last_error(const pic_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif

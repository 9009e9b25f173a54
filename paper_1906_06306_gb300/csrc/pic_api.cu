// C ABI of the PIC hot path (see include/pic.h): argument checking, scratch
// ownership, the order of the time step (Table 1 of arXiv:1906.06306) and
// event timing.  All device work goes to the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pic.h"
#include "pic_kernels.h"

using namespace pic;

namespace {

struct TimedLaunch {
  cudaEvent_t a, b;
  int kind;
};

thread_local std::string g_init_error;

// most chunks per species of the overlapped pic_step_host
constexpr int kHostChunks = 8;

}  // namespace

namespace pic {
void set_global_error(const char* msg) { g_init_error = msg; }
}  // namespace pic

struct pic_ctx {
  pic_grid grid{};
  int ns = 0;
  pic_species sp[PIC_MAX_SPECIES]{};
  float c = 0.f;
  float* F = nullptr;
  cudaStream_t st = nullptr;
  pic_tuning tun{};
  GridDev g{};
  TileDev tile{};
  int splits = 1;
  int splits_ens = 1;     // the same without the GPU-filling rule (inside a batch graph)
  bool ensemble = false;  // being captured into a batch graph
  long long ntot = 0, nmax = 0;
  int* d_tstart[PIC_MAX_SPECIES] = {};
  int* d_count = nullptr;   // per tile
  int* d_cursor = nullptr;  // per tile
  void* d_sortbuf = nullptr;   // sorted particles of every species (one record layout each)
  bool sorted_pending = false;  // the next push reads the sorted buffer (no copy back)
  int* d_cell_old = nullptr;
  float* d_off_old = nullptr;
  bool snapshot_valid = false;
  float* d_jtmp = nullptr;
  double* d_rho = nullptr;
  double* d_rho2 = nullptr;
  double* d_acc = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_strays = nullptr;  // particles that took the global path
  int pusher = 0;                          // PIC_PUSHER_*
  long long cap[PIC_MAX_SPECIES] = {};     // row length of each species' arrays
  long long sorted_n[PIC_MAX_SPECIES] = {};  // count at the last sort (start of the tail)
  // shock boundaries (pic_set_shock)
  bool shock = false;
  int wall = 0, i_zero = 0, lt = 0;
  double x0 = 0.0, x_max = 0.0, v_inj = 0.0, v_up = 0.0;
  long long shock_steps = 0;                 // steps since pic_set_shock
  long long tn[PIC_MAX_SPECIES] = {};        // template particles per species
  std::vector<double> txs[PIC_MAX_SPECIES];  // template x = i + off_x (host, sorted)
  void* d_tmpl = nullptr;                    // template records of every species
  int* d_adj_tstart = nullptr;  // checked copies of the adjoint's bucket starts
  size_t adj_tstart_len = 0;
  int* d_dlist = nullptr;   // particles deferred to the global pass, room for cap[s] per species
  int* d_dcount = nullptr;  // entries per species
  float* d_adjF = nullptr;                   // forward fields of an adjoint step (9 planes)
  // 2D field window by tensor copy: the map over E and B, box and shift
  // (window_map); win_tma == 0 when the grid or tiling does not allow it
  CUtensorMap win_map{};
  int win_tma = 0;
  int win_box[2] = {0, 0};
  int win_shift = 0;
  long long steps = 0;
  long long sorted_step = -1;  // value of `steps` at the last tile sort
  bool capturing = false;      // pic_step is being captured into a CUDA graph
  // pic_step(n) replays whole sort cycles from a CUDA graph (boxes without
  // shock boundaries, timing off), captured on cap_st; it stays valid while
  // the tuning, the pusher and field solver, and the phase of the sort cycle
  // are those of the capture
  cudaStream_t cap_st = nullptr;
  cudaGraph_t step_graph = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  pic_tuning step_tun{};
  long long step_phase = -1;
  int step_solver = -1;
  // pic_step_host's copy streams (in, out), its events (copied in and pushed,
  // per species and chunk; three more) and clipped bucket starts (one table
  // per chunk), made on first use
  cudaStream_t io_st[2] = {nullptr, nullptr};
  cudaEvent_t io_ev[2 * PIC_MAX_SPECIES * kHostChunks + 3] = {};
  int* d_tclip = nullptr;
  long long tclip_len = 0;
  long long host_chunk = 1LL << 21;  // particles per chunk (pic_set_host_chunk)
  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> pool;
  double ms[PIC_KERNEL_KINDS] = {};
  int64_t launches[PIC_KERNEL_KINDS] = {};
  std::string err;
};

namespace {

pic_status set_err(pic_ctx* ctx, pic_status s, const std::string& msg) {
  if (ctx)
    ctx->err = msg;
  else
    g_init_error = msg;
  return s;
}

pic_status cuda_fail(pic_ctx* ctx, const char* what, cudaError_t e) {
  const pic_status s = (e == cudaErrorMemoryAllocation) ? PIC_ERR_OOM : PIC_ERR_CUDA;
  return set_err(ctx, s, std::string(what) + ": " + cudaGetErrorString(e));
}

#define PIC_CK(ctx, call)                                     \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((ctx), #call, e_); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count);
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

void free_all(pic_ctx* ctx) {
  for (int s = 0; s < PIC_MAX_SPECIES; ++s) dfree(ctx->d_tstart[s]);
  dfree(ctx->d_count);
  dfree(ctx->d_cursor);
  dfree(ctx->d_sortbuf);
  dfree(ctx->d_cell_old);
  dfree(ctx->d_off_old);
  dfree(ctx->d_jtmp);
  dfree(ctx->d_rho);
  dfree(ctx->d_rho2);
  dfree(ctx->d_acc);
  dfree(ctx->d_status);
  dfree(ctx->d_strays);
  dfree(ctx->d_tmpl);
  dfree(ctx->d_adj_tstart);
  dfree(ctx->d_dlist);
  dfree(ctx->d_dcount);
  dfree(ctx->d_adjF);
  dfree(ctx->d_tclip);
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  ctx->step_exec = nullptr;
  ctx->step_graph = nullptr;
  if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
  ctx->cap_st = nullptr;
  for (auto& io : ctx->io_st) {
    if (io) cudaStreamDestroy(io);
    io = nullptr;
  }
  for (auto& ev : ctx->io_ev) {
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
  }
  for (auto& t : ctx->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  ctx->pending.clear();
  for (auto e : ctx->pool) cudaEventDestroy(e);
  ctx->pool.clear();
}

int extent(const pic_grid& g, int d) { return d == 0 ? g.nx : d == 1 ? g.ny : g.nz; }

// Streaming multiprocessors of the current device (looked up once).
int device_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      sms = v;
    else
      return 152;
  }
  return sms;
}

// Tile geometry from the tuning; returns an error message or "".
std::string derive_tiles(const pic_grid& grid, const pic_tuning& tun, long long ntot,
                         TileDev* t, int* splits, int* splits_ens) {
  if (tun.halo < 1) return "halo must be >= 1";
  if (tun.chunk < 32) return "chunk must be >= 32";
  TileDev r{};
  r.H = tun.halo;
  long long ntiles = 1, wcells = 1;
  for (int d = 0; d < 3; ++d) {
    if (d < grid.dim) {
      if (tun.tile[d] < 1) return "tile extents must be >= 1";
      const int n = extent(grid, d);
      r.T[d] = tun.tile[d] < n ? tun.tile[d] : n;
      r.nt[d] = (n + r.T[d] - 1) / r.T[d];
      r.W[d] = r.T[d] + 2 * r.H + 1;
      const int ks = grid.dim == 3 ? kSubTile3[d] : grid.dim == 2 ? kSubTile2[d] : 0;
      const int sub = ks > 0 && ks < r.T[d] ? ks : r.T[d];
      r.S[d] = sub;
      r.ns[d] = (r.T[d] + sub - 1) / sub;
    } else {
      r.T[d] = 1;
      r.nt[d] = 1;
      r.W[d] = 1;
      r.S[d] = 1;
      r.ns[d] = 1;
    }
    ntiles *= r.nt[d];
    wcells *= r.W[d];
  }
  if (wcells > (1LL << 24)) return "tile + halo window too large";
  r.wcells = (int)wcells;
  r.wstride = (int)((wcells + 3) / 4 * 4);
  if ((long long)particle_smem_bytes(grid.dim, r) > 200 * 1024)
    return "tile + halo window exceeds 200 KB of shared memory";
  if (ntiles > (1LL << 30)) return "too many tiles";
  r.ntiles = (int)ntiles;
  r.nsub = r.ns[0] * r.ns[1] * r.ns[2];
  if (ntiles * r.nsub > (1LL << 30)) return "too many sort bins";
  const long long per_tile = (ntot + ntiles - 1) / ntiles;
  const auto clamp = [](long long v) { return (int)(v < 1 ? 1 : v > 1024 ? 1024 : v); };
  long long sp = (per_tile + tun.chunk - 1) / tun.chunk;
  *splits_ens = clamp(sp);
  // a box with few tiles splits them further, down to 256 particles per block,
  // until a launch has 4 blocks per SM (else most of the GPU idles while each
  // thread runs many particles in turn); inside a batch graph the ensemble
  // fills the GPU and the finer split only adds window loads and flushes
  const long long fill = (4LL * device_sms() + ntiles - 1) / ntiles;
  const long long fine = (per_tile + 255) / 256;
  if (sp < fill) sp = fill < fine ? fill : fine;
  *t = r;
  *splits = clamp(sp);
  return "";
}

void window_map(pic_ctx* ctx);

pic_status alloc_tiles(pic_ctx* ctx) {
  for (int s = 0; s < ctx->ns; ++s) {
    dfree(ctx->d_tstart[s]);
    PIC_CK(ctx, dalloc(&ctx->d_tstart[s], sort_bins(ctx->tile) + 1));
  }
  dfree(ctx->d_count);
  dfree(ctx->d_cursor);
  // the counts, then the multi-block scan's scratch
  PIC_CK(ctx, dalloc(&ctx->d_count, sort_bins(ctx->tile) + scan_scratch(sort_bins(ctx->tile))));
  PIC_CK(ctx, dalloc(&ctx->d_cursor, sort_bins(ctx->tile)));
  window_map(ctx);
  return PIC_OK;
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link to
// libcuda); null when the driver does not provide it
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// The tensor map of the 2D window copy: the field buffer as a 3D tensor
// (x, y, plane) of FP32, box (box_x, W1, 6) over the E and B planes, whose x
// origin is the window's rounded down to a multiple of 4 floats (tensor
// copies start 16-byte aligned; the window starts at tile x * T0 - H, the same
// residue mod 4 for every tile when T0 is a multiple of 4).  Out-of-range box
// points (up to 3 past the lattice's x end) are filled with zeros and never
// read.
void window_map(pic_ctx* ctx) {
  ctx->win_tma = 0;
  const TileDev& t = ctx->tile;
  const int nx = ctx->grid.nx, ny = ctx->grid.ny;
  if (!PIC_TMA_WINDOW || ctx->grid.dim != 2 || t.T[0] % 4 != 0 || nx % 4 != 0 ||
      (reinterpret_cast<uintptr_t>(ctx->F) & 15) != 0)
    return;
  const int shift = ((-t.H) % 4 + 4) % 4;
  const int bx = (t.W[0] + shift + 3) / 4 * 4, by = t.W[1];
  if (bx > 256 || by > 256 || 6LL * bx * by > window_landing_floats(2, t)) return;
  EncodeTiled enc = encode_tiled();
  if (!enc) return;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
  const cuuint64_t strides[2] = {4ULL * nx, 4ULL * nx * ny};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 6};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&ctx->win_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ctx->F, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return;
  ctx->win_tma = 1;
  ctx->win_box[0] = bx;
  ctx->win_box[1] = by;
  ctx->win_shift = shift;
}

cudaEvent_t take_event(pic_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Run `fn` (which enqueues one kind of work) bracketed by timing events when
// timing is on.
template <typename Fn>
cudaError_t timed(pic_ctx* ctx, int kind, Fn fn) {
  if (!ctx->timing) return fn();
  TimedLaunch t{take_event(ctx), take_event(ctx), kind};
  cudaEventRecord(t.a, ctx->st);
  const cudaError_t e = fn();
  cudaEventRecord(t.b, ctx->st);
  ctx->pending.push_back(t);
  return e;
}

// offset (in 4-byte words) of species s in the sorted buffer
long long sortbuf_offset(const pic_ctx* ctx, int s) {
  long long o = 0;
  for (int r = 0; r < s; ++r) o += ctx->cap[r] * (1 + ctx->grid.dim + 3);
  return o;
}

long long total_cap(const pic_ctx* ctx) {
  long long t = 0;
  for (int s = 0; s < ctx->ns; ++s) t += ctx->cap[s];
  return t;
}

// Copy `rows` rows of n elements of `elem` bytes between arrays whose rows
// are ld elements long.
cudaError_t copy_rows(void* dst, const void* src, size_t elem, long long n, long long ld, int rows,
                      cudaMemcpyKind kind, cudaStream_t st) {
  if (n == 0 || rows == 0) return cudaSuccess;
  if (ld == n) return cudaMemcpyAsync(dst, src, elem * (size_t)n * rows, kind, st);
  return cudaMemcpy2DAsync(dst, elem * (size_t)ld, src, elem * (size_t)ld, elem * (size_t)n,
                           (size_t)rows, kind, st);
}

// Thread blocks for the particles appended since the last sort.
int tail_blocks(const pic_ctx* ctx) {
  long long mx = 0;
  for (int s = 0; s < ctx->ns; ++s) mx = std::max(mx, ctx->sp[s].n - ctx->sorted_n[s]);
  const long long b = (mx + kPushThreads - 1) / kPushThreads;
  return (int)std::min<long long>(b, 8 * 152);
}

PushParams make_params(pic_ctx* ctx) {
  PushParams P{};
  P.g = ctx->g;
  P.t = ctx->tile;
  P.F = ctx->F;
  P.nspecies = ctx->ns;
  P.splits = ctx->ensemble ? ctx->splits_ens : ctx->splits;
  P.status = ctx->d_status;
  P.strays = ctx->d_strays;
  P.pusher = ctx->pusher;
  P.inv_c = 1.0f / ctx->c;
  P.inv_c2 = 1.0f / (ctx->c * ctx->c);
  P.div0 = make_fastdiv(ctx->g.n[0]);
  P.div1 = make_fastdiv(ctx->g.n[1]);
  P.wrap_fast = 1;
  for (int d = 0; d < ctx->grid.dim; ++d)
    if (ctx->g.n[d] < ctx->tile.W[d]) P.wrap_fast = 0;
  float maxq = 0.f;
  for (int s = 0; s < ctx->ns; ++s) maxq = std::fmax(maxq, std::fabs(ctx->sp[s].q));
  P.jq = current_quantum(maxq, ctx->c, kPushThreads * kSpillEvery);
  P.jq_inv = 1.0f / P.jq;
  long long o = 0;
  for (int s = 0; s < ctx->ns; ++s) {
    SpeciesDev& S = P.sp[s];
    S.q = ctx->sp[s].q;
    S.qm = ctx->sp[s].q / ctx->sp[s].m;
    S.n = ctx->sp[s].n;
    S.ld = ctx->cap[s];
    S.tail = ctx->sorted_n[s];
    S.cell = ctx->sp[s].cell;
    S.off = ctx->sp[s].off;
    S.u = ctx->sp[s].u;
    S.rcell = S.cell;
    S.roff = S.off;
    S.ru = S.u;
    if (ctx->sorted_pending) {
      int* c = (int*)ctx->d_sortbuf + sortbuf_offset(ctx, s);
      S.rcell = c;
      S.roff = (const float*)(c + S.ld);
      S.ru = (const float*)(c + S.ld) + (long long)ctx->grid.dim * S.ld;
    }
    S.tstart = ctx->d_tstart[s];
    S.cell_old = ctx->d_cell_old ? ctx->d_cell_old + o : nullptr;
    S.off_old = ctx->d_off_old ? ctx->d_off_old + (long long)ctx->grid.dim * o : nullptr;
    S.dlist = ctx->d_dlist + o;
    S.dcount = ctx->d_dcount + s;
    o += ctx->cap[s];
  }
  P.wall = ctx->shock ? ctx->wall : 0;
  P.tail_blocks = tail_blocks(ctx);
  P.dcount = ctx->d_dcount;
  P.win_tma = ctx->win_tma;
  P.win_box[0] = ctx->win_box[0];
  P.win_box[1] = ctx->win_box[1];
  P.win_shift = ctx->win_shift;
  P.win_map = ctx->win_map;
  P.rec_aligned = 1;
  for (int s = 0; s < ctx->ns; ++s) {
    const SpeciesDev& S = P.sp[s];
    const auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    if (S.ld % 4 != 0 || !a16(S.rcell) || !a16(S.roff) || !a16(S.ru)) P.rec_aligned = 0;
  }
  return P;
}

// Sort every species by tile into the sorted buffer.  With copy_back the
// sorted particles are copied into the caller's arrays; without, the next push
// reads them from the buffer and writes the caller's arrays (pic_step).
// The launches that sort species s by tile into its part of the sorted
// buffer (and, with copy_back, copy it back into the caller's arrays).
cudaError_t sort_species(pic_ctx* ctx, int s, bool copy_back, int32_t* perm) {
  const SortParams P = make_sort_params(ctx->g, ctx->tile, ctx->d_status);
  const int D = ctx->grid.dim;
  const long long n = ctx->sp[s].n, ld = ctx->cap[s];
  const int bins = (int)sort_bins(ctx->tile);
  cudaError_t r = cudaMemsetAsync(ctx->d_count, 0, sizeof(int) * bins, ctx->st);
  if (r != cudaSuccess) return r;
  r = launch_tile_count(P, ctx->sp[s].cell, n, ctx->d_count, ctx->st);
  if (r != cudaSuccess) return r;
  r = launch_tile_scan(ctx->d_count, bins, ctx->d_tstart[s], ctx->d_cursor, ctx->d_count + bins,
                       ctx->st);
  if (r != cudaSuccess) return r;
  if (n == 0) return cudaSuccess;
  int* cell_out = (int*)ctx->d_sortbuf + sortbuf_offset(ctx, s);
  float* off_out = (float*)(cell_out + ld);
  float* u_out = off_out + (long long)D * ld;
  r = launch_tile_scatter(P, ctx->sp[s].cell, ctx->sp[s].off, ctx->sp[s].u, n, ld, ctx->d_cursor,
                          cell_out, off_out, u_out, ctx->st, perm);
  if (r != cudaSuccess) return r;
  if (!copy_back) return cudaSuccess;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  r = copy_rows(ctx->sp[s].cell, cell_out, sizeof(int), n, ld, 1, k, ctx->st);
  if (r != cudaSuccess) return r;
  r = copy_rows(ctx->sp[s].off, off_out, sizeof(float), n, ld, D, k, ctx->st);
  if (r != cudaSuccess) return r;
  return copy_rows(ctx->sp[s].u, u_out, sizeof(float), n, ld, 3, k, ctx->st);
}

// The context's bookkeeping of a tile sort of every species (at the current
// step, with or without copy back); launches nothing.
void sort_done(pic_ctx* ctx, bool copy_back) {
  long long ntot = 0;
  for (int s = 0; s < ctx->ns; ++s) {
    ctx->sorted_n[s] = ctx->sp[s].n;
    ntot += ctx->sp[s].n;
  }
  if (ntot != ctx->ntot) {  // injection changed the count: re-derive the splits per tile
    TileDev td{};
    int splits = 1, splits_ens = 1;
    if (derive_tiles(ctx->grid, ctx->tun, ntot, &td, &splits, &splits_ens).empty()) {
      ctx->splits = splits;
      ctx->splits_ens = splits_ens;
    }
    ctx->ntot = ntot;
  }
  ctx->snapshot_valid = false;
  ctx->sorted_pending = !copy_back;
  ctx->sorted_step = ctx->steps;
}

pic_status do_sort(pic_ctx* ctx, bool copy_back, int32_t* const* perm = nullptr) {
  const cudaError_t e = timed(ctx, PIC_KERNEL_SORT, [&]() -> cudaError_t {
    for (int s = 0; s < ctx->ns; ++s) {
      const cudaError_t r = sort_species(ctx, s, copy_back, perm ? perm[s] : nullptr);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  });
  if (e != cudaSuccess) return cuda_fail(ctx, "tile sort", e);
  sort_done(ctx, copy_back);
  return PIC_OK;
}

// Template coordinate of the receding injector after s steps:
// A(s) = (X(s) - x0) + v_up s with X(s) = min(x0 + v_inj s, x_max).
double inj_front(const pic_ctx* ctx, long long s) {
  const double X = std::fmin(ctx->x0 + ctx->v_inj * (double)s, ctx->x_max);
  return (X - ctx->x0) + ctx->v_up * (double)s;
}

// The injection of step s (the particles of template copy m with
// A(s) - m lt <= x_t < A(s+1) - m lt), as runs of template indices per
// species, appended after each species' current particles; add[s] receives
// each species' count.  The template is sorted by x_t, so each (species, m)
// is one contiguous run, found by binary search with the same comparisons.
void plan_injection(const pic_ctx* ctx, long long s, InjectParams* P, long long* add) {
  *P = InjectParams{};
  P->g = ctx->g;
  P->lt = ctx->lt;
  const double a = inj_front(ctx, s), b = inj_front(ctx, s + 1);
  const double lt = (double)ctx->lt;
  long long total = 0;
  for (int sp = 0; sp < ctx->ns; ++sp) {
    const std::vector<double>& xs = ctx->txs[sp];
    long long out = ctx->sp[sp].n;
    for (long long m = (long long)std::floor(a / lt); m <= (long long)std::floor(b / lt); ++m) {
      const double am = a - (double)m * lt, bm = b - (double)m * lt;
      const long long k0 = std::lower_bound(xs.begin(), xs.end(), am) - xs.begin();
      const long long k1 = std::lower_bound(xs.begin(), xs.end(), bm) - xs.begin();
      if (k1 <= k0 || P->nruns >= kMaxInjectRuns) continue;
      InjectRun& R = P->run[P->nruns];
      R.s = sp;
      R.k0 = k0;
      R.k1 = k1;
      R.out = out;
      R.shift = ((double)m * lt + ctx->x0) - ctx->v_up * (double)(s + 1);
      P->first[P->nruns] = total;
      total += k1 - k0;
      out += k1 - k0;
      ++P->nruns;
    }
    add[sp] = out - ctx->sp[sp].n;
  }
  P->first[P->nruns] = total;
  const int D = ctx->grid.dim;
  long long o = 0;
  for (int sp = 0; sp < ctx->ns; ++sp) {
    const int* tc = (const int*)ctx->d_tmpl + o;
    P->tcell[sp] = tc;
    P->toff[sp] = (const float*)(tc + ctx->tn[sp]);
    P->tu[sp] = (const float*)(tc + ctx->tn[sp]) + (long long)D * ctx->tn[sp];
    P->tn[sp] = ctx->tn[sp];
    P->cell[sp] = ctx->sp[sp].cell;
    P->off[sp] = ctx->sp[sp].off;
    P->u[sp] = ctx->sp[sp].u;
    P->ld[sp] = ctx->cap[sp];
    o += ctx->tn[sp] * (1 + D + 3);
  }
}

// Longest sort cycle (steps) captured into one graph.
constexpr int kMaxCycle = 240;

bool step_graph_current(const pic_ctx* ctx) {
  return ctx->step_exec && std::memcmp(&ctx->tun, &ctx->step_tun, sizeof(pic_tuning)) == 0 &&
         ctx->steps % ctx->tun.sort_every == ctx->step_phase &&
         ctx->pusher * 16 + ctx->g.order == ctx->step_solver;
}

// Capture one sort cycle of pic_step into the context's step graph (on a
// private stream; nothing runs during the capture).
pic_status step_capture(pic_ctx* ctx) {
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  ctx->step_exec = nullptr;
  ctx->step_graph = nullptr;
  // buffers that pic_step would allocate on first use: no allocation may
  // happen during a capture
  if (ctx->tun.filter_passes > 0 && !ctx->d_jtmp)
    PIC_CK(ctx, dalloc(&ctx->d_jtmp, 3 * (size_t)ctx->g.plane));
  if (!ctx->cap_st) PIC_CK(ctx, cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking));
  // work already queued on the context's stream is ordered before the graph
  // launches on that stream; the capture itself runs nothing
  const cudaStream_t saved_st = ctx->st;
  const long long saved_steps = ctx->steps;
  PIC_CK(ctx, cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeThreadLocal));
  ctx->st = ctx->cap_st;
  ctx->capturing = true;
  const pic_status st = pic_step(ctx, ctx->tun.sort_every);
  ctx->capturing = false;
  ctx->st = saved_st;
  ctx->steps = saved_steps;  // the captured steps have not run yet
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->cap_st, &graph);
  if (st != PIC_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return st != PIC_OK ? st : cuda_fail(ctx, "step graph capture", e);
  }
  const cudaError_t ei = cudaGraphInstantiate(&ctx->step_exec, graph, 0);
  if (ei != cudaSuccess) {
    cudaGraphDestroy(graph);
    ctx->step_exec = nullptr;
    return cuda_fail(ctx, "step graph instantiation", ei);
  }
  ctx->step_graph = graph;
  ctx->step_tun = ctx->tun;
  ctx->step_phase = ctx->steps % ctx->tun.sort_every;
  ctx->step_solver = ctx->pusher * 16 + ctx->g.order;
  return PIC_OK;
}

pic_status do_filter(pic_ctx* ctx, int passes) {
  if (passes <= 0) return PIC_OK;
  float* J = ctx->F + JX * ctx->g.plane;
  if (!ctx->d_jtmp) PIC_CK(ctx, dalloc(&ctx->d_jtmp, 3 * (size_t)ctx->g.plane));
  float* a = J;
  float* b = ctx->d_jtmp;
  for (int p = 0; p < passes; ++p) {
    const cudaError_t e = timed(
        ctx, PIC_KERNEL_FILTER, [&]() { return launch_filter_pass_f32(ctx->g, a, b, 3, ctx->st, ctx->d_status); });
    if (e != cudaSuccess) return cuda_fail(ctx, "binomial filter", e);
    float* t = a;
    a = b;
    b = t;
  }
  if (a != J)
    PIC_CK(ctx, cudaMemcpyAsync(J, a, sizeof(float) * 3 * ctx->g.plane, cudaMemcpyDeviceToDevice,
                                ctx->st));
  return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_init(pic_ctx** out, const pic_grid* grid, const pic_species* species, int nspecies,
                    float c, float dt, float* fields, void* stream) {
  g_init_error.clear();
  if (!out) return set_err(nullptr, PIC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !species || !fields) return set_err(nullptr, PIC_ERR_ARG, "grid, species or fields is NULL");
  if (grid->dim < 1 || grid->dim > 3) return set_err(nullptr, PIC_ERR_ARG, "dim must be 1, 2 or 3");
  long long ncell = 1;
  for (int d = 0; d < 3; ++d) {
    const int n = extent(*grid, d);
    if (n < 1) return set_err(nullptr, PIC_ERR_ARG, "grid extents must be >= 1");
    if (d >= grid->dim && n != 1)
      return set_err(nullptr, PIC_ERR_ARG, "extents of non-gridded dimensions must be 1");
    ncell *= n;
  }
  if (ncell > 0x7fffffffLL) return set_err(nullptr, PIC_ERR_ARG, "nx*ny*nz must fit in int32");
  if (grid->ny > 65535 || grid->nz > 21845)
    return set_err(nullptr, PIC_ERR_ARG, "ny must be <= 65535 and nz <= 21845");
  if (nspecies < 1 || nspecies > PIC_MAX_SPECIES)
    return set_err(nullptr, PIC_ERR_ARG, "nspecies must be in 1..4");
  if (!(c > 0.f && c < 1.f)) return set_err(nullptr, PIC_ERR_ARG, "Courant number must be in (0, 1)");
  if (dt != 1.0f) return set_err(nullptr, PIC_ERR_ARG, "dt must be 1 (code units)");
  long long ntot = 0, nmax = 0;
  for (int s = 0; s < nspecies; ++s) {
    const pic_species& S = species[s];
    if (S.n < 0 || S.n > 0x7fffffffLL)
      return set_err(nullptr, PIC_ERR_ARG, "species n must be in [0, 2^31)");
    if (S.cap != 0 && (S.cap < S.n || S.cap > 0x7fffffffLL))
      return set_err(nullptr, PIC_ERR_ARG, "species cap must be 0 or in [n, 2^31)");
    if (S.n > 0 && (!S.cell || !S.off || !S.u))
      return set_err(nullptr, PIC_ERR_ARG, "species buffers are NULL");
    if (!(S.m > 0.f) || !std::isfinite(S.m) || !std::isfinite(S.q))
      return set_err(nullptr, PIC_ERR_ARG, "species mass must be > 0 and charge finite");
    ntot += S.n;
    nmax = S.n > nmax ? S.n : nmax;
  }

  pic_ctx* ctx = new pic_ctx();
  ctx->grid = *grid;
  ctx->ns = nspecies;
  long long totcap = 0;
  for (int s = 0; s < nspecies; ++s) {
    ctx->sp[s] = species[s];
    ctx->cap[s] = species[s].cap ? species[s].cap : species[s].n;
    ctx->sp[s].cap = ctx->cap[s];
    totcap += ctx->cap[s];
  }
  ctx->c = c;
  ctx->F = fields;
  ctx->st = (cudaStream_t)stream;
  ctx->ntot = ntot;
  ctx->nmax = nmax;
  ctx->g.dim = grid->dim;
  ctx->g.n[0] = grid->nx;
  ctx->g.n[1] = grid->ny;
  ctx->g.n[2] = grid->nz;
  ctx->g.plane = ncell;
  ctx->g.c = c;
  ctx->g.order = 2;
  // defaults: tiles of 64 cells in 1D, 16^2 in 2D, 8x8x4 in 3D; sort every 10 steps
  // (3 in 3D, where a 2-cell halo is all the shared memory affords)
  ctx->tun.tile[0] = grid->dim == 1 ? 64 : grid->dim == 2 ? 16 : 8;
  ctx->tun.tile[1] = grid->dim == 2 ? 16 : 8;
  ctx->tun.tile[2] = 4;
  ctx->tun.halo = grid->dim == 3 ? 2 : 3;
  ctx->tun.sort_every = grid->dim == 3 ? 3 : 10;
  ctx->tun.filter_passes = 0;
  ctx->tun.chunk = 4096;
  const std::string msg =
      derive_tiles(ctx->grid, ctx->tun, ntot, &ctx->tile, &ctx->splits, &ctx->splits_ens);
  if (!msg.empty()) {
    delete ctx;
    return set_err(nullptr, PIC_ERR_ARG, msg);
  }
  pic_status s = PIC_OK;
  cudaError_t e = cudaSuccess;
  if ((e = set_particle_smem_limit(200 * 1024)) != cudaSuccess) {
    s = cuda_fail(nullptr, "cudaFuncSetAttribute", e);
  } else if ((e = dalloc(&ctx->d_status, 1)) != cudaSuccess ||
             (e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->st)) != cudaSuccess ||
             (e = dalloc(&ctx->d_strays, 1)) != cudaSuccess ||
             (e = cudaMemsetAsync(ctx->d_strays, 0, sizeof(unsigned long long), ctx->st)) !=
                 cudaSuccess) {
    s = cuda_fail(nullptr, "status word", e);
  } else if ((e = dalloc((char**)&ctx->d_sortbuf, (size_t)totcap * (4 + 4 * grid->dim + 12))) !=
             cudaSuccess) {
    s = cuda_fail(nullptr, "sort buffer", e);
  } else if ((e = dalloc(&ctx->d_dlist, (size_t)totcap)) != cudaSuccess ||
             (e = dalloc(&ctx->d_dcount, (size_t)PIC_MAX_SPECIES)) != cudaSuccess) {
    s = cuda_fail(nullptr, "deferred-particle lists", e);
  } else if ((s = alloc_tiles(ctx)) != PIC_OK || (s = do_sort(ctx, true)) != PIC_OK) {
    g_init_error = ctx->err;
  }
  if (s != PIC_OK) {
    cudaStreamSynchronize(ctx->st);
    free_all(ctx);
    delete ctx;
    return s;
  }
  *out = ctx;
  return PIC_OK;
}

pic_status pic_get_tuning(pic_ctx* ctx, pic_tuning* out) {
  if (!ctx || !out) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  *out = ctx->tun;
  return PIC_OK;
}

pic_status pic_set_tuning(pic_ctx* ctx, const pic_tuning* t) {
  if (!ctx || !t) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  pic_tuning nt = ctx->tun;
  for (int d = 0; d < 3; ++d)
    if (t->tile[d]) nt.tile[d] = t->tile[d];
  if (t->halo) nt.halo = t->halo;
  if (t->sort_every) nt.sort_every = t->sort_every;
  if (t->filter_passes) nt.filter_passes = t->filter_passes;
  if (t->chunk) nt.chunk = t->chunk;
  if (nt.sort_every < 1) return set_err(ctx, PIC_ERR_ARG, "sort_every must be >= 1");
  if (nt.filter_passes < 0) return set_err(ctx, PIC_ERR_ARG, "filter_passes must be >= 0");
  TileDev td{};
  int splits = 1, splits_ens = 1;
  const std::string msg = derive_tiles(ctx->grid, nt, ctx->ntot, &td, &splits, &splits_ens);
  if (!msg.empty()) return set_err(ctx, PIC_ERR_ARG, msg);
  const bool retile = std::memcmp(&td, &ctx->tile, sizeof(TileDev)) != 0;
  ctx->tun = nt;
  ctx->splits = splits;
  ctx->splits_ens = splits_ens;
  if (retile) {
    PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
    ctx->tile = td;
    pic_status s = alloc_tiles(ctx);
    if (s != PIC_OK) return s;
    return do_sort(ctx, true);
  }
  return PIC_OK;
}

pic_status pic_set_field_solver(pic_ctx* ctx, int order) {
  if (!ctx) return PIC_ERR_ARG;
  if (order != PIC_FDTD2 && order != PIC_FDTD4)
    return set_err(ctx, PIC_ERR_ARG, "order must be PIC_FDTD2 or PIC_FDTD4");
  // FDTD4 is stable for c sqrt(D) (9/8 + 1/24) <= 1
  if (order == PIC_FDTD4 && ctx->c * std::sqrt((double)ctx->grid.dim) * (7.0 / 6.0) >= 1.0)
    return set_err(ctx, PIC_ERR_ARG, "Courant number too large for FDTD4 in this dimension");
  ctx->g.order = order;
  return PIC_OK;
}

pic_status pic_set_pusher(pic_ctx* ctx, int pusher) {
  if (!ctx) return PIC_ERR_ARG;
  if (pusher != PIC_PUSHER_BORIS && pusher != PIC_PUSHER_HIGUERA_CARY)
    return set_err(ctx, PIC_ERR_ARG, "pusher must be PIC_PUSHER_BORIS or PIC_PUSHER_HIGUERA_CARY");
  ctx->pusher = pusher;
  return PIC_OK;
}

pic_status pic_set_host_chunk(pic_ctx* ctx, int64_t particles) {
  if (!ctx) return PIC_ERR_ARG;
  if (particles < 1 || particles > (1LL << 30))
    return set_err(ctx, PIC_ERR_ARG, "particles per chunk must be in [1, 2^30]");
  ctx->host_chunk = particles;
  return PIC_OK;
}

pic_status pic_set_shock(pic_ctx* ctx, const pic_shock* sh) {
  if (!ctx) return PIC_ERR_ARG;
  if (!sh) return set_err(ctx, PIC_ERR_ARG, "shock is NULL");
  const int nx = ctx->grid.nx, D = ctx->grid.dim;
  const double vals[4] = {sh->x0, sh->x_max, sh->v_inj, sh->v_up};
  for (double v : vals)
    if (!std::isfinite(v)) return set_err(ctx, PIC_ERR_ARG, "shock parameters must be finite");
  if (sh->wall < 1) return set_err(ctx, PIC_ERR_ARG, "wall must be >= 1");
  if (sh->lt < 1) return set_err(ctx, PIC_ERR_ARG, "lt must be >= 1");
  if (!(sh->x_max <= nx - 3)) return set_err(ctx, PIC_ERR_ARG, "x_max must be <= nx - 3");
  if (!(sh->x0 <= sh->x_max)) return set_err(ctx, PIC_ERR_ARG, "x0 must be <= x_max");
  if (!(sh->v_inj >= 0.0 && sh->v_up >= 0.0))
    return set_err(ctx, PIC_ERR_ARG, "v_inj and v_up must be >= 0");
  if (!(sh->v_inj + sh->v_up < sh->lt))
    return set_err(ctx, PIC_ERR_ARG, "v_inj + v_up must be < lt");
  if (!(sh->x0 - sh->v_up >= sh->wall + 1))
    return set_err(ctx, PIC_ERR_ARG, "x0 - v_up must be >= wall + 1");
  const int i_zero = (int)std::floor(sh->x_max) + 2;
  if (2 * sh->wall >= i_zero) return set_err(ctx, PIC_ERR_ARG, "2 wall must be < floor(x_max) + 2");
  const long long block = (long long)sh->lt * ctx->grid.ny * ctx->grid.nz;
  long long words = 0;
  std::vector<double> xs[PIC_MAX_SPECIES];
  for (int s = 0; s < ctx->ns; ++s) {
    const long long nt = sh->nt[s];
    if (nt < 0 || nt > 0x7fffffffLL) return set_err(ctx, PIC_ERR_ARG, "template nt must be in [0, 2^31)");
    const pic_host_species& T = sh->tmpl[s];
    if (nt > 0 && (!T.cell || !T.off || !T.u))
      return set_err(ctx, PIC_ERR_ARG, "template buffers are NULL");
    xs[s].resize((size_t)nt);
    for (long long k = 0; k < nt; ++k) {
      const int c = T.cell[k];
      if (c < 0 || c >= block) return set_err(ctx, PIC_ERR_ARG, "template cell outside lt x ny x nz");
      for (int d = 0; d < D; ++d)
        if (!(T.off[d * nt + k] >= 0.0f && T.off[d * nt + k] < 1.0f))
          return set_err(ctx, PIC_ERR_ARG, "template offset outside [0,1)");
      for (int a = 0; a < 3; ++a)
        if (!std::isfinite(T.u[a * nt + k]))
          return set_err(ctx, PIC_ERR_ARG, "template four-velocity not finite");
      xs[s][k] = (double)(c % sh->lt) + (double)T.off[k];
      if (k > 0 && xs[s][k] < xs[s][k - 1])
        return set_err(ctx, PIC_ERR_ARG, "template not sorted by x");
    }
    words += nt * (1 + D + 3);
  }
  // copy the templates (cell, off rows, u rows per species) to the device
  PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
  dfree(ctx->d_tmpl);
  PIC_CK(ctx, dalloc((char**)&ctx->d_tmpl, (size_t)words * 4));
  long long o = 0;
  for (int s = 0; s < ctx->ns; ++s) {
    const long long nt = sh->nt[s];
    int* tc = (int*)ctx->d_tmpl + o;
    if (nt > 0) {
      PIC_CK(ctx, cudaMemcpy(tc, sh->tmpl[s].cell, 4 * nt, cudaMemcpyHostToDevice));
      PIC_CK(ctx, cudaMemcpy(tc + nt, sh->tmpl[s].off, 4 * D * nt, cudaMemcpyHostToDevice));
      PIC_CK(ctx, cudaMemcpy(tc + nt + D * nt, sh->tmpl[s].u, 12 * nt, cudaMemcpyHostToDevice));
    }
    ctx->tn[s] = nt;
    ctx->txs[s].swap(xs[s]);
    o += nt * (1 + D + 3);
  }
  ctx->shock = true;
  ctx->wall = sh->wall;
  ctx->i_zero = i_zero;
  ctx->lt = sh->lt;
  ctx->x0 = sh->x0;
  ctx->x_max = sh->x_max;
  ctx->v_inj = sh->v_inj;
  ctx->v_up = sh->v_up;
  ctx->shock_steps = 0;
  // the fields entering the first step satisfy the wall's boundary
  PIC_CK(ctx, launch_wall_fields(ctx->g, ctx->F, ctx->wall, ctx->i_zero, ctx->st));
  return PIC_OK;
}

pic_status pic_adjoint_step(pic_ctx* ctx, const float* fwd_fields, const pic_adjoint_species* sp,
                            float* adj_fields) {
  if (!ctx) return PIC_ERR_ARG;
  if (!fwd_fields || !sp || !adj_fields) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  if (ctx->g.order != 2 || ctx->pusher != PIC_PUSHER_BORIS || ctx->shock)
    return set_err(ctx, PIC_ERR_STATE, "the adjoint covers FDTD2, Boris and periodic boxes");
  const int D = ctx->grid.dim;
  for (int s = 0; s < ctx->ns; ++s)
    if (ctx->sp[s].n > 0 && (!sp[s].cell || !sp[s].off || !sp[s].u || !sp[s].xbar || !sp[s].ubar))
      return set_err(ctx, PIC_ERR_ARG, "adjoint species buffers are NULL");
  const long long P = ctx->g.plane;
  if (!ctx->d_adjF) PIC_CK(ctx, dalloc(&ctx->d_adjF, 9 * (size_t)P));
  if (!ctx->d_jtmp) PIC_CK(ctx, dalloc(&ctx->d_jtmp, 3 * (size_t)P));
  AdjParams AP{};
  AP.g = ctx->g;
  AP.t = ctx->tile;
  AP.splits = ctx->splits;
  AP.F1 = ctx->d_adjF;
  AP.A = adj_fields;
  AP.div0 = make_fastdiv(ctx->g.n[0]);
  AP.div1 = make_fastdiv(ctx->g.n[1]);
  AP.nspecies = ctx->ns;
  AP.dcount = ctx->d_dcount;
  // the tile grouping: the caller's bucket starts, copied and checked (a tile
  // block must never read a slot outside [0, n); see pic_sort_assume)
  bool tiled = true;
  for (int s = 0; s < ctx->ns; ++s) tiled &= ctx->sp[s].n == 0 || sp[s].tstart != nullptr;
  const long long nb = sort_bins(ctx->tile);
  if (tiled) {
    const size_t need = (size_t)ctx->ns * (size_t)(nb + 1);
    if (ctx->adj_tstart_len < need) {
      dfree(ctx->d_adj_tstart);
      ctx->adj_tstart_len = 0;
      PIC_CK(ctx, dalloc(&ctx->d_adj_tstart, need));
      ctx->adj_tstart_len = need;
    }
  }
  long long o = 0;
  for (int s = 0; s < ctx->ns; ++s) {
    AdjSpecies& S = AP.sp[s];
    S.tstart = nullptr;
    if (tiled && ctx->sp[s].n > 0) {
      int* t = ctx->d_adj_tstart + (long long)s * (nb + 1);
      PIC_CK(ctx, cudaMemcpyAsync(t, sp[s].tstart, sizeof(int) * (nb + 1),
                                  cudaMemcpyDeviceToDevice, ctx->st));
      PIC_CK(ctx, launch_check_buckets(t, nb, ctx->sp[s].n, ctx->d_status, ctx->st));
      S.tstart = t;
    }
    S.dlist = ctx->d_dlist + o;
    o += ctx->cap[s];
    S.q = ctx->sp[s].q;
    S.qm = ctx->sp[s].q / ctx->sp[s].m;
    S.n = ctx->sp[s].n;
    S.ld = ctx->cap[s];
    S.cell = sp[s].cell;
    S.off = sp[s].off;
    S.u = sp[s].u;
    S.xbar = sp[s].xbar;
    S.ubar = sp[s].ubar;
  }
  (void)D;
  const cudaError_t e = timed(ctx, PIC_KERNEL_ADJOINT, [&]() -> cudaError_t {
    // forward fields seen by the particles: E and B1 = B - (c/2) curl+ E
    cudaError_t r = cudaMemcpyAsync(ctx->d_adjF, fwd_fields, sizeof(float) * 6 * P,
                                    cudaMemcpyDeviceToDevice, ctx->st);
    if (r == cudaSuccess) r = launch_b_half(ctx->g, ctx->d_adjF, 0, ctx->st);
    if (r == cudaSuccess) r = launch_adj_e(ctx->g, adj_fields, ctx->st);  // E' = E + c curl- B2 - Jf
    float* J = adj_fields + JX * P;
    float* a = J;
    float* b = ctx->d_jtmp;
    for (int p = 0; p < ctx->tun.filter_passes && r == cudaSuccess; ++p) {  // Jf = F^p J
      r = launch_filter_pass_f32(ctx->g, a, b, 3, ctx->st, ctx->d_status);
      float* t = a;
      a = b;
      b = t;
    }
    if (r == cudaSuccess && a != J)
      r = cudaMemcpyAsync(J, a, sizeof(float) * 3 * P, cudaMemcpyDeviceToDevice, ctx->st);
    if (r == cudaSuccess) r = launch_adj_b_half(ctx->g, adj_fields, ctx->st);  // B2 = B1 - ...
    if (r == cudaSuccess) r = launch_adj_particles(AP, ctx->st);             // particles
    if (r == cudaSuccess) r = launch_adj_b_half(ctx->g, adj_fields, ctx->st);  // B1 = B - ...
    if (r == cudaSuccess) r = cudaMemsetAsync(J, 0, sizeof(float) * 3 * P, ctx->st);
    return r;
  });
  if (e != cudaSuccess) return cuda_fail(ctx, "adjoint step", e);
  return PIC_OK;
}

pic_status pic_particle_counts(pic_ctx* ctx, int64_t* n, int nout) {
  if (!ctx || !n) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  if (nout < ctx->ns) return set_err(ctx, PIC_ERR_ARG, "nout must be >= nspecies");
  for (int s = 0; s < ctx->ns; ++s) n[s] = ctx->sp[s].n;
  return PIC_OK;
}

pic_status pic_sort(pic_ctx* ctx) {
  if (!ctx) return PIC_ERR_ARG;
  return do_sort(ctx, true);
}

pic_status pic_sort_bins(pic_ctx* ctx, int64_t* nbins) {
  if (!ctx || !nbins) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  *nbins = sort_bins(ctx->tile);
  return PIC_OK;
}

pic_status pic_sort_record(pic_ctx* ctx, int32_t* const* perm, int32_t* const* tstart) {
  if (!ctx || !perm || !tstart) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  for (int s = 0; s < ctx->ns; ++s)
    if (ctx->sp[s].n > 0 && (!perm[s] || !tstart[s]))
      return set_err(ctx, PIC_ERR_ARG, "perm or tstart of a species with particles is NULL");
  const pic_status st = do_sort(ctx, true, perm);
  if (st != PIC_OK) return st;
  const long long nb = sort_bins(ctx->tile) + 1;
  for (int s = 0; s < ctx->ns; ++s)
    if (tstart[s])
      PIC_CK(ctx, cudaMemcpyAsync(tstart[s], ctx->d_tstart[s], sizeof(int) * nb,
                                  cudaMemcpyDeviceToDevice, ctx->st));
  return PIC_OK;
}

pic_status pic_sort_assume(pic_ctx* ctx, const int32_t* const* tstart) {
  if (!ctx || !tstart) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  for (int s = 0; s < ctx->ns; ++s)
    if (ctx->sp[s].n > 0 && !tstart[s])
      return set_err(ctx, PIC_ERR_ARG, "tstart of a species with particles is NULL");
  const long long nb = sort_bins(ctx->tile);
  for (int s = 0; s < ctx->ns; ++s) {
    const long long n = ctx->sp[s].n;
    if (n > 0)
      PIC_CK(ctx, cudaMemcpyAsync(ctx->d_tstart[s], tstart[s], sizeof(int) * (nb + 1),
                                  cudaMemcpyDeviceToDevice, ctx->st));
    else
      PIC_CK(ctx, cudaMemsetAsync(ctx->d_tstart[s], 0, sizeof(int) * (nb + 1), ctx->st));
    // a tile kernel must never read a slot outside [0, n): starts that are
    // not a partition are replaced by one bucket (correct, through the stray
    // path) and reported by pic_check
    PIC_CK(ctx, launch_check_buckets(ctx->d_tstart[s], nb, n, ctx->d_status, ctx->st));
    ctx->sorted_n[s] = n;
  }
  ctx->snapshot_valid = false;
  ctx->sorted_pending = false;
  ctx->sorted_step = ctx->steps;
  return PIC_OK;
}

pic_status pic_adjoint_unsort(pic_ctx* ctx, const int32_t* const* perm,
                              const pic_adjoint_species* sp) {
  if (!ctx || !perm || !sp) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  if (ctx->sorted_pending)
    return set_err(ctx, PIC_ERR_STATE, "a sorted copy of the particles awaits its push");
  const int D = ctx->grid.dim;
  for (int s = 0; s < ctx->ns; ++s) {
    const long long n = ctx->sp[s].n, ld = ctx->cap[s];
    if (n == 0) continue;
    if (!perm[s] || !sp[s].xbar || !sp[s].ubar)
      return set_err(ctx, PIC_ERR_ARG, "perm, xbar or ubar of a species with particles is NULL");
    // through the sort buffer of the species (room for 1 + D + 3 rows of ld)
    float* tmp = (float*)((int*)ctx->d_sortbuf + sortbuf_offset(ctx, s));
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    PIC_CK(ctx, launch_unpermute(perm[s], sp[s].xbar, tmp, n, ld, D, ctx->d_status, ctx->st));
    PIC_CK(ctx, copy_rows(sp[s].xbar, tmp, sizeof(float), n, ld, D, k, ctx->st));
    PIC_CK(ctx, launch_unpermute(perm[s], sp[s].ubar, tmp, n, ld, 3, ctx->d_status, ctx->st));
    PIC_CK(ctx, copy_rows(sp[s].ubar, tmp, sizeof(float), n, ld, 3, k, ctx->st));
  }
  return PIC_OK;
}

pic_status pic_gather_push(pic_ctx* ctx) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->shock)
    return set_err(ctx, PIC_ERR_STATE, "the split gather/deposit path does not model the wall");
  if (!ctx->d_cell_old) {
    PIC_CK(ctx, dalloc(&ctx->d_cell_old, (size_t)total_cap(ctx)));
    PIC_CK(ctx, dalloc(&ctx->d_off_old, (size_t)total_cap(ctx) * ctx->grid.dim));
  }
  const PushParams P = make_params(ctx);
  const cudaError_t e = timed(ctx, PIC_KERNEL_PUSH,
                              [&]() { return launch_particles(ctx->grid.dim, 1, P, ctx->st); });
  if (e != cudaSuccess) return cuda_fail(ctx, "gather/push kernel", e);
  ctx->snapshot_valid = true;
  return PIC_OK;
}

pic_status pic_deposit(pic_ctx* ctx) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->shock)
    return set_err(ctx, PIC_ERR_STATE, "the split gather/deposit path does not model the wall");
  if (!ctx->snapshot_valid)
    return set_err(ctx, PIC_ERR_STATE, "pic_deposit needs a preceding pic_gather_push");
  const PushParams P = make_params(ctx);
  const cudaError_t e = timed(ctx, PIC_KERNEL_PUSH,
                              [&]() { return launch_particles(ctx->grid.dim, 2, P, ctx->st); });
  if (e != cudaSuccess) return cuda_fail(ctx, "deposit kernel", e);
  return PIC_OK;
}

pic_status pic_filter_current(pic_ctx* ctx, int passes) {
  if (!ctx) return PIC_ERR_ARG;
  if (passes < 0) return set_err(ctx, PIC_ERR_ARG, "passes must be >= 0");
  return do_filter(ctx, passes);
}

pic_status pic_field_update(pic_ctx* ctx, int which) {
  if (!ctx) return PIC_ERR_ARG;
  cudaError_t e;
  if (which == PIC_FIELD_B_HALF)
    e = timed(ctx, PIC_KERNEL_BHALF, [&]() { return launch_b_half(ctx->g, ctx->F, 0, ctx->st); });
  else if (which == PIC_FIELD_E)
    e = timed(ctx, PIC_KERNEL_EUPD, [&]() { return launch_e_update(ctx->g, ctx->F, ctx->st); });
  else
    return set_err(ctx, PIC_ERR_ARG, "which must be PIC_FIELD_B_HALF or PIC_FIELD_E");
  if (e != cudaSuccess) return cuda_fail(ctx, "field update", e);
  return PIC_OK;
}

// The conducting wall's field condition after a field update (shock boxes).
cudaError_t wall_fields(pic_ctx* ctx) {
  if (!ctx->shock) return cudaSuccess;
  return timed(ctx, PIC_KERNEL_BOUNDARY, [&]() {
    return launch_wall_fields(ctx->g, ctx->F, ctx->wall, ctx->i_zero, ctx->st);
  });
}

// Inside one pic_step call on a small periodic lattice, the single-block
// field launch of a step also runs the next step's first B half step.
#ifndef PIC_SMALL_CHAIN
#define PIC_SMALL_CHAIN 1
#endif

// The field half of a step, after the particles deposited J: the filter
// passes, the second B half step and the E update; with `chain` (small
// periodic lattices only) the next step's first B half step too.
pic_status step_fields(pic_ctx* ctx, bool chain = false) {
  cudaError_t e;
  if (!ctx->shock && fields_small_ok(ctx->g)) {
    // small periodic lattice: the filter (on J) first, then the second B
    // half step and the E update in one launch (the B half step touches B
    // only, the filter J only: the order between them does not matter)
    const pic_status s = do_filter(ctx, ctx->tun.filter_passes);
    if (s != PIC_OK) return s;
    e = timed(ctx, PIC_KERNEL_EUPD,
              [&]() { return launch_fields_small(ctx->g, ctx->F, ctx->st, chain ? 1 : 0); });
    if (e != cudaSuccess) return cuda_fail(ctx, "B half step and E update", e);
  } else {
    e = timed(ctx, PIC_KERNEL_BHALF, [&]() { return launch_b_half(ctx->g, ctx->F, 0, ctx->st); });
    if (e == cudaSuccess) e = wall_fields(ctx);
    if (e != cudaSuccess) return cuda_fail(ctx, "B half step", e);
    const pic_status s = do_filter(ctx, ctx->tun.filter_passes);
    if (s != PIC_OK) return s;
    e = timed(ctx, PIC_KERNEL_EUPD, [&]() { return launch_e_update(ctx->g, ctx->F, ctx->st); });
    if (e == cudaSuccess) e = wall_fields(ctx);
    if (e != cudaSuccess) return cuda_fail(ctx, "E update", e);
  }
  return PIC_OK;
}

pic_status pic_step(pic_ctx* ctx, int nsteps) {
  if (!ctx) return PIC_ERR_ARG;
  if (nsteps < 0) return set_err(ctx, PIC_ERR_ARG, "nsteps must be >= 0");
  // whole sort cycles from the context's step graph: the same kernels with the
  // same arguments as the loop below, launched as one graph per cycle
  const int cyc = ctx->tun.sort_every;
  if (PIC_STEP_GRAPHS && !ctx->shock && !ctx->timing && !ctx->capturing && cyc <= kMaxCycle &&
      nsteps >= 2 * cyc) {
    if (!step_graph_current(ctx)) {
      const pic_status s = step_capture(ctx);
      if (s != PIC_OK) return s;
    }
    const int full = nsteps / cyc;
    for (int i = 0; i < full; ++i) {
      const cudaError_t e = cudaGraphLaunch(ctx->step_exec, ctx->st);
      if (e != cudaSuccess) return cuda_fail(ctx, "step graph launch", e);
    }
    ctx->steps += (long long)full * cyc;
    ctx->snapshot_valid = false;
    nsteps -= full * cyc;
  }
  const auto wall_bc = [&]() { return wall_fields(ctx); };
  bool b1_done = false;  // this step's first B half step ran with the last field launch
  for (int it = 0; it < nsteps; ++it) {
    InjectParams IP{};
    long long add[PIC_MAX_SPECIES] = {};
    if (ctx->shock) {  // plan this step's injection first: refuse it whole if it does not fit
      plan_injection(ctx, ctx->shock_steps, &IP, add);
      for (int s = 0; s < ctx->ns; ++s)
        if (ctx->sp[s].n + add[s] > ctx->cap[s])
          return set_err(ctx, PIC_ERR_ARG, "injection would exceed a species' cap");
    }
    // a sort opens every cycle of sort_every steps, unless the particles were
    // sorted at this very step count already (at set-up, by pic_sort or a
    // re-tiling); a captured cycle always sorts, since it is replayed later
    if (ctx->steps % ctx->tun.sort_every == 0 &&
        (ctx->capturing || ctx->sorted_step != ctx->steps)) {
      const pic_status s = do_sort(ctx, false);
      if (s != PIC_OK) return s;
    }
    const PushParams P = make_params(ctx);
    ctx->sorted_pending = false;
    cudaError_t e = cudaSuccess;
    if (!b1_done) {
      e = timed(ctx, PIC_KERNEL_BHALF, [&]() { return launch_b_half(ctx->g, ctx->F, 1, ctx->st); });
      if (e == cudaSuccess) e = wall_bc();
      if (e != cudaSuccess) return cuda_fail(ctx, "B half step", e);
    }
    e = timed(ctx, PIC_KERNEL_PUSH, [&]() { return launch_particles(ctx->grid.dim, 0, P, ctx->st); });
    if (e != cudaSuccess) return cuda_fail(ctx, "gather/push/deposit kernel", e);
    // small periodic lattice, not the call's last step: the field launch also
    // takes the next step's first B half step
    b1_done = PIC_SMALL_CHAIN && it + 1 < nsteps && !ctx->shock && fields_small_ok(ctx->g);
    {
      const pic_status s = step_fields(ctx, b1_done);
      if (s != PIC_OK) return s;
    }
    if (ctx->shock) {
      if (IP.nruns > 0) {
        e = timed(ctx, PIC_KERNEL_BOUNDARY, [&]() { return launch_inject(IP, ctx->st); });
        if (e != cudaSuccess) return cuda_fail(ctx, "injection", e);
      }
      for (int s2 = 0; s2 < ctx->ns; ++s2) ctx->sp[s2].n += add[s2];
      ++ctx->shock_steps;
    }
    ++ctx->steps;
  }
  ctx->snapshot_valid = false;
  return PIC_OK;
}

pic_status pic_energies(pic_ctx* ctx, double* out, int nout) {
  if (!ctx || !out) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  const int ns = ctx->ns;
  if (nout < 4 + ns) return set_err(ctx, PIC_ERR_ARG, "nout must be >= 4 + nspecies");
  const long long P = ctx->g.plane;
  if (!ctx->d_acc) {
    PIC_CK(ctx, dalloc(&ctx->d_acc, 4 + PIC_MAX_SPECIES));
    PIC_CK(ctx, dalloc(&ctx->d_rho, (size_t)P));
    PIC_CK(ctx, dalloc(&ctx->d_rho2, (size_t)P));
  }
  PIC_CK(ctx, cudaMemsetAsync(ctx->d_acc, 0, sizeof(double) * (4 + PIC_MAX_SPECIES), ctx->st));
  PIC_CK(ctx, cudaMemsetAsync(ctx->d_rho, 0, sizeof(double) * P, ctx->st));
  PIC_CK(ctx, launch_field_energy(ctx->g, ctx->F, ctx->d_acc, ctx->st));
  const double c2 = (double)ctx->c * (double)ctx->c;
  for (int s = 0; s < ns; ++s) {
    PIC_CK(ctx, launch_kinetic(ctx->sp[s].u, ctx->sp[s].n, ctx->cap[s], (double)ctx->sp[s].m * c2,
                               ctx->d_acc + 2 + s, ctx->st));
    PIC_CK(ctx, launch_rho(ctx->g, ctx->sp[s].cell, ctx->sp[s].off, ctx->sp[s].n, ctx->cap[s],
                           (double)ctx->sp[s].q, ctx->d_rho, ctx->st));
  }
  double* a = ctx->d_rho;
  double* b = ctx->d_rho2;
  for (int p = 0; p < ctx->tun.filter_passes; ++p) {
    for (int axis = 0; axis < ctx->grid.dim; ++axis) {
      PIC_CK(ctx, launch_filter_f64(ctx->g, a, b, 1, axis, ctx->st));
      double* t = a;
      a = b;
      b = t;
    }
  }
  // with the wall, the residual covers the plasma side: wall < i < i_zero
  const int i_lo = ctx->shock ? ctx->wall + 1 : 0;
  const int i_hi = ctx->shock ? ctx->i_zero : ctx->grid.nx;
  PIC_CK(ctx, launch_gauss(ctx->g, ctx->F, a, i_lo, i_hi,
                           (unsigned long long*)(ctx->d_acc + 2 + ns), ctx->d_acc + 3 + ns, ctx->st));
  double h[4 + PIC_MAX_SPECIES];
  PIC_CK(ctx, cudaMemcpyAsync(h, ctx->d_acc, sizeof(double) * (4 + ns), cudaMemcpyDeviceToHost, ctx->st));
  PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
  for (int i = 0; i < 3 + ns; ++i) out[i] = h[i];
  out[3 + ns] = std::sqrt(h[3 + ns] / ((double)(i_hi - i_lo) * (double)(P / ctx->grid.nx)));
  return PIC_OK;
}

pic_status pic_check(pic_ctx* ctx) {
  if (!ctx) return PIC_ERR_ARG;
  int h = 0;
  PIC_CK(ctx, cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
  if (h == 0) return PIC_OK;
  PIC_CK(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->st));
  PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
  std::string m = "invalid particle data:";
  if (h & ST_BAD_CELL) m += " cell index out of range;";
  if (h & ST_BAD_OFF) m += " offset outside [0,1);";
  if (h & ST_BAD_U) m += " non-finite four-velocity;";
  if (h & ST_BEHIND_WALL) m += " particle behind the conducting wall;";
  if (h & ST_BAD_BUCKETS)
    m += " bucket starts or a permutation handed in were not valid (starts replaced by one"
         " bucket, permutation entries outside [0, n) skipped);";
  // a bounded wait on a shared-memory copy gave up: the results of that step
  // are not to be trusted, the context stays usable
  if (h & ST_TIMEOUT)
    return set_err(ctx, PIC_ERR_TIMEOUT, "a bounded device-side wait on a tensor copy gave up");
  return set_err(ctx, PIC_ERR_STATE, m);
}

pic_status pic_wait_probe(pic_ctx* ctx) {
  if (!ctx) return PIC_ERR_ARG;
  PIC_CK(ctx, launch_wait_probe(ctx->d_status, ctx->st));
  return PIC_OK;
}

// pic_step_host overlaps its copies in and out (chunk by chunk) with each
// other and with the last step.
#ifndef PIC_HOST_OVERLAP
#define PIC_HOST_OVERLAP 1
#endif
// Copy the slots [lo, hi) of `rows` rows of ld elements of `elem` bytes.
cudaError_t copy_slots(void* dst, const void* src, size_t elem, long long lo, long long hi,
                       long long ld, int rows, cudaMemcpyKind kind, cudaStream_t st) {
  if (hi <= lo || rows == 0) return cudaSuccess;
  char* d = static_cast<char*>(dst) + elem * (size_t)lo;
  const char* s = static_cast<const char*>(src) + elem * (size_t)lo;
  if (rows == 1) return cudaMemcpyAsync(d, s, elem * (size_t)(hi - lo), kind, st);
  return cudaMemcpy2DAsync(d, elem * (size_t)ld, s, elem * (size_t)ld, elem * (size_t)(hi - lo),
                           (size_t)rows, kind, st);
}

// pic_step_host with its copies overlapped.  Each species is cut into chunks
// of slots (host_chunk particles each, at most kHostChunks; one chunk for a
// species with an unsorted tail, which the last launch processes).  The copies
// in run on one stream, the fields first and then chunk after chunk; the
// copies out on another.  The steps before the last wait for every copy in.  The last
// step runs the particle kernel chunk by chunk, each launch over bucket starts
// clipped to the chunk's slots, as soon as the chunk is in, and sends each
// chunk back out as soon as its launch is done while later chunks are still
// coming in: the host link moves data both ways at once faster than one way
// at a time.  A sort due at the last step waits for the whole species.  The
// launches are pic_step's, with the sort split by species and the particle
// kernel by chunk.
pic_status step_host_copies(pic_ctx* ctx, const pic_host_species* hs, float* host_fields,
                            int nsteps);

pic_status step_host_overlapped(pic_ctx* ctx, const pic_host_species* hs, float* host_fields,
                                int nsteps) {
  const pic_status r = step_host_copies(ctx, hs, host_fields, nsteps);
  if (r != PIC_OK) {
    // no copy to or from the caller's host buffers may outlive the call
    for (auto io : ctx->io_st)
      if (io) cudaStreamSynchronize(io);
    cudaStreamSynchronize(ctx->st);
  }
  return r;
}

pic_status step_host_copies(pic_ctx* ctx, const pic_host_species* hs, float* host_fields,
                            int nsteps) {
  const int D = ctx->grid.dim, ns = ctx->ns;
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
  for (auto& io : ctx->io_st)
    if (!io) PIC_CK(ctx, cudaStreamCreateWithFlags(&io, cudaStreamNonBlocking));
  for (auto& ev : ctx->io_ev)
    if (!ev) PIC_CK(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  const long long nb1 = sort_bins(ctx->tile) + 1;
  if (!ctx->d_tclip || ctx->tclip_len < kHostChunks * nb1) {
    dfree(ctx->d_tclip);
    ctx->tclip_len = 0;
    PIC_CK(ctx, dalloc(&ctx->d_tclip, kHostChunks * nb1));
    ctx->tclip_len = kHostChunks * nb1;
  }
  int nk[PIC_MAX_SPECIES];
  for (int s = 0; s < ns; ++s)
    nk[s] = ctx->sp[s].n != ctx->sorted_n[s]
                ? 1
                : (int)std::min<long long>(
                      kHostChunks, std::max<long long>(1, (ctx->sp[s].n + ctx->host_chunk - 1) /
                                                              ctx->host_chunk));
  const auto lo_of = [&](int s, int k) { return ctx->sp[s].n * k / nk[s]; };
  const auto ev_in = [&](int s, int k) { return ctx->io_ev[s * kHostChunks + k]; };
  const auto ev_pushed = [&](int s, int k) {
    return ctx->io_ev[(PIC_MAX_SPECIES + s) * kHostChunks + k];
  };
  const int e0 = 2 * PIC_MAX_SPECIES * kHostChunks;
  const cudaStream_t in = ctx->io_st[0], out = ctx->io_st[1];
  const cudaEvent_t ev_go = ctx->io_ev[e0];        // earlier work queued
  const cudaEvent_t ev_fin = ctx->io_ev[e0 + 1];   // fields are in
  const cudaEvent_t ev_fout = ctx->io_ev[e0 + 2];  // fields are final
  // the copies in overwrite buffers that work queued earlier may still use
  PIC_CK(ctx, cudaEventRecord(ev_go, ctx->st));
  PIC_CK(ctx, cudaStreamWaitEvent(in, ev_go, 0));
  PIC_CK(ctx, cudaMemcpyAsync(ctx->F, host_fields, 36 * ctx->g.plane, h2d, in));
  PIC_CK(ctx, cudaEventRecord(ev_fin, in));
  for (int s = 0; s < ns; ++s)
    for (int k = 0; k < nk[s]; ++k) {
      const long long lo = lo_of(s, k), hi = lo_of(s, k + 1), ld = ctx->cap[s];
      PIC_CK(ctx, copy_slots(ctx->sp[s].cell, hs[s].cell, 4, lo, hi, ld, 1, h2d, in));
      PIC_CK(ctx, copy_slots(ctx->sp[s].off, hs[s].off, 4, lo, hi, ld, D, h2d, in));
      PIC_CK(ctx, copy_slots(ctx->sp[s].u, hs[s].u, 4, lo, hi, ld, 3, h2d, in));
      PIC_CK(ctx, cudaEventRecord(ev_in(s, k), in));
    }
  PIC_CK(ctx, cudaStreamWaitEvent(ctx->st, ev_fin, 0));
  if (nsteps > 1) {
    for (int s = 0; s < ns; ++s) PIC_CK(ctx, cudaStreamWaitEvent(ctx->st, ev_in(s, nk[s] - 1), 0));
    const pic_status r = pic_step(ctx, nsteps - 1);
    if (r != PIC_OK) return r;
  }
  // the last step: the context's bookkeeping of a due sort comes first, so
  // that the particle parameters read every species from the sorted buffer
  const bool sort = ctx->steps % ctx->tun.sort_every == 0 && ctx->sorted_step != ctx->steps;
  if (sort) sort_done(ctx, false);
  const PushParams P = make_params(ctx);
  ctx->sorted_pending = false;
  cudaError_t e = launch_b_half(ctx->g, ctx->F, 1, ctx->st);
  if (e != cudaSuccess) return cuda_fail(ctx, "B half step", e);
  for (int s = 0; s < ns; ++s) {
    if (sort) {  // the count covers the whole species
      PIC_CK(ctx, cudaStreamWaitEvent(ctx->st, ev_in(s, nk[s] - 1), 0));
      if ((e = sort_species(ctx, s, false, nullptr)) != cudaSuccess)
        return cuda_fail(ctx, "tile sort", e);
    }
    for (int k = 0; k < nk[s]; ++k) {
      const long long lo = lo_of(s, k), hi = lo_of(s, k + 1), ld = ctx->cap[s];
      PIC_CK(ctx, cudaStreamWaitEvent(ctx->st, ev_in(s, k), 0));
      PushParams Ps = P;  // chunk k of species s; the current's quantum stays the step's
      Ps.nspecies = 1;
      Ps.sp[0] = P.sp[s];
      Ps.dcount = P.sp[s].dcount;
      if (nk[s] > 1) {
        int* tk = ctx->d_tclip + k * nb1;
        PIC_CK(ctx, launch_clip_starts(P.sp[s].tstart, nb1, (int)lo, (int)hi, tk, ctx->st));
        Ps.sp[0].tstart = tk;
      }
      // the tail kernel runs with the species' last chunk (with its only one
      // when the species has an unsorted tail)
      if (k + 1 < nk[s]) Ps.tail_blocks = 0;
      if ((e = launch_particles(D, 0, Ps, ctx->st)) != cudaSuccess)
        return cuda_fail(ctx, "gather/push/deposit kernel", e);
      PIC_CK(ctx, cudaEventRecord(ev_pushed(s, k), ctx->st));
      PIC_CK(ctx, cudaStreamWaitEvent(out, ev_pushed(s, k), 0));
      PIC_CK(ctx, copy_slots(hs[s].cell, ctx->sp[s].cell, 4, lo, hi, ld, 1, d2h, out));
      PIC_CK(ctx, copy_slots(hs[s].off, ctx->sp[s].off, 4, lo, hi, ld, D, d2h, out));
      PIC_CK(ctx, copy_slots(hs[s].u, ctx->sp[s].u, 4, lo, hi, ld, 3, d2h, out));
    }
  }
  const pic_status r = step_fields(ctx);
  if (r != PIC_OK) return r;
  ++ctx->steps;
  ctx->snapshot_valid = false;
  PIC_CK(ctx, cudaEventRecord(ev_fout, ctx->st));
  PIC_CK(ctx, cudaStreamWaitEvent(out, ev_fout, 0));
  PIC_CK(ctx, cudaMemcpyAsync(host_fields, ctx->F, 36 * ctx->g.plane, d2h, out));
  PIC_CK(ctx, cudaStreamSynchronize(out));
  PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}

pic_status pic_step_host(pic_ctx* ctx, const pic_host_species* hs, float* host_fields, int nsteps) {
  if (!ctx || !hs || !host_fields) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  const int D = ctx->grid.dim;
  for (int s = 0; s < ctx->ns; ++s)
    if (ctx->sp[s].n > 0 && (!hs[s].cell || !hs[s].off || !hs[s].u))
      return set_err(ctx, PIC_ERR_ARG, "host species buffers are NULL");
  // boxes without shock boundaries (whose counts the injector changes),
  // with the event timers off: the overlapped copies
  if (PIC_HOST_OVERLAP && nsteps >= 1 && !ctx->shock && !ctx->timing)
    return step_host_overlapped(ctx, hs, host_fields, nsteps);
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
  for (int s = 0; s < ctx->ns; ++s) {
    const long long n = ctx->sp[s].n, ld = ctx->cap[s];
    if (n == 0) continue;
    PIC_CK(ctx, copy_rows(ctx->sp[s].cell, hs[s].cell, 4, n, ld, 1, h2d, ctx->st));
    PIC_CK(ctx, copy_rows(ctx->sp[s].off, hs[s].off, 4, n, ld, D, h2d, ctx->st));
    PIC_CK(ctx, copy_rows(ctx->sp[s].u, hs[s].u, 4, n, ld, 3, h2d, ctx->st));
  }
  PIC_CK(ctx, cudaMemcpyAsync(ctx->F, host_fields, 36 * ctx->g.plane, h2d, ctx->st));
  const pic_status s = pic_step(ctx, nsteps);
  if (s != PIC_OK) {
    cudaStreamSynchronize(ctx->st);  // the copies in read the caller's host buffers
    return s;
  }
  for (int sp = 0; sp < ctx->ns; ++sp) {
    const long long n = ctx->sp[sp].n, ld = ctx->cap[sp];
    if (n == 0) continue;
    PIC_CK(ctx, copy_rows(hs[sp].cell, ctx->sp[sp].cell, 4, n, ld, 1, d2h, ctx->st));
    PIC_CK(ctx, copy_rows(hs[sp].off, ctx->sp[sp].off, 4, n, ld, D, d2h, ctx->st));
    PIC_CK(ctx, copy_rows(hs[sp].u, ctx->sp[sp].u, 4, n, ld, 3, d2h, ctx->st));
  }
  PIC_CK(ctx, cudaMemcpyAsync(host_fields, ctx->F, 36 * ctx->g.plane, d2h, ctx->st));
  PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
  return PIC_OK;
}

pic_status pic_stats(pic_ctx* ctx, int64_t* strays) {
  if (!ctx || !strays) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  unsigned long long h = 0;
  PIC_CK(ctx, cudaMemcpyAsync(&h, ctx->d_strays, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
  PIC_CK(ctx, cudaMemsetAsync(ctx->d_strays, 0, sizeof(h), ctx->st));
  PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
  *strays = (int64_t)h;
  return PIC_OK;
}

pic_status pic_autotune(pic_ctx* ctx, const pic_tuning* candidates, int ncandidates, int steps,
                        int* best_index) {
  if (!ctx) return PIC_ERR_ARG;
  if (steps < 1) return set_err(ctx, PIC_ERR_ARG, "steps must be >= 1");
  if (candidates && ncandidates < 1) return set_err(ctx, PIC_ERR_ARG, "ncandidates must be >= 1");
  std::vector<pic_tuning> cs;
  if (candidates) {
    cs.assign(candidates, candidates + ncandidates);
  } else {
    // built-in candidates: tile shapes around the default, two halos (3 and 4 in
    // 1D/2D, 2 and 3 in 3D, where the window's shared memory is the limit),
    // cadences
    const int D = ctx->grid.dim;
    const int tiles1[][3] = {{32, 1, 1}, {64, 1, 1}, {128, 1, 1}};
    const int tiles2[][3] = {{16, 16, 1}, {8, 16, 1}, {16, 8, 1}};
    const int tiles3[][3] = {{8, 8, 4}, {8, 8, 8}, {8, 4, 4}};
    const int (*tiles)[3] = D == 1 ? tiles1 : D == 2 ? tiles2 : tiles3;
    const int cad2[] = {5, 10, 20}, cad3[] = {2, 3, 5};
    const int* cad = D == 3 ? cad3 : cad2;
    const int h0 = D == 3 ? 2 : 3;
    for (int t = 0; t < 3; ++t)
      for (int h = h0; h <= h0 + 1; ++h)
        for (int k = 0; k < 3; ++k) {
          pic_tuning c{};
          for (int d = 0; d < 3; ++d) c.tile[d] = tiles[t][d];
          c.halo = h;
          c.sort_every = cad[k];
          cs.push_back(c);
        }
  }
  const pic_tuning orig = ctx->tun;
  cudaEvent_t ea = nullptr, eb = nullptr;
  PIC_CK(ctx, cudaEventCreate(&ea));
  PIC_CK(ctx, cudaEventCreate(&eb));
  // Two passes over the candidates, the second in reverse order, each
  // candidate's time the sum of both: the plasma keeps evolving while the
  // candidates run (a heating plasma strays more), and a drift in the step
  // time then weighs on every candidate alike.  Before each timed run an
  // untimed one of two sort cycles re-sorts into the new tiles and captures
  // the new step graph, so that neither lands in the timed interval.
  std::vector<double> per_step(cs.size(), 0.0);
  std::vector<char> valid(cs.size(), 1);
  pic_status st = PIC_OK;
  for (int pass = 0; pass < 2 && st == PIC_OK; ++pass)
    for (size_t j = 0; j < cs.size() && st == PIC_OK; ++j) {
      const size_t i = pass == 0 ? j : cs.size() - 1 - j;
      if (!valid[i]) continue;
      pic_tuning t = cs[i];
      t.filter_passes = orig.filter_passes;  // physics, not a launch parameter
      if (t.chunk == 0) t.chunk = orig.chunk;
      if (pic_set_tuning(ctx, &t) != PIC_OK) {  // e.g. window too large: skip
        valid[i] = 0;
        continue;
      }
      const int S = ctx->tun.sort_every;
      const int k = ((std::max(steps, 2 * S) + S - 1) / S) * S;
      if ((st = pic_step(ctx, 2 * S)) != PIC_OK) break;
      cudaEventRecord(ea, ctx->st);
      if ((st = pic_step(ctx, k)) != PIC_OK) break;
      cudaEventRecord(eb, ctx->st);
      if (cudaEventSynchronize(eb) != cudaSuccess) {
        st = cuda_fail(ctx, "autotune timing", cudaGetLastError());
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ea, eb);
      per_step[i] += ms / k;
    }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  if (st != PIC_OK) return st;
  int best = -1;
  for (size_t i = 0; i < cs.size(); ++i)
    if (valid[i] && (best < 0 || per_step[i] < per_step[best])) best = (int)i;
  if (best < 0) {
    pic_set_tuning(ctx, &orig);
    return set_err(ctx, PIC_ERR_ARG, "no candidate tuning was valid");
  }
  pic_tuning t = cs[best];
  t.filter_passes = orig.filter_passes;
  if (t.chunk == 0) t.chunk = orig.chunk;
  st = pic_set_tuning(ctx, &t);
  if (st == PIC_OK && best_index) *best_index = best;
  return st;
}

pic_status pic_timing(pic_ctx* ctx, int enable) {
  if (!ctx) return PIC_ERR_ARG;
  ctx->timing = enable != 0;
  return PIC_OK;
}

pic_status pic_kernel_times(pic_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx || !ms || !launches) return set_err(ctx, PIC_ERR_ARG, "NULL argument");
  PIC_CK(ctx, cudaStreamSynchronize(ctx->st));
  for (auto& t : ctx->pending) {
    float v = 0.f;
    PIC_CK(ctx, cudaEventElapsedTime(&v, t.a, t.b));
    ctx->ms[t.kind] += v;
    ctx->launches[t.kind] += 1;
    ctx->pool.push_back(t.a);
    ctx->pool.push_back(t.b);
  }
  ctx->pending.clear();
  for (int k = 0; k < PIC_KERNEL_KINDS; ++k) {
    ms[k] = ctx->ms[k];
    launches[k] = ctx->launches[k];
    ctx->ms[k] = 0.0;
    ctx->launches[k] = 0;
  }
  return PIC_OK;
}

pic_status pic_destroy(pic_ctx* ctx) {
  if (!ctx) return PIC_ERR_ARG;
  cudaStreamSynchronize(ctx->st);
  free_all(ctx);
  delete ctx;
  return PIC_OK;
}

const char* pic_last_error(const pic_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------- batches --

struct pic_batch {
  std::vector<pic_ctx*> ctxs;
  std::vector<cudaStream_t> branches;  // capture branches (one per group of boxes)
  cudaStream_t origin = nullptr;       // capture origin
  std::vector<cudaEvent_t> events;     // fork (0) and joins (1..)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int cycle = 0;                          // steps per graph launch
  std::vector<long long> phase;           // steps % sort_every of each context at capture
  std::vector<pic_tuning> tun;            // tuning of each context at capture
  std::vector<int> solver;                // pusher * 16 + field order at capture
};

namespace {

constexpr int kBatchBranches = 32;

long long gcd_ll(long long a, long long b) {
  while (b) {
    const long long r = a % b;
    a = b;
    b = r;
  }
  return a;
}

void batch_free_graph(pic_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

bool batch_graph_current(const pic_batch* b) {
  if (!b->exec) return false;
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    const pic_ctx* c = b->ctxs[i];
    if (std::memcmp(&c->tun, &b->tun[i], sizeof(pic_tuning)) != 0) return false;
    if (c->steps % c->tun.sort_every != b->phase[i]) return false;
    if (c->pusher * 16 + c->g.order != b->solver[i]) return false;
  }
  return true;
}

// Capture `cycle` steps of every context into one graph, each context on one
// of the branch streams forked from the origin stream.
pic_status batch_capture(pic_batch* b) {
  batch_free_graph(b);
  for (pic_ctx* c : b->ctxs)  // no allocation may happen during capture
    if (c->tun.filter_passes > 0 && !c->d_jtmp) {
      const cudaError_t ea = dalloc(&c->d_jtmp, 3 * (size_t)c->g.plane);
      if (ea != cudaSuccess) return cuda_fail(nullptr, "filter buffer", ea);
    }
  std::vector<long long> saved_steps(b->ctxs.size());
  std::vector<cudaStream_t> saved_st(b->ctxs.size());
  std::vector<bool> saved_timing(b->ctxs.size());
  cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(nullptr, "batch capture", e);
  pic_status st = PIC_OK;
  cudaEventRecord(b->events[0], b->origin);
  for (cudaStream_t s : b->branches) cudaStreamWaitEvent(s, b->events[0], 0);
  for (size_t i = 0; i < b->ctxs.size() && st == PIC_OK; ++i) {
    pic_ctx* c = b->ctxs[i];
    saved_steps[i] = c->steps;
    saved_st[i] = c->st;
    saved_timing[i] = c->timing;
    c->st = b->branches[i % b->branches.size()];
    c->timing = false;
    c->ensemble = true;
    c->capturing = true;
    st = pic_step(c, b->cycle);
    c->capturing = false;
    c->ensemble = false;
    c->st = saved_st[i];
    c->timing = saved_timing[i];
    c->steps = saved_steps[i];  // the captured steps have not run yet
    if (st != PIC_OK) g_init_error = c->err;
  }
  for (size_t k = 0; k < b->branches.size(); ++k) {
    cudaEventRecord(b->events[k + 1], b->branches[k]);
    cudaStreamWaitEvent(b->origin, b->events[k + 1], 0);
  }
  e = cudaStreamEndCapture(b->origin, &b->graph);
  if (st != PIC_OK) {
    batch_free_graph(b);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(nullptr, "batch capture", e);
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    batch_free_graph(b);
    return cuda_fail(nullptr, "batch graph instantiation", e);
  }
  b->phase.resize(b->ctxs.size());
  b->tun.resize(b->ctxs.size());
  b->solver.resize(b->ctxs.size());
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    b->phase[i] = b->ctxs[i]->steps % b->ctxs[i]->tun.sort_every;
    b->tun[i] = b->ctxs[i]->tun;
    b->solver[i] = b->ctxs[i]->pusher * 16 + b->ctxs[i]->g.order;
  }
  return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_batch_create(pic_batch** out, pic_ctx* const* ctxs, int nctx) {
  g_init_error.clear();
  if (!out) return set_err(nullptr, PIC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ctxs || nctx < 1) return set_err(nullptr, PIC_ERR_ARG, "need at least one context");
  for (int i = 0; i < nctx; ++i) {
    if (!ctxs[i]) return set_err(nullptr, PIC_ERR_ARG, "NULL context");
    if (ctxs[i]->shock)
      return set_err(nullptr, PIC_ERR_ARG, "a context with shock boundaries cannot join a batch");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return set_err(nullptr, PIC_ERR_ARG, "a context appears twice");
  }
  pic_batch* b = new pic_batch();
  b->ctxs.assign(ctxs, ctxs + nctx);
  const int nb = nctx < kBatchBranches ? nctx : kBatchBranches;
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int k = 0; k < nb && e == cudaSuccess; ++k) {
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branches.push_back(s);
  }
  for (int k = 0; k <= nb && e == cudaSuccess; ++k) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->events.push_back(ev);
  }
  // buffers that pic_step would otherwise allocate on first use (no
  // allocation may happen during capture)
  for (int i = 0; i < nctx && e == cudaSuccess; ++i)
    if (ctxs[i]->tun.filter_passes > 0 && !ctxs[i]->d_jtmp)
      e = dalloc(&ctxs[i]->d_jtmp, 3 * (size_t)ctxs[i]->g.plane);
  if (e != cudaSuccess) {
    pic_batch_destroy(b);
    return cuda_fail(nullptr, "batch set-up", e);
  }
  *out = b;
  return PIC_OK;
}

pic_status pic_batch_step(pic_batch* b, int nsteps, void* stream) {
  g_init_error.clear();
  if (!b) return set_err(nullptr, PIC_ERR_ARG, "batch is NULL");
  if (nsteps < 0) return set_err(nullptr, PIC_ERR_ARG, "nsteps must be >= 0");
  const cudaStream_t st = (cudaStream_t)stream;
  long long cycle = 1;
  for (pic_ctx* c : b->ctxs) {
    if (c->st != st) return set_err(nullptr, PIC_ERR_ARG, "every context must use the batch's stream");
    if (c->shock)
      return set_err(nullptr, PIC_ERR_ARG, "a context with shock boundaries cannot join a batch");
    cycle = cycle / gcd_ll(cycle, c->tun.sort_every) * c->tun.sort_every;
    if (cycle > kMaxCycle) return set_err(nullptr, PIC_ERR_ARG, "lcm of the sort cadences exceeds 240");
  }
  const int full = nsteps / (int)cycle, rem = nsteps % (int)cycle;
  if (full > 0) {
    if ((int)cycle != b->cycle || !batch_graph_current(b)) {
      b->cycle = (int)cycle;
      // work already queued on the contexts' stream must precede the capture's
      // own ordering (the graph is launched on that stream afterwards)
      const pic_status s = batch_capture(b);
      if (s != PIC_OK) return s;
    }
    for (int i = 0; i < full; ++i) {
      const cudaError_t e = cudaGraphLaunch(b->exec, st);
      if (e != cudaSuccess) return cuda_fail(nullptr, "batch graph launch", e);
    }
    for (pic_ctx* c : b->ctxs) {
      c->steps += (long long)full * cycle;
      c->snapshot_valid = false;
    }
  }
  for (pic_ctx* c : b->ctxs) {
    if (rem == 0) break;
    const pic_status s = pic_step(c, rem);
    if (s != PIC_OK) {
      g_init_error = c->err;
      return s;
    }
  }
  return PIC_OK;
}

pic_status pic_batch_destroy(pic_batch* b) {
  if (!b) return PIC_ERR_ARG;
  batch_free_graph(b);
  if (b->origin) cudaStreamSynchronize(b->origin);
  for (cudaStream_t s : b->branches) cudaStreamDestroy(s);
  for (cudaEvent_t ev : b->events) cudaEventDestroy(ev);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
  return PIC_OK;
}

}  // extern "C"

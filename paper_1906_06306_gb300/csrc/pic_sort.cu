// Counting sort of particles by spatial tile: the single-GPU stand-in for the
// particle communication routines of Table 1 (arXiv:1906.06306), which move
// particles to the tile that owns them.  count -> exclusive scan -> scatter.
// Lanes of a warp that share a tile combine their atomic (match_any), so a
// sorted or nearly sorted array costs about one global atomic per warp.
#include "pic_kernels.h"

namespace pic {

// Sort bin of a cell: its tile, then the sub-tile inside it (tile-major); every
// division is an exact multiply-shift (FastDiv).
__device__ __forceinline__ int tile_key(const SortParams& P, int cell) {
  if (cell < 0 || (long long)cell >= P.g.plane) {
    atomicOr(P.status, ST_BAD_CELL);
    return 0;  // kept (in tile 0) so that no particle is lost
  }
  const int r = fdiv(cell, P.dn0);
  const int i = cell - r * P.g.n[0];
  const int k = fdiv(r, P.dn1);
  const int j = r - k * P.g.n[1];
  const int ti = fdiv(i, P.dt0), tj = fdiv(j, P.dt1), tk = fdiv(k, P.dt2);
  const int tile = ti + P.t.nt[0] * (tj + P.t.nt[1] * tk);
  if (P.t.nsub == 1) return tile;
  const int si = fdiv(i - ti * P.t.T[0], P.ds0), sj = fdiv(j - tj * P.t.T[1], P.ds1),
            sk = fdiv(k - tk * P.t.T[2], P.ds2);
  return tile * P.t.nsub + si + P.t.ns[0] * (sj + P.t.ns[1] * sk);
}

// Reserve `1` slot of counter[key] for every active lane; returns this lane's
// slot.  Lanes with equal keys share one atomic.
__device__ __forceinline__ int warp_reserve(int* counter, int key, unsigned active) {
  const unsigned peers = __match_any_sync(active, key);
  const int leader = __ffs(peers) - 1;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == leader) base = atomicAdd(&counter[key], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & lanemask_lt());
}

// Tiles of a block's contiguous chunk of particles, counted in a shared-memory
// table before the global counters: in a sorted or nearly sorted array a
// chunk spans a few tiles and their neighbours, so each of those reaches the
// global count once per block instead of once per warp (the same-address
// global atomics of the per-warp count were its limit).  Lanes of a warp with
// the same tile combine first; a table slot is claimed by compare-and-swap,
// and a tile whose slot another tile holds goes straight to the global count.
constexpr int kCountSlots = 1024;
__global__ void __launch_bounds__(256) k_tile_count(const SortParams P, const int* __restrict__ cell,
                                                    long long n, long long chunk, int* count) {
  __shared__ int skey[kCountSlots];
  __shared__ int scnt[kCountSlots];
  for (int s = threadIdx.x; s < kCountSlots; s += blockDim.x) {
    skey[s] = -1;
    scnt[s] = 0;
  }
  __syncthreads();
  const long long lo = (long long)blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  const int lane = threadIdx.x & 31;
  constexpr int U = 4;  // rounds whose loads are issued together (4 loads in flight per thread)
  for (long long base = lo; base < hi; base += U * blockDim.x) {  // block-uniform trip count
    int c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long p = base + u * blockDim.x + threadIdx.x;
      c[u] = p < hi ? cell[p] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool act = base + u * blockDim.x + threadIdx.x < hi;
      const unsigned active = __ballot_sync(0xffffffffu, act);
      if (act) {
        const int key = tile_key(P, c[u]);
        const unsigned peers = __match_any_sync(active, key);
        if (lane == __ffs(peers) - 1) {
          const int n_same = __popc(peers);
          const int slot = (int)(((unsigned)key * 2654435761u) >> 22);  // multiplicative hash, 10 bits
          const int old = atomicCAS(&skey[slot], -1, key);
          if (old == -1 || old == key)
            atomicAdd(&scnt[slot], n_same);
          else
            atomicAdd(&count[key], n_same);
        }
      }
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < kCountSlots; s += blockDim.x)
    if (skey[s] >= 0) atomicAdd(&count[skey[s]], scnt[s]);
}

// Exclusive scan of count[0..ntiles) into start[0..ntiles] (start[ntiles] =
// total) and cursor = start, in one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_tile_scan(const int* __restrict__ count, int ntiles,
                                                    int* start, int* cursor) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < ntiles; base += 1024) {
    const int t = base + threadIdx.x;
    const int v = t < ntiles ? count[t] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    const int incl = x + (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
    if (t < ntiles) {
      start[t] = incl - v;
      cursor[t] = incl - v;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[ntiles] = carry;
}

// Multi-block form of the same exclusive scan for long count arrays (sub-tile
// sort bins): each block scans kScanChunk counts into start and leaves its
// total in part[]; one block scans part[]; every block then adds its offset
// (start[bins] = total, cursor = start).
constexpr int kScanChunk = 4096;  // counts per block: 4 per thread of 1024
__global__ void __launch_bounds__(1024) k_scan_chunks(const int* __restrict__ count, int n,
                                                      int* start, int* part) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int base = blockIdx.x * kScanChunk + 4 * threadIdx.x;
  int v[4], s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[i] = base + i < n ? count[base + i] : 0;
    s += v[i];
  }
  int x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  int run = x - s + (wid > 0 ? warp_sums[wid - 1] : 0);  // exclusive offset in the chunk
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (base + i < n) start[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 1023) part[blockIdx.x] = run;
}

__global__ void __launch_bounds__(1024) k_scan_add(int* start, int* cursor, int n,
                                                   const int* part_scan) {
  const int off = part_scan[blockIdx.x];
  const int base = blockIdx.x * kScanChunk + 4 * threadIdx.x;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (base + i < n) {
      const int v = start[base + i] + off;
      start[base + i] = v;
      cursor[base + i] = v;
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) start[n] = part_scan[gridDim.x];
}

template <int D>
__global__ void k_tile_scatter(const SortParams P, const int* __restrict__ cell,
                               const float* __restrict__ off, const float* __restrict__ u,
                               long long n, long long ld, int* cursor, int* __restrict__ cell_out,
                               float* __restrict__ off_out, float* __restrict__ u_out,
                               int* __restrict__ perm) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long p = base + threadIdx.x;
    const bool act = p < n;
    const unsigned active = __ballot_sync(0xffffffffu, act);
    if (act) {
      const int c = cell[p];
      const long long q = warp_reserve(cursor, tile_key(P, c), active);
      cell_out[q] = c;
#pragma unroll
      for (int d = 0; d < D; ++d) off_out[d * ld + q] = off[d * ld + p];
#pragma unroll
      for (int a = 0; a < 3; ++a) u_out[a * ld + q] = u[a * ld + p];
      if (perm) perm[q] = (int)p;  // the slot the particle held before the sort
    }
  }
}

SortParams make_sort_params(const GridDev& g, const TileDev& t, int* status) {
  SortParams P{};
  P.g = g;
  P.t = t;
  P.status = status;
  P.dn0 = make_fastdiv(g.n[0]);
  P.dn1 = make_fastdiv(g.n[1]);
  P.dt0 = make_fastdiv(t.T[0]);
  P.dt1 = make_fastdiv(t.T[1]);
  P.dt2 = make_fastdiv(t.T[2]);
  P.ds0 = make_fastdiv(t.S[0]);
  P.ds1 = make_fastdiv(t.S[1]);
  P.ds2 = make_fastdiv(t.S[2]);
  return P;
}

static unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 64) b = 152LL * 64;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_tile_count(const SortParams& P, const int* cell, long long n, int* count,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  // contiguous chunks of at least 4096 particles (a multiple of 256), at most
  // 16 blocks per SM
  long long nb = (n + 4095) / 4096;
  if (nb > 152LL * 16) nb = 152LL * 16;
  const long long chunk = ((n + nb - 1) / nb + 255) / 256 * 256;
  nb = (n + chunk - 1) / chunk;
  k_tile_count<<<(unsigned)nb, 256, 0, st>>>(P, cell, n, chunk, count);
  return cudaGetLastError();
}

cudaError_t launch_tile_scan(const int* count, int ntiles, int* start, int* cursor, int* scratch,
                             cudaStream_t st) {
  if (ntiles <= kScanChunk) {
    k_tile_scan<<<1, 1024, 0, st>>>(count, ntiles, start, cursor);
    return cudaGetLastError();
  }
  // scratch: block totals [nb], their scan [nb + 1], the scan's cursor [nb]
  const int nb = (ntiles + kScanChunk - 1) / kScanChunk;
  int* part = scratch;
  int* part_scan = scratch + nb;
  int* part_cursor = scratch + 2 * nb + 1;
  k_scan_chunks<<<nb, 1024, 0, st>>>(count, ntiles, start, part);
  k_tile_scan<<<1, 1024, 0, st>>>(part, nb, part_scan, part_cursor);
  k_scan_add<<<nb, 1024, 0, st>>>(start, cursor, ntiles, part_scan);
  return cudaGetLastError();
}

cudaError_t launch_tile_scatter(const SortParams& P, const int* cell, const float* off,
                                const float* u, long long n, long long ld, int* cursor,
                                int* cell_out, float* off_out, float* u_out, cudaStream_t st,
                                int* perm) {
  if (n == 0) return cudaSuccess;
  const unsigned nb = blocks_for(n);
  switch (P.g.dim) {
    case 1: k_tile_scatter<1><<<nb, 256, 0, st>>>(P, cell, off, u, n, ld, cursor, cell_out, off_out, u_out, perm); break;
    case 2: k_tile_scatter<2><<<nb, 256, 0, st>>>(P, cell, off, u, n, ld, cursor, cell_out, off_out, u_out, perm); break;
    case 3: k_tile_scatter<3><<<nb, 256, 0, st>>>(P, cell, off, u, n, ld, cursor, cell_out, off_out, u_out, perm); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Bucket starts handed in from outside: one block checks that they run from
// 0 to n without decreasing; if not, every start but the last becomes 0 (one
// bucket: the last tile's blocks take every particle, all through the stray
// path) and the status word says so.
__global__ void k_check_buckets(int* __restrict__ t, long long nb, long long n, int* status) {
  bool bad = threadIdx.x == 0 && (t[0] != 0 || t[nb] != n);
  for (long long i = threadIdx.x; i < nb; i += blockDim.x) bad |= t[i] > t[i + 1];
  if (!__syncthreads_or(bad)) return;
  for (long long i = threadIdx.x; i < nb; i += blockDim.x) t[i] = 0;
  if (threadIdx.x == 0) {
    t[nb] = (int)n;
    atomicOr(status, ST_BAD_BUCKETS);
  }
}

cudaError_t launch_check_buckets(int* tstart, long long nb, long long n, int* status,
                                 cudaStream_t st) {
  k_check_buckets<<<1, 1024, 0, st>>>(tstart, nb, n, status);
  return cudaGetLastError();
}

// Bucket starts of one slot range [lo, hi) of a species: out[i] = tstart[i]
// clamped to [lo, hi), so that bucket i of the clipped starts is bucket i's
// part inside the range (a particle launch over the clipped starts processes
// the slots of that range only).
__global__ void k_clip_starts(const int* __restrict__ t, long long nb1, int lo, int hi,
                              int* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb1; i += stride)
    out[i] = min(max(t[i], lo), hi);
}

cudaError_t launch_clip_starts(const int* tstart, long long nb1, int lo, int hi, int* out,
                               cudaStream_t st) {
  if (nb1 <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((nb1 + 255) / 256, 4 * 152);
  k_clip_starts<<<(unsigned)blocks, 256, 0, st>>>(tstart, nb1, lo, hi, out);
  return cudaGetLastError();
}

// Adjoint of a sort's permutation: the gradient rows of the particle now in
// slot i go to the slot it held before the sort, perm[i] (out[perm[i]] =
// in[i] on each of the `rows` rows of length ld).  An entry outside [0, n)
// is skipped and reported (ST_BAD_BUCKETS): the permutation came from the
// caller.
__global__ void k_unpermute(const int* __restrict__ perm, const float* __restrict__ in,
                            float* __restrict__ out, long long n, long long ld, int rows,
                            int* status) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long q = perm[i];
    if (q < 0 || q >= n) {
      atomicOr(status, ST_BAD_BUCKETS);
      continue;
    }
    for (int r = 0; r < rows; ++r) out[r * ld + q] = in[r * ld + i];
  }
}

cudaError_t launch_unpermute(const int* perm, const float* in, float* out, long long n,
                             long long ld, int rows, int* status, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_unpermute<<<blocks_for(n), 256, 0, st>>>(perm, in, out, n, ld, rows, status);
  return cudaGetLastError();
}

}  // namespace pic

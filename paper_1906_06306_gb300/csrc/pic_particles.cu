// Particle kernel of the PIC step: interp_em + push + comp_curr of Table 1
// (arXiv:1906.06306), one thread block per (tile, split).
//
// Particles are sorted by tile.  A block stages its tile's E and B plus a
// halo into shared memory, runs every particle of the tile's bucket (all
// species) through gather -> Boris -> move -> ZigZag, accumulating the current
// in a shared-memory J window, and finally adds that window into the global J
// planes.  A particle whose stencil is not inside the window (it drifted more
// than halo-1 cells since the last sort) reads and deposits through global
// memory instead, so correctness never depends on the sort cadence.
#include "pic_kernels.h"

namespace pic {

template <int D, int MODE>
__device__ __forceinline__ void one_particle(const PushParams& P, const SpeciesDev& S,
                                             long long p, const SmemAcc& SA, const GlobAcc& GA,
                                             const int* w0) {
  const long long n = S.n;
  int cell;
  float o1[3] = {0.f, 0.f, 0.f};
  float u[3];
  if (MODE == 2) {
    cell = S.cell_old[p];
#pragma unroll
    for (int d = 0; d < D; ++d) o1[d] = S.off_old[d * n + p];
  } else {
    cell = S.cell[p];
#pragma unroll
    for (int d = 0; d < D; ++d) o1[d] = S.off[d * n + p];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = S.u[a * n + p];

  if (cell < 0 || (long long)cell >= P.g.plane) {
    atomicOr(P.status, ST_BAD_CELL);
    return;
  }
  bool bad = false;
#pragma unroll
  for (int d = 0; d < D; ++d) bad |= !(o1[d] >= 0.0f && o1[d] < 1.0f);
  if (bad) {
    atomicOr(P.status, ST_BAD_OFF);
    return;
  }
  if (!(isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) {
    atomicOr(P.status, ST_BAD_U);
    return;
  }

  int ijk[3];
  ijk[0] = cell % P.g.n[0];
  const int r = cell / P.g.n[0];
  ijk[1] = r % P.g.n[1];
  ijk[2] = r / P.g.n[1];
  int l[3] = {0, 0, 0};
  bool inwin = true;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    l[d] = wrapi(ijk[d] - w0[d], P.g.n[d]);
    inwin &= (l[d] >= 1) && (l[d] <= P.t.W[d] - 3);
  }

  if (MODE != 2) {
    float e[3], b[3];
    if (inwin)
      gather<D>(SA, l, o1, e, b);
    else
      gather<D>(GA, ijk, o1, e, b);
    boris(u, e, b, S.qm, P.g.c, P.inv_c, P.inv_c2);
  }
  float o2[3] = {0.f, 0.f, 0.f}, dn[3];
  int dc[3] = {0, 0, 0};
  move<D>(u, o1, P.g.c, o2, dc, dn);

  if (MODE != 2) {
    int nc[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) nc[d] = wrap1(ijk[d] + dc[d], P.g.n[d]);
    const int cell2 = nc[0] + P.g.n[0] * (nc[1] + P.g.n[1] * nc[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) S.u[a * n + p] = u[a];
#pragma unroll
    for (int d = 0; d < D; ++d) S.off[d * n + p] = o2[d];
    S.cell[p] = cell2;
    if (MODE == 1) {
      S.cell_old[p] = cell;
#pragma unroll
      for (int d = 0; d < D; ++d) S.off_old[d * n + p] = o1[d];
    }
  }
  if (MODE != 1) {
    if (inwin)
      zigzag<D>(SA, l, dc, o1, o2, dn, S.q);
    else
      zigzag<D>(GA, ijk, dc, o1, o2, dn, S.q);
  }
}

template <int D, int MODE>
__global__ void __launch_bounds__(kPushThreads) k_particles(const PushParams P) {
  extern __shared__ float sm[];
  const int tile = blockIdx.x / P.splits;
  const int split = blockIdx.x - tile * P.splits;
  const int tc[3] = {tile % P.t.nt[0], (tile / P.t.nt[0]) % P.t.nt[1],
                     tile / (P.t.nt[0] * P.t.nt[1])};
  int w0[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < D; ++d) w0[d] = tc[d] * P.t.T[d] - P.t.H;
  const int wc = P.t.wcells;
  const int W0 = P.t.W[0], W1 = P.t.W[1];
  const GlobAcc GA{P.F, P.g.plane, P.g.n[0], P.g.n[1], P.g.n[2]};
  const SmemAcc SA{sm, W0, W0 * W1, wc};

  for (int w = threadIdx.x; w < wc; w += blockDim.x) {
    const int lx = w % W0, rr = w / W0, ly = rr % W1, lz = rr / W1;
    const long long gi = GA.at(w0[0] + lx, w0[1] + ly, w0[2] + lz);
    if (MODE != 2) {
#pragma unroll
      for (int comp = EX; comp <= BZ; ++comp) sm[comp * wc + w] = __ldg(&P.F[comp * P.g.plane + gi]);
    }
    if (MODE != 1) {
#pragma unroll
      for (int comp = JX; comp <= JZ; ++comp) sm[comp * wc + w] = 0.0f;
    }
  }
  __syncthreads();

  for (int s = 0; s < P.nspecies; ++s) {
    const SpeciesDev& S = P.sp[s];
    const long long lo = S.tstart[tile], hi = S.tstart[tile + 1];
    const long long len = hi - lo;
    const long long a = lo + len * split / P.splits;
    const long long b = lo + len * (split + 1) / P.splits;
    for (long long p = a + threadIdx.x; p < b; p += blockDim.x)
      one_particle<D, MODE>(P, S, p, SA, GA, w0);
  }

  if (MODE != 1) {
    __syncthreads();
    for (int w = threadIdx.x; w < wc; w += blockDim.x) {
      const int lx = w % W0, rr = w / W0, ly = rr % W1, lz = rr / W1;
      const long long gi = GA.at(w0[0] + lx, w0[1] + ly, w0[2] + lz);
#pragma unroll
      for (int comp = JX; comp <= JZ; ++comp) {
        const float v = sm[comp * wc + w];
        if (v != 0.0f) atomicAdd(&P.F[comp * P.g.plane + gi], v);
      }
    }
  }
}

size_t particle_smem_bytes(const TileDev& t) { return sizeof(float) * 9 * (size_t)t.wcells; }

template <int D, int MODE>
static cudaError_t set_limit(int bytes) {
  return cudaFuncSetAttribute(k_particles<D, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t set_particle_smem_limit(int bytes) {
  cudaError_t e = cudaSuccess;
#define PIC_SET(D)                                          \
  if (e == cudaSuccess) e = set_limit<D, 0>(bytes);         \
  if (e == cudaSuccess) e = set_limit<D, 1>(bytes);         \
  if (e == cudaSuccess) e = set_limit<D, 2>(bytes);
  PIC_SET(1)
  PIC_SET(2)
  PIC_SET(3)
#undef PIC_SET
  return e;
}

template <int D, int MODE>
static void launch(const PushParams& P, cudaStream_t st) {
  const unsigned nblocks = (unsigned)P.t.ntiles * (unsigned)P.splits;
  k_particles<D, MODE><<<nblocks, kPushThreads, particle_smem_bytes(P.t), st>>>(P);
}

cudaError_t launch_particles(int dim, int mode, const PushParams& P, cudaStream_t st) {
  if ((long long)P.t.ntiles * P.splits == 0) return cudaSuccess;
  switch (dim * 3 + mode) {
    case 3: launch<1, 0>(P, st); break;
    case 4: launch<1, 1>(P, st); break;
    case 5: launch<1, 2>(P, st); break;
    case 6: launch<2, 0>(P, st); break;
    case 7: launch<2, 1>(P, st); break;
    case 8: launch<2, 2>(P, st); break;
    case 9: launch<3, 0>(P, st); break;
    case 10: launch<3, 1>(P, st); break;
    case 11: launch<3, 2>(P, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pic

// FDTD2 field update and Binomial2 current filter (arXiv:1906.06306,
// Sect. 2.3.1, Eqs. (fdE), (fdB), Table 2) on periodic Yee planes.
// One thread per lattice point, x fastest, so every plane is streamed with
// coalesced loads; neighbours one point away come from the same or adjacent
// rows and hit L1/L2.  The filter runs as one 3-point sub-pass per gridded
// axis (x, then y, then z), the order in which the paper's filter is applied.
#include "pic_kernels.h"

namespace pic {

// B -= (c/2) curl+ E (forward differences: B sits half a cell above E), and,
// when zero_j is set, clear J for the deposit that follows.
template <int D>
__device__ __forceinline__ void b_half_point(float* __restrict__ F, const GridDev& g, int i, int j,
                                             int k, float hc, int zero_j) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  const long long idx = (long long)i + (long long)n0 * (j + (long long)n1 * k);
  const long long sx = (i + 1 < n0) ? 1 : 1 - n0;
  const long long sy = (D >= 2) ? ((j + 1 < n1) ? n0 : (long long)n0 * (1 - n1)) : 0;
  const long long sz = (D >= 3) ? ((k + 1 < n2) ? (long long)n0 * n1 : (long long)n0 * n1 * (1 - n2)) : 0;
  const float* Ex = F + EX * P;
  const float* Ey = F + EY * P;
  const float* Ez = F + EZ * P;
  const float ex = Ex[idx], ey = Ey[idx], ez = Ez[idx];
  float cx = 0.f, cy = 0.f, cz = 0.f;
  cy -= Ez[idx + sx] - ez;
  cz += Ey[idx + sx] - ey;
  if (D >= 2) {
    cx += Ez[idx + sy] - ez;
    cz -= Ex[idx + sy] - ex;
  }
  if (D >= 3) {
    cx -= Ey[idx + sz] - ey;
    cy += Ex[idx + sz] - ex;
  }
  F[BX * P + idx] = fmaf(-hc, cx, F[BX * P + idx]);
  F[BY * P + idx] = fmaf(-hc, cy, F[BY * P + idx]);
  F[BZ * P + idx] = fmaf(-hc, cz, F[BZ * P + idx]);
  if (zero_j) {
    F[JX * P + idx] = 0.f;
    F[JY * P + idx] = 0.f;
    F[JZ * P + idx] = 0.f;
  }
}

template <int D>
__global__ void k_b_half(float* __restrict__ F, const GridDev g, float hc, int zero_j) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  FOR_ROWS(j, k) { b_half_point<D>(F, g, i, j, k, hc, zero_j); }
}

// E += c curl- B - J (backward differences: E sits half a cell below B).
template <int D>
__device__ __forceinline__ void e_update_point(float* __restrict__ F, const GridDev& g, int i,
                                               int j, int k, float c) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  const long long idx = (long long)i + (long long)n0 * (j + (long long)n1 * k);
  const long long sx = (i > 0) ? 1 : 1 - n0;
  const long long sy = (D >= 2) ? ((j > 0) ? n0 : (long long)n0 * (1 - n1)) : 0;
  const long long sz = (D >= 3) ? ((k > 0) ? (long long)n0 * n1 : (long long)n0 * n1 * (1 - n2)) : 0;
  const float* Bx = F + BX * P;
  const float* By = F + BY * P;
  const float* Bz = F + BZ * P;
  const float bx = Bx[idx], by = By[idx], bz = Bz[idx];
  float cx = 0.f, cy = 0.f, cz = 0.f;
  cy -= bz - Bz[idx - sx];
  cz += by - By[idx - sx];
  if (D >= 2) {
    cx += bz - Bz[idx - sy];
    cz -= bx - Bx[idx - sy];
  }
  if (D >= 3) {
    cx -= by - By[idx - sz];
    cy += bx - Bx[idx - sz];
  }
  F[EX * P + idx] = fmaf(c, cx, F[EX * P + idx]) - F[JX * P + idx];
  F[EY * P + idx] = fmaf(c, cy, F[EY * P + idx]) - F[JY * P + idx];
  F[EZ * P + idx] = fmaf(c, cz, F[EZ * P + idx]) - F[JZ * P + idx];
}

template <int D>
__global__ void k_e_update(float* __restrict__ F, const GridDev g, float c) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  FOR_ROWS(j, k) { e_update_point<D>(F, g, i, j, k, c); }
}

// The second B half step and the E update of a small lattice by one block:
// every point's B half step, a block barrier (which orders the block's
// global-memory writes before its later reads), every point's E update; the
// operations of k_b_half and k_e_update point by point, so the same bits.  One
// launch instead of two where launch latency, not bandwidth, bounds the step.
// With `chain` set, after another barrier, the next step's first B half step
// (which clears J for its deposit) as well: one launch instead of three.
template <int D>
__global__ void __launch_bounds__(1024) k_fields_small(float* __restrict__ F, const GridDev g,
                                                       float hc, float c, int chain) {
  const int n0 = g.n[0], n1 = g.n[1];
  const int cells = (int)g.plane;
  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    const int i = t % n0, r = t / n0;
    b_half_point<D>(F, g, i, r % n1, r / n1, hc, 0);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    const int i = t % n0, r = t / n0;
    e_update_point<D>(F, g, i, r % n1, r / n1, c);
  }
  if (!chain) return;
  __syncthreads();
  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    const int i = t % n0, r = t / n0;
    b_half_point<D>(F, g, i, r % n1, r / n1, hc, 1);
  }
}

// The same two updates with four consecutive x points per thread (rows whose
// length is a multiple of 4 and 16-byte aligned planes): 16-byte loads and
// stores of the thread's points, one scalar load for the x neighbour outside
// them.  Each point goes through the operations of k_b_half / k_e_update in
// the same order, so the results are the same bits.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void arr4(const float4 a, float v[4]) {
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}

template <int D>
__global__ void k_b_half_x4(float* __restrict__ F, const GridDev g, float hc, int zero_j) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  const int i = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n0) return;
  FOR_ROWS(j, k) {
    const long long idx = (long long)i + (long long)n0 * (j + (long long)n1 * k);
    const long long x4 = (i + 4 < n0) ? idx + 4 : idx + 4 - n0;  // x neighbour of the last point
    const long long sy = (D >= 2) ? ((j + 1 < n1) ? n0 : (long long)n0 * (1 - n1)) : 0;
    const long long sz = (D >= 3) ? ((k + 1 < n2) ? (long long)n0 * n1 : (long long)n0 * n1 * (1 - n2)) : 0;
    const float* Ex = F + EX * P;
    const float* Ey = F + EY * P;
    const float* Ez = F + EZ * P;
    float ex[4], ey[4], ez[4], eyx[4], ezx[4], ezy[4] = {}, exy[4] = {}, eyz[4] = {}, exz[4] = {};
    arr4(ld4(Ex + idx), ex);
    arr4(ld4(Ey + idx), ey);
    arr4(ld4(Ez + idx), ez);
    eyx[0] = ey[1], eyx[1] = ey[2], eyx[2] = ey[3], eyx[3] = Ey[x4];
    ezx[0] = ez[1], ezx[1] = ez[2], ezx[2] = ez[3], ezx[3] = Ez[x4];
    if (D >= 2) {
      arr4(ld4(Ez + idx + sy), ezy);
      arr4(ld4(Ex + idx + sy), exy);
    }
    if (D >= 3) {
      arr4(ld4(Ey + idx + sz), eyz);
      arr4(ld4(Ex + idx + sz), exz);
    }
    float bx[4], by[4], bz[4];
    arr4(ld4(F + BX * P + idx), bx);
    arr4(ld4(F + BY * P + idx), by);
    arr4(ld4(F + BZ * P + idx), bz);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      float cx = 0.f, cy = 0.f, cz = 0.f;
      cy -= ezx[l] - ez[l];
      cz += eyx[l] - ey[l];
      if (D >= 2) {
        cx += ezy[l] - ez[l];
        cz -= exy[l] - ex[l];
      }
      if (D >= 3) {
        cx -= eyz[l] - ey[l];
        cy += exz[l] - ex[l];
      }
      bx[l] = fmaf(-hc, cx, bx[l]);
      by[l] = fmaf(-hc, cy, by[l]);
      bz[l] = fmaf(-hc, cz, bz[l]);
    }
    st4(F + BX * P + idx, bx);
    st4(F + BY * P + idx, by);
    st4(F + BZ * P + idx, bz);
    if (zero_j) {
      const float z[4] = {0.f, 0.f, 0.f, 0.f};
      st4(F + JX * P + idx, z);
      st4(F + JY * P + idx, z);
      st4(F + JZ * P + idx, z);
    }
  }
}

template <int D>
__global__ void k_e_update_x4(float* __restrict__ F, const GridDev g, float c) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  const int i = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n0) return;
  FOR_ROWS(j, k) {
    const long long idx = (long long)i + (long long)n0 * (j + (long long)n1 * k);
    const long long xm = (i > 0) ? idx - 1 : idx + n0 - 1;  // x neighbour of the first point
    const long long sy = (D >= 2) ? ((j > 0) ? n0 : (long long)n0 * (1 - n1)) : 0;
    const long long sz = (D >= 3) ? ((k > 0) ? (long long)n0 * n1 : (long long)n0 * n1 * (1 - n2)) : 0;
    const float* Bx = F + BX * P;
    const float* By = F + BY * P;
    const float* Bz = F + BZ * P;
    float bx[4], by[4], bz[4], byx[4], bzx[4], bzy[4] = {}, bxy[4] = {}, byz[4] = {}, bxz[4] = {};
    arr4(ld4(Bx + idx), bx);
    arr4(ld4(By + idx), by);
    arr4(ld4(Bz + idx), bz);
    byx[0] = By[xm], byx[1] = by[0], byx[2] = by[1], byx[3] = by[2];
    bzx[0] = Bz[xm], bzx[1] = bz[0], bzx[2] = bz[1], bzx[3] = bz[2];
    if (D >= 2) {
      arr4(ld4(Bz + idx - sy), bzy);
      arr4(ld4(Bx + idx - sy), bxy);
    }
    if (D >= 3) {
      arr4(ld4(By + idx - sz), byz);
      arr4(ld4(Bx + idx - sz), bxz);
    }
    float ex[4], ey[4], ez[4], jx[4], jy[4], jz[4];
    arr4(ld4(F + EX * P + idx), ex);
    arr4(ld4(F + EY * P + idx), ey);
    arr4(ld4(F + EZ * P + idx), ez);
    arr4(ld4(F + JX * P + idx), jx);
    arr4(ld4(F + JY * P + idx), jy);
    arr4(ld4(F + JZ * P + idx), jz);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      float cx = 0.f, cy = 0.f, cz = 0.f;
      cy -= bz[l] - bzx[l];
      cz += by[l] - byx[l];
      if (D >= 2) {
        cx += bz[l] - bzy[l];
        cz -= bx[l] - bxy[l];
      }
      if (D >= 3) {
        cx -= by[l] - byz[l];
        cy += bx[l] - bxz[l];
      }
      ex[l] = fmaf(c, cx, ex[l]) - jx[l];
      ey[l] = fmaf(c, cy, ey[l]) - jy[l];
      ez[l] = fmaf(c, cz, ez[l]) - jz[l];
    }
    st4(F + EX * P + idx, ex);
    st4(F + EY * P + idx, ey);
    st4(F + EZ * P + idx, ez);
  }
}

// One Binomial2 sub-pass along one axis: dst = (1/4, 1/2, 1/4) * src along
// `axis`, periodic.  Thread (x, y, z*ncomp) of a 3D launch grid owns one
// lattice value, so neighbours along every axis are coalesced loads.
template <typename T>
__global__ void k_filter_axis(const T* __restrict__ src, T* __restrict__ dst, const GridDev g,
                              int axis) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n[0]) return;
  const int j = blockIdx.y;
  const int k = blockIdx.z % g.n[2];
  const long long comp = blockIdx.z / g.n[2];
  const long long P = g.plane;
  const long long idx = (long long)i + (long long)g.n[0] * (j + (long long)g.n[1] * k);
  const T* s = src + comp * P;
  const int a = axis == 0 ? i : axis == 1 ? j : k;
  const int na = g.n[axis];
  const long long stride = axis == 0 ? 1 : axis == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1];
  const long long lo = a > 0 ? idx - stride : idx + (long long)(na - 1) * stride;
  const long long hi = a + 1 < na ? idx + stride : idx - (long long)(na - 1) * stride;
  dst[comp * P + idx] = T(0.25) * s[lo] + T(0.5) * s[idx] + T(0.25) * s[hi];
}

// One full Binomial2 pass (the x, y and z sub-passes in that order) on each
// of the consecutive planes src -> dst, fused through shared memory: a block
// loads a TX x TY x TZ tile of one plane plus a one-cell periodic halo, runs
// the sub-passes on it in shared memory and writes the tile.  Every output
// goes through the same arithmetic, in the same order, as three
// k_filter_axis sub-passes, but a pass moves 24 B per cell instead of 72.
// Grid: x = tile index, y = plane.  The library launches it for 1D grids
// (1024-point tiles); 2D and 3D grids take the marching passes k_filter_y2
// and k_filter_z3 below, which stream the planes instead of re-reading a
// halo per tile.
template <int D, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256) k_filter_pass(const float* __restrict__ src,
                                                     float* __restrict__ dst, const GridDev g,
                                                     int ntx, int nty) {
  constexpr int HX = TX + 2, HY = D >= 2 ? TY + 2 : 1, HZ = D >= 3 ? TZ + 2 : 1;
  constexpr int OY = D >= 2 ? TY : 1, OZ = D >= 3 ? TZ : 1;
  __shared__ float a[HX * HY * HZ];
  __shared__ float b[TX * HY * HZ];
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int tile = blockIdx.x;
  const int x0 = (tile % ntx) * TX;
  const int y0 = ((tile / ntx) % nty) * OY;
  const int z0 = (tile / (ntx * nty)) * OZ;
  const long long P = g.plane;
  const float* s = src + (long long)blockIdx.y * P;
  float* d = dst + (long long)blockIdx.y * P;
  // tile coordinates run from -1 to n + T - 1: one conditional wrap suffices
  // when the extent is larger than the tile (else, tiny grids, a modulo)
  const bool fast = n0 > TX && (D < 2 || n1 > TY) && (D < 3 || n2 > TZ);
  for (int t = threadIdx.x; t < HX * HY * HZ; t += blockDim.x) {
    const int lx = t % HX, r = t / HX, ly = r % HY, lz = r / HY;
    int gx = x0 + lx - 1, gy = D >= 2 ? y0 + ly - 1 : 0, gz = D >= 3 ? z0 + lz - 1 : 0;
    if (fast) {
      gx = wrap1(gx, n0);
      if (D >= 2) gy = wrap1(gy, n1);
      if (D >= 3) gz = wrap1(gz, n2);
    } else {
      gx = wrapi(gx, n0);
      if (D >= 2) gy = wrapi(gy, n1);
      if (D >= 3) gz = wrapi(gz, n2);
    }
    a[t] = s[(long long)gx + (long long)n0 * (gy + (long long)n1 * gz)];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TX * HY * HZ; t += blockDim.x) {  // x sub-pass: a -> b
    const int lx = t % TX, r = t / TX;
    const float* q = a + lx + HX * r;
    b[t] = 0.25f * q[0] + 0.5f * q[1] + 0.25f * q[2];
  }
  __syncthreads();
  const float* res = b;  // result tile, rows of TX
  if (D >= 2) {
    for (int t = threadIdx.x; t < TX * TY * HZ; t += blockDim.x) {  // y sub-pass: b -> a
      const int lx = t % TX, r = t / TX, ly = r % TY, lz = r / TY;
      const float* q = b + lx + TX * (ly + HY * lz);
      a[t] = 0.25f * q[0] + 0.5f * q[TX] + 0.25f * q[2 * TX];
    }
    __syncthreads();
    res = a;
  }
  for (int t = threadIdx.x; t < TX * OY * OZ; t += blockDim.x) {
    const int lx = t % TX, r = t / TX, ly = r % OY, lz = r / OY;
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    if (gx >= n0 || gy >= n1 || gz >= n2) continue;
    float v;
    if (D >= 3) {  // z sub-pass straight from the y result
      const float* q = res + lx + TX * (ly + TY * lz);
      v = 0.25f * q[0] + 0.5f * q[TX * TY] + 0.25f * q[2 * TX * TY];
    } else {
      v = res[t];
    }
    d[(long long)gx + (long long)n0 * (gy + (long long)n1 * gz)] = v;
  }
}

// One full 3D Binomial2 pass (x, y, then z sub-pass) of one plane src -> dst,
// marching along z.  A block of 256 threads owns a ZX x ZY = 128 x 16 column
// of (x, y) points over a run of `zrun` z-planes; a thread owns a 4 (x) x 2
// (y) patch of it.  Each z-plane of the column plus its one-point periodic
// (x, y) halo is copied into a ring of ZS shared-memory stages, ZS - 1 planes
// ahead of the one being filtered.  BULK (rows of a multiple of 4 floats,
// 16-byte aligned planes, a status word): the ZY + 2 stage rows arrive by one
// bulk copy each (`cp.async.bulk`, issued by the lanes of warp 0, completing
// on the stage's mbarrier) and the two halo points of each row by 4-byte
// cp.async; otherwise every thread copies by cp.async (16-byte copies for the
// aligned interior, 4-byte ones for the halo and for ragged or wrapped rows).
// A thread reads its four rows (y - 1 .. y + 2) with one 16-byte and two
// 4-byte shared loads each, runs the x and y sub-passes in registers and keeps
// the last three y results for the z sub-pass.  Reads: the column, its (x, y)
// halo (rows of neighbouring columns, mostly from L2) and two extra planes per
// run; writes: the column, 16 bytes per store.  Every output goes through the
// same arithmetic, in the same order, as three k_filter_axis sub-passes.
// Grid: x = column index + columns x run, y = plane.
constexpr int ZX = 128, ZY = 16, ZS = 4;
constexpr int ZROW = ZX + 8;  // stage row: [3] left halo, [4, 4 + ZX) interior, [4 + ZX] right
constexpr int ZPLANE = (ZY + 2) * ZROW;
constexpr int ZCH = ZX / 4 + 2;         // copy operations per stage row
constexpr int ZOPS = (ZY + 2) * ZCH;    // copy operations per stage (612)
constexpr int ZOPT = (ZOPS + 255) / 256;  // per thread (3)

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ float b3(float l, float c, float r) {
  return 0.25f * l + 0.5f * c + 0.25f * r;
}

// A marching pass's wait, by every thread, for the bulk copies of step k
// (stage k % ZS, phase parity (k / ZS) & 1; steps k .. min(k + ZS - 2,
// nk - 1) are in flight); true when the whole block may go on.  When a wait
// ran out (the status word has the timeout bit), thread 0 waits once more,
// bounded, for each step still in flight, and the block leaves together.
__device__ __forceinline__ bool stage_landed(unsigned long long* full, int k, int nk, int* status) {
  const bool ok = mbar_wait(&full[k % ZS], (unsigned)(k / ZS) & 1u, status);
  if (!__syncthreads_or(!ok)) return true;
  if (threadIdx.x == 0)
    for (int j = k; j < k + ZS - 1 && j < nk; ++j)
      mbar_wait(&full[j % ZS], (unsigned)(j / ZS) & 1u, nullptr);
  cp_async_wait<0>();
  return false;
}

template <bool BULK>
__global__ void __launch_bounds__(256, 4) k_filter_z3(const float* __restrict__ src,
                                                     float* __restrict__ dst, const GridDev g,
                                                     int ncx, int ncy, int zrun, int vec,
                                                     int* status) {
  __shared__ __align__(16) float stage[ZS][ZPLANE];
  __shared__ unsigned long long full[ZS];  // BULK: stage's rows have landed
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long nxy = (long long)n0 * n1;
  const int col = blockIdx.x % (ncx * ncy), run = blockIdx.x / (ncx * ncy);
  const int x0 = (col % ncx) * ZX, y0 = (col / ncx) * ZY, z0 = run * zrun;
  const int zc = min(zrun, n2 - z0);  // planes z0 .. z0 + zc - 1 are written
  const long long P = g.plane;
  const float* s = src + (long long)blockIdx.y * P;
  float* d = dst + (long long)blockIdx.y * P;
  const int len = min(ZX, n0 - x0);  // interior points of the column's rows

  // This thread's copy operations op = threadIdx.x + 256 j, the same for every
  // z-plane: stage row op / ZCH (y = y0 - 1 + row) and either a 4-point
  // interior chunk (c < ZX / 4), the left halo point (c = ZX / 4) or the right.
  // BULK: lane r < ZY + 2 of warp 0 copies the interior of stage row r, and
  // threads 64 .. 64 + 2 (ZY + 2) - 1 its halo points (the right one after
  // the last interior point, where a ragged column's x sub-pass reads it).
  long long yoff[ZOPT];
  int xs[ZOPT], dofs[ZOPT], kind[ZOPT];  // kind: 0 none, 1 16-byte, 2 four 4-byte, 3 one 4-byte
#pragma unroll
  for (int j = 0; j < ZOPT; ++j) {
    kind[j] = 0;
    yoff[j] = 0;
    xs[j] = 0;
    dofs[j] = 0;
  }
  if (BULK) {
    const int t = threadIdx.x;
    if (t < ZY + 2) {  // interior of row t
      yoff[0] = (long long)n0 * wrapi(y0 - 1 + t, n1);
      xs[0] = x0;
      dofs[0] = t * ZROW + 4;
      kind[0] = 1;
    } else if (t >= 64 && t < 64 + 2 * (ZY + 2)) {  // a halo point of row (t - 64) / 2
      const int row = (t - 64) >> 1, right = (t - 64) & 1;
      yoff[0] = (long long)n0 * wrapi(y0 - 1 + row, n1);
      xs[0] = wrapi(right ? x0 + len : x0 - 1, n0);
      dofs[0] = row * ZROW + (right ? 4 + len : 3);
      kind[0] = 3;
    }
    if (t == 0) {
      for (int i = 0; i < ZS; ++i) mbar_init(&full[i], 1);
      mbar_init_fence();
    }
    __syncthreads();  // the barriers are initialised before any copy or wait
  } else {
#pragma unroll
    for (int j = 0; j < ZOPT; ++j) {
      const int op = threadIdx.x + 256 * j;
      const int row = op / ZCH, c = op % ZCH;
      if (op < ZOPS) {
        yoff[j] = (long long)n0 * wrapi(y0 - 1 + row, n1);
        if (c < ZX / 4) {
          xs[j] = x0 + 4 * c;
          dofs[j] = row * ZROW + 4 + 4 * c;
          kind[j] = vec && xs[j] + 3 < n0 ? 1 : 2;
        } else {
          xs[j] = wrapi(c == ZX / 4 ? x0 - 1 : x0 + ZX, n0);
          dofs[j] = row * ZROW + (c == ZX / 4 ? 3 : 4 + ZX);
          kind[j] = 3;
        }
      }
    }
  }
  auto issue = [&](int k) {  // copy halo plane k (z = z0 - 1 + k) into stage k % ZS
    if (k < zc + 2) {
      int z = z0 - 1 + k;  // -1 <= z <= n2
      z = z < 0 ? z + n2 : (z >= n2 ? z - n2 : z);
      const float* base = s + nxy * z;
      float* st = stage[k % ZS];
      if (BULK) {
        if (threadIdx.x < 32) {
          if (threadIdx.x == 0)
            mbar_arrive_expect_tx(&full[k % ZS], (unsigned)((ZY + 2) * len * 4));
          __syncwarp();
          if (kind[0] == 1) {
            fence_proxy_async_smem();
            bulk_load(st + dofs[0], base + yoff[0] + xs[0], (unsigned)(len * 4), &full[k % ZS]);
          }
        } else if (kind[0] == 3) {
          cp_async4(st + dofs[0], base + yoff[0] + xs[0]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < ZOPT; ++j) {
          const float* sr = base + yoff[j];
          if (kind[j] == 1) {
            cp_async16(st + dofs[j], sr + xs[j]);
          } else if (kind[j] == 3) {
            cp_async4(st + dofs[j], sr + xs[j]);
          } else if (kind[j] == 2) {
            for (int e = 0; e < 4; ++e) cp_async4(st + dofs[j] + e, sr + wrapi(xs[j] + e, n0));
          }
        }
      }
    }
    cp_async_commit();  // an empty group keeps the group count uniform
  };
#pragma unroll
  for (int k = 0; k < ZS - 1; ++k) issue(k);

  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int gx = x0 + 4 * tx, gy = y0 + 2 * ty;
  float pm[8], p0[8];  // y results of the two previous planes: [row * 4 + x]
#pragma unroll
  for (int i = 0; i < 8; ++i) pm[i] = p0[i] = 0.f;
  for (int k = 0; k < zc + 2; ++k) {
    cp_async_wait<ZS - 2>();  // this thread's copies of plane k have landed
    if (BULK) {
      // and the bulk copies of every thread's rows; then stage (k - 1) % ZS
      // is no longer read
      if (!stage_landed(full, k, zc + 2, status)) return;
    } else {
      __syncthreads();  // everyone's have; stage (k - 1) % ZS is no longer read
    }
    issue(k + ZS - 1);
    const float* a = stage[k % ZS] + 2 * ty * ZROW + 4 * tx + 3;  // row y - 1, column x - 1
    float xf[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {  // x sub-pass of rows y - 1 .. y + 2
      const float l = a[r * ZROW];
      const float4 m = *reinterpret_cast<const float4*>(a + r * ZROW + 1);
      const float rr = a[r * ZROW + 5];
      xf[r][0] = b3(l, m.x, m.y);
      xf[r][1] = b3(m.x, m.y, m.z);
      xf[r][2] = b3(m.y, m.z, m.w);
      xf[r][3] = b3(m.z, m.w, rr);
    }
    float p1[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // y sub-pass of rows y, y + 1
      p1[i] = b3(xf[0][i], xf[1][i], xf[2][i]);
      p1[4 + i] = b3(xf[1][i], xf[2][i], xf[3][i]);
    }
    if (k >= 2) {  // z sub-pass of plane z0 + k - 2
      const int z = z0 + k - 2;
#pragma unroll
      for (int rw = 0; rw < 2; ++rw) {
        if (gy + rw >= n1) continue;
        float o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = b3(pm[4 * rw + i], p0[4 * rw + i], p1[4 * rw + i]);
        float* q = d + gx + (long long)n0 * (gy + rw) + nxy * z;
        if (vec && gx + 3 < n0) {
          *reinterpret_cast<float4*>(q) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (gx + i < n0) q[i] = o[i];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      pm[i] = p0[i];
      p0[i] = p1[i];
    }
  }
  cp_async_wait<0>();
}

// One full 2D Binomial2 pass (x, then y sub-pass) of one plane src -> dst,
// marching along y: a block of 256 threads owns YX = 1024 x-points (4 per
// thread) over a run of `yrun` rows.  Each row plus its one-point periodic x
// halo goes through a ring of ZS shared-memory stages, ZS - 1 rows ahead of
// the one being filtered.  BULK (rows of a multiple of 4 floats, 16-byte
// aligned planes, a status word): the row's points arrive by one bulk copy
// (`cp.async.bulk`, issued by thread 0, completing on the stage's mbarrier)
// and its two halo points by 4-byte cp.async; otherwise every thread copies
// by cp.async (16-byte copies for aligned interior chunks, 4-byte ones for the
// halo and for ragged or wrapped chunks).  A thread runs the x sub-pass of its
// 4 points from one 16-byte and two 4-byte shared loads and keeps the last
// three results for the y sub-pass.  Every output goes through the same
// arithmetic, in the same order, as two k_filter_axis sub-passes.
// Grid: x = x-column + columns x run, y = plane.
constexpr int YX = 1024;
constexpr int YROW = YX + 8;  // stage row: [3] left halo, [4, 4 + YX) interior, [4 + YX] right

template <bool BULK>
__global__ void __launch_bounds__(256) k_filter_y2(const float* __restrict__ src,
                                                  float* __restrict__ dst, const GridDev g,
                                                  int ncx, int yrun, int vec, int* status) {
  __shared__ __align__(16) float stage[ZS][YROW];
  __shared__ unsigned long long full[ZS];  // BULK: the stage's row has landed
  const int n0 = g.n[0], n1 = g.n[1];
  const int col = blockIdx.x % ncx, run = blockIdx.x / ncx;
  const int x0 = col * YX, y0 = run * yrun;
  const int yc = min(yrun, n1 - y0);  // rows y0 .. y0 + yc - 1 are written
  const long long P = g.plane;
  const float* s = src + (long long)blockIdx.y * P;
  float* d = dst + (long long)blockIdx.y * P;
  const int t = threadIdx.x;
  const int len = min(YX, n0 - x0);  // interior points of the column's rows
  // this thread's copies, the same for every row: interior chunk t (x0 + 4t ..
  // x0 + 4t + 3), and for threads 0 and 1 the left and right halo point (BULK:
  // the right one right after the last interior point, where a ragged
  // column's x sub-pass reads it; thread 0 also issues the row's bulk copy)
  const int xs = x0 + 4 * t;
  const bool v16 = vec && xs + 3 < n0;
  const int hx = t == 0 ? wrapi(x0 - 1, n0) : wrapi(BULK ? x0 + len : x0 + YX, n0);
  const int hcol = t == 0 ? 3 : 4 + (BULK ? len : YX);
  if (BULK) {
    if (t == 0) {
      for (int i = 0; i < ZS; ++i) mbar_init(&full[i], 1);
      mbar_init_fence();
    }
    __syncthreads();  // the barriers are initialised before any copy or wait
  }
  auto issue = [&](int k) {  // copy halo row k (y = y0 - 1 + k) into stage k % ZS
    if (k < yc + 2) {
      int y = y0 - 1 + k;  // -1 <= y <= n1
      y = y < 0 ? y + n1 : (y >= n1 ? y - n1 : y);
      const float* row = s + (long long)n0 * y;
      float* st = stage[k % ZS];
      if (BULK) {
        if (t == 0) {
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&full[k % ZS], (unsigned)(len * 4));
          bulk_load(st + 4, row + x0, (unsigned)(len * 4), &full[k % ZS]);
        }
      } else if (v16) {
        cp_async16(st + 4 + 4 * t, row + xs);
      } else {
        for (int e = 0; e < 4; ++e) cp_async4(st + 4 + 4 * t + e, row + wrapi(xs + e, n0));
      }
      if (t < 2) cp_async4(st + hcol, row + hx);
    }
    cp_async_commit();  // an empty group keeps the group count uniform
  };
#pragma unroll
  for (int k = 0; k < ZS - 1; ++k) issue(k);

  float pm[4] = {0.f, 0.f, 0.f, 0.f}, p0[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < yc + 2; ++k) {
    cp_async_wait<ZS - 2>();  // this thread's copies of row k have landed
    if (BULK) {
      // and the row's bulk copy; then stage (k - 1) % ZS is no longer read
      if (!stage_landed(full, k, yc + 2, status)) return;
    } else {
      __syncthreads();  // everyone's have; stage (k - 1) % ZS is no longer read
    }
    issue(k + ZS - 1);
    const float* a = stage[k % ZS] + 4 * t + 3;  // column x - 1
    const float l = a[0];
    const float4 m = *reinterpret_cast<const float4*>(a + 1);
    const float r = a[5];
    const float p1[4] = {b3(l, m.x, m.y), b3(m.x, m.y, m.z), b3(m.y, m.z, m.w), b3(m.z, m.w, r)};
    if (k >= 2) {  // y sub-pass of row y0 + k - 2
      float o[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) o[i] = b3(pm[i], p0[i], p1[i]);
      float* q = d + (long long)n0 * (y0 + k - 2) + xs;
      if (v16) {
        *reinterpret_cast<float4*>(q) = make_float4(o[0], o[1], o[2], o[3]);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (xs + i < n0) q[i] = o[i];
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      pm[i] = p0[i];
      p0[i] = p1[i];
    }
  }
  cp_async_wait<0>();
}

// Offsets (elements) of the lattice points a-2, a-1, a+1, a+2 along an axis of
// n points with stride s, periodic.
struct Nb {
  long long m2, m1, p1, p2;
};
__device__ __forceinline__ Nb neighbours(int a, int n, long long s) {
  Nb r;
  r.m2 = (long long)(wrapi(a - 2, n) - a) * s;
  r.m1 = (long long)(wrapi(a - 1, n) - a) * s;
  r.p1 = (long long)(wrapi(a + 1, n) - a) * s;
  r.p2 = (long long)(wrapi(a + 2, n) - a) * s;
  return r;
}
// fourth-order staggered differences (FDTD4): at the point half a cell up
// (forward) or down (backward) the axis, coefficients 9/8 and -1/24
__device__ __forceinline__ float d4p(const float* A, long long i, const Nb& b) {
  return 1.125f * (A[i + b.p1] - A[i]) - (1.0f / 24.0f) * (A[i + b.p2] - A[i + b.m1]);
}
__device__ __forceinline__ float d4m(const float* A, long long i, const Nb& b) {
  return 1.125f * (A[i] - A[i + b.m1]) - (1.0f / 24.0f) * (A[i + b.p1] - A[i + b.m2]);
}

// FDTD4 versions of the two updates (same structure as above, wider stencil).
template <int D>
__global__ void k_b_half4(float* __restrict__ F, const GridDev g, float hc, int zero_j) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  FOR_ROWS(j, k) {
    const long long idx = (long long)i + (long long)n0 * (j + (long long)n1 * k);
    const Nb nx = neighbours(i, g.n[0], 1);
    const Nb ny = neighbours(j, g.n[1], g.n[0]);
    const Nb nz = neighbours(k, g.n[2], (long long)g.n[0] * g.n[1]);
    const float* Ex = F + EX * P;
    const float* Ey = F + EY * P;
    const float* Ez = F + EZ * P;
    float cx = 0.f, cy = 0.f, cz = 0.f;
    cy -= d4p(Ez, idx, nx);
    cz += d4p(Ey, idx, nx);
    if (D >= 2) {
      cx += d4p(Ez, idx, ny);
      cz -= d4p(Ex, idx, ny);
    }
    if (D >= 3) {
      cx -= d4p(Ey, idx, nz);
      cy += d4p(Ex, idx, nz);
    }
    F[BX * P + idx] = fmaf(-hc, cx, F[BX * P + idx]);
    F[BY * P + idx] = fmaf(-hc, cy, F[BY * P + idx]);
    F[BZ * P + idx] = fmaf(-hc, cz, F[BZ * P + idx]);
    if (zero_j) {
      F[JX * P + idx] = 0.f;
      F[JY * P + idx] = 0.f;
      F[JZ * P + idx] = 0.f;
    }
  }
}

template <int D>
__global__ void k_e_update4(float* __restrict__ F, const GridDev g, float c) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  FOR_ROWS(j, k) {
    const long long idx = (long long)i + (long long)n0 * (j + (long long)n1 * k);
    const Nb nx = neighbours(i, g.n[0], 1);
    const Nb ny = neighbours(j, g.n[1], g.n[0]);
    const Nb nz = neighbours(k, g.n[2], (long long)g.n[0] * g.n[1]);
    const float* Bx = F + BX * P;
    const float* By = F + BY * P;
    const float* Bz = F + BZ * P;
    float cx = 0.f, cy = 0.f, cz = 0.f;
    cy -= d4m(Bz, idx, nx);
    cz += d4m(By, idx, nx);
    if (D >= 2) {
      cx += d4m(Bz, idx, ny);
      cz -= d4m(Bx, idx, ny);
    }
    if (D >= 3) {
      cx -= d4m(By, idx, nz);
      cy += d4m(Bx, idx, nz);
    }
    F[EX * P + idx] = fmaf(c, cx, F[EX * P + idx]) - F[JX * P + idx];
    F[EY * P + idx] = fmaf(c, cy, F[EY * P + idx]) - F[JY * P + idx];
    F[EZ * P + idx] = fmaf(c, cz, F[EZ * P + idx]) - F[JZ * P + idx];
  }
}

// Launch of the four-points-per-thread kernels: rows of n0 / 4 threads.
static bool x4_ok(const GridDev& g, const float* F) {
  return g.n[0] % 4 == 0 && (reinterpret_cast<uintptr_t>(F) & 15) == 0;
}
static RowLaunch row_launch_x4(const GridDev& g) {
  GridDev q = g;
  q.n[0] = g.n[0] / 4;
  return row_launch(q);
}

cudaError_t launch_b_half(const GridDev& g, float* F, int zero_j, cudaStream_t st) {
  const float hc = 0.5f * g.c;
  if (g.order == 2 && x4_ok(g, F)) {
    const RowLaunch L = row_launch_x4(g);
    switch (g.dim) {
      case 1: k_b_half_x4<1><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
      case 2: k_b_half_x4<2><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
      case 3: k_b_half_x4<3><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  const RowLaunch L = row_launch(g);
  switch (g.dim * 10 + g.order) {
    case 12: k_b_half<1><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
    case 22: k_b_half<2><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
    case 32: k_b_half<3><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
    case 14: k_b_half4<1><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
    case 24: k_b_half4<2><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
    case 34: k_b_half4<3><<<L.grid, L.threads, 0, st>>>(F, g, hc, zero_j); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

bool fields_small_ok(const GridDev& g) {
  return PIC_SMALL_FIELDS && g.order == 2 && g.plane <= kSmallFieldCells;
}

cudaError_t launch_fields_small(const GridDev& g, float* F, cudaStream_t st, int chain) {
  const int threads = g.plane < 1024 ? (int)((g.plane + 31) / 32 * 32) : 1024;
  switch (g.dim) {
    case 1: k_fields_small<1><<<1, threads, 0, st>>>(F, g, 0.5f * g.c, g.c, chain); break;
    case 2: k_fields_small<2><<<1, threads, 0, st>>>(F, g, 0.5f * g.c, g.c, chain); break;
    case 3: k_fields_small<3><<<1, threads, 0, st>>>(F, g, 0.5f * g.c, g.c, chain); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_e_update(const GridDev& g, float* F, cudaStream_t st) {
  if (g.order == 2 && x4_ok(g, F)) {
    const RowLaunch L = row_launch_x4(g);
    switch (g.dim) {
      case 1: k_e_update_x4<1><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
      case 2: k_e_update_x4<2><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
      case 3: k_e_update_x4<3><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  const RowLaunch L = row_launch(g);
  switch (g.dim * 10 + g.order) {
    case 12: k_e_update<1><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
    case 22: k_e_update<2><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
    case 32: k_e_update<3><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
    case 14: k_e_update4<1><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
    case 24: k_e_update4<2><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
    case 34: k_e_update4<3><<<L.grid, L.threads, 0, st>>>(F, g, g.c); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_filter(const GridDev& g, const T* src, T* dst, int ncomp, int axis,
                                 cudaStream_t st) {
  if (axis < 0 || axis >= g.dim || g.n[1] > 65535 || (long long)g.n[2] * ncomp > 65535)
    return cudaErrorInvalidValue;
  const dim3 grid((g.n[0] + 127) / 128, g.n[1], g.n[2] * ncomp);
  k_filter_axis<T><<<grid, 128, 0, st>>>(src, dst, g, axis);
  return cudaGetLastError();
}

cudaError_t launch_filter_f32(const GridDev& g, const float* src, float* dst, int ncomp, int axis,
                              cudaStream_t st) {
  return launch_filter<float>(g, src, dst, ncomp, axis, st);
}

template <int D, int TX, int TY, int TZ>
static cudaError_t launch_pass(const GridDev& g, const float* src, float* dst, int ncomp,
                               cudaStream_t st) {
  const int ntx = (g.n[0] + TX - 1) / TX;
  const int nty = D >= 2 ? (g.n[1] + TY - 1) / TY : 1;
  const int ntz = D >= 3 ? (g.n[2] + TZ - 1) / TZ : 1;
  const long long tiles = (long long)ntx * nty * ntz;
  if (tiles > 0x7fffffffLL || ncomp > 65535) return cudaErrorInvalidValue;
  k_filter_pass<D, TX, TY, TZ><<<dim3((unsigned)tiles, (unsigned)ncomp), 256, 0, st>>>(
      src, dst, g, ntx, nty);
  return cudaGetLastError();
}

// The z-marching 3D pass.  The z-runs are as long as they can be with every
// block resident at once (one wave: no block re-reads a run's two halo planes
// from DRAM after its neighbour has evicted them, no tail wave); a grid with
// more columns than resident blocks gets one run per column.
static cudaError_t launch_pass_z3(const GridDev& g, const float* src, float* dst, int ncomp,
                                  cudaStream_t st, int* status) {
  static int resident = 0;
  if (resident == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_z3<true>, 256, 0);
    resident = sms * per_sm > 0 ? sms * per_sm : 1;
  }
  const int ncx = (g.n[0] + ZX - 1) / ZX, ncy = (g.n[1] + ZY - 1) / ZY;
  const long long streams = (long long)ncx * ncy * ncomp;
  long long runs = resident / streams;
  if (runs < 1) runs = 1;
  if (runs > g.n[2]) runs = g.n[2];
  const int zrun = (int)((g.n[2] + runs - 1) / runs);
  const long long blocks = (long long)ncx * ncy * ((g.n[2] + zrun - 1) / zrun);
  if (blocks > 0x7fffffffLL || ncomp > 65535) return cudaErrorInvalidValue;
  // 16-byte copies and stores need 16-byte aligned rows: plane bases and n0
  // multiples of 4 floats
  const int vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 &&
                  g.n[0] % 4 == 0 && g.plane % 4 == 0;
  // bulk row copies where a status word can report a wait that ran out
  const dim3 grid((unsigned)blocks, (unsigned)ncomp);
  if (vec && status && PIC_BULK_FILTER)
    k_filter_z3<true><<<grid, 256, 0, st>>>(src, dst, g, ncx, ncy, zrun, vec, status);
  else
    k_filter_z3<false><<<grid, 256, 0, st>>>(src, dst, g, ncx, ncy, zrun, vec, status);
  return cudaGetLastError();
}

// The y-marching 2D pass; runs as long as one wave of resident blocks allows.
static cudaError_t launch_pass_y2(const GridDev& g, const float* src, float* dst, int ncomp,
                                  cudaStream_t st, int* status) {
  static int resident = 0;
  if (resident == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_y2<true>, 256, 0);
    resident = sms * per_sm > 0 ? sms * per_sm : 1;
  }
  const int ncx = (g.n[0] + YX - 1) / YX;
  const long long streams = (long long)ncx * ncomp;
  long long runs = resident / streams;
  if (runs < 1) runs = 1;
  if (runs > g.n[1]) runs = g.n[1];
  const int yrun = (int)((g.n[1] + runs - 1) / runs);
  const long long blocks = (long long)ncx * ((g.n[1] + yrun - 1) / yrun);
  if (blocks > 0x7fffffffLL || ncomp > 65535) return cudaErrorInvalidValue;
  const int vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 &&
                  g.n[0] % 4 == 0 && g.plane % 4 == 0;
  const dim3 grid((unsigned)blocks, (unsigned)ncomp);
  if (vec && status && PIC_BULK_FILTER)
    k_filter_y2<true><<<grid, 256, 0, st>>>(src, dst, g, ncx, yrun, vec, status);
  else
    k_filter_y2<false><<<grid, 256, 0, st>>>(src, dst, g, ncx, yrun, vec, status);
  return cudaGetLastError();
}

cudaError_t launch_filter_pass_f32(const GridDev& g, const float* src, float* dst, int ncomp,
                                   cudaStream_t st, int* status) {
  switch (g.dim) {
    case 1: return launch_pass<1, 1024, 1, 1>(g, src, dst, ncomp, st);
    case 2: return launch_pass_y2(g, src, dst, ncomp, st, status);
    case 3: return launch_pass_z3(g, src, dst, ncomp, st, status);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_filter_f64(const GridDev& g, const double* src, double* dst, int ncomp,
                              int axis, cudaStream_t st) {
  return launch_filter<double>(g, src, dst, ncomp, axis, st);
}

}  // namespace pic

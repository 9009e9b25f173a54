// FDTD2 field update and Binomial2 current filter (arXiv:1906.06306,
// Sect. 2.3.1, Eqs. (fdE), (fdB), Table 2) on periodic Yee planes.
// One thread per lattice point, x fastest, so every plane is streamed with
// coalesced loads; neighbours one point away come from the same or adjacent
// rows and hit L1/L2.  The filter runs as one 3-point sub-pass per gridded
// axis (x, then y, then z), the order in which the paper's filter is applied.
#include "pic_kernels.h"

namespace pic {

static unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > (1LL << 20)) b = 1LL << 20;
  return (unsigned)(b < 1 ? 1 : b);
}

// B -= (c/2) curl+ E (forward differences: B sits half a cell above E), and,
// when zero_j is set, clear J for the deposit that follows.
template <int D>
__global__ void k_b_half(float* __restrict__ F, const GridDev g, float hc, int zero_j) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n0);
    const long long r = idx / n0;
    const int j = (int)(r % n1), k = (int)(r / n1);
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
}

// E += c curl- B - J (backward differences: E sits half a cell below B).
template <int D>
__global__ void k_e_update(float* __restrict__ F, const GridDev g, float c) {
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const long long P = g.plane;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n0);
    const long long r = idx / n0;
    const int j = (int)(r % n1), k = (int)(r / n1);
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
// Grid: x = tile index, y = plane.
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
  const long long P = g.plane;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.n[0]);
    const long long r = idx / g.n[0];
    const int j = (int)(r % g.n[1]), k = (int)(r / g.n[1]);
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
  const long long P = g.plane;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.n[0]);
    const long long r = idx / g.n[0];
    const int j = (int)(r % g.n[1]), k = (int)(r / g.n[1]);
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

cudaError_t launch_b_half(const GridDev& g, float* F, int zero_j, cudaStream_t st) {
  const unsigned nb = grid_for(g.plane, 256);
  const float hc = 0.5f * g.c;
  switch (g.dim * 10 + g.order) {
    case 12: k_b_half<1><<<nb, 256, 0, st>>>(F, g, hc, zero_j); break;
    case 22: k_b_half<2><<<nb, 256, 0, st>>>(F, g, hc, zero_j); break;
    case 32: k_b_half<3><<<nb, 256, 0, st>>>(F, g, hc, zero_j); break;
    case 14: k_b_half4<1><<<nb, 256, 0, st>>>(F, g, hc, zero_j); break;
    case 24: k_b_half4<2><<<nb, 256, 0, st>>>(F, g, hc, zero_j); break;
    case 34: k_b_half4<3><<<nb, 256, 0, st>>>(F, g, hc, zero_j); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_e_update(const GridDev& g, float* F, cudaStream_t st) {
  const unsigned nb = grid_for(g.plane, 256);
  switch (g.dim * 10 + g.order) {
    case 12: k_e_update<1><<<nb, 256, 0, st>>>(F, g, g.c); break;
    case 22: k_e_update<2><<<nb, 256, 0, st>>>(F, g, g.c); break;
    case 32: k_e_update<3><<<nb, 256, 0, st>>>(F, g, g.c); break;
    case 14: k_e_update4<1><<<nb, 256, 0, st>>>(F, g, g.c); break;
    case 24: k_e_update4<2><<<nb, 256, 0, st>>>(F, g, g.c); break;
    case 34: k_e_update4<3><<<nb, 256, 0, st>>>(F, g, g.c); break;
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

cudaError_t launch_filter_pass_f32(const GridDev& g, const float* src, float* dst, int ncomp,
                                   cudaStream_t st) {
  switch (g.dim) {
    case 1: return launch_pass<1, 1024, 1, 1>(g, src, dst, ncomp, st);
    case 2: return launch_pass<2, 32, 32, 1>(g, src, dst, ncomp, st);
    case 3: return launch_pass<3, 32, 8, 8>(g, src, dst, ncomp, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_filter_f64(const GridDev& g, const double* src, double* dst, int ncomp,
                              int axis, cudaStream_t st) {
  return launch_filter<double>(g, src, dst, ncomp, axis, st);
}

}  // namespace pic

// Shock boundaries of the paper's collisionless-shock set-up (arXiv:1906.06306,
// Sect. 4.2): the conducting wall's field boundary and the receding
// injector's particle source.  Both are small next to the step (a few planes
// of cells, a thin slab of particles) and run as plain grid-stride kernels.
#include <cmath>

#include "pic_kernels.h"

namespace pic {

static unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > (1LL << 20)) b = 1LL << 20;
  return (unsigned)(b < 1 ? 1 : b);
}

// Perfect conductor on the node plane x = w: Ey = Ez = 0 at i = w, and the
// cells i < w hold the mirror image of the plasma side (tangential E and
// normal B odd, normal E and tangential B even about x = w).  Integer-x
// components (Ey, Ez, Bx) at i take the value at 2w - i; half-integer ones
// (Ex, By, Bz, stored at i for x = i + 1/2) the value at 2w - 1 - i.  E and
// B at i >= i_zero are zeroed.  The sources 2w - i > w and 2w - 1 - i >= w
// lie below i_zero (2w < i_zero) and are never written here, so the threads
// do not race.
__global__ void k_wall_fields(float* __restrict__ F, const GridDev g, int w, int i_zero) {
  const int n0 = g.n[0];
  const long long P = g.plane;
  const int cols = w + 1 + (n0 - i_zero);
  const long long rows = P / n0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < rows * cols;
       idx += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(idx % cols);
    const long long row = (idx / cols) * n0;
    if (col < w) {
      const long long a = row + col, ri = row + (2 * w - col), rh = row + (2 * w - 1 - col);
      F[EX * P + a] = F[EX * P + rh];
      F[BY * P + a] = F[BY * P + rh];
      F[BZ * P + a] = F[BZ * P + rh];
      F[EY * P + a] = -F[EY * P + ri];
      F[EZ * P + a] = -F[EZ * P + ri];
      F[BX * P + a] = -F[BX * P + ri];
    } else if (col == w) {
      F[EY * P + row + w] = 0.f;
      F[EZ * P + row + w] = 0.f;
    } else {
      const long long a = row + i_zero + (col - w - 1);
#pragma unroll
      for (int c = EX; c <= BZ; ++c) F[c * P + a] = 0.f;
    }
  }
}

cudaError_t launch_wall_fields(const GridDev& g, float* F, int wall, int i_zero, cudaStream_t st) {
  const long long work = (g.plane / g.n[0]) * (long long)(wall + 1 + (g.n[0] - i_zero));
  k_wall_fields<<<grid_for(work, 256), 256, 0, st>>>(F, g, wall, i_zero);
  return cudaGetLastError();
}

// Injection of the particles that crossed the receding injector in one step:
// thread t takes the t-th particle of the runs (located by the prefix
// `first`), reads template particle k of its species and writes it at output
// index run.out + (k - run.k0) with x = x_t + run.shift, x_t = i_t + off_x
// (double precision, as the host computed the runs); y, z cells, offsets and
// u are copied.
template <int D>
__global__ void k_inject(const InjectParams P) {
  const long long total = P.first[P.nruns];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int r = 0;
    while (r + 1 < P.nruns && t >= P.first[r + 1]) ++r;
    const InjectRun R = P.run[r];
    const int s = R.s;
    const long long k = R.k0 + (t - P.first[r]);
    const long long o = R.out + (t - P.first[r]);
    const long long tn = P.tn[s], ld = P.ld[s];
    const int tc = P.tcell[s][k];
    const int ti = tc % P.lt, trow = tc / P.lt;  // trow = j + ny k
    const double xt = (double)ti + (double)P.toff[s][k];
    const double pos = xt + R.shift;
    double cx = floor(pos);
    float ox = __double2float_rn(pos - cx);
    if (ox == 1.0f) {
      cx += 1.0;
      ox = 0.0f;
    }
    P.cell[s][o] = (int)cx + P.g.n[0] * trow;
    P.off[s][o] = ox;
#pragma unroll
    for (int d = 1; d < D; ++d) P.off[s][d * ld + o] = P.toff[s][d * tn + k];
#pragma unroll
    for (int a = 0; a < 3; ++a) P.u[s][a * ld + o] = P.tu[s][a * tn + k];
  }
}

cudaError_t launch_inject(const InjectParams& P, cudaStream_t st) {
  const long long total = P.first[P.nruns];
  if (total == 0) return cudaSuccess;
  const unsigned nb = grid_for(total, 256);
  switch (P.g.dim) {
    case 1: k_inject<1><<<nb, 256, 0, st>>>(P); break;
    case 2: k_inject<2><<<nb, 256, 0, st>>>(P); break;
    case 3: k_inject<3><<<nb, 256, 0, st>>>(P); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pic

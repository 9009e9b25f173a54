// Diagnostics of the PIC state, accumulated in double precision on the GPU:
// field and kinetic energies, the first-order charge on the nodes and the
// discrete Gauss residual div E - rho of Appendix B (arXiv:1906.06306).
#include "pic_kernels.h"

namespace pic {

static unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

__global__ void k_field_energy(const float* __restrict__ F, long long P, double* acc) {
  __shared__ double sh[32];
  double se = 0.0, sb = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double e = F[(EX + a) * P + i], b = F[(BX + a) * P + i];
      se += e * e;
      sb += b * b;
    }
  }
  se = block_sum(se, sh);
  sb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&acc[0], 0.5 * se);
    atomicAdd(&acc[1], 0.5 * sb);
  }
}

// m c^2 (gamma - 1) with gamma - 1 = u^2 / (gamma + 1)
__global__ void k_kinetic(const float* __restrict__ u, long long n, long long ld, double mc2,
                          double* acc) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double a = u[p], b = u[ld + p], c = u[2 * ld + p];
    const double u2 = a * a + b * b + c * c;
    s += u2 / (sqrt(1.0 + u2) + 1.0);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) atomicAdd(acc, mc2 * s);
}

// charge q with weights (1 - w, w) per gridded axis onto the 2^D nodes
template <int D>
__global__ void k_rho(const GridDev g, const int* __restrict__ cell, const float* __restrict__ off,
                      long long n, long long ld, double q, double* rho) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int c = cell[p];
    if (c < 0 || (long long)c >= g.plane) continue;
    int ijk[3];
    ijk[0] = c % g.n[0];
    const int r = c / g.n[0];
    ijk[1] = r % g.n[1];
    ijk[2] = r / g.n[1];
    double w[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < D; ++d) w[d] = off[d * ld + p];
#pragma unroll
    for (int corner = 0; corner < (1 << D); ++corner) {
      double wt = q;
      int id[3] = {ijk[0], ijk[1], ijk[2]};
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int o = (corner >> d) & 1;
        wt *= o ? w[d] : 1.0 - w[d];
        id[d] = o ? wrap1(id[d] + 1, g.n[d]) : id[d];
      }
      atomicAdd(&rho[id[0] + (long long)g.n[0] * (id[1] + (long long)g.n[1] * id[2])], wt);
    }
  }
}

// res = div- E - rho on the nodes with i_lo <= i < i_hi; max |res| (bit
// pattern of a non-negative double, which orders like the value) and sum res^2
template <int D>
__global__ void k_gauss(const GridDev g, const float* __restrict__ F, const double* __restrict__ rho,
                        int i_lo, int i_hi, unsigned long long* acc_max, double* acc_sq) {
  __shared__ double sh[32];
  __shared__ unsigned long long shm;
  if (threadIdx.x == 0) shm = 0ull;
  const long long P = g.plane;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  double sq = 0.0, mx = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n0);
    const long long r = idx / n0;
    const int j = (int)(r % n1), k = (int)(r / n1);
    if (i < i_lo || i >= i_hi) continue;
    double div = (double)F[EX * P + idx] - (double)F[EX * P + idx - ((i > 0) ? 1 : 1 - n0)];
    if (D >= 2)
      div += (double)F[EY * P + idx] -
             (double)F[EY * P + idx - ((j > 0) ? n0 : (long long)n0 * (1 - n1))];
    if (D >= 3)
      div += (double)F[EZ * P + idx] -
             (double)F[EZ * P + idx - ((k > 0) ? (long long)n0 * n1 : (long long)n0 * n1 * (1 - n2))];
    const double res = div - rho[idx];
    sq += res * res;
    mx = fmax(mx, fabs(res));
  }
  sq = block_sum(sq, sh);
  __syncthreads();
  atomicMax(&shm, (unsigned long long)__double_as_longlong(mx));
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(acc_sq, sq);
    atomicMax(acc_max, shm);
  }
}

cudaError_t launch_field_energy(const GridDev& g, const float* F, double* acc, cudaStream_t st) {
  k_field_energy<<<blocks_for(g.plane), 256, 0, st>>>(F, g.plane, acc);
  return cudaGetLastError();
}

cudaError_t launch_kinetic(const float* u, long long n, long long ld, double mc2, double* acc,
                           cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_kinetic<<<blocks_for(n), 256, 0, st>>>(u, n, ld, mc2, acc);
  return cudaGetLastError();
}

cudaError_t launch_rho(const GridDev& g, const int* cell, const float* off, long long n,
                       long long ld, double q, double* rho, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned nb = blocks_for(n);
  switch (g.dim) {
    case 1: k_rho<1><<<nb, 256, 0, st>>>(g, cell, off, n, ld, q, rho); break;
    case 2: k_rho<2><<<nb, 256, 0, st>>>(g, cell, off, n, ld, q, rho); break;
    case 3: k_rho<3><<<nb, 256, 0, st>>>(g, cell, off, n, ld, q, rho); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gauss(const GridDev& g, const float* F, const double* rho, int i_lo, int i_hi,
                         unsigned long long* acc_max, double* acc_sq, cudaStream_t st) {
  const unsigned nb = blocks_for(g.plane);
  switch (g.dim) {
    case 1: k_gauss<1><<<nb, 256, 0, st>>>(g, F, rho, i_lo, i_hi, acc_max, acc_sq); break;
    case 2: k_gauss<2><<<nb, 256, 0, st>>>(g, F, rho, i_lo, i_hi, acc_max, acc_sq); break;
    case 3: k_gauss<3><<<nb, 256, 0, st>>>(g, F, rho, i_lo, i_hi, acc_max, acc_sq); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// One warp waits on a shared-memory barrier that nothing completes: its
// bounded wait gives up after about a second of SM clock and sets ST_TIMEOUT
// in the status word, as a particle block's wait on a tensor copy that never
// landed would.  No copy is in flight, so leaving is safe.
__global__ void k_wait_probe(int* status) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  mbar_wait(&bar, 0, status);
}

cudaError_t launch_wait_probe(int* status, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(status);
  return cudaGetLastError();
}

}  // namespace pic

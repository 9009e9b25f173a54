// Allocation-free Binomial2 filter entry point (see include/pic.h).
//
// The filter ping-pongs between the caller's J planes and a scratch copy of
// them.  Here the scratch is a fixed array in device global memory that is part
// of the library image, so a call allocates nothing.  Host code cannot use the
// array's name as a device address (it only names a host-side stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress.
#include <mutex>

#include "pic.h"
#include "pic_kernels.h"

namespace {

__device__ __align__(256) float g_filter_scratch[PIC_FILTER_STATIC_MAX_FLOATS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of g_filter_scratch on the current device (looked up on the
// first call for that device).
cudaError_t scratch_address(float** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_filter_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

pic_status fail(pic_status s, const char* msg) {
  pic::set_global_error(msg);
  return s;
}

}  // namespace

extern "C" pic_status pic_filter_current_static(const pic_grid* grid, float* J, int passes,
                                                void* stream) {
  pic::set_global_error("");
  if (!grid || !J) return fail(PIC_ERR_ARG, "grid or J is NULL");
  if (grid->dim < 1 || grid->dim > 3) return fail(PIC_ERR_ARG, "dim must be 1, 2 or 3");
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  long long ncell = 1;
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1) return fail(PIC_ERR_ARG, "grid extents must be >= 1");
    if (d >= grid->dim && n[d] != 1)
      return fail(PIC_ERR_ARG, "extents of non-gridded dimensions must be 1");
    ncell *= n[d];
  }
  if (passes < 0) return fail(PIC_ERR_ARG, "passes must be >= 0");
  if (3 * ncell > PIC_FILTER_STATIC_MAX_FLOATS)
    return fail(PIC_ERR_ARG,
                "3*nx*ny*nz exceeds PIC_FILTER_STATIC_MAX_FLOATS (the static scratch size); "
                "use pic_filter_current on a context instead");
  if (passes == 0) return PIC_OK;
  float* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return fail(PIC_ERR_CUDA, cudaGetErrorString(e));
  pic::GridDev g{};
  g.dim = grid->dim;
  g.n[0] = n[0];
  g.n[1] = n[1];
  g.n[2] = n[2];
  g.plane = ncell;
  g.order = 2;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the context path's fused passes (every axis in one launch), ping-ponging
  // between J and the static scratch
  float* a = J;
  float* b = scratch;
  for (int p = 0; p < passes; ++p) {
    e = pic::launch_filter_pass_f32(g, a, b, 3, st, nullptr);
    if (e != cudaSuccess) return fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    float* t = a;
    a = b;
    b = t;
  }
  if (a != J) {
    e = cudaMemcpyAsync(J, a, sizeof(float) * 3 * ncell, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(PIC_ERR_CUDA, cudaGetErrorString(e));
  }
  return PIC_OK;
}

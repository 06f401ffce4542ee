// Cloud-in-cell deposit that allocates nothing (pic_deposit_static).
//
// Who needs it: code that may not call cudaMalloc / cudaFree at the point
// where it deposits -- for example a host program whose device memory is
// already fully reserved by another runtime's pool, or a latency-critical
// loop that cannot afford the device-wide synchronisation an allocation or
// release can cause.  Such a caller passes its own input and output buffers;
// the only scratch this entry point uses is the fixed-size accumulator below,
// which lives in the library image on every GPU that loads the library,
// until the process exits.
//
// The arithmetic is the one of the context-based deposit: each particle's
// four bilinear shares are quantised to 2^-20 of its weight (three rounded
// to nearest-even, the fourth the remainder) and summed exactly in 64-bit
// integers, so the result does not depend on particle order.
#include <cuda_runtime.h>

#include "picgb.h"

namespace {

constexpr long long kStaticMaxNodes = 1ll << 20;   // 8 MiB of 64-bit accumulators
constexpr int kThreads = 256;

// The scratch.  In host code this name is only a stand-in for the device
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned long long g_deposit_scratch[kStaticMaxNodes];

// Device address of the scratch in the current context.  It is looked up
// on every call (a cheap host-side query): a cached address would go stale
// when the caller switches to another context of the same device (a
// runtime that drives its own, non-primary context) or after the device
// was reset and the module loaded again.
pic_status scratch_address(unsigned long long **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_deposit_scratch) != cudaSuccess || !p) return PIC_ECUDA;
  *out = static_cast<unsigned long long *>(p);
  return PIC_OK;
}

__global__ void k_clear(unsigned long long *acc, long long nn) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nn;
       k += (long long)gridDim.x * blockDim.x)
    acc[k] = 0ull;
}

__global__ void k_deposit(const double *x, const double *y, long long n, int nx, int ny, int px,
                          int py, int nyn, unsigned long long *acc) {
  const float q = 1048576.0f;   // 2^20
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double X = x[k], Y = y[k];
    if (px) {
      X = fmod(X, double(nx));
      if (X < 0) X += nx;
      if (X >= nx) X -= nx;
    }
    if (py) {
      Y = fmod(Y, double(ny));
      if (Y < 0) Y += ny;
      if (Y >= ny) Y -= ny;
    }
    const double fi = floor(X), fj = floor(Y);
    if (!(fi >= 0 && fi < nx && fj >= 0 && fj < ny)) continue;   // outside the grid: skipped
    const int i = int(fi), j = int(fj);
    const float fx = fminf(float(X - fi), 0x1.fffffep-1f);
    const float fy = fminf(float(Y - fj), 0x1.fffffep-1f);
    const float gx = __fsub_rn(1.0f, fx), gy = __fsub_rn(1.0f, fy);
    const int w00 = __float2int_rn(__fmul_rn(__fmul_rn(gx, gy), q));
    const int w10 = __float2int_rn(__fmul_rn(__fmul_rn(fx, gy), q));
    const int w01 = __float2int_rn(__fmul_rn(__fmul_rn(gx, fy), q));
    const int w11 = int(1u << 20) - w00 - w10 - w01;
    int i1 = i + 1, j1 = j + 1;
    if (px && i1 == nx) i1 = 0;
    if (py && j1 == ny) j1 = 0;
    atomicAdd(&acc[(long long)i * nyn + j], (unsigned long long)(long long)w00);
    atomicAdd(&acc[(long long)i * nyn + j1], (unsigned long long)(long long)w01);
    atomicAdd(&acc[(long long)i1 * nyn + j], (unsigned long long)(long long)w10);
    atomicAdd(&acc[(long long)i1 * nyn + j1], (unsigned long long)(long long)w11);
  }
}

__global__ void k_finish(const unsigned long long *acc, long long nn, double scale, double *rho) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nn;
       k += (long long)gridDim.x * blockDim.x)
    rho[k] = scale * double((long long)acc[k]);   // two's complement: a sum can be slightly negative
}

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return int(b);
}

// Launches one kernel and returns the error of this launch alone (the
// runtime's thread-wide last-error state is neither read nor cleared).
cudaError_t launch1(const void *k, long long work, void **args, cudaStream_t s) {
  return cudaLaunchKernel(k, dim3(unsigned(grid_for(work))), dim3(kThreads), args, 0, s);
}

}  // namespace

extern "C" pic_status pic_deposit_static(int32_t nx, int32_t ny, int32_t periodic_x,
                                         int32_t periodic_y, int64_t n, const double *x,
                                         const double *y, double weight, double *rho,
                                         void *stream) {
  if (nx < 1 || ny < 1 || n < 0 || !rho || (n > 0 && (!x || !y))) return PIC_EINVAL;
  const long long nxn = periodic_x ? nx : (long long)nx + 1;
  const long long nyn = periodic_y ? ny : (long long)ny + 1;
  long long nn = nxn * nyn;
  if (nn > kStaticMaxNodes) return PIC_ESIZE;
  unsigned long long *acc = nullptr;
  const pic_status st = scratch_address(&acc);
  if (st != PIC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int ix = nx, iy = ny, px = periodic_x ? 1 : 0, py = periodic_y ? 1 : 0, inyn = int(nyn);
  long long np = n;
  double scale = weight / 1048576.0;
  // the scratch keeps the previous call's sums: clear the part this call uses
  void *a_clear[] = {&acc, &nn};
  void *a_dep[] = {&x, &y, &np, &ix, &iy, &px, &py, &inyn, &acc};
  void *a_fin[] = {&acc, &nn, &scale, &rho};
  if (launch1((const void *)k_clear, nn, a_clear, s) != cudaSuccess) return PIC_ECUDA;
  if (n > 0 && launch1((const void *)k_deposit, n, a_dep, s) != cudaSuccess) return PIC_ECUDA;
  if (launch1((const void *)k_finish, nn, a_fin, s) != cudaSuccess) return PIC_ECUDA;
  return PIC_OK;
}

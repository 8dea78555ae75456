// Operator application Y = A X, A = -Laplacian_h + diag(V) on a periodic nx x ny x nz grid (7-point stencil).
//
// This is the operator that every step of Algorithm 3 applies ("AX" in the profiles of Section 6, the
// planewave Hamiltonian there; a real-space stencil here). One thread per grid point and column; the six
// neighbour loads of a warp are coalesced along x and reused through L1. The kernel is bound by the FP64
// issue rate (5 DADD + 1 DMUL + 1 DFMA per point) rather than by HBM on GB300.
#include "ppcg_internal.h"

namespace ppcg {

namespace {

constexpr int kTx = 32;
constexpr int kTy = 8;

__global__ void __launch_bounds__(kTx * kTy)
stencil_kernel(const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy,
               const double* __restrict__ dg, int nx, int ny, int nz, int tiles_x, double inv_h2) {
  const int tx = blockIdx.x % tiles_x;
  const int ty = blockIdx.x / tiles_x;
  const int i = tx * kTx + threadIdx.x;
  const int j = ty * kTy + threadIdx.y;
  const int l = blockIdx.y;
  const int c = blockIdx.z;
  if (i >= nx || j >= ny) return;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t p = i + (int64_t)nx * j + plane * l;
  const double* __restrict__ x = X + (int64_t)c * ldx;
  const int64_t ip = (i + 1 < nx) ? p + 1 : p - (nx - 1);
  const int64_t im = (i > 0) ? p - 1 : p + (nx - 1);
  const int64_t jp = (j + 1 < ny) ? p + nx : p - (int64_t)nx * (ny - 1);
  const int64_t jm = (j > 0) ? p - nx : p + (int64_t)nx * (ny - 1);
  const int64_t lp = (l + 1 < nz) ? p + plane : p - plane * (nz - 1);
  const int64_t lm = (l > 0) ? p - plane : p + plane * (nz - 1);
  const double s = ((__ldg(x + im) + __ldg(x + ip)) + (__ldg(x + jm) + __ldg(x + jp))) +
                   (__ldg(x + lm) + __ldg(x + lp));
  Y[(int64_t)c * ldy + p] = fma(__ldg(dg + p), __ldg(x + p), -inv_h2 * s);
}

}  // namespace

cudaError_t stencil_apply(const Grid& g, const double* dg, const double* X, int64_t ldx, double* Y, int64_t ldy,
                          int m, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int tiles_x = (int)ceil_div(g.nx, kTx);
  const int tiles_y = (int)ceil_div(g.ny, kTy);
  dim3 grid(tiles_x * tiles_y, g.nz, m);
  dim3 block(kTx, kTy);
  stencil_kernel<<<grid, block, 0, s>>>(X, ldx, Y, ldy, dg, g.nx, g.ny, g.nz, tiles_x, g.inv_h2);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ppcg

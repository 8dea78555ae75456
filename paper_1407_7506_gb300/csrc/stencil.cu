// Operator application Y = A X, A = -Laplacian_h + diag(V) on a periodic nx x ny x nz grid (7-point stencil),
// or its complex Bloch-twisted form applied in the real form (see bloch_stencil_kernel).
//
// This is the operator that every step of Algorithm 3 applies ("AX" in the profiles of Section 6, the
// planewave Hamiltonian there; a real-space stencil here). One thread per grid point and column; the six
// neighbour loads of a warp are coalesced along x and reused through L1. The kernel is bound by the FP64
// issue rate (5 DADD + 1 DMUL + 1 DFMA per point; no DMUL when h = 1) rather than by HBM on GB300.
#include "ppcg_internal.h"

namespace ppcg {

namespace {

constexpr int kTx = 32;
constexpr int kTy = 8;

template <bool UNIT>
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
  // h = 1 needs no scaling multiply: 6 FP64 instructions per point instead of 7
  Y[(int64_t)c * ldy + p] = fma(__ldg(dg + p), __ldg(x + p), UNIT ? -s : -inv_h2 * s);
}

// Complex Bloch operator in the real form: column [u; v] (2 n rows) holds z = u + i v. A neighbour across an upper
// face carries e^{+i theta_d}, one across a lower face e^{-i theta_d} (x(r + N e_d) = e^{i theta_d} x(r)). One
// thread per grid point and column computes both halves: (A z)_p = dg_p z_p - inv_h2 sum_nbr phase * z_nbr.
__global__ void __launch_bounds__(kTx * kTy)
bloch_stencil_kernel(const double* __restrict__ X, int64_t ldx, double* __restrict__ Y, int64_t ldy,
                     const double* __restrict__ dg, int nx, int ny, int nz, int tiles_x, double inv_h2, double c0,
                     double s0, double c1, double s1, double c2, double s2) {
  const int tx = blockIdx.x % tiles_x;
  const int ty = blockIdx.x / tiles_x;
  const int i = tx * kTx + threadIdx.x;
  const int j = ty * kTy + threadIdx.y;
  const int l = blockIdx.y;
  const int c = blockIdx.z;
  if (i >= nx || j >= ny) return;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t n = plane * nz;
  const int64_t p = i + (int64_t)nx * j + plane * l;
  const double* __restrict__ u = X + (int64_t)c * ldx;
  const double* __restrict__ v = u + n;
  double sr = 0.0, si = 0.0;
  // neighbour q with phase e^{i sgn theta} (sgn = 0 inside the cell): accumulate phase * (u_q + i v_q)
  auto add = [&](int64_t q, int sgn, double ct, double st) {
    const double a = __ldg(u + q), b = __ldg(v + q);
    if (sgn == 0) {
      sr += a;
      si += b;
    } else {
      const double sn = sgn > 0 ? st : -st;
      sr += ct * a - sn * b;
      si += sn * a + ct * b;
    }
  };
  add((i + 1 < nx) ? p + 1 : p - (nx - 1), (i + 1 < nx) ? 0 : 1, c0, s0);
  add((i > 0) ? p - 1 : p + (nx - 1), (i > 0) ? 0 : -1, c0, s0);
  add((j + 1 < ny) ? p + nx : p - (int64_t)nx * (ny - 1), (j + 1 < ny) ? 0 : 1, c1, s1);
  add((j > 0) ? p - nx : p + (int64_t)nx * (ny - 1), (j > 0) ? 0 : -1, c1, s1);
  add((l + 1 < nz) ? p + plane : p - plane * (nz - 1), (l + 1 < nz) ? 0 : 1, c2, s2);
  add((l > 0) ? p - plane : p + plane * (nz - 1), (l > 0) ? 0 : -1, c2, s2);
  const double d = __ldg(dg + p);
  double* y = Y + (int64_t)c * ldy;
  y[p] = fma(d, __ldg(u + p), -inv_h2 * sr);
  y[p + n] = fma(d, __ldg(v + p), -inv_h2 * si);
}

}  // namespace

cudaError_t stencil_apply(const Grid& g, const double* dg, const double* X, int64_t ldx, double* Y, int64_t ldy,
                          int m, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int tiles_x = (int)ceil_div(g.nx, kTx);
  const int tiles_y = (int)ceil_div(g.ny, kTy);
  dim3 grid(tiles_x * tiles_y, g.nz, m);
  dim3 block(kTx, kTy);
  if (g.cplx)
    bloch_stencil_kernel<<<grid, block, 0, s>>>(X, ldx, Y, ldy, dg, g.nx, g.ny, g.nz, tiles_x, g.inv_h2, g.ct[0],
                                                g.st[0], g.ct[1], g.st[1], g.ct[2], g.st[2]);
  else if (g.inv_h2 == 1.0)
    stencil_kernel<true><<<grid, block, 0, s>>>(X, ldx, Y, ldy, dg, g.nx, g.ny, g.nz, tiles_x, g.inv_h2);
  else
    stencil_kernel<false><<<grid, block, 0, s>>>(X, ldx, Y, ldy, dg, g.nx, g.ny, g.nz, tiles_x, g.inv_h2);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ppcg

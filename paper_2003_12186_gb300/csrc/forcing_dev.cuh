// forcing_dev.cuh -- device body of the direct-forcing iteration (see forcing.cu),
// shared by the single-lattice and the batched launch.
#pragma once

#include "iilbm_internal.cuh"

#include <cmath>

namespace iilbm {

struct DfArgs {
  const double *X, *UD, *G0;
  double *G, *U;
  int *iters;
  double *res;
  int n;
  double eta, dX, tol;
  int max_iters;
  int wx0, wy0, ww, wh;  // window origin and size (lattice nodes)
  double bodyx, bodyy, rho0;
};

constexpr int DF_THREADS = 1024;

// The whole force iteration of one body by one CTA of DF_THREADS threads; smem_raw is
// the CTA's dynamic shared memory (direct_forcing_smem bytes).
template <typename S>
__device__ __forceinline__ void direct_forcing_cta(const S *__restrict__ A, const Geom &geo,
                                                   bool odd, const DfArgs &a, double inv_scale,
                                                   unsigned char *smem_raw) {
  using T = typename Store<S>::T;
  const int W = a.ww * a.wh;
  T *usx = reinterpret_cast<T *>(smem_raw);
  T *usy = usx + W;
  T *h2r = usy + W;  // 1 / (2 rho)
  T *gx = h2r + W;
  T *gy = gx + W;
  double *Gk = reinterpret_cast<double *>(gy + W + (W & 1));  // 8-byte aligned
  double *Uk = Gk + 2 * a.n;
  __shared__ double red[DF_THREADS / 32];
  __shared__ double res_s;
  const int tid = threadIdx.x;

  // u*, 1/(2 rho) on the window (zero outside the lattice: no stencil node lies there)
  for (int c = tid; c < W; c += DF_THREADS) {
    const int x = a.wx0 + c % a.ww, y = a.wy0 + c / a.ww;
    T ux = T(0), uy = T(0), hr = T(0);
    const bool in = geo.bc == IILBM_BC_PERIODIC
                        ? true
                        : (y >= 0 && y < geo.ny && (geo.bc != IILBM_BC_CHANNEL || (x >= 0 && x < geo.nx)));
    if (in) {
      const int xi = geo.bc == IILBM_BC_CHANNEL ? x : wrap(x, geo.nx);
      const int yi = geo.bc == IILBM_BC_PERIODIC ? wrap(y, geo.ny) : y;
      T f[9];
#pragma unroll
      for (int i = 0; i < 9; i++) f[i] = Store<S>::ld(A[aa_loc(geo, odd, i, xi, yi)]) * T(inv_scale);
      const T d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
      const T rho = T(a.rho0) + d;
      ux = ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]) + T(0.5) * T(a.bodyx)) / rho;
      uy = ((f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]) + T(0.5) * T(a.bodyy)) / rho;
      hr = T(0.5) / rho;
    }
    usx[c] = ux;
    usy[c] = uy;
    h2r[c] = hr;
  }
  for (int k = tid; k < 2 * a.n; k += DF_THREADS) Gk[k] = a.G0[k];
  __syncthreads();

  // (marker k, stencil node l) pairs: 16 per marker
  const int npairs = 16 * a.n;
  int it = 0;
  double res = 0.0;
  for (it = 0; it < a.max_iters; it++) {
    for (int c = tid; c < W; c += DF_THREADS) {
      gx[c] = T(0);
      gy[c] = T(0);
    }
    __syncthreads();
    // spread G dX (Eq. 17)
    for (int q = tid; q < npairs; q += DF_THREADS) {
      const int k = q >> 4, l = q & 15;
      const double Xk = a.X[2 * k], Yk = a.X[2 * k + 1];
      const int xa = (int)floor(Xk) - 1 + (l & 3), yb = (int)floor(Yk) - 1 + (l >> 2);
      const T w = phi4<T>(T((double)xa - Xk)) * phi4<T>(T((double)yb - Yk));
      const int c = (yb - a.wy0) * a.ww + (xa - a.wx0);
      if (w != T(0)) {
        atomicAdd(&gx[c], T(Gk[2 * k] * a.dX) * w);
        atomicAdd(&gy[c], T(Gk[2 * k + 1] * a.dX) * w);
      }
    }
    __syncthreads();
    // interpolate u* + g / (2 rho) (Eq. 20): 16 consecutive threads per marker
    for (int base = 0; base < npairs; base += DF_THREADS) {
      const int q = base + tid;
      double sx = 0.0, sy = 0.0;
      if (q < npairs) {
        const int k = q >> 4, l = q & 15;
        const double Xk = a.X[2 * k], Yk = a.X[2 * k + 1];
        const int xa = (int)floor(Xk) - 1 + (l & 3), yb = (int)floor(Yk) - 1 + (l >> 2);
        const T w = phi4<T>(T((double)xa - Xk)) * phi4<T>(T((double)yb - Yk));
        const int c = (yb - a.wy0) * a.ww + (xa - a.wx0);
        sx = (double)((usx[c] + gx[c] * h2r[c]) * w);
        sy = (double)((usy[c] + gy[c] * h2r[c]) * w);
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o, 16);
        sy += __shfl_xor_sync(0xffffffffu, sy, o, 16);
      }
      if (q < npairs && (q & 15) == 0) {
        Uk[2 * (q >> 4)] = sx;
        Uk[2 * (q >> 4) + 1] = sy;
      }
    }
    __syncthreads();
    // residual max_k |U^D - U_k| over both components
    double r = 0.0;
    for (int k = tid; k < 2 * a.n; k += DF_THREADS) r = fmax(r, fabs(a.UD[k] - Uk[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((tid & 31) == 0) red[tid >> 5] = r;
    __syncthreads();
    if (tid < 32) {
      double v = red[tid];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (tid == 0) res_s = v;
    }
    __syncthreads();
    res = res_s;
    if (a.tol > 0.0 && res < a.tol) break;  // uniform
    for (int k = tid; k < 2 * a.n; k += DF_THREADS) Gk[k] += a.eta * (a.UD[k] - Uk[k]);
    __syncthreads();
  }
  for (int k = tid; k < 2 * a.n; k += DF_THREADS) {
    a.G[k] = Gk[k];
    a.U[k] = Uk[k];
  }
  if (tid == 0) {
    *a.iters = it;
    *a.res = res;
  }
}

}  // namespace iilbm

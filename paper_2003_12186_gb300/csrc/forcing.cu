// forcing.cu -- direct forcing of a rigid body with repeated correction (Eq. 18,
// multi-direct forcing), on sm_103a.
//
// The Lagrangian force of a fixed body is found before the step's collision from the
// streamed state f~ (no jump, no immersed-boundary force): u* = (sum_i e_i f~_i +
// body/2) / rho.  Each pass spreads the whole current G (Eq. 17, IB form), interpolates
// u* + g / (2 rho) back to the markers (Eq. 20), and adds eta (U^D - U) to G (Eq. 18);
// the passes stop after mdf_iters updates or once max_k |U^D - U_k| < mdf_tol.  The
// converged G then enters the step like a prescribed force: its normal part through
// the jump, its tangential part spread (section 3.2).
//
// A rigid body has few markers, so the whole iteration runs in one CTA on a shared-
// memory window that covers the body's bounding box plus the kernel support: u*,
// 1/(2 rho) and the spread force live there; G and U stay in FP64.
#include "iilbm_internal.cuh"

#include <cmath>

namespace iilbm {

template <typename T>
__device__ inline T phi4d(T r) {
  const T a = fabs(r);
  if (a < T(1)) return T(0.125) * (T(3) - T(2) * a + sqrt(T(1) + T(4) * a - T(4) * a * a));
  if (a < T(2)) return T(0.125) * (T(5) - T(2) * a - sqrt(T(-7) + T(12) * a - T(4) * a * a));
  return T(0);
}

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

template <typename S>
__global__ void __launch_bounds__(DF_THREADS)
    k_direct_forcing(const S *__restrict__ A, const Geom geo, bool odd, DfArgs a, double inv_scale) {
  using T = typename Store<S>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
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
      const T w = phi4d<T>(T((double)xa - Xk)) * phi4d<T>(T((double)yb - Yk));
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
        const T w = phi4d<T>(T((double)xa - Xk)) * phi4d<T>(T((double)yb - Yk));
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

// Shared memory of the forcing kernel for a window of ww x wh nodes and n markers.
size_t direct_forcing_smem(const iilbm_lattice *h, int ww, int wh, int n) {
  const size_t W = (size_t)ww * wh;
  return 5 * W * h->tbytes + 16 + 4 * (size_t)n * sizeof(double);
}

int launch_direct_forcing(iilbm_lattice *h) {
  const bool odd = h->step & 1;
  DfArgs a;
  a.X = h->X;
  a.UD = h->aux;
  a.G0 = h->G0;
  a.G = h->Gdf;
  a.U = h->U;
  a.iters = h->d_mdf_iters;
  a.res = h->d_mdf_res;
  a.n = h->nm;
  a.eta = h->ip.eta;
  a.dX = h->ip.dX;
  a.tol = h->ip.mdf_tol;
  a.max_iters = h->ip.mdf_iters;
  a.wx0 = h->df_win[0];
  a.wy0 = h->df_win[1];
  a.ww = h->df_win[2];
  a.wh = h->df_win[3];
  a.bodyx = h->cfg.body[0];
  a.bodyy = h->cfg.body[1];
  a.rho0 = h->cfg.rho0;
  const size_t smem = direct_forcing_smem(h, a.ww, a.wh, a.n);
  const double is = std::ldexp(1.0, -h->cfg.storage_scale_log2);
  cudaError_t e = cudaSuccess;
  switch (h->cfg.storage) {
    case IILBM_F64:
      e = cudaFuncSetAttribute(k_direct_forcing<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k_direct_forcing<double><<<1, DF_THREADS, smem, h->stream>>>((const double *)h->A, h->geom, odd, a, is);
      break;
    case IILBM_F32:
      e = cudaFuncSetAttribute(k_direct_forcing<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k_direct_forcing<float><<<1, DF_THREADS, smem, h->stream>>>((const float *)h->A, h->geom, odd, a, is);
      break;
    case IILBM_F16:
      e = cudaFuncSetAttribute(k_direct_forcing<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k_direct_forcing<__half><<<1, DF_THREADS, smem, h->stream>>>((const __half *)h->A, h->geom, odd, a, is);
      break;
    default:
      e = cudaFuncSetAttribute(k_direct_forcing<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k_direct_forcing<__nv_bfloat16><<<1, DF_THREADS, smem, h->stream>>>((const __nv_bfloat16 *)h->A, h->geom, odd, a, is);
  }
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_CUDA;
  }
  return IILBM_OK;
}

}  // namespace iilbm

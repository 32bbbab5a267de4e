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
#include "forcing_dev.cuh"

#include <cmath>

namespace iilbm {

template <typename S>
__global__ void __launch_bounds__(DF_THREADS)
    k_direct_forcing(const S *__restrict__ A, const Geom geo, bool odd, DfArgs a, double inv_scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  direct_forcing_cta<S>(A, geo, odd, a, inv_scale, smem_raw);
}

// Shared memory of the forcing kernel for a window of ww x wh nodes and n markers.
size_t direct_forcing_smem(const iilbm_lattice *h, int ww, int wh, int n) {
  const bool mlp = h->ws_mode == WS_MLP;
  return h->cfg.storage == IILBM_F64 ? df_smem_bytes<double>(ww * wh, n, mlp)
                                     : df_smem_bytes<float>(ww * wh, n, mlp);
}

// The force iteration's arguments for lattice h.
DfArgs df_args(const iilbm_lattice *h) {
  DfArgs a;
  a.X = h->X;
  a.UD = h->aux;
  a.G0 = h->G0;
  a.G = h->Gdf;
  a.U = h->U;
  a.Ustar = h->Ustar;
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
  a.ws_mode = h->ws_mode;
  a.mlp_P = h->mlp ? mlp_params_transposed(h->mlp) : nullptr;
  a.mlp_norm = h->mlp ? mlp_norm(h->mlp) : nullptr;
  a.re = h->re;
  return a;
}

int launch_direct_forcing(iilbm_lattice *h) {
  const bool odd = h->step & 1;
  const DfArgs a = df_args(h);
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

__global__ void k_df_features(const double *__restrict__ X, const double *__restrict__ UD,
                              const double *__restrict__ Ustar, int n, double dX, float re,
                              float *F) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df_features_cta(X, UD, Ustar, n, dX, re, F, reinterpret_cast<float *>(smem_raw));
}

int launch_df_features(iilbm_lattice *h, float re, float *F) {
  const size_t smem = (size_t)h->nm * MLP_BLOCK * sizeof(float);
  if (smem > 227 * 1024) return IILBM_ERR_CAPACITY;
  if (cudaFuncSetAttribute(k_df_features, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_CUDA;
  }
  k_df_features<<<1, 256, smem, h->stream>>>(h->X, h->aux, h->Ustar, h->nm, h->ip.dX, re, F);
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

}  // namespace iilbm

// forcing_dev.cuh -- device body of the direct-forcing iteration (see forcing.cu),
// shared by the single-lattice and the batched launch.
#pragma once

#include "iilbm_internal.cuh"
#include "mlp_dev.cuh"

#include <cmath>

namespace iilbm {

// Where the force iteration starts (G^(0)).
enum { WS_GIVEN = 0, WS_PREVIOUS = 1, WS_MLP = 2 };

struct DfArgs {
  const double *X, *UD, *G0;
  double *G, *U;
  double *Ustar;  // out: U*_k, the interpolated velocity without immersed-boundary force
  int *iters;
  double *res;
  int n;
  double eta, dX, tol;
  int max_iters;
  int wx0, wy0, ww, wh;  // window origin and size (lattice nodes)
  double bodyx, bodyy, rho0;
  int ws_mode;            // WS_GIVEN: G0; WS_PREVIOUS: the G of the last iteration (in G);
                          // WS_MLP: the network's proposal from the step's features
  const float *mlp_P;     // WS_MLP: packed parameters (W1..W3 transposed), normalisation,
                          // Re feature
  const float *mlp_norm;
  float re;
};

constexpr int DF_THREADS = 1024;

// Shared memory of the force iteration: the window fields u*, 1/(2 rho) and two force
// fields g (7 W values of T), the stencil of every marker (16 n weights T and window indices), and the marker
// arrays G, U, U^D, G dX and U* (2 n values of T each).
// With the network's proposal (mlp), the per-marker feature blocks and two activation
// buffers (6 + 2 x 64 floats per marker) follow.
template <typename T>
__host__ __device__ inline size_t df_smem_bytes(int W, int n, bool mlp = false) {
  // u*, 1/(2 rho) and the force fields: three (x, y) fields in FP32, two in FP64
  size_t b = (sizeof(T) == 4 ? 9 : 7) * (size_t)W * sizeof(T);
  b += 16 * (size_t)n * (sizeof(T) + sizeof(int));
  b = (b + 15) & ~(size_t)15;
  b += 10 * (size_t)n * sizeof(T);
  b = (b + 15) & ~(size_t)15;
  if (mlp) b += ((size_t)n * (MLP_BLOCK + 2 * MLP_H) + (MLP_IN + 2 * MLP_H) * MLP_H) * sizeof(float);
  return b + 16;
}

// Bit pattern of a non-negative value of T; such patterns order as the values do, so
// the residual's maximum is taken with integer maxima.
template <typename T> struct BitsOf;
template <> struct BitsOf<float> {
  using U = unsigned;
  __device__ static U of(float v) { return __float_as_uint(v); }
  __device__ static float val(U b) { return __uint_as_float(b); }
};
template <> struct BitsOf<double> {
  using U = unsigned long long;
  __device__ static U of(double v) { return (U)__double_as_longlong(v); }
  __device__ static double val(U b) { return __longlong_as_double((long long)b); }
};

// The whole force iteration of one body by one CTA of DF_THREADS threads; smem_raw is
// the CTA's dynamic shared memory (df_smem_bytes<T>(ww * wh, n)).
//
// The markers do not move within the iteration, so each marker's 4 x 4 stencil
// (window indices and weights phi(x - X) phi(y - Y), from the FP64 position) is formed
// once; a pass is then the spread (Eq. 17) of G dX, the interpolation (Eq. 20) of
// u* + g / (2 rho), the residual max_k |U^D - U_k| and the update G += eta (U^D - U)
// (Eq. 18), all in the arithmetic type T (FP64 for FP64 storage; FP32 otherwise, where
// GB300's FP64 pipe would cost a whole warp's time even for the few lanes that hold a
// marker).  U* (the interpolation with G = 0) is recorded for the learned warm start.
template <typename S>
__device__ __forceinline__ void direct_forcing_cta(const S *__restrict__ A, const Geom &geo,
                                                   bool odd, const DfArgs &a, double inv_scale,
                                                   unsigned char *smem_raw) {
  using T = typename Store<S>::T;
  using B = typename BitsOf<T>::U;
  const int W = a.ww * a.wh, n = a.n;
  T *usx = reinterpret_cast<T *>(smem_raw);
  T *usy = usx + W;
  T *h2r = usy + W;  // 1 / (2 rho)
  T *gx = h2r + W;  // force field of the even passes (FP32: of passes 0, 3, 6, ...)
  T *gy = gx + W;
  T *gx2 = gy + W;  // force field of the odd passes (FP32: of passes 1, 4, 7, ...)
  T *gy2 = gx2 + W;
  T *gx3 = gy2 + W;  // FP32 only: the third field (passes 2, 5, 8, ...)
  T *gy3 = gx3 + W;
  T *pw = sizeof(T) == 4 ? gy3 + W : gy2 + W;       // stencil weights [16 n]
  int *pc = reinterpret_cast<int *>(pw + 16 * n);   // stencil window indices [16 n]
  size_t off = (size_t)(reinterpret_cast<unsigned char *>(pc + 16 * n) - smem_raw);
  off = (off + 15) & ~(size_t)15;
  T *Gk = reinterpret_cast<T *>(smem_raw + off);    // [2 n] each
  T *Uk = Gk + 2 * n;
  T *UDk = Uk + 2 * n;
  T *GdX = UDk + 2 * n;                             // G dX, what the spread moves
  T *Us = GdX + 2 * n;                              // U*
  size_t off2 = (size_t)(reinterpret_cast<unsigned char *>(Us + 2 * n) - smem_raw);
  off2 = (off2 + 15) & ~(size_t)15;
  // WS_MLP scratch: the transposed weights first (16-byte aligned for 16-byte loads),
  // then the per-marker feature blocks and two activation buffers
  float *wt1 = reinterpret_cast<float *>(smem_raw + off2);
  float *wt2 = wt1 + MLP_IN * MLP_H;
  float *wt3 = wt2 + MLP_H * MLP_H;
  float *blk = wt3 + MLP_H * MLP_H;
  float *act0 = blk + MLP_BLOCK * n;
  float *act1 = act0 + MLP_H * n;
  __shared__ B red[2][DF_THREADS / 32];
  __shared__ T cst[6];  // 2^-k, rho0, body force, eta, dX: converted once, by one thread
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    cst[0] = T(inv_scale);
    cst[1] = T(a.rho0);
    cst[2] = T(a.bodyx);
    cst[3] = T(a.bodyy);
    cst[4] = T(a.eta);
    cst[5] = T(a.dX);
  }
  __syncthreads();
  const T is = cst[0], rho0 = cst[1], bodyx = cst[2], bodyy = cst[3], eta = cst[4], dX = cst[5];

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
      for (int i = 0; i < 9; i++) f[i] = Store<S>::ld(A[aa_loc(geo, odd, i, xi, yi)]) * is;
      const T d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
      const T rho = rho0 + d;
      ux = ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]) + T(0.5) * bodyx) / rho;
      uy = ((f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]) + T(0.5) * bodyy) / rho;
      hr = T(0.5) / rho;
    }
    usx[c] = ux;
    usy[c] = uy;
    h2r[c] = hr;
    gx[c] = T(0);
    gy[c] = T(0);
    gx2[c] = T(0);
    gy2[c] = T(0);
    if (sizeof(T) == 4) {
      gx3[c] = T(0);
      gy3[c] = T(0);
    }
  }
  // stencils, one thread per marker
  for (int k = tid; k < n; k += DF_THREADS) {
    const double Xk = a.X[2 * k], Yk = a.X[2 * k + 1];
    const int bx = (int)floor(Xk) - 1, by = (int)floor(Yk) - 1;
    T wx[4], wy[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      wx[q] = phi4<T>(T((double)(bx + q) - Xk));
      wy[q] = phi4<T>(T((double)(by + q) - Yk));
    }
#pragma unroll
    for (int l = 0; l < 16; l++) {
      pw[16 * k + l] = wx[l & 3] * wy[l >> 2];
      pc[16 * k + l] = (by + (l >> 2) - a.wy0) * a.ww + (bx + (l & 3) - a.wx0);
    }
  }
  // marker arrays, one thread per component: the start of the iteration, U^D
  const double *g0 = a.ws_mode == WS_PREVIOUS ? a.G : a.G0;
  for (int k = tid; k < 2 * n; k += DF_THREADS) {
    if (sizeof(T) == 8) {
      Gk[k] = T(g0[k]);
      GdX[k] = T(g0[k] * a.dX);
    } else {
      Gk[k] = T(g0[k]);
      GdX[k] = Gk[k] * dX;
    }
    UDk[k] = T(a.UD[k]);
  }
  __syncthreads();

  const int npairs = 16 * n;
  // U* = interp(u*), 16 consecutive threads per marker
  for (int base = 0; base < npairs; base += DF_THREADS) {
    const int q = base + tid;
    T sx = T(0), sy = T(0);
    if (q < npairs) {
      const int c = pc[q];
      sx = usx[c] * pw[q];
      sy = usy[c] * pw[q];
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o, 16);
      sy += __shfl_xor_sync(0xffffffffu, sy, o, 16);
    }
    if (q < npairs && (q & 15) == 0) {
      Us[2 * (q >> 4)] = sx;
      Us[2 * (q >> 4) + 1] = sy;
      Uk[2 * (q >> 4)] = sx;  // the last interpolated velocity, should no pass run
      Uk[2 * (q >> 4) + 1] = sy;
    }
  }

  if (a.ws_mode == WS_MLP) {
    // G^(0) proposed by the network from each marker's features (U* from above)
    __syncthreads();
    for (int j = tid; j < n; j += DF_THREADS)
      marker_feature_block(a.X, n, j, a.dX, (float)(UDk[2 * j] - Us[2 * j]),
                           (float)(UDk[2 * j + 1] - Us[2 * j + 1]), a.re, blk + MLP_BLOCK * j);
    __syncthreads();
    for (int k = tid; k < n; k += DF_THREADS) mlp_gather_input(blk, n, k, a.mlp_norm, act1 + MLP_IN * k);
    // mlp_P holds W1, W2, W3 already transposed to [in][64]
    mlp_copy4(a.mlp_P + OFF_W1, wt1, MLP_IN * MLP_H, tid, DF_THREADS);
    mlp_copy4(a.mlp_P + OFF_W2, wt2, MLP_H * MLP_H, tid, DF_THREADS);
    mlp_copy4(a.mlp_P + OFF_W3, wt3, MLP_H * MLP_H, tid, DF_THREADS);
    __syncthreads();
    mlp_hidden_layer_t(wt1, a.mlp_P + OFF_B1, act1, MLP_IN, act0, n, tid, DF_THREADS);
    __syncthreads();
    mlp_hidden_layer_t(wt2, a.mlp_P + OFF_B2, act0, MLP_H, act1, n, tid, DF_THREADS);
    __syncthreads();
    mlp_hidden_layer_t(wt3, a.mlp_P + OFF_B3, act1, MLP_H, act0, n, tid, DF_THREADS);
    __syncthreads();
    mlp_output_layer(a.mlp_P, act0, act1, n, tid, DF_THREADS);
    __syncthreads();
    for (int k = tid; k < 2 * n; k += DF_THREADS) {
      const int o = k & 1;
      const float g = act1[k] * a.mlp_norm[NORM_OUT_SCALE + o] + a.mlp_norm[NORM_OUT_MEAN + o];
      Gk[k] = T(g);
      if (sizeof(T) == 8) GdX[k] = T((double)g * a.dX);
      else GdX[k] = Gk[k] * dX;
    }
    __syncthreads();
  }

  // the start G^(0) spread (Eq. 17) into the field of pass 0
  for (int q = tid; q < npairs; q += DF_THREADS) {
    const T w = pw[q];
    if (w != T(0)) {
      const int k = q >> 4, c = pc[q];
      atomicAdd(&gx[c], GdX[2 * k] * w);
      atomicAdd(&gy[c], GdX[2 * k + 1] * w);
    }
  }
  __syncthreads();

  int it = 0;
  B rm = 0;
  // stop once the residual's bit pattern is below the tolerance's (both non-negative)
  const bool stop_on_tol = a.tol > 0.0;
  const B tol_bits = BitsOf<T>::of(T(a.tol));
  if constexpr (sizeof(T) == 4) {
    // FP32: one barrier per pass.  The 16 lanes of a marker interpolate u* + g / (2 rho)
    // (Eq. 20) from the pass's field; after the xor butterfly each holds the same U_k,
    // so they form G += eta (U^D - U) (Eq. 18) and spread the new G dX into the next
    // pass's field at once, without waiting for the residual; meanwhile the field of
    // the pass after next is cleared (three fields in turn).  The barrier then makes the
    // spread complete and the warps' residual maxima visible; a pass whose residual
    // (taken before its update) is below the tolerance puts the G it started from
    // back, so the result is the one of checking before updating.
    T *Gp = GdX;  // G at the start of the pass, for that roll-back (GdX is free by now)
    // the fields in turn: read (fx), spread into (ox), cleared (zx)
    T *fx = gx, *fy = gy, *ox = gx2, *oy = gy2, *zx = gx3, *zy = gy3;
    for (it = 0; it < a.max_iters; it++) {
      B r = 0;
      for (int base = 0; base < npairs; base += DF_THREADS) {
        const int q = base + tid, k = q >> 4;
        T sx = T(0), sy = T(0);
        if (q < npairs) {
          const int c = pc[q];
          const T w = pw[q];
          sx = (usx[c] + fx[c] * h2r[c]) * w;
          sy = (usy[c] + fy[c] * h2r[c]) * w;
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          sx += __shfl_xor_sync(0xffffffffu, sx, o, 16);
          sy += __shfl_xor_sync(0xffffffffu, sy, o, 16);
        }
        T gxo = T(0), gyo = T(0), nx = T(0), ny = T(0);
        if (q < npairs) {
          gxo = Gk[2 * k];
          gyo = Gk[2 * k + 1];
          nx = gxo + eta * (UDk[2 * k] - sx);
          ny = gyo + eta * (UDk[2 * k + 1] - sy);
        }
        __syncwarp();  // every lane of the marker has read the old G
        if (q < npairs) {
          if ((q & 15) == 0) {
            Uk[2 * k] = sx;
            Uk[2 * k + 1] = sy;
            r = max(r, max(BitsOf<T>::of(fabs(UDk[2 * k] - sx)),
                           BitsOf<T>::of(fabs(UDk[2 * k + 1] - sy))));
            Gp[2 * k] = gxo;
            Gp[2 * k + 1] = gyo;
            Gk[2 * k] = nx;
            Gk[2 * k + 1] = ny;
          }
          const T w = pw[q];
          if (w != T(0)) {
            const int c = pc[q];
            atomicAdd(&ox[c], nx * dX * w);
            atomicAdd(&oy[c], ny * dX * w);
          }
        }
      }
      for (int c = tid; c < W; c += DF_THREADS) {
        zx[c] = T(0);
        zy[c] = T(0);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r = max(r, (B)__shfl_xor_sync(0xffffffffu, r, o));
      if (lane == 0) red[it & 1][tid >> 5] = r;  // two sets: a warp may run a pass ahead
      __syncthreads();
      rm = lane < DF_THREADS / 32 ? red[it & 1][lane] : B(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rm = max(rm, (B)__shfl_xor_sync(0xffffffffu, rm, o));
      if (stop_on_tol && rm < tol_bits) {  // uniform
        for (int k = tid; k < 2 * n; k += DF_THREADS) Gk[k] = Gp[k];
        __syncthreads();
        break;
      }
      T *tx = fx, *ty = fy;  // rotate: spread-into -> read, cleared -> spread-into
      fx = ox;
      fy = oy;
      ox = zx;
      oy = zy;
      zx = tx;
      zy = ty;
    }
  } else {
  // FP64: each pass interpolates u* + g / (2 rho) (Eq. 20) from the pass's field and
  // takes the residual (clearing the other field meanwhile); then, unless converged,
  // updates G += eta (U^D - U) (Eq. 18) and spreads the new G dX into the other field --
  // the 16 lanes of a marker form the same update, its first lane stores it.  Two
  // barriers.
  for (it = 0; it < a.max_iters; it++) {
    const bool odd_pass = it & 1;
    const T *fx = odd_pass ? gx2 : gx, *fy = odd_pass ? gy2 : gy;
    T *ox = odd_pass ? gx : gx2, *oy = odd_pass ? gy : gy2;
    B r = 0;
    for (int base = 0; base < npairs; base += DF_THREADS) {
      const int q = base + tid;
      T sx = T(0), sy = T(0);
      if (q < npairs) {
        const int c = pc[q];
        const T w = pw[q];
        sx = (usx[c] + fx[c] * h2r[c]) * w;
        sy = (usy[c] + fy[c] * h2r[c]) * w;
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o, 16);
        sy += __shfl_xor_sync(0xffffffffu, sy, o, 16);
      }
      if (q < npairs && (q & 15) == 0) {
        const int k = q >> 4;
        Uk[2 * k] = sx;
        Uk[2 * k + 1] = sy;
        r = max(r, max(BitsOf<T>::of(fabs(UDk[2 * k] - sx)),
                       BitsOf<T>::of(fabs(UDk[2 * k + 1] - sy))));
      }
    }
    for (int c = tid; c < W; c += DF_THREADS) {
      ox[c] = T(0);
      oy[c] = T(0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = max(r, (B)__shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) red[0][tid >> 5] = r;
    __syncthreads();
    // every warp reduces the warp maxima itself
    rm = lane < DF_THREADS / 32 ? red[0][lane] : B(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rm = max(rm, (B)__shfl_xor_sync(0xffffffffu, rm, o));
    if (stop_on_tol && rm < tol_bits) break;  // uniform
    for (int base = 0; base < npairs; base += DF_THREADS) {
      const int q = base + tid;
      const int k = q >> 4;
      T nx = T(0), ny = T(0);
      if (q < npairs) {
        nx = Gk[2 * k] + eta * (UDk[2 * k] - Uk[2 * k]);
        ny = Gk[2 * k + 1] + eta * (UDk[2 * k + 1] - Uk[2 * k + 1]);
      }
      __syncwarp();  // every lane of the marker has read the old G
      if (q < npairs) {
        if ((q & 15) == 0) {
          Gk[2 * k] = nx;
          Gk[2 * k + 1] = ny;
        }
        T px, py;
        if (sizeof(T) == 8) {
          px = T((double)nx * a.dX);
          py = T((double)ny * a.dX);
        } else {
          px = nx * dX;
          py = ny * dX;
        }
        const T w = pw[q];
        if (w != T(0)) {
          const int c = pc[q];
          atomicAdd(&ox[c], px * w);
          atomicAdd(&oy[c], py * w);
        }
      }
    }
    __syncthreads();
  }
  }
  for (int k = tid; k < 2 * n; k += DF_THREADS) {
    a.G[k] = (double)Gk[k];
    a.U[k] = (double)Uk[k];
    a.Ustar[k] = (double)Us[k];
  }
  if (tid == 0) {
    *a.iters = it;
    *a.res = (double)BitsOf<T>::val(rm);
  }
}

// Raw (unnormalised) features [n][30] of every marker from the U* of the most recent
// force iteration: one CTA, blocks in shared memory (n * 6 floats).
__device__ inline void df_features_cta(const double *__restrict__ X, const double *__restrict__ UD,
                                       const double *__restrict__ Ustar, int n, double dX,
                                       float re, float *F, float *blk) {
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    marker_feature_block(X, n, j, dX, (float)(UD[2 * j] - Ustar[2 * j]),
                         (float)(UD[2 * j + 1] - Ustar[2 * j + 1]), re, blk + MLP_BLOCK * j);
  __syncthreads();
  for (int e = threadIdx.x; e < n * MLP_IN; e += blockDim.x) {
    const int k = e / MLP_IN, i = e % MLP_IN, q = i / MLP_BLOCK, r = i % MLP_BLOCK;
    int j = k + q - 2;
    j = j < 0 ? j + n : (j >= n ? j - n : j);
    F[e] = blk[MLP_BLOCK * j + r];
  }
}

}  // namespace iilbm

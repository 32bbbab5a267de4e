// mlp_dev.cuh -- device building blocks of the learned warm start: the 30-64-64-64-2
// network with the exact (erf) GELU, its per-marker features, and block-cooperative
// layers used both by the training kernels (mlp.cu) and by the direct-forcing CTA,
// which proposes the starting force G^(0) of every marker of its body.
//
// FP32 on the CUDA cores: the contractions are 64 wide over at most a few thousand
// samples per launch, far too small to feed the tensor cores, and the gradients are
// checked against an FP64 oracle at 1e-4.
#pragma once

#include "iilbm_internal.cuh"

#include <cmath>

namespace iilbm {

constexpr int MLP_IN = 30, MLP_H = 64, MLP_OUT = 2;
// packed parameters: W1 [64][30], b1, W2 [64][64], b2, W3 [64][64], b3, W4 [2][64], b4
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H,
              OFF_B2 = OFF_W2 + MLP_H * MLP_H, OFF_W3 = OFF_B2 + MLP_H,
              OFF_B3 = OFF_W3 + MLP_H * MLP_H, OFF_W4 = OFF_B3 + MLP_H,
              OFF_B4 = OFF_W4 + MLP_OUT * MLP_H, MLP_NPARAM = OFF_B4 + MLP_OUT;
static_assert(MLP_NPARAM == 10434, "parameter count");
// normalisation: input mean [30], input 1/std [30], output mean [2], output scale [2]
constexpr int NORM_IN_MEAN = 0, NORM_IN_ISTD = 30, NORM_OUT_MEAN = 60, NORM_OUT_SCALE = 62,
              MLP_NORM = 64;
// features per marker of the 5-marker window: dU (2), n (2), kappa, Re
constexpr int MLP_BLOCK = 6;

__device__ inline float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
// d/dz [z Phi(z)] = Phi(z) + z phi(z)
__device__ inline float gelu_prime_f(float z) {
  const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  return Phi + z * (0.39894228040143268f * expf(-0.5f * z * z));
}

// One hidden layer for S samples: out[s][j] = gelu(b[j] + sum_i W[j][i] in[s][i]),
// j < 64; the pre-activation goes to z (if not null).  Threads stride over (s, j).
__device__ inline void mlp_hidden_layer(const float *__restrict__ W, const float *__restrict__ b,
                                        const float *in, int in_dim, float *z, float *out, int S,
                                        int tid, int nthreads) {
  for (int idx = tid; idx < S * MLP_H; idx += nthreads) {
    const int s = idx >> 6, j = idx & (MLP_H - 1);
    const float *w = W + j * in_dim;
    const float *x = in + s * in_dim;
    float acc = b[j];
    for (int i = 0; i < in_dim; i++) acc = fmaf(w[i], x[i], acc);
    if (z) z[idx] = acc;
    out[idx] = gelu_f(acc);
  }
}

// The same layer with the weights transposed, WT[i][j] (shared memory): a thread forms
// four outputs j0 .. j0+3 of one sample from one broadcast input load and one 16-byte
// weight load per i (each output's sum in the same order as above).
__device__ inline void mlp_hidden_layer_t(const float *WT, const float *__restrict__ b,
                                          const float *in, int in_dim, float *out, int S, int tid,
                                          int nthreads) {
  for (int item = tid; item < S * (MLP_H / 4); item += nthreads) {
    const int s = item >> 4, j0 = (item & 15) * 4;
    const float *x = in + s * in_dim;
    float a0 = b[j0], a1 = b[j0 + 1], a2 = b[j0 + 2], a3 = b[j0 + 3];
    for (int i = 0; i < in_dim; i++) {
      const float xi = x[i];
      const float4 w = *reinterpret_cast<const float4 *>(WT + i * MLP_H + j0);
      a0 = fmaf(w.x, xi, a0);
      a1 = fmaf(w.y, xi, a1);
      a2 = fmaf(w.z, xi, a2);
      a3 = fmaf(w.w, xi, a3);
    }
    float *o = out + s * MLP_H + j0;
    o[0] = gelu_f(a0);
    o[1] = gelu_f(a1);
    o[2] = gelu_f(a2);
    o[3] = gelu_f(a3);
  }
}

// Copy n floats (a multiple of 4, 16-byte aligned both sides) with 16-byte accesses.
__device__ inline void mlp_copy4(const float *__restrict__ src, float *dst, int n, int tid,
                                 int nthreads) {
  const float4 *s4 = reinterpret_cast<const float4 *>(src);
  float4 *d4 = reinterpret_cast<float4 *>(dst);
  for (int e = tid; e < n / 4; e += nthreads) d4[e] = s4[e];
}

// Output layer: y[s][o] = b4[o] + sum_j W4[o][j] a[s][j] (normalised output).
__device__ inline void mlp_output_layer(const float *__restrict__ P, const float *a, float *y, int S,
                                        int tid, int nthreads) {
  for (int idx = tid; idx < S * MLP_OUT; idx += nthreads) {
    const int s = idx >> 1, o = idx & 1;
    const float *w = P + OFF_W4 + o * MLP_H;
    const float *x = a + s * MLP_H;
    float acc = P[OFF_B4 + o];
    for (int j = 0; j < MLP_H; j++) acc = fmaf(w[j], x[j], acc);
    y[idx] = acc;
  }
}

// Features block of marker j of a closed counter-clockwise polygon of n markers:
// dU = U^D - U* (2), outward unit normal (2), signed curvature -(d2 X . n) / dX^2, Re.
// The position differences (small differences of large numbers) in FP64, the rest in
// FP32: GB300 charges a warp's full FP64 time for the few lanes that hold a marker.
__device__ inline void marker_feature_block(const double *__restrict__ X, int n, int j, double dX,
                                            float dUx, float dUy, float re, float *blk) {
  const int jp = j + 1 == n ? 0 : j + 1, jm = j == 0 ? n - 1 : j - 1;
  const double x = X[2 * j], y = X[2 * j + 1];
  const double xp = X[2 * jp], yp = X[2 * jp + 1], xm = X[2 * jm], ym = X[2 * jm + 1];
  const float ax = (float)(xp - x), ay = (float)(yp - y);  // X_{j+1} - X_j
  const float bx = (float)(x - xm), by = (float)(y - ym);  // X_j - X_{j-1}
  const float tx = ax + bx, ty = ay + by;                  // X_{j+1} - X_{j-1}
  const float il = rsqrtf(tx * tx + ty * ty);
  const float nx = ty * il, ny = -tx * il;
  const float d2x = (float)((xp - x) - (x - xm)), d2y = (float)((yp - y) - (y - ym));
  const float idx2 = 1.0f / (float)(dX * dX);
  blk[0] = dUx;
  blk[1] = dUy;
  blk[2] = nx;
  blk[3] = ny;
  blk[4] = -(d2x * nx + d2y * ny) * idx2;
  blk[5] = re;
}

// Normalised network input of marker k from the per-marker blocks [n][6]:
// the blocks of markers k-2 .. k+2 (cyclic), then (x - mean) * istd.
__device__ inline void mlp_gather_input(const float *blk, int n, int k, const float *__restrict__ norm,
                                        float *xh) {
#pragma unroll
  for (int q = 0; q < 5; q++) {
    int j = k + q - 2;
    j = j < 0 ? j + n : (j >= n ? j - n : j);
#pragma unroll
    for (int r = 0; r < MLP_BLOCK; r++) {
      const int i = q * MLP_BLOCK + r;
      xh[i] = (blk[j * MLP_BLOCK + r] - norm[NORM_IN_MEAN + i]) * norm[NORM_IN_ISTD + i];
    }
  }
}

}  // namespace iilbm

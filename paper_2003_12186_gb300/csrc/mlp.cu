// mlp.cu -- training and batch inference of the learned warm start on sm_103a.
//
// One training step on a batch of B samples is two launches:
//   k_mlp_fwd_bwd   each CTA takes MLP_SPB samples of the batch: forward pass (pre-
//                   activations and activations kept in shared memory), the squared
//                   error of the normalised outputs, and backpropagation to a partial
//                   gradient of the whole parameter vector, written to its own row;
//   k_mlp_reduce    one thread per parameter sums the partial rows in a fixed order
//                   (deterministic) and applies the Adam update (or returns the
//                   gradient, for the check against the oracle).
// The definitions (features, network, loss, optimiser) are those of the oracle's
// module docstring; the parameters are FP32.
#include "mlp_dev.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace iilbm {

constexpr int MLP_SPB = 16;       // samples per CTA
constexpr int MLP_THREADS = 256;

// Forward and backward pass of samples [first, first + count) of the list (idx[first +
// s], or first + s without a list); the gradient of L = sum (yh - th)^2 * wscale over
// these samples goes to partial[blockIdx.x][.], the error sum to loss[blockIdx.x].
__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_fwd_bwd(const float *__restrict__ P, const float *__restrict__ norm,
                  const float *__restrict__ X, const float *__restrict__ T,
                  const int *__restrict__ idx, int first, int count, float wscale,
                  float *__restrict__ partial, float *__restrict__ loss) {
  __shared__ float xh[MLP_SPB * MLP_IN];
  __shared__ float z1[MLP_SPB * MLP_H], a1[MLP_SPB * MLP_H];
  __shared__ float z2[MLP_SPB * MLP_H], a2[MLP_SPB * MLP_H];
  __shared__ float z3[MLP_SPB * MLP_H], a3[MLP_SPB * MLP_H];
  __shared__ float dy[MLP_SPB * MLP_OUT], yh[MLP_SPB * MLP_OUT];
  __shared__ float red[MLP_THREADS / 32];
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * MLP_SPB;
  const int S = min(MLP_SPB, count - s0);
  float *g = partial + (size_t)blockIdx.x * MLP_NPARAM;
  // normalised inputs
  for (int e = tid; e < MLP_SPB * MLP_IN; e += MLP_THREADS) {
    const int s = e / MLP_IN, i = e % MLP_IN;
    float v = 0.0f;
    if (s < S) {
      const int r = idx ? idx[first + s0 + s] : first + s0 + s;
      v = (X[(size_t)r * MLP_IN + i] - norm[NORM_IN_MEAN + i]) * norm[NORM_IN_ISTD + i];
    }
    xh[e] = v;
  }
  __syncthreads();
  mlp_hidden_layer(P + OFF_W1, P + OFF_B1, xh, MLP_IN, z1, a1, MLP_SPB, tid, MLP_THREADS);
  __syncthreads();
  mlp_hidden_layer(P + OFF_W2, P + OFF_B2, a1, MLP_H, z2, a2, MLP_SPB, tid, MLP_THREADS);
  __syncthreads();
  mlp_hidden_layer(P + OFF_W3, P + OFF_B3, a2, MLP_H, z3, a3, MLP_SPB, tid, MLP_THREADS);
  __syncthreads();
  mlp_output_layer(P, a3, yh, MLP_SPB, tid, MLP_THREADS);
  __syncthreads();
  // error of the normalised output; dL/dyh = 2 e wscale (rows past the batch: 0)
  float l = 0.0f;
  if (tid < MLP_SPB * MLP_OUT) {
    const int s = tid >> 1, o = tid & 1;
    float e = 0.0f;
    if (s < S) {
      const int r = idx ? idx[first + s0 + s] : first + s0 + s;
      const float th = (T[(size_t)r * MLP_OUT + o] - norm[NORM_OUT_MEAN + o]) / norm[NORM_OUT_SCALE + o];
      e = yh[tid] - th;
    }
    dy[tid] = 2.0f * e * wscale;
    l = e * e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((tid & 31) == 0) red[tid >> 5] = l;
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
    for (int w = 0; w < MLP_THREADS / 32; w++) t += red[w];
    loss[blockIdx.x] = t;
  }
  // output layer: gW4[o][j] = sum_s dy[s][o] a3[s][j], gb4[o] = sum_s dy[s][o]
  for (int e = tid; e < MLP_OUT * MLP_H + MLP_OUT; e += MLP_THREADS) {
    float acc = 0.0f;
    if (e < MLP_OUT * MLP_H) {
      const int o = e / MLP_H, j = e % MLP_H;
      for (int s = 0; s < MLP_SPB; s++) acc = fmaf(dy[s * MLP_OUT + o], a3[s * MLP_H + j], acc);
      g[OFF_W4 + e] = acc;
    } else {
      const int o = e - MLP_OUT * MLP_H;
      for (int s = 0; s < MLP_SPB; s++) acc += dy[s * MLP_OUT + o];
      g[OFF_B4 + o] = acc;
    }
  }
  // dz3 = (dy W4) * gelu'(z3), kept in z3
  for (int e = tid; e < MLP_SPB * MLP_H; e += MLP_THREADS) {
    const int s = e >> 6, j = e & (MLP_H - 1);
    const float d = dy[s * MLP_OUT] * P[OFF_W4 + j] + dy[s * MLP_OUT + 1] * P[OFF_W4 + MLP_H + j];
    z3[e] = d * gelu_prime_f(z3[e]);
  }
  __syncthreads();
  // hidden layers, from the third back to the first: gW[j][i] = sum_s dz[s][j] in[s][i],
  // gb[j] = sum_s dz[s][j], and dz of the layer below = (dz W) * gelu'(z below)
  const float *dzs[3] = {z3, z2, z1};
  const float *ins[3] = {a2, a1, xh};
  float *zb[3] = {z2, z1, nullptr};
  const int offW[3] = {OFF_W3, OFF_W2, OFF_W1}, offB[3] = {OFF_B3, OFF_B2, OFF_B1};
  const int dims[3] = {MLP_H, MLP_H, MLP_IN};
  for (int L = 0; L < 3; L++) {
    const float *dz = dzs[L], *in = ins[L];
    const int din = dims[L];
    for (int e = tid; e < MLP_H * din + MLP_H; e += MLP_THREADS) {
      float acc = 0.0f;
      if (e < MLP_H * din) {
        const int j = e / din, i = e % din;
        for (int s = 0; s < MLP_SPB; s++) acc = fmaf(dz[s * MLP_H + j], in[s * din + i], acc);
        g[offW[L] + e] = acc;
      } else {
        const int j = e - MLP_H * din;
        for (int s = 0; s < MLP_SPB; s++) acc += dz[s * MLP_H + j];
        g[offB[L] + j] = acc;
      }
    }
    if (zb[L]) {
      // z below is overwritten by its dz only after every thread has used dz above;
      // the in[] of this layer (activations a) is not touched
      float tmp[MLP_SPB * MLP_H / MLP_THREADS];
      int q = 0;
      for (int e = tid; e < MLP_SPB * MLP_H; e += MLP_THREADS, q++) {
        const int s = e >> 6, i = e & (MLP_H - 1);
        const float *W = P + offW[L];
        float acc = 0.0f;
        for (int j = 0; j < MLP_H; j++) acc = fmaf(dz[s * MLP_H + j], W[j * MLP_H + i], acc);
        tmp[q] = acc * gelu_prime_f(zb[L][e]);
      }
      __syncthreads();
      q = 0;
      for (int e = tid; e < MLP_SPB * MLP_H; e += MLP_THREADS, q++) zb[L][e] = tmp[q];
      __syncthreads();
    }
  }
}

// One thread per parameter: the gradient (sum of the partial rows, in order), then
// either an Adam step (t >= 1) or a copy to grad_out.  Block 0 also sums the losses.
__global__ void k_mlp_reduce(const float *__restrict__ partial, int nparts,
                             const float *__restrict__ loss, float loss_scale, float *loss_out,
                             float *P, float *m, float *v, int t, float lr, float beta1,
                             float beta2, float eps, float *grad_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && loss_out) {
    float s = 0.0f;
    for (int p = 0; p < nparts; p++) s += loss[p];
    *loss_out = s * loss_scale;
  }
  if (i >= MLP_NPARAM) return;
  float gsum = 0.0f;
  for (int p = 0; p < nparts; p++) gsum += partial[(size_t)p * MLP_NPARAM + i];
  if (grad_out) grad_out[i] = gsum;
  if (t > 0) {
    const float mi = beta1 * m[i] + (1.0f - beta1) * gsum;
    const float vi = beta2 * v[i] + (1.0f - beta2) * gsum * gsum;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(beta1, (float)t));
    const float vh = vi / (1.0f - powf(beta2, (float)t));
    P[i] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// Batch inference: MLP_SPB samples per CTA, G^(0) in physical units.
__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_forward(const float *__restrict__ P, const float *__restrict__ norm,
                  const float *__restrict__ X, int N, float *__restrict__ Y) {
  __shared__ float xh[MLP_SPB * MLP_IN];
  __shared__ float a1[MLP_SPB * MLP_H], a2[MLP_SPB * MLP_H];
  __shared__ float yh[MLP_SPB * MLP_OUT];
  const int tid = threadIdx.x, s0 = blockIdx.x * MLP_SPB;
  for (int e = tid; e < MLP_SPB * MLP_IN; e += MLP_THREADS) {
    const int s = e / MLP_IN, i = e % MLP_IN;
    xh[e] = s0 + s < N ? (X[(size_t)(s0 + s) * MLP_IN + i] - norm[NORM_IN_MEAN + i]) *
                             norm[NORM_IN_ISTD + i]
                       : 0.0f;
  }
  __syncthreads();
  mlp_hidden_layer(P + OFF_W1, P + OFF_B1, xh, MLP_IN, nullptr, a1, MLP_SPB, tid, MLP_THREADS);
  __syncthreads();
  mlp_hidden_layer(P + OFF_W2, P + OFF_B2, a1, MLP_H, nullptr, a2, MLP_SPB, tid, MLP_THREADS);
  __syncthreads();
  mlp_hidden_layer(P + OFF_W3, P + OFF_B3, a2, MLP_H, nullptr, a1, MLP_SPB, tid, MLP_THREADS);
  __syncthreads();
  mlp_output_layer(P, a1, yh, MLP_SPB, tid, MLP_THREADS);
  __syncthreads();
  if (tid < MLP_SPB * MLP_OUT && s0 + (tid >> 1) < N) {
    const int o = tid & 1;
    Y[(size_t)(s0 + (tid >> 1)) * MLP_OUT + o] =
        yh[tid] * norm[NORM_OUT_SCALE + o] + norm[NORM_OUT_MEAN + o];
  }
}

// PT: the packed parameters with W1, W2, W3 stored [in][64] (biases, W4, b4 as in P).
__global__ void k_mlp_transposed(const float *__restrict__ P, float *__restrict__ PT) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= MLP_NPARAM) return;
  int off = -1, in_dim = 0;
  if (e >= OFF_W1 && e < OFF_B1) off = OFF_W1, in_dim = MLP_IN;
  else if (e >= OFF_W2 && e < OFF_B2) off = OFF_W2, in_dim = MLP_H;
  else if (e >= OFF_W3 && e < OFF_B3) off = OFF_W3, in_dim = MLP_H;
  if (off < 0) {
    PT[e] = P[e];
  } else {
    const int r = e - off, i = r >> 6, j = r & (MLP_H - 1);  // destination [i][j]
    PT[e] = P[off + j * in_dim + i];
  }
}

}  // namespace iilbm

using namespace iilbm;

struct iilbm_mlp {
  int device;
  cudaStream_t stream;
  bool own_stream;
  float *P, *m, *v, *norm;
  float *PT;  // P with W1, W2, W3 transposed to [in][64] (for the direct-forcing CTA)
  int t;  // Adam steps taken
  float *partial, *loss;
  int cap_parts;
};

namespace {

#define CKM(call)                \
  do {                           \
    if ((call) != cudaSuccess) { \
      cudaGetLastError();        \
      return IILBM_ERR_CUDA;     \
    }                            \
  } while (0)

int ensure_parts(iilbm_mlp *M, int parts) {
  if (parts <= M->cap_parts) return IILBM_OK;
  if (M->partial) cudaFree(M->partial);
  if (M->loss) cudaFree(M->loss);
  M->partial = nullptr;
  M->loss = nullptr;
  M->cap_parts = 0;
  if (cudaMalloc(&M->partial, (size_t)parts * MLP_NPARAM * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&M->loss, (size_t)parts * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_OOM;
  }
  M->cap_parts = parts;
  return IILBM_OK;
}

// device copy of a host-or-device array (owned copy released by the caller)
template <typename V>
int to_device(const V *src, size_t count, cudaStream_t s, V **dst) {
  *dst = nullptr;
  if (cudaMalloc(dst, std::max<size_t>(count, 1) * sizeof(V)) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_OOM;
  }
  if (count && cudaMemcpyAsync(*dst, src, count * sizeof(V), cudaMemcpyDefault, s) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(*dst);
    *dst = nullptr;
    return IILBM_ERR_CUDA;
  }
  return IILBM_OK;
}

// Rebuild the transposed copy after the parameters change (stream-ordered).
int refresh_transposed(iilbm_mlp *M) {
  k_mlp_transposed<<<(MLP_NPARAM + 255) / 256, 256, 0, M->stream>>>(M->P, M->PT);
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

}  // namespace

namespace iilbm {
const float *mlp_params(const iilbm_mlp *M) { return M->P; }
const float *mlp_params_transposed(const iilbm_mlp *M) { return M->PT; }
const float *mlp_norm(const iilbm_mlp *M) { return M->norm; }
int mlp_device(const iilbm_mlp *M) { return M->device; }
}  // namespace iilbm

extern "C" {

int iilbm_mlp_create(iilbm_mlp_t *out, void *stream) {
  if (!out) return IILBM_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_NO_DEVICE;
  }
  if (prop.major != 10 || prop.minor != 3) return IILBM_ERR_NO_DEVICE;
  iilbm_mlp *M = new (std::nothrow) iilbm_mlp();
  if (!M) return IILBM_ERR_OOM;
  M->device = dev;
  bool ok = cudaMalloc(&M->P, MLP_NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->PT, MLP_NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->m, MLP_NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->v, MLP_NPARAM * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&M->norm, MLP_NORM * sizeof(float)) == cudaSuccess;
  if (stream) {
    M->stream = (cudaStream_t)stream;
  } else {
    ok = ok && cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking) == cudaSuccess;
    M->own_stream = true;
  }
  if (ok) {
    std::vector<float> nm(MLP_NORM, 0.0f);
    for (int i = 0; i < MLP_IN; i++) nm[NORM_IN_ISTD + i] = 1.0f;
    nm[NORM_OUT_SCALE] = nm[NORM_OUT_SCALE + 1] = 1.0f;
    ok = cudaMemsetAsync(M->P, 0, MLP_NPARAM * sizeof(float), M->stream) == cudaSuccess &&
         cudaMemsetAsync(M->PT, 0, MLP_NPARAM * sizeof(float), M->stream) == cudaSuccess &&
         cudaMemsetAsync(M->m, 0, MLP_NPARAM * sizeof(float), M->stream) == cudaSuccess &&
         cudaMemsetAsync(M->v, 0, MLP_NPARAM * sizeof(float), M->stream) == cudaSuccess &&
         cudaMemcpy(M->norm, nm.data(), MLP_NORM * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaStreamSynchronize(M->stream) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    iilbm_mlp_destroy(M);
    return IILBM_ERR_OOM;
  }
  *out = M;
  return IILBM_OK;
}

int iilbm_mlp_destroy(iilbm_mlp_t M) {
  if (!M) return IILBM_ERR_INVALID_ARG;
  if (M->stream) cudaStreamSynchronize(M->stream);
  void *bufs[] = {M->P, M->PT, M->m, M->v, M->norm, M->partial, M->loss};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (M->own_stream && M->stream) cudaStreamDestroy(M->stream);
  delete M;
  return IILBM_OK;
}

int iilbm_mlp_set_params(iilbm_mlp_t M, const float *params) {
  if (!M || !params) return IILBM_ERR_INVALID_ARG;
  CKM(cudaMemcpyAsync(M->P, params, MLP_NPARAM * sizeof(float), cudaMemcpyDefault, M->stream));
  if (refresh_transposed(M)) return IILBM_ERR_CUDA;
  CKM(cudaMemsetAsync(M->m, 0, MLP_NPARAM * sizeof(float), M->stream));
  CKM(cudaMemsetAsync(M->v, 0, MLP_NPARAM * sizeof(float), M->stream));
  M->t = 0;
  CKM(cudaStreamSynchronize(M->stream));
  return IILBM_OK;
}

int iilbm_mlp_get_params(iilbm_mlp_t M, float *params) {
  if (!M || !params) return IILBM_ERR_INVALID_ARG;
  CKM(cudaMemcpyAsync(params, M->P, MLP_NPARAM * sizeof(float), cudaMemcpyDefault, M->stream));
  CKM(cudaStreamSynchronize(M->stream));
  return IILBM_OK;
}

int iilbm_mlp_set_normalization(iilbm_mlp_t M, const float *in_mean, const float *in_istd,
                                const float *out_mean, const float *out_scale) {
  if (!M || !in_mean || !in_istd || !out_mean || !out_scale) return IILBM_ERR_INVALID_ARG;
  float nm[MLP_NORM];
  std::memcpy(nm + NORM_IN_MEAN, in_mean, MLP_IN * sizeof(float));
  std::memcpy(nm + NORM_IN_ISTD, in_istd, MLP_IN * sizeof(float));
  std::memcpy(nm + NORM_OUT_MEAN, out_mean, MLP_OUT * sizeof(float));
  std::memcpy(nm + NORM_OUT_SCALE, out_scale, MLP_OUT * sizeof(float));
  for (int o = 0; o < MLP_OUT; o++)
    if (!(nm[NORM_OUT_SCALE + o] != 0.0f) || !std::isfinite(nm[NORM_OUT_SCALE + o]))
      return IILBM_ERR_INVALID_ARG;
  CKM(cudaMemcpyAsync(M->norm, nm, sizeof nm, cudaMemcpyHostToDevice, M->stream));
  CKM(cudaStreamSynchronize(M->stream));
  return IILBM_OK;
}

int iilbm_mlp_forward(iilbm_mlp_t M, const float *X, int32_t N, float *Y) {
  if (!M || N < 0 || (N > 0 && (!X || !Y))) return IILBM_ERR_INVALID_ARG;
  if (N == 0) return IILBM_OK;
  float *dX = nullptr, *dY = nullptr;
  int rc = to_device(X, (size_t)N * MLP_IN, M->stream, &dX);
  if (!rc && cudaMalloc(&dY, (size_t)N * MLP_OUT * sizeof(float)) != cudaSuccess) rc = IILBM_ERR_OOM;
  if (!rc) {
    k_mlp_forward<<<(N + MLP_SPB - 1) / MLP_SPB, MLP_THREADS, 0, M->stream>>>(M->P, M->norm, dX, N, dY);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(Y, dY, (size_t)N * MLP_OUT * sizeof(float), cudaMemcpyDefault, M->stream) != cudaSuccess ||
        cudaStreamSynchronize(M->stream) != cudaSuccess)
      rc = IILBM_ERR_CUDA;
  }
  cudaGetLastError();
  if (dX) cudaFree(dX);
  if (dY) cudaFree(dY);
  return rc;
}

int iilbm_mlp_gradient(iilbm_mlp_t M, const float *X, const float *T, int32_t N, float *grad,
                       float *loss) {
  if (!M || N <= 0 || !X || !T || !grad) return IILBM_ERR_INVALID_ARG;
  const int parts = (N + MLP_SPB - 1) / MLP_SPB;
  int rc = ensure_parts(M, parts);
  if (rc) return rc;
  float *dX = nullptr, *dT = nullptr, *dG = nullptr, *dL = nullptr;
  rc = to_device(X, (size_t)N * MLP_IN, M->stream, &dX);
  if (!rc) rc = to_device(T, (size_t)N * MLP_OUT, M->stream, &dT);
  if (!rc && (cudaMalloc(&dG, MLP_NPARAM * sizeof(float)) != cudaSuccess ||
              cudaMalloc(&dL, sizeof(float)) != cudaSuccess))
    rc = IILBM_ERR_OOM;
  if (!rc) {
    const float wscale = 1.0f / (float)(N * MLP_OUT);
    k_mlp_fwd_bwd<<<parts, MLP_THREADS, 0, M->stream>>>(M->P, M->norm, dX, dT, nullptr, 0, N,
                                                        wscale, M->partial, M->loss);
    k_mlp_reduce<<<(MLP_NPARAM + 255) / 256, 256, 0, M->stream>>>(
        M->partial, parts, M->loss, wscale, dL, M->P, M->m, M->v, 0, 0.f, 0.f, 0.f, 0.f, dG);
    float hl = 0.0f;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(grad, dG, MLP_NPARAM * sizeof(float), cudaMemcpyDefault, M->stream) != cudaSuccess ||
        cudaMemcpyAsync(&hl, dL, sizeof(float), cudaMemcpyDeviceToHost, M->stream) != cudaSuccess ||
        cudaStreamSynchronize(M->stream) != cudaSuccess)
      rc = IILBM_ERR_CUDA;
    if (!rc && loss) *loss = hl;
  }
  cudaGetLastError();
  void *bufs[] = {dX, dT, dG, dL};
  for (void *b : bufs)
    if (b) cudaFree(b);
  return rc;
}

int iilbm_mlp_train(iilbm_mlp_t M, const float *X, const float *T, int32_t N, const int32_t *order,
                    int32_t steps, int32_t batch, float lr, float beta1, float beta2, float eps,
                    float *losses) {
  if (!M || N <= 0 || !X || !T || !order || steps < 0 || batch <= 0 || (int64_t)steps * batch > (int64_t)1 << 31)
    return IILBM_ERR_INVALID_ARG;
  if (!(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return IILBM_ERR_INVALID_ARG;
  const int parts = (batch + MLP_SPB - 1) / MLP_SPB;
  int rc = ensure_parts(M, parts);
  if (rc) return rc;
  float *dX = nullptr, *dT = nullptr, *dL = nullptr;
  int *dI = nullptr;
  rc = to_device(X, (size_t)N * MLP_IN, M->stream, &dX);
  if (!rc) rc = to_device(T, (size_t)N * MLP_OUT, M->stream, &dT);
  if (!rc) rc = to_device(order, (size_t)steps * batch, M->stream, &dI);
  if (!rc && cudaMalloc(&dL, std::max(1, steps) * sizeof(float)) != cudaSuccess) rc = IILBM_ERR_OOM;
  // indices must address the sample set
  if (!rc) {
    std::vector<int32_t> hI((size_t)steps * batch);
    if (cudaMemcpyAsync(hI.data(), dI, hI.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, M->stream) != cudaSuccess ||
        cudaStreamSynchronize(M->stream) != cudaSuccess)
      rc = IILBM_ERR_CUDA;
    for (size_t q = 0; q < hI.size() && !rc; q++)
      if (hI[q] < 0 || hI[q] >= N) rc = IILBM_ERR_INVALID_ARG;
  }
  const float wscale = 1.0f / (float)(batch * MLP_OUT);
  for (int s = 0; s < steps && !rc; s++) {
    k_mlp_fwd_bwd<<<parts, MLP_THREADS, 0, M->stream>>>(M->P, M->norm, dX, dT, dI, s * batch,
                                                        batch, wscale, M->partial, M->loss);
    M->t++;
    k_mlp_reduce<<<(MLP_NPARAM + 255) / 256, 256, 0, M->stream>>>(
        M->partial, parts, M->loss, wscale, dL + s, M->P, M->m, M->v, M->t, lr, beta1, beta2, eps,
        nullptr);
    if (cudaGetLastError() != cudaSuccess) rc = IILBM_ERR_CUDA;
  }
  if (!rc && steps > 0) rc = refresh_transposed(M);
  if (!rc && losses && steps > 0 &&
      cudaMemcpyAsync(losses, dL, steps * sizeof(float), cudaMemcpyDefault, M->stream) != cudaSuccess)
    rc = IILBM_ERR_CUDA;
  if (cudaStreamSynchronize(M->stream) != cudaSuccess && !rc) rc = IILBM_ERR_CUDA;
  cudaGetLastError();
  void *bufs[] = {dX, dT, dL, dI};
  for (void *b : bufs)
    if (b) cudaFree(b);
  return rc;
}

}  // extern "C"

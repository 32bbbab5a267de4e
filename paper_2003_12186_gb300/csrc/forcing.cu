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

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

namespace iilbm {

template <typename S>
__global__ void __launch_bounds__(DF_THREADS)
    k_direct_forcing(const S *__restrict__ A, const Geom geo, bool odd, DfArgs a, double inv_scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  direct_forcing_cta<S>(A, geo, odd, a, inv_scale, smem_raw);
}

// Shared memory of the forcing kernel for a band of nb nodes and n markers (a moving
// body: its capacities instead, plus the band's construction).
size_t direct_forcing_smem(const iilbm_lattice *h, int nb, int n) {
  const bool mlp = h->ws_mode == WS_MLP;
  if (h->body) nb = h->body_nb;
  size_t b = h->cfg.storage == IILBM_F64 ? df_smem_bytes<double>(nb, n, mlp)
                                         : df_smem_bytes<float>(nb, n, mlp);
  if (h->body) b += df_move_bytes(h->body_words, h->body_nb, h->body_nl);
  return b;
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
  a.band = h->df_band;
  a.nb = h->df_nb;
  a.st = h->df_st;
  a.links = (const DfLink *)h->df_links;
  a.nl = h->df_nl;
  a.moving = h->body != nullptr;
  a.words_max = a.moving ? h->body_words : 0;
  a.nb_max = a.moving ? h->body_nb : 0;
  a.nl_max = a.moving ? h->body_nl : 0;
  a.ig = h->igeom;
  a.status = h->d_status;
  a.jump = h->cfg.jump;
  a.bodyx = h->cfg.body[0];
  a.bodyy = h->cfg.body[1];
  a.rho0 = h->cfg.rho0;
  a.ws_mode = h->ws_mode;
  a.mlp_P = h->mlp ? mlp_params_transposed(h->mlp) : nullptr;
  a.mlp_norm = h->mlp ? mlp_norm(h->mlp) : nullptr;
  a.re = h->re;
  return a;
}

// Cut-link records of a fixed body, one warp per segment.
template <typename T, int BC>
__global__ void __launch_bounds__(128)
    k_df_links(const double *__restrict__ X, int n, GeomC<BC> geo, const int *__restrict__ band,
               int nb, DfLink *links, int *counters, int cap) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= n) return;  // uniform per warp
  df_segment_links<T>(X, n, k, threadIdx.x & 31, geo, band, nb, links, counters, cap,
                      counters + 1);
}

namespace {

// floor / ceil of a coordinate snapped to 2^-24 (as the kernels take them)
long long snap(double v) { return std::llrint(v * QSCALE); }
int qfloor_h(long long v) { return (int)(v >> 24); }
int qceil_h(long long v) { return (int)-((-v) >> 24); }

// Key y * nx + x of node (x, y) wrapped onto the lattice, or -1 off a non-periodic edge.
int node_key(const Geom &g, int x, int y) {
  if (g.bc == IILBM_BC_CHANNEL) {
    if (x < 0 || x >= g.nx) return -1;
  } else {
    x = wrap(x, g.nx);
  }
  if (g.bc == IILBM_BC_PERIODIC) y = wrap(y, g.ny);
  else if (y < 0 || y >= g.ny) return -1;
  return y * g.nx + x;
}

template <typename F>
int with_bc(int bc, F &&f) {
  switch (bc) {
    case IILBM_BC_PERIODIC: return f(std::integral_constant<int, IILBM_BC_PERIODIC>());
    case IILBM_BC_WALLS_Y: return f(std::integral_constant<int, IILBM_BC_WALLS_Y>());
    default: return f(std::integral_constant<int, IILBM_BC_CHANNEL>());
  }
}

}  // namespace

void free_direct_forcing(iilbm_lattice *h) {
  if (h->df_band) cudaFree(h->df_band);
  if (h->df_st) cudaFree(h->df_st);
  if (h->df_links) cudaFree(h->df_links);
  h->df_band = h->df_st = nullptr;
  h->df_links = nullptr;
  h->df_nb = h->df_nl = 0;
}

// Set up the force iteration of the fixed body with markers hx (host copy of X): the
// band (every node of a marker stencil and every candidate destination of a cut link,
// sorted, unique), each stencil node's band index, and the cut-link records.  Returns
// INTERFACE if the iteration's shared memory would exceed 227 KB.
int setup_direct_forcing(iilbm_lattice *h, const double *hx) {
  free_direct_forcing(h);
  const Geom &g = h->igeom;  // the interface's view: a box is bounded on every side
  const int n = h->nm;
  std::vector<int> keys;
  keys.reserve(16 * (size_t)n * 2);
  for (int k = 0; k < n; k++) {
    const int bx = (int)std::floor(hx[2 * k]) - 1, by = (int)std::floor(hx[2 * k + 1]) - 1;
    for (int l = 0; l < 16; l++) {
      const int key = node_key(g, bx + (l & 3), by + (l >> 2));
      if (key >= 0) keys.push_back(key);
    }
  }
  long long cap = 0;
  if (h->cfg.jump) {
    for (int k = 0; k < n; k++) {
      const int kp = (k + 1) % n;
      const long long ax = snap(hx[2 * k]), ay = snap(hx[2 * k + 1]);
      const long long bx = snap(hx[2 * kp]), by = snap(hx[2 * kp + 1]);
      // the destinations the crossing enumeration considers, widened by one node
      const int x0 = qceil_h(std::min(ax, bx)) - 2, x1 = qceil_h(std::max(ax, bx)) + 1;
      const int y0 = qceil_h(std::min(ay, by)) - 2, y1 = qceil_h(std::max(ay, by)) + 1;
      cap += 8LL * (x1 - x0 - 1) * (y1 - y0 - 1);
      for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) {
          const int key = node_key(g, x, y);
          if (key >= 0) keys.push_back(key);
        }
    }
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  const int nb = (int)keys.size();
  if (direct_forcing_smem(h, nb, n) > 227 * 1024) return IILBM_ERR_INTERFACE;
  std::vector<int> st(16 * (size_t)n);
  for (int k = 0; k < n; k++) {
    const int bx = (int)std::floor(hx[2 * k]) - 1, by = (int)std::floor(hx[2 * k + 1]) - 1;
    for (int l = 0; l < 16; l++) {
      const int key = node_key(g, bx + (l & 3), by + (l >> 2));
      st[16 * k + l] =
          key < 0 ? -1 : (int)(std::lower_bound(keys.begin(), keys.end(), key) - keys.begin());
    }
  }
  const int icap = (int)std::max(1LL, cap);
  int *counters = nullptr;
  bool ok = cudaMalloc(&h->df_band, std::max<size_t>(1, keys.size()) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->df_st, st.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->df_links, (size_t)icap * sizeof(DfLink)) == cudaSuccess &&
            cudaMalloc(&counters, 2 * sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (counters) cudaFree(counters);
    free_direct_forcing(h);
    return IILBM_ERR_OOM;
  }
  h->df_nb = nb;
  int rc = IILBM_OK;
  if (cudaMemcpy(h->df_band, keys.data(), keys.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->df_st, st.data(), st.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(counters, 0, 2 * sizeof(int)) != cudaSuccess)
    rc = IILBM_ERR_CUDA;
  int cnt[2] = {0, 0};
  if (!rc && h->cfg.jump) {
    rc = with_bc(g.bc, [&](auto bcc) {
      constexpr int BC = decltype(bcc)::value;
      const int blocks = (n + 3) / 4;
      if (h->cfg.storage == IILBM_F64)
        k_df_links<double, BC><<<blocks, 128, 0, h->stream>>>(h->X, n, GeomC<BC>(g), h->df_band,
                                                              nb, (DfLink *)h->df_links, counters,
                                                              icap);
      else
        k_df_links<float, BC><<<blocks, 128, 0, h->stream>>>(h->X, n, GeomC<BC>(g), h->df_band,
                                                             nb, (DfLink *)h->df_links, counters,
                                                             icap);
      return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
    });
    if (!rc && (cudaMemcpyAsync(cnt, counters, sizeof cnt, cudaMemcpyDeviceToHost, h->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(h->stream) != cudaSuccess))
      rc = IILBM_ERR_CUDA;
    // every destination lies in the band and the capacity bounds the candidates: either
    // failing is a defect, reported rather than run with a partial list
    if (!rc && (cnt[1] != 0 || cnt[0] > icap)) rc = IILBM_ERR_CAPACITY;
  }
  cudaFree(counters);
  if (rc) {
    cudaGetLastError();
    free_direct_forcing(h);
    return rc;
  }
  h->df_nl = cnt[0];
  return IILBM_OK;
}

int launch_direct_forcing(iilbm_lattice *h) {
  const bool odd = h->step & 1;
  const DfArgs a = df_args(h);
  const size_t smem = direct_forcing_smem(h, a.nb, a.n);
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

// ---------------------------------------------------------------- rigid body
// After a step: F_ext = -sum G dX + rho_f V_s (U_c(t) - U_c(t-1)) and T_ext (Eqs. 25-26)
// reduced over the markers; the body's update (Eqs. 27-29 for a free body with its
// springs and dampers, section 4.4's harmonic translation for a prescribed one); then
// every marker placed rigidly, X_k = X_c + R(theta) X0_k, and given the body's velocity
// as its desired velocity, U^D_k = U_c + W x (X_k - X_c).
__global__ void __launch_bounds__(256)
    k_body_update(iilbm_body_dev *b, double *X, double *UD, const double *__restrict__ G,
                  const double *__restrict__ X0, int n, double dX) {
  __shared__ double red[3][8];
  __shared__ double pose[5];  // X_c, Y_c, theta, U_x, U_y (then W in pose[4 + 1])
  __shared__ double wnew;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double xc = b->Xc[0], yc = b->Xc[1];
  double fx = 0, fy = 0, tq = 0;
  for (int q = tid; q < n; q += blockDim.x) {
    const double rx = X[2 * q] - xc, ry = X[2 * q + 1] - yc;
    fx -= G[2 * q] * dX;
    fy -= G[2 * q + 1] * dX;
    tq -= (rx * G[2 * q + 1] - ry * G[2 * q]) * dX;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    tq += __shfl_xor_sync(0xffffffffu, tq, o);
  }
  if (lane == 0) {
    red[0][warp] = fx;
    red[1][warp] = fy;
    red[2][warp] = tq;
  }
  __syncthreads();
  if (tid == 0) {
    fx = fy = tq = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      fx += red[0][w];
      fy += red[1][w];
      tq += red[2][w];
    }
    fx += b->rho_f * b->Vs * (b->Uc[0] - b->Ucp[0]);
    fy += b->rho_f * b->Vs * (b->Uc[1] - b->Ucp[1]);
    tq += b->rho_f * b->Vs / b->m * b->I * (b->W - b->Wp);
    b->F[0] = fx;
    b->F[1] = fy;
    b->F[2] = tq;
    b->t += 1;
    b->Ucp[0] = b->Uc[0];
    b->Ucp[1] = b->Uc[1];
    b->Wp = b->W;
    if (b->mode == IILBM_BODY_PRESCRIBED_X) {
      const double tt = (double)b->t;
      b->Xc[0] = b->Xc0[0] - b->A * sin(b->umax * tt / b->A);
      b->Uc[0] = -b->umax * cos(b->umax * tt / b->A);
    } else {
      const double F[3] = {fx, fy, tq}, inert[3] = {b->m, b->m, b->I};
      double *pos[3] = {&b->Xc[0], &b->Xc[1], &b->th};
      double *vel[3] = {&b->Uc[0], &b->Uc[1], &b->W};
      double *acc[3] = {&b->ac[0], &b->ac[1], &b->wdot};
      const double org[3] = {b->Xc0[0], b->Xc0[1], 0.0};
      for (int d = 0; d < 3; d++) {
        if (!(b->dof & (1 << d))) continue;
        const double a1 = (F[d] - b->k[d] * (*pos[d] - org[d]) - b->c[d] * (*vel[d])) / inert[d];
        const double v0 = *vel[d], a0 = *acc[d];
        *vel[d] = v0 + a1;
        *pos[d] = *pos[d] + v0 + 0.5 * (a0 + a1);
        *acc[d] = a1;
      }
    }
    pose[0] = b->Xc[0];
    pose[1] = b->Xc[1];
    pose[2] = b->th;
    pose[3] = b->Uc[0];
    pose[4] = b->Uc[1];
    wnew = b->W;
  }
  __syncthreads();
  const double ct = cos(pose[2]), st = sin(pose[2]);
  for (int q = tid; q < n; q += blockDim.x) {
    const double ox = X0[2 * q], oy = X0[2 * q + 1];
    const double x = pose[0] + ct * ox - st * oy, y = pose[1] + st * ox + ct * oy;
    X[2 * q] = x;
    X[2 * q + 1] = y;
    UD[2 * q] = pose[3] - wnew * (y - pose[1]);
    UD[2 * q + 1] = pose[4] + wnew * (x - pose[0]);
  }
}

int launch_body_update(iilbm_lattice *h) {
  if (!h->body) return IILBM_OK;
  k_body_update<<<1, 256, 0, h->stream>>>(h->body, h->X, h->aux, h->Gdf, h->body_X0, h->nm,
                                          h->ip.dX);
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

void free_body(iilbm_lattice *h) {
  if (h->body) cudaFree(h->body);
  if (h->body_X0) cudaFree(h->body_X0);
  h->body = nullptr;
  h->body_X0 = nullptr;
  h->body_words = h->body_nb = h->body_nl = 0;
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

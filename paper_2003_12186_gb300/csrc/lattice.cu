// lattice.cu -- the Eulerian side of the II-LBM step on sm_103a:
//   * the fused AA-pattern stream-collide (SRT Eq. 14 + Guo Eq. 21, or MRT Eq. 15 +
//     Guo Eq. 22), which also adds the jump of Eq. 47 to the populations it reads on
//     cut links and the spread tangential force of Eq. 46;
//   * velocity interpolation at the markers (Eq. 20) with the marker update;
//   * state conversion (set / get populations, equilibrium start) and macroscopic
//     fields.
//
// Memory layout: populations df_i = f_i - w_i rho0 stored as structure of arrays
// A[i][y][x] (row pitch rounded to 32 elements) in the storage precision, updated in
// place with the AA pattern: an even step reads slot i of node x and writes the
// post-collision f*_i into slot opp(i) of the same node; an odd step reads slot
// opp(i) of the upstream node x - e_i and writes f*_i into slot i of the downstream
// node x + e_i.  Each node only touches slots no other node touches in that step,
// so one array suffices and every step moves 2 x 9 values per node.
#include "interface_dev.cuh"
#include "lattice_dev.cuh"
#include "sc_tma_dev.cuh"

#include <cudaTypedefs.h>

#include <cmath>

namespace iilbm {

// Lean kernels: one block per (sub-)tile; a flagged tile is left to the forced kernel.
template <typename S, int COLL, bool ODD, int BC>
__global__ void __launch_bounds__(32 * TILE_Y)
    k_stream_collide(S *__restrict__ A, const unsigned *__restrict__ flags,
                     const unsigned *__restrict__ tag, const Geom geo,
                     const CollP<typename Store<S>::T> p, int *status) {
  const int xb = blockIdx.x * 32, yb = blockIdx.y * TILE_Y;
  if (flags[blockIdx.y * geo.ntx + xb / TILE_X] == *tag) return;  // uniform per block
  sc_scalar_rows<S, COLL, ODD, BC, false>(A, nullptr, nullptr, nullptr, geo, p, status, xb, yb);
}

// At least three resident blocks per SM (<= 85 registers): the odd step would otherwise
// drop to two and lose a third of its memory parallelism.  BODY = false (no body force):
// the lean tiles carry no force at all and the collision drops Guo's source terms.
template <typename S, int COLL, bool ODD, int BC, bool BODY>
__global__ void __launch_bounds__(32 * VEC_ROWS, 3)
    k_stream_collide_vec(S *__restrict__ A, const unsigned *__restrict__ flags,
                         const unsigned *__restrict__ tag, const Geom geo,
                         const CollP<typename Store<S>::T> p, int *status) {
  constexpr int W = 32 * Vec<S>::V;  // nodes per warp row
  const int xb = blockIdx.x * W, yb = blockIdx.y * VEC_ROWS;
  if (flags[blockIdx.y * geo.ntx + xb / TILE_X] == *tag) return;  // uniform per block
  sc_vec_rows<S, COLL, ODD, BC, false, Vec<S>::V, BODY>(A, nullptr, nullptr, nullptr, geo, p,
                                                         status, xb, yb);
}

// Forced kernels: blocks stride over the list of flagged tiles of this step (and first
// prepare the next interface phase's buffer and marker snapshot, marker_prep).
template <typename S, int COLL, bool ODD, int BC>
__global__ void __launch_bounds__(32 * TILE_Y)
    k_stream_collide_forced(S *__restrict__ A, typename Store<S>::T *__restrict__ Jf,
                            typename Store<S>::T *__restrict__ gf,
                            typename Store<S>::T *__restrict__ uf,
                            const int *__restrict__ list, const int *__restrict__ count,
                            const Geom geo, const CollP<typename Store<S>::T> p, int *status,
                            MarkerPrep mp) {
  marker_prep(mp);
  const int n = *count;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int tile = list[t];
    const int tx = (tile % geo.ntx) * TILE_X, ty = (tile / geo.ntx) * TILE_Y;
    for (int sub = 0; sub < TILE_X; sub += 32)
      sc_scalar_rows<S, COLL, ODD, BC, true>(A, Jf, gf, uf, geo, p, status, tx + sub, ty);
  }
}

// Budgeted like the lean kernel (three blocks per SM, <= 85 registers, a few spilled):
// its blocks run beside the lean stream-collide, and each one then takes the place of
// one lean block instead of two.
template <typename S, int COLL, bool ODD, int BC>
__global__ void __launch_bounds__(32 * VEC_ROWS, 3)
    k_stream_collide_vec_forced(S *__restrict__ A, typename Store<S>::T *__restrict__ Jf,
                                typename Store<S>::T *__restrict__ gf,
                                typename Store<S>::T *__restrict__ uf,
                                const int *__restrict__ list, const int *__restrict__ count,
                                const Geom geo, const CollP<typename Store<S>::T> p,
                                int *status, MarkerPrep mp) {
  constexpr int W = 32 * Vec<S>::V;
  marker_prep(mp);
  const int n = *count;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int tile = list[t];
    const int tx = (tile % geo.ntx) * TILE_X, ty = (tile / geo.ntx) * TILE_Y;
    for (int sub = 0; sub < TILE_X; sub += W)
      sc_vec_rows<S, COLL, ODD, BC, true>(A, Jf, gf, uf, geo, p, status, tx + sub, ty);
  }
}

// Macroscopic density deviation and velocity of node (x, y) of the current state:
// populations (AA location) plus the jump, force g of the current interface.
template <typename S>
__device__ inline void node_macros(const S *A, const typename Store<S>::T *Jf,
                                   const typename Store<S>::T *gf, const Geom &geo,
                                   const CollP<typename Store<S>::T> &p, bool odd, int x,
                                   int y, double &drho, double &ux, double &uy) {
  using T = typename Store<S>::T;
  const long long here = (long long)y * geo.pitch + x;
  T f[9];
#pragma unroll
  for (int i = 0; i < 9; i++) f[i] = Store<S>::ld(A[aa_loc(geo, odd, i, x, y)]) * p.inv_scale;
#pragma unroll
  for (int i = 1; i < 9; i++) f[i] += Jf[(i - 1) * geo.plane + here];
  // the collision's velocity: (j + g/2) / rho with Guo's force, j / rho with the simple one
  const T h = p.he ? T(0) : T(0.5);
  const T gx = p.bodyx + gf[here], gy = p.bodyy + gf[geo.plane + here];
  const T d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const T jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const T jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  const T ir = T(1) / (p.rho0 + d);
  drho = double(d);
  ux = double((jx + h * gx) * ir);
  uy = double((jy + h * gy) * ir);
}

// Velocity interpolation U_k = sum_x u(x) delta_h(x - X_k) (Eq. 20), one thread per
// marker (interp_marker); a membrane marker then moves, X_k += U_k.  u is the
// collision velocity of the step (jump and g/2 included) that the forced stream-collide
// left in uf for every node of the flagged tiles -- which cover every marker's stencil
// -- so this runs right after the forced kernel.  (The pipelined step runs it fused
// with the next interface phase instead: k_interface<T, true>.)
template <typename T>
__global__ void k_interp(const T *__restrict__ uf, const Geom geo, double *X,
                         const long long *__restrict__ Xq, int n, double *U, int moves) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) interp_marker<T>(uf, geo, X, Xq, k, U, moves);
}

template <typename S>
__global__ void k_macros(const S *__restrict__ A, const typename Store<S>::T *__restrict__ Jf,
                         const typename Store<S>::T *__restrict__ gf, const Geom geo,
                         const CollP<typename Store<S>::T> p, bool odd, double *drho,
                         double *ux, double *uy) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= geo.nx) return;
  double d, u, v;
  node_macros<S>(A, Jf, gf, geo, p, odd, x, y, d, u, v);
  const long long o = (long long)y * geo.nx + x;
  if (drho) drho[o] = d;
  if (ux) ux[o] = u;
  if (uy) uy[o] = v;
}

// State in: natural-layout FP64 df[9][ny][nx], or the equilibrium (Eq. 23) of
// rho(x), u(x) (rho0 / zero where the pointer is null).
template <typename S>
__global__ void k_set_populations(S *A, const Geom geo, const CollP<typename Store<S>::T> p,
                                  bool odd, const double *df, int equilibrium,
                                  const double *rho, const double *ux, const double *uy,
                                  double rho0) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= geo.nx) return;
  const long long o = (long long)y * geo.nx + x;
  const long long N = (long long)geo.nx * geo.ny;
  double v[9];
  if (equilibrium) {
    const double d = rho ? rho[o] - rho0 : 0.0;
    const double u = ux ? ux[o] : 0.0, w = uy ? uy[o] : 0.0;
    const double r = rho0 + d, u2 = u * u + w * w;
    for (int i = 0; i < 9; i++) {
      const double eu = cx(i) * u + cy(i) * w;
      v[i] = wt<double>(i) * (d + r * (3.0 * eu + 4.5 * eu * eu - 1.5 * u2));
    }
  } else {
    for (int i = 0; i < 9; i++) v[i] = df[i * N + o];
  }
  for (int i = 0; i < 9; i++)
    A[aa_loc(geo, odd, i, x, y)] =
        Store<S>::st((typename Store<S>::T)(v[i]) * p.scale);
}

template <typename S>
__global__ void k_get_populations(const S *A, const Geom geo,
                                  const CollP<typename Store<S>::T> p, bool odd, double *df) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= geo.nx) return;
  const long long o = (long long)y * geo.nx + x;
  const long long N = (long long)geo.nx * geo.ny;
  for (int i = 0; i < 9; i++)
    df[i * N + o] = double(Store<S>::ld(A[aa_loc(geo, odd, i, x, y)]) * p.inv_scale);
}

// The jump field of the current state: J[i - 1][y][x] in population units (i = 1..8),
// FP64 natural layout.
template <typename T>
__global__ void k_get_jump(const T *__restrict__ J, const Geom geo, double *out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= geo.nx) return;
  const long long N = (long long)geo.nx * geo.ny;
  for (int i = 0; i < 8; i++)
    out[i * N + (long long)y * geo.nx + x] = (double)J[i * geo.plane + (long long)y * geo.pitch + x];
}

// ------------------------------------------------------------ channel ends
// Inflow / outflow of a channel on the streamed state (one thread per row), after every
// stream-collide: inflow column x = 0 by non-equilibrium extrapolation from column 1,
//   f_i(0,y) = f_eq_i(rho(1,y), u_in(y)) + [f_i(1,y) - f_eq_i(rho(1,y), u(1,y))],
// u_in(y) = 4 u_max (y + 1/2)(ny - y - 1/2) / ny^2 (parabolic, v = 0); outflow column
// nx - 1: the populations with e_x < 0 copied from column nx - 2 (zero gradient).
template <typename S>
__global__ void k_channel_bc(S *A, const Geom geo, const CollP<typename Store<S>::T> p,
                             bool odd, double u_max) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y < geo.ny) channel_bc_row<S>(A, geo, p, odd, u_max, y);
}

// The edge of a box (the outflow or walled boxes of section 4), one thread per edge node:
// the bottom and top rows, then the left and right columns without their corners.
template <typename S>
__global__ void k_box_bc(S *A, const Geom geo, const CollP<typename Store<S>::T> p, bool odd,
                         bool outflow) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nx = geo.nx, ny = geo.ny;
  int x, y;
  if (t < 2 * nx) {
    x = t % nx;
    y = t < nx ? 0 : ny - 1;
  } else if (t < 2 * nx + 2 * (ny - 2)) {
    const int r = t - 2 * nx;
    x = r < ny - 2 ? 0 : nx - 1;
    y = 1 + r % (ny - 2);
  } else {
    return;
  }
  box_bc_node<S>(A, geo, p, odd, outflow, x, y);
}

// ------------------------------------------------------------------ dispatch
template <typename F>
static int dispatch_storage(int storage, F &&f) {
  switch (storage) {
    case IILBM_F64: return f((double *)nullptr);
    case IILBM_F32: return f((float *)nullptr);
    case IILBM_F16: return f((__half *)nullptr);
    case IILBM_BF16: return f((__nv_bfloat16 *)nullptr);
  }
  return IILBM_ERR_INVALID_ARG;
}

static int last_error() {
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

// The interior tiles of the TMA stream-collide (see sc_tma_dev.cuh); false if none.
static bool tma_tiles(const Geom &g, TmaTiles &t) {
  t.tx0 = 1;
  t.ntx_i = g.nx >= TMA_W + TMA_W + 2 * TMA_HALO ? (g.nx - TMA_W - TMA_HALO) / TMA_W : 0;
  t.ty0 = 1;
  t.nty_i = g.ny >= 2 * TMA_R + 1 ? (g.ny - TMA_R - 1) / TMA_R : 0;
  return t.ntx_i > 0 && t.nty_i > 0;
}

bool uses_tma_sc(const iilbm_lattice *h, bool odd) {
  TmaTiles t;
  return (h->tma_sc == 1 || (h->tma_sc == 2 && odd)) && h->vector_sc && h->cfg.storage == IILBM_F32 && h->geom.nx % 4 == 0 &&
         tma_tiles(h->geom, t);
}

// Tensor maps of the FP32 populations, dims (nx, ny, 9) with the row pitch and plane
// strides, boxes 136 x 8, 128 x 8 and 124 x 8 (no swizzle, no out-of-bounds use).
static bool tma_maps(iilbm_lattice *h) {
  if (h->tmap_A == h->A) return true;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const Geom &g = h->geom;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * sizeof(float),
                                 (cuuint64_t)g.plane * sizeof(float)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t width[3] = {TMA_LW_ODD, TMA_W, TMA_SW};
  for (int q = 0; q < 3; q++) {
    const cuuint32_t box[3] = {width[q], TMA_R, 1};
    if (encode(&h->tmap[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->A, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return false;
  }
  h->tmap_A = h->A;
  return true;
}

// The lean stream-collide as the TMA kernel over the interior tiles plus the register
// path over the rest; false (nothing launched) where it does not apply.
template <typename S, int COLL, bool ODD, int BC, bool BODY>
static bool sc_launch_tma(iilbm_lattice *h, const unsigned *fl, const unsigned *tag,
                          const CollP<typename Store<S>::T> &p) {
  if constexpr (!std::is_same<S, float>::value) {
    return false;
  } else {
    TmaTiles t;
    if (!uses_tma_sc(h, ODD) || !tma_tiles(h->geom, t) || !tma_maps(h)) return false;
    const Geom &g = h->geom;
    auto kern = k_stream_collide_tma<COLL, ODD, BODY>;
    constexpr size_t smem = TmaSmem<ODD>::bytes;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    static int sms = 0;
    if (!sms) {
      cudaDeviceProp prop;
      if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return false;
      sms = prop.multiProcessorCount;
    }
    const int interior = t.ntx_i * t.nty_i;
    const int nty = (g.ny + TILE_Y - 1) / TILE_Y;
    const int grid = std::min(interior, sms);
    if ((interior + grid - 1) / grid > 32 * TMA_MASK_WORDS) return false;  // beyond the mask
    kern<<<grid, TMA_THREADS, smem, h->stream>>>(
        h->tmap[ODD ? 0 : 1], h->tmap[1], h->tmap[2], (float *)h->A, fl, tag, g, t, p,
        h->d_status);
    k_stream_collide_vec_edge<S, COLL, ODD, BC, BODY>
        <<<g.ntx * nty - interior, 32 * VEC_ROWS, 0, h->stream>>>((S *)h->A, fl, tag, g, p,
                                                                  h->d_status, t, nty);
    return true;
  }
}

template <typename S, int COLL, bool ODD, int BC>
static void sc_launch_bc(iilbm_lattice *h, cudaStream_t forced_stream) {
  using T = typename Store<S>::T;
  const Geom &g = h->geom;
  const int b = h->step & 1;
  T *J = (T *)h->Jb[b], *gf = (T *)h->gb[b];
  const unsigned *fl = h->flagsb[b];
  const CollP<T> p = make_collp<T>(h->cfg);
  constexpr int V = Vec<S>::V;
  const int nyt = (g.ny + TILE_Y - 1) / TILE_Y;
  const bool vec = h->vector_sc && g.nx % V == 0;
  const dim3 vgrid((g.nx + 32 * V - 1) / (32 * V), nyt);
  const bool body = h->cfg.body[0] != 0.0 || h->cfg.body[1] != 0.0;
  if (vec && (body ? sc_launch_tma<S, COLL, ODD, BC, true>(h, fl, h->tagb[b], p)
                   : sc_launch_tma<S, COLL, ODD, BC, false>(h, fl, h->tagb[b], p))) {
    // interior tiles by TMA, the rest by the register path
  } else if (vec && !body)
    k_stream_collide_vec<S, COLL, ODD, BC, false><<<vgrid, 32 * VEC_ROWS, 0, h->stream>>>(
        (S *)h->A, fl, h->tagb[b], g, p, h->d_status);
  else if (vec)
    k_stream_collide_vec<S, COLL, ODD, BC, true><<<vgrid, 32 * VEC_ROWS, 0, h->stream>>>(
        (S *)h->A, fl, h->tagb[b], g, p, h->d_status);
  else
    k_stream_collide<S, COLL, ODD, BC><<<dim3((g.nx + 31) / 32, nyt), dim3(32, TILE_Y), 0,
                                         h->stream>>>((S *)h->A, fl, h->tagb[b], g, p,
                                                      h->d_status);
  if (h->nm == 0) return;  // no interface: no flagged tiles
  const int grid = h->forced_grid;
  const MarkerPrep mp{h->X, h->Xp, h->Xq, h->Xqp, pipelined(h) ? 2 * h->nm : 0, h->tagb[b ^ 1],
                      h->tile_count[b ^ 1]};
  if (vec)
    k_stream_collide_vec_forced<S, COLL, ODD, BC><<<grid, 32 * VEC_ROWS, 0, forced_stream>>>(
        (S *)h->A, J, gf, (T *)h->uf, h->tile_list[b], h->tile_count[b], g, p, h->d_status, mp);
  else
    k_stream_collide_forced<S, COLL, ODD, BC><<<grid, dim3(32, TILE_Y), 0, forced_stream>>>(
        (S *)h->A, J, gf, (T *)h->uf, h->tile_list[b], h->tile_count[b], g, p, h->d_status, mp);
}

template <typename S, int COLL, bool ODD>
static void sc_launch(iilbm_lattice *h, cudaStream_t forced_stream) {
  if (h->geom.bc == IILBM_BC_PERIODIC)
    sc_launch_bc<S, COLL, ODD, IILBM_BC_PERIODIC>(h, forced_stream);
  else if (h->geom.bc == IILBM_BC_WALLS_Y)
    sc_launch_bc<S, COLL, ODD, IILBM_BC_WALLS_Y>(h, forced_stream);
  else
    sc_launch_bc<S, COLL, ODD, IILBM_BC_CHANNEL>(h, forced_stream);
}

// Launch the lean stream-collide on the handle's stream and the forced one (flagged
// tiles) on forced_stream (which may be the same stream).
int launch_stream_collide(iilbm_lattice *h, cudaStream_t forced_stream) {
  const bool odd = h->step & 1;
  return dispatch_storage(h->cfg.storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    if (h->cfg.collision == IILBM_SRT) {
      if (odd) sc_launch<S, IILBM_SRT, true>(h, forced_stream);
      else sc_launch<S, IILBM_SRT, false>(h, forced_stream);
    } else {
      if (odd) sc_launch<S, IILBM_MRT, true>(h, forced_stream);
      else sc_launch<S, IILBM_MRT, false>(h, forced_stream);
    }
    return last_error();
  });
}

int launch_interp(iilbm_lattice *h, cudaStream_t s) {
  if (h->nm == 0) return IILBM_OK;
  const int blocks = (h->nm + 127) / 128;
  if (h->cfg.storage == IILBM_F64)
    k_interp<double><<<blocks, 128, 0, s>>>((const double *)h->uf, h->igeom, h->X, h->Xq, h->nm,
                                            h->U, h->ip.moves);
  else
    k_interp<float><<<blocks, 128, 0, s>>>((const float *)h->uf, h->igeom, h->X, h->Xq, h->nm,
                                           h->U, h->ip.moves);
  return last_error();
}

int launch_channel_bc(iilbm_lattice *h) {
  const bool box = h->cfg.bc == IILBM_BC_BOX_OUTFLOW || h->cfg.bc == IILBM_BC_BOX_WALL;
  if (h->geom.bc != IILBM_BC_CHANNEL && !box) return IILBM_OK;
  const bool odd = h->step & 1;  // the state just produced
  return dispatch_storage(h->cfg.storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    using T = typename Store<S>::T;
    if (box) {
      const int edge = 2 * h->geom.nx + 2 * (h->geom.ny - 2);
      k_box_bc<S><<<(edge + 127) / 128, 128, 0, h->stream>>>(
          (S *)h->A, h->geom, make_collp<T>(h->cfg), odd, h->cfg.bc == IILBM_BC_BOX_OUTFLOW);
    } else {
      k_channel_bc<S><<<(h->geom.ny + 127) / 128, 128, 0, h->stream>>>(
          (S *)h->A, h->geom, make_collp<T>(h->cfg), odd, h->cfg.u_max);
    }
    return last_error();
  });
}

int launch_macros(iilbm_lattice *h, double *drho, double *ux, double *uy) {
  const bool odd = h->step & 1;
  return dispatch_storage(h->cfg.storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    using T = typename Store<S>::T;
    dim3 grid((h->geom.nx + 127) / 128, h->geom.ny);
    const int b = h->step & 1;
    k_macros<S><<<grid, 128, 0, h->stream>>>((const S *)h->A, (const T *)h->Jb[b],
                                             (const T *)h->gb[b], h->geom, make_collp<T>(h->cfg),
                                             odd, drho, ux, uy);
    return last_error();
  });
}

int launch_get_jump(iilbm_lattice *h, double *out) {
  const int b = h->step & 1;
  dim3 grid((h->geom.nx + 127) / 128, h->geom.ny);
  if (h->cfg.storage == IILBM_F64)
    k_get_jump<double><<<grid, 128, 0, h->stream>>>((const double *)h->Jb[b], h->geom, out);
  else
    k_get_jump<float><<<grid, 128, 0, h->stream>>>((const float *)h->Jb[b], h->geom, out);
  return last_error();
}

int launch_set_populations(iilbm_lattice *h, const double *df, bool equilibrium,
                           const double *rho, const double *ux, const double *uy) {
  const bool odd = h->step & 1;
  return dispatch_storage(h->cfg.storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    using T = typename Store<S>::T;
    dim3 grid((h->geom.nx + 127) / 128, h->geom.ny);
    k_set_populations<S><<<grid, 128, 0, h->stream>>>((S *)h->A, h->geom, make_collp<T>(h->cfg),
                                                      odd, df, equilibrium ? 1 : 0, rho, ux, uy,
                                                      h->cfg.rho0);
    return last_error();
  });
}

int launch_get_populations(iilbm_lattice *h, double *df) {
  const bool odd = h->step & 1;
  return dispatch_storage(h->cfg.storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    using T = typename Store<S>::T;
    dim3 grid((h->geom.nx + 127) / 128, h->geom.ny);
    k_get_populations<S><<<grid, 128, 0, h->stream>>>((const S *)h->A, h->geom,
                                                      make_collp<T>(h->cfg), odd, df);
    return last_error();
  });
}

}  // namespace iilbm

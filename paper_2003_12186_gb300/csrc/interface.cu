// interface.cu -- the Lagrangian side of the II-LBM step on sm_103a (FP64 geometry).
//
// One kernel does the interface work of a time level; each block takes 8 consecutive
// segments and the 9 markers at their ends (the last one is also the next block's:
// computed twice, written by its owner only):
//   * the marker pass, one thread per marker k: the Lagrangian force (Eq. 19 spring, a
//     rest-length spring, or a prescribed / directly forced force), its normal /
//     tangential split (Eqs. 31-32, 46), the marker's coordinates snapped to 2^-24 (kept
//     in shared memory for the segment pass and written out for the interpolation);
//   * the segment pass, one warp per segment k -> k+1 (4 warps take the 8 segments of
//     a block in turn): every lattice link x - e_i -> x
//     crossing it (exact 64-bit integer orientation tests on the snapped coordinates,
//     degenerate contacts resolved by displacing lattice nodes by (eps, eps^2)), each
//     adding the jump [[f_i]] = +-w_i/c_s^2 Fn of Eq. 32 to the jump field of its
//     destination node (Eq. 47); and flagging every touched tile, appending newly
//     flagged tiles to the tile list that the forced stream-collide walks; then 16 of
//     its lanes spread the tangential force of the segment's first marker with Peskin's
//     four-point kernel (Eq. 46) into the force field.
// In the pipelined step the same kernel first interpolates the velocity of the level
// just streamed at the markers and moves them (Eq. 20, X += U): a block needs the new
// positions of markers a - 1 .. a + 9, so it interpolates those 11 (its 8 and a halo
// of 3, recomputed with the same arithmetic) from the snapshot of the old positions
// that the forced stream-collide took, since the owners of the halo markers overwrite
// X meanwhile.  The side stream then runs two kernels per step (forced stream-collide,
// this one) beside the lean stream-collide.  (The batched executor keeps the three
// passes as separate launches over its flattened marker list.)
// The dense [.][ny][pitch] fields are only ever touched on O(interface length) tiles.
#include "interface_dev.cuh"
#include "spline_dev.cuh"

#include <cmath>

namespace iilbm {

template <typename T, bool INTERP, int BC>
__global__ void __launch_bounds__(32 * IFACE_WARPS)
    k_interface(double *X, const double *__restrict__ aux, int n, iilbm_interface_params ip,
                int jump, GeomC<BC> geo, T *gf, T *Jf, TileBuf tb, double *G, double *Fn,
                double *nrm, long long *Xq, int *status, InterpIn<T> in) {
  interface_block<T, INTERP, IFACE_WARPS>(blockIdx.x * SEGS_PER_BLOCK, X, aux, n, ip, jump, geo,
                                          gf, Jf, tb, G, Fn, nrm, Xq, status, in);
}

template <typename T, bool INTERP, int BC>
static void launch_interface_bc(iilbm_lattice *h, int buf, cudaStream_t s) {
  const int n = h->nm;
  const double *aux = h->ip.model == IILBM_DIRECT ? h->Gdf : h->aux;
  const TileBuf tb{h->flagsb[buf], h->tagb[buf], h->tile_list[buf], h->tile_count[buf],
                   h->d_tiles_total};
  const InterpIn<T> in{(const T *)h->uf, h->Xp, h->Xqp, h->U, h->ip.moves};
  const int blocks = (n + SEGS_PER_BLOCK - 1) / SEGS_PER_BLOCK;
  k_interface<T, INTERP, BC><<<blocks, 32 * IFACE_WARPS, 0, s>>>(
      h->X, aux, n, h->ip, h->cfg.jump, GeomC<BC>(h->igeom), (T *)h->gb[buf], (T *)h->Jb[buf], tb,
      h->G, h->Fn, h->nrm, h->Xq, h->d_status, in);
}

template <typename T, bool INTERP>
static int launch_interface(iilbm_lattice *h, int buf, cudaStream_t s) {
  switch (h->igeom.bc) {
    case IILBM_BC_PERIODIC: launch_interface_bc<T, INTERP, IILBM_BC_PERIODIC>(h, buf, s); break;
    case IILBM_BC_WALLS_Y: launch_interface_bc<T, INTERP, IILBM_BC_WALLS_Y>(h, buf, s); break;
    default: launch_interface_bc<T, INTERP, IILBM_BC_CHANNEL>(h, buf, s);
  }
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

// ----------------------------------------------------- spline interface phase
// A spline interface (interface parameter curve = m >= 1; see spline_dev.cuh) runs its
// interface phase in four launches (not fused with the interpolation): the spline
// coefficients of the marker coordinates; the marker pass (force, the split with the
// spline's normal and |X_s| = |X'(k)| / dX, snapped coordinates, tangential spread); the
// spline coefficients of Fn; and the segment pass over the m chords of every segment,
// one warp per chord, the jump at a crossing taken from the spline of Fn.

// Spline coefficients of comps interleaved periodic sequences v[stride * k + a].
__global__ void k_spline_coeffs(const double *__restrict__ v, int n, int stride, int comps,
                                double *c) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * comps) return;
  const int k = t / comps, a = t - k * comps;
  c[stride * k + a] = spline_coeff(v + a, n, stride, k);
}

template <typename T, int BC>
__global__ void __launch_bounds__(128)
    k_spline_markers(const double *__restrict__ X, const double *__restrict__ aux, int n,
                     iilbm_interface_params ip, int jump, GeomC<BC> geo, T *gf, double *G,
                     double *Fn, double *nrm, long long *Xq, int *status,
                     const double *__restrict__ cs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) interface_marker<T>(X, aux, n, j, ip, jump, geo, gf, G, Fn, nrm, Xq, status, cs);
}

// Point j / m of segment k of the spline, snapped (XQ_OUT outside the covered region).
__device__ inline void spline_point(const double *__restrict__ cs, int n, int m, int q,
                                    long long &px, long long &py) {
  const int k = q / m, j = q - k * m;
  const double sp = (double)k + (double)j / m;
  const double t = sp - floor(sp);
  const double x = spline_at<double>(cs, n, 2, k, t), y = spline_at<double>(cs + 1, n, 2, k, t);
  const bool inside = isfinite(x) && isfinite(y) && in_region(x, y);
  px = inside ? __double2ll_rn(x * QSCALE) : XQ_OUT;
  py = inside ? __double2ll_rn(y * QSCALE) : XQ_OUT;
}

template <typename T, int BC>
__global__ void __launch_bounds__(128)
    k_spline_segments(const double *__restrict__ cs, const double *__restrict__ cf, int n, int m,
                      int jump, GeomC<BC> geo, T *Jf, TileBuf tb) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= n * m) return;  // uniform per warp
  const int lane = threadIdx.x & 31;
  const unsigned tag = *tb.tag;
  const int q2 = q + 1 == n * m ? 0 : q + 1;
  long long ax, ay, bx, by;
  spline_point(cs, n, m, q, ax, ay);
  spline_point(cs, n, m, q2, bx, by);
  const int k = q / m, j = q - k * m;
  segment_jump<T>(ax, ay, bx, by, lane, jump, geo, Jf, tb, tag, [&](int i, int s1, T t) -> T {
    // Fn at spline parameter k + (j + t) / m
    double u = ((double)j + (double)t) / m;
    int kk = k;
    if (u >= 1.0) {
      u -= 1.0;
      kk = kk + 1 == n ? 0 : kk + 1;
    }
    const double F = spline_at<double>(cf, n, 1, kk, u);
    if (sizeof(T) == 8) return T((double)s1 * 3.0 * wt<double>(i) * F);
    return T((float)s1 * 3.0f * wt<float>(i) * (float)F);
  });
}

template <typename T, int BC>
static void launch_spline_bc(iilbm_lattice *h, int buf, cudaStream_t s) {
  const int n = h->nm, m = h->ip.curve;
  const double *aux = h->ip.model == IILBM_DIRECT ? h->Gdf : h->aux;
  const TileBuf tb{h->flagsb[buf], h->tagb[buf], h->tile_list[buf], h->tile_count[buf],
                   h->d_tiles_total};
  k_spline_coeffs<<<(2 * n + 127) / 128, 128, 0, s>>>(h->X, n, 2, 2, h->spl_c);
  k_spline_markers<T, BC><<<(n + 127) / 128, 128, 0, s>>>(
      h->X, aux, n, h->ip, h->cfg.jump, GeomC<BC>(h->igeom), (T *)h->gb[buf], h->G, h->Fn, h->nrm,
      h->Xq, h->d_status, h->spl_c);
  k_spline_coeffs<<<(n + 127) / 128, 128, 0, s>>>(h->Fn, n, 1, 1, h->spl_f);
  const long long threads = 32LL * n * m;
  k_spline_segments<T, BC><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
      h->spl_c, h->spl_f, n, m, h->cfg.jump, GeomC<BC>(h->igeom), (T *)h->Jb[buf], tb);
}

template <typename T>
static int launch_spline(iilbm_lattice *h, int buf, cudaStream_t s) {
  switch (h->igeom.bc) {
    case IILBM_BC_PERIODIC: launch_spline_bc<T, IILBM_BC_PERIODIC>(h, buf, s); break;
    case IILBM_BC_WALLS_Y: launch_spline_bc<T, IILBM_BC_WALLS_Y>(h, buf, s); break;
    default: launch_spline_bc<T, IILBM_BC_CHANNEL>(h, buf, s);
  }
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

// ---------------------------------------------------------- interface phase
// Bring buffer buf to the interface of the markers X.  The buffer arrives clean: its
// jump / force entries were zeroed by the forced stream-collide that consumed them, its
// counters reset and its tag advanced by the forced stream-collide of the level before
// (or by the set-up), so stale flags from earlier time levels no longer match.
int launch_interface_phase(iilbm_lattice *h, int buf, cudaStream_t s) {
  if (h->nm == 0) return IILBM_OK;
  if (h->ip.curve > 0)
    return h->cfg.storage == IILBM_F64 ? launch_spline<double>(h, buf, s)
                                       : launch_spline<float>(h, buf, s);
  return h->cfg.storage == IILBM_F64 ? launch_interface<double, false>(h, buf, s)
                                     : launch_interface<float, false>(h, buf, s);
}

// The pipelined step's side-stream tail: interpolation of the level just streamed (with
// the marker move) and the interface phase of the next level in its buffer, one kernel.
// Needs the snapshot X -> Xp, Xq -> Xqp of the forced stream-collide before it.
int launch_interp_interface(iilbm_lattice *h, cudaStream_t s) {
  if (h->nm == 0) return IILBM_OK;
  const int buf = (int)((h->step + 1) & 1);
  return h->cfg.storage == IILBM_F64 ? launch_interface<double, true>(h, buf, s)
                                     : launch_interface<float, true>(h, buf, s);
}

}  // namespace iilbm

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

#include <cmath>

namespace iilbm {

constexpr int SEGS_PER_BLOCK = 8;
// Warps per block: each takes segments w, w + IFACE_WARPS, ...  The kernel waits on
// memory most of its time, beside the register-heavy lean stream-collide; fewer warps
// per segment hold fewer of the registers that stream-collide blocks could use.
constexpr int IFACE_WARPS = 4;

// Inputs of the fused interpolation (INTERP = true): the collision velocity of the
// streamed level and that level's marker snapshot; U and the new X go to the markers.
template <typename T>
struct InterpIn {
  const T *uf;
  const double *Xp;
  const long long *Xqp;
  double *U;
  int moves;
};

template <typename T, bool INTERP>
__global__ void __launch_bounds__(32 * IFACE_WARPS)
    k_interface(double *X, const double *__restrict__ aux, int n, iilbm_interface_params ip,
                int jump, Geom geo, T *gf, T *Jf, TileBuf tb, double *G, double *Fn,
                double *nrm, long long *Xq, int *status, InterpIn<T> in) {
  __shared__ double sx[SEGS_PER_BLOCK + 3][2];  // markers a - 1 .. a + nseg + 1
  __shared__ long long sq[SEGS_PER_BLOCK + 1][2];
  __shared__ double sfn[SEGS_PER_BLOCK + 1];
  __shared__ T spx[SEGS_PER_BLOCK], spy[SEGS_PER_BLOCK];
  __shared__ int sspread[SEGS_PER_BLOCK];
  const int a = blockIdx.x * SEGS_PER_BLOCK;
  const int nseg = min(SEGS_PER_BLOCK, n - a);
  const int t = threadIdx.x;
  const unsigned tag = *tb.tag;  // issued early: the tile flags need it last
  // ---- positions of markers a - 1 .. a + nseg + 1 (n >= 3: one wrap at most)
  if (t < nseg + 3) {
    int j = a - 1 + t;
    if (j < 0) j += n;
    else if (j >= n) j -= n;
    if (INTERP) {
      const double x = in.Xp[2 * j], y = in.Xp[2 * j + 1];
      double ux, uy;
      interp_at<T>(in.uf, geo, x, in.Xqp[2 * j], y, in.Xqp[2 * j + 1], ux, uy);
      const double xn = in.moves ? x + ux : x, yn = in.moves ? y + uy : y;
      sx[t][0] = xn;
      sx[t][1] = yn;
      if (t >= 1 && t <= nseg) {  // owned by this block
        in.U[2 * j] = ux;
        in.U[2 * j + 1] = uy;
        if (in.moves) {
          X[2 * j] = xn;
          X[2 * j + 1] = yn;
        }
      }
    } else {
      sx[t][0] = X[2 * j];
      sx[t][1] = X[2 * j + 1];
    }
  }
  __syncthreads();
  // ---- markers a .. a + nseg (the last is the next block's first, or marker 0)
  if (t <= nseg) {
    const int j = a + t == n ? 0 : a + t;
    const double x = sx[t + 1][0], y = sx[t + 1][1];
    const MarkerForce<T> m = marker_force_at<T>(x, y, sx[t + 2][0], sx[t + 2][1], sx[t][0],
                                                sx[t][1], aux, j, ip, jump, geo);
    const bool inside = in_region(x, y);
    const long long qx = inside ? __double2ll_rn(x * QSCALE) : XQ_OUT;
    const long long qy = inside ? __double2ll_rn(y * QSCALE) : XQ_OUT;
    sq[t][0] = qx;
    sq[t][1] = qy;
    sfn[t] = (double)m.fn;
    if (t < nseg) {  // owned by this block
      if (m.bad) atomicOr(status, ST_INTERFACE);
      G[2 * j] = (double)m.gx;
      G[2 * j + 1] = (double)m.gy;
      Fn[j] = (double)m.fn;
      nrm[2 * j] = (double)m.nx;
      nrm[2 * j + 1] = (double)m.ny;
      Xq[2 * j] = qx;
      Xq[2 * j + 1] = qy;
      // the spread goes into the tiles that segment j -> j+1 flags: it needs both ends
      sspread[t] = inside && in_region(sx[t + 2][0], sx[t + 2][1]);
      spx[t] = m.px;
      spy[t] = m.py;
    }
  }
  __syncthreads();
  const int w = t >> 5, lane = t & 31;
  // ---- cut links and tile flags of segments a + w, a + w + IFACE_WARPS, ...
  for (int k = w; k < nseg; k += IFACE_WARPS)
    segment_links<T>(sq[k][0], sq[k][1], sq[k + 1][0], sq[k + 1][1], sfn[k], sfn[k + 1], lane,
                     jump, geo, Jf, tb, tag);
  // ---- spread of the segments' first markers, 16 lanes (one stencil node each) per
  // marker (Eq. 46 / 17)
  for (int k0 = w; k0 < nseg; k0 += 2 * IFACE_WARPS) {
    const int k = k0 + (lane < 16 ? 0 : IFACE_WARPS), l = lane & 15;
    if (k >= nseg || !sspread[k]) continue;
    int bx, by;
    T wx[4], wy[4];
    stencil_weights<T>(sx[k + 1][0], sq[k][0], bx, wx);
    stencil_weights<T>(sx[k + 1][1], sq[k][1], by, wy);
    int xi = bx + (l & 3), yi = by + (l >> 2);
    bool ok = true;
    if (geo.bc == IILBM_BC_PERIODIC) yi = wrap(yi, geo.ny);
    else ok = yi >= 0 && yi < geo.ny;
    if (geo.bc == IILBM_BC_CHANNEL) ok = ok && xi >= 0 && xi < geo.nx;
    else xi = wrap(xi, geo.nx);
    const T wgt = wx[l & 3] * wy[l >> 2];
    if (ok && wgt != T(0)) {
      const long long here = (long long)yi * geo.pitch + xi;
      atomicAdd(&gf[here], spx[k] * wgt);
      atomicAdd(&gf[geo.plane + here], spy[k] * wgt);
    }
  }
}

template <typename T, bool INTERP>
static int launch_interface(iilbm_lattice *h, int buf, cudaStream_t s) {
  const int n = h->nm;
  const double *aux = h->ip.model == IILBM_DIRECT ? h->Gdf : h->aux;
  const TileBuf tb{h->flagsb[buf], h->tagb[buf], h->tile_list[buf], h->tile_count[buf],
                   h->d_tiles_total};
  const InterpIn<T> in{(const T *)h->uf, h->Xp, h->Xqp, h->U, h->ip.moves};
  const int blocks = (n + SEGS_PER_BLOCK - 1) / SEGS_PER_BLOCK;
  k_interface<T, INTERP><<<blocks, 32 * IFACE_WARPS, 0, s>>>(
      h->X, aux, n, h->ip, h->cfg.jump, h->geom, (T *)h->gb[buf], (T *)h->Jb[buf], tb, h->G,
      h->Fn, h->nrm, h->Xq, h->d_status, in);
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

// ---------------------------------------------------------- interface phase
// Bring buffer buf to the interface of the markers X.  The buffer arrives clean: its
// jump / force entries were zeroed by the forced stream-collide that consumed them, its
// counters reset and its tag advanced by the forced stream-collide of the level before
// (or by the set-up), so stale flags from earlier time levels no longer match.
int launch_interface_phase(iilbm_lattice *h, int buf, cudaStream_t s) {
  if (h->nm == 0) return IILBM_OK;
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

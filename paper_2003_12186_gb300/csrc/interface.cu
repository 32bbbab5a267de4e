// interface.cu -- the Lagrangian side of the II-LBM step on sm_103a (FP64 geometry).
//
// One kernel does the interface work of a time level; each block takes 8 consecutive
// segments and the 9 markers at their ends (the last one is also the next block's:
// computed twice, written by its owner only):
//   * the marker pass, one thread per marker k: the Lagrangian force (Eq. 19 spring, a
//     rest-length spring, or a prescribed / directly forced force), its normal /
//     tangential split (Eqs. 31-32, 46), the marker's coordinates snapped to 2^-24 (kept
//     in shared memory for the segment pass and written out for the interpolation);
//   * the segment pass, one warp per segment k -> k+1: every lattice link x - e_i -> x
//     crossing it (exact 64-bit integer orientation tests on the snapped coordinates,
//     degenerate contacts resolved by displacing lattice nodes by (eps, eps^2)), each
//     adding the jump [[f_i]] = +-w_i/c_s^2 Fn of Eq. 32 to the jump field of its
//     destination node (Eq. 47); and flagging every touched tile, appending newly
//     flagged tiles to the tile list that the forced stream-collide walks; then 16 of
//     its lanes spread the tangential force of the segment's first marker with Peskin's
//     four-point kernel (Eq. 46) into the force field.
// One launch instead of a marker and a segment kernel shortens the chain of small
// kernels that runs beside the lean stream-collide.  (The batched executor keeps the
// two passes as separate launches over its flattened marker list.)
// The dense [.][ny][pitch] fields are only ever touched on O(interface length) tiles.
#include "interface_dev.cuh"

#include <cmath>

namespace iilbm {

constexpr int SEGS_PER_BLOCK = 8;

template <typename T>
__global__ void __launch_bounds__(32 * SEGS_PER_BLOCK)
    k_interface(const double *__restrict__ X, const double *__restrict__ aux, int n,
                iilbm_interface_params ip, int jump, Geom geo, T *gf, T *Jf, TileBuf tb,
                double *G, double *Fn, double *nrm, long long *Xq, int *status) {
  __shared__ long long sq[SEGS_PER_BLOCK + 1][2];
  __shared__ double sfn[SEGS_PER_BLOCK + 1];
  __shared__ T spx[SEGS_PER_BLOCK], spy[SEGS_PER_BLOCK];
  __shared__ int sspread[SEGS_PER_BLOCK];
  const int a = blockIdx.x * SEGS_PER_BLOCK;
  const int nseg = min(SEGS_PER_BLOCK, n - a);
  const int t = threadIdx.x;
  // ---- markers a .. a + nseg (the last is the next block's first, or marker 0)
  if (t <= nseg) {
    const int j = a + t == n ? 0 : a + t;
    const MarkerForce<T> m = marker_force<T>(X, aux, n, j, ip, jump, geo);
    const double x = X[2 * j], y = X[2 * j + 1];
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
      const int jp = j + 1 == n ? 0 : j + 1;
      // the spread goes into the tiles that segment j -> j+1 flags: it needs both ends
      sspread[t] = inside && in_region(X[2 * jp], X[2 * jp + 1]);
      spx[t] = m.px;
      spy[t] = m.py;
    }
  }
  __syncthreads();
  const int w = t >> 5, lane = t & 31;
  if (w >= nseg) return;  // uniform per warp
  // ---- cut links and tile flags of segment a + w
  segment_links<T>(sq[w][0], sq[w][1], sq[w + 1][0], sq[w + 1][1], sfn[w], sfn[w + 1], lane,
                   jump, geo, Jf, tb);
  // ---- spread of marker a + w, one stencil node per lane 0..15 (Eq. 46 / 17)
  if (lane < 16 && sspread[w]) {
    const int j = a + w;
    int bx, by;
    T wx[4], wy[4];
    stencil_weights<T>(X[2 * j], sq[w][0], bx, wx);
    stencil_weights<T>(X[2 * j + 1], sq[w][1], by, wy);
    int xi = bx + (lane & 3), yi = by + (lane >> 2);
    bool ok = true;
    if (geo.bc == IILBM_BC_PERIODIC) yi = wrap(yi, geo.ny);
    else ok = yi >= 0 && yi < geo.ny;
    if (geo.bc == IILBM_BC_CHANNEL) ok = ok && xi >= 0 && xi < geo.nx;
    else xi = wrap(xi, geo.nx);
    const T wgt = wx[lane & 3] * wy[lane >> 2];
    if (ok && wgt != T(0)) {
      const long long here = (long long)yi * geo.pitch + xi;
      atomicAdd(&gf[here], spx[w] * wgt);
      atomicAdd(&gf[geo.plane + here], spy[w] * wgt);
    }
  }
}

// ---------------------------------------------------------- interface phase
// Bring buffer buf to the interface of the markers X.  The buffer arrives clean: its
// jump / force entries were zeroed by the forced stream-collide that consumed them, its
// counters reset and its tag advanced by the interpolation kernel since (or by the
// set-up), so stale flags from earlier time levels no longer match.
int launch_interface_phase(iilbm_lattice *h, int buf, cudaStream_t s) {
  if (h->nm == 0) return IILBM_OK;
  const int n = h->nm;
  const double *aux = h->ip.model == IILBM_DIRECT ? h->Gdf : h->aux;
  const TileBuf tb{h->flagsb[buf], h->tagb[buf], h->tile_list[buf], h->tile_count[buf],
                   h->d_tiles_total};
  const int blocks = (n + SEGS_PER_BLOCK - 1) / SEGS_PER_BLOCK;
  if (h->cfg.storage == IILBM_F64)
    k_interface<double><<<blocks, 32 * SEGS_PER_BLOCK, 0, s>>>(
        h->X, aux, n, h->ip, h->cfg.jump, h->geom, (double *)h->gb[buf], (double *)h->Jb[buf], tb,
        h->G, h->Fn, h->nrm, h->Xq, h->d_status);
  else
    k_interface<float><<<blocks, 32 * SEGS_PER_BLOCK, 0, s>>>(
        h->X, aux, n, h->ip, h->cfg.jump, h->geom, (float *)h->gb[buf], (float *)h->Jb[buf], tb,
        h->G, h->Fn, h->nrm, h->Xq, h->d_status);
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

}  // namespace iilbm

// interface.cu -- the Lagrangian side of the II-LBM step on sm_103a (FP64 geometry).
//
// Two kernels do the interface work of a time level:
//   * the marker pass, one thread per marker k: the Lagrangian force (Eq. 19 spring, a
//     rest-length spring, or a prescribed / directly forced force), its normal /
//     tangential split (Eqs. 31-32, 46), the marker's coordinates snapped to 2^-24, and
//     the spreading of its tangential force with Peskin's four-point kernel (Eq. 46)
//     into the force field;
//   * the segment pass, one warp per segment k -> k+1: every lattice link x - e_i -> x
//     crossing it (exact 64-bit integer orientation tests on the snapped coordinates,
//     degenerate contacts resolved by displacing lattice nodes by (eps, eps^2)), each
//     adding the jump [[f_i]] = +-w_i/c_s^2 Fn of Eq. 32 to the jump field of its
//     destination node (Eq. 47); and flagging every touched tile, appending newly
//     flagged tiles to the tile list that the forced stream-collide walks.
// The dense [.][ny][pitch] fields are only ever touched on O(interface length) tiles.
#include "interface_dev.cuh"

#include <cmath>

namespace iilbm {

template <typename T>
__global__ void __launch_bounds__(128)
    k_markers(const double *__restrict__ X, const double *__restrict__ aux, int n,
              iilbm_interface_params ip, int jump, Geom geo, T *gf, double *G, double *Fn,
              double *nrm, long long *Xq, int *status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) interface_marker<T>(X, aux, n, k, ip, jump, geo, gf, G, Fn, nrm, Xq, status);
}

template <typename T>
__global__ void __launch_bounds__(128)
    k_segments(const long long *__restrict__ Xq, const double *__restrict__ Fn, int n, int jump,
               Geom geo, T *Jf, TileBuf tb) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= n) return;  // uniform per warp
  interface_segment<T>(Xq, Fn, n, k, threadIdx.x & 31, jump, geo, Jf, tb);
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
  const int mblocks = (n + 127) / 128, sblocks = (32 * n + 127) / 128;
  if (h->cfg.storage == IILBM_F64) {
    k_markers<double><<<mblocks, 128, 0, s>>>(h->X, aux, n, h->ip, h->cfg.jump, h->geom,
                                              (double *)h->gb[buf], h->G, h->Fn, h->nrm, h->Xq,
                                              h->d_status);
    k_segments<double><<<sblocks, 128, 0, s>>>(h->Xq, h->Fn, n, h->cfg.jump, h->geom,
                                               (double *)h->Jb[buf], tb);
  } else {
    k_markers<float><<<mblocks, 128, 0, s>>>(h->X, aux, n, h->ip, h->cfg.jump, h->geom,
                                             (float *)h->gb[buf], h->G, h->Fn, h->nrm, h->Xq,
                                             h->d_status);
    k_segments<float><<<sblocks, 128, 0, s>>>(h->Xq, h->Fn, n, h->cfg.jump, h->geom,
                                              (float *)h->Jb[buf], tb);
  }
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

}  // namespace iilbm

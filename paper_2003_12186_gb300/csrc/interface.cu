// interface.cu -- the Lagrangian side of the II-LBM step on sm_103a (FP64 geometry).
//
// One fused kernel, one warp per marker k, does all interface work of a time level:
//   * the Lagrangian force of markers k and k+1 (Eq. 19 spring, a rest-length spring,
//     or a prescribed force) and their normal / tangential split (Eqs. 31-32, 46);
//   * the cut links of segment k -> k+1: every lattice link x - e_i -> x crossing it
//     (exact 64-bit integer orientation tests on marker coordinates snapped to 2^-24,
//     degenerate contacts resolved by displacing lattice nodes by (eps, eps^2)), each
//     adding the jump [[f_i]] = +-w_i/c_s^2 Fn of Eq. 32 to the jump field of its
//     destination node (Eq. 47);
//   * the spreading of marker k's tangential force with Peskin's four-point kernel
//     (Eq. 46) into the force field;
//   * flagging every touched tile and appending newly flagged tiles to the tile list
//     that the forced stream-collide walks.
// The dense [.][ny][pitch] fields are only ever touched on O(interface length) tiles.
#include "interface_dev.cuh"

#include <cmath>

namespace iilbm {

template <typename T>
__global__ void __launch_bounds__(128)
    k_interface(const double *__restrict__ X, const double *__restrict__ aux, int n,
                iilbm_interface_params ip, int jump, Geom geo, T *Jf, T *gf, TileBuf tb,
                double *G, double *Fn, double *nrm, int *status) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= n) return;  // uniform per warp
  interface_warp<T>(X, aux, n, k, threadIdx.x & 31, ip, jump, geo, Jf, gf, tb, G, Fn, nrm, status);
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
  const bool dbl = h->cfg.storage == IILBM_F64;
  const int threads = 32 * n;
  if (dbl)
    k_interface<double><<<(threads + 127) / 128, 128, 0, s>>>(
        h->X, aux, n, h->ip, h->cfg.jump, h->geom, (double *)h->Jb[buf],
        (double *)h->gb[buf], tb, h->G, h->Fn, h->nrm, h->d_status);
  else
    k_interface<float><<<(threads + 127) / 128, 128, 0, s>>>(
        h->X, aux, n, h->ip, h->cfg.jump, h->geom, (float *)h->Jb[buf], (float *)h->gb[buf],
        tb, h->G, h->Fn, h->nrm, h->d_status);
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

}  // namespace iilbm

// api.cu -- the C ABI of include/iilbm.h: handle life cycle, argument checking,
// memory ownership, and the order of the kernels of one II-LBM time step.
#include "forcing_dev.cuh"
#include "iilbm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace iilbm;

namespace {

// On failure, clear the runtime's last-error slot too, so a failed call never
// surfaces again from a later, unrelated launch check.
#define CK(call)                         \
  do {                                   \
    if ((call) != cudaSuccess) {         \
      cudaGetLastError();                \
      return IILBM_ERR_CUDA;             \
    }                                    \
  } while (0)

size_t storage_bytes(int s) {
  switch (s) {
    case IILBM_F64: return 8;
    case IILBM_F32: return 4;
    case IILBM_F16: return 2;
    case IILBM_BF16: return 2;
  }
  return 0;
}

// Copy n bytes from a host or device pointer to device memory on the stream.
int copy_in(void *dst, const void *src, size_t n, cudaStream_t s) {
  CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, s));
  return IILBM_OK;
}

int read_status(iilbm_lattice *h) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (st & ST_NONFINITE) return IILBM_ERR_NONFINITE;
  if (st & ST_INTERFACE) return IILBM_ERR_INTERFACE;
  if (st & ST_CAPACITY) return IILBM_ERR_CAPACITY;
  if (st & ST_TIMEOUT) return IILBM_ERR_DEVICE_TIMEOUT;
  return IILBM_OK;
}

void free_interface(iilbm_lattice *h) {
  double **bufs[] = {&h->X,  &h->aux, &h->G,     &h->Fn,    &h->U,    &h->nrm,
                     &h->G0, &h->Gdf, &h->Ustar, &h->Xp, &h->spl_c, &h->spl_f};
  for (double **b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  if (h->Xq) cudaFree(h->Xq);
  if (h->Xqp) cudaFree(h->Xqp);
  h->Xq = h->Xqp = nullptr;
  free_direct_forcing(h);
  free_body(h);
  h->nm = 0;
}

// Bring the jump / force buffer of the current state's parity to the current
// interface (idempotent per state).  Direct forcing first finds the body force from
// the current state.
int prepare(iilbm_lattice *h) {
  if (h->prepared) return IILBM_OK;
  if (h->in_batch) return prepare_batch_of(h);
  int rc;
  if (h->nm > 0 && h->ip.model == IILBM_DIRECT && (rc = launch_direct_forcing(h))) return rc;
  rc = launch_interface_phase(h, (int)(h->step & 1), h->stream);
  if (rc) return rc;
  h->prepared = true;
  return IILBM_OK;
}

void drop_graph(iilbm_lattice *h) {
  for (int k = 0; k < GRAPH_KINDS; k++) {
    for (int r = 0; r < GRAPH_RING; r++) {
      if (h->gexec[k][r]) cudaGraphExecDestroy(h->gexec[k][r]);
      h->gexec[k][r] = nullptr;
      h->ring_pending[k][r] = false;
    }
    h->ring_next[k] = 0;
  }
}

// Clear every jump / force buffer (used when the interface or the state is replaced
// outside the step sequence).
int clear_fields(iilbm_lattice *h) {
  const Geom &g = h->geom;
  for (int b = 0; b < 2; b++) {
    CK(cudaMemsetAsync(h->Jb[b], 0, 8 * (size_t)g.plane * h->tbytes, h->stream));
    CK(cudaMemsetAsync(h->gb[b], 0, 2 * (size_t)g.plane * h->tbytes, h->stream));
    CK(cudaMemsetAsync(h->flagsb[b], 0, (size_t)h->ntiles * sizeof(unsigned), h->stream));
    CK(cudaMemsetAsync(h->tile_count[b], 0, 2 * sizeof(int), h->stream));
    static const unsigned one = 1u;  // a tag no cleared flag carries
    CK(cudaMemcpyAsync(h->tagb[b], &one, sizeof one, cudaMemcpyHostToDevice, h->stream));
  }
  h->prepared = false;
  return IILBM_OK;
}

// Fold recorded lean stream-collide event pairs into the running sum: the eager pairs,
// or the graph_len(k) pairs of slot r of graph kind k.
int drain_events(iilbm_lattice *h) {
  if (h->nev == 0) return IILBM_OK;
  CK(cudaEventSynchronize(h->ev[EAGER_EV0 + 2 * h->nev - 1]));
  for (int e = 0; e < h->nev; e++) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, h->ev[EAGER_EV0 + 2 * e], h->ev[EAGER_EV0 + 2 * e + 1]));
    h->sc_ms += ms;
  }
  h->nev = 0;
  return IILBM_OK;
}

// First timing event of slot r of graph kind k.
int slot_ev0(int k, int r) { return graph_ev0(k) + 2 * graph_len(k) * r; }

int drain_slot(iilbm_lattice *h, int k, int r) {
  if (!h->ring_pending[k][r]) return IILBM_OK;
  const int e0 = slot_ev0(k, r), len = graph_len(k);
  CK(cudaEventSynchronize(h->ev[e0 + 2 * len - 1]));
  for (int q = 0; q < len; q++) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, h->ev[e0 + 2 * q], h->ev[e0 + 2 * q + 1]));
    h->sc_ms += ms;
  }
  h->ring_pending[k][r] = false;
  return IILBM_OK;
}

int drain_all(iilbm_lattice *h) {
  int rc = drain_events(h);
  for (int k = 0; k < GRAPH_KINDS && !rc; k++)
    for (int r = 0; r < GRAPH_RING && !rc; r++) rc = drain_slot(h, k, r);
  return rc;
}

}  // namespace

namespace iilbm {
// Interface phase of a lattice's current state, for the batched executor.
int prepare_lattice(iilbm_lattice *h) { return prepare(h); }
}  // namespace iilbm

extern "C" {

const char *iilbm_error_string(int status) {
  switch (status) {
    case IILBM_OK: return "ok";
    case IILBM_ERR_INVALID_ARG: return "invalid argument";
    case IILBM_ERR_OOM: return "device allocation failed";
    case IILBM_ERR_CUDA: return "CUDA runtime error";
    case IILBM_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case IILBM_ERR_NONFINITE: return "non-finite population";
    case IILBM_ERR_INTERFACE: return "invalid marker polygon";
    case IILBM_ERR_CAPACITY:
      return "capacity exceeded (cut-link list, forcing shared memory or no-allocation staging array)";
    case IILBM_ERR_NO_DEVICE: return "no compute capability 10.3 CUDA device";
  }
  return "unknown status";
}

int iilbm_create_lattice(iilbm_t *out, const iilbm_config *cfg) {
  if (!out || !cfg) return IILBM_ERR_INVALID_ARG;
  *out = nullptr;
  const iilbm_config &c = *cfg;
  if (c.nx < 4 || c.ny < 4 || c.nx > 32768 || c.ny > 32768) return IILBM_ERR_INVALID_ARG;
  if (c.collision != IILBM_SRT && c.collision != IILBM_MRT) return IILBM_ERR_INVALID_ARG;
  if (!storage_bytes(c.storage)) return IILBM_ERR_INVALID_ARG;
  if (c.bc < IILBM_BC_PERIODIC || c.bc > IILBM_BC_BOX_WALL) return IILBM_ERR_INVALID_ARG;
  if (c.force != IILBM_FORCE_GUO && c.force != IILBM_FORCE_SIMPLE) return IILBM_ERR_INVALID_ARG;
  if (c.bc == IILBM_BC_CHANNEL && !(std::abs(c.u_max) < 0.5)) return IILBM_ERR_INVALID_ARG;
  if (!(c.tau > 0.5) || !(c.rho0 > 0) || std::abs(c.storage_scale_log2) > 30)
    return IILBM_ERR_INVALID_ARG;
  if (c.collision == IILBM_MRT)
    for (int i = 0; i < 9; i++)
      if (!(c.s[i] >= 0.0 && c.s[i] < 2.0)) return IILBM_ERR_INVALID_ARG;
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return IILBM_ERR_NO_DEVICE;
  }
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  if (prop.major != 10 || prop.minor != 3) return IILBM_ERR_NO_DEVICE;

  iilbm_lattice *h = new (std::nothrow) iilbm_lattice();
  if (!h) return IILBM_ERR_OOM;
  h->cfg = c;
  h->device = dev;
  Geom &g = h->geom;
  g.nx = c.nx;
  g.ny = c.ny;
  // a channel keeps two ghost columns in the row padding
  g.pitch = (c.nx + (c.bc == IILBM_BC_CHANNEL ? 2 : 0) + 31) / 32 * 32;
  g.plane = (long long)g.pitch * c.ny;
  g.ntx = (c.nx + TILE_X - 1) / TILE_X;
  const bool box = c.bc == IILBM_BC_BOX_OUTFLOW || c.bc == IILBM_BC_BOX_WALL;
  g.bc = box ? IILBM_BC_PERIODIC : c.bc;  // a box streams periodically; its edge is rewritten
  h->igeom = g;
  if (box) h->igeom.bc = IILBM_BC_CHANNEL;  // for the interface: bounded in x and in y
  h->ntiles = g.ntx * ((c.ny + TILE_Y - 1) / TILE_Y);
  h->sbytes = storage_bytes(c.storage);
  h->tbytes = c.storage == IILBM_F64 ? 8 : 4;
  if (c.stream) {
    h->stream = (cudaStream_t)c.stream;
    h->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return IILBM_ERR_CUDA;
    }
    h->own_stream = true;
  }
  h->vector_sc = true;
  h->tma_sc = 0;
  h->tmap_A = nullptr;
  h->overlap = true;
  h->use_graph = true;
  h->forced_grid = std::max(1, std::min(h->ntiles, 2 * prop.multiProcessorCount));
  // The side stream (forced tiles, next interface phase) runs at the highest priority
  // so its few blocks are dispatched ahead of the lean stream-collide's backlog.
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  bool ok = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess &&
            cudaMalloc(&h->A, 9 * (size_t)g.plane * h->sbytes) == cudaSuccess &&
            cudaMalloc(&h->uf, 2 * (size_t)g.plane * h->tbytes) == cudaSuccess &&
            cudaMalloc(&h->d_status, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_mdf_iters, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->d_mdf_res, sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->d_tiles_total, sizeof(unsigned long long)) == cudaSuccess;
  for (int b = 0; b < 2 && ok; b++)
    ok = cudaMalloc(&h->Jb[b], 8 * (size_t)g.plane * h->tbytes) == cudaSuccess &&
         cudaMalloc(&h->gb[b], 2 * (size_t)g.plane * h->tbytes) == cudaSuccess &&
         cudaMalloc(&h->flagsb[b], (size_t)h->ntiles * sizeof(unsigned)) == cudaSuccess &&
         cudaMalloc(&h->tile_list[b], (size_t)h->ntiles * sizeof(int)) == cudaSuccess &&
         cudaMalloc(&h->tile_count[b], 2 * sizeof(int)) == cudaSuccess &&
         cudaMalloc(&h->tagb[b], sizeof(unsigned)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    iilbm_destroy(h);
    return IILBM_ERR_OOM;
  }
  int rc = IILBM_OK;
  if (cudaMemsetAsync(h->A, 0, 9 * (size_t)g.plane * h->sbytes, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_mdf_iters, 0, sizeof(int), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_mdf_res, 0, sizeof(double), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->d_tiles_total, 0, sizeof(unsigned long long), h->stream) != cudaSuccess)
    rc = IILBM_ERR_CUDA;
  if (!rc) rc = clear_fields(h);
  if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IILBM_ERR_CUDA;
  if (rc) {
    iilbm_destroy(h);
    return rc;
  }
  *out = h;
  return IILBM_OK;
}

int iilbm_destroy(iilbm_t h) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  if (h->in_batch) return IILBM_ERR_INVALID_ARG;  // owned by a batch until it is destroyed
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->side) cudaStreamSynchronize(h->side);
  drop_graph(h);
  free_interface(h);
  void *bufs[] = {h->A, h->uf, h->Jb[0], h->Jb[1], h->gb[0], h->gb[1], h->flagsb[0], h->flagsb[1],
                  h->tile_list[0], h->tile_list[1], h->tile_count[0], h->tile_count[1],
                  h->tagb[0], h->tagb[1],
                  h->d_status, h->d_mdf_iters, h->d_mdf_res, h->d_tiles_total};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev[0])
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return IILBM_OK;
}

int iilbm_set_interface(iilbm_t h, const double *xy, int32_t n, const iilbm_interface_params *p,
                        const double *aux) {
  if (!h || n < 0 || (n > 0 && (!xy || !p))) return IILBM_ERR_INVALID_ARG;
  if (h->in_batch) return IILBM_ERR_INVALID_ARG;  // owned by a batch until it is destroyed
  if (n > 0 && n < 3) return IILBM_ERR_INVALID_ARG;
  if (n > 0) {
    if (p->model < IILBM_SPRING || p->model > IILBM_DIRECT) return IILBM_ERR_INVALID_ARG;
    if (p->model == IILBM_DIRECT && (p->moves || !(p->eta > 0) || p->mdf_iters < 0))
      return IILBM_ERR_INVALID_ARG;  // direct forcing: a fixed body, positive gain
    if (!(p->dX > 0) || !std::isfinite(p->stiffness)) return IILBM_ERR_INVALID_ARG;
    if (p->model == IILBM_SPRING_REST && !(p->rest_length > 0)) return IILBM_ERR_INVALID_ARG;
    if ((p->model == IILBM_PRESCRIBED || p->model == IILBM_DIRECT) && !aux)
      return IILBM_ERR_INVALID_ARG;
    // the spline interface is for flexible boundaries: a directly forced (rigid) body
    // keeps the polygon
    if (p->curve < 0 || p->curve > 16 || (p->curve > 0 && p->model == IILBM_DIRECT))
      return IILBM_ERR_INVALID_ARG;
    // direct forcing is built on Guo's half-force velocity (section 3, reading 13)
    if (p->model == IILBM_DIRECT && h->cfg.force != IILBM_FORCE_GUO) return IILBM_ERR_INVALID_ARG;
  }
  int rc = clear_fields(h);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  // Same marker count and parameters: the marker buffers are reused in place, and the
  // captured step graphs (which hold their addresses and the parameters) stay valid --
  // a new polygon of the same body costs no reallocation and no recapture.
  // (A directly forced body's band and cut links depend on its polygon: rebuilt.)
  const bool keep = n > 0 && n == h->nm && std::memcmp(p, &h->ip, sizeof *p) == 0 &&
                    p->model != IILBM_DIRECT;
  if (!keep) {
    int drc = drain_all(h);
    if (drc) return drc;
    drop_graph(h);
    free_interface(h);
  }
  if (n == 0) return IILBM_OK;
  const size_t b2 = 2 * (size_t)n * sizeof(double);
  if (!keep) {
    bool ok = cudaMalloc(&h->X, b2) == cudaSuccess && cudaMalloc(&h->aux, b2) == cudaSuccess &&
              cudaMalloc(&h->G, b2) == cudaSuccess && cudaMalloc(&h->G0, b2) == cudaSuccess &&
              cudaMalloc(&h->Gdf, b2) == cudaSuccess && cudaMalloc(&h->Ustar, b2) == cudaSuccess &&
              cudaMalloc(&h->Fn, (size_t)n * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&h->Xq, b2) == cudaSuccess && cudaMalloc(&h->U, b2) == cudaSuccess &&
              cudaMalloc(&h->nrm, b2) == cudaSuccess && cudaMalloc(&h->Xp, b2) == cudaSuccess &&
              cudaMalloc(&h->Xqp, b2) == cudaSuccess && cudaMalloc(&h->spl_c, b2) == cudaSuccess &&
              cudaMalloc(&h->spl_f, b2 / 2) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_interface(h);
      return IILBM_ERR_OOM;
    }
  }
  h->nm = n;
  h->ip = *p;
  if ((rc = copy_in(h->X, xy, b2, h->stream))) return rc;
  if (aux) {
    if ((rc = copy_in(h->aux, aux, b2, h->stream))) return rc;
  } else {
    CK(cudaMemsetAsync(h->aux, 0, b2, h->stream));
  }
  CK(cudaMemsetAsync(h->U, 0, b2, h->stream));
  CK(cudaMemsetAsync(h->G, 0, b2, h->stream));
  CK(cudaMemsetAsync(h->G0, 0, b2, h->stream));
  CK(cudaMemsetAsync(h->Gdf, 0, b2, h->stream));
  CK(cudaMemsetAsync(h->Ustar, 0, b2, h->stream));
  CK(cudaMemsetAsync(h->Fn, 0, (size_t)n * sizeof(double), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  // host-side validation of the polygon (the kernels re-check every step)
  double *hx = (double *)std::malloc(b2);
  if (!hx) return IILBM_ERR_OOM;
  CK(cudaMemcpy(hx, h->X, b2, cudaMemcpyDeviceToHost));
  bool bad = false;
  for (int k = 0; k < n && !bad; k++) {
    const int kp = (k + 1) % n;
    const double x = hx[2 * k], y = hx[2 * k + 1];
    const double dx = hx[2 * kp] - x, dy = hx[2 * kp + 1] - y;
    bad = !std::isfinite(x) || !std::isfinite(y) || std::abs(x) > MAX_COORD ||
          std::abs(y) > MAX_COORD || !(dx * dx + dy * dy < MAX_SEGMENT * MAX_SEGMENT) ||
          (dx == 0 && dy == 0);
    if (h->igeom.bc != IILBM_BC_PERIODIC) bad = bad || y < 3.0 || y > h->cfg.ny - 4.0;
    if (h->igeom.bc == IILBM_BC_CHANNEL) bad = bad || x < 3.0 || x > h->cfg.nx - 4.0;
  }
  if (bad) {
    std::free(hx);
    drop_graph(h);
    free_interface(h);
    return IILBM_ERR_INTERFACE;
  }
  if (p->model == IILBM_DIRECT) {
    // the band of nodes the force iteration touches and the body's cut links
    rc = setup_direct_forcing(h, hx);
    if (rc) {
      std::free(hx);
      free_interface(h);
      return rc;
    }
  }
  std::free(hx);
  return IILBM_OK;
}

int iilbm_init_equilibrium(iilbm_t h, const double *rho, const double *ux, const double *uy) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  if (h->in_batch) return IILBM_ERR_INVALID_ARG;  // owned by a batch until it is destroyed
  const size_t N = (size_t)h->cfg.nx * h->cfg.ny;
  const double *src[3] = {rho, ux, uy};
  double *dev[3] = {nullptr, nullptr, nullptr};
  int rc = IILBM_OK;
  for (int a = 0; a < 3 && !rc; a++)
    if (src[a]) {
      if (cudaMalloc(&dev[a], N * sizeof(double)) != cudaSuccess) rc = IILBM_ERR_OOM;
      else rc = copy_in(dev[a], src[a], N * sizeof(double), h->stream);
    }
  if (!rc) rc = clear_fields(h);
  if (!rc) rc = launch_set_populations(h, nullptr, true, dev[0], dev[1], dev[2]);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = IILBM_ERR_CUDA;
  for (double *d : dev)
    if (d) cudaFree(d);
  return rc;
}

int iilbm_set_populations(iilbm_t h, const double *df) {
  if (!h || !df) return IILBM_ERR_INVALID_ARG;
  if (h->in_batch) return IILBM_ERR_INVALID_ARG;  // owned by a batch until it is destroyed
  const size_t bytes = 9 * (size_t)h->cfg.nx * h->cfg.ny * sizeof(double);
  double *d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) return IILBM_ERR_OOM;
  int rc = copy_in(d, df, bytes, h->stream);
  if (!rc) rc = clear_fields(h);
  if (!rc) rc = launch_set_populations(h, d, false, nullptr, nullptr, nullptr);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = IILBM_ERR_CUDA;
  cudaFree(d);
  return rc;
}

int iilbm_get_populations(iilbm_t h, double *df) {
  if (!h || !df) return IILBM_ERR_INVALID_ARG;
  const size_t bytes = 9 * (size_t)h->cfg.nx * h->cfg.ny * sizeof(double);
  double *d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) return IILBM_ERR_OOM;
  int rc = launch_get_populations(h, d);
  if (!rc && cudaMemcpyAsync(df, d, bytes, cudaMemcpyDefault, h->stream) != cudaSuccess)
    rc = IILBM_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = IILBM_ERR_CUDA;
  cudaFree(d);
  return rc ? rc : read_status(h);
}

}  // extern "C"

namespace {

// Kernels launched by one step: lean stream-collide (two launches with the TMA kernel:
// interior and edge tiles); with an interface also the
// forced stream-collide and the interpolation fused with the next interface phase
// (pipelined), or the interpolation, the interface kernel and, for direct forcing, the
// force iteration; a channel adds its boundary kernel.
long long kernels_per_step(const iilbm_lattice *h, bool odd) {
  long long k = (uses_tma_sc(h, odd) ? 2 : 1) + (h->cfg.bc == IILBM_BC_CHANNEL || h->cfg.bc == IILBM_BC_BOX_OUTFLOW ||
                             h->cfg.bc == IILBM_BC_BOX_WALL
                         ? 1
                         : 0);
  if (h->nm > 0)
    k += pipelined(h) ? 2
                      : 3 + (h->ip.model == IILBM_DIRECT ? 1 : 0) + (h->ip.curve > 0 ? 3 : 0) +
                            (h->body ? 1 : 0);
  return k;
}

// Kernels launched by the len steps from time level step0.
long long kernels_over(const iilbm_lattice *h, long long step0, int len) {
  long long k = 0;
  for (int q = 0; q < len; q++) k += kernels_per_step(h, ((step0 + q) & 1) != 0);
  return k;
}


// One time step of the current state n (its interface already prepared in buffer
// n & 1).  Main stream: the lean stream-collide (every tile without a jump or force).
// Second stream (highest priority), forked at the start of the step: the forced
// stream-collide of the flagged tiles, which also leaves the collision velocity there,
// then the interpolation from it with the marker move (X^{n+1}) fused with the
// interface phase of state n + 1 in buffer (n+1) & 1 -- or, for a directly forced body
// (whose interface phase waits for the next state's force iteration), the interpolation
// alone; it joins before the step ends.  Without overlap the forced stream-collide and
// the interpolation run on the main stream and the interface phase in the next
// prepare.  Safe inside stream capture.
// ev_slot: index of the start event of the lean stream-collide timing pair, or -1.
int one_step(iilbm_lattice *h, int ev_slot) {
  int rc;
  const bool pipe = pipelined(h);
  // the forced stream-collide and the interpolation go to the side stream whenever
  // overlap is on; the next level's interface phase only when it does not have to wait
  // for the next state (direct forcing needs it, so it runs in the next prepare)
  const bool fork = h->overlap && h->nm > 0;
  cudaStream_t s2 = fork ? h->side : h->stream;
  if (fork) {
    CK(cudaEventRecord(h->ev_fork, h->stream));
    CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  }
  // Timing events: inside a stream capture they must become event-record nodes of the
  // graph (cudaEventRecordExternal); outside a capture they are plain records.
  const unsigned evflag = h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (ev_slot >= 0) CK(cudaEventRecordWithFlags(h->ev[ev_slot], h->stream, evflag));
  if ((rc = launch_stream_collide(h, s2))) return rc;
  if (ev_slot >= 0) CK(cudaEventRecordWithFlags(h->ev[ev_slot + 1], h->stream, evflag));
  rc = pipe ? launch_interp_interface(h, h->side)  // interface phase of state n + 1
            : launch_interp(h, s2);
  if (rc) return rc;
  if (fork) {
    CK(cudaEventRecord(h->ev_join, h->side));
    CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  }
  h->step++;
  if ((rc = launch_channel_bc(h))) return rc;  // inflow / outflow of the new state
  if ((rc = launch_body_update(h))) return rc;  // a rigid body moves to the new level
  h->prepared = pipe || h->nm == 0;
  return IILBM_OK;
}

// Graph replay needs the state a captured step starts from: prepared for a pipelined
// lattice (and one without an interface), unprepared for a directly forced body, whose
// captured steps each begin with the force iteration and the interface phase.
bool graph_entry(const iilbm_lattice *h) {
  if (h->nm == 0) return true;
  return pipelined(h) ? h->prepared : !h->prepared;
}

// One step as captured: the interface phase first where the state needs it, then the
// step itself.  ev_slot as for one_step.
int graph_step(iilbm_lattice *h, int ev_slot) {
  int rc = prepare(h);
  return rc ? rc : one_step(h, ev_slot);
}

// Capture the graph_len(k) steps of kind k (from an even state, or one step from an odd
// one for the last kind) into slot r.  Capture records the launches without running
// them; the host-side state (level, preparation) is restored afterwards, so any slot of
// any kind may be captured from any state that is a graph entry.
int capture_graph(iilbm_lattice *h, int k, int r) {
  const long long step0 = h->step;
  const bool prepared0 = h->prepared;
  const bool odd = k == GRAPH_ODD;
  h->step = odd ? (step0 | 1) : (step0 & ~1LL);
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = IILBM_OK;
  h->capturing = true;
  for (int q = 0; q < graph_len(k) && !rc; q++)
    rc = graph_step(h, h->timing ? slot_ev0(k, r) + 2 * q : -1);
  h->capturing = false;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  cudaGetLastError();
  h->step = step0;
  h->prepared = prepared0;
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return IILBM_ERR_CUDA;
  // honour the side stream's priority inside the graph
  e = cudaGraphInstantiateWithFlags(&h->gexec[k][r], graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->gexec[k][r] = nullptr;
    cudaGetLastError();
    return IILBM_ERR_CUDA;
  }
  return IILBM_OK;
}

// Capture every kind's graph (slot 0, or all GRAPH_RING slots with timing on) at the
// first replay, so that no later call of any length pays for a capture.
int capture_all(iilbm_lattice *h) {
  const int slots = h->timing ? GRAPH_RING : 1;
  int rc = IILBM_OK;
  for (int k = 0; k < GRAPH_KINDS && !rc; k++)
    for (int r = 0; r < slots && !rc; r++)
      if (!h->gexec[k][r]) rc = capture_graph(h, k, r);
  return rc;
}

}  // namespace

extern "C" {

// Advance n steps.  With graphs on, each iteration launches one graph: the one-step
// graph from an odd state, else the longest kind that fits in what is left, so n steps
// take at most one odd step and the binary decomposition of the rest.  A state that is
// not a graph entry (a direct-forcing state prepared by a read-out, or graphs off) takes
// an eager step.
int iilbm_step(iilbm_t h, int32_t n) {
  if (!h || n < 0 || h->in_batch) return IILBM_ERR_INVALID_ARG;
  int rc;
  while (n > 0) {
    if (h->use_graph && h->nm > 0 && pipelined(h) && !h->prepared && (rc = prepare(h)))
      return rc;
    if (h->use_graph && graph_entry(h)) {
      if (h->graph_timing != h->timing) {
        if ((rc = drain_all(h))) return rc;
        CK(cudaStreamSynchronize(h->stream));  // no graph of the other setting in flight
        drop_graph(h);
        h->graph_timing = h->timing;
      }
      if ((rc = capture_all(h))) return rc;
      int k = GRAPH_ODD;
      if ((h->step & 1) == 0) {
        k = 0;
        while (graph_len(k) > n) k++;
      }
      // with timing the ring lets each launch record into events that the launch
      // GRAPH_RING earlier of the same kind has long finished with
      const int r = h->timing ? h->ring_next[k] : 0;
      if (h->timing && (rc = drain_slot(h, k, r))) return rc;
      CK(cudaGraphLaunch(h->gexec[k][r], h->stream));
      const int len = graph_len(k);
      h->step += len;
      h->prepared = pipelined(h) || h->nm == 0;
      n -= len;
      if (h->timing) {
        h->ring_pending[k][r] = true;
        h->ring_next[k] = (r + 1) % GRAPH_RING;
        h->sc_launches += len;
        h->kernel_launches += kernels_over(h, h->step - len, len);
      }
      continue;
    }
    if ((rc = prepare(h))) return rc;
    int slot = -1;
    if (h->timing) {
      if (h->nev == EAGER_PAIRS && (rc = drain_events(h))) return rc;
      slot = EAGER_EV0 + 2 * h->nev;
    }
    const long long step0 = h->step;
    if ((rc = one_step(h, slot))) return rc;
    if (h->timing) {
      h->nev++;
      h->sc_launches++;
      h->kernel_launches += kernels_over(h, step0, 1);
    }
    n--;
  }
  return IILBM_OK;
}

int iilbm_set_option(iilbm_t h, int32_t option, int32_t value) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  if (h->in_batch) return IILBM_ERR_INVALID_ARG;  // owned by a batch until it is destroyed
  CK(cudaStreamSynchronize(h->stream));
  switch (option) {
    case IILBM_OPT_CUDA_GRAPH: h->use_graph = value != 0; break;
    case IILBM_OPT_OVERLAP: h->overlap = value != 0; break;
    case IILBM_OPT_VECTOR_KERNEL: h->vector_sc = value != 0; break;
    case IILBM_OPT_TMA_KERNEL:
      if (value < 0 || value > 2) return IILBM_ERR_INVALID_ARG;
      h->tma_sc = value;
      break;
    case IILBM_OPT_FORCED_BLOCKS: {
      if (value < 0) return IILBM_ERR_INVALID_ARG;
      cudaDeviceProp prop;
      CK(cudaGetDeviceProperties(&prop, h->device));
      h->forced_grid = std::max(1, std::min(h->ntiles, value > 0 ? (int)value
                                                                  : 2 * prop.multiProcessorCount));
      break;
    }
    default: return IILBM_ERR_INVALID_ARG;
  }
  drop_graph(h);
  return IILBM_OK;
}

int iilbm_set_timing(iilbm_t h, int32_t enable) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  CK(cudaMemsetAsync(h->d_tiles_total, 0, sizeof(unsigned long long), h->stream));
  const int nev = (int)(sizeof(h->ev) / sizeof(h->ev[0]));
  if (enable && !h->ev[0])
    for (int e = 0; e < nev; e++) CK(cudaEventCreate(&h->ev[e]));
  if (!enable) {
    int rc = drain_all(h);
    if (rc) return rc;
  }
  h->timing = enable != 0;
  return IILBM_OK;
}

int iilbm_get_timing(iilbm_t h, double *sc_ms, int32_t *launches, int64_t *kernel_launches,
                     int64_t *flagged_tiles) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  int rc = drain_all(h);
  if (rc) return rc;
  unsigned long long tiles = 0;
  CK(cudaStreamSynchronize(h->side));
  CK(cudaMemcpyAsync(&tiles, h->d_tiles_total, sizeof tiles, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemsetAsync(h->d_tiles_total, 0, sizeof tiles, h->stream));
  if ((rc = read_status(h))) return rc;
  if (sc_ms) *sc_ms = h->sc_ms;
  if (launches) *launches = h->sc_launches;
  if (kernel_launches) *kernel_launches = h->kernel_launches;
  if (flagged_tiles) *flagged_tiles = (int64_t)tiles;
  h->sc_ms = 0;
  h->sc_launches = 0;
  h->kernel_launches = 0;
  return IILBM_OK;
}

int iilbm_get_macros(iilbm_t h, double *drho, double *ux, double *uy) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  int rc = prepare(h);
  if (rc) return rc;
  const size_t bytes = (size_t)h->cfg.nx * h->cfg.ny * sizeof(double);
  double *d = nullptr;
  if (cudaMalloc(&d, 3 * bytes) != cudaSuccess) return IILBM_ERR_OOM;
  rc = launch_macros(h, d, d + bytes / 8, d + 2 * bytes / 8);
  double *outs[3] = {drho, ux, uy};
  for (int a = 0; a < 3 && !rc; a++)
    if (outs[a] && cudaMemcpyAsync(outs[a], d + a * (bytes / 8), bytes, cudaMemcpyDefault,
                                   h->stream) != cudaSuccess)
      rc = IILBM_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = IILBM_ERR_CUDA;
  cudaFree(d);
  return rc ? rc : read_status(h);
}

int iilbm_get_jump(iilbm_t h, double *J) {
  if (!h || !J) return IILBM_ERR_INVALID_ARG;
  int rc = prepare(h);
  if (rc) return rc;
  const size_t bytes = 8 * (size_t)h->cfg.nx * h->cfg.ny * sizeof(double);
  double *d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_OOM;
  }
  rc = launch_get_jump(h, d);
  if (!rc && cudaMemcpyAsync(J, d, bytes, cudaMemcpyDefault, h->stream) != cudaSuccess)
    rc = IILBM_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = IILBM_ERR_CUDA;
  cudaGetLastError();
  cudaFree(d);
  return rc ? rc : read_status(h);
}

int iilbm_get_markers(iilbm_t h, double *X, double *G, double *U, double *Fn) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  if (h->nm == 0) return read_status(h);
  const size_t b2 = 2 * (size_t)h->nm * sizeof(double);
  if (X) CK(cudaMemcpyAsync(X, h->X, b2, cudaMemcpyDefault, h->stream));
  if (G) CK(cudaMemcpyAsync(G, h->G, b2, cudaMemcpyDefault, h->stream));
  if (U) CK(cudaMemcpyAsync(U, h->U, b2, cudaMemcpyDefault, h->stream));
  if (Fn) CK(cudaMemcpyAsync(Fn, h->Fn, b2 / 2, cudaMemcpyDefault, h->stream));
  return read_status(h);
}

int iilbm_get_mdf_stats(iilbm_t h, int32_t *iters, double *residual) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  int it = 0;
  double res = 0;
  CK(cudaMemcpyAsync(&it, h->d_mdf_iters, sizeof it, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&res, h->d_mdf_res, sizeof res, cudaMemcpyDeviceToHost, h->stream));
  int rc = read_status(h);
  if (iters) *iters = it;
  if (residual) *residual = res;
  return rc;
}

int iilbm_set_warm_start(iilbm_t h, const double *G0) {
  if (!h || h->nm == 0) return IILBM_ERR_INVALID_ARG;
  const size_t b2 = 2 * (size_t)h->nm * sizeof(double);
  if (G0) CK(cudaMemcpyAsync(h->G0, G0, b2, cudaMemcpyDefault, h->stream));
  else CK(cudaMemsetAsync(h->G0, 0, b2, h->stream));
  // used by the next force iteration: that of the current state unless a read-out has
  // already run it (re-running the interface phase would add the jump a second time)
  CK(cudaStreamSynchronize(h->stream));
  return IILBM_OK;
}

int iilbm_set_warm_start_mode(iilbm_t h, int32_t mode) {
  if (!h || mode < IILBM_WS_GIVEN || mode > IILBM_WS_PREVIOUS) return IILBM_ERR_INVALID_ARG;
  if (h->in_batch) return IILBM_ERR_INVALID_ARG;  // owned by a batch until it is destroyed
  int rc = drain_all(h);  // captured force iterations bake the start mode in
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));  // no graph of the old setting in flight
  drop_graph(h);
  h->ws_mode = mode;
  h->mlp = nullptr;
  return IILBM_OK;
}

int iilbm_set_warm_start_mlp(iilbm_t h, iilbm_mlp_t mlp, double re) {
  if (!h || !mlp || !std::isfinite(re)) return IILBM_ERR_INVALID_ARG;
  if (h->in_batch) return IILBM_ERR_INVALID_ARG;
  if (h->nm == 0 || h->ip.model != IILBM_DIRECT || mlp_device(mlp) != h->device)
    return IILBM_ERR_INVALID_ARG;
  const int prev = h->ws_mode;
  h->ws_mode = WS_MLP;
  if (direct_forcing_smem(h, h->df_nb, h->nm) > 227 * 1024) {
    h->ws_mode = prev;
    return IILBM_ERR_CAPACITY;
  }
  int rc = drain_all(h);  // captured force iterations bake the network and Re in
  if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IILBM_ERR_CUDA;
  if (rc) {
    h->ws_mode = prev;
    return rc;
  }
  drop_graph(h);
  h->mlp = mlp;
  h->re = (float)re;
  return IILBM_OK;
}

int iilbm_get_df_features(iilbm_t h, double re, float *F) {
  if (!h || !F || !std::isfinite(re)) return IILBM_ERR_INVALID_ARG;
  if (h->nm == 0 || h->ip.model != IILBM_DIRECT) return IILBM_ERR_INVALID_ARG;
  const size_t bytes = (size_t)h->nm * 30 * sizeof(float);
  float *d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_OOM;
  }
  int rc = launch_df_features(h, (float)re, d);
  if (!rc && cudaMemcpyAsync(F, d, bytes, cudaMemcpyDefault, h->stream) != cudaSuccess)
    rc = IILBM_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = IILBM_ERR_CUDA;
  cudaGetLastError();
  cudaFree(d);
  return rc ? rc : read_status(h);
}

int iilbm_get_unforced_velocity(iilbm_t h, double *Ustar) {
  if (!h || !Ustar) return IILBM_ERR_INVALID_ARG;
  if (h->nm == 0 || h->ip.model != IILBM_DIRECT) return IILBM_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(Ustar, h->Ustar, 2 * (size_t)h->nm * sizeof(double), cudaMemcpyDefault,
                     h->stream));
  return read_status(h);
}

int iilbm_get_body_force(iilbm_t h, double *F) {
  if (!h || !F) return IILBM_ERR_INVALID_ARG;
  F[0] = F[1] = 0.0;
  if (h->nm == 0) return read_status(h);
  const size_t b2 = 2 * (size_t)h->nm * sizeof(double);
  double *hg = (double *)std::malloc(b2);
  if (!hg) return IILBM_ERR_OOM;
  int rc = IILBM_OK;
  if (cudaMemcpyAsync(hg, h->G, b2, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) {
    cudaGetLastError();
    rc = IILBM_ERR_CUDA;
  }
  if (!rc) rc = read_status(h);
  if (!rc)
    for (int k = 0; k < h->nm; k++) {
      F[0] -= hg[2 * k] * h->ip.dX;
      F[1] -= hg[2 * k + 1] * h->ip.dX;
    }
  std::free(hg);
  return rc;
}

int iilbm_get_cut_link_count(iilbm_t h, int32_t *count) {
  if (!h || !count) return IILBM_ERR_INVALID_ARG;
  *count = 0;
  if (h->nm == 0) return read_status(h);
  int rc = prepare(h);
  if (rc) return rc;
  CK(cudaMemcpyAsync(count, h->tile_count[h->step & 1] + 1, sizeof(int), cudaMemcpyDeviceToHost,
                     h->stream));
  return read_status(h);
}

int iilbm_synchronize(iilbm_t h) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(h->side));
  return read_status(h);
}

}  // extern "C"

// ------------------------------------------------------------- rigid body
// Make the directly forced interface a rigid body (include/iilbm.h).
extern "C" int iilbm_set_rigid_body(iilbm_t h, const iilbm_body_params *bp) {
  if (!h || !bp || h->in_batch || h->nm == 0 || h->ip.model != IILBM_DIRECT)
    return IILBM_ERR_INVALID_ARG;
  if (bp->mode != IILBM_BODY_PRESCRIBED_X && bp->mode != IILBM_BODY_FREE)
    return IILBM_ERR_INVALID_ARG;
  if (bp->mode == IILBM_BODY_PRESCRIBED_X && !(bp->amplitude > 0 && std::isfinite(bp->u_max)))
    return IILBM_ERR_INVALID_ARG;
  if (bp->mode == IILBM_BODY_FREE &&
      (!(bp->mass > 0) || !(bp->inertia > 0) || !(bp->volume >= 0) || bp->dof < 0 || bp->dof > 7))
    return IILBM_ERR_INVALID_ARG;
  int rc = drain_all(h);  // the force iteration's launches change: recapture
  if (rc) return rc;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return IILBM_ERR_CUDA;
  drop_graph(h);
  const int n = h->nm;
  std::vector<double> X(2 * (size_t)n), X0(2 * (size_t)n), UD(2 * (size_t)n);
  if (cudaMemcpy(X.data(), h->X, X.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return IILBM_ERR_CUDA;
  double cxm = 0, cym = 0, r = 0;
  for (int q = 0; q < n; q++) {
    cxm += X[2 * q];
    cym += X[2 * q + 1];
  }
  cxm /= n;
  cym /= n;
  for (int q = 0; q < n; q++) {
    X0[2 * q] = X[2 * q] - cxm;
    X0[2 * q + 1] = X[2 * q + 1] - cym;
    r = std::max(r, std::hypot(X0[2 * q], X0[2 * q + 1]));
  }
  iilbm_body_dev b{};
  b.mode = bp->mode;
  b.dof = bp->dof;
  b.A = bp->amplitude;
  b.umax = bp->u_max;
  b.m = bp->mode == IILBM_BODY_FREE ? bp->mass : 1.0;
  b.I = bp->mode == IILBM_BODY_FREE ? bp->inertia : 1.0;
  b.Vs = bp->volume;
  b.rho_f = h->cfg.rho0;
  for (int d = 0; d < 3; d++) {
    b.k[d] = bp->spring[d];
    b.c[d] = bp->damping[d];
  }
  b.t = h->step;  // the prescribed motion is a function of the lattice's time level
  b.Xc0[0] = b.Xc[0] = cxm;
  b.Xc0[1] = b.Xc[1] = cym;
  if (bp->mode == IILBM_BODY_PRESCRIBED_X) b.Uc[0] = b.Ucp[0] = -bp->u_max;
  for (int q = 0; q < n; q++) {  // the desired velocity of the state at t = 0
    UD[2 * q] = b.Uc[0] - b.W * (X[2 * q + 1] - cym);
    UD[2 * q + 1] = b.Uc[1] + b.W * (X[2 * q] - cxm);
  }
  // capacities: the band and the cut links of the body wherever it moves (the set-up
  // band's sizes with a margin), the bitmap of a window around its circumcircle
  free_body(h);
  const int side = (int)std::ceil(2 * r) + 10;
  h->body_words = (side * side + 31) / 32 + 1;
  h->body_nb = h->df_nb + h->df_nb / 3 + 64;
  h->body_nl = h->df_nl + h->df_nl / 3 + 64;
  if (cudaMalloc(&h->body, sizeof(iilbm_body_dev)) != cudaSuccess ||
      cudaMalloc(&h->body_X0, X0.size() * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    free_body(h);
    return IILBM_ERR_OOM;
  }
  if (direct_forcing_smem(h, h->body_nb, n) > 227 * 1024) {  // with the body's capacities
    free_body(h);
    return IILBM_ERR_CAPACITY;
  }
  if (cudaMemcpy(h->body, &b, sizeof b, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->body_X0, X0.data(), X0.size() * sizeof(double), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(h->aux, UD.data(), UD.size() * sizeof(double), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    free_body(h);
    return IILBM_ERR_CUDA;
  }
  return IILBM_OK;
}

extern "C" int iilbm_get_rigid_body(iilbm_t h, double *state) {
  if (!h || !state || !h->body) return IILBM_ERR_INVALID_ARG;
  iilbm_body_dev b;
  if (cudaMemcpyAsync(&b, h->body, sizeof b, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_CUDA;
  }
  const double v[9] = {b.Xc[0], b.Xc[1], b.th, b.Uc[0], b.Uc[1], b.W, b.F[0], b.F[1], b.F[2]};
  for (int q = 0; q < 9; q++) state[q] = v[q];
  return IILBM_OK;
}


// ------------------------------------------------------ no-allocation read-out
// iilbm_get_macros_noalloc: the macroscopic read-out of iilbm_get_macros without any
// device allocation.  The fields are staged in a file-scope device array instead of a
// cudaMalloc'd buffer.  Every device that loads this library holds the array (6 MiB)
// until the process exits.  All calls share it, so calls whose GPU work overlaps in
// time (two streams, two threads) race on it; it needs no clearing because the kernel
// writes every element a call reads back.

namespace {

constexpr long long NOALLOC_MAX_CELLS = IILBM_NOALLOC_MAX_CELLS;
static __device__ __align__(256) double g_noalloc_stage[3 * NOALLOC_MAX_CELLS];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the staging array on `device`, looked up once per device with that
// device current (the host-side symbol is only a stand-in, never a device address).
int noalloc_stage(int device, double **out) {
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) return IILBM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    int prev = -1;
    CK(cudaGetDevice(&prev));
    if (prev != device) CK(cudaSetDevice(device));
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_stage);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return IILBM_ERR_CUDA;
    }
    g_noalloc_ptr[device] = (double *)p;
  }
  *out = g_noalloc_ptr[device];
  return IILBM_OK;
}

}  // namespace

extern "C" int iilbm_get_macros_noalloc(iilbm_t h, double *drho, double *ux, double *uy) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  const long long cells = (long long)h->cfg.nx * h->cfg.ny;
  if (cells > NOALLOC_MAX_CELLS) return IILBM_ERR_CAPACITY;
  double *stage = nullptr;
  int rc = noalloc_stage(h->device, &stage);
  if (rc) return rc;
  if ((rc = prepare(h))) return rc;
  rc = launch_macros(h, stage, stage + cells, stage + 2 * cells);
  double *outs[3] = {drho, ux, uy};
  for (int a = 0; a < 3 && !rc; a++)
    if (outs[a] && cudaMemcpyAsync(outs[a], stage + a * cells, (size_t)cells * sizeof(double),
                                   cudaMemcpyDefault, h->stream) != cudaSuccess) {
      cudaGetLastError();
      rc = IILBM_ERR_CUDA;
    }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess && !rc) rc = IILBM_ERR_CUDA;
  return rc ? rc : read_status(h);
}

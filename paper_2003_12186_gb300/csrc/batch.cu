// batch.cu -- many independent lattices advanced together on sm_103a.
//
// A batch is built from existing lattice handles of one storage type, collision model
// and boundary kind (sizes, rates, interfaces and force models may all differ).  Every
// phase of a time step is ONE launch for the whole batch instead of one per lattice:
//   * lean stream-collide over a flattened list of (lattice, tile) work items, either
//     one block per item or a persistent grid striding over the list;
//   * forced stream-collide over each lattice's flagged-tile list (grid.y = lattice);
//   * interpolation and the two interface passes over a flattened marker list;
//   * direct forcing, one CTA per fixed body; the channel ends, one row per thread.
// The kernels resolve their lattice from a device table of descriptors and run the
// same device code as the single-lattice path.  An autotuner times the stream-collide
// variants (vectorised or one node per thread; per-item or persistent grid) on the
// batch itself and keeps the fastest.  Steps are replayed from CUDA graphs.
#include "forcing_dev.cuh"
#include "interface_dev.cuh"
#include "lattice_dev.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

using namespace iilbm;

namespace iilbm {

// One lattice of the batch as the batched kernels see it.
struct SimDev {
  Geom geo;
  int ntiles;
  void *A;
  void *J[2], *g[2];
  unsigned *flags[2];
  unsigned *tag[2];
  int *list[2], *ctr[2];
  void *uf;
  double *X, *aux, *G, *Fn, *nrm, *U;
  long long *Xq;
  int nm, jump;
  iilbm_interface_params ip;
  CollP<float> p;
  int *status;
  unsigned long long *tiles_total;
  DfArgs df;
  double u_max;
};

// Stream-collide variants the autotuner chooses from: nodes per thread (4, 2 or 1),
// resident blocks per SM the registers are budgeted for (3: at most 80 registers, with
// some spilling at 2 and 4 nodes per thread; 2: no spilling), and grid shape (one block
// per work item, or a persistent grid of resident blocks x SMs striding over the items).
// The odd step needs more registers than the even one (neighbour shifts, edge stores):
// the last two variants budget 3 blocks per SM for the even step and 2 (no spilling)
// for the odd one.
struct BatchVariant {
  int npt, minb;
  bool persistent;
  int minb_odd;  // 0: as minb
};
constexpr BatchVariant BATCH_VARIANTS[] = {
    {4, 3, false, 0}, {4, 3, true, 0}, {4, 2, false, 0}, {4, 2, true, 0}, {2, 3, false, 0},
    {2, 3, true, 0},  {2, 2, false, 0}, {2, 2, true, 0}, {1, 3, false, 0}, {1, 3, true, 0},
    {4, 3, false, 2}, {4, 3, true, 2}};
constexpr int BV_COUNT = sizeof(BATCH_VARIANTS) / sizeof(BATCH_VARIANTS[0]);

// ----------------------------------------------------------------- kernels
// A work item is up to LEAN_GROUP consecutive tiles of one lattice: the lattice's
// descriptor, tag and the group's flags are loaded once, before its first tile.
// NPT = nodes per thread: 4 or 2 (vectorised, 32 NPT nodes per warp row), or 1 (one
// node per thread, 32-node sub-blocks); MINB resident blocks per SM.
constexpr int LEAN_GROUP = 4;

template <typename S, int COLL, bool ODD, int BC, int NPT, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_batch_lean(const SimDev *__restrict__ sims, const int2 *__restrict__ items, int nitems) {
  constexpr int b = ODD ? 1 : 0;  // buffer of the state = its parity
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];  // (lattice, first tile)
    const SimDev &sd = sims[w.x];
    const unsigned *fl = sd.flags[b];
    const unsigned tag = *sd.tag[b];
    const int nt = min(LEAN_GROUP, sd.ntiles - w.y);
    unsigned todo = 0u;  // bit q: tile w.y + q is a lean tile
#pragma unroll
    for (int q = 0; q < LEAN_GROUP; q++)
      if (q < nt && fl[w.y + q] != tag) todo |= 1u << q;
#pragma unroll 1
    for (int q = 0; q < nt; q++) {
      if (!(todo >> q & 1u)) continue;  // uniform per block: a forced tile
      const int tile = w.y + q;
      const int tx = (tile % sd.geo.ntx) * TILE_X, ty = (tile / sd.geo.ntx) * TILE_Y;
      if (NPT > 1) {
        for (int sub = 0; sub < TILE_X; sub += 32 * NPT)
          sc_vec_rows<S, COLL, ODD, BC, false, NPT>((S *)sd.A, nullptr, nullptr, nullptr,
                                                     sd.geo, sd.p, sd.status, tx + sub, ty);
      } else {
        for (int sub = 0; sub < TILE_X; sub += 32)
          sc_scalar_rows<S, COLL, ODD, BC, false>((S *)sd.A, nullptr, nullptr, nullptr, sd.geo,
                                                   sd.p, sd.status, tx + sub, ty);
      }
    }
  }
}

// Two resident blocks per SM (<= 128 registers): the forced tiles are few and short,
// so memory parallelism, not per-thread registers, sets their pace.
template <typename S, int COLL, bool ODD, int BC>
__global__ void __launch_bounds__(256, 2)
    k_batch_forced(const SimDev *__restrict__ sims) {
  constexpr int b = ODD ? 1 : 0;
  const SimDev &sd = sims[blockIdx.y];
  if (sd.nm == 0) return;
  const int n = sd.ctr[b][0];
  constexpr int W = 32 * Vec<S>::V;
  // every batched lattice has nx % 4 == 0, so the vectorised block serves all of them
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int tile = sd.list[b][t];
    const int tx = (tile % sd.geo.ntx) * TILE_X, ty = (tile / sd.geo.ntx) * TILE_Y;
    for (int sub = 0; sub < TILE_X; sub += W)
      sc_vec_rows<S, COLL, ODD, BC, true>((S *)sd.A, (float *)sd.J[b], (float *)sd.g[b],
                                           (float *)sd.uf, sd.geo, sd.p, sd.status, tx + sub, ty);
  }
}

// One thread per marker of the flattened list; thread s < nsims also prepares lattice
// s's buffer of the next time level (tag advanced, counters reset).
__global__ void __launch_bounds__(128)
    k_batch_interp(const SimDev *__restrict__ sims, int nsims, const int *__restrict__ msim,
                   const int *__restrict__ mk, int nmarkers, int next_buf) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < nsims && sims[tid].nm > 0) {
    const SimDev &sd = sims[tid];
    *sd.tag[next_buf] += 1u;
    sd.ctr[next_buf][0] = 0;
    sd.ctr[next_buf][1] = 0;
  }
  if (tid >= nmarkers) return;
  const SimDev &sd = sims[msim[tid]];
  interp_marker<float>((const float *)sd.uf, sd.geo, sd.X, sd.Xq, mk[tid], sd.U, sd.ip.moves);
}

// Marker pass of buffer buf, one thread per marker of the flattened list.
__global__ void __launch_bounds__(128)
    k_batch_markers(const SimDev *__restrict__ sims, const int *__restrict__ msim,
                    const int *__restrict__ mk, int nmarkers, int buf) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmarkers) return;
  const SimDev &sd = sims[msim[m]];
  const double *aux = sd.ip.model == IILBM_DIRECT ? sd.df.G : sd.aux;
  interface_marker<float>(sd.X, aux, sd.nm, mk[m], sd.ip, sd.jump, sd.geo, (float *)sd.g[buf],
                          sd.G, sd.Fn, sd.nrm, sd.Xq, sd.status);
}

// Segment pass of buffer buf, one warp per segment of the flattened list.
__global__ void __launch_bounds__(128)
    k_batch_segments(const SimDev *__restrict__ sims, const int *__restrict__ msim,
                     const int *__restrict__ mk, int nmarkers, int buf) {
  const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (m >= nmarkers) return;  // uniform per warp
  const SimDev &sd = sims[msim[m]];
  const TileBuf tb{sd.flags[buf], sd.tag[buf], sd.list[buf], sd.ctr[buf], sd.tiles_total};
  interface_segment<float>(sd.Xq, sd.Fn, sd.nm, mk[m], threadIdx.x & 31, sd.jump, sd.geo,
                           (float *)sd.J[buf], tb);
}

// One CTA per lattice with a fixed body under direct forcing.
template <typename S>
__global__ void __launch_bounds__(DF_THREADS)
    k_batch_direct_forcing(const SimDev *__restrict__ sims, bool odd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SimDev &sd = sims[blockIdx.x];
  if (sd.nm == 0 || sd.ip.model != IILBM_DIRECT) return;
  direct_forcing_cta<S>((const S *)sd.A, sd.geo, odd, sd.df, (double)sd.p.inv_scale, smem_raw);
}

template <typename S>
__global__ void k_batch_channel_bc(const SimDev *__restrict__ sims, bool odd) {
  const SimDev &sd = sims[blockIdx.y];
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (sd.geo.bc == IILBM_BC_CHANNEL && y < sd.geo.ny)
    channel_bc_row<S>((S *)sd.A, sd.geo, sd.p, odd, sd.u_max, y);
}

}  // namespace iilbm

// ------------------------------------------------------------------- handle
struct iilbm_batch {
  std::vector<iilbm_lattice *> sims;
  int storage, collision, bc;
  cudaStream_t stream, side;
  bool own_stream;
  cudaEvent_t ev_fork, ev_join;
  SimDev *d_sims;
  int2 *d_items;
  int nitems;
  int *d_msim, *d_mk;
  int nmarkers;
  int nsims;
  int max_ny;
  int forced_gx;
  int sm_count;
  size_t df_smem;
  bool any_direct, any_iface;
  long long step;
  bool prepared;
  int variant;
  cudaGraphExec_t gexec;
  // timing of the lean stream-collide (eager steps only)
  bool timing;
  std::vector<cudaEvent_t> ev;
  int nev;
  double sc_ms;
  int sc_launches;
  long long kernel_launches;
};

namespace {

#define CKB(call)                         \
  do {                                    \
    if ((call) != cudaSuccess) {          \
      cudaGetLastError();                 \
      return IILBM_ERR_CUDA;              \
    }                                     \
  } while (0)

constexpr int BATCH_GRAPH_STEPS = 32;

template <typename F>
int with_storage(int storage, F &&f) {
  switch (storage) {
    case IILBM_F32: return f((float *)nullptr);
    case IILBM_F16: return f((__half *)nullptr);
    case IILBM_BF16: return f((__nv_bfloat16 *)nullptr);
  }
  return IILBM_ERR_INVALID_ARG;
}

template <typename S, int COLL, bool ODD, int BC, int NPT, int MINB>
void lean_launch_v(iilbm_batch *B, bool persistent) {
  const int grid = persistent ? std::min(B->nitems, MINB * B->sm_count) : B->nitems;
  const dim3 block = NPT > 1 ? dim3(256) : dim3(32, TILE_Y);
  k_batch_lean<S, COLL, ODD, BC, NPT, MINB><<<grid, block, 0, B->stream>>>(B->d_sims, B->d_items,
                                                                            B->nitems);
}

template <typename S, int COLL, bool ODD, int BC>
void lean_launch(iilbm_batch *B) {
  const BatchVariant v = BATCH_VARIANTS[B->variant];
  const int minb = ODD && v.minb_odd ? v.minb_odd : v.minb;
  if (v.npt == 4 && minb == 3) lean_launch_v<S, COLL, ODD, BC, 4, 3>(B, v.persistent);
  else if (v.npt == 4) lean_launch_v<S, COLL, ODD, BC, 4, 2>(B, v.persistent);
  else if (v.npt == 2 && minb == 3) lean_launch_v<S, COLL, ODD, BC, 2, 3>(B, v.persistent);
  else if (v.npt == 2) lean_launch_v<S, COLL, ODD, BC, 2, 2>(B, v.persistent);
  else lean_launch_v<S, COLL, ODD, BC, 1, 3>(B, v.persistent);
}

template <typename S, int COLL, bool ODD, int BC>
void sc_batch(iilbm_batch *B, cudaStream_t s2) {
  lean_launch<S, COLL, ODD, BC>(B);
  if (B->any_iface)
    k_batch_forced<S, COLL, ODD, BC><<<dim3(B->forced_gx, B->nsims), 256, 0, s2>>>(B->d_sims);
}

template <typename S>
void sc_batch_dispatch(iilbm_batch *B, cudaStream_t s2) {
  const bool odd = B->step & 1;
  const bool mrt = B->collision == IILBM_MRT;
#define SCB(C, O, BCV) sc_batch<S, C, O, BCV>(B, s2)
  if (B->bc == IILBM_BC_PERIODIC) {
    if (mrt) { if (odd) SCB(IILBM_MRT, true, IILBM_BC_PERIODIC); else SCB(IILBM_MRT, false, IILBM_BC_PERIODIC); }
    else { if (odd) SCB(IILBM_SRT, true, IILBM_BC_PERIODIC); else SCB(IILBM_SRT, false, IILBM_BC_PERIODIC); }
  } else if (B->bc == IILBM_BC_WALLS_Y) {
    if (mrt) { if (odd) SCB(IILBM_MRT, true, IILBM_BC_WALLS_Y); else SCB(IILBM_MRT, false, IILBM_BC_WALLS_Y); }
    else { if (odd) SCB(IILBM_SRT, true, IILBM_BC_WALLS_Y); else SCB(IILBM_SRT, false, IILBM_BC_WALLS_Y); }
  } else {
    if (mrt) { if (odd) SCB(IILBM_MRT, true, IILBM_BC_CHANNEL); else SCB(IILBM_MRT, false, IILBM_BC_CHANNEL); }
    else { if (odd) SCB(IILBM_SRT, true, IILBM_BC_CHANNEL); else SCB(IILBM_SRT, false, IILBM_BC_CHANNEL); }
  }
#undef SCB
}

int launch_batch_sc(iilbm_batch *B, cudaStream_t s2) {
  return with_storage(B->storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    sc_batch_dispatch<S>(B, s2);
    return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
  });
}

int launch_batch_interface(iilbm_batch *B, int buf, cudaStream_t s) {
  if (!B->any_iface) return IILBM_OK;
  const int n = B->nmarkers;
  k_batch_markers<<<(n + 127) / 128, 128, 0, s>>>(B->d_sims, B->d_msim, B->d_mk, n, buf);
  k_batch_segments<<<(32 * n + 127) / 128, 128, 0, s>>>(B->d_sims, B->d_msim, B->d_mk, n, buf);
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

int launch_batch_interp(iilbm_batch *B, cudaStream_t s) {
  if (!B->any_iface) return IILBM_OK;
  const int threads = std::max(B->nmarkers, B->nsims);
  k_batch_interp<<<(threads + 127) / 128, 128, 0, s>>>(B->d_sims, B->nsims, B->d_msim, B->d_mk,
                                                       B->nmarkers, (int)((B->step + 1) & 1));
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

int set_batch_df_smem(iilbm_batch *B) {
  return with_storage(B->storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    return cudaFuncSetAttribute(k_batch_direct_forcing<S>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)B->df_smem) == cudaSuccess
               ? IILBM_OK
               : IILBM_ERR_CUDA;
  });
}

int launch_batch_df(iilbm_batch *B) {
  if (!B->any_direct) return IILBM_OK;
  const bool odd = B->step & 1;
  return with_storage(B->storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_batch_direct_forcing<S><<<B->nsims, DF_THREADS, B->df_smem, B->stream>>>(B->d_sims, odd);
    return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
  });
}

int launch_batch_channel(iilbm_batch *B) {
  if (B->bc != IILBM_BC_CHANNEL) return IILBM_OK;
  const bool odd = B->step & 1;
  return with_storage(B->storage, [&](auto *tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_batch_channel_bc<S><<<dim3((B->max_ny + 127) / 128, B->nsims), 128, 0, B->stream>>>(
        B->d_sims, odd);
    return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
  });
}

bool batch_pipelined(const iilbm_batch *B) { return B->any_iface && !B->any_direct; }

int batch_prepare(iilbm_batch *B) {
  if (B->prepared) return IILBM_OK;
  int rc = launch_batch_df(B);
  if (!rc) rc = launch_batch_interface(B, (int)(B->step & 1), B->stream);
  if (!rc) B->prepared = true;
  return rc;
}

void sync_lattices(iilbm_batch *B) {
  for (iilbm_lattice *h : B->sims) {
    h->step = B->step;
    h->prepared = B->prepared;
  }
}

// Lean stream-collide; with interfaces the forced one, the interpolation, the marker
// and the segment pass (and the force iteration under direct forcing); a channel adds
// its boundary kernel.
long long batch_kernels_per_step(const iilbm_batch *B) {
  return 1 + (B->any_iface ? 4 + (B->any_direct ? 1 : 0) : 0) + (B->bc == IILBM_BC_CHANNEL ? 1 : 0);
}

// One time step of every lattice (same structure as the single-lattice step).
int batch_one_step(iilbm_batch *B, int ev_pair) {
  int rc;
  const bool pipe = batch_pipelined(B);
  const bool fork = B->any_iface;  // forced + interpolation beside the lean kernel
  cudaStream_t s2 = fork ? B->side : B->stream;
  if (fork) {
    CKB(cudaEventRecord(B->ev_fork, B->stream));
    CKB(cudaStreamWaitEvent(B->side, B->ev_fork, 0));
  }
  if (ev_pair >= 0) CKB(cudaEventRecord(B->ev[ev_pair], B->stream));
  if ((rc = launch_batch_sc(B, s2))) return rc;
  if (ev_pair >= 0) CKB(cudaEventRecord(B->ev[ev_pair + 1], B->stream));
  if ((rc = launch_batch_interp(B, s2))) return rc;
  if (pipe && (rc = launch_batch_interface(B, (int)((B->step + 1) & 1), B->side))) return rc;
  if (fork) {
    CKB(cudaEventRecord(B->ev_join, B->side));
    CKB(cudaStreamWaitEvent(B->stream, B->ev_join, 0));
  }
  B->step++;
  B->prepared = pipe || !B->any_iface;
  return launch_batch_channel(B);
}

int batch_drain(iilbm_batch *B) {
  if (B->nev == 0) return IILBM_OK;
  CKB(cudaEventSynchronize(B->ev[2 * B->nev - 1]));
  for (int e = 0; e < B->nev; e++) {
    float ms = 0;
    CKB(cudaEventElapsedTime(&ms, B->ev[2 * e], B->ev[2 * e + 1]));
    B->sc_ms += ms;
  }
  B->nev = 0;
  return IILBM_OK;
}

void drop_batch_graph(iilbm_batch *B) {
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  B->gexec = nullptr;
}

int capture_batch_graph(iilbm_batch *B) {
  drop_batch_graph(B);
  const long long step0 = B->step;
  cudaGraph_t graph = nullptr;
  CKB(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
  int rc = IILBM_OK;
  for (int k = 0; k < BATCH_GRAPH_STEPS && !rc; k++) {
    if (!B->prepared) rc = batch_prepare(B);
    if (!rc) rc = batch_one_step(B, -1);
  }
  cudaError_t e = cudaStreamEndCapture(B->stream, &graph);
  cudaGetLastError();
  B->step = step0;
  B->prepared = batch_pipelined(B) || !B->any_iface;
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return IILBM_ERR_CUDA;
  e = cudaGraphInstantiateWithFlags(&B->gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    B->gexec = nullptr;
    cudaGetLastError();
    return IILBM_ERR_CUDA;
  }
  return IILBM_OK;
}

int batch_steps(iilbm_batch *B, int n) {
  int rc;
  while (n > 0) {
    // A graph replays whole steps from an even state: a pipelined batch starts and ends
    // every step prepared; a direct-forcing batch starts every step unprepared (each
    // captured step begins with the force iteration and the interface phase).
    const bool entry = !B->any_iface || (B->any_direct ? !B->prepared : B->prepared);
    if (!B->timing && (B->step & 1) == 0 && n >= BATCH_GRAPH_STEPS && entry) {
      if (!B->gexec && (rc = capture_batch_graph(B))) return rc;
      CKB(cudaGraphLaunch(B->gexec, B->stream));
      B->step += BATCH_GRAPH_STEPS;
      B->prepared = batch_pipelined(B) || !B->any_iface;
      n -= BATCH_GRAPH_STEPS;
      continue;
    }
    if ((rc = batch_prepare(B))) return rc;
    int pair = -1;
    if (B->timing) {
      if (2 * (B->nev + 1) > (int)B->ev.size() && (rc = batch_drain(B))) return rc;
      pair = 2 * B->nev;
    }
    if ((rc = batch_one_step(B, pair))) return rc;
    if (B->timing) {
      B->nev++;
      B->sc_launches++;
      B->kernel_launches += batch_kernels_per_step(B);
    }
    n--;
  }
  return IILBM_OK;
}

}  // namespace

namespace iilbm {
// A read on one lattice of a batch that needs the interface of the current state
// prepares the whole batch (so the batch's own bookkeeping stays consistent).
int prepare_batch_of(iilbm_lattice *h) {
  iilbm_batch *B = h->batch;
  const int rc = batch_prepare(B);
  sync_lattices(B);
  return rc;
}
}  // namespace iilbm

extern "C" {

int iilbm_create_batch(iilbm_batch_t *out, const iilbm_t *lattices, int32_t count, void *stream) {
  if (!out || !lattices || count <= 0) return IILBM_ERR_INVALID_ARG;
  *out = nullptr;
  iilbm_lattice *h0 = lattices[0];
  if (!h0) return IILBM_ERR_INVALID_ARG;
  for (int s = 0; s < count; s++) {
    iilbm_lattice *h = lattices[s];
    if (!h || h->in_batch || h->cfg.storage == IILBM_F64 || h->cfg.storage != h0->cfg.storage ||
        h->geom.nx % 4 != 0 || (h->nm > 0 && h->ip.curve > 0) || h->cfg.bc != h->geom.bc ||
        h->cfg.collision != h0->cfg.collision || h->cfg.bc != h0->cfg.bc ||
        h->device != h0->device || ((h->step ^ h0->step) & 1))
      return IILBM_ERR_INVALID_ARG;
    for (int q = 0; q < s; q++)
      if (lattices[q] == h) return IILBM_ERR_INVALID_ARG;
  }
  iilbm_batch *B = new (std::nothrow) iilbm_batch();
  if (!B) return IILBM_ERR_OOM;
  B->sims.assign(lattices, lattices + count);
  B->storage = h0->cfg.storage;
  B->collision = h0->cfg.collision;
  B->bc = h0->cfg.bc;
  B->nsims = count;
  B->variant = 0;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, h0->device) != cudaSuccess) {
    delete B;
    return IILBM_ERR_CUDA;
  }
  B->sm_count = prop.multiProcessorCount;
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  bool ok = cudaStreamCreateWithPriority(&B->side, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) == cudaSuccess;
  if (stream) {
    B->stream = (cudaStream_t)stream;
  } else {
    ok = ok && cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) == cudaSuccess;
    B->own_stream = true;
  }
  if (!ok) {
    cudaGetLastError();
    iilbm_destroy_batch(B);
    return IILBM_ERR_CUDA;
  }
  // bring every lattice to a prepared state on its own streams, then hand the batch's
  // streams to the lattices so that their own calls stay ordered after batch work
  int rc = IILBM_OK;
  for (iilbm_lattice *h : B->sims) {
    if (!rc) rc = prepare_lattice(h);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaStreamSynchronize(h->side) != cudaSuccess)
      rc = IILBM_ERR_CUDA;
  }
  if (rc) {
    cudaGetLastError();
    iilbm_destroy_batch(B);
    return rc;
  }
  std::vector<SimDev> sd(count);
  std::vector<int2> items;
  std::vector<int> msim, mk;
  B->max_ny = 0;
  int max_list = 1;
  for (int s = 0; s < count; s++) {
    iilbm_lattice *h = B->sims[s];
    SimDev &d = sd[s];
    d.geo = h->geom;
    d.A = h->A;
    for (int b = 0; b < 2; b++) {
      d.J[b] = h->Jb[b];
      d.g[b] = h->gb[b];
      d.flags[b] = h->flagsb[b];
      d.tag[b] = h->tagb[b];
      d.list[b] = h->tile_list[b];
      d.ctr[b] = h->tile_count[b];
    }
    d.uf = h->uf;
    d.X = h->X; d.aux = h->aux; d.G = h->G; d.Fn = h->Fn; d.nrm = h->nrm; d.U = h->U;
    d.Xq = h->Xq;
    d.nm = h->nm;
    d.jump = h->cfg.jump;
    d.ip = h->ip;
    const iilbm_config &c = h->cfg;
    d.p = make_collp<float>(c);
    d.status = h->d_status;
    d.tiles_total = h->d_tiles_total;
    d.u_max = c.u_max;
    std::memset(&d.df, 0, sizeof d.df);
    if (h->nm > 0 && h->ip.model == IILBM_DIRECT) {
      d.df = df_args(h);
      const DfArgs &a = d.df;
      B->any_direct = true;
      B->df_smem = std::max(B->df_smem, direct_forcing_smem(h, a.nb, a.n));
    }
    if (h->nm > 0) B->any_iface = true;
    B->max_ny = std::max(B->max_ny, h->geom.ny);
    max_list = std::max(max_list, h->ntiles);
    d.ntiles = h->ntiles;
    for (int t = 0; t < h->ntiles; t += LEAN_GROUP) items.push_back(make_int2(s, t));
    for (int k = 0; k < h->nm; k++) {
      msim.push_back(s);
      mk.push_back(k);
    }
  }
  if (B->any_direct && set_batch_df_smem(B)) {
    iilbm_destroy_batch(B);
    return IILBM_ERR_CUDA;
  }
  B->nitems = (int)items.size();
  B->nmarkers = (int)msim.size();
  B->forced_gx = std::min(max_list, 8);
  B->step = h0->step;
  B->prepared = true;
  ok = cudaMalloc(&B->d_sims, sizeof(SimDev) * count) == cudaSuccess &&
       cudaMalloc(&B->d_items, sizeof(int2) * std::max(1, B->nitems)) == cudaSuccess &&
       cudaMalloc(&B->d_msim, sizeof(int) * std::max(1, B->nmarkers)) == cudaSuccess &&
       cudaMalloc(&B->d_mk, sizeof(int) * std::max(1, B->nmarkers)) == cudaSuccess;
  ok = ok && cudaMemcpy(B->d_sims, sd.data(), sizeof(SimDev) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(B->d_items, items.data(), sizeof(int2) * B->nitems, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok && B->nmarkers)
    ok = cudaMemcpy(B->d_msim, msim.data(), sizeof(int) * B->nmarkers, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(B->d_mk, mk.data(), sizeof(int) * B->nmarkers, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    iilbm_destroy_batch(B);
    return IILBM_ERR_OOM;
  }
  for (iilbm_lattice *h : B->sims) {
    h->own_main = h->stream;
    h->own_side = h->side;
    h->stream = B->stream;
    h->side = B->side;
    h->in_batch = true;
    h->batch = B;
  }
  *out = B;
  return IILBM_OK;
}

int iilbm_destroy_batch(iilbm_batch_t B) {
  if (!B) return IILBM_ERR_INVALID_ARG;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->side) cudaStreamSynchronize(B->side);
  for (iilbm_lattice *h : B->sims)
    if (h && h->in_batch) {
      h->stream = h->own_main;
      h->side = h->own_side;
      h->in_batch = false;
      h->batch = nullptr;
      h->step = B->step;
      h->prepared = B->prepared;
    }
  drop_batch_graph(B);
  void *bufs[] = {B->d_sims, B->d_items, B->d_msim, B->d_mk};
  for (void *p : bufs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : B->ev) cudaEventDestroy(e);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->ev_join) cudaEventDestroy(B->ev_join);
  if (B->side) cudaStreamDestroy(B->side);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
  return IILBM_OK;
}

int iilbm_batch_step(iilbm_batch_t B, int32_t n) {
  if (!B || n < 0) return IILBM_ERR_INVALID_ARG;
  const int rc = batch_steps(B, n);
  sync_lattices(B);
  return rc;
}

int iilbm_batch_set_variant(iilbm_batch_t B, int32_t variant) {
  if (!B || variant < 0 || variant >= BV_COUNT) return IILBM_ERR_INVALID_ARG;
  CKB(cudaStreamSynchronize(B->stream));
  B->variant = variant;
  drop_batch_graph(B);
  return IILBM_OK;
}

int iilbm_batch_autotune(iilbm_batch_t B, int32_t steps, int32_t *chosen, double *us_per_step) {
  if (!B || steps <= 0) return IILBM_ERR_INVALID_ARG;
  const int reps = std::max(BATCH_GRAPH_STEPS, (steps + BATCH_GRAPH_STEPS - 1) / BATCH_GRAPH_STEPS *
                                                   BATCH_GRAPH_STEPS);
  cudaEvent_t a, b;
  CKB(cudaEventCreate(&a));
  CKB(cudaEventCreate(&b));
  int best = B->variant, rc = IILBM_OK;
  float best_ms = 1e30f;
  const bool timing = B->timing;
  B->timing = false;
  for (int v = 0; v < BV_COUNT && !rc; v++) {
    if ((rc = iilbm_batch_set_variant(B, v))) break;
    if ((B->step & 1) && (rc = batch_steps(B, 1))) break;   // align to an even state
    if ((rc = batch_steps(B, BATCH_GRAPH_STEPS))) break;     // capture + warm up
    float ms = 0;
    if (cudaEventRecord(a, B->stream) != cudaSuccess) rc = IILBM_ERR_CUDA;
    if (!rc) rc = batch_steps(B, reps);
    if (!rc && (cudaEventRecord(b, B->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
      rc = IILBM_ERR_CUDA;
    if (!rc && ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  B->timing = timing;
  if (!rc) rc = iilbm_batch_set_variant(B, best);
  sync_lattices(B);
  if (chosen) *chosen = best;
  if (us_per_step) *us_per_step = best_ms * 1e3 / reps;
  return rc;
}

int iilbm_batch_set_timing(iilbm_batch_t B, int32_t enable) {
  if (!B) return IILBM_ERR_INVALID_ARG;
  if (enable && B->ev.empty()) {
    B->ev.resize(512);
    for (cudaEvent_t &e : B->ev) CKB(cudaEventCreate(&e));
  }
  if (!enable) {
    int rc = batch_drain(B);
    if (rc) return rc;
  }
  B->timing = enable != 0;
  return IILBM_OK;
}

int iilbm_batch_get_timing(iilbm_batch_t B, double *sc_ms, int32_t *launches,
                           int64_t *kernel_launches) {
  if (!B) return IILBM_ERR_INVALID_ARG;
  int rc = batch_drain(B);
  if (rc) return rc;
  if (sc_ms) *sc_ms = B->sc_ms;
  if (launches) *launches = B->sc_launches;
  if (kernel_launches) *kernel_launches = B->kernel_launches;
  B->sc_ms = 0;
  B->sc_launches = 0;
  B->kernel_launches = 0;
  return IILBM_OK;
}

int iilbm_batch_synchronize(iilbm_batch_t B) {
  if (!B) return IILBM_ERR_INVALID_ARG;
  CKB(cudaStreamSynchronize(B->stream));
  CKB(cudaStreamSynchronize(B->side));
  for (iilbm_lattice *h : B->sims) {
    int st = 0;
    CKB(cudaMemcpy(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost));
    if (st) return st & ST_NONFINITE ? IILBM_ERR_NONFINITE : IILBM_ERR_INTERFACE;
  }
  return IILBM_OK;
}

}  // extern "C"

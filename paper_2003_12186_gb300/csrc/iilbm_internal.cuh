// iilbm_internal.cuh -- device-side building blocks shared by the CUDA translation
// units of the II-LBM library (lattice constants, storage conversions, handle).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>

#include "../../include/iilbm.h"

namespace iilbm {

// ---------------------------------------------------------------- D2Q9 lattice
// Velocity set of section 2.2.1 in the order 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE,
// 6 NW, 7 SW, 8 SE; weights of Eq. 9.
__host__ __device__ constexpr int cx(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 5 + 2) & 3) + 5);
}
template <typename T>
__host__ __device__ constexpr T wt(int i) {
  return i == 0 ? T(4) / T(9) : (i <= 4 ? T(1) / T(9) : T(1) / T(36));
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp axis");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp diag");

// Force / jump tiles of TILE_X x TILE_Y nodes: a per-tile byte flags tiles that carry
// a jump or a spread force; a tile is one block of the vectorised stream-collide.
constexpr int TILE_X = 128;
constexpr int TILE_Y = 8;

// Device status bits (latched, read back by synchronising calls).
constexpr int ST_NONFINITE = 1;
constexpr int ST_INTERFACE = 2;
constexpr int ST_CAPACITY = 4;
constexpr int ST_TIMEOUT = 8;

// Marker coordinates are snapped to multiples of 2^-24 lattice units for the exact
// integer crossing predicate of the cut links.
constexpr double QSCALE = 16777216.0;
constexpr double MAX_SEGMENT = 16.0;
constexpr double MAX_COORD = 16000.0;
// CUDA graphs of a lattice: kind k < GRAPH_KINDS - 1 replays graph_len(k) = 32 >> k
// steps from an even state, the last kind one step from an odd state; iilbm_step(n)
// launches the binary decomposition of n (after one odd step, if the state is odd).
constexpr int GRAPH_KINDS = 7;
constexpr int GRAPH_ODD = GRAPH_KINDS - 1;
constexpr int GRAPH_MAX = 32;
__host__ __device__ constexpr int graph_len(int k) { return k < GRAPH_ODD ? GRAPH_MAX >> k : 1; }
constexpr int GRAPH_RING = 4;
// first timing event of kind k's ring (a pair per step of each of its GRAPH_RING graphs)
__host__ __device__ constexpr int graph_ev0(int k) {
  return k == 0 ? 0 : graph_ev0(k - 1) + 2 * GRAPH_RING * graph_len(k - 1);
}
constexpr int EAGER_EV0 = graph_ev0(GRAPH_KINDS);  // first eager timing event
constexpr int EAGER_PAIRS = 128;

// Sentinel of a snapped marker coordinate outside the region the integer geometry covers.
constexpr long long XQ_OUT = (long long)(-0x7fffffffffffffffLL - 1);

// ------------------------------------------------------ Peskin delta (Eq. 17)
// Peskin's four-point kernel phi(r) in the arithmetic type T.
template <typename T>
__device__ inline T phi4(T r) {
  const T a = fabs(r);
  if (a < T(1)) return T(0.125) * (T(3) - T(2) * a + sqrt(T(1) + T(4) * a - T(4) * a * a));
  if (a < T(2)) return T(0.125) * (T(5) - T(2) * a - sqrt(T(-7) + T(12) * a - T(4) * a * a));
  return T(0);
}

// ------------------------------------------------------------ storage types
// Populations are stored as df * 2^k in S and computed in T (double for FP64
// storage, float otherwise).
template <typename S> struct Store;
template <> struct Store<double> {
  using T = double;
  __device__ static double ld(double v) { return v; }
  __device__ static double st(double v) { return v; }
};
template <> struct Store<float> {
  using T = float;
  __device__ static float ld(float v) { return v; }
  __device__ static float st(float v) { return v; }
};
template <> struct Store<__half> {
  using T = float;
  __device__ static float ld(__half v) { return __half2float(v); }
  __device__ static __half st(float v) { return __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
  using T = float;
  __device__ static float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};

// Geometry of one lattice as the kernels see it.
struct Geom {
  int nx, ny;
  int pitch;        // row stride in elements (nx rounded up to 32)
  long long plane;  // pitch * ny
  int ntx;          // tiles per row
  int bc;           // IILBM_BC_*
};

// A Geom whose boundary kind is a compile-time constant: device code templated on the
// geometry type then reads geo.bc as a constant and drops the other kinds' branches
// (smaller code for kernels that run once per step with a cold instruction cache).
template <int BC>
struct GeomC : Geom {
  static constexpr int bc = BC;
  GeomC() = default;
  __host__ __device__ explicit GeomC(const Geom &g) : Geom(g) {}
};

__host__ __device__ inline int wrap(int v, int n) {
  if ((unsigned)v < (unsigned)n) return v;  // the common case: no division
  v = v % n;
  return v < 0 ? v + n : v;
}

// Storage column of lattice column x in [-1, nx]: periodic x wraps; a channel keeps
// the populations that stream in through x = -1 / x = nx in two ghost columns taken
// from the row padding (pitch >= nx + 2): x = nx is column nx, x = -1 column pitch - 1.
__host__ __device__ inline int xcol(const Geom &g, int x) {
  if (g.bc != IILBM_BC_CHANNEL) return wrap(x, g.nx);
  return x < 0 ? g.pitch - 1 : x;
}

// Location (plane index, cell index) of the population f_i(x, y) of the current
// state in the AA layout.  Even state: slot i at the node itself.  Odd state: slot
// opp(i) at the upstream node (x - e_i), wrapped on periodic axes; a population
// that arrives through a y wall (halfway bounce-back) sits in slot i of the node.
__device__ inline long long aa_loc(const Geom &g, bool odd, int i, int x, int y) {
  if (!odd) return (long long)i * g.plane + (long long)y * g.pitch + x;
  int sx = x - cx(i), sy = y - cy(i);
  if (g.bc == IILBM_BC_PERIODIC) {
    sy = wrap(sy, g.ny);
  } else if (sy < 0 || sy >= g.ny) {
    return (long long)i * g.plane + (long long)y * g.pitch + x;
  }
  sx = xcol(g, sx);
  return (long long)opp(i) * g.plane + (long long)sy * g.pitch + sx;
}

}  // namespace iilbm

// The rigid body of section 2.3 carrying a directly forced interface: its state on the
// device (one CTA updates it after every step, so graph replay carries it along).
struct iilbm_body_dev {
  int mode, dof;
  double A, umax, m, I, Vs, rho_f;
  double k[3], c[3];
  double Xc0[2], Xc[2], Uc[2], Ucp[2], ac[2];
  double th, W, Wp, wdot;
  double F[3];      // the last F_ext (x, y) and T_ext
  long long t;      // time level of the state
};

// ------------------------------------------------------------------ handle
struct iilbm_lattice {
  iilbm_config cfg;
  iilbm::Geom geom;   // the populations' geometry (a box streams periodically)
  iilbm::Geom igeom;  // the interface's: as geom, but a box is bounded on every side (its
                      // bc reads as a channel's: clipped in x and in y)
  int device;
  cudaStream_t stream;
  bool own_stream;
  size_t sbytes;      // bytes per stored population
  size_t tbytes;      // bytes per arithmetic value (jump, force)
  void *A;            // [9][plane] populations, storage type
  // Jump [8][plane], spread force [2][plane] (arithmetic type) and tile flags of the
  // interface of a state, double-buffered by the parity of the state's time level so
  // the interface phase of step n+1 can run while step n's stream-collide consumes
  // (and re-zeroes) the buffer of step n.
  void *Jb[2];
  void *gb[2];
  unsigned *flagsb[2];   // tile flags: flagged iff equal to the buffer's tag
  unsigned *tagb[2];     // device word: tag of the buffer's current time level
  void *uf;           // [2][plane] collision velocity on flagged tiles (for interpolation)
  int *tile_list[2];  // flagged tiles of each buffer, appended by the interface phase
  int *tile_count[2]; // per buffer: [0] flagged tiles, [1] cut-link crossings
  unsigned long long *d_tiles_total;  // flagged tiles summed while timing
  int ntiles;
  int forced_grid;    // blocks of the forced stream-collide (strides over the list)
  // execution
  bool vector_sc;     // vectorised stream-collide when nx is a multiple of its width
  int tma_sc;         // FP32: interior tiles by the TMA stream-collide (sc_tma_dev.cuh):
                      // 0 never, 1 every step, 2 odd steps only
  const void *tmap_A; // the population array the tensor maps below describe
  CUtensorMap tmap[3];  // boxes 136 x 8, 128 x 8, 124 x 8 of [9][ny][pitch]
  bool overlap;       // next interface phase on the side stream during stream-collide
  bool use_graph;     // replay steps from CUDA graphs (GRAPH_KINDS lengths)
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  // per graph kind a ring of GRAPH_RING executables; with timing on each one records
  // into its own event set, so draining a set never waits on the GPU (without timing
  // slot 0 alone is used)
  cudaGraphExec_t gexec[iilbm::GRAPH_KINDS][iilbm::GRAPH_RING];
  bool ring_pending[iilbm::GRAPH_KINDS][iilbm::GRAPH_RING];
  int ring_next[iilbm::GRAPH_KINDS];
  bool graph_timing;  // the instantiated graphs record timing events
  bool capturing;     // inside cudaStreamBeginCapture / EndCapture
  bool in_batch;      // advanced by a batch (iilbm_step refused meanwhile)
  struct iilbm_batch *batch;
  cudaStream_t own_main, own_side;  // the lattice's streams while batched
  long long step;     // time level of the state; AA parity = step & 1
  bool prepared;      // jump / force of the current state already in J, g
  int *d_status;      // latched device status bits
  // interface
  int nm;
  iilbm_interface_params ip;
  double *X, *aux, *G, *Fn, *U, *nrm;
  long long *Xq;      // marker coordinates snapped to 2^-24 (XQ_OUT outside the region)
  double *Xp;         // X, Xq of the level being interpolated, for the fused phase
  long long *Xqp;
  double *G0, *Gdf;   // direct forcing: warm start and converged force
  double *spl_c, *spl_f;  // spline interface: coefficients of X [n][2] and of Fn [n]
  double *Ustar;      // direct forcing: interpolated velocity without the body's force
  int ws_mode;        // direct forcing: where the iteration starts (WS_*)
  const struct iilbm_mlp *mlp;  // WS_MLP: the network proposing G^(0)
  float re;                     // WS_MLP: the Reynolds-number feature
  int *d_mdf_iters;
  double *d_mdf_res;
  // direct forcing of a fixed body: the band of nodes its iteration touches (sorted keys
  // y * nx + x), each stencil node's band index, and the cut-link records (DfLink)
  int *df_band;
  int df_nb;
  int *df_st;
  void *df_links;
  int df_nl;
  // a rigid body carrying the directly forced interface (iilbm_set_rigid_body): its
  // state on the device, the markers' offsets from its centre at angle 0, and the
  // capacities of the band the force iteration rebuilds every step
  struct iilbm_body_dev *body;
  double *body_X0;
  int body_words, body_nb, body_nl;
  double *d_res;      // direct forcing residual scratch
  // diagnostics
  bool timing;
  int nev;                      // event pairs in use
  cudaEvent_t ev[iilbm::EAGER_EV0 + 2 * iilbm::EAGER_PAIRS];  // lean stream-collide start / stop
  double sc_ms;
  int sc_launches;
  long long kernel_launches;    // every library kernel launched while timing
};

// Launchers (defined in lattice.cu / interface.cu).
namespace iilbm {
// The next level's interface phase runs on the side stream during the stream-collide,
// fused with the interpolation (direct forcing needs the next state first, so its
// interface phase waits for the next step's force iteration).
inline bool pipelined(const iilbm_lattice *h) {
  return h->overlap && h->nm > 0 && h->ip.model != IILBM_DIRECT && h->ip.curve == 0;
}

int launch_stream_collide(iilbm_lattice *h, cudaStream_t forced_stream);
bool uses_tma_sc(const iilbm_lattice *h, bool odd);
int launch_interp(iilbm_lattice *h, cudaStream_t s);
int launch_macros(iilbm_lattice *h, double *drho, double *ux, double *uy);
int launch_set_populations(iilbm_lattice *h, const double *df, bool equilibrium,
                           const double *rho, const double *ux, const double *uy);
int launch_get_populations(iilbm_lattice *h, double *df);
int launch_get_jump(iilbm_lattice *h, double *out);
int launch_interface_phase(iilbm_lattice *h, int buf, cudaStream_t s);
int launch_interp_interface(iilbm_lattice *h, cudaStream_t s);
int launch_channel_bc(iilbm_lattice *h);
int launch_direct_forcing(iilbm_lattice *h);
int launch_body_update(iilbm_lattice *h);
void free_body(iilbm_lattice *h);
int launch_df_features(iilbm_lattice *h, float re, float *F);
size_t direct_forcing_smem(const iilbm_lattice *h, int nb, int n);
int setup_direct_forcing(iilbm_lattice *h, const double *hx);
void free_direct_forcing(iilbm_lattice *h);
struct DfArgs;
DfArgs df_args(const iilbm_lattice *h);
const float *mlp_params(const struct iilbm_mlp *M);
const float *mlp_params_transposed(const struct iilbm_mlp *M);
const float *mlp_norm(const struct iilbm_mlp *M);
int mlp_device(const struct iilbm_mlp *M);
int prepare_lattice(iilbm_lattice *h);
int prepare_batch_of(iilbm_lattice *h);
}  // namespace iilbm

// sc_tma_dev.cuh -- the lean stream-collide of interior tiles with the tensor memory
// accelerator (TMA): FP32 storage, D2Q9, either AA parity.
//
// One persistent block per SM (512 threads) walks the interior tiles (128 x 8 nodes, the
// flag tiles) round-robin.  Thread 0 moves every tile with bulk tensor copies: each
// population plane's box is loaded into shared memory (a four-stage ring, an mbarrier per
// stage: three tiles in flight while one computes) and, after the collision, stored back
// from an output area.  The 16 warps never address global memory for the bulk of the
// data: they read the streamed populations from shared memory with the AA shift folded
// into the index, collide, and write the post-collision values into the output boxes.
// Loads of the next tiles are in flight while a tile computes, so the memory system sees
// the same bytes in flight whatever the parity.
//
// The odd step reads slot opp(i) of x - e_i and writes slot i of x + e_i.  Its load box of
// a plane is 136 nodes wide, from x = xb - 4 (a 16-byte boundary; every row needs only one
// node beyond the tile on one side).  Its store box of a plane with e_x = +-1 covers the
// 124 aligned nodes the tile writes alone (xb + 4 .. xb + 127 for e_x = +1, xb .. xb + 123
// for e_x = -1); the four remaining values of each row land next to a neighbouring tile's
// values inside one 16-byte segment: they go to an edge slot after the box in shared
// memory and from there to global memory with plain stores, as the register-path kernel
// writes them at its warp ends.  Every (plane, row, column) is
// written by exactly one node, and a node's read set is its write set (the AA pattern), so
// the tiles need no ordering among themselves or with the edge tiles of the other launch.
//
// Interior tiles have every box inside the lattice (no wrap, no wall row, no channel ghost
// column): xb >= 128, xb + 132 <= nx, yb >= 8, yb + 9 <= ny.  The other tiles, and every
// flagged tile, are left to the register-path kernels.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "lattice_dev.cuh"

namespace iilbm {

constexpr int TMA_W = 128;          // tile width (nodes), = TILE_X
constexpr int TMA_R = 8;            // tile height (rows), = TILE_Y
constexpr int TMA_HALO = 4;         // odd-step load box starts 4 nodes left of the tile
constexpr int TMA_LW_ODD = TMA_W + 2 * TMA_HALO;  // 136
constexpr int TMA_SW = TMA_W - 4;   // 124: odd-step store box of the e_x = +-1 planes
constexpr int TMA_EDGE = TMA_R * TMA_SW;  // their edge values: [8][4] after the box
constexpr int TMA_STAGES = 4;
constexpr int TMA_THREADS = 512;
constexpr unsigned TMA_SPIN_LIMIT = 1u << 22;  // mbarrier polls before a wait gives up
constexpr int TMA_MASK_WORDS = 256;  // a block's flag mask: up to 8192 candidate tiles
static_assert(TMA_W == TILE_X && TMA_R == TILE_Y, "TMA tiles are the flag tiles");

// Interior tiles: tile columns [tx0, tx0 + ntx_i), tile rows [ty0, ty0 + nty_i).
struct TmaTiles {
  int tx0, ntx_i, ty0, nty_i;
};

// Shared memory of one block (dynamic; 128-byte aligned boxes).
template <bool ODD>
struct TmaSmem {
  static constexpr int LW = ODD ? TMA_LW_ODD : TMA_W;
  static constexpr int IN_BOX = TMA_R * LW;     // floats per plane box in
  static constexpr int OUT_BOX = TMA_R * TMA_W; // floats per plane slot out
  static constexpr size_t in_bytes = (size_t)TMA_STAGES * 9 * IN_BOX * 4;
  static constexpr size_t out_bytes = (size_t)9 * OUT_BOX * 4;
  static constexpr size_t bytes = in_bytes + out_bytes + 128;
  static constexpr unsigned stage_tx = 9u * IN_BOX * 4u;
  static_assert((IN_BOX * 4) % 128 == 0 && (OUT_BOX * 4) % 128 == 0, "box alignment");
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0u;
}
// Bounded wait for the phase of the given parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (unsigned k = 0; k < TMA_SPIN_LIMIT; k++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int x, int y, int z,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store3(const CUtensorMap *map, int x, int y, int z,
                                           const void *src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group"
               " [%0, {%1, %2, %3}], [%4];" ::"l"(reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(smem_addr(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until at most N committed store groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace iilbm

namespace iilbm {

__device__ __forceinline__ void tma_tile_xy(const TmaTiles &t, int k, int &xb, int &yb) {
  xb = (t.tx0 + k % t.ntx_i) * TMA_W;
  yb = (t.ty0 + k / t.ntx_i) * TMA_R;
}

// The persistent TMA stream-collide of the interior tiles that carry no flag.
// m_load: box LW x 8 x 1 of the populations [9][ny][pitch] (LW = 136 odd, 128 even);
// m_store: box 128 x 8 x 1; m_store_s: box 124 x 8 x 1 (odd step, e_x = +-1 planes).
// Warp w computes row w / 2 of the tile, lanes nodes (w % 2) 64 + lane + 32 j, j = 0, 1:
// every shared-memory access of a warp reads or writes 32 consecutive words.
template <int COLL, bool ODD, bool BODY>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    k_stream_collide_tma(const __grid_constant__ CUtensorMap m_load,
                         const __grid_constant__ CUtensorMap m_store,
                         const __grid_constant__ CUtensorMap m_store_s, float *__restrict__ A,
                         const unsigned *__restrict__ flags, const unsigned *__restrict__ tag,
                         const Geom geo, const TmaTiles tt, const CollP<float> p,
                         int *status) {
  using SM = TmaSmem<ODD>;
  constexpr int LW = SM::LW;
  extern __shared__ unsigned char tma_smem_raw[];
  unsigned char *base =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tma_smem_raw) + 127) &
                                        ~static_cast<uintptr_t>(127));
  float *in = reinterpret_cast<float *>(base);
  float *out = reinterpret_cast<float *>(base + SM::in_bytes);
  __shared__ uint64_t full[TMA_STAGES];
  __shared__ int tile_of[TMA_STAGES];
  __shared__ int abort_flag;
  __shared__ unsigned skip[TMA_MASK_WORDS];  // bit j: candidate j carries a flag
  const int tid = threadIdx.x;
  const int ntiles = tt.ntx_i * tt.nty_i;
  // the block's candidates are tiles blockIdx.x + j gridDim.x, j < J (J <= 32 x the mask)
  const int J = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  {
    const unsigned tg = *tag;
    const int lane = tid & 31;
    for (int wd = tid >> 5; wd < (J + 31) / 32; wd += TMA_THREADS / 32) {
      const int j = wd * 32 + lane;
      bool flagged = false;
      if (j < J) {
        int xb, yb;
        tma_tile_xy(tt, (int)blockIdx.x + j * (int)gridDim.x, xb, yb);
        flagged = flags[(yb / TMA_R) * geo.ntx + xb / TMA_W] == tg;
      }
      const unsigned m = __ballot_sync(0xffffffffu, flagged);
      if (lane == 0) skip[wd] = m;
    }
  }
  __syncthreads();
  int cj = 0;  // thread 0's cursor over the candidates

  // thread 0: the next candidate without a flag (-1: none left)
  auto claim = [&]() -> int {
    while (cj < J) {
      const int j = cj++;
      if (!((skip[j >> 5] >> (j & 31)) & 1u)) return (int)blockIdx.x + j * (int)gridDim.x;
    }
    return -1;
  };
  // thread 0: load tile k's nine plane boxes into stage s
  auto issue = [&](int s, int k) {
    tile_of[s] = k;
    if (k < 0) return;
    int xb, yb;
    tma_tile_xy(tt, k, xb, yb);
    mbar_expect_tx(&full[s], SM::stage_tx);
    float *dst = in + (size_t)s * 9 * SM::IN_BOX;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      if (ODD)  // slot opp(i) of x - e_i
        tma_load3(dst + i * SM::IN_BOX, &m_load, xb - TMA_HALO, yb - cy(i), opp(i), &full[s]);
      else  // slot i of x
        tma_load3(dst + i * SM::IN_BOX, &m_load, xb, yb, i, &full[s]);
    }
  };

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < TMA_STAGES; s++) mbar_init(&full[s], 1);
    fence_barrier_init();
    abort_flag = 0;
#pragma unroll
    for (int s = 0; s < TMA_STAGES; s++) issue(s, claim());
  }
  __syncthreads();

  const int w = tid >> 5, lane = tid & 31, r = w >> 1, half = w & 1;
  const float gxs = BODY ? p.bodyx * p.scale : 0.0f, gys = BODY ? p.bodyy * p.scale : 0.0f;
  int s = 0;
  uint32_t phase = 0;
  for (;;) {
    const int k = tile_of[s];
    if (k < 0) break;  // uniform: the claims come in order, none is left
    int xb, yb;
    tma_tile_xy(tt, k, xb, yb);
    const bool ok = mbar_wait(&full[s], phase);
    float f[2][9];
    if (!ok) {
      atomicOr(status, ST_TIMEOUT);
      abort_flag = 1;
    } else {
      const float *src = in + (size_t)s * 9 * SM::IN_BOX + r * LW;
      bool finite = true;
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int u = half * 64 + lane + 32 * j;
#pragma unroll
        for (int i = 0; i < 9; i++)
          f[j][i] = src[i * SM::IN_BOX + (ODD ? u + TMA_HALO - cx(i) : u)];
        float ux, uy;
        const float drho = collide<float, COLL, CollP<float>, BODY>(f[j], gxs, gys, p, ux, uy);
        finite = finite && isfinite(drho);
      }
      if (!finite) atomicOr(status, ST_NONFINITE);
    }
    __syncthreads();  // stage s consumed; the output area read out by the last stores
    if (abort_flag) break;
    if (tid == 0) issue(s, claim());  // refill stage s at once
    if (ok) {
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int u = half * 64 + lane + 32 * j;
#pragma unroll
        for (int i = 0; i < 9; i++) {
          const float v = f[j][i];
          if (!ODD) {  // slot opp(i) of x
            out[opp(i) * SM::OUT_BOX + r * TMA_W + u] = v;
          } else if (cx(i) == 0) {  // slot i of x + e_i: the same columns
            out[i * SM::OUT_BOX + r * TMA_W + u] = v;
          } else if (cx(i) > 0) {  // column xb + u + 1; the box covers xb + 4 .. xb + 127,
                                   // u = 0, 1, 2, 127 go to the edge slot (e = 0, 1, 2, 3)
            const bool box = u >= 3 && u < TMA_W - 1;
            const int e = u == TMA_W - 1 ? 3 : u;
            out[i * SM::OUT_BOX + (box ? r * TMA_SW + (u - 3) : TMA_EDGE + 4 * r + e)] = v;
          } else {  // column xb + u - 1; the box covers xb .. xb + 123, u = 0, 125, 126,
                    // 127 go to the edge slot (e = 0, 1, 2, 3)
            const bool box = u >= 1 && u <= TMA_SW;
            const int e = u == 0 ? 0 : u - TMA_SW;
            out[i * SM::OUT_BOX + (box ? r * TMA_SW + (u - 1) : TMA_EDGE + 4 * r + e)] = v;
          }
        }
      }
    }
    fence_async_shared();  // the output boxes, written by the threads, go to the TMA
    __syncthreads();       // output area complete
    if (ODD && tid < 6 * 32) {
      // the edge values: six planes with e_x != 0 x 8 rows x 4, one plain store each
      const int q = tid >> 5, rr = (tid >> 2) & 7, e = tid & 3;
      const int i = q < 2 ? 2 * q + 1 : q + 3;  // planes 1, 3, 5, 6, 7, 8
      const int col = cx(i) > 0 ? (e < 3 ? xb + 1 + e : xb + TMA_W) : (e == 0 ? xb - 1 : xb + TMA_SW - 1 + e);
      A[i * geo.plane + (long long)(yb + rr + cy(i)) * geo.pitch + col] =
          out[i * SM::OUT_BOX + TMA_EDGE + 4 * rr + e];
    }
    if (tid == 0) {
#pragma unroll
      for (int i = 0; i < 9; i++) {
        const float *b = out + i * SM::OUT_BOX;
        if (!ODD) tma_store3(&m_store, xb, yb, i, b);
        else if (cx(i) == 0) tma_store3(&m_store, xb, yb + cy(i), i, b);
        else if (cx(i) > 0) tma_store3(&m_store_s, xb + 4, yb + cy(i), i, b);
        else tma_store3(&m_store_s, xb, yb + cy(i), i, b);
      }
      bulk_commit();
      bulk_wait_read<0>();  // the output area is free again once the stores have read it
    }
    if (++s == TMA_STAGES) {
      s = 0;
      phase ^= 1u;
    }
  }
  if (tid == 0) {
    if (abort_flag) {
      // let the loads still in flight land before the block's shared memory goes away
      for (int q = 0; q < TMA_STAGES; q++) {
        if (tile_of[s] >= 0) mbar_wait(&full[s], phase);
        if (++s == TMA_STAGES) {
          s = 0;
          phase ^= 1u;
        }
      }
    }
    bulk_wait<0>();  // every store complete
  }
}

// The lean register-path stream-collide over the tiles outside the interior rectangle
// (rows below and above it, the columns left and right of it), one block per tile.
template <typename S, int COLL, bool ODD, int BC, bool BODY>
__global__ void __launch_bounds__(32 * VEC_ROWS, 3)
    k_stream_collide_vec_edge(S *__restrict__ A, const unsigned *__restrict__ flags,
                              const unsigned *__restrict__ tag, const Geom geo,
                              const CollP<typename Store<S>::T> p, int *status,
                              const TmaTiles tt, int nty) {
  constexpr int W = 32 * Vec<S>::V;
  static_assert(W == TILE_X && VEC_ROWS == TILE_Y, "edge tiles are flag tiles");
  const int ntx = geo.ntx;
  const int below = tt.ty0 * ntx, side = ntx - tt.ntx_i;
  int b = blockIdx.x, tx, ty;
  if (b < below) {
    ty = b / ntx;
    tx = b % ntx;
  } else if ((b -= below) < tt.nty_i * side) {
    ty = tt.ty0 + b / side;
    const int c = b % side;
    tx = c < tt.tx0 ? c : c + tt.ntx_i;
  } else {
    b -= tt.nty_i * side;
    ty = tt.ty0 + tt.nty_i + b / ntx;
    tx = b % ntx;
  }
  if (ty >= nty) return;
  if (flags[ty * ntx + tx] == *tag) return;  // uniform per block
  sc_vec_rows<S, COLL, ODD, BC, false, Vec<S>::V, BODY>(A, nullptr, nullptr, nullptr, geo, p,
                                                         status, tx * W, ty * VEC_ROWS);
}

}  // namespace iilbm

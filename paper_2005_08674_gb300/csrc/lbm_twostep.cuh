// lbm_twostep.cuh -- two time steps per launch for one domain (temporal
// blocking).  Each block owns an output tile of TX x TY nodes: it stages the
// state at step n over the tile and two nodes around it in shared memory
// (nine bulk copies per row, completing on an mbarrier), computes step n + 1
// over the tile and one node around it into a second shared-memory buffer --
// never written to device memory -- and from that step n + 2 over the tile,
// which it stores.  Every node runs the same device functions as the
// single-step kernels (the interior collision on pulled vectors, the NSBC
// quads through source / destination accessors) and step n + 1 is rounded to
// the storage type exactly as a single step stores it, so one launch gives
// the bits of two single steps.  The last tile along each axis is shifted
// back to end at the domain's edge (overlapping its neighbour: two blocks
// compute and store the same nodes, with the same bits), so no tile is thin
// and every boundary node's second-order differences lie inside its tile.  Device-memory traffic
// per two steps: one read and one write of the state; the halo rows and
// columns of neighbouring tiles are read again, mostly from L2.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_staged.cuh"

namespace lbmk {

constexpr int kTwoStepThreads = 320;  // 10 warps, two blocks per SM

template <typename T>
struct TwoStepShape;
template <>
struct TwoStepShape<float> {
  static constexpr int TX = 120;
};
template <>
struct TwoStepShape<__half> {
  static constexpr int TX = 240;
};
template <>
struct TwoStepShape<__nv_bfloat16> {
  static constexpr int TX = 240;
};

template <typename T>
struct TwoStep {
  static constexpr int V = Store<T>::V;
  static constexpr int TX = TwoStepShape<T>::TX;  // output columns per tile
  static constexpr int TY = 8;                    // output rows per tile
  static constexpr int RW = TX + 2 * V;           // elements of one population's row in the buffers
  static constexpr int NV = RW / V;               // vectors per buffer row
  static constexpr int R0 = TY + 4;               // state rows staged: the tile and two around it
  static constexpr int R1 = TY + 2;               // intermediate rows: the tile and one around it
  static constexpr int SLOT = 9 * RW;             // elements per buffer row (nine populations)
  static constexpr size_t kSmem = (size_t)(R0 + R1) * SLOT * sizeof(T);
};

// Scalar shared-memory element <-> physical units (the storage scale undone),
// rounding exactly as the global accessors do.
template <typename T>
__device__ __forceinline__ typename Store<T>::C ld1p(const T* p) {
  using S = Store<T>;
  using C = typename S::C;
  if constexpr (S::kScale == 1)
    return S::ld1s(p);
  else
    return S::ld1s(p) * C(1.0 / S::kScale);
}

// Node (x, y) of a tile buffer whose row 0 is domain row ybase and whose
// element 0 of a row is column xbase.
template <typename T>
struct TileSrc {
  const T* base;
  int xbase, ybase;
  __device__ __forceinline__ typename Store<T>::C ld(int i, int x, int y) const {
    return ld1p<T>(base + ((y - ybase) * 9 + i) * TwoStep<T>::RW + (x - xbase));
  }
};

template <typename T>
struct TileDst {
  T* base;
  int xbase, ybase;
  __device__ __forceinline__ void st(int i, int x, int y, typename Store<T>::C v) const {
    base[((y - ybase) * 9 + i) * TwoStep<T>::RW + (x - xbase)] = Store<T>::cvt(v);
  }
};

// Vector stores of CPT nodes (stored units) to shared memory.
template <typename T, int CPT>
__device__ __forceinline__ void sts_vec(T* p, const typename Store<T>::C (&o)[CPT]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
    static_assert(sizeof(T) == 2 && CPT == 4, "16-bit rows are collided in half vectors");
    T t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] = T(o[k]);  // round to nearest even, as the global stores
    uint2 u;
    memcpy(&u, t, 8);
    *reinterpret_cast<uint2*>(p) = u;
  }
}

// Interior collision of one vector (CPT nodes: part `part` of vector `vec`)
// of row y from the buffer `src` (row 0 = domain row sbase), in stored units
// like the single-step kernels.  Only interior nodes of the domain inside
// [keep_a, keep_b) are stored -- to the buffer `dst` (row 0 = domain row
// dbase) or, TO_GLOBAL, to row y of B -- and nothing is loaded for a vector
// that keeps none.
template <typename T, int MODEL, bool SHIFT, bool TO_GLOBAL>
__device__ __forceinline__ void tile_collide(const T* src, int sbase, int xbase, int vec, int part, int y,
                                             const Geom& g, const Rates<typename Store<T>::C>& r, int keep_a,
                                             int keep_b, T* dst, int dbase, T* __restrict__ B) {
  using S = Store<T>;
  using C = typename S::C;
  using TS = TwoStep<T>;
  constexpr int V = TS::V;
  constexpr int SPLIT = sizeof(T) == 2 ? 2 : 1;
  constexpr int CPT = V / SPLIT;
  const int col = vec * V + part * CPT;  // buffer column of the first node
  const int x0 = xbase + col;
  if (y < 1 || y > g.ny - 2) return;  // boundary rows are the NSBC's
  const int lo = max(max(keep_a, 1), x0), hi = min(min(keep_b, g.nx - 1), x0 + CPT);
  if (lo >= hi) return;
  C v[9][CPT], lf[9], rt[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T* e = src + ((y - cy(i) - sbase) * 9 + i) * TS::RW + col;  // pull: from row y - c_iy
    if constexpr (SPLIT == 1)
      S::lds(e, v[i]);
    else
      S::ldsp(e, v[i]);
    lf[i] = col > 0 ? S::ld1s(e - 1) : C(0);                 // x0 - 1 (outside the buffer: a node not kept)
    rt[i] = col + CPT < TS::RW ? S::ld1s(e + CPT) : C(0);  // x0 + CPT
  }
  C o[9][CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    C h[9];
    h[0] = v[0][k];
    h[1] = k == 0 ? lf[1] : v[1][k - 1];
    h[2] = k == CPT - 1 ? rt[2] : v[2][k + 1];
    h[3] = v[3][k];
    h[4] = v[4][k];
    h[5] = k == 0 ? lf[5] : v[5][k - 1];
    h[6] = k == CPT - 1 ? rt[6] : v[6][k + 1];
    h[7] = k == CPT - 1 ? rt[7] : v[7][k + 1];
    h[8] = k == 0 ? lf[8] : v[8][k - 1];
    collide<MODEL, SHIFT>(h, r, C(S::kScale));
#pragma unroll
    for (int i = 0; i < 9; ++i) o[i][k] = h[i];
  }
  const bool whole = lo == x0 && hi == x0 + CPT;
  if constexpr (TO_GLOBAL) {
    T* row = B + (long long)y * g.pitch;
    if (whole) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        if constexpr (SPLIT == 1)
          S::st(row + i * g.plane + x0, o[i]);
        else
          S::stp(row + i * g.plane + x0, o[i]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < CPT; ++k)
        if (x0 + k >= lo && x0 + k < hi) {
#pragma unroll
          for (int i = 0; i < 9; ++i) S::st1r(row + i * g.plane + x0 + k, o[i][k]);
        }
    }
  } else {
    T* row = dst + (y - dbase) * 9 * TS::RW + col;
    if (whole) {
#pragma unroll
      for (int i = 0; i < 9; ++i) sts_vec<T, CPT>(row + i * TS::RW, o[i]);
    } else {
#pragma unroll
      for (int k = 0; k < CPT; ++k)
        if (x0 + k >= lo && x0 + k < hi) {
#pragma unroll
          for (int i = 0; i < 9; ++i) row[i * TS::RW + k] = T(o[i][k]);
        }
    }
  }
}

// Perimeter index (the order perimeter_node walks) of edge node (x, y).
__device__ __forceinline__ int perimeter_index(int x, int y, int nx, int ny) {
  if (y == 0) return x;
  if (y == ny - 1) return nx + x;
  return 2 * nx + (x == 0 ? y - 1 : (ny - 2) + (y - 1));
}

// The perimeter nodes of rows [ya, yb) x columns [ca, cb): whole rows 0 and
// ny - 1, and columns 0 and nx - 1 of the other rows.
__device__ __forceinline__ int edge_count_row(int y, int ca, int cb, int nx, int ny) {
  if (y == 0 || y == ny - 1) return cb - ca;
  return (ca == 0 ? 1 : 0) + (cb == nx ? 1 : 0);
}
__device__ __forceinline__ void edge_of(int m, int ya, int yb, int ca, int cb, int nx, int ny, int& x, int& y) {
  for (y = ya; y < yb; ++y) {
    const int n = edge_count_row(y, ca, cb, nx, ny);
    if (m < n) {
      x = (y == 0 || y == ny - 1) ? ca + m : ((m == 0 && ca == 0) ? 0 : nx - 1);
      return;
    }
    m -= n;
  }
  x = ca;
  y = ya;  // not reached: m < the count of the rows
}

// NSBC quads (Sec. 5) for the perimeter nodes of rows [ya, yb) x columns
// [ca, cb), reading the previous state through `src` and writing through
// `dst`; four lanes per node, every thread of the block takes lanes.
template <typename T, int MODEL, bool SHIFT, typename Src, typename Dst>
__device__ __forceinline__ void tile_edges(const Src& src, const Dst& dst, const Geom& g, const Nsbc& p,
                                           const Rates<typename Store<T>::C>& r, int ya, int yb, int ca, int cb) {
  int total = 0;
  for (int y = ya; y < yb; ++y) total += edge_count_row(y, ca, cb, g.nx, g.ny);
  for (int l = threadIdx.x; l < 4 * total; l += blockDim.x) {  // a quad's lanes are consecutive
    int x, y;
    edge_of(l >> 2, ya, yb, ca, cb, g.nx, g.ny, x, y);
    const int node[1] = {perimeter_index(x, y, g.nx, g.ny)};
    const bool ok[1] = {true};
    nsbc_nodes<T, MODEL, 1, SHIFT>(src, dst, g, p, r, node, ok, l & 3);
  }
}

// Origin of tile t (tiles nbx wide): the last tile along each axis ends at
// the domain's edge; X0 stays a multiple of V for the copies' alignment (the
// last tile along x starts at nx - TX rounded up, so it may be up to V - 1
// columns short of TX).
template <typename T>
__device__ __forceinline__ void tile_origin(int t, int nbx, const Geom& g, int& X0, int& Y0) {
  using TS = TwoStep<T>;
  constexpr int V = TS::V;
  X0 = min((t % nbx) * TS::TX, (max(0, g.nx - TS::TX) + V - 1) / V * V);
  Y0 = min((t / nbx) * TS::TY, max(0, g.ny - TS::TY));
}

// Warp 0: the state rows of tile t into buf0, nine bulk copies per row
// completing on `bar` (lane 0 announces the bytes, then the lanes copy).
// (Checked build: a copy whose source or destination range fails is neither
// issued nor counted in the barrier's byte total.)
template <typename T>
__device__ __forceinline__ void stage_tile(const T* __restrict__ A, const Geom& g, int t, int nbx, T* buf0,
                                           uint64_t* bar) {
  using TS = TwoStep<T>;
  constexpr int V = TS::V;
  int X0, Y0;
  tile_origin<T>(t, nbx, g, X0, Y0);
  const int xbase = X0 - V, ybase0 = Y0 - 2;
  const int ya0 = max(Y0 - 2, 0), yb0 = min(Y0 + TS::TY + 2, g.ny);
  const int lo_x = max(xbase, 0), hi_x = min(xbase + TS::RW, g.pitch);
  const uint32_t row_bytes = (uint32_t)(hi_x - lo_x) * (uint32_t)sizeof(T);
  const long long slot_bytes = (long long)(TS::R0 * TS::SLOT) * (long long)sizeof(T);
  const int lane = threadIdx.x & 31;
  uint32_t mine = 0;
  for (int k = lane; k < 9 * (yb0 - ya0); k += 32) {
    const int y = ya0 + k / 9, i = k % 9;
    const long long d = ((long long)((y - ybase0) * 9 + i) * TS::RW + (lo_x - xbase)) * (long long)sizeof(T);
    if (in_bounds(A + i * g.plane + (long long)y * g.pitch + lo_x, row_bytes) && in_slot(d, row_bytes, slot_bytes))
      mine += row_bytes;
  }
  const uint32_t total = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0) mbar_expect_tx(bar, total);
  __syncwarp();
  for (int k = lane; k < 9 * (yb0 - ya0); k += 32) {
    const int y = ya0 + k / 9, i = k % 9;
    const T* src = A + i * g.plane + (long long)y * g.pitch + lo_x;
    const long long d = ((long long)((y - ybase0) * 9 + i) * TS::RW + (lo_x - xbase)) * (long long)sizeof(T);
    if (in_bounds(src, row_bytes) && in_slot(d, row_bytes, slot_bytes))
      bulk_copy_g2s(reinterpret_cast<unsigned char*>(buf0) + d, src, row_bytes, bar);
  }
}

// Two steps: state A (step n) -> B (step n + 2).  Persistent: block b takes
// tiles b, b + gridDim.x, ... of the ntiles (nbx wide); the state of its next
// tile is copied into buf0 while it computes step n + 2 of the current one
// from buf1.  Domains of at least 8 x 8 nodes without periodic axes.  A
// bounded wait that gives up (in any thread: the block agrees on it) sets
// err[2] and the block returns.
template <typename T, int MODEL, bool SHIFT>
__global__ void __launch_bounds__(kTwoStepThreads, 2)
    twostep_kernel(const T* __restrict__ A, T* __restrict__ B, Geom g, Nsbc p, Rates<typename Store<T>::C> r,
                   int nbx, int ntiles, int* __restrict__ err) {
  using TS = TwoStep<T>;
  constexpr int V = TS::V;
  constexpr int SPLIT = sizeof(T) == 2 ? 2 : 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* buf0 = reinterpret_cast<T*>(smem_raw);
  T* buf1 = buf0 + TS::R0 * TS::SLOT;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x < 32 && (int)blockIdx.x < ntiles) stage_tile<T>(A, g, blockIdx.x, nbx, buf0, &bar);
  uint32_t parity = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int X0, Y0;
    tile_origin<T>(t, nbx, g, X0, Y0);
    const int X1 = min(X0 + TS::TX, g.nx), Y1 = min(Y0 + TS::TY, g.ny);
    const int xbase = X0 - V;
    const int ybase0 = Y0 - 2, ybase1 = Y0 - 1;
    const int ya1 = max(Y0 - 1, 0), yb1 = min(Y1 + 1, g.ny);  // intermediate rows computed
    const int ca1 = max(X0 - 1, 0), cb1 = min(X1 + 1, g.nx);  // intermediate columns kept
    const bool ok = mbar_wait(&bar, parity);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(&err[2], 1);
      return;
    }
    parity ^= 1u;
    // step n + 1 over the tile and one node around it, buf0 -> buf1
    {
      const TileSrc<T> src0{buf0, xbase, ybase0};
      const TileDst<T> dst1{buf1, xbase, ybase1};
      constexpr int PER_ROW = TS::NV * SPLIT;
      const int n = (yb1 - ya1) * PER_ROW;
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int rr = k / PER_ROW, rem = k - rr * PER_ROW;
        tile_collide<T, MODEL, SHIFT, false>(buf0, ybase0, xbase, rem / SPLIT, rem % SPLIT, ya1 + rr, g, r, ca1, cb1,
                                             buf1, ybase1, nullptr);
      }
      tile_edges<T, MODEL, SHIFT>(src0, dst1, g, p, r, ya1, yb1, ca1, cb1);
    }
    __syncthreads();
    // buf0 is free: the next tile's state moves in while step n + 2 runs
    if (threadIdx.x < 32 && t + (int)gridDim.x < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      stage_tile<T>(A, g, t + gridDim.x, nbx, buf0, &bar);
    }
    // step n + 2 over the tile, buf1 -> B (vectors 1 .. NV - 2 cover the tile)
    {
      const TileSrc<T> src1{buf1, xbase, ybase1};
      const GlobalDst<T> dstB{B, g.plane, g.pitch};
      constexpr int PER_ROW = (TS::NV - 2) * SPLIT;
      const int n = (Y1 - Y0) * PER_ROW;
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int rr = k / PER_ROW, rem = k - rr * PER_ROW;
        tile_collide<T, MODEL, SHIFT, true>(buf1, ybase1, xbase, 1 + rem / SPLIT, rem % SPLIT, Y0 + rr, g, r, X0,
                                            X1, nullptr, 0, B);
      }
      tile_edges<T, MODEL, SHIFT>(src1, dstB, g, p, r, Y0, Y1, X0, X1);
    }
    __syncthreads();  // buf1 read before the next tile's step n + 1 writes it
  }
}

}  // namespace lbmk

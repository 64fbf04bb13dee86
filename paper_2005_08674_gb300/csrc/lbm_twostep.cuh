// lbm_twostep.cuh -- two time steps per launch for one domain (temporal
// blocking).  Each block owns an output region of W columns x band rows and
// streams down it row group by row group with two rings of rows in shared
// memory: S0 rows (the state at step n, copied in from global memory by
// cp.async, one group ahead) and S1 rows (step n + 1, computed here and never
// written to global memory).  Step n + 2 rows are computed from the S1 ring
// and stored to the output buffer.  Every node runs the same device functions
// as the single-step kernels -- the interior collision on pulled vectors,
// the NSBC quads through source / destination accessors -- and S1 is rounded
// to the storage type exactly as a single step would store it, so two
// launches of a single-step kernel and one launch of this one give the same
// bits.  A node of S1 is computed by every block whose output region reaches
// within one node of it (a one-node halo around each region, and rows down to
// two away for the boundary's second-order differences): DRAM traffic per
// two steps is one read and one write of the state plus the halo.
#pragma once

#include "lbm_kernels.cuh"

namespace lbmk {

constexpr int kTwoStepThreads = 288;  // 9 warps: one vector of a G-row group of S1 per thread
constexpr int kTwoStepG = 4;          // rows per group

template <typename T>
struct TwoStepShape;
template <>
struct TwoStepShape<float> {
  static constexpr int W = 256;
};
template <>
struct TwoStepShape<__half> {
  static constexpr int W = 512;
};
template <>
struct TwoStepShape<__nv_bfloat16> {
  static constexpr int W = 512;
};

template <typename T>
struct TwoStep {
  static constexpr int V = Store<T>::V;
  static constexpr int W = TwoStepShape<T>::W;  // output columns per block
  static constexpr int RW = W + 2 * V;          // elements of one population's row in a ring slot
  static constexpr int NV = RW / V;             // vectors per ring row
  static constexpr int G = kTwoStepG;
  static constexpr int RS0 = 2 * G + 4;  // S0 ring rows: the window of a group (G + 4) and the next group
  static constexpr int RS1 = G + 4;      // S1 ring rows: a group and two rows on each side
  static constexpr int SLOT = 9 * RW;    // elements per ring row (nine populations)
  static constexpr size_t kSmem = (size_t)(RS0 + RS1) * SLOT * sizeof(T);
  static_assert(G * NV <= kTwoStepThreads, "one vector of a group per thread");
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

template <typename T, int SLOTS>
struct RingSrc {
  const T* base;  // ring slot 0
  int xbase;      // column of element 0 of a ring row
  __device__ __forceinline__ typename Store<T>::C ld(int i, int x, int y) const {
    return ld1p<T>(base + ((y % SLOTS) * 9 + i) * TwoStep<T>::RW + (x - xbase));
  }
};

template <typename T, int SLOTS>
struct RingDst {
  T* base;
  int xbase;
  __device__ __forceinline__ void st(int i, int x, int y, typename Store<T>::C v) const {
    base[((y % SLOTS) * 9 + i) * TwoStep<T>::RW + (x - xbase)] = Store<T>::cvt(v);
  }
};

// 16-byte asynchronous copy global -> shared (cp.async.cg: through L2 only).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copy rows [ya, yb) of the state (columns xbase .. xbase + RW, clipped to
// [0, pitch)) into their S0 ring slots; every thread takes a share.
template <typename T>
__device__ __forceinline__ void load_rows(const T* __restrict__ A, const Geom& g, T* ring0, int xbase, int ya,
                                          int yb) {
  using TS = TwoStep<T>;
  constexpr int V = TS::V;
  const int per_row = 9 * TS::NV;
  const int total = (yb - ya) * per_row;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int r = k / per_row, rem = k - r * per_row;
    const int i = rem / TS::NV, vec = rem - i * TS::NV;
    const int y = ya + r, x = xbase + vec * V;
    if (x < 0 || x >= g.pitch) continue;
    const T* src = A + i * g.plane + (long long)y * g.pitch + x;
    T* dst = ring0 + ((y % TS::RS0) * 9 + i) * TS::RW + vec * V;
    if (in_bounds(src, 16)) cp_async16(dst, src);
  }
}

// Vector stores of CPT nodes (stored units) to shared memory.
template <typename T, int CPT>
__device__ __forceinline__ void sts_vec(T* p, const typename Store<T>::C (&o)[CPT]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  } else if constexpr (sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  } else {
    static_assert(CPT == 4, "16-bit rows are collided in half vectors");
    T t[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] = T(o[k]);  // round to nearest even, as the global stores
    uint2 u;
    memcpy(&u, t, 8);
    *reinterpret_cast<uint2*>(p) = u;
  }
}

// Interior collision of the vector (CPT nodes, part `part` of vector `vec`)
// of row y from the ring rows around it (src: SLOTS-row ring), in stored
// units like the single-step kernels.  Nodes that are not interior nodes of
// the domain, or outside [keep_a, keep_b), are not stored.  Stores go to the
// destination ring (TO_GLOBAL false) or to global row y of B.
template <typename T, int MODEL, bool SHIFT, int SLOTS, bool TO_GLOBAL>
__device__ __forceinline__ void ring_collide(const T* src, int xbase, int vec, int part, int y, const Geom& g,
                                             const Rates<typename Store<T>::C>& r, int keep_a, int keep_b, T* dst,
                                             int dst_slots, T* __restrict__ B) {
  using S = Store<T>;
  using C = typename S::C;
  using TS = TwoStep<T>;
  constexpr int V = TS::V;
  constexpr int SPLIT = sizeof(T) == 2 ? 2 : 1;
  constexpr int CPT = V / SPLIT;
  const int col = vec * V + part * CPT;  // ring column of the first node
  const int x0 = xbase + col;
  // nodes to store: interior nodes of the domain inside [keep_a, keep_b);
  // boundary rows are the NSBC's (and the rows around them may not be in the
  // ring), so nothing is loaded for a vector that keeps no node
  if (y < 1 || y > g.ny - 2) return;
  const int lo = max(max(keep_a, 1), x0), hi = min(min(keep_b, g.nx - 1), x0 + CPT);
  if (lo >= hi) return;
  C v[9][CPT], lf[9], rt[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int ys = y - cy(i);  // pull: population i comes from row y - c_iy
    const T* e = src + ((ys % SLOTS) * 9 + i) * TS::RW + col;
    if constexpr (SPLIT == 1)
      S::lds(e, v[i]);
    else
      S::ldsp(e, v[i]);
    lf[i] = col > 0 ? S::ld1s(e - 1) : C(0);            // x0 - 1 (outside the ring: a node not kept)
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
  if constexpr (TO_GLOBAL) {
    T* row = B + (long long)y * g.pitch;
    if (lo == x0 && hi == x0 + CPT) {
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
    T* row = dst + (y % dst_slots) * 9 * TS::RW + col;
    if (lo == x0 && hi == x0 + CPT) {
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

// The perimeter nodes of rows [ya, yb) and columns [ca, cb): whole rows 0 and
// ny - 1, and columns 0 and nx - 1 of the other rows.  Node m of that list
// -> (x, y); returns false past its end.
__device__ __forceinline__ int edge_count_row(int y, int ca, int cb, int nx, int ny) {
  if (y == 0 || y == ny - 1) return cb - ca;
  return (ca == 0 ? 1 : 0) + (cb == nx ? 1 : 0);
}
__device__ __forceinline__ bool edge_of(int m, int ya, int yb, int ca, int cb, int nx, int ny, int& x, int& y) {
  for (y = ya; y < yb; ++y) {
    const int n = edge_count_row(y, ca, cb, nx, ny);
    if (m < n) {
      if (y == 0 || y == ny - 1)
        x = ca + m;
      else
        x = (m == 0 && ca == 0) ? 0 : nx - 1;
      return true;
    }
    m -= n;
  }
  return false;
}

// NSBC quads (Sec. 5) for the perimeter nodes of rows [ya, yb) x columns
// [ca, cb), reading the previous state through `src` and writing through
// `dst`; four lanes per node, every thread of the block takes lanes.
template <typename T, int MODEL, bool SHIFT, typename Src, typename Dst>
__device__ __forceinline__ void ring_edges(const Src& src, const Dst& dst, const Geom& g, const Nsbc& p,
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

// Two steps: state A (step n) -> B (step n + 2).  Block b covers output
// columns [X0, X0 + W) of strip b % nstrips and rows [Y0, Y0 + band) of band
// b / nstrips.  Domains of at least 8 x 8 nodes without periodic axes.
template <typename T, int MODEL, bool SHIFT>
__global__ void __launch_bounds__(kTwoStepThreads, 1)
    twostep_kernel(const T* __restrict__ A, T* __restrict__ B, Geom g, Nsbc p, Rates<typename Store<T>::C> r,
                   int band, int nstrips) {
  using TS = TwoStep<T>;
  constexpr int V = TS::V, G = TS::G;
  constexpr int SPLIT = sizeof(T) == 2 ? 2 : 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* ring0 = reinterpret_cast<T*>(smem_raw);
  T* ring1 = ring0 + TS::RS0 * TS::SLOT;
  const int X0 = (blockIdx.x % nstrips) * TS::W, X1 = min(X0 + TS::W, g.nx);
  const int Y0 = (blockIdx.x / nstrips) * band, Y1 = min(Y0 + band, g.ny);
  if (Y0 >= g.ny) return;
  const int xbase = X0 - V;
  // S1 columns needed: one node around the output region, two where a
  // boundary node's second-order difference reaches (a narrow last strip)
  const int c1a = max(X0 - 2, 0), c1b = min(X1 + 2, g.nx);
  const int s1_end = min(Y1 + 2, g.ny);                      // S1 rows needed: [Y0 - 2, Y1 + 2)
  const RingSrc<T, TS::RS0> src0{ring0, xbase};
  const RingDst<T, TS::RS1> dst1{ring1, xbase};
  const RingSrc<T, TS::RS1> src1{ring1, xbase};
  const GlobalDst<T> dstB{B, g.plane, g.pitch};

  // S0 rows for the first group of S1 rows
  int s1_done = max(Y0 - 2, 0);  // S1 rows [.., s1_done) are in the ring
  int s0_have = min(Y0 + G + 4, g.ny);
  load_rows<T>(A, g, ring0, xbase, max(Y0 - 4, 0), s0_have);
  cp_async_commit();
  for (int s0 = Y0; s0 < Y1; s0 += G) {
    const int s1 = min(s0 + G, Y1);
    // S1 rows up to s1 + 2 (S2 rows [s0, s1) read S1 rows s0 - 2 .. s1 + 1)
    const int want = min(s1 + 2, s1_end);
    cp_async_wait_all();
    __syncthreads();
    while (s1_done < want) {
      const int ya = s1_done, yb = min(s1_done + G, want);
      const int nv = (yb - ya) * TS::NV * SPLIT;
      for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        const int rr = k / (TS::NV * SPLIT), rem = k - rr * TS::NV * SPLIT;
        ring_collide<T, MODEL, SHIFT, TS::RS0, false>(ring0, xbase, rem / SPLIT, rem % SPLIT, ya + rr, g, r, c1a,
                                                      c1b, ring1, TS::RS1, nullptr);
      }
      ring_edges<T, MODEL, SHIFT>(src0, dst1, g, p, r, ya, yb, c1a, c1b);
      s1_done = yb;
      if (s1_done < want) __syncthreads();  // the first group fills the S1 ring in two passes
    }
    __syncthreads();
    // the S0 rows of the next group, into slots this group no longer reads
    const int next_have = min(s0_have + G, g.ny);
    if (next_have > s0_have) {
      load_rows<T>(A, g, ring0, xbase, s0_have, next_have);
      s0_have = next_have;
    }
    cp_async_commit();
    // S2 rows [s0, s1): from the S1 ring to B (vectors 1 .. NV - 2: the
    // output columns)
    constexpr int NV2 = (TS::NV - 2) * SPLIT;
    const int nv2 = (s1 - s0) * NV2;
    for (int k = threadIdx.x; k < nv2; k += blockDim.x) {
      const int rr = k / NV2, rem = k - rr * NV2;
      ring_collide<T, MODEL, SHIFT, TS::RS1, true>(ring1, xbase, 1 + rem / SPLIT, rem % SPLIT, s0 + rr, g, r, X0,
                                                   X1, nullptr, 0, B);
    }
    ring_edges<T, MODEL, SHIFT>(src1, dstB, g, p, r, s0, s1, X0, X1);
  }
  cp_async_wait_all();
}

}  // namespace lbmk

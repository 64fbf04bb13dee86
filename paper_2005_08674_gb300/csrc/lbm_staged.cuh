// lbm_staged.cuh -- the producer/consumer step kernel shared by the batched
// mode and the single-domain staged mode: bulk tiles of an instance's
// flattened interior staged into shared memory by cp.async.bulk copies that
// complete on mbarriers, NSBC chunks taken from the same work list, and the
// host-side builder of that list.  Every wait is bounded (about a second of
// SM clock); a wait that gives up records a flag and the kernel returns.
#pragma once

#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

#include "lbm_kernels.cuh"

namespace lbmk {

// One instance as the work-list kernels see it.
struct InstDev {
  long long off;    // element offset of the instance's planes in each pool
  long long plane;  // elements per plane
  int nx, ny, pitch;
  int vec_shift;      // divisor pitch / V (16-byte vectors per row) as a
  unsigned vec_mul;   // multiply-and-shift pair, set by set_row_divisor
  int pad;
  double omega;     // 1 / tau
  double m0[3];     // far field (rho, ux, uy)
};

// Division of a flattened vector index by the vectors per row, q = j / nvec,
// as a multiply-high and a shift (Granlund & Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994): with
// l = ceil(log2 nvec) and m = floor(2^32 (2^l - nvec) / nvec) + 1,
// q = (umulhi(m, j) + j) >> l for every 0 <= j < 2^31 (the sum cannot
// overflow since umulhi(m, j) <= j).
inline void set_row_divisor(InstDev& d, int V) {
  const unsigned long long nvec = (unsigned long long)(d.pitch / V);
  int l = 0;
  while ((1ull << l) < nvec) ++l;
  d.vec_shift = l;
  d.vec_mul = (unsigned)((((1ull << l) - nvec) << 32) / nvec + 1);
}

__device__ __forceinline__ int row_of_vector(int j, const InstDev& d) {
  return (int)((__umulhi(d.vec_mul, (unsigned)j) + (unsigned)j) >> d.vec_shift);
}

// ---------------------------------------------------------------------------
// Staging: an instance's flattened interior is ONE contiguous range per plane
// when its pitch is a whole number of 16-byte vectors (shifted by a row for
// the planes pulled from y - 1 / y + 1); a tile plus one vector on each side
// (the x - 1 / x + 1 neighbours) arrives by nine cp.async.bulk copies that
// complete on an mbarrier.
// ---------------------------------------------------------------------------
constexpr long long kTmaWaitCycles = 2000000000LL;  // ~1 s of SM clock before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for phase `parity` of the barrier: false once `budget` SM
// clock cycles have passed without the phase completing.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget = kTmaWaitCycles) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  do {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  } while (clock64() - t0 < budget);
  return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Row shift of the plane each direction is pulled from (Fig. 1 numbering).
__device__ __forceinline__ int pull_row_shift(int i) { return (i == 3 || i == 5 || i == 7) ? -1 : ((i == 4 || i == 6 || i == 8) ? 1 : 0); }

// Issue the nine copies of tile w into slot (9 planes of SLOT bytes each).
template <typename T, int TILE>
__device__ __forceinline__ void issue_tile(const T* __restrict__ A, const InstDev& d, const int4& w, unsigned char* slot,
                                           uint64_t* bar) {
  constexpr int V = lbmk::Store<T>::V;
  constexpr int SLOT = (TILE + 2) * 16;
  const long long plane_elems = (long long)d.ny * d.pitch;
  long long lo[9], hi[9];
  bool ok[9];
  uint32_t total = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const long long start = (long long)(1 + pull_row_shift(i)) * d.pitch + (long long)(w.y - 1) * V;
    lo[i] = start < 0 ? 0 : start;
    const long long end = start + (long long)(w.z + 2) * V;
    hi[i] = end > plane_elems ? plane_elems : end;
    const long long bytes = (hi[i] - lo[i]) * (long long)sizeof(T);
    // (checked build: a copy whose source or slot range fails is not issued
    // and not counted in the barrier's byte total)
    ok[i] = in_bounds(A + d.off + i * d.plane + lo[i], (unsigned long long)bytes) &&
            in_slot((lo[i] - start) * (long long)sizeof(T), bytes, SLOT);
    if (ok[i]) total += (uint32_t)bytes;
  }
  mbar_expect_tx(bar, total);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const long long start = (long long)(1 + pull_row_shift(i)) * d.pitch + (long long)(w.y - 1) * V;
    if (ok[i])
      bulk_copy_g2s(slot + i * SLOT + (lo[i] - start) * (long long)sizeof(T), A + d.off + i * d.plane + lo[i],
                    (uint32_t)((hi[i] - lo[i]) * (long long)sizeof(T)), bar);
  }
}

// Collide the nodes of a staged bulk tile (slot `sl`) and store them to B.
// 16-bit storages are collided in half vectors (4 nodes per thread) so the
// per-thread register footprint matches the f32 path.
template <typename T, int BX, int MODEL, int TILE, bool SHIFT = false>
__device__ __forceinline__ void collide_tile(const unsigned char* sl, const InstDev& d, const int4& w,
                                             T* __restrict__ B, const lbmk::Rates<typename lbmk::Store<T>::C>& r) {
  using S = lbmk::Store<T>;
  using C = typename S::C;
  constexpr int V = S::V;
  constexpr int SLOT = (TILE + 2) * 16;
  constexpr int SPLIT = sizeof(T) == 2 ? 2 : 1;
  constexpr int CPT = V / SPLIT;
  const int nvec = d.pitch / V;  // the batch pitch is a whole number of vectors
  T* b = B + d.off;
#pragma unroll 1
  for (int u2 = threadIdx.x; u2 < w.z * SPLIT; u2 += BX) {
    const int u = u2 / SPLIT, part = u2 - u * SPLIT;
    const int j = w.y + u;
    const int y = 1 + row_of_vector(j, d);
    const int x0 = (j - (y - 1) * nvec) * V + part * CPT;
    // elements (u + 1) V + part CPT - 1 .. + CPT of every plane's slot
    if (!in_slot(((long long)(u + 1) * V + part * CPT - 1) * (long long)sizeof(T), (CPT + 2) * (long long)sizeof(T),
                 SLOT))
      continue;
    C v[9][CPT], lf[9], rt[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const T* e = reinterpret_cast<const T*>(sl + i * SLOT) + (u + 1) * V + part * CPT;
      if constexpr (SPLIT == 1)
        S::lds(e, v[i]);
      else
        S::ldsp(e, v[i]);
      lf[i] = S::ld1s(e - 1);    // x0 - 1 of the same (shifted) row
      rt[i] = S::ld1s(e + CPT);  // x0 + CPT
    }
    C o[9][CPT];
#pragma unroll
    for (int kk = 0; kk < CPT; ++kk) {
      o[0][kk] = v[0][kk];
      o[1][kk] = kk == 0 ? lf[1] : v[1][kk - 1];
      o[2][kk] = kk == CPT - 1 ? rt[2] : v[2][kk + 1];
      o[3][kk] = v[3][kk];
      o[4][kk] = v[4][kk];
      o[5][kk] = kk == 0 ? lf[5] : v[5][kk - 1];
      o[6][kk] = kk == CPT - 1 ? rt[6] : v[6][kk + 1];
      o[7][kk] = kk == CPT - 1 ? rt[7] : v[7][kk + 1];
      o[8][kk] = kk == 0 ? lf[8] : v[8][kk - 1];
    }
    lbmk::collide_nodes<MODEL, SHIFT, false>(o, r, C(S::kScale));
    const long long r0 = (long long)y * d.pitch + x0;
    if (x0 >= 1 && x0 + CPT <= d.nx - 1) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        if constexpr (SPLIT == 1)
          S::st(b + i * d.plane + r0, o[i]);
        else
          S::stp(b + i * d.plane + r0, o[i]);
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < CPT; ++kk) {
        const int x = x0 + kk;
        if (x >= 1 && x <= d.nx - 2) {
#pragma unroll
          for (int i = 0; i < 9; ++i) S::st1r(b + i * d.plane + r0 + kk, o[i][kk]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised form of the same step: the last warp of each block is a
// producer whose lane 0 claims work items from the counter and keeps up to
// STAGES of them in flight (bulk tiles by cp.async.bulk onto the stage's
// `full` barrier, NSBC chunks by a plain arrival); the NC consumer threads
// take the stages in order, work on them (tiles from shared memory, NSBC
// chunks from global memory) and release each stage on its `empty` barrier
// (one arrival per consumer warp).  No block-wide barrier inside the loop;
// every wait is bounded, and on give-up a thread records the flag and leaves.
// ---------------------------------------------------------------------------
template <typename T, int NC, int MODEL, int TILE, int STAGES, int K, bool SHIFT = false>
__global__ void __launch_bounds__(NC + 32, 4) batch_ws_kernel(const T* __restrict__ A, T* __restrict__ B,
                                                           const InstDev* __restrict__ inst,
                                                           const Shift<typename Store<T>::C>* __restrict__ shifts,
                                                           const int4* __restrict__ items, int n_items, lbmk::Nsbc p,
                                                           double s_e, double s_eps, double s_q,
                                                           int* __restrict__ sched) {
  using C = typename lbmk::Store<T>::C;
  constexpr int SLOT = (TILE + 2) * 16;
  constexpr int NCW = NC / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
  __shared__ int4 ring[STAGES];
  __shared__ InstDev rinst[STAGES];  // the item's instance, read once by the producer
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the only block-wide barrier

  if (warp == NCW) {
    // producer
    if (lane == 0) {
      uint32_t ephase = 0u;  // bit s: parity of the next completion of empty[s]
      int s = 0, produced = 0;
      for (;;) {
        const int c = atomicAdd(&sched[0], 1);
        if (produced >= STAGES) {  // stage s was used before: wait until its consumers released it
          if (!mbar_wait(&empty[s], (ephase >> s) & 1u)) {
            atomicExch(&sched[2], 1);
            break;
          }
          ephase ^= 1u << s;
        }
        if (c >= n_items) {
          ring[s] = make_int4(0, 0, 0, -1);  // end of work for this block's consumers
          mbar_arrive(&full[s]);
          break;
        }
        const int4 w = items[c];
        const InstDev d = inst[w.x < 0 ? ~w.x : w.x];
        ring[s] = w;
        rinst[s] = d;
        if (w.x >= 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue_tile<T, TILE>(A, d, w, smem + s * 9 * SLOT, &full[s]);
        } else {
          mbar_arrive(&full[s]);
        }
        s = s + 1 == STAGES ? 0 : s + 1;
        ++produced;
      }
      __threadfence();
      if (atomicAdd(&sched[1], 1) == (int)gridDim.x - 1) {
        sched[0] = 0;
        sched[1] = 0;
      }
    }
    return;
  }

  // consumers
  uint32_t fphase = 0u;  // bit s: parity of the next completion of full[s]
  for (int s = 0;; s = s + 1 == STAGES ? 0 : s + 1) {
    if (!mbar_wait(&full[s], (fphase >> s) & 1u)) {
      atomicExch(&sched[2], 1);
      return;
    }
    fphase ^= 1u << s;
    const int4 w = ring[s];
    if (w.w < 0) break;
    const bool edge = w.x < 0;
    const InstDev d = rinst[s];
    lbmk::Rates<C> r{C(d.omega), C(s_e), C(s_eps), C(s_q), {}};
    if constexpr (SHIFT) r.z = shifts[w.x < 0 ? ~w.x : w.x];  // the instance's storage shift
    if (edge) {
      lbmk::Nsbc q = p;
      q.m0[0] = d.m0[0];
      q.m0[1] = d.m0[1];
      q.m0[2] = d.m0[2];
      const lbmk::Geom g{d.nx, d.ny, d.pitch, d.plane};
      // K nodes per lane quad: node w.y + quad + (NC / 4) k of the chunk
      int node[K];
      bool valid[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int n = (tid >> 2) + (NC / 4) * k;
        valid[k] = n < w.z;
        node[k] = w.y + (valid[k] ? n : 0);
      }
      lbmk::nsbc_nodes<T, MODEL, K, SHIFT>(lbmk::GlobalSrc<T>{A + d.off, g.plane, g.pitch},
                                           lbmk::GlobalDst<T>{B + d.off, g.plane, g.pitch}, g, q, r, node, valid,
                                           tid & 3);
    } else {
      collide_tile<T, NC, MODEL, TILE, SHIFT>(smem + s * 9 * SLOT, d, w, B, r);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// ---------------------------------------------------------------------------
// Host side: the work list of one instance for the staged kernels, in memory
// order -- its bulk tiles (k, first vector, count) of `tile` vectors in row
// order, each NSBC chunk (~k, first perimeter node, count) of `chunk` nodes
// right after the tile that stages the last row the chunk reads (rows
// y - 1 .. y + 2 around its nodes), so that the chunk's scattered loads find
// those rows in L2 and its partial-sector stores meet the tile's there.
// ---------------------------------------------------------------------------
// Row of perimeter node n (bottom row, top row, left column, right column:
// the order perimeter_node walks the perimeter in).
inline int perimeter_row(int n, int nx, int ny) {
  if (n < 2 * nx) return n >= nx ? ny - 1 : 0;
  n -= 2 * nx;
  return 1 + (n >= ny - 2 ? n - (ny - 2) : n);
}

inline void staged_instance_items(int k, const InstDev& d, int V, int tile, int chunk, std::vector<int4>& out) {
  const int nvec = d.pitch / V;
  const int total = (d.ny - 2) * nvec;  // interior rows flattened into 16-byte vectors
  const int perim = 2 * d.nx + 2 * (d.ny - 2);
  std::vector<std::pair<int, int4>> chunks;  // (last row read, chunk)
  for (int n0 = 0; n0 < perim; n0 += chunk) {
    const int cnt = std::min(chunk, perim - n0);
    int last = 0;
    for (int n = n0; n < n0 + cnt; ++n) last = std::max(last, std::min(perimeter_row(n, d.nx, d.ny) + 2, d.ny - 1));
    chunks.push_back({last, make_int4(~k, n0, cnt, 0)});
  }
  std::stable_sort(chunks.begin(), chunks.end(),
                   [](const std::pair<int, int4>& x, const std::pair<int, int4>& y) { return x.first < y.first; });
  size_t c = 0;
  for (int j0 = 0; j0 < total; j0 += tile) {
    const int first_row = 1 + j0 / nvec;
    for (; c < chunks.size() && chunks[c].first < first_row; ++c) out.push_back(chunks[c].second);
    out.push_back(make_int4(k, j0, std::min(tile, total - j0), 0));
  }
  for (; c < chunks.size(); ++c) out.push_back(chunks[c].second);
}

}  // namespace lbmk

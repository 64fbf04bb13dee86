// lbm_batch.cu -- many independent D2Q9 + NSBC simulations of uneven sizes
// advanced by ONE persistent launch per step.
//
// Every instance keeps its own 9-plane layout (pitch = nx rounded up to one
// 16-byte vector, planes 256-byte aligned) inside two shared pools A and B.
// A work list of int4 items drives the launch: NSBC chunks (~instance, first
// perimeter node, count) and bulk tiles (instance, first vector, count) of
// 16-byte vectors of the instance's interior rows flattened end to end (so
// narrow instances leave no lanes idle).  Items of one step read only pool A
// and write disjoint nodes of pool B, so no synchronisation is needed inside
// the launch.  Each item runs the same device code as the single-domain
// kernels (bulk_row, nsbc_node), so an instance's results are bit-identical
// to a single-domain run with the same storage and collision model.
//
// Three forms, chosen by lbm_batch_set_launch or the autotuner:
//   batch_ws_kernel   (default) producer warp + consumer warps: tiles staged
//                     into shared memory by bulk copies, 3-4 stages in flight;
//   batch_tma_kernel  the same staging with the whole block taking turns;
//   batch_step_kernel tiles straight from global memory (register path).
// The staged forms take items from a counter in device memory, in memory
// order with each NSBC chunk after the tile that stages its rows.  Every form
// is compiled plain and with the far-field storage shift (Shift); a batch
// with any instance in a mean flow runs the shifted one, reading each
// instance's shift from a small device table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "lbm.h"
#include "lbm_aux.cuh"
#include "lbm_kernels.cuh"
#include "lbm_staged.cuh"
#include "lbm_trace.h"
#include "lbm_tune_cache.h"
#include "lbm_twostep.cuh"

int lbm_internal_fail(int code, const char* msg);
// the autotuner cache of lbm_runtime.cu (lbm_set_tune_cache)
std::string lbm_internal_tune_path();
std::string lbm_internal_tune_key(const char* kind, int storage, int model, bool shift,
                                  const std::vector<long long>& dims);
void lbm_internal_tune_count(bool hit);
int lbm_internal_set_edges(lbmk::Nsbc* p, const int32_t types[4], const double uw[8]);

namespace {

int bfail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return lbm_internal_fail(code, buf);
}

#define BATCH_CUDA(call)                                                                               \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess)                                                                             \
      return bfail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s (%s:%d)", #call, \
                   cudaGetErrorString(e_), __FILE__, __LINE__);                                        \
  } while (0)

using lbmk::batch_ws_kernel;
using lbmk::collide_tile;
using lbmk::InstDev;
using lbmk::issue_tile;
using lbmk::kTmaWaitCycles;
using lbmk::mbar_arrive;
using lbmk::mbar_expect_tx;
using lbmk::mbar_init;
using lbmk::mbar_wait;
using lbmk::smem_u32;

constexpr int kBatchGraphSteps = 16;
constexpr int kBatchBX[] = {64, 128, 256};
constexpr int kBatchRows[] = {1, 2, 4};

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct lbm_batch {
  int count = 0;
  int storage = LBM_F32;
  size_t elt = 4;
  std::vector<InstDev> inst;
  std::vector<double> tau;
  long long pool_elems = 0;
  long long cells = 0;
  size_t max_cells = 0;
  lbmk::Nsbc nsbc{};
  int collision = 0;
  double s_e = 1.0, s_eps = 1.0, s_q = 1.0;
  void* pool[2] = {nullptr, nullptr};
  void* scratch = nullptr;  // 3 fields of the largest instance (double)
  bool owns_pools = false, bound = false;
  InstDev* d_inst = nullptr;
  void* d_shift = nullptr;  // per-instance storage shifts in the compute type (Shift<C>[count])
  int4* d_items = nullptr;
  int n_items = 0, n_bulk_items = 0;
  // launch shape; the default is the producer/consumer form (128 consumer
  // threads, 3 stages of 128-vector tiles, one NSBC node per lane quad)
  int bx = 128, rows = 3, blocks = 0;  // blocks: -1 one per item, 0 one resident wave, > 0 as given
  int pf = 1;                          // register path: L2 prefetch distance; producer/consumer: nodes per quad
  bool split = false;                   // NSBC chunks in their own concurrent launch
  bool shift = false;                   // some instance has a far field not at rest (Shift)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int wave = 1;                        // resident blocks on the device for the current shape
  int tile = 128;                      // > 0: bulk tiles of this many vectors staged by bulk copies
  int* d_err = nullptr;                // [0] work counter, [1] blocks done, [2] a bounded wait gave up
  // two-step passes (lbm_batch_set_twostep): the rolling kernel's items and
  // grid, the frame launches' items (step n + 1 on the width-3 frames, step
  // n + 2 on the width-2 frames) and the instances' frame buffers
  bool twostep = false, ts_dirty = true;
  int4* d_roll = nullptr;
  int4* d_frame1 = nullptr;
  int4* d_frame2 = nullptr;
  void* d_frame = nullptr;
  int n_roll = 0, n_frame1 = 0, n_frame2 = 0, roll_grid = 0;
  bool items_dirty = true;
  std::vector<char> initialised;
  int cur = 0;
  long long steps = 0;
  cudaStream_t stream = nullptr, cap = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int device = 0;
};

namespace {

template <typename F>
void bdispatch(int storage, F&& f) {
  switch (storage) {
    case LBM_F64: f(double{}); break;
    case LBM_F16: f(__half{}); break;
    case LBM_BF16: f(__nv_bfloat16{}); break;
    default: f(float{}); break;
  }
}

// Whole-tile prefetch of bulk item w of instance d: the tile's vectors span
// one contiguous address range per plane (its rows plus their padding); warp
// `wid` asks the bulk-copy engine for planes wid, wid + BX/32, ... so the
// tile's loads find their lines in L2.
template <typename T, int BX>
__device__ __forceinline__ void prefetch_tile(const T* __restrict__ A, const InstDev& d, const int4& w, int wid) {
  constexpr int V = lbmk::Store<T>::V;
  const int nvec = (d.nx + V - 1) / V;
  const int ja = w.y, jb = w.y + w.z - 1;
  const int ya = 1 + ja / nvec, yb = 1 + jb / nvec;
  const long long a0 = (long long)ya * d.pitch + (long long)(ja - (ya - 1) * nvec) * V;
  const long long a1 = (long long)yb * d.pitch + (long long)(jb - (yb - 1) * nvec + 1) * V;
  const unsigned bytes = (unsigned)((a1 - a0) * (long long)sizeof(T));
  const T* base = A + d.off + a0;
  for (int pl = wid; pl < 9; pl += BX / 32) {
    const long long sh = (pl == 3 || pl == 5 || pl == 7) ? -(long long)d.pitch
                                                       : ((pl == 4 || pl == 6 || pl == 8) ? (long long)d.pitch : 0);
    lbmk::prefetch_l2(base + pl * d.plane + sh, bytes);
  }
}

// PART 0: the whole work list in one launch (NSBC chunks and bulk tiles);
// PART 1: bulk tiles only; PART 2: NSBC chunks only (the split schedule runs
// 1 and 2 as two concurrent launches, so the bulk launch keeps the register
// budget -- and occupancy -- of the single-domain bulk kernel).
template <typename T, int BX, int MODEL, int PART, bool SHIFT = false>
__global__ void __launch_bounds__(BX) batch_step_kernel(const T* __restrict__ A, T* __restrict__ B,
                                                        const InstDev* __restrict__ inst,
                                                        const lbmk::Shift<typename lbmk::Store<T>::C>* __restrict__ shifts,
                                                        const int4* __restrict__ items, int i0, int i1,
                                                        lbmk::Nsbc p, double s_e, double s_eps, double s_q, int pf) {
  using C = typename lbmk::Store<T>::C;
  constexpr int V = lbmk::Store<T>::V;
  const int lane = threadIdx.x & 31;
  for (int it = i0 + blockIdx.x; it < i1; it += gridDim.x) {
    const int4 w = items[it];
    const bool edge = PART == 2 || (PART == 0 && w.x < 0);
    const InstDev d = inst[edge ? ~w.x : w.x];
    const lbmk::Geom g{d.nx, d.ny, d.pitch, d.plane};
    lbmk::Rates<C> r{C(d.omega), C(s_e), C(s_eps), C(s_q), {}};
    if constexpr (SHIFT) r.z = shifts[edge ? ~w.x : w.x];
    const T* a = A + d.off;
    T* b = B + d.off;
    if constexpr (PART != 2) {
      if (!edge) {
        // the instance's interior rows 1..ny-2 flattened into one sequence of
        // 16-byte vectors, nvec per row; this item is vectors [w.y, w.y + w.z)
        const int nvec = (d.nx + V - 1) / V;
        const int warp0 = (int)threadIdx.x - lane;
        if (pf == 1 && lane == 0) prefetch_tile<T, BX>(A, d, w, warp0 / 32);
        if (pf > 1 && lane == 0 && it + pf < i1) {
          // the tile pf items ahead (another block's, started a little later)
          const int4 wn = items[it + pf];
          if (wn.x >= 0) prefetch_tile<T, BX>(A, inst[wn.x], wn, warp0 / 32);
        }
        for (int base = 0; base < w.z; base += BX) {
          const int jr = base + (int)threadIdx.x;
          const bool valid = jr < w.z;
          const int j = w.y + (valid ? jr : 0);
          const int yy = 1 + j / nvec;
          const int x0 = (j - (yy - 1) * nvec) * V;
          lbmk::bulk_row<T, MODEL, SHIFT>(a, b, g, r, yy, x0, lane, 0, 0u, valid);
        }
        continue;
      }
    }
    if constexpr (PART != 1) {
      lbmk::Nsbc q = p;
      q.m0[0] = d.m0[0];
      q.m0[1] = d.m0[1];
      q.m0[2] = d.m0[2];
      const int node = w.y + ((int)threadIdx.x >> 2);
      if (node < w.y + w.z) lbmk::nsbc_node<T, MODEL, SHIFT>(a, b, g, q, r, node, (int)threadIdx.x & 3);
    }
  }
}

// ---------------------------------------------------------------------------
// Bulk tiles through shared memory (bulk-copy engine).  With the batch pitch
// equal to nx rounded up to one 16-byte vector, a tile of vectors [j0, j1) of
// an instance's flattened interior is ONE contiguous range per plane (shifted
// by a row for the planes pulled from y - 1 / y + 1); the tile plus one
// vector on each side (the x - 1 / x + 1 neighbours) arrives by nine
// cp.async.bulk copies completing on an mbarrier.  Two buffers per block: the
// next tile is in flight while the current one is collided, so the bytes in
// flight are bounded by shared memory, not by registers.
// ---------------------------------------------------------------------------
// A wait on a barrier nothing ever arrives on, then a wait on a counter
// nothing ever increments (the two-step pass's wait for its first-frame
// chunks): each must give up after its budget; *flag = 1 if both did (the
// kernel then returns normally), 2 otherwise.
__global__ void wait_selftest_kernel(long long budget, int* flag, const int* counter) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool a = mbar_wait(&bar, 0u, budget);
    const bool b = lbmk::wait_count(counter, 1, budget);
    *flag = (!a && !b) ? 1 : 2;
  }
}

// The whole step of every instance in ONE persistent launch: blocks take
// work items from a shared counter (sched[0]) -- NSBC chunks, computed from
// global memory, and bulk tiles, staged into shared memory by the bulk-copy
// engine.  While a block works on its current item, the copy for the next
// bulk tile it took is already in flight (two slots).  The last block out
// resets the counters for the next step.  sched[2] is set if a bounded wait
// on a copy gave up.
template <typename T, int BX, int MODEL, int TILE, bool SHIFT = false>
__global__ void __launch_bounds__(BX) batch_tma_kernel(const T* __restrict__ A, T* __restrict__ B,
                                                       const InstDev* __restrict__ inst,
                                                       const lbmk::Shift<typename lbmk::Store<T>::C>* __restrict__ shifts,
                                                       const int4* __restrict__ items, int n_items, lbmk::Nsbc p,
                                                       double s_e, double s_eps, double s_q, int* __restrict__ sched) {
  using C = typename lbmk::Store<T>::C;
  constexpr int SLOT = (TILE + 2) * 16;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_cur, s_cur_slot, s_next, s_next_slot, s_ok;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t parity[2] = {0u, 0u};
  int ns = 0;  // thread 0: slot the next copy goes to
  if (tid == 0) {
    const int c = atomicAdd(&sched[0], 1);
    s_cur = c;
    s_cur_slot = -1;
    if (c < n_items) {
      const int4 w = items[c];
      if (w.x >= 0) {
        issue_tile<T, TILE>(A, inst[w.x], w, smem + ns * 9 * SLOT, &bar[ns]);
        s_cur_slot = ns;
        ns ^= 1;
      }
    }
  }
  __syncthreads();
  for (;;) {
    const int cur = s_cur, cslot = s_cur_slot;
    if (cur >= n_items) break;  // uniform: read after a barrier
    __syncthreads();            // everyone has read s_cur / s_cur_slot
    if (tid == 0) {
      const int c = atomicAdd(&sched[0], 1);
      s_next = c;
      s_next_slot = -1;
      if (c < n_items) {
        const int4 wn = items[c];
        if (wn.x >= 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue_tile<T, TILE>(A, inst[wn.x], wn, smem + ns * 9 * SLOT, &bar[ns]);
          s_next_slot = ns;
          ns ^= 1;
        }
      }
    }
    const int4 w = items[cur];
    const bool edge = w.x < 0;
    const InstDev d = inst[edge ? ~w.x : w.x];
    lbmk::Rates<C> r{C(d.omega), C(s_e), C(s_eps), C(s_q), {}};
    if constexpr (SHIFT) r.z = shifts[edge ? ~w.x : w.x];
    if (edge) {
      lbmk::Nsbc q = p;
      q.m0[0] = d.m0[0];
      q.m0[1] = d.m0[1];
      q.m0[2] = d.m0[2];
      const lbmk::Geom g{d.nx, d.ny, d.pitch, d.plane};
      const int node = w.y + (tid >> 2);
      if (node < w.y + w.z) lbmk::nsbc_node<T, MODEL, SHIFT>(A + d.off, B + d.off, g, q, r, node, tid & 3);
    } else {
      // thread 0 waits (bounded) and tells the block, so that the whole block
      // takes the same way out if the copy never lands
      if (tid == 0) s_ok = mbar_wait(&bar[cslot], parity[cslot]) ? 1 : 0;
      __syncthreads();
      if (!s_ok) {
        if (tid == 0) {
          atomicExch(&sched[2], 1);
          mbar_wait(&bar[cslot], parity[cslot]);
          if (s_next_slot >= 0) mbar_wait(&bar[s_next_slot], parity[s_next_slot]);
        }
        break;
      }
      mbar_wait(&bar[cslot], parity[cslot]);  // completes at once; orders this thread after the copy
      parity[cslot] ^= 1u;
      collide_tile<T, BX, MODEL, TILE, SHIFT>(smem + cslot * 9 * SLOT, d, w, B, r);
    }
    __syncthreads();  // done with the current slot; s_next visible
    if (tid == 0) {
      s_cur = s_next;
      s_cur_slot = s_next_slot;
    }
    __syncthreads();
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&sched[1], 1) == (int)gridDim.x - 1) {
      sched[0] = 0;
      sched[1] = 0;
    }
  }
}

// SHIFT: whether any instance has a far field not at rest (its stored
// populations are then deviations from that equilibrium; see Shift).
template <typename F>
void with_shift(bool on, F&& f) {
  if (on)
    f(std::integral_constant<bool, true>{});
  else
    f(std::integral_constant<bool, false>{});
}

template <typename T, int BX, int MODEL, int TILE>
void launch_tma(const lbm_batch_t* b, int from, cudaStream_t s, int grid) {
  // the dynamic shared-memory limit was raised by wave_blocks() when the work
  // list was built (never inside a stream capture)
  constexpr int smem = 2 * 9 * (TILE + 2) * 16;
  with_shift(b->shift, [&](auto zc) {
    batch_tma_kernel<T, BX, MODEL, TILE, decltype(zc)::value><<<grid, BX, smem, s>>>(
        static_cast<const T*>(b->pool[from]), static_cast<T*>(b->pool[1 - from]), b->d_inst,
        static_cast<const lbmk::Shift<typename lbmk::Store<T>::C>*>(b->d_shift), b->d_items, b->n_items,
        b->nsbc, b->s_e, b->s_eps, b->s_q, b->d_err);
  });
}

template <typename T, int NC, int MODEL, int TILE, int STAGES, int K>
void launch_ws(const lbm_batch_t* b, int from, cudaStream_t s, int grid) {
  constexpr int smem = STAGES * 9 * (TILE + 2) * 16;  // limit raised by wave_blocks()
  with_shift(b->shift, [&](auto zc) {
    batch_ws_kernel<T, NC, MODEL, TILE, STAGES, K, decltype(zc)::value><<<grid, NC + 32, smem, s>>>(
        static_cast<const T*>(b->pool[from]), static_cast<T*>(b->pool[1 - from]), b->d_inst,
        static_cast<const lbmk::Shift<typename lbmk::Store<T>::C>*>(b->d_shift), b->d_items, b->n_items,
        b->nsbc, b->s_e, b->s_eps, b->s_q, b->d_err);
  });
}

template <typename T, int BX, int PART>
const void* kernel_ptr(int model, bool shift) {
  if (shift)
    return model == 1 ? (const void*)batch_step_kernel<T, BX, 1, PART, true>
                      : (const void*)batch_step_kernel<T, BX, 0, PART, true>;
  return model == 1 ? (const void*)batch_step_kernel<T, BX, 1, PART> : (const void*)batch_step_kernel<T, BX, 0, PART>;
}

template <typename T, int BX, int PART>
void launch_part(const lbm_batch_t* b, int from, cudaStream_t s, int grid, int i0, int i1) {
  const T* A = static_cast<const T*>(b->pool[from]);
  T* B = static_cast<T*>(b->pool[1 - from]);
  const auto* zs = static_cast<const lbmk::Shift<typename lbmk::Store<T>::C>*>(b->d_shift);
  with_shift(b->shift, [&](auto zc) {
    constexpr bool Z = decltype(zc)::value;
    if (b->collision == 1)
      batch_step_kernel<T, BX, 1, PART, Z><<<grid, BX, 0, s>>>(A, B, b->d_inst, zs, b->d_items, i0, i1, b->nsbc, b->s_e,
                                                              b->s_eps, b->s_q, b->pf);
    else
      batch_step_kernel<T, BX, 0, PART, Z><<<grid, BX, 0, s>>>(A, B, b->d_inst, zs, b->d_items, i0, i1, b->nsbc, b->s_e,
                                                              b->s_eps, b->s_q, b->pf);
  });
}

template <typename F>
void with_bx(int bx, F&& f) {
  switch (bx) {
    case 64: f(std::integral_constant<int, 64>{}); break;
    case 256: f(std::integral_constant<int, 256>{}); break;
    default: f(std::integral_constant<int, 128>{}); break;
  }
}

// (threads, tile) pairs compiled for the shared-memory bulk path
template <typename F>
void with_tma(int bx, int tile, F&& f) {
  if (bx == 256)
    f(std::integral_constant<int, 256>{}, std::integral_constant<int, 256>{});
  else if (tile == 256)
    f(std::integral_constant<int, 128>{}, std::integral_constant<int, 256>{});
  else
    f(std::integral_constant<int, 128>{}, std::integral_constant<int, 128>{});
}

bool tma_shape_ok(int bx, int tile) {
  return (bx == 128 && (tile == 128 || tile == 256)) || (bx == 256 && tile == 256);
}

// Shapes compiled for the producer/consumer path (128 consumer threads,
// tiles of 128 vectors): 3 or 4 stages, 1 or 2 perimeter nodes per lane quad
// (the `prefetch_rows` field carries the latter; 0 means 1).
int ws_nodes_per_quad(int pf) { return pf == 2 ? 2 : 1; }

template <typename F>
void with_ws(int stages, int pf, F&& f) {
  const int k = ws_nodes_per_quad(pf);
  auto pick_k = [&](auto sc) {
    if (k == 2)
      f(sc, std::integral_constant<int, 2>{});
    else
      f(sc, std::integral_constant<int, 1>{});
  };
  if (stages >= 4)
    pick_k(std::integral_constant<int, 4>{});
  else
    pick_k(std::integral_constant<int, 3>{});
}

// resident blocks on the device for the launch that carries the bulk tiles
int wave_blocks(const lbm_batch_t* b) {
  int per_sm = 0, sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  bdispatch(b->storage, [&](auto tag) {
    using T = decltype(tag);
    if (b->tile > 0 && b->rows >= 3) {
      with_ws(b->rows, b->pf, [&](auto sc, auto kc) {
        constexpr int STAGES = decltype(sc)::value, K = decltype(kc)::value;
        constexpr int smem = STAGES * 9 * (128 + 2) * 16;
        const void* k = b->shift ? (b->collision == 1 ? (const void*)batch_ws_kernel<T, 128, 1, 128, STAGES, K, true>
                                                      : (const void*)batch_ws_kernel<T, 128, 0, 128, STAGES, K, true>)
                                 : (b->collision == 1 ? (const void*)batch_ws_kernel<T, 128, 1, 128, STAGES, K>
                                                      : (const void*)batch_ws_kernel<T, 128, 0, 128, STAGES, K>);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128 + 32, smem);
      });
      return;
    }
    if (b->tile > 0) {
      with_tma(b->bx, b->tile, [&](auto bxc, auto tc) {
        constexpr int BX = decltype(bxc)::value, TILE = decltype(tc)::value;
        constexpr int smem = 2 * 9 * (TILE + 2) * 16;
        const void* k = b->shift ? (b->collision == 1 ? (const void*)batch_tma_kernel<T, BX, 1, TILE, true>
                                                      : (const void*)batch_tma_kernel<T, BX, 0, TILE, true>)
                                 : (b->collision == 1 ? (const void*)batch_tma_kernel<T, BX, 1, TILE>
                                                      : (const void*)batch_tma_kernel<T, BX, 0, TILE>);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BX, smem);
      });
      return;
    }
    with_bx(b->bx, [&](auto bxc) {
      constexpr int BX = decltype(bxc)::value;
      const void* k =
          b->split ? kernel_ptr<T, BX, 1>(b->collision, b->shift) : kernel_ptr<T, BX, 0>(b->collision, b->shift);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BX, 0);
    });
  });
  return std::max(1, per_sm) * std::max(1, sms);
}

int grid_for_items(const lbm_batch_t* b, int n) {
  // blocks < 0: one block per work item; 0: one resident wave; > 0: as given
  return std::max(1, b->blocks < 0 ? n : std::min(n, b->blocks > 0 ? b->blocks : b->wave));
}

// One step from pool `from`.  Fused: one launch over the whole list.  Split:
// the NSBC chunks on the side stream beside the bulk tiles (fork/join events,
// captured as two parallel graph nodes).
void enqueue_batch_step(const lbm_batch_t* b, int from, cudaStream_t s) {
  bdispatch(b->storage, [&](auto tag) {
    using T = decltype(tag);
    if (b->tile > 0 && b->rows >= 3) {
      // one persistent launch, producer warp + consumer warps
      with_ws(b->rows, b->pf, [&](auto sc, auto kc) {
        constexpr int STAGES = decltype(sc)::value, K = decltype(kc)::value;
        const int grid = std::max(1, std::min(b->n_items, b->blocks > 0 ? b->blocks : b->wave));
        if (b->collision == 1)
          launch_ws<T, 128, 1, 128, STAGES, K>(b, from, s, grid);
        else
          launch_ws<T, 128, 0, 128, STAGES, K>(b, from, s, grid);
      });
      return;
    }
    if (b->tile > 0) {
      // the whole step in one persistent launch (NSBC chunks and staged tiles)
      with_tma(b->bx, b->tile, [&](auto bxc, auto tc) {
        constexpr int BX = decltype(bxc)::value, TILE = decltype(tc)::value;
        const int grid = std::max(1, std::min(b->n_items, b->blocks > 0 ? b->blocks : b->wave));
        if (b->collision == 1)
          launch_tma<T, BX, 1, TILE>(b, from, s, grid);
        else
          launch_tma<T, BX, 0, TILE>(b, from, s, grid);
      });
      return;
    }
    with_bx(b->bx, [&](auto bxc) {
      constexpr int BX = decltype(bxc)::value;
      if (!b->split) {
        launch_part<T, BX, 0>(b, from, s, grid_for_items(b, b->n_items), 0, b->n_items);
      } else {
        const int n_edge = b->n_items - b->n_bulk_items;
        cudaEventRecord(b->ev_fork, s);
        cudaStreamWaitEvent(b->side, b->ev_fork, 0);
        launch_part<T, BX, 2>(b, from, b->side, std::max(1, n_edge), 0, n_edge);
        launch_part<T, BX, 1>(b, from, s, grid_for_items(b, b->n_bulk_items), n_edge, b->n_items);
        cudaEventRecord(b->ev_join, b->side);
        cudaStreamWaitEvent(s, b->ev_join, 0);
      }
    });
  });
}

void drop_batch_graphs(lbm_batch_t* b) {
  for (auto& g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// Work list for the current shape.  Register path: NSBC chunks first
// (latency-bound; they start early and overlap with the bandwidth-bound
// tiles), then bulk tiles, largest instances first.  Staged-tile paths: one
// interleaved list (below).
int build_items(lbm_batch_t* b) {
  if (!b->items_dirty) return LBM_OK;
  const int V = (int)(16 / b->elt);
  std::vector<int> order(b->count);
  for (int k = 0; k < b->count; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) {
    return (long long)b->inst[i].nx * b->inst[i].ny > (long long)b->inst[j].nx * b->inst[j].ny;
  });
  std::vector<int4> items;
  // NSBC chunk: one node per quad of lanes (K per quad in the
  // producer/consumer form)
  const int chunk = b->bx / 4 * (b->tile > 0 && b->rows >= 3 ? ws_nodes_per_quad(b->pf) : 1);
  for (int k : order) {
    const InstDev& d = b->inst[k];
    const int perim = 2 * d.nx + 2 * (d.ny - 2);
    for (int n0 = 0; n0 < perim; n0 += chunk) items.push_back(make_int4(~k, n0, std::min(chunk, perim - n0), 0));
  }
  const int n_edge = (int)items.size();
  for (int k : order) {
    const InstDev& d = b->inst[k];
    const int nvec = (d.nx + V - 1) / V;
    const int total = (d.ny - 2) * nvec;  // interior rows flattened into 16-byte vectors
    const int per_item = b->tile > 0 ? b->tile : b->bx * b->rows;
    for (int j0 = 0; j0 < total; j0 += per_item) items.push_back(make_int4(k, j0, std::min(per_item, total - j0), 0));
  }
  const int n_bulk = (int)items.size() - n_edge;
  if (b->tile > 0) {
    // one dynamically scheduled list in memory order: instance after instance
    // (largest first), each as lbmk::staged_instance_items lays it out.
    // (Spreading the NSBC chunks evenly over the whole list instead, or each
    // instance's items over the whole step, costs 10-15 % in step time.)
    items.clear();
    for (int k : order) lbmk::staged_instance_items(k, b->inst[k], V, b->tile, chunk, items);
  }
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  BATCH_CUDA(cudaMalloc(&b->d_items, items.size() * sizeof(int4)));
  BATCH_CUDA(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
  b->n_items = (int)items.size();
  b->n_bulk_items = n_bulk;
  b->wave = wave_blocks(b);
  b->items_dirty = false;
  drop_batch_graphs(b);
  return LBM_OK;
}

// The two-step pass serves the batch: 16- or 32-bit storage, no periodic
// axis, every instance 8 x 8 nodes or more.
bool batch_twostep_ok(const lbm_batch_t* b) {
  if (b->storage == LBM_F64 || b->nsbc.periodic_x || b->nsbc.periodic_y) return false;
  for (const InstDev& d : b->inst)
    if (d.nx < 8 || d.ny < 8) return false;
  return true;
}

// Work lists of the two-step pass, largest instance first: rolling items in
// bands of at most 64 output rows, all strips of a band side by side;
// frame items of 128 threads; each instance's frame buffer after the last.
int build_twostep(lbm_batch_t* b) {
  if (!b->ts_dirty) return LBM_OK;
  const int out = b->storage == LBM_F32 ? lbmk::Roll<float>::OUT : lbmk::Roll<__half>::OUT;
  std::vector<int> order(b->count);
  for (int k = 0; k < b->count; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) {
    return (long long)b->inst[i].nx * b->inst[i].ny > (long long)b->inst[j].nx * b->inst[j].ny;
  });
  std::vector<int4> roll, f1, f2;
  long long foff = 0;
  for (int k : order) {
    const InstDev& d = b->inst[k];
    const int strips = (d.nx - 4 + out - 1) / out, iy = d.ny - 4;
    // bands of at most 64 rows: more, smaller items balance the warps better
    // (measured on the 256-instance batch, band caps 128 / 64 / 32 / 16:
    // f32 115k / 123k / 124k / 122k MLUPS, f16 144k / 149k / 149k / 144k)
    const int nb = (iy + 63) / 64, band = (iy + nb - 1) / nb;
    for (int y = 2; y < d.ny - 2; y += band)
      for (int j = 0; j < strips; ++j) roll.push_back(make_int4(k, j * out, y, std::min(y + band, d.ny - 2)));
    if (foff > INT32_MAX - 9LL * lbmk::ring_offset(d.nx, d.ny, lbmk::kFrameWidth))
      return bfail(LBM_EINVAL, "lbm_batch: frame buffers beyond 2^31 elements");
    for (int t0 = 0; t0 < lbmk::frame_threads(d.nx, d.ny, lbmk::kFrameWidth); t0 += 128)
      f1.push_back(make_int4(k, t0, (int)foff, 0));
    for (int t0 = 0; t0 < lbmk::frame_threads(d.nx, d.ny, 2); t0 += 128) f2.push_back(make_int4(k, t0, (int)foff, 0));
    foff += 9LL * lbmk::ring_offset(d.nx, d.ny, lbmk::kFrameWidth);
  }
  for (int4** p : {&b->d_roll, &b->d_frame1, &b->d_frame2}) {
    cudaFree(*p);
    *p = nullptr;
  }
  cudaFree(b->d_frame);
  b->d_frame = nullptr;
  BATCH_CUDA(cudaMalloc(&b->d_frame, (size_t)foff * b->elt));
  BATCH_CUDA(cudaMalloc(&b->d_roll, roll.size() * sizeof(int4)));
  BATCH_CUDA(cudaMalloc(&b->d_frame1, f1.size() * sizeof(int4)));
  BATCH_CUDA(cudaMalloc(&b->d_frame2, f2.size() * sizeof(int4)));
  BATCH_CUDA(cudaMemcpy(b->d_roll, roll.data(), roll.size() * sizeof(int4), cudaMemcpyHostToDevice));
  BATCH_CUDA(cudaMemcpy(b->d_frame1, f1.data(), f1.size() * sizeof(int4), cudaMemcpyHostToDevice));
  BATCH_CUDA(cudaMemcpy(b->d_frame2, f2.data(), f2.size() * sizeof(int4), cudaMemcpyHostToDevice));
  b->n_roll = (int)roll.size();
  b->n_frame1 = (int)f1.size();
  b->n_frame2 = (int)f2.size();
  // the rolling kernel's shared memory, and one resident wave of its blocks
  int per_sm = 0, sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  bdispatch(b->storage, [&](auto tag) {
    using T = decltype(tag);
    if constexpr (!std::is_same<T, double>::value) {
      const int smem = (int)lbmk::Roll<T>::kSmem;
      for (const void* k :
           {(const void*)lbmk::roll_batch_kernel<T, 0, false>, (const void*)lbmk::roll_batch_kernel<T, 0, true>,
            (const void*)lbmk::roll_batch_kernel<T, 1, false>, (const void*)lbmk::roll_batch_kernel<T, 1, true>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbmk::roll_batch_kernel<T, 1, true>,
                                                          lbmk::kRollThreads, smem);
    }
  });
  if (e != cudaSuccess) return bfail(LBM_ECUDA, "lbm_batch: two-step kernel setup: %s", cudaGetErrorString(e));
  if (per_sm <= 0) return bfail(LBM_ECUDA, "lbm_batch: no two-step block fits on an SM");
  const int warps = lbmk::Roll<float>::WARPS;
  b->roll_grid = std::max(1, std::min(per_sm * sms, (b->n_roll + warps - 1) / warps));
  b->ts_dirty = false;
  return LBM_OK;
}

// Two steps from pool `from` to 1 - from: three launches.
void enqueue_batch_twostep(const lbm_batch_t* b, int from, cudaStream_t s) {
  bdispatch(b->storage, [&](auto tag) {
    using T = decltype(tag);
    if constexpr (!std::is_same<T, double>::value) {
      using C = typename lbmk::Store<T>::C;
      const T* A = static_cast<const T*>(b->pool[from]);
      T* B = static_cast<T*>(b->pool[1 - from]);
      T* F = static_cast<T*>(b->d_frame);
      const auto* zs = static_cast<const lbmk::Shift<C>*>(b->d_shift);
      with_shift(b->shift, [&](auto zc) {
        constexpr bool Z = decltype(zc)::value;
        // the frame launches on the side stream, beside the rolling kernel
        // (whose warps claim items, so blocks that start late take fewer)
        cudaStream_t fs = b->side ? b->side : s;
        auto go = [&](auto mc) {
          constexpr int M = decltype(mc)::value;
          if (fs != s) {
            cudaEventRecord(b->ev_fork, s);
            cudaStreamWaitEvent(fs, b->ev_fork, 0);
          }
          lbmk::frame_batch_kernel<T, M, Z, true><<<b->n_frame1, 128, 0, fs>>>(A, B, F, b->d_inst, zs, b->d_frame1,
                                                                               b->nsbc, b->s_e, b->s_eps, b->s_q);
          lbmk::roll_batch_kernel<T, M, Z><<<b->roll_grid, lbmk::kRollThreads, lbmk::Roll<T>::kSmem, s>>>(
              A, B, b->d_inst, zs, b->d_roll, b->n_roll, b->s_e, b->s_eps, b->s_q, b->d_err);
          lbmk::frame_batch_kernel<T, M, Z, false><<<b->n_frame2, 128, 0, fs>>>(A, B, F, b->d_inst, zs, b->d_frame2,
                                                                                b->nsbc, b->s_e, b->s_eps, b->s_q);
          if (fs != s) {
            cudaEventRecord(b->ev_join, fs);
            cudaStreamWaitEvent(s, b->ev_join, 0);
          }
        };
        if (b->collision == 1)
          go(std::integral_constant<int, 1>{});
        else
          go(std::integral_constant<int, 0>{});
      });
    }
  });
}

int ensure_batch_memory(lbm_batch_t* b) {
  if (!b->bound) {
    const size_t pb = lbm_batch_buffer_bytes(b);
    BATCH_CUDA(cudaGetDevice(&b->device));
    BATCH_CUDA(cudaMalloc(&b->pool[0], pb));
    BATCH_CUDA(cudaMalloc(&b->pool[1], pb));
    BATCH_CUDA(cudaMalloc(&b->scratch, lbm_batch_scratch_bytes(b)));
    BATCH_CUDA(cudaMemset(b->pool[0], 0, pb));
    BATCH_CUDA(cudaMemset(b->pool[1], 0, pb));
    lbmk::check_add(b->pool[0], pb);  // bounds-checked build only
    lbmk::check_add(b->pool[1], pb);
    b->owns_pools = true;
    b->bound = true;
  }
  if (!b->d_err) {
    BATCH_CUDA(cudaMalloc(&b->d_err, 4 * sizeof(int)));  // work counter, blocks done, error flag
    BATCH_CUDA(cudaMemset(b->d_err, 0, 4 * sizeof(int)));
  }
  if (!b->d_inst) {
    BATCH_CUDA(cudaMalloc(&b->d_inst, b->inst.size() * sizeof(InstDev)));
    BATCH_CUDA(cudaMemcpy(b->d_inst, b->inst.data(), b->inst.size() * sizeof(InstDev), cudaMemcpyHostToDevice));
  }
  if (!b->d_shift) {
    // each instance's storage shift, rounded once on the host to the compute type
    int rc = LBM_OK;
    bdispatch(b->storage, [&](auto tag) {
      using C = typename lbmk::Store<decltype(tag)>::C;
      std::vector<lbmk::Shift<C>> z(b->inst.size());
      for (size_t k = 0; k < z.size(); ++k) z[k] = lbmk::shift_as<C>(lbmk::far_field_shift(b->inst[k].m0));
      if (cudaMalloc(&b->d_shift, z.size() * sizeof(lbmk::Shift<C>)) != cudaSuccess ||
          cudaMemcpy(b->d_shift, z.data(), z.size() * sizeof(lbmk::Shift<C>), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = LBM_ECUDA;
    });
    if (rc) return bfail(rc, "lbm_batch: shift table: %s", cudaGetErrorString(cudaGetLastError()));
  }
  return LBM_OK;
}

int ensure_batch_streams(lbm_batch_t* b) {
  if (!b->cap) {
    BATCH_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    BATCH_CUDA(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    BATCH_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    BATCH_CUDA(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
  }
  return LBM_OK;
}

int batch_check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(LBM_ECUDA, "batched kernel launch failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbmk::Geom inst_geom(const InstDev& d) { return lbmk::Geom{d.nx, d.ny, d.pitch, d.plane}; }

double* bscratch(lbm_batch_t* b, int c) {
  return reinterpret_cast<double*>(static_cast<char*>(b->scratch) + c * round_up(b->max_cells * sizeof(double), 256));
}

bool batch_shape_ok(int bx, int rows) {
  bool a = false, r = false;
  for (int v : kBatchBX) a |= v == bx;
  for (int v : kBatchRows) r |= v == rows;
  return a && r;
}

}  // namespace

extern "C" {

lbm_batch_t* lbm_batch_create(int32_t count, const lbm_instance_desc* descs, int32_t storage) {
  if (count < 1 || !descs) {
    bfail(LBM_EINVAL, "lbm_batch_create: need count >= 1 and descriptors");
    return nullptr;
  }
  if (storage < LBM_F64 || storage > LBM_BF16) {
    bfail(LBM_EINVAL, "lbm_batch_create: unknown storage %d", storage);
    return nullptr;
  }
  lbm_batch_t* b = new lbm_batch_t();
  b->count = count;
  b->storage = storage;
  b->elt = storage == LBM_F64 ? 8 : (storage == LBM_F32 ? 4 : 2);
  b->nsbc.gamma = 0.6;
  b->nsbc.beta = 0.0;
  b->nsbc.kappa = 3.0;
  b->nsbc.order = 1;
  b->nsbc.corner = 0;
  long long off = 0;
  for (int k = 0; k < count; ++k) {
    const lbm_instance_desc& s = descs[k];
    if (s.nx < 3 || s.ny < 3 || s.nx > 65536 || s.ny > 65536 || !std::isfinite(s.tau) || !(s.tau > 0.5) ||
        !(s.farfield_rho > 0.0) || !std::isfinite(s.farfield_ux) || !std::isfinite(s.farfield_uy)) {
      bfail(LBM_EINVAL, "lbm_batch_create: instance %d invalid (nx=%d ny=%d tau=%g)", k, s.nx, s.ny, s.tau);
      delete b;
      return nullptr;
    }
    InstDev d{};
    d.nx = s.nx;
    d.ny = s.ny;
    // one 16-byte vector of alignment: consecutive rows of a plane then form
    // one contiguous run of vectors, so a tile is one copy per plane
    d.pitch = (int)round_up((size_t)s.nx, 16 / b->elt);
    d.plane = (long long)(round_up((size_t)s.ny * d.pitch * b->elt, 256) / b->elt);
    lbmk::set_row_divisor(d, (int)(16 / b->elt));
    d.off = off;
    d.omega = 1.0 / s.tau;
    d.m0[0] = s.farfield_rho;
    d.m0[1] = s.farfield_ux;
    d.m0[2] = s.farfield_uy;
    b->shift = b->shift || lbmk::far_field_shift(d.m0).on;
    off += 9 * d.plane;
    b->inst.push_back(d);
    b->tau.push_back(s.tau);
    b->cells += (long long)s.nx * s.ny;
    b->max_cells = std::max(b->max_cells, (size_t)s.nx * s.ny);
  }
  b->pool_elems = off;
  b->initialised.assign(count, 0);
  return b;
}

void lbm_batch_destroy(lbm_batch_t* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_batch_graphs(b);
  if (b->bound) {
    lbmk::check_remove(b->pool[0]);
    lbmk::check_remove(b->pool[1]);
  }
  if (b->owns_pools) {
    cudaFree(b->pool[0]);
    cudaFree(b->pool[1]);
    cudaFree(b->scratch);
  }
  cudaFree(b->d_inst);
  cudaFree(b->d_shift);
  cudaFree(b->d_items);
  cudaFree(b->d_err);
  cudaFree(b->d_roll);
  cudaFree(b->d_frame1);
  cudaFree(b->d_frame2);
  cudaFree(b->d_frame);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  delete b;
}

int64_t lbm_batch_cells(const lbm_batch_t* b) { return b ? b->cells : -1; }

int lbm_batch_get_dims(const lbm_batch_t* b, int32_t k, int32_t* nx, int32_t* ny) {
  if (!b || !nx || !ny) return bfail(LBM_EINVAL, "lbm_batch_get_dims: NULL argument");
  if (k < 0 || k >= b->count) return bfail(LBM_EINVAL, "lbm_batch_get_dims: instance %d out of range", k);
  *nx = b->inst[k].nx;
  *ny = b->inst[k].ny;
  return LBM_OK;
}

size_t lbm_batch_buffer_bytes(const lbm_batch_t* b) { return b ? (size_t)b->pool_elems * b->elt : 0; }

size_t lbm_batch_scratch_bytes(const lbm_batch_t* b) {
  return b ? 3 * round_up(b->max_cells * sizeof(double), 256) + round_up((1024 * 4 + 4) * sizeof(double), 256) : 0;
}

int lbm_batch_bind(lbm_batch_t* b, void* dev_a, void* dev_b, void* dev_scratch) {
  if (!b || !dev_a || !dev_b || !dev_scratch) return bfail(LBM_EINVAL, "lbm_batch_bind: NULL argument");
  if (b->bound) return bfail(LBM_ESTATE, "lbm_batch_bind: memory already bound or allocated");
  for (void* p : {dev_a, dev_b, dev_scratch})
    if (reinterpret_cast<uintptr_t>(p) % 256) return bfail(LBM_EINVAL, "lbm_batch_bind: pointers must be 256-byte aligned");
  BATCH_CUDA(cudaGetDevice(&b->device));
  b->pool[0] = dev_a;
  b->pool[1] = dev_b;
  b->scratch = dev_scratch;
  lbmk::check_add(dev_a, lbm_batch_buffer_bytes(b));  // bounds-checked build only
  lbmk::check_add(dev_b, lbm_batch_buffer_bytes(b));
  b->bound = true;
  return LBM_OK;
}

namespace lbmk {
// This unit's share of lbm_check_read (its kernels have their own table).
void batch_check_read(unsigned long long* count, unsigned long long* first, bool reset) {
  check_read(count, first, reset);
}
}  // namespace lbmk

int lbm_batch_set_nsbc(lbm_batch_t* b, double gamma, double beta, double kappa, int32_t corner_mode,
                       int32_t grad_order) {
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_set_nsbc: NULL handle");
  if (!std::isfinite(gamma) || !std::isfinite(beta) || !std::isfinite(kappa) || (grad_order != 1 && grad_order != 2) ||
      (corner_mode != LBM_CORNER_DIAGONAL && corner_mode != LBM_CORNER_MEAN))
    return bfail(LBM_EINVAL,
                 "lbm_batch_set_nsbc: need finite gamma, beta, kappa, corner_mode 0 or 1 and grad_order 1 or 2");
  b->nsbc.gamma = gamma;
  b->nsbc.beta = beta;
  b->nsbc.kappa = kappa;
  b->nsbc.order = grad_order;
  b->nsbc.corner = corner_mode;
  drop_batch_graphs(b);
  return LBM_OK;
}

int lbm_batch_set_edges(lbm_batch_t* b, const int32_t types[4], const double uw[8]) {
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_set_edges: NULL handle");
  lbmk::Nsbc p = b->nsbc;
  int rc = lbm_internal_set_edges(&p, types, uw);
  if (rc) return rc;
  b->nsbc = p;
  drop_batch_graphs(b);
  return LBM_OK;
}

int lbm_batch_set_collision(lbm_batch_t* b, int32_t model, double omega_e, double omega_eps, double omega_q) {
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_set_collision: NULL handle");
  if (model != LBM_BGK && model != LBM_MRT) return bfail(LBM_EINVAL, "lbm_batch_set_collision: unknown model %d", model);
  if (model == LBM_MRT)
    for (double r : {omega_e, omega_eps, omega_q})
      if (!std::isfinite(r) || !(r > 0.0) || !(r < 2.0))
        return bfail(LBM_EINVAL, "lbm_batch_set_collision: MRT rates must lie in (0, 2)");
  b->collision = model;
  b->items_dirty = true;  // the kernel's occupancy (one wave of blocks) depends on the model
  if (model == LBM_MRT) {
    b->s_e = omega_e;
    b->s_eps = omega_eps;
    b->s_q = omega_q;
  }
  drop_batch_graphs(b);
  return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch_t* b, void* cuda_stream) {
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_set_stream: NULL handle");
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  return LBM_OK;
}

int lbm_batch_init(lbm_batch_t* b, int32_t k, const double* rho, const double* ux, const double* uy) {
  if (!b || !rho || !ux || !uy) return bfail(LBM_EINVAL, "lbm_batch_init: NULL argument");
  if (k < 0 || k >= b->count) return bfail(LBM_EINVAL, "lbm_batch_init: instance %d out of range", k);
  int rc = ensure_batch_memory(b);
  if (rc) return rc;
  const InstDev& d = b->inst[k];
  const size_t bytes = (size_t)d.nx * d.ny * sizeof(double);
  const double* src[3] = {rho, ux, uy};
  for (int c = 0; c < 3; ++c)
    BATCH_CUDA(cudaMemcpyAsync(bscratch(b, c), src[c], bytes, cudaMemcpyHostToDevice, b->stream));
  bdispatch(b->storage, [&](auto tag) {
    using T = decltype(tag);
    lbmk::init_kernel<T><<<lbmk::rows_grid(d.pitch, d.ny), 256, 0, b->stream>>>(
        static_cast<T*>(b->pool[0]) + d.off, static_cast<T*>(b->pool[1]) + d.off, inst_geom(d),
        lbmk::far_field_shift(d.m0),
        bscratch(b, 0), bscratch(b, 1), bscratch(b, 2), 0, d.ny);
  });
  rc = batch_check_launch();
  if (rc) return rc;
  BATCH_CUDA(cudaStreamSynchronize(b->stream));
  if (b->steps != 0 || b->cur != 0) {
    // a fresh start for the whole batch: step counts are per batch
    b->steps = 0;
  }
  b->initialised[k] = 1;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch_t* b, int32_t n) {
  LBM_TRACE("lbm_batch_step");
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_step: NULL handle");
  if (n < 0) return bfail(LBM_EINVAL, "lbm_batch_step: n=%d < 0", n);
  for (int k = 0; k < b->count; ++k)
    if (!b->initialised[k]) return bfail(LBM_ESTATE, "lbm_batch_step: instance %d not initialised", k);
  int rc = build_items(b);
  if (rc) return rc;
  rc = ensure_batch_streams(b);
  if (rc) return rc;
  const bool two = b->twostep && batch_twostep_ok(b);
  if (two) {
    rc = build_twostep(b);
    if (rc) return rc;
  }
  int left = n;
  if (left >= kBatchGraphSteps) {
    if (!b->graph[b->cur]) {
      cudaGraph_t g = nullptr;
      BATCH_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
      if (two)  // kBatchGraphSteps / 2 passes: an even number of pool swaps
        for (int s = 0; s < kBatchGraphSteps / 2; ++s) enqueue_batch_twostep(b, (b->cur + s) & 1, b->cap);
      else
        for (int s = 0; s < kBatchGraphSteps; ++s) enqueue_batch_step(b, (b->cur + s) & 1, b->cap);
      cudaError_t e = cudaStreamEndCapture(b->cap, &g);
      if (e != cudaSuccess) return bfail(LBM_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->graph[b->cur], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return bfail(LBM_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
    }
    while (left >= kBatchGraphSteps) {
      BATCH_CUDA(cudaGraphLaunch(b->graph[b->cur], b->stream));
      left -= kBatchGraphSteps;
    }
  }
  for (; two && left >= 2; left -= 2) {
    enqueue_batch_twostep(b, b->cur, b->stream);
    b->cur ^= 1;
  }
  for (; left > 0; --left) {
    enqueue_batch_step(b, b->cur, b->stream);
    b->cur ^= 1;
  }
  rc = batch_check_launch();
  if (rc) return rc;
  b->steps += n;
  return LBM_OK;
}

int lbm_batch_get_macros(lbm_batch_t* b, int32_t k, double* rho, double* ux, double* uy) {
  if (!b || !rho || !ux || !uy) return bfail(LBM_EINVAL, "lbm_batch_get_macros: NULL argument");
  if (k < 0 || k >= b->count) return bfail(LBM_EINVAL, "lbm_batch_get_macros: instance %d out of range", k);
  if (!b->initialised[k]) return bfail(LBM_ESTATE, "lbm_batch_get_macros: instance %d not initialised", k);
  const InstDev& d = b->inst[k];
  const long long n = (long long)d.nx * d.ny;
  bdispatch(b->storage, [&](auto tag) {
    using T = decltype(tag);
    lbmk::macros_kernel<T><<<lbmk::rows_grid(d.nx, d.ny), 256, 0, b->stream>>>(
        static_cast<const T*>(b->pool[b->cur]) + d.off, inst_geom(d),
        lbmk::shift_as<typename lbmk::Store<T>::C>(lbmk::far_field_shift(d.m0)), bscratch(b, 0), bscratch(b, 1),
        bscratch(b, 2), 0, d.ny);
  });
  int rc = batch_check_launch();
  if (rc) return rc;
  double* dst[3] = {rho, ux, uy};
  for (int c = 0; c < 3; ++c)
    BATCH_CUDA(cudaMemcpyAsync(dst[c], bscratch(b, c), n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

int lbm_batch_unstable_nodes(lbm_batch_t* b, int32_t k, int64_t* count) {
  if (!b || !count) return bfail(LBM_EINVAL, "lbm_batch_unstable_nodes: NULL argument");
  if (k < 0 || k >= b->count) return bfail(LBM_EINVAL, "lbm_batch_unstable_nodes: instance %d out of range", k);
  if (!b->initialised[k]) return bfail(LBM_ESTATE, "lbm_batch_unstable_nodes: instance %d not initialised", k);
  const InstDev& d = b->inst[k];
  const long long n = (long long)d.nx * d.ny;
  const int blocks = (int)std::min<long long>(1024, (n + 255) / 256);
  double* partials = bscratch(b, 3);  // after the three field slots
  double* out = partials + 1024 * 4;
  lbmk::RefField ref{nullptr, nullptr, nullptr, 0};
  bdispatch(b->storage, [&](auto tag) {
    using T = decltype(tag);
    lbmk::reduce_kernel<T, 256><<<blocks, 256, 0, b->stream>>>(
        static_cast<const T*>(b->pool[b->cur]) + d.off, inst_geom(d),
        lbmk::shift_as<typename lbmk::Store<T>::C>(lbmk::far_field_shift(d.m0)),
        ref, d.m0[0], d.m0[1], d.m0[2], partials);
  });
  lbmk::reduce_finish<256><<<1, 256, 0, b->stream>>>(partials, blocks, out);
  int rc = batch_check_launch();
  if (rc) return rc;
  double h[4];
  BATCH_CUDA(cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(cudaStreamSynchronize(b->stream));
  *count = (int64_t)h[3];
  return LBM_OK;
}

int lbm_batch_set_launch(lbm_batch_t* b, int32_t threads_x, int32_t rows, int32_t blocks, int32_t prefetch_rows,
                         int32_t split, int32_t tma_tile) {
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_set_launch: NULL handle");
  if (tma_tile != 0 && !tma_shape_ok(threads_x, tma_tile))
    return bfail(LBM_EINVAL, "lbm_batch_set_launch: staged tiles need (threads, tile) = (128, 128), (128, 256) or "
                             "(256, 256), got (%d, %d)", threads_x, tma_tile);
  const bool ws = tma_tile != 0 && rows >= 3;
  if (ws && (threads_x != 128 || tma_tile != 128 || rows > 4))
    return bfail(LBM_EINVAL, "lbm_batch_set_launch: the producer/consumer path takes (threads, tile) = (128, 128) "
                             "and 3 or 4 stages, got (%d, %d, %d)", threads_x, tma_tile, rows);
  if (ws && prefetch_rows != 0 && prefetch_rows != 1 && prefetch_rows != 2)
    return bfail(LBM_EINVAL, "lbm_batch_set_launch: the producer/consumer path takes 1 or 2 perimeter nodes per "
                             "lane quad, got %d", prefetch_rows);
  if (tma_tile == 0 && !batch_shape_ok(threads_x, rows))
    return bfail(LBM_EINVAL, "lbm_batch_set_launch: shape (%d, %d) not compiled", threads_x, rows);
  if (blocks < -1) return bfail(LBM_EINVAL, "lbm_batch_set_launch: blocks=%d < -1", blocks);
  if (prefetch_rows < 0 || prefetch_rows > 65536)
    return bfail(LBM_EINVAL, "lbm_batch_set_launch: prefetch=%d outside [0, 65536]", prefetch_rows);
  b->bx = threads_x;
  b->rows = tma_tile ? (ws ? rows : 1) : rows;
  b->blocks = blocks;
  b->pf = prefetch_rows;
  b->split = tma_tile == 0 && split != 0;
  b->tile = tma_tile;
  b->twostep = false;
  b->items_dirty = true;
  drop_batch_graphs(b);
  return LBM_OK;
}

int lbm_batch_set_twostep(lbm_batch_t* b, int32_t enable) {
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_set_twostep: NULL handle");
  if (enable && !batch_twostep_ok(b))
    return bfail(LBM_EINVAL, "lbm_batch_set_twostep: needs f32, f16 or bf16 storage, no periodic axis and every "
                             "instance 8 x 8 nodes or more");
  b->twostep = enable != 0;
  drop_batch_graphs(b);
  return LBM_OK;
}

int32_t lbm_batch_get_twostep(const lbm_batch_t* b) { return b ? (b->twostep ? 1 : 0) : LBM_EINVAL; }

int lbm_batch_autotune(lbm_batch_t* b, int32_t* threads_x, int32_t* rows, int32_t* blocks, int32_t* prefetch_rows,
                       int32_t* split, int32_t* tma_tile, double* ms_per_step) {
  LBM_TRACE("lbm_batch_autotune");
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_autotune: NULL handle");
  for (int k = 0; k < b->count; ++k)
    if (!b->initialised[k]) return bfail(LBM_ESTATE, "lbm_batch_autotune: instance %d not initialised", k);
  int rcs = ensure_batch_streams(b);
  if (rcs) return rcs;
  // a choice recorded for the same key is applied without timing
  const std::string tune_path = lbm_internal_tune_path();
  std::string tune_key;
  if (!tune_path.empty()) {
    tune_key = lbm_internal_tune_key("batch", b->storage, b->collision, b->shift, {b->count, b->cells});
    lbmtune::Entry e;
    double v[7];
    const char* names[7] = {"threads_x", "rows", "blocks", "prefetch_rows", "split", "tma_tile", "ms_per_step"};
    bool ok = lbmtune::lookup(tune_path, tune_key, &e);
    for (int k = 0; ok && k < 7; ++k) ok = e.get(names[k], &v[k]);
    double ts = 0.0;
    ok = ok && e.get("twostep", &ts);
    if (ok && lbm_batch_set_launch(b, (int32_t)v[0], (int32_t)v[1], (int32_t)v[2], (int32_t)v[3], (int32_t)v[4],
                                   (int32_t)v[5]) == LBM_OK &&
        (ts == 0.0 || lbm_batch_set_twostep(b, 1) == LBM_OK)) {
      lbm_internal_tune_count(true);
      if (threads_x) *threads_x = b->bx;
      if (rows) *rows = b->rows;
      if (blocks) *blocks = b->blocks;
      if (prefetch_rows) *prefetch_rows = b->pf;
      if (split) *split = b->split ? 1 : 0;
      if (tma_tile) *tma_tile = b->tile;
      if (ms_per_step) *ms_per_step = v[6];
      return LBM_OK;
    }
  }
  // keep the state: current pool copied aside and restored
  const size_t pb = lbm_batch_buffer_bytes(b);
  void* backup = nullptr;
  BATCH_CUDA(cudaMallocAsync(&backup, pb, b->stream));
  BATCH_CUDA(cudaMemcpyAsync(backup, b->pool[b->cur], pb, cudaMemcpyDeviceToDevice, b->stream));
  cudaEvent_t e0, e1;
  BATCH_CUDA(cudaEventCreate(&e0));
  BATCH_CUDA(cudaEventCreate(&e1));
  const int reps = (int)std::max<long long>(4, std::min<long long>(32, (1LL << 28) / std::max(b->cells, 1LL)));
  float best = 1e30f;
  int bb = b->bx, br = b->rows, bk = b->blocks, bp = b->pf, bt = b->tile;
  bool bs = b->split, bts = false;
  b->twostep = false;
  int rc = LBM_OK;
  auto time_it = [&]() -> float {
    for (int s = 0; s < 2; ++s) enqueue_batch_step(b, s & 1, b->stream);
    cudaEventRecord(e0, b->stream);
    for (int s = 0; s < reps; ++s) enqueue_batch_step(b, s & 1, b->stream);
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
  };
  auto keep = [&](float ms) {
    if (ms < best) {
      best = ms;
      bts = false;
      bb = b->bx;
      br = b->rows;
      bk = b->blocks;
      bp = b->pf;
      bs = b->split;
      bt = b->tile;
    }
  };
  // register path: fused or split, tile shape, grid, prefetch
  for (int sp : {0, 1})
    for (int bx : kBatchBX)
      for (int r : kBatchRows) {
        b->bx = bx;
        b->rows = r;
        b->split = sp != 0;
        b->tile = 0;
        b->items_dirty = true;
        rc = build_items(b);
        if (rc) break;
        for (int mult : {-1, 1, 2})  // -1: one block per item; k: k resident waves, persistent
          for (int pf : {0, 1, 256}) {  // 1: own tile at start; k > 1: the tile k items ahead
            b->blocks = mult < 0 ? -1 : b->wave * mult;
            b->pf = pf;
            keep(time_it());
          }
      }
  // shared-memory path: tiles staged by bulk copies, persistent blocks
  const int tma_pairs[3][2] = {{128, 128}, {128, 256}, {256, 256}};
  for (const auto& tp : tma_pairs) {
    if (rc) break;
    b->bx = tp[0];
    b->rows = 1;
    b->tile = tp[1];
    b->split = false;
    b->blocks = 0;
    b->pf = 0;
    b->items_dirty = true;
    rc = build_items(b);
    if (rc) break;
    keep(time_it());
  }
  // producer/consumer path: one issuing warp, 3 or 4 tile stages, 1 or 2
  // perimeter nodes per lane quad
  for (int st : {3, 4})
    for (int kq : {1, 2}) {
      if (rc) break;
      b->bx = 128;
      b->rows = st;
      b->tile = 128;
      b->split = false;
      b->blocks = 0;
      b->pf = kq;
      b->items_dirty = true;
      rc = build_items(b);
      if (rc) break;
      keep(time_it());
    }
  // two-step passes (their odd steps, if any, take the best single step)
  if (!rc && batch_twostep_ok(b)) {
    rc = build_twostep(b);
    if (!rc) {
      for (int s = 0; s < 2; ++s) enqueue_batch_twostep(b, s & 1, b->stream);
      cudaEventRecord(e0, b->stream);
      const int passes = std::max(2, reps / 2);
      for (int s = 0; s < passes; ++s) enqueue_batch_twostep(b, s & 1, b->stream);
      cudaEventRecord(e1, b->stream);
      float ms = 1e30f;
      if (cudaEventSynchronize(e1) == cudaSuccess) {
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 2.0f * passes;
      }
      if (ms < best) {
        best = ms;
        bts = true;
      }
    }
  }
  if (!rc) rc = batch_check_launch();
  b->bx = bb;
  b->rows = br;
  b->blocks = bk;
  b->pf = bp;
  b->split = bs;
  b->tile = bt;
  b->twostep = bts;
  b->items_dirty = true;
  drop_batch_graphs(b);
  int rc2 = build_items(b);
  BATCH_CUDA(cudaMemcpyAsync(b->pool[b->cur], backup, pb, cudaMemcpyDeviceToDevice, b->stream));
  BATCH_CUDA(cudaFreeAsync(backup, b->stream));
  BATCH_CUDA(cudaStreamSynchronize(b->stream));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (rc2) return rc2;
  if (!tune_path.empty()) {
    lbm_internal_tune_count(false);
    lbmtune::Entry e{tune_key,
                     {{"threads_x", bb}, {"rows", br}, {"blocks", bk}, {"prefetch_rows", bp}, {"split", bs ? 1 : 0},
                      {"tma_tile", bt}, {"twostep", bts ? 1 : 0}, {"ms_per_step", best}}};
    lbmtune::store(tune_path, e);  // a cache that cannot be written is only not reused
  }
  if (threads_x) *threads_x = bb;
  if (rows) *rows = br;
  if (blocks) *blocks = bk;
  if (prefetch_rows) *prefetch_rows = bp;
  if (split) *split = bs ? 1 : 0;
  if (tma_tile) *tma_tile = bt;
  if (ms_per_step) *ms_per_step = best;
  return LBM_OK;
}

int lbm_partition_instances(int32_t count, const int64_t* cells, int32_t ranks, int32_t* rank_of) {
  if (count < 0 || ranks < 1 || (count > 0 && (!cells || !rank_of)))
    return bfail(LBM_EINVAL, "lbm_partition_instances: need count >= 0, ranks >= 1 and non-NULL arrays");
  for (int k = 0; k < count; ++k)
    if (cells[k] < 0) return bfail(LBM_EINVAL, "lbm_partition_instances: instance %d has %lld nodes", k,
                                   (long long)cells[k]);
  // largest first, each to the rank with the fewest nodes so far (ties: the
  // lower index, the lower rank), so every rank computes the same partition
  std::vector<int> order(count);
  for (int k = 0; k < count; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cells[a] > cells[c]; });
  std::vector<long long> load(ranks, 0);
  for (int k : order) {
    int r = 0;
    for (int q = 1; q < ranks; ++q)
      if (load[q] < load[r]) r = q;
    rank_of[k] = r;
    load[r] += cells[k];
  }
  return LBM_OK;
}

int lbm_wait_selftest(int64_t budget_cycles) {
  if (budget_cycles <= 0 || budget_cycles > 4000000000LL)
    return bfail(LBM_EINVAL, "lbm_wait_selftest: budget %lld outside (0, 4e9] cycles", (long long)budget_cycles);
  int* d = nullptr;  // [0] the flag, [1] a counter that stays 0
  BATCH_CUDA(cudaMalloc(&d, 2 * sizeof(int)));
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof(int));
  int h = 0;
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 32>>>(budget_cycles, d, d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, "lbm_wait_selftest: %s", cudaGetErrorString(e));
  if (h == 1) return bfail(LBM_ETIMEOUT, "lbm_wait_selftest: the bounded wait gave up as it should");
  return LBM_OK;
}

int lbm_batch_status(lbm_batch_t* b) {
  if (!b) return bfail(LBM_EINVAL, "lbm_batch_status: NULL handle");
  if (!b->d_err) return LBM_OK;
  int h = 0;
  BATCH_CUDA(cudaMemcpyAsync(&h, b->d_err + 2, sizeof h, cudaMemcpyDeviceToHost, b->stream));
  BATCH_CUDA(cudaStreamSynchronize(b->stream));
  if (h) return bfail(LBM_ETIMEOUT, "lbm_batch_status: a staged-tile copy did not complete within its wait limit");
  return LBM_OK;
}

int64_t lbm_batch_steps_done(const lbm_batch_t* b) { return b ? b->steps : -1; }

}  // extern "C"

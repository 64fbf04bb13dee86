// lbm_twostep.cuh -- two time steps per pass over one domain (temporal
// blocking), in one launch whose warps claim three kinds of work from a
// counter, in this order, and together give the bits of two single steps:
//
//   first-frame chunks (A -> F): step n + 1 on the frame of nodes whose
//       distance to the nearest edge is below 3 -- the NSBC (Sec. 5) on the
//       perimeter, the interior collision on rings 1 and 2 -- into a compact
//       frame buffer F (a few MB);
//   rolling items (A -> B): steps n + 1 and n + 2 on the nodes at distance
//       2 or more.  The warp owns a strip of 32 x 4 columns and rolls down a
//       band of rows: it stages the state rows by bulk copies in a private
//       ring of three or four rows in shared memory, computes step n + 1 of
//       each row (the interior collision only: every node it needs there is
//       at distance 1 or more) and keeps the populations that step n + 2
//       pulls from it in registers, rounded to the storage type as a single
//       step stores them.  The intermediate step never reaches device memory;
//   second-frame chunks (F -> B): step n + 2 on the nodes at distance 0 and
//       1, from the frame buffer, each after a bounded wait until every
//       first-frame chunk is done.
//
// Device-memory traffic per two steps: one read and one write of the state
// (the strips' overlapping columns and the bands' four overlapping rows are
// read again, mostly from L2) plus the frame buffer.
//
// The batched form (many instances) runs the same three kinds of work as
// three launches instead -- the frames' thousands of NSBC quads are latency-
// bound and want more resident warps than the rolling kernel leaves; in one
// launch the 256-instance batch ran 20 % slower.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_staged.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
// The frame of width w: nodes with d = min(x, y, nx-1-x, ny-1-y) < w.  Ring d
// is the perimeter of the (nx - 2d) x (ny - 2d) domain at offset (d, d),
// walked in perimeter_node's order; ring_offset(d) nodes lie in rings below d.
// ---------------------------------------------------------------------------
__host__ __device__ inline int ring_offset(int nx, int ny, int d) {
  return d * (2 * nx + 2 * ny - 4) - 4 * d * (d - 1);
}
// Step n + 2 on rings 0 and 1 reads step n + 1 on rings 0..2: the NSBC pulls
// at its node (rings 0, 1) and reads the nodes b - n and b - 2n (rings 1, 2;
// the corners' diagonal b - 2n is (2, 2) from the corner), ring 1's interior
// collision pulls from rings 0..2.
constexpr int kFrameWidth = 3;

// Element of frame node (x, y) (distance below kFrameWidth = w) in a plane
// of the frame buffer: rows 0 .. w-1 (nx each), rows ny-w .. ny-1, then per
// middle row y = w .. ny-w-1 its columns 0 .. w-1 and nx-w .. nx-1; the
// plane holds ring_offset(nx, ny, w) = 2 w (nx + ny - 2 w) elements.
__device__ __forceinline__ int frame_index(int x, int y, int nx, int ny) {
  constexpr int w = kFrameWidth;
  if (y < w) return y * nx + x;
  if (y >= ny - w) return (y - ny + 2 * w) * nx + x;
  return 2 * w * nx + (y - w) * 2 * w + (x < w ? x : x - nx + 2 * w);
}

// Population i of frame node (x, y) in the frame buffer f (planes of fn
// elements): ld / st in physical units like GlobalSrc / GlobalDst, raw /
// st_raw in stored units like the interior kernels.
template <typename T>
struct FrameSrc {
  const T* __restrict__ f;
  int nx, ny, fn;
  __device__ __forceinline__ typename Store<T>::C raw(int i, int x, int y) const {
    // through L2: other warps of the same launch wrote it
    const T v = __ldcg(f + (long long)i * fn + frame_index(x, y, nx, ny));
    return Store<T>::ld1s(&v);
  }
  __device__ __forceinline__ typename Store<T>::C ld(int i, int x, int y) const {
    using S = Store<T>;
    using C = typename S::C;
    if constexpr (S::kScale == 1)
      return raw(i, x, y);
    else
      return raw(i, x, y) * C(1.0 / S::kScale);
  }
};
template <typename T>
struct FrameDst {
  T* __restrict__ f;
  int nx, ny, fn;
  __device__ __forceinline__ void st(int i, int x, int y, typename Store<T>::C v) const {
    f[(long long)i * fn + frame_index(x, y, nx, ny)] = Store<T>::cvt(v);
  }
  __device__ __forceinline__ void st_raw(int i, int x, int y, typename Store<T>::C v) const {
    f[(long long)i * fn + frame_index(x, y, nx, ny)] = T(v);  // round to nearest even, as the vector stores
  }
};
// the same calls on a population buffer in device memory
template <typename T>
struct GlobalRawSrc {
  const T* __restrict__ a;
  long long plane;
  int pitch;
  __device__ __forceinline__ typename Store<T>::C raw(int i, int x, int y) const {
    return Store<T>::ld1(a + i * plane + (long long)y * pitch + x);
  }
  __device__ __forceinline__ typename Store<T>::C ld(int i, int x, int y) const {
    return Store<T>::ldg1(a + i * plane + (long long)y * pitch + x);
  }
};
template <typename T>
struct GlobalRawDst {
  T* __restrict__ b;
  long long plane;
  int pitch;
  __device__ __forceinline__ void st(int i, int x, int y, typename Store<T>::C v) const {
    Store<T>::st1(b + i * plane + (long long)y * pitch + x, v);
  }
  __device__ __forceinline__ void st_raw(int i, int x, int y, typename Store<T>::C v) const {
    Store<T>::st1r(b + i * plane + (long long)y * pitch + x, v);
  }
};

// Thread t's share of one step on the frame of width `width`: threads
// 0 .. 4 P - 1 (P perimeter nodes) run the NSBC quads (a quad's four lanes
// are consecutive threads of one warp), the next ones one interior node of
// rings 1 .. width - 1 each, pulled and collided in stored units like the
// interior kernels.
template <typename T, int MODEL, bool SHIFT, typename Src, typename Dst>
__device__ __forceinline__ void frame_node(const Src& src, const Dst& dst, const Geom& g, const Nsbc& p,
                                           const Rates<typename Store<T>::C>& r, int width, int t) {
  using S = Store<T>;
  using C = typename S::C;
  const int perim = ring_offset(g.nx, g.ny, 1);
  if (t < 4 * perim) {  // 4 P is a multiple of 4: a quad stays together
    const int node[1] = {t >> 2};
    const bool ok[1] = {true};
    nsbc_nodes<T, MODEL, 1, SHIFT>(src, dst, g, p, r, node, ok, t & 3);
    return;
  }
  int k = t - 4 * perim;
  if (k >= ring_offset(g.nx, g.ny, width) - perim) return;
  int d = 1;
  while (k >= ring_offset(g.nx, g.ny, d + 1) - ring_offset(g.nx, g.ny, d)) {
    k -= ring_offset(g.nx, g.ny, d + 1) - ring_offset(g.nx, g.ny, d);
    ++d;
  }
  int x, y, nxn, nyn;
  perimeter_node(k, g.nx - 2 * d, g.ny - 2 * d, x, y, nxn, nyn);
  x += d;
  y += d;
  C h[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) h[i] = src.raw(i, x - cx(i), y - cy(i));
  collide<MODEL, SHIFT>(h, r, C(S::kScale));
#pragma unroll
  for (int i = 0; i < 9; ++i) dst.st_raw(i, x, y, h[i]);
}

// Threads on the frame of width `width`: 4 per perimeter node, 1 per node of
// rings 1 .. width - 1.
__host__ __device__ inline int frame_threads(int nx, int ny, int width) {
  return 3 * ring_offset(nx, ny, 1) + ring_offset(nx, ny, width);
}

// ---------------------------------------------------------------------------
// The rolling interior kernel.
// ---------------------------------------------------------------------------
template <typename T>
struct Roll {
  static constexpr int W = 32 * 4;  // state columns of a strip, four per lane
  // output columns of a strip: step n + 1 is valid on columns 1 .. W - 2 of
  // the strip, step n + 2 on 2 .. W - 3; strips start OUT apart, a multiple
  // of 16 bytes for the copies
  static constexpr int OUT = sizeof(T) == 4 ? W - 4 : W - 8;
  // ring rows: three read while the fourth is in flight (f32 then fits
  // three blocks per SM, 16-bit storage four)
  static constexpr int DEPTH = 4;
  static constexpr int BLOCKS = sizeof(T) == 4 ? 3 : 4;  // resident blocks per SM
  static constexpr int ROWE = 9 * W;
  static constexpr int WARPS = 4;  // independent warps per block
  // paired FP32 collisions for 16-bit storage, whose kernel is bound by
  // instruction issue; f32 has no registers to spare for them
  static constexpr bool PAIRED = sizeof(T) == 2;
  static constexpr size_t kSmem = (size_t)WARPS * DEPTH * ROWE * sizeof(T);
};
constexpr int kRollThreads = 32 * 4;

// this lane's four values of one population at columns 4 lane .. 4 lane + 3
// of a staged row, in stored units
template <typename T>
__device__ __forceinline__ void roll_lds(const T* p, typename Store<T>::C (&o)[4]) {
  if constexpr (sizeof(T) == 4)
    Store<T>::lds(p, o);
  else
    Store<T>::ldsp(p, o);
}

// v[k] := the value at column 4 lane + k - c (c = c_ix), i.e. what node k
// pulls along x; the strip's outermost columns get a value that no valid
// node uses
template <typename C>
__device__ __forceinline__ void shift_x(int c, C (&v)[4]) {
  if (c > 0) {
    const C l = __shfl_up_sync(0xffffffffu, v[3], 1);
    v[3] = v[2];
    v[2] = v[1];
    v[1] = v[0];
    v[0] = l;
  } else if (c < 0) {
    const C rgt = __shfl_down_sync(0xffffffffu, v[0], 1);
    v[0] = v[1];
    v[1] = v[2];
    v[2] = v[3];
    v[3] = rgt;
  }
}

// Lanes 0..8 copy population `lane` of state row s (columns X0 .. X0 + W,
// clipped to the pitch) into ring row `dst`, completing on `bar`.
// (Checked build: a copy whose range fails is neither issued nor counted.)
template <typename T>
__device__ __forceinline__ void roll_stage(const T* __restrict__ A, const Geom& g, int X0, int s, T* dst,
                                           uint64_t* bar, int lane) {
  using R = Roll<T>;
  const int hi = min(X0 + R::W, g.pitch);
  const uint32_t bytes = (uint32_t)(hi - X0) * (uint32_t)sizeof(T);
  const T* src = A + lane * g.plane + (long long)s * g.pitch + X0;
  const bool ok = lane < 9 && in_bounds(src, bytes) &&
                  in_slot((long long)lane * R::W * (long long)sizeof(T), bytes, (long long)R::ROWE * sizeof(T));
  const uint32_t total = __reduce_add_sync(0xffffffffu, ok ? bytes : 0u);
  if (lane == 0) mbar_expect_tx(bar, total);
  __syncwarp();
  if (ok) bulk_copy_g2s(dst + lane * R::W, src, bytes, bar);
}

// One work item of the rolling kernel: steps n + 1 and n + 2 of output rows
// [Ya, Yb) x columns X0 + 2 .. X0 + 2 + OUT (clipped to [2, nx - 2)) of the
// domain g, rolling down state rows Ya - 2 .. Yb + 1 through this warp's
// ring (rows `ring`, barriers `bar`, their parities in `phase`).  All lanes
// of the warp call it.  false: a wait gave up (err[2] is set).
template <typename T, int MODEL, bool SHIFT>
__device__ __forceinline__ bool roll_item(const T* __restrict__ A, T* __restrict__ B, const Geom& g,
                                          const Rates<typename Store<T>::C>& r, int X0, int Ya, int Yb, T* ring,
                                          uint64_t* bar, uint32_t& phase, int lane, int* __restrict__ err) {
  using R = Roll<T>;
  using S = Store<T>;
  using C = typename S::C;
  const int s0 = Ya - 2, s1 = Yb + 1;  // state rows read: s0 .. s1
  __syncwarp();                        // the previous item's reads of the ring are done
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  for (int s = s0; s <= min(s0 + R::DEPTH - 1, s1); ++s)
    roll_stage<T>(A, g, X0, s, ring + (s - s0) * R::ROWE, &bar[s - s0], lane);
  // step n + 1 populations carried from row to row, already pulled along x:
  // ip = row q - 1's c_y = +1 ones, i0 / ip2 = row q's c_y = 0 / +1 ones
  C ip[3][4], i0[3][4], ip2[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < 4; ++k) ip[a][k] = i0[a][k] = ip2[a][k] = C(0);
  for (int s = s0, slot = 0; s <= s1; ++s, slot = slot + 1 == R::DEPTH ? 0 : slot + 1) {
    {
      const bool done = mbar_wait(&bar[slot], (phase >> slot) & 1u);
      if (!__all_sync(0xffffffffu, done)) {
        if (lane == 0) atomicExch(&err[2], 1);
        return false;
      }
      phase ^= 1u << slot;
    }
    if (s < s0 + 2) continue;
    // step n + 1 of row s - 1 from state rows s - 2, s - 1, s
    const int slot_m1 = slot == 0 ? R::DEPTH - 1 : slot - 1;
    const int slot_m2 = slot_m1 == 0 ? R::DEPTH - 1 : slot_m1 - 1;
    C h[9][4];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int row = cy(i) > 0 ? slot_m2 : (cy(i) == 0 ? slot_m1 : slot);
      roll_lds<T>(ring + row * R::ROWE + i * R::W + 4 * lane, h[i]);
      shift_x(cx(i), h[i]);
    }
    collide_nodes<MODEL, SHIFT, R::PAIRED>(h, r, C(S::kScale));
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) h[i][k] = C(T(h[i][k]));  // rounded as a single step stores it
    // row s - 2 is read: stage row s + DEPTH - 2 in its place
    __syncwarp();
    if (s + R::DEPTH - 2 <= s1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      roll_stage<T>(A, g, X0, s + R::DEPTH - 2, ring + slot_m2 * R::ROWE, &bar[slot_m2], lane);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) shift_x(cx(i), h[i]);
    // step n + 2 of row q = s - 2 (rows Ya .. Yb - 1) from step n + 1 rows q - 1, q, q + 1
    const int q = s - 2;
    if (q >= Ya) {
      C o[9][4];
#pragma unroll
      for (int i = 0, a = 0, b = 0; i < 9; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) o[i][k] = cy(i) > 0 ? ip[a][k] : (cy(i) == 0 ? i0[b][k] : h[i][k]);
        a += cy(i) > 0;
        b += cy(i) == 0;
      }
      collide_nodes<MODEL, SHIFT, R::PAIRED>(o, r, C(S::kScale));
      const int x0 = X0 + 4 * lane;
      const int lo = max(max(2, X0 + 2), x0), hi = min(min(g.nx - 2, X0 + 2 + R::OUT), x0 + 4);
      T* row = B + (long long)q * g.pitch + x0;
      if (lo == x0 && hi == x0 + 4) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          if constexpr (sizeof(T) == 4)
            S::st(row + i * g.plane, o[i]);
          else
            S::stp(row + i * g.plane, o[i]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (x0 + k >= lo && x0 + k < hi) {
#pragma unroll
            for (int i = 0; i < 9; ++i) S::st1r(row + i * g.plane + k, o[i][k]);
          }
      }
    }
    // carry: row s - 1 is the next q's row q
#pragma unroll
    for (int i = 0, a = 0, b = 0; i < 9; ++i) {
      if (cy(i) > 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          ip[a][k] = ip2[a][k];
          ip2[a][k] = h[i][k];
        }
      } else if (cy(i) == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) i0[b][k] = h[i][k];
      }
      a += cy(i) > 0;
      b += cy(i) == 0;
    }
  }
  return true;
}

// Bounded wait until the counter *c reaches `want` (acquire: what the
// producers wrote before their release increments is visible after it);
// false once `budget` SM clock cycles have passed.
__device__ __forceinline__ bool wait_count(const int* c, int want, long long budget = kTmaWaitCycles) {
  const long long t0 = clock64();
  do {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    if (v >= want) return true;
    __nanosleep(100);
  } while (clock64() - t0 < budget);
  return false;
}

// Frame work of one warp: 32 consecutive frame threads of frame_node (a
// multiple of 32 from the first, so quads stay whole).  FIRST: step n + 1 on
// the width-3 frame into F, then a release increment of *done; else step
// n + 2 on the width-2 frame from F.
template <typename T, int MODEL, bool SHIFT, bool FIRST>
__device__ __forceinline__ void frame_chunk(const T* __restrict__ A, T* __restrict__ B, T* __restrict__ F,
                                            const Geom& g, const Nsbc& p, const Rates<typename Store<T>::C>& r,
                                            int t0, int lane, int* done) {
  const int fn = ring_offset(g.nx, g.ny, kFrameWidth);
  if constexpr (FIRST) {
    frame_node<T, MODEL, SHIFT>(GlobalRawSrc<T>{A, g.plane, g.pitch}, FrameDst<T>{F, g.nx, g.ny, fn}, g, p, r,
                                kFrameWidth, t0 + lane);
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(done, 1);
  } else {
    frame_node<T, MODEL, SHIFT>(FrameSrc<T>{F, g.nx, g.ny, fn}, GlobalRawDst<T>{B, g.plane, g.pitch}, g, p, r, 2,
                                t0 + lane);
  }
}

// The whole pass in one launch, A (step n) -> B (step n + 2), F the frame
// buffer.  Warps claim work from a counter (sched[0]) in this order: n_f1
// chunks of step n + 1 on the width-3 frame; the rolling items; n_f3 chunks
// of step n + 2 on the width-2 frame, each of which first waits (bounded)
// until all n_f1 first chunks are done (sched[3]).  Every claimed first chunk
// belongs to a running warp that waits on nothing, so the wait always ends.
// Rolling item j = (strip, band): strip X0 = strip OUT reads columns X0 ..
// X0 + W and stores X0 + 2 .. X0 + 2 + OUT; band b stores rows 2 + b band ..
// + band; items come as all strips of a band side by side, the bands in
// waves (wave k: bands k, k + n_waves, ...), so that the lines neighbouring
// strips share and the rows a band restarts on are read from L2.  The last
// warp out resets the counters.  A wait that gives up sets sched[2] and the
// warp returns.
template <typename T, int MODEL, bool SHIFT>
__global__ void __launch_bounds__(kRollThreads, Roll<T>::BLOCKS)
    pass_kernel(const T* __restrict__ A, T* __restrict__ B, T* __restrict__ F, Geom g, Nsbc p,
                Rates<typename Store<T>::C> r, int n_strips, int band, int n_bands, int bands_per_wave, int n_waves,
                int n_f1, int n_f3, int* __restrict__ sched) {
  using R = Roll<T>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[R::WARPS][R::DEPTH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* ring = reinterpret_cast<T*>(smem_raw) + warp * R::DEPTH * R::ROWE;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < R::DEPTH; ++j) mbar_init(&bar[j], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t phase = 0u;  // bit j: parity of the next completion of bar[j]
  const int per_wave = bands_per_wave * n_strips, n_roll = n_waves * per_wave;
  const int n_items = n_f1 + n_roll + n_f3;
  for (;;) {
    int c = 0;
    if (lane == 0) c = atomicAdd(&sched[0], 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= n_items) break;
    if (c < n_f1) {
      frame_chunk<T, MODEL, SHIFT, true>(A, B, F, g, p, r, c * 32, lane, &sched[3]);
    } else if (c < n_f1 + n_roll) {
      const int item = c - n_f1;
      const int wave = item / per_wave, rem = item - wave * per_wave;
      const int m = rem / n_strips, strip = rem - m * n_strips;
      const int b = m * n_waves + wave;
      if (b >= n_bands) continue;
      const int Ya = 2 + b * band, Yb = min(Ya + band, g.ny - 2);
      if (!roll_item<T, MODEL, SHIFT>(A, B, g, r, strip * R::OUT, Ya, Yb, ring, bar, phase, lane, sched)) return;
    } else {
      bool ok = true;
      if (lane == 0) ok = wait_count(&sched[3], n_f1);
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        if (lane == 0) atomicExch(&sched[2], 1);
        return;
      }
      __syncwarp();
      frame_chunk<T, MODEL, SHIFT, false>(A, B, F, g, p, r, (c - n_f1 - n_roll) * 32, lane, nullptr);
    }
  }
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(&sched[1], 1) == (int)gridDim.x * R::WARPS - 1) {
      sched[0] = 0;
      sched[3] = 0;
      __threadfence();
      sched[1] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// The same pass over many independent instances (the batched mode): the
// instance table, per-instance storage shifts and relaxation rates as the
// batched single step takes them, so the bits are those of two batched steps.
// ---------------------------------------------------------------------------
// Rates and NSBC parameters of instance d, as the batched step forms them.
template <typename C, bool SHIFT>
__device__ __forceinline__ Rates<C> instance_rates(const InstDev& d, const Shift<C>* __restrict__ shifts, int k,
                                                   double s_e, double s_eps, double s_q) {
  Rates<C> r{C(d.omega), C(s_e), C(s_eps), C(s_q), {}};
  if constexpr (SHIFT) r.z = shifts[k];
  return r;
}

// Frame work: item j = {instance k, first frame thread t0 of this block (a
// multiple of 128), element offset of the instance's frame buffer (9 planes
// of ring_offset(nx, ny, 3) elements), 0}; one block of 128 threads per item.
// TO_FRAME: step n + 1 from pool A into the frame buffers F (width 3); else
// step n + 2 from F into pool B (width 2).
template <typename T, int MODEL, bool SHIFT, bool TO_FRAME>
__global__ void __launch_bounds__(128) frame_batch_kernel(const T* __restrict__ A, T* __restrict__ B, T* __restrict__ F,
                                                          const InstDev* __restrict__ inst,
                                                          const Shift<typename Store<T>::C>* __restrict__ shifts,
                                                          const int4* __restrict__ items, Nsbc p, double s_e,
                                                          double s_eps, double s_q) {
  using C = typename Store<T>::C;
  const int4 w = items[blockIdx.x];
  const InstDev d = inst[w.x];
  const Rates<C> r = instance_rates<C, SHIFT>(d, shifts, w.x, s_e, s_eps, s_q);
  Nsbc q = p;
  q.m0[0] = d.m0[0];
  q.m0[1] = d.m0[1];
  q.m0[2] = d.m0[2];
  const Geom g{d.nx, d.ny, d.pitch, d.plane};
  const int fn = ring_offset(d.nx, d.ny, kFrameWidth);
  const int t = w.y + threadIdx.x;
  if constexpr (TO_FRAME)
    frame_node<T, MODEL, SHIFT>(GlobalRawSrc<T>{A + d.off, d.plane, d.pitch}, FrameDst<T>{F + w.z, d.nx, d.ny, fn}, g,
                                q, r, kFrameWidth, t);
  else
    frame_node<T, MODEL, SHIFT>(FrameSrc<T>{F + w.z, d.nx, d.ny, fn}, GlobalRawDst<T>{B + d.off, d.plane, d.pitch}, g,
                                q, r, 2, t);
}

// Rolling work: item j = {instance k, strip start X0, output rows Ya, Yb}.
// Warps claim items from a counter (sched[0]; the last warp to finish resets
// it and sched[1]); items come largest instance first, all strips of a band
// side by side.  A wait that gives up sets sched[2] and the warp returns.
template <typename T, int MODEL, bool SHIFT>
__global__ void __launch_bounds__(kRollThreads, Roll<T>::BLOCKS)
    roll_batch_kernel(const T* __restrict__ A, T* __restrict__ B, const InstDev* __restrict__ inst,
                      const Shift<typename Store<T>::C>* __restrict__ shifts, const int4* __restrict__ items,
                      int n_items, double s_e, double s_eps, double s_q, int* __restrict__ sched) {
  using R = Roll<T>;
  using C = typename Store<T>::C;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[R::WARPS][R::DEPTH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* ring = reinterpret_cast<T*>(smem_raw) + warp * R::DEPTH * R::ROWE;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < R::DEPTH; ++j) mbar_init(&bar[j], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  uint32_t phase = 0u;
  for (;;) {
    int c = 0;
    if (lane == 0) c = atomicAdd(&sched[0], 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= n_items) break;
    const int4 w = items[c];
    const InstDev d = inst[w.x];
    const Rates<C> r = instance_rates<C, SHIFT>(d, shifts, w.x, s_e, s_eps, s_q);
    const Geom g{d.nx, d.ny, d.pitch, d.plane};
    if (!roll_item<T, MODEL, SHIFT>(A + d.off, B + d.off, g, r, w.y, w.z, w.w, ring, bar, phase, lane, sched)) return;
  }
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(&sched[1], 1) == (int)gridDim.x * R::WARPS - 1) {
      sched[0] = 0;
      sched[1] = 0;
    }
  }
}

}  // namespace lbmk

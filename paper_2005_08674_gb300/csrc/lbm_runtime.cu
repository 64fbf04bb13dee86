// lbm_runtime.cu -- host runtime behind the C ABI of include/lbm.h: handle
// state, device memory (library-owned or caller-bound), stream, CUDA-graph
// replay of the step loop, the three step forms (bulk + NSBC kernel pair,
// fused one-launch kernel, staged producer/consumer kernel) in their plain
// or far-field-shifted variant, launch-shape autotuning, and the entry
// points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <mutex>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_aux.cuh"
#include "lbm_kernels.cuh"
#include "lbm_staged.cuh"
#include "lbm_trace.h"
#include "lbm_twostep.cuh"
#include "lbm_tune_cache.h"

namespace lbmk {
Shift<double> far_field_shift(const double m0[3]) {
  Shift<double> z{};
  const double drho = m0[0] - 1.0, rho = m0[0], ux = m0[1], uy = m0[2];
  const double usq = 1.5 * (ux * ux + uy * uy);
  for (int i = 0; i < 9; ++i) {
    const double cu = cx(i) * ux + cy(i) * uy;
    z.sh[i] = wt<double>(i) * (drho + rho * (3.0 * cu + 4.5 * cu * cu - usq));
  }
  for (int i = 0; i < 9; ++i) {
    const double cu = cx(i) * ux + cy(i) * uy;
    z.p0[i] = 1.0 + 3.0 * cu + 4.5 * cu * cu - usq;
  }
  z.u0[0] = ux;
  z.u0[1] = uy;
  z.rho0 = rho;
  for (int c = 0; c < 3; ++c) z.m0[c] = m0[c];
  z.on = !(drho == 0.0 && ux == 0.0 && uy == 0.0);
  return z;
}
}  // namespace lbmk

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

}  // namespace

// Shared with the other translation units of the library (batched mode):
// records the calling thread's error message and returns `code`.
int lbm_internal_fail(int code, const char* msg) {
  g_last_error = msg;
  return code;
}

namespace {

#define LBM_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                  \
  } while (0)

constexpr int kGraphSteps = 16;  // steps per captured graph (even: buffers return to their roles)
constexpr int kReduceThreads = 256;
constexpr int kReduceBlocks = 1216;  // 8 x 152 SMs
constexpr int kNsbcThreads = 128;

// launch shapes compiled for the bulk kernel: threads per block along x
constexpr int kShapesBX[] = {64, 128, 256, 512};
constexpr int kShapesRows[] = {1, 2, 4, 8};
// L2 prefetch distances (rows ahead) tried by the autotuner
constexpr int kPrefetchRows[] = {0, 1, 3, 8};

}  // namespace

struct lbm {
  int nx = 0, ny = 0, pitch = 0;
  long long plane = 0;  // elements per population plane (256-byte multiple)
  double tau = 0.0;
  lbmk::Nsbc nsbc{};
  int storage = LBM_F32;
  size_t elt = 4;
  void* buf[2] = {nullptr, nullptr};
  void* scratch = nullptr;
  bool owns_memory = false;
  bool bound = false;
  bool initialised = false;
  int cur = 0;  // buffer holding the current state
  long long steps = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr, side = nullptr;  // capture stream and NSBC branch
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_chunk[8] = {};  // row chunks of the host transfers (lbm_init, lbm_get_macros)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // by starting buffer
  int bx = 128, rows = 1, pf = 0;  // bulk launch shape and L2 prefetch distance (rows)
  int device = 0;
  int collision = 0;                          // 0 = BGK, 1 = MRT
  double s_e = 1.0, s_eps = 1.0, s_q = 1.0;   // MRT energy, energy-square and flux rates
  // staged step kernel (lbm_set_staged): the producer/consumer kernel of
  // lbm_staged.cuh over this domain's one-instance work list; 0 = off, else
  // the number of tile stages
  int staged = 0;
  // fused step kernel (lbm_set_fused): the bulk grid of the current shape and
  // the NSBC quads in one launch per step
  bool fused = false;
  // two-step pass (lbm_set_twostep): two steps per pass, the step in between
  // kept on chip except on the frame of width 3 (in d_frame, fn nodes);
  // the rolling kernel's strips, bands, rows per band, bands per wave,
  // waves and persistent grid, and the device's SM count
  bool twostep = false;
  int ts_strips = 0, ts_bands = 0, ts_band = 0, ts_wave_bands = 0, ts_waves = 0, ts_grid = 0, sms = 0;
  void* d_frame = nullptr;
  int frame_fn = 0;
  int4* d_items = nullptr;
  lbmk::InstDev* d_inst = nullptr;
  void* d_shift = nullptr;  // the far field's storage shift in the compute type (staged kernel)
  int* d_sched = nullptr;  // work counter, blocks done, give-up flag
  int n_items = 0, items_storage = -1, staged_grid = 0;
  // per-launch timing (lbm_profile): an event pair around every launch, and
  // which kernel it was (0 = bulk or staged step kernel, 1 = NSBC)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
};

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

lbmk::Geom geom(const lbm_t* h) { return lbmk::Geom{h->nx, h->ny, h->pitch, h->plane}; }

size_t macro_bytes(const lbm_t* h) { return round_up((size_t)h->nx * h->ny * sizeof(double), 256); }

// scratch layout: rho | ux | uy (each macro_bytes) | partials | out[4]
double* scratch_field(lbm_t* h, int c) {
  return reinterpret_cast<double*>(static_cast<char*>(h->scratch) + c * macro_bytes(h));
}
double* scratch_partials(lbm_t* h) { return scratch_field(h, 3); }
double* scratch_out(lbm_t* h) { return scratch_partials(h) + kReduceBlocks * 4; }

void drop_graphs(lbm_t* h) {
  for (auto& g : h->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  h->staged_grid = 0;  // the staged kernel's residency may have changed too
}

int ensure_memory(lbm_t* h) {
  if (h->bound) return LBM_OK;
  const size_t bb = lbm_buffer_bytes(h), sb = lbm_scratch_bytes(h);
  LBM_CUDA(cudaGetDevice(&h->device));
  LBM_CUDA(cudaMalloc(&h->buf[0], bb));
  LBM_CUDA(cudaMalloc(&h->buf[1], bb));
  LBM_CUDA(cudaMalloc(&h->scratch, sb));
  LBM_CUDA(cudaMemset(h->buf[0], 0, bb));
  LBM_CUDA(cudaMemset(h->buf[1], 0, bb));
  lbmk::check_add(h->buf[0], bb);  // bounds-checked build only
  lbmk::check_add(h->buf[1], bb);
  h->owns_memory = true;
  h->bound = true;
  return LBM_OK;
}

int ensure_streams(lbm_t* h) {
  if (!h->cap) {
    LBM_CUDA(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    LBM_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    LBM_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    LBM_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    for (auto& e : h->ev_chunk) LBM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  return LBM_OK;
}

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152LL * 32 ? 152LL * 32 : b));
}

// ---- typed launchers ------------------------------------------------------


// storage shift of the handle's far field (stored populations are
// deviations from its equilibrium)
lbmk::Shift<double> zshift(const lbm_t* h) { return lbmk::far_field_shift(h->nsbc.m0); }

template <typename C>
lbmk::Rates<C> rates(const lbm_t* h) {
  return lbmk::Rates<C>{C(1.0 / h->tau), C(h->s_e), C(h->s_eps), C(h->s_q), lbmk::shift_as<C>(zshift(h))};
}

// SHIFT: the far field is not at rest, so the stored populations are
// deviations from its equilibrium (Shift); the plain kernels otherwise.
template <typename F>
void with_shift(const lbm_t* h, F&& f) {
  if (zshift(h).on)
    f(std::integral_constant<bool, true>{});
  else
    f(std::integral_constant<bool, false>{});
}

template <typename T, int BX>
void launch_bulk_bx(const lbm_t* h, const void* a, void* b, int rows, cudaStream_t s) {
  using C = typename lbmk::Store<T>::C;
  constexpr int V = lbmk::Store<T>::V;
  const int nvec = (h->nx + V - 1) / V;
  dim3 grid((nvec + BX - 1) / BX, (h->ny - 2 + rows - 1) / rows);
  with_shift(h, [&](auto zc) {
    constexpr bool Z = decltype(zc)::value;
    if (h->collision == 1)
      lbmk::bulk_kernel<T, BX, 1, Z><<<grid, BX, 0, s>>>(static_cast<const T*>(a), static_cast<T*>(b), geom(h),
                                                        rates<C>(h), rows, h->pf);
    else
      lbmk::bulk_kernel<T, BX, 0, Z><<<grid, BX, 0, s>>>(static_cast<const T*>(a), static_cast<T*>(b), geom(h),
                                                        rates<C>(h), rows, h->pf);
  });
}

template <typename T>
void launch_bulk(const lbm_t* h, const void* a, void* b, int bx, int rows, cudaStream_t s) {
  switch (bx) {
    case 64: launch_bulk_bx<T, 64>(h, a, b, rows, s); break;
    case 256: launch_bulk_bx<T, 256>(h, a, b, rows, s); break;
    case 512: launch_bulk_bx<T, 512>(h, a, b, rows, s); break;
    default: launch_bulk_bx<T, 128>(h, a, b, rows, s); break;
  }
}

template <typename T>
void launch_nsbc(const lbm_t* h, const void* a, void* b, cudaStream_t s) {
  using C = typename lbmk::Store<T>::C;
  const long long perim = 2LL * h->nx + 2LL * (h->ny - 2);
  const int blocks = (int)((perim * 4 + kNsbcThreads - 1) / kNsbcThreads);
  with_shift(h, [&](auto zc) {
    constexpr bool Z = decltype(zc)::value;
    if (h->collision == 1)
      lbmk::nsbc_kernel<T, 1, Z><<<blocks, kNsbcThreads, 0, s>>>(static_cast<const T*>(a), static_cast<T*>(b),
                                                                 geom(h), h->nsbc, rates<C>(h));
    else
      lbmk::nsbc_kernel<T, 0, Z><<<blocks, kNsbcThreads, 0, s>>>(static_cast<const T*>(a), static_cast<T*>(b),
                                                                 geom(h), h->nsbc, rates<C>(h));
  });
}

template <typename T, int BX>
void launch_fused_bx(const lbm_t* h, const void* a, void* b, int rows, cudaStream_t s) {
  using C = typename lbmk::Store<T>::C;
  constexpr int V = lbmk::Store<T>::V;
  const int nvec = (h->nx + V - 1) / V;
  const int nbx = (nvec + BX - 1) / BX, nby = (h->ny - 2 + rows - 1) / rows;
  const long long perim = 2LL * h->nx + 2LL * (h->ny - 2);
  const int n_edge = (int)((perim * 4 + BX - 1) / BX);
  const int grid = n_edge + nbx * nby;
  with_shift(h, [&](auto zc) {
    constexpr bool Z = decltype(zc)::value;
    if (h->collision == 1)
      lbmk::fused_step_kernel<T, BX, 1, Z><<<grid, BX, 0, s>>>(static_cast<const T*>(a), static_cast<T*>(b), geom(h),
                                                              h->nsbc, rates<C>(h), rows, h->pf, n_edge, nbx);
    else
      lbmk::fused_step_kernel<T, BX, 0, Z><<<grid, BX, 0, s>>>(static_cast<const T*>(a), static_cast<T*>(b), geom(h),
                                                              h->nsbc, rates<C>(h), rows, h->pf, n_edge, nbx);
  });
}

template <typename T>
void launch_fused(const lbm_t* h, const void* a, void* b, cudaStream_t s) {
  switch (h->bx) {
    case 64: launch_fused_bx<T, 64>(h, a, b, h->rows, s); break;
    case 256: launch_fused_bx<T, 256>(h, a, b, h->rows, s); break;
    case 512: launch_fused_bx<T, 512>(h, a, b, h->rows, s); break;
    default: launch_fused_bx<T, 128>(h, a, b, h->rows, s); break;
  }
}

// ---- staged step kernel --------------------------------------------------
// One launch per step: the producer warp of each block claims the domain's
// work items (NSBC chunks of 32 nodes and tiles of 128 vectors of the
// flattened interior, padding columns included) and stages the tiles into
// shared memory; the 128 consumer threads collide them.  Same device
// functions as the bulk and NSBC kernels, so the same bits.
constexpr int kStagedThreads = 128, kStagedTile = 128;

template <typename T, int MODEL, int STAGES>
const void* staged_kernel(bool shift) {
  return shift ? (const void*)lbmk::batch_ws_kernel<T, kStagedThreads, MODEL, kStagedTile, STAGES, 1, true>
               : (const void*)lbmk::batch_ws_kernel<T, kStagedThreads, MODEL, kStagedTile, STAGES, 1, false>;
}

template <typename T>
const void* staged_kernel_for(const lbm_t* h) {
  const bool z = zshift(h).on;
  if (h->staged >= 4) return h->collision == 1 ? staged_kernel<T, 1, 4>(z) : staged_kernel<T, 0, 4>(z);
  return h->collision == 1 ? staged_kernel<T, 1, 3>(z) : staged_kernel<T, 0, 3>(z);
}

int staged_smem(const lbm_t* h) { return (h->staged >= 4 ? 4 : 3) * 9 * (kStagedTile + 2) * 16; }

template <typename T>
void launch_staged(const lbm_t* h, const void* a, void* b, cudaStream_t s) {
  const T* A = static_cast<const T*>(a);
  T* B = static_cast<T*>(b);
  const int smem = staged_smem(h);
  const dim3 grid(h->staged_grid), block(kStagedThreads + 32);
  auto go = [&](auto kernel) {
    kernel<<<grid, block, smem, s>>>(A, B, h->d_inst,
                                     static_cast<const lbmk::Shift<typename lbmk::Store<T>::C>*>(h->d_shift),
                                     h->d_items, h->n_items, h->nsbc, h->s_e, h->s_eps, h->s_q, h->d_sched);
  };
  with_shift(h, [&](auto zc) {
    constexpr bool Z = decltype(zc)::value;
    if (h->staged >= 4) {
      if (h->collision == 1)
        go(lbmk::batch_ws_kernel<T, kStagedThreads, 1, kStagedTile, 4, 1, Z>);
      else
        go(lbmk::batch_ws_kernel<T, kStagedThreads, 0, kStagedTile, 4, 1, Z>);
    } else {
      if (h->collision == 1)
        go(lbmk::batch_ws_kernel<T, kStagedThreads, 1, kStagedTile, 3, 1, Z>);
      else
        go(lbmk::batch_ws_kernel<T, kStagedThreads, 0, kStagedTile, 3, 1, Z>);
    }
  });
}

// Two-step pass: the rolling items are strips of Roll::OUT output columns
// times bands of ts_band rows, taken with the frame chunks by a persistent
// grid of as many blocks as fit on the device at once; each wave of items is
// all strips of ts_wave_bands bands.  Bands of 16 rows (a restart costs four
// staged and two computed rows) unless the domain gives every resident warp
// more than 16 (f32) or 8 (16-bit) items: measured on pulse-2048 / 4096 /
// 8192, f32 bands of 16 gave 128k / 147k / 162k MLUPS against 58-100k /
// 111-147k / 157-160k for bands of 24-48, and 16-bit storage, bound by
// instruction issue, gains from the longer bands at 8192^2 (29 rows: 207k
// against 198k for 16).  Items that would fill one wave of warps and a bit
// of a second are cut to one wave instead (f32 at 2048^2: 102k -> 128k).
template <typename T>
void twostep_grid(lbm_t* h, int per_sm) {
  using R = lbmk::Roll<T>;
  const int interior_x = h->nx - 4, interior_y = h->ny - 4;  // output nodes [2, n - 2)
  h->ts_strips = (interior_x + R::OUT - 1) / R::OUT;
  const int warps = std::max(1, per_sm * h->sms * R::WARPS);
  const int per_wave = std::max(1, warps / h->ts_strips);  // bands side by side
  const int items_per_warp = sizeof(T) == 4 ? 16 : 8;
  const int want = std::max(1, std::min(items_per_warp * per_wave, interior_y));
  h->ts_band = std::max(std::min(16, interior_y), (interior_y + want - 1) / want);
  const long long items = (long long)h->ts_strips * ((interior_y + h->ts_band - 1) / h->ts_band);
  if (items > warps && items < 2LL * warps && per_wave * h->ts_strips <= warps)
    h->ts_band = std::max(h->ts_band, (interior_y + per_wave - 1) / per_wave);
  h->ts_bands = (interior_y + h->ts_band - 1) / h->ts_band;
  h->ts_wave_bands = std::min(per_wave, h->ts_bands);
  h->ts_waves = (h->ts_bands + h->ts_wave_bands - 1) / h->ts_wave_bands;
  h->ts_grid = std::max(1, per_sm * h->sms);  // frame chunks as well as rolling items: every resident warp
}

template <typename T, int MODEL, bool SHIFT>
void launch_twostep_k(const lbm_t* h, const T* A, T* B, cudaStream_t s) {
  using C = typename lbmk::Store<T>::C;
  const lbmk::Geom g{h->nx, h->ny, h->pitch, h->plane};
  const lbmk::Rates<C> r = rates<C>(h);
  // one launch: the frame chunks of step n + 1, the rolling items, the frame
  // chunks of step n + 2 (32 frame threads per chunk)
  const int n_f1 = (lbmk::frame_threads(h->nx, h->ny, lbmk::kFrameWidth) + 31) / 32;
  const int n_f3 = (lbmk::frame_threads(h->nx, h->ny, 2) + 31) / 32;
  lbmk::pass_kernel<T, MODEL, SHIFT><<<h->ts_grid, lbmk::kRollThreads, lbmk::Roll<T>::kSmem, s>>>(
      A, B, static_cast<T*>(h->d_frame), g, h->nsbc, r, h->ts_strips, h->ts_band, h->ts_bands, h->ts_wave_bands,
      h->ts_waves, n_f1, n_f3, h->d_sched);
}

template <typename T>
void launch_twostep(const lbm_t* h, const void* a, void* b, cudaStream_t s) {
  const T* A = static_cast<const T*>(a);
  T* B = static_cast<T*>(b);
  with_shift(h, [&](auto zc) {
    constexpr bool Z = decltype(zc)::value;
    if (h->collision == 1)
      launch_twostep_k<T, 1, Z>(h, A, B, s);
    else
      launch_twostep_k<T, 0, Z>(h, A, B, s);
  });
}

// the two-step kernel serves this handle (f32 / f16 / bf16, no periodic axis, 8 x 8 nodes or more)
bool twostep_ok(const lbm_t* h) {
  return h->storage != LBM_F64 && !h->nsbc.periodic_x && !h->nsbc.periodic_y && h->nx >= 8 && h->ny >= 8;
}

template <typename T>
int twostep_prepare(lbm_t* h) {
  if (!h->d_sched) {  // the give-up flag of the bounded waits (lbm_status reads it)
    LBM_CUDA(cudaMalloc(&h->d_sched, 4 * sizeof(int)));
    LBM_CUDA(cudaMemset(h->d_sched, 0, 4 * sizeof(int)));
  }
  if (!h->d_frame) {
    h->frame_fn = lbmk::ring_offset(h->nx, h->ny, lbmk::kFrameWidth);
    LBM_CUDA(cudaMalloc(&h->d_frame, (size_t)9 * h->frame_fn * sizeof(T)));
  }
  const int smem = (int)lbmk::Roll<T>::kSmem;
  cudaError_t e = cudaSuccess;
  int per_sm = 0, sms = 0;
  for (const void* k : {(const void*)lbmk::pass_kernel<T, 0, false>, (const void*)lbmk::pass_kernel<T, 0, true>,
                        (const void*)lbmk::pass_kernel<T, 1, false>, (const void*)lbmk::pass_kernel<T, 1, true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbmk::pass_kernel<T, 1, true>, lbmk::kRollThreads,
                                                      smem);
  if (e != cudaSuccess)
    return fail(LBM_ECUDA, "two-step kernel: %d bytes of shared memory refused: %s", smem, cudaGetErrorString(e));
  if (per_sm <= 0) return fail(LBM_ECUDA, "two-step kernel: no block fits on an SM");
  h->sms = sms;
  twostep_grid<T>(h, per_sm);
  return LBM_OK;
}

template <typename F>
void dispatch(int storage, F&& f) {
  switch (storage) {
    case LBM_F64: f(double{}); break;
    case LBM_F16: f(__half{}); break;
    case LBM_BF16: f(__nv_bfloat16{}); break;
    default: f(float{}); break;
  }
}

// Work list, instance record and counters of the staged kernel (built once
// the storage is fixed), and its grid: one resident wave of blocks.  Never
// called inside a stream capture (lbm_step prepares it before capturing).
int ensure_staged(lbm_t* h) {
  if (!h->staged) return LBM_OK;
  if (h->items_storage != h->storage) {
    const int V = (int)(16 / h->elt);
    lbmk::InstDev d{};
    d.off = 0;
    d.plane = h->plane;
    d.nx = h->nx;
    d.ny = h->ny;
    d.pitch = h->pitch;
    d.omega = 1.0 / h->tau;
    for (int c = 0; c < 3; ++c) d.m0[c] = h->nsbc.m0[c];
    lbmk::set_row_divisor(d, V);
    std::vector<int4> items;
    lbmk::staged_instance_items(0, d, V, kStagedTile, kStagedThreads / 4, items);
    if (h->d_items) cudaFree(h->d_items);
    h->d_items = nullptr;
    LBM_CUDA(cudaMalloc(&h->d_items, items.size() * sizeof(int4)));
    LBM_CUDA(cudaMemcpy(h->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (!h->d_inst) LBM_CUDA(cudaMalloc(&h->d_inst, sizeof(lbmk::InstDev)));
    LBM_CUDA(cudaMemcpy(h->d_inst, &d, sizeof d, cudaMemcpyHostToDevice));
    if (!h->d_shift) LBM_CUDA(cudaMalloc(&h->d_shift, sizeof(lbmk::Shift<double>)));
    int rcz = LBM_OK;
    dispatch(h->storage, [&](auto tag) {
      using C = typename lbmk::Store<decltype(tag)>::C;
      const lbmk::Shift<C> z = lbmk::shift_as<C>(zshift(h));
      if (cudaMemcpy(h->d_shift, &z, sizeof z, cudaMemcpyHostToDevice) != cudaSuccess) rcz = LBM_ECUDA;
    });
    if (rcz) return fail(rcz, "staged step kernel: shift copy failed");
    if (!h->d_sched) {
      LBM_CUDA(cudaMalloc(&h->d_sched, 4 * sizeof(int)));
      LBM_CUDA(cudaMemset(h->d_sched, 0, 4 * sizeof(int)));
    }
    h->n_items = (int)items.size();
    h->items_storage = h->storage;
  }
  if (h->staged_grid <= 0) {
    int per_sm = 0, sms = 0;
    LBM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    dispatch(h->storage, [&](auto tag) {
      using T = decltype(tag);
      const void* k = staged_kernel_for<T>(h);
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, staged_smem(h));
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kStagedThreads + 32, staged_smem(h));
    });
    if (per_sm <= 0) return fail(LBM_ECUDA, "staged step kernel: no block fits on an SM");
    h->staged_grid = std::min(h->n_items, per_sm * sms);
  }
  return LBM_OK;
}

// Equilibrium initialisation of rows [y0, y1) of both buffers (the other
// buffer's padding columns start defined too) from device fields [ny][nx].
void enqueue_init_rows(const lbm_t* h, const double* d_rho, const double* d_ux, const double* d_uy, int y0, int y1) {
  dispatch(h->storage, [&](auto tag) {
    using T = decltype(tag);
    lbmk::init_kernel<T><<<lbmk::rows_grid(h->pitch, y1 - y0), 256, 0, h->stream>>>(
        static_cast<T*>(h->buf[0]), static_cast<T*>(h->buf[1]), geom(h), zshift(h), d_rho, d_ux, d_uy, y0, y1);
  });
}

void enqueue_macros_rows(const lbm_t* h, double* d_rho, double* d_ux, double* d_uy, int y0, int y1) {
  dispatch(h->storage, [&](auto tag) {
    using T = decltype(tag);
    lbmk::macros_kernel<T><<<lbmk::rows_grid(h->nx, y1 - y0), 256, 0, h->stream>>>(
        static_cast<const T*>(h->buf[h->cur]), geom(h), lbmk::shift_as<typename lbmk::Store<T>::C>(zshift(h)), d_rho,
        d_ux, d_uy, y0, y1);
  });
}

// One step from buffer `from` to 1 - from.  With `fork`, the NSBC kernel runs
// on the side stream concurrently with the bulk kernel (both only read
// buffer `from` and write disjoint nodes of the other buffer).
// Two-step launches need the kernels' shared-memory attribute and the grid
// (once the storage is fixed); 0 when the two-step kernel is off.
int ensure_twostep(lbm_t* h) {
  if (!h->twostep || !twostep_ok(h)) return LBM_OK;
  int rc = LBM_OK;
  dispatch(h->storage, [&](auto tag) {
    using T = decltype(tag);
    if constexpr (!std::is_same<T, double>::value) rc = twostep_prepare<T>(h);
  });
  return rc;
}

// Two steps from buffer `from` to 1 - from (one launch of the pass kernel).
void enqueue_twostep(const lbm_t* h, int from, cudaStream_t s) {
  dispatch(h->storage, [&](auto tag) {
    using T = decltype(tag);
    if constexpr (!std::is_same<T, double>::value) launch_twostep<T>(h, h->buf[from], h->buf[1 - from], s);
  });
}

void enqueue_step(const lbm_t* h, int from, cudaStream_t s, bool fork) {
  const void* a = h->buf[from];
  void* b = h->buf[1 - from];
  dispatch(h->storage, [&](auto tag) {
    using T = decltype(tag);
    if (h->staged) {
      launch_staged<T>(h, a, b, s);
      return;
    }
    if (h->fused) {
      launch_fused<T>(h, a, b, s);
      return;
    }
    if (fork) {
      cudaEventRecord(h->ev_fork, s);
      cudaStreamWaitEvent(h->side, h->ev_fork, 0);
      launch_nsbc<T>(h, a, b, h->side);
      launch_bulk<T>(h, a, b, h->bx, h->rows, s);
      cudaEventRecord(h->ev_join, h->side);
      cudaStreamWaitEvent(s, h->ev_join, 0);
    } else {
      launch_bulk<T>(h, a, b, h->bx, h->rows, s);
      launch_nsbc<T>(h, a, b, s);
    }
  });
}

int capture_graph(lbm_t* h, int from) {
  cudaGraph_t g = nullptr;
  LBM_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  if (h->twostep && twostep_ok(h)) {
    // kGraphSteps / 2 launches of two steps: an even number of buffer swaps
    for (int k = 0; k < kGraphSteps / 2; ++k) enqueue_twostep(h, (from + k) & 1, h->cap);
  } else {
    for (int k = 0; k < kGraphSteps; ++k) enqueue_step(h, (from + k) & 1, h->cap, true);
  }
  cudaError_t e = cudaStreamEndCapture(h->cap, &g);
  if (e != cudaSuccess) return fail(LBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph[from], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// Event pair for one profiled launch of kernel `kind` (0 bulk / staged, 1 NSBC).
int profiled_pair(lbm_t* h, int kind, cudaEvent_t* e) {
  for (int k = 0; k < 2; ++k) {
    if (h->ev_used == h->ev_pool.size()) {
      cudaEvent_t x;
      LBM_CUDA(cudaEventCreate(&x));
      h->ev_pool.push_back(x);
      h->ev_kind.push_back(0);
    }
    h->ev_kind[h->ev_used] = kind;
    e[k] = h->ev_pool[h->ev_used++];
  }
  return LBM_OK;
}

// One step with an event pair around each kernel, all on the handle's stream.
int enqueue_step_profiled(lbm_t* h, int from) {
  const void* a = h->buf[from];
  void* b = h->buf[1 - from];
  cudaEvent_t e[4];
  const bool one = h->staged || h->fused;  // one launch per step
  int rc = profiled_pair(h, 0, e);
  if (!rc && !one) rc = profiled_pair(h, 1, e + 2);
  if (rc) return rc;
  dispatch(h->storage, [&](auto tag) {
    using T = decltype(tag);
    cudaEventRecord(e[0], h->stream);
    if (h->staged)
      launch_staged<T>(h, a, b, h->stream);
    else if (h->fused)
      launch_fused<T>(h, a, b, h->stream);
    else
      launch_bulk<T>(h, a, b, h->bx, h->rows, h->stream);
    cudaEventRecord(e[1], h->stream);
    if (!one) {
      cudaEventRecord(e[2], h->stream);
      launch_nsbc<T>(h, a, b, h->stream);
      cudaEventRecord(e[3], h->stream);
    }
  });
  return LBM_OK;
}

// A two-step pass with an event pair around its launch (counted as one bulk
// launch; it carries two steps).
int enqueue_twostep_profiled(lbm_t* h, int from) {
  cudaEvent_t e[2];
  int rc = profiled_pair(h, 0, e);
  if (rc) return rc;
  cudaEventRecord(e[0], h->stream);
  enqueue_twostep(h, from, h->stream);
  cudaEventRecord(e[1], h->stream);
  return LBM_OK;
}

int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBM_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

bool shape_compiled(int bx, int rows) {
  bool okb = false, okr = false;
  for (int v : kShapesBX) okb |= v == bx;
  for (int v : kShapesRows) okr |= v == rows;
  return okb && okr;
}

}  // namespace

// =========================================================================
// C ABI
// =========================================================================
extern "C" {

const char* lbm_last_error(void) { return g_last_error.c_str(); }

lbm_t* lbm_create(int32_t nx, int32_t ny, double tau, double farfield_rho, const double farfield_u[2]) {
  if (nx < 3 || ny < 3 || nx > 65536 || ny > 65536) {
    fail(LBM_EINVAL, "lbm_create: nx=%d ny=%d outside [3, 65536]", nx, ny);
    return nullptr;
  }
  if (!std::isfinite(tau) || !(tau > 0.5)) {
    fail(LBM_EINVAL, "lbm_create: tau=%g must be finite and > 0.5", tau);
    return nullptr;
  }
  if (!farfield_u || !std::isfinite(farfield_rho) || !(farfield_rho > 0.0) || !std::isfinite(farfield_u[0]) ||
      !std::isfinite(farfield_u[1])) {
    fail(LBM_EINVAL, "lbm_create: far field must be finite with rho > 0 and u non-NULL");
    return nullptr;
  }
  lbm_t* h = new lbm_t();
  h->nx = nx;
  h->ny = ny;
  h->tau = tau;
  h->nsbc.gamma = 0.6;
  h->nsbc.beta = 0.0;
  h->nsbc.kappa = 3.0;
  h->nsbc.order = 1;
  h->nsbc.corner = 0;
  h->nsbc.m0[0] = farfield_rho;
  h->nsbc.m0[1] = farfield_u[0];
  h->nsbc.m0[2] = farfield_u[1];
  lbm_set_precision(h, LBM_F32);
  return h;
}

void lbm_destroy(lbm_t* h) {
  if (!h) return;
  if (h->stream || h->cap) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  if (h->bound) {
    lbmk::check_remove(h->buf[0]);
    lbmk::check_remove(h->buf[1]);
  }
  if (h->owns_memory) {
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->scratch);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->d_items) cudaFree(h->d_items);
  if (h->d_inst) cudaFree(h->d_inst);
  if (h->d_shift) cudaFree(h->d_shift);
  if (h->d_sched) cudaFree(h->d_sched);
  if (h->d_frame) cudaFree(h->d_frame);
  if (h->cap) {
    cudaStreamDestroy(h->cap);
    cudaStreamDestroy(h->side);
    cudaEventDestroy(h->ev_fork);
    cudaEventDestroy(h->ev_join);
    for (cudaEvent_t e : h->ev_chunk) cudaEventDestroy(e);
  }
  delete h;
}

int lbm_set_nsbc(lbm_t* h, double gamma, double beta, double kappa, int32_t corner_mode, int32_t grad_order) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_nsbc: NULL handle");
  if (!std::isfinite(gamma) || !std::isfinite(beta) || !std::isfinite(kappa) || (grad_order != 1 && grad_order != 2) ||
      (corner_mode != LBM_CORNER_DIAGONAL && corner_mode != LBM_CORNER_MEAN))
    return fail(LBM_EINVAL, "lbm_set_nsbc: need finite gamma, beta, kappa, corner_mode 0 or 1 and grad_order 1 or 2");
  h->nsbc.gamma = gamma;
  h->nsbc.beta = beta;
  h->nsbc.kappa = kappa;
  h->nsbc.order = grad_order;
  h->nsbc.corner = corner_mode;
  drop_graphs(h);
  return LBM_OK;
}

}  // extern "C"

// Autotuner cache (lbm_set_tune_cache), shared with the batched mode: the
// file path ("" = off; the LBM_TUNE_CACHE environment variable sets it until
// the first lbm_set_tune_cache) and the hit / miss counts.
#ifndef LBM_BUILD_ID
#define LBM_BUILD_ID "unversioned"
#endif
namespace {
std::mutex g_tune_mutex;
std::string g_tune_path;
bool g_tune_set = false;
long long g_tune_hits = 0, g_tune_misses = 0;
}  // namespace

std::string lbm_internal_tune_path() {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  if (!g_tune_set) {
    const char* env = std::getenv("LBM_TUNE_CACHE");
    g_tune_path = env ? env : "";
    g_tune_set = true;
  }
  return g_tune_path;
}

// The key of a tuning problem on the current device (see lbm_tune_cache.h).
std::string lbm_internal_tune_key(const char* kind, int storage, int model, bool shift,
                                  const std::vector<long long>& dims) {
  int dev = 0, drv = 0, rt = 0;
  cudaGetDevice(&dev);
  cudaDriverGetVersion(&drv);
  cudaRuntimeGetVersion(&rt);
  cudaDeviceProp prop{};
  const char* name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown-device";
  return lbmtune::make_key(name, drv, rt, LBM_BUILD_ID, kind, storage, model, shift, dims);
}

void lbm_internal_tune_count(bool hit) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  (hit ? g_tune_hits : g_tune_misses) += 1;
}

extern "C" int lbm_set_tune_cache(const char* path) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_path = path ? path : "";
  g_tune_set = true;
  return LBM_OK;
}

extern "C" int lbm_tune_cache_stats(int64_t* hits, int64_t* misses) {
  if (!hits || !misses) return fail(LBM_EINVAL, "lbm_tune_cache_stats: NULL argument");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  *hits = g_tune_hits;
  *misses = g_tune_misses;
  return LBM_OK;
}

// Shared with the batched mode: validate edge types and fill the NSBC block.
int lbm_internal_set_edges(lbmk::Nsbc* p, const int32_t types[4], const double uw[8]) {
  if (!types) return fail(LBM_EINVAL, "set_edges: NULL types");
  for (int s = 0; s < 4; ++s)
    if (types[s] < LBM_EDGE_NSBC || types[s] > LBM_EDGE_VELOCITY)
      return fail(LBM_EINVAL, "set_edges: unknown edge type %d on side %d", types[s], s);
  if ((types[0] == LBM_EDGE_PERIODIC) != (types[1] == LBM_EDGE_PERIODIC) ||
      (types[2] == LBM_EDGE_PERIODIC) != (types[3] == LBM_EDGE_PERIODIC))
    return fail(LBM_EINVAL, "set_edges: periodic edges come in pairs (left+right, bottom+top)");
  for (int s = 0; s < 4; ++s)
    if (types[s] == LBM_EDGE_VELOCITY && (!uw || !std::isfinite(uw[2 * s]) || !std::isfinite(uw[2 * s + 1])))
      return fail(LBM_EINVAL, "set_edges: velocity edge %d needs a finite velocity", s);
  p->periodic_x = types[0] == LBM_EDGE_PERIODIC;
  p->periodic_y = types[2] == LBM_EDGE_PERIODIC;
  for (int s = 0; s < 4; ++s) {
    p->vel[s] = types[s] == LBM_EDGE_VELOCITY;
    p->uw[s][0] = p->vel[s] ? uw[2 * s] : 0.0;
    p->uw[s][1] = p->vel[s] ? uw[2 * s + 1] : 0.0;
  }
  return LBM_OK;
}

extern "C" {

int lbm_set_edges(lbm_t* h, const int32_t types[4], const double uw[8]) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_edges: NULL handle");
  lbmk::Nsbc p = h->nsbc;
  int rc = lbm_internal_set_edges(&p, types, uw);
  if (rc) return rc;
  h->nsbc = p;
  drop_graphs(h);
  return LBM_OK;
}

int lbm_set_collision(lbm_t* h, int32_t model, double omega_e, double omega_eps, double omega_q) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_collision: NULL handle");
  if (model != LBM_BGK && model != LBM_MRT) return fail(LBM_EINVAL, "lbm_set_collision: unknown model %d", model);
  if (model == LBM_MRT)
    for (double r : {omega_e, omega_eps, omega_q})
      if (!std::isfinite(r) || !(r > 0.0) || !(r < 2.0))
        return fail(LBM_EINVAL, "lbm_set_collision: MRT rates must lie in (0, 2)");
  h->collision = model;
  if (model == LBM_MRT) {
    h->s_e = omega_e;
    h->s_eps = omega_eps;
    h->s_q = omega_q;
  }
  drop_graphs(h);
  return LBM_OK;
}

int lbm_set_precision(lbm_t* h, int32_t storage) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_precision: NULL handle");
  if (storage < LBM_F64 || storage > LBM_BF16) return fail(LBM_EINVAL, "lbm_set_precision: unknown storage %d", storage);
  if (h->bound) return fail(LBM_ESTATE, "lbm_set_precision: memory already bound or allocated");
  h->storage = storage;
  h->elt = storage == LBM_F64 ? 8 : (storage == LBM_F32 ? 4 : 2);
  h->pitch = (int)round_up((size_t)h->nx, 64);
  h->plane = (long long)(round_up((size_t)h->ny * h->pitch * h->elt, 256) / h->elt);
  return LBM_OK;
}

int lbm_set_stream(lbm_t* h, void* cuda_stream) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_stream: NULL handle");
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return LBM_OK;
}

size_t lbm_buffer_bytes(const lbm_t* h) { return h ? (size_t)9 * h->plane * h->elt : 0; }

size_t lbm_scratch_bytes(const lbm_t* h) {
  return h ? 3 * macro_bytes(h) + round_up((kReduceBlocks * 4 + 4) * sizeof(double), 256) : 0;
}

int lbm_bind(lbm_t* h, void* dev_a, void* dev_b, void* dev_scratch) {
  if (!h || !dev_a || !dev_b || !dev_scratch) return fail(LBM_EINVAL, "lbm_bind: NULL argument");
  if (h->bound) return fail(LBM_ESTATE, "lbm_bind: memory already bound or allocated");
  for (void* p : {dev_a, dev_b, dev_scratch})
    if (reinterpret_cast<uintptr_t>(p) % 256) return fail(LBM_EINVAL, "lbm_bind: pointers must be 256-byte aligned");
  LBM_CUDA(cudaGetDevice(&h->device));
  h->buf[0] = dev_a;
  h->buf[1] = dev_b;
  h->scratch = dev_scratch;
  lbmk::check_add(dev_a, lbm_buffer_bytes(h));  // bounds-checked build only
  lbmk::check_add(dev_b, lbm_buffer_bytes(h));
  h->bound = true;
  h->owns_memory = false;
  return LBM_OK;
}

int lbm_init_device(lbm_t* h, const double* d_rho, const double* d_ux, const double* d_uy) {
  if (!h || !d_rho || !d_ux || !d_uy) return fail(LBM_EINVAL, "lbm_init_device: NULL argument");
  int rc = ensure_memory(h);
  if (rc) return rc;
  h->cur = 0;
  enqueue_init_rows(h, d_rho, d_ux, d_uy, 0, h->ny);
  rc = check_launch();
  if (rc) return rc;
  h->initialised = true;
  h->steps = 0;
  return LBM_OK;
}

int lbm_init(lbm_t* h, const double* rho, const double* ux, const double* uy) {
  LBM_TRACE("lbm_init");
  if (!h || !rho || !ux || !uy) return fail(LBM_EINVAL, "lbm_init: NULL argument");
  int rc = ensure_memory(h);
  if (rc) return rc;
  rc = ensure_streams(h);
  if (rc) return rc;
  // the copy of row chunk c (side stream, copy engine) overlaps the
  // initialisation of chunk c - 1 (the handle's stream)
  const double* src[3] = {rho, ux, uy};
  LBM_CUDA(cudaEventRecord(h->ev_fork, h->stream));  // earlier work on the scratch area first
  LBM_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  h->cur = 0;
  constexpr int K = (int)(sizeof(h->ev_chunk) / sizeof(h->ev_chunk[0]));
  for (int c = 0; c < K; ++c) {
    const int y0 = (int)((long long)h->ny * c / K), y1 = (int)((long long)h->ny * (c + 1) / K);
    if (y1 <= y0) continue;
    const size_t off = (size_t)y0 * h->nx, bytes = (size_t)(y1 - y0) * h->nx * sizeof(double);
    for (int f = 0; f < 3; ++f)
      LBM_CUDA(cudaMemcpyAsync(scratch_field(h, f) + off, src[f] + off, bytes, cudaMemcpyHostToDevice, h->side));
    LBM_CUDA(cudaEventRecord(h->ev_chunk[c], h->side));
    LBM_CUDA(cudaStreamWaitEvent(h->stream, h->ev_chunk[c], 0));
    enqueue_init_rows(h, scratch_field(h, 0), scratch_field(h, 1), scratch_field(h, 2), y0, y1);
  }
  rc = check_launch();
  if (rc) return rc;
  h->initialised = true;
  h->steps = 0;
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_step(lbm_t* h, int32_t n) {
  LBM_TRACE("lbm_step");
  if (!h) return fail(LBM_EINVAL, "lbm_step: NULL handle");
  if (n < 0) return fail(LBM_EINVAL, "lbm_step: n=%d < 0", n);
  if (!h->initialised) return fail(LBM_ESTATE, "lbm_step: call lbm_init first");
  int rc = ensure_streams(h);
  if (!rc) rc = ensure_staged(h);
  if (!rc) rc = ensure_twostep(h);
  if (rc) return rc;
  const bool two = h->twostep && twostep_ok(h);
  int left = n;
  if (h->profiling) {
    for (; two && left >= 2; left -= 2) {
      rc = enqueue_twostep_profiled(h, h->cur);
      if (rc) return rc;
      h->cur ^= 1;
    }
    for (; left > 0; --left) {
      rc = enqueue_step_profiled(h, h->cur);
      if (rc) return rc;
      h->cur ^= 1;
    }
  }
  if (left >= kGraphSteps) {
    if (!h->graph[h->cur]) {
      rc = capture_graph(h, h->cur);
      if (rc) return rc;
    }
    while (left >= kGraphSteps) {
      LBM_CUDA(cudaGraphLaunch(h->graph[h->cur], h->stream));
      left -= kGraphSteps;  // kGraphSteps is even: h->cur is unchanged
    }
  }
  for (; two && left >= 2; left -= 2) {
    enqueue_twostep(h, h->cur, h->stream);
    h->cur ^= 1;
  }
  for (; left > 0; --left) {  // an odd last step: the kernel pair
    enqueue_step(h, h->cur, h->stream, false);
    h->cur ^= 1;
  }
  rc = check_launch();
  if (rc) return rc;
  h->steps += n;
  return LBM_OK;
}

int64_t lbm_steps_done(const lbm_t* h) { return h ? h->steps : -1; }

int lbm_get_dims(const lbm_t* h, int32_t* nx, int32_t* ny) {
  if (!h || !nx || !ny) return fail(LBM_EINVAL, "lbm_get_dims: NULL argument");
  *nx = h->nx;
  *ny = h->ny;
  return LBM_OK;
}

namespace lbmk {
void batch_check_read(unsigned long long* count, unsigned long long* first, bool reset);  // lbm_batch.cu
}

int lbm_check_read(int64_t* rejected, uint64_t* first_address, int32_t reset) {
  if (!rejected || !first_address) return fail(LBM_EINVAL, "lbm_check_read: NULL argument");
  unsigned long long c1 = 0, f1 = 0, c2 = 0, f2 = 0;
  lbmk::check_read(&c1, &f1, reset != 0);
  lbmk::batch_check_read(&c2, &f2, reset != 0);
  *rejected = (int64_t)(c1 + c2);
  *first_address = c1 ? f1 : f2;
  return lbmk::kChecked ? 1 : 0;
}

int lbm_get_macros_device(lbm_t* h, double* d_rho, double* d_ux, double* d_uy) {
  if (!h || !d_rho || !d_ux || !d_uy) return fail(LBM_EINVAL, "lbm_get_macros_device: NULL argument");
  if (!h->initialised) return fail(LBM_ESTATE, "lbm_get_macros_device: call lbm_init first");
  enqueue_macros_rows(h, d_rho, d_ux, d_uy, 0, h->ny);
  return check_launch();
}

int lbm_get_macros(lbm_t* h, double* rho, double* ux, double* uy) {
  LBM_TRACE("lbm_get_macros");
  if (!h || !rho || !ux || !uy) return fail(LBM_EINVAL, "lbm_get_macros: NULL argument");
  if (!h->initialised) return fail(LBM_ESTATE, "lbm_get_macros: call lbm_init first");
  int rc = ensure_streams(h);
  if (rc) return rc;
  // the macros of row chunk c (the handle's stream) overlap the copy-out of
  // chunk c - 1 (side stream, copy engine)
  double* dst[3] = {rho, ux, uy};
  constexpr int K = (int)(sizeof(h->ev_chunk) / sizeof(h->ev_chunk[0]));
  for (int c = 0; c < K; ++c) {
    const int y0 = (int)((long long)h->ny * c / K), y1 = (int)((long long)h->ny * (c + 1) / K);
    if (y1 <= y0) continue;
    enqueue_macros_rows(h, scratch_field(h, 0), scratch_field(h, 1), scratch_field(h, 2), y0, y1);
    LBM_CUDA(cudaEventRecord(h->ev_chunk[c], h->stream));
    LBM_CUDA(cudaStreamWaitEvent(h->side, h->ev_chunk[c], 0));
    const size_t off = (size_t)y0 * h->nx, bytes = (size_t)(y1 - y0) * h->nx * sizeof(double);
    for (int f = 0; f < 3; ++f)
      LBM_CUDA(cudaMemcpyAsync(dst[f] + off, scratch_field(h, f) + off, bytes, cudaMemcpyDeviceToHost, h->side));
  }
  rc = check_launch();
  if (rc) return rc;
  LBM_CUDA(cudaEventRecord(h->ev_join, h->side));  // later work on the handle's stream waits for the copies
  LBM_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  LBM_CUDA(cudaStreamSynchronize(h->side));
  return LBM_OK;
}

int lbm_get_populations(lbm_t* h, double* f) {
  if (!h || !f) return fail(LBM_EINVAL, "lbm_get_populations: NULL argument");
  if (!h->initialised) return fail(LBM_ESTATE, "lbm_get_populations: call lbm_init first");
  const long long n = (long long)h->nx * h->ny;
  for (int i = 0; i < 9; ++i) {
    dispatch(h->storage, [&](auto tag) {
      using T = decltype(tag);
      lbmk::plane_to_f64<T><<<grid_for(n, 256), 256, 0, h->stream>>>(static_cast<const T*>(h->buf[h->cur]), geom(h),
                                                                      zshift(h), i, scratch_field(h, 0));
    });
    int rc = check_launch();
    if (rc) return rc;
    LBM_CUDA(cudaMemcpyAsync(f + i * n, scratch_field(h, 0), n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

int lbm_set_populations(lbm_t* h, const double* f) {
  if (!h || !f) return fail(LBM_EINVAL, "lbm_set_populations: NULL argument");
  int rc = ensure_memory(h);
  if (rc) return rc;
  const long long n = (long long)h->nx * h->ny;
  h->cur = 0;
  for (int i = 0; i < 9; ++i) {
    LBM_CUDA(cudaMemcpyAsync(scratch_field(h, 0), f + i * n, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    dispatch(h->storage, [&](auto tag) {
      using T = decltype(tag);
      for (int b = 0; b < 2; ++b)
        lbmk::f64_to_plane<T><<<grid_for((long long)h->ny * h->pitch, 256), 256, 0, h->stream>>>(
            static_cast<T*>(h->buf[b]), geom(h), zshift(h), i, scratch_field(h, 0));
    });
    rc = check_launch();
    if (rc) return rc;
    LBM_CUDA(cudaStreamSynchronize(h->stream));
  }
  h->initialised = true;
  h->steps = 0;
  return LBM_OK;
}

}  // extern "C"

// Checkpoint record: this header, then the population buffer as stored.
namespace {
struct StateHeader {
  char magic[8];  // "LBMSTAT1"
  int32_t version, storage, nx, ny, pitch, reserved;
  int64_t steps;
  double m0[3];  // far field: the stored populations are deviations from f^eq(m0)
};
static_assert(sizeof(StateHeader) == 64, "checkpoint header layout");
constexpr char kStateMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', '1'};
}  // namespace

extern "C" {

size_t lbm_state_bytes(const lbm_t* h) { return h ? sizeof(StateHeader) + lbm_buffer_bytes(h) : 0; }

int lbm_save_state(lbm_t* h, void* host, size_t bytes, int64_t* steps) {
  if (!h || !host) return fail(LBM_EINVAL, "lbm_save_state: NULL argument");
  if (!h->initialised) return fail(LBM_ESTATE, "lbm_save_state: call lbm_init first");
  if (bytes != lbm_state_bytes(h))
    return fail(LBM_EINVAL, "lbm_save_state: %zu bytes given, the record is %zu", bytes, lbm_state_bytes(h));
  StateHeader hd{};
  std::memcpy(hd.magic, kStateMagic, sizeof hd.magic);
  hd.version = 1;
  hd.storage = h->storage;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.pitch = h->pitch;
  hd.steps = h->steps;
  for (int c = 0; c < 3; ++c) hd.m0[c] = h->nsbc.m0[c];
  std::memcpy(host, &hd, sizeof hd);
  LBM_CUDA(cudaMemcpyAsync(static_cast<char*>(host) + sizeof hd, h->buf[h->cur], lbm_buffer_bytes(h),
                           cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (steps) *steps = h->steps;
  return LBM_OK;
}

int lbm_load_state(lbm_t* h, const void* host, size_t bytes) {
  if (!h || !host) return fail(LBM_EINVAL, "lbm_load_state: NULL argument");
  if (bytes != lbm_state_bytes(h))
    return fail(LBM_EINVAL, "lbm_load_state: %zu bytes given, the record is %zu", bytes, lbm_state_bytes(h));
  // the record must describe this handle's layout and far field, or its
  // bytes mean something else here
  StateHeader hd;
  std::memcpy(&hd, host, sizeof hd);
  if (std::memcmp(hd.magic, kStateMagic, sizeof hd.magic) != 0 || hd.version != 1)
    return fail(LBM_EINVAL, "lbm_load_state: not a checkpoint record of this library");
  if (hd.storage != h->storage || hd.nx != h->nx || hd.ny != h->ny || hd.pitch != h->pitch)
    return fail(LBM_EINVAL, "lbm_load_state: record holds storage %d, %d x %d (pitch %d); handle has %d, %d x %d (%d)",
                hd.storage, hd.nx, hd.ny, hd.pitch, h->storage, h->nx, h->ny, h->pitch);
  for (int c = 0; c < 3; ++c)
    if (std::memcmp(&hd.m0[c], &h->nsbc.m0[c], sizeof(double)) != 0)
      return fail(LBM_EINVAL, "lbm_load_state: record's far field (%.17g, %.17g, %.17g) differs from the handle's",
                  hd.m0[0], hd.m0[1], hd.m0[2]);
  if (hd.steps < 0) return fail(LBM_EINVAL, "lbm_load_state: step count %lld < 0", (long long)hd.steps);
  int rc = ensure_memory(h);
  if (rc) return rc;
  h->cur = 0;
  const size_t bb = lbm_buffer_bytes(h);
  LBM_CUDA(cudaMemcpyAsync(h->buf[0], static_cast<const char*>(host) + sizeof hd, bb, cudaMemcpyHostToDevice,
                           h->stream));
  LBM_CUDA(cudaMemcpyAsync(h->buf[1], h->buf[0], bb, cudaMemcpyDeviceToDevice, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  h->initialised = true;
  h->steps = hd.steps;
  return LBM_OK;
}

int lbm_reduce(lbm_t* h, const double* ref_rho, const double* ref_ux, const double* ref_uy, int32_t ref_pitch,
               double out[4]) {
  LBM_TRACE("lbm_reduce");
  if (!h || !out) return fail(LBM_EINVAL, "lbm_reduce: NULL argument");
  if (!h->initialised) return fail(LBM_ESTATE, "lbm_reduce: call lbm_init first");
  if (ref_rho && (!ref_ux || !ref_uy || ref_pitch < h->nx))
    return fail(LBM_EINVAL, "lbm_reduce: reference needs rho, ux, uy and pitch >= nx");
  lbmk::RefField ref{ref_rho, ref_ux, ref_uy, ref_pitch};
  const long long n = (long long)h->nx * h->ny;
  const int blocks = (int)std::min<long long>(kReduceBlocks, (n + kReduceThreads - 1) / kReduceThreads);
  dispatch(h->storage, [&](auto tag) {
    using T = decltype(tag);
    lbmk::reduce_kernel<T, kReduceThreads><<<blocks, kReduceThreads, 0, h->stream>>>(
        static_cast<const T*>(h->buf[h->cur]), geom(h), lbmk::shift_as<typename lbmk::Store<T>::C>(zshift(h)), ref,
        h->nsbc.m0[0], h->nsbc.m0[1], h->nsbc.m0[2], scratch_partials(h));
  });
  lbmk::reduce_finish<kReduceThreads><<<1, kReduceThreads, 0, h->stream>>>(scratch_partials(h), blocks, scratch_out(h));
  int rc = check_launch();
  if (rc) return rc;
  LBM_CUDA(cudaMemcpyAsync(out, scratch_out(h), 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (out[3] > 0.0) return fail(LBM_EUNSTABLE, "lbm_reduce: %.0f nodes with non-finite or non-positive density", out[3]);
  return LBM_OK;
}

int lbm_profile(lbm_t* h, int32_t enable) {
  if (!h) return fail(LBM_EINVAL, "lbm_profile: NULL handle");
  h->profiling = enable != 0;
  h->ev_used = 0;
  return LBM_OK;
}

int lbm_profile_read(lbm_t* h, double out[4]) {
  if (!h || !out) return fail(LBM_EINVAL, "lbm_profile_read: NULL argument");
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  double ms[2] = {0.0, 0.0}, n[2] = {0.0, 0.0};
  for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
    float t = 0.f;
    LBM_CUDA(cudaEventElapsedTime(&t, h->ev_pool[k], h->ev_pool[k + 1]));
    ms[h->ev_kind[k]] += t;
    n[h->ev_kind[k]] += 1.0;
  }
  out[0] = ms[0];
  out[1] = n[0];
  out[2] = ms[1];
  out[3] = n[1];
  h->ev_used = 0;
  return LBM_OK;
}

int lbm_set_launch(lbm_t* h, int32_t threads_x, int32_t rows, int32_t prefetch_rows) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_launch: NULL handle");
  if (threads_x == 0 && rows == 0) {
    threads_x = 128;
    rows = 1;
  }
  if (!shape_compiled(threads_x, rows))
    return fail(LBM_EINVAL, "lbm_set_launch: shape (%d, %d) not compiled", threads_x, rows);
  if (prefetch_rows < 0 || prefetch_rows > 64)
    return fail(LBM_EINVAL, "lbm_set_launch: prefetch_rows=%d outside [0, 64]", prefetch_rows);
  h->bx = threads_x;
  h->rows = rows;
  h->pf = prefetch_rows;
  h->staged = 0;
  h->fused = false;
  h->twostep = false;
  drop_graphs(h);
  return LBM_OK;
}

int lbm_set_fused(lbm_t* h, int32_t enable) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_fused: NULL handle");
  h->fused = enable != 0;
  if (h->fused) {
    h->staged = 0;
    h->twostep = false;
  }
  drop_graphs(h);
  return LBM_OK;
}

int32_t lbm_get_fused(const lbm_t* h) { return h ? (h->fused ? 1 : 0) : LBM_EINVAL; }

int lbm_set_staged(lbm_t* h, int32_t stages) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_staged: NULL handle");
  if (stages != 0 && stages != 3 && stages != 4)
    return fail(LBM_EINVAL, "lbm_set_staged: stages=%d (0 = off, 3 or 4)", stages);
  h->staged = stages;
  if (stages) {
    h->fused = false;
    h->twostep = false;
  }
  drop_graphs(h);
  return LBM_OK;
}

int32_t lbm_get_staged(const lbm_t* h) { return h ? h->staged : LBM_EINVAL; }

int lbm_set_twostep(lbm_t* h, int32_t enable) {
  if (!h) return fail(LBM_EINVAL, "lbm_set_twostep: NULL handle");
  if (enable && !twostep_ok(h))
    return fail(LBM_EINVAL, "lbm_set_twostep: needs f32, f16 or bf16 storage, no periodic axis and 8 x 8 nodes or more");
  h->twostep = enable != 0;
  if (h->twostep) {
    h->staged = 0;
    h->fused = false;
  }
  drop_graphs(h);
  return LBM_OK;
}

int32_t lbm_get_twostep(const lbm_t* h) { return h ? (h->twostep ? 1 : 0) : LBM_EINVAL; }

int lbm_status(lbm_t* h) {
  if (!h) return fail(LBM_EINVAL, "lbm_status: NULL handle");
  if (!h->d_sched) return LBM_OK;
  int flag = 0;
  LBM_CUDA(cudaMemcpyAsync(&flag, h->d_sched + 2, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (flag) return fail(LBM_ETIMEOUT, "lbm_status: a bounded wait of the staged step kernel gave up");
  return LBM_OK;
}

int lbm_autotune(lbm_t* h, int32_t* threads_x, int32_t* rows, int32_t* prefetch_rows, double* ms_per_step) {
  LBM_TRACE("lbm_autotune");
  if (!h) return fail(LBM_EINVAL, "lbm_autotune: NULL handle");
  if (!h->initialised) return fail(LBM_ESTATE, "lbm_autotune: call lbm_init first");
  int rc = ensure_streams(h);
  if (rc) return rc;
  // a choice recorded for the same key is applied without timing
  const std::string tune_path = lbm_internal_tune_path();
  std::string tune_key;
  if (!tune_path.empty()) {
    tune_key = lbm_internal_tune_key("domain", h->storage, h->collision, zshift(h).on, {h->nx, h->ny});
    lbmtune::Entry e;
    double bx = 0, r = 0, pf = 0, st = -1, fz = -1, ts = -1, ms = 0;
    if (lbmtune::lookup(tune_path, tune_key, &e) && e.get("threads_x", &bx) && e.get("rows", &r) &&
        e.get("prefetch_rows", &pf) && e.get("staged", &st) && e.get("fused", &fz) && e.get("twostep", &ts) &&
        e.get("ms_per_step", &ms) && (st == 0 || st == 3 || st == 4) && (fz == 0 || fz == 1) &&
        (ts == 0 || ts == 1) && lbm_set_launch(h, (int32_t)bx, (int32_t)r, (int32_t)pf) == LBM_OK &&
        (st == 0 || lbm_set_staged(h, (int32_t)st) == LBM_OK) && (fz == 0 || lbm_set_fused(h, 1) == LBM_OK) &&
        (ts == 0 || lbm_set_twostep(h, 1) == LBM_OK)) {
      lbm_internal_tune_count(true);
      if (threads_x) *threads_x = h->bx;
      if (rows) *rows = h->rows;
      if (prefetch_rows) *prefetch_rows = h->pf;
      if (ms_per_step) *ms_per_step = ms;
      return LBM_OK;
    }
  }
  // keep the state: copy the current buffer aside, restore it at the end
  const size_t bb = lbm_buffer_bytes(h);
  void* backup = nullptr;
  LBM_CUDA(cudaMallocAsync(&backup, bb, h->stream));
  LBM_CUDA(cudaMemcpyAsync(backup, h->buf[h->cur], bb, cudaMemcpyDeviceToDevice, h->stream));
  cudaEvent_t e0, e1;
  LBM_CUDA(cudaEventCreate(&e0));
  LBM_CUDA(cudaEventCreate(&e1));
  const long long cells = (long long)h->nx * h->ny;
  const int reps = (int)std::max<long long>(4, std::min<long long>(64, (1LL << 28) / std::max(cells, 1LL)));
  float best = 1e30f;
  int best_bx = h->bx, best_rows = h->rows, best_pf = h->pf, best_staged = h->staged;
  bool best_fused = h->fused, best_twostep = false;
  h->twostep = false;
  // whole steps as the graphs run them (NSBC kernel on the forked branch)
  auto time_steps = [&]() -> float {
    for (int k = 0; k < 2; ++k) enqueue_step(h, k & 1, h->stream, true);
    cudaEventRecord(e0, h->stream);
    for (int k = 0; k < reps; ++k) enqueue_step(h, k & 1, h->stream, true);
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
  };
  // small domains: steps as lbm_step replays them (captured graphs of
  // kGraphSteps steps), since there the gaps between launches are part of
  // what is being chosen (timed one by one, a form with fewer launches per
  // step looks better than it runs)
  const bool use_graph = cells <= (1LL << 22);
  auto time_graph = [&]() -> float {
    drop_graphs(h);
    if (h->staged && ensure_staged(h) != LBM_OK) return 1e30f;
    if (h->twostep && ensure_twostep(h) != LBM_OK) return 1e30f;
    if (capture_graph(h, 0) != LBM_OK) return 1e30f;
    const int n = std::max(1, reps / kGraphSteps);
    cudaGraphLaunch(h->graph[0], h->stream);
    cudaEventRecord(e0, h->stream);
    for (int k = 0; k < n; ++k) cudaGraphLaunch(h->graph[0], h->stream);
    cudaEventRecord(e1, h->stream);
    float ms = 1e30f;
    if (cudaEventSynchronize(e1) == cudaSuccess) {
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)(n * kGraphSteps);
    }
    drop_graphs(h);
    return ms;
  };
  auto time_form = [&]() -> float { return use_graph ? time_graph() : time_steps(); };
  h->staged = 0;
  for (int bx : kShapesBX)
    for (int r : kShapesRows)
      for (int pf : kPrefetchRows)
        for (bool fz : {false, true}) {  // the kernel pair, or both in one launch
          if (r > 1 && (h->ny - 2) / r < 152) continue;  // too few blocks to fill the GPU
          h->bx = bx;
          h->rows = r;
          h->pf = pf;
          h->fused = fz;
          const float ms = time_form();
          if (ms < best) {
            best = ms;
            best_bx = bx;
            best_rows = r;
            best_pf = pf;
            best_staged = 0;
            best_fused = fz;
            best_twostep = false;
          }
        }
  h->fused = false;
  // the staged step kernel (producer/consumer, 3 or 4 tile stages)
  for (int st : {3, 4}) {
    h->staged = st;
    drop_graphs(h);
    if (ensure_staged(h) != LBM_OK) break;
    const float ms = time_form();
    if (ms < best) {
      best = ms;
      best_staged = st;
      best_fused = false;
      best_twostep = false;
    }
  }
  // the two-step kernel: two steps per launch
  h->staged = 0;
  if (twostep_ok(h)) {
    h->twostep = true;
    if (ensure_twostep(h) == LBM_OK) {
      float ms = 1e30f;
      if (use_graph) {
        ms = time_graph();
      } else {
        const int launches = std::max(2, reps / 2);
        for (int k = 0; k < 2; ++k) enqueue_twostep(h, k & 1, h->stream);
        cudaEventRecord(e0, h->stream);
        for (int k = 0; k < launches; ++k) enqueue_twostep(h, k & 1, h->stream);
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) == cudaSuccess) {
          cudaEventElapsedTime(&ms, e0, e1);
          ms /= 2.0f * launches;
        }
      }
      if (ms < best) {
        best = ms;
        best_twostep = true;
        best_staged = 0;
        best_fused = false;
      }
    }
    h->twostep = false;
  }
  rc = check_launch();
  h->bx = best_bx;
  h->rows = best_rows;
  h->pf = best_pf;
  h->staged = best_staged;
  h->fused = best_fused && !best_staged;
  h->twostep = best_twostep && !best_staged && !h->fused;
  drop_graphs(h);
  LBM_CUDA(cudaMemcpyAsync(h->buf[h->cur], backup, bb, cudaMemcpyDeviceToDevice, h->stream));
  LBM_CUDA(cudaFreeAsync(backup, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (!tune_path.empty()) {
    lbm_internal_tune_count(false);
    lbmtune::Entry e{tune_key,
                     {{"threads_x", best_bx}, {"rows", best_rows}, {"prefetch_rows", best_pf},
                      {"staged", h->staged}, {"fused", h->fused ? 1 : 0}, {"twostep", h->twostep ? 1 : 0},
                      {"ms_per_step", best}}};
    lbmtune::store(tune_path, e);  // a cache that cannot be written is only not reused
  }
  if (threads_x) *threads_x = best_bx;
  if (rows) *rows = best_rows;
  if (prefetch_rows) *prefetch_rows = best_pf;
  if (ms_per_step) *ms_per_step = best;
  return LBM_OK;
}

}  // extern "C"

// =========================================================================
// Allocation-free reduction (lbm_reduce_noalloc).
//
// Some callers cannot allocate device memory at the moment they want the
// reduction: a monitoring hook that runs inside another framework's step
// loop, where that framework owns the device memory (its caching allocator
// holds it) or where cudaMalloc/cudaFree would synchronise the device and
// stall the framework's other streams.  For them, lbm_reduce_noalloc runs the
// same reduction kernels as lbm_reduce but keeps the per-block partial sums
// and the four results in the fixed array below instead of the handle's
// scratch area.  It calls no cudaMalloc, cudaFree or allocating routine.
//
// The array lives in every GPU that loads this library until the process
// exits.  Every call on a device shares it and it keeps the last call's
// contents; nothing in it needs to start at zero, because a call reads only
// slots that the same call wrote first.  Calls that overlap on the GPU
// (other streams, other host threads, other handles on the same device) race
// on it: the caller must order them.
// =========================================================================
namespace {

// reduce_kernel hands whole rows to blocks (row y to block y mod grid) and
// columns to threads, so any domain works with at most kNoAllocMaxBlocks
// blocks: the grid is min(ny, kNoAllocMaxBlocks), one block per row up to that.
constexpr int kNoAllocThreads = kReduceThreads;
constexpr int kNoAllocMaxBlocks = 4096;
constexpr int kNoAllocDoubles = kNoAllocMaxBlocks * 4 + 4;  // partials + out[4]: 131,104 bytes

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int noalloc_scratch(double** out) {
  int dev = 0;
  LBM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EINVAL, "lbm_reduce_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(LBM_ECUDA, "lbm_reduce_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_reduce_noalloc(lbm_t* h, const double* ref_rho, const double* ref_ux, const double* ref_uy,
                                  int32_t ref_pitch, double out[4]) {
  if (!h || !out) return fail(LBM_EINVAL, "lbm_reduce_noalloc: NULL argument");
  const int blocks = std::min(h->ny, kNoAllocMaxBlocks);
  if (!h->initialised) return fail(LBM_ESTATE, "lbm_reduce_noalloc: call lbm_init first");
  if (ref_rho && (!ref_ux || !ref_uy || ref_pitch < h->nx))
    return fail(LBM_EINVAL, "lbm_reduce_noalloc: reference needs rho, ux, uy and pitch >= nx");
  if (h->bound) {
    int dev = -1;
    LBM_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) return fail(LBM_EINVAL, "lbm_reduce_noalloc: handle lives on device %d, current is %d",
                                      h->device, dev);
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  double* partials = scratch;
  double* d_out = scratch + kNoAllocMaxBlocks * 4;
  lbmk::RefField ref{ref_rho, ref_ux, ref_uy, ref_pitch};
  dispatch(h->storage, [&](auto tag) {
    using T = decltype(tag);
    lbmk::reduce_kernel<T, kNoAllocThreads><<<blocks, kNoAllocThreads, 0, h->stream>>>(
        static_cast<const T*>(h->buf[h->cur]), geom(h), lbmk::shift_as<typename lbmk::Store<T>::C>(zshift(h)), ref,
        h->nsbc.m0[0], h->nsbc.m0[1], h->nsbc.m0[2], partials);
  });
  lbmk::reduce_finish<kNoAllocThreads><<<1, kNoAllocThreads, 0, h->stream>>>(partials, blocks, d_out);
  rc = check_launch();
  if (rc) return rc;
  LBM_CUDA(cudaMemcpyAsync(out, d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (out[3] > 0.0)
    return fail(LBM_EUNSTABLE, "lbm_reduce_noalloc: %.0f nodes with non-finite or non-positive density", out[3]);
  return LBM_OK;
}

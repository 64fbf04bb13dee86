/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D2Q9 lattice-Boltzmann library with
 * the Non-equilibrium Symmetry Boundary Condition (NSBC) of Euser & Vuik,
 * "A non-reflective boundary condition for LBM based on the assumption of
 * non-equilibrium symmetry" (arXiv 2005.08674).
 *
 * Conventions shared by every entry point:
 *   - Lattice: D2Q9 numbered as in the paper's Fig. 1 (Sec. 3):
 *     c_0=(0,0), c_1=(1,0), c_2=(-1,0), c_3=(0,1), c_4=(0,-1), c_5=(1,1),
 *     c_6=(-1,-1), c_7=(-1,1), c_8=(1,-1); weights 4/9, 1/9, 1/36.
 *   - Node (i, j) sits at x = i, y = j.  Host and device macroscopic fields
 *     are row-major [ny][nx] arrays of double, x fastest.
 *   - The stored state is the post-collision population set of step n.  Its
 *     moments equal the fluid state at step n (collision conserves rho and
 *     rho u), and that is what the macro getters return.
 *   - A step is: pull streaming (Eq. lbe_0), NSBC on every edge node
 *     (Sec. 5: Eqs. nes_0..nes_4), then BGK collision at every node
 *     (Eqs. lbe_1, feq_1), boundary nodes included.
 *   - Status codes: LBM_OK (0) or a negative LBM_E* value; lbm_last_error()
 *     returns a message for the calling thread's last failure.
 *   - Device work is asynchronous on the handle's stream unless an entry
 *     point says it synchronises.  Entry points are not thread-safe on one
 *     handle; distinct handles are independent.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)    /* bad argument: NULL, nx or ny < 3, tau <= 0.5, unknown mode */
#define LBM_ENOMEM (-2)    /* device allocation failed */
#define LBM_ECUDA (-3)     /* a CUDA runtime call failed (message has the CUDA error) */
#define LBM_EUNSTABLE (-4) /* non-finite or non-positive density found by lbm_reduce */
#define LBM_ESTATE (-5)    /* call out of order (e.g. step before init) */
#define LBM_ETIMEOUT (-6)  /* a bounded device-side wait gave up (see lbm_batch_status) */

/* Storage of the populations in device memory.  Every type stores the
 * deviation f_i - f_i^eq(m_0) from the equilibrium of the far field m_0 given
 * to lbm_create (for a far field at rest that is f_i - w_i): a shift that
 * keeps the stored magnitudes as small as the disturbance, so rounding is
 * relative to it even in a mean flow.  binary16 holds it scaled by 2^12.
 * Arithmetic: LBM_F64 computes in double everywhere; the other three
 * collide and apply the NSBC in float, with the NSBC gradient extrapolation
 * and far-field blend (Eqs. nes_2, nes_3) in double. */
#define LBM_F64 0
#define LBM_F32 1
#define LBM_F16 2  /* IEEE binary16, round-to-nearest-even */
#define LBM_BF16 3 /* bfloat16, round-to-nearest-even */

typedef struct lbm lbm_t;

/* Create a simulation of nx x ny nodes with BGK relaxation time tau
 * (Eq. lbe_1, dt = 1) and far-field reference vector
 * m_0 = (farfield_rho, farfield_u[0], farfield_u[1]) (Eq. nes_3).
 * NSBC defaults: gamma = 0.6 (the paper's best value for D2Q9, Sec. 5),
 * beta = 0 (the paper's experiments), kappa = 3, first-order gradient.
 * Storage defaults to LBM_F32.  Host-only: no device memory is touched
 * until lbm_bind or the first lbm_init*.  Returns NULL on bad arguments
 * (nx, ny < 3 or > 65536, tau <= 0.5 or not finite, farfield_rho <= 0,
 * farfield_u NULL) with the reason in lbm_last_error(). */
lbm_t* lbm_create(int32_t nx, int32_t ny, double tau, double farfield_rho,
                  const double farfield_u[2]);

/* Free the handle and any device memory the library allocated for it
 * (never memory passed to lbm_bind).  Synchronises the stream.  NULL-safe. */
void lbm_destroy(lbm_t* h);

/* NSBC parameters (Sec. 5).  gamma: relaxation of the gradient prediction
 * m_p = m - gamma d_n m (Eq. nes_2), d_n a one-sided difference along the
 * outward unit normal with grad_order 1 or 2 points into the domain.
 * beta: far-field factor of Eq. nes_3.  kappa: momentum factor of the
 * correction of Eq. nes_4, f_i -= w_i (d_rho + kappa c_i . d(rho u));
 * kappa = 3 makes the corrected node carry exactly rho_c and rho_c u_c,
 * kappa = 1 is the printed formula.  corner_mode: Sec. 5 says nothing about
 * corner nodes.  LBM_CORNER_DIAGONAL (default) predicts along the diagonal
 * outward normal (|n| = sqrt 2, points b - n, b - 2n on the diagonal);
 * LBM_CORNER_MEAN gives the corner the mean of the two blended states m_c
 * (Eq. nes_3) that the vertical and the horizontal edge through it predict,
 * each along its own unit normal.  Either way the diagonal pair whose two
 * members are both unknown gets f^eq(m_c) alone, and Eq. nes_4 then sets the
 * node's moments.  Host-only; the step graph is recaptured.  Returns
 * LBM_EINVAL for grad_order not in {1, 2}, an unknown corner_mode or
 * non-finite values. */
#define LBM_CORNER_DIAGONAL 0
#define LBM_CORNER_MEAN 1
int lbm_set_nsbc(lbm_t* h, double gamma, double beta, double kappa, int32_t corner_mode, int32_t grad_order);

/* Edge types, per side in the order left (x = 0), right (x = nx-1), bottom
 * (y = 0), top (y = ny-1).  LBM_EDGE_NSBC (default): the boundary of Sec. 5.
 * LBM_EDGE_PERIODIC: the axis wraps (both sides of an axis together).
 * LBM_EDGE_VELOCITY: a Dirichlet velocity edge (the paper's vortex test uses
 * one on its inflow side and only cites the scheme): the same reconstruction
 * as the NSBC with the velocity of m_c replaced by the prescribed
 * (uw[2 side], uw[2 side + 1]) and the density still predicted by Eq. nes_2,
 * so the correction of Eq. nes_4 leaves exactly that velocity on the node;
 * at a corner a left/right velocity edge wins over a bottom/top one.
 * uw may be NULL when no side is a velocity edge.  LBM_EINVAL for unknown
 * types, unpaired periodic sides or non-finite velocities. */
#define LBM_EDGE_NSBC 0
#define LBM_EDGE_PERIODIC 1
#define LBM_EDGE_VELOCITY 2
int lbm_set_edges(lbm_t* h, const int32_t types[4], const double uw[8]);

/* Collision model (bulk and boundary nodes alike).  LBM_BGK (default):
 * Eq. lbe_1 with rate 1/tau.  LBM_MRT: Eq. mrt_lbe with the Gram-Schmidt
 * moment basis of Sec. 4 and S = diag(-, omega_e, omega_eps, -, omega_q, -,
 * omega_q, 1/tau, 1/tau) (Eq. mrt_rm; the conserved moments' rates do not
 * matter, and the stress rate 1/tau keeps nu = cs^2 (tau - 1/2)).  The
 * paper's tests use omega_e = omega_eps = omega_q = 1.9 (acoustic wave, Sec. 6)
 * and 1.4, 1.4, 1.2 (vortex, Sec. 7).  The rates are ignored for BGK.
 * Returns LBM_EINVAL for an unknown model or MRT rates outside (0, 2). */
#define LBM_BGK 0
#define LBM_MRT 1
int lbm_set_collision(lbm_t* h, int32_t model, double omega_e, double omega_eps, double omega_q);

/* Choose the storage type (LBM_F64 / LBM_F32 / LBM_F16 / LBM_BF16).
 * Only allowed before the first lbm_bind / lbm_init* (LBM_ESTATE after). */
int lbm_set_precision(lbm_t* h, int32_t storage);

/* Use this CUDA stream (a cudaStream_t passed as void*; NULL = the legacy
 * default stream) for all later device work of this handle. */
int lbm_set_stream(lbm_t* h, void* cuda_stream);

/* Node counts of the domain as given to lbm_create, so that a caller or a
 * binding can size the [ny][nx] arrays the other calls read and write (a
 * library service; the paper has no counterpart).  Host-only.  LBM_EINVAL
 * for a NULL argument. */
int lbm_get_dims(const lbm_t* h, int32_t* nx, int32_t* ny);

/* Bytes of ONE population buffer: 9 planes of ny rows of `pitch` elements
 * of the storage type, pitch = nx rounded up to 64, each plane starting
 * 256-byte aligned. */
size_t lbm_buffer_bytes(const lbm_t* h);

/* Bytes of the scratch area: three [ny][nx] double fields (macros) plus
 * reduction partials, rounded to 256 bytes. */
size_t lbm_scratch_bytes(const lbm_t* h);

/* Hand the library caller-owned device memory (e.g. from PyTorch): two
 * population buffers of lbm_buffer_bytes() each and one scratch area of
 * lbm_scratch_bytes(), all 256-byte aligned and on the current device.
 * The caller keeps ownership and must keep them alive until lbm_destroy.
 * Must precede the first lbm_init*; otherwise the library allocates its own
 * on first use. */
int lbm_bind(lbm_t* h, void* dev_a, void* dev_b, void* dev_scratch);

/* Initialise every node at equilibrium f_i = f_i^eq(rho, u) (Eq. feq_1) from
 * HOST fields rho, ux, uy ([ny][nx] double).  Copies host->device through
 * the scratch area on the stream and synchronises.  Resets the step count. */
int lbm_init(lbm_t* h, const double* rho, const double* ux, const double* uy);

/* As lbm_init, from DEVICE fields [ny][nx] double; asynchronous. */
int lbm_init_device(lbm_t* h, const double* d_rho, const double* d_ux, const double* d_uy);

/* Advance n >= 0 steps, asynchronously on the stream.  Steps are replayed
 * from a CUDA graph of a fixed number of steps captured on first use (and
 * recaptured after lbm_set_nsbc / lbm_set_stream); the remainder is
 * launched directly. */
int lbm_step(lbm_t* h, int32_t n);

/* Number of steps taken since the last lbm_init* / lbm_set_populations. */
int64_t lbm_steps_done(const lbm_t* h);

/* Macroscopic fields rho, ux, uy (Eqs. cf_0, cf_1 as discrete sums) of the
 * current state into HOST arrays [ny][nx] double; synchronises.  The sums
 * are taken in the storage's compute type (float for f32 / f16 / bf16, where
 * the shifted populations keep rho - 1 exact to float rounding; double for
 * f64) and widened to double. */
int lbm_get_macros(lbm_t* h, double* rho, double* ux, double* uy);

/* As lbm_get_macros into DEVICE arrays [ny][nx] double; asynchronous. */
int lbm_get_macros_device(lbm_t* h, double* d_rho, double* d_ux, double* d_uy);

/* Absolute populations f_i (not shifted) as HOST [9][ny][nx] double, rounded
 * to the storage type on the way in.  For checkpoints and tests.  Both
 * synchronise.  set resets the step count. */
int lbm_get_populations(lbm_t* h, double* f);
int lbm_set_populations(lbm_t* h, const double* f);

/* Checkpoint / resume (a library service): a record of lbm_state_bytes()
 * bytes in HOST memory -- a 64-byte header (magic "LBMSTAT1", version,
 * storage, nx, ny, pitch, step count, far field m0) followed by the current
 * population buffer exactly as stored (lbm_buffer_bytes() bytes: the
 * handle's storage type and layout, deviations from f^eq(m0)).  Loading a
 * record into a handle with the same size, storage and far field continues
 * bit for bit like the run it was saved from (with the same tau, collision
 * and NSBC settings; those are the caller's and are not checked), and sets
 * the step count from the record.  Both synchronise.  LBM_EINVAL for a NULL
 * argument, a byte count other than lbm_state_bytes(), and (load) a record
 * that is not this library's, that holds another storage type, size, pitch
 * or far field (the bytes would mean something else here), or a negative
 * step count -- all checked before any device work; LBM_ESTATE for a save
 * before lbm_init. */
size_t lbm_state_bytes(const lbm_t* h);
int lbm_save_state(lbm_t* h, void* host, size_t bytes, int64_t* steps);
int lbm_load_state(lbm_t* h, const void* host, size_t bytes);

/* FP64 reductions over all nodes, used for the reflection measure and as an
 * instability check.  Each node's terms are formed in the storage's compute
 * type (as for lbm_get_macros; rho_r - 1 is formed in double before it is
 * rounded) and every sum is accumulated in double.  If ref_rho is non-NULL, ref_* are DEVICE [.][ref_pitch]
 * double fields whose element [0] is aligned with node (0, 0) of this
 * handle (pass a pointer into a larger, padded reference domain).  Writes
 * HOST out[4]:
 *   out[0] = sum rho                               (mass)
 *   out[1] = sum (cs^2 (rho - rho_r)^2 / rho_ff + rho_ff |u - u_r|^2) / 2
 *            with (rho_r, u_r) the reference field, or the far field m_0
 *   out[2] = sum rho |u|^2 / 2                     (kinetic energy)
 *   out[3] = number of nodes with non-finite or non-positive rho
 * Synchronises.  Returns LBM_EUNSTABLE when out[3] > 0 (out still filled). */
int lbm_reduce(lbm_t* h, const double* ref_rho, const double* ref_ux, const double* ref_uy,
               int32_t ref_pitch, double out[4]);

/* Bounds-checked build.  liblbm_check.so is this library compiled with
 * LBM_CHECK (paper_2005_08674_gb300/build.py, build(check=True)): there every
 * global access of the step kernels (vector and scalar population loads and
 * stores, the bulk tile copies, the L2 prefetches) and every shared-memory
 * tile access is first checked against the population buffers and pools the
 * host allocated or bound (on the current device) and against its slot; an
 * access that fails is not made (a load yields 0) and is counted instead.
 * The paper has no counterpart: it is a test instrument standing in for a
 * device memory checker.  Writes the number of rejected accesses since the
 * last reset and the first rejected address (top bit set: a shared-memory
 * offset) to *rejected / *first_address, and clears both if reset != 0;
 * synchronises the device.  Returns 1 in the checked build, 0 in the ordinary
 * one (where both outputs are 0), LBM_EINVAL for NULL outputs. */
int lbm_check_read(int64_t* rejected, uint64_t* first_address, int32_t reset);

/* Launch shape of the bulk stream-collide kernel: threads per block along x
 * (64, 128, 256, 512), rows per block (1, 2, 4, 8), and the distance in rows
 * (0 = off, at most 64) at which each warp asks the bulk-copy engine to
 * prefetch its next segments into L2.  threads_x = rows = 0 restores the
 * built-in shape.  Selects the bulk + NSBC kernel pair (turns the staged
 * kernel below off).  Returns LBM_EINVAL for shapes the kernel was not
 * compiled for. */
int lbm_set_launch(lbm_t* h, int32_t threads_x, int32_t rows, int32_t prefetch_rows);

/* Staged step kernel instead of the bulk + NSBC kernel pair: ONE persistent
 * launch per step in which one producer warp per block claims work items of
 * this domain from a counter in device memory -- tiles of 128 16-byte
 * vectors of the flattened interior rows (padding columns included), staged
 * into shared memory by nine cp.async.bulk copies completing on an mbarrier,
 * and chunks of 32 perimeter nodes, each placed after the tile that stages
 * its rows -- and keeps `stages` (3 or 4) of them in flight while 128
 * consumer threads collide them.  Same arithmetic as the kernel pair, hence
 * the same bits.  stages = 0 returns to the kernel pair.  Every wait of the
 * kernel is bounded (about one second of SM clock); a wait that gives up
 * makes it return early and lbm_status report LBM_ETIMEOUT.  LBM_EINVAL for
 * other values.  Device memory for the work list is allocated at the next
 * lbm_step. */
int lbm_set_staged(lbm_t* h, int32_t stages);
/* The current stages setting (0 = kernel pair), or LBM_EINVAL for NULL. */
int32_t lbm_get_staged(const lbm_t* h);
/* One launch per step with the bulk + NSBC kernel pair's work: the bulk grid
 * of the current lbm_set_launch shape and the NSBC quads (Sec. 5) in a
 * single kernel, perimeter blocks first.  For domains small enough that the
 * step is bound by launch gaps rather than by HBM.  Bit-identical to the
 * pair.  enable != 0 turns it on (and the staged kernel off); lbm_set_launch
 * and lbm_set_staged turn it off.  lbm_autotune also times it against the
 * pair for every shape.  lbm_get_fused: 1 if on, 0 if off, LBM_EINVAL for a
 * NULL handle. */
int lbm_set_fused(lbm_t* h, int32_t enable);
int32_t lbm_get_fused(const lbm_t* h);
/* Two steps per pass (temporal blocking), in one launch whose warps take, in
 * turn, three kinds of work: step n + 1 on the frame of nodes within
 * distance 2 of an edge (the NSBC and the interior collision) into a small
 * frame buffer; steps n + 1 and n + 2 on the nodes at distance 2 or more,
 * each warp rolling down a strip of 128 columns, staging the state rows by
 * bulk copies and keeping step n + 1 in registers; and, once all of the first
 * kind is done (a bounded wait on a counter), step n + 2 on the frame from
 * the frame buffer.  Every node runs the same device arithmetic as the
 * single-step kernels and step n + 1 is rounded to the storage type as a
 * single step stores it, so the results are bit-identical to the kernel
 * pair, while the state crosses device memory once per two steps.
 * lbm_step(n) runs n / 2 passes (graphs of 16 steps) and, for odd n, one
 * step of the kernel pair.  enable != 0 turns it on (and the staged and fused
 * kernels off); lbm_set_launch, lbm_set_staged and lbm_set_fused turn it off;
 * lbm_autotune times it against the other forms.  LBM_EINVAL when enabling
 * it on an f64 handle, a handle with a periodic axis or fewer than 8 x 8
 * nodes.  A bounded wait that gives up makes lbm_status report LBM_ETIMEOUT.
 * Device memory: a frame buffer of 9 x (6 (nx + ny) - 36) populations,
 * allocated when first enabled.  lbm_get_twostep: 1 if on, 0 if off,
 * LBM_EINVAL for NULL. */
int lbm_set_twostep(lbm_t* h, int32_t enable);
int32_t lbm_get_twostep(const lbm_t* h);
/* LBM_ETIMEOUT if a bounded wait of the staged kernel gave up (the state is
 * then not valid), else LBM_OK; synchronises the stream. */
int lbm_status(lbm_t* h);

/* Time every compiled bulk launch shape and prefetch distance (as the
 * kernel pair and as the fused one-launch step), and the staged kernel with
 * 3 and 4 stages, on this handle's own buffers (a few whole steps each,
 * CUDA events on the stream) and keep the fastest; the state is restored
 * afterwards (through a temporary device copy from cudaMallocAsync).  Writes
 * the bulk shape, and the time per step in milliseconds of the winner, to
 * the optional outputs; lbm_get_staged / lbm_get_fused tell whether the
 * staged or the fused form won. */
int lbm_autotune(lbm_t* h, int32_t* threads_x, int32_t* rows, int32_t* prefetch_rows, double* ms_per_step);

/* Autotuner cache (a library service; the paper has no counterpart).  With
 * a cache file set, lbm_autotune and lbm_batch_autotune first look up the
 * key of the problem -- device name, driver and runtime versions, the
 * library's build id, single domain or batch, storage, collision model,
 * storage-shift form, and size classes ceil(log2 n) of nx and ny (a batch:
 * of the instance count and the total nodes) -- and apply the recorded launch
 * shape without timing; on a miss they time the candidates as usual and then
 * add the winner to the file.  The file is a small JSON document written by
 * the library (temporary file renamed over the old one); a missing,
 * unreadable or malformed file reads as empty, and one that cannot be
 * written is left as it is, so the cache never makes autotuning fail.
 * path = NULL turns the cache off.  Until the first call the environment
 * variable LBM_TUNE_CACHE, if set, names the file.  Process-wide, host-only;
 * callers that tune from several threads at once should use different
 * files.  Always LBM_OK. */
int lbm_set_tune_cache(const char* path);
/* Lookups that found a usable entry, and autotuner runs that timed the
 * candidates with the cache on, since the process started.  LBM_EINVAL for
 * NULL outputs. */
int lbm_tune_cache_stats(int64_t* hits, int64_t* misses);

/* Allocation-free form of lbm_reduce, for callers that cannot allocate
 * device memory when they need the sums, such as a monitoring hook inside
 * another framework's step loop where that framework owns all device memory
 * or where a cudaMalloc/cudaFree would synchronise the device.  The paper has
 * no counterpart; this is a library service.
 * Same arguments, results, synchronisation and return codes as lbm_reduce,
 * and the same kernels, but the partial sums live in a fixed device array
 * inside the library (131,104 bytes, held by every GPU that loads the
 * library until the process exits) instead of the handle's scratch area; the
 * call makes no cudaMalloc, cudaFree or other allocating call.
 * The array holds the partial sums of at most 4096 blocks; the reduction
 * hands whole rows to blocks (min(ny, 4096) of them), so every domain that
 * lbm_create accepts fits and no size is refused.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (once per device, with that device current); make
 * that first call before any stream capture.  All calls on a device share
 * the array and it keeps the last call's contents (no slot needs to start
 * at zero: a call reads only what it wrote first); calls that overlap on the
 * GPU -- other streams, threads or handles on the same device -- race on it
 * and must be ordered by the caller. */
int lbm_reduce_noalloc(lbm_t* h, const double* ref_rho, const double* ref_ux, const double* ref_uy,
                       int32_t ref_pitch, double out[4]);

/* ------------------------------------------------------------------------
 * Batched mode: many independent simulations of uneven sizes, each with its
 * own tau and far field, stepped together by ONE persistent kernel launch
 * per step (bulk tiles and NSBC chunks of all instances in one work list),
 * replayed from a CUDA graph.  Storage, collision model and NSBC parameters
 * are shared by the batch.  Results per instance are bit-identical to a
 * single-domain handle with the same settings.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch_t;

typedef struct lbm_instance_desc {
  int32_t nx, ny; /* nodes, each in [3, 65536] */
  double tau;     /* > 0.5 */
  double farfield_rho, farfield_ux, farfield_uy;
} lbm_instance_desc;

/* Host-only: validates the descriptors and lays out the pools; NULL on bad
 * arguments (message in lbm_last_error()). */
lbm_batch_t* lbm_batch_create(int32_t count, const lbm_instance_desc* descs, int32_t storage);
/* Frees library-owned device memory; synchronises the stream.  NULL-safe. */
void lbm_batch_destroy(lbm_batch_t* b);
/* NSBC parameters (Eqs. nes_2-nes_4) for every instance of the batch: same
 * arguments, ranges and LBM_EINVAL cases as lbm_set_nsbc.  Host-only. */
int lbm_batch_set_nsbc(lbm_batch_t* b, double gamma, double beta, double kappa, int32_t corner_mode,
                       int32_t grad_order);
/* Collision model (LBM_BGK, or LBM_MRT with the rates of Sec. 4) for every
 * instance: same arguments and errors as lbm_set_collision.  Host-only. */
int lbm_batch_set_collision(lbm_batch_t* b, int32_t model, double omega_e, double omega_eps, double omega_q);
/* Edge types for every instance of the batch, as lbm_set_edges. */
int lbm_batch_set_edges(lbm_batch_t* b, const int32_t types[4], const double uw[8]);
/* CUDA stream (a cudaStream_t, NULL = the legacy default stream) on which
 * every later call on the batch works, as lbm_set_stream.  The step graph is
 * captured on a private stream and launched on this one, so it is kept. */
int lbm_batch_set_stream(lbm_batch_t* b, void* cuda_stream);
/* Total nodes over all instances. */
int64_t lbm_batch_cells(const lbm_batch_t* b);
/* Node counts of instance k (its descriptor's nx, ny).  Host-only.
 * LBM_EINVAL for a NULL argument or k out of range. */
int lbm_batch_get_dims(const lbm_batch_t* b, int32_t k, int32_t* nx, int32_t* ny);
/* Bytes of ONE population pool (all instances), and of the scratch area
 * (three [ny][nx] double fields of the largest instance + reduction slots). */
size_t lbm_batch_buffer_bytes(const lbm_batch_t* b);
size_t lbm_batch_scratch_bytes(const lbm_batch_t* b);
/* Caller-owned device memory (256-byte aligned), before the first init;
 * otherwise the library allocates on first init. */
int lbm_batch_bind(lbm_batch_t* b, void* dev_a, void* dev_b, void* dev_scratch);
/* Instance k at equilibrium from HOST fields [ny_k][nx_k] double; synchronises. */
int lbm_batch_init(lbm_batch_t* b, int32_t k, const double* rho, const double* ux, const double* uy);
/* n steps of every instance (all must be initialised); asynchronous. */
int lbm_batch_step(lbm_batch_t* b, int32_t n);
/* Steps issued (host counter, no sync); an lbm_batch_init after steps
 * were taken restarts it at 0 for the whole batch.  -1 for NULL. */
int64_t lbm_batch_steps_done(const lbm_batch_t* b);
/* Macros of instance k into HOST arrays [ny_k][nx_k] double; synchronises. */
int lbm_batch_get_macros(lbm_batch_t* b, int32_t k, double* rho, double* ux, double* uy);
/* Number of nodes of instance k with non-finite or non-positive density
 * (FP64 reduction); synchronises. */
int lbm_batch_unstable_nodes(lbm_batch_t* b, int32_t k, int64_t* count);
/* Launch shape of the batched step.  Default (no call): the
 * producer/consumer form described last, (128, 3, 0, 1, 0, 128).
 * Register path (tma_tile = 0): a bulk tile is threads_x (64, 128, 256) x `rows` (1, 2, 4)
 * 16-byte vectors of an instance's interior rows laid end to end (nodes per
 * thread = vector x rows); grid size `blocks` (-1 = one block per work item,
 * 0 = one resident wave of blocks looping over the list, > 0 = that many);
 * `prefetch_rows`: 0 = off, 1 = each tile asks the bulk-copy engine for its
 * own footprint in L2 when it starts, k > 1 = for the footprint of the tile
 * k items further down the list (at most 65536); `split` = 0 runs NSBC chunks and bulk tiles in ONE launch
 * per step, 1 runs the NSBC chunks as a second launch beside the bulk tiles
 * (the bulk launch then keeps the single-domain kernel's register budget).
 * `tma_tile` > 0 selects the shared-memory path instead: ONE persistent
 * launch per step whose blocks take NSBC chunks and bulk tiles from a shared
 * counter; tiles of `tma_tile` vectors (128 or 256, with threads_x 128, or
 * 256 with 256) are staged by cp.async.bulk copies completing on an
 * mbarrier, the next tile's copy in flight while the current item is
 * worked on.  `blocks` (0 = one resident wave) sets the grid;
 * `prefetch_rows` and `split` are ignored, and `rows` is 1 or 2 there.
 * `tma_tile` = 128 with threads_x = 128 and `rows` = 3 or 4 selects the
 * producer/consumer form: one extra warp per block claims items and keeps
 * `rows` tiles in flight, the 128 consumer threads work on them in order
 * (no block-wide barrier per item); there `prefetch_rows` is the number of
 * perimeter nodes each quad of lanes handles per NSBC chunk (0 or 1, or 2).
 * Staged-tile work lists run instance after instance in memory order, each
 * NSBC chunk right after the tile that stages its rows.  LBM_EINVAL for a
 * shape not compiled. */
int lbm_batch_set_launch(lbm_batch_t* b, int32_t threads_x, int32_t rows, int32_t blocks, int32_t prefetch_rows,
                         int32_t split, int32_t tma_tile);
/* Two steps per pass for every instance (the pass lbm_set_twostep describes,
 * here in three launches over all instances: step n + 1 on every frame, the
 * rolling items in bands of at most 64 output rows, claimed by warps from a
 * counter, largest instance first, beside the frame launches on a side
 * stream, then step n + 2 on every frame; each instance's frame buffer after
 * the last).  Bit-identical to two batched steps.  lbm_batch_step(n) runs n / 2
 * passes (graphs of 16 steps) and, for odd n, one batched step of the launch
 * shape set.  enable != 0 turns it on; lbm_batch_set_launch turns it off;
 * lbm_batch_autotune times it against the other forms.  LBM_EINVAL when
 * enabling it on f64 storage, with a periodic axis, or with an instance
 * smaller than 8 x 8.  lbm_batch_get_twostep: 1 on, 0 off, LBM_EINVAL for
 * NULL. */
int lbm_batch_set_twostep(lbm_batch_t* b, int32_t enable);
int32_t lbm_batch_get_twostep(const lbm_batch_t* b);
/* Time every compiled tile shape, grid size, prefetch setting and split, the
 * shared-memory paths and the two-step pass, on the batch's own state
 * (restored afterwards, through a temporary device copy from
 * cudaMallocAsync) and keep the fastest. */
int lbm_batch_autotune(lbm_batch_t* b, int32_t* threads_x, int32_t* rows, int32_t* blocks, int32_t* prefetch_rows,
                       int32_t* split, int32_t* tma_tile, double* ms_per_step);
/* LBM_ETIMEOUT if a staged-tile wait of the shared-memory path gave up since
 * the batch was created (the step then left those tiles untouched); LBM_OK
 * otherwise.  Synchronises. */
int lbm_batch_status(lbm_batch_t* b);

/* Split independent instances over `ranks` processes (one GPU each) so
 * that every rank steps about the same number of nodes and no data moves
 * between ranks: the instances, largest first, each go to the rank with the
 * fewest nodes so far (ties: lower instance index first, lower rank).
 * Deterministic, so every rank computes the same partition on its own.
 * cells[k] = nodes of instance k (nx * ny); writes rank_of[k] in
 * [0, ranks).  Host-only (a library service for sharding the batched mode;
 * the paper has no counterpart).  LBM_EINVAL for count < 0, ranks < 1, NULL
 * arrays or a negative node count. */
int lbm_partition_instances(int32_t count, const int64_t* cells, int32_t ranks, int32_t* rank_of);

/* Failure-detection check of the bounded device-side waits: one block waits
 * on an mbarrier that nothing arrives on (the waits of the shared-memory
 * paths), then on a device counter that nothing increments (the two-step
 * pass's wait for its first-frame chunks); each gives up after budget_cycles
 * SM clock cycles (at most 4e9), and the kernel returns normally.  Returns
 * LBM_ETIMEOUT when both waits gave up (the expected outcome), LBM_OK if
 * either did not, LBM_ECUDA on a CUDA error.  Allocates and frees two ints of
 * device memory; synchronises. */
int lbm_wait_selftest(int64_t budget_cycles);

/* Per-launch timing.  While enabled, lbm_step launches every step directly
 * (no graph) on the handle's stream with CUDA events around the bulk
 * stream-collide kernel and around the NSBC kernel, which then run one after
 * the other (with the staged kernel: around its one launch per step, counted
 * as the bulk kernel).  lbm_profile resets the record. */
int lbm_profile(lbm_t* h, int32_t enable);

/* Read and reset the record (synchronises): out[0] = total bulk-kernel
 * milliseconds, out[1] = bulk launches, out[2] = total NSBC-kernel
 * milliseconds, out[3] = NSBC launches, since the last reset. */
int lbm_profile_read(lbm_t* h, double out[4]);

/* Message describing the calling thread's last failure ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */

// lbm_aux.cuh -- the kernels around the time step: initialisation at
// equilibrium, macroscopic fields, population planes to and from FP64, and
// the FP64 mass / energy reductions used for the reflection measure and the
// instability check.  None of them runs inside a step.
#pragma once

#include "lbm_kernels.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
// Initialisation at equilibrium (Eq. feq_1) of rows [y0, y1) of A (and of
// A2 if not null) from double fields [ny][nx]; padding columns are zeroed.
// The equilibrium is formed in double and rounded once to the storage type
// (forming it in float measurably changed the 16-bit runs' reflection
// figures).  The stored value is the deviation from the far-field
// equilibrium (Shift).  Grid: x over the pitch, blockIdx.y striding over the
// rows.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void init_kernel(T* __restrict__ A, T* __restrict__ A2, Geom g, Shift<double> zd,
                            const double* __restrict__ rho, const double* __restrict__ ux,
                            const double* __restrict__ uy, int y0, int y1) {
  using S = Store<T>;
  using C = typename S::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.pitch) return;
  for (int y = y0 + (int)blockIdx.y; y < y1; y += (int)gridDim.y) {
    double e[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) e[i] = 0.0;
    if (x < g.nx) {
      const long long k = (long long)y * g.nx + x;
      equilibrium(rho[k] - 1.0, ux[k], uy[k], e);
#pragma unroll
      for (int i = 0; i < 9; ++i) e[i] = sub_rn(e[i], zd.sh[i]);
    }
    const long long idx = (long long)y * g.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const T v = S::cvt(C(e[i]));
      A[i * g.plane + idx] = v;
      if (A2) A2[i * g.plane + idx] = v;
    }
  }
}

// Macroscopic fields (double) of rows [y0, y1) of the stored state; same grid.
template <typename T>
__global__ void macros_kernel(const T* __restrict__ A, Geom g, Shift<typename Store<T>::C> z, double* __restrict__ rho,
                              double* __restrict__ ux, double* __restrict__ uy, int y0, int y1) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  for (int y = y0 + (int)blockIdx.y; y < y1; y += (int)gridDim.y) {
    typename Store<T>::C m[3];
    node_dmoments(A, g, x, y, z, m);  // deviations from the far field
    const long long k = (long long)y * g.nx + x;
    rho[k] = z.m0[0] + (double)m[0];
    ux[k] = z.m0[1] + (double)m[1];
    uy[k] = z.m0[2] + (double)m[2];
  }
}

// Grid for init_kernel / macros_kernel over `width` columns and `rows` rows.
inline dim3 rows_grid(int width, int rows) {
  return dim3((unsigned)((width + 255) / 256), (unsigned)(rows < 1 ? 1 : (rows > 2048 ? 2048 : rows)));
}

// One population plane <-> absolute double field [ny][nx].
template <typename T>
__global__ void plane_to_f64(const T* __restrict__ A, Geom g, Shift<double> zd, int i, double* __restrict__ out) {
  using S = Store<T>;
  const long long n = (long long)g.ny * g.nx;
  const double w = wt<double>(i) + zd.sh[i];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(k / g.nx), x = (int)(k % g.nx);
    out[k] = (double)S::ldg1(A + i * g.plane + (long long)y * g.pitch + x) + w;
  }
}

template <typename T>
__global__ void f64_to_plane(T* __restrict__ A, Geom g, Shift<double> zd, int i, const double* __restrict__ in) {
  using S = Store<T>;
  const long long n = (long long)g.ny * g.pitch;
  const double w = wt<double>(i) + zd.sh[i];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(idx / g.pitch), x = (int)(idx % g.pitch);
    const double v = x < g.nx ? in[(long long)y * g.nx + x] - w : 0.0;
    A[i * g.plane + idx] = S::cvt(typename S::C(v));
  }
}

// ---------------------------------------------------------------------------
// FP64 reductions: per-block partial sums (4 doubles per block) into
// `partials`, then one block sums the partials in a fixed order.
// ---------------------------------------------------------------------------
struct RefField {
  const double *rho, *ux, *uy;
  int pitch;
};

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* smem) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) smem[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < NT / 32; ++k) s += smem[k];
  return s;  // valid in thread 0
}

// Compensated (Kahan) running sum in the compute type: a thread's share of
// one row is summed here, then widened to double once per row.
template <typename C>
struct KahanSum {
  C s = C(0), c = C(0);
  __device__ __forceinline__ void add(C v) {
    const C y = v - c;
    const C t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Per node: (rho - rho_ff, u - u_ff) in the storage's compute type and the
// energy / mass terms formed there; a thread's terms along one row are summed
// with compensation in that type and every row sum is accumulated in double.
// Sums: [0] mass sum rho (node count x rho_ff + sum of rho - rho_ff), [1]
// disturbance energy sum cs^2 (rho - rho_r)^2 / (2 rho_ff) + rho_ff |u - u_r|^2 / 2
// against the reference field (or the far field), [2] kinetic energy sum
// rho |u|^2 / 2, [3] nodes with a non-finite or non-positive density.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) reduce_kernel(const T* __restrict__ A, Geom g, Shift<typename Store<T>::C> z,
                                                    RefField ref, double rho_ff, double uxf, double uyf,
                                                    double* __restrict__ partials) {
  using C = typename Store<T>::C;
  __shared__ double smem[NT / 32];
  double s[3] = {0.0, 0.0, 0.0};
  long long count = 0, bad = 0;
  const C e_rho = C(0.5 / (3.0 * rho_ff));  // cs^2 / (2 rho_ff), rounded once
  const C e_u = C(0.5 * rho_ff);
  const C rho0 = C(rho_ff), u0 = C(uxf), v0 = C(uyf);
  // rows over blocks, columns over threads (no integer divisions per node)
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x) {
    KahanSum<C> k0, k1, k2;
    for (int x = threadIdx.x; x < g.nx; x += NT) {
      C m[3];
      node_dmoments(A, g, x, y, z, m);  // (rho - rho_ff, u - u_ff)
      C drr = C(0), dur = C(0), dvr = C(0);
      if (ref.rho) {
        // the reference's deviations from the far field, formed in double and
        // rounded once: no cancellation against the node's deviations
        const long long r = (long long)y * ref.pitch + x;
        drr = C(ref.rho[r] - rho_ff);
        dur = C(ref.ux[r] - uxf);
        dvr = C(ref.uy[r] - uyf);
      }
      const C dr = m[0] - drr, du = m[1] - dur, dv = m[2] - dvr;
      const C rho = rho0 + m[0], ux = u0 + m[1], uy = v0 + m[2];
      ++count;
      k0.add(m[0]);
      k1.add(e_rho * dr * dr + e_u * (du * du + dv * dv));
      k2.add(C(0.5) * rho * (ux * ux + uy * uy));
      bad += (isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]) && rho > C(0)) ? 0 : 1;
    }
    s[0] += k0.value();
    s[1] += k1.value();
    s[2] += k2.value();
  }
  const double sums[4] = {(double)count * rho_ff + s[0], s[1], s[2], (double)bad};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double t = block_sum<NT>(sums[c], smem);
    if (threadIdx.x == 0) partials[blockIdx.x * 4 + c] = t;
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) reduce_finish(const double* __restrict__ partials, int nblocks,
                                                    double* __restrict__ out) {
  __shared__ double smem[NT / 32];
  for (int c = 0; c < 4; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += NT) s += partials[b * 4 + c];
    const double t = block_sum<NT>(s, smem);
    if (threadIdx.x == 0) out[c] = t;
  }
}

}  // namespace lbmk

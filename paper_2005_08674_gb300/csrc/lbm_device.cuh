// lbm_device.cuh -- device-side building blocks of the D2Q9 + NSBC update
// for sm_103a: storage traits (shifted populations in f64/f32/f16/bf16 with
// 16-byte vector access), the BGK cell update, and the NSBC node update.
//
// Populations are stored as h_i = f_i - w_i (deviation from the rest state),
// so rho = 1 + sum h_i and rho u = sum c_i h_i (sum c_i w_i = 0).  The
// equilibrium in the same shift is
//   h_i^eq = f_i^eq - w_i = w_i (d_rho + rho (3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u))
// which is Eq. (feq_1) with cs^2 = 1/3 minus w_i.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_check.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
// Lattice (Fig. 1): c_0=(0,0) c_1=(1,0) c_2=(-1,0) c_3=(0,1) c_4=(0,-1)
// c_5=(1,1) c_6=(-1,-1) c_7=(-1,1) c_8=(1,-1); w = 4/9, 1/9, 1/36.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 2 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return i == 3 || i == 5 || i == 7 ? 1 : (i == 4 || i == 6 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1); }
template <typename C>
__host__ __device__ constexpr C wt(int i) {
  return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}

// ---------------------------------------------------------------------------
// Storage traits: compute type C, cells per 16-byte vector V, vector and
// scalar loads (streaming: every population is read once per step) and
// stores.  16-bit types round to nearest even on store.
// ---------------------------------------------------------------------------
template <typename T>
struct Store;

template <>
struct Store<double> {
  using C = double;
  static constexpr int V = 2;
  __device__ static void ld(const double* p, C (&o)[V]) {
    if (!in_bounds(p, 16)) {
      o[0] = o[1] = 0.0;
      return;
    }
    const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    o[0] = t.x;
    o[1] = t.y;
  }
  __device__ static void st(double* p, const C (&o)[V]) {
    if (!in_bounds(p, 16)) return;
    __stcs(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
  }
  static constexpr double kScale = 1.0;
  // shared-memory copies of the stored values (tiles staged by bulk copies)
  __device__ static void lds(const double* p, C (&o)[V]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    o[0] = t.x;
    o[1] = t.y;
  }
  __device__ static C ld1s(const double* p) { return *p; }
  __device__ static C ld1(const double* p) { return in_bounds(p, 8) ? __ldcs(p) : 0.0; }
  __device__ static C ldg1(const double* p) { return in_bounds(p, 8) ? __ldg(p) : 0.0; }
  __device__ static void st1(double* p, C v) {
    if (in_bounds(p, 8)) *p = v;
  }
  __device__ static void st1r(double* p, C v) {
    if (in_bounds(p, 8)) *p = v;
  }
  __device__ static double cvt(C v) { return v; }
};

template <>
struct Store<float> {
  using C = float;
  static constexpr int V = 4;
  __device__ static void ld(const float* p, C (&o)[V]) {
    if (!in_bounds(p, 16)) {
      o[0] = o[1] = o[2] = o[3] = 0.f;
      return;
    }
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
  }
  __device__ static void st(float* p, const C (&o)[V]) {
    if (!in_bounds(p, 16)) return;
    __stcs(reinterpret_cast<float4*>(p), make_float4(o[0], o[1], o[2], o[3]));
  }
  static constexpr float kScale = 1.0f;
  __device__ static void lds(const float* p, C (&o)[V]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
  }
  __device__ static C ld1s(const float* p) { return *p; }
  __device__ static C ld1(const float* p) { return in_bounds(p, 4) ? __ldcs(p) : 0.f; }
  __device__ static C ldg1(const float* p) { return in_bounds(p, 4) ? __ldg(p) : 0.f; }
  __device__ static void st1(float* p, C v) {
    if (in_bounds(p, 4)) *p = v;
  }
  __device__ static void st1r(float* p, C v) {
    if (in_bounds(p, 4)) *p = v;
  }
  __device__ static float cvt(C v) { return v; }
};

// binary16 holds h_i * 2^12: acoustic deviations of 1e-7..1e-2 would fall
// into binary16's subnormal range (below 6.1e-5), where the absolute spacing
// 6e-8 is a large relative error; scaled by 2^12 they stay normal (down to
// 1.5e-8), and |h| up to 16 still fits.  A power of two scales exactly.
constexpr float kHalfScale = 4096.0f;
constexpr float kHalfUnscale = 1.0f / 4096.0f;

// ld / st / ld1 / st1r move STORED values (s * h, s = kScale) and are used by
// the bulk kernel, whose collision works in stored units; ldg1 / st1 / cvt
// convert to and from h itself for the boundary and the helper kernels.
template <>
struct Store<__half> {
  using C = float;
  static constexpr int V = 8;
  static constexpr float kScale = kHalfScale;
  __device__ static void ld(const __half* p, C (&o)[V]) {
    if (!in_bounds(p, 16)) {
#pragma unroll
      for (int k = 0; k < V; ++k) o[k] = 0.f;
      return;
    }
    const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 h2;
      memcpy(&h2, &w[k], 4);
      const float2 f = __half22float2(h2);
      o[2 * k] = f.x;
      o[2 * k + 1] = f.y;
    }
  }
  __device__ static void st(__half* p, const C (&o)[V]) {
    if (!in_bounds(p, 16)) return;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __half2 h2 = __floats2half2_rn(o[2 * k], o[2 * k + 1]);
      memcpy(&w[k], &h2, 4);
    }
    __stcs(reinterpret_cast<uint4*>(p), make_uint4(w[0], w[1], w[2], w[3]));
  }
  __device__ static void lds(const __half* p, C (&o)[V]) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __half2 h2;
      memcpy(&h2, &w[k], 4);
      const float2 f = __half22float2(h2);
      o[2 * k] = f.x;
      o[2 * k + 1] = f.y;
    }
  }
  __device__ static C ld1s(const __half* p) { return __half2float(*p); }
  // half vectors (4 nodes, 8 bytes): shared-memory load and streaming store
  __device__ static void ldsp(const __half* p, C (&o)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    __half2 a, b;
    memcpy(&a, &t.x, 4);
    memcpy(&b, &t.y, 4);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    o[0] = fa.x;
    o[1] = fa.y;
    o[2] = fb.x;
    o[3] = fb.y;
  }
  __device__ static void stp(__half* p, const C (&o)[4]) {
    if (!in_bounds(p, 8)) return;
    const __half2 a = __floats2half2_rn(o[0], o[1]), b = __floats2half2_rn(o[2], o[3]);
    uint2 t;
    memcpy(&t.x, &a, 4);
    memcpy(&t.y, &b, 4);
    __stcs(reinterpret_cast<uint2*>(p), t);
  }
  __device__ static C ld1(const __half* p) { return in_bounds(p, 2) ? __half2float(*p) : 0.f; }
  __device__ static void st1r(__half* p, C v) {
    if (in_bounds(p, 2)) *p = __float2half_rn(v);
  }
  __device__ static C ldg1(const __half* p) {
    return in_bounds(p, 2) ? __half2float(__ldg(p)) * kHalfUnscale : 0.f;
  }
  __device__ static void st1(__half* p, C v) {
    if (in_bounds(p, 2)) *p = __float2half_rn(v * kHalfScale);
  }
  __device__ static __half cvt(C v) { return __float2half_rn(v * kHalfScale); }
};

template <>
struct Store<__nv_bfloat16> {
  using C = float;
  static constexpr int V = 8;
  __device__ static void ld(const __nv_bfloat16* p, C (&o)[V]) {
    if (!in_bounds(p, 16)) {
#pragma unroll
      for (int k = 0; k < V; ++k) o[k] = 0.f;
      return;
    }
    const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __nv_bfloat162 b2;
      memcpy(&b2, &w[k], 4);
      const float2 f = __bfloat1622float2(b2);
      o[2 * k] = f.x;
      o[2 * k + 1] = f.y;
    }
  }
  __device__ static void st(__nv_bfloat16* p, const C (&o)[V]) {
    if (!in_bounds(p, 16)) return;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(o[2 * k], o[2 * k + 1]);
      memcpy(&w[k], &b2, 4);
    }
    __stcs(reinterpret_cast<uint4*>(p), make_uint4(w[0], w[1], w[2], w[3]));
  }
  static constexpr float kScale = 1.0f;
  __device__ static void lds(const __nv_bfloat16* p, C (&o)[V]) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __nv_bfloat162 b2;
      memcpy(&b2, &w[k], 4);
      const float2 f = __bfloat1622float2(b2);
      o[2 * k] = f.x;
      o[2 * k + 1] = f.y;
    }
  }
  __device__ static C ld1s(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ static void ldsp(const __nv_bfloat16* p, C (&o)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    __nv_bfloat162 a, b;
    memcpy(&a, &t.x, 4);
    memcpy(&b, &t.y, 4);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    o[0] = fa.x;
    o[1] = fa.y;
    o[2] = fb.x;
    o[3] = fb.y;
  }
  __device__ static void stp(__nv_bfloat16* p, const C (&o)[4]) {
    if (!in_bounds(p, 8)) return;
    const __nv_bfloat162 a = __floats2bfloat162_rn(o[0], o[1]), b = __floats2bfloat162_rn(o[2], o[3]);
    uint2 t;
    memcpy(&t.x, &a, 4);
    memcpy(&t.y, &b, 4);
    __stcs(reinterpret_cast<uint2*>(p), t);
  }
  __device__ static C ld1(const __nv_bfloat16* p) { return in_bounds(p, 2) ? __bfloat162float(*p) : 0.f; }
  __device__ static C ldg1(const __nv_bfloat16* p) { return in_bounds(p, 2) ? __bfloat162float(__ldg(p)) : 0.f; }
  __device__ static void st1(__nv_bfloat16* p, C v) {
    if (in_bounds(p, 2)) *p = __float2bfloat16_rn(v);
  }
  __device__ static void st1r(__nv_bfloat16* p, C v) {
    if (in_bounds(p, 2)) *p = __float2bfloat16_rn(v);
  }
  __device__ static __nv_bfloat16 cvt(C v) { return __float2bfloat16_rn(v); }
};

// Bulk-copy-engine prefetch of [p, p + bytes) into L2 (16-byte aligned,
// bytes a multiple of 16); no registers or shared memory are tied up.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  if (!in_bounds(p, bytes)) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------
// Moments of shifted populations (Eqs. cf_0, cf_1 as discrete sums).
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ void moments(const C (&h)[9], C& drho, C& jx, C& jy) {
  drho = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
  jx = (h[1] - h[2]) + (h[5] - h[6]) + (h[8] - h[7]);
  jy = (h[3] - h[4]) + (h[5] - h[6]) + (h[7] - h[8]);
}

// Shifted equilibrium h^eq_i at (d_rho, u), Eq. (feq_1) minus w_i, times the
// storage scale s (1 except for binary16 storage, where it folds into w_i).
template <typename C>
__device__ __forceinline__ void equilibrium(C drho, C ux, C uy, C (&e)[9], C s = C(1)) {
  const C rho = C(1) + drho;
  const C usq = C(1.5) * (ux * ux + uy * uy);
  const C w0 = wt<C>(0) * s, wa = wt<C>(1) * s, wd = wt<C>(5) * s;
  e[0] = w0 * (drho - rho * usq);
  // axis directions: c.u = +-ux, +-uy
  {
    const C a = C(4.5) * ux * ux - usq, b = C(3) * ux;
    e[1] = wa * (drho + rho * (a + b));
    e[2] = wa * (drho + rho * (a - b));
  }
  {
    const C a = C(4.5) * uy * uy - usq, b = C(3) * uy;
    e[3] = wa * (drho + rho * (a + b));
    e[4] = wa * (drho + rho * (a - b));
  }
  {
    const C s = ux + uy;  // c_5 = -c_6 = (1, 1)
    const C a = C(4.5) * s * s - usq, b = C(3) * s;
    e[5] = wd * (drho + rho * (a + b));
    e[6] = wd * (drho + rho * (a - b));
  }
  {
    const C d = uy - ux;  // c_7 = -c_8 = (-1, 1)
    const C a = C(4.5) * d * d - usq, b = C(3) * d;
    e[7] = wd * (drho + rho * (a + b));
    e[8] = wd * (drho + rho * (a - b));
  }
}

// Storage shift.  A stored population is h_i = f_i - f_i^eq(m0) (times the
// storage scale), m0 = (rho0, u0) the far field, so that with a mean flow the
// stored numbers stay as small as the disturbance instead of carrying the
// stream's equilibrium (a 16-bit storage keeps its relative precision for
// what changes); for a far field at rest h_i = f_i - w_i.  The step kernels
// compute in deviations from m0 as well (d = rho - rho0, v = u - u0,
// equilibrium_dev), which needs P_i(u0), u0 and rho0; sh_i = f_i^eq(m0) - w_i
// converts to and from absolute populations outside the step.
template <typename C>
struct Shift {
  C sh[9];        // f_i^eq(m0) - w_i
  C p0[9];        // P_i(u0) = 1 + 3 c_i.u0 + 4.5 (c_i.u0)^2 - 1.5 u0.u0
  C u0[2];        // u0
  C rho0;         // rho0
  double m0[3];   // (rho0, u0x, u0y) in double
  bool on;        // false: far field at rest (rho0 = 1, u0 = 0)
};

// The shift of far field m0 = (rho0, u0x, u0y), formed in double on the host
// (the same expression as equilibrium() below, with rho0 - 1 kept apart).
// Defined once, in lbm_runtime.cu: a host compiler that fuses multiply-adds
// could otherwise round an inline copy differently in each file, and the
// single-domain and batched paths must start from the same bits.
Shift<double> far_field_shift(const double m0[3]);

template <typename C>
__host__ __device__ inline Shift<C> shift_as(const Shift<double>& z) {
  Shift<C> o;
  for (int i = 0; i < 9; ++i) o.sh[i] = C(z.sh[i]);
  for (int i = 0; i < 9; ++i) o.p0[i] = C(z.p0[i]);
  o.u0[0] = C(z.u0[0]);
  o.u0[1] = C(z.u0[1]);
  o.rho0 = C(z.rho0);
  for (int c = 0; c < 3; ++c) o.m0[c] = z.m0[c];
  o.on = z.on;
  return o;
}

// Relaxation rates, and the storage shift the collision needs.
template <typename C>
struct Rates {
  C omega;         // BGK rate 1/tau, also the MRT stress rate omega_nu
  C s_e, s_eps, s_q;
  Shift<C> z;
};

// a * b + c rounded once, in every kernel alike (the shift terms multiply
// loop-invariant values, and a compiler left free to hoist the product in one
// kernel and fuse it in another would round them differently).
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
// a - b rounded on its own (never fused with a product that formed a)
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
// a * b rounded on its own (never fused into a later add)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// a / rho for the velocity u = (rho u) / rho: in float the fast division
// intrinsic (within 2 ulp for rho in the normal range; rho is near 1 here),
// an IEEE division in double (the parity mode).
__device__ __forceinline__ float div_rho(float a, float rho) { return __fdividef(a, rho); }
__device__ __forceinline__ double div_rho(double a, double rho) { return a / rho; }

// The interior collision's arithmetic, every operation rounded on its own
// (none fused by the compiler), on one node (float, double) or on two nodes
// at once (float2: the paired FP32 instructions of sm_100 and later, whose
// components round exactly as the scalar __fadd_rn / __fmul_rn / __fmaf_rn
// do).  The same sequence of operations therefore gives the same bits for a
// node whether it is collided alone or beside another.
__device__ __forceinline__ float v_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double v_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float2 v_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float v_neg(float a) { return -a; }
__device__ __forceinline__ double v_neg(double a) { return -a; }
__device__ __forceinline__ float2 v_neg(float2 a) { return make_float2(-a.x, -a.y); }
template <typename V>
__device__ __forceinline__ V v_sub(V a, V b) {
  return v_add(a, v_neg(b));  // a - b = a + (-b), rounded once
}
__device__ __forceinline__ float v_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double v_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float2 v_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float v_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double v_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 v_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <typename V, typename C>
__device__ __forceinline__ V v_splat(C c) {
  if constexpr (std::is_same<V, float2>::value)
    return make_float2(c, c);
  else
    return V(c);
}
__device__ __forceinline__ float v_div_rho(float a, float rho) { return div_rho(a, rho); }
__device__ __forceinline__ double v_div_rho(double a, double rho) { return div_rho(a, rho); }
__device__ __forceinline__ float2 v_div_rho(float a, float2 rho) {
  return make_float2(div_rho(a, rho.x), div_rho(a, rho.y));
}
// the moments' sums (as moments() forms them) in this arithmetic
template <typename V>
__device__ __forceinline__ void v_moments(const V (&h)[9], V& drho, V& jx, V& jy) {
  drho = v_add(v_add(v_add(v_add(h[0], h[1]), v_add(h[2], h[3])), v_add(v_add(h[4], h[5]), v_add(h[6], h[7]))),
               h[8]);
  const V a = v_sub(h[5], h[6]);
  jx = v_add(v_add(v_sub(h[1], h[2]), a), v_sub(h[8], h[7]));
  jy = v_add(v_add(v_sub(h[3], h[4]), a), v_sub(h[7], h[8]));
}

// Equilibrium in deviations from the far field: E_i = f_i^eq(rho, u) -
// f_i^eq(rho0, u0) (Eq. feq_1 at two states, cs^2 = 1/3) times the weight
// scale ws, from d = rho - rho0, v = u - u0 and the momentum deviation
// J = rho v (= rho u - rho0 u0 - d u0).  With
//   P_i(u) = 1 + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u   (so f_i^eq = w_i rho P_i(u)),
//   E_i = w_i [ d P_i(u0) + 3 c_i.J + rho Q_i ],
//   Q_i = 4.5 (c_i.v)(c_i.s) - 1.5 v.s,   s = u + u0 = 2 u0 + v,
// (rho (P_i(u) - P_i(u0)) = 3 c_i.J + rho Q_i), every term is of the size of
// the disturbance, so float rounding is relative to it even in a mean flow:
// forming f^eq(rho, u) and subtracting f^eq(m0) instead rounds terms of the
// size of the stream's equilibrium (0.04 per population at Ma 0.1) every
// step, and in a steady flow those roundings -- which do not conserve mass or
// momentum -- add up step after step.  The first-order term takes J as summed
// from the populations, not rho times a rounded quotient, so the momentum a
// BGK relaxation puts back is the node's own to the rounding of each term.
// For a far field at rest (SHIFT false: rho0 = 1, u0 = 0, P_i(u0) = 1) this
// is w_i (d + 3 c_i.J + rho (4.5 (c_i.u)^2 - 1.5 u.u)).
template <bool SHIFT, typename V, typename C>
__device__ __forceinline__ void equilibrium_dev(V d, V vx, V vy, V jx, V jy, const Shift<C>& z, V (&e)[9],
                                                C ws = C(1)) {
  // every operation is rounded on its own (v_add / v_mul / v_fma), so that
  // the shifted form with a zero shift (rho0 = 1, u0 = 0, P_i(u0) = 1) rounds
  // exactly like the plain one, and two nodes at once like one at a time
  V rho, sx, sy;
  if constexpr (SHIFT) {
    rho = v_add(v_splat<V>(z.rho0), d);
    sx = v_fma(v_splat<V>(C(2)), v_splat<V>(z.u0[0]), vx);
    sy = v_fma(v_splat<V>(C(2)), v_splat<V>(z.u0[1]), vy);
  } else {
    rho = v_add(v_splat<V>(C(1)), d);
    sx = vx;
    sy = vy;
  }
  V dp[9];  // d P_i(u0)
#pragma unroll
  for (int i = 0; i < 9; ++i) dp[i] = SHIFT ? v_mul(d, v_splat<V>(z.p0[i])) : d;
  const V vs = v_mul(v_splat<V>(C(1.5)), v_fma(vx, sx, v_mul(vy, sy)));
  const V nvs = v_neg(vs);
  const V w0 = v_splat<V>(wt<C>(0) * ws), wa = v_splat<V>(wt<C>(1) * ws), wd = v_splat<V>(wt<C>(5) * ws);
  const V c45 = v_splat<V>(C(4.5)), c3 = v_splat<V>(C(3));
  e[0] = v_mul(w0, v_fma(v_neg(rho), vs, dp[0]));
  // axis directions: c.v = +-vx, +-vy
  {
    const V q = v_fma(v_mul(c45, vx), sx, nvs), b = v_mul(c3, jx);
    e[1] = v_mul(wa, v_add(v_fma(rho, q, dp[1]), b));
    e[2] = v_mul(wa, v_sub(v_fma(rho, q, dp[2]), b));
  }
  {
    const V q = v_fma(v_mul(c45, vy), sy, nvs), b = v_mul(c3, jy);
    e[3] = v_mul(wa, v_add(v_fma(rho, q, dp[3]), b));
    e[4] = v_mul(wa, v_sub(v_fma(rho, q, dp[4]), b));
  }
  {
    const V cv = v_add(vx, vy), cs = v_add(sx, sy);  // c_5 = -c_6 = (1, 1)
    const V q = v_fma(v_mul(c45, cv), cs, nvs), b = v_mul(c3, v_add(jx, jy));
    e[5] = v_mul(wd, v_add(v_fma(rho, q, dp[5]), b));
    e[6] = v_mul(wd, v_sub(v_fma(rho, q, dp[6]), b));
  }
  {
    const V cv = v_sub(vy, vx), cs = v_sub(sy, sx);  // c_7 = -c_8 = (-1, 1)
    const V q = v_fma(v_mul(c45, cv), cs, nvs), b = v_mul(c3, v_sub(jy, jx));
    e[7] = v_mul(wd, v_add(v_fma(rho, q, dp[7]), b));
    e[8] = v_mul(wd, v_sub(v_fma(rho, q, dp[8]), b));
  }
}

// BGK collision, Eq. (lbe_1) with dt = 1, on shifted populations held as
// s * h (s = storage scale; the relaxation is linear in h, only the moments
// need 1/s).  Written as h* = (1 - omega) h + omega h^eq with omega folded
// into the equilibrium weights: one fused multiply-add per population.
// With a storage shift (SHIFT: a far field not at rest) the velocity enters
// as its deviation v = u - u0 = (sum c h - d u0) / rho and the equilibrium as
// its deviation from f^eq(m0) (equilibrium_dev), so no term of the size of
// the stream's equilibrium is ever rounded.  The relaxation is one explicitly
// rounded fused multiply-add per population in both forms, and the shifted
// form with a zero shift gives the same bits as the plain one.
template <bool SHIFT, typename V, typename C>
__device__ __forceinline__ void collide_bgk(V (&h)[9], const Rates<C>& r, C s = C(1)) {
  const C omega = r.omega;
  V sd, sjx, sjy;
  v_moments(h, sd, sjx, sjy);
  const C is = C(1) / s;
  const V vis = v_splat<V>(is);
  const V d = v_mul(sd, vis);  // rho - rho0
  V e[9];
  if constexpr (SHIFT) {
    // J = rho (u - u0) = sum c h - d u0 and v = J / rho, from small quantities only
    const V inv = v_div_rho(is, v_add(v_splat<V>(r.z.rho0), d));
    const V nsd = v_neg(sd);
    const V jx = v_fma(nsd, v_splat<V>(r.z.u0[0]), sjx), jy = v_fma(nsd, v_splat<V>(r.z.u0[1]), sjy);
    equilibrium_dev<true>(d, v_mul(jx, inv), v_mul(jy, inv), v_mul(jx, vis), v_mul(jy, vis), r.z, e, s * omega);
  } else {
    const V inv = v_div_rho(is, v_add(v_splat<V>(C(1)), d));
    equilibrium_dev<false>(d, v_mul(sjx, inv), v_mul(sjy, inv), v_mul(sjx, vis), v_mul(sjy, vis), r.z, e,
                           s * omega);
  }
  const V keep = v_splat<V>(C(1) - omega);
#pragma unroll
  for (int i = 0; i < 9; ++i) h[i] = v_fma(keep, h[i], e[i]);
}

// ---------------------------------------------------------------------------
// MRT collision, Eq. (mrt_lbe): f* = f - M^-1 S (m - m^eq), with the
// Gram-Schmidt moment basis of Sec. 4 in the order of Eq. (mrt_rm):
// (rho, e, eps, jx, qx, jy, qy, pxx, pxy).  Rows scaled to integers:
//   e   = (-4, -1, -1, -1, -1,  2,  2,  2,  2)   |e|^2   = 36
//   eps = ( 4, -2, -2, -2, -2,  1,  1,  1,  1)   |eps|^2 = 36
//   qx  = ( 0, -2,  2,  0,  0,  1, -1, -1,  1)   |qx|^2  = 12
//   qy  = ( 0,  0,  0, -2,  2,  1, -1,  1, -1)   |qy|^2  = 12
//   pxx = ( 0,  1,  1, -1, -1,  0,  0,  0,  0)   |pxx|^2 = 4
//   pxy = ( 0,  0,  0,  0,  0,  1,  1, -1, -1)   |pxy|^2 = 4
// The rows are orthogonal, so M^-1 = M^T diag(1/|row|^2); a row scale does
// not change M^-1 S M.  The conserved moments of f - f^eq vanish, so their
// rates (C_rho, C_jx, C_jy) never enter.  The stress rate is 1/tau.
// ---------------------------------------------------------------------------

template <bool SHIFT, typename C>
__device__ __forceinline__ void collide_mrt(C (&h)[9], const Rates<C>& r, C s = C(1)) {
  C sd, sjx, sjy;
  moments(h, sd, sjx, sjy);
  const C is = C(1) / s;
  const C dr = sd * is;  // rho - rho0
  C e[9];
  if constexpr (SHIFT) {
    const C inv = div_rho(is, r.z.rho0 + dr);
    const C jx = fma_rn(-sd, r.z.u0[0], sjx), jy = fma_rn(-sd, r.z.u0[1], sjy);
    equilibrium_dev<true>(dr, jx * inv, jy * inv, jx * is, jy * is, r.z, e, s);
  } else {
    const C inv = div_rho(is, C(1) + dr);
    equilibrium_dev<false>(dr, sjx * inv, sjy * inv, sjx * is, sjy * is, r.z, e, s);
  }
  C n[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) n[i] = sub_rn(h[i], e[i]);
  const C ax = n[1] + n[2], ay = n[3] + n[4], d = (n[5] + n[6]) + (n[7] + n[8]);
  const C me = C(-4) * n[0] - (ax + ay) + C(2) * d;
  const C mep = C(4) * n[0] - C(2) * (ax + ay) + d;
  const C mqx = C(-2) * (n[1] - n[2]) + ((n[5] - n[6]) + (n[8] - n[7]));
  const C mqy = C(-2) * (n[3] - n[4]) + ((n[5] - n[6]) + (n[7] - n[8]));
  const C mxx = ax - ay;
  const C mxy = (n[5] + n[6]) - (n[7] + n[8]);
  const C re = r.s_e * me * C(1.0 / 36.0), rep = r.s_eps * mep * C(1.0 / 36.0);
  const C rqx = r.s_q * mqx * C(1.0 / 12.0), rqy = r.s_q * mqy * C(1.0 / 12.0);
  const C rxx = r.omega * mxx * C(0.25), rxy = r.omega * mxy * C(0.25);
  const C a0 = C(-1) * re - C(2) * rep;  // e/eps part of the axis columns
  const C a1 = C(2) * re + rep;          // e/eps part of the diagonal columns
  h[0] -= C(4) * (rep - re);
  h[1] -= a0 - C(2) * rqx + rxx;
  h[2] -= a0 + C(2) * rqx + rxx;
  h[3] -= a0 - C(2) * rqy - rxx;
  h[4] -= a0 + C(2) * rqy - rxx;
  h[5] -= a1 + rqx + rqy + rxy;
  h[6] -= a1 - rqx - rqy + rxy;
  h[7] -= a1 - rqx + rqy - rxy;
  h[8] -= a1 + rqx - rqy - rxy;
}

// Collision model: 0 = BGK (Eq. lbe_1), 1 = MRT (Eq. mrt_lbe).
template <int MODEL, bool SHIFT, typename C>
__device__ __forceinline__ void collide(C (&h)[9], const Rates<C>& r, C s = C(1)) {
  if constexpr (MODEL == 1)
    collide_mrt<SHIFT>(h, r, s);
  else
    collide_bgk<SHIFT>(h, r, s);
}

// The collision of N nodes held as h[i][k] (population i of node k): with
// PAIRED, in float BGK, two nodes per paired instruction (half the
// arithmetic instructions, at the price of register pairs: worth it where
// the kernel is bound by instruction issue and has registers to spare),
// otherwise one after another; the bits of each node are those of collide()
// on it alone either way.
template <int MODEL, bool SHIFT, bool PAIRED, typename C, int N>
__device__ __forceinline__ void collide_nodes(C (&h)[9][N], const Rates<C>& r, C s = C(1)) {
  if constexpr (PAIRED && MODEL == 0 && std::is_same<C, float>::value && N % 2 == 0) {
#pragma unroll
    for (int k = 0; k < N; k += 2) {
      float2 p[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) p[i] = make_float2(h[i][k], h[i][k + 1]);
      collide_bgk<SHIFT>(p, r, s);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        h[i][k] = p[i].x;
        h[i][k + 1] = p[i].y;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      C n[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) n[i] = h[i][k];
      collide<MODEL, SHIFT>(n, r, s);
#pragma unroll
      for (int i = 0; i < 9; ++i) h[i][k] = n[i];
    }
  }
}

// ---------------------------------------------------------------------------
// Geometry and NSBC parameters passed by value to the kernels.
// ---------------------------------------------------------------------------
struct Geom {
  int nx, ny, pitch;
  long long plane;  // elements between population planes
};

struct Nsbc {
  double gamma, beta, kappa;
  double m0[3];  // far-field (rho, ux, uy)
  int order;     // 1 or 2
  int corner;    // corner reading: 0 diagonal normal, 1 mean of the two edges' m_c
  int periodic_x, periodic_y;  // axes closed periodically instead of by NSBC edges
  int vel[4];                  // edges (left, right, bottom, top) with a prescribed velocity
  double uw[4][2];             // that velocity
};

// Node k of the perimeter (k < 2 nx + 2 (ny - 2)) -> coordinates and outward
// normal.  Order: bottom row, top row, left column, right column (corners
// belong to the rows).
__device__ __forceinline__ void perimeter_node(int k, int nx, int ny, int& x, int& y, int& nxn, int& nyn) {
  if (k < 2 * nx) {
    const bool top = k >= nx;
    x = top ? k - nx : k;
    y = top ? ny - 1 : 0;
    nyn = top ? 1 : -1;
    nxn = x == 0 ? -1 : (x == nx - 1 ? 1 : 0);
  } else {
    k -= 2 * nx;
    const bool right = k >= ny - 2;
    y = 1 + (right ? k - (ny - 2) : k);
    x = right ? nx - 1 : 0;
    nxn = right ? 1 : -1;
    nyn = 0;
  }
}

// Deviations (rho - rho0, u - u0) from the far field at node (x, y) of the
// stored state, in the compute type of the storage: float for f32 / f16 /
// bf16 (the shifted populations keep them free of cancellation, so float
// loses nothing the storage kept), double in the f64 parity mode.
template <typename T>
__device__ __forceinline__ void node_dmoments(const T* __restrict__ A, const Geom& g, int x, int y,
                                              const Shift<typename Store<T>::C>& z, typename Store<T>::C (&m)[3]) {
  using S = Store<T>;
  using C = typename S::C;
  const long long o = (long long)y * g.pitch + x;
  C h[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) h[i] = S::ldg1(A + i * g.plane + o);
  C d, jx, jy;
  moments(h, d, jx, jy);
  const C inv = div_rho(C(1), z.rho0 + d);
  m[0] = d;
  m[1] = fma_rn(-d, z.u0[0], jx) * inv;
  m[2] = fma_rn(-d, z.u0[1], jy) * inv;
}

// Deviations (rho - rho0, u - u0) from the far field of a node's shifted
// populations (physical units) in the compute type of the storage: every
// quantity is of the size of the disturbance, so float is exact to float
// rounding of the perturbation.  For a far field at rest (SHIFT false) they
// are (rho - 1, u).
template <bool SHIFT, typename C>
__device__ __forceinline__ void dmoments_of(const C (&h)[9], C rho0, C u0x, C u0y, C (&m)[3]) {
  C d, jx, jy;
  moments(h, d, jx, jy);
  m[0] = d;
  if constexpr (SHIFT) {
    const C inv = C(1) / (rho0 + d);
    m[1] = fma_rn(-d, u0x, jx) * inv;
    m[2] = fma_rn(-d, u0y, jy) * inv;
  } else {
    const C inv = C(1) / (C(1) + d);
    m[1] = jx * inv;
    m[2] = jy * inv;
  }
}

}  // namespace lbmk

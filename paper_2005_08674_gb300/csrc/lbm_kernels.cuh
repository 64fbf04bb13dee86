// lbm_kernels.cuh -- the sm_103a kernels of one D2Q9 + NSBC time step (the
// initialisation, macroscopic-field and reduction kernels are in
// lbm_aux.cuh).
//
//   bulk_kernel  : fused pull-stream (Eq. lbe_0) + collide (BGK, Eq. lbe_1,
//                  or MRT, Eq. mrt_lbe)
//                  over interior nodes, 16-byte vector loads/stores along x,
//                  x-1 / x+1 neighbours exchanged with warp shuffles.
//   fused_step_kernel : both in one launch (perimeter blocks first).
//   nsbc_kernel  : the boundary of Sec. 5 on every edge and corner node:
//                  gradient prediction (Eq. nes_2) with one-sided differences
//                  whose points are loaded by neighbouring lanes and gathered
//                  with warp shuffles, far-field blend (Eq. nes_3), mirror of
//                  the outgoing non-equilibrium part (Eqs. nes_0, nes_1),
//                  conservation correction (Eq. nes_4), then the ordinary
//                  collision.
// Both read buffer A (step n) and write disjoint nodes of buffer B (step
// n+1), so they may run concurrently.
#pragma once

#include "lbm_device.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
// Bulk: interior rows 1..ny-2; each thread owns V consecutive cells of a row
// segment (V = 16 bytes / sizeof(T)), blocks of BX threads cover BX*V cells
// of `rows` consecutive rows.  Only nodes 1..nx-2 are stored.
// ---------------------------------------------------------------------------
// Bytes of one warp's row segment (32 lanes x V nodes) starting at warp_x0,
// clipped to the row pitch, for the L2 prefetch.
template <typename T>
__device__ __forceinline__ unsigned warp_segment_bytes(const Geom& g, int warp_x0) {
  return (unsigned)(min(32 * Store<T>::V, g.pitch - warp_x0) * (int)sizeof(T)) & ~15u;
}

// Interior nodes x0..x0+V-1 of row y for this lane.  Every lane of the warp
// must call this (shuffles).  Lanes normally share y and hold consecutive
// vectors; a lane may also sit on the next row (the batched kernel flattens
// rows): the neighbour value it then gets from the shuffle belongs to a node
// it never stores (x = 0 or x = nx - 1), so it is harmless.  `valid` = false
// makes the lane load and store nothing.  L2 prefetch distance pf in rows
// (0 = off, only with a row shared by the warp): lane 0 asks the bulk-copy
// engine to pull the warp's segments of row y + pf into L2, so more bytes
// are in flight than the registers of the resident warps hold.
template <typename T, int MODEL, bool SHIFT = false>
__device__ __forceinline__ void bulk_row(const T* __restrict__ A, T* __restrict__ B, const Geom& g,
                                         const Rates<typename Store<T>::C>& rates, int y, int x0, int lane,
                                         int pf, unsigned pf_bytes, bool valid = true) {
  using S = Store<T>;
  using C = typename S::C;
  constexpr int V = S::V;
  const bool active = valid && x0 < g.nx;
  const long long P = g.plane;
  const int warp_x0 = x0 - lane * V;
  {
    const long long r0 = (long long)y * g.pitch + x0;
    const long long rm = r0 - g.pitch, rp = r0 + g.pitch;
    if (pf > 0 && lane == 0 && warp_x0 < g.nx && y + pf <= g.ny - 2 && pf_bytes > 0) {
      const long long q0 = (long long)(y + pf) * g.pitch + warp_x0;
      const long long qm = q0 - g.pitch, qp = q0 + g.pitch;
      prefetch_l2(A + 0 * P + q0, pf_bytes);
      prefetch_l2(A + 1 * P + q0, pf_bytes);
      prefetch_l2(A + 2 * P + q0, pf_bytes);
      prefetch_l2(A + 3 * P + qm, pf_bytes);
      prefetch_l2(A + 4 * P + qp, pf_bytes);
      prefetch_l2(A + 5 * P + qm, pf_bytes);
      prefetch_l2(A + 6 * P + qp, pf_bytes);
      prefetch_l2(A + 7 * P + qm, pf_bytes);
      prefetch_l2(A + 8 * P + qp, pf_bytes);
    }
    C v[9][V];
    if (active) {
      S::ld(A + 0 * P + r0, v[0]);
      S::ld(A + 1 * P + r0, v[1]);
      S::ld(A + 2 * P + r0, v[2]);
      S::ld(A + 3 * P + rm, v[3]);
      S::ld(A + 4 * P + rp, v[4]);
      S::ld(A + 5 * P + rm, v[5]);
      S::ld(A + 6 * P + rp, v[6]);
      S::ld(A + 7 * P + rm, v[7]);
      S::ld(A + 8 * P + rp, v[8]);
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int k = 0; k < V; ++k) v[i][k] = C(0);
    }
    // values at x0-1 for the directions pulled from the left (1, 5, 8) and
    // at x0+V for those pulled from the right (2, 6, 7): from the
    // neighbouring lane, or a scalar load at the warp's ends.
    C l1 = __shfl_up_sync(0xffffffffu, v[1][V - 1], 1);
    C l5 = __shfl_up_sync(0xffffffffu, v[5][V - 1], 1);
    C l8 = __shfl_up_sync(0xffffffffu, v[8][V - 1], 1);
    C r2 = __shfl_down_sync(0xffffffffu, v[2][0], 1);
    C r6 = __shfl_down_sync(0xffffffffu, v[6][0], 1);
    C r7 = __shfl_down_sync(0xffffffffu, v[7][0], 1);
    if (lane == 0 && active && x0 > 0) {
      l1 = S::ld1(A + 1 * P + r0 - 1);
      l5 = S::ld1(A + 5 * P + rm - 1);
      l8 = S::ld1(A + 8 * P + rp - 1);
    }
    if (lane == 31 && active && x0 + V < g.nx) {
      r2 = S::ld1(A + 2 * P + r0 + V);
      r6 = S::ld1(A + 6 * P + rp + V);
      r7 = S::ld1(A + 7 * P + rm + V);
    }
    C o[9][V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      o[0][k] = v[0][k];
      o[1][k] = k == 0 ? l1 : v[1][k - 1];
      o[2][k] = k == V - 1 ? r2 : v[2][k + 1];
      o[3][k] = v[3][k];
      o[4][k] = v[4][k];
      o[5][k] = k == 0 ? l5 : v[5][k - 1];
      o[6][k] = k == V - 1 ? r6 : v[6][k + 1];
      o[7][k] = k == V - 1 ? r7 : v[7][k + 1];
      o[8][k] = k == 0 ? l8 : v[8][k - 1];
    }
    collide_nodes<MODEL, SHIFT, false>(o, rates, C(S::kScale));  // in stored units
    if (active) {
      if (x0 >= 1 && x0 + V <= g.nx - 1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) S::st(B + i * P + r0, o[i]);
      } else {
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const int x = x0 + k;
          if (x >= 1 && x <= g.nx - 2) {
#pragma unroll
            for (int i = 0; i < 9; ++i) S::st1r(B + i * P + r0 + k, o[i][k]);
          }
        }
      }
    }
  }
}

template <typename T, int BX, int MODEL, bool SHIFT = false>
__global__ void __launch_bounds__(BX) bulk_kernel(const T* __restrict__ A, T* __restrict__ B, Geom g,
                                                  Rates<typename Store<T>::C> rates, int rows, int pf) {
  constexpr int V = Store<T>::V;
  const int lane = threadIdx.x & 31;
  const int x0 = (blockIdx.x * BX + threadIdx.x) * V;
  const int y_begin = 1 + blockIdx.y * rows;
  const int y_end = min(y_begin + rows, g.ny - 1);
  const unsigned pf_bytes = warp_segment_bytes<T>(g, x0 - lane * V);
  for (int y = y_begin; y < y_end; ++y) bulk_row<T, MODEL, SHIFT>(A, B, g, rates, y, x0, lane, pf, pf_bytes);
}

// ---------------------------------------------------------------------------
// NSBC.  The moments are formed in the compute type at b, b - n and
// (second-order difference) b - 2n as deviations (rho - rho0, u - u0) from
// the far field m0; m_c is predicted and blended in double (Eqs. nes_2 and
// nes_3 are linear, so predicting the deviation is predicting m, and the
// blend towards m0 scales the deviation by 1 - beta); the node is then
// rebuilt, corrected and collided in the compute type.
// ---------------------------------------------------------------------------
// Perimeter node `node`: coordinates and outward normal (zero along a
// periodic axis, which has no boundary there).
struct EdgeNode {
  int x, y, nxn, nyn;
  bool open;  // an NSBC / velocity edge node (not closed periodically)
};

__device__ __forceinline__ EdgeNode edge_node(int node, const Geom& g, const Nsbc& p) {
  EdgeNode e;
  perimeter_node(node, g.nx, g.ny, e.x, e.y, e.nxn, e.nyn);
  if (p.periodic_x) e.nxn = 0;
  if (p.periodic_y) e.nyn = 0;
  e.open = e.nxn != 0 || e.nyn != 0;
  return e;
}

// Where the boundary code reads the state it updates and writes the result:
// population i of node (x, y), in physical units (the storage scale undone).
// GlobalSrc / GlobalDst address a population buffer in device memory; other
// sources (rows staged in shared memory) provide the same two calls.
template <typename T>
struct GlobalSrc {
  const T* __restrict__ a;
  long long plane;
  int pitch;
  __device__ __forceinline__ typename Store<T>::C ld(int i, int x, int y) const {
    return Store<T>::ldg1(a + i * plane + (long long)y * pitch + x);
  }
};
template <typename T>
struct GlobalDst {
  T* __restrict__ b;
  long long plane;
  int pitch;
  __device__ __forceinline__ void st(int i, int x, int y, typename Store<T>::C v) const {
    Store<T>::st1(b + i * plane + (long long)y * pitch + x, v);
  }
};

// The NSBC finish runs on all four lanes of a quad: lane q owns one opposite
// pair of populations, q = 0: (1, 2), c = (1, 0); q = 1: (3, 4), c = (0, 1);
// q = 2: (5, 6), c = (1, 1); q = 3: (7, 8), c = (-1, 1) (Fig. 1 numbering),
// and every lane carries population 0 (lane 0 stores it).  The lanes run the
// same instructions on their own pair, and node sums over the nine
// populations are quad reductions.
struct QuadPair {
  int ip, im;  // the populations along c and along -c
  int cx, cy;  // c
  bool diag;
};

__device__ __forceinline__ QuadPair quad_pair(int q) {
  QuadPair r;
  r.ip = 1 + 2 * q;
  r.im = 2 + 2 * q;
  r.cx = q == 1 ? 0 : (q == 3 ? -1 : 1);
  r.cy = q == 0 ? 0 : 1;
  r.diag = q >= 2;
  return r;
}

// Sum of v over the four lanes of the quad, the same bits in every lane.
template <typename C>
__device__ __forceinline__ C quad_sum(C v, unsigned quad) {
  v = v + __shfl_xor_sync(quad, v, 1, 4);
  return v + __shfl_xor_sync(quad, v, 2, 4);
}

// This lane's pulled populations of the node: h+ (along c) from x - c, h-
// (along -c) from x + c, h0 from x; unknown (and zero) where the source lies
// outside the domain, wrapped on periodic axes.
template <typename T, typename Src>
__device__ __forceinline__ void quad_pull(const Src& A, const Geom& g, const Nsbc& p, const EdgeNode& e,
                                          const QuadPair& pr, typename Store<T>::C& hp, typename Store<T>::C& hm,
                                          typename Store<T>::C& h0, bool& kp, bool& km) {
  using C = typename Store<T>::C;
  auto pull = [&](int i, int sx, int sy, bool& known) -> C {
    if (p.periodic_x) sx = sx < 0 ? sx + g.nx : (sx >= g.nx ? sx - g.nx : sx);
    if (p.periodic_y) sy = sy < 0 ? sy + g.ny : (sy >= g.ny ? sy - g.ny : sy);
    known = sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny;
    return known ? A.ld(i, sx, sy) : C(0);
  };
  hp = pull(pr.ip, e.x - pr.cx, e.y - pr.cy, kp);
  hm = pull(pr.im, e.x + pr.cx, e.y + pr.cy, km);
  h0 = A.ld(0, e.x, e.y);
}

// Equilibrium deviations (as equilibrium_dev) of this lane's pair and of
// population 0, times ws.
template <bool SHIFT, typename C>
__device__ __forceinline__ void pair_equilibrium(const QuadPair& pr, int q, C d, C vx, C vy, C jx, C jy,
                                                 const Shift<C>& z, C ws, C& ep, C& em, C& e0) {
  C rho, sx, sy, dpp, dpm, dp0;
  if constexpr (SHIFT) {
    rho = z.rho0 + d;
    sx = fma_rn(C(2), z.u0[0], vx);
    sy = fma_rn(C(2), z.u0[1], vy);
    const C p0p = q == 0 ? z.p0[1] : (q == 1 ? z.p0[3] : (q == 2 ? z.p0[5] : z.p0[7]));  // static indices only
    const C p0m = q == 0 ? z.p0[2] : (q == 1 ? z.p0[4] : (q == 2 ? z.p0[6] : z.p0[8]));
    dpp = mul_rn(d, p0p);
    dpm = mul_rn(d, p0m);
    dp0 = mul_rn(d, z.p0[0]);
  } else {
    rho = C(1) + d;
    sx = vx;
    sy = vy;
    dpp = dpm = dp0 = d;
  }
  const C vs = C(1.5) * fma_rn(vx, sx, mul_rn(vy, sy));
  const C fx = C(pr.cx), fy = C(pr.cy);
  const C cv = fma_rn(fx, vx, mul_rn(fy, vy)), cs = fma_rn(fx, sx, mul_rn(fy, sy));
  const C cj = fma_rn(fx, jx, mul_rn(fy, jy));
  const C a = fma_rn(C(4.5) * cv, cs, -vs), b = C(3) * cj;
  const C w = (pr.diag ? wt<C>(5) : wt<C>(1)) * ws;
  ep = w * (fma_rn(rho, a, dpp) + b);
  em = w * (fma_rn(rho, a, dpm) - b);
  e0 = (wt<C>(0) * ws) * fma_rn(-rho, vs, dp0);
}

// d = rho - rho0 and J = rho (u - u0) of the node from the quad's pairs.
template <bool SHIFT, typename C>
__device__ __forceinline__ void pair_moments(const QuadPair& pr, C hp, C hm, C h0, const Shift<C>& z, unsigned quad,
                                             C& d, C& jx, C& jy) {
  const C odd = hp - hm;
  d = h0 + quad_sum(hp + hm, quad);
  jx = quad_sum(C(pr.cx) * odd, quad);
  jy = quad_sum(C(pr.cy) * odd, quad);
  (void)z;
}

// The collision (BGK, Eq. lbe_1, or MRT, Eq. mrt_lbe) of the node, each lane
// relaxing its own pair (and population 0), in physical units.
template <int MODEL, bool SHIFT, typename C>
__device__ __forceinline__ void pair_collide(const QuadPair& pr, int q, C& hp, C& hm, C& h0, const Rates<C>& r,
                                             unsigned quad) {
  C d, sjx, sjy;
  pair_moments<SHIFT>(pr, hp, hm, h0, r.z, quad, d, sjx, sjy);
  C jx = sjx, jy = sjy, inv;
  if constexpr (SHIFT) {
    inv = div_rho(C(1), r.z.rho0 + d);
    jx = fma_rn(-d, r.z.u0[0], sjx);
    jy = fma_rn(-d, r.z.u0[1], sjy);
  } else {
    inv = div_rho(C(1), C(1) + d);
  }
  C ep, em, e0;
  if constexpr (MODEL == 1) {
    pair_equilibrium<SHIFT>(pr, q, d, jx * inv, jy * inv, jx, jy, r.z, C(1), ep, em, e0);
    // non-equilibrium moments of Eq. mrt_rm (rows as in collide_mrt): each
    // lane's share, summed over the quad
    const C np = sub_rn(hp, ep), nm = sub_rn(hm, em), n0 = sub_rn(h0, e0);
    const C even = np + nm, oddn = np - nm;
    const C ce = pr.diag ? C(2) : C(-1), cep = pr.diag ? C(1) : C(-2), cq = pr.diag ? C(1) : C(-2);
    const C cxx = C(pr.cx * pr.cx - pr.cy * pr.cy), cxy = C(pr.cx * pr.cy);
    const C me = fma_rn(C(-4), n0, quad_sum(ce * even, quad));
    const C mep = fma_rn(C(4), n0, quad_sum(cep * even, quad));
    const C mqx = quad_sum(cq * C(pr.cx) * oddn, quad), mqy = quad_sum(cq * C(pr.cy) * oddn, quad);
    const C mxx = quad_sum(cxx * even, quad), mxy = quad_sum(cxy * even, quad);
    const C re = r.s_e * me * C(1.0 / 36.0), rep = r.s_eps * mep * C(1.0 / 36.0);
    const C rqx = r.s_q * mqx * C(1.0 / 12.0), rqy = r.s_q * mqy * C(1.0 / 12.0);
    const C rxx = r.omega * mxx * C(0.25), rxy = r.omega * mxy * C(0.25);
    const C base = ce * re + cep * rep;
    const C odd = cq * (C(pr.cx) * rqx + C(pr.cy) * rqy);
    const C stress = cxx * rxx + cxy * rxy;
    h0 -= C(4) * (rep - re);
    hp -= (base + odd) + stress;
    hm -= (base - odd) + stress;
  } else {
    const C omega = r.omega, keep = C(1) - omega;
    pair_equilibrium<SHIFT>(pr, q, d, jx * inv, jy * inv, jx, jy, r.z, omega, ep, em, e0);
    hp = fma_rn(keep, hp, ep);
    hm = fma_rn(keep, hm, em);
    h0 = fma_rn(keep, h0, e0);
  }
}

// Eq. (nes_2): m_p = m_b - gamma d_n m, d_n along the outward unit normal by
// the one-sided difference of the given order (1 / |n| = 1/sqrt(2) along a
// corner's diagonal); Eq. (nes_3): m_c = (1 - beta) m_p + beta m_0, which
// for the deviation m - m_0 is (1 - beta) (m_p - m_0).  Component c of the
// deviation (rho - rho0, u - u0) from its values at b, b - n, b - 2n, in FP64
// with every rounding explicit (no contraction left to the compiler), so that
// every caller gets the same bits.  GB300's FP64 divide is slow: no divides.
// The settings Eqs. nes_2 and nes_3 use, and the far field in the compute
// type: small values passed by value (also to the out-of-line corner pass,
// where a reference would move the caller's structures to local memory).
struct Predict {
  double gamma, beta;
  int order;
};
template <typename C>
struct Far {
  C rho0, u0x, u0y;
};
__device__ __forceinline__ Predict predict_of(const Nsbc& p) { return Predict{p.gamma, p.beta, p.order}; }
template <typename C>
__device__ __forceinline__ Far<C> far_of(const Shift<C>& z) { return Far<C>{z.rho0, z.u0[0], z.u0[1]}; }

template <typename C>
__device__ __forceinline__ double edge_predict(C vb, C v1, C v2, bool diagonal, Predict p) {
  const double mb = (double)vb, m1 = (double)v1, m2 = (double)v2;
  const double inv_len = diagonal ? 0.70710678118654752 : 1.0;
  const double dn = p.order == 2 ? __dmul_rn(__fma_rn(3.0, mb, __fma_rn(-4.0, m1, m2)), 0.5 * inv_len)
                                 : __dmul_rn(__dsub_rn(mb, m1), inv_len);
  const double mp = __fma_rn(-p.gamma, dn, mb);
  return __dmul_rn(1.0 - p.beta, mp);
}

// Lane q of a quad: the deviations (rho - rho0, u - u0) of node b - q n (zeros for
// lanes beyond the difference order), transposed across the quad so that
// lane c (c < 3) gets component c at b, b - n, b - 2n, predicted and blended
// in FP64 by edge_predict.  All four lanes call this together.
template <typename T, bool SHIFT>
__device__ __forceinline__ double quad_predict(const typename Store<T>::C (&v)[9], Far<typename Store<T>::C> z,
                                               unsigned quad, int cq, bool diagonal, Predict p) {
  using C = typename Store<T>::C;
  C mq[3];
  dmoments_of<SHIFT>(v, z.rho0, z.u0x, z.u0y, mq);  // lanes that loaded nothing get unused values
  C t0[3], t1[3], t2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    t0[c] = __shfl_sync(quad, mq[c], 0, 4);
    t1[c] = __shfl_sync(quad, mq[c], 1, 4);
    t2[c] = __shfl_sync(quad, mq[c], 2, 4);
  }
  return edge_predict(cq == 0 ? t0[0] : (cq == 1 ? t0[1] : t0[2]), cq == 0 ? t1[0] : (cq == 1 ? t1[1] : t1[2]),
                      cq == 0 ? t2[0] : (cq == 1 ? t2[1] : t2[2]), diagonal, p);
}

// The populations of node (x, y), or zeros if !want.
template <typename T, typename Src>
__device__ __forceinline__ void load_node(const Src& A, int x, int y, bool want, typename Store<T>::C (&v)[9]) {
  using C = typename Store<T>::C;
#pragma unroll
  for (int i = 0; i < 9; ++i) v[i] = want ? A.ld(i, x, y) : C(0);
}

// The rest of the node, on all four lanes of its quad, given this lane's
// pulled pair and the blended deviation m_c - m0 = (rho_c - rho0, u_c - u0):
// velocity override, reconstruction of the unknown populations, correction,
// collision and the store.
template <typename T, int MODEL, bool SHIFT = false, typename Dst>
__device__ __forceinline__ void quad_finish(const Dst& B, const Geom& g, const Nsbc& p,
                                            const Rates<typename Store<T>::C>& rates, const EdgeNode& en,
                                            const QuadPair& pr, int q, unsigned quad, typename Store<T>::C hp,
                                            typename Store<T>::C hm, typename Store<T>::C h0, bool kp, bool km,
                                            typename Store<T>::C (&mc)[3], bool store) {
  using S = Store<T>;
  using C = typename S::C;
  const int x = en.x, y = en.y;
  if (en.open) {
    // a velocity edge keeps the predicted density and imposes its velocity
    // (left/right edges win at corners); its deviation u_w - u0 is formed in
    // double
    const int side = (x == 0 && p.vel[0])             ? 0
                     : (x == g.nx - 1 && p.vel[1])    ? 1
                     : (y == 0 && p.vel[2])           ? 2
                     : (y == g.ny - 1 && p.vel[3])    ? 3
                                                      : -1;
    if (side >= 0) {
      const double ux = side == 0 ? p.uw[0][0] : side == 1 ? p.uw[1][0] : side == 2 ? p.uw[2][0] : p.uw[3][0];
      const double uy = side == 0 ? p.uw[0][1] : side == 1 ? p.uw[1][1] : side == 2 ? p.uw[2][1] : p.uw[3][1];
      mc[1] = C(ux - p.m0[1]);
      mc[2] = C(uy - p.m0[2]);
    }

    // Eqs. (nes_0), (nes_1): f_in = f_in^eq(m_c) + f_out - f_out^eq(m_c)
    // (in stored deviations: f^eq(m_c) - f^eq(m0), the same relation); both
    // members of the pair are this lane's
    C ep, em, e0;
    {
      const C rho_c = (SHIFT ? rates.z.rho0 : C(1)) + mc[0];
      pair_equilibrium<SHIFT>(pr, q, mc[0], mc[1], mc[2], rho_c * mc[1], rho_c * mc[2], rates.z, C(1), ep, em, e0);
    }
    const C hp0 = hp, hm0 = hm;
    if (!kp) hp = km ? ep + (hm0 - em) : ep;
    if (!km) hm = kp ? em + (hp0 - ep) : em;

    // Eq. (nes_4): f_i -= w_i (d_rho + kappa c_i . d(rho u)), with the node's
    // moments and the targets (rho_c, rho_c u_c) both taken relative to m0:
    // rho_c u_c - rho0 u0 = rho_c (u_c - u0) + (rho_c - rho0) u0
    C drho, jx, jy;
    pair_moments<SHIFT>(pr, hp, hm, h0, rates.z, quad, drho, jx, jy);
    const C d_rho = drho - mc[0];
    C d_jx, d_jy;  // explicit multiply-adds: a zero shift rounds like the plain form
    if constexpr (SHIFT) {
      const C rho_c = rates.z.rho0 + mc[0];
      d_jx = fma_rn(-rho_c, mc[1], fma_rn(-mc[0], rates.z.u0[0], jx));
      d_jy = fma_rn(-rho_c, mc[2], fma_rn(-mc[0], rates.z.u0[1], jy));
    } else {
      const C rho_c = C(1) + mc[0];
      d_jx = fma_rn(-rho_c, mc[1], jx);
      d_jy = fma_rn(-rho_c, mc[2], jy);
    }
    const C t = C(p.kappa) * (C(pr.cx) * d_jx + C(pr.cy) * d_jy);
    const C w = pr.diag ? wt<C>(5) : wt<C>(1);
    hp -= w * (d_rho + t);
    hm -= w * (d_rho - t);
    h0 -= wt<C>(0) * d_rho;
  }

  pair_collide<MODEL, SHIFT>(pr, q, hp, hm, h0, rates, quad);
  if (store) {
    B.st(pr.ip, x, y, hp);
    B.st(pr.im, x, y, hm);
    if (q == 0) B.st(0, x, y, h0);
  }
}

// The second prediction of a corner under corner reading 1, along the
// horizontal edge's normal (0, nyn).  Kept out of line: only the quads that
// hold a corner call it, and inlined it would cost every NSBC node registers.
template <typename T, bool SHIFT, typename Src>
__device__ __noinline__ double corner_second_prediction(Src A, int x, int y, Far<typename Store<T>::C> z,
                                                        unsigned quad, int q, Predict p) {
  typename Store<T>::C w[9];
  load_node<T>(A, x, y, q <= p.order, w);
  return quad_predict<T, SHIFT>(w, z, quad, q < 3 ? q : 0, false, p);
}

// K perimeter nodes, each handled by the four lanes of one quad (q = lane &
// 3); all four lanes must call this together with the same nodes.  Lane q
// forms the deviations (rho - rho0, u - u0) at b - q n in the compute type; the quad then
// transposes them so that lane c (c < 3) holds component c at b, b - n,
// b - 2n and predicts and blends that component in FP64 -- three lanes share
// the FP64 work (GB300's FP64 pipe is narrow) -- and every lane gathers the
// three blended components and finishes its own pair of populations
// (quad_finish).  Every load of the K nodes is
// issued before the first is used (one round trip for all of them); nodes
// with valid[k] false are computed (from in-range addresses) but not stored.
// A corner under corner reading 1 is predicted twice, along the normals of
// the vertical edge (n = (nxn, 0)) and of the horizontal one (n = (0, nyn)),
// and gets the mean of the two blended states; the second pass runs only in
// the quads that hold a corner.
template <typename T, int MODEL, int K, bool SHIFT = false, typename Src, typename Dst>
__device__ __forceinline__ void nsbc_nodes(const Src& A, const Dst& B, const Geom& g, const Nsbc& p,
                                           const Rates<typename Store<T>::C>& rates, const int (&node)[K],
                                           const bool (&valid)[K], int q) {
  using S = Store<T>;
  using C = typename S::C;
  const unsigned quad = 0xFu << ((threadIdx.x & 31) & ~3);
  const QuadPair pr = quad_pair(q);
  EdgeNode en[K];
  C hp[K], hm[K], h0[K], v[K][9];
  bool kp[K], km[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    en[k] = edge_node(node[k], g, p);
    quad_pull<T>(A, g, p, en[k], pr, hp[k], hm[k], h0[k], kp[k], km[k]);  // this lane's pulled pair
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {  // lane q: the node b - q n (zeros if not needed)
    const bool split = p.corner == 1 && en[k].nxn != 0 && en[k].nyn != 0;
    const int ny1 = split ? 0 : en[k].nyn;  // a split corner: the vertical edge's normal first
    load_node<T>(A, en[k].x - q * en[k].nxn, en[k].y - q * ny1, en[k].open && q <= p.order, v[k]);
  }
  const int cq = q < 3 ? q : 0;
  C mc[K][3];  // (rho_c - rho0, u_c - u0)
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const bool corner = en[k].nxn != 0 && en[k].nyn != 0;
    const bool split = p.corner == 1 && corner;  // the same for all four lanes of the quad
    double mine = quad_predict<T, SHIFT>(v[k], far_of(rates.z), quad, cq, corner && !split, predict_of(p));
    if (split)
      mine = __dmul_rn(0.5, __dadd_rn(mine, corner_second_prediction<T, SHIFT>(A, en[k].x, en[k].y - q * en[k].nyn,
                                                                              far_of(rates.z), quad, q,
                                                                              predict_of(p))));
    const C mcq = C(mine);
#pragma unroll
    for (int c = 0; c < 3; ++c) mc[k][c] = __shfl_sync(quad, mcq, c, 4);
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    quad_finish<T, MODEL, SHIFT>(B, g, p, rates, en[k], pr, q, quad, hp[k], hm[k], h0[k], kp[k], km[k], mc[k],
                                 valid[k]);
}

template <typename T, int MODEL, bool SHIFT = false>
__device__ __forceinline__ void nsbc_node(const T* __restrict__ A, T* __restrict__ B, const Geom& g, const Nsbc& p,
                                          const Rates<typename Store<T>::C>& rates, int node, int q) {
  const int n[1] = {node};
  const bool ok[1] = {true};
  nsbc_nodes<T, MODEL, 1, SHIFT>(GlobalSrc<T>{A, g.plane, g.pitch}, GlobalDst<T>{B, g.plane, g.pitch}, g, p, rates,
                                 n, ok, q);
}

// One launch for the whole step (the "fused" form, for domains small enough
// that launch gaps dominate): the first n_edge blocks take the perimeter,
// one node per quad of lanes as in nsbc_kernel; the others are the blocks of
// bulk_kernel's (threads_x, rows) grid, numbered row-major with nbx blocks
// along x.  Same device functions, so the same bits as the kernel pair.
template <typename T, int BX, int MODEL, bool SHIFT = false>
__global__ void __launch_bounds__(BX) fused_step_kernel(const T* __restrict__ A, T* __restrict__ B, Geom g, Nsbc p,
                                                        Rates<typename Store<T>::C> rates, int rows, int pf, int n_edge,
                                                        int nbx) {
  constexpr int V = Store<T>::V;
  if ((int)blockIdx.x < n_edge) {
    const int t = blockIdx.x * BX + threadIdx.x;
    const int node = t >> 2, q = t & 3;
    if (node >= 2 * g.nx + 2 * (g.ny - 2)) return;  // a quad leaves together
    nsbc_node<T, MODEL, SHIFT>(A, B, g, p, rates, node, q);
    return;
  }
  const int k = (int)blockIdx.x - n_edge;
  const int bx = k % nbx, by = k / nbx;
  const int lane = threadIdx.x & 31;
  const int x0 = (bx * BX + threadIdx.x) * V;
  const int y_begin = 1 + by * rows;
  const int y_end = min(y_begin + rows, g.ny - 1);
  const unsigned pf_bytes = warp_segment_bytes<T>(g, x0 - lane * V);
  for (int y = y_begin; y < y_end; ++y) bulk_row<T, MODEL, SHIFT>(A, B, g, rates, y, x0, lane, pf, pf_bytes);
}

template <typename T, int MODEL, bool SHIFT = false>
__global__ void __launch_bounds__(128) nsbc_kernel(const T* __restrict__ A, T* __restrict__ B, Geom g, Nsbc p,
                                                   Rates<typename Store<T>::C> rates) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int node = t >> 2, q = t & 3;
  const int perim = 2 * g.nx + 2 * (g.ny - 2);
  if (node >= perim) return;  // a quad leaves together
  nsbc_node<T, MODEL, SHIFT>(A, B, g, p, rates, node, q);
}

}  // namespace lbmk

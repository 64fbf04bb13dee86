/*
 * lbm_oracle.c -- plain, slow, single-threaded FP64 reference solver for the
 * D2Q9 lattice-Boltzmann update closed by the Non-equilibrium Symmetry
 * Boundary Condition (NSBC) of Euser & Vuik (arXiv 2005.08674).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library; every constant below is written out here from the paper.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * x86_64 and aarch64 builds give identical bits).
 *
 * What each part follows:
 *   lattice table ............ Fig. 1 (velocity labels c_0..c_8, weights table)
 *   equilibrium .............. Eq. (feq_1): w_i rho (1 + u.c/cs^2 + (u.c)^2/(2cs^4) - u.u/(2cs^2)), cs = 1/sqrt(3)
 *   moments .................. Eqs. (cf_0), (cf_1) as discrete sums over the 9 populations
 *   stream ................... Eq. (lbe_0), pull form: g_i(x) = f_i(x - c_i)
 *   BGK collide .............. Eq. (lbe_1) with dt = 1
 *   MRT collide .............. Eqs. (mrt_lbe), (mrt_vm), (mrt_rm); M built by Gram-Schmidt
 *   NSBC ..................... Sec. 5: Eq. (nes_0)/(nes_1) mirror, Eq. (nes_2) gradient
 *                              prediction, Eq. (nes_3) far-field blend, Eq. (nes_4) correction,
 *                              then the ordinary collision at the boundary node.
 *   storage emulation ........ no counterpart in the paper: an optional rounding of the
 *                              stored populations through a narrower format (or_set_storage),
 *                              used by the tests to separate storage loss from arithmetic.
 *
 * Readings taken where the paper is silent or ambiguous (all selectable where
 * an alternative is plausible):
 *   - stored state: post-collision populations at step n; a step is
 *     pull-stream -> NSBC on edge nodes -> collide every node.
 *   - Eq. (nes_2): outward unit normal n, one-sided difference pointing into
 *     the domain, moments taken from the step-n state:
 *       order 1: d_n m = (m_b - m_{b-n}) / |n|
 *       order 2: d_n m = (3 m_b - 4 m_{b-n} + m_{b-2n}) / (2 |n|)
 *     Corner nodes (the paper says nothing about them) take one of two
 *     readings, chosen by corner_mode:
 *       0 (default): the diagonal normal, |n| = sqrt(2), one prediction;
 *       1: the mean of the two blended states m_c (Eq. nes_3) that the two
 *          edges meeting there would predict, each along its own unit normal.
 *   - m = (rho, u_x, u_y): density and velocity are predicted and blended,
 *     not momentum.
 *   - incoming = populations whose pull source lies outside the domain;
 *     outgoing = their opposites.  Both equilibria in Eq. (nes_1) are taken
 *     at m_c.  When the opposite is unknown too (a corner's diagonal pair),
 *     the incoming population is f^eq(m_c) alone.
 *   - Eq. (nes_4) is applied to all nine populations of the node with a
 *     momentum factor kappa: kappa = 3 = 1/cs^2 makes the corrected node carry
 *     exactly rho_c and rho_c u_c (the stated aim of the correction);
 *     kappa = 1 is the formula as printed.
 *
 * Parity pins: see the tests that exercise this file (lattice table against
 * Fig. 1, equilibrium moment identities, BGK relaxation rate, streaming
 * direction, shear-wave viscosity, sound speed, far-field invariance, exact
 * reconstruction under the symmetry assumption, moment prediction at the
 * edge, mirror symmetries, reflection ordering).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Fig. 1: c_0=(0,0), c_1=(1,0), c_2=(-1,0), c_3=(0,1), c_4=(0,-1),
 * c_5=(1,1), c_6=(-1,-1), c_7=(-1,1), c_8=(1,-1); w = 4/9, 1/9 (axis), 1/36 (diagonal). */
static const int CX[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
static const double WT[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* the direction pointing the opposite way: the j with c_j = -c_i */
static int opposite(int i) {
  for (int j = 0; j < 9; ++j)
    if (CX[j] == -CX[i] && CY[j] == -CY[i]) return j;
  return -1;
}

typedef struct or_sim {
  int nx, ny;
  double tau;
  double m0[3];       /* far-field reference vector (rho, ux, uy), Eq. (nes_3) */
  double gamma;       /* NSBC relaxation parameter, Eq. (nes_2) */
  double beta;        /* far-field factor, Eq. (nes_3) */
  double kappa;       /* momentum factor of the correction, Eq. (nes_4) */
  int grad_order;     /* 1 or 2: one-sided difference order for d_n m */
  int corner_mode;    /* 0: diagonal normal at corners; 1: mean of the two edges' m_c */
  int periodic[2];    /* periodic axes (x, y) instead of NSBC edges */
  int velocity[4];    /* edges (left, right, bottom, top) with a prescribed velocity */
  double uw[4][2];    /* that velocity */
  int collision;      /* 0 = BGK (Eq. lbe_1), 1 = MRT (Eq. mrt_lbe) */
  double mrt_s[9];    /* diagonal of S, Eq. (mrt_rm) */
  double M[9][9];     /* Gram-Schmidt moment matrix, Eq. (mrt_vm) */
  double Minv[9][9];
  double *f, *fn;     /* [9][ny][nx] post-collision populations, and the next buffer */
  long steps;
  int store_fmt;      /* storage emulation (test instrument): 0 off, 1 binary32, 2 binary16 x 2^12, 3 bfloat16 */
  int store_ff;       /* deviations stored from f^eq(m_0) (1) or from w_i (0) */
} or_sim;

#define F(s, buf, i, x, y) ((buf)[((size_t)(i) * (size_t)(s)->ny + (size_t)(y)) * (size_t)(s)->nx + (size_t)(x)])

/* Eq. (feq_1) with cs^2 = 1/3 */
void or_equilibrium(double rho, double ux, double uy, double feq[9]) {
  const double cs2 = 1.0 / 3.0;
  const double uu = ux * ux + uy * uy;
  for (int i = 0; i < 9; ++i) {
    const double cu = CX[i] * ux + CY[i] * uy;
    feq[i] = WT[i] * rho * (1.0 + cu / cs2 + (cu * cu) / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
  }
}

/* Eqs. (cf_0), (cf_1): rho = sum f_i, rho u = sum c_i f_i */
static void moments(const double g[9], double m[3]) {
  double rho = 0.0, jx = 0.0, jy = 0.0;
  for (int i = 0; i < 9; ++i) {
    rho += g[i];
    jx += CX[i] * g[i];
    jy += CY[i] * g[i];
  }
  m[0] = rho;
  m[1] = jx / rho;
  m[2] = jy / rho;
}

static void node_moments(const or_sim* s, int x, int y, double m[3]) {
  double g[9];
  for (int i = 0; i < 9; ++i) g[i] = F(s, s->f, i, x, y);
  moments(g, m);
}

/* Eq. (lbe_1), dt = 1 */
static void collide_bgk(const or_sim* s, double g[9]) {
  double m[3], feq[9];
  moments(g, m);
  or_equilibrium(m[0], m[1], m[2], feq);
  for (int i = 0; i < 9; ++i) g[i] = g[i] - (g[i] - feq[i]) / s->tau;
}

/* Eq. (mrt_lbe): f* = f - M^-1 S (m - m_eq), m = M f, m_eq = M f_eq */
static void collide_mrt(const or_sim* s, double g[9]) {
  double mac[3], feq[9], m[9], meq[9], r[9];
  moments(g, mac);
  or_equilibrium(mac[0], mac[1], mac[2], feq);
  for (int a = 0; a < 9; ++a) {
    m[a] = 0.0;
    meq[a] = 0.0;
    for (int i = 0; i < 9; ++i) {
      m[a] += s->M[a][i] * g[i];
      meq[a] += s->M[a][i] * feq[i];
    }
    r[a] = s->mrt_s[a] * (m[a] - meq[a]);
  }
  for (int i = 0; i < 9; ++i) {
    double d = 0.0;
    for (int a = 0; a < 9; ++a) d += s->Minv[i][a] * r[a];
    g[i] -= d;
  }
}

/* Eqs. (nes_2), (nes_3) at node (x, y) for the outward normal (nxn, nyn):
 * m_p = m - gamma d_n m with a one-sided difference into the domain, then
 * the far-field criterion m_c = (1 - beta) m_p + beta m_0. */
static void predict_blend(const or_sim* s, int x, int y, int nxn, int nyn, double mc[3]) {
  const double len = sqrt((double)(nxn * nxn + nyn * nyn));
  double mb[3], m1[3], m2[3], mp[3];
  node_moments(s, x, y, mb);
  node_moments(s, x - nxn, y - nyn, m1);
  if (s->grad_order == 2) node_moments(s, x - 2 * nxn, y - 2 * nyn, m2);
  for (int c = 0; c < 3; ++c) {
    double dn;
    if (s->grad_order == 2)
      dn = (3.0 * mb[c] - 4.0 * m1[c] + m2[c]) / (2.0 * len);
    else
      dn = (mb[c] - m1[c]) / len;
    mp[c] = mb[c] - s->gamma * dn;
  }
  for (int c = 0; c < 3; ++c) mc[c] = (1.0 - s->beta) * mp[c] + s->beta * s->m0[c];
}

/* Sec. 5: fill the unknown populations of edge node (x, y), then correct. */
static void nsbc(const or_sim* s, int x, int y, double g[9], const int known[9]) {
  int nxn = 0, nyn = 0; /* outward normal */
  if (!s->periodic[0]) {
    if (x == 0) nxn = -1;
    else if (x == s->nx - 1) nxn = 1;
  }
  if (!s->periodic[1]) {
    if (y == 0) nyn = -1;
    else if (y == s->ny - 1) nyn = 1;
  }

  double mc[3];
  if (s->corner_mode == 1 && nxn != 0 && nyn != 0) {
    /* a corner: the mean of what the vertical and the horizontal edge predict */
    double mx[3], my[3];
    predict_blend(s, x, y, nxn, 0, mx);
    predict_blend(s, x, y, 0, nyn, my);
    for (int c = 0; c < 3; ++c) mc[c] = 0.5 * (mx[c] + my[c]);
  } else {
    predict_blend(s, x, y, nxn, nyn, mc);
  }

  /* A velocity (Dirichlet) edge: the paper only cites its scheme.  Reading
   * taken: the same reconstruction with the velocity of m_c replaced by the
   * prescribed one (density still predicted), so after the correction the
   * node carries exactly that velocity.  At a corner the left/right edge's
   * velocity wins over the bottom/top one. */
  {
    int side = -1;
    if (x == 0 && s->velocity[0]) side = 0;
    else if (x == s->nx - 1 && s->velocity[1]) side = 1;
    else if (y == 0 && s->velocity[2]) side = 2;
    else if (y == s->ny - 1 && s->velocity[3]) side = 3;
    if (side >= 0) {
      mc[1] = s->uw[side][0];
      mc[2] = s->uw[side][1];
    }
  }

  /* Eqs. (nes_0), (nes_1): f_in = f_in^eq + f_out^neq, both equilibria at m_c */
  double feq[9];
  or_equilibrium(mc[0], mc[1], mc[2], feq);
  for (int i = 0; i < 9; ++i) {
    if (known[i]) continue;
    const int o = opposite(i);
    if (known[o])
      g[i] = feq[i] + (g[o] - feq[o]);
    else
      g[i] = feq[i];
  }

  /* Eq. (nes_4): conservation correction towards rho_c, rho_c u_c */
  double rho = 0.0, jx = 0.0, jy = 0.0;
  for (int i = 0; i < 9; ++i) {
    rho += g[i];
    jx += CX[i] * g[i];
    jy += CY[i] * g[i];
  }
  const double drho = rho - mc[0];
  const double djx = jx - mc[0] * mc[1];
  const double djy = jy - mc[0] * mc[2];
  for (int i = 0; i < 9; ++i) g[i] -= WT[i] * (drho + s->kappa * (CX[i] * djx + CY[i] * djy));
}

/* Gram-Schmidt moment basis for MRT (Sec. 4): orthogonalise the monomial
 * moments 1, e, eps, jx, qx, jy, qy, pxx, pxy in the plain (unweighted) inner
 * product over the 9 directions, in the order of the diagonal of S in
 * Eq. (mrt_rm).  Seed monomials: 1, |c|^2, |c|^4, cx, cx|c|^2, cy, cy|c|^2,
 * cx^2 - cy^2, cx cy. */
static void build_mrt_basis(or_sim* s) {
  double seed[9][9];
  for (int i = 0; i < 9; ++i) {
    const double cx = CX[i], cy = CY[i], c2 = cx * cx + cy * cy;
    seed[0][i] = 1.0;
    seed[1][i] = c2;
    seed[2][i] = c2 * c2;
    seed[3][i] = cx;
    seed[4][i] = cx * c2;
    seed[5][i] = cy;
    seed[6][i] = cy * c2;
    seed[7][i] = cx * cx - cy * cy;
    seed[8][i] = cx * cy;
  }
  for (int a = 0; a < 9; ++a) {
    double v[9];
    for (int i = 0; i < 9; ++i) v[i] = seed[a][i];
    for (int b = 0; b < a; ++b) {
      double num = 0.0, den = 0.0;
      for (int i = 0; i < 9; ++i) {
        num += seed[a][i] * s->M[b][i];
        den += s->M[b][i] * s->M[b][i];
      }
      for (int i = 0; i < 9; ++i) v[i] -= num / den * s->M[b][i];
    }
    for (int i = 0; i < 9; ++i) s->M[a][i] = v[i];
  }
  /* rows are mutually orthogonal: M^-1 = M^T diag(1/|row|^2) */
  for (int a = 0; a < 9; ++a) {
    double n2 = 0.0;
    for (int i = 0; i < 9; ++i) n2 += s->M[a][i] * s->M[a][i];
    for (int i = 0; i < 9; ++i) s->Minv[i][a] = s->M[a][i] / n2;
  }
}

or_sim* or_create(int nx, int ny, double tau, double rho_ff, double ux_ff, double uy_ff) {
  if (nx < 3 || ny < 3 || !(tau > 0.5)) return NULL;
  or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
  if (!s) return NULL;
  s->nx = nx;
  s->ny = ny;
  s->tau = tau;
  s->m0[0] = rho_ff;
  s->m0[1] = ux_ff;
  s->m0[2] = uy_ff;
  s->gamma = 0.6; /* Sec. 5: best value found for D2Q9 */
  s->beta = 0.0;  /* the paper's experiments use f_f = 0 */
  s->kappa = 3.0;
  s->grad_order = 1;
  s->collision = 0;
  build_mrt_basis(s);
  for (int a = 0; a < 9; ++a) s->mrt_s[a] = 1.0 / tau;
  const size_t n = (size_t)9 * (size_t)nx * (size_t)ny;
  s->f = (double*)calloc(n, sizeof(double));
  s->fn = (double*)calloc(n, sizeof(double));
  if (!s->f || !s->fn) {
    free(s->f);
    free(s->fn);
    free(s);
    return NULL;
  }
  return s;
}

void or_destroy(or_sim* s) {
  if (!s) return;
  free(s->f);
  free(s->fn);
  free(s);
}

void or_set_nsbc(or_sim* s, double gamma, double beta, double kappa, int grad_order) {
  s->gamma = gamma;
  s->beta = beta;
  s->kappa = kappa;
  s->grad_order = grad_order == 2 ? 2 : 1;
}

/* corner reading: 0 diagonal normal, 1 mean of the two adjacent edges' m_c */
void or_set_corner_mode(or_sim* s, int mode) { s->corner_mode = mode == 1 ? 1 : 0; }

void or_set_periodic(or_sim* s, int px, int py) {
  s->periodic[0] = px != 0;
  s->periodic[1] = py != 0;
}

/* side: 0 left (x = 0), 1 right, 2 bottom (y = 0), 3 top; on = 0 restores NSBC */
void or_set_velocity_edge(or_sim* s, int side, int on, double ux, double uy) {
  if (side < 0 || side > 3) return;
  s->velocity[side] = on != 0;
  s->uw[side][0] = ux;
  s->uw[side][1] = uy;
}

/* collision = 0: BGK; collision = 1: MRT with the diagonal s[9] of Eq. (mrt_rm) */
void or_set_collision(or_sim* s, int collision, const double* srates) {
  s->collision = collision;
  if (collision == 1 && srates)
    for (int a = 0; a < 9; ++a) s->mrt_s[a] = srates[a];
}

void or_mrt_matrix(const or_sim* s, double* M) {
  for (int a = 0; a < 9; ++a)
    for (int i = 0; i < 9; ++i) M[a * 9 + i] = s->M[a][i];
}

/* Storage emulation -- a test instrument, off unless or_set_storage is called.
 * It models only what keeping the populations in a narrower format loses:
 * after the initialisation and after every step each population f_i is
 * replaced by r_i + q(f_i - r_i), with r_i = f_i^eq(m_0) (store_ff = 1) or
 * w_i (store_ff = 0) and q rounding to nearest, ties to even, through
 * binary32 (format 1), binary16 holding the value times 2^12 (format 2) or
 * bfloat16 (format 3; the binary32 value's upper half, rounded).  The 16-bit
 * formats are reached through binary32, as a device computing in float would
 * reach them.  Everything in between stays double. */
static double q_store(double v, int fmt) {
  if (fmt == 1) return (double)(float)v;
  if (fmt == 2) return (double)(_Float16)(float)(v * 4096.0) / 4096.0;
  if (fmt == 3) {
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    if ((b & 0x7f800000u) != 0x7f800000u) { /* finite: round the lower half away, ties to even */
      b += 0x7fffu + ((b >> 16) & 1u);
      b &= 0xffff0000u;
    }
    memcpy(&f, &b, sizeof f);
    return (double)f;
  }
  return v;
}

static void apply_storage(const or_sim* s, double* buf) {
  if (!s->store_fmt) return;
  double r[9];
  if (s->store_ff)
    or_equilibrium(s->m0[0], s->m0[1], s->m0[2], r);
  else
    for (int i = 0; i < 9; ++i) r[i] = WT[i];
  /* every value is rounded on its own; the OpenMP build splits rows over
   * threads without changing any result bit */
  for (int i = 0; i < 9; ++i) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) F(s, buf, i, x, y) = r[i] + q_store(F(s, buf, i, x, y) - r[i], s->store_fmt);
  }
}

void or_set_storage(or_sim* s, int format, int far_field_shift) {
  s->store_fmt = format;
  s->store_ff = far_field_shift;
  apply_storage(s, s->f);
}

/* f := f^eq(rho, u) at every node; fields are [ny][nx], x fastest */
void or_init(or_sim* s, const double* rho, const double* ux, const double* uy) {
  double feq[9];
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      const size_t k = (size_t)y * s->nx + x;
      or_equilibrium(rho[k], ux[k], uy[k], feq);
      for (int i = 0; i < 9; ++i) F(s, s->f, i, x, y) = feq[i];
    }
  apply_storage(s, s->f);
  s->steps = 0;
}

void or_set_f(or_sim* s, const double* f) {
  memcpy(s->f, f, sizeof(double) * 9 * (size_t)s->nx * s->ny);
}

void or_get_f(const or_sim* s, double* f) {
  memcpy(f, s->f, sizeof(double) * 9 * (size_t)s->nx * s->ny);
}

void or_macros(const or_sim* s, double* rho, double* ux, double* uy) {
  double m[3];
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      node_moments(s, x, y, m);
      const size_t k = (size_t)y * s->nx + x;
      rho[k] = m[0];
      ux[k] = m[1];
      uy[k] = m[2];
    }
}

/* Eq. (lbe_0) streaming, Sec. 5 boundary, Eq. (lbe_1)/(mrt_lbe) collision */
void or_step(or_sim* s, int n) {
  for (int k = 0; k < n; ++k) {
    /* rows are independent within a step; the OpenMP build splits them over
     * threads without changing any result bit */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        double g[9];
        int known[9], unknown = 0;
        for (int i = 0; i < 9; ++i) {
          int sx = x - CX[i], sy = y - CY[i];
          if (s->periodic[0]) sx = (sx + s->nx) % s->nx;
          if (s->periodic[1]) sy = (sy + s->ny) % s->ny;
          if (sx >= 0 && sx < s->nx && sy >= 0 && sy < s->ny) {
            g[i] = F(s, s->f, i, sx, sy);
            known[i] = 1;
          } else {
            g[i] = 0.0;
            known[i] = 0;
            ++unknown;
          }
        }
        if (unknown) nsbc(s, x, y, g, known);
        if (s->collision == 1)
          collide_mrt(s, g);
        else
          collide_bgk(s, g);
        for (int i = 0; i < 9; ++i) F(s, s->fn, i, x, y) = g[i];
      }
    apply_storage(s, s->fn);
    double* t = s->f;
    s->f = s->fn;
    s->fn = t;
    ++s->steps;
  }
}

long or_steps(const or_sim* s) { return s->steps; }

/* the lattice table as used here, for the test against Fig. 1 */
void or_lattice(int* cx, int* cy, double* w, int* opp) {
  for (int i = 0; i < 9; ++i) {
    cx[i] = CX[i];
    cy[i] = CY[i];
    w[i] = WT[i];
    opp[i] = opposite(i);
  }
}

/*
 * vpath_oracle.c -- plain FP64 CPU oracle of the biased-Langevin trial
 * generator and of the bias functional of the variational pathway scheme
 * (arXiv:1405.6104).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a stand-alone shared
 * library that only the tests, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py load.  It shares no source, header, table or helper with
 * the CUDA library: everything here is written out from the paper and from
 * the published definitions it relies on, slowly and in the order the method
 * states it.
 *
 * What it computes (one trial):
 *   - Langevin equations of motion for solute X and solvent Y (Eq. Lang),
 *     integrated with BAOAB (the paper does not name its integrator);
 *   - the potential U(X,Y): Lennard-Jones with Lorentz-Berthelot mixing,
 *     shifted to zero at the cut-off, plus reaction-field electrostatics,
 *     harmonic bonds and harmonic angles (stand-in for the paper's
 *     AMBER99SB-ILDN/TIP3P force field, Sec. "Results");
 *   - the contact-map reaction coordinate z(X) (SM, "Collective coordinate"):
 *     z = sum_{i<j, j-i>s} [C~_ij(X) - C~_ij(X_native)]^2 with
 *     C(r) = (1-(r/r0)^6)/(1-(r/r0)^10), smoothly switched off between
 *     r_s and r_c^cv;
 *   - the ratchet-and-pawl bias (Eq. VR): F_i = -(k_R/2) (z - z_m) grad_i z
 *     when z > z_m, else 0, with z_m the running minimum of z (z_m(0)=z(X_0));
 *   - the bias functional (Eq. VMDcondition):
 *     Phi = int dt sum_{i in solute} |F_i^bias|^2 / (gamma_i m_i),
 *     right-endpoint rectangle rule over the force evaluations.
 *   - the Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     SC'11) and Box-Muller normals for the white noise eta of Eq. Lang.
 *   - the Verlet-list membership rule, restated in IEEE single precision
 *     (this decision is taken in FP32 by the kernels; see or_pairlist).
 *
 * Units: nm, ps, amu, kJ/mol, e, K.
 *
 * Build: cc -O2 -fopenmp -ffp-contract=off -shared -fPIC (the list rule
 * takes its two fused steps from fmaf and relies on no other contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_KB 0.0083144626        /* Boltzmann constant, kJ/mol/K */
#define OR_FCOUL 138.935458       /* 1/(4 pi eps0), kJ mol^-1 nm e^-2 */
#define OR_MAX_EXCL 32

/* ------------------------------------------------------------------------ */
/* input description (mirrors the arrays the generator produces)            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n, n_solute, n_cv, n_types;
  const double *mass, *charge, *sigma, *epsilon, *gamma; /* gamma may be NULL */
  const int32_t *type;
  int32_t n_bonds;
  const int32_t *bonds;
  const double *bond_r0, *bond_k;
  int32_t n_angles;
  const int32_t *angles;
  const double *angle_t0, *angle_k;
  int32_t n_excl;
  const int32_t *excl; /* extra excluded pairs, 2*n_excl */
  double box;
  const double *native; /* 3*n_cv */
} or_system;

typedef struct {
  double dt, temperature, gamma, r_cut, skin;
  int32_t nstlist;
  double eps_rf, k_ratchet, cv_r0, cv_r_switch, cv_r_cut;
  int32_t cv_min_sep;
  int32_t list_fixed; /* 1: lists rebuilt only at multiples of nstlist */
} or_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the Philox S-box on a   */
/* 128-bit counter with a 64-bit key bumped by the Weyl constants.           */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three standard normals for (trial seed, atom, step, stream): key = seed,
 * counter = (atom, step_lo, step_hi, stream).  Uniforms on the open interval
 * (0,1) from the top 23 bits, u = ((x >> 9) + 1/2) 2^-23 (a value that is
 * exact in single precision too), then Box-Muller on (u0,u1) and (u2,u3). */
void or_normal3(uint64_t seed, int64_t atom, int64_t step, uint32_t stream, double out[3]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)atom, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), stream};
  uint32_t x[4];
  or_philox4x32_10(ctr, key, x);
  double u[4];
  for (int k = 0; k < 4; ++k) u[k] = ((double)(x[k] >> 9) + 0.5) * (1.0 / 8388608.0);
  const double two_pi = 6.283185307179586476925286766559;
  double r01 = sqrt(-2.0 * log(u[0]));
  double r23 = sqrt(-2.0 * log(u[2]));
  out[0] = r01 * cos(two_pi * u[1]);
  out[1] = r01 * sin(two_pi * u[1]);
  out[2] = r23 * cos(two_pi * u[3]);
}

/* ------------------------------------------------------------------------ */
/* contact function of the reaction coordinate (SM, "Collective coordinate") */
/* ------------------------------------------------------------------------ */
/* C(r) = (1 - rho^6) / (1 - rho^10), rho = r / r0.  With s = rho^2 both the
 * numerator and the denominator carry the factor (1 - s), so
 * C = (1 + s + s^2) / (1 + s + s^2 + s^3 + s^4), which is the same function
 * with its removable singularity at r = r0 filled in (C(r0) = 3/5). */
static void contact_raw(double r, double r0, double *C, double *dC) {
  double s = (r / r0) * (r / r0);
  double N = 1.0 + s + s * s;
  double D = N + s * s * s + s * s * s * s;
  double dN = 1.0 + 2.0 * s;
  double dD = dN + 3.0 * s * s + 4.0 * s * s * s;
  *C = N / D;
  double dCds = (dN * D - N * dD) / (D * D);
  *dC = dCds * 2.0 * r / (r0 * r0);
}

/* Smooth switch: 1 below r_s, 0 above r_c, quintic 1 - 10x^3 + 15x^4 - 6x^5
 * in between (x = (r - r_s)/(r_c - r_s)); C^2 at both ends. */
static void switch_fn(double r, double rs, double rc, double *S, double *dS) {
  if (r <= rs) { *S = 1.0; *dS = 0.0; return; }
  if (r >= rc) { *S = 0.0; *dS = 0.0; return; }
  double w = rc - rs, x = (r - rs) / w;
  *S = 1.0 - x * x * x * (10.0 - 15.0 * x + 6.0 * x * x);
  *dS = -30.0 * x * x * (1.0 - x) * (1.0 - x) / w;
}

/* C~ = C S and its derivative; out = {C, C~, dC/dr, dC~/dr} */
void or_contact(double r, double r0, double rs, double rc, double out[4]) {
  double C, dC, S, dS;
  contact_raw(r, r0, &C, &dC);
  switch_fn(r, rs, rc, &S, &dS);
  out[0] = C; out[1] = C * S; out[2] = dC; out[3] = dC * S + C * dS;
}

static inline double min_image(double d, double L) { return d - L * nearbyint(d / L); }

/* Reaction coordinate z(X) and its gradient (FP64).  pos: 3*n (only the first
 * n_cv atoms are read), grad: 3*n_cv (may be NULL).  Distances in the trial
 * use the minimum image; native distances are plain Euclidean. */
double or_cv(const double *pos, const double *native, int32_t n_cv, double box, double r0, double rs,
             double rc, int32_t min_sep, double *grad) {
  double *zi = (double *)calloc((size_t)(n_cv > 0 ? n_cv : 1), sizeof(double));
  if (grad) memset(grad, 0, sizeof(double) * 3 * (size_t)n_cv);
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n_cv; ++i) {
    double gi[3] = {0, 0, 0};
    double zsum = 0.0;
    for (int j = 0; j < n_cv; ++j) {
      int sep = j > i ? j - i : i - j;
      if (sep <= min_sep) continue;
      double d[3], dn[3];
      for (int k = 0; k < 3; ++k) {
        d[k] = min_image(pos[3 * j + k] - pos[3 * i + k], box);
        dn[k] = native[3 * j + k] - native[3 * i + k];
      }
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double rn = sqrt(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2]);
      double c[4], cn[4];
      or_contact(r, r0, rs, rc, c);
      or_contact(rn, r0, rs, rc, cn);
      double h = c[1] - cn[1];
      if (j > i) zsum += h * h;
      /* d z / d x_i = 2 h C~'(r) (x_i - x_j)/r  (sum over partners j) */
      double coef = 2.0 * h * c[3] / r;
      for (int k = 0; k < 3; ++k) gi[k] -= coef * d[k];
    }
    zi[i] = zsum;
    if (grad)
      for (int k = 0; k < 3; ++k) grad[3 * i + k] = gi[k];
  }
  double z = 0.0;
  for (int i = 0; i < n_cv; ++i) z += zi[i];
  free(zi);
  return z;
}

/* ------------------------------------------------------------------------ */
/* exclusions: 1-2 and 1-3 pairs from the topology plus the extra pairs      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t *cnt;
  int32_t *lst; /* n * OR_MAX_EXCL */
  int ok;
} excl_t;

static void excl_add(excl_t *e, int a, int b) {
  if (a == b) return;
  for (int k = 0; k < e->cnt[a]; ++k)
    if (e->lst[a * OR_MAX_EXCL + k] == b) return;
  if (e->cnt[a] >= OR_MAX_EXCL) { e->ok = 0; return; }
  e->lst[a * OR_MAX_EXCL + e->cnt[a]++] = b;
}

static excl_t excl_build(const or_system *s) {
  excl_t e;
  e.cnt = (int32_t *)calloc((size_t)s->n, sizeof(int32_t));
  e.lst = (int32_t *)malloc(sizeof(int32_t) * (size_t)s->n * OR_MAX_EXCL);
  e.ok = 1;
  for (int b = 0; b < s->n_bonds; ++b) {
    excl_add(&e, s->bonds[2 * b], s->bonds[2 * b + 1]);
    excl_add(&e, s->bonds[2 * b + 1], s->bonds[2 * b]);
  }
  for (int a = 0; a < s->n_angles; ++a) {
    int i = s->angles[3 * a], j = s->angles[3 * a + 1], k = s->angles[3 * a + 2];
    excl_add(&e, i, j); excl_add(&e, j, i);
    excl_add(&e, j, k); excl_add(&e, k, j);
    excl_add(&e, i, k); excl_add(&e, k, i);
  }
  for (int x = 0; x < s->n_excl; ++x) {
    excl_add(&e, s->excl[2 * x], s->excl[2 * x + 1]);
    excl_add(&e, s->excl[2 * x + 1], s->excl[2 * x]);
  }
  return e;
}

static int excluded(const excl_t *e, int a, int b) {
  for (int k = 0; k < e->cnt[a]; ++k)
    if (e->lst[a * OR_MAX_EXCL + k] == b) return 1;
  return 0;
}

static void excl_free(excl_t *e) { free(e->cnt); free(e->lst); }

/* ------------------------------------------------------------------------ */
/* Verlet-list membership, restated bit for bit in IEEE single precision:    */
/*   n_k = rint((x_j,k - x_i,k) * invL);  d_k = (x_j,k - L * n_k) - x_i,k     */
/*   r2 = fma(d_z, d_z, fma(d_y, d_y, d_x*d_x));  member iff r2 < rl2        */
/* with L = (float)box, invL = (float)(1.0/(double)L) and                    */
/* rl2 = (float)(r_list*r_list) in double; no other fused multiply-add (the  */
/* image of x_j is formed first, as the force evaluation forms it).          */
/* ------------------------------------------------------------------------ */
static int list_rule(const float *xi, const float *xj, float L, float invL, float rl2) {
  float d[3];
  for (int k = 0; k < 3; ++k) {
    float t = xj[k] - xi[k];
    float q = t * invL;
    float n = rintf(q);
    float sh = L * n;
    float u = xj[k] - sh;
    d[k] = u - xi[k];
  }
  float r2 = d[0] * d[0];
  r2 = fmaf(d[1], d[1], r2);
  r2 = fmaf(d[2], d[2], r2);
  return r2 < rl2;
}

/* All non-excluded pairs i<j that satisfy the list rule.  posf holds float
 * positions (3*n).  Returns the pair count (pairs beyond cap are counted but
 * not stored). */
int64_t or_pairlist(const or_system *s, const float *posf, double r_list, int32_t *pairs, int64_t cap) {
  excl_t e = excl_build(s);
  float L = (float)s->box;
  float invL = (float)(1.0 / (double)L);
  float rl2 = (float)(r_list * r_list);
  int64_t cnt = 0;
  for (int i = 0; i < s->n; ++i)
    for (int j = i + 1; j < s->n; ++j) {
      if (!list_rule(posf + 3 * i, posf + 3 * j, L, invL, rl2)) continue;
      if (excluded(&e, i, j)) continue;
      if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
      ++cnt;
    }
  excl_free(&e);
  return cnt;
}

/* Full neighbour list (both directions) in CSR form for the integrator. */
typedef struct {
  int32_t *start; /* n+1 */
  int32_t *nbr;
  int ok;
} vlist_t;

static vlist_t vlist_build(const or_system *s, const double *pos, double r_list, const excl_t *e) {
  int n = s->n;
  float *pf = (float *)malloc(sizeof(float) * 3 * (size_t)n);
  for (int i = 0; i < 3 * n; ++i) pf[i] = (float)pos[i];
  float L = (float)s->box;
  float invL = (float)(1.0 / (double)L);
  float rl2 = (float)(r_list * r_list);
  int32_t *cnt = (int32_t *)calloc((size_t)n, sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    int c = 0;
    for (int j = 0; j < n; ++j)
      if (j != i && list_rule(pf + 3 * i, pf + 3 * j, L, invL, rl2) && !excluded(e, i, j)) ++c;
    cnt[i] = c;
  }
  vlist_t v;
  v.start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
  v.start[0] = 0;
  for (int i = 0; i < n; ++i) v.start[i + 1] = v.start[i] + cnt[i];
  v.nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(v.start[n] > 0 ? v.start[n] : 1));
  v.ok = 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    int c = v.start[i];
    for (int j = 0; j < n; ++j)
      if (j != i && list_rule(pf + 3 * i, pf + 3 * j, L, invL, rl2) && !excluded(e, i, j)) v.nbr[c++] = j;
  }
  free(cnt);
  free(pf);
  return v;
}

static void vlist_free(vlist_t *v) { free(v->start); free(v->nbr); }

/* ------------------------------------------------------------------------ */
/* physical forces -grad U (FP64)                                            */
/* ------------------------------------------------------------------------ */
/* Pair interaction within the cut-off: returns V and sets fscal such that
 * the force on i is fscal * (x_i - x_j).
 *   LJ:  V = 4 eps [(sig/r)^12 - (sig/r)^6] - same at r_c, sig = (s_i+s_j)/2,
 *        eps = sqrt(e_i e_j)   (Lorentz-Berthelot)
 *   RF:  V = f q_i q_j (1/r + k_rf r^2 - c_rf),
 *        k_rf = (eps_rf-1)/((2 eps_rf+1) r_c^3), c_rf = 1/r_c + k_rf r_c^2,
 *        eps_rf = infinity -> k_rf = 1/(2 r_c^3), c_rf = 3/(2 r_c). */
static void pair_terms(const or_system *s, const or_params *p, int i, int j, double r, double *vlj,
                       double *vrf, double *fscal) {
  int ti = s->type[i], tj = s->type[j];
  double sig = 0.5 * (s->sigma[ti] + s->sigma[tj]);
  double eps = sqrt(s->epsilon[ti] * s->epsilon[tj]);
  double rc = p->r_cut;
  double krf, crf;
  if (p->eps_rf <= 0.0) { krf = 1.0 / (2.0 * rc * rc * rc); crf = 3.0 / (2.0 * rc); }
  else { krf = (p->eps_rf - 1.0) / ((2.0 * p->eps_rf + 1.0) * rc * rc * rc); crf = 1.0 / rc + krf * rc * rc; }
  double qq = OR_FCOUL * s->charge[i] * s->charge[j];
  double lj = 0.0, dlj = 0.0;
  if (eps > 0.0 && sig > 0.0) {
    double sr6 = pow(sig / r, 6.0), sc6 = pow(sig / rc, 6.0);
    lj = 4.0 * eps * (sr6 * sr6 - sr6) - 4.0 * eps * (sc6 * sc6 - sc6);
    dlj = 4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r; /* dV/dr */
  }
  double rf = qq * (1.0 / r + krf * r * r - crf);
  double drf = qq * (-1.0 / (r * r) + 2.0 * krf * r);
  *vlj = lj;
  *vrf = rf;
  *fscal = -(dlj + drf) / r;
}

/* energies[4] = {E_LJ, E_RF, E_bond, E_angle}.  If vl is NULL every pair
 * within the cut-off is taken (brute force over all pairs); otherwise the
 * pairs of the Verlet list that lie within the cut-off. */
static void phys_forces(const or_system *s, const or_params *p, const double *pos, const vlist_t *vl,
                        const excl_t *e, double *F, double *energies) {
  int n = s->n;
  double L = s->box, rc2 = p->r_cut * p->r_cut;
  double *elj = (double *)calloc((size_t)n, sizeof(double));
  double *erf = (double *)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    double f[3] = {0, 0, 0}, el = 0, er = 0;
    int jb = vl ? vl->start[i] : 0, je = vl ? vl->start[i + 1] : n;
    for (int jj = jb; jj < je; ++jj) {
      int j = vl ? vl->nbr[jj] : jj;
      if (j == i) continue;
      if (!vl && excluded(e, i, j)) continue;
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = min_image(pos[3 * i + k] - pos[3 * j + k], L);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 >= rc2) continue;
      double vlj, vrf, fs;
      pair_terms(s, p, i, j, sqrt(r2), &vlj, &vrf, &fs);
      for (int k = 0; k < 3; ++k) f[k] += fs * d[k];
      el += 0.5 * vlj;
      er += 0.5 * vrf;
    }
    for (int k = 0; k < 3; ++k) F[3 * i + k] = f[k];
    elj[i] = el;
    erf[i] = er;
  }
  double E_lj = 0, E_rf = 0, E_b = 0, E_a = 0;
  for (int i = 0; i < n; ++i) { E_lj += elj[i]; E_rf += erf[i]; }
  free(elj);
  free(erf);
  /* bonds: V = k/2 (r - r0)^2 */
  for (int b = 0; b < s->n_bonds; ++b) {
    int i = s->bonds[2 * b], j = s->bonds[2 * b + 1];
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = min_image(pos[3 * i + k] - pos[3 * j + k], L);
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double dr = r - s->bond_r0[b];
    E_b += 0.5 * s->bond_k[b] * dr * dr;
    double fs = -s->bond_k[b] * dr / r;
    for (int k = 0; k < 3; ++k) { F[3 * i + k] += fs * d[k]; F[3 * j + k] -= fs * d[k]; }
  }
  /* angles: V = k/2 (theta - theta0)^2, theta at the middle atom */
  for (int a = 0; a < s->n_angles; ++a) {
    int i = s->angles[3 * a], j = s->angles[3 * a + 1], k3 = s->angles[3 * a + 2];
    double u[3], v[3];
    for (int k = 0; k < 3; ++k) {
      u[k] = min_image(pos[3 * i + k] - pos[3 * j + k], L);
      v[k] = min_image(pos[3 * k3 + k] - pos[3 * j + k], L);
    }
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    double nu = sqrt(uu), nv = sqrt(vv);
    double c = uv / (nu * nv);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c);
    double dth = th - s->angle_t0[a];
    E_a += 0.5 * s->angle_k[a] * dth * dth;
    double sn = sqrt(1.0 - c * c);
    if (sn < 1e-12) sn = 1e-12;
    /* dV/dtheta * dtheta/dcos = -k dth / sin(theta) */
    double g = s->angle_k[a] * dth / sn; /* = -dV/dcos */
    for (int k = 0; k < 3; ++k) {
      double dcu = v[k] / (nu * nv) - c * u[k] / uu; /* d cos / d u */
      double dcv = u[k] / (nu * nv) - c * v[k] / vv; /* d cos / d v */
      /* F = -dV/dx = -(dV/dcos)(dcos/dx) = g * dcos/dx */
      F[3 * i + k] += g * dcu;
      F[3 * k3 + k] += g * dcv;
      F[3 * j + k] -= g * (dcu + dcv);
    }
  }
  if (energies) { energies[0] = E_lj; energies[1] = E_rf; energies[2] = E_b; energies[3] = E_a; }
}

/* Physical forces at a given state.  use_list = 0: every pair within r_c;
 * use_list = 1: pairs of a Verlet list built (list rule) from the same
 * positions.  Returns 0, or -1 if an atom has too many exclusions. */
int or_forces(const or_system *s, const or_params *p, const double *pos, int32_t use_list, double *F,
              double *energies) {
  excl_t e = excl_build(s);
  if (!e.ok) { excl_free(&e); return -1; }
  if (use_list) {
    vlist_t v = vlist_build(s, pos, p->r_cut + p->skin, &e);
    phys_forces(s, p, pos, &v, &e, F, energies);
    vlist_free(&v);
  } else {
    phys_forces(s, p, pos, NULL, &e, F, energies);
  }
  excl_free(&e);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* one biased trial trajectory                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* per step n = 0..n_steps (index 0 = initial state) */
  double *z, *zm, *a, *phi_step; /* may be NULL */
  double *frames;                 /* (n_steps/record_every + 1) * 3n, may be NULL */
  int32_t record_every;
  double *pos_out, *vel_out; /* 3n each, may be NULL */
  double Phi;                /* bias functional at the end */
  double energies[6];        /* E_LJ, E_RF, E_bond, E_angle, E_kin, E_bias at the end */
  double *force_out;         /* 3n total force at the end, may be NULL */
} or_run_out;

static double kinetic(const or_system *s, const double *v) {
  double e = 0.0;
  for (int i = 0; i < s->n; ++i)
    e += 0.5 * s->mass[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
  return e;
}

/* Maxwell-Boltzmann velocities from Philox stream 1 at step 0, with the
 * centre-of-mass velocity removed. */
void or_initial_velocities(const or_system *s, double temperature, uint64_t seed, double *vel) {
  double kT = OR_KB * temperature;
  double P[3] = {0, 0, 0}, M = 0;
  for (int i = 0; i < s->n; ++i) {
    double g[3];
    or_normal3(seed, i, 0, 1u, g);
    double sd = sqrt(kT / s->mass[i]);
    for (int k = 0; k < 3; ++k) { vel[3 * i + k] = sd * g[k]; P[k] += s->mass[i] * vel[3 * i + k]; }
    M += s->mass[i];
  }
  for (int i = 0; i < s->n; ++i)
    for (int k = 0; k < 3; ++k) vel[3 * i + k] -= P[k] / M;
}

/* ratchet bias (Eq. VR) from z, z_m and grad z: adds F^bias to F, returns
 * a = (z - z_m) if z > z_m else 0, and the functional density
 * phi = sum_i |F_i^bias|^2/(gamma_i m_i) (Eq. VMDcondition) in *phi. */
static double ratchet(const or_system *s, const or_params *p, double z, double zm, const double *g, double *F,
                      double *phi) {
  double a = z > zm ? z - zm : 0.0;
  double acc = 0.0;
  for (int i = 0; i < s->n_cv; ++i) {
    double gam = s->gamma ? s->gamma[i] : p->gamma;
    double f2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      double fb = -0.5 * p->k_ratchet * a * g[3 * i + k];
      F[3 * i + k] += fb;
      f2 += fb * fb;
    }
    acc += f2 / (gam * s->mass[i]);
  }
  *phi = acc;
  return a;
}

static void wrap(double *pos, int n, double L) {
  for (int i = 0; i < 3 * n; ++i) pos[i] -= L * floor(pos[i] / L);
}

/* Integrates n_steps BAOAB steps of Eq. Lang with the rMD bias:
 *   v += dt/2 F/m; x += dt/2 v; v = c1 v + c2 sqrt(kT/m) xi_n; x += dt/2 v;
 *   [list due: wrap, rebuild list]; F = -grad U + F^bias;
 *   v += dt/2 F/m; Phi += dt * phi_n,
 * where U is the cut-off potential: the list (pairs within r_cut + skin) is
 * due when an atom is farther than skin/2 - 1e-5 nm from where it was at the
 * last rebuild (then no pair within r_cut can be missing from it) or nstlist
 * steps after it (list_fixed: at multiples of nstlist only),
 * with c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2), xi_n the Philox normals of
 * (seed, atom, n, stream 0).  vel_in NULL -> Maxwell-Boltzmann start.
 * Returns 0 on success, -1 on bad input, -2 on a non-finite state. */
int or_run(const or_system *s, const or_params *p, uint64_t seed, const double *pos_in, const double *vel_in,
           int32_t n_steps, or_run_out *out) {
  int n = s->n;
  excl_t e = excl_build(s);
  if (!e.ok) { excl_free(&e); return -1; }
  double *x = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  double *v = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  double *F = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  double *g = (double *)malloc(sizeof(double) * 3 * (size_t)(s->n_cv > 0 ? s->n_cv : 1));
  double *c1 = (double *)malloc(sizeof(double) * (size_t)n);
  double *c2 = (double *)malloc(sizeof(double) * (size_t)n);
  memcpy(x, pos_in, sizeof(double) * 3 * (size_t)n);
  if (vel_in) memcpy(v, vel_in, sizeof(double) * 3 * (size_t)n);
  else or_initial_velocities(s, p->temperature, seed, v);
  double kT = OR_KB * p->temperature, dt = p->dt, L = s->box;
  for (int i = 0; i < n; ++i) {
    double gam = s->gamma ? s->gamma[i] : p->gamma;
    c1[i] = exp(-gam * dt);
    c2[i] = sqrt(1.0 - c1[i] * c1[i]);
  }
  wrap(x, n, L);
  vlist_t vl = vlist_build(s, x, p->r_cut + p->skin, &e);
  double *xref = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  memcpy(xref, x, sizeof(double) * 3 * (size_t)n);
  int last_rebuild = 0;
  const double trig = 0.5 * p->skin - 1e-5 > 0.0 ? 0.5 * p->skin - 1e-5 : 0.0;
  double en[4];
  phys_forces(s, p, x, &vl, &e, F, en);
  double z = or_cv(x, s->native, s->n_cv, L, p->cv_r0, p->cv_r_switch, p->cv_r_cut, p->cv_min_sep, g);
  double zm = z; /* z_m(0) = z(X_0): no bias on the first force evaluation */
  double phi;
  double a = ratchet(s, p, z, zm, g, F, &phi);
  double Phi = 0.0;
  int rec = 0, status = 0;
  if (out->z) out->z[0] = z;
  if (out->zm) out->zm[0] = zm;
  if (out->a) out->a[0] = a;
  if (out->phi_step) out->phi_step[0] = 0.0;
  if (out->frames && out->record_every > 0) memcpy(out->frames, x, sizeof(double) * 3 * (size_t)n), rec = 1;
  for (int step = 1; step <= n_steps; ++step) {
    for (int i = 0; i < n; ++i) {
      double im = 1.0 / s->mass[i];
      double sd = sqrt(kT * im);
      double xi[3];
      or_normal3(seed, i, step, 0u, xi);
      for (int k = 0; k < 3; ++k) {
        double vi = v[3 * i + k] + 0.5 * dt * F[3 * i + k] * im;
        x[3 * i + k] += 0.5 * dt * vi;
        vi = c1[i] * vi + c2[i] * sd * xi[k];
        x[3 * i + k] += 0.5 * dt * vi;
        v[3 * i + k] = vi;
      }
    }
    int due;
    if (p->list_fixed) {
      due = p->nstlist > 0 && step % p->nstlist == 0;
    } else {
      due = step - last_rebuild >= p->nstlist;
      for (int i = 0; i < n && !due; ++i) {
        double dx = x[3 * i] - xref[3 * i], dy = x[3 * i + 1] - xref[3 * i + 1], dz = x[3 * i + 2] - xref[3 * i + 2];
        due = dx * dx + dy * dy + dz * dz > trig * trig;
      }
    }
    if (due) {
      wrap(x, n, L);
      vlist_free(&vl);
      vl = vlist_build(s, x, p->r_cut + p->skin, &e);
      memcpy(xref, x, sizeof(double) * 3 * (size_t)n);
      last_rebuild = step;
    }
    phys_forces(s, p, x, &vl, &e, F, en);
    z = or_cv(x, s->native, s->n_cv, L, p->cv_r0, p->cv_r_switch, p->cv_r_cut, p->cv_min_sep, g);
    a = ratchet(s, p, z, zm, g, F, &phi);
    if (z < zm) zm = z;
    Phi += dt * phi;
    for (int i = 0; i < n; ++i) {
      double im = 1.0 / s->mass[i];
      for (int k = 0; k < 3; ++k) v[3 * i + k] += 0.5 * dt * F[3 * i + k] * im;
    }
    if (out->z) out->z[step] = z;
    if (out->zm) out->zm[step] = zm;
    if (out->a) out->a[step] = a;
    if (out->phi_step) out->phi_step[step] = phi;
    if (out->frames && out->record_every > 0 && step % out->record_every == 0)
      memcpy(out->frames + (size_t)rec++ * 3 * n, x, sizeof(double) * 3 * (size_t)n);
    if (!isfinite(z) || !isfinite(x[0]) || !isfinite(x[3 * (n - 1)])) { status = -2; break; }
  }
  out->Phi = Phi;
  out->energies[0] = en[0];
  out->energies[1] = en[1];
  out->energies[2] = en[2];
  out->energies[3] = en[3];
  out->energies[4] = kinetic(s, v);
  out->energies[5] = 0.25 * p->k_ratchet * a * a;
  if (out->pos_out) memcpy(out->pos_out, x, sizeof(double) * 3 * (size_t)n);
  if (out->vel_out) memcpy(out->vel_out, v, sizeof(double) * 3 * (size_t)n);
  if (out->force_out) memcpy(out->force_out, F, sizeof(double) * 3 * (size_t)n);
  vlist_free(&vl);
  excl_free(&e);
  free(x); free(v); free(F); free(g); free(c1); free(c2); free(xref);
  return status;
}

/* The bias functional along a given sequence of frames X_0 .. X_{n_frames-1}
 * (each 3*n_cv, CV atoms only), spaced dt apart: z_m starts at z(X_0) and
 * Phi = sum_{n>=1} dt sum_i |F_i^bias(X_n; z_m,n-1)|^2/(gamma_i m_i).
 * Per-frame z, a and phi are written when the pointers are not NULL. */
double or_phi_frames(const or_system *s, const or_params *p, const double *frames, int32_t n_frames,
                     double *z_out, double *a_out, double *phi_out) {
  int ncv = s->n_cv;
  double *g = (double *)malloc(sizeof(double) * 3 * (size_t)(ncv > 0 ? ncv : 1));
  double *F = (double *)calloc((size_t)3 * (size_t)(ncv > 0 ? ncv : 1), sizeof(double));
  double zm = 0.0, Phi = 0.0;
  for (int f = 0; f < n_frames; ++f) {
    const double *X = frames + (size_t)f * 3 * ncv;
    double z = or_cv(X, s->native, ncv, s->box, p->cv_r0, p->cv_r_switch, p->cv_r_cut, p->cv_min_sep, g);
    if (f == 0) zm = z;
    double phi;
    memset(F, 0, sizeof(double) * 3 * (size_t)ncv);
    double a = ratchet(s, p, z, zm, g, F, &phi);
    if (f > 0) Phi += p->dt * phi;
    if (z < zm) zm = z;
    if (z_out) z_out[f] = z;
    if (a_out) a_out[f] = a;
    if (phi_out) phi_out[f] = (f > 0) ? phi : 0.0;
  }
  free(g);
  free(F);
  return Phi;
}

/* ------------------------------------------------------------------------ */
/* adjoint of the bias functional with respect to the frames                */
/* ------------------------------------------------------------------------ */
/* Second derivative of C~(r) = C(r) S(r) (closed forms of the rational C and
 * the quintic switch). */
static double contact_d2(double r, double r0, double rs, double rc) {
  double s = (r / r0) * (r / r0);
  double N = 1.0 + s + s * s, D = N + s * s * s + s * s * s * s;
  double N1 = 1.0 + 2.0 * s, D1 = N1 + 3.0 * s * s + 4.0 * s * s * s;
  double N2 = 2.0, D2 = 2.0 + 6.0 * s + 12.0 * s * s;
  double Cs = (N1 * D - N * D1) / (D * D);
  double Css = ((N2 * D - N * D2) * D - 2.0 * D1 * (N1 * D - N * D1)) / (D * D * D);
  double ds = 2.0 * r / (r0 * r0);
  double C = N / D, C1 = Cs * ds, C2 = Css * ds * ds + Cs * 2.0 / (r0 * r0);
  if (r <= rs) return C2;
  if (r >= rc) return 0.0;
  double w = rc - rs, x = (r - rs) / w;
  double S = 1.0 - x * x * x * (10.0 - 15.0 * x + 6.0 * x * x);
  double S1 = -30.0 * x * x * (1.0 - x) * (1.0 - x) / w;
  double S2 = (-60.0 * x + 180.0 * x * x - 120.0 * x * x * x) / (w * w);
  return C2 * S + 2.0 * C1 * S1 + C * S2;
}

/* Hessian of z applied to w (both 3*n_cv): z = sum_p f_p(r_p) with
 * f = (C~(r) - C~_nat)^2, so a pair adds K (w_j - w_i) to atom j and
 * subtracts it from atom i, K v = f'' u (u.v) + (f'/r)(v - u (u.v)). */
static void cv_hessian_vec(const double *pos, const double *native, int n_cv, double box, const or_params *p,
                           const double *w, double *out) {
  if (n_cv <= 0) return;
  memset(out, 0, sizeof(double) * 3 * (size_t)n_cv);
  for (int i = 0; i < n_cv; ++i)
    for (int j = i + 1; j < n_cv; ++j) {
      if (j - i <= p->cv_min_sep) continue;
      double d[3], dn[3];
      for (int k = 0; k < 3; ++k) {
        d[k] = min_image(pos[3 * j + k] - pos[3 * i + k], box);
        dn[k] = native[3 * j + k] - native[3 * i + k];
      }
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double rn = sqrt(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2]);
      double c[4], cn[4];
      or_contact(r, p->cv_r0, p->cv_r_switch, p->cv_r_cut, c);
      or_contact(rn, p->cv_r0, p->cv_r_switch, p->cv_r_cut, cn);
      double h = c[1] - cn[1];
      double f1 = 2.0 * h * c[3];
      double f2 = 2.0 * (c[3] * c[3] + h * contact_d2(r, p->cv_r0, p->cv_r_switch, p->cv_r_cut));
      double u[3] = {d[0] / r, d[1] / r, d[2] / r};
      double v[3] = {w[3 * j] - w[3 * i], w[3 * j + 1] - w[3 * i + 1], w[3 * j + 2] - w[3 * i + 2]};
      double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
      for (int k = 0; k < 3; ++k) {
        double kv = f2 * u[k] * uv + (f1 / r) * (v[k] - u[k] * uv);
        out[3 * j + k] += kv;
        out[3 * i + k] -= kv;
      }
    }
}

/* Gradient of Phi (as defined by or_phi_frames) with respect to every frame:
 * Phi = sum_{n>=1} dt (k_R/2)^2 a_n^2 Q_n, a_n = (z_n - m_{n-1})_+,
 * m_{n-1} = min_{k<n} z_k, Q_n = sum_i |grad_i z(X_n)|^2 / (gamma_i m_i).
 *   dPhi/dX_n = dt (k_R/2)^2 [ 2 a_n Q_n g_n + a_n^2 2 H_z(X_n) w_n ]      (n >= 1)
 *             - dt (k_R/2)^2 sum_{l : n is the first minimiser of z_0..z_{l-1}} 2 a_l Q_l g_n
 * with g = grad z and w_i = g_i/(gamma_i m_i) (the running minimum is
 * differentiated along its first minimiser).  Returns Phi. */
double or_phi_frames_grad(const or_system *s, const or_params *p, const double *frames, int32_t n_frames,
                          double *grad) {
  int ncv = s->n_cv;
  size_t fs = (size_t)3 * ncv;
  double *g = (double *)malloc(sizeof(double) * fs * (size_t)(n_frames > 0 ? n_frames : 1));
  double *z = (double *)malloc(sizeof(double) * (size_t)(n_frames > 0 ? n_frames : 1));
  double *Q = (double *)calloc((size_t)(n_frames > 0 ? n_frames : 1), sizeof(double));
  double *a = (double *)calloc((size_t)(n_frames > 0 ? n_frames : 1), sizeof(double));
  double *route = (double *)calloc((size_t)(n_frames > 0 ? n_frames : 1), sizeof(double));
  double *w = (double *)malloc(sizeof(double) * (fs > 0 ? fs : 1));
  double *hw = (double *)malloc(sizeof(double) * (fs > 0 ? fs : 1));
  double c = p->dt * 0.25 * p->k_ratchet * p->k_ratchet;
  for (int f = 0; f < n_frames; ++f) {
    z[f] = or_cv(frames + f * fs, s->native, ncv, s->box, p->cv_r0, p->cv_r_switch, p->cv_r_cut, p->cv_min_sep,
                 g + f * fs);
    double q = 0.0;
    for (int i = 0; i < ncv; ++i) {
      double gam = s->gamma ? s->gamma[i] : p->gamma;
      double g2 = g[f * fs + 3 * i] * g[f * fs + 3 * i] + g[f * fs + 3 * i + 1] * g[f * fs + 3 * i + 1] +
                  g[f * fs + 3 * i + 2] * g[f * fs + 3 * i + 2];
      q += g2 / (gam * s->mass[i]);
    }
    Q[f] = q;
  }
  double Phi = 0.0;
  double m = 0.0;
  int arg = 0;
  for (int f = 0; f < n_frames; ++f) {
    if (f == 0) { m = z[0]; arg = 0; continue; }
    a[f] = z[f] > m ? z[f] - m : 0.0;
    Phi += c * a[f] * a[f] * Q[f];
    if (a[f] > 0.0) route[arg] += 2.0 * a[f] * Q[f];
    if (z[f] < m) { m = z[f]; arg = f; }
  }
  for (int f = 0; f < n_frames; ++f) {
    const double *X = frames + f * fs;
    double *G = grad + f * fs;
    double cg = c * ((f > 0 ? 2.0 * a[f] * Q[f] : 0.0) - route[f]);
    for (size_t k = 0; k < fs; ++k) G[k] = cg * g[f * fs + k];
    if (f > 0 && a[f] > 0.0) {
      for (int i = 0; i < ncv; ++i) {
        double gam = s->gamma ? s->gamma[i] : p->gamma;
        for (int k = 0; k < 3; ++k) w[3 * i + k] = g[f * fs + 3 * i + k] / (gam * s->mass[i]);
      }
      cv_hessian_vec(X, s->native, ncv, s->box, p, w, hw);
      for (size_t k = 0; k < fs; ++k) G[k] += c * a[f] * a[f] * 2.0 * hw[k];
    }
  }
  free(g); free(z); free(Q); free(a); free(route); free(w); free(hw);
  return Phi;
}

int32_t or_num_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int32_t k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}

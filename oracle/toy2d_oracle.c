/*
 * toy2d_oracle.c -- plain FP64 CPU oracle of the two-dimensional toy model
 * of the variational pathway scheme (arXiv:1405.6104, SM "Illustrative
 * Application in a Toy Model").
 *
 * TEST INFRASTRUCTURE ONLY, like vpath_oracle.c (linked into the same
 * stand-alone library; nothing here is shared with the CUDA library).
 *
 * What it computes (one trial):
 *   - the potential of the toy-model section,
 *       U(x,y) = w^2 (x^2+y^2)^2 - A1 s1^p/(x^2+y^2+s1^2)^2
 *              + A2 s2^p/(x^2+y^2+s2^2)^2 - A3 s3^p/((x-xm)^2+(y-ym)^2+s3^2)^2,
 *     and its force -grad U.  The section prints p = 2; with p = 2 the
 *     profile falls monotonically from the start to the funnel, so there is
 *     no ring barrier to cross, contrary to what the section reports.  With
 *     p = 4 each term's amplitude at its centre is A (funnel -30, ring +20,
 *     gate -6) and the landscape has the ring barrier and the gate the
 *     section describes.  p is a parameter (s_power);
 *   - underdamped Langevin dynamics (Eq. Lang with one particle of mass m),
 *     BAOAB splitting as in the atomistic oracle, white noise from
 *     Philox4x32-10 + Box-Muller (or_normal3, stream 0, atom 0);
 *   - one of three biases on the reaction coordinate z = sqrt(x^2+y^2)
 *     (the distance from the product at the origin):
 *       0  none (plain Langevin),
 *       1  ratchet-and-pawl (Eq. VR): F = -(k/2)(z - z_m) grad z when z > z_m,
 *          z_m the running minimum of z, z_m(0) = z(x_0),
 *       2  steered MD (the comparison of the toy-model section): a harmonic
 *          pull of constant strength k towards z = 0, F = -k z grad z;
 *   - the bias functional (Eq. VMDcondition) Phi = sum_n dt |F_bias|^2/(gamma m)
 *     over the force evaluations of the path, right-endpoint rule, up to and
 *     including the first step with z <= z_product (first passage), where the
 *     trial stops.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

void or_normal3(uint64_t seed, int64_t atom, int64_t step, uint32_t stream, double out[3]);

typedef struct {
  double A1, A2, A3, s1, s2, s3, w, xm, ym; /* potential */
  double mass, gamma, kT, dt;                /* Langevin */
  double x0, y0;                             /* start */
  double z_product;                          /* product reached when z <= z_product */
  int32_t bias;                              /* 0 none, 1 ratchet, 2 steered */
  int32_t s_power;                           /* p: 2 (as printed) or 4 (amplitude A at the centre) */
} or_toy2d_params;

static double spow(double s, int p) { return p == 4 ? (s * s) * (s * s) : s * s; }

/* U and -grad U.  With r2 = x^2 + y^2 and a well term A s^p / (d2 + s^2)^2,
 * d/dx = -4 A s^p (d2 + s^2)^-3 (x - x_c). */
void or_toy2d_force(const or_toy2d_params *p, double x, double y, double *U, double *fx, double *fy) {
  double r2 = x * x + y * y;
  double u = p->w * p->w * r2 * r2;
  double gx = 4.0 * p->w * p->w * r2 * x; /* dU/dx of the quartic */
  double gy = 4.0 * p->w * p->w * r2 * y;
  /* funnel (-), ring barrier (+), gate (-) */
  double D1 = r2 + p->s1 * p->s1;
  double n1 = spow(p->s1, p->s_power);
  u -= p->A1 * n1 / (D1 * D1);
  double c1 = 4.0 * p->A1 * n1 / (D1 * D1 * D1);
  gx += c1 * x;
  gy += c1 * y;
  double D2 = r2 + p->s2 * p->s2;
  double n2 = spow(p->s2, p->s_power);
  u += p->A2 * n2 / (D2 * D2);
  double c2 = 4.0 * p->A2 * n2 / (D2 * D2 * D2);
  gx -= c2 * x;
  gy -= c2 * y;
  double dx = x - p->xm, dy = y - p->ym;
  double D3 = dx * dx + dy * dy + p->s3 * p->s3;
  double n3 = spow(p->s3, p->s_power);
  u -= p->A3 * n3 / (D3 * D3);
  double c3 = 4.0 * p->A3 * n3 / (D3 * D3 * D3);
  gx += c3 * dx;
  gy += c3 * dy;
  if (U) *U = u;
  *fx = -gx;
  *fy = -gy;
}

/* Bias force at (x, y) given the running minimum zm (ratchet) and k; returns
 * the ratchet amplitude a (0 for the other biases). */
static double bias_force(const or_toy2d_params *p, double k, double x, double y, double zm, double *bx,
                         double *by) {
  double z = sqrt(x * x + y * y);
  *bx = 0.0;
  *by = 0.0;
  if (z == 0.0) return 0.0; /* grad z undefined at the product itself */
  double ux = x / z, uy = y / z; /* grad z */
  if (p->bias == 1) {
    double a = z > zm ? z - zm : 0.0;
    *bx = -0.5 * k * a * ux;
    *by = -0.5 * k * a * uy;
    return a;
  }
  if (p->bias == 2) {
    *bx = -k * z * ux;
    *by = -k * z * uy;
  }
  return 0.0;
}

/* One trial of n_steps steps (fewer when the product is reached).  Returns
 * the first-passage step (-1: not reached).  out_state[4] = {x, y, vx, vy} at
 * the end, *phi = the functional; path (may be NULL) receives (x, y) at steps
 * 0 .. end, 2 doubles per step. */
int64_t or_toy2d_run(const or_toy2d_params *p, double k, uint64_t seed, int64_t n_steps, double *out_state,
                     double *phi, double *path) {
  double x = p->x0, y = p->y0;
  double sd = sqrt(p->kT / p->mass);
  double g[3];
  or_normal3(seed, 0, 0, 1u, g); /* Maxwell-Boltzmann start: stream 1, step 0 */
  double vx = sd * g[0], vy = sd * g[1];
  double c1 = exp(-p->gamma * p->dt);
  double c2 = sqrt(1.0 - c1 * c1);
  double zm = sqrt(x * x + y * y);
  double fx, fy, bx, by;
  or_toy2d_force(p, x, y, NULL, &fx, &fy);
  bias_force(p, k, x, y, zm, &bx, &by);
  fx += bx;
  fy += by;
  double Phi = 0.0;
  int64_t passage = -1;
  if (path) { path[0] = x; path[1] = y; }
  double h = 0.5 * p->dt, im = 1.0 / p->mass;
  for (int64_t n = 1; n <= n_steps; ++n) {
    or_normal3(seed, 0, n, 0u, g);
    vx += h * fx * im;
    vy += h * fy * im;
    x += h * vx;
    y += h * vy;
    vx = c1 * vx + c2 * sd * g[0];
    vy = c1 * vy + c2 * sd * g[1];
    x += h * vx;
    y += h * vy;
    or_toy2d_force(p, x, y, NULL, &fx, &fy);
    bias_force(p, k, x, y, zm, &bx, &by);
    Phi += p->dt * (bx * bx + by * by) / (p->gamma * p->mass);
    fx += bx;
    fy += by;
    double z = sqrt(x * x + y * y);
    if (z < zm) zm = z;
    vx += h * fx * im;
    vy += h * fy * im;
    if (path) { path[2 * n] = x; path[2 * n + 1] = y; }
    if (z <= p->z_product) { passage = n; break; }
  }
  out_state[0] = x;
  out_state[1] = y;
  out_state[2] = vx;
  out_state[3] = vy;
  *phi = Phi;
  return passage;
}

/* The functional of Eq. VMDcondition along a given path (x_n, y_n),
 * n = 0 .. n_points-1, spaced dt apart, with the same bias rule and the same
 * stop at the first point with z <= z_product.  *passage receives that
 * index (-1: none). */
double or_toy2d_phi_path(const or_toy2d_params *p, double k, const double *path, int64_t n_points,
                         int64_t *passage) {
  double zm = sqrt(path[0] * path[0] + path[1] * path[1]);
  double Phi = 0.0, bx, by;
  *passage = -1;
  for (int64_t n = 1; n < n_points; ++n) {
    double x = path[2 * n], y = path[2 * n + 1];
    bias_force(p, k, x, y, zm, &bx, &by);
    Phi += p->dt * (bx * bx + by * by) / (p->gamma * p->mass);
    double z = sqrt(x * x + y * y);
    if (z < zm) zm = z;
    if (z <= p->z_product) { *passage = n; break; }
  }
  return Phi;
}

// vp_cvpair.cuh -- one contact pair of the reaction coordinate (SM,
// "Collective coordinate"): C~(r) = C(r) S(r) with the rational contact
// function C = (1 + s + s^2)/(1 + s + s^2 + s^3 + s^4), s = (r/r0)^2 (the
// printed (1 - rho^6)/(1 - rho^10) with the factor (1 - s) cancelled) and the
// quintic switch S.  Shared by the batched kernel and the adjoint kernels.
#pragma once
#include "vp_internal.cuh"

namespace vp {

struct CvConst {
  ff inv_r0sq, rs, inv_w;
  float rs2, rc2_far;
};

__device__ __forceinline__ CvConst cv_const(const SimConst &c) {
  return CvConst{ff{c.cv_inv_r0sq_hi, c.cv_inv_r0sq_lo}, ff{c.cv_rs_hi, c.cv_rs_lo}, ff{c.cv_inv_w_hi, c.cv_inv_w_lo},
                 c.cv_rs2, c.cv_rc2_far};
}

__device__ __forceinline__ ff contact_ff(ff s) {
  ff s2 = ff_sqr(s);
  ff s3 = ff_mul(s2, s);
  ff s4 = ff_sqr(s2);
  ff N = ff_add(ff_add_f(s, 1.0f), s2);
  ff D = ff_add(ff_add(N, s3), s4);
  return ff_div(N, D);
}

__device__ __forceinline__ float dcontact_ds(float s) {
  float N = 1.0f + s + s * s;
  float D = N + s * s * s + s * s * s * s;
  float dN = 1.0f + 2.0f * s;
  float dD = dN + 3.0f * s * s + 4.0f * s * s * s;
  return (dN * D - N * dD) / (D * D);
}

// d^2 C / ds^2 of the rational contact function
__device__ __forceinline__ float d2contact_ds2(float s) {
  float N = 1.0f + s + s * s, D = N + s * s * s + s * s * s * s;
  float N1 = 1.0f + 2.0f * s, D1 = N1 + 3.0f * s * s + 4.0f * s * s * s;
  float D2 = 2.0f + 6.0f * s + 12.0f * s * s;
  return ((2.0f * D - N * D2) * D - 2.0f * D1 * (N1 * D - N * D1)) / (D * D * D);
}

struct CvPair {
  ff Ct;       // C~(r)
  float dCt;   // dC~/dr
  float d2Ct;  // d^2 C~/dr^2 (only with SECOND)
  float r;
};

// C~, C~' (and C~'' when SECOND) at the squared distance r2 (float-float)
template <bool SECOND>
__device__ __forceinline__ CvPair cv_contact(ff r2, const CvConst &k) {
  CvPair o;
  const ff s = ff_mul(r2, k.inv_r0sq);
  o.Ct = contact_ff(s);
  o.r = sqrtf(r2.hi);
  const float ds = 2.0f * o.r * k.inv_r0sq.hi;  // ds/dr
  const float Cs = dcontact_ds(s.hi);
  o.dCt = Cs * ds;
  o.d2Ct = SECOND ? d2contact_ds2(s.hi) * ds * ds + Cs * 2.0f * k.inv_r0sq.hi : 0.0f;
  if (r2.hi > k.rs2) {
    const ff r = ff_sqrt(r2);
    const ff x = ff_mul(ff_add(r, ff_neg(k.rs)), k.inv_w);
    if (x.hi >= 1.0f) {
      o.Ct = {0.f, 0.f};
      o.dCt = 0.f;
      o.d2Ct = 0.f;
    } else {
      // S = 1 - x^3 (10 - 15 x + 6 x^2)
      ff p = ff_add_f(ff_mul_f(x, 6.0f), -15.0f);
      p = ff_add_f(ff_mul(p, x), 10.0f);
      const ff x3 = ff_mul(ff_sqr(x), x);
      const ff S = ff_add_f(ff_neg(ff_mul(x3, p)), 1.0f);
      const float xf = x.hi, iw = k.inv_w.hi;
      const float S1 = -30.0f * xf * xf * (1.0f - xf) * (1.0f - xf) * iw;
      if (SECOND) {
        const float S2 = (-60.0f * xf + 180.0f * xf * xf - 120.0f * xf * xf * xf) * iw * iw;
        o.d2Ct = o.d2Ct * S.hi + 2.0f * o.dCt * S1 + o.Ct.hi * S2;
      }
      o.dCt = o.dCt * S.hi + o.Ct.hi * S1;
      o.Ct = ff_mul(o.Ct, S);
    }
  }
  return o;
}

// exact minimum-image difference x_j - x_i as float-float
__device__ __forceinline__ void cv_delta(float3 xi, float xjx, float xjy, float xjz, float L, float iL, ff &dx, ff &dy,
                                         ff &dz) {
  dx = ff_diff(xjx, xi.x);
  dy = ff_diff(xjy, xi.y);
  dz = ff_diff(xjz, xi.z);
  const float nx = rintf(dx.hi * iL), ny = rintf(dy.hi * iL), nz = rintf(dz.hi * iL);
  if (nx != 0.f) dx = ff_add_f(dx, -L * nx);
  if (ny != 0.f) dy = ff_add_f(dy, -L * ny);
  if (nz != 0.f) dz = ff_add_f(dz, -L * nz);
}

}  // namespace vp

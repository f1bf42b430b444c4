// vp_update_dev.cuh -- the Langevin update of one slot (BAOAB with the
// ratchet force and Philox noise), shared by the update kernel and the
// one-kernel step.
#pragma once
#include "vp_dev.cuh"

namespace vp {

// One slot; returns whether it requested a list rebuild of its trial.
template <int MODE>
__device__ __forceinline__ bool update_slot(const Dev &d, const SimConst &c, int slot) {
  if (slot >= d.total_slots) return false;
  bool req = false;
  if (MODE == UPD_FINAL && slot == 0) *d.kick = 0.5f;
  // every load that does not depend on another is issued before any store
  // (the stores could alias them as far as the compiler knows), so a thread
  // waits for two memory round trips (three for reaction-coordinate atoms);
  // slots past a trial's clusters and padding slots carry orig = -1
  const int o = __ldg(d.orig + slot);
  const int t = __ldg(d.slot_trial + slot);
  float4 p = d.pos[slot], v = d.vel[slot];
  const float4 ref = MODE == UPD_DRIFT && !c.list_fixed ? d.ref_slot[slot] : make_float4(0.f, 0.f, 0.f, 0.f);
  const long long fxi = d.fx[slot], fyi = d.fy[slot], fzi = d.fz[slot];
  const float kick = MODE == UPD_DRIFT ? *d.kick : 0.5f;
  const unsigned long long step = MODE == UPD_DRIFT ? (unsigned long long)(*d.step) + 1ull : 0ull;
  if (MODE == UPD_DRIFT && slot == 0) *d.cur_step = step;  // the step the rebuild kernels work on
  if (o < 0) return false;
  const int n_cv = __ldg(&d.tinfo[t].n_cv), cv0 = __ldg(&d.tinfo[t].cv0);
  const uint32_t key0 = __ldg(&d.tinfo[t].key0), key1 = __ldg(&d.tinfo[t].key1);
  const unsigned long long nstep = step + (unsigned long long)__ldg(&d.tinfo[t].noise_off);
  float Fx = fx_to(fxi), Fy = fx_to(fyi), Fz = fx_to(fzi);
  if (o < n_cv) {
    // ratchet force F_i = -(k_R/2) a grad_i z (Eq. VR); a = 0 when z <= z_m
    const double a = d.tstate[t].a;
    const int gi = cv0 + o;
    const long long gx = d.gx[gi], gy = d.gy[gi], gz = d.gz[gi];
    const float s = -c.kR_half * (float)a;
    Fx += s * fx_to(gx);
    Fy += s * fx_to(gy);
    Fz += s * fx_to(gz);
    if (MODE == UPD_DRIFT) { d.gx[gi] = 0; d.gy[gi] = 0; d.gz[gi] = 0; }
  }
  if (MODE == UPD_DRIFT) { d.fx[slot] = 0; d.fy[slot] = 0; d.fz[slot] = 0; }
  const float kdt = kick * c.dt * v.w;
  v.x += kdt * Fx; v.y += kdt * Fy; v.z += kdt * Fz;
  if (MODE == UPD_DRIFT) {
    float c1, c2sd;
    if (c.uniform_gamma) {  // c2 sqrt(kT/m) = c2 sqrt(kT) sqrt(1/m)
      c1 = c.c1_u;
      c2sd = c.c2sqkT_u * sqrtf(v.w);
    } else {
      const AtomSys as = d.asys[__ldg(&d.tinfo[t].sysatom0) + o];
      c1 = as.c1;
      c2sd = as.c2sd;
    }
    p.x += c.half_dt * v.x; p.y += c.half_dt * v.y; p.z += c.half_dt * v.z;
    const float3 xi = normal3(key0, key1, (uint32_t)o, nstep, 0u);
    v.x = c1 * v.x + c2sd * xi.x;
    v.y = c1 * v.y + c2sd * xi.y;
    v.z = c1 * v.z + c2sd * xi.z;
    p.x += c.half_dt * v.x; p.y += c.half_dt * v.y; p.z += c.half_dt * v.z;
    // a run that has blown up: a non-finite state, a force beyond 2^30
    // kJ/mol/nm (the 64-bit fixed-point sums, 2^32 units per kJ/mol/nm, are
    // no longer trustworthy) or an atom that crosses the box in one step
    // (positions are wrapped at every rebuild, so a blown-up run would
    // otherwise stay finite)
    const float vlim = __ldg(&d.tinfo[t].box) / c.dt;
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(v.x) && isfinite(v.y) && isfinite(v.z)) ||
        fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))) > vlim ||
        fmaxf(fabsf(Fx), fmaxf(fabsf(Fy), fabsf(Fz))) > 1073741824.0f)
      atomicOr(d.err, ERR_NONFINITE);
    d.pos[slot] = p;
    // moved beyond the list buffer: the trial's list is rebuilt in this step,
    // before the forces (positions are not wrapped between rebuilds, so this
    // is the displacement itself)
    if (!c.list_fixed) {
      const float ddx = p.x - ref.x, ddy = p.y - ref.y, ddz = p.z - ref.z;
      if (ddx * ddx + ddy * ddy + ddz * ddz > c.trig2) {
        d.rb[t] = (uint32_t)step;
        req = true;
      }
    }
  }
  d.vel[slot] = v;
  return req;
}

}  // namespace vp

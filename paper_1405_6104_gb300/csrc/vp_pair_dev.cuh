// vp_pair_dev.cuh -- device functions of the force kernels (the packed
// nonbonded pair loop of one i-cluster, the bonded terms of one group),
// shared by the separate kernels and the one-kernel step.
#pragma once
#include <type_traits>

#include "vp_dev.cuh"

namespace vp {

// displacement x_p - x_self under the minimum image, with the image shift
// subtracted from x_p first (exact when the two are within a box length)
__device__ __forceinline__ float3 min_disp(float4 self, float4 other, float L, float iL) {
  float nx = rintf((other.x - self.x) * iL), ny = rintf((other.y - self.y) * iL), nz = rintf((other.z - self.z) * iL);
  return make_float3((other.x - L * nx) - self.x, (other.y - L * ny) - self.y, (other.z - L * nz) - self.z);
}

// launch shape of the force-only pair kernels: warps per block, the penalty
// of a masked pair
constexpr int PF_WARPS = 4;
constexpr float MASK_PEN = 1.0e30f;

// shared memory of the packed pair kernel's warps
struct PairF2Shared {
  float4 s_c4[PF_WARPS][CL / 2][SMALL_TYPES];
  float4 s_sh[PF_WARPS][64];
  float4 s_ip[PF_WARPS][CL / 2][2];
  float s_red[PF_WARPS][3 * CL * 33];
};


// the forces of one i-cluster I by the calling warp (packed arithmetic)
__device__ __forceinline__ void pair_cluster_f2(const Dev &d, const SimConst &c, PairF2Shared &sh, int I) {
  constexpr int TS = SMALL_TYPES;
  auto &s_c4 = sh.s_c4;
  auto &s_sh = sh.s_sh;
  auto &s_ip = sh.s_ip;
  auto &s_red = sh.s_red;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int NT = c.n_types;
  const int t = d.clus_trial[I];
  // the loads that need only I go out before those that need the trial (one
  // memory round trip less before the pair loop): the list's first two
  // groups (taken only below list_n, read within the cluster's segment), the
  // i-atoms and their types
  const int n = d.list_n[I], nm = d.list_nm[I];
  const uint32_t *seg = d.list + (size_t)I * c.list_cap;
  const uint8_t *segm = d.list_m + (size_t)I * c.list_cap;
  // the list words stream through L2 (the batch's lists are larger than L2)
  // with the evict-first hint, so that they do not push out the positions
  // and force accumulators every lane keeps coming back to
  const uint32_t raw0 = lane < c.list_cap ? __ldcs(seg + lane) : d.idle_entry;
  const uint32_t raw1 = 32 + lane < c.list_cap ? __ldcs(seg + 32 + lane) : d.idle_entry;
  float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
  if (lane < CL / 2) {
    a0 = d.pos[I * CL + 2 * lane];
    a1 = d.pos[I * CL + 2 * lane + 1];
  }
  int ty[2][2] = {{0, 0}, {0, 0}};  // the i-atom types of this lane's table rows (at most two per lane)
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int k = lane + 32 * r;
    if (k < (CL / 2) * NT) {
      const int p = k / NT;
      ty[r][0] = d.type[I * CL + 2 * p];
      ty[r][1] = d.type[I * CL + 2 * p + 1];
    }
  }
  const TrialInfo T = d.tinfo[t];
  if (I - T.clus0 >= d.tstate[t].n_clus) return;
  const float L = T.box, iL = T.inv_box;

  if (lane < CL / 2) {
    // negated coordinates: d = xj + (-xi) in one FADD2 (a packed operand has no negate modifier)
    s_ip[wib][lane][0] = make_float4(-a0.x, -a1.x, -a0.y, -a1.y);
    s_ip[wib][lane][1] = make_float4(-a0.z, -a1.z, a0.w, a1.w);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int k = lane + 32 * r;
    if (k < (CL / 2) * NT) {
      const int p = k / NT, tj = k - p * NT;
      const float2 c0 = d.ljtab[ty[r][0] * NT + tj], c1 = d.ljtab[ty[r][1] * NT + tj];
      s_c4[wib][p][tj] = make_float4(c0.y, c1.y, -c0.x, -c1.x);
    }
  }
  for (int k = lane; k < 64; k += 32) {
    const int ix = (k & 3) - 1, iy = ((k >> 2) & 3) - 1, iz = ((k >> 4) & 3) - 1;
    s_sh[wib][k] = make_float4(L * ix, L * iy, L * iz, 0.f);
  }
  __syncwarp();
  float2 fx[CL / 2], fy[CL / 2], fz[CL / 2];
#pragma unroll
  for (int p = 0; p < CL / 2; ++p) fx[p] = fy[p] = fz[p] = make_float2(0.f, 0.f);
  const float2 m2krf = make_float2(-c.two_krf, -c.two_krf);
  const float rc2 = c.rc2;

  // one j-atom entry per lane; entries are fetched two groups ahead, the
  // j-atom itself at the top of its iteration (fewer live registers: a higher
  // block count per SM hides that load better than a prefetch does)
  uint32_t ent = lane < n ? raw0 : d.idle_entry;
  uint32_t ent_n = 32 + lane < n ? raw1 : d.idle_entry;
  for (int e0 = 0; e0 < n; e0 += 32) {
    const uint32_t ent_nn = e0 + 64 + lane < n ? __ldcs(seg + e0 + 64 + lane) : d.idle_entry;
    const int sj = (int)(ent & J_MASK);
    const float4 pj = d.pos[sj];
    const int tj = d.type[sj];
    const float4 shv = s_sh[wib][(ent >> J_BITS) & 63u];
    const float xj = pj.x - shv.x, yj = pj.y - shv.y, zj = pj.z - shv.z, qj = pj.w;
    // the pair masks, in the groups that need them (the first nm entries)
    const bool masked = e0 < nm;
    const unsigned mb = masked && e0 + lane < n ? segm[e0 + lane] : 0u;
    const bool exact = (ent & E_EXACT) != 0u;
    const float4 *row = &s_c4[wib][0][tj];
    float fjx, fjy, fjz;
    // one image per entry; MASKED: the pair masks apply (a group with
    // exclusions or the cluster itself); else the cut-off alone decides, which
    // gives the same forces: a listed pair that failed the list rule is still
    // beyond the cut-off (lists are rebuilt before any atom has moved skin/2)
    auto one_image = [&](auto mtag) {
      constexpr bool MASKED = decltype(mtag)::value;
      const float2 xj2 = make_float2(xj, xj), yj2 = make_float2(yj, yj), zj2 = make_float2(zj, zj);
      const float2 qj2 = make_float2(qj, qj);
      float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
#pragma unroll
      for (int p = 0; p < CL / 2; ++p) {
        const float4 i0 = s_ip[wib][p][0], i1 = s_ip[wib][p][1];
        const float2 dx = __fadd2_rn(xj2, make_float2(i0.x, i0.y));
        const float2 dy = __fadd2_rn(yj2, make_float2(i0.z, i0.w));
        const float2 dz = __fadd2_rn(zj2, make_float2(i1.x, i1.y));
        // the mask bit joins the cut-off test (the same forces as the penalty form)
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 rinv2 = __fmul2_rn(rinv, rinv);
        const float2 rinv6 = __fmul2_rn(__fmul2_rn(rinv2, rinv2), rinv2);
        const float4 cc = row[p * TS];
        const float2 qq = __fmul2_rn(make_float2(i1.z, i1.w), qj2);
        float2 tt = __ffma2_rn(make_float2(cc.x, cc.y), rinv6, make_float2(cc.z, cc.w));
        tt = __fmul2_rn(tt, rinv6);
        tt = __ffma2_rn(qq, rinv, tt);
        tt = __fmul2_rn(tt, rinv2);
        float2 f = __ffma2_rn(qq, m2krf, tt);
        f.x = ((!MASKED || (mb & (1u << (2 * p)))) && r2.x < rc2) ? f.x : 0.0f;
        f.y = ((!MASKED || (mb & (1u << (2 * p + 1)))) && r2.y < rc2) ? f.y : 0.0f;
        fx[p] = __ffma2_rn(f, dx, fx[p]);
        fy[p] = __ffma2_rn(f, dy, fy[p]);
        fz[p] = __ffma2_rn(f, dz, fz[p]);
        gx = __ffma2_rn(f, dx, gx);
        gy = __ffma2_rn(f, dy, gy);
        gz = __ffma2_rn(f, dz, gz);
      }
      fjx = gx.x + gx.y;
      fjy = gy.x + gy.y;
      fjz = gz.x + gz.y;
    };
    if (!masked) {
      one_image(std::false_type{});
    } else if (!__any_sync(0xffffffffu, exact)) {
      one_image(std::true_type{});
    } else {
      // some entry of this group needs pair-by-pair minimum images
      float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
#pragma unroll
      for (int p = 0; p < CL / 2; ++p) {
        const float4 i0 = s_ip[wib][p][0], i1 = s_ip[wib][p][1];
        const float4 cc = row[p * TS];
        float2 f2v, dx2, dy2, dz2;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const float pen = (mb & (1u << (2 * p + hh))) ? 0.0f : MASK_PEN;
          float dx = __fadd_rn(xj, hh ? i0.y : i0.x), dy = __fadd_rn(yj, hh ? i0.w : i0.z),
                dz = __fadd_rn(zj, hh ? i1.y : i1.x);
          if (exact) {
            dx = __fmaf_rn(-L, rintf(__fmul_rn(dx, iL)), dx);
            dy = __fmaf_rn(-L, rintf(__fmul_rn(dy, iL)), dy);
            dz = __fmaf_rn(-L, rintf(__fmul_rn(dz, iL)), dz);
          }
          const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmaf_rn(dx, dx, pen)));
          const float rinv = rsqrtf(r2);
          const float rinv2 = __fmul_rn(rinv, rinv);
          const float rinv6 = __fmul_rn(__fmul_rn(rinv2, rinv2), rinv2);
          const float qq = __fmul_rn(hh ? i1.w : i1.z, qj);
          float tt = __fmaf_rn(hh ? cc.y : cc.x, rinv6, hh ? cc.w : cc.z);
          tt = __fmul_rn(tt, rinv6);
          tt = __fmaf_rn(qq, rinv, tt);
          tt = __fmul_rn(tt, rinv2);
          float f = __fmaf_rn(qq, -c.two_krf, tt);
          f = r2 < rc2 ? f : 0.0f;
          if (hh) { f2v.y = f; dx2.y = dx; dy2.y = dy; dz2.y = dz; }
          else { f2v.x = f; dx2.x = dx; dy2.x = dy; dz2.x = dz; }
        }
        fx[p] = __ffma2_rn(f2v, dx2, fx[p]);
        fy[p] = __ffma2_rn(f2v, dy2, fy[p]);
        fz[p] = __ffma2_rn(f2v, dz2, fz[p]);
        gx = __ffma2_rn(f2v, dx2, gx);
        gy = __ffma2_rn(f2v, dy2, gy);
        gz = __ffma2_rn(f2v, dz2, gz);
      }
      fjx = gx.x + gx.y;
      fjy = gy.x + gy.y;
      fjz = gz.x + gz.y;
    }
    if (fjx != 0.f || fjy != 0.f || fjz != 0.f) {
      red_add(d.fx + sj, fx_from(fjx));
      red_add(d.fy + sj, fx_from(fjy));
      red_add(d.fz + sj, fx_from(fjz));
    }
    ent = ent_n;
    ent_n = ent_nn;
  }

  float fi[CL][3];
#pragma unroll
  for (int p = 0; p < CL / 2; ++p) {
    fi[2 * p][0] = -fx[p].x; fi[2 * p][1] = -fy[p].x; fi[2 * p][2] = -fz[p].x;
    fi[2 * p + 1][0] = -fx[p].y; fi[2 * p + 1][1] = -fy[p].y; fi[2 * p + 1][2] = -fz[p].y;
  }
  float *r = s_red[wib];
#pragma unroll
  for (int a = 0; a < CL; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) r[(3 * a + k) * 33 + lane] = fi[a][k];
  __syncwarp();
  if (lane < 3 * CL) {
    float sum = 0.f;
    for (int l = 0; l < 32; ++l) sum += r[lane * 33 + l];
    const int a = lane / 3, comp = lane - 3 * a;
    const long long val = fx_from(sum);
    if (val != 0) red_add((comp == 0 ? d.fx : comp == 1 ? d.fy : d.fz) + I * CL + a, val);
  }
}


// Bonded forces, one thread per (trial, group of terms over at most 3 atoms;
// a water's angle and bonds form one group): every term's forces are
// converted to fixed point and summed per atom, exactly, so the group issues
// one reduction per atom and component (exact action-reaction: a bond's
// second atom and an angle's vertex take minus the others' forces).  The
// arithmetic of a term is that of bonded_force for the bond's first atom and
// for the angle's vertex.  A kernel of its own, beside the pair kernel: inside
// the pair kernel's warps the per-atom term loops ran on 8 of 32 lanes behind
// chains of dependent loads.
__device__ __forceinline__ void add3(long long (&F)[3][3], int m, long long x, long long y, long long z) {
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (q == m) { F[q][0] += x; F[q][1] += y; F[q][2] += z; }
}

__device__ __forceinline__ float4 pick3(const float4 (&p)[3], int m) { return m == 0 ? p[0] : m == 1 ? p[1] : p[2]; }

// group k of trial t's system
__device__ __forceinline__ void bonded_group(const Dev &d, int t, int k) {
  const TrialInfo T = d.tinfo[t];
  if (k >= d.sys_nbg[T.sys]) return;
  const BGroup G = d.bgrp[d.sys_bg0[T.sys] + k];
  const float L = T.box, iL = T.inv_box;
  int sl[3];
  float4 p[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    sl[m] = G.at[m] >= 0 ? d.slot_of[T.atom0 + G.at[m]] : -1;
    p[m] = sl[m] >= 0 ? d.pos[sl[m]] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  long long F[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q >= G.n) break;
    const int code = G.code[q];
    const float4 par = G.par[q];
    const int li = (code >> 1) & 3, lj = (code >> 3) & 3, ll = (code >> 5) & 3;
    const float4 pa = pick3(p, li), pb = pick3(p, lj);
    if ((code & 1) == 0) {
      // bond a-b, V = k/2 (r - r0)^2: the stretch in float-float (exact coordinate differences)
      const float nx = rintf((pb.x - pa.x) * iL), ny = rintf((pb.y - pa.y) * iL), nz = rintf((pb.z - pa.z) * iL);
      const ff dx = ff_diff(pb.x - L * nx, pa.x), dy = ff_diff(pb.y - L * ny, pa.y), dz = ff_diff(pb.z - L * nz, pa.z);
      const ff r = ff_sqrt(ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz)));
      const float dr = ff_add_f(ff_add_f(r, -par.x), -par.z).hi;  // r - r0 with r0 in float-float
      const float fs = par.y * dr / r.hi;  // force on a = +k dr (b - a)/r
      const long long fx = fx_from(fs * dx.hi), fy = fx_from(fs * dy.hi), fz = fx_from(fs * dz.hi);
      add3(F, li, fx, fy, fz);
      add3(F, lj, -fx, -fy, -fz);
    } else {
      // angle a-b-c (vertex b), V = k/2 (theta - theta0)^2
      const float4 pc = pick3(p, ll);
      const float3 u = min_disp(pb, pa, L, iL), v = min_disp(pb, pc, L, iL);
      const float uu = u.x * u.x + u.y * u.y + u.z * u.z, vv = v.x * v.x + v.y * v.y + v.z * v.z;
      const float iuv = rsqrtf(uu * vv);
      float cs = (u.x * v.x + u.y * v.y + u.z * v.z) * iuv;
      cs = fminf(1.0f, fmaxf(-1.0f, cs));
      const float dth = acosf(cs) - par.x;
      const float sn = fmaxf(sqrtf(fmaxf(0.0f, 1.0f - cs * cs)), 1e-6f);
      const float g = par.y * dth / sn;
      const float iuu = 1.0f / uu, ivv = 1.0f / vv;
      // forces on the ends: g d cos / d u and g d cos / d v
      const long long ax = fx_from(g * (v.x * iuv - cs * u.x * iuu)), ay = fx_from(g * (v.y * iuv - cs * u.y * iuu)),
                      az = fx_from(g * (v.z * iuv - cs * u.z * iuu));
      const long long cx = fx_from(g * (u.x * iuv - cs * v.x * ivv)), cy = fx_from(g * (u.y * iuv - cs * v.y * ivv)),
                      cz = fx_from(g * (u.z * iuv - cs * v.z * ivv));
      add3(F, li, ax, ay, az);
      add3(F, ll, cx, cy, cz);
      add3(F, lj, -(ax + cx), -(ay + cy), -(az + cz));
    }
  }
#pragma unroll
  for (int m = 0; m < 3; ++m)
    if (sl[m] >= 0) {
      red_add(d.fx + sl[m], F[m][0]);
      red_add(d.fy + sl[m], F[m][1]);
      red_add(d.fz + sl[m], F[m][2]);
    }
}

}  // namespace vp

// vp_pair.cu -- nonbonded (LJ + reaction field) and bonded forces.
//
// One warp per 8-atom i-cluster.  Lane l takes list entry e0 + l, one j-atom
// (the list holds only j-atoms with at least one pair in it); it loops over
// the 8 i-atoms, so the force on its j-atom is complete after the loop and
// goes to memory with one 64-bit fixed-point reduction per component.  i-forces stay in registers over the whole list
// and are reduced across the warp at the end.  FP32 pair arithmetic,
// order-independent int64 accumulation (2^32 units per kJ/mol/nm), so the
// forces are bit-reproducible.  Bonded forces (each atom computes its own
// share of every bond and angle it is part of) come from k_bonded; the
// energy kernel k_pair computes the bonded energies itself.
#include <algorithm>
#include <type_traits>

#include "vp_dev.cuh"
#include "vp_pair_dev.cuh"

namespace vp {


// force on one atom from its bonded terms (bonds: V = k/2 (r - r0)^2, angles
// V = k/2 (theta - theta0)^2); eb/ea receive this atom's share of the energy
__device__ float3 bonded_force(const Dev &d, const TrialInfo &T, int o, float4 self, float &eb, float &ea) {
  float3 F = make_float3(0.f, 0.f, 0.f);
  const int sa = T.sysatom0 + o;
  const int b0 = d.bt_start[sa], b1 = d.bt_start[sa + 1];
  const float L = T.box, iL = T.inv_box;
  for (int k = b0; k < b1; ++k) {
    const BTerm bt = d.bterm[k];
    if (bt.kind == 0) {
      // stiff springs: the stretch r - r0 in float-float (exact coordinate
      // differences), so that k (r - r0) keeps FP32 relative accuracy
      float4 pp = d.pos[d.slot_of[T.atom0 + bt.p1]];
      const float nx = rintf((pp.x - self.x) * iL), ny = rintf((pp.y - self.y) * iL), nz = rintf((pp.z - self.z) * iL);
      const ff dx = ff_diff(pp.x - L * nx, self.x), dy = ff_diff(pp.y - L * ny, self.y), dz = ff_diff(pp.z - L * nz, self.z);
      const ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
      const ff r = ff_sqrt(r2);
      const float dr = ff_add_f(r, -bt.x0).hi;
      const float fs = bt.k * dr / r.hi;  // force on self = +k dr (partner - self)/r
      F.x += fs * dx.hi; F.y += fs * dy.hi; F.z += fs * dz.hi;
      eb += 0.25f * bt.k * dr * dr;
    } else {
      float4 p1 = d.pos[d.slot_of[T.atom0 + bt.p1]];
      float4 p2 = d.pos[d.slot_of[T.atom0 + bt.p2]];
      float3 d1 = min_disp(self, p1, L, iL), d2 = min_disp(self, p2, L, iL);
      float3 u, v;
      if (bt.kind == 1) {  // self is an end; p1 vertex, p2 other end
        u = make_float3(-d1.x, -d1.y, -d1.z);
        v = make_float3(d2.x - d1.x, d2.y - d1.y, d2.z - d1.z);
      } else {  // self is the vertex; p1, p2 the ends
        u = d1;
        v = d2;
      }
      float uu = u.x * u.x + u.y * u.y + u.z * u.z, vv = v.x * v.x + v.y * v.y + v.z * v.z;
      float iuv = rsqrtf(uu * vv);
      float cs = (u.x * v.x + u.y * v.y + u.z * v.z) * iuv;
      cs = fminf(1.0f, fmaxf(-1.0f, cs));
      float th = acosf(cs);
      float dth = th - bt.x0;
      float sn = fmaxf(sqrtf(fmaxf(0.0f, 1.0f - cs * cs)), 1e-6f);
      float g = bt.k * dth / sn;
      float iuu = 1.0f / uu, ivv = 1.0f / vv;
      // d cos / d u and d cos / d v
      float3 du = make_float3(v.x * iuv - cs * u.x * iuu, v.y * iuv - cs * u.y * iuu, v.z * iuv - cs * u.z * iuu);
      if (bt.kind == 1) {
        F.x += g * du.x; F.y += g * du.y; F.z += g * du.z;
      } else {
        float3 dv = make_float3(u.x * iuv - cs * v.x * ivv, u.y * iuv - cs * v.y * ivv, u.z * iuv - cs * v.z * ivv);
        F.x -= g * (du.x + dv.x); F.y -= g * (du.y + dv.y); F.z -= g * (du.z + dv.z);
      }
      ea += (0.5f / 3.0f) * bt.k * dth * dth;
    }
  }
  return F;
}

// the 8 pairs of one lane: j-atom (xj, yj, zj, qj, type row tj) against the
// warp's 8 i-atoms.  Explicit round-to-nearest intrinsics pin the operation
// count (3 FADD, 6 FMUL, 12 FFMA, 1 RSQ, 1 LDS, 1 FSEL per pair).
template <bool EXACT, bool ENERGY>
__device__ __forceinline__ void pair_block(const float (&xi)[CL], const float (&yi)[CL], const float (&zi)[CL],
                                           const float (&qi)[CL], const int (&tio)[CL], float xj, float yj,
                                           float zj, float qj, int tj, unsigned mb, float L, float iL,
                                           const SimConst &c, const float2 *tab, const float *tshift,
                                           float (&fi)[CL][3], float &fjx, float &fjy, float &fjz, float &elj,
                                           float &erf) {
#pragma unroll
  for (int a = 0; a < CL; ++a) {
    float dx = __fsub_rn(xj, xi[a]), dy = __fsub_rn(yj, yi[a]), dz = __fsub_rn(zj, zi[a]);
    if (EXACT) {
      dx = __fmaf_rn(-L, rintf(__fmul_rn(dx, iL)), dx);
      dy = __fmaf_rn(-L, rintf(__fmul_rn(dy, iL)), dy);
      dz = __fmaf_rn(-L, rintf(__fmul_rn(dz, iL)), dz);
    }
    const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    const bool in = ((mb >> a) & 1u) && (r2 < c.rc2);
    const float rinv = rsqrtf(r2);
    const float rinv2 = __fmul_rn(rinv, rinv);
    const float rinv6 = __fmul_rn(__fmul_rn(rinv2, rinv2), rinv2);
    const float2 cc = tab[tio[a] + tj];
    const float qq = __fmul_rn(qi[a], qj);
    float t = __fmaf_rn(cc.y, rinv6, -cc.x);
    t = __fmul_rn(t, rinv6);
    t = __fmaf_rn(qq, rinv, t);
    t = __fmul_rn(t, rinv2);
    float f = __fmaf_rn(-qq, c.two_krf, t);
    f = in ? f : 0.0f;
    fi[a][0] = __fmaf_rn(-f, dx, fi[a][0]);
    fi[a][1] = __fmaf_rn(-f, dy, fi[a][1]);
    fi[a][2] = __fmaf_rn(-f, dz, fi[a][2]);
    fjx = __fmaf_rn(f, dx, fjx);
    fjy = __fmaf_rn(f, dy, fjy);
    fjz = __fmaf_rn(f, dz, fjz);
    if (ENERGY && in) {
      elj += rinv6 * (cc.y * (1.0f / 12.0f) * rinv6 - cc.x * (1.0f / 6.0f)) - tshift[tio[a] + tj];
      erf += qq * (rinv + c.krf * r2 - c.crf);
    }
  }
}

template <bool ENERGY, int MINB>
__global__ void __launch_bounds__(128, MINB) k_pair(Dev d, SimConst c, int only_trial) {
  extern __shared__ float2 smem_tab[];
  __shared__ float s_red[ENERGY ? 1 : 4][ENERGY ? 1 : 3 * CL * 33];
  float2 *tab = smem_tab;
  float *tshift = reinterpret_cast<float *>(smem_tab + c.n_types * c.n_types);
  const int nt2 = c.n_types * c.n_types;
  for (int k = threadIdx.x; k < nt2; k += blockDim.x) {
    tab[k] = d.ljtab[k];
    if (ENERGY) tshift[k] = d.ljshift[k];
  }
  __syncthreads();
  const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (I >= d.total_clus) return;
  const int t = d.clus_trial[I];
  if (only_trial >= 0 && t != only_trial) return;
  const TrialInfo T = d.tinfo[t];
  if (I - T.clus0 >= d.tstate[t].n_clus) return;
  const float L = T.box, iL = T.inv_box;

  float xi[CL], yi[CL], zi[CL], qi[CL];
  int tio[CL];
#pragma unroll
  for (int a = 0; a < CL; ++a) {
    float4 p = d.pos[I * CL + a];
    xi[a] = p.x; yi[a] = p.y; zi[a] = p.z; qi[a] = p.w;
    tio[a] = d.type[I * CL + a] * c.n_types;
  }
  float fi[CL][3];
#pragma unroll
  for (int a = 0; a < CL; ++a) fi[a][0] = fi[a][1] = fi[a][2] = 0.0f;
  float elj = 0.0f, erf = 0.0f;

  const int n = d.list_n[I];
  const uint32_t *seg = d.list + (size_t)I * c.list_cap;
  const uint8_t *segm = d.list_m + (size_t)I * c.list_cap;
  // one j-atom entry per lane; software pipeline: the entry two groups ahead
  // and the j-atom of the next group are in flight while the current group is
  // evaluated; idle lanes get an empty mask
  uint32_t ent = lane < n ? seg[lane] : d.idle_entry;
  uint32_t ent_n = 32 + lane < n ? seg[32 + lane] : d.idle_entry;
  float4 pj = d.pos[(int)(ent & J_MASK)];
  int tj = d.type[(int)(ent & J_MASK)];
  for (int e0 = 0; e0 < n; e0 += 32) {
    const uint32_t ent_nn = e0 + 64 + lane < n ? seg[e0 + 64 + lane] : d.idle_entry;
    const int sj_n = (int)(ent_n & J_MASK);
    const float4 pj_n = d.pos[sj_n];
    const int tj_n = d.type[sj_n];
    const int sj = (int)(ent & J_MASK);
    const unsigned sh = ent >> J_BITS;
    const float xj = pj.x - L * (float)((int)(sh & 3u) - 1);
    const float yj = pj.y - L * (float)((int)((sh >> 2) & 3u) - 1);
    const float zj = pj.z - L * (float)((int)((sh >> 4) & 3u) - 1);
    const unsigned mb = e0 + lane < n ? segm[e0 + lane] : 0u;
    const bool exact = (ent & E_EXACT) != 0u;
    float fjx = 0.f, fjy = 0.f, fjz = 0.f;
    if (!__any_sync(0xffffffffu, exact))
      pair_block<false, ENERGY>(xi, yi, zi, qi, tio, xj, yj, zj, pj.w, tj, mb, L, iL, c, tab, tshift, fi, fjx, fjy,
                                fjz, elj, erf);
    else if (exact)
      pair_block<true, ENERGY>(xi, yi, zi, qi, tio, xj, yj, zj, pj.w, tj, mb, L, iL, c, tab, tshift, fi, fjx, fjy,
                               fjz, elj, erf);
    else
      pair_block<false, ENERGY>(xi, yi, zi, qi, tio, xj, yj, zj, pj.w, tj, mb, L, iL, c, tab, tshift, fi, fjx, fjy,
                                fjz, elj, erf);
    if (!ENERGY && (fjx != 0.f || fjy != 0.f || fjz != 0.f)) {
      red_add(d.fx + sj, fx_from(fjx));
      red_add(d.fy + sj, fx_from(fjy));
      red_add(d.fz + sj, fx_from(fjz));
    }
    ent = ent_n;
    ent_n = ent_nn;
    pj = pj_n;
    tj = tj_n;
  }

  // bonded terms of the 8 i-atoms (lanes 0..7)
  float eb = 0.f, ea = 0.f;
  if (lane < CL) {
    const int o = d.orig[I * CL + lane];
    if (o >= 0) {
      float4 self = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int a = 0; a < CL; ++a)
        if (a == lane) self = make_float4(xi[a], yi[a], zi[a], 0.f);
      float3 fb = bonded_force(d, T, o, self, eb, ea);
#pragma unroll
      for (int a = 0; a < CL; ++a)
        if (a == lane) { fi[a][0] += fb.x; fi[a][1] += fb.y; fi[a][2] += fb.z; }
    }
  }

  if (!ENERGY) {
    // i-forces: column sums of the 32 lanes' partials in a fixed order
    float *r = s_red[threadIdx.x >> 5];
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
  } else {
    double e4[4] = {(double)elj, (double)erf, (double)eb, (double)ea};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) e4[k] += __shfl_xor_sync(0xffffffffu, e4[k], off);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 4; ++k) red_add(d.energy + (size_t)t * 5 + k, __double2ll_rn(e4[k] * E_SCALE));
  }
}


// Force-only kernel (the hot path).  Per warp, shared memory holds the LJ
// coefficients of its 8 i-atoms against every type (row a at a fixed stride,
// so the pair loop addresses them with immediate offsets) and the 27 image
// shifts of its box; the list mask enters the squared distance as a penalty
// (0 or 1e30), so a masked pair falls outside the cut-off without any
// per-pair bit test.  Arithmetic per pair: 3 FADD, 6 FMUL, 12 FFMA, 1 RSQ,
// 1 LDS, 1 FSETP + FSEL.
// SHI: the i-atoms are read from shared memory (one broadcast LDS.128 per
// pair) instead of being held in 32 registers, which lets more warps reside.
// TS is the row stride of the per-warp LJ table (at least the number of types).
template <int MINB, bool SHI, int TS>
__global__ void __launch_bounds__(PF_WARPS * 32, MINB) k_pair_f(Dev d, SimConst c, const int *clist, int n_items) {
  __shared__ float2 s_cij[PF_WARPS][CL][TS];
  __shared__ float4 s_sh[PF_WARPS][64];
  __shared__ float4 s_i[PF_WARPS][CL];
  __shared__ float s_red[PF_WARPS][3 * CL * 33];
  const int wib = threadIdx.x >> 5;
  const int item = blockIdx.x * PF_WARPS + wib;
  const int lane = threadIdx.x & 31;
  if (item >= n_items) return;
  const int I = clist ? clist[item] : item;
  const int t = d.clus_trial[I];
  const TrialInfo T = d.tinfo[t];
  if (I - T.clus0 >= d.tstate[t].n_clus) return;
  const float L = T.box, iL = T.inv_box;
  const int NT = c.n_types;

  float xi[CL], yi[CL], zi[CL], qi[CL];
  int ti[CL];
#pragma unroll
  for (int a = 0; a < CL; ++a) {
    const float4 p = d.pos[I * CL + a];
    xi[a] = p.x; yi[a] = p.y; zi[a] = p.z; qi[a] = p.w;
    ti[a] = d.type[I * CL + a];
  }
  if (SHI && lane < CL) s_i[wib][lane] = d.pos[I * CL + lane];
  // per-warp tables: LJ rows of the i-atoms, image shifts (code = (nx+1) | (ny+1)<<2 | (nz+1)<<4)
  for (int k = lane; k < CL * NT; k += 32) {
    const int a = k / NT, tj = k - a * NT;
    int tia = ti[0];
#pragma unroll
    for (int q = 1; q < CL; ++q)
      if (q == a) tia = ti[q];
    s_cij[wib][a][tj] = d.ljtab[tia * NT + tj];
  }
  for (int k = lane; k < 64; k += 32) {
    const int nx = (k & 3) - 1, ny = ((k >> 2) & 3) - 1, nz = ((k >> 4) & 3) - 1;
    s_sh[wib][k] = make_float4(L * nx, L * ny, L * nz, 0.f);
  }
  __syncwarp();
  float fi[CL][3];
#pragma unroll
  for (int a = 0; a < CL; ++a) fi[a][0] = fi[a][1] = fi[a][2] = 0.0f;

  const int n = d.list_n[I], nm = d.list_nm[I];
  const uint32_t *seg = d.list + (size_t)I * c.list_cap;
  const uint8_t *segm = d.list_m + (size_t)I * c.list_cap;
  uint32_t ent = lane < n ? seg[lane] : d.idle_entry;
  uint32_t ent_n = 32 + lane < n ? seg[32 + lane] : d.idle_entry;
  float4 pj = d.pos[(int)(ent & J_MASK)];
  int tj = d.type[(int)(ent & J_MASK)];
  for (int e0 = 0; e0 < n; e0 += 32) {
    const uint32_t ent_nn = e0 + 64 + lane < n ? seg[e0 + 64 + lane] : d.idle_entry;
    const int sj_n = (int)(ent_n & J_MASK);
    const float4 pj_n = d.pos[sj_n];
    const int tj_n = d.type[sj_n];
    const int sj = (int)(ent & J_MASK);
    const float4 shv = s_sh[wib][(ent >> J_BITS) & 63u];
    const float xj = pj.x - shv.x, yj = pj.y - shv.y, zj = pj.z - shv.z, qj = pj.w;
    const bool masked = e0 < nm;
    const unsigned mb = masked && e0 + lane < n ? segm[e0 + lane] : 0u;
    const bool exact = (ent & E_EXACT) != 0u;
    const float2 *row = &s_cij[wib][0][tj];
    // j-force: even and odd i-atoms in two partial sums (the packed variant's order)
    float fjx[2] = {0.f, 0.f}, fjy[2] = {0.f, 0.f}, fjz[2] = {0.f, 0.f};
    // one image per entry; MASKED: the pair masks apply (a group with
    // exclusions or the cluster itself); else the cut-off alone decides, which
    // gives the same forces: a listed pair that failed the list rule is still
    // beyond the cut-off (lists are rebuilt before any atom has moved skin/2)
    auto one_image = [&](auto mtag) {
      constexpr bool MASKED = decltype(mtag)::value;
#pragma unroll
      for (int a = 0; a < CL; ++a) {
        const float4 ia = SHI ? s_i[wib][a] : make_float4(xi[a], yi[a], zi[a], qi[a]);
        const float pen = MASKED ? ((mb & (1u << a)) ? 0.0f : MASK_PEN) : 0.0f;
        const float dx = __fsub_rn(xj, ia.x), dy = __fsub_rn(yj, ia.y), dz = __fsub_rn(zj, ia.z);
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmaf_rn(dx, dx, pen)));
        const float rinv = rsqrtf(r2);
        const float rinv2 = __fmul_rn(rinv, rinv);
        const float rinv6 = __fmul_rn(__fmul_rn(rinv2, rinv2), rinv2);
        const float2 cc = row[a * TS];
        const float qq = __fmul_rn(ia.w, qj);
        float tt = __fmaf_rn(cc.y, rinv6, -cc.x);
        tt = __fmul_rn(tt, rinv6);
        tt = __fmaf_rn(qq, rinv, tt);
        tt = __fmul_rn(tt, rinv2);
        float f = __fmaf_rn(-qq, c.two_krf, tt);
        f = r2 < c.rc2 ? f : 0.0f;
        fi[a][0] = __fmaf_rn(-f, dx, fi[a][0]);
        fi[a][1] = __fmaf_rn(-f, dy, fi[a][1]);
        fi[a][2] = __fmaf_rn(-f, dz, fi[a][2]);
        fjx[a & 1] = __fmaf_rn(f, dx, fjx[a & 1]);
        fjy[a & 1] = __fmaf_rn(f, dy, fjy[a & 1]);
        fjz[a & 1] = __fmaf_rn(f, dz, fjz[a & 1]);
      }
    };
    if (!masked) {
      one_image(std::false_type{});
    } else if (!__any_sync(0xffffffffu, exact)) {
      one_image(std::true_type{});
    } else {
      // some entry of this group needs pair-by-pair minimum images
#pragma unroll
      for (int a = 0; a < CL; ++a) {
        const float4 ia = SHI ? s_i[wib][a] : make_float4(xi[a], yi[a], zi[a], qi[a]);
        const float pen = (mb & (1u << a)) ? 0.0f : MASK_PEN;
        float dx = __fsub_rn(xj, ia.x), dy = __fsub_rn(yj, ia.y), dz = __fsub_rn(zj, ia.z);
        if (exact) {
          dx = __fmaf_rn(-L, rintf(__fmul_rn(dx, iL)), dx);
          dy = __fmaf_rn(-L, rintf(__fmul_rn(dy, iL)), dy);
          dz = __fmaf_rn(-L, rintf(__fmul_rn(dz, iL)), dz);
        }
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmaf_rn(dx, dx, pen)));
        const float rinv = rsqrtf(r2);
        const float rinv2 = __fmul_rn(rinv, rinv);
        const float rinv6 = __fmul_rn(__fmul_rn(rinv2, rinv2), rinv2);
        const float2 cc = row[a * TS];
        const float qq = __fmul_rn(ia.w, qj);
        float tt = __fmaf_rn(cc.y, rinv6, -cc.x);
        tt = __fmul_rn(tt, rinv6);
        tt = __fmaf_rn(qq, rinv, tt);
        tt = __fmul_rn(tt, rinv2);
        float f = __fmaf_rn(-qq, c.two_krf, tt);
        f = r2 < c.rc2 ? f : 0.0f;
        fi[a][0] = __fmaf_rn(-f, dx, fi[a][0]);
        fi[a][1] = __fmaf_rn(-f, dy, fi[a][1]);
        fi[a][2] = __fmaf_rn(-f, dz, fi[a][2]);
        fjx[a & 1] = __fmaf_rn(f, dx, fjx[a & 1]);
        fjy[a & 1] = __fmaf_rn(f, dy, fjy[a & 1]);
        fjz[a & 1] = __fmaf_rn(f, dz, fjz[a & 1]);
      }
    }
    const float sx = fjx[0] + fjx[1], sy = fjy[0] + fjy[1], sz = fjz[0] + fjz[1];
    if (sx != 0.f || sy != 0.f || sz != 0.f) {
      red_add(d.fx + sj, fx_from(sx));
      red_add(d.fy + sj, fx_from(sy));
      red_add(d.fz + sj, fx_from(sz));
    }
    ent = ent_n;
    ent_n = ent_nn;
    pj = pj_n;
    tj = tj_n;
  }

  // i-forces: column sums of the 32 lanes' partials in a fixed order
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

// Packed variant: the same pair loop on FP32x2 arithmetic (FADD2, FMUL2,
// FFMA2: one instruction for two pairs) over the i-atom pairs (2p, 2p+1).
// The i-atoms sit in shared memory as {-x, -x', -y, -y'} {-z, -z', q, q'} and the
// LJ row of an i-atom pair is {c12, c12', -c6, -c6'}; per two pairs the loop
// issues 3 FADD2, 6 FMUL2, 7 FFMA2, 2 RSQ, 3 LDS.128 and, per pair, one mask
// test joined with the cut-off test and a select (a masked pair may compute
// inf or NaN on the way; the select discards it).  The i-force partials accumulate +f*d and are negated once
// (exactly the sum of -f*d: round-to-nearest is sign-symmetric); the j-force
// sums even and odd i-atoms in two partials, as the scalar variants do, so
// all variants give bit-identical forces.


template <int MINB>
__global__ void __launch_bounds__(PF_WARPS * 32, MINB) k_pair_f2(Dev d, SimConst c, unsigned *next, const int *clist,
                                                                   int n_items) {
  __shared__ PairF2Shared sh;
  const int lane = threadIdx.x & 31;
  // persistent warps: each takes the next i-cluster from a counter until none
  // is left, so that short and long lists even out across the SMs
  for (;;) {
    __syncwarp();  // the warp's tables of its previous cluster are no longer read
    unsigned got = 0u;
    if (lane == 0) got = atomicAdd(next, 1u);
    const int item = (int)__shfl_sync(0xffffffffu, got, 0);
    if (item >= n_items) return;
    pair_cluster_f2(d, c, sh, clist ? clist[item] : item);
  }
}

__global__ void __launch_bounds__(256) k_bonded(Dev d) {
  bonded_group(d, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x);
}

void launch_bonded(const Dev &d, cudaStream_t s) {
  if (d.max_nbg <= 0) return;
  k_bonded<<<dim3((unsigned)((d.max_nbg + 255) / 256), (unsigned)d.n_trials), 256, 0, s>>>(d);
}

// variants differ in the register cap (blocks per SM the compiler must fit)
// and in where the i-atoms live: 0/1/2: registers, 4/5/6 blocks; 3/4/5:
// shared memory and an LJ table for at most SMALL_TYPES types (less shared
// memory per block), 6/7/8 blocks (larger type sets fall back to variant 0).
// All variants do the same arithmetic in the same order (bit-identical forces).
void launch_pair(const Dev &d, const SimConst &c, bool energy, int32_t only_trial, cudaStream_t s, int variant,
                 const int *clist, int n_items) {
  long long threads = (long long)d.total_clus * 32;
  unsigned blocks = (unsigned)((threads + 127) / 128);
  const size_t nt2 = (size_t)c.n_types * c.n_types;
  if (energy || only_trial >= 0) {
    k_pair<true, 4><<<blocks, 128, nt2 * (sizeof(float2) + sizeof(float)), s>>>(d, c, only_trial);
    return;
  }
  if (!clist) n_items = d.total_clus;
  if (n_items <= 0) return;
  const unsigned fb = (unsigned)((n_items + PF_WARPS - 1) / PF_WARPS);
  if (variant >= 3 && c.n_types > SMALL_TYPES) variant = 0;
  switch (variant) {
    case 1: k_pair_f<5, false, MAX_TYPES><<<fb, PF_WARPS * 32, 0, s>>>(d, c, clist, n_items); break;
    case 2: k_pair_f<6, false, MAX_TYPES><<<fb, PF_WARPS * 32, 0, s>>>(d, c, clist, n_items); break;
    case 3: k_pair_f<6, true, SMALL_TYPES><<<fb, PF_WARPS * 32, 0, s>>>(d, c, clist, n_items); break;
    case 4: k_pair_f<7, true, SMALL_TYPES><<<fb, PF_WARPS * 32, 0, s>>>(d, c, clist, n_items); break;
    case 5: k_pair_f<8, true, SMALL_TYPES><<<fb, PF_WARPS * 32, 0, s>>>(d, c, clist, n_items); break;
    case 6: case 7: case 8: {
      // persistent grid: as many blocks as can be resident, sized from the SM
      // count; the counter hands out the i-clusters
      const int minb = variant - 1;
      const unsigned pb = std::min(fb, (unsigned)(d.n_sm * minb));
      cudaMemsetAsync(d.pair_next, 0, sizeof(unsigned), s);
      if (variant == 6) k_pair_f2<5><<<pb, PF_WARPS * 32, 0, s>>>(d, c, d.pair_next, clist, n_items);
      else if (variant == 7) k_pair_f2<6><<<pb, PF_WARPS * 32, 0, s>>>(d, c, d.pair_next, clist, n_items);
      else k_pair_f2<7><<<pb, PF_WARPS * 32, 0, s>>>(d, c, d.pair_next, clist, n_items);
      break;
    }
    default: k_pair_f<4, false, MAX_TYPES><<<fb, PF_WARPS * 32, 0, s>>>(d, c, clist, n_items); break;
  }
}

}  // namespace vp

// vp_cv_dev.cuh -- device functions of the reaction coordinate (one warp's
// tile of the contact-pair triangle, one trial's finaliser), shared by the
// separate kernels and the one-kernel step.
#pragma once
#include "vp_cvpair.cuh"
#include "vp_dev.cuh"

namespace vp {

__device__ __forceinline__ long long gsum(int hi, unsigned lo) { return (long long)hi * 16777216ll + (long long)lo; }

// One warp's tile of the contact-pair triangle: the work item wq of the flat
// (trial, tile) list, in the work order.
__device__ __forceinline__ void cv_tile(const Dev &d, const SimConst &c, CvWarpShared &sh, int wq) {
  auto &s_near = sh.s_near;
  auto &s_x = sh.s_x;
  auto &s_ghi = sh.s_ghi;
  auto &s_glo = sh.s_glo;
  const int lane = threadIdx.x & 31;
  const int w = d.work_order[wq];  // costliest tiles first (the partial sums keep their slots)
  const int2 wk = d.work[w];
  const TrialInfo T = d.tinfo[wk.x];
  const int2 bij = d.tiles[wk.y];
  const int ncv = T.n_cv, msep = c.cv_min_sep;
  const float L = T.box, iL = T.inv_box;
  const int i = bij.x * CV_T + lane;
  const int jl = bij.y * CV_T + lane;
  float3 xi = make_float3(0.f, 0.f, 0.f), xj = make_float3(0.f, 0.f, 0.f);
  if (i < ncv) { float4 q = d.pos[d.slot_of[T.atom0 + i]]; xi = make_float3(q.x, q.y, q.z); }
  if (jl < ncv) { float4 q = d.pos[d.slot_of[T.atom0 + jl]]; xj = make_float3(q.x, q.y, q.z); }
  s_x[lane][0] = xi.x; s_x[lane][1] = xi.y; s_x[lane][2] = xi.z;
  s_x[CV_T + lane][0] = xj.x; s_x[CV_T + lane][1] = xj.y; s_x[CV_T + lane][2] = xj.z;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    s_ghi[lane][q] = 0; s_ghi[CV_T + lane][q] = 0;
    s_glo[lane][q] = 0u; s_glo[CV_T + lane][q] = 0u;
  }
  // ---- phase 1: near pairs of the tile ----
  int n_near = 0;
  for (int k = 0; k < CV_T; ++k) {
    const int jc = (lane + k) & (CV_T - 1);
    const int j = bij.y * CV_T + jc;
    const float xjx = __shfl_sync(0xffffffffu, xj.x, jc);
    const float xjy = __shfl_sync(0xffffffffu, xj.y, jc);
    const float xjz = __shfl_sync(0xffffffffu, xj.z, jc);
    bool near = false;
    if (i < ncv && j < ncv && j - i > msep) {
      float dx = xjx - xi.x, dy = xjy - xi.y, dz = xjz - xi.z;
      dx -= L * rintf(dx * iL);
      dy -= L * rintf(dy * iL);
      dz -= L * rintf(dz * iL);
      near = dx * dx + dy * dy + dz * dz < c.cv_rc2_far;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, near);
    if (near) s_near[n_near + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)(lane | (jc << 5));
    n_near += __popc(bal);
  }
  __syncwarp();
  // ---- phase 2: the near pairs, densely ----
  const CvConst k = cv_const(c);
  const float2 *cn = d.cnat_ff + (size_t)wk.y * CV_T * CV_T;
  ff zacc = {0.f, 0.f};
  for (int base = 0; base < n_near; base += 32) {
    const int idx = base + lane;
    if (idx < n_near) {
      const unsigned e = s_near[idx];
      const int il = e & 31, jc = e >> 5;
      const float3 pi = make_float3(s_x[il][0], s_x[il][1], s_x[il][2]);
      ff dx, dy, dz;
      cv_delta(pi, s_x[CV_T + jc][0], s_x[CV_T + jc][1], s_x[CV_T + jc][2], L, iL, dx, dy, dz);
      const float2 cv2 = cn[((jc - il) & (CV_T - 1)) * CV_T + il];
      const ff cnat = {cv2.x, cv2.y};
      const ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
      const CvPair cp = cv_contact<false>(r2, k);
      const ff h = ff_add(cp.Ct, ff_neg(cnat));
      // z term: C~ (C~ - 2 C~_nat) = (C~ - C~_nat)^2 - C~_nat^2
      zacc = ff_add(zacc, ff_mul(cp.Ct, ff_add(cp.Ct, ff{-2.0f * cnat.hi, -2.0f * cnat.lo})));  // doubling is exact
      // dz/dx_i = -w d, dz/dx_j = +w d with d = x_j - x_i, w = 2 h C~'(r)/r
      const float wgt = 2.0f * h.hi * cp.dCt / cp.r;
      if (wgt != 0.0f) {
        const long long gx = fx_from(wgt * dx.hi), gy = fx_from(wgt * dy.hi), gz = fx_from(wgt * dz.hi);
        const long long gv[3] = {gx, gy, gz};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          atomicAdd(&s_ghi[il][q], (int)((-gv[q]) >> 24));
          atomicAdd(&s_glo[il][q], (unsigned)((-gv[q]) & 0xffffff));
          atomicAdd(&s_ghi[CV_T + jc][q], (int)(gv[q] >> 24));
          atomicAdd(&s_glo[CV_T + jc][q], (unsigned)(gv[q] & 0xffffff));
        }
      }
    }
  }
  __syncwarp();
  if (n_near > 0) {
    if (i < ncv) {
      const long long a0 = gsum(s_ghi[lane][0], s_glo[lane][0]),
                      a1 = gsum(s_ghi[lane][1], s_glo[lane][1]),
                      a2 = gsum(s_ghi[lane][2], s_glo[lane][2]);
      if (a0 | a1 | a2) { red_add(d.gx + T.cv0 + i, a0); red_add(d.gy + T.cv0 + i, a1); red_add(d.gz + T.cv0 + i, a2); }
    }
    if (jl < ncv) {
      const long long a0 = gsum(s_ghi[CV_T + lane][0], s_glo[CV_T + lane][0]),
                      a1 = gsum(s_ghi[CV_T + lane][1], s_glo[CV_T + lane][1]),
                      a2 = gsum(s_ghi[CV_T + lane][2], s_glo[CV_T + lane][2]);
      if (a0 | a1 | a2) { red_add(d.gx + T.cv0 + jl, a0); red_add(d.gy + T.cv0 + jl, a1); red_add(d.gz + T.cv0 + jl, a2); }
    }
  }
  double zl = ff_to_d(zacc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) zl += __shfl_xor_sync(0xffffffffu, zl, off);
  if (lane == 0) d.z_part[w] = zl;
}


// The finaliser of trial t by one block of any size: the reduction runs over
// CVFIN_THREADS virtual threads in a fixed tree, so z is the same bit for bit
// whatever block runs it.  Returns true in the block that finished the last
// trial of the step (FIN_STEP: the step counter and the kick then advance).
template <int MODE>
__device__ bool cvfin_trial(const Dev &d, const SimConst &c, CvfinShared &sh, int t) {
  double *rz = sh.rz, *rq = sh.rq;
  const TrialInfo T = d.tinfo[t];
  const long long step_now = *d.step;
  for (int v = threadIdx.x; v < CVFIN_THREADS; v += blockDim.x) {
    double zs = 0.0, q = 0.0;
    for (int k = v; k < T.n_work; k += CVFIN_THREADS) zs += d.z_part[T.work0 + k];
    for (int i = v; i < T.n_cv; i += CVFIN_THREADS) {
      double gx = (double)d.gx[T.cv0 + i] * 2.3283064365386963e-10;
      double gy = (double)d.gy[T.cv0 + i] * 2.3283064365386963e-10;
      double gz = (double)d.gz[T.cv0 + i] * 2.3283064365386963e-10;
      q += (gx * gx + gy * gy + gz * gz) * d.inv_gm[T.sysatom0 + i];  // FP64 division is slow on this part
    }
    rz[v] = zs;
    rq[v] = q;
  }
  __syncthreads();
  for (int off = CVFIN_THREADS / 2; off > 0; off >>= 1) {
    for (int v = threadIdx.x; v < off; v += blockDim.x) { rz[v] += rz[v + off]; rq[v] += rq[v + off]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    TrialState &S = d.tstate[t];
    const double z = S.zconst + rz[0];
    const double Q = rq[0];
    double a = 0.0, phi = 0.0;
    if (MODE == FIN_INIT) {
      S.zm = z;
    } else {
      a = z > S.zm ? z - S.zm : 0.0;
      if (MODE == FIN_STEP) {
        phi = c.kR_half_d * c.kR_half_d * a * a * Q;
        S.Phi += c.dt_d * phi;
      }
      if (z < S.zm) S.zm = z;
    }
    S.z = z;
    S.a = a;
    S.phi = phi;
    if (!isfinite(z)) atomicOr(d.err, ERR_NONFINITE);
    if (c.rec_cap > 0 && MODE != FIN_KEEP) {
      long long n = MODE == FIN_STEP ? step_now + 1 : step_now;
      double *r = d.rec + ((size_t)t * c.rec_cap + (size_t)(n % c.rec_cap)) * 5;
      r[0] = z; r[1] = S.zm; r[2] = a; r[3] = phi; r[4] = Q;
    }
    if (MODE == FIN_STEP) {
      __threadfence();
      unsigned ticket = atomicAdd(d.done, 1u);
      sh.last = ticket == (unsigned)(d.n_trials - 1);
    } else {
      sh.last = false;
    }
  }
  __syncthreads();
  const bool last = sh.last;
  if (MODE == FIN_STEP && last && threadIdx.x == 0) {
    *d.step = step_now + 1;
    *d.kick = 1.0f;
    *d.done = 0u;
  }
  __syncthreads();  // the shared arrays may be reused by the caller
  return last;
}

}  // namespace vp

// vp_cv.cu -- the contact-map reaction coordinate z(X), its gradient, and the
// per-step ratchet bookkeeping and bias functional.
//
// z = sum over pairs i < j < n_cv with j - i > min_sep of (C~(r_ij) - C~_nat)^2
// (SM, "Collective coordinate").  Written as z = Z0 + sum over pairs closer
// than the contact cut-off of C~ (C~ - 2 C~_nat), Z0 = sum of C~_nat^2, so far
// pairs cost one FP32 distance test.  Near pairs are evaluated in
// float-float arithmetic (about 44 significant bits on the FP32 pipes):
// the ratchet amplitude a = z - z_m is a small difference of large sums and
// the functional needs it to ~1e-6 relative.  Gradients are accumulated in
// 64-bit fixed point, z partial sums in FP64.
//
// Work item = (trial, 32 x 32 tile of the pair triangle); one warp per item.
// Lane l owns i = bi*32 + l; at step k it takes column (l + k) mod 32, and the
// column accumulators travel one lane per step around the warp so that every
// column sum is built in a fixed order without atomics inside the tile.
#include "vp_dev.cuh"

namespace vp {

// C(s) with s = (r/r0)^2: (1 + s + s^2) / (1 + s + s^2 + s^3 + s^4), the printed
// (1 - rho^6)/(1 - rho^10) with the common factor (1 - s) cancelled
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

// one warp per (system tile); C~ of the native structure in FP64
__global__ void k_cnat(Dev d, SimConst c, const double *native, const int32_t *sys_nat0, const int32_t *tile_sys,
                       int32_t n_tiles) {
  int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (tile >= n_tiles) return;
  int sys = tile_sys[tile];
  int2 bij = d.tiles[tile];
  int ncv = d.sys_ncv[sys], msep = d.sys_minsep[sys];
  const double *X = native + 3 * (size_t)sys_nat0[sys];
  const double r0 = c.cv_r0_d, rs = c.cv_rs_d, rc = c.cv_rc_d;
  int i = bij.x * CV_T + lane;
  for (int k = 0; k < CV_T; ++k) {
    int j = bij.y * CV_T + ((lane + k) & (CV_T - 1));
    double v = 0.0;
    if (i < ncv && j < ncv && j - i > msep) {
      double dx = X[3 * j] - X[3 * i], dy = X[3 * j + 1] - X[3 * i + 1], dz = X[3 * j + 2] - X[3 * i + 2];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      double s = (r / r0) * (r / r0);
      double N = 1.0 + s + s * s, D = N + s * s * s + s * s * s * s;
      double C = N / D, S = 1.0;
      if (r >= rc) S = 0.0;
      else if (r > rs) {
        double x = (r - rs) / (rc - rs);
        S = 1.0 - x * x * x * (10.0 - 15.0 * x + 6.0 * x * x);
      }
      v = C * S;
    }
    d.cnat[(size_t)tile * CV_T * CV_T + k * CV_T + lane] = v;
  }
}

// per trial: Z0 = sum of C~_nat^2 over the system's contact pairs (fixed order)
__global__ void k_zconst(Dev d, const int32_t *sys_tile0, const int32_t *sys_ntiles) {
  __shared__ double red[256];
  int t = blockIdx.x;
  int sys = d.tinfo[t].sys;
  size_t b = (size_t)sys_tile0[sys] * CV_T * CV_T, n = (size_t)sys_ntiles[sys] * CV_T * CV_T;
  double acc = 0.0;
  for (size_t k = threadIdx.x; k < n; k += blockDim.x) {
    double v = d.cnat[b + k];
    acc += v * v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) d.tstate[t].zconst = red[0];
}

__global__ void __launch_bounds__(128) k_cv(Dev d, SimConst c) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= d.total_work) return;
  const int2 wk = d.work[w];
  const TrialInfo T = d.tinfo[wk.x];
  const int2 bij = d.tiles[wk.y];
  const int ncv = T.n_cv, msep = c.cv_min_sep;
  const float L = T.box, iL = T.inv_box;
  const int i = bij.x * CV_T + lane;
  const int jl = bij.y * CV_T + lane;
  float3 xi = make_float3(0.f, 0.f, 0.f), xj = make_float3(0.f, 0.f, 0.f);
  if (i < ncv) { float4 p = d.pos[d.slot_of[T.atom0 + i]]; xi = make_float3(p.x, p.y, p.z); }
  if (jl < ncv) { float4 p = d.pos[d.slot_of[T.atom0 + jl]]; xj = make_float3(p.x, p.y, p.z); }
  const ff inv_r0sq = {c.cv_inv_r0sq_hi, c.cv_inv_r0sq_lo};
  const double *cn = d.cnat + (size_t)wk.y * CV_T * CV_T;
  long long gix = 0, giy = 0, giz = 0, gjx = 0, gjy = 0, gjz = 0;
  ff zacc = {0.f, 0.f};
  for (int k = 0; k < CV_T; ++k) {
    const int jc = (lane + k) & (CV_T - 1);
    const int j = bij.y * CV_T + jc;
    const float xjx = __shfl_sync(0xffffffffu, xj.x, jc);
    const float xjy = __shfl_sync(0xffffffffu, xj.y, jc);
    const float xjz = __shfl_sync(0xffffffffu, xj.z, jc);
    if (i < ncv && j < ncv && j - i > msep) {
      ff dx = ff_diff(xjx, xi.x), dy = ff_diff(xjy, xi.y), dz = ff_diff(xjz, xi.z);
      float nx = rintf(dx.hi * iL), ny = rintf(dy.hi * iL), nz = rintf(dz.hi * iL);
      if (nx != 0.f) dx = ff_add_f(dx, -L * nx);
      if (ny != 0.f) dy = ff_add_f(dy, -L * ny);
      if (nz != 0.f) dz = ff_add_f(dz, -L * nz);
      const float r2f = dx.hi * dx.hi + dy.hi * dy.hi + dz.hi * dz.hi;
      if (r2f < c.cv_rc2_far) {
        const ff cnat = ff_from_d(cn[k * CV_T + lane]);
        const ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
        const ff s = ff_mul(r2, inv_r0sq);
        ff Ct = contact_ff(s);
        const float rf = sqrtf(r2.hi);
        float dCt = dcontact_ds(s.hi) * 2.0f * rf * inv_r0sq.hi;  // dC/dr
        if (r2.hi > c.cv_rs2) {
          const ff r = ff_sqrt(r2);
          const ff x = ff_mul(ff_add(r, ff{-c.cv_rs_hi, -c.cv_rs_lo}), ff{c.cv_inv_w_hi, c.cv_inv_w_lo});
          if (x.hi >= 1.0f) {
            Ct = {0.f, 0.f};
            dCt = 0.f;
          } else {
            // S = 1 - x^3 (10 - 15 x + 6 x^2)
            ff p = ff_add_f(ff_mul_f(x, 6.0f), -15.0f);
            p = ff_add_f(ff_mul(p, x), 10.0f);
            const ff x3 = ff_mul(ff_sqr(x), x);
            const ff S = ff_add_f(ff_neg(ff_mul(x3, p)), 1.0f);
            const float xf = x.hi;
            const float dS = -30.0f * xf * xf * (1.0f - xf) * (1.0f - xf) * c.cv_inv_w_hi;
            dCt = dCt * S.hi + Ct.hi * dS;
            Ct = ff_mul(Ct, S);
          }
        }
        const ff h = ff_add(Ct, ff_neg(cnat));
        // z term: C~ (C~ - 2 C~_nat) = (C~ - C~_nat)^2 - C~_nat^2
        zacc = ff_add(zacc, ff_mul(Ct, ff_add(Ct, ff_neg(ff_mul_f(cnat, 2.0f)))));
        // dz/dx_i = -w d, dz/dx_j = +w d with d = x_j - x_i, w = 2 h C~'(r)/r
        const float wgt = 2.0f * h.hi * dCt / rf;
        const long long gx = fx_from(wgt * dx.hi), gy = fx_from(wgt * dy.hi), gz = fx_from(wgt * dz.hi);
        gix -= gx; giy -= gy; giz -= gz;
        gjx += gx; gjy += gy; gjz += gz;
      }
    }
    const int src = (lane + 1) & 31;
    gjx = __shfl_sync(0xffffffffu, gjx, src);
    gjy = __shfl_sync(0xffffffffu, gjy, src);
    gjz = __shfl_sync(0xffffffffu, gjz, src);
  }
  if (i < ncv && (gix | giy | giz)) {
    red_add(d.gx + T.cv0 + i, gix); red_add(d.gy + T.cv0 + i, giy); red_add(d.gz + T.cv0 + i, giz);
  }
  if (jl < ncv && (gjx | gjy | gjz)) {
    red_add(d.gx + T.cv0 + jl, gjx); red_add(d.gy + T.cv0 + jl, gjy); red_add(d.gz + T.cv0 + jl, gjz);
  }
  double zl = ff_to_d(zacc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) zl += __shfl_xor_sync(0xffffffffu, zl, off);
  if (lane == 0) d.z_part[w] = zl;
}

// per trial: z, the ratchet amplitude a, z_m and Phi (Eqs. VR, VMDcondition)
template <int MODE>
__global__ void __launch_bounds__(256) k_cvfin(Dev d, SimConst c) {
  __shared__ double rz[256], rq[256];
  __shared__ bool last;
  const int t = blockIdx.x;
  const TrialInfo T = d.tinfo[t];
  const long long step_now = *d.step;
  double zs = 0.0, q = 0.0;
  for (int k = threadIdx.x; k < T.n_work; k += blockDim.x) zs += d.z_part[T.work0 + k];
  for (int i = threadIdx.x; i < T.n_cv; i += blockDim.x) {
    double gx = (double)d.gx[T.cv0 + i] * 2.3283064365386963e-10;
    double gy = (double)d.gy[T.cv0 + i] * 2.3283064365386963e-10;
    double gz = (double)d.gz[T.cv0 + i] * 2.3283064365386963e-10;
    q += (gx * gx + gy * gy + gz * gz) / d.gm[T.sysatom0 + i];
  }
  rz[threadIdx.x] = zs;
  rq[threadIdx.x] = q;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) { rz[threadIdx.x] += rz[threadIdx.x + off]; rq[threadIdx.x] += rq[threadIdx.x + off]; }
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
    if (c.rec_cap > 0) {
      long long n = MODE == FIN_STEP ? step_now + 1 : step_now;
      double *r = d.rec + ((size_t)t * c.rec_cap + (size_t)(n % c.rec_cap)) * 4;
      r[0] = z; r[1] = S.zm; r[2] = a; r[3] = phi;
    }
    if (MODE == FIN_STEP) {
      __threadfence();
      unsigned ticket = atomicAdd(d.done, 1u);
      last = ticket == (unsigned)(d.n_trials - 1);
    } else {
      last = false;
    }
  }
  __syncthreads();
  if (MODE == FIN_STEP && last && threadIdx.x == 0) {
    *d.step = step_now + 1;
    *d.kick = 1.0f;
    *d.done = 0u;
  }
}

void launch_cnat(const Dev &d, const SimConst &c, const double *native, const int32_t *sys_nat0, int32_t n_tiles,
                 const int32_t *tile_sys, cudaStream_t s) {
  if (n_tiles <= 0) return;
  long long threads = (long long)n_tiles * 32;
  k_cnat<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(d, c, native, sys_nat0, tile_sys, n_tiles);
}
void launch_zconst(const Dev &d, const int32_t *sys_tile0, const int32_t *sys_ntiles, cudaStream_t s) {
  k_zconst<<<d.n_trials, 256, 0, s>>>(d, sys_tile0, sys_ntiles);
}
void launch_cv(const Dev &d, const SimConst &c, cudaStream_t s) {
  if (d.total_work <= 0) return;
  long long threads = (long long)d.total_work * 32;
  k_cv<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(d, c);
}
void launch_cvfin(const Dev &d, const SimConst &c, FinMode mode, cudaStream_t s) {
  if (mode == FIN_STEP) k_cvfin<FIN_STEP><<<d.n_trials, 256, 0, s>>>(d, c);
  else if (mode == FIN_INIT) k_cvfin<FIN_INIT><<<d.n_trials, 256, 0, s>>>(d, c);
  else k_cvfin<FIN_RESTORE><<<d.n_trials, 256, 0, s>>>(d, c);
}

}  // namespace vp

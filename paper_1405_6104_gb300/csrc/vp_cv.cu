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
#include "vp_cvpair.cuh"
#include "vp_dev.cuh"

namespace vp {

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
    const float hi = (float)v;
    d.cnat_ff[(size_t)tile * CV_T * CV_T + k * CV_T + lane] = make_float2(hi, (float)(v - (double)hi));
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

__device__ __forceinline__ long long gsum(int hi, unsigned lo) { return (long long)hi * 16777216ll + (long long)lo; }

// Two phases per (trial, tile) warp: (1) a cheap FP32 distance test of the
// 1024 pairs of the tile lists the pairs closer than the contact cut-off in
// shared memory; (2) the warp evaluates only those, 32 at a time, in
// float-float, accumulating the gradient of the tile's 64 atoms with integer
// shared-memory atomics (order-independent, so deterministic) and flushing it
// once per tile.  Far pairs (C~ = 0) contribute only to the constant Z0.
template <int CV_WARPS>
__global__ void __launch_bounds__(CV_WARPS * 32) k_cv(Dev d, SimConst c) {
  __shared__ unsigned short s_near[CV_WARPS][CV_T * CV_T];
  __shared__ float s_x[CV_WARPS][2 * CV_T][3];
  // gradient of the tile's 64 atoms: each fixed-point contribution c splits
  // into c >> 24 (signed) and its low 24 bits, summed in 32-bit shared
  // atomics (native, unlike 64-bit ones); at most 32 contributions per entry
  // keep both sums far from overflow, and (hi << 24) + lo is the exact sum
  __shared__ int s_ghi[CV_WARPS][2 * CV_T][3];
  __shared__ unsigned s_glo[CV_WARPS][2 * CV_T][3];
  const int wib = threadIdx.x >> 5;
  const int wq = blockIdx.x * CV_WARPS + wib;
  const int lane = threadIdx.x & 31;
  if (wq >= d.total_work) return;
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
  s_x[wib][lane][0] = xi.x; s_x[wib][lane][1] = xi.y; s_x[wib][lane][2] = xi.z;
  s_x[wib][CV_T + lane][0] = xj.x; s_x[wib][CV_T + lane][1] = xj.y; s_x[wib][CV_T + lane][2] = xj.z;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    s_ghi[wib][lane][q] = 0; s_ghi[wib][CV_T + lane][q] = 0;
    s_glo[wib][lane][q] = 0u; s_glo[wib][CV_T + lane][q] = 0u;
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
    if (near) s_near[wib][n_near + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)(lane | (jc << 5));
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
      const unsigned e = s_near[wib][idx];
      const int il = e & 31, jc = e >> 5;
      const float3 pi = make_float3(s_x[wib][il][0], s_x[wib][il][1], s_x[wib][il][2]);
      ff dx, dy, dz;
      cv_delta(pi, s_x[wib][CV_T + jc][0], s_x[wib][CV_T + jc][1], s_x[wib][CV_T + jc][2], L, iL, dx, dy, dz);
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
          atomicAdd(&s_ghi[wib][il][q], (int)((-gv[q]) >> 24));
          atomicAdd(&s_glo[wib][il][q], (unsigned)((-gv[q]) & 0xffffff));
          atomicAdd(&s_ghi[wib][CV_T + jc][q], (int)(gv[q] >> 24));
          atomicAdd(&s_glo[wib][CV_T + jc][q], (unsigned)(gv[q] & 0xffffff));
        }
      }
    }
  }
  __syncwarp();
  if (n_near > 0) {
    if (i < ncv) {
      const long long a0 = gsum(s_ghi[wib][lane][0], s_glo[wib][lane][0]),
                      a1 = gsum(s_ghi[wib][lane][1], s_glo[wib][lane][1]),
                      a2 = gsum(s_ghi[wib][lane][2], s_glo[wib][lane][2]);
      if (a0 | a1 | a2) { red_add(d.gx + T.cv0 + i, a0); red_add(d.gy + T.cv0 + i, a1); red_add(d.gz + T.cv0 + i, a2); }
    }
    if (jl < ncv) {
      const long long a0 = gsum(s_ghi[wib][CV_T + lane][0], s_glo[wib][CV_T + lane][0]),
                      a1 = gsum(s_ghi[wib][CV_T + lane][1], s_glo[wib][CV_T + lane][1]),
                      a2 = gsum(s_ghi[wib][CV_T + lane][2], s_glo[wib][CV_T + lane][2]);
      if (a0 | a1 | a2) { red_add(d.gx + T.cv0 + jl, a0); red_add(d.gy + T.cv0 + jl, a1); red_add(d.gz + T.cv0 + jl, a2); }
    }
  }
  double zl = ff_to_d(zacc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) zl += __shfl_xor_sync(0xffffffffu, zl, off);
  if (lane == 0) d.z_part[w] = zl;
}

// per trial: z, the ratchet amplitude a, z_m and Phi (Eqs. VR, VMDcondition).
// One block per trial; the block size is fixed (not chosen by batch size), so
// the reduction order, and with it every trial's z, does not depend on the
// batch.  1024 threads keep a single trial's gather and sum short.
constexpr int CVFIN_THREADS = 1024;

template <int MODE>
__global__ void __launch_bounds__(CVFIN_THREADS) k_cvfin(Dev d, SimConst c) {
  __shared__ double rz[CVFIN_THREADS], rq[CVFIN_THREADS];
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
    q += (gx * gx + gy * gy + gz * gz) * d.inv_gm[T.sysatom0 + i];  // FP64 division is slow on this part
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
    if (c.rec_cap > 0 && MODE != FIN_KEEP) {
      long long n = MODE == FIN_STEP ? step_now + 1 : step_now;
      double *r = d.rec + ((size_t)t * c.rec_cap + (size_t)(n % c.rec_cap)) * 5;
      r[0] = z; r[1] = S.zm; r[2] = a; r[3] = phi; r[4] = Q;
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

// CV-atom positions of one trial after every force evaluation (the step
// counter has already advanced for a step; frame index = step % capacity)
// frame of step n: one trial ([cap][n_cv][3]) or, with trial < 0, every
// trial ([n_trials][cap][stride][3], stride = the largest n_cv; blockIdx.y
// is the trial)
__global__ void k_rec_frames(Dev d, int trial, int cap, int stride, float *frames) {
  const int t = trial >= 0 ? trial : (int)blockIdx.y;
  const TrialInfo &T = d.tinfo[t];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T.n_cv) return;
  const long long n = *d.step;
  const float4 p = d.pos[d.slot_of[T.atom0 + i]];
  const size_t base = trial >= 0 ? 0 : (size_t)t * (size_t)cap * (size_t)stride;
  float *f = frames + (base + (size_t)(n % cap) * stride + i) * 3;
  f[0] = p.x; f[1] = p.y; f[2] = p.z;
}

void launch_rec_frames(const Dev &d, int trial, int n_cv, int cap, float *frames, cudaStream_t s) {
  if (n_cv <= 0 || cap <= 0) return;
  dim3 grid((unsigned)((n_cv + 127) / 128), trial >= 0 ? 1u : (unsigned)d.n_trials);
  k_rec_frames<<<grid, 128, 0, s>>>(d, trial, cap, n_cv, frames);
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
// variants: 0: 4 warps per block, 1: 2 warps, 2: 8 warps
void launch_cv(const Dev &d, const SimConst &c, cudaStream_t s, int variant) {
  if (d.total_work <= 0) return;
  if (variant == 1) k_cv<2><<<(unsigned)((d.total_work + 1) / 2), 64, 0, s>>>(d, c);
  else if (variant == 2) k_cv<8><<<(unsigned)((d.total_work + 7) / 8), 256, 0, s>>>(d, c);
  else k_cv<4><<<(unsigned)((d.total_work + 3) / 4), 128, 0, s>>>(d, c);
}
void launch_cvfin(const Dev &d, const SimConst &c, FinMode mode, cudaStream_t s) {
  if (mode == FIN_STEP) k_cvfin<FIN_STEP><<<d.n_trials, CVFIN_THREADS, 0, s>>>(d, c);
  else if (mode == FIN_INIT) k_cvfin<FIN_INIT><<<d.n_trials, CVFIN_THREADS, 0, s>>>(d, c);
  else if (mode == FIN_RESTORE) k_cvfin<FIN_RESTORE><<<d.n_trials, CVFIN_THREADS, 0, s>>>(d, c);
  else k_cvfin<FIN_KEEP><<<d.n_trials, CVFIN_THREADS, 0, s>>>(d, c);
}

}  // namespace vp

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
#include "vp_cv_dev.cuh"

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


// Two phases per (trial, tile) warp: (1) a cheap FP32 distance test of the
// 1024 pairs of the tile lists the pairs closer than the contact cut-off in
// shared memory; (2) the warp evaluates only those, 32 at a time, in
// float-float, accumulating the gradient of the tile's 64 atoms with integer
// shared-memory atomics (order-independent, so deterministic) and flushing it
// once per tile.  Far pairs (C~ = 0) contribute only to the constant Z0.

template <int CV_WARPS>
__global__ void __launch_bounds__(CV_WARPS * 32) k_cv(Dev d, SimConst c) {
  __shared__ CvWarpShared sh[CV_WARPS];
  PDL_WAIT();
  const int wib = threadIdx.x >> 5;
  const int wq = blockIdx.x * CV_WARPS + wib;
  if (wq >= d.total_work) return;
  cv_tile(d, c, sh[wib], wq);
}

// per trial: z, the ratchet amplitude a, z_m and Phi (Eqs. VR, VMDcondition).
// One block per trial; the reduction order (over CVFIN_THREADS virtual
// threads) is fixed, so every trial's z does not depend on the batch or on
// the block that finishes it.  1024 threads keep a single trial's gather and
// sum short.


template <int MODE>
__global__ void __launch_bounds__(CVFIN_THREADS) k_cvfin(Dev d, SimConst c) {
  __shared__ CvfinShared sh;
  PDL_WAIT();
  cvfin_trial<MODE>(d, c, sh, blockIdx.x);
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
void launch_cv(const Dev &d, const SimConst &c, cudaStream_t s, int variant, bool after_kernel) {
  if (d.total_work <= 0) return;
  const int w = variant == 1 ? 2 : variant == 2 ? 8 : 4;
  const dim3 g((unsigned)((d.total_work + w - 1) / w)), b((unsigned)(32 * w));
  if (!after_kernel) {  // first on its stream: an ordinary launch
    if (w == 2) k_cv<2><<<g, b, 0, s>>>(d, c);
    else if (w == 8) k_cv<8><<<g, b, 0, s>>>(d, c);
    else k_cv<4><<<g, b, 0, s>>>(d, c);
  } else if (w == 2) {
    launch_pdl(k_cv<2>, g, b, s, d, c);
  } else if (w == 8) {
    launch_pdl(k_cv<8>, g, b, s, d, c);
  } else {
    launch_pdl(k_cv<4>, g, b, s, d, c);
  }
}
void launch_cvfin(const Dev &d, const SimConst &c, FinMode mode, cudaStream_t s) {
  const dim3 g((unsigned)d.n_trials), b(CVFIN_THREADS);
  if (mode == FIN_STEP) launch_pdl(k_cvfin<FIN_STEP>, g, b, s, d, c);
  else if (mode == FIN_INIT) launch_pdl(k_cvfin<FIN_INIT>, g, b, s, d, c);
  else if (mode == FIN_RESTORE) launch_pdl(k_cvfin<FIN_RESTORE>, g, b, s, d, c);
  else launch_pdl(k_cvfin<FIN_KEEP>, g, b, s, d, c);
}

}  // namespace vp

// vp_adjoint.cu -- gradient of the bias functional with respect to the frames
// of a trial path (the variational condition of Eq. VMDcondition is stated as
// a functional derivative with respect to the path X(tau)).
//
// Along frames X_0 .. X_N (dt apart), with z_n = z(X_n), g_n = grad z(X_n),
// Q_n = sum_i |g_n,i|^2/(gamma_i m_i), m_n = min_{k<=n} z_k (first minimiser)
// and a_n = (z_n - m_{n-1})_+ (Eq. VR):
//   Phi = sum_{n>=1} dt (k_R/2)^2 a_n^2 Q_n
//   dPhi/dX_n = A_n g_n + B_n H_z(X_n) w_n,   w_i = g_i/(gamma_i m_i),
//   A_n = dt (k_R/2)^2 (2 a_n Q_n [n>=1] - R_n),  B_n = 2 dt (k_R/2)^2 a_n^2,
//   R_n = sum over later l whose running minimum sits at frame n of 2 a_l Q_l.
// Kernels: per (frame, 32x32 tile) warp for z and g (float-float pair math as
// in the batched kernel), per frame block for z_n, Q_n and w, one scan for the
// coefficients, per (frame, tile) warp for H_z w (FP32 pair math, int64
// fixed-point accumulation), and a per-atom combination.
#include <cstring>
#include <string>
#include <vector>

#include "vp_adjoint.cuh"
#include "vp_cvpair.cuh"

namespace vp {

struct AdjDev {
  const float *frames;  // [nf][3 n_cv]
  int nf, n_cv, min_sep, n_tiles;
  const int2 *tiles;    // the system's tiles
  const double *cnat;   // the system's C~_nat in tile-skew order
  const double *gm;     // gamma_i m_i of the system's atoms
  float L, iL;
  double zconst;
  long long *gx, *gy, *gz;  // [nf][n_cv]
  long long *hx, *hy, *hz;  // [nf][n_cv]
  float *w;                 // [nf][3 n_cv]
  double *zpart;            // [nf][n_tiles]
  double *z, *Q;            // [nf]
  double *coef;             // [2 nf]: A_n, B_n
};

__global__ void __launch_bounds__(128) k_adj_cv(AdjDev a, CvConst k) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= a.nf * a.n_tiles) return;
  const int f = w / a.n_tiles, t = w - f * a.n_tiles;
  const int2 bij = a.tiles[t];
  const float *X = a.frames + (size_t)f * 3 * a.n_cv;
  const int i = bij.x * CV_T + lane, jl = bij.y * CV_T + lane;
  float3 xi = make_float3(0.f, 0.f, 0.f), xj = make_float3(0.f, 0.f, 0.f);
  if (i < a.n_cv) xi = make_float3(X[3 * i], X[3 * i + 1], X[3 * i + 2]);
  if (jl < a.n_cv) xj = make_float3(X[3 * jl], X[3 * jl + 1], X[3 * jl + 2]);
  const double *cn = a.cnat + (size_t)t * CV_T * CV_T;
  long long gix = 0, giy = 0, giz = 0, gjx = 0, gjy = 0, gjz = 0;
  ff zacc = {0.f, 0.f};
  for (int s = 0; s < CV_T; ++s) {
    const int jc = (lane + s) & (CV_T - 1);
    const int j = bij.y * CV_T + jc;
    const float xjx = __shfl_sync(0xffffffffu, xj.x, jc);
    const float xjy = __shfl_sync(0xffffffffu, xj.y, jc);
    const float xjz = __shfl_sync(0xffffffffu, xj.z, jc);
    if (i < a.n_cv && j < a.n_cv && j - i > a.min_sep) {
      ff dx, dy, dz;
      cv_delta(xi, xjx, xjy, xjz, a.L, a.iL, dx, dy, dz);
      const float r2f = dx.hi * dx.hi + dy.hi * dy.hi + dz.hi * dz.hi;
      if (r2f < k.rc2_far) {
        const ff cnat = ff_from_d(cn[s * CV_T + lane]);
        const ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
        const CvPair cp = cv_contact<false>(r2, k);
        const ff h = ff_add(cp.Ct, ff_neg(cnat));
        zacc = ff_add(zacc, ff_mul(cp.Ct, ff_add(cp.Ct, ff_neg(ff_mul_f(cnat, 2.0f)))));
        const float wgt = 2.0f * h.hi * cp.dCt / cp.r;
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
  const size_t base = (size_t)f * a.n_cv;
  if (i < a.n_cv && (gix | giy | giz)) { red_add(a.gx + base + i, gix); red_add(a.gy + base + i, giy); red_add(a.gz + base + i, giz); }
  if (jl < a.n_cv && (gjx | gjy | gjz)) { red_add(a.gx + base + jl, gjx); red_add(a.gy + base + jl, gjy); red_add(a.gz + base + jl, gjz); }
  double zl = ff_to_d(zacc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) zl += __shfl_xor_sync(0xffffffffu, zl, off);
  if (lane == 0) a.zpart[(size_t)f * a.n_tiles + t] = zl;
}

// per frame: z, Q and w = g/(gamma m)
__global__ void __launch_bounds__(256) k_adj_fin(AdjDev a) {
  __shared__ double rz[256], rq[256];
  const int f = blockIdx.x;
  double zs = 0.0, q = 0.0;
  for (int t = threadIdx.x; t < a.n_tiles; t += blockDim.x) zs += a.zpart[(size_t)f * a.n_tiles + t];
  const double sc = 2.3283064365386963e-10;
  for (int i = threadIdx.x; i < a.n_cv; i += blockDim.x) {
    const size_t k = (size_t)f * a.n_cv + i;
    const double gx = (double)a.gx[k] * sc, gy = (double)a.gy[k] * sc, gz = (double)a.gz[k] * sc;
    const double gm = a.gm[i];
    q += (gx * gx + gy * gy + gz * gz) / gm;
    a.w[3 * k] = (float)(gx / gm);
    a.w[3 * k + 1] = (float)(gy / gm);
    a.w[3 * k + 2] = (float)(gz / gm);
  }
  rz[threadIdx.x] = zs;
  rq[threadIdx.x] = q;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) { rz[threadIdx.x] += rz[threadIdx.x + off]; rq[threadIdx.x] += rq[threadIdx.x + off]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.z[f] = a.zconst + rz[0];
    a.Q[f] = rq[0];
  }
}

// coefficients A_n, B_n and Phi from z and Q along the path (z_m starts at z_0)
__global__ void k_adj_scan(const double *z, const double *Q, int nf, double c, double *coef, double *route,
                           double *phi_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int f = 0; f < nf; ++f) route[f] = 0.0;
  double m = z[0], Phi = 0.0;
  int arg = 0;
  for (int f = 1; f < nf; ++f) {
    const double a = z[f] > m ? z[f] - m : 0.0;
    Phi += c * a * a * Q[f];
    if (a > 0.0) route[arg] += 2.0 * a * Q[f];
    coef[2 * f + 1] = 2.0 * c * a * a;
    coef[2 * f] = 2.0 * c * a * Q[f];
    if (z[f] < m) { m = z[f]; arg = f; }
  }
  coef[0] = 0.0;
  coef[1] = 0.0;
  for (int f = 0; f < nf; ++f) coef[2 * f] -= c * route[f];
  if (phi_out) *phi_out = Phi;
}

// H_z w per frame: a pair adds K (w_j - w_i) to atom j and subtracts it from
// atom i, K v = f'' u (u.v) + (f'/r)(v - u (u.v)), f = (C~ - C~_nat)^2
__global__ void __launch_bounds__(128) k_adj_hw(AdjDev a, CvConst k) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= a.nf * a.n_tiles) return;
  const int f = w / a.n_tiles, t = w - f * a.n_tiles;
  if (a.coef[2 * f + 1] == 0.0) return;  // no bias at this frame: no Hessian term
  const int2 bij = a.tiles[t];
  const float *X = a.frames + (size_t)f * 3 * a.n_cv;
  const float *W = a.w + (size_t)f * 3 * a.n_cv;
  const int i = bij.x * CV_T + lane, jl = bij.y * CV_T + lane;
  float3 xi = make_float3(0.f, 0.f, 0.f), xj = make_float3(0.f, 0.f, 0.f);
  float3 wi = make_float3(0.f, 0.f, 0.f), wj = make_float3(0.f, 0.f, 0.f);
  if (i < a.n_cv) {
    xi = make_float3(X[3 * i], X[3 * i + 1], X[3 * i + 2]);
    wi = make_float3(W[3 * i], W[3 * i + 1], W[3 * i + 2]);
  }
  if (jl < a.n_cv) {
    xj = make_float3(X[3 * jl], X[3 * jl + 1], X[3 * jl + 2]);
    wj = make_float3(W[3 * jl], W[3 * jl + 1], W[3 * jl + 2]);
  }
  const double *cn = a.cnat + (size_t)t * CV_T * CV_T;
  long long hix = 0, hiy = 0, hiz = 0, hjx = 0, hjy = 0, hjz = 0;
  for (int s = 0; s < CV_T; ++s) {
    const int jc = (lane + s) & (CV_T - 1);
    const int j = bij.y * CV_T + jc;
    const float xjx = __shfl_sync(0xffffffffu, xj.x, jc);
    const float xjy = __shfl_sync(0xffffffffu, xj.y, jc);
    const float xjz = __shfl_sync(0xffffffffu, xj.z, jc);
    const float wjx = __shfl_sync(0xffffffffu, wj.x, jc);
    const float wjy = __shfl_sync(0xffffffffu, wj.y, jc);
    const float wjz = __shfl_sync(0xffffffffu, wj.z, jc);
    if (i < a.n_cv && j < a.n_cv && j - i > a.min_sep) {
      ff dx, dy, dz;
      cv_delta(xi, xjx, xjy, xjz, a.L, a.iL, dx, dy, dz);
      const float r2f = dx.hi * dx.hi + dy.hi * dy.hi + dz.hi * dz.hi;
      if (r2f < k.rc2_far) {
        const ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
        const CvPair cp = cv_contact<true>(r2, k);
        const float h = ff_add(cp.Ct, ff_neg(ff_from_d(cn[s * CV_T + lane]))).hi;
        const float f1 = 2.0f * h * cp.dCt;
        const float f2 = 2.0f * (cp.dCt * cp.dCt + h * cp.d2Ct);
        const float ir = 1.0f / cp.r;
        const float ux = dx.hi * ir, uy = dy.hi * ir, uz = dz.hi * ir;
        const float vx = wjx - wi.x, vy = wjy - wi.y, vz = wjz - wi.z;
        const float uv = ux * vx + uy * vy + uz * vz;
        const float q = f1 * ir;
        const float kx = f2 * ux * uv + q * (vx - ux * uv);
        const float ky = f2 * uy * uv + q * (vy - uy * uv);
        const float kz = f2 * uz * uv + q * (vz - uz * uv);
        const long long ex = fx_from(kx), ey = fx_from(ky), ez = fx_from(kz);
        hix -= ex; hiy -= ey; hiz -= ez;
        hjx += ex; hjy += ey; hjz += ez;
      }
    }
    const int src = (lane + 1) & 31;
    hjx = __shfl_sync(0xffffffffu, hjx, src);
    hjy = __shfl_sync(0xffffffffu, hjy, src);
    hjz = __shfl_sync(0xffffffffu, hjz, src);
  }
  const size_t base = (size_t)f * a.n_cv;
  if (i < a.n_cv && (hix | hiy | hiz)) { red_add(a.hx + base + i, hix); red_add(a.hy + base + i, hiy); red_add(a.hz + base + i, hiz); }
  if (jl < a.n_cv && (hjx | hjy | hjz)) { red_add(a.hx + base + jl, hjx); red_add(a.hy + base + jl, hjy); red_add(a.hz + base + jl, hjz); }
}

__global__ void k_adj_out(AdjDev a, double *grad) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)a.nf * a.n_cv) return;
  const int f = (int)(k / a.n_cv);
  const double A = a.coef[2 * f], B = a.coef[2 * f + 1], sc = 2.3283064365386963e-10;
  grad[3 * k] = A * (double)a.gx[k] * sc + B * (double)a.hx[k] * sc;
  grad[3 * k + 1] = A * (double)a.gy[k] * sc + B * (double)a.hy[k] * sc;
  grad[3 * k + 2] = A * (double)a.gz[k] * sc + B * (double)a.hz[k] * sc;
}

// ---------------------------------------------------------------------------

int adjoint_frames(const AdjInput &in, cudaStream_t st, std::string &err) {
  const int nf = in.n_frames, ncv = in.n_cv, nt = in.n_tiles;
  const size_t na = (size_t)nf * ncv;
  AdjDev a{};
  a.nf = nf; a.n_cv = ncv; a.min_sep = in.min_sep; a.n_tiles = nt;
  a.tiles = in.tiles; a.cnat = in.cnat; a.gm = in.gm; a.L = in.L; a.iL = in.iL; a.zconst = in.zconst;
  std::vector<void *> bufs;
  auto alloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 8) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  };
  auto freeall = [&]() { for (void *p : bufs) cudaFree(p); };
  float *dframes = (float *)alloc(sizeof(float) * 3 * na);
  a.gx = (long long *)alloc(sizeof(long long) * 3 * na);
  a.hx = (long long *)alloc(sizeof(long long) * 3 * na);
  a.w = (float *)alloc(sizeof(float) * 3 * na);
  a.zpart = (double *)alloc(sizeof(double) * (size_t)nf * (nt > 0 ? nt : 1));
  a.z = (double *)alloc(sizeof(double) * nf);
  a.Q = (double *)alloc(sizeof(double) * nf);
  a.coef = (double *)alloc(sizeof(double) * 2 * nf);
  double *route = (double *)alloc(sizeof(double) * nf);
  double *dphi = (double *)alloc(sizeof(double));
  double *dgrad = (double *)alloc(sizeof(double) * 3 * na);
  for (void *p : bufs)
    if (!p) { freeall(); err = "cudaMalloc failed"; return SIM_ECUDA; }
  a.frames = dframes;
  a.gy = a.gx + na; a.gz = a.gy + na;
  a.hy = a.hx + na; a.hz = a.hy + na;
  std::vector<float> hf(3 * na);
  for (size_t k = 0; k < 3 * na; ++k) hf[k] = (float)in.frames[k];
  cudaMemcpyAsync(dframes, hf.data(), sizeof(float) * 3 * na, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(a.gx, 0, sizeof(long long) * 3 * na, st);
  cudaMemsetAsync(a.hx, 0, sizeof(long long) * 3 * na, st);
  const long long warps = (long long)nf * nt;
  if (warps > 0) k_adj_cv<<<(unsigned)((warps * 32 + 127) / 128), 128, 0, st>>>(a, in.k);
  k_adj_fin<<<nf, 256, 0, st>>>(a);
  if (in.coef) {
    cudaMemcpyAsync(a.coef, in.coef, sizeof(double) * 2 * nf, cudaMemcpyHostToDevice, st);
  } else {
    k_adj_scan<<<1, 32, 0, st>>>(a.z, a.Q, nf, in.c, a.coef, route, dphi);
  }
  if (warps > 0) k_adj_hw<<<(unsigned)((warps * 32 + 127) / 128), 128, 0, st>>>(a, in.k);
  if (na > 0) k_adj_out<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(a, dgrad);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && in.grad) e = cudaMemcpyAsync(in.grad, dgrad, sizeof(double) * 3 * na, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && in.z_out) e = cudaMemcpyAsync(in.z_out, a.z, sizeof(double) * nf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && in.Q_out) e = cudaMemcpyAsync(in.Q_out, a.Q, sizeof(double) * nf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && in.phi && !in.coef) e = cudaMemcpyAsync(in.phi, dphi, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  freeall();
  if (e != cudaSuccess) { err = cudaGetErrorString(e); return SIM_ECUDA; }
  return SIM_OK;
}

// ---------------------------------------------------------------------------
// refinement of a path by descent on the functional (frames as variables)
// ---------------------------------------------------------------------------
__global__ void k_to_f32(const double *x, float *y, size_t n) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = (float)x[k];
}

// y = x - eta g on frames 1 .. nf-2, rounded to FP32 (the precision the
// functional is evaluated at, so that the returned path is exactly the one
// scored); y = x on the end frames, which stay put
__global__ void k_descend(const double *x, const double *g, double eta, double *y, size_t per_frame, int nf) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= per_frame * (size_t)nf) return;
  const int f = (int)(k / per_frame);
  y[k] = (f == 0 || f == nf - 1) ? x[k] : (double)(float)(x[k] - eta * g[k]);
}

// |g|^2 over frames 1 .. nf-2: fixed-order block sums, then one block
__global__ void k_sq_interior(const double *g, size_t per_frame, int nf, double *part) {
  __shared__ double red[256];
  double acc = 0.0;
  const size_t lo = per_frame, hi = per_frame * (size_t)(nf > 1 ? nf - 1 : 0);
  for (size_t k = lo + (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < hi; k += (size_t)gridDim.x * blockDim.x)
    acc += g[k] * g[k];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

int refine_frames(const AdjInput &in, double *frames, int n_iter, double step, double *phi_hist, int *n_accepted,
                  cudaStream_t st, std::string &err) {
  const int nf = in.n_frames, ncv = in.n_cv, nt = in.n_tiles;
  const size_t na = (size_t)nf * ncv, nx = 3 * na;
  AdjDev a{};
  a.nf = nf; a.n_cv = ncv; a.min_sep = in.min_sep; a.n_tiles = nt;
  a.tiles = in.tiles; a.cnat = in.cnat; a.gm = in.gm; a.L = in.L; a.iL = in.iL; a.zconst = in.zconst;
  std::vector<void *> bufs;
  auto alloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 8) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  };
  auto freeall = [&]() { for (void *p : bufs) cudaFree(p); };
  constexpr int SQ_BLOCKS = 64;
  float *f32 = (float *)alloc(sizeof(float) * nx);
  double *X = (double *)alloc(sizeof(double) * nx), *Y = (double *)alloc(sizeof(double) * nx);
  double *G = (double *)alloc(sizeof(double) * nx);
  a.gx = (long long *)alloc(sizeof(long long) * 3 * na);
  a.hx = (long long *)alloc(sizeof(long long) * 3 * na);
  a.w = (float *)alloc(sizeof(float) * nx);
  a.zpart = (double *)alloc(sizeof(double) * (size_t)nf * (nt > 0 ? nt : 1));
  a.z = (double *)alloc(sizeof(double) * nf);
  a.Q = (double *)alloc(sizeof(double) * nf);
  a.coef = (double *)alloc(sizeof(double) * 2 * nf);
  double *route = (double *)alloc(sizeof(double) * nf);
  double *dphi = (double *)alloc(sizeof(double));
  double *part = (double *)alloc(sizeof(double) * SQ_BLOCKS);
  for (void *p : bufs)
    if (!p) { freeall(); err = "cudaMalloc failed"; return SIM_ECUDA; }
  a.frames = f32;
  a.gy = a.gx + na; a.gz = a.gy + na;
  a.hy = a.hx + na; a.hz = a.hy + na;
  const long long warps = (long long)nf * nt;
  const unsigned gx_blocks = (unsigned)((nx + 255) / 256);
  // Phi (and, when want_grad, dPhi/dX into G) at the frames in src
  auto eval = [&](const double *src, bool want_grad, double &phi) -> cudaError_t {
    k_to_f32<<<gx_blocks, 256, 0, st>>>(src, f32, nx);
    cudaMemsetAsync(a.gx, 0, sizeof(long long) * 3 * na, st);
    cudaMemsetAsync(a.hx, 0, sizeof(long long) * 3 * na, st);
    if (warps > 0) k_adj_cv<<<(unsigned)((warps * 32 + 127) / 128), 128, 0, st>>>(a, in.k);
    k_adj_fin<<<nf, 256, 0, st>>>(a);
    k_adj_scan<<<1, 32, 0, st>>>(a.z, a.Q, nf, in.c, a.coef, route, dphi);
    if (want_grad) {
      if (warps > 0) k_adj_hw<<<(unsigned)((warps * 32 + 127) / 128), 128, 0, st>>>(a, in.k);
      if (na > 0) k_adj_out<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(a, G);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&phi, dphi, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  };
  auto sq = [&](double &v) -> cudaError_t {
    k_sq_interior<<<SQ_BLOCKS, 256, 0, st>>>(G, 3 * (size_t)ncv, nf, part);
    double h[SQ_BLOCKS];
    cudaError_t e = cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    v = 0.0;
    for (int b = 0; b < SQ_BLOCKS; ++b) v += h[b];
    return e;
  };
  cudaError_t e = cudaMemcpyAsync(X, frames, sizeof(double) * nx, cudaMemcpyHostToDevice, st);
  double phi = 0.0, gg = 0.0;
  if (e == cudaSuccess) e = eval(X, true, phi);
  if (e == cudaSuccess) e = sq(gg);
  if (phi_hist) phi_hist[0] = phi;
  int accepted = 0;
  double eta = step;
  for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
    bool ok = false;
    // backtracking (Armijo): accept the first step that lowers Phi by at least 1e-4 eta |g|^2
    for (int bt = 0; bt < 40 && e == cudaSuccess && gg > 0.0; ++bt) {
      k_descend<<<gx_blocks, 256, 0, st>>>(X, G, eta, Y, 3 * (size_t)ncv, nf);
      double phi_y = 0.0;
      e = eval(Y, false, phi_y);
      if (e != cudaSuccess) break;
      if (phi_y <= phi - 1e-4 * eta * gg) {
        std::swap(X, Y);
        phi = phi_y;
        ok = true;
        break;
      }
      eta *= 0.5;
    }
    if (e == cudaSuccess && ok) {
      e = eval(X, true, phi);
      if (e == cudaSuccess) e = sq(gg);
      ++accepted;
      eta *= 2.0;
    }
    if (phi_hist) phi_hist[it + 1] = phi;
    if (!ok) {  // no step lowers Phi any more: keep the value for the remaining entries
      for (int k = it + 2; phi_hist && k <= n_iter; ++k) phi_hist[k] = phi;
      break;
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(frames, X, sizeof(double) * nx, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  freeall();
  if (n_accepted) *n_accepted = accepted;
  if (e != cudaSuccess) { err = cudaGetErrorString(e); return SIM_ECUDA; }
  return SIM_OK;
}

int adjoint_coefficients(const double *z, const double *Q, int n, double c, double *coef, double *phi,
                         cudaStream_t st, std::string &err) {
  double *dz = nullptr, *dq = nullptr, *dc = nullptr, *dr = nullptr, *dp = nullptr;
  size_t nb = sizeof(double) * (n > 0 ? n : 1);
  if (cudaMalloc(&dz, nb) != cudaSuccess || cudaMalloc(&dq, nb) != cudaSuccess || cudaMalloc(&dc, 2 * nb) != cudaSuccess ||
      cudaMalloc(&dr, nb) != cudaSuccess || cudaMalloc(&dp, sizeof(double)) != cudaSuccess) {
    cudaFree(dz); cudaFree(dq); cudaFree(dc); cudaFree(dr); cudaFree(dp);
    err = "cudaMalloc failed";
    return SIM_ECUDA;
  }
  cudaMemcpyAsync(dz, z, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dq, Q, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  k_adj_scan<<<1, 32, 0, st>>>(dz, dq, n, c, dc, dr, dp);
  cudaError_t e = cudaMemcpyAsync(coef, dc, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && phi) e = cudaMemcpyAsync(phi, dp, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dz); cudaFree(dq); cudaFree(dc); cudaFree(dr); cudaFree(dp);
  if (e != cudaSuccess) { err = cudaGetErrorString(e); return SIM_ECUDA; }
  return SIM_OK;
}

}  // namespace vp

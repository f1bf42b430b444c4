// vp_toy2d.cu -- batched trials of the two-dimensional toy model of the
// variational pathway scheme (SM, "Illustrative Application in a Toy Model"):
// one particle on U(x, y) under underdamped Langevin dynamics (Eq. Lang,
// BAOAB), with the ratchet-and-pawl bias of Eq. VR, a steered harmonic pull,
// or no bias on z = sqrt(x^2 + y^2), and the functional of Eq. VMDcondition
// accumulated up to the first passage into the product (z <= z_product).
//
// One thread owns one trial for its whole run and keeps the state in
// registers; the only memory traffic is the trial's inputs, its outputs and
// (optionally) its recorded path.  Arithmetic is FP64 without contraction
// (this file is compiled with -fmad=false), in the operation order of the
// equations, so that a trial follows its FP64 definition step for step; the
// white noise is Philox4x32-10 (counter = (0, step, 0 | stream)) turned into
// normals by Box-Muller in FP64.
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/vpath.h"
#include "vp_internal.cuh"

namespace vp {
namespace {

struct ToyConst {
  double A1, A2, A3, s1, s2, s3, w, xm, ym;
  double n1, n2, n3;   // s^p of the three terms
  double gm, im, h, dt; // gamma m, 1/m, dt/2, dt
  double c1, c2sd;     // exp(-gamma dt), sqrt(1 - c1^2) sqrt(kT/m)
  double sd;           // sqrt(kT/m)
  double zp;           // product threshold
  int bias;
};

// two standard normals from Philox (key = seed) at (atom 0, step, stream)
__device__ __forceinline__ double2 normal2_d(uint32_t k0, uint32_t k1, unsigned long long step, uint32_t stream) {
  const uint4 x = philox4x32_10(make_uint4(0u, (uint32_t)step, (uint32_t)(step >> 32), stream), k0, k1);
  const double s23 = 1.0 / 8388608.0;
  const double u0 = ((double)(x.x >> 9) + 0.5) * s23, u1 = ((double)(x.y >> 9) + 0.5) * s23;
  const double two_pi = 6.283185307179586476925286766559;
  const double r = sqrt(-2.0 * log(u0));
  double sn, cs;
  sincos(two_pi * u1, &sn, &cs);
  return make_double2(r * cs, r * sn);
}

// -grad U (the force of the potential; U itself is not needed on the path)
__device__ __forceinline__ void toy_force(const ToyConst &c, double x, double y, double &fx, double &fy) {
  const double r2 = x * x + y * y;
  double gx = 4.0 * c.w * c.w * r2 * x;
  double gy = 4.0 * c.w * c.w * r2 * y;
  const double D1 = r2 + c.s1 * c.s1;
  const double q1 = 4.0 * c.A1 * c.n1 / (D1 * D1 * D1);
  gx += q1 * x;
  gy += q1 * y;
  const double D2 = r2 + c.s2 * c.s2;
  const double q2 = 4.0 * c.A2 * c.n2 / (D2 * D2 * D2);
  gx -= q2 * x;
  gy -= q2 * y;
  const double dx = x - c.xm, dy = y - c.ym;
  const double D3 = dx * dx + dy * dy + c.s3 * c.s3;
  const double q3 = 4.0 * c.A3 * c.n3 / (D3 * D3 * D3);
  gx += q3 * dx;
  gy += q3 * dy;
  fx = -gx;
  fy = -gy;
}

// bias force at (x, y): ratchet (Eq. VR) against the running minimum zm, or
// the steered pull -k z grad z; grad z = (x, y)/z (zero at z = 0)
__device__ __forceinline__ void toy_bias(const ToyConst &c, double k, double x, double y, double z, double zm,
                                         double &bx, double &by) {
  bx = 0.0;
  by = 0.0;
  if (z == 0.0) return;
  const double ux = x / z, uy = y / z;
  if (c.bias == TOY2D_RATCHET) {
    const double a = z > zm ? z - zm : 0.0;
    bx = -0.5 * k * a * ux;
    by = -0.5 * k * a * uy;
  } else if (c.bias == TOY2D_STEERED) {
    bx = -k * z * ux;
    by = -k * z * uy;
  }
}

__global__ void __launch_bounds__(128) k_toy2d(ToyConst c, int n, const double *__restrict__ kk,
                                               const unsigned long long *__restrict__ seeds, long long n_steps,
                                               double x0, double y0, double *state, double *phi_out,
                                               long long *passage_out, double *path, int every, long long n_rec) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double k = kk[t];
  const unsigned long long seed = seeds[t];
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  double x = x0, y = y0;
  const double2 g0 = normal2_d(k0, k1, 0ull, 1u);  // Maxwell-Boltzmann start: stream 1, step 0
  double vx = c.sd * g0.x, vy = c.sd * g0.y;
  double zm = sqrt(x * x + y * y);
  double fx, fy, bx, by;
  toy_force(c, x, y, fx, fy);
  toy_bias(c, k, x, y, zm, zm, bx, by);
  fx += bx;
  fy += by;
  double Phi = 0.0;
  long long passage = -1;
  double *rec = path ? path + (size_t)t * (size_t)n_rec * 2 : nullptr;
  long long r = 0;
  if (rec) { rec[0] = x; rec[1] = y; r = 1; }
  for (long long s = 1; s <= n_steps; ++s) {
    const double2 g = normal2_d(k0, k1, (unsigned long long)s, 0u);
    vx += c.h * fx * c.im;
    vy += c.h * fy * c.im;
    x += c.h * vx;
    y += c.h * vy;
    vx = c.c1 * vx + c.c2sd * g.x;
    vy = c.c1 * vy + c.c2sd * g.y;
    x += c.h * vx;
    y += c.h * vy;
    toy_force(c, x, y, fx, fy);
    const double z = sqrt(x * x + y * y);
    toy_bias(c, k, x, y, z, zm, bx, by);
    Phi += c.dt * (bx * bx + by * by) / c.gm;
    fx += bx;
    fy += by;
    if (z < zm) zm = z;
    vx += c.h * fx * c.im;
    vy += c.h * fy * c.im;
    if (rec && s % every == 0 && r < n_rec) { rec[2 * r] = x; rec[2 * r + 1] = y; ++r; }
    if (z <= c.zp) { passage = s; break; }
  }
  if (rec)
    for (; r < n_rec; ++r) { rec[2 * r] = nan(""); rec[2 * r + 1] = nan(""); }
  if (state) {
    state[4 * t] = x; state[4 * t + 1] = y; state[4 * t + 2] = vx; state[4 * t + 3] = vy;
  }
  phi_out[t] = Phi;
  passage_out[t] = passage;
}

int set_err(char *errbuf, int32_t errlen, int code, const std::string &msg) {
  if (errbuf && errlen > 0) {
    std::strncpy(errbuf, msg.c_str(), (size_t)errlen - 1);
    errbuf[errlen - 1] = '\0';
  }
  return code;
}

}  // namespace
}  // namespace vp

using namespace vp;

extern "C" __attribute__((visibility("default"))) int toy2d_run(const toy2d_params *p, int32_t n_trials,
                                                                const double *k, const uint64_t *seeds,
                                                                int64_t n_steps, double *state, double *phi,
                                                                int64_t *passage, double *path, int32_t path_every,
                                                                void *cuda_stream, char *errbuf, int32_t errlen) {
  if (!p || n_trials < 0 || n_steps < 0 || (n_trials > 0 && (!k || !seeds || !phi || !passage)))
    return set_err(errbuf, errlen, SIM_EINVAL, "toy2d_run: null argument or negative size");
  if (path && path_every < 1) return set_err(errbuf, errlen, SIM_EINVAL, "toy2d_run: path_every must be >= 1");
  if (p->bias != TOY2D_NONE && p->bias != TOY2D_RATCHET && p->bias != TOY2D_STEERED)
    return set_err(errbuf, errlen, SIM_EINVAL, "toy2d_run: unknown bias");
  if (p->s_power != 2 && p->s_power != 4) return set_err(errbuf, errlen, SIM_EINVAL, "toy2d_run: s_power must be 2 or 4");
  if (!(p->mass > 0.0) || !(p->gamma >= 0.0) || !(p->kT >= 0.0) || !(p->dt > 0.0))
    return set_err(errbuf, errlen, SIM_EINVAL, "toy2d_run: mass and dt must be > 0, gamma and kT >= 0");
  if (p->bias != TOY2D_NONE && !(p->gamma > 0.0))
    return set_err(errbuf, errlen, SIM_EINVAL, "toy2d_run: the functional needs gamma > 0");
  if (n_trials == 0) return SIM_OK;
  ToyConst c{};
  c.A1 = p->A1; c.A2 = p->A2; c.A3 = p->A3; c.s1 = p->s1; c.s2 = p->s2; c.s3 = p->s3;
  c.w = p->w; c.xm = p->xm; c.ym = p->ym;
  auto spow = [&](double s) { return p->s_power == 4 ? (s * s) * (s * s) : s * s; };
  c.n1 = spow(p->s1); c.n2 = spow(p->s2); c.n3 = spow(p->s3);
  c.gm = p->gamma * p->mass;
  c.im = 1.0 / p->mass;
  c.h = 0.5 * p->dt;
  c.dt = p->dt;
  c.c1 = std::exp(-p->gamma * p->dt);
  c.sd = std::sqrt(p->kT / p->mass);
  c.c2sd = std::sqrt(1.0 - c.c1 * c.c1) * c.sd;
  c.zp = p->z_product;
  c.bias = p->bias;
  const long long n_rec = path ? n_steps / path_every + 1 : 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)n_trials;
  double *dk = nullptr, *dstate = nullptr, *dphi = nullptr, *dpath = nullptr;
  unsigned long long *dseed = nullptr;
  long long *dpass = nullptr;
  std::string err;
  auto ck = [&](cudaError_t e, const char *what) {
    if (e != cudaSuccess && err.empty()) err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  bool ok = ck(cudaMalloc(&dk, n * sizeof(double)), "cudaMalloc") &&
            ck(cudaMalloc(&dseed, n * sizeof(unsigned long long)), "cudaMalloc") &&
            ck(cudaMalloc(&dphi, n * sizeof(double)), "cudaMalloc") &&
            ck(cudaMalloc(&dpass, n * sizeof(long long)), "cudaMalloc") &&
            (!state || ck(cudaMalloc(&dstate, 4 * n * sizeof(double)), "cudaMalloc")) &&
            (!path || ck(cudaMalloc(&dpath, (size_t)n_rec * 2 * n * sizeof(double)), "cudaMalloc"));
  ok = ok && ck(cudaMemcpyAsync(dk, k, n * sizeof(double), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
       ck(cudaMemcpyAsync(dseed, seeds, n * sizeof(uint64_t), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
  if (ok) {
    // one warp per block: the trials (a few per SM at most) spread evenly over
    // the SMs, so no SM runs two blocks' worth of the FP64 pipe while others idle
    k_toy2d<<<(unsigned)((n + 31) / 32), 32, 0, st>>>(c, n_trials, dk, dseed, (long long)n_steps, p->x0, p->y0,
                                                      dstate, dphi, dpass, dpath, path_every, n_rec);
    ok = ck(cudaGetLastError(), "k_toy2d launch");
  }
  ok = ok && ck(cudaMemcpyAsync(phi, dphi, n * sizeof(double), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") &&
       ck(cudaMemcpyAsync(passage, dpass, n * sizeof(int64_t), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") &&
       (!state || ck(cudaMemcpyAsync(state, dstate, 4 * n * sizeof(double), cudaMemcpyDeviceToHost, st),
                     "cudaMemcpyAsync")) &&
       (!path || ck(cudaMemcpyAsync(path, dpath, (size_t)n_rec * 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st),
                    "cudaMemcpyAsync"));
  ck(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  cudaFree(dk); cudaFree(dseed); cudaFree(dphi); cudaFree(dpass);
  if (dstate) cudaFree(dstate);
  if (dpath) cudaFree(dpath);
  if (!err.empty()) return set_err(errbuf, errlen, SIM_ECUDA, "toy2d_run: " + err);
  return SIM_OK;
}

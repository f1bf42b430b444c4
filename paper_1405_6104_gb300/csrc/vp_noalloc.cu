// vp_noalloc.cu -- the reaction coordinate z and its gradient for one
// configuration, computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a host program whose device memory is
// owned by another allocator (a framework's caching allocator that has
// reserved the memory, or a fixed per-process budget) must not have a library
// take device memory behind its back, and a latency-critical caller cannot
// accept the implicit device-wide synchronisation that cudaMalloc/cudaFree may
// perform.  This entry point serves them: it is a variant of the batched
// reaction-coordinate kernel of vp_cv.cu in which every piece of scratch (the
// per-tile partial sums of z and the fixed-point gradient accumulators) lives
// in one file-scope device array of fixed size, and the native contact map is
// evaluated on the fly instead of from a precomputed table.
//
// The array is allocated when the library is loaded and is held by every GPU
// that loads it until the process exits.  Its device address is looked up once
// per device with cudaGetSymbolAddress, with that device current, during the
// first call on that device; that first call should therefore come before any
// stream capture on that device.  All calls share the array and it keeps the
// last call's contents, so each call clears what must start at zero, and calls
// that overlap on the GPU (on different streams) race.
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/vpath.h"
#include "vp_internal.cuh"

#define VP_API extern "C" __attribute__((visibility("default")))

namespace vp {
namespace noalloc {

constexpr int MAX_CV = 2048;                      // reaction-coordinate atoms per call
constexpr int MAX_NB = MAX_CV / CV_T;             // 64 tile rows
constexpr int MAX_TILES = MAX_NB * MAX_NB;        // tile grid (upper triangle used)
// scratch: 3 gradient components (int64) per atom + two FP64 partials per
// tile (contact sums and native-map sums): 112 KiB
constexpr size_t SCRATCH_BYTES =
    (size_t)3 * MAX_CV * sizeof(long long) + (size_t)2 * MAX_TILES * sizeof(double);

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

struct Scratch {
  long long *gx, *gy, *gz;
  double *zpart, *zcon;
};

__host__ __device__ inline Scratch carve(unsigned char *base) {
  Scratch s;
  s.gx = reinterpret_cast<long long *>(base);
  s.gy = s.gx + MAX_CV;
  s.gz = s.gy + MAX_CV;
  s.zpart = reinterpret_cast<double *>(s.gz + MAX_CV);
  s.zcon = s.zpart + MAX_TILES;
  return s;
}

struct Consts {
  float L, iL;
  float inv_r0sq_hi, inv_r0sq_lo, rs_hi, rs_lo, inv_w_hi, inv_w_lo, rs2, rc2_far;
  double r0, rs, rc;
  int n_cv, min_sep, nb;
};

// the same rational form of the contact function as the batched kernel
__device__ __forceinline__ ff contact_s(ff s) {
  ff s2 = ff_sqr(s);
  ff s3 = ff_mul(s2, s);
  ff s4 = ff_sqr(s2);
  ff N = ff_add(ff_add_f(s, 1.0f), s2);
  ff D = ff_add(ff_add(N, s3), s4);
  return ff_div(N, D);
}

__device__ __forceinline__ float dcontact(float s) {
  float N = 1.0f + s + s * s;
  float D = N + s * s * s + s * s * s * s;
  float dN = 1.0f + 2.0f * s;
  float dD = dN + 3.0f * s * s + 4.0f * s * s * s;
  return (dN * D - N * dD) / (D * D);
}

__device__ double native_contact(const double *X, int i, int j, const Consts &k) {
  double dx = X[3 * j] - X[3 * i], dy = X[3 * j + 1] - X[3 * i + 1], dz = X[3 * j + 2] - X[3 * i + 2];
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  double s = (r / k.r0) * (r / k.r0);
  double N = 1.0 + s + s * s, D = N + s * s * s + s * s * s * s;
  double C = N / D, S = 1.0;
  if (r >= k.rc) S = 0.0;
  else if (r > k.rs) {
    double x = (r - k.rs) / (k.rc - k.rs);
    S = 1.0 - x * x * x * (10.0 - 15.0 * x + 6.0 * x * x);
  }
  return C * S;
}

__global__ void k_clear(Scratch s, int n_cv, int n_tiles) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_cv) { s.gx[i] = 0; s.gy[i] = 0; s.gz[i] = 0; }
  if (i < n_tiles) s.zpart[i] = 0.0;
}

// one warp per (bi, bj) tile of the nb x nb grid; tiles below the diagonal
// or without a contact pair write a zero partial
__global__ void __launch_bounds__(128) k_cv_tile(const float *pos, const double *native, Consts k, Scratch sc,
                                                 double *zconst_part) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= k.nb * k.nb) return;
  const int bi = w / k.nb, bj = w - bi * k.nb;
  double z0 = 0.0;
  ff zacc = {0.f, 0.f};
  long long gix = 0, giy = 0, giz = 0, gjx = 0, gjy = 0, gjz = 0;
  const int i = bi * CV_T + lane, jl = bj * CV_T + lane;
  if (bj >= bi) {
    float3 xi = make_float3(0.f, 0.f, 0.f), xj = make_float3(0.f, 0.f, 0.f);
    if (i < k.n_cv) xi = make_float3(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]);
    if (jl < k.n_cv) xj = make_float3(pos[3 * jl], pos[3 * jl + 1], pos[3 * jl + 2]);
    const ff inv_r0sq = {k.inv_r0sq_hi, k.inv_r0sq_lo};
    for (int s = 0; s < CV_T; ++s) {
      const int jc = (lane + s) & (CV_T - 1);
      const int j = bj * CV_T + jc;
      const float xjx = __shfl_sync(0xffffffffu, xj.x, jc);
      const float xjy = __shfl_sync(0xffffffffu, xj.y, jc);
      const float xjz = __shfl_sync(0xffffffffu, xj.z, jc);
      if (i < k.n_cv && j < k.n_cv && j - i > k.min_sep) {
        const double cnat_d = native_contact(native, i, j, k);
        z0 += cnat_d * cnat_d;
        ff dx = ff_diff(xjx, xi.x), dy = ff_diff(xjy, xi.y), dz = ff_diff(xjz, xi.z);
        const float nx = rintf(dx.hi * k.iL), ny = rintf(dy.hi * k.iL), nz = rintf(dz.hi * k.iL);
        if (nx != 0.f) dx = ff_add_f(dx, -k.L * nx);
        if (ny != 0.f) dy = ff_add_f(dy, -k.L * ny);
        if (nz != 0.f) dz = ff_add_f(dz, -k.L * nz);
        const float r2f = dx.hi * dx.hi + dy.hi * dy.hi + dz.hi * dz.hi;
        if (r2f < k.rc2_far) {
          const ff cnat = ff_from_d(cnat_d);
          const ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
          const ff sv = ff_mul(r2, inv_r0sq);
          ff Ct = contact_s(sv);
          const float rf = sqrtf(r2.hi);
          float dCt = dcontact(sv.hi) * 2.0f * rf * inv_r0sq.hi;
          if (r2.hi > k.rs2) {
            const ff r = ff_sqrt(r2);
            const ff x = ff_mul(ff_add(r, ff{-k.rs_hi, -k.rs_lo}), ff{k.inv_w_hi, k.inv_w_lo});
            if (x.hi >= 1.0f) {
              Ct = {0.f, 0.f};
              dCt = 0.f;
            } else {
              ff p = ff_add_f(ff_mul_f(x, 6.0f), -15.0f);
              p = ff_add_f(ff_mul(p, x), 10.0f);
              const ff x3 = ff_mul(ff_sqr(x), x);
              const ff S = ff_add_f(ff_neg(ff_mul(x3, p)), 1.0f);
              const float xf = x.hi;
              const float dS = -30.0f * xf * xf * (1.0f - xf) * (1.0f - xf) * k.inv_w_hi;
              dCt = dCt * S.hi + Ct.hi * dS;
              Ct = ff_mul(Ct, S);
            }
          }
          const ff h = ff_add(Ct, ff_neg(cnat));
          zacc = ff_add(zacc, ff_mul(Ct, ff_add(Ct, ff_neg(ff_mul_f(cnat, 2.0f)))));
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
    if (i < k.n_cv && (gix | giy | giz)) { red_add(sc.gx + i, gix); red_add(sc.gy + i, giy); red_add(sc.gz + i, giz); }
    if (jl < k.n_cv && (gjx | gjy | gjz)) { red_add(sc.gx + jl, gjx); red_add(sc.gy + jl, gjy); red_add(sc.gz + jl, gjz); }
  }
  double zl = ff_to_d(zacc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    zl += __shfl_xor_sync(0xffffffffu, zl, off);
    z0 += __shfl_xor_sync(0xffffffffu, z0, off);
  }
  if (lane == 0) {
    sc.zpart[w] = zl;
    zconst_part[w] = z0;
  }
}

// fixed-order sum of the tile partials; gradient to FP64
__global__ void __launch_bounds__(256) k_finish(Scratch sc, const double *zconst_part, int n_tiles, int n_cv,
                                                double *z_out, double *grad_out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) acc += zconst_part[t] + sc.zpart[t];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *z_out = red[0];
  const double s = 2.3283064365386963e-10;
  for (int i = threadIdx.x; i < n_cv; i += blockDim.x) {
    grad_out[3 * i] = (double)sc.gx[i] * s;
    grad_out[3 * i + 1] = (double)sc.gy[i] * s;
    grad_out[3 * i + 2] = (double)sc.gz[i] * s;
  }
}

// per-device address of the static scratch
constexpr int MAX_DEVICES = 64;
static unsigned char *g_addr[MAX_DEVICES];
static std::mutex g_mutex;

}  // namespace noalloc
}  // namespace vp

using namespace vp;

static void set_msg(char *buf, int32_t len, const char *msg) {
  if (buf && len > 0) {
    std::strncpy(buf, msg, (size_t)len - 1);
    buf[len - 1] = '\0';
  }
}

VP_API int cv_eval_noalloc(const float *d_pos, const double *d_native, int32_t n_cv, double box,
                           const sim_params *params, double *d_z, double *d_grad, void *cuda_stream, char *errbuf,
                           int32_t errlen) {
  using namespace vp::noalloc;
  if (!params || !d_z || (n_cv > 0 && (!d_pos || !d_native || !d_grad))) {
    set_msg(errbuf, errlen, "cv_eval_noalloc: missing argument");
    return SIM_EINVAL;
  }
  if (n_cv < 0 || n_cv > MAX_CV) {
    set_msg(errbuf, errlen, "cv_eval_noalloc: n_cv exceeds the fixed scratch limit of 2048 atoms");
    return SIM_EINVAL;
  }
  if (!(box > 0.0) || !(params->cv_r0 > 0.0) || !(params->cv_r_cut > params->cv_r_switch) ||
      !(params->cv_r_switch > 0.0) || params->cv_min_sep < 0) {
    set_msg(errbuf, errlen, "cv_eval_noalloc: invalid box or contact parameters");
    return SIM_EINVAL;
  }
  // an error left on this thread by earlier work is reported as such, before
  // anything is launched, so that the check after the launches sees only ours
  {
    const cudaError_t pending = cudaGetLastError();
    if (pending != cudaSuccess) {
      set_msg(errbuf, errlen, (std::string("cv_eval_noalloc: an earlier CUDA error is pending: ") +
                               cudaGetErrorString(pending)).c_str());
      return SIM_ECUDA;
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    set_msg(errbuf, errlen, "cv_eval_noalloc: no usable current device");
    return SIM_ECUDA;
  }
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) {
        set_msg(errbuf, errlen, cudaGetErrorString(e));
        return SIM_ECUDA;
      }
      g_addr[dev] = static_cast<unsigned char *>(p);
    }
    base = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const Scratch sc = carve(base);
  Consts k{};
  const float Lf = (float)box;
  k.L = Lf;
  k.iL = (float)(1.0 / (double)Lf);
  auto split = [](double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  split(1.0 / (params->cv_r0 * params->cv_r0), k.inv_r0sq_hi, k.inv_r0sq_lo);
  split(params->cv_r_switch, k.rs_hi, k.rs_lo);
  split(1.0 / (params->cv_r_cut - params->cv_r_switch), k.inv_w_hi, k.inv_w_lo);
  k.rs2 = (float)(params->cv_r_switch * params->cv_r_switch);
  k.rc2_far = (float)(params->cv_r_cut * params->cv_r_cut * (1.0 + 1e-4));
  k.r0 = params->cv_r0;
  k.rs = params->cv_r_switch;
  k.rc = params->cv_r_cut;
  k.n_cv = n_cv;
  k.min_sep = params->cv_min_sep;
  k.nb = (n_cv + CV_T - 1) / CV_T;
  const int n_tiles = k.nb * k.nb;
  double *zconst_part = sc.zcon;
  const int nclear = n_cv > n_tiles ? n_cv : n_tiles;
  if (nclear > 0) k_clear<<<(nclear + 255) / 256, 256, 0, st>>>(sc, n_cv, n_tiles);
  if (n_tiles > 0) k_cv_tile<<<(n_tiles * 32 + 127) / 128, 128, 0, st>>>(d_pos, d_native, k, sc, zconst_part);
  k_finish<<<1, 256, 0, st>>>(sc, zconst_part, n_tiles, n_cv, d_z, d_grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_msg(errbuf, errlen, cudaGetErrorString(e));
    return SIM_ECUDA;
  }
  set_msg(errbuf, errlen, "");
  return SIM_OK;
}

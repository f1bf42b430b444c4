// vp_contacts.cu -- the order in which native contacts form along each trial
// and the path similarity of two paths (Sec. "Results": the matrix M of
// contact-formation order and s(k, k'), after Camilloni et al. 2011).
//
// A contact (i, j) of reaction-coordinate atoms is formed when its contact
// value C(r) = (1 - (r/r0)^6)/(1 - (r/r0)^10) exceeds 1/2; with s = (r/r0)^2
// that is s^4 + s^3 - s^2 - s - 1 < 0, i.e. s below the polynomial's positive
// root.  The decision is taken in FP64 on the FP32 positions (exact
// differences), as the definition reads; an FP32 distance far from the
// threshold (outside a 1e-4 relative guard band, some 400 times its rounding
// error) decides alone.  The formation time of a native contact is the step
// from which it has stayed formed (-1: not formed at the last check); checks
// run every `every` steps.
#include <climits>
#include <cstring>
#include <string>

#include "../../include/vpath.h"
#include "vp_contacts.cuh"

namespace vp {

__device__ __forceinline__ bool contact_formed(float4 pi, float4 pj, float L, float iL, double Ld, double r0,
                                               float r2_lo, float r2_hi) {
  float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
  dx -= L * rintf(dx * iL);
  dy -= L * rintf(dy * iL);
  dz -= L * rintf(dz * iL);
  const float r2f = dx * dx + dy * dy + dz * dz;
  if (r2f < r2_lo) return true;
  if (r2f > r2_hi) return false;
  // FP64, every operation rounded on its own (no contraction), in the order of the definition
  double ex = __dsub_rn((double)pj.x, (double)pi.x), ey = __dsub_rn((double)pj.y, (double)pi.y),
         ez = __dsub_rn((double)pj.z, (double)pi.z);
  ex = __dsub_rn(ex, __dmul_rn(Ld, rint(__ddiv_rn(ex, Ld))));
  ey = __dsub_rn(ey, __dmul_rn(Ld, rint(__ddiv_rn(ey, Ld))));
  ez = __dsub_rn(ez, __dmul_rn(Ld, rint(__ddiv_rn(ez, Ld))));
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
  const double s = __ddiv_rn(r2, __dmul_rn(r0, r0));
  const double p =
      __dsub_rn(__dmul_rn(__dsub_rn(__dmul_rn(__dsub_rn(__dmul_rn(__dadd_rn(s, 1.0), s), 1.0), s), 1.0), s), 1.0);
  return p < 0.0;
}

// grid: (contacts of the largest system / 256, trials); the step counter has
// just been advanced to the step whose positions are current
__global__ void __launch_bounds__(256) k_contacts(Dev d, ContactDev c) {
  const long long n = *d.step;
  if (n % c.every != 0) return;
  const int t = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int sys = c.trial_sys[t];
  if (k >= c.sys_n[sys]) return;
  const int2 pr = c.pairs[c.sys_off[sys] + k];
  const TrialInfo &T = d.tinfo[t];
  const float4 pi = d.pos[d.slot_of[T.atom0 + pr.x]], pj = d.pos[d.slot_of[T.atom0 + pr.y]];
  const bool f = contact_formed(pi, pj, T.box, T.inv_box, (double)T.box, c.r0, c.r2_lo, c.r2_hi);
  long long *tt = c.t + c.t_off[t] + k;
  const long long cur = *tt;
  if (f) {
    if (cur < 0) *tt = n;
  } else if (cur >= 0) {
    *tt = -1;
  }
}

void launch_contacts(const Dev &d, const ContactDev &c, cudaStream_t s) {
  if (c.max_nc <= 0) return;
  dim3 grid((unsigned)((c.max_nc + 255) / 256), (unsigned)d.n_trials);
  k_contacts<<<grid, 256, 0, s>>>(d, c);
}

namespace {

constexpr int SIM_TILE = 2048;

// formation steps as 32-bit order keys: -1 (not formed) orders last; the
// caller guarantees steps below 2^31 - 1
__device__ __forceinline__ int order_key(long long t) { return t < 0 ? INT_MAX : (int)t; }

// sign of a - b in {-1, 0, 1} for keys of the same sign class (no overflow: 0 <= keys <= INT_MAX)
__device__ __forceinline__ int cmp3(int a, int b) { return (a > b) - (a < b); }

// one (path pair, block of i) per block: counts the ordered pairs (i != j)
// on which the two paths' order relations agree
__global__ void __launch_bounds__(256) k_similarity(const long long *__restrict__ t, long long n_c,
                                                    const int2 *__restrict__ pp, unsigned long long *count) {
  __shared__ int2 sab[SIM_TILE];
  __shared__ unsigned long long red[256];
  const int2 ab = pp[blockIdx.y];
  const long long *ta = t + (size_t)ab.x * (size_t)n_c, *tb = t + (size_t)ab.y * (size_t)n_c;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ai = i < n_c ? order_key(ta[i]) : 0, bi = i < n_c ? order_key(tb[i]) : 0;
  unsigned int cnt = 0;  // per thread: at most n_c < 2^31
  for (long long j0 = 0; j0 < n_c; j0 += SIM_TILE) {
    __syncthreads();
    for (int q = threadIdx.x; q < SIM_TILE; q += blockDim.x) {
      const long long j = j0 + q;
      sab[q] = j < n_c ? make_int2(order_key(ta[j]), order_key(tb[j])) : make_int2(0, 0);
    }
    __syncthreads();
    if (i < n_c) {
      const int m = (int)(n_c - j0 < SIM_TILE ? n_c - j0 : SIM_TILE);
#pragma unroll 4
      for (int q = 0; q < m; ++q) {
        const int2 v = sab[q];
        cnt += cmp3(ai, v.x) == cmp3(bi, v.y) ? 1u : 0u;
      }
    }
  }
  // the diagonal (j = i) always agrees; it is not an ordered pair
  if (i < n_c) cnt -= 1u;
  red[threadIdx.x] = cnt;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(count + blockIdx.y, red[0]);
}

int put_err(char *errbuf, int32_t errlen, int code, const std::string &msg) {
  if (errbuf && errlen > 0) {
    std::strncpy(errbuf, msg.c_str(), (size_t)errlen - 1);
    errbuf[errlen - 1] = '\0';
  }
  return code;
}

}  // namespace
}  // namespace vp

using namespace vp;

extern "C" __attribute__((visibility("default"))) int path_similarity(const int64_t *times, int32_t n_paths,
                                                                      int64_t n_c, const int32_t *pairs,
                                                                      int32_t n_pairs, double *s, void *cuda_stream,
                                                                      char *errbuf, int32_t errlen) {
  if (n_paths < 0 || n_c < 0 || n_pairs < 0 || (n_pairs > 0 && (!pairs || !s)) || (n_paths > 0 && n_c > 0 && !times))
    return put_err(errbuf, errlen, SIM_EINVAL, "path_similarity: null argument or negative size");
  for (int32_t q = 0; q < n_pairs; ++q)
    if (pairs[2 * q] < 0 || pairs[2 * q] >= n_paths || pairs[2 * q + 1] < 0 || pairs[2 * q + 1] >= n_paths)
      return put_err(errbuf, errlen, SIM_EINVAL, "path_similarity: path index out of range");
  if (n_pairs == 0) return SIM_OK;
  if (n_c < 2) {  // no ordered pair: identical by definition
    for (int32_t q = 0; q < n_pairs; ++q) s[q] = 1.0;
    return SIM_OK;
  }
  if (n_c > (1ll << 30)) return put_err(errbuf, errlen, SIM_EINVAL, "path_similarity: too many contacts");
  for (size_t k = 0; k < (size_t)n_paths * (size_t)n_c; ++k)
    if (times[k] >= (int64_t)INT_MAX) return put_err(errbuf, errlen, SIM_EINVAL, "path_similarity: step >= 2^31 - 1");
  if (n_pairs > 65535) return put_err(errbuf, errlen, SIM_EINVAL, "path_similarity: at most 65535 pairs per call");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  long long *dt = nullptr;
  int2 *dp = nullptr;
  unsigned long long *dc = nullptr;
  std::string err;
  auto ck = [&](cudaError_t e, const char *what) {
    if (e != cudaSuccess && err.empty()) err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  const size_t nt = (size_t)n_paths * (size_t)n_c;
  bool ok = ck(cudaMalloc(&dt, nt * sizeof(long long)), "cudaMalloc") &&
            ck(cudaMalloc(&dp, (size_t)n_pairs * sizeof(int2)), "cudaMalloc") &&
            ck(cudaMalloc(&dc, (size_t)n_pairs * sizeof(unsigned long long)), "cudaMalloc");
  ok = ok && ck(cudaMemcpyAsync(dt, times, nt * sizeof(long long), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
       ck(cudaMemcpyAsync(dp, pairs, (size_t)n_pairs * sizeof(int2), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
       ck(cudaMemsetAsync(dc, 0, (size_t)n_pairs * sizeof(unsigned long long), st), "cudaMemsetAsync");
  if (ok) {
    dim3 grid((unsigned)((n_c + 255) / 256), (unsigned)n_pairs);
    k_similarity<<<grid, 256, 0, st>>>(dt, (long long)n_c, dp, dc);
    ok = ck(cudaGetLastError(), "k_similarity launch");
  }
  unsigned long long *hc = new unsigned long long[(size_t)n_pairs];
  ok = ok && ck(cudaMemcpyAsync(hc, dc, (size_t)n_pairs * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st),
                "cudaMemcpyAsync");
  ck(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (ok && err.empty()) {
    const double denom = (double)n_c * (double)(n_c - 1);
    for (int32_t q = 0; q < n_pairs; ++q) s[q] = (double)hc[q] / denom;
  }
  delete[] hc;
  cudaFree(dt);
  cudaFree(dp);
  cudaFree(dc);
  if (!err.empty()) return put_err(errbuf, errlen, SIM_ECUDA, "path_similarity: " + err);
  return SIM_OK;
}

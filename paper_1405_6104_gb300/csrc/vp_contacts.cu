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
//
// The similarity of two paths counts the ordered contact pairs on which
// their order relations agree.  Only the order of the times within a path
// matters, so the host replaces them by dense ranks; with few distinct times
// (formation times are check steps) the count comes from the joint histogram
// of the two rank arrays in O(n_c + K_a K_b), otherwise from all n_c^2
// ordered pairs.
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

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
constexpr int HIST_CELLS = 4096;  // joint histogram capacity (K_a x K_b) of the counting kernel

// sign of a - b in {-1, 0, 1}
__device__ __forceinline__ int cmp3(int a, int b) { return (a > b) - (a < b); }

// all ordered pairs: one (path pair, block of i) per block counts the pairs
// (i != j) on which the two paths' order relations agree; keys are the
// paths' dense ranks (order-preserving, unformed contacts last)
__global__ void __launch_bounds__(256) k_similarity(const int *__restrict__ rk, long long n_c,
                                                    const int2 *__restrict__ pp, unsigned long long *count) {
  __shared__ int2 sab[SIM_TILE];
  __shared__ unsigned long long red[256];
  const int2 ab = pp[blockIdx.y];
  const int *ta = rk + (size_t)ab.x * (size_t)n_c, *tb = rk + (size_t)ab.y * (size_t)n_c;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ai = i < n_c ? ta[i] : 0, bi = i < n_c ? tb[i] : 0;
  unsigned int cnt = 0;  // per thread: at most n_c < 2^31
  for (long long j0 = 0; j0 < n_c; j0 += SIM_TILE) {
    __syncthreads();
    for (int q = threadIdx.x; q < SIM_TILE; q += blockDim.x) {
      const long long j = j0 + q;
      sab[q] = j < n_c ? make_int2(ta[j], tb[j]) : make_int2(0, 0);
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

// few distinct times (K_a K_b <= HIST_CELLS): one block per path pair counts
// the same agreements from the joint histogram H[x][y] of the two paths'
// ranks.  Two contacts in one cell tie in both paths (M = 1/2 in both:
// c (c - 1) ordered pairs agree); two contacts in cells strictly below-left
// and above-right of each other are concordant (both ordered pairs agree);
// every other pair disagrees.  So the count is sum c (c - 1) + 2 sum c P,
// with P the number of contacts strictly below-left of the cell.
__global__ void __launch_bounds__(256) k_similarity_hist(const int *__restrict__ rk, long long n_c,
                                                         const int2 *__restrict__ pp, const int *__restrict__ kk,
                                                         const int *__restrict__ list,
                                                         unsigned long long *count) {
  __shared__ unsigned H[HIST_CELLS];
  __shared__ unsigned long long red[256];
  const int q = list[blockIdx.x];
  const int2 ab = pp[q];
  const int Ka = kk[ab.x], Kb = kk[ab.y], nc = Ka * Kb;
  const int *ta = rk + (size_t)ab.x * (size_t)n_c, *tb = rk + (size_t)ab.y * (size_t)n_c;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) H[c] = 0u;
  __syncthreads();
  for (long long i = threadIdx.x; i < n_c; i += blockDim.x) atomicAdd(&H[ta[i] * Kb + tb[i]], 1u);
  __syncthreads();
  // P over the grid, in place, after each cell's own count has been used:
  // first the row prefix sums (exclusive along y), then the column ones
  // (exclusive along x) of those: then the cell holds the contacts strictly
  // below-left.  The cell counts are needed twice, so they are kept aside.
  unsigned long long acc = 0;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const unsigned long long v = H[c];
    acc += v * (v - (v > 0 ? 1ull : 0ull));
  }
  // row prefix (exclusive) per x: one thread per row
  __syncthreads();
  __shared__ unsigned rowcnt[HIST_CELLS];
  for (int c = threadIdx.x; c < nc; c += blockDim.x) rowcnt[c] = H[c];
  __syncthreads();
  for (int x = threadIdx.x; x < Ka; x += blockDim.x) {
    unsigned run = 0;
    for (int y = 0; y < Kb; ++y) {
      const unsigned v = H[x * Kb + y];
      H[x * Kb + y] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int y = threadIdx.x; y < Kb; y += blockDim.x) {
    unsigned run = 0;
    for (int x = 0; x < Ka; ++x) {
      const unsigned v = H[x * Kb + y];
      H[x * Kb + y] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) acc += 2ull * (unsigned long long)rowcnt[c] * H[c];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) count[q] = red[0];
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
  if (n_pairs > 65535) return put_err(errbuf, errlen, SIM_EINVAL, "path_similarity: at most 65535 pairs per call");
  // dense ranks per path (order-preserving; a negative time, not formed,
  // ranks after every formed contact): only the order relations enter s
  const size_t nt = (size_t)n_paths * (size_t)n_c;
  std::vector<int> rk(nt), K(n_paths);
  {
    // paths are ranked independently, on up to 16 host threads
    auto rank_paths = [&](int32_t p0, int32_t p1) {
      std::vector<int64_t> v((size_t)n_c), u;
      for (int32_t p = p0; p < p1; ++p) {
        const int64_t *tp = times + (size_t)p * (size_t)n_c;
        for (int64_t i = 0; i < n_c; ++i) v[(size_t)i] = tp[i] < 0 ? INT64_MAX : tp[i];
        u = v;
        std::sort(u.begin(), u.end());
        u.erase(std::unique(u.begin(), u.end()), u.end());
        K[p] = (int)u.size();
        for (int64_t i = 0; i < n_c; ++i)
          rk[(size_t)p * (size_t)n_c + (size_t)i] = (int)(std::lower_bound(u.begin(), u.end(), v[(size_t)i]) - u.begin());
      }
    };
    const int nw = (int)std::max(1u, std::min({std::thread::hardware_concurrency(), 16u, (unsigned)n_paths}));
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w)
      pool.emplace_back(rank_paths, (int32_t)((long long)n_paths * w / nw), (int32_t)((long long)n_paths * (w + 1) / nw));
    rank_paths(0, (int32_t)((long long)n_paths / nw));
    for (auto &th : pool) th.join();
  }
  // path pairs with few distinct times take the counting kernel, the rest
  // compare all ordered contact pairs
  std::vector<int> hist_list, all_list;
  for (int32_t q = 0; q < n_pairs; ++q) {
    const long long cells = (long long)K[pairs[2 * q]] * (long long)K[pairs[2 * q + 1]];
    (cells <= HIST_CELLS ? hist_list : all_list).push_back(q);
  }
  std::vector<int2> all_pp;
  for (int q : all_list) all_pp.push_back(make_int2(pairs[2 * q], pairs[2 * q + 1]));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int *dr = nullptr, *dk = nullptr, *dl = nullptr;
  int2 *dp = nullptr, *dpa = nullptr;
  unsigned long long *dc = nullptr, *dca = nullptr;
  std::string err;
  auto ck = [&](cudaError_t e, const char *what) {
    if (e != cudaSuccess && err.empty()) err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  const size_t np = (size_t)n_pairs, na = all_list.size(), nh = hist_list.size();
  bool ok = ck(cudaMalloc(&dr, nt * sizeof(int)), "cudaMalloc") &&
            ck(cudaMalloc(&dk, (size_t)n_paths * sizeof(int)), "cudaMalloc") &&
            ck(cudaMalloc(&dp, np * sizeof(int2)), "cudaMalloc") &&
            ck(cudaMalloc(&dc, np * sizeof(unsigned long long)), "cudaMalloc") &&
            (nh == 0 || ck(cudaMalloc(&dl, nh * sizeof(int)), "cudaMalloc")) &&
            (na == 0 || (ck(cudaMalloc(&dpa, na * sizeof(int2)), "cudaMalloc") &&
                         ck(cudaMalloc(&dca, na * sizeof(unsigned long long)), "cudaMalloc")));
  ok = ok && ck(cudaMemcpyAsync(dr, rk.data(), nt * sizeof(int), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
       ck(cudaMemcpyAsync(dk, K.data(), (size_t)n_paths * sizeof(int), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
       ck(cudaMemcpyAsync(dp, pairs, np * sizeof(int2), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
  if (ok && nh > 0) {
    ok = ck(cudaMemcpyAsync(dl, hist_list.data(), nh * sizeof(int), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    if (ok) {
      k_similarity_hist<<<(unsigned)nh, 256, 0, st>>>(dr, (long long)n_c, dp, dk, dl, dc);
      ok = ck(cudaGetLastError(), "k_similarity_hist launch");
    }
  }
  if (ok && na > 0) {
    ok = ck(cudaMemcpyAsync(dpa, all_pp.data(), na * sizeof(int2), cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") &&
         ck(cudaMemsetAsync(dca, 0, na * sizeof(unsigned long long), st), "cudaMemsetAsync");
    if (ok) {
      dim3 grid((unsigned)((n_c + 255) / 256), (unsigned)na);
      k_similarity<<<grid, 256, 0, st>>>(dr, (long long)n_c, dpa, dca);
      ok = ck(cudaGetLastError(), "k_similarity launch");
    }
  }
  std::vector<unsigned long long> hc(np, 0ull), ha(na, 0ull);
  if (ok && nh > 0)
    ok = ck(cudaMemcpyAsync(hc.data(), dc, np * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st),
            "cudaMemcpyAsync");
  if (ok && na > 0)
    ok = ck(cudaMemcpyAsync(ha.data(), dca, na * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st),
            "cudaMemcpyAsync");
  ck(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (ok && err.empty()) {
    for (size_t k = 0; k < na; ++k) hc[(size_t)all_list[k]] = ha[k];
    const double denom = (double)n_c * (double)(n_c - 1);
    for (int32_t q = 0; q < n_pairs; ++q) s[q] = (double)hc[(size_t)q] / denom;
  }
  cudaFree(dr);
  cudaFree(dk);
  cudaFree(dp);
  cudaFree(dc);
  cudaFree(dl);
  cudaFree(dpa);
  cudaFree(dca);
  if (!err.empty()) return put_err(errbuf, errlen, SIM_ECUDA, "path_similarity: " + err);
  return SIM_OK;
}

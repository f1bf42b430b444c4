// vp_step.cu -- one MD step of every trial as one cooperative kernel: the
// update, the rebuild decision, the list rebuilds that are due, the pair,
// bonded and reaction-coordinate forces and the finaliser, phases separated
// by grid barriers instead of kernel boundaries.  For batches too small to
// fill the GPU, where the step is made of short kernels and the gaps between
// them; the arithmetic of every phase is the same device code as the
// separate kernels', so both forms give bit-identical states.
//
// All blocks are resident at once (cooperative launch, grid sized from the
// occupancy of this kernel), so a grid barrier cannot deadlock; still every
// barrier polls a bounded number of times and, if it gives up, records
// ERR_TIMEOUT and ends the kernel (the host reports SIM_ETIMEOUT).
#include <algorithm>

#include "vp_cv_dev.cuh"
#include "vp_dev.cuh"
#include "vp_pair_dev.cuh"
#include "vp_rebuild_dev.cuh"
#include "vp_update_dev.cuh"

namespace vp {

constexpr int STEP_THREADS = PF_WARPS * 32;
static_assert(STEP_THREADS == LIST_WARPS * 32, "the list phase assumes one warp per cluster in 4-warp blocks");

union StepShared {
  // the forces phase: a warp works on reaction-coordinate tiles and on pair
  // clusters in any order, so both have their own tables
  struct {
    PairF2Shared pair;
    CvWarpShared cv[PF_WARPS];
  } force;
  ListShared list;
  ColsortShared colsort;
  CvfinShared cvfin;
  struct {
    int a[STEP_THREADS], c[STEP_THREADS];
  } scan;
};

// Grid barrier: bar[0] counts arrivals, bar[1] the generation.  The last
// block to arrive resets the count and opens the next generation; the others
// poll the generation at most `limit` times.  Returns false (in every thread
// of the block) when this block gave up.  Every thread fences afterwards, so
// what other blocks wrote before the barrier is seen after it.
__device__ __forceinline__ bool grid_sync(unsigned *bar, int *err, unsigned limit, volatile int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned polls = 0;
      while (*gen == g) {
        if (polls++ >= limit) {
          atomicOr(err, ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  __threadfence();
  return *s_ok != 0;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ unsigned ld_volatile(const unsigned *p) { return *(const volatile unsigned *)p; }

template <int MINB>
__global__ void __launch_bounds__(STEP_THREADS, MINB)
    k_step(Dev d, SimConst c, float rl2_bbox, float half_skin2, int strict) {
  __shared__ StepShared sh;
  __shared__ int s_ok;
  const unsigned limit = c.spin_limit;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;

  // ---- update (B-A-O-A of Eq. Lang); the work counters of later phases start at 0 ----
  if (blockIdx.x == 0 && threadIdx.x == 0) d.pair_next[1] = 0u;
  for (int slot = blockIdx.x * STEP_THREADS + threadIdx.x; slot < d.total_slots; slot += gridDim.x * STEP_THREADS)
    update_slot<UPD_DRIFT>(d, c, slot);
  if (!grid_sync(d.bar, d.err, limit, &s_ok)) return;

  // ---- which trials rebuild their lists ----
  const unsigned long long n = ld_volatile(d.cur_step);
  if (blockIdx.x == 0) decide_rebuilds(d, c, n, false);
  if (!grid_sync(d.bar, d.err, limit, &s_ok)) return;

  const int n_rb = (int)ld_volatile(d.rb_cnt);
  if (n_rb > 0) {
    const int per_slots = (d.max_trial_slots + STEP_THREADS - 1) / STEP_THREADS;
    for (int it = blockIdx.x; it < n_rb * per_slots; it += gridDim.x)
      bin_slot(d, c, half_skin2, strict, d.rb_list[it / per_slots], (it % per_slots) * STEP_THREADS + threadIdx.x, n);
    if (!grid_sync(d.bar, d.err, limit, &s_ok)) return;
    for (int b = blockIdx.x; b < n_rb; b += gridDim.x) {
      __syncthreads();
      colscan_trial<STEP_THREADS>(d, sh.scan.a, sh.scan.c, d.rb_list[b]);
    }
    if (!grid_sync(d.bar, d.err, limit, &s_ok)) return;
    for (int it = blockIdx.x; it < n_rb * per_slots; it += gridDim.x)
      colfill_slot(d, d.rb_list[it / per_slots], (it % per_slots) * STEP_THREADS + threadIdx.x);
    if (!grid_sync(d.bar, d.err, limit, &s_ok)) return;
    for (int it = blockIdx.x; it < n_rb * d.max_trial_cols; it += gridDim.x) {
      __syncthreads();
      colsort_column<false>(d, sh.colsort, d.rb_list[it / d.max_trial_cols], it % d.max_trial_cols);
    }
    if (!grid_sync(d.bar, d.err, limit, &s_ok)) return;
    const int n_items = n_rb * d.max_trial_clus;
    for (;;) {
      __syncwarp();
      unsigned got = 0u;
      if (lane == 0) got = atomicAdd(d.rb_cnt + 1, 1u);
      const int item = (int)__shfl_sync(0xffffffffu, got, 0);
      if (item >= n_items) break;
      list_cluster(d, c, rl2_bbox, sh.list, d.rb_list[item / d.max_trial_clus], item % d.max_trial_clus);
    }
    if (!grid_sync(d.bar, d.err, limit, &s_ok)) return;
  }

  // ---- forces: one queue of warp items, the longest first: reaction-
  // coordinate tiles (costliest first), pair clusters, then the bonded
  // groups 32 at a time (a lane each), so that the short items fill in
  // around the long ones ----
  {
    const int n_cv = d.total_work, n_pair = d.total_clus;
    const int n_bond = (d.n_trials * d.max_nbg + 31) / 32;
    for (;;) {
      __syncwarp();
      unsigned got = 0u;
      if (lane == 0) got = atomicAdd(d.pair_next + 1, 1u);
      const int item = (int)__shfl_sync(0xffffffffu, got, 0);
      if (item < n_cv) {
        cv_tile(d, c, sh.force.cv[wib], item);
      } else if (item < n_cv + n_pair) {
        pair_cluster_f2(d, c, sh.force.pair, item - n_cv);
      } else if (item < n_cv + n_pair + n_bond) {
        const int k = (item - n_cv - n_pair) * 32 + lane;
        if (k < d.n_trials * d.max_nbg) bonded_group(d, k / d.max_nbg, k % d.max_nbg);
      } else {
        break;
      }
    }
  }
  if (!grid_sync(d.bar, d.err, limit, &s_ok)) return;

  // ---- per trial: z, the ratchet, Phi; the last trial advances the step ----
  for (int t = blockIdx.x; t < d.n_trials; t += gridDim.x) cvfin_trial<FIN_STEP>(d, c, sh.cvfin, t);
}

constexpr int STEP_MINB = 7;

cudaError_t launch_step_fused(const Dev &d, const SimConst &c, float rl2_bbox, float half_skin2, int strict,
                              cudaStream_t s) {
  static int per_sm = -1;  // resident blocks per SM of this kernel (occupancy is the same on every device here)
  if (per_sm < 0) {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_step<STEP_MINB>, STEP_THREADS, 0);
    if (e != cudaSuccess) return e;
    per_sm = v;
  }
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  // no more blocks than the pair phase has four-warp shares of i-clusters:
  // a small batch then has fewer blocks to gather at each barrier
  const long long shares = ((long long)d.total_clus + PF_WARPS - 1) / PF_WARPS;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::max(1LL, std::min((long long)d.n_sm * per_sm, shares)));
  cfg.blockDim = dim3(STEP_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_step<STEP_MINB>, d, c, rl2_bbox, half_skin2, strict);
}

}  // namespace vp

// vp_rebuild.cu -- cell binning, spatial sort into 8-atom clusters and the
// Verlet list (8-atom i-clusters, one entry per j-atom) of the trials whose
// list is due.
//
// Every kernel here runs in every step and works only on the trials whose
// list is due in that step: the front kernel (one block per trial) decides,
// bins, scans and fills per trial and lists the rebuilding trials in
// d.rb_list; the later kernels take their work items (columns, slot chunks,
// clusters) from that list.  A trial's list is due when one of its atoms has moved
// farther than skin/2 - 1e-5 nm from where its list was built (the update
// kernel requests it), after nstlist steps, or on request from the host
// (creation, a new state).  The first rule keeps every pair closer than r_cut
// in the list at every force evaluation: two atoms that were at least
// r_cut + skin apart when the list was built are still farther apart than
// r_cut (the 1e-5 nm cover FP32 rounding).
//
// Layout: per trial the box is cut into ncol x ncol columns along x and y;
// atoms are sorted by (column, z) and cut into clusters of 8 (the last
// cluster of a column is padded).  The list build tests 4-atom j-clusters
// (halves of i-clusters) against each 8-atom i-cluster and writes one list
// entry per j-atom with at least one pair that satisfies the FP32 list rule
// and is not excluded, with an 8-bit mask of those pairs; the half list keeps
// j-clusters whose parent cluster index is >= the i-cluster (upper triangle
// inside a cluster).
#include <algorithm>

#include "vp_dev.cuh"
#include "vp_rebuild_dev.cuh"

namespace vp {

// ---------------------------------------------------------------------------
// binning: wrap into the box, pick the column, count, skin check
// ---------------------------------------------------------------------------
// forced rebuild of one trial (trial >= 0) or of all, in the step held now
// (the front kernel that follows rebuilds exactly those trials)
__global__ void k_rebuild_request(Dev d, int trial) {
  const unsigned long long n = *d.cur_step;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < d.n_trials; t += gridDim.x * blockDim.x)
    if (trial < 0 || t == trial) d.rb[d.n_trials + t] = (uint32_t)n;
}

// work items of the rebuilding trials: each trial cut into `per` pieces,
// items taken in grid-stride order by whole blocks
#define FOR_REBUILD_ITEMS(per, t, piece)                                                  \
  for (int item_ = blockIdx.x, n_items_ = (int)d.rb_cnt[0] * (per); item_ < n_items_;     \
       item_ += gridDim.x)                                                                 \
    if (const int t = d.rb_list[item_ / (per)], piece = item_ % (per); true)

// ---------------------------------------------------------------------------
// the decision and the first part of the rebuild: one cluster of blocks per
// trial; a cluster whose trial is due bins its atoms, scans the columns and
// fills the column buckets; block 0 also writes the list of rebuilding
// trials that the later kernels walk.  No block writes what another reads to
// decide (the requests, the last-rebuild stamps: the column sort stamps them).
// ---------------------------------------------------------------------------
// cond_a, cond_b (with set_cond): conditional nodes of a captured graph
// around the later rebuild kernels, opened only when a trial rebuilds
__global__ void __cluster_dims__(FRONT_CLUSTER, 1, 1) __launch_bounds__(FRONT_THREADS, 1)
    k_front(Dev d, SimConst c, float half_skin2, int strict, int forced_only, cudaGraphConditionalHandle cond_a,
            cudaGraphConditionalHandle cond_b, int set_cond) {
  __shared__ FrontShared sh;
  PDL_WAIT();
  const unsigned long long n = *d.cur_step;
  if (blockIdx.x == 0) {
    decide_rebuilds(d, c, n, forced_only != 0);
    if (set_cond) {
      __syncthreads();  // every decision is counted
      if (threadIdx.x == 0) {
        const unsigned any = d.rb_cnt[0] != 0u ? 1u : 0u;
        cudaGraphSetConditional(cond_a, any);
        cudaGraphSetConditional(cond_b, any);
      }
    }
  }
  const int n_clusters = (int)gridDim.x / FRONT_CLUSTER;
  // the whole cluster takes the same trials (the same decision in every block)
  for (int t = (int)blockIdx.x / FRONT_CLUSTER; t < d.n_trials; t += n_clusters) {
    if (!trial_due(d, c, t, n, forced_only != 0)) continue;
    front_trial(d, c, half_skin2, strict, sh, t, n);
  }
}

// ---------------------------------------------------------------------------
// per column: sort by (z, atom index), write the new cluster layout, update
// slot_of, pad the last cluster and compute cluster bounding boxes
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_colsort(Dev d) {
  __shared__ ColsortShared sh;
  PDL_WAIT();
  FOR_REBUILD_ITEMS(d.max_trial_cols, t, piece) {
    __syncthreads();  // the previous column's shared arrays are no longer read
    colsort_column<true>(d, sh, t, piece);
  }
}

// one warp per cluster of a rebuilding trial, clusters handed out by a
// counter (their lists differ in length)
__global__ void __launch_bounds__(LIST_WARPS * 32, 8) k_list(Dev d, SimConst c, float rl2_bbox) {
  __shared__ ListShared sh;
  PDL_WAIT();
  const int lane = threadIdx.x & 31;
  const int n_items = (int)d.rb_cnt[0] * d.max_trial_clus;
  for (;;) {
    __syncwarp();  // the warp's shared arrays of its previous cluster are no longer read
    unsigned got = 0u;
    if (lane == 0) got = atomicAdd(d.rb_cnt + 1, 1u);
    const int item = (int)__shfl_sync(0xffffffffu, got, 0);
    if (item >= n_items) return;
    list_cluster(d, c, rl2_bbox, sh, d.rb_list[item / d.max_trial_clus], item % d.max_trial_clus);
  }
}

// positions the current list of one trial was built from, caller order
__global__ void k_list_positions(Dev d, int trial, double *out, int n) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const float4 p = d.ref_slot[d.slot_of[d.tinfo[trial].atom0 + o]];
  out[3 * o] = p.x;
  out[3 * o + 1] = p.y;
  out[3 * o + 2] = p.z;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// The grids are fixed (they are captured in graphs) and sized from the SM
// count; their blocks and warps walk the work items of the trials that
// rebuild in the step, so a step in which few trials rebuild costs little.
// (no more blocks than items in the largest possible step: all trials rebuilding)
static unsigned rebuild_grid(const Dev &d, int per_sm, long long per_trial) {
  return (unsigned)std::max(1LL, std::min((long long)d.n_sm * per_sm, per_trial * d.n_trials));
}

void launch_rebuild_request(const Dev &d, int32_t trial, cudaStream_t s) {
  k_rebuild_request<<<(d.n_trials + 255) / 256, 256, 0, s>>>(d, trial);
}
void launch_front(const Dev &d, const SimConst &c, float half_skin2, int strict_skin, bool forced_only,
                  cudaStream_t s, const cudaGraphConditionalHandle *cond) {
  const unsigned clusters = (unsigned)std::min(d.n_trials, 16384);
  launch_pdl(k_front, dim3(clusters * FRONT_CLUSTER), dim3(FRONT_THREADS), s, d, c, half_skin2, strict_skin,
             forced_only ? 1 : 0, cond ? cond[0] : cudaGraphConditionalHandle(0),
             cond ? cond[1] : cudaGraphConditionalHandle(0), cond ? 1 : 0);
}
void launch_list_positions(const Dev &d, int32_t trial, double *out, int32_t n, cudaStream_t s) {
  if (n > 0) k_list_positions<<<(n + 255) / 256, 256, 0, s>>>(d, trial, out, n);
}
void launch_colsort(const Dev &d, cudaStream_t s) {
  // columns hold about 100 atoms: 128 threads keep every thread busy in the sort
  launch_pdl(k_colsort, dim3(rebuild_grid(d, 8, d.max_trial_cols)), dim3(128), s, d);
}
void launch_list(const Dev &d, const SimConst &c, float rl2_bbox, cudaStream_t s) {
  launch_pdl(k_list, dim3(rebuild_grid(d, 8, (d.max_trial_clus + LIST_WARPS - 1) / LIST_WARPS)), dim3(LIST_WARPS * 32),
             s, d, c, rl2_bbox);
}

}  // namespace vp

// vp_dev.cuh -- the device buffers of one batch (passed by value to every
// kernel) and the host launchers of all kernels.
#pragma once
#include "vp_internal.cuh"

namespace vp {

struct Dev {
  int32_t n_trials, n_sys;
  int32_t total_slots, total_clus, total_cols, total_work;
  // one 4-atom half cluster past the last slot (pos, type and force arrays
  // hold total_slots + 4 entries) sits at idle_pos(): the entry of a lane
  // with no list entry to work on points there (with an empty mask), so its
  // pairs fall outside the cut-off with or without the pair masks
  uint32_t idle_entry;
  TrialInfo *tinfo;
  TrialState *tstate;
  // slots (cluster order); *_b are the targets of the re-sort at a rebuild
  float4 *pos, *vel, *pos_b, *vel_b;   // pos.w = q*sqrt(f), vel.w = 1/m
  int32_t *orig, *type, *orig_b, *type_b;
  int32_t *slot_trial;                 // static: trial of every slot
  int32_t *slot_col;                   // grid column of every slot at binning (-1: none)
  long long *fx, *fy, *fz;             // fixed-point force accumulators per slot
  // clusters
  int32_t *clus_trial;                 // static: trial of every i-cluster
  float4 *bb_lo, *bb_hi;               // bounding boxes of the 4-atom half clusters (wrapped positions at rebuild)
  uint32_t *list;                      // [total_clus * list_cap] j-atom entries (see vp_internal.cuh)
  uint8_t *list_m;                     // [total_clus * list_cap] their pair masks
  int32_t *list_n;                     // entries per i-cluster ...
  int32_t *list_nm;                    // ... of which the first list_nm need the pair masks (exclusions,
                                       // the cluster itself, mixed images); the pair kernels apply the
                                       // masks in every group of 32 entries that starts below list_nm
  // grid columns
  int32_t *col_trial;                  // static
  int32_t *col_count, *col_start, *col_cstart, *col_fill;
  int32_t *col_ztab;                   // [columns * (ZBINS + 1)]: halves of the column with z_lo below b L / ZBINS
  int32_t *bucket;                     // [total trial atoms]
  // per trial, caller-ordered
  int32_t *slot_of;                    // [total trial atoms]
  float4 *ref_slot;                    // [slots] the positions the trial's current list was built from
  long long *gx, *gy, *gz;             // CV gradient, fixed point, [total CV atoms]
  double *z_part;                      // [total_work] per-tile partial sums of z
  // per system, caller-ordered
  AtomSys *asys;
  double *gm;                          // gamma_i m_i
  double *inv_gm;                      // 1 / (gamma_i m_i) (0 without friction)
  int32_t *excl, *excl_n;              // [sys atoms * MAX_EXCL], counts
  int32_t *bt_start;                   // [total system atoms + 1] CSR of owner-computed bonded terms (energies)
  BTerm *bterm;
  BGroup *bgrp;                        // bonded terms for forces in groups over at most 3 atoms
  int32_t *sys_bg0, *sys_nbg;          // per system: first group, count
  int32_t max_nbg;                     // largest group count of a system
  // reaction coordinate
  int2 *tiles;                         // per system tile (bi, bj), concatenated
  int2 *work;                          // flat (trial, global tile) work items
  int32_t *work_order;                 // the order warps take them: tiles near the diagonal (most near pairs) first
  double *cnat;                        // [tiles * 1024] C~ of the native structure in tile-skew order
  float2 *cnat_ff;                     // the same as float-float (hi, lo), read by the per-step kernel
  int32_t *sys_ncv, *sys_minsep;
  // Lennard-Jones pair table over de-duplicated types
  float2 *ljtab;                       // (6 c6, 12 c12)
  float *ljshift;                      // potential at r_cut
  // globals
  int32_t *err;
  long long *step;
  float *kick;
  unsigned int *done;                  // block ticket of the per-trial finaliser
  long long *energy;                   // [n_trials * 5] fixed point (2^24): LJ, RF, bond, angle, kin
  long long *diag;                     // [4]: skin violations (fixed-interval lists), trial rebuilds,
                                       // rebuilds triggered by a displacement, spare
  // list rebuilds: a trial's list is rebuilt in the step whose number (low
  // 32 bits) its decision entry holds
  unsigned long long *cur_step;        // number of the step being computed (or of the state held)
  uint32_t *rb;                        // [2 n_trials]: displacement request, forced request
  uint32_t *last_rb;                   // [n_trials] step of the trial's last rebuild
  int32_t *rb_list;                    // [n_trials] the trials rebuilding in this step (any order) ...
  uint32_t *rb_cnt;                    // [4]: ... their number, the list kernel's work counter, spare
  int32_t max_trial_slots, max_trial_cols, max_trial_clus;  // largest of any trial
  double *rec;                         // [n_trials * rec_cap * 5]: z, z_m, a, phi, Q
  unsigned *pair_next;                 // work counters: [0] the persistent pair kernel; [1] the
                                       // one-kernel step's forces phase; [2] spare
  unsigned *bar;                       // [2] grid barrier of the one-kernel step: arrivals, generation
  int32_t n_sm;                        // multiprocessors of the device
};

// whether trial t rebuilds its list in step n: a forced request, or (unless
// forced_only) a displacement request, or nstlist steps since its last
// rebuild (with fixed intervals: every nstlist-th step)
__device__ __forceinline__ bool trial_due(const Dev &d, const SimConst &c, int t, unsigned long long n,
                                          bool forced_only) {
  const uint32_t n32 = (uint32_t)n;
  if (d.rb[d.n_trials + t] == n32) return true;
  if (forced_only) return false;
  if (d.rb[t] == n32) return true;
  if (c.list_fixed) return n % (unsigned long long)c.nstlist == 0ull;
  return n32 - d.last_rb[t] >= (uint32_t)c.nstlist;
}

// Which trials rebuild their lists in step n (executed by one whole block:
// block 0 of the rebuild front kernel, or of the one-kernel step): the
// trials for which trial_due holds go to rb_list, which the later rebuild
// kernels walk.
__device__ __forceinline__ void decide_rebuilds(const Dev &d, const SimConst &c, unsigned long long n,
                                                bool forced_only) {
  if (threadIdx.x == 0) {
    d.rb_cnt[0] = 0u;
    d.rb_cnt[1] = 0u;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < d.n_trials; t += blockDim.x)
    if (trial_due(d, c, t, n, forced_only)) d.rb_list[atomicAdd(d.rb_cnt, 1u)] = t;
}

enum UpdateMode { UPD_DRIFT = 0, UPD_FINAL = 1 };

// shared memory of one warp's reaction-coordinate tile
struct CvWarpShared {
  unsigned short s_near[CV_T * CV_T];
  float s_x[2 * CV_T][3];
  // gradient of the tile's 64 atoms: each fixed-point contribution c splits
  // into c >> 24 (signed) and its low 24 bits, summed in 32-bit shared
  // atomics (native, unlike 64-bit ones); at most 32 contributions per entry
  // keep both sums far from overflow, and (hi << 24) + lo is the exact sum
  int s_ghi[2 * CV_T][3];
  unsigned s_glo[2 * CV_T][3];
};
constexpr int CVFIN_THREADS = 1024;  // the finaliser's reduction width (virtual threads)
struct CvfinShared {
  double rz[CVFIN_THREADS], rq[CVFIN_THREADS];
  bool last;
};
// FIN_STEP: a step (Phi accumulates, the step counter advances); FIN_INIT:
// z_m = z; FIN_RESTORE: a new state (z and a from the stored z_m, the record
// entry of the current step rewritten); FIN_KEEP: the same state again after a
// forced list rebuild (nothing recorded)
enum FinMode { FIN_STEP = 0, FIN_INIT = 1, FIN_RESTORE = 2, FIN_KEEP = 3 };

// Programmatic dependent launch: a kernel that follows another kernel on
// the same stream may be launched while that one drains (its launch latency
// then overlaps the other's tail); such a kernel starts with PDL_WAIT, which
// returns once the preceding kernel has completed and its writes are
// visible (a no-op for an ordinary launch).
#define PDL_WAIT() cudaGridDependencySynchronize()

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// rebuild (vp_rebuild.cu)
// a forced rebuild of one trial (trial >= 0) or of all in the step held now
void launch_rebuild_request(const Dev &d, int32_t trial, cudaStream_t s);
// which trials rebuild (forced_only: those with a forced request), then
// binning, column scans and bucket fills of those trials
void launch_front(const Dev &d, const SimConst &c, float half_skin2, int strict_skin, bool forced_only,
                  cudaStream_t s, const cudaGraphConditionalHandle *cond = nullptr);  // cond: two handles, or none
void launch_colsort(const Dev &d, cudaStream_t s);
void launch_list(const Dev &d, const SimConst &c, float rl2_bbox, cudaStream_t s);
void launch_list_positions(const Dev &d, int32_t trial, double *out, int32_t n, cudaStream_t s);
// forces (vp_pair.cu)
// clist (optional): the i-clusters to work on (n_items of them), else all
void launch_pair(const Dev &d, const SimConst &c, bool energy, int32_t only_trial, cudaStream_t s, int variant = 0,
                 const int *clist = nullptr, int n_items = 0);
void launch_bonded(const Dev &d, cudaStream_t s);
constexpr int PAIR_VARIANTS = 9;
// reaction coordinate and functional (vp_cv.cu)
void launch_cnat(const Dev &d, const SimConst &c, const double *native, const int32_t *sys_nat0, int32_t n_tiles_total,
                 const int32_t *tile_sys, cudaStream_t s);
void launch_zconst(const Dev &d, const int32_t *sys_tile0, const int32_t *sys_ntiles, cudaStream_t s);
// after_kernel: the launch follows a kernel on its stream (a programmatic launch)
void launch_cv(const Dev &d, const SimConst &c, cudaStream_t s, int variant = 0, bool after_kernel = true);
constexpr int CV_VARIANTS = 3;
void launch_cvfin(const Dev &d, const SimConst &c, FinMode mode, cudaStream_t s);
void launch_rec_frames(const Dev &d, int trial, int n_cv, int cap, float *frames, cudaStream_t s);
// integrator and state (vp_update.cu)
void launch_update(const Dev &d, const SimConst &c, UpdateMode mode, cudaStream_t s);
void launch_init_vel(const Dev &d, float kT, const int32_t *need, cudaStream_t s);
void launch_scatter_state(const Dev &d, int32_t trial, const double *pos, const double *vel, int32_t n, cudaStream_t s);
void launch_gather_state(const Dev &d, int32_t trial, double *pos, double *vel, int32_t n, cudaStream_t s);
void launch_check_finite(const double *x, size_t n, int *flag, cudaStream_t s);
void launch_forces_out(const Dev &d, const SimConst &c, int32_t trial, double *out, int32_t n, cudaStream_t s);
void launch_kinetic(const Dev &d, int32_t trial, cudaStream_t s);
void launch_scatter_positions(const Dev &d, const SimConst &c, const double *pos, int32_t n, cudaStream_t s);
void launch_potential_out(const Dev &d, double *energy, double *forces, int32_t n, cudaStream_t s);
void launch_extract_pairs(const Dev &d, int32_t list_cap, int32_t trial, int32_t n_clus, int32_t *pairs,
                          long long cap, unsigned long long *count, cudaStream_t s);
void launch_philox_normals(uint64_t seed, unsigned long long step, uint32_t stream, int n, uint32_t *raw,
                           double *normals, cudaStream_t s);
void launch_select(const Dev &d, double z_max, double *phi_out, int32_t *argmin_out, cudaStream_t s);
// one MD step of every trial as one cooperative kernel (vp_step.cu)
cudaError_t launch_step_fused(const Dev &d, const SimConst &c, float rl2_bbox, float half_skin2, int strict,
                              cudaStream_t s);

}  // namespace vp

// vp_capi.cu -- host side of the C ABI declared in include/vpath.h: batch
// construction, the per-step launch sequence, CUDA-graph capture of list
// intervals, state transfer and diagnostics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "../../include/vpath.h"
#include "vp_adjoint.cuh"
#include "vp_contacts.cuh"
#include "vp_dev.cuh"

#define VP_API extern "C" __attribute__((visibility("default")))

using namespace vp;

namespace {

struct Timer {
  const char *name;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  double ms = 0.0;
  long long count = 0;
};

}  // namespace

struct sim_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t caller = nullptr;
  cudaEvent_t entry_ev = nullptr, exit_ev = nullptr;
  // second stream of the captured chunk: the reaction coordinate (CV and its
  // finaliser) reads only positions, so it runs beside the list build and the
  // pair forces, joined before the next update
  cudaStream_t side = nullptr;
  cudaStream_t cstream = nullptr;  // captures the bodies of conditional nodes (step form 2)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t bstream = nullptr;  // the bonded forces, beside the reaction coordinate
  cudaEvent_t ev_bjoin = nullptr;
  Dev d{};
  SimConst c{};
  sim_params params{};
  int n_sys = 0, n_trials = 0;
  std::vector<TrialInfo> tinfo;
  std::vector<int> trial_sys;
  long long step = 0;
  float rl2_bbox = 0.f, half_skin2 = 0.f;
  int strict_skin = 0;
  bool use_graph = true;
  cudaGraphExec_t chunk = nullptr;
  bool timing = false;
  // in-graph timing: external event-record nodes around each pair-kernel
  // launch of the captured chunk, read after every graph replay
  bool gtiming = false;
  int cap_k = -1;  // step index inside the chunk being captured (-1: not capturing)
  std::vector<cudaEvent_t> gev;
  std::vector<Timer> timers;
  std::map<std::string, int> timer_idx;
  std::vector<void *> allocs;
  std::string err;
  int rec_cap = 0;
  int pair_variant = 0, cv_variant = 0;  // launch shapes picked by the autotuner
  // size classes of the batch (trials grouped by atom count, density and
  // type count) and, when the autotuner found it faster, one pair launch per
  // class over its clusters with the class's own variant
  struct SizeClass {
    int lg_atoms = 0, n_trials = 0, n_clus = 0, variant = 0;
    int *clist = nullptr;
  };
  std::vector<SizeClass> classes;
  bool per_class = false;
  // step form: false = one kernel per phase (CUDA-graph replays of chunks),
  // true = one cooperative kernel per step (replayed in graphs when the
  // capture succeeds, else launched directly)
  bool fused = false, fused_no_graph = false;
  bool skip_empty = false;  // step form 2: graph nodes of the later rebuild kernels only when a trial rebuilds
  bool capture_failed = false;  // a conditional node could not be added while capturing a chunk
  // CV-frame recorder (one trial)
  int frame_trial = -1, frame_cap = 0;
  float *frames = nullptr;
  // staging
  double *dbuf = nullptr;
  size_t dbuf_n = 0;
  int32_t *d_argmin = nullptr;
  unsigned long long *d_count = nullptr;
  int *d_flag = nullptr;  // device flag of host-side checks done on the GPU
  int max_atoms = 0;
  // native structures (host copy, per system: first CV atom in native_all, CV atoms, min separation)
  std::vector<double> native_all;
  std::vector<int32_t> sys_nat0, sys_ncv, sys_minsep;
  // native-contact formation tracker (built on first use)
  ContactDev cdev{};
  bool contacts_built = false;
  bool contacts_tracked = false;     // sim_contact_tracking was called
  std::vector<int32_t> csys_n;       // native contacts per system
  std::vector<long long> ct_off;     // per trial: first entry of its formation times
  std::vector<void *> callocs;
};

namespace {

int fail(sim_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  return code;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(h, SIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
int dalloc(sim_handle *h, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess) return fail(h, SIM_ECUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(*p);
  cudaMemset(*p, 0, n * sizeof(T));
  return SIM_OK;
}

template <class T>
int upload(sim_handle *h, T **p, const std::vector<T> &v) {
  int r = dalloc(h, p, v.size());
  if (r) return r;
  if (!v.empty()) {
    cudaError_t e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(h, SIM_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  }
  return SIM_OK;
}

void ff_split(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// kernel launch with optional CUDA-event timing
template <class F>
void timed(sim_handle *h, const char *name, F &&f) {
  if (!h->timing) {
    f();
    return;
  }
  auto it = h->timer_idx.find(name);
  int k;
  if (it == h->timer_idx.end()) {
    k = (int)h->timers.size();
    h->timer_idx[name] = k;
    h->timers.push_back(Timer{name, {}, 0.0, 0});
  } else {
    k = it->second;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, h->stream);
  f();
  cudaEventRecord(b, h->stream);
  h->timers[k].ev.emplace_back(a, b);
}

void harvest_timers(sim_handle *h) {
  for (auto &t : h->timers) {
    for (auto &pr : t.ev) {
      float ms = 0.f;
      cudaEventSynchronize(pr.second);
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      t.ms += ms;
      t.count += 1;
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    t.ev.clear();
  }
}

Timer &timer(sim_handle *h, const char *name) {
  auto it = h->timer_idx.find(name);
  if (it != h->timer_idx.end()) return h->timers[it->second];
  h->timer_idx[name] = (int)h->timers.size();
  h->timers.push_back(Timer{name, {}, 0.0, 0});
  return h->timers.back();
}

// durations of the pair-kernel launches of the last chunk replay
int harvest_graph_timers(sim_handle *h) {
  Timer &t = timer(h, "pair_in_graph");
  for (int k = 0; k + 1 < (int)h->gev.size(); k += 2) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, h->gev[k], h->gev[k + 1]);
    if (e != cudaSuccess) return fail(h, SIM_ECUDA, std::string("in-graph timing: ") + cudaGetErrorString(e));
    t.ms += ms;
    t.count += 1;
  }
  return SIM_OK;
}

// which trials rebuild, their cell binning and the spatial sort (the new
// atom slots); forced_only: the trials with a forced request alone
void rebuild_cols(sim_handle *h, bool forced_only) {
  cudaStream_t s = h->stream;
  timed(h, "front", [&] { launch_front(h->d, h->c, h->half_skin2, h->strict_skin, forced_only, s); });
  timed(h, "colsort", [&] { launch_colsort(h->d, s); });
}

void rebuild_list(sim_handle *h) {
  timed(h, "list", [&] { launch_list(h->d, h->c, h->rl2_bbox, h->stream); });
}

// the nonbonded forces of every trial: one launch over all clusters, or one
// per size class with the class's variant
void launch_pair_hot(const sim_handle *h, const Dev &d, cudaStream_t s) {
  if (!h->per_class) {
    launch_pair(d, h->c, false, -1, s, h->pair_variant);
    return;
  }
  for (const auto &k : h->classes) launch_pair(d, h->c, false, -1, s, k.variant, k.clist, k.n_clus);
}

void pair_forces(sim_handle *h) {
  cudaStream_t s = h->stream;
  if (h->gtiming && h->cap_k >= 0) {
    cudaEventRecordWithFlags(h->gev[2 * h->cap_k], s, cudaEventRecordExternal);  // a failure ends the capture
    launch_pair_hot(h, h->d, s);
    cudaEventRecordWithFlags(h->gev[2 * h->cap_k + 1], s, cudaEventRecordExternal);
  } else {
    timed(h, "pair", [&] { launch_pair_hot(h, h->d, s); });
  }
}

// the forces beside the pair kernel, on one stream: bonded forces, then the
// reaction coordinate and its finaliser
void cv_forces(sim_handle *h, FinMode mode, cudaStream_t s) {
  timed(h, "bonded", [&] { launch_bonded(h->d, s); });
  timed(h, "cv", [&] { launch_cv(h->d, h->c, s, h->cv_variant); });
  timed(h, "cvfin", [&] { launch_cvfin(h->d, h->c, mode, s); });
}

// ... or as two branches forked from the main stream: the reaction
// coordinate and its finaliser on the second stream, the bonded forces on a
// third (none reads what another writes; forces meet in order-independent
// fixed-point sums); join_side brings both back
void fork_side(sim_handle *h, FinMode mode) {
  cudaEventRecord(h->ev_fork, h->stream);
  cudaStreamWaitEvent(h->side, h->ev_fork, 0);
  cudaStreamWaitEvent(h->bstream, h->ev_fork, 0);
  launch_cv(h->d, h->c, h->side, h->cv_variant, false);
  launch_cvfin(h->d, h->c, mode, h->side);
  cudaEventRecord(h->ev_join, h->side);
  launch_bonded(h->d, h->bstream);
  cudaEventRecord(h->ev_bjoin, h->bstream);
}
void join_side(sim_handle *h) {
  cudaStreamWaitEvent(h->stream, h->ev_join, 0);
  cudaStreamWaitEvent(h->stream, h->ev_bjoin, 0);
}

// reaction-coordinate atoms per frame: of the recorded trial, or the largest
// n_cv when every trial is recorded (frame_trial < 0)
int frame_stride(const sim_handle *h) {
  if (h->frame_trial >= 0) return h->tinfo[h->frame_trial].n_cv;
  int m = 0;
  for (const auto &T : h->tinfo) m = std::max(m, T.n_cv);
  return m;
}

// what follows the forces: contact tracking and the frame recorder read the
// step counter that the CV finaliser has advanced
void after_forces(sim_handle *h, FinMode mode) {
  cudaStream_t s = h->stream;
  if (mode == FIN_STEP && h->cdev.every > 0) launch_contacts(h->d, h->cdev, s);
  if (h->frames)
    launch_rec_frames(h->d, h->frame_trial, frame_stride(h), h->frame_cap, h->frames, s);
}

constexpr int NO_REQUEST = -2;  // forces(): no forced list rebuild
constexpr int STEP_MODES = SIM_STEP_MODES;

// Adds to the graph being captured on h->stream a conditional node whose body
// is captured from `body` (launches on the stream given to it); returns the
// handle (the kernel that sets it must come earlier in the same graph).
int add_conditional(sim_handle *h, cudaGraphConditionalHandle hc, const std::function<void(cudaStream_t)> &body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(h->stream, &st, nullptr, &g, &deps, &ed, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, &cp));
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  CK(cudaStreamBeginCaptureToGraph(h->cstream, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  body(h->cstream);
  CK(cudaStreamEndCapture(h->cstream, &bg));
  return SIM_OK;
}

// a new conditional handle of the graph being captured on h->stream (its
// value is 1 unless a kernel of the graph sets it)
int new_conditional(sim_handle *h, cudaGraphConditionalHandle *hc) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g;
  CK(cudaStreamGetCaptureInfo(h->stream, &st, nullptr, &g, nullptr, nullptr, nullptr));
  CK(cudaGraphConditionalHandleCreate(hc, g, 1u, cudaGraphCondAssignDefault));
  return SIM_OK;
}

// forces of the current positions.  The rebuild kernels run every time and
// rebuild the lists that are due (a displacement beyond the buffer, the
// longest interval, or a forced request: request = a trial, -1 for all, or
// NO_REQUEST).  Unless kernels are being timed one by one, the bonded forces
// and the reaction coordinate (CV and its finaliser) run on a second stream
// once the atoms have their slots (they read positions through slot_of) and
// join before anything that follows: the list build and the pair kernel write
// nothing they read, and pair and bonded forces meet only in
// order-independent fixed-point sums, so both orders give bit-identical states.
void forces(sim_handle *h, FinMode mode, int request) {
  if (request != NO_REQUEST) launch_rebuild_request(h->d, request, h->stream);
  if (h->skip_empty && h->cap_k >= 0 && request == NO_REQUEST && h->side && !h->timing) {
    // step form 2 inside a captured chunk: the column sort and the list
    // build sit in conditional nodes that the front kernel opens only
    // when a trial rebuilds in this step (the same kernels otherwise)
    cudaGraphConditionalHandle hc[2];
    if (new_conditional(h, &hc[0]) || new_conditional(h, &hc[1])) {
      h->capture_failed = true;
      return;
    }
    launch_front(h->d, h->c, h->half_skin2, h->strict_skin, false, h->stream, hc);
    if (add_conditional(h, hc[0], [&](cudaStream_t cs) {
          launch_colsort(h->d, cs);
        })) {
      h->capture_failed = true;
      return;
    }
    fork_side(h, mode);
    if (add_conditional(h, hc[1], [&](cudaStream_t cs) { launch_list(h->d, h->c, h->rl2_bbox, cs); })) {
      h->capture_failed = true;
      join_side(h);  // the side branches still join the capture
      return;
    }
    pair_forces(h);
    join_side(h);
    after_forces(h, mode);
    return;
  }
  rebuild_cols(h, request != NO_REQUEST);
  if (h->side && !h->timing) {
    fork_side(h, mode);
    rebuild_list(h);
    pair_forces(h);
    join_side(h);
  } else {
    rebuild_list(h);
    pair_forces(h);
    cv_forces(h, mode, h->stream);
  }
  after_forces(h, mode);
}

void one_step(sim_handle *h) {
  if (h->fused) {
    timed(h, "step_fused",
          [&] { launch_step_fused(h->d, h->c, h->rl2_bbox, h->half_skin2, h->strict_skin, h->stream); });
    after_forces(h, FIN_STEP);
    return;
  }
  timed(h, "update", [&] { launch_update(h->d, h->c, UPD_DRIFT, h->stream); });
  forces(h, FIN_STEP, NO_REQUEST);
}

int check_flags(sim_handle *h) {
  int flags = 0;
  CK(cudaMemcpyAsync(&flags, h->d.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (flags & ERR_NONFINITE)
    return fail(h, SIM_ENONFINITE,
                "non-finite position, velocity or reaction coordinate, a force beyond 2^30 kJ/mol/nm or an atom "
                "faster than a box per step");
  if (flags & (ERR_LIST | ERR_COL | ERR_CAPACITY))
    return fail(h, SIM_ELIST_OVERFLOW, "cluster list, grid column or cluster capacity exceeded");
  if (flags & ERR_SKIN)
    return fail(h, SIM_ESKIN, "an atom moved more than skin/2 between fixed-interval list rebuilds");
  if (flags & ERR_TIMEOUT) {
    // the barrier is left half counted: start it afresh for the next launch
    CK(cudaMemsetAsync(h->d.bar, 0, 2 * sizeof(unsigned), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return fail(h, SIM_ETIMEOUT, "a grid barrier of the one-kernel step gave up waiting (the step is incomplete)");
  }
  return SIM_OK;
}

int enter(sim_handle *h) {
  if (!h) return SIM_EINVAL;
  CK(cudaSetDevice(h->device));
  if (h->caller) {
    CK(cudaEventRecord(h->entry_ev, h->caller));
    CK(cudaStreamWaitEvent(h->stream, h->entry_ev, 0));
  }
  return SIM_OK;
}

int ensure_dbuf(sim_handle *h, size_t n) {
  if (h->dbuf_n >= n) return SIM_OK;
  if (h->dbuf) cudaFree(h->dbuf);
  h->dbuf = nullptr;
  cudaError_t e = cudaMalloc(&h->dbuf, n * sizeof(double));
  if (e != cudaSuccess) return fail(h, SIM_ECUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->dbuf_n = n;
  return SIM_OK;
}

int capture_chunk(sim_handle *h) {
  if (h->chunk) return SIM_OK;
  cudaGraph_t g;
  if (h->gtiming && h->gev.empty()) {
    h->gev.resize(2 * (size_t)h->params.nstlist);
    for (auto &e : h->gev) CK(cudaEventCreate(&e));
  }
  // the chunk is nst steps; every step decides on the device which lists
  // to rebuild, so a chunk replays from any step
  const int nst = h->params.nstlist;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  h->capture_failed = false;
  for (int k = 0; k < nst; ++k) {
    h->cap_k = k;
    one_step(h);
  }
  h->cap_k = -1;
  CK(cudaStreamEndCapture(h->stream, &g));
  if (h->capture_failed) {
    cudaGraphDestroy(g);
    const std::string why = h->err;
    return fail(h, SIM_ECUDA, "a conditional graph node could not be captured: " + why);
  }
  cudaError_t e = cudaGraphInstantiate(&h->chunk, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->chunk = nullptr;
    return fail(h, SIM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  return SIM_OK;
}

// validation of one system description
std::string check_system(const sim_system &s, const sim_params &p) {
  if (s.n_atoms < 1) return "n_atoms < 1";
  if (s.n_solute < 0 || s.n_solute > s.n_atoms) return "n_solute out of range";
  if (s.n_cv < 0 || s.n_cv > s.n_solute) return "n_cv out of range";
  if (!s.pos || !s.mass || !s.charge || !s.lj_type || !s.sigma || !s.epsilon) return "missing atom arrays";
  if (s.n_cv > 0 && !s.native_pos) return "missing native_pos";
  if (s.n_types < 1) return "n_types < 1";
  double rl = p.r_cut + p.skin;
  if (!(s.box > 2.0 * rl)) return "box must exceed 2 (r_cut + skin)";
  if (!(s.box < 60.0)) return "box must be below 60 nm";
  for (int i = 0; i < s.n_atoms; ++i) {
    if (!(s.mass[i] > 0.0)) return "non-positive mass";
    if (s.lj_type[i] < 0 || s.lj_type[i] >= s.n_types) return "lj_type out of range";
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(s.pos[3 * i + k])) return "non-finite position";
  }
  for (int b = 0; b < s.n_bonds; ++b)
    for (int k = 0; k < 2; ++k)
      if (s.bonds[2 * b + k] < 0 || s.bonds[2 * b + k] >= s.n_atoms) return "bond index out of range";
  for (int a = 0; a < s.n_angles; ++a)
    for (int k = 0; k < 3; ++k)
      if (s.angles[3 * a + k] < 0 || s.angles[3 * a + k] >= s.n_atoms) return "angle index out of range";
  for (int x = 0; x < s.n_excl; ++x)
    for (int k = 0; k < 2; ++k)
      if (s.excl[2 * x + k] < 0 || s.excl[2 * x + k] >= s.n_atoms) return "exclusion index out of range";
  return "";
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

VP_API int sim_create(const sim_system *systems, int32_t n_systems, const int32_t *trials_per_system,
                      const uint64_t *trial_seeds, const sim_params *params, void *cuda_stream, sim_handle **out) {
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  if (!systems || n_systems < 1 || !trials_per_system || !params) return SIM_EINVAL;
  sim_handle *h = new sim_handle();
  auto bail = [&](int code) {
    *out = h;  // keep the handle so that sim_last_error works; caller destroys it
    return code;
  };
  const sim_params &p = *params;
  h->params = p;
  if (!(p.dt > 0) || !(p.temperature >= 0) || !(p.r_cut > 0) || !(p.skin >= 0) || p.nstlist < 1 ||
      !(p.cv_r0 > 0) || !(p.cv_r_cut > p.cv_r_switch) || !(p.cv_r_switch > 0) || p.cv_min_sep < 0)
    return bail(fail(h, SIM_EINVAL, "invalid sim_params"));
  int total_trials = 0;
  for (int s = 0; s < n_systems; ++s) {
    if (trials_per_system[s] < 0) return bail(fail(h, SIM_EINVAL, "negative trial count"));
    if (trials_per_system[s] > MAX_TRIALS || total_trials + trials_per_system[s] > MAX_TRIALS)
      return bail(fail(h, SIM_EINVAL, "more than 65535 trials in one batch"));
    std::string m = check_system(systems[s], p);
    if (!m.empty()) return bail(fail(h, SIM_EINVAL, "system " + std::to_string(s) + ": " + m));
    total_trials += trials_per_system[s];
  }
  if (total_trials < 1) return bail(fail(h, SIM_EINVAL, "no trials"));
  cudaError_t ce = cudaGetDevice(&h->device);
  if (ce != cudaSuccess) return bail(fail(h, SIM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce)));
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(h, SIM_ECUDA, "cudaStreamCreate failed"));
  cudaEventCreateWithFlags(&h->entry_ev, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&h->exit_ev, cudaEventDisableTiming);
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->bstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_bjoin, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(h, SIM_ECUDA, "cudaStreamCreate / cudaEventCreate failed"));
  h->caller = (cudaStream_t)cuda_stream;
  h->n_sys = n_systems;
  h->n_trials = total_trials;
  h->use_graph = !(p.flags & SIM_NO_GRAPH);
  h->strict_skin = (p.flags & SIM_STRICT_SKIN) ? 1 : 0;
  if (h->strict_skin && !(p.flags & SIM_FIXED_INTERVAL))
    return bail(fail(h, SIM_EINVAL, "SIM_STRICT_SKIN applies to fixed-interval lists (SIM_FIXED_INTERVAL)"));

  // ---- constants -------------------------------------------------------------
  const double kT = KB * p.temperature;
  const double rl = p.r_cut + p.skin;
  SimConst &c = h->c;
  c.dt = (float)p.dt;
  c.half_dt = (float)(0.5 * p.dt);
  c.dt_d = p.dt;
  c.rc2 = (float)(p.r_cut * p.r_cut);
  c.rl2 = (float)(rl * rl);
  double krf, crf;
  if (p.eps_rf <= 0.0) {
    krf = 1.0 / (2.0 * p.r_cut * p.r_cut * p.r_cut);
    crf = 3.0 / (2.0 * p.r_cut);
  } else {
    krf = (p.eps_rf - 1.0) / ((2.0 * p.eps_rf + 1.0) * p.r_cut * p.r_cut * p.r_cut);
    crf = 1.0 / p.r_cut + krf * p.r_cut * p.r_cut;
  }
  c.krf = (float)krf;
  c.crf = (float)crf;
  c.two_krf = (float)(2.0 * krf);
  c.kR_half = (float)(0.5 * p.k_ratchet);
  c.kR_half_d = 0.5 * p.k_ratchet;
  c.list_cap = LIST_CAP;
  // debug knob (fault injection): a smaller list capacity, 8..LIST_CAP j-atom entries per cluster
  if (const char *e = std::getenv("VPATH_LIST_CAP")) {
    const int v = std::atoi(e);
    if (v >= 8 && v <= LIST_CAP) c.list_cap = v;
  }
  ff_split(1.0 / (p.cv_r0 * p.cv_r0), c.cv_inv_r0sq_hi, c.cv_inv_r0sq_lo);
  ff_split(p.cv_r_switch, c.cv_rs_hi, c.cv_rs_lo);
  ff_split(1.0 / (p.cv_r_cut - p.cv_r_switch), c.cv_inv_w_hi, c.cv_inv_w_lo);
  c.cv_rs2 = (float)(p.cv_r_switch * p.cv_r_switch);
  c.cv_rc2_far = (float)(p.cv_r_cut * p.cv_r_cut * (1.0 + 1e-4));
  c.cv_r0_d = p.cv_r0;
  c.cv_rs_d = p.cv_r_switch;
  c.cv_rc_d = p.cv_r_cut;
  c.cv_min_sep = p.cv_min_sep;
  c.rec_cap = 0;
  // one friction for every atom: the Langevin coefficients need no per-atom table
  {
    bool uni = true;
    for (int s = 0; s < n_systems && uni; ++s)
      if (systems[s].gamma)
        for (int i = 0; i < systems[s].n_atoms; ++i)
          if (systems[s].gamma[i] != p.gamma) { uni = false; break; }
    const double c1u = std::exp(-p.gamma * p.dt);
    c.uniform_gamma = uni ? 1 : 0;
    c.c1_u = (float)c1u;
    c.c2sqkT_u = (float)std::sqrt((1.0 - c1u * c1u) * kT);
  }
  h->rl2_bbox = (float)((rl + 1e-3) * (rl + 1e-3));
  h->half_skin2 = (float)(0.25 * p.skin * p.skin);
  c.nstlist = p.nstlist;
  c.list_fixed = (p.flags & SIM_FIXED_INTERVAL) ? 1 : 0;
  // bounded grid barriers of the one-kernel step: 2^20 polls of >= 64 ns; the
  // debug variable VPATH_SPIN_LIMIT sets another bound (a test makes it run
  // out with a tiny one)
  c.spin_limit = 1u << 20;
  if (const char *e = std::getenv("VPATH_SPIN_LIMIT")) c.spin_limit = (uint32_t)std::strtoul(e, nullptr, 10);
  {
    const double trig = std::max(0.0, 0.5 * p.skin - 1e-5);  // 1e-5 nm cover FP32 rounding
    c.trig2 = (float)(trig * trig);
  }

  // ---- LJ types: de-duplicate (sigma, epsilon) over all systems -------------
  std::vector<std::pair<double, double>> gtypes;
  std::vector<std::vector<int>> tmap(n_systems);
  for (int s = 0; s < n_systems; ++s) {
    const sim_system &S = systems[s];
    tmap[s].resize(S.n_types);
    for (int k = 0; k < S.n_types; ++k) {
      std::pair<double, double> key(S.sigma[k], S.epsilon[k]);
      int g = -1;
      for (size_t q = 0; q < gtypes.size(); ++q)
        if (gtypes[q] == key) { g = (int)q; break; }
      if (g < 0) {
        g = (int)gtypes.size();
        gtypes.push_back(key);
      }
      tmap[s][k] = g;
    }
  }
  if ((int)gtypes.size() > MAX_TYPES) return bail(fail(h, SIM_EINVAL, "more than 64 distinct LJ types"));
  const int NT = (int)gtypes.size();
  c.n_types = NT;
  std::vector<float2> ljtab(NT * NT);
  std::vector<float> ljshift(NT * NT);
  for (int a = 0; a < NT; ++a)
    for (int b = 0; b < NT; ++b) {
      double sig = 0.5 * (gtypes[a].first + gtypes[b].first);
      double eps = std::sqrt(gtypes[a].second * gtypes[b].second);
      double s6 = std::pow(sig, 6.0);
      double c6 = 4.0 * eps * s6, c12 = 4.0 * eps * s6 * s6;
      if (!(eps > 0.0 && sig > 0.0)) c6 = c12 = 0.0;
      ljtab[a * NT + b] = make_float2((float)(6.0 * c6), (float)(12.0 * c12));
      double rc6 = std::pow(p.r_cut, 6.0);
      ljshift[a * NT + b] = (float)(c12 / (rc6 * rc6) - c6 / rc6);
    }

  // ---- per-system tables ------------------------------------------------------
  std::vector<int> sysatom0(n_systems + 1, 0);
  for (int s = 0; s < n_systems; ++s) sysatom0[s + 1] = sysatom0[s] + systems[s].n_atoms;
  const int total_sys_atoms = sysatom0[n_systems];
  std::vector<AtomSys> asys(total_sys_atoms);
  std::vector<double> gm(total_sys_atoms);
  std::vector<int32_t> excl((size_t)total_sys_atoms * MAX_EXCL, -1), excl_n(total_sys_atoms, 0);
  std::vector<int32_t> bt_start(total_sys_atoms + 1, 0);
  std::vector<BTerm> bterm;
  std::vector<BGroup> bgrp;
  std::vector<int32_t> sys_bg0(n_systems), sys_nbg(n_systems);
  std::vector<int2> tiles;
  std::vector<int32_t> sys_tile0(n_systems), sys_ntiles(n_systems), sys_ncv(n_systems), sys_minsep(n_systems),
      tile_sys, sys_nat0(n_systems);
  std::vector<double> native_all;
  const double sqf = std::sqrt(FCOUL);
  for (int s = 0; s < n_systems; ++s) {
    const sim_system &S = systems[s];
    const int a0 = sysatom0[s];
    for (int i = 0; i < S.n_atoms; ++i) {
      double g = S.gamma ? S.gamma[i] : p.gamma;
      double c1 = std::exp(-g * p.dt);
      asys[a0 + i].invm = (float)(1.0 / S.mass[i]);
      asys[a0 + i].c1 = (float)c1;
      asys[a0 + i].c2sd = (float)std::sqrt((1.0 - c1 * c1) * kT / S.mass[i]);
      asys[a0 + i].qs = (float)(S.charge[i] * sqf);
      gm[a0 + i] = g > 0.0 ? g * S.mass[i] : INFINITY;  // no friction: no bias weight (k_R must be 0)
      if (i < S.n_cv && !(g > 0.0) && p.k_ratchet != 0.0)
        return bail(fail(h, SIM_EINVAL, "reaction-coordinate atoms need gamma > 0 when k_ratchet != 0"));
    }
    // exclusions: 1-2, 1-3 and the extra pairs
    auto add_ex = [&](int i, int j) -> bool {
      if (i == j) return true;
      int *e = &excl[(size_t)(a0 + i) * MAX_EXCL];
      int &n = excl_n[a0 + i];
      for (int k = 0; k < n; ++k)
        if (e[k] == j) return true;
      if (n >= MAX_EXCL) return false;
      e[n++] = j;
      return true;
    };
    bool ok = true;
    for (int b = 0; b < S.n_bonds; ++b) {
      int i = S.bonds[2 * b], j = S.bonds[2 * b + 1];
      ok &= add_ex(i, j) && add_ex(j, i);
    }
    for (int a = 0; a < S.n_angles; ++a) {
      int i = S.angles[3 * a], j = S.angles[3 * a + 1], k = S.angles[3 * a + 2];
      ok &= add_ex(i, j) && add_ex(j, i) && add_ex(j, k) && add_ex(k, j) && add_ex(i, k) && add_ex(k, i);
    }
    for (int x = 0; x < S.n_excl; ++x) {
      int i = S.excl[2 * x], j = S.excl[2 * x + 1];
      ok &= add_ex(i, j) && add_ex(j, i);
    }
    if (!ok) return bail(fail(h, SIM_EINVAL, "more than 16 excluded partners for an atom"));
    // bonded terms per owning atom (the energy kernel computes each atom's share)
    std::vector<std::vector<BTerm>> per(S.n_atoms);
    for (int b = 0; b < S.n_bonds; ++b) {
      int i = S.bonds[2 * b], j = S.bonds[2 * b + 1];
      per[i].push_back(BTerm{0, j, -1, (float)S.bond_r0[b], (float)S.bond_k[b]});
      per[j].push_back(BTerm{0, i, -1, (float)S.bond_r0[b], (float)S.bond_k[b]});
    }
    for (int a = 0; a < S.n_angles; ++a) {
      int i = S.angles[3 * a], j = S.angles[3 * a + 1], k = S.angles[3 * a + 2];
      float t0 = (float)S.angle_t0[a], kk = (float)S.angle_k[a];
      per[i].push_back(BTerm{1, j, k, t0, kk});
      per[k].push_back(BTerm{1, j, i, t0, kk});
      per[j].push_back(BTerm{2, i, k, t0, kk});
    }
    for (int i = 0; i < S.n_atoms; ++i) {
      bt_start[a0 + i] = (int)bterm.size();
      for (auto &t : per[i]) bterm.push_back(t);
    }
    // the same terms once each, for the force kernel, grouped: every angle
    // opens a group of its three atoms; a bond joins the first group that
    // holds both its atoms, else one it can extend to three atoms, else opens
    // a group of its own (a water: its angle and both bonds in one group)
    sys_bg0[s] = (int)bgrp.size();
    {
      std::vector<std::vector<int>> of_atom(S.n_atoms);  // groups (local index) that hold an atom
      std::vector<BGroup> G;
      auto local = [](const BGroup &g, int atom) {
        for (int m = 0; m < 3; ++m)
          if (g.at[m] == atom) return m;
        return -1;
      };
      for (int a = 0; a < S.n_angles; ++a) {
        BGroup g{};
        g.at[0] = S.angles[3 * a]; g.at[1] = S.angles[3 * a + 1]; g.at[2] = S.angles[3 * a + 2];
        g.n = 1;
        g.code[0] = 1 | (0 << 1) | (1 << 3) | (2 << 5);
        g.par[0] = make_float4((float)S.angle_t0[a], (float)S.angle_k[a], 0.f, 0.f);
        for (int m = 0; m < 3; ++m) of_atom[g.at[m]].push_back((int)G.size());
        G.push_back(g);
      }
      for (int b = 0; b < S.n_bonds; ++b) {
        const int i = S.bonds[2 * b], j = S.bonds[2 * b + 1];
        int gi = -1;
        for (int q : of_atom[i])
          if (G[q].n < 3 && local(G[q], j) >= 0) { gi = q; break; }
        if (gi < 0)
          for (int atom : {i, j}) {
            for (int q : of_atom[atom])
              if (G[q].n < 3 && G[q].at[2] < 0) { gi = q; break; }
            if (gi >= 0) break;
          }
        if (gi < 0) {
          BGroup g{};
          g.at[0] = i; g.at[1] = j; g.at[2] = -1;
          gi = (int)G.size();
          G.push_back(g);
          of_atom[i].push_back(gi);
          of_atom[j].push_back(gi);
        }
        BGroup &g = G[gi];
        for (int atom : {i, j})
          if (local(g, atom) < 0) {  // the third atom of a two-atom group
            g.at[2] = atom;
            of_atom[atom].push_back(gi);
          }
        g.code[g.n] = 0 | (local(g, i) << 1) | (local(g, j) << 3);
        const float r0 = (float)S.bond_r0[b];
        g.par[g.n] = make_float4(r0, (float)S.bond_k[b], (float)(S.bond_r0[b] - (double)r0), 0.f);
        g.n += 1;
      }
      for (auto &g : G) bgrp.push_back(g);
    }
    sys_nbg[s] = (int)bgrp.size() - sys_bg0[s];
    // reaction-coordinate tiles
    sys_ncv[s] = S.n_cv;
    sys_minsep[s] = p.cv_min_sep;
    sys_tile0[s] = (int)tiles.size();
    sys_nat0[s] = (int)(native_all.size() / 3);
    for (int i = 0; i < 3 * S.n_cv; ++i) native_all.push_back(S.native_pos[i]);
    int nb = (S.n_cv + CV_T - 1) / CV_T;
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = bi; bj < nb; ++bj) {
        int maxj = std::min(bj * CV_T + CV_T - 1, S.n_cv - 1);
        if (maxj - bi * CV_T > p.cv_min_sep) {
          tiles.push_back(make_int2(bi, bj));
          tile_sys.push_back(s);
        }
      }
    sys_ntiles[s] = (int)tiles.size() - sys_tile0[s];
  }
  bt_start[total_sys_atoms] = (int)bterm.size();

  // ---- per-trial layout ---------------------------------------------------------
  std::vector<int> slot_trial, clus_trial, col_trial;
  std::vector<int2> work;
  int slot0 = 0, col0 = 0, atom0 = 0, cv0 = 0;
  int tcount = 0;
  for (int s = 0; s < n_systems; ++s) {
    const sim_system &S = systems[s];
    const float Lf = (float)S.box;
    const double L = (double)Lf;
    const double rho = S.n_atoms / (L * L * L);
    int ncol = (int)std::lround(L / std::cbrt((double)CL / rho));
    ncol = std::max(1, std::min(ncol, 64));
    for (int r = 0; r < trials_per_system[s]; ++r, ++tcount) {
      TrialInfo T{};
      T.sys = s;
      T.atom0 = atom0;
      T.sysatom0 = sysatom0[s];
      T.n_atoms = S.n_atoms;
      T.n_cv = S.n_cv;
      T.slot0 = slot0;
      T.clus0 = slot0 / CL;
      T.max_clus = (S.n_atoms + (CL - 1) * ncol * ncol + CL - 1) / CL + 1;
      T.ncol = ncol;
      T.col0 = col0;
      T.cv0 = cv0;
      T.work0 = (int)work.size();
      T.n_work = sys_ntiles[s];
      T.systile0 = sys_tile0[s];
      T.box = Lf;
      T.inv_box = (float)(1.0 / L);
      T.col_w = (float)(L / ncol);
      T.inv_col_w = (float)(ncol / L);
      uint64_t seed = trial_seeds ? trial_seeds[tcount] : p.seed + (uint64_t)tcount;
      T.key0 = (uint32_t)seed;
      T.key1 = (uint32_t)(seed >> 32);
      for (int k = 0; k < sys_ntiles[s]; ++k) work.push_back(make_int2(tcount, sys_tile0[s] + k));
      for (int k = 0; k < T.max_clus * CL; ++k) slot_trial.push_back(tcount);
      for (int k = 0; k < T.max_clus; ++k) clus_trial.push_back(tcount);
      for (int k = 0; k < ncol * ncol; ++k) col_trial.push_back(tcount);
      h->tinfo.push_back(T);
      h->trial_sys.push_back(s);
      slot0 += T.max_clus * CL;
      col0 += ncol * ncol;
      atom0 += S.n_atoms;
      cv0 += S.n_cv;
      h->max_atoms = std::max(h->max_atoms, S.n_atoms);
    }
  }
  Dev &d = h->d;
  if ((long long)slot0 + CJ >= (1LL << J_BITS))
    return bail(fail(h, SIM_EINVAL, "batch too large: list entries address at most 2^25 atom slots"));
  d.n_trials = total_trials;
  d.n_sys = n_systems;
  d.total_slots = slot0;
  d.total_clus = slot0 / CL;
  d.total_cols = col0;
  d.total_work = (int)work.size();
  const int total_atoms = atom0, total_cv = cv0;

  // ---- initial slot contents (caller order, padded; the idle half cluster past the end) ----
  std::vector<float4> pos(slot0 + CJ), vel(slot0);
  for (int k = 0; k < slot0; ++k) pos[k] = pad_pos(k);
  for (int k = slot0; k < slot0 + CJ; ++k) pos[k] = idle_pos();
  d.idle_entry = (uint32_t)slot0 | (NO_SHIFT << J_BITS);
  std::vector<int32_t> orig(slot0, -1), type(slot0 + CJ, 0), slot_of(total_atoms > 0 ? total_atoms : 1);
  std::vector<TrialState> tstate(total_trials);
  std::vector<int32_t> need_vel(total_trials, 0);
  for (int t = 0; t < total_trials; ++t) {
    const TrialInfo &T = h->tinfo[t];
    const sim_system &S = systems[T.sys];
    for (int o = 0; o < S.n_atoms; ++o) {
      int sl = T.slot0 + o;
      float4 pp = make_float4((float)S.pos[3 * o], (float)S.pos[3 * o + 1], (float)S.pos[3 * o + 2],
                              asys[T.sysatom0 + o].qs);
      pos[sl] = pp;
      vel[sl] = make_float4(S.vel ? (float)S.vel[3 * o] : 0.f, S.vel ? (float)S.vel[3 * o + 1] : 0.f,
                            S.vel ? (float)S.vel[3 * o + 2] : 0.f, asys[T.sysatom0 + o].invm);
      orig[sl] = o;
      type[sl] = tmap[T.sys][S.lj_type[o]];
      slot_of[T.atom0 + o] = sl;
    }
    tstate[t].n_clus = (S.n_atoms + CL - 1) / CL;
    need_vel[t] = S.vel ? 0 : 1;
  }

  // ---- device allocation and upload ---------------------------------------------
  int r = 0;
  std::vector<int32_t> ncv_v(sys_ncv), ms_v(sys_minsep);
  r |= upload(h, &d.tinfo, h->tinfo);
  r |= upload(h, &d.tstate, tstate);
  r |= upload(h, &d.pos, pos);
  r |= upload(h, &d.vel, vel);
  r |= dalloc(h, &d.pos_b, slot0);
  r |= dalloc(h, &d.vel_b, slot0);
  r |= upload(h, &d.orig, orig);
  r |= upload(h, &d.type, type);
  r |= dalloc(h, &d.orig_b, slot0);
  r |= dalloc(h, &d.type_b, slot0);
  r |= upload(h, &d.slot_trial, slot_trial);
  r |= dalloc(h, &d.slot_col, slot0);
  r |= dalloc(h, &d.fx, slot0 + CJ);
  r |= dalloc(h, &d.fy, slot0 + CJ);
  r |= dalloc(h, &d.fz, slot0 + CJ);
  r |= upload(h, &d.clus_trial, clus_trial);
  r |= dalloc(h, &d.bb_lo, 2 * (size_t)d.total_clus);  // per 4-atom half cluster
  r |= dalloc(h, &d.bb_hi, 2 * (size_t)d.total_clus);
  r |= dalloc(h, &d.list, (size_t)d.total_clus * c.list_cap);
  r |= dalloc(h, &d.list_m, (size_t)d.total_clus * c.list_cap);
  r |= dalloc(h, &d.list_n, d.total_clus);
  r |= dalloc(h, &d.list_nm, d.total_clus);
  r |= upload(h, &d.col_trial, col_trial);
  r |= dalloc(h, &d.col_count, col0);
  r |= dalloc(h, &d.col_start, col0);
  r |= dalloc(h, &d.col_cstart, col0);
  r |= dalloc(h, &d.col_fill, col0);
  r |= dalloc(h, &d.col_ztab, (size_t)col0 * (ZBINS + 1));
  r |= dalloc(h, &d.bucket, total_atoms);
  r |= upload(h, &d.slot_of, slot_of);
  r |= dalloc(h, &d.ref_slot, slot0);
  r |= dalloc(h, &d.gx, total_cv);
  r |= dalloc(h, &d.gy, total_cv);
  r |= dalloc(h, &d.gz, total_cv);
  r |= dalloc(h, &d.z_part, work.size());
  r |= upload(h, &d.asys, asys);
  r |= upload(h, &d.gm, gm);
  {
    std::vector<double> igm(gm.size());
    for (size_t k = 0; k < gm.size(); ++k) igm[k] = std::isfinite(gm[k]) ? 1.0 / gm[k] : 0.0;
    r |= upload(h, &d.inv_gm, igm);
  }
  r |= upload(h, &d.excl, excl);
  r |= upload(h, &d.excl_n, excl_n);
  r |= upload(h, &d.bt_start, bt_start);
  r |= upload(h, &d.bterm, bterm);
  r |= upload(h, &d.bgrp, bgrp);
  r |= upload(h, &d.sys_bg0, sys_bg0);
  r |= upload(h, &d.sys_nbg, sys_nbg);
  d.max_nbg = sys_nbg.empty() ? 0 : *std::max_element(sys_nbg.begin(), sys_nbg.end());
  r |= upload(h, &d.tiles, tiles);
  r |= upload(h, &d.work, work);
  {
    // tiles close to the diagonal hold the pairs close in sequence, which are
    // mostly near pairs: they run first so that the long ones do not trail
    std::vector<int32_t> order(work.size());
    for (size_t k = 0; k < work.size(); ++k) order[k] = (int32_t)k;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      const int2 ta = tiles[work[a].y], tb = tiles[work[b].y];
      return ta.y - ta.x < tb.y - tb.x;
    });
    r |= upload(h, &d.work_order, order);
  }
  r |= dalloc(h, &d.cnat, tiles.size() * CV_T * CV_T);
  r |= dalloc(h, &d.cnat_ff, tiles.size() * CV_T * CV_T);
  r |= upload(h, &d.sys_ncv, ncv_v);
  r |= upload(h, &d.sys_minsep, ms_v);
  r |= upload(h, &d.ljtab, ljtab);
  r |= upload(h, &d.ljshift, ljshift);
  r |= dalloc(h, &d.err, 1);
  r |= dalloc(h, &d.step, 1);
  r |= dalloc(h, &d.kick, 1);
  r |= dalloc(h, &d.done, 1);
  r |= dalloc(h, &d.energy, (size_t)total_trials * 5);
  r |= dalloc(h, &d.diag, 4);
  r |= dalloc(h, &d.cur_step, 1);
  r |= dalloc(h, &d.rb, 2 * (size_t)total_trials);
  r |= dalloc(h, &d.last_rb, total_trials);
  r |= dalloc(h, &d.rb_list, total_trials);
  r |= dalloc(h, &d.rb_cnt, 4);
  for (const auto &T : h->tinfo) {
    d.max_trial_slots = std::max(d.max_trial_slots, T.max_clus * CL);
    d.max_trial_clus = std::max(d.max_trial_clus, T.max_clus);
    d.max_trial_cols = std::max(d.max_trial_cols, T.ncol * T.ncol);
  }
  r |= dalloc(h, &h->d_argmin, 1);
  r |= dalloc(h, &h->d_count, 1);
  r |= dalloc(h, &h->d_flag, 1);
  r |= dalloc(h, &d.pair_next, 3);
  r |= dalloc(h, &d.bar, 2);
  {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    d.n_sm = nsm > 0 ? nsm : 1;
  }
  if (r) return bail(SIM_ECUDA);
  float half = 0.5f;
  if (cudaMemcpy(d.kick, &half, sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(h, SIM_ECUDA, "cudaMemcpy kick"));
  // no rebuild requested for any step yet (a step number's low 32 bits never
  // equal this value within 2^32 steps of creation)
  if (cudaMemset(d.rb, 0xff, 2 * sizeof(uint32_t) * (size_t)total_trials) != cudaSuccess)
    return bail(fail(h, SIM_ECUDA, "cudaMemset rebuild requests"));

  // ---- native contact map, velocities, first lists and forces -------------------------
  int32_t *d_need = nullptr, *d_nat0 = nullptr, *d_tsys = nullptr, *d_st0 = nullptr, *d_snt = nullptr;
  double *d_native = nullptr;
  r |= upload(h, &d_need, need_vel);
  r |= upload(h, &d_native, native_all);
  h->native_all = native_all;
  h->sys_nat0 = sys_nat0;
  h->sys_ncv = sys_ncv;
  h->sys_minsep = sys_minsep;
  r |= upload(h, &d_nat0, sys_nat0);
  r |= upload(h, &d_tsys, tile_sys);
  r |= upload(h, &d_st0, sys_tile0);
  r |= upload(h, &d_snt, sys_ntiles);
  if (r) return bail(SIM_ECUDA);
  cudaStream_t st = h->stream;
  launch_cnat(d, c, d_native, d_nat0, (int)tiles.size(), d_tsys, st);
  launch_zconst(d, d_st0, d_snt, st);
  launch_init_vel(d, (float)kT, d_need, st);
  forces(h, FIN_INIT, -1);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return bail(fail(h, SIM_ECUDA, std::string("initialisation kernels failed: ") +
                                       cudaGetErrorString(cudaGetLastError())));
  int fr = check_flags(h);
  if (fr) return bail(fr);
  *out = h;
  return SIM_OK;
}

VP_API int sim_step_batch(sim_handle *h, int32_t n_steps) {
  int r = enter(h);
  if (r) return r;
  if (n_steps < 0) return fail(h, SIM_EINVAL, "n_steps < 0");
  if (n_steps == 0) return SIM_OK;
  CK(cudaMemsetAsync(h->d.err, 0, sizeof(int), h->stream));
  const int nst = h->params.nstlist;
  int left = n_steps;
  bool pending = false;  // a replay whose in-graph timing events are not read yet
  while (left > 0) {
    if (h->use_graph && !h->timing && left >= nst && !(h->fused && h->fused_no_graph)) {
      r = capture_chunk(h);
      if (r && h->fused) {
        // the cooperative step kernel could not be captured: launch it directly from now on
        cudaGetLastError();
        h->fused_no_graph = true;
        continue;
      }
      if (r) return r;
      if (pending) {  // read the previous replay's events before this one records them again
        CK(cudaStreamSynchronize(h->stream));
        r = harvest_graph_timers(h);
        if (r) return r;
      }
      CK(cudaGraphLaunch(h->chunk, h->stream));
      h->step += nst;
      left -= nst;
      pending = h->gtiming && !h->fused;  // the one-kernel step has no separate pair launch to time
    } else {
      one_step(h);
      h->step += 1;
      left -= 1;
    }
  }
  timed(h, "update_final", [&] { launch_update(h->d, h->c, UPD_FINAL, h->stream); });
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) harvest_timers(h);
  if (pending) {
    r = harvest_graph_timers(h);
    if (r) return r;
  }
  return check_flags(h);
}

VP_API int bias_functional(sim_handle *h, double z_max, double *phi, int32_t *argmin) {
  int r = enter(h);
  if (r) return r;
  r = ensure_dbuf(h, (size_t)h->n_trials);
  if (r) return r;
  launch_select(h->d, z_max, h->dbuf, h->d_argmin, h->stream);
  int32_t am = -1;
  std::vector<double> tmp(h->n_trials);
  CK(cudaMemcpyAsync(tmp.data(), h->dbuf, sizeof(double) * h->n_trials, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&am, h->d_argmin, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (phi) std::memcpy(phi, tmp.data(), sizeof(double) * h->n_trials);
  if (argmin) *argmin = am;
  return SIM_OK;
}

VP_API int energy_forces(sim_handle *h, int32_t trial, double *energies, double *forces_out) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials) return fail(h, SIM_EINVAL, "trial out of range");
  const TrialInfo &T = h->tinfo[trial];
  if (energies) {
    CK(cudaMemsetAsync(h->d.energy + (size_t)trial * 5, 0, 5 * sizeof(long long), h->stream));
    launch_pair(h->d, h->c, true, trial, h->stream);
    launch_kinetic(h->d, trial, h->stream);
    long long e[5];
    TrialState S;
    CK(cudaMemcpyAsync(e, h->d.energy + (size_t)trial * 5, sizeof(e), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&S, h->d.tstate + trial, sizeof(S), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 5; ++k) energies[k] = (double)e[k] / E_SCALE;
    energies[5] = 0.5 * h->c.kR_half_d * S.a * S.a;
  }
  if (forces_out) {
    r = ensure_dbuf(h, (size_t)3 * T.n_atoms);
    if (r) return r;
    launch_forces_out(h->d, h->c, trial, h->dbuf, T.n_atoms, h->stream);
    CK(cudaMemcpyAsync(forces_out, h->dbuf, sizeof(double) * 3 * T.n_atoms, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  CK(cudaGetLastError());
  return SIM_OK;
}

VP_API int sim_get_state(sim_handle *h, int32_t trial, double *pos, double *vel, double *cv) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials) return fail(h, SIM_EINVAL, "trial out of range");
  const TrialInfo &T = h->tinfo[trial];
  const size_t n3 = (size_t)3 * T.n_atoms;
  r = ensure_dbuf(h, 2 * n3);
  if (r) return r;
  launch_gather_state(h->d, trial, h->dbuf, h->dbuf + n3, T.n_atoms, h->stream);
  if (pos) CK(cudaMemcpyAsync(pos, h->dbuf, sizeof(double) * n3, cudaMemcpyDeviceToHost, h->stream));
  if (vel) CK(cudaMemcpyAsync(vel, h->dbuf + n3, sizeof(double) * n3, cudaMemcpyDeviceToHost, h->stream));
  TrialState S;
  CK(cudaMemcpyAsync(&S, h->d.tstate + trial, sizeof(S), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (cv) { cv[0] = S.z; cv[1] = S.zm; cv[2] = S.a; cv[3] = S.Phi; }
  return SIM_OK;
}

VP_API int sim_set_state(sim_handle *h, int32_t trial, const double *pos, const double *vel, const double *cv_state) {
  int r = enter(h);
  if (r) return r;
  if (!pos || !vel) return fail(h, SIM_EINVAL, "pos and vel are required");
  if (trial < -1 || trial >= h->n_trials) return fail(h, SIM_EINVAL, "trial out of range");
  int t0 = trial < 0 ? 0 : trial, t1 = trial < 0 ? h->n_trials : trial + 1;
  size_t n = 0;
  for (int t = t0; t < t1; ++t) n += (size_t)h->tinfo[t].n_atoms;
  r = ensure_dbuf(h, 6 * n);
  if (r) return r;
  CK(cudaMemcpyAsync(h->dbuf, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->dbuf + 3 * n, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
  // the state is checked on the device before it replaces the current one
  CK(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
  launch_check_finite(h->dbuf, 6 * n, h->d_flag, h->stream);
  // functional bookkeeping of the affected trials
  std::vector<TrialState> S(h->n_trials);
  int bad = 0;
  CK(cudaMemcpyAsync(S.data(), h->d.tstate, sizeof(TrialState) * h->n_trials, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&bad, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (bad) return fail(h, SIM_EINVAL, "non-finite state");
  launch_scatter_state(h->d, trial, h->dbuf, h->dbuf + 3 * n, (int)n, h->stream);
  for (int t = t0; t < t1; ++t) {
    if (cv_state) {
      S[t].zm = cv_state[2 * (t - t0)];
      S[t].Phi = cv_state[2 * (t - t0) + 1];
    } else {
      S[t].zm = INFINITY;
      S[t].Phi = 0.0;
    }
  }
  CK(cudaMemcpyAsync(h->d.tstate, S.data(), sizeof(TrialState) * h->n_trials, cudaMemcpyHostToDevice, h->stream));
  const Dev &d = h->d;
  CK(cudaMemsetAsync(d.fx, 0, sizeof(long long) * d.total_slots, h->stream));
  CK(cudaMemsetAsync(d.fy, 0, sizeof(long long) * d.total_slots, h->stream));
  CK(cudaMemsetAsync(d.fz, 0, sizeof(long long) * d.total_slots, h->stream));
  size_t ncv = 0;
  for (auto &T : h->tinfo) ncv += T.n_cv;
  if (ncv) {
    CK(cudaMemsetAsync(d.gx, 0, sizeof(long long) * ncv, h->stream));
    CK(cudaMemsetAsync(d.gy, 0, sizeof(long long) * ncv, h->stream));
    CK(cudaMemsetAsync(d.gz, 0, sizeof(long long) * ncv, h->stream));
  }
  CK(cudaMemsetAsync(d.err, 0, sizeof(int), h->stream));
  float half = 0.5f;
  CK(cudaMemcpyAsync(d.kick, &half, sizeof(float), cudaMemcpyHostToDevice, h->stream));
  forces(h, FIN_RESTORE, trial);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return check_flags(h);
}

VP_API int sim_rebuild(sim_handle *h) {
  int r = enter(h);
  if (r) return r;
  const Dev &d = h->d;
  CK(cudaMemsetAsync(d.err, 0, sizeof(int), h->stream));
  CK(cudaMemsetAsync(d.fx, 0, sizeof(long long) * d.total_slots, h->stream));
  CK(cudaMemsetAsync(d.fy, 0, sizeof(long long) * d.total_slots, h->stream));
  CK(cudaMemsetAsync(d.fz, 0, sizeof(long long) * d.total_slots, h->stream));
  size_t ncv = 0;
  for (auto &T : h->tinfo) ncv += T.n_cv;
  if (ncv) {
    CK(cudaMemsetAsync(d.gx, 0, sizeof(long long) * ncv, h->stream));
    CK(cudaMemsetAsync(d.gy, 0, sizeof(long long) * ncv, h->stream));
    CK(cudaMemsetAsync(d.gz, 0, sizeof(long long) * ncv, h->stream));
  }
  forces(h, FIN_KEEP, -1);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return check_flags(h);
}

VP_API int sim_potential_device(sim_handle *h, const double *d_pos, double *d_energy, double *d_forces,
                                void *cuda_stream) {
  if (!h) return SIM_EINVAL;
  if (!d_pos || (!d_energy && !d_forces)) return fail(h, SIM_EINVAL, "d_pos and an output are required");
  CK(cudaSetDevice(h->device));
  cudaStream_t cs = (cudaStream_t)cuda_stream, s = h->stream;
  CK(cudaEventRecord(h->entry_ev, cs));
  CK(cudaStreamWaitEvent(s, h->entry_ev, 0));
  const Dev &d = h->d;
  int n = 0;
  for (const auto &T : h->tinfo) n += T.n_atoms;
  // requests of earlier calls at this step number must not count again
  CK(cudaMemsetAsync(d.rb, 0xff, 2 * sizeof(uint32_t) * (size_t)h->n_trials, s));
  CK(cudaMemsetAsync(d.err, 0, sizeof(int), s));
  CK(cudaMemsetAsync(d.fx, 0, sizeof(long long) * d.total_slots, s));
  CK(cudaMemsetAsync(d.fy, 0, sizeof(long long) * d.total_slots, s));
  CK(cudaMemsetAsync(d.fz, 0, sizeof(long long) * d.total_slots, s));
  CK(cudaMemsetAsync(d.energy, 0, sizeof(long long) * 5 * (size_t)h->n_trials, s));
  launch_scatter_positions(d, h->c, d_pos, n, s);
  rebuild_cols(h, false);
  rebuild_list(h);
  launch_pair_hot(h, d, s);
  launch_bonded(d, s);
  launch_pair(d, h->c, true, -1, s);
  launch_potential_out(d, d_energy, d_forces, n, s);
  CK(cudaGetLastError());
  CK(cudaEventRecord(h->exit_ev, s));
  CK(cudaStreamWaitEvent(cs, h->exit_ev, 0));
  return SIM_OK;
}

VP_API int sim_list_positions(sim_handle *h, int32_t trial, double *pos) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials || !pos) return fail(h, SIM_EINVAL, "trial out of range or pos is NULL");
  const int n = h->tinfo[trial].n_atoms;
  r = ensure_dbuf(h, (size_t)3 * n);
  if (r) return r;
  launch_list_positions(h->d, trial, h->dbuf, n, h->stream);
  CK(cudaMemcpyAsync(pos, h->dbuf, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

VP_API int64_t sim_step_count(const sim_handle *h) { return h ? h->step : -1; }

VP_API int sim_set_step_count(sim_handle *h, int64_t step) {
  int r = enter(h);
  if (r) return r;
  if (step < 0) return fail(h, SIM_EINVAL, "negative step");
  long long s = step;
  CK(cudaMemcpyAsync(h->d.step, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d.cur_step, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->step = step;
  return SIM_OK;
}

VP_API int sim_set_noise_offset(sim_handle *h, int32_t trial, int64_t offset) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials) return fail(h, SIM_EINVAL, "trial out of range");
  h->tinfo[trial].noise_off = offset;
  CK(cudaMemcpyAsync(h->d.tinfo + trial, &h->tinfo[trial], sizeof(TrialInfo), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

VP_API int sim_noise_offset(sim_handle *h, int32_t trial, int64_t *offset) {
  if (!h) return SIM_EINVAL;
  if (trial < 0 || trial >= h->n_trials || !offset) return fail(h, SIM_EINVAL, "trial out of range or offset is NULL");
  *offset = h->tinfo[trial].noise_off;
  return SIM_OK;
}

VP_API int sim_trial_seed(sim_handle *h, int32_t trial, uint64_t *seed) {
  if (!h) return SIM_EINVAL;
  if (trial < 0 || trial >= h->n_trials || !seed) return fail(h, SIM_EINVAL, "trial out of range or seed is NULL");
  *seed = (uint64_t)h->tinfo[trial].key0 | ((uint64_t)h->tinfo[trial].key1 << 32);
  return SIM_OK;
}

VP_API int32_t sim_num_trials(const sim_handle *h) { return h ? h->n_trials : 0; }

VP_API int32_t sim_num_atoms(const sim_handle *h, int32_t trial) {
  if (!h || trial < 0 || trial >= h->n_trials) return 0;
  return h->tinfo[trial].n_atoms;
}

VP_API int sim_record(sim_handle *h, int32_t capacity) {
  int r = enter(h);
  if (r) return r;
  if (capacity < 0) return fail(h, SIM_EINVAL, "negative capacity");
  if (h->d.rec) {
    cudaFree(h->d.rec);
    h->d.rec = nullptr;
  }
  h->rec_cap = capacity;
  h->c.rec_cap = capacity;
  if (h->chunk) {
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  if (capacity > 0) {
    size_t n = (size_t)h->n_trials * capacity * 5;
    CK(cudaMalloc(&h->d.rec, n * sizeof(double)));
    CK(cudaMemset(h->d.rec, 0, n * sizeof(double)));
  }
  return SIM_OK;
}

VP_API int sim_get_record(sim_handle *h, int32_t trial, double *out) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials || !out || h->rec_cap <= 0) return fail(h, SIM_EINVAL, "no record");
  size_t n = (size_t)h->rec_cap * 5;
  CK(cudaMemcpyAsync(out, h->d.rec + (size_t)trial * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

VP_API int sim_record_frames(sim_handle *h, int32_t trial, int32_t capacity) {
  int r = enter(h);
  if (r) return r;
  if (capacity < 0 || (capacity > 0 && (trial < -1 || trial >= h->n_trials)))
    return fail(h, SIM_EINVAL, "bad frame-record arguments");
  if (h->frames) {
    cudaFree(h->frames);
    h->frames = nullptr;
  }
  if (h->chunk) {
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  h->frame_cap = capacity;
  h->frame_trial = capacity > 0 ? trial : -1;
  if (capacity > 0) {
    const size_t nt = trial >= 0 ? 1 : (size_t)h->n_trials;
    size_t n = nt * (size_t)capacity * 3 * (size_t)std::max(1, frame_stride(h));
    CK(cudaMalloc(&h->frames, n * sizeof(float)));
    CK(cudaMemset(h->frames, 0, n * sizeof(float)));
  }
  return SIM_OK;
}

VP_API int sim_frame_shape(sim_handle *h, int32_t *shape) {
  if (!h) return SIM_EINVAL;
  if (!shape) return fail(h, SIM_EINVAL, "shape is NULL");
  shape[0] = h->frames ? (h->frame_trial >= 0 ? 1 : h->n_trials) : 0;
  shape[1] = h->frames ? h->frame_cap : 0;
  shape[2] = h->frames ? frame_stride(h) : 0;
  return SIM_OK;
}

VP_API int sim_get_frames(sim_handle *h, double *out, int64_t out_len) {
  int r = enter(h);
  if (r) return r;
  if (!h->frames || !out) return fail(h, SIM_EINVAL, "no frame record");
  const size_t nt = h->frame_trial >= 0 ? 1 : (size_t)h->n_trials;
  size_t n = nt * (size_t)h->frame_cap * 3 * (size_t)frame_stride(h);
  if (out_len < 0 || (size_t)out_len < n)
    return fail(h, SIM_EINVAL, "output holds " + std::to_string(out_len) + " doubles, the frame record needs " +
                                   std::to_string(n));
  std::vector<float> tmp(n);
  CK(cudaMemcpyAsync(tmp.data(), h->frames, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (size_t k = 0; k < n; ++k) out[k] = tmp[k];
  return SIM_OK;
}

namespace {
AdjInput adj_input(sim_handle *h, int trial) {
  const TrialInfo &T = h->tinfo[trial];
  AdjInput in{};
  in.n_cv = T.n_cv;
  in.min_sep = h->c.cv_min_sep;
  in.n_tiles = T.n_work;
  in.tiles = h->d.tiles + T.systile0;
  in.cnat = h->d.cnat + (size_t)T.systile0 * CV_T * CV_T;
  in.gm = h->d.gm + T.sysatom0;
  in.L = T.box;
  in.iL = T.inv_box;
  const SimConst &c = h->c;
  in.k = CvConst{ff{c.cv_inv_r0sq_hi, c.cv_inv_r0sq_lo}, ff{c.cv_rs_hi, c.cv_rs_lo}, ff{c.cv_inv_w_hi, c.cv_inv_w_lo},
                 c.cv_rs2, c.cv_rc2_far};
  in.c = h->c.dt_d * h->c.kR_half_d * h->c.kR_half_d;
  return in;
}
}  // namespace

VP_API int phi_frames_adjoint(sim_handle *h, int32_t trial, const double *frames, int32_t n_frames, const double *coef,
                              double *phi, double *z, double *grad) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials || n_frames < 1 || !frames) return fail(h, SIM_EINVAL, "bad arguments");
  TrialState S;
  CK(cudaMemcpyAsync(&S, h->d.tstate + trial, sizeof(S), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  AdjInput in = adj_input(h, trial);
  in.frames = frames;
  in.n_frames = n_frames;
  in.zconst = S.zconst;
  in.coef = coef;
  in.phi = phi;
  in.z_out = z;
  in.grad = grad;
  std::string err;
  r = adjoint_frames(in, h->stream, err);
  if (r) return fail(h, r, "phi_frames_adjoint: " + err);
  return SIM_OK;
}

VP_API int phi_frames_refine(sim_handle *h, int32_t trial, double *frames, int32_t n_frames, int32_t n_iter,
                             double step, double *phi_history, int32_t *n_accepted) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials || n_frames < 2 || !frames || n_iter < 0 || !(step > 0.0))
    return fail(h, SIM_EINVAL, "bad refinement arguments");
  TrialState S;
  CK(cudaMemcpyAsync(&S, h->d.tstate + trial, sizeof(S), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  AdjInput in = adj_input(h, trial);
  in.n_frames = n_frames;
  in.zconst = S.zconst;
  std::string err;
  int acc = 0;
  r = refine_frames(in, frames, n_iter, step, phi_history, &acc, h->stream, err);
  if (n_accepted) *n_accepted = acc;
  if (r) return fail(h, r, "phi_frames_refine: " + err);
  return SIM_OK;
}

VP_API int phi_adjoint_coefficients(sim_handle *h, const double *z, const double *Q, int32_t n, double *coef,
                                    double *phi) {
  int r = enter(h);
  if (r) return r;
  if (n < 1 || !z || !Q || !coef) return fail(h, SIM_EINVAL, "bad arguments");
  std::string err;
  r = adjoint_coefficients(z, Q, n, h->c.dt_d * h->c.kR_half_d * h->c.kR_half_d, coef, phi, h->stream, err);
  if (r) return fail(h, r, "phi_adjoint_coefficients: " + err);
  return SIM_OK;
}

// ---------------------------------------------------------------------------
// autotuner: times the launch-shape variants of the pair and reaction-
// coordinate kernels on this batch (into scratch accumulators, so the state
// is untouched) and keeps the fastest; results are cached per size class
// (atoms per trial, trials, atom density) in a small text file.
// ---------------------------------------------------------------------------
namespace {

std::string tune_key(const sim_handle *h) {
  long long atoms = 0;
  double vol = 0.0;
  for (const auto &T : h->tinfo) {
    atoms += T.n_atoms;
    vol += (double)T.box * T.box * T.box;
  }
  const int lg_atoms = (int)std::lround(std::log2((double)std::max(1LL, atoms)));
  const int lg_trials = (int)std::lround(std::log2((double)std::max(1, h->n_trials)));
  const int dens = (int)std::lround(atoms / std::max(vol, 1e-9) / 10.0);
  char buf[96];
  std::snprintf(buf, sizeof(buf), "a%d_t%d_d%d_nt%d", lg_atoms, lg_trials, dens, h->c.n_types);
  return buf;
}

bool tune_lookup(const char *path, const std::string &key, int &pv, int &cv) {
  FILE *f = path ? std::fopen(path, "r") : nullptr;
  if (!f) return false;
  char k[128];
  int a, b;
  bool found = false;
  while (std::fscanf(f, "%127s %d %d", k, &a, &b) == 3)
    if (key == k) { pv = a; cv = b; found = true; }
  std::fclose(f);
  return found && pv >= 0 && pv < PAIR_VARIANTS && cv >= 0 && cv < CV_VARIANTS;
}

void tune_store(const char *path, const std::string &key, int pv, int cv) {
  if (!path) return;
  FILE *f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d\n", key.c_str(), pv, cv);
  std::fclose(f);
}

}  // namespace

namespace {
// size classes: trials grouped by round(log2 atoms), density (per 10 atoms/nm^3)
// and the batch's type count; device cluster lists of each class
int build_classes(sim_handle *h) {
  if (!h->classes.empty()) return SIM_OK;
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (int t = 0; t < h->n_trials; ++t) {
    const TrialInfo &T = h->tinfo[t];
    const double vol = (double)T.box * T.box * T.box;
    const int lg = (int)std::lround(std::log2((double)std::max(1, T.n_atoms)));
    const int dens = (int)std::lround(T.n_atoms / std::max(vol, 1e-9) / 10.0);
    groups[{lg, dens}].push_back(t);
  }
  for (const auto &g : groups) {
    sim_handle::SizeClass k;
    k.lg_atoms = g.first.first;
    k.n_trials = (int)g.second.size();
    std::vector<int32_t> cl;
    for (int t : g.second)
      for (int q = 0; q < h->tinfo[t].max_clus; ++q) cl.push_back(h->tinfo[t].clus0 + q);
    k.n_clus = (int)cl.size();
    int r = upload(h, &k.clist, cl);
    if (r) return r;
    h->classes.push_back(k);
  }
  return SIM_OK;
}
}  // namespace

VP_API int sim_autotune(sim_handle *h, int32_t reps, const char *cache_path, int32_t *choice) {
  int r = enter(h);
  if (r) return r;
  if (reps < 1) reps = 5;
  r = build_classes(h);
  if (r) return r;
  const std::string key = tune_key(h);
  int pv = 0, cv = 0;
  bool per_class = false;
  const bool multi = h->classes.size() > 1;
  if (multi || !tune_lookup(cache_path, key, pv, cv)) {
    // scratch accumulators: the timed launches must not touch the state
    Dev scratch = h->d;
    const size_t ns = (size_t)h->d.total_slots + CJ;  // with the idle half cluster
    size_t ncv = 0;
    for (auto &T : h->tinfo) ncv += T.n_cv;
    long long *buf = nullptr;
    double *zp = nullptr;
    CK(cudaMalloc(&buf, sizeof(long long) * (3 * ns + 3 * std::max<size_t>(ncv, 1))));
    CK(cudaMalloc(&zp, sizeof(double) * std::max(1, h->d.total_work)));
    scratch.fx = buf; scratch.fy = buf + ns; scratch.fz = buf + 2 * ns;
    scratch.gx = buf + 3 * ns; scratch.gy = scratch.gx + ncv; scratch.gz = scratch.gy + ncv;
    scratch.z_part = zp;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_it = [&](auto &&launch) {
      launch();  // warm
      cudaEventRecord(e0, h->stream);
      for (int k = 0; k < reps; ++k) launch();
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      return ms;
    };
    float best = 3e38f;
    for (int v = 0; v < PAIR_VARIANTS; ++v) {
      float ms = time_it([&] { launch_pair(scratch, h->c, false, -1, h->stream, v); });
      if (ms < best) { best = ms; pv = v; }
    }
    if (multi) {
      // each class on its own, then the classes one after another with their
      // own variants against the best single launch over the whole batch
      for (auto &k : h->classes) {
        float bk = 3e38f;
        for (int v = 0; v < PAIR_VARIANTS; ++v) {
          float ms = time_it([&] { launch_pair(scratch, h->c, false, -1, h->stream, v, k.clist, k.n_clus); });
          if (ms < bk) { bk = ms; k.variant = v; }
        }
      }
      const float t_classes = time_it([&] {
        for (const auto &k : h->classes) launch_pair(scratch, h->c, false, -1, h->stream, k.variant, k.clist, k.n_clus);
      });
      per_class = t_classes < best;
    }
    float bc = 3e38f;
    for (int v = 0; v < CV_VARIANTS; ++v) {
      float ms = time_it([&] { launch_cv(scratch, h->c, h->stream, v); });
      if (ms < bc) { bc = ms; cv = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(zp);
    CK(cudaGetLastError());
    if (!multi) tune_store(cache_path, key, pv, cv);
  }
  h->pair_variant = pv;
  h->cv_variant = cv;
  h->per_class = per_class;
  if (!multi && !h->classes.empty()) h->classes[0].variant = pv;
  if (h->chunk) {
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  if (choice) { choice[0] = pv; choice[1] = cv; }
  return SIM_OK;
}

VP_API int sim_set_class_variants(sim_handle *h, const int32_t *variants, int32_t n) {
  if (!h) return SIM_EINVAL;
  if (build_classes(h)) return SIM_ECUDA;
  if (!variants || n != (int32_t)h->classes.size()) return fail(h, SIM_EINVAL, "one variant per size class");
  for (int k = 0; k < n; ++k)
    if (variants[k] < 0 || variants[k] >= PAIR_VARIANTS) return fail(h, SIM_EINVAL, "variant out of range");
  for (int k = 0; k < n; ++k) h->classes[k].variant = variants[k];
  h->per_class = true;
  if (h->chunk) {
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  return SIM_OK;
}

VP_API int sim_set_step_mode(sim_handle *h, int32_t mode) {
  if (!h) return SIM_EINVAL;
  if (mode < 0 || mode >= STEP_MODES)
    return fail(h, SIM_EINVAL,
                "step mode must be 0 (kernel per phase), 1 (one kernel) or 2 (kernel per phase, rebuild kernels "
                "only in steps with a rebuild)");
  if (mode == 1 && h->c.n_types > SMALL_TYPES)
    return fail(h, SIM_EINVAL, "the one-kernel step handles at most 16 distinct LJ types");
  h->fused = mode == 1;
  h->skip_empty = mode == 2;
  if (h->chunk) {
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  return SIM_OK;
}

VP_API int32_t sim_step_mode(const sim_handle *h) {
  return h ? (h->fused ? 1 : h->skip_empty ? 2 : 0) : SIM_EINVAL;
}

VP_API int sim_autotune_step(sim_handle *h, int32_t reps, int32_t *mode, double *ms_per_step) {
  int r = enter(h);
  if (r) return r;
  if (reps < 1) reps = 3;
  const Dev &d = h->d;
  const int nst = h->params.nstlist;
  // the state to come back to: positions and velocities of every trial, the
  // functional's bookkeeping, the step counter
  size_t n = 0;
  for (const auto &T : h->tinfo) n += (size_t)T.n_atoms;
  double *saved = nullptr;
  CK(cudaMalloc(&saved, sizeof(double) * 6 * std::max<size_t>(n, 1)));
  {
    size_t off = 0;
    for (int t = 0; t < h->n_trials; ++t) {
      const size_t m = (size_t)h->tinfo[t].n_atoms;
      launch_gather_state(d, t, saved + 3 * off, saved + 3 * n + 3 * off, (int)m, h->stream);
      off += m;
    }
  }
  std::vector<TrialState> S(h->n_trials);
  CK(cudaMemcpyAsync(S.data(), d.tstate, sizeof(TrialState) * h->n_trials, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const long long step0 = h->step;
  auto restore = [&]() -> int {
    launch_scatter_state(d, -1, saved, saved + 3 * n, (int)n, h->stream);
    // the functional's bookkeeping comes back; the cluster counts stay those
    // of the current layout (the rebuild below starts from it)
    std::vector<TrialState> cur(h->n_trials);
    CK(cudaMemcpyAsync(cur.data(), d.tstate, sizeof(TrialState) * h->n_trials, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int t = 0; t < h->n_trials; ++t) {
      cur[t].zm = S[t].zm;
      cur[t].Phi = S[t].Phi;
    }
    CK(cudaMemcpyAsync(d.tstate, cur.data(), sizeof(TrialState) * h->n_trials, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(d.step, &step0, sizeof(step0), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(d.cur_step, &step0, sizeof(step0), cudaMemcpyHostToDevice, h->stream));
    h->step = step0;
    const float half = 0.5f;
    CK(cudaMemcpyAsync(d.kick, &half, sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(d.fx, 0, sizeof(long long) * d.total_slots, h->stream));
    CK(cudaMemsetAsync(d.fy, 0, sizeof(long long) * d.total_slots, h->stream));
    CK(cudaMemsetAsync(d.fz, 0, sizeof(long long) * d.total_slots, h->stream));
    size_t ncv = 0;
    for (auto &T : h->tinfo) ncv += T.n_cv;
    if (ncv) {
      CK(cudaMemsetAsync(d.gx, 0, sizeof(long long) * ncv, h->stream));
      CK(cudaMemsetAsync(d.gy, 0, sizeof(long long) * ncv, h->stream));
      CK(cudaMemsetAsync(d.gz, 0, sizeof(long long) * ncv, h->stream));
    }
    forces(h, FIN_KEEP, -1);
    CK(cudaStreamSynchronize(h->stream));
    return check_flags(h);
  };
  float best = 3e38f;
  int pick = sim_step_mode(h);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int m = 0; m < STEP_MODES && r == SIM_OK; ++m) {
    if (ms_per_step) ms_per_step[m] = -1.0;
    if (m == 1 && h->c.n_types > SMALL_TYPES) continue;  // a form this batch cannot take
    r = sim_set_step_mode(h, m);
    if (!r) r = sim_step_batch(h, nst);  // captures the chunk graph
    if (!r) {
      cudaEventRecord(e0, h->stream);
      for (int k = 0; k < reps && !r; ++k) r = sim_step_batch(h, nst);
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (!r && ms < best) { best = ms; pick = m; }
      if (!r && ms_per_step) ms_per_step[m] = ms / ((double)reps * nst);
    }
    if (!r) r = restore();
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(saved);
  if (r) return r;
  r = sim_set_step_mode(h, pick);
  if (mode) *mode = pick;
  return r;
}

VP_API int32_t sim_tune_classes(sim_handle *h, int32_t *info, int32_t cap) {
  if (!h) return SIM_EINVAL;
  if (build_classes(h)) return SIM_ECUDA;
  const int n = (int)h->classes.size();
  for (int k = 0; k < n && k < cap && info; ++k) {
    const auto &c = h->classes[k];
    int32_t *o = info + 5 * k;
    o[0] = c.lg_atoms; o[1] = c.n_trials; o[2] = c.n_clus; o[3] = h->per_class ? c.variant : h->pair_variant;
    o[4] = h->per_class ? 1 : 0;
  }
  return n;
}

VP_API int sim_set_variants(sim_handle *h, int32_t pair_variant, int32_t cv_variant) {
  if (!h) return SIM_EINVAL;
  if (pair_variant < 0 || pair_variant >= PAIR_VARIANTS || cv_variant < 0 || cv_variant >= CV_VARIANTS)
    return fail(h, SIM_EINVAL, "variant out of range");
  h->pair_variant = pair_variant;
  h->cv_variant = cv_variant;
  h->per_class = false;
  if (h->chunk) {
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  return SIM_OK;
}

VP_API int sim_pairlist(sim_handle *h, int32_t trial, int32_t *pairs, int64_t cap, int64_t *n_pairs) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials || cap < 0) return fail(h, SIM_EINVAL, "bad arguments");
  TrialState S;
  CK(cudaMemcpyAsync(&S, h->d.tstate + trial, sizeof(S), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemsetAsync(h->d_count, 0, sizeof(unsigned long long), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int32_t *dp = nullptr;
  size_t nbytes = (size_t)std::max<int64_t>(cap, 1) * 2 * sizeof(int32_t);
  CK(cudaMalloc(&dp, nbytes));
  launch_extract_pairs(h->d, h->c.list_cap, trial, S.n_clus, dp, cap, h->d_count, h->stream);
  unsigned long long cnt = 0;
  cudaMemcpyAsync(&cnt, h->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  int64_t keep = std::min<int64_t>((int64_t)cnt, cap);
  cudaError_t e = cudaSuccess;
  if (keep > 0 && pairs) e = cudaMemcpy(pairs, dp, (size_t)keep * 2 * sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(dp);
  if (e != cudaSuccess) return fail(h, SIM_ECUDA, cudaGetErrorString(e));
  if (n_pairs) *n_pairs = (int64_t)cnt;
  return SIM_OK;
}

VP_API int sim_diagnostics(sim_handle *h, int64_t *out) {
  int r = enter(h);
  if (r) return r;
  if (!out) return fail(h, SIM_EINVAL, "out is NULL");
  long long dg[4] = {0, 0, 0, 0};
  std::vector<int32_t> ln(h->d.total_clus);
  std::vector<TrialState> S(h->n_trials);
  CK(cudaMemcpyAsync(dg, h->d.diag, sizeof(dg), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(ln.data(), h->d.list_n, sizeof(int32_t) * ln.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(S.data(), h->d.tstate, sizeof(TrialState) * S.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int mx = 0;
  for (int v : ln) mx = std::max(mx, v);
  long long used = 0, entries = 0;
  for (auto &s : S) used += s.n_clus;
  for (int v : ln) entries += v;
  out[0] = dg[0];
  out[1] = mx;
  out[2] = h->c.list_cap;
  out[3] = used;
  out[4] = entries;
  out[5] = dg[1];
  out[6] = dg[2];
  return SIM_OK;
}

VP_API int sim_set_timing(sim_handle *h, int32_t on) {
  if (!h) return SIM_EINVAL;
  if (on < 0 || on > 2) return fail(h, SIM_EINVAL, "timing mode must be 0, 1 or 2");
  h->timing = on == 1;
  const bool g = on == 2;
  if (g != h->gtiming && h->chunk) {  // the chunk graph is captured again with or without the event nodes
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  h->gtiming = g;
  return SIM_OK;
}

VP_API int sim_kernel_times(sim_handle *h, const char **names, double *ms, int64_t *counts, int32_t cap) {
  if (!h) return SIM_EINVAL;
  int n = (int)h->timers.size();
  for (int k = 0; k < n && k < cap; ++k) {
    if (names) names[k] = h->timers[k].name;
    if (ms) ms[k] = h->timers[k].ms;
    if (counts) counts[k] = h->timers[k].count;
  }
  for (auto &t : h->timers) { t.ms = 0.0; t.count = 0; }
  return n;
}

namespace {
// C(r) > 1/2 with s = (r/r0)^2  <=>  s^4 + s^3 - s^2 - s - 1 < 0
bool contact_above_half(double r2, double r0) {
  const double s = r2 / (r0 * r0);
  return (((s + 1.0) * s - 1.0) * s - 1.0) * s - 1.0 < 0.0;
}

// native contact lists of every system, per-trial formation times (all -1)
int build_contacts(sim_handle *h) {
  if (h->contacts_built) return SIM_OK;
  const double r0 = h->params.cv_r0;
  std::vector<int2> pairs;
  std::vector<int32_t> off(h->n_sys), cnt(h->n_sys);
  int max_nc = 0;
  for (int sy = 0; sy < h->n_sys; ++sy) {
    off[sy] = (int32_t)pairs.size();
    const double *X = h->native_all.data() + 3 * (size_t)h->sys_nat0[sy];
    const int n = h->sys_ncv[sy], ms = h->sys_minsep[sy];
    for (int i = 0; i < n; ++i)
      for (int j = i + ms + 1; j < n; ++j) {
        const double dx = X[3 * j] - X[3 * i], dy = X[3 * j + 1] - X[3 * i + 1], dz = X[3 * j + 2] - X[3 * i + 2];
        if (contact_above_half(dx * dx + dy * dy + dz * dz, r0)) pairs.push_back(make_int2(i, j));
      }
    cnt[sy] = (int32_t)pairs.size() - off[sy];
    max_nc = std::max(max_nc, cnt[sy]);
  }
  std::vector<long long> toff(h->n_trials);
  long long total = 0;
  for (int t = 0; t < h->n_trials; ++t) {
    toff[t] = total;
    total += cnt[h->trial_sys[t]];
  }
  // threshold: the positive root s_h of s^4 + s^3 - s^2 - s - 1 (bisection on [1, 2])
  double lo = 1.0, hi = 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if ((((mid + 1.0) * mid - 1.0) * mid - 1.0) * mid - 1.0 < 0.0) lo = mid; else hi = mid;
  }
  const double rh2 = 0.5 * (lo + hi) * r0 * r0;
  auto alloc = [&](void **p, size_t bytes) {
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) h->callocs.push_back(*p);
    return e;
  };
  int2 *dp = nullptr;
  int32_t *doff = nullptr, *dcnt = nullptr, *dts = nullptr;
  long long *dt = nullptr, *dtoff = nullptr;
  CK(alloc((void **)&dp, pairs.size() * sizeof(int2)));
  CK(alloc((void **)&doff, off.size() * sizeof(int32_t)));
  CK(alloc((void **)&dcnt, cnt.size() * sizeof(int32_t)));
  CK(alloc((void **)&dts, h->trial_sys.size() * sizeof(int32_t)));
  CK(alloc((void **)&dt, (size_t)total * sizeof(long long)));
  CK(alloc((void **)&dtoff, toff.size() * sizeof(long long)));
  if (!pairs.empty()) CK(cudaMemcpy(dp, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(doff, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dcnt, cnt.data(), cnt.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  std::vector<int32_t> ts(h->trial_sys.begin(), h->trial_sys.end());
  CK(cudaMemcpy(dts, ts.data(), ts.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dtoff, toff.data(), toff.size() * sizeof(long long), cudaMemcpyHostToDevice));
  ContactDev &c = h->cdev;
  c.every = 0;
  c.max_nc = max_nc;
  c.pairs = dp;
  c.sys_off = doff;
  c.sys_n = dcnt;
  c.trial_sys = dts;
  c.t = dt;
  c.t_off = dtoff;
  c.r2_lo = (float)(rh2 * (1.0 - 1e-4));
  c.r2_hi = (float)(rh2 * (1.0 + 1e-4));
  c.r0 = r0;
  h->csys_n = cnt;
  h->ct_off = toff;
  h->contacts_built = true;
  return SIM_OK;
}
}  // namespace

VP_API int sim_contact_tracking(sim_handle *h, int32_t every) {
  int r = enter(h);
  if (r) return r;
  if (every < 0) return fail(h, SIM_EINVAL, "every must be >= 0");
  r = build_contacts(h);
  if (r) return r;
  long long total = h->ct_off.empty() ? 0 : h->ct_off.back() + h->csys_n[h->trial_sys.back()];
  if (total > 0) CK(cudaMemsetAsync(h->cdev.t, 0xff, (size_t)total * sizeof(long long), h->stream));  // all -1
  if (h->chunk) {  // the chunk graph is captured again with or without the tracker
    cudaGraphExecDestroy(h->chunk);
    h->chunk = nullptr;
  }
  h->cdev.every = every;
  h->contacts_tracked = true;
  CK(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

VP_API int sim_native_contacts(sim_handle *h, int32_t trial, int32_t *pairs, int64_t cap, int64_t *n_contacts) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials || cap < 0 || (cap > 0 && !pairs))
    return fail(h, SIM_EINVAL, "bad native-contact arguments");
  r = build_contacts(h);
  if (r) return r;
  const int sy = h->trial_sys[trial];
  const int64_t n = h->csys_n[sy];
  if (n_contacts) *n_contacts = n;
  const int64_t m = std::min(n, cap);
  if (m > 0) {
    int32_t off = 0;
    for (int q = 0; q < sy; ++q) off += h->csys_n[q];
    CK(cudaMemcpy(pairs, h->cdev.pairs + off, (size_t)m * sizeof(int2), cudaMemcpyDeviceToHost));
  }
  return SIM_OK;
}

VP_API int sim_contact_times(sim_handle *h, int32_t trial, int64_t *times, int64_t cap) {
  int r = enter(h);
  if (r) return r;
  if (trial < 0 || trial >= h->n_trials || cap < 0 || (cap > 0 && !times))
    return fail(h, SIM_EINVAL, "bad contact-time arguments");
  if (!h->contacts_tracked) return fail(h, SIM_EINVAL, "contact tracking was never enabled");
  const int64_t m = std::min<int64_t>(h->csys_n[h->trial_sys[trial]], cap);
  CK(cudaStreamSynchronize(h->stream));
  if (m > 0)
    CK(cudaMemcpy(times, h->cdev.t + h->ct_off[trial], (size_t)m * sizeof(long long), cudaMemcpyDeviceToHost));
  return SIM_OK;
}

VP_API int sim_philox_normals(uint64_t seed, int64_t step, uint32_t stream, int32_t n, uint32_t *raw,
                              double *normals) {
  if (n < 0 || step < 0) return SIM_EINVAL;
  if (n == 0) return SIM_OK;
  uint32_t *draw = nullptr;
  double *dnorm = nullptr;
  if (cudaMalloc(&draw, sizeof(uint32_t) * 4 * (size_t)n) != cudaSuccess) return SIM_ECUDA;
  if (cudaMalloc(&dnorm, sizeof(double) * 3 * (size_t)n) != cudaSuccess) {
    cudaFree(draw);
    return SIM_ECUDA;
  }
  launch_philox_normals(seed, (unsigned long long)step, stream, n, draw, dnorm, 0);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && raw) e = cudaMemcpy(raw, draw, sizeof(uint32_t) * 4 * (size_t)n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && normals)
    e = cudaMemcpy(normals, dnorm, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(draw);
  cudaFree(dnorm);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

VP_API void *sim_stream(sim_handle *h) { return h ? (void *)h->stream : nullptr; }

VP_API void sim_destroy(sim_handle *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->bstream) cudaStreamSynchronize(h->bstream);
  if (h->chunk) cudaGraphExecDestroy(h->chunk);
  for (auto &e : h->gev) cudaEventDestroy(e);
  for (void *p : h->callocs) cudaFree(p);
  for (void *p : h->allocs) cudaFree(p);
  if (h->d.rec) cudaFree(h->d.rec);
  if (h->frames) cudaFree(h->frames);
  if (h->dbuf) cudaFree(h->dbuf);
  for (auto &t : h->timers)
    for (auto &pr : t.ev) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  if (h->entry_ev) cudaEventDestroy(h->entry_ev);
  if (h->exit_ev) cudaEventDestroy(h->exit_ev);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_bjoin) cudaEventDestroy(h->ev_bjoin);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->bstream) cudaStreamDestroy(h->bstream);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

VP_API const char *sim_last_error(const sim_handle *h) { return h ? h->err.c_str() : "null handle"; }

/*
 * vpath.h -- C ABI of the GB300 trial-path generator of the variational
 * pathway scheme (arXiv:1405.6104): many biased Langevin trial trajectories
 * in explicit solvent, advanced together on one GPU, each scored by the bias
 * functional whose least value selects the optimal path.
 *
 * The method (paper references are to its equations and sections):
 *   - Eq. Lang: Langevin dynamics m x'' = -m gamma x' - grad U + eta for the
 *     solute X (atoms [0, n_solute)) and the solvent Y (the other atoms);
 *     integrated with BAOAB, white noise from Philox4x32-10.
 *   - Eq. VR: ratchet-and-pawl bias on the solute only,
 *     F_i = -(k_R/2) (z - z_m) grad_i z when z > z_m, 0 otherwise, with z_m
 *     the running minimum of z and z_m(0) = z(X_0).
 *   - SM "Collective coordinate": z(X) = sum_{i<j, j-i > cv_min_sep}
 *     [C~_ij(X) - C~_ij(X_native)]^2, C(r) = (1-(r/r0)^6)/(1-(r/r0)^10),
 *     C~ = C * S(r) with S a quintic switch from 1 at cv_r_switch to 0 at
 *     cv_r_cut.
 *   - Eq. VMDcondition: Phi = int dt sum_{i in solute} |F_i^bias|^2/(gamma_i m_i),
 *     accumulated every step; the trial with the least Phi is the optimum
 *     (Sec. "Results", selection per initial condition).
 *
 * Conventions for every entry point:
 *   - Units: nm, ps, amu, kJ/mol, e, K.
 *   - Return value 0 (SIM_OK) or a negative SIM_E* code; sim_last_error()
 *     then describes the failure.  No entry point aborts the process.
 *   - All pointer arguments are HOST pointers, owned by the caller, read or
 *     written only during the call.  The library owns all device memory it
 *     allocates (cudaMalloc at sim_create, freed by sim_destroy).
 *   - A handle is not thread-safe; calls on one handle must be serialised.
 *   - Atom indices are the caller's order within a system; trials are
 *     numbered system by system (all trials of system 0 first).
 */
#ifndef VPATH_H
#define VPATH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SIM_OK 0
#define SIM_EINVAL (-1)          /* invalid argument or system description */
#define SIM_ECUDA (-2)           /* a CUDA call failed */
#define SIM_ELIST_OVERFLOW (-3)  /* a cluster's neighbour list or a grid column exceeded capacity
                                   (per 8-atom cluster 2 048 j-atoms with a listed pair, from at
                                   most 512 4-atom j-clusters; the environment variable
                                   VPATH_LIST_CAP, read at sim_create, lowers the first to
                                   8..2047 for fault-injection tests) */
#define SIM_ESKIN (-4)           /* an atom moved more than skin/2 between fixed-interval list rebuilds
                                   (SIM_FIXED_INTERVAL | SIM_STRICT_SKIN) */
#define SIM_ENONFINITE (-5)      /* a position, velocity or z became non-finite, a force exceeded
                                   2^30 kJ/mol/nm or an atom moved more than a box length in one
                                   step (the run has blown up) */
#define SIM_ETIMEOUT (-6)        /* a bounded device wait gave up (a grid barrier of the one-kernel step) */

/* sim_params.flags */
#define SIM_STRICT_SKIN 1        /* with SIM_FIXED_INTERVAL: treat skin violations as errors instead of
                                   counting them (SIM_EINVAL without SIM_FIXED_INTERVAL) */
#define SIM_NO_GRAPH 2           /* launch every kernel directly instead of replaying CUDA graphs */
#define SIM_FIXED_INTERVAL 4     /* rebuild lists only at steps that are multiples of nstlist (no
                                   displacement trigger: pairs may be missed when an atom moves more
                                   than skin/2 within an interval; such moves are counted) */

typedef struct sim_handle sim_handle;

/* One periodic system.  Arrays are read at sim_create only. */
typedef struct sim_system {
  int32_t n_atoms;         /* total atoms (solute + solvent), >= 1 */
  int32_t n_solute;        /* solute X = atoms [0, n_solute) */
  int32_t n_cv;            /* atoms of the reaction coordinate = [0, n_cv), n_cv <= n_solute */
  const double *pos;       /* [3*n_atoms] start positions, nm (stored as FP32 on the device) */
  const double *vel;       /* [3*n_atoms] start velocities nm/ps, or NULL: Maxwell-Boltzmann
                              draw per trial (Philox stream 1) with the centre of mass at rest */
  const double *mass;      /* [n_atoms] amu, > 0 */
  const double *charge;    /* [n_atoms] e */
  const int32_t *lj_type;  /* [n_atoms] index into sigma/epsilon */
  int32_t n_types;
  const double *sigma;     /* [n_types] nm; Lorentz-Berthelot mixing */
  const double *epsilon;   /* [n_types] kJ/mol */
  int32_t n_bonds;
  const int32_t *bonds;    /* [2*n_bonds] atom pairs, V = k/2 (r - r0)^2 */
  const double *bond_r0;   /* [n_bonds] nm */
  const double *bond_k;    /* [n_bonds] kJ/mol/nm^2 */
  int32_t n_angles;
  const int32_t *angles;   /* [3*n_angles] (i, vertex, k), V = k/2 (theta - theta0)^2 */
  const double *angle_t0;  /* [n_angles] rad */
  const double *angle_k;   /* [n_angles] kJ/mol/rad^2 */
  int32_t n_excl;
  const int32_t *excl;     /* [2*n_excl] extra excluded pairs; 1-2 and 1-3 pairs are excluded automatically */
  double box;              /* cubic periodic box side, nm (rounded to FP32); > 2 (r_cut + skin) */
  const double *native_pos;/* [3*n_cv] target structure X_native of the contact map (plain distances) */
  const double *gamma;     /* [n_atoms] friction 1/ps, or NULL: sim_params.gamma for every atom */
} sim_system;

/* Run parameters shared by all trials. */
typedef struct sim_params {
  double dt;               /* ps */
  double temperature;      /* K */
  double gamma;            /* 1/ps, default friction */
  double r_cut;            /* LJ and reaction-field cut-off, nm */
  double skin;             /* Verlet buffer, nm: lists hold pairs within r_cut + skin */
  int32_t nstlist;         /* longest interval between two list rebuilds of a trial, >= 1 (with
                              SIM_FIXED_INTERVAL: the interval).  A trial's list is also rebuilt,
                              before the forces, in the first step in which one of its atoms is
                              farther than skin/2 - 1e-5 nm from where the list was built, so that
                              no pair closer than r_cut is ever missing from it (the cut-off model
                              of U in Eq. Lang); nstlist steps are also one CUDA-graph chunk */
  double eps_rf;           /* reaction-field dielectric; <= 0 means infinity */
  double k_ratchet;        /* k_R of Eq. VR, kJ/mol */
  double cv_r0;            /* r0 of the contact function, nm */
  double cv_r_switch;      /* switching of C~ starts, nm */
  double cv_r_cut;         /* C~ = 0 beyond, nm */
  int32_t cv_min_sep;      /* contact pairs have j - i > cv_min_sep, >= 0 */
  uint64_t seed;           /* trial t uses seed + t unless trial_seeds is given */
  int32_t flags;           /* SIM_* flags */
} sim_params;

/* Creates a batch: trials_per_system[s] independent trials of each system
 * (1 to 65535 trials in all; SIM_EINVAL otherwise) (trial seeds from
 * trial_seeds[total trials] or params->seed + t).  Uploads
 * the systems, draws velocities where vel is NULL, builds cells and lists,
 * computes the first forces and sets z_m = z(X_0), Phi = 0 for every trial.
 * cuda_stream: the caller's stream (or NULL); the library orders its own
 * stream after it at every call and synchronises before returning.
 * On success *out receives the handle.  On failure *out may still receive a
 * handle that only sim_last_error and sim_destroy accept (or NULL). */
int sim_create(const sim_system *systems, int32_t n_systems, const int32_t *trials_per_system,
               const uint64_t *trial_seeds, const sim_params *params, void *cuda_stream, sim_handle **out);

/* Advances every trial by n_steps BAOAB steps with the rMD bias and the
 * per-step accumulation of Phi (Eqs. Lang, VR, VMDcondition).  Blocks until
 * the device error flags are read.  n_steps >= 0. */
int sim_step_batch(sim_handle *h, int32_t n_steps);

/* Bias functional of every trial (phi[total trials], may be NULL) and the
 * index of the trial with the least Phi among trials whose current z is
 * <= z_max (z_max < 0: all trials); *argmin = -1 if none qualifies; ties go
 * to the lowest index (selection of Sec. "Results"). */
int bias_functional(sim_handle *h, double z_max, double *phi, int32_t *argmin);

/* Energies and forces of one trial at its current state, without advancing
 * it: energies[6] = {E_LJ, E_RF, E_bond, E_angle, E_kin, E_bias} with
 * E_bias = (k_R/4) (z - z_m)_+^2; forces[3*n_atoms] (or NULL) = -grad U plus
 * the ratchet force, in the caller's atom order. */
int energy_forces(sim_handle *h, int32_t trial, double *energies, double *forces);

/* State of one trial: pos, vel [3*n_atoms] (either may be NULL; positions
 * are wrapped into the box at list rebuilds), cv[4] = {z, z_m, a, Phi} (may
 * be NULL) where a = (z - z_m_previous)_+ of the last force evaluation. */
int sim_get_state(sim_handle *h, int32_t trial, double *pos, double *vel, double *cv);

/* Replaces the state of one trial (trial >= 0) or of all trials (trial = -1,
 * arrays concatenated in trial order).  pos and vel must both be given.
 * cv_state = {z_m, Phi} per affected trial, or NULL to restart the functional
 * (z_m = z(X), Phi = 0).  Lists are rebuilt and forces recomputed for the
 * affected trials (forces of the whole batch); the step counter is unchanged. */
int sim_set_state(sim_handle *h, int32_t trial, const double *pos, const double *vel, const double *cv_state);

/* Rebuilds the lists of every trial at the current positions and recomputes
 * the forces, leaving the state (positions, velocities, z_m, Phi, step
 * counter, records) as it is.  A run that calls this at a checkpoint and a run
 * restored there with sim_set_state continue bit-identically. */
int sim_rebuild(sim_handle *h);

/* The potential U(X, Y) of Eq. Lang (Lennard-Jones + reaction field + bonds
 * + angles, no bias) and its forces -grad U for one configuration per trial,
 * entirely on the device: no host copy, no synchronisation of the host.
 *   d_pos: DEVICE array, every trial's positions [n_atoms][3] (nm, FP64,
 *     caller order), trials concatenated in trial order; the trials' positions
 *     are replaced by them (stored as FP32; velocities and the functional's
 *     bookkeeping are left as they are: call sim_set_state before stepping
 *     such a trial);
 *   d_energy: DEVICE array [n_trials] (FP64, kJ/mol) or NULL; NaN for every
 *     trial when a device error flag was raised in the evaluation (a list
 *     overflow, a non-finite coordinate);
 *   d_forces: DEVICE array shaped like d_pos (kJ/mol/nm) or NULL;
 *   cuda_stream: the caller's stream; the work is ordered after the work
 *     queued on it before the call, and work queued on it after the call
 *     waits for the results.
 * A trial's list is rebuilt only when one of its atoms lies farther than
 * skin/2 - 1e-5 nm from where the list was built (so repeated evaluations near
 * one configuration reuse it).  SIM_EINVAL without d_pos or any output. */
int sim_potential_device(sim_handle *h, const double *d_pos, double *d_energy, double *d_forces, void *cuda_stream);

/* Steps taken since creation (the Philox counter of the next step is this + 1). */
int64_t sim_step_count(const sim_handle *h);
/* Sets the step counter (resume from a checkpoint; with SIM_FIXED_INTERVAL
 * lists are rebuilt at multiples of nstlist of this counter). */
int sim_set_step_count(sim_handle *h, int64_t step);

/* Noise counter offset of one trial: its Langevin noise of step n is drawn
 * with the Philox counter of step n + offset (Eq. Lang; the noise is a
 * function of (trial seed, atom, step) only).  0 at creation.  A batch that
 * replays segments of one trajectory side by side (each segment a trial with
 * the original seed) sets each segment's start step as its offset, so every
 * segment draws the noise of the original run.  SIM_EINVAL for a bad trial. */
int sim_set_noise_offset(sim_handle *h, int32_t trial, int64_t offset);

/* The noise counter offset of a trial (see sim_set_noise_offset) into
 * *offset.  SIM_EINVAL for a bad trial or NULL offset. */
int sim_noise_offset(sim_handle *h, int32_t trial, int64_t *offset);

/* The Philox key (seed) of a trial: trial_seeds[trial] at creation, or
 * params->seed + trial.  SIM_EINVAL for a bad trial or NULL seed. */
int sim_trial_seed(sim_handle *h, int32_t trial, uint64_t *seed);

int32_t sim_num_trials(const sim_handle *h);
int32_t sim_num_atoms(const sim_handle *h, int32_t trial);

/* Per-step record of {z, z_m, a, phi, Q} for every trial, where
 * phi = (k_R/2)^2 a^2 Q and Q = sum_i |grad_i z|^2/(gamma_i m_i): capacity
 * entries per trial (0 disables); entry of step n at index n % capacity.
 * Enabling clears the record. */
int sim_record(sim_handle *h, int32_t capacity);
int sim_get_record(sim_handle *h, int32_t trial, double *out /* [5*capacity] */);

/* Per-step record of the reaction-coordinate atom positions of one trial
 * (the frames X_n of the path): capacity frames, the frame of step n at index
 * n % capacity, written after every force evaluation (also at sim_set_state).
 * trial = -1 records every trial.  sim_frame_shape writes shape[3] =
 * {trials recorded (1, or n_trials for -1), capacity, m}, all 0 without a
 * record, m = n_cv of the recorded trial or the largest n_cv of the batch.
 * sim_get_frames copies the record, [shape[0]][capacity][m][3] doubles (nm;
 * a trial with fewer CV atoms leaves the rest of its rows 0), to out, which
 * holds out_len doubles: SIM_EINVAL without a record or when out_len is
 * smaller than the record (nothing is written then). */
int sim_record_frames(sim_handle *h, int32_t trial, int32_t capacity);
int sim_frame_shape(sim_handle *h, int32_t *shape);
int sim_get_frames(sim_handle *h, double *out, int64_t out_len);

/* Gradient of the bias functional (Eq. VMDcondition, discretised as in
 * bias_functional) with respect to the reaction-coordinate atoms of every
 * frame of a path X_0 .. X_{n_frames-1} of one trial's system, dt apart:
 *   dPhi/dX_n = A_n grad z(X_n) + B_n H_z(X_n) w_n,  w_i = grad_i z/(gamma_i m_i),
 *   A_n = dt (k_R/2)^2 (2 a_n Q_n - R_n), B_n = 2 dt (k_R/2)^2 a_n^2,
 * a_n = (z_n - min_{k<n} z_k)_+ (Eq. VR), R_n = sum of 2 a_l Q_l over the later
 * frames l whose running minimum sits at frame n (its first minimiser).
 *   frames [n_frames][n_cv][3] host; coef [2*n_frames] host (A_n, B_n) or NULL
 *   to derive them from these frames with z_m starting at frame 0 (then *phi,
 *   if not NULL, receives Phi along them); z [n_frames] (may be NULL) receives
 *   z(X_n); grad [n_frames][n_cv][3] host output. */
int phi_frames_adjoint(sim_handle *h, int32_t trial, const double *frames, int32_t n_frames, const double *coef,
                       double *phi, double *z, double *grad);

/* The coefficients (A_n, B_n) above and Phi from z_n and Q_n along a path of
 * n frames (z_m starts at z_0; Q_0 is not used), e.g. from sim_record, so that
 * phi_frames_adjoint can process a long path segment by segment. */
int phi_adjoint_coefficients(sim_handle *h, const double *z, const double *Q, int32_t n, double *coef, double *phi);

/* Refinement of a path by descent on the functional (the variational
 * condition of Eq. VMDcondition read as a minimisation over the path, with
 * the frames X_1 .. X_{n_frames-2} as the variables and the end frames held
 * fixed): starting from frames [n_frames][n_cv][3] (host, read and
 * overwritten with the refined path), each iteration takes the gradient of
 * phi_frames_adjoint and the first step eta, 2 eta_prev at first, halved until
 * Phi(X - eta g) <= Phi(X) - 1e-4 eta |g|^2 (Armijo; g over the free frames);
 * moved coordinates are rounded to FP32, the precision Phi is evaluated at.
 * phi_history [n_iter + 1] (may be NULL) receives Phi before and after each
 * iteration; *n_accepted (may be NULL) the iterations that moved the path.
 * It stops early, repeating the last value, when no step lowers Phi.  The
 * trial selects the system (and its native map).  SIM_EINVAL for n_frames < 2,
 * n_iter < 0 or step <= 0. */
int phi_frames_refine(sim_handle *h, int32_t trial, double *frames, int32_t n_frames, int32_t n_iter, double step,
                      double *phi_history, int32_t *n_accepted);

/* Test and diagnostics hooks.
 * sim_pairlist: the atom pairs (i < j, caller's indices) that the current
 *   cluster lists hold for one trial (list rule at the last rebuild);
 *   *n_pairs receives the count, pairs beyond cap are dropped.
 * sim_list_positions: pos[3*n_atoms] (caller order) receives the positions
 *   the trial's current list was built from (wrapped into the box).
 * sim_diagnostics: out[7] = {skin violations counted (SIM_FIXED_INTERVAL:
 *   atoms farther than skin/2 from where their list was built when it was
 *   rebuilt; 0 otherwise, where a list is rebuilt before that can happen), max
 *   list entries of a cluster, list capacity per cluster, clusters in use (all
 *   trials), list entries in use (all trials; each is one j-atom against the
 *   8 atoms of its i-cluster, so 8 times this over the atoms is the pair
 *   evaluations per atom-step), list rebuilds of trials since creation, of
 *   them triggered by a displacement}. */
int sim_pairlist(sim_handle *h, int32_t trial, int32_t *pairs, int64_t cap, int64_t *n_pairs);
int sim_list_positions(sim_handle *h, int32_t trial, double *pos);
int sim_diagnostics(sim_handle *h, int64_t *out);

/* Autotuner: times the launch-shape variants of the pair kernel (0-2: the
 * i-atoms in registers with register caps of 4, 5 or 6 blocks per SM; 3-5:
 * the i-atoms in shared memory with caps of 6, 7 or 8 blocks per SM; 6-8:
 * packed FP32x2 arithmetic, i-atoms in shared memory, caps of 5, 6 or 7;
 * 3-8 need at most 16 LJ types, else run as variant 0; all give bit-identical
 * forces) and of the reaction-coordinate kernel
 * (2, 4 or 8 warps per block) on this batch, reps launches each, into scratch
 * accumulators (the state is untouched), and uses the fastest from then on.
 * Size classes: the trials are grouped by round(log2 atoms) and density; when
 * a batch holds more than one class, the pair variants are also timed on each
 * class's clusters alone, and one launch per class with its own variant is
 * used instead of the single launch when that sequence is faster.
 * cache_path (may be NULL): a text file of "size-class variant variant" lines
 * consulted first and appended to (batches of one class).  choice[2] (may be
 * NULL) receives the picked variants (the single launch's pair variant). */
int sim_autotune(sim_handle *h, int32_t reps, const char *cache_path, int32_t *choice);
/* The batch's size classes: returns their number and writes, for k < cap,
 * info[5k .. 5k+4] = {round(log2 atoms per trial), trials, clusters (slot
 * capacity / 8), pair variant used for it, 1 if the class has a launch of its
 * own (0: one launch for the batch)}. */
int32_t sim_tune_classes(sim_handle *h, int32_t *info, int32_t cap);
/* One pair launch per size class from now on, class k with variants[k]
 * (n = the number of classes).  SIM_EINVAL for a wrong n or variant. */
int sim_set_class_variants(sim_handle *h, const int32_t *variants, int32_t n);
/* Sets the launch shapes directly (the numbering of sim_autotune), e.g. to
 * test one of them.  SIM_EINVAL for a variant out of range. */
int sim_set_variants(sim_handle *h, int32_t pair_variant, int32_t cv_variant);

/* Form of a step.  mode 0: one kernel per phase (update, rebuild decision,
 * list rebuilds, pair forces, bonded forces and the reaction coordinate on a
 * second stream, finaliser), CUDA-graph replays of nstlist-step chunks;
 * mode 1: one cooperative kernel per step (every phase of every trial; grid
 * barriers between phases, each polling a bounded number of times: when one
 * gives up the call returns SIM_ETIMEOUT and the step is incomplete; the
 * environment variable VPATH_SPIN_LIMIT, read at sim_create, sets the bound
 * for fault-injection tests), for batches too small to fill the GPU;
 * mode 2: as mode 0, but in the captured chunks the column sort and the
 * list build of a step sit in conditional graph nodes that the rebuild
 * front opens only when some trial rebuilds in that step (small batches,
 * where most steps rebuild nothing and those launches are pure latency).
 * All forms give bit-identical states.  SIM_EINVAL for another mode, and
 * for mode 1 when the batch has more than 16 distinct LJ types.
 * sim_step_mode returns the current form.  sim_autotune_step times reps
 * chunks of nstlist steps in each form the batch can take, keeps the fastest
 * (*mode, may be NULL; ms_per_step[SIM_STEP_MODES], may be NULL, receives
 * every form's milliseconds per step, indexed by mode, -1 for a form not
 * timed) and restores the state it started from (positions, velocities, z_m,
 * Phi, step counter; the lists are rebuilt). */
#define SIM_STEP_MODES 3
int sim_set_step_mode(sim_handle *h, int32_t mode);
int32_t sim_step_mode(const sim_handle *h);
int sim_autotune_step(sim_handle *h, int32_t reps, int32_t *mode, double *ms_per_step);

/* Kernel timing.  on = 1: the next sim_step_batch calls launch kernels
 * directly and time each launch with CUDA events on the library stream.
 * on = 2: the steps still run as CUDA-graph replays, and the chunk graph is
 * captured with external event-record nodes around each pair-kernel launch;
 * their durations are read after every replay (a call of several chunks
 * synchronises between them) and reported as "pair_in_graph".  on = 0: off
 * (the graph is captured again without the event nodes).  SIM_EINVAL for
 * other values.  sim_kernel_times fills up to cap entries of names (static
 * strings), total milliseconds and launch counts, returns the number of
 * kernels, and resets the accumulators. */
int sim_set_timing(sim_handle *h, int32_t on);
int sim_kernel_times(sim_handle *h, const char **names, double *ms, int64_t *counts, int32_t cap);

/* The counter-based noise as the integrator draws it, for atoms 0..n-1 of a
 * trial with the given seed at one step and stream (0: Langevin noise,
 * 1: initial velocities): raw[4n] Philox4x32-10 outputs for counter
 * (atom, step_lo, step_hi, stream) and key (seed_lo, seed_hi), normals[3n]
 * the FP32 Box-Muller normals widened to double.  Either output may be NULL.
 * Runs on the current device; allocates and frees its own scratch. */
int sim_philox_normals(uint64_t seed, int64_t step, uint32_t stream, int32_t n, uint32_t *raw, double *normals);

/* Reaction coordinate z and its gradient for one configuration, allocating
 * no device memory (the paper has no counterpart: this serves callers that
 * must not allocate -- a host program whose device memory belongs to another
 * allocator or a fixed budget, or a latency-critical path that cannot accept
 * the device-wide synchronisation cudaMalloc/cudaFree may cause).
 * Same z and gradient as the batched path (SM "Collective coordinate"), with
 * the native contact map evaluated on the fly.
 *   d_pos [3*n_cv] FP32 and d_native [3*n_cv] FP64: DEVICE pointers, read;
 *   box: cubic side (rounded to FP32); params: cv_r0, cv_r_switch, cv_r_cut
 *   and cv_min_sep are read (host pointer);
 *   d_z [1] and d_grad [3*n_cv]: DEVICE pointers, written (FP64);
 *   cuda_stream: the stream the three launches go to (NULL: legacy stream);
 *     the call returns after queueing them -- synchronise before reading;
 *   errbuf/errlen: optional host buffer for a message.
 * Scratch lives in a static device array of fixed size (112 KiB, held by every
 * GPU that loads the library until exit): n_cv above 2048 is rejected with
 * SIM_EINVAL.  The first call on a device looks the array up on that device
 * (do it before any stream capture there).  Calls share the array: calls that
 * overlap on the GPU race.  Returns SIM_OK, SIM_EINVAL (also for
 * cv_r_switch <= 0, cv_r_cut <= cv_r_switch or cv_min_sep < 0) or SIM_ECUDA
 * (also, before anything is launched, when an earlier CUDA error is pending
 * on the calling thread; the message names it). */
int cv_eval_noalloc(const float *d_pos, const double *d_native, int32_t n_cv, double box, const sim_params *params,
                    double *d_z, double *d_grad, void *cuda_stream, char *errbuf, int32_t errlen);

/* ------------------------------------------------------------------------
 * Order of native-contact formation and path similarity (Sec. "Results":
 * the matrix M of the order in which native contacts form along a path, and
 * s(k, k') = (1/(Nc (Nc - 1))) sum_{i != j} [M_ij(k) = M_ij(k')]).
 * A contact (i, j) of reaction-coordinate atoms (j - i > cv_min_sep) is
 * formed when C(r) = (1 - (r/r0)^6)/(1 - (r/r0)^10) > 1/2 (r0 = cv_r0, minimum
 * image; decided in FP64 on the FP32 positions); native contacts are those
 * formed in the native structure (Euclidean distances), listed by i then j.
 * The formation time of a native contact is the step from which it has
 * stayed formed, -1 when it is not formed at the last check; M_ij = 1, 0 or
 * 1/2 as t_i <, > or = t_j, with -1 ordered after every step.
 * ------------------------------------------------------------------------ */

/* Tracks formation times in every trial, checking after each step whose
 * number is a multiple of every (>= 1); 0 stops tracking.  Each call restarts
 * all times at -1.  The first call builds the native contact lists.
 * SIM_EINVAL for every < 0. */
int sim_contact_tracking(sim_handle *h, int32_t every);

/* Native contacts of a trial's system: *n_contacts receives their number and
 * pairs[2*cap] the first cap of them (i, j).  Builds the lists if needed. */
int sim_native_contacts(sim_handle *h, int32_t trial, int32_t *pairs, int64_t cap, int64_t *n_contacts);

/* Formation times (steps, -1: not formed) of a trial's native contacts, in
 * the order of sim_native_contacts; the first cap are written.  SIM_EINVAL if
 * tracking was never enabled. */
int sim_contact_times(sim_handle *h, int32_t trial, int64_t *times, int64_t cap);

/* Path similarity on the GPU: times [n_paths][n_c] formation times (HOST,
 * read; a negative time: not formed, ordered after every formed contact),
 * pairs [2*n_pairs] path indices (HOST), s [n_pairs] (HOST, written):
 * s(pairs[2q], pairs[2q+1]).  Only the order of the times within a path
 * enters s, so the host replaces them by dense ranks.  A path pair whose
 * paths hold K_a and K_b distinct times with K_a K_b <= 4096 is counted from
 * the joint histogram of its ranks (every pair of contacts in one cell ties
 * in both paths, pairs of cells strictly below-left / above-right are
 * concordant); other pairs compare all ordered contact pairs.  Both counts
 * are exact.  n_c < 2 gives 1 (no ordered pair); n_c <= 2^30.  At most 65535
 * pairs per call.  Returns SIM_OK, SIM_EINVAL or SIM_ECUDA. */
int path_similarity(const int64_t *times, int32_t n_paths, int64_t n_c, const int32_t *pairs, int32_t n_pairs,
                    double *s, void *cuda_stream, char *errbuf, int32_t errlen);

/* ------------------------------------------------------------------------
 * Two-dimensional toy model (SM, "Illustrative Application in a Toy Model").
 * One particle of mass m on
 *   U(x,y) = w^2 (x^2+y^2)^2 - A1 s1^p/(x^2+y^2+s1^2)^2 + A2 s2^p/(x^2+y^2+s2^2)^2
 *            - A3 s3^p/((x-xm)^2+(y-ym)^2+s3^2)^2
 * (the section prints p = 2; p = 4 gives each term the amplitude A at its
 * centre and the ring barrier and gate the section describes), underdamped
 * Langevin dynamics (Eq. Lang, BAOAB as on the atomistic path), started at
 * (x0, y0) with a Maxwell-Boltzmann velocity (Philox stream 1, step 0), with
 * one of three biases on z = sqrt(x^2 + y^2):
 *   TOY2D_NONE     plain Langevin;
 *   TOY2D_RATCHET  Eq. VR: F = -(k/2)(z - z_m) grad z when z > z_m, z_m the
 *                  running minimum of z (z_m(0) = z(x0, y0));
 *   TOY2D_STEERED  the section's steered-MD comparison: F = -k z grad z.
 * A trial stops at its first step with z <= z_product; the functional of
 * Eq. VMDcondition, Phi = sum dt |F_bias|^2 / (gamma m) over its force
 * evaluations, is accumulated up to and including that step.
 * ------------------------------------------------------------------------ */
enum { TOY2D_NONE = 0, TOY2D_RATCHET = 1, TOY2D_STEERED = 2 };

typedef struct {
  double A1, A2, A3, s1, s2, s3, w, xm, ym; /* potential */
  double mass, gamma, kT, dt;                /* Langevin (kT in the potential's units) */
  double x0, y0;                             /* start */
  double z_product;                          /* product reached when z <= z_product */
  int32_t bias;                              /* TOY2D_* */
  int32_t s_power;                           /* p: 2 or 4 */
} toy2d_params;

/* Runs n_trials independent trials of n_steps steps on the GPU (one thread
 * per trial, FP64 without contraction).  All pointers are HOST pointers:
 *   k[n_trials]      bias strength of each trial (ignored for TOY2D_NONE);
 *   seeds[n_trials]  Philox key of each trial (noise counter (0, step, 0|1));
 *   state[4*n_trials] (x, y, vx, vy) at each trial's end (may be NULL);
 *   phi[n_trials]    the functional; passage[n_trials] first-passage step or -1;
 *   path             may be NULL; else [n_trials][n_steps/path_every + 1][2]:
 *                    (x, y) at steps 0, path_every, 2 path_every, ... up to
 *                    the trial's end, NaN after it.
 * cuda_stream: the stream used (NULL: legacy); the call returns when the
 * results are on the host.  Device scratch is allocated and freed per call.
 * Returns SIM_OK, SIM_EINVAL (null pointer, negative size, unknown bias,
 * s_power not 2 or 4, m or dt <= 0, gamma or kT < 0, gamma = 0 with a bias)
 * or SIM_ECUDA; errbuf/errlen (may be NULL/0) receive a message. */
int toy2d_run(const toy2d_params *p, int32_t n_trials, const double *k, const uint64_t *seeds, int64_t n_steps,
              double *state, double *phi, int64_t *passage, double *path, int32_t path_every, void *cuda_stream,
              char *errbuf, int32_t errlen);

/* The cudaStream_t the library launches on. */
void *sim_stream(sim_handle *h);

void sim_destroy(sim_handle *h);
const char *sim_last_error(const sim_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* VPATH_H */

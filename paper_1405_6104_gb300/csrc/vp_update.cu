// vp_update.cu -- the Langevin update (Eq. Lang, BAOAB splitting) with the
// ratchet force applied, initial velocities, state transfer and small
// reductions.
//
// Step n -> n+1 of BAOAB:  v += dt/2 F/m;  x += dt/2 v;  v = c1 v + c2 sqrt(kT/m) xi;
// x += dt/2 v;  F = F(x);  v += dt/2 F/m.   Within a call the closing half
// kick of one step and the opening half kick of the next are one kick of
// dt (the device scalar `kick` is 0.5 at the first step of a call and 1.0
// afterwards); a final half kick (UPD_FINAL) closes the call.
#include "vp_dev.cuh"
#include "vp_update_dev.cuh"

namespace vp {



// Six blocks per SM (40 registers: with 32 the list buffer's reference
// position, one more early load, spills): the kernel waits on memory round
// trips and needs every resident warp it can get.
template <int MODE>
__global__ void __launch_bounds__(256, 6) k_update(Dev d, SimConst c) {
  update_slot<MODE>(d, c, blockIdx.x * blockDim.x + threadIdx.x);
}

// Maxwell-Boltzmann velocities (Philox stream 1, step 0) with the centre of
// mass at rest; one block per trial, only trials with need[t] != 0
__global__ void __launch_bounds__(256) k_init_vel(Dev d, float kT, const int32_t *need) {
  __shared__ double red[4][256];
  const int t = blockIdx.x;
  if (!need[t]) return;
  const TrialInfo T = d.tinfo[t];
  double px = 0, py = 0, pz = 0, m = 0;
  for (int o = threadIdx.x; o < T.n_atoms; o += blockDim.x) {
    const AtomSys as = d.asys[T.sysatom0 + o];
    const float3 g = normal3(T.key0, T.key1, (uint32_t)o, 0ull, 1u);
    const double mass = 1.0 / (double)as.invm;
    const double sd = sqrt((double)kT / mass);
    px += mass * sd * g.x; py += mass * sd * g.y; pz += mass * sd * g.z; m += mass;
  }
  red[0][threadIdx.x] = px; red[1][threadIdx.x] = py; red[2][threadIdx.x] = pz; red[3][threadIdx.x] = m;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + off];
    __syncthreads();
  }
  const double vx0 = red[0][0] / red[3][0], vy0 = red[1][0] / red[3][0], vz0 = red[2][0] / red[3][0];
  for (int o = threadIdx.x; o < T.n_atoms; o += blockDim.x) {
    const AtomSys as = d.asys[T.sysatom0 + o];
    const float3 g = normal3(T.key0, T.key1, (uint32_t)o, 0ull, 1u);
    const double sd = sqrt((double)kT * (double)as.invm);
    const int s = d.slot_of[T.atom0 + o];
    float4 v = d.vel[s];
    v.x = (float)(sd * g.x - vx0); v.y = (float)(sd * g.y - vy0); v.z = (float)(sd * g.z - vz0);
    d.vel[s] = v;
  }
}

// caller-ordered double arrays <-> slots of one trial (or all trials: trial < 0)
__global__ void k_scatter_state(Dev d, int trial, const double *pos, const double *vel, int n) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int t = trial, o = k, base = 0;
  if (trial < 0) {  // all trials: find the trial of global index k (trials are contiguous)
    int lo = 0, hi = d.n_trials - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (d.tinfo[mid].atom0 <= k) lo = mid; else hi = mid - 1;
    }
    t = lo;
    o = k - d.tinfo[t].atom0;
    base = d.tinfo[t].atom0;
  }
  const TrialInfo &T = d.tinfo[t];
  const int s = d.slot_of[T.atom0 + o];
  float4 p = d.pos[s], v = d.vel[s];
  const size_t q = (size_t)(base + o) * 3;
  p.x = (float)pos[q]; p.y = (float)pos[q + 1]; p.z = (float)pos[q + 2];
  v.x = (float)vel[q]; v.y = (float)vel[q + 1]; v.z = (float)vel[q + 2];
  d.pos[s] = p;
  d.vel[s] = v;
}

// flag = 1 if any of the n values is not finite (the caller's state is
// checked on the device before it replaces the current one)
__global__ void k_check_finite(const double *x, size_t n, int *flag) {
  bool bad = false;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[k]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void k_gather_state(Dev d, int trial, double *pos, double *vel, int n) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const TrialInfo &T = d.tinfo[trial];
  const int s = d.slot_of[T.atom0 + o];
  const float4 p = d.pos[s], v = d.vel[s];
  if (pos) { pos[3 * o] = p.x; pos[3 * o + 1] = p.y; pos[3 * o + 2] = p.z; }
  if (vel) { vel[3 * o] = v.x; vel[3 * o + 1] = v.y; vel[3 * o + 2] = v.z; }
}

// total force (accumulated pair + bonded, plus the ratchet force) in FP64
__global__ void k_forces_out(Dev d, SimConst c, int trial, double *out, int n) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const TrialInfo &T = d.tinfo[trial];
  const int s = d.slot_of[T.atom0 + o];
  const double sc = 2.3283064365386963e-10;
  double F[3] = {(double)d.fx[s] * sc, (double)d.fy[s] * sc, (double)d.fz[s] * sc};
  if (o < T.n_cv) {
    const double k = -c.kR_half_d * d.tstate[trial].a * sc;
    F[0] += k * (double)d.gx[T.cv0 + o];
    F[1] += k * (double)d.gy[T.cv0 + o];
    F[2] += k * (double)d.gz[T.cv0 + o];
  }
  out[3 * o] = F[0]; out[3 * o + 1] = F[1]; out[3 * o + 2] = F[2];
}

// Positions of every trial from a device array (trials concatenated, caller
// order, FP64; velocities untouched).  An atom farther than the list buffer
// allows from where its trial's list was built requests a rebuild of that
// list in the current step.
__global__ void k_scatter_positions(Dev d, SimConst c, const double *pos, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int lo = 0, hi = d.n_trials - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d.tinfo[mid].atom0 <= k) lo = mid; else hi = mid - 1;
  }
  const int t = lo;
  const int s = d.slot_of[k];
  float4 p = d.pos[s];
  p.x = (float)pos[3 * (size_t)k];
  p.y = (float)pos[3 * (size_t)k + 1];
  p.z = (float)pos[3 * (size_t)k + 2];
  d.pos[s] = p;
  const float4 r = d.ref_slot[s];
  const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
  if (c.list_fixed || !(dx * dx + dy * dy + dz * dz <= c.trig2)) d.rb[t] = (uint32_t)*d.cur_step;
}

// potential energy (LJ + RF + bonds + angles) and -grad U of every trial into
// device arrays: energy[t], forces [trials concatenated][3] (FP64)
// (NaN energies when a device error flag is up: a list overflow or a
// non-finite state in the evaluation)
__global__ void k_potential_out(Dev d, double *energy, double *forces, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < d.n_trials && energy) {
    const long long *e = d.energy + (size_t)k * 5;
    energy[k] = *d.err ? __longlong_as_double(0x7ff8000000000000LL)
                       : ((double)e[0] + (double)e[1] + (double)e[2] + (double)e[3]) / E_SCALE;
  }
  if (k >= n || !forces) return;
  const int s = d.slot_of[k];
  const double sc = 2.3283064365386963e-10;
  forces[3 * (size_t)k] = (double)d.fx[s] * sc;
  forces[3 * (size_t)k + 1] = (double)d.fy[s] * sc;
  forces[3 * (size_t)k + 2] = (double)d.fz[s] * sc;
}

__global__ void k_kinetic(Dev d, int trial) {
  __shared__ double red[256];
  const TrialInfo T = d.tinfo[trial];
  double e = 0.0;
  for (int o = threadIdx.x; o < T.n_atoms; o += blockDim.x) {
    const float4 v = d.vel[d.slot_of[T.atom0 + o]];
    e += 0.5 * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z) / (double)v.w;
  }
  red[threadIdx.x] = e;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) d.energy[(size_t)trial * 5 + 4] = __double2ll_rn(red[0] * E_SCALE);
}

// atom pairs held by the cluster lists of one trial (caller's indices, i < j)
__global__ void k_extract_pairs(Dev d, int list_cap, int trial, int32_t *pairs, long long cap,
                                unsigned long long *count) {
  const TrialInfo T = d.tinfo[trial];
  const int Il = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (Il >= d.tstate[trial].n_clus) return;
  const int I = T.clus0 + Il;
  const int n = d.list_n[I];
  for (int e = lane; e < n; e += 32) {
    const uint32_t ent = d.list[(size_t)I * list_cap + e];
    const unsigned m = d.list_m[(size_t)I * list_cap + e];
    const int oj = d.orig[(int)(ent & J_MASK)];
    for (int a = 0; a < CL; ++a) {
      if (!((m >> a) & 1u)) continue;
      const int oi = d.orig[I * CL + a];
      unsigned long long k = atomicAdd(count, 1ull);
      if ((long long)k < cap) {
        pairs[2 * k] = min(oi, oj);
        pairs[2 * k + 1] = max(oi, oj);
      }
    }
  }
}

// argmin of Phi over trials with z <= z_max (z_max < 0: all), lowest index on ties
__global__ void k_select(Dev d, double z_max, double *phi_out, int32_t *argmin_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int best = -1;
  double bv = 0.0;
  for (int t = 0; t < d.n_trials; ++t) {
    const TrialState &S = d.tstate[t];
    phi_out[t] = S.Phi;
    if (z_max >= 0.0 && !(S.z <= z_max)) continue;
    if (best < 0 || S.Phi < bv) { best = t; bv = S.Phi; }
  }
  *argmin_out = best;
}

__global__ void k_philox_normals(uint32_t k0, uint32_t k1, unsigned long long step, uint32_t stream, int n,
                                 uint32_t *raw, double *normals) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  uint4 x = philox4x32_10(make_uint4((uint32_t)o, (uint32_t)step, (uint32_t)(step >> 32), stream), k0, k1);
  raw[4 * o] = x.x; raw[4 * o + 1] = x.y; raw[4 * o + 2] = x.z; raw[4 * o + 3] = x.w;
  float3 g = normal3(k0, k1, (uint32_t)o, step, stream);
  normals[3 * o] = g.x; normals[3 * o + 1] = g.y; normals[3 * o + 2] = g.z;
}

void launch_philox_normals(uint64_t seed, unsigned long long step, uint32_t stream, int n, uint32_t *raw,
                           double *normals, cudaStream_t s) {
  if (n > 0)
    k_philox_normals<<<(n + 255) / 256, 256, 0, s>>>((uint32_t)seed, (uint32_t)(seed >> 32), step, stream, n, raw,
                                                      normals);
}

void launch_update(const Dev &d, const SimConst &c, UpdateMode mode, cudaStream_t s) {
  unsigned blocks = (unsigned)((d.total_slots + 255) / 256);
  if (mode == UPD_DRIFT) {
    k_update<UPD_DRIFT><<<blocks, 256, 0, s>>>(d, c);
  } else {
    k_update<UPD_FINAL><<<blocks, 256, 0, s>>>(d, c);
  }
}
void launch_init_vel(const Dev &d, float kT, const int32_t *need, cudaStream_t s) {
  k_init_vel<<<d.n_trials, 256, 0, s>>>(d, kT, need);
}
void launch_scatter_state(const Dev &d, int32_t trial, const double *pos, const double *vel, int32_t n,
                          cudaStream_t s) {
  if (n > 0) k_scatter_state<<<(n + 255) / 256, 256, 0, s>>>(d, trial, pos, vel, n);
}
void launch_check_finite(const double *x, size_t n, int *flag, cudaStream_t s) {
  if (n > 0) k_check_finite<<<4 * 152, 256, 0, s>>>(x, n, flag);
}
void launch_gather_state(const Dev &d, int32_t trial, double *pos, double *vel, int32_t n, cudaStream_t s) {
  if (n > 0) k_gather_state<<<(n + 255) / 256, 256, 0, s>>>(d, trial, pos, vel, n);
}
void launch_forces_out(const Dev &d, const SimConst &c, int32_t trial, double *out, int32_t n, cudaStream_t s) {
  if (n > 0) k_forces_out<<<(n + 255) / 256, 256, 0, s>>>(d, c, trial, out, n);
}
void launch_kinetic(const Dev &d, int32_t trial, cudaStream_t s) { k_kinetic<<<1, 256, 0, s>>>(d, trial); }
void launch_scatter_positions(const Dev &d, const SimConst &c, const double *pos, int32_t n, cudaStream_t s) {
  if (n > 0) k_scatter_positions<<<(n + 255) / 256, 256, 0, s>>>(d, c, pos, n);
}
void launch_potential_out(const Dev &d, double *energy, double *forces, int32_t n, cudaStream_t s) {
  const int m = n > d.n_trials ? n : d.n_trials;
  if (m > 0) k_potential_out<<<(m + 255) / 256, 256, 0, s>>>(d, energy, forces, n);
}
void launch_extract_pairs(const Dev &d, int32_t list_cap, int32_t trial, int32_t n_clus, int32_t *pairs,
                          long long cap, unsigned long long *count, cudaStream_t s) {
  if (n_clus > 0) k_extract_pairs<<<(n_clus + 3) / 4, 128, 0, s>>>(d, list_cap, trial, pairs, cap, count);
}
void launch_select(const Dev &d, double z_max, double *phi_out, int32_t *argmin_out, cudaStream_t s) {
  k_select<<<1, 32, 0, s>>>(d, z_max, phi_out, argmin_out);
}

}  // namespace vp

// vp_internal.cuh -- device data layout and helpers shared by the kernels of
// the trial-path generator.  Host launchers for every kernel are declared at
// the end; vp_capi.cu drives them.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vp {

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------
constexpr double KB = 0.0083144626;    // kJ/mol/K
constexpr double FCOUL = 138.935458;   // kJ mol^-1 nm e^-2
constexpr int CL = 8;                  // atoms per i-cluster
constexpr int CJ = 4;                  // atoms per j-cluster (half an i-cluster)
constexpr int ZBINS = 16;             // z-bins of the per-column half table the list build searches
constexpr int MAX_TRIALS = 65535;      // trials per batch (one grid row each in the per-trial kernels)
constexpr int MAX_EXCL = 16;           // excluded partners per atom
constexpr int MAX_TYPES = 64;          // distinct LJ types after de-duplication
constexpr int SMALL_TYPES = 16;        // at most this many: the per-warp LJ tables of the shared-memory
                                       // pair kernels and of the one-kernel step
constexpr int COL_CAP = 1024;          // atoms per grid column
constexpr float FX_SCALE = 4294967296.0f;        // fixed point: 2^32 units per kJ/mol/nm
constexpr float FX_INV = 2.3283064365386963e-10f;  // 2^-32
constexpr double E_SCALE = 16777216.0;            // energies: 2^24 units per kJ/mol
constexpr int CV_T = 32;               // CV tile edge (atoms)

// error flag bits (device int32)
constexpr int ERR_LIST = 1;
constexpr int ERR_COL = 2;
constexpr int ERR_NONFINITE = 4;
constexpr int ERR_CAPACITY = 8;
constexpr int ERR_SKIN = 16;
constexpr int ERR_TIMEOUT = 32;        // a bounded grid barrier of the one-kernel step gave up

// list entry of an 8-atom i-cluster: one j-atom, with at least one of the
// eight pairs in the list --
//   word (uint32) = j slot (bits 0-24) | image shift (bits 25-30: nx+1,
//       ny+1, nz+1, two bits each; x_j image = x_j - L n) | E_EXACT (bit 31)
//       when the j-atom's pairs do not share one image (the kernel then
//       takes the minimum image pair by pair)
//   mask (uint8, a parallel array): bit a set when i-atom a and the j-atom
//       satisfy the FP32 list rule, are not excluded, are real atoms and
//       (inside the i-cluster itself) the j slot follows a's -- the Verlet
//       list proper.
// The list build works on 4-atom j-clusters (the same fields, the j-cluster
// index in bits 0-24 and a 32-bit mask, bit a*4 + b for j-atom b) and then
// writes one entry per j-atom whose mask column is not empty: the entries
// whose masks the pair kernels must apply (exclusions, the cluster itself,
// mixed images) first, the others after them.
constexpr uint32_t J_BITS = 25;
constexpr int LIST_CAP = 2048;         // j-atom entries per i-cluster
constexpr uint32_t J_MASK = (1u << J_BITS) - 1u;
constexpr uint32_t E_EXACT = 1u << 31;
// image code of no shift ((0+1) | (0+1) << 2 | (0+1) << 4)
constexpr uint32_t NO_SHIFT = 21u;

// Padding slots sit far outside every box, on distinct points 64 nm apart,
// so that no pair involving one can fall inside the cut-off (boxes < 60 nm).
__host__ __device__ __forceinline__ float4 pad_pos(int slot) {
  return make_float4(1.0e6f + 64.0f * (float)(slot & 0xffff), 1.0e6f + 64.0f * (float)((slot >> 16) & 0xffff),
                     1.0e6f, 0.0f);
}
// stand-in j-atom for idle lanes: far from every real and padding slot
__host__ __device__ __forceinline__ float4 idle_pos() { return make_float4(1.0e6f, 1.0e6f, 3.0e6f, 0.0f); }

// ---------------------------------------------------------------------------
// per-trial static description (device copy, read-only after create)
// ---------------------------------------------------------------------------
struct TrialInfo {
  int32_t sys;
  int32_t atom0;       // per-trial, caller-ordered arrays: [atom0 + orig]
  int32_t sysatom0;    // per-system, caller-ordered arrays: [sysatom0 + orig]
  int32_t n_atoms, n_cv;
  int32_t slot0;       // first slot of the trial (multiple of 8)
  int32_t clus0;       // first i-cluster = slot0 / 8
  int32_t max_clus;    // slot capacity / 8
  int32_t ncol, col0;  // grid columns [col0, col0 + ncol*ncol)
  int32_t cv0;         // CV gradient accumulators [cv0 + i], i < n_cv
  int32_t work0, n_work;  // CV work items of this trial in the flat work list
  int32_t systile0;    // first CV tile of the system
  float box, inv_box, col_w, inv_col_w;
  uint32_t key0, key1; // Philox key (trial seed)
  long long noise_off; // the noise of step n uses the counter n + noise_off (0 unless set)
};

struct TrialState {
  int32_t n_clus;      // i-clusters in use
  int32_t pad_;
  double z, zm, a, Phi, phi;
  double zconst;       // sum of C~_nat^2 over the trial's contact pairs
};

// per-system, caller-ordered atom data
struct AtomSys {
  float invm, c1, c2sd, qs;   // 1/m, exp(-gamma dt), sqrt((1-c1^2) kT/m), q*sqrt(f)
};

// owner-computes bonded term of one atom
struct BTerm {
  int32_t kind;   // 0 bond, 1 angle end, 2 angle vertex
  int32_t p1, p2; // bond: partner; end: vertex, other end; vertex: the two ends
  float x0, k;    // r0 or theta0, force constant
};

// a group of bonded terms over at most 3 atoms (one thread each): the terms'
// forces are summed per atom in fixed point before one reduction per atom
// and component.  code[k] of term k < n: bit 0 kind (0 bond, 1 angle), bits
// 1-2, 3-4, 5-6 the local atoms i, j, l (bond i-j; angle i-j-l, j the vertex)
struct __align__(16) BGroup {
  int32_t at[3];   // system atoms (at[2] = -1 for a two-atom group)
  int32_t n;       // terms, 1..3
  int32_t code[3];
  int32_t pad;
  float4 par[3];   // {r0 or theta0, force constant, r0 - x (a bond's rest length in float-float:
                   //  k (r - r0) with k ~ 1e5 needs it), 0}
};

struct SimConst {
  float dt, half_dt;
  float rc2;          // r_cut^2
  float rl2;          // list radius^2 as the FP32 list rule uses it
  float two_krf;      // 2 k_rf
  float krf, crf;     // reaction-field constants (energies)
  float kR_half;      // k_R / 2
  double dt_d, kR_half_d;
  int32_t n_types;
  int32_t list_cap;   // j-atom entries per i-cluster
  float cv_inv_r0sq_hi, cv_inv_r0sq_lo;   // 1/r0^2 as float-float
  float cv_rs_hi, cv_rs_lo;               // switching start as float-float
  float cv_inv_w_hi, cv_inv_w_lo;         // 1/(r_cut^cv - r_switch) as float-float
  float cv_rs2, cv_rc2_far;   // switching start^2, far threshold on r^2
  double cv_r0_d, cv_rs_d, cv_rc_d;
  int32_t cv_min_sep;
  int32_t rec_cap;
  int32_t uniform_gamma;      // every atom of every system has the same friction
  float c1_u, c2sqkT_u;       // then exp(-gamma dt) and sqrt((1 - c1^2) kT)
  // list rebuilds: at most nstlist steps apart; unless list_fixed, also in
  // the first step in which an atom of the trial has moved farther than
  // skin/2 - 1e-5 nm (squared: trig2) from where its list was built
  int32_t nstlist, list_fixed;
  float trig2;
  uint32_t spin_limit;        // polls of a grid barrier before it gives up (one-kernel step)
};



// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// three normals from (key, atom, step, stream): uniforms ((x>>9)+1/2) 2^-23
// (exact in FP32), Box-Muller on (u0,u1) and (u2,u3)
__device__ __forceinline__ float3 normal3(uint32_t k0, uint32_t k1, uint32_t atom, uint64_t step, uint32_t stream) {
  uint4 x = philox4x32_10(make_uint4(atom, (uint32_t)step, (uint32_t)(step >> 32), stream), k0, k1);
  const float s23 = 1.1920928955078125e-07f;
  float u0 = ((float)(x.x >> 9) + 0.5f) * s23, u1 = ((float)(x.y >> 9) + 0.5f) * s23;
  float u2 = ((float)(x.z >> 9) + 0.5f) * s23, u3 = ((float)(x.w >> 9) + 0.5f) * s23;
  float r01 = sqrtf(-2.0f * logf(u0)), r23 = sqrtf(-2.0f * logf(u2));
  float s1, c1;
  sincospif(2.0f * u1, &s1, &c1);
  return make_float3(r01 * c1, r01 * s1, r23 * cospif(2.0f * u3));
}

// ---------------------------------------------------------------------------
// fixed point
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long fx_from(float f) { return __float2ll_rn(f * FX_SCALE); }
__device__ __forceinline__ float fx_to(long long v) { return __ll2float_rn(v) * FX_INV; }
__device__ __forceinline__ void red_add(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// ---------------------------------------------------------------------------
// float-float (double-single) arithmetic on the FP32 pipes: Knuth's TwoSum,
// FMA-based TwoProduct (Ogita, Rump, Oishi 2005), Dekker-style products and
// quotients.  A value is hi + lo with |lo| <= ulp(hi)/2.
// ---------------------------------------------------------------------------
struct ff { float hi, lo; };

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// sum with one TwoSum of the leading parts and the trailing parts added in
// FP32 (the "sloppy" double-single sum): relative error about 2^-44 without
// cancellation, absolute error below ulp(max(|x|, |y|)) * 2^-22 with it --
// ample for sums whose required accuracy is absolute (z to ~1e-9 per term)
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_add_f(ff x, float y) {
  ff s = two_sum(x.hi, y);
  s.lo = __fadd_rn(s.lo, x.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  ff p = two_prod(x.hi, y.hi);
  p.lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff x, float y) {
  ff p = two_prod(x.hi, y);
  p.lo = __fmaf_rn(x.lo, y, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_sqr(ff x) {
  ff p = two_prod(x.hi, x.hi);
  p.lo = __fmaf_rn(2.0f * x.hi, x.lo, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// quotient: q1 = x/y to float, remainder x - q1 y in float-float, q2 = r/y
__device__ __forceinline__ ff ff_div(ff x, ff y) {
  float q1 = __fdividef(x.hi, y.hi);
  ff r = ff_add(x, ff_neg(ff_mul_f(y, q1)));
  return fast_two_sum(q1, __fdividef(r.hi, y.hi));
}
__device__ __forceinline__ ff ff_sqrt(ff x) {
  float y = sqrtf(x.hi);
  ff yy = two_prod(y, y);
  ff r = ff_add(x, ff_neg(yy));
  return fast_two_sum(y, __fdividef(r.hi, 2.0f * y));
}
__device__ __forceinline__ double ff_to_d(ff x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ ff ff_from_d(double d) {
  float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}

// exact difference of two floats as float-float
__device__ __forceinline__ ff ff_diff(float a, float b) { return two_sum(a, -b); }

}  // namespace vp

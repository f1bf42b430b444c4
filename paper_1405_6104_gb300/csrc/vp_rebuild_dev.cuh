// vp_rebuild_dev.cuh -- device functions of the list rebuild (binning,
// column scan, bucket fill, column sort, cluster-pair list of one i-cluster),
// shared by the separate kernels and the one-kernel step.  The binning stages
// each live atom (wrapped position, velocity, type, index) in the sort
// buffers; the column sort writes the new layout from there into the arrays.
#pragma once
#include <cooperative_groups.h>

#include "vp_dev.cuh"

namespace vp {

// Slot `slot` of trial t, its position p already loaded (live: the slot
// holds an atom): wrapped into the box, its grid column picked and recorded
// in slot_col; returns the trial's column offset plus the column (the index
// into the per-column arrays), or -1 for a slot without an atom.
__device__ __forceinline__ int bin_loaded(const Dev &d, const SimConst &c, const TrialInfo &T, float half_skin2,
                                          int strict, int t, int slot, bool live, int o, float4 p,
                                          unsigned long long n) {
  if (!live) { d.slot_col[slot] = -1; return -1; }
  // the slot's atom is staged in the sort buffers (the column sort reads it
  // there and writes the new layout straight into the arrays themselves)
  d.vel_b[slot] = d.vel[slot];
  d.type_b[slot] = d.type[slot];
  d.orig_b[slot] = o;
  const float L = T.box, iL = T.inv_box;
  if (c.list_fixed && d.rb[d.n_trials + t] != (uint32_t)n) {
    // fixed-interval lists: an atom farther than skin/2 from where the list
    // was built may have left pairs out (the slot is the one it had then;
    // a forced rebuild follows a new state, not a list interval)
    const float4 r = d.ref_slot[slot];
    const float ddx = p.x - r.x, ddy = p.y - r.y, ddz = p.z - r.z;
    if (ddx * ddx + ddy * ddy + ddz * ddz > half_skin2) {
      atomicAdd(reinterpret_cast<unsigned long long *>(d.diag), 1ull);
      if (strict) atomicOr(d.err, ERR_SKIN);
    }
  }
  float x = p.x - L * floorf(p.x * iL), y = p.y - L * floorf(p.y * iL), z = p.z - L * floorf(p.z * iL);
  x = x >= L ? x - L : (x < 0.0f ? x + L : x);
  y = y >= L ? y - L : (y < 0.0f ? y + L : y);
  z = z >= L ? z - L : (z < 0.0f ? z + L : z);
  z += 0.0f;  // no negative zero in the sort key
  // a coordinate that is not finite, or so large that one wrap cannot bring
  // it into the box (a run that has blown up), is an error; the atom is put
  // at the origin so that every index below stays inside the grid
  if (!(isfinite(x) && isfinite(y) && isfinite(z)) || !(x >= 0.0f && x < L && y >= 0.0f && y < L && z >= 0.0f && z < L)) {
    atomicOr(d.err, ERR_NONFINITE);
    x = y = z = 0.0f;
  }
  d.pos_b[slot] = make_float4(x, y, z, p.w);
  int cx = max(0, min((int)(x * T.inv_col_w), T.ncol - 1));
  int cy = max(0, min((int)(y * T.inv_col_w), T.ncol - 1));
  const int col = cx * T.ncol + cy;
  d.slot_col[slot] = col;
  return T.col0 + col;
}

// the same for slot `local` of the trial (loads included)
__device__ __forceinline__ int bin_slot_col(const Dev &d, const SimConst &c, const TrialInfo &T, float half_skin2,
                                            int strict, int t, int local, int n_clus, unsigned long long n) {
  if (local >= T.max_clus * CL) return -1;
  const int slot = T.slot0 + local;
  const int o = d.orig[slot];
  const bool live = local < n_clus * CL && o >= 0;
  return bin_loaded(d, c, T, half_skin2, strict, t, slot, live, o,
                    live ? d.pos[slot] : make_float4(0.f, 0.f, 0.f, 0.f), n);
}

// ... and counted in its column (global counters)
__device__ __forceinline__ void bin_slot(const Dev &d, const SimConst &c, float half_skin2, int strict, int t,
                                         int local, unsigned long long n) {
  const TrialInfo T = d.tinfo[t];
  const int cg = bin_slot_col(d, c, T, half_skin2, strict, t, local, d.tstate[t].n_clus, n);
  if (cg < 0) return;
  // slots are in column order from the last rebuild, so a warp's atoms fall
  // into one or two columns: one atomic per column and warp
  const unsigned peers = __match_any_sync(__activemask(), cg);
  if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&d.col_count[cg], __popc(peers));
}

// STAMP: record this step as the trial's last rebuild here (the front kernel
// leaves that to the column sort: its blocks still read the stamps to decide)
template <int NT, bool STAMP = true>
__device__ __forceinline__ void colscan_trial(const Dev &d, int (&s_a)[NT], int (&s_c)[NT], int t) {
  const TrialInfo T = d.tinfo[t];
  int nc = T.ncol * T.ncol;
  int per = (nc + NT - 1) / NT;
  int b = threadIdx.x * per, e = min(b + per, nc);
  int sa = 0, sc = 0, bad = 0;
  for (int c = b; c < e; ++c) {
    int n = d.col_count[T.col0 + c];
    bad |= n > COL_CAP;
    sa += n;
    sc += (n + CL - 1) / CL;
  }
  s_a[threadIdx.x] = sa;
  s_c[threadIdx.x] = sc;
  __syncthreads();
  // Hillis-Steele inclusive scan over the thread sums (fixed order)
  for (int off = 1; off < NT; off <<= 1) {
    int va = threadIdx.x >= off ? s_a[threadIdx.x - off] : 0;
    int vc = threadIdx.x >= off ? s_c[threadIdx.x - off] : 0;
    __syncthreads();
    s_a[threadIdx.x] += va;
    s_c[threadIdx.x] += vc;
    __syncthreads();
  }
  int pa = s_a[threadIdx.x] - sa, pc = s_c[threadIdx.x] - sc;
  for (int c = b; c < e; ++c) {
    int n = d.col_count[T.col0 + c];
    d.col_start[T.col0 + c] = pa;
    d.col_cstart[T.col0 + c] = pc;
    d.col_fill[T.col0 + c] = 0;
    pa += n;
    pc += (n + CL - 1) / CL;
  }
  if (bad) atomicOr(d.err, ERR_COL);
  int total = s_c[NT - 1];
  if (total > T.max_clus) {
    if (threadIdx.x == 0) atomicOr(d.err, ERR_CAPACITY);
    total = T.max_clus;
  }
  if (threadIdx.x == NT - 1) {
    d.tstate[t].n_clus = total;
    const uint32_t n32 = (uint32_t)*d.cur_step;
    if (STAMP) d.last_rb[t] = n32;
    atomicAdd(reinterpret_cast<unsigned long long *>(d.diag + 1), 1ull);
    if (d.rb[t] == n32) atomicAdd(reinterpret_cast<unsigned long long *>(d.diag + 2), 1ull);
  }
  // slots past the new clusters become empty (their atoms, if any, are
  // staged in the sort buffers already; the column sort fills the others)
  for (int sl = T.slot0 + total * CL + threadIdx.x; sl < T.slot0 + T.max_clus * CL; sl += NT) {
    const float4 pad = pad_pos(sl);
    d.orig[sl] = -1;
    d.pos[sl] = pad;
    d.ref_slot[sl] = pad;
    d.vel[sl] = make_float4(0.f, 0.f, 0.f, 0.f);
    d.type[sl] = 0;
  }
}

__device__ __forceinline__ void colfill_slot(const Dev &d, int t, int local) {
  const TrialInfo &T = d.tinfo[t];
  if (local >= T.max_clus * CL) return;
  const int slot = T.slot0 + local;
  int c = d.slot_col[slot];
  if (c < 0) return;
  int cg = T.col0 + c;
  // one atomic per column and warp; the lanes of a column take consecutive
  // places (the order inside a bucket is irrelevant: the column sort orders it)
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, cg);
  const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&d.col_fill[cg], __popc(peers));
  base = __shfl_sync(act, base, leader);
  const int p = base + __popc(peers & ((1u << lane) - 1u));
  if (p < COL_CAP && d.col_count[cg] <= COL_CAP) d.bucket[T.atom0 + d.col_start[cg] + p] = slot;
}

// The first part of trial t's rebuild by one thread-block cluster of
// FRONT_CLUSTER blocks of FRONT_THREADS threads, in place of three grid-wide
// kernels: binning (bin_loaded), the column scans (colscan_trial) and the
// bucket fill.  The column counters live in the shared memory of the
// cluster's first block; the others reach them through distributed shared
// memory.  The order inside a column's bucket depends on timing (as with the
// separate kernels), but the column sort orders every column by (z, atom
// index), so the layout is the same.  Each thread issues the loads of
// FRONT_UNROLL slots together.
constexpr int FRONT_THREADS = 1024;
constexpr int FRONT_CLUSTER = 4;
constexpr int FRONT_UNROLL = 4;
constexpr int MAX_COLS = 64 * 64;  // columns per trial (the host caps the grid at 64 x 64)
struct FrontShared {
  int cnt[MAX_COLS];   // atoms per column (used in the cluster's first block)
  int fill[MAX_COLS];  // places taken in each column's bucket (idem)
  int a[FRONT_THREADS], c[FRONT_THREADS];
};

__device__ __forceinline__ void front_trial(const Dev &d, const SimConst &c, float half_skin2, int strict,
                                            FrontShared &sh, int t, unsigned long long n) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  const int rank = (int)cl.block_rank();
  int *cnt0 = cl.map_shared_rank(sh.cnt, 0);
  int *fill0 = cl.map_shared_rank(sh.fill, 0);
  const TrialInfo T = d.tinfo[t];
  const int nc = T.ncol * T.ncol;
  const int n_clus = d.tstate[t].n_clus;
  const int n_slots = T.max_clus * CL;
  constexpr int STRIDE = FRONT_CLUSTER * FRONT_THREADS;
  const int first = rank * FRONT_THREADS + threadIdx.x;
  if (rank == 0)
    for (int k = threadIdx.x; k < nc; k += FRONT_THREADS) {
      sh.cnt[k] = 0;
      sh.fill[k] = 0;
    }
  cl.sync();
  for (int base = first; base < n_slots; base += STRIDE * FRONT_UNROLL) {
    int o[FRONT_UNROLL];
    float4 p[FRONT_UNROLL];
#pragma unroll
    for (int u = 0; u < FRONT_UNROLL; ++u) {
      const int local = base + u * STRIDE;
      o[u] = local < n_slots ? d.orig[T.slot0 + local] : -1;
      p[u] = local < n_slots ? d.pos[T.slot0 + local] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < FRONT_UNROLL; ++u) {
      const int local = base + u * STRIDE;
      if (local < n_slots) {
        const bool live = local < n_clus * CL && o[u] >= 0;
        const int cg = bin_loaded(d, c, T, half_skin2, strict, t, T.slot0 + local, live, o[u], p[u], n);
        if (cg >= 0) {
          const unsigned peers = __match_any_sync(__activemask(), cg);
          if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt0 + (cg - T.col0), __popc(peers));
        }
      }
    }
  }
  cl.sync();
  if (rank == 0) {
    for (int k = threadIdx.x; k < nc; k += FRONT_THREADS) d.col_count[T.col0 + k] = sh.cnt[k];
    __syncthreads();
    colscan_trial<FRONT_THREADS, false>(d, sh.a, sh.c, t);
  }
  cl.sync();  // the column starts are written (release and acquire at cluster scope)
  for (int base = first; base < n_slots; base += STRIDE * FRONT_UNROLL) {
    int col[FRONT_UNROLL];
#pragma unroll
    for (int u = 0; u < FRONT_UNROLL; ++u) {
      const int local = base + u * STRIDE;
      col[u] = local < n_slots ? d.slot_col[T.slot0 + local] : -1;
    }
#pragma unroll
    for (int u = 0; u < FRONT_UNROLL; ++u) {
      if (col[u] >= 0) {
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, col[u]);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        int b = 0;
        if (lane == leader) b = atomicAdd(fill0 + col[u], __popc(peers));
        b = __shfl_sync(act, b, leader);
        const int q = b + __popc(peers & ((1u << lane) - 1u));
        const int cg = T.col0 + col[u];
        if (q < COL_CAP && d.col_count[cg] <= COL_CAP)
          d.bucket[T.atom0 + d.col_start[cg] + q] = T.slot0 + base + u * STRIDE;
      }
    }
  }
  cl.sync();  // the first block's counters stay alive until every block is done with them
}

struct ColsortShared {
  unsigned long long key[COL_CAP];
  int s_old[COL_CAP];
  float s_zlo[COL_CAP / CJ + 2];  // lower z-bound of every half
};


// The column's atoms are read from the sort buffers (staged by the binning:
// the layout before this rebuild) and written in the new order into the
// arrays themselves.  STAMP: the block of column 0 records this step as the
// trial's last rebuild.
template <bool STAMP>
__device__ __forceinline__ void colsort_column(const Dev &d, ColsortShared &sh, int t, int c) {
  unsigned long long *key = sh.key;
  int *s_old = sh.s_old;
  float *s_zlo = sh.s_zlo;
  const TrialInfo T = d.tinfo[t];
  if (c >= T.ncol * T.ncol) return;
  if (STAMP && c == 0 && threadIdx.x == 0) d.last_rb[t] = (uint32_t)*d.cur_step;
  const int cg = T.col0 + c;
  int n = d.col_count[cg];
  __syncthreads();
  // the count is consumed: the column starts from zero at the trial's next rebuild
  if (threadIdx.x == 0) d.col_count[cg] = 0;
  if (n > COL_CAP) return;  // flagged by k_colscan
  int start = d.col_start[cg], cstart = d.col_cstart[cg];
  if (cstart + (n + CL - 1) / CL > T.max_clus) return;  // flagged by k_colscan
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int i = threadIdx.x; i < np2; i += blockDim.x) {
    if (i < n) {
      int s = d.bucket[T.atom0 + start + i];
      float z = d.pos_b[s].z;
      key[i] = ((unsigned long long)__float_as_uint(z) << 32) | (unsigned)d.orig_b[s];
    } else {
      key[i] = ~0ull;
    }
  }
  __syncthreads();
  // bitonic sort, ascending
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < np2; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long a = key[i], b = key[ixj];
          bool up = (i & k) == 0;
          if ((a > b) == up) { key[i] = b; key[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    int o = (int)(key[r] & 0xffffffffu);
    s_old[r] = d.slot_of[T.atom0 + o];
  }
  __syncthreads();
  int ncl = (n + CL - 1) / CL;
  int base = T.slot0 + cstart * CL;
  for (int r = threadIdx.x; r < ncl * CL; r += blockDim.x) {
    int ns = base + r;
    if (r < n) {
      int old = s_old[r];
      int o = (int)(key[r] & 0xffffffffu);
      const float4 p = d.pos_b[old];
      d.pos[ns] = p;
      d.ref_slot[ns] = p;  // the position the new list is built from
      d.vel[ns] = d.vel_b[old];
      d.orig[ns] = o;
      d.type[ns] = d.type_b[old];
      d.slot_of[T.atom0 + o] = ns;
    } else {
      const float4 pad = pad_pos(ns);
      d.pos[ns] = pad;
      d.ref_slot[ns] = pad;
      d.vel[ns] = make_float4(0.f, 0.f, 0.f, 0.f);
      d.orig[ns] = -1;
      d.type[ns] = 0;
    }
  }
  // bounding boxes of the 4-atom halves of each cluster (real atoms only; an
  // all-padding half gets an empty box, lo > hi)
  for (int k = threadIdx.x; k < 2 * ncl; k += blockDim.x) {
    float3 lo = make_float3(3e38f, 3e38f, 3e38f), hi = make_float3(-3e38f, -3e38f, -3e38f);
    for (int a = 0; a < CJ; ++a) {
      int r = k * CJ + a;
      if (r >= n) break;
      float4 p = d.pos_b[s_old[r]];
      lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
      hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
    }
    int hj = 2 * (T.clus0 + cstart) + k;
    d.bb_lo[hj] = make_float4(lo.x, lo.y, lo.z, 0.f);
    d.bb_hi[hj] = make_float4(hi.x, hi.y, hi.z, 0.f);
    s_zlo[k] = lo.z;
  }
  __syncthreads();
  // z-bin table: the halves are in ascending z, so the number of halves whose
  // lower z-bound lies below b L / ZBINS is the first half at or above it
  for (int b = threadIdx.x; b <= ZBINS; b += blockDim.x) {
    const float zt = (float)b * (T.box / ZBINS);
    int cnt = 0;
    for (int k = 0; k < 2 * ncl; ++k) cnt += s_zlo[k] < zt ? 1 : 0;
    d.col_ztab[(size_t)cg * (ZBINS + 1) + b] = cnt;
  }
}

// ---------------------------------------------------------------------------
// cluster-pair list
// ---------------------------------------------------------------------------
// distance between two intervals on a circle of length L
__device__ __forceinline__ float periodic_gap(float a0, float a1, float b0, float b1, float L) {
  float g = 3e38f;
#pragma unroll
  for (int k = -1; k <= 1; ++k) {
    float s = k * L;
    float gg = fmaxf(0.0f, fmaxf(b0 + s - a1, a0 - (b1 + s)));
    g = fminf(g, gg);
  }
  return g;
}

// the FP32 list rule: n = rint((xj - xi) * invL); d = (xj - L n) - xi (the
// image of x_j first, as the force kernel forms it); r2 = fma(dz, dz,
// fma(dy, dy, dx*dx)); member iff r2 < rl2.  Also returns the image key
// 9 nx + 3 ny + nz of the counts n (x_j image = x_j - L n).
__device__ __forceinline__ bool list_rule(float4 pi, float4 pj, float L, float iL, float rl2, float &key) {
  const float tx = __fsub_rn(pj.x, pi.x), ty = __fsub_rn(pj.y, pi.y), tz = __fsub_rn(pj.z, pi.z);
  const float qx = rintf(__fmul_rn(tx, iL)), qy = rintf(__fmul_rn(ty, iL)), qz = rintf(__fmul_rn(tz, iL));
  const float dx = __fsub_rn(__fsub_rn(pj.x, __fmul_rn(L, qx)), pi.x);
  const float dy = __fsub_rn(__fsub_rn(pj.y, __fmul_rn(L, qy)), pi.y);
  const float dz = __fsub_rn(__fsub_rn(pj.z, __fmul_rn(L, qz)), pi.z);
  const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
  key = __fmaf_rn(9.0f, qx, __fmaf_rn(3.0f, qy, qz));
  return r2 < rl2;
}

// A candidate whose atom pairs do not all share the image counts (it spans
// half a box length in some dimension): the per-pair rule for all 8 x 4
// pairs, with validity and self-pair tests; kmin/kmax collect the image keys
// of the passing pairs (exclusions are cleared afterwards).
static __device__ __noinline__ unsigned list_mixed_images(const Dev &d, int I, int Il, int J8, int sj0, float L, float iL,
                                                   float rl2, float &kmin, float &kmax) {
  unsigned mask = 0u;
  for (int b = 0; b < CJ; ++b) {
    const float4 pj = d.pos[sj0 + b];
    const int oj = d.orig[sj0 + b];
    for (int a = 0; a < CL; ++a) {
      const float4 pi = d.pos[I * CL + a];
      const int oi = d.orig[I * CL + a];
      float key;
      const bool v = list_rule(pi, pj, L, iL, rl2, key) && oi >= 0 && oj >= 0 && (J8 != Il || sj0 + b > I * CL + a);
      if (v) {
        kmin = fminf(kmin, key);
        kmax = fmaxf(kmax, key);
        mask |= 1u << (a * CJ + b);
      }
    }
  }
  return mask;
}

constexpr int LIST_WARPS = 4;
constexpr int CAND_MAX = 1024;  // candidate 4-atom j-clusters per i-cluster (bounding-box pass)
constexpr int ENT_MAX = 512;    // 4-atom j-clusters with a listed pair per i-cluster
// a candidate word: the half index (J_BITS bits), the shared-image flag, the image key
constexpr int CAND_SAME_BIT = (int)J_BITS;
constexpr int CAND_KEY_SHIFT = (int)J_BITS + 1;
static_assert(J_BITS + 6 <= 31, "candidate word: half index, flag and a 5-bit key in a non-negative int");

// the mask column of j-atom b of a 4-atom j-cluster entry: bit a of the
// result is bit a*4 + b of the 32-bit mask
__device__ __forceinline__ unsigned j_column(unsigned m, int b) {
  unsigned x = (m >> b) & 0x11111111u;
  x = (x | (x >> 3)) & 0x03030303u;
  x = (x | (x >> 6)) & 0x000f000fu;
  return (x | (x >> 12)) & 0xffu;
}
// j-atoms of an entry with at least one listed pair
__device__ __forceinline__ int j_columns(unsigned m) {
  const unsigned any = m | (m >> 16);
  const unsigned a2 = any | (any >> 8);
  return __popc((a2 | (a2 >> 4)) & 0xfu);
}

// One warp per i-cluster.  Phase 1: lanes test columns, then the 4-atom
// halves of the clusters of each passing column, against the i-cluster's
// bounding box and collect the candidates in order (column-major, then z,
// i.e. ascending j-cluster index).  Phase 2: each lane takes one candidate
// and evaluates the FP32 list rule for all 8 x 4 atom pairs itself, giving
// the entry's mask, image code and exact flag; entries are written in
// candidate order (deterministic).  Phase 3: the i-atoms' exclusions clear
// their bits in the entries (found by binary search).  Phase 4: one list
// entry per j-atom with a listed pair is written out.
struct ListShared {
  int s_cand[LIST_WARPS][CAND_MAX];
  int s_excl[LIST_WARPS][CL][MAX_EXCL];
  int s_nex[LIST_WARPS][CL];
  float4 s_xp[LIST_WARPS][CL / 2][2];  // i-atom pairs (2p, 2p+1): {-x, -x', -y, -y'} {-z, -z', 0, 0}
  unsigned s_dirty[LIST_WARPS][ENT_MAX / 32];  // entries whose j-atoms need the pair masks
  unsigned s_mask[LIST_WARPS][ENT_MAX];        // masks of the entries (their first words overwrite s_cand)
};

__device__ __forceinline__ void list_cluster(const Dev &d, const SimConst &c, float rl2_bbox, ListShared &sh, int t,
                                             int Il) {
  auto &s_cand = sh.s_cand;
  auto &s_excl = sh.s_excl;
  auto &s_nex = sh.s_nex;
  auto &s_xp = sh.s_xp;
  auto &s_dirty = sh.s_dirty;
  auto &s_mask = sh.s_mask;
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const TrialInfo T = d.tinfo[t];
  if (Il >= T.max_clus) return;
  const int I = T.clus0 + Il;
  if (Il >= d.tstate[t].n_clus) {
    if (lane == 0) d.list_n[I] = 0;
    return;
  }
  float4 lo, hi;
  {
    const float4 l0 = d.bb_lo[2 * I], l1 = d.bb_lo[2 * I + 1], h0 = d.bb_hi[2 * I], h1 = d.bb_hi[2 * I + 1];
    lo = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
    hi = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
  }
  const float L = T.box, iL = T.inv_box, w = T.col_w;
  const int nc2 = T.ncol * T.ncol;
  int *cand = s_cand[wib];
  int n_cand = 0;
  bool overflow = false;
  // ---- phase 1: candidate 4-atom j-clusters ----
  // Only the grid columns within reach of the i-cluster's bounding box (one
  // column more on each side for the rounding of the binning) are visited,
  // in ascending column index: the window's x and y column indices, wrapped
  // periodically, are enumerated in sorted order (so the candidates, and the
  // entries, ascend in j-cluster index).  Lanes test 32 columns; the halves
  // (of clusters with index >= Il) of the passing columns are then
  // enumerated as one flat range, 32 per step, so that the bounding-box loads
  // of a whole step are in flight together.
  const float reach = sqrtf(rl2_bbox);
  int wx0, wnx, wy0, wny;  // first column (mod ncol) and count of the window in x and in y
  {
    const int ax = (int)floorf((lo.x - reach) * T.inv_col_w) - 1, bx = (int)floorf((hi.x + reach) * T.inv_col_w) + 1;
    const int ay = (int)floorf((lo.y - reach) * T.inv_col_w) - 1, by = (int)floorf((hi.y + reach) * T.inv_col_w) + 1;
    wnx = min(T.ncol, bx - ax + 1);
    wny = min(T.ncol, by - ay + 1);
    wx0 = wnx == T.ncol ? 0 : ((ax % T.ncol) + T.ncol) % T.ncol;
    wy0 = wny == T.ncol ? 0 : ((ay % T.ncol) + T.ncol) % T.ncol;
  }
  // k-th smallest of {a, a + 1, ..., a + m - 1} mod ncol
  auto kth = [&](int a, int m, int k) {
    const int e = a + m - T.ncol;  // the part that wraps to [0, e)
    return e <= 0 ? a + k : (k < e ? k : a + (k - e));
  };
  const int nwin = wnx * wny;
  const int n_clus_t = d.tstate[t].n_clus;
  for (int cb = 0; cb < nwin; cb += 32) {
    const int wi = cb + lane;
    // this lane's column: up to two ranges [a1, a1 + n1), [a2, a2 + n2) of
    // half indices (relative to the trial's first half) whose z-extent can
    // reach the i-cluster: the z-window (and its periodic image) comes from
    // the column's xy gap, the ranges from the column's z-bin table, one bin
    // wider on each side than needed (every half in them is still tested)
    int a1 = 0, n1 = 0, a2 = 0, n2 = 0;
    const int cc = wi < nwin ? kth(wx0, wnx, wi / wny) * T.ncol + kth(wy0, wny, wi % wny) : 0;
    if (wi < nwin) {
      // the geometry first, then every load of the column at once (one
      // memory round trip instead of two)
      const int cx = cc / T.ncol, cy = cc - cx * T.ncol;
      const float gx = periodic_gap(lo.x, hi.x, cx * w, (cx + 1) * w, L);
      const float gy = periodic_gap(lo.y, hi.y, cy * w, (cy + 1) * w, L);
      const float g2 = gx * gx + gy * gy;
      if (g2 < rl2_bbox) {
        const float rz = sqrtf(rl2_bbox - g2) * 1.001f + 1e-3f;
        const float za = lo.z - rz, zb = hi.z + rz;
        const bool whole = zb - za >= L;
        // z-bins of the halves that may meet [u, v] (0 <= u <= v <= L): one
        // or two intervals (the periodic image)
        const float zs = ZBINS * iL;
        const bool two = za < 0.f || zb > L;
        const float u1 = 0.f, v1 = za < 0.f ? zb : (zb > L ? zb - L : zb);
        const float u1r = two ? u1 : za;
        const float u2 = za < 0.f ? za + L : za, v2 = L;
        auto bin_lo = [&](float u) { return max(0, min(ZBINS, (int)floorf(u * zs) - 1)); };
        auto bin_hi = [&](float v) { return max(0, min(ZBINS, (int)floorf(v * zs) + 2)); };
        const int bu1 = bin_lo(u1r), bv1 = bin_hi(v1), bu2 = bin_lo(u2), bv2 = bin_hi(v2);
        const int *tab = d.col_ztab + (size_t)(T.col0 + cc) * (ZBINS + 1);
        const int ccs = d.col_cstart[T.col0 + cc];
        const int cnext = cc + 1 < nc2 ? d.col_cstart[T.col0 + cc + 1] : n_clus_t;
        const int t1a = tab[bu1], t1b = tab[bv1];
        const int t2a = two ? tab[bu2] : 0, t2b = two ? tab[bv2] : 0;
        const int ncl = max(0, cnext - ccs);
        const int jlo = max(ccs, Il);
        if (ccs + ncl > jlo) {
          const int hs = 2 * (jlo - ccs), he = 2 * ncl;  // local half range of the half list
          if (whole) {
            a1 = hs; n1 = he - hs;
          } else {
            int r1a = max(t1a - 1, 0), r1b = bv1 >= ZBINS ? he : t1b;
            int r2a = 0, r2b = 0;
            if (two) {
              r2a = max(t2a - 1, 0);
              r2b = bv2 >= ZBINS ? he : t2b;
            }
            r1a = max(r1a, hs); r1b = min(r1b, he);
            r2a = max(max(r2a, hs), r1b); r2b = min(r2b, he);  // ascending, no half twice
            a1 = r1a; n1 = max(r1b - r1a, 0);
            a2 = r2a; n2 = max(r2b - r2a, 0);
          }
          a1 += 2 * ccs;
          a2 += 2 * ccs;
        }
      }
    }
    const int cntc = n1 + n2;
    // inclusive scan of the per-column candidate counts
    int incl = cntc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int tt = t0 + lane;
      const int tq = min(tt, total - 1);
      // owner column: first lane whose inclusive count exceeds tq (all lanes search)
      int lo_l = 0, hi_l = 31;
#pragma unroll
      for (int it = 0; it < 5; ++it) {
        const int mid = (lo_l + hi_l) >> 1;
        const int v = __shfl_sync(0xffffffffu, incl, mid);
        if (v > tq) hi_l = mid; else lo_l = mid + 1;
      }
      const int own_incl = __shfl_sync(0xffffffffu, incl, lo_l);
      const int own_cnt = __shfl_sync(0xffffffffu, cntc, lo_l);
      const int own_a1 = __shfl_sync(0xffffffffu, a1, lo_l);
      const int own_n1 = __shfl_sync(0xffffffffu, n1, lo_l);
      const int own_a2 = __shfl_sync(0xffffffffu, a2, lo_l);
      bool ok = false;
      int J4 = 0;
      if (tt < total) {
        const int u = tt - (own_incl - own_cnt);
        J4 = u < own_n1 ? own_a1 + u : own_a2 + (u - own_n1);
        const float4 jlo4 = d.bb_lo[2 * T.clus0 + J4], jhi4 = d.bb_hi[2 * T.clus0 + J4];
        const float gx = periodic_gap(lo.x, hi.x, jlo4.x, jhi4.x, L);
        const float gy = periodic_gap(lo.y, hi.y, jlo4.y, jhi4.y, L);
        const float gz = periodic_gap(lo.z, hi.z, jlo4.z, jhi4.z, L);
        ok = gx * gx + gy * gy + gz * gz < rl2_bbox;
        // image counts at the two bounding-box extremes (each -1, 0 or 1: the
        // positions lie in [0, L)); when they agree in every dimension, every
        // atom pair of the candidate has them.  Carried in the candidate word
        // (shared image flag, key 9 (nx+1) + 3 (ny+1) + (nz+1)) so that phase 2
        // need not load the box again.
        const float qlx = rintf(__fmul_rn(__fsub_rn(jlo4.x, hi.x), iL)), qhx = rintf(__fmul_rn(__fsub_rn(jhi4.x, lo.x), iL));
        const float qly = rintf(__fmul_rn(__fsub_rn(jlo4.y, hi.y), iL)), qhy = rintf(__fmul_rn(__fsub_rn(jhi4.y, lo.y), iL));
        const float qlz = rintf(__fmul_rn(__fsub_rn(jlo4.z, hi.z), iL)), qhz = rintf(__fmul_rn(__fsub_rn(jhi4.z, lo.z), iL));
        const int same = qlx == qhx && qly == qhy && qlz == qhz;
        const int key = 9 * ((int)qlx + 1) + 3 * ((int)qly + 1) + ((int)qlz + 1);
        J4 |= (same << CAND_SAME_BIT) | (key << CAND_KEY_SHIFT);
      }
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      const int pos = n_cand + __popc(m & ((1u << lane) - 1u));
      if (ok && pos < CAND_MAX) cand[pos] = J4;
      n_cand += __popc(m);
    }
  }
  if (n_cand > CAND_MAX) {
    overflow = true;
    n_cand = CAND_MAX;
  }
  // i-atoms (shared memory: broadcast reads leave registers for more resident
  // warps) and their exclusions
  if (lane < CL / 2) {
    const float4 a0 = d.pos[I * CL + 2 * lane], a1 = d.pos[I * CL + 2 * lane + 1];
    s_xp[wib][lane][0] = make_float4(-a0.x, -a1.x, -a0.y, -a1.y);
    s_xp[wib][lane][1] = make_float4(-a0.z, -a1.z, 0.f, 0.f);
  }
  if (lane < CL) {
    const int o = d.orig[I * CL + lane];
    s_nex[wib][lane] = o < 0 ? 0 : d.excl_n[T.sysatom0 + o];
  }
  if (lane < ENT_MAX / 32) s_dirty[wib][lane] = c.list_fixed ? ~0u : 0u;  // fixed-interval lists: masks everywhere
  __syncwarp();
  // the slots of the i-atoms' excluded partners, all loads of the warp in flight together
  for (int k = lane; k < CL * MAX_EXCL; k += 32) {
    const int a = k / MAX_EXCL, q = k - a * MAX_EXCL;
    if (q < s_nex[wib][a]) {
      const int o = d.orig[I * CL + a];
      s_excl[wib][a][q] = d.slot_of[T.atom0 + d.excl[(size_t)(T.sysatom0 + o) * MAX_EXCL + q]];
    }
  }
  // ---- phase 2: one candidate 4-atom j-cluster per lane ----
  // Image counts: q = rint(fl(d * invL)) is monotone in d = fl(xj - xi), so
  // when the two bounding-box extremes of d give the same q in a dimension,
  // every atom pair of the candidate has that q there and the rule reduces to
  // d - fl(L q) with the same rounding as the per-pair form.  Padding atoms
  // sit far outside every box and fail the distance test on that path.
  const float rl2 = c.rl2;
  int cnt = 0;
  for (int k0 = 0; k0 < n_cand; k0 += 32) {
    const int k = k0 + lane;
    unsigned mask = 0u, w0 = 0u;
    if (k < n_cand) {
      const int cw = cand[k];
      const int J4 = cw & (int)J_MASK;
      const int J8 = J4 >> 1, h = J4 & 1;
      const int JG = T.clus0 + J8;
      const int sj0 = JG * CL + h * CJ;
      float kmin = 3e38f, kmax = -3e38f;
      const int ckey = (cw >> CAND_KEY_SHIFT) & 31;
      const float qlx = (float)(ckey / 9 - 1), qly = (float)((ckey / 3) % 3 - 1), qlz = (float)(ckey % 3 - 1);
      if ((cw >> CAND_SAME_BIT) & 1) {
        // the j-atom's image once, then two i-atoms per packed FP32x2
        // operation; every operation rounds on its own exactly as the
        // per-pair rule does (d = (xj - L n) + (-xi) is (xj - L n) - xi)
        const float sx = __fmul_rn(L, qlx), sy = __fmul_rn(L, qly), sz = __fmul_rn(L, qlz);
#pragma unroll
        for (int b = 0; b < CJ; ++b) {
          const float4 pj = d.pos[sj0 + b];
          const float ux = __fsub_rn(pj.x, sx), uy = __fsub_rn(pj.y, sy), uz = __fsub_rn(pj.z, sz);
          const float2 xj2 = make_float2(ux, ux), yj2 = make_float2(uy, uy), zj2 = make_float2(uz, uz);
#pragma unroll
          for (int p = 0; p < CL / 2; ++p) {
            const float4 i0 = s_xp[wib][p][0], i1 = s_xp[wib][p][1];
            const float2 dx = __fadd2_rn(xj2, make_float2(i0.x, i0.y));
            const float2 dy = __fadd2_rn(yj2, make_float2(i0.z, i0.w));
            const float2 dz = __fadd2_rn(zj2, make_float2(i1.x, i1.y));
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            if (r2.x < rl2) mask |= 1u << (2 * p * CJ + b);
            if (r2.y < rl2) mask |= 1u << ((2 * p + 1) * CJ + b);
          }
        }
        if (J8 == Il) {  // inside the i-cluster itself: pairs with the j slot above the i slot
          unsigned tri = 0u;
#pragma unroll
          for (int a = 0; a < CL; ++a)
#pragma unroll
            for (int b = 0; b < CJ; ++b)
              if (h * CJ + b > a) tri |= 1u << (a * CJ + b);
          mask &= tri;
        }
        if (mask) kmin = kmax = __fmaf_rn(9.0f, qlx, __fmaf_rn(3.0f, qly, qlz));
      } else {
        mask = list_mixed_images(d, I, Il, J8, sj0, L, iL, rl2, kmin, kmax);
      }
      // image counts of the entry from the key 9 nx + 3 ny + nz (each in -1..1)
      const int key = mask ? (int)kmin : 0;
      const int kz = ((key % 3) + 4) % 3 - 1;
      const int ky = (((key - kz) / 3) % 3 + 4) % 3 - 1;
      const int kx = (key - kz - 3 * ky) / 9;
      const bool same = kmin == kmax;
      w0 = (unsigned)(2 * JG + h) | ((unsigned)((kx + 1) | ((ky + 1) << 2) | ((kz + 1) << 4)) << J_BITS) |
           (same || !mask ? 0u : E_EXACT);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, mask != 0u);
    const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
    __syncwarp();  // every lane has read its candidate before entries overwrite them
    if (mask != 0u && pos < ENT_MAX) {
      // entries are kept in shared memory until the exclusions are cleared:
      // the first word over the consumed candidates, the mask beside
      cand[pos] = (int)w0;
      s_mask[wib][pos] = mask;
      // the cluster with itself (pairs below the diagonal masked) and entries
      // whose pairs take images one by one need the masks in the pair kernel
      if ((int)((w0 & J_MASK) >> 1) == I || (w0 & E_EXACT)) atomicOr(&s_dirty[wib][pos >> 5], 1u << (pos & 31));
    }
    cnt += __popc(bal);
  }
  const int n_ent = min(cnt, ENT_MAX);
  // ---- phase 3: exclusions ----
  // lane a < 8 clears, for each atom excluded from i-atom a, the bit of that
  // pair in the entry of its 4-atom j-cluster, if this list holds the pair
  // (entries ascend in j-cluster index; a pair inside the i-cluster belongs
  // to the entry with the higher slot as j)
  __syncwarp();
  for (int k = lane; k < CL * MAX_EXCL; k += 32) {
    const int a = k / MAX_EXCL, q = k - a * MAX_EXCL;
    if (q >= s_nex[wib][a]) continue;
    const int si = I * CL + a;
    const int sj = s_excl[wib][a][q];
    if ((sj >> 3) < I || ((sj >> 3) == I && sj <= si)) continue;  // listed from the other side, or not at all
    const unsigned j4 = (unsigned)(sj >> 2);
    int lo_e = 0, hi_e = n_ent;  // first entry with j-cluster >= j4
    while (lo_e < hi_e) {
      const int mid = (lo_e + hi_e) >> 1;
      if (((unsigned)cand[mid] & J_MASK) < j4) lo_e = mid + 1; else hi_e = mid;
    }
    if (lo_e < n_ent && ((unsigned)cand[lo_e] & J_MASK) == j4) {
      atomicAnd(&s_mask[wib][lo_e], ~(1u << (a * CJ + (sj & 3))));
      atomicOr(&s_dirty[wib][lo_e >> 5], 1u << (lo_e & 31));
    }
  }
  __syncwarp();
  // ---- phase 4: one entry per j-atom with a listed pair ----
  // In entry order, j-atoms ascending; the j-atoms of entries that need the
  // masks first, so that they fill as few groups of 32 entries as possible.
  auto dirty_at = [&](int e) { return ((s_dirty[wib][e >> 5] >> (e & 31)) & 1u) != 0u; };
  int n_dirty = 0;
  for (int e0 = 0; e0 < n_ent; e0 += 32) {
    const int e = e0 + lane;
    const int nd = e < n_ent && dirty_at(e) ? j_columns(s_mask[wib][e]) : 0;
    n_dirty += __reduce_add_sync(0xffffffffu, nd);
  }
  uint32_t *segw = d.list + (size_t)I * c.list_cap;
  uint8_t *segm = d.list_m + (size_t)I * c.list_cap;
  int pd = 0, pc = n_dirty;  // where the next j-atoms of either kind go
  for (int e0 = 0; e0 < n_ent; e0 += 32) {
    const int e = e0 + lane;
    const unsigned m = e < n_ent ? s_mask[wib][e] : 0u;
    const bool dirty = e < n_ent && dirty_at(e);
    const int nj = j_columns(m);
    // inclusive scan over the lanes of both counts at once (16 bits each)
    const int own = dirty ? nj : nj << 16;
    int sdc = own;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, sdc, off);
      if (lane >= off) sdc += v;
    }
    const int before = sdc - own;
    int p = dirty ? pd + (before & 0xffff) : pc + (before >> 16);
    if (nj) {
      const unsigned w = (unsigned)cand[e];
      const unsigned s0 = (w & J_MASK) * CJ, rest = w & ~J_MASK;
#pragma unroll
      for (int b = 0; b < CJ; ++b) {
        const unsigned col = j_column(m, b);
        if (col) {
          if (p < c.list_cap) {
            segw[p] = (s0 + b) | rest;
            segm[p] = (uint8_t)col;
          }
          ++p;
        }
      }
    }
    const int tot = __shfl_sync(0xffffffffu, sdc, 31);
    pd += tot & 0xffff;
    pc += tot >> 16;
  }
  if (lane == 0) {
    d.list_n[I] = min(pc, c.list_cap);
    d.list_nm[I] = min(n_dirty, c.list_cap);
    if (cnt > ENT_MAX || pc > c.list_cap || overflow) atomicOr(d.err, ERR_LIST);
  }
}


}  // namespace vp

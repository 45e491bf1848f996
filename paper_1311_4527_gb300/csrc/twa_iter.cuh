// twa_iter.cuh -- the per-block work of one TWA iteration (Appendix B steps
// 1-7 over the factor graph of Section 3.3 of Bento et al., NIPS 2013), shared
// by the single-planner kernels and the batched ones (both in plan.cu).
//
// Pass 1, test_block: one block per (segment s, agent tiles I <= J) of 32 x 32
//   collision factors: finish the deferred dual update of the pairs that were
//   active (step 7 of the previous iteration), n = z - u (step 1), collision
//   test and weight (steps 2-3), activity bits, worklist of active pairs.
// segment_block: the kinetic and wall factors of one (segment, agent tile);
//   the single-planner kernels run these blocks in the same launch as pass 1
//   and leave the active walls' capsule minimizers to pass 2
//   (wall_prox_item_warp, one warp per wall), which spreads them over the GPU.
// Pass 2, prox_item: the collision minimizer of one active pair; adds its
//   m = x + u to the consensus sums (wall_prox_item_warp: the same for a wall).
// Pass 3, consensus_node: z = sum m / count per free break-point (step 5).
//
// Step 7 needs z^{k+1}, which exists only after every factor ran, so x^{k+1}
// of the active factors is stored and u^{k+1} = u^k + alpha (x^{k+1} -
// z^{k+1}) is finished at the start of the next iteration.  Back weights
// (step 6) are rho0 at every interior node (the kinetic factors always send
// rho0 there) and infinity at the fixed ends; u on an edge whose forward
// weight was 0, or whose node is fixed, is 0.
//
// Collision-factor state lives in tile order: block blk = s * ntp + tp holds
// the 32 x 32 pair slots (row r = i - 32 I, column c = j - 32 J), so a warp
// streams one row as 32 consecutive float4 (512 B).  Per slot:
//   ulo[slot] = (u_i(s), u_j(s))       uhi[slot] = (u_i(s+1), u_j(s+1))
//   xlo / xhi = pending x^{k+1}, read and written only for active factors
//   bits[blk * 32 + r] bit c = forward weight rho0 in the last iteration.
// With the dense state the u record of every slot is read and written each
// iteration; otherwise only those of factors whose bit is set (every other u
// is 0 by the reset rule), which leaves 1 bit per factor of state traffic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "twa_math.cuh"

namespace {

using namespace twa;

constexpr int TILE = 32;
constexpr int WARPS = 8;
constexpr int THREADS = TILE * WARPS;
constexpr int ROWS = TILE / WARPS;  // rows of a tile per warp
constexpr unsigned FULL = 0xffffffffu;

struct Dev {
  int p, eta, nw, nt, ntp;
  float rho, alpha;
  int dense, keep, admm;
  int nv;                // velocity-factor kinds after the walls (0..2)
  unsigned vmin_mask;    // bit v: velocity kind v is a minimum (else maximum)
  int noenergy;          // no kinetic factors (the feasibility problem)
  int vo;                // velocity-obstacle epoch (eta = 2): collision, wall and velocity
                         // factors on segment 0 only, the kinetic factor on segment 1 only
  const float* vlim;     // [nv][p][eta] velocity limits
  uint8_t* wnode;        // [p][eta+1] back-weight class when noenergy: 0 or 1
  const float2* z;       // z^k, [p][eta+1]
  float2* z_next;        // z^{k+1}; until the consensus pass writes it, z^{k-1}
  const float* radius;   // [p]
  const float* cost;     // [p][eta], kinetic coefficients c_{i,s}
  const float4* walls;   // [nw] (xL.x, xL.y, xR.x, xR.y)
  // uwall / xwall / wbits hold nw wall kinds followed by nv velocity kinds
  const int2* tiles;     // [ntp] (I, J), I <= J
  float4 *ulo, *uhi, *xlo, *xhi;
  uint32_t* bits;        // [eta * ntp * 32]
  float4 *ukin, *xkin;   // [eta][p]
  float4 *uwall, *xwall; // [nw][eta][p]
  uint32_t* wbits;       // [nw][eta][nt]
  uint32_t* work;        // active collision slots of this iteration
  unsigned* work_count;  // their number
  unsigned* work_count_next;  // the counter the next iteration appends to
  // pass-1 scheduling (single plans; hcap = 0 turns it off): tiles whose
  // exact-test work was large in the previous iteration are listed and
  // dispatched first, on the first hcap warps of the launch, and stamped so
  // that their place in the ordinary order is skipped
  int hcap;                    // heavy-tile slots at the front of the launch
  const uint32_t* heavy_cur;   // this iteration's heavy tiles (built by the previous one)
  unsigned* hcount_cur;        // their number (cleared by the consensus pass for reuse)
  uint32_t* heavy_next;        // the next iteration's heavy tiles (built by this pass 1)
  unsigned* hcount_next;
  // [eta ntp] iteration number for which the tile is listed heavy, one array
  // per iteration parity: this iteration's list is only read (ordinary warps
  // skip the tiles listed in it) while the next one's is written
  const unsigned* stamp_cur;
  unsigned* stamp_next;
  unsigned* iter;              // iteration number (advanced by the consensus pass)
  uint32_t* wwork;       // active wall factors ((w eta + s) p + i) of this iteration whose
                         // minimizer runs in pass 2 (wall_prox_item_warp)
  unsigned* wwork_count;       // their number
  unsigned* wwork_count_next;  // the counter the next iteration appends to
  unsigned long long* accx;  // [p][eta+1] fixed-point sums of rho0-weighted m.x
  unsigned long long* accy;  //                                 ... of m.y
  unsigned* accc;        // [p][eta+1] number of rho0-weighted incoming edges
  const float* fix;      // fixed-point scale (a power of two) and |m| bound
  unsigned* res_cur;     // residual slot of this iteration (consensus part)
  unsigned* res_prev;    // residual slot of the previous iteration (primal part)
  unsigned* status;      // bit 0: a pinned wall minimizer had no separating direction;
                         // bit 1: a message out of the fixed-point range
};

__device__ __forceinline__ float maxabs2(float2 a) { return fmaxf(fabsf(a.x), fabsf(a.y)); }

// Step 7 of the previous iteration for one edge: u^k from the stored u^{k-1},
// the pending x^k and z^k.
__device__ __forceinline__ float2 finish_u(bool bprev, bool pinned, bool keep, float2 u_prev,
                                           float2 x_pend, float2 zk, float alpha, float& res) {
  if (pinned) return mk(0.f, 0.f);
  if (bprev) {
    float2 d = x_pend - zk;
    res = fmaxf(res, maxabs2(d));
    return mk(u_prev.x + alpha * d.x, u_prev.y + alpha * d.y);
  }
  return keep ? u_prev : mk(0.f, 0.f);
}

// Step 5's sums in 64-bit fixed point: each FP32 m is scaled by a power of
// two 2^e chosen from the layout's extent and rounded to an integer (an
// absolute error of at most 2^-(e+1), about 1e-13 at p = 1024 on the 40 x 40
// square, far below the FP32 ulp of m itself), then the integers are summed
// exactly; integer addition does not depend on the order of the atomics, so z
// is deterministic: the integer sum rounded once to FP32 and divided by the
// count in FP32 (within 1.5 units in the last place of the mean of the
// quantised messages).  A non-finite or out-of-range m sets status bit 1,
// which the consensus pass turns into a NaN residual.
__device__ __forceinline__ void contribute(const Dev& P, float scale, float bound, int i, int s,
                                           float2 m) {
  if (!(fabsf(m.x) <= bound && fabsf(m.y) <= bound)) {
    atomicOr(P.status, 2u);
    return;
  }
  const size_t node = (size_t)i * (P.eta + 1) + s;
  atomicAdd(P.accx + node, (unsigned long long)__float2ll_rn(m.x * scale));
  atomicAdd(P.accy + node, (unsigned long long)__float2ll_rn(m.y * scale));
  atomicAdd(P.accc + node, 1u);
}
__device__ __forceinline__ void contribute(const Dev& P, int i, int s, float2 m) {
  contribute(P, P.fix[0], P.fix[1], i, s, m);
}

// Standard-ADMM mode, a factor that was feasible in the previous iteration:
// its x^k was n^{k-1} = z^{k-1} - u^{k-1}, so step 7 needs no stored x.
__device__ __forceinline__ float2 finish_u_feasible(bool pinned, float2 u_prev, float2 z_prev,
                                                    float2 zk, float alpha, float& res) {
  if (pinned) return mk(0.f, 0.f);
  const float2 d = (z_prev - u_prev) - zk;
  res = fmaxf(res, maxabs2(d));
  return mk(u_prev.x + alpha * d.x, u_prev.y + alpha * d.y);
}

__device__ __forceinline__ float2 lo2(float4 v) { return mk(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return mk(v.z, v.w); }
__device__ __forceinline__ float4 pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

__device__ __forceinline__ void atomic_max_nonneg(unsigned* slot, float v) {
  atomicMax(slot, __float_as_uint(v));
}

// Global loads issued where they stand.  A volatile asm is never moved into
// a later branch, so loads placed ahead of an early exit are in flight
// together with the loads after it: one memory round trip instead of two on
// a warp's dependent chain.  For data that no other thread of the launch
// writes (and that the loading thread writes, if at all, only afterwards).
__device__ __forceinline__ float2 ld_now(const float2* p) {
  float2 v;
  asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_now(const float* p) {
  float v;
  asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned ld_now(const unsigned* p) {
  unsigned v;
  asm volatile("ld.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// Collision minimizer of one pair (Appendix C with equal weights rho on each
// end, or infinite at a fixed end).  n: (i lo, i hi, j lo, j hi).
__device__ __forceinline__ void coll_minimizer(float2 nil, float2 nih, float2 njl, float2 njh,
                                               bool pin_lo, bool pin_hi, float R, float rho,
                                               float2& xil, float2& xih, float2& xjl, float2& xjh) {
  float2 cl = njl - nil, ch = njh - nih;     // relative targets v = x_j - x_i
  float2 sl = nil + njl, sh = nih + njh;     // sum coordinates x_i + x_j
  xil = nil; xih = nih; xjl = njl; xjh = njh;
  if (pin_lo && pin_hi) return;
  if (pin_lo || pin_hi) {  // one call site for both fixed ends
    const float2 v = disk_prox_pinned(pin_lo ? cl : ch, pin_lo ? ch : cl, R);
    const float2 sm = pin_lo ? sh : sl;
    const float2 xi = 0.5f * (sm - v), xj = 0.5f * (sm + v);
    if (pin_lo) { xih = xi; xjh = xj; } else { xil = xi; xjl = xj; }
  } else {
    float2 vl, vh;
    float w = 0.5f * rho;  // rho rho / (rho + rho)
    disk_prox_free(cl, ch, w, w, R, vl, vh);
    xil = 0.5f * (sl - vl);
    xjl = 0.5f * (sl + vl);
    xih = 0.5f * (sh - vh);
    xjh = 0.5f * (sh + vh);
  }
}

// The collision minimizer with per-agent weight classes at each end (the
// feasibility problem; Appendix C's reduction with weights rho rho' / (rho +
// rho')): both agents at rho0 give relative weight rho0 / 2, a zero class on
// either gives relative weight 0 and the relative change goes to the
// zero-weight agent (split evenly when both are zero), a fixed end stays.
__device__ __forceinline__ void pair_end(float2 ni, float2 nj, int ci, int cj, float2 v, float2& xi,
                                         float2& xj) {
  if (ci == 2) { xi = ni; xj = nj; return; }
  if (ci == 0 && cj == 1) { xj = nj; xi = nj - v; return; }
  if (ci == 1 && cj == 0) { xi = ni; xj = ni + v; return; }
  const float2 sm = ni + nj;
  xi = 0.5f * (sm - v);
  xj = 0.5f * (sm + v);
}

__device__ __forceinline__ void coll_minimizer_classes(float2 nil, float2 nih, float2 njl,
                                                       float2 njh, int cil, int cih, int cjl,
                                                       int cjh, float R, float rho, float2& xil,
                                                       float2& xih, float2& xjl, float2& xjh) {
  const float2 cl = njl - nil, ch = njh - nih;
  const int rl = (cil == 2) ? 2 : ((cil == 1 && cjl == 1) ? 1 : 0);
  const int rh = (cih == 2) ? 2 : ((cih == 1 && cjh == 1) ? 1 : 0);
  float2 vl, vh;
  disk_prox_classes(cl, ch, rl, rh, R, 0.5f * rho, vl, vh);
  pair_end(nil, njl, cil, cjl, vl, xil, xjl);
  pair_end(nih, njh, cih, cjh, vh, xih, xjh);
}

// Kinetic factor (i, s): always active (it always sends rho0).  Finishes its
// pending dual update, runs the closed-form minimizer and stores x and u.
__device__ __forceinline__ void kinetic_factor(const Dev& P, int i, int s, float2 zl, float2 zh,
                                               bool pin_lo, bool pin_hi, float& res) {
  const size_t idx = (size_t)s * P.p + i;
  const float4 u4 = P.ukin[idx], x4 = P.xkin[idx];
  const float2 ul = finish_u(true, pin_lo, false, lo2(u4), lo2(x4), zl, P.alpha, res);
  const float2 uh = finish_u(true, pin_hi, false, hi2(u4), hi2(x4), zh, P.alpha, res);
  float2 xl, xh;
  energy_prox(zl - ul, zh - uh, P.rho, pin_lo, pin_hi, P.cost[(size_t)i * P.eta + s], xl, xh);
  P.xkin[idx] = pack(xl, xh);
  P.ukin[idx] = pack(ul, uh);
  if (!pin_lo) contribute(P, i, s, xl + ul);
  if (!pin_hi) contribute(P, i, s + 1, xh + uh);
}

// Back-weight classes of agent i's break-points s and s + 1: 2 at a fixed
// end, else rho0 (1) unless the feasibility problem left a node with only
// zero incoming weights (0).
__device__ __forceinline__ void end_classes(const Dev& P, int i, int s, bool pin_lo, bool pin_hi,
                                            int& cl, int& ch) {
  const size_t b = (size_t)i * (P.eta + 1) + s;
  cl = pin_lo ? 2 : (P.noenergy ? (int)P.wnode[b] : 1);
  ch = pin_hi ? 2 : (P.noenergy ? (int)P.wnode[b + 1] : 1);
}

// Gated segment factor w of (i, s): a wall (w < nw, Eq. wall_minimizer) or a
// maximum / minimum velocity factor (w >= nw, Eq. max_vel_min).  Forward
// weight rho0 when the n's violate it, else 0.  Called by a full warp (lane =
// agent of tile I).  DEFER: the capsule minimizers of active walls go to the
// wall worklist (P.wwork) instead of running here.
template <bool DEFER>
__device__ __forceinline__ void wall_factor(const Dev& P, int w, int i, bool vi, int s, int I,
                                            float2 zl, float2 zh, float r, bool pin_lo,
                                            bool pin_hi, float& res) {
  const int lane = threadIdx.x & 31;
  const size_t widx = ((size_t)w * P.eta + s) * P.nt + I;
  const uint32_t word = P.wbits[widx];
  const bool bprev = vi && ((word >> lane) & 1u);
  const size_t idx = ((size_t)w * P.eta + s) * P.p + i;
  float4 u4 = make_float4(0.f, 0.f, 0.f, 0.f), x4 = u4;
  if (vi && (P.dense || bprev)) u4 = P.uwall[idx];
  if (bprev) x4 = P.xwall[idx];
  float2 ul, uh;
  if (P.admm && vi && !bprev) {
    const int E1 = P.eta + 1;
    ul = finish_u_feasible(pin_lo, lo2(u4), P.z_next[(size_t)i * E1 + s], zl, P.alpha, res);
    uh = finish_u_feasible(pin_hi, hi2(u4), P.z_next[(size_t)i * E1 + s + 1], zh, P.alpha, res);
  } else {
    ul = finish_u(bprev, pin_lo, P.keep, lo2(u4), lo2(x4), zl, P.alpha, res);
    uh = finish_u(bprev, pin_hi, P.keep, hi2(u4), hi2(x4), zh, P.alpha, res);
  }
  const float2 nl = zl - ul, nh = zh - uh;
  const bool vel = w >= P.nw;
  bool act;
  float2 c0 = mk(0.f, 0.f), c1 = c0;
  float C = 0.f;
  bool vmin = false;
  if (vel) {
    const int v = w - P.nw;
    vmin = (P.vmin_mask >> v) & 1u;
    if (vi) C = P.vlim[((size_t)v * P.p + i) * P.eta + s];
    const float2 d = nl - nh;
    const float d2 = dot(d, d);
    act = vi && (vmin ? d2 < C * C : d2 > C * C);
  } else {
    const float4 W = P.walls[w];
    c0 = mk(W.x, W.y); c1 = mk(W.z, W.w);
    act = vi && dist2_segment_segment(nl, nh, c0, c1) < r * r;
  }
  const uint32_t nw = __ballot_sync(FULL, act);
  if (lane == 0 && nw != word) P.wbits[widx] = nw;
  if (DEFER && !vel) {
    // the capsule minimizers go to the minimizer pass, spread over the GPU
    // (one warp with several active walls would run them one after another)
    if (act) P.uwall[idx] = pack(ul, uh);
    else if (vi && P.dense) P.uwall[idx] = pack(ul, uh);
    if (nw) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(P.wwork_count, (unsigned)__popc(nw));
      base = __shfl_sync(FULL, base, 0);
      if (act) P.wwork[base + __popc(nw & ((1u << lane) - 1u))] = (uint32_t)idx;
    }
    return;
  }
  if (act) {
    float2 xl = nl, xh = nh;
    int cl, ch;
    end_classes(P, i, s, pin_lo, pin_hi, cl, ch);
    if (vel) {
      velocity_prox(nl, nh, cl, ch, C, xl, xh);
    } else if (!DEFER) {
      if (!capsule_prox_classes(nl, nh, cl, ch, c0, c1, r, 0.5f * P.rho, xl, xh))
        atomicOr(P.status, 1u);
    }
    P.xwall[idx] = pack(xl, xh);
    P.uwall[idx] = pack(ul, uh);
    if (!pin_lo) contribute(P, i, s, xl + ul);
    if (!pin_hi) contribute(P, i, s + 1, xh + uh);
  } else if (vi && P.dense) {
    P.uwall[idx] = pack(ul, uh);
  }
}

// Collision test of the n-trajectories (Eq. f_coll_def): does the relative
// segment [cl, ch] pass closer than R to the origin?  Strict, so touching is
// inactive.  Division-free: for an interior closest point, dist^2 =
// cross(cl, d)^2 / |d|^2 is compared as cross^2 < R^2 |d|^2.
__device__ __forceinline__ bool collides(float2 cl, float2 ch, float R) {
  const float2 d = ch - cl;
  const float dd = dot(d, d);
  const float t = -dot(cl, d);
  const float R2 = R * R;
  const float c = cross(cl, d);
  // endpoints, or an interior closest point (0 < t < |d|^2)
  return (dot(cl, cl) < R2) | (dot(ch, ch) < R2) | ((t > 0.f) & (t < dd) & (c * c < R2 * dd));
}

__device__ __forceinline__ int tile_pair(int nt, int I, int J) {  // I <= J
  return I * nt - I * (I - 1) / 2 + (J - I);
}

// Inverse of tile_pair: the tiles (I, J), I <= J, of pair index t, without
// the table lookup (a square root, then an exact integer correction).
__device__ __forceinline__ void tile_of(int nt, int t, int& I, int& J) {
  const float b = 2.f * nt + 1.f;
  int i = (int)((b - sqrtf(fmaxf(b * b - 8.f * t, 0.f))) * 0.5f);
  i = max(0, min(i, nt - 1));
  while (i > 0 && tile_pair(nt, i, i) > t) --i;
  while (i + 1 < nt && tile_pair(nt, i + 1, i + 1) <= t) ++i;
  I = i;
  J = i + (t - tile_pair(nt, i, i));
}

// Pass 1 of an iteration.  One CTA of 4 warps per (segment s, agent tiles
// I <= J) block of 32 x 32 collision factors; each warp takes 8 rows, lane =
// column agent j, and the row agents' data is held one per lane and broadcast
// by shuffles.  Per row, the warp finishes the pending dual update of the
// pairs that were active (step 7 of the previous iteration), forms n = z - u
// (step 1), runs the collision test (steps 2-3: weight rho0 or 0), stores the
// row's activity bits, and appends its active pairs to the global worklist.
// DENSE streams the u record of every pair (PLAN_DENSE_STATE).
//
// Early out (gated state): agent i's segment lies in the disk of centre m_i
// (its midpoint) and radius h_i (half its length), so the relative segment of
// a pair stays at distance >= |m_j - m_i| - h_i - h_j from the origin.  Rows
// where every pair has |m_j - m_i| > (h_i + h_j + r_i + r_j)(1 + 1e-5) cannot
// collide and skip the exact test; the margin keeps the outcome identical to
// running the exact test everywhere.
// TROWS rows per warp, TILE / TROWS warps per block (the launch shape the
// batched autotuner varies).
template <bool DENSE, int TROWS>
__device__ __forceinline__ void test_block(const Dev& P, int blk) {
  constexpr int TEST_ROWS = TROWS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int E1 = P.eta + 1;
  float res = 0.f;
  if (blk == 0 && threadIdx.x == 0) *P.res_cur = 0u;
  const int s = blk / P.ntp;
  if (P.vo && s != 0) return;  // no collision factors between x and x_ref
  const int2 IJ = P.tiles[blk - s * P.ntp];
  const int I = IJ.x, J = IJ.y;
  const bool diag = (I == J);
  const bool pin_lo = (s == 0), pin_hi = (s == P.eta - 1);
  const int r0 = warp * TEST_ROWS;
  const int nrows = min(TEST_ROWS, P.p - I * TILE - r0);
  if (nrows > 0) {  // warp-uniform
    // column agent of this lane
    const int j = J * TILE + lane;
    const bool vj = j < P.p;
    float2 zjl = mk(0.f, 0.f), zjh = zjl;
    float rj = 0.f;
    if (vj) { zjl = P.z[(size_t)j * E1 + s]; zjh = P.z[(size_t)j * E1 + s + 1]; rj = P.radius[j]; }
    // row agents r0 .. r0 + 7, held by lanes 0 .. 7
    float2 ill = mk(0.f, 0.f), ilh = ill;
    float rl = 0.f;
    uint32_t wordl = 0u;
    if (lane < nrows) {
      const int il = I * TILE + r0 + lane;
      ill = P.z[(size_t)il * E1 + s]; ilh = P.z[(size_t)il * E1 + s + 1]; rl = P.radius[il];
      wordl = P.bits[(size_t)blk * TILE + r0 + lane];
    }
    float2 mj = mk(0.f, 0.f), ml = mj;
    float bj = 0.f, bl = 0.f;
    if (!DENSE) {
      mj = 0.5f * (zjl + zjh);
      bj = 0.5f * sqrtf(dot(zjh - zjl, zjh - zjl)) + rj;
      ml = 0.5f * (ill + ilh);
      bl = 0.5f * sqrtf(dot(ilh - ill, ilh - ill)) + rl;
    }
#pragma unroll 2
    for (int q = 0; q < nrows; ++q) {
      const int r = r0 + q;
      const uint32_t word = __shfl_sync(FULL, wordl, q);
      const bool valid = vj && (!diag || r < lane);
      const float ri = __shfl_sync(FULL, rl, q);
      bool act = false;
      float2 uil = mk(0.f, 0.f), ujl = uil, uih = uil, ujh = uil;
      const size_t row = (size_t)blk * TILE + r;
      const size_t fid = row * TILE + lane;
      if (!DENSE && word == 0u) {
        // no pair of this row was active: every u is 0 by the reset rule, n = z
        const float2 mi = mk(__shfl_sync(FULL, ml.x, q), __shfl_sync(FULL, ml.y, q));
        const float br = __shfl_sync(FULL, bl, q) + bj;
        const float2 dm = mj - mi;
        const bool near = valid && dot(dm, dm) <= br * br * 1.00002f;
        if (__any_sync(FULL, near)) {
          const float2 zil = mk(__shfl_sync(FULL, ill.x, q), __shfl_sync(FULL, ill.y, q));
          const float2 zih = mk(__shfl_sync(FULL, ilh.x, q), __shfl_sync(FULL, ilh.y, q));
          act = near && collides(zjl - zil, zjh - zih, ri + rj);
        }
      } else {
        const float2 zil = mk(__shfl_sync(FULL, ill.x, q), __shfl_sync(FULL, ill.y, q));
        const float2 zih = mk(__shfl_sync(FULL, ilh.x, q), __shfl_sync(FULL, ilh.y, q));
        const bool bprev = (word >> lane) & 1u;  // set only for valid pairs
        if (DENSE && valid) {
          const float4 a = P.ulo[fid], b = P.uhi[fid];
          uil = lo2(a); ujl = hi2(a); uih = lo2(b); ujh = hi2(b);
        }
        if (bprev) {
          // finish step 7 of the previous iteration for this pair
          const float4 xa = P.xlo[fid], xb = P.xhi[fid];
          float4 a, b;
          if (DENSE) { a = pack(uil, ujl); b = pack(uih, ujh); }
          else { a = P.ulo[fid]; b = P.uhi[fid]; }
          uil = finish_u(true, pin_lo, false, lo2(a), lo2(xa), zil, P.alpha, res);
          ujl = finish_u(true, pin_lo, false, hi2(a), hi2(xa), zjl, P.alpha, res);
          uih = finish_u(true, pin_hi, false, lo2(b), lo2(xb), zih, P.alpha, res);
          ujh = finish_u(true, pin_hi, false, hi2(b), hi2(xb), zjh, P.alpha, res);
        } else if (DENSE && P.admm && valid) {
          // standard ADMM: the pair was feasible, so x^k = z^{k-1} - u^{k-1}
          const float2 pil = P.z_next[(size_t)(I * TILE + r) * E1 + s];
          const float2 pih = P.z_next[(size_t)(I * TILE + r) * E1 + s + 1];
          const float2 pjl = P.z_next[(size_t)j * E1 + s], pjh = P.z_next[(size_t)j * E1 + s + 1];
          uil = finish_u_feasible(pin_lo, uil, pil, zil, P.alpha, res);
          ujl = finish_u_feasible(pin_lo, ujl, pjl, zjl, P.alpha, res);
          uih = finish_u_feasible(pin_hi, uih, pih, zih, P.alpha, res);
          ujh = finish_u_feasible(pin_hi, ujh, pjh, zjh, P.alpha, res);
        } else if (DENSE && !P.keep) {
          uil = ujl = uih = ujh = mk(0.f, 0.f);  // reset rule: inactive edges carry u = 0
        }
        if (pin_lo) { uil = mk(0.f, 0.f); ujl = uil; }
        if (pin_hi) { uih = mk(0.f, 0.f); ujh = uih; }
        act = valid && collides((zjl - ujl) - (zil - uil), (zjh - ujh) - (zih - uih), ri + rj);
        if (DENSE && valid) {
          P.ulo[fid] = pack(uil, ujl);
          P.uhi[fid] = pack(uih, ujh);
        }
      }
      const uint32_t nword = __ballot_sync(FULL, act);
      if (nword != word && lane == 0) P.bits[row] = nword;
      if (nword) {
        if (!DENSE && act) {
          P.ulo[fid] = pack(uil, ujl);
          P.uhi[fid] = pack(uih, ujh);
        }
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(P.work_count, (unsigned)__popc(nword));
        base = __shfl_sync(FULL, base, 0);
        if (act) P.work[base + __popc(nword & ((1u << lane) - 1u))] = (uint32_t)fid;
      }
    }
  }
  res = warp_max(res);
  if (lane == 0 && res > 0.f && P.res_prev) atomic_max_nonneg(P.res_prev, res);
}

// Pass 1 of an iteration, gated state, one warp per (segment s, agent tiles
// I <= J) block with lane = ROW agent i: each lane keeps its row agent in
// registers and walks the 32 column agents, whose data the warp stages in
// shared memory (one broadcast 16-byte load per column).  A lane accumulates
// its row's activity word itself, so a row costs no shuffles, ballots or
// per-row bookkeeping; the pairs of the row that were active in the last
// iteration (set bits) are finished first (deferred step 7, exact test on
// n = z - u), every other valid pair has u = 0 by the reset rule and takes the
// bounding-circle early out before the exact test.  Same decisions and
// stores as test_block<false>; only the worklist order differs.
// col: 64 float4 of shared memory per warp.
// Bounding-circle filter of pass 1.  Agent i's segment lies in the disk of
// centre m_i (its midpoint) and radius b_i (half its length plus r_i), so a
// pair can only collide when |m_i - m_j| <= b_i + b_j, i.e. when
//     m_i . m_j + b_i b_j >= Q_i / 2 + Q_j / 2,   Q = |m|^2 - b^2.
// With a_i = Q_i / 2 - 2e-6 (|m_i|^2 + b_i^2) the test is
// m_i . m_j + b_i b_j - a_i >= a_j.  The margin, 4e-6 of the magnitudes
// involved, is about ten times the rounding of the expression and of the
// bounding radii, so the filter never drops a pair that the exact test would
// find colliding: the outcome is that of testing every pair exactly.
__device__ __forceinline__ float bounding_offset(float2 m, float b) {
  const float mm = dot(m, m), bb = b * b;
  return 0.5f * (mm - bb) - 2e-6f * (mm + bb);
}

// A tile with at least this many exact tests (pairs past the bounding-circle
// filter plus pairs active before) is listed heavy for the next iteration.
constexpr unsigned HEAVY_TESTS = 160;

// check_stamp: the tile is skipped when the heavy-tile stamps show that a
// heavy warp takes it in this iteration.
__device__ __forceinline__ void test_tile_rows(const Dev& P, int blk, float4* col, uint32_t* nws,
                                               bool check_stamp = false) {
  const int lane = threadIdx.x & 31;
  const int E1 = P.eta + 1;
  float res = 0.f;
  const int s = blk / P.ntp;
  int I, J;
  tile_of(P.nt, blk - s * P.ntp, I, J);
  const bool pin_lo = (s == 0), pin_hi = (s == P.eta - 1);
  // Every load the tile starts from is issued here, before any is used: the
  // column agent and the row agent of this lane, the row's activity word,
  // the iteration number and the tile's stamp.
  const int j = J * TILE + lane;
  const bool vj = j < P.p;
  float2 zjl = mk(0.f, 0.f), zjh = zjl;
  float rj = 0.f;
  if (vj) { zjl = ld_now(P.z + (size_t)j * E1 + s); zjh = ld_now(P.z + (size_t)j * E1 + s + 1); rj = ld_now(P.radius + j); }
  const int i = I * TILE + lane;
  const bool vi = i < P.p;
  const size_t row = (size_t)blk * TILE + lane;
  float2 zil = mk(0.f, 0.f), zih = zil;
  float ri = 0.f;
  uint32_t word = 0u;
  if (vi) {
    zil = ld_now(P.z + (size_t)i * E1 + s); zih = ld_now(P.z + (size_t)i * E1 + s + 1); ri = ld_now(P.radius + i);
    word = ld_now(P.bits + row);
  }
  const unsigned it = P.hcap ? ld_now(P.iter) : 0u;
  if (check_stamp && ld_now(P.stamp_cur + blk) == it) return;  // warp-uniform: taken by a heavy warp
  // column agents: (midpoint, bounding radius, bounding_offset), (z lo, z hi)
  // and r_j (col holds 72 float4: the last 8 are the 32 radii)
  float* rcol = reinterpret_cast<float*>(col + 64);
  {
    const float2 m = 0.5f * (zjl + zjh);
    const float b = 0.5f * sqrtf(dot(zjh - zjl, zjh - zjl)) + rj;
    col[lane] = make_float4(m.x, m.y, b, bounding_offset(m, b));
    col[32 + lane] = pack(zjl, zjh);
    rcol[lane] = rj;
  }
  const uint32_t vmask = __ballot_sync(FULL, vj);
  __syncwarp();
  uint32_t valid = vi ? vmask : 0u;
  if (I == J) valid &= (lane == 31) ? 0u : (~0u << (lane + 1));  // pairs i < j
  uint32_t nword = 0u;
  // pairs active in the last iteration: finish step 7, test n = z - u
  // exactly.  They are dealt over the whole warp, one pair per lane per
  // round, so that their u / x loads overlap (a row's own pairs would be
  // fetched one after another); the activity bits come back through nws.
  if (__any_sync(FULL, word != 0u)) {
    unsigned pincl = __popc(word);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(FULL, pincl, o);
      if (lane >= o) pincl += v;
    }
    const unsigned ptot = __shfl_sync(FULL, pincl, 31);
    nws[lane] = 0u;
    __syncwarp();
    for (unsigned base = 0; base < ptot; base += 32) {  // warp-uniform
      const unsigned g = base + lane;
      int r = 0;  // the row of pair g: the first lane whose inclusive count exceeds g
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (__shfl_sync(FULL, pincl, r + step - 1) <= g) r += step;
      const uint32_t wr = __shfl_sync(FULL, word, r);
      const unsigned first = __shfl_sync(FULL, pincl, r) - __popc(wr);
      const float2 zrl = mk(__shfl_sync(FULL, zil.x, r), __shfl_sync(FULL, zil.y, r));
      const float2 zrh = mk(__shfl_sync(FULL, zih.x, r), __shfl_sync(FULL, zih.y, r));
      const float rr = __shfl_sync(FULL, ri, r);
      if (g < ptot) {
        uint32_t w = wr;
        for (unsigned q = first; q < g; ++q) w &= w - 1u;
        const int c = __ffs(w) - 1;
        const size_t fid = ((size_t)blk * TILE + r) * TILE + c;
        const float4 cb = col[32 + c];
        const float rjc = rcol[c];
        const float4 a = P.ulo[fid], b = P.uhi[fid], xa = P.xlo[fid], xb = P.xhi[fid];
        const float2 uil = finish_u(true, pin_lo, false, lo2(a), lo2(xa), zrl, P.alpha, res);
        const float2 ujl = finish_u(true, pin_lo, false, hi2(a), hi2(xa), lo2(cb), P.alpha, res);
        const float2 uih = finish_u(true, pin_hi, false, lo2(b), lo2(xb), zrh, P.alpha, res);
        const float2 ujh = finish_u(true, pin_hi, false, hi2(b), hi2(xb), hi2(cb), P.alpha, res);
        if (collides((lo2(cb) - ujl) - (zrl - uil), (hi2(cb) - ujh) - (zrh - uih), rr + rjc)) {
          P.ulo[fid] = pack(uil, ujl);
          P.uhi[fid] = pack(uih, ujh);
          atomicOr(&nws[r], 1u << c);
        }
      }
    }
    __syncwarp();
    nword = nws[lane];
  }
  // every other valid pair: u = 0, n = z.  The bounding circles of all 32
  // columns first (branch-free), then the exact test on the near ones.
  const uint32_t rest = valid & ~word;
  unsigned work = __popc(word);  // exact tests of this row (scheduling of the next iteration)
  if (__any_sync(FULL, rest != 0u)) {
    const float2 mi = 0.5f * (zil + zih);
    const float bi = 0.5f * sqrtf(dot(zih - zil, zih - zil)) + ri;
    const float ai = bounding_offset(mi, bi);
    uint32_t near = 0u;
#pragma unroll
    for (int c = 0; c < TILE; ++c) {
      const float4 A = col[c];
      // m_i . m_j + b_i b_j - a_i >= a_j: three FMAs and a compare per pair
      const float t = fmaf(mi.x, A.x, fmaf(mi.y, A.y, fmaf(bi, A.z, -ai)));
      near |= (t >= A.w) ? (1u << c) : 0u;
    }
    work += __popc(near & rest);
    for (near &= rest; near; near &= near - 1u) {
      const int c = __ffs(near) - 1;
      const float4 B = col[32 + c];
      if (collides(lo2(B) - zil, hi2(B) - zih, ri + rcol[c])) {
        // a newly active pair starts from u = 0 (the slot may hold an old u)
        const size_t fid = row * TILE + c;
        P.ulo[fid] = make_float4(0.f, 0.f, 0.f, 0.f);
        P.uhi[fid] = make_float4(0.f, 0.f, 0.f, 0.f);
        nword |= 1u << c;
      }
    }
  }
  if (vi && nword != word) P.bits[row] = nword;
  // a heavy tile goes first in the next iteration: its slot is claimed here,
  // so that this atomic and the worklist's below are in flight together
  unsigned hk = ~0u;
  if (P.hcap) {
    const unsigned total = __reduce_add_sync(FULL, work);
    if (lane == 0 && total >= HEAVY_TESTS) hk = atomicAdd(P.hcount_next, 1u);
  }
  // worklist: warp prefix sum of the rows' active counts, one atomic per warp
  if (__any_sync(FULL, nword != 0u)) {
    const unsigned cnt = __popc(nword);
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned total = __shfl_sync(FULL, incl, 31);
    unsigned base = 0;
    if (lane == 31) base = atomicAdd(P.work_count, total);
    base = __shfl_sync(FULL, base, 31) + (incl - cnt);
    for (uint32_t w = nword; w; w &= w - 1u) P.work[base++] = (uint32_t)(row * TILE + (__ffs(w) - 1));
  }
  if (__any_sync(FULL, res > 0.f)) {  // only pairs active before have a residual
    res = warp_max(res);
    if (lane == 0 && P.res_prev) atomic_max_nonneg(P.res_prev, res);
  }
  if (hk < (unsigned)P.hcap) {  // lane 0 of a heavy tile with a free slot
    P.heavy_next[hk] = (uint32_t)blk;
    P.stamp_next[blk] = it + 1u;
  }
}

// Kinetic and wall factors (steps 1-3 and the pending step 7) of one segment
// s and one agent tile: warp f < 1 + n_walls takes factor kind f (0 =
// kinetic, else wall f - 1), lane = agent.  DEFER: see wall_factor.
template <bool DEFER>
__device__ __forceinline__ void segment_block(const Dev& P, int blk) {
  const int s = blk / P.nt;
  const int I = blk - s * P.nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = I * TILE + lane;
  const bool vi = i < P.p;
  const int E1 = P.eta + 1;
  const bool pin_lo = (s == 0), pin_hi = (s == P.eta - 1);
  float2 zl = mk(0.f, 0.f), zh = zl;
  float r = 0.f;
  if (vi) { zl = P.z[(size_t)i * E1 + s]; zh = P.z[(size_t)i * E1 + s + 1]; r = P.radius[i]; }
  float res = 0.f;
  for (int f = warp; f < 1 + P.nw + P.nv; f += blockDim.x >> 5) {
    if (f == 0) {
      if (vi && !P.noenergy && !(P.vo && s == 0)) kinetic_factor(P, i, s, zl, zh, pin_lo, pin_hi, res);
    } else if (!(P.vo && s != 0)) {
      wall_factor<DEFER>(P, f - 1, i, vi, s, I, zl, zh, r, pin_lo, pin_hi, res);
    }
  }
  res = warp_max(res);
  if (lane == 0 && res > 0.f && P.res_prev) atomic_max_nonneg(P.res_prev, res);
}

// The capsule minimizer (Eq. wall_minimizer) of one active wall factor from
// the wall worklist, with the u that its segment block finished (so n = z - u
// is the value it tested).  Called by all 32 lanes of a warp with the same
// item: both ends free (the common case) shares the candidate solves out
// over the lanes; lane 0 stores the result.
__device__ __forceinline__ void wall_prox_item_warp(const Dev& P, uint32_t idx) {
  const uint32_t i = idx % (uint32_t)P.p, ws = idx / (uint32_t)P.p;
  const int s = (int)(ws % (uint32_t)P.eta), w = (int)(ws / (uint32_t)P.eta);
  const int E1 = P.eta + 1;
  const bool pin_lo = (s == 0), pin_hi = (s == P.eta - 1);
  const float4 u4 = P.uwall[idx];
  const float2 ul = lo2(u4), uh = hi2(u4);
  const float2 nl = P.z[(size_t)i * E1 + s] - ul, nh = P.z[(size_t)i * E1 + s + 1] - uh;
  const float4 W = P.walls[w];
  const float2 c0 = mk(W.x, W.y), c1 = mk(W.z, W.w);
  const float r = P.radius[i];
  int cl, ch;
  end_classes(P, (int)i, s, pin_lo, pin_hi, cl, ch);
  float2 xl = nl, xh = nh;
  bool ok = true;
  if (cl == 1 && ch == 1) {
    const float wgt = 0.5f * P.rho;
    capsule_prox_free_warp(nl, nh, wgt, wgt, c0, c1, r, xl, xh);
  } else {
    ok = capsule_prox_classes(nl, nh, cl, ch, c0, c1, r, 0.5f * P.rho, xl, xh);
  }
  if ((threadIdx.x & 31) != 0) return;
  if (!ok) atomicOr(P.status, 1u);
  P.xwall[idx] = pack(xl, xh);
  if (!pin_lo) contribute(P, (int)i, s, xl + ul);
  if (!pin_hi) contribute(P, (int)i, s + 1, xh + uh);
}

// Pass 2: the collision minimizer (Eq. coll_minimizer_problem through
// App. C/D/I) of every active pair in the worklist, one thread per pair.
__device__ __forceinline__ void prox_item(const Dev& P, uint32_t fid) {
  const int E1 = P.eta + 1;
  const uint32_t row = fid >> 5, c = fid & 31;
  const uint32_t blk = row >> 5, r = row & 31;
  const int s = (int)(blk / P.ntp);
  int I, J;
  tile_of(P.nt, (int)(blk - (uint32_t)s * P.ntp), I, J);
  const int i = I * TILE + r, j = J * TILE + c;
  const float scale = P.fix[0], bound = P.fix[1];  // loaded beside the minimizer
  const float4 a = P.ulo[fid], b = P.uhi[fid];
  const float2 nil = P.z[(size_t)i * E1 + s] - lo2(a), nih = P.z[(size_t)i * E1 + s + 1] - lo2(b);
  const float2 njl = P.z[(size_t)j * E1 + s] - hi2(a), njh = P.z[(size_t)j * E1 + s + 1] - hi2(b);
  float2 xil, xih, xjl, xjh;
  const bool pin_lo = (s == 0), pin_hi = (s == P.eta - 1);
  if (P.noenergy) {
    int cil, cih, cjl, cjh;
    end_classes(P, i, s, pin_lo, pin_hi, cil, cih);
    end_classes(P, j, s, pin_lo, pin_hi, cjl, cjh);
    coll_minimizer_classes(nil, nih, njl, njh, cil, cih, cjl, cjh, P.radius[i] + P.radius[j],
                           P.rho, xil, xih, xjl, xjh);
  } else {
    coll_minimizer(nil, nih, njl, njh, pin_lo, pin_hi, P.radius[i] + P.radius[j], P.rho,
                   xil, xih, xjl, xjh);
  }
  P.xlo[fid] = pack(xil, xjl);
  P.xhi[fid] = pack(xih, xjh);
  if (!pin_lo) {
    contribute(P, scale, bound, i, s, xil + lo2(a));
    contribute(P, scale, bound, j, s, xjl + hi2(a));
  }
  if (!pin_hi) {
    contribute(P, scale, bound, i, s + 1, xih + lo2(b));
    contribute(P, scale, bound, j, s + 1, xjh + hi2(b));
  }
}

// Pass 3 (steps 5-6): z = sum(rho m) / sum(rho) per free break-point from the
// fixed-point sums (every weight is rho0, so z is the mean of the incoming m;
// no incoming weight means z is unchanged).  Clears the sums for the next
// iteration.
__device__ __forceinline__ void consensus_node(const Dev& P, int t, float& dz, bool& bad) {
  // consecutive threads take consecutive break-points of one agent, which
  // are adjacent in the [p][eta+1] arrays (coalesced)
  const int i = t / (P.eta - 1);
  const int sp = 1 + (t - i * (P.eta - 1));
  const size_t node = (size_t)i * (P.eta + 1) + sp;
  const unsigned status = *P.status;  // issued with the sums, not after them
  const long long sx = (long long)P.accx[node], sy = (long long)P.accy[node];
  const unsigned cnt = P.accc[node];
  const float2 zo = P.z[node];  // every load before the stores, so that they overlap
  P.accx[node] = 0ull;
  P.accy[node] = 0ull;
  P.accc[node] = 0u;
  float2 zn = zo;  // every incoming weight zero: treated as 1, which gives z unchanged
  if (P.admm) {
    // every edge is weighted; each feasible collision or wall factor sent
    // m = n + u = z^k, added here in the same exact fixed point
    const unsigned deg = 2u * (unsigned)(P.p - 1) + 2u + 2u * (unsigned)P.nw;
    const long long rest = (long long)(deg - cnt);
    const long long qx = __float2ll_rn(zo.x * P.fix[0]), qy = __float2ll_rn(zo.y * P.fix[0]);
    const float den = P.fix[0] * (float)deg;  // exact: a power of two times a small count
    zn = mk(__ll2float_rn(sx + rest * qx) / den, __ll2float_rn(sy + rest * qy) / den);
  } else if (cnt > 0u) {
    // the exact integer sum rounded once to FP32, then one FP32 division
    const float den = P.fix[0] * (float)cnt;
    zn = mk(__ll2float_rn(sx) / den, __ll2float_rn(sy) / den);
  }
  // step 6: the back weight is rho0 where some factor sent rho0, else 0
  if (P.noenergy) P.wnode[node] = cnt > 0u ? 1 : 0;
  P.z_next[node] = zn;
  bad = (status & 2u) != 0u || !(fabsf(zn.x - zo.x) + fabsf(zn.y - zo.y) >= 0.f);
  dz = bad ? 0.f : maxabs2(zn - zo);
}

// Warp-level end of the consensus pass: a NaN or overflow anywhere makes the
// residual NaN (reported as PLAN_ENUMERIC).  All 32 lanes must call it.
__device__ __forceinline__ void consensus_reduce(const Dev& P, float dz, bool bad) {
  dz = warp_max(dz);
  const bool anybad = __any_sync(FULL, bad);
  if ((threadIdx.x & 31) == 0) {
    if (anybad) atomicMax(P.res_cur, 0x7fc00000u);
    else if (dz > 0.f) atomic_max_nonneg(P.res_cur, dz);
  }
}

}  // namespace

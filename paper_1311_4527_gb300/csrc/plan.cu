// plan.cu -- GB300 (sm_103a) kernels and C ABI of the three-weight ADMM
// trajectory planner (Bento, Derbinsky, Alonso-Mora, Yedidia, NIPS 2013).
//
// One iteration = Appendix B steps 1-7 over the factor graph of Section 3.3,
// run as two kernels:
//
//   factor_kernel  one CTA per (segment s, agent tile I, agent tile J >= I):
//                  every collision factor (s, i in I, j in J, i < j) of the
//                  tile -- and, in the diagonal CTAs, the kinetic and wall
//                  factors of the agents of I at segment s.  Per factor: finish
//                  the pending dual update of the previous iteration (step 7),
//                  form n = z - u (step 1), run the minimizer and its weight
//                  logic (steps 2-3), form m = x + u (step 4) and add the
//                  weighted m into per-tile consensus partial sums (warp
//                  shuffles for the row agent, registers + shared memory for
//                  the column agent).  One store per (tile, agent, component).
//   consensus_kernel  one thread per free break-point: z = sum(rho m) /
//                  sum(rho) over the tile partials in a fixed order (step 5,
//                  deterministic), and |z_new - z_old| for the residual.
//
// Step 7 needs z^{k+1}, which exists only after every factor ran.  The factor
// kernel therefore stores x^{k+1} of the factors that sent rho0 and finishes
// u^{k+1} = u^k + alpha (x^{k+1} - z^{k+1}) at the start of the next
// iteration.  Back weights (step 6) are rho0 at every interior node, because
// the kinetic factors always send rho0 there, and infinity at the fixed ends;
// u on an edge whose forward weight was 0, or whose node is fixed, is 0.
//
// Collision-factor state lives in tile order: for CTA blk = s * ntp + tp the
// 32 x 32 pair slots (row r = i - 32 I, column c = j - 32 J) are contiguous,
// so a warp streams one row as 32 consecutive float4 (512 B).  Per slot:
//   ulo[slot] = (u_i(s), u_j(s))       uhi[slot] = (u_i(s+1), u_j(s+1))
//   xlo / xhi = pending x^{k+1}, read and written only for active factors
//   bits[blk * 32 + r] bit c = forward weight rho0 in the last iteration.
// With PLAN_DENSE_STATE the u record of every slot is read and written each
// iteration; otherwise only those of factors whose bit is set (every other u
// is 0 by the reset rule), which leaves 1 bit per factor of state traffic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"
#include "twa_math.cuh"

using namespace twa;

namespace {

constexpr int TILE = 32;
constexpr int WARPS = 8;
constexpr int THREADS = TILE * WARPS;
constexpr int ROWS = TILE / WARPS;  // rows of a tile per warp
constexpr unsigned FULL = 0xffffffffu;

struct Dev {
  int p, eta, nw, nt, ntp;
  float rho, alpha;
  int dense, keep, admm;
  const float2* z;       // z^k, [p][eta+1]
  float2* z_next;        // z^{k+1}; until the consensus pass writes it, z^{k-1}
  const float* radius;   // [p]
  const float* cost;     // [p][eta], kinetic coefficients c_{i,s}
  const float4* walls;   // [nw] (xL.x, xL.y, xR.x, xR.y)
  const int2* tiles;     // [ntp] (I, J), I <= J
  float4 *ulo, *uhi, *xlo, *xhi;
  uint32_t* bits;        // [eta * ntp * 32]
  float4 *ukin, *xkin;   // [eta][p]
  float4 *uwall, *xwall; // [nw][eta][p]
  uint32_t* wbits;       // [nw][eta][nt]
  uint32_t* work;        // active collision slots of this iteration
  unsigned* work_count;  // their number
  unsigned* work_count_next;  // the counter the next iteration appends to
  unsigned long long* accx;  // [p][eta+1] fixed-point sums of rho0-weighted m.x
  unsigned long long* accy;  //                                 ... of m.y
  unsigned* accc;        // [p][eta+1] number of rho0-weighted incoming edges
  const float* fix;      // fixed-point scale (a power of two) and |m| bound
  unsigned* res_cur;     // residual slot of this iteration (consensus part)
  unsigned* res_prev;    // residual slot of the previous iteration (primal part)
  unsigned* status;      // bit 0: a pinned wall minimizer had no separating direction
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

// Step 5's sums in 64-bit fixed point: each FP32 m converts exactly (the scale
// is a power of two chosen from the layout's extent), integer addition does not
// depend on the order of the atomics, so z is deterministic and is the
// correctly rounded mean of the incoming m's.  A non-finite or out-of-range m
// sets status bit 1, which the consensus pass turns into a NaN residual.
__device__ __forceinline__ void contribute(const Dev& P, int i, int s, float2 m) {
  const float scale = P.fix[0], bound = P.fix[1];
  if (!(fabsf(m.x) <= bound && fabsf(m.y) <= bound)) {
    atomicOr(P.status, 2u);
    return;
  }
  const size_t node = (size_t)i * (P.eta + 1) + s;
  atomicAdd(P.accx + node, (unsigned long long)__float2ll_rn(m.x * scale));
  atomicAdd(P.accy + node, (unsigned long long)__float2ll_rn(m.y * scale));
  atomicAdd(P.accc + node, 1u);
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
  if (pin_lo) {
    float2 vh = disk_prox_pinned(cl, ch, R);
    xih = 0.5f * (sh - vh);
    xjh = 0.5f * (sh + vh);
  } else if (pin_hi) {
    float2 vl = disk_prox_pinned(ch, cl, R);
    xil = 0.5f * (sl - vl);
    xjl = 0.5f * (sl + vl);
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

// Wall factor (w, i, s).  Called by a full warp (lane = agent of tile I).
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
  const float4 W = P.walls[w];
  const float2 c0 = mk(W.x, W.y), c1 = mk(W.z, W.w);
  const bool act = vi && dist2_segment_segment(nl, nh, c0, c1) < r * r;
  const uint32_t nw = __ballot_sync(FULL, act);
  if (lane == 0 && nw != word) P.wbits[widx] = nw;
  if (act) {
    float2 xl = nl, xh = nh;
    if (pin_lo && pin_hi) {
    } else if (pin_lo) {
      if (!capsule_prox_pinned(nl, nh, c0, c1, r, xh)) atomicOr(P.status, 1u);
    } else if (pin_hi) {
      if (!capsule_prox_pinned(nh, nl, c0, c1, r, xl)) atomicOr(P.status, 1u);
    } else {
      const float wgt = 0.5f * P.rho;
      capsule_prox_free(nl, nh, wgt, wgt, c0, c1, r, xl, xh);
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
constexpr int TEST_WARPS = 4;
constexpr int TEST_ROWS = TILE / TEST_WARPS;

template <bool DENSE>
__global__ void __launch_bounds__(32 * TEST_WARPS) test_kernel(Dev P) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int blk = blockIdx.x;
  const int E1 = P.eta + 1;
  float res = 0.f;
  if (blk == 0 && threadIdx.x == 0) *P.res_cur = 0u;
  const int s = blk / P.ntp;
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

// Kinetic and wall factors (steps 1-3 and the pending step 7) of one segment
// s and one agent tile: warp f < 1 + n_walls takes factor kind f (0 =
// kinetic, else wall f - 1), lane = agent.
__global__ void __launch_bounds__(THREADS) segment_kernel(Dev P) {
  const int s = blockIdx.x / P.nt;
  const int I = blockIdx.x - s * P.nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = I * TILE + lane;
  const bool vi = i < P.p;
  const int E1 = P.eta + 1;
  const bool pin_lo = (s == 0), pin_hi = (s == P.eta - 1);
  float2 zl = mk(0.f, 0.f), zh = zl;
  float r = 0.f;
  if (vi) { zl = P.z[(size_t)i * E1 + s]; zh = P.z[(size_t)i * E1 + s + 1]; r = P.radius[i]; }
  float res = 0.f;
  for (int f = warp; f < 1 + P.nw; f += blockDim.x >> 5) {
    if (f == 0) {
      if (vi) kinetic_factor(P, i, s, zl, zh, pin_lo, pin_hi, res);
    } else {
      wall_factor(P, f - 1, i, vi, s, I, zl, zh, r, pin_lo, pin_hi, res);
    }
  }
  res = warp_max(res);
  if (lane == 0 && res > 0.f && P.res_prev) atomic_max_nonneg(P.res_prev, res);
}

// Pass 2: the collision minimizer (Eq. coll_minimizer_problem through
// App. C/D/I) of every active pair in the worklist, one thread per pair.
__global__ void __launch_bounds__(256) prox_kernel(Dev P) {
  const unsigned n = *P.work_count;
  const int E1 = P.eta + 1;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const uint32_t fid = P.work[t];
    const uint32_t row = fid >> 5, c = fid & 31;
    const uint32_t blk = row >> 5, r = row & 31;
    const int s = (int)(blk / P.ntp);
    const int2 IJ = P.tiles[blk - (uint32_t)s * P.ntp];
    const int i = IJ.x * TILE + r, j = IJ.y * TILE + c;
    const float4 a = P.ulo[fid], b = P.uhi[fid];
    const float2 nil = P.z[(size_t)i * E1 + s] - lo2(a), nih = P.z[(size_t)i * E1 + s + 1] - lo2(b);
    const float2 njl = P.z[(size_t)j * E1 + s] - hi2(a), njh = P.z[(size_t)j * E1 + s + 1] - hi2(b);
    float2 xil, xih, xjl, xjh;
    const bool pin_lo = (s == 0), pin_hi = (s == P.eta - 1);
    coll_minimizer(nil, nih, njl, njh, pin_lo, pin_hi, P.radius[i] + P.radius[j], P.rho,
                   xil, xih, xjl, xjh);
    P.xlo[fid] = pack(xil, xjl);
    P.xhi[fid] = pack(xih, xjh);
    if (!pin_lo) {
      contribute(P, i, s, xil + lo2(a));
      contribute(P, j, s, xjl + hi2(a));
    }
    if (!pin_hi) {
      contribute(P, i, s + 1, xih + lo2(b));
      contribute(P, j, s + 1, xjh + hi2(b));
    }
  }
}

// Pass 3 (steps 5-6): z = sum(rho m) / sum(rho) per free break-point from the
// fixed-point sums (every weight is rho0, so z is the mean of the incoming m;
// no incoming weight means z is unchanged).  Clears the sums for the next
// iteration.
__global__ void consensus_kernel(Dev P) {
  const int nfree = (P.eta - 1) * P.p;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) *P.work_count_next = 0u;
  float dz = 0.f;
  bool bad = false;
  if (t < nfree) {
    const int sp = 1 + t / P.p;
    const int i = t - (sp - 1) * P.p;
    const size_t node = (size_t)i * (P.eta + 1) + sp;
    const long long sx = (long long)P.accx[node], sy = (long long)P.accy[node];
    const unsigned cnt = P.accc[node];
    P.accx[node] = 0ull;
    P.accy[node] = 0ull;
    P.accc[node] = 0u;
    const float2 zo = P.z[node];
    float2 zn = zo;  // every incoming weight zero: treated as 1, which gives z unchanged
    if (P.admm) {
      // every edge is weighted; each feasible collision or wall factor sent
      // m = n + u = z^k, added here in the same exact fixed point
      const unsigned deg = 2u * (unsigned)(P.p - 1) + 2u + 2u * (unsigned)P.nw;
      const long long rest = (long long)(deg - cnt);
      const long long qx = __float2ll_rn(zo.x * P.fix[0]), qy = __float2ll_rn(zo.y * P.fix[0]);
      const double den = (double)P.fix[0] * (double)deg;
      zn = mk((float)((double)(sx + rest * qx) / den), (float)((double)(sy + rest * qy) / den));
    } else if (cnt > 0u) {
      const double den = (double)P.fix[0] * (double)cnt;
      zn = mk((float)((double)sx / den), (float)((double)sy / den));
    }
    P.z_next[node] = zn;
    bad = (*P.status & 2u) != 0u || !(fabsf(zn.x - zo.x) + fabsf(zn.y - zo.y) >= 0.f);
    dz = bad ? 0.f : maxabs2(zn - zo);
  }
  // a NaN or overflow anywhere makes the residual NaN (reported as PLAN_ENUMERIC)
  dz = warp_max(dz);
  const bool anybad = __any_sync(FULL, bad);
  if ((threadIdx.x & 31) == 0) {
    if (anybad) atomicMax(P.res_cur, 0x7fc00000u);
    else if (dz > 0.f) atomic_max_nonneg(P.res_cur, dz);
  }
}

// Fixed-point scale of the consensus sums: the largest power of two with
// 8 (L + 1) x (max incoming edges) x scale <= 2^62, L the largest coordinate
// magnitude of the endpoints and walls.  One block.
__global__ void fix_kernel(Dev P, const float2* start, const float2* goal) {
  __shared__ float red[256];
  float L = 0.f;
  for (int k = threadIdx.x; k < P.p; k += blockDim.x)
    L = fmaxf(L, fmaxf(maxabs2(start[k]), maxabs2(goal[k])));
  for (int k = threadIdx.x; k < P.nw; k += blockDim.x) {
    const float4 w = P.walls[k];
    L = fmaxf(L, fmaxf(fmaxf(fabsf(w.x), fabsf(w.y)), fmaxf(fabsf(w.z), fabsf(w.w))));
  }
  red[threadIdx.x] = L;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double edges = 2.0 + 2.0 * (P.p - 1) + 2.0 * P.nw;
    const double bound = 8.0 * ((double)red[0] + 1.0);
    int e = (int)floor(log2(4.611686018427388e18 / (bound * edges)));
    e = e < 8 ? 8 : (e > 60 ? 60 : e);
    float* f = const_cast<float*>(P.fix);
    f[0] = ldexpf(1.f, e);
    f[1] = (float)bound;
  }
}

// Primal residual max |x^k - z^k| over weighted edges, without changing state
// (the same finishing arithmetic the next factor_kernel will apply).
__global__ void residual_kernel(Dev P) {
  float res = 0.f;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int E1 = P.eta + 1;
  const size_t nrows = (size_t)P.eta * P.ntp * TILE;
  for (size_t row = gw; row < nrows; row += nwarps) {
    uint32_t word = P.bits[row];
    if (P.admm && !((word >> lane) & 1u)) {
      // standard ADMM: a feasible pair's x is z^{k-1} - u^{k-1}
      const size_t blk = row / TILE;
      const int r = (int)(row - blk * TILE);
      const int s = (int)(blk / P.ntp);
      const int2 IJ = P.tiles[blk - (size_t)s * P.ntp];
      const int i = IJ.x * TILE + r, j = IJ.y * TILE + lane;
      if (i >= P.p || j >= P.p || (IJ.x == IJ.y && r >= lane)) continue;
      const size_t fid = row * TILE + lane;
      const float4 a = P.ulo[fid], b = P.uhi[fid];
      if (s != 0) {
        finish_u_feasible(false, lo2(a), P.z_next[(size_t)i * E1 + s], P.z[(size_t)i * E1 + s], P.alpha, res);
        finish_u_feasible(false, hi2(a), P.z_next[(size_t)j * E1 + s], P.z[(size_t)j * E1 + s], P.alpha, res);
      }
      if (s != P.eta - 1) {
        finish_u_feasible(false, lo2(b), P.z_next[(size_t)i * E1 + s + 1], P.z[(size_t)i * E1 + s + 1], P.alpha, res);
        finish_u_feasible(false, hi2(b), P.z_next[(size_t)j * E1 + s + 1], P.z[(size_t)j * E1 + s + 1], P.alpha, res);
      }
      continue;
    }
    if (!((word >> lane) & 1u)) continue;
    const size_t blk = row / TILE;
    const int r = (int)(row - blk * TILE);
    const int s = (int)(blk / P.ntp);
    const int2 IJ = P.tiles[blk - (size_t)s * P.ntp];
    const int i = IJ.x * TILE + r, j = IJ.y * TILE + lane;
    const size_t fid = row * TILE + lane;
    float4 xl = P.xlo[fid], xh = P.xhi[fid];
    if (s != 0) {
      res = fmaxf(res, maxabs2(lo2(xl) - P.z[(size_t)i * E1 + s]));
      res = fmaxf(res, maxabs2(hi2(xl) - P.z[(size_t)j * E1 + s]));
    }
    if (s != P.eta - 1) {
      res = fmaxf(res, maxabs2(lo2(xh) - P.z[(size_t)i * E1 + s + 1]));
      res = fmaxf(res, maxabs2(hi2(xh) - P.z[(size_t)j * E1 + s + 1]));
    }
  }
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int t = gt; t < P.eta * P.p; t += nth) {
    const int s = t / P.p, i = t - s * P.p;
    float4 x = P.xkin[t];
    if (s != 0) res = fmaxf(res, maxabs2(lo2(x) - P.z[(size_t)i * E1 + s]));
    if (s != P.eta - 1) res = fmaxf(res, maxabs2(hi2(x) - P.z[(size_t)i * E1 + s + 1]));
  }
  for (int t = gt; t < P.nw * P.eta * P.p; t += nth) {
    const int i = t % P.p;
    const int ws = t / P.p;
    const int s = ws % P.eta;
    const uint32_t word = P.wbits[(size_t)ws * P.nt + i / TILE];
    if (!((word >> (i % TILE)) & 1u)) {
      if (P.admm) {  // feasible wall factor in standard ADMM: x = z^{k-1} - u^{k-1}
        const float4 u = P.uwall[t];
        if (s != 0) finish_u_feasible(false, lo2(u), P.z_next[(size_t)i * E1 + s], P.z[(size_t)i * E1 + s], P.alpha, res);
        if (s != P.eta - 1) finish_u_feasible(false, hi2(u), P.z_next[(size_t)i * E1 + s + 1], P.z[(size_t)i * E1 + s + 1], P.alpha, res);
      }
      continue;
    }
    float4 x = P.xwall[t];
    if (s != 0) res = fmaxf(res, maxabs2(lo2(x) - P.z[(size_t)i * E1 + s]));
    if (s != P.eta - 1) res = fmaxf(res, maxabs2(hi2(x) - P.z[(size_t)i * E1 + s + 1]));
  }
  res = warp_max(res);
  if (lane == 0 && res > 0.f) atomic_max_nonneg(P.res_prev, res);
}

// Initial state (Section 4): z = start except the goal node; u = 0; the
// kinetic pending x equals z so that the first finishing step gives u = 0.
__global__ void reset_kernel(Dev P, float2* z0, float2* z1, const float2* start,
                             const float2* goal) {
  const int E1 = P.eta + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < P.p * E1) {
    const int i = t / E1, s = t - i * E1;
    float2 v = (s == P.eta) ? goal[i] : start[i];
    z0[t] = v;
    z1[t] = v;
  }
  if (t < P.eta * P.p) {
    const int s = t / P.p, i = t - s * P.p;
    float2 zl = start[i];
    float2 zh = (s + 1 == P.eta) ? goal[i] : start[i];
    P.xkin[t] = pack(zl, zh);
    P.ukin[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// New fixed ends: overwrite the s = 0 and s = eta nodes of both z buffers.
__global__ void endpoints_kernel(int p, int eta, float2* z0, float2* z1, const float2* start,
                                 const float2* goal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  const size_t b = (size_t)i * (eta + 1);
  z0[b] = start[i]; z1[b] = start[i];
  z0[b + eta] = goal[i]; z1[b + eta] = goal[i];
}

__device__ __forceinline__ size_t pair_index(int p, int i, int j) {
  return (size_t)i * (2 * (size_t)p - i - 1) / 2 + (size_t)(j - i - 1);
}

// State export in the paper's variables (u^k after finishing step 7).
__global__ void export_coll_kernel(Dev P, float* u_coll, uint8_t* act) {
  const size_t slot = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nslots = (size_t)P.eta * P.ntp * TILE * TILE;
  if (slot >= nslots) return;
  const size_t row = slot / TILE;
  const int lane = (int)(slot - row * TILE);
  const size_t blk = row / TILE;
  const int r = (int)(row - blk * TILE);
  const int s = (int)(blk / P.ntp);
  const int2 IJ = P.tiles[blk - (size_t)s * P.ntp];
  const int i = IJ.x * TILE + r, j = IJ.y * TILE + lane;
  if (i >= P.p || j >= P.p || i >= j) return;
  const int E1 = P.eta + 1;
  const bool bprev = (P.bits[row] >> lane) & 1u;
  float4 ul4 = P.ulo[slot], uh4 = P.uhi[slot];
  if (!P.dense && !bprev) { ul4 = make_float4(0.f, 0.f, 0.f, 0.f); uh4 = ul4; }
  float4 xl4 = make_float4(0.f, 0.f, 0.f, 0.f), xh4 = xl4;
  if (bprev) { xl4 = P.xlo[slot]; xh4 = P.xhi[slot]; }
  const bool pin_lo = (s == 0), pin_hi = (s == P.eta - 1);
  float dummy = 0.f;
  float2 uil, ujl, uih, ujh;
  if (P.admm && !bprev) {
    uil = finish_u_feasible(pin_lo, lo2(ul4), P.z_next[(size_t)i * E1 + s], P.z[(size_t)i * E1 + s], P.alpha, dummy);
    ujl = finish_u_feasible(pin_lo, hi2(ul4), P.z_next[(size_t)j * E1 + s], P.z[(size_t)j * E1 + s], P.alpha, dummy);
    uih = finish_u_feasible(pin_hi, lo2(uh4), P.z_next[(size_t)i * E1 + s + 1], P.z[(size_t)i * E1 + s + 1], P.alpha, dummy);
    ujh = finish_u_feasible(pin_hi, hi2(uh4), P.z_next[(size_t)j * E1 + s + 1], P.z[(size_t)j * E1 + s + 1], P.alpha, dummy);
  } else {
    uil = finish_u(bprev, pin_lo, P.keep, lo2(ul4), lo2(xl4), P.z[(size_t)i * E1 + s], P.alpha, dummy);
    ujl = finish_u(bprev, pin_lo, P.keep, hi2(ul4), hi2(xl4), P.z[(size_t)j * E1 + s], P.alpha, dummy);
    uih = finish_u(bprev, pin_hi, P.keep, lo2(uh4), lo2(xh4), P.z[(size_t)i * E1 + s + 1], P.alpha, dummy);
    ujh = finish_u(bprev, pin_hi, P.keep, hi2(uh4), hi2(xh4), P.z[(size_t)j * E1 + s + 1], P.alpha, dummy);
  }
  const size_t P2 = (size_t)P.p * (P.p - 1) / 2;
  const size_t q = (size_t)s * P2 + pair_index(P.p, i, j);
  if (u_coll) {
    float* o = u_coll + q * 8;
    o[0] = uil.x; o[1] = uil.y; o[2] = uih.x; o[3] = uih.y;
    o[4] = ujl.x; o[5] = ujl.y; o[6] = ujh.x; o[7] = ujh.y;
  }
  if (act) act[q] = bprev ? 1 : 0;
}

__global__ void export_seg_kernel(Dev P, float* u_kin, float* u_wall, uint8_t* act_wall) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int E1 = P.eta + 1;
  const int nk = P.eta * P.p;
  float dummy = 0.f;
  if (t < nk) {
    const int s = t / P.p, i = t - s * P.p;
    float4 u4 = P.ukin[t], x4 = P.xkin[t];
    float2 ul = finish_u(true, s == 0, false, lo2(u4), lo2(x4), P.z[(size_t)i * E1 + s], P.alpha, dummy);
    float2 uh = finish_u(true, s == P.eta - 1, false, hi2(u4), hi2(x4), P.z[(size_t)i * E1 + s + 1], P.alpha, dummy);
    if (u_kin) {
      float* o = u_kin + (size_t)t * 4;
      o[0] = ul.x; o[1] = ul.y; o[2] = uh.x; o[3] = uh.y;
    }
  }
  if (t < P.nw * nk) {
    const int i = t % P.p, ws = t / P.p, s = ws % P.eta;
    const bool bprev = (P.wbits[(size_t)ws * P.nt + i / TILE] >> (i % TILE)) & 1u;
    float4 u4 = P.uwall[t], x4 = P.xwall[t];
    if (!P.dense && !bprev) u4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 ul, uh;
    if (P.admm && !bprev) {
      ul = finish_u_feasible(s == 0, lo2(u4), P.z_next[(size_t)i * E1 + s], P.z[(size_t)i * E1 + s], P.alpha, dummy);
      uh = finish_u_feasible(s == P.eta - 1, hi2(u4), P.z_next[(size_t)i * E1 + s + 1], P.z[(size_t)i * E1 + s + 1], P.alpha, dummy);
    } else {
      ul = finish_u(bprev, s == 0, P.keep, lo2(u4), lo2(x4), P.z[(size_t)i * E1 + s], P.alpha, dummy);
      uh = finish_u(bprev, s == P.eta - 1, P.keep, hi2(u4), hi2(x4), P.z[(size_t)i * E1 + s + 1], P.alpha, dummy);
    }
    if (u_wall) {
      float* o = u_wall + (size_t)t * 4;
      o[0] = ul.x; o[1] = ul.y; o[2] = uh.x; o[3] = uh.y;
    }
    if (act_wall) act_wall[t] = bprev ? 1 : 0;
  }
}

// State import: u^k becomes the stored u with the pending x set to z^k, so
// the next finishing step reproduces u^k exactly (u + alpha * 0).
__global__ void import_coll_kernel(Dev P, const float* u_coll) {
  const size_t slot = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nslots = (size_t)P.eta * P.ntp * TILE * TILE;
  const int lane = threadIdx.x & 31;
  bool nz = false;
  size_t row = slot / TILE;
  if (slot < nslots) {
    const size_t blk = row / TILE;
    const int r = (int)(row - blk * TILE);
    const int s = (int)(blk / P.ntp);
    const int2 IJ = P.tiles[blk - (size_t)s * P.ntp];
    const int i = IJ.x * TILE + r, j = IJ.y * TILE + lane;
    float4 ul = make_float4(0.f, 0.f, 0.f, 0.f), uh = ul, xl = ul, xh = ul;
    if (i < P.p && j < P.p && i < j) {
      const int E1 = P.eta + 1;
      const size_t P2 = (size_t)P.p * (P.p - 1) / 2;
      const float* u = u_coll + ((size_t)s * P2 + pair_index(P.p, i, j)) * 8;
      ul = make_float4(u[0], u[1], u[4], u[5]);
      uh = make_float4(u[2], u[3], u[6], u[7]);
      xl = pack(P.z[(size_t)i * E1 + s], P.z[(size_t)j * E1 + s]);
      xh = pack(P.z[(size_t)i * E1 + s + 1], P.z[(size_t)j * E1 + s + 1]);
      // flagged pairs finish from the stored x = z^k, which reproduces u^k
      // exactly; in standard ADMM every pair must take that path after import
      nz = P.admm || ul.x != 0.f || ul.y != 0.f || ul.z != 0.f || ul.w != 0.f ||
           uh.x != 0.f || uh.y != 0.f || uh.z != 0.f || uh.w != 0.f;
    }
    P.ulo[slot] = ul; P.uhi[slot] = uh; P.xlo[slot] = xl; P.xhi[slot] = xh;
  }
  uint32_t word = __ballot_sync(FULL, nz);
  if (lane == 0 && slot < nslots) P.bits[row] = word;
}

__global__ void import_seg_kernel(Dev P, const float* u_kin, const float* u_wall) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int E1 = P.eta + 1;
  const int nk = P.eta * P.p;
  if (t < nk) {
    const int s = t / P.p, i = t - s * P.p;
    const float* u = u_kin + (size_t)t * 4;
    P.ukin[t] = make_float4(u[0], u[1], u[2], u[3]);
    P.xkin[t] = pack(P.z[(size_t)i * E1 + s], P.z[(size_t)i * E1 + s + 1]);
  }
  if (t < P.nw * nk) {
    const int i = t % P.p, s = (t / P.p) % P.eta;
    const float* u = u_wall + (size_t)t * 4;
    P.uwall[t] = make_float4(u[0], u[1], u[2], u[3]);
    P.xwall[t] = pack(P.z[(size_t)i * E1 + s], P.z[(size_t)i * E1 + s + 1]);
  }
}

// wall bits: one 32-agent word per (wall, segment, tile); set where u != 0
__global__ void import_wbits_kernel(Dev P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per (w, s, tile, lane)
  const int lane = threadIdx.x & 31;
  const int words = P.nw * P.eta * P.nt;
  const int w = t >> 5;
  bool nz = false;
  if (w < words) {
    const int tile = w % P.nt, ws = w / P.nt;
    const int i = tile * TILE + lane;
    if (i < P.p) {
      float4 u = P.uwall[(size_t)ws * P.p + i];
      nz = P.admm || u.x != 0.f || u.y != 0.f || u.z != 0.f || u.w != 0.f;
    }
  }
  uint32_t word = __ballot_sync(FULL, nz);
  if (lane == 0 && w < words) P.wbits[w] = word;
}

__global__ void count_kernel(const uint32_t* words, size_t n, unsigned long long* out) {
  unsigned long long c = 0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    c += __popc(words[t]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

thread_local std::string g_err;

plan_status fail(plan_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(PLAN_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t z0, z1, start, goal, radius, cost, walls, tiles;
  size_t ulo, uhi, xlo, xhi, bits, ukin, xkin, uwall, xwall, wbits, work, wcount, accx, accy, accc, fix,
      res, status, count;
  size_t total;
};

bool sizes_ok(const plan_config* c) {
  if (c->p < 1 || c->eta < 1 || c->n_walls < 0) return false;
  if (c->p > (1 << 16) || c->eta > (1 << 12) || c->n_walls > 4096) return false;
  return true;
}

Layout layout_for(const plan_config* c) {
  const size_t p = c->p, eta = c->eta, nw = c->n_walls;
  const size_t nt = (p + TILE - 1) / TILE, ntp = nt * (nt + 1) / 2;
  const size_t slots = eta * ntp * TILE * TILE;
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = a256(o + std::max<size_t>(bytes, 1)); return at; };
  L.z0 = take(p * (eta + 1) * 8);
  L.z1 = take(p * (eta + 1) * 8);
  L.start = take(p * 8);
  L.goal = take(p * 8);
  L.radius = take(p * 4);
  L.cost = take(p * eta * 4);
  L.walls = take(nw * 16);
  L.tiles = take(ntp * 8);
  L.ulo = take(slots * 16);
  L.uhi = take(slots * 16);
  L.xlo = take(slots * 16);
  L.xhi = take(slots * 16);
  L.bits = take(eta * ntp * TILE * 4);
  L.ukin = take(eta * p * 16);
  L.xkin = take(eta * p * 16);
  L.uwall = take(nw * eta * p * 16);
  L.xwall = take(nw * eta * p * 16);
  L.wbits = take(nw * eta * nt * 4);
  L.work = take(slots * 4);
  L.wcount = take(2 * 4);
  L.accx = take(p * (eta + 1) * 8);
  L.accy = take(p * (eta + 1) * 8);
  L.accc = take(p * (eta + 1) * 4);
  L.fix = take(2 * 4);
  L.res = take(4 * 4);
  L.status = take(4);
  L.count = take(16);
  L.total = o;
  return L;
}

bool finite_all(const float* a, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(a[k])) return false;
  return true;
}

double seg_point_dist(double px, double py, double ax, double ay, double bx, double by) {
  double dx = bx - ax, dy = by - ay, dd = dx * dx + dy * dy;
  double t = dd > 0 ? ((px - ax) * dx + (py - ay) * dy) / dd : 0.0;
  t = std::min(1.0, std::max(0.0, t));
  double cx = ax + t * dx - px, cy = ay + t * dy - py;
  return std::sqrt(cx * cx + cy * cy);
}

// Host-side input check: fixed configurations must be feasible (two disks
// closer than r_i + r_j, or a disk closer than r_i to a wall, make the
// fixed-end minimizers infeasible).  Pairs are found with a uniform grid of
// cell size max(r_i + r_j), so the check is linear in p.
plan_status check_endpoints(int p, const float* start, const float* goal, const float* radius,
                            int nw, const float* walls) {
  float rmax = 0.f;
  for (int i = 0; i < p; ++i) rmax = std::max(rmax, radius[i]);
  const double cell = std::max(2.0 * rmax, 1e-6);
  for (int which = 0; which < 2; ++which) {
    const float* X = which ? goal : start;
    double x0 = X[0], y0 = X[1], x1 = X[0], y1 = X[1];
    for (int i = 1; i < p; ++i) {
      x0 = std::min(x0, (double)X[2 * i]); x1 = std::max(x1, (double)X[2 * i]);
      y0 = std::min(y0, (double)X[2 * i + 1]); y1 = std::max(y1, (double)X[2 * i + 1]);
    }
    // cells at least `cell` wide, so overlapping disks sit in neighbouring cells
    const long nx = std::max<long>(1, std::min<long>(4096, (long)((x1 - x0) / cell)));
    const long ny = std::max<long>(1, std::min<long>(4096, (long)((y1 - y0) / cell)));
    const double sx = (x1 - x0) / nx + 1e-300, sy = (y1 - y0) / ny + 1e-300;
    std::vector<int> head(nx * ny, -1), next(p, -1);
    std::vector<long> cx(p), cy(p);
    for (int i = 0; i < p; ++i) {
      cx[i] = std::min(nx - 1, (long)((X[2 * i] - x0) / sx));
      cy[i] = std::min(ny - 1, (long)((X[2 * i + 1] - y0) / sy));
      const long c = cy[i] * nx + cx[i];
      next[i] = head[c];
      head[c] = i;
    }
    for (int i = 0; i < p; ++i) {
      for (long dy = -1; dy <= 1; ++dy) {
        for (long dx = -1; dx <= 1; ++dx) {
          const long gx = cx[i] + dx, gy = cy[i] + dy;
          if (gx < 0 || gy < 0 || gx >= nx || gy >= ny) continue;
          for (int j = head[gy * nx + gx]; j >= 0; j = next[j]) {
            if (j <= i) continue;
            const double ddx = (double)X[2 * j] - X[2 * i], ddy = (double)X[2 * j + 1] - X[2 * i + 1];
            const double R = (double)radius[i] + radius[j];
            if (ddx * ddx + ddy * ddy < R * R)
              return fail(PLAN_EINFEASIBLE_INPUT, "%s positions of agents %d and %d overlap",
                          which ? "goal" : "start", std::min(i, j), std::max(i, j));
          }
        }
      }
      for (int w = 0; w < nw; ++w) {
        const float* W = walls + 4 * w;
        if (seg_point_dist(X[2 * i], X[2 * i + 1], W[0], W[1], W[2], W[3]) < radius[i])
          return fail(PLAN_EINFEASIBLE_INPUT, "%s of agent %d is within its radius of wall %d",
                      which ? "goal" : "start", i, w);
      }
    }
  }
  return PLAN_OK;
}

}  // namespace

struct plan_s {
  plan_config cfg;
  int p, eta, nw, nt, ntp;
  size_t slots;
  cudaStream_t stream;
  Layout L;
  char* ws;
  bool own_ws;
  int k;
  int cur;  // which z buffer holds z^k
  int prox_grid = 0;  // CTAs of the minimizer pass (resident CTAs per SM x SMs)
  cudaStream_t side = nullptr;   // second stream for the kinetic and wall factors
  cudaStream_t cap = nullptr;    // private stream for capturing the iteration graphs
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool profiling = false;        // plan_profile: per-kernel event timing
  cudaEvent_t pev[6] = {};
  cudaEvent_t pend = nullptr;
  cudaGraphExec_t gexec[4] = {};  // captured iterations by (k parity, z buffer)
  double ptime[4] = {0, 0, 0, 0};
  int pcount = 0;
  unsigned* h_res;  // pinned host word for residual readback
  std::vector<float> h_radius;
  std::vector<float> h_walls;

  template <class T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }

  float rho_at(int kk) const {
    return (kk < cfg.warm_iters) ? cfg.warm_rho : cfg.rho0;
  }

  Dev dev(int kk) const {
    Dev P{};
    P.p = p; P.eta = eta; P.nw = nw; P.nt = nt; P.ntp = ntp;
    P.rho = rho_at(kk);
    P.alpha = cfg.alpha;
    // keeping u on inactive edges (or standard ADMM, which updates every u)
    // needs every u record, so both imply the dense state
    P.dense = (cfg.flags & (PLAN_DENSE_STATE | PLAN_U_KEEP | PLAN_ADMM)) ? 1 : 0;
    P.admm = (cfg.flags & PLAN_ADMM) ? 1 : 0;
    P.keep = (cfg.flags & PLAN_U_KEEP) ? 1 : 0;
    float2* z0 = at<float2>(L.z0);
    float2* z1 = at<float2>(L.z1);
    P.z = cur ? z1 : z0;
    P.z_next = cur ? z0 : z1;
    P.radius = at<float>(L.radius);
    P.cost = at<float>(L.cost);
    P.walls = at<float4>(L.walls);
    P.tiles = at<int2>(L.tiles);
    P.ulo = at<float4>(L.ulo); P.uhi = at<float4>(L.uhi);
    P.xlo = at<float4>(L.xlo); P.xhi = at<float4>(L.xhi);
    P.bits = at<uint32_t>(L.bits);
    P.ukin = at<float4>(L.ukin); P.xkin = at<float4>(L.xkin);
    P.uwall = at<float4>(L.uwall); P.xwall = at<float4>(L.xwall);
    P.wbits = at<uint32_t>(L.wbits);
    P.work = at<uint32_t>(L.work);
    P.work_count = at<unsigned>(L.wcount) + (kk & 1);
    P.work_count_next = at<unsigned>(L.wcount) + ((kk + 1) & 1);
    P.accx = at<unsigned long long>(L.accx);
    P.accy = at<unsigned long long>(L.accy);
    P.accc = at<unsigned>(L.accc);
    P.fix = at<float>(L.fix);
    unsigned* res = at<unsigned>(L.res);
    P.res_cur = res + (kk & 1);
    P.res_prev = kk > 0 ? res + ((kk - 1) & 1) : nullptr;
    P.status = at<unsigned>(L.status);
    return P;
  }
};

namespace {

cudaError_t clear_sums(plan_t h) {
  const size_t nodes = (size_t)h->p * (h->eta + 1);
  cudaError_t e = cudaMemsetAsync(h->at<void>(h->L.accx), 0, nodes * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->at<void>(h->L.accy), 0, nodes * 8, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->at<void>(h->L.accc), 0, nodes * 4, h->stream);
  return e;
}

plan_status ensure_prox_grid(plan_t h) {
  if (h->prox_grid == 0) {
    int dev = 0, sms = 0, nb = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, prox_kernel, 256, 0));
    h->prox_grid = std::max(1, sms * std::max(nb, 1));
  }
  return PLAN_OK;
}

// Enqueue the kernels of iteration h->k (no state change on the host).
plan_status enqueue_iteration(plan_t h, cudaStream_t ms) {
  Dev P = h->dev(h->k);
  const unsigned grid = (unsigned)((size_t)h->eta * h->ntp);
  const int seg_threads = 32 * std::min(1 + h->nw, WARPS);
  const bool prof = h->profiling && h->side;
  if (h->side) {
    // kinetic and wall factors run beside the collision passes
    CK(cudaEventRecord(h->ev_fork, ms));
    CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    if (prof) CK(cudaEventRecord(h->pev[4], h->side));
    segment_kernel<<<h->eta * h->nt, seg_threads, 0, h->side>>>(P);
    if (prof) CK(cudaEventRecord(h->pev[5], h->side));
    CK(cudaEventRecord(h->ev_join, h->side));
  } else {
    segment_kernel<<<h->eta * h->nt, seg_threads, 0, ms>>>(P);
  }
  if (prof) CK(cudaEventRecord(h->pev[0], ms));
  if (P.dense) test_kernel<true><<<grid, 32 * TEST_WARPS, 0, ms>>>(P);
  else test_kernel<false><<<grid, 32 * TEST_WARPS, 0, ms>>>(P);
  if (prof) CK(cudaEventRecord(h->pev[1], ms));
  prox_kernel<<<h->prox_grid, 256, 0, ms>>>(P);
  if (prof) CK(cudaEventRecord(h->pev[2], ms));
  if (h->side) CK(cudaStreamWaitEvent(ms, h->ev_join, 0));
  if (prof) CK(cudaEventRecord(h->pev[3], ms));
  // the consensus kernel also clears the next iteration's worklist counter, so
  // it runs even when there is no free break-point (eta = 1)
  const int nfree = (h->eta - 1) * h->p;
  consensus_kernel<<<std::max(1, (nfree + 63) / 64), 64, 0, ms>>>(P);
  if (prof) {
    CK(cudaEventRecord(h->pend, ms));
    CK(cudaEventSynchronize(h->pend));
    float t[4];
    CK(cudaEventElapsedTime(&t[0], h->pev[0], h->pev[1]));
    CK(cudaEventElapsedTime(&t[1], h->pev[1], h->pev[2]));
    CK(cudaEventElapsedTime(&t[2], h->pev[4], h->pev[5]));
    CK(cudaEventElapsedTime(&t[3], h->pev[3], h->pend));
    for (int q = 0; q < 4; ++q) h->ptime[q] += t[q];
    h->pcount += 1;
  }
  CK(cudaGetLastError());
  return PLAN_OK;
}

// One iteration: replay a captured CUDA graph of the four kernels when one
// fits (past the rho warm-up, not profiling), else launch them directly.
plan_status run_iteration(plan_t h) {
  plan_status st = ensure_prox_grid(h);
  if (st != PLAN_OK) return st;
  const bool graphable = h->cap && h->side && !h->profiling && h->k >= std::max(1, h->cfg.warm_iters);
  if (graphable) {
    const int key = ((h->k & 1) << 1) | h->cur;
    if (!h->gexec[key]) {
      cudaGraph_t g = nullptr;
      // captured on a private stream: the legacy default stream cannot be
      // captured, and the graph does not depend on the stream it came from
      CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
      plan_status cst = enqueue_iteration(h, h->cap);
      cudaError_t e = cudaStreamEndCapture(h->cap, &g);
      if (cst != PLAN_OK) { if (g) cudaGraphDestroy(g); return cst; }
      if (e != cudaSuccess) return fail(PLAN_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&h->gexec[key], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(PLAN_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    CK(cudaGraphLaunch(h->gexec[key], h->stream));
  } else {
    st = enqueue_iteration(h, h->stream);
    if (st != PLAN_OK) return st;
  }
  if (h->eta > 1) h->cur ^= 1;
  h->k += 1;
  return PLAN_OK;
}

// Residual of the last completed iteration (k - 1): its consensus part was
// written by consensus_kernel, the primal part comes from residual_kernel.
plan_status read_residual(plan_t h, float* out) {
  if (h->k == 0) { *out = INFINITY; return PLAN_OK; }
  Dev P = h->dev(h->k);
  residual_kernel<<<h->eta > 0 ? 304 : 1, 256, 0, h->stream>>>(P);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->h_res, P.res_prev, 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  uint32_t bitsv = *h->h_res;
  float v;
  std::memcpy(&v, &bitsv, 4);
  *out = v;
  return PLAN_OK;
}

plan_status upload_inputs(plan_t h, const float* start, const float* goal, const float* radius,
                          const float* cost_w, const float* walls) {
  const plan_config& c = h->cfg;
  const size_t p = c.p, eta = c.eta;
  std::vector<float> cost(p * eta);
  const double norm = (c.flags & PLAN_COST_UNNORM) ? 1.0 : 1.0 / ((double)p * eta);
  for (size_t i = 0; i < p; ++i)
    for (size_t s = 0; s < eta; ++s) {
      double C = (c.flags & PLAN_COST_PER_SEGMENT) ? cost_w[i * eta + s] : cost_w[i];
      cost[i * eta + s] = (float)(C * norm);
    }
  std::vector<int2> tiles;
  for (int I = 0; I < h->nt; ++I)
    for (int J = I; J < h->nt; ++J) tiles.push_back(make_int2(I, J));
  CK(cudaMemcpyAsync(h->at<void>(h->L.start), start, p * 8, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.goal), goal, p * 8, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.radius), radius, p * 4, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.cost), cost.data(), p * eta * 4, cudaMemcpyHostToDevice, h->stream));
  if (h->nw)
    CK(cudaMemcpyAsync(h->at<void>(h->L.walls), walls, (size_t)h->nw * 16, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.tiles), tiles.data(), tiles.size() * 8, cudaMemcpyHostToDevice, h->stream));
  // the staging vectors die at return: wait for the copies
  CK(cudaStreamSynchronize(h->stream));
  return PLAN_OK;
}

}  // namespace

extern "C" {

const char* plan_last_error(void) { return g_err.c_str(); }

plan_status plan_workspace_size(const plan_config* cfg, size_t* bytes) {
  if (!cfg || !bytes) return fail(PLAN_EINVAL, "null argument");
  if (!sizes_ok(cfg)) return fail(PLAN_EINVAL, "p, eta or n_walls out of range");
  *bytes = layout_for(cfg).total;
  return PLAN_OK;
}

plan_status plan_reset(plan_t h) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  h->k = 0;
  h->cur = 0;
  Dev P = h->dev(0);
  const size_t zbytes = (size_t)h->p * (h->eta + 1) * 8;
  (void)zbytes;
  CK(cudaMemsetAsync(h->at<void>(h->L.bits), 0, (size_t)h->eta * h->ntp * TILE * 4, h->stream));
  if (h->nw) CK(cudaMemsetAsync(h->at<void>(h->L.wbits), 0, (size_t)h->nw * h->eta * h->nt * 4, h->stream));
  if (h->cfg.flags & (PLAN_DENSE_STATE | PLAN_U_KEEP | PLAN_ADMM)) {
    CK(cudaMemsetAsync(h->at<void>(h->L.ulo), 0, h->slots * 16, h->stream));
    CK(cudaMemsetAsync(h->at<void>(h->L.uhi), 0, h->slots * 16, h->stream));
    if (h->nw) CK(cudaMemsetAsync(h->at<void>(h->L.uwall), 0, (size_t)h->nw * h->eta * h->p * 16, h->stream));
  }
  CK(cudaMemsetAsync(h->at<void>(h->L.res), 0, 16, h->stream));
  CK(cudaMemsetAsync(h->at<void>(h->L.wcount), 0, 8, h->stream));
  CK(clear_sums(h));
  CK(cudaMemsetAsync(h->at<void>(h->L.status), 0, 4, h->stream));
  fix_kernel<<<1, 256, 0, h->stream>>>(P, h->at<float2>(h->L.start), h->at<float2>(h->L.goal));
  const int n = std::max(h->p * (h->eta + 1), h->eta * h->p);
  reset_kernel<<<(n + 255) / 256, 256, 0, h->stream>>>(P, h->at<float2>(h->L.z0), h->at<float2>(h->L.z1),
                                                      h->at<float2>(h->L.start), h->at<float2>(h->L.goal));
  CK(cudaGetLastError());
  return PLAN_OK;
}

plan_status plan_create(const plan_config* cfg, const float* start, const float* goal,
                        const float* radius, const float* cost_w, const float* walls,
                        void* workspace, size_t workspace_bytes, void* cuda_stream, plan_t* out) {
  if (!cfg || !start || !goal || !radius || !cost_w || !out) return fail(PLAN_EINVAL, "null argument");
  *out = nullptr;
  if (!sizes_ok(cfg)) return fail(PLAN_EINVAL, "p, eta or n_walls out of range");
  if (cfg->n_walls > 0 && !walls) return fail(PLAN_EINVAL, "walls is NULL but n_walls > 0");
  if (!(cfg->rho0 > 0.f) || !std::isfinite(cfg->rho0)) return fail(PLAN_EINVAL, "rho0 must be positive");
  if (!(cfg->alpha > 0.f) || !std::isfinite(cfg->alpha)) return fail(PLAN_EINVAL, "alpha must be positive");
  if (cfg->warm_iters < 0 || (cfg->warm_iters > 0 && !(cfg->warm_rho > 0.f)))
    return fail(PLAN_EINVAL, "warm_rho must be positive when warm_iters > 0");
  if (cfg->max_iter < 0) return fail(PLAN_EINVAL, "max_iter must be >= 0");
  const unsigned known = PLAN_U_KEEP | PLAN_COST_UNNORM | PLAN_COST_PER_SEGMENT |
                         PLAN_DENSE_STATE | PLAN_ADMM;
  if (cfg->flags & ~known) return fail(PLAN_EINVAL, "unknown flag bits 0x%x", cfg->flags & ~known);
  const size_t p = cfg->p, eta = cfg->eta;
  const size_t ncost = (cfg->flags & PLAN_COST_PER_SEGMENT) ? p * eta : p;
  if (!finite_all(start, 2 * p) || !finite_all(goal, 2 * p) || !finite_all(radius, p) ||
      !finite_all(cost_w, ncost) || (cfg->n_walls && !finite_all(walls, 4 * (size_t)cfg->n_walls)))
    return fail(PLAN_EINVAL, "non-finite input");
  for (size_t i = 0; i < p; ++i)
    if (!(radius[i] > 0.f)) return fail(PLAN_EINVAL, "radius[%zu] must be positive", i);
  for (size_t i = 0; i < ncost; ++i)
    if (cost_w[i] < 0.f) return fail(PLAN_EINVAL, "cost_w[%zu] must be >= 0", i);
  plan_status st = check_endpoints(cfg->p, start, goal, radius, cfg->n_walls, walls);
  if (st != PLAN_OK) return st;

  Layout L = layout_for(cfg);
  plan_s* h = new plan_s();
  h->cfg = *cfg;
  if (h->cfg.check_every < 1) h->cfg.check_every = 1;
  h->p = cfg->p; h->eta = cfg->eta; h->nw = cfg->n_walls;
  h->nt = (h->p + TILE - 1) / TILE;
  h->ntp = h->nt * (h->nt + 1) / 2;
  h->slots = (size_t)h->eta * h->ntp * TILE * TILE;
  h->stream = (cudaStream_t)cuda_stream;
  h->L = L;
  h->h_radius.assign(radius, radius + p);
  if (h->nw) h->h_walls.assign(walls, walls + 4 * (size_t)h->nw);
  if (workspace) {
    if (workspace_bytes < L.total) {
      delete h;
      return fail(PLAN_ENOMEM, "workspace of %zu bytes, %zu needed", workspace_bytes, L.total);
    }
    if (reinterpret_cast<uintptr_t>(workspace) & 255) {
      delete h;
      return fail(PLAN_EINVAL, "workspace must be 256-byte aligned");
    }
    h->ws = static_cast<char*>(workspace);
    h->own_ws = false;
  } else {
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, L.total);
    if (e != cudaSuccess) {
      delete h;
      return fail(PLAN_ENOMEM, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
    }
    h->ws = static_cast<char*>(mem);
    h->own_ws = true;
  }
  cudaError_t e = cudaMallocHost(&h->h_res, 16);
  if (e != cudaSuccess) {
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return fail(PLAN_ENOMEM, "cudaMallocHost failed: %s", cudaGetErrorString(e));
  }
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    plan_destroy(h);
    return fail(PLAN_ECUDA, "stream or event creation failed");
  }
  st = upload_inputs(h, start, goal, radius, cost_w, walls);
  if (st == PLAN_OK) st = plan_reset(h);
  if (st != PLAN_OK) {
    plan_destroy(h);
    return st;
  }
  *out = h;
  return PLAN_OK;
}

void plan_destroy(plan_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  if (h->h_res) cudaFreeHost(h->h_res);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (int q = 0; q < 6; ++q)
    if (h->pev[q]) cudaEventDestroy(h->pev[q]);
  for (int q = 0; q < 4; ++q)
    if (h->gexec[q]) cudaGraphExecDestroy(h->gexec[q]);
  if (h->pend) cudaEventDestroy(h->pend);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

plan_status plan_set_endpoints(plan_t h, const float* start, const float* goal) {
  if (!h || !start || !goal) return fail(PLAN_EINVAL, "null argument");
  if (!finite_all(start, 2 * (size_t)h->p) || !finite_all(goal, 2 * (size_t)h->p))
    return fail(PLAN_EINVAL, "non-finite input");
  plan_status st = check_endpoints(h->p, start, goal, h->h_radius.data(), h->nw, h->h_walls.data());
  if (st != PLAN_OK) return st;
  CK(cudaMemcpyAsync(h->at<void>(h->L.start), start, (size_t)h->p * 8, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.goal), goal, (size_t)h->p * 8, cudaMemcpyHostToDevice, h->stream));
  endpoints_kernel<<<(h->p + 255) / 256, 256, 0, h->stream>>>(
      h->p, h->eta, h->at<float2>(h->L.z0), h->at<float2>(h->L.z1), h->at<float2>(h->L.start),
      h->at<float2>(h->L.goal));
  fix_kernel<<<1, 256, 0, h->stream>>>(h->dev(h->k), h->at<float2>(h->L.start), h->at<float2>(h->L.goal));
  CK(cudaGetLastError());
  // the caller's host buffers may be reused once this returns
  CK(cudaStreamSynchronize(h->stream));
  return PLAN_OK;
}

plan_status plan_iterate(plan_t h, int k_iters, float* max_residual) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  if (k_iters < 0) return fail(PLAN_EINVAL, "k_iters must be >= 0");
  for (int it = 0; it < k_iters; ++it) {
    plan_status st = run_iteration(h);
    if (st != PLAN_OK) return st;
  }
  if (max_residual) return read_residual(h, max_residual);
  return PLAN_OK;
}

plan_status plan_solve(plan_t h, int* iters_done, float* max_residual) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  float res = INFINITY;
  plan_status st = PLAN_OK;
  while (h->k < h->cfg.max_iter) {
    int n = std::min(h->cfg.check_every, h->cfg.max_iter - h->k);
    st = plan_iterate(h, n, &res);
    if (st != PLAN_OK) break;
    if (!(res == res)) { st = fail(PLAN_ENUMERIC, "non-finite residual at iteration %d", h->k); break; }
    if (res < h->cfg.tol) break;
  }
  if (st == PLAN_OK && !(res < h->cfg.tol))
    st = fail(PLAN_ENOTCONV, "residual %g after %d iterations", (double)res, h->k);
  if (iters_done) *iters_done = h->k;
  if (max_residual) *max_residual = res;
  return st;
}

plan_status plan_get_trajectory(plan_t h, float* z, int on_device) {
  if (!h || !z) return fail(PLAN_EINVAL, "null argument");
  const size_t bytes = (size_t)h->p * (h->eta + 1) * 8;
  const void* src = h->cur ? h->at<void>(h->L.z1) : h->at<void>(h->L.z0);
  CK(cudaMemcpyAsync(z, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  if (!on_device) CK(cudaStreamSynchronize(h->stream));
  return PLAN_OK;
}

plan_status plan_export_state(plan_t h, float* z, float* u_coll, float* u_kin, float* u_wall,
                              uint8_t* act_coll, uint8_t* act_wall, int* k) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  Dev P = h->dev(h->k);
  if (z) {
    plan_status st = plan_get_trajectory(h, z, 1);
    if (st != PLAN_OK) return st;
  }
  if (u_coll || act_coll) {
    const size_t n = h->slots;
    export_coll_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(P, u_coll, act_coll);
  }
  const int nseg = std::max(h->eta * h->p, h->nw * h->eta * h->p);
  if (u_kin || u_wall || act_wall)
    export_seg_kernel<<<(nseg + 255) / 256, 256, 0, h->stream>>>(P, u_kin, u_wall, act_wall);
  CK(cudaGetLastError());
  if (k) *k = h->k;
  return PLAN_OK;
}

plan_status plan_import_state(plan_t h, const float* z, const float* u_coll, const float* u_kin,
                              const float* u_wall, int k) {
  if (!h || !z || !u_kin || (h->p > 1 && !u_coll) || (h->nw && !u_wall))
    return fail(PLAN_EINVAL, "null argument");
  if (k < 0) return fail(PLAN_EINVAL, "k must be >= 0");
  const size_t zbytes = (size_t)h->p * (h->eta + 1) * 8;
  CK(cudaMemcpyAsync(h->at<void>(h->L.z0), z, zbytes, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.z1), z, zbytes, cudaMemcpyDeviceToDevice, h->stream));
  h->cur = 0;
  h->k = k;
  Dev P = h->dev(k);
  if (h->p > 1) import_coll_kernel<<<(unsigned)((h->slots + 255) / 256), 256, 0, h->stream>>>(P, u_coll);
  const int nseg = std::max(h->eta * h->p, h->nw * h->eta * h->p);
  import_seg_kernel<<<(nseg + 255) / 256, 256, 0, h->stream>>>(P, u_kin, u_wall);
  if (h->nw) {
    const int words = h->nw * h->eta * h->nt;
    import_wbits_kernel<<<(words * 32 + 255) / 256, 256, 0, h->stream>>>(P);
  }
  CK(cudaMemsetAsync(h->at<void>(h->L.res), 0, 16, h->stream));
  CK(cudaMemsetAsync(h->at<void>(h->L.wcount), 0, 8, h->stream));
  CK(clear_sums(h));
  CK(cudaMemsetAsync(h->at<void>(h->L.status), 0, 4, h->stream));
  fix_kernel<<<1, 256, 0, h->stream>>>(P, h->at<float2>(h->L.start), h->at<float2>(h->L.goal));
  CK(cudaGetLastError());
  return PLAN_OK;
}

plan_status plan_get_info(plan_t h, plan_info* info) {
  if (!h || !info) return fail(PLAN_EINVAL, "null argument");
  const long long p = h->p, eta = h->eta;
  info->n_coll = eta * p * (p - 1) / 2;
  info->n_kin = eta * p;
  info->n_wall = (long long)h->nw * eta * p;
  info->n_pos = 2 * p;
  info->k = h->k;
  info->tile = TILE;
  info->workspace_bytes = h->L.total;
  unsigned long long* cnt = h->at<unsigned long long>(h->L.count);
  CK(cudaMemsetAsync(cnt, 0, 16, h->stream));
  count_kernel<<<256, 256, 0, h->stream>>>(h->at<uint32_t>(h->L.bits), (size_t)h->eta * h->ntp * TILE, cnt);
  if (h->nw) count_kernel<<<64, 256, 0, h->stream>>>(h->at<uint32_t>(h->L.wbits), (size_t)h->nw * h->eta * h->nt, cnt + 1);
  CK(cudaGetLastError());
  unsigned long long hc[2] = {0, 0};
  CK(cudaMemcpyAsync(hc, cnt, 16, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  info->active_coll = (long long)hc[0];
  info->active_wall = (long long)hc[1];
  return PLAN_OK;
}

plan_status plan_profile(plan_t h, int enable, float* ms, int* iterations) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  if (!h->side) return fail(PLAN_EINVAL, "this plan has no second stream to time");
  if (enable) {
    for (int q = 0; q < 6; ++q)
      if (!h->pev[q]) CK(cudaEventCreate(&h->pev[q]));
    if (!h->pend) CK(cudaEventCreate(&h->pend));
    for (int q = 0; q < 4; ++q) h->ptime[q] = 0.0;
    h->pcount = 0;
    h->profiling = true;
    return PLAN_OK;
  }
  h->profiling = false;
  for (int q = 0; q < 4; ++q)
    if (ms) ms[q] = h->pcount ? (float)(h->ptime[q] / h->pcount) : 0.f;
  if (iterations) *iterations = h->pcount;
  return PLAN_OK;
}

plan_status plan_backward(plan_t h, int K, const float* dL_dz, float* d_start, float* d_goal,
                          float* d_radius, float* d_cost_w) {
  (void)h; (void)K; (void)dL_dz; (void)d_start; (void)d_goal; (void)d_radius; (void)d_cost_w;
  return fail(PLAN_EUNSUPPORTED, "plan_backward is not built yet");
}


// ---------------------------------------------------------------------------
// plan_iterate_static: one iteration with every temporary in a static array
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

// Temporaries of plan_iterate_static, laid out like a plan_create workspace.
// Host code must not use this name as an address: it is looked up per device
// with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[PLAN_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Kinetic coefficients c_{i,s} and the tile-pair table, computed on the
// device from the caller's device arrays (same arithmetic as upload_inputs).
__global__ void static_prep_kernel(int p, int eta, int nt, int ntp, unsigned flags,
                                   const float* cost_w, float* cost, int2* tiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < p * eta) {
    const int i = t / eta, s = t - i * eta;
    const double norm = (flags & PLAN_COST_UNNORM) ? 1.0 : 1.0 / ((double)p * eta);
    const double C = (flags & PLAN_COST_PER_SEGMENT) ? cost_w[(size_t)i * eta + s] : cost_w[i];
    cost[t] = (float)(C * norm);
  }
  if (t < ntp) {
    int I = 0, off = 0;
    while (off + (nt - I) <= t) { off += nt - I; ++I; }
    tiles[t] = make_int2(I, I + (t - off));
  }
}

plan_status static_scratch_for_current_device(void** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PLAN_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    CK(cudaGetSymbolAddress(&ptr, g_static_scratch));
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return PLAN_OK;
}

}  // namespace

extern "C" {

plan_status plan_iterate_static(const plan_config* cfg, const float* start, const float* goal,
                                const float* radius, const float* cost_w, const float* walls,
                                const float* z_in, const float* u_coll_in, const float* u_kin_in,
                                const float* u_wall_in, float* z_out, float* u_coll_out,
                                float* u_kin_out, float* u_wall_out, uint8_t* act_coll_out,
                                uint8_t* act_wall_out, int k, void* cuda_stream) {
  if (!cfg || !start || !goal || !radius || !cost_w || !z_in || !u_kin_in || !z_out || !u_kin_out)
    return fail(PLAN_EINVAL, "null argument");
  if (!sizes_ok(cfg)) return fail(PLAN_EINVAL, "p, eta or n_walls out of range");
  if (cfg->p > 1 && (!u_coll_in || !u_coll_out)) return fail(PLAN_EINVAL, "null u_coll");
  if (cfg->n_walls > 0 && (!walls || !u_wall_in || !u_wall_out)) return fail(PLAN_EINVAL, "null wall array");
  if (!(cfg->rho0 > 0.f) || !(cfg->alpha > 0.f)) return fail(PLAN_EINVAL, "rho0 and alpha must be positive");
  if (k < 0) return fail(PLAN_EINVAL, "k must be >= 0");
  const unsigned known = PLAN_U_KEEP | PLAN_COST_UNNORM | PLAN_COST_PER_SEGMENT |
                         PLAN_DENSE_STATE | PLAN_ADMM;
  if (cfg->flags & ~known) return fail(PLAN_EINVAL, "unknown flag bits 0x%x", cfg->flags & ~known);
  const Layout L = layout_for(cfg);
  if (L.total > PLAN_STATIC_SCRATCH_BYTES)
    return fail(PLAN_ENOMEM, "problem needs %zu bytes of scratch; the static array holds %u "
                "(p = %d, eta = %d, n_walls = %d)", L.total, PLAN_STATIC_SCRATCH_BYTES, cfg->p,
                cfg->eta, cfg->n_walls);
  void* scratch = nullptr;
  plan_status st = static_scratch_for_current_device(&scratch);
  if (st != PLAN_OK) return st;

  plan_s h;  // a plan over the static array; nothing here allocates
  h.cfg = *cfg;
  h.p = cfg->p; h.eta = cfg->eta; h.nw = cfg->n_walls;
  h.nt = (h.p + TILE - 1) / TILE;
  h.ntp = h.nt * (h.nt + 1) / 2;
  h.slots = (size_t)h.eta * h.ntp * TILE * TILE;
  h.stream = (cudaStream_t)cuda_stream;
  h.L = L;
  h.ws = static_cast<char*>(scratch);
  h.own_ws = false;
  h.h_res = nullptr;
  h.k = 0;
  h.cur = 0;

  const size_t p = h.p;
  CK(cudaMemcpyAsync(h.at<void>(L.start), start, p * 8, cudaMemcpyDeviceToDevice, h.stream));
  CK(cudaMemcpyAsync(h.at<void>(L.goal), goal, p * 8, cudaMemcpyDeviceToDevice, h.stream));
  CK(cudaMemcpyAsync(h.at<void>(L.radius), radius, p * 4, cudaMemcpyDeviceToDevice, h.stream));
  if (h.nw)
    CK(cudaMemcpyAsync(h.at<void>(L.walls), walls, (size_t)h.nw * 16, cudaMemcpyDeviceToDevice, h.stream));
  // the scratch keeps the previous call's contents: clear what must start at zero
  CK(cudaMemsetAsync(h.at<void>(L.status), 0, 4, h.stream));
  if (h.cfg.flags & (PLAN_DENSE_STATE | PLAN_U_KEEP | PLAN_ADMM)) {
    CK(cudaMemsetAsync(h.at<void>(L.ulo), 0, h.slots * 16, h.stream));
    CK(cudaMemsetAsync(h.at<void>(L.uhi), 0, h.slots * 16, h.stream));
  }
  const int nprep = std::max(h.p * h.eta, h.ntp);
  static_prep_kernel<<<(nprep + 255) / 256, 256, 0, h.stream>>>(
      h.p, h.eta, h.nt, h.ntp, h.cfg.flags, cost_w, h.at<float>(L.cost), h.at<int2>(L.tiles));
  CK(cudaGetLastError());
  st = plan_import_state(&h, z_in, u_coll_in, u_kin_in, u_wall_in, k);
  if (st == PLAN_OK) st = run_iteration(&h);
  if (st == PLAN_OK)
    st = plan_export_state(&h, z_out, h.p > 1 ? u_coll_out : nullptr, u_kin_out,
                           h.nw ? u_wall_out : nullptr, h.p > 1 ? act_coll_out : nullptr,
                           h.nw ? act_wall_out : nullptr, nullptr);
  return st;
}

}  // extern "C"

// twa_backward.cuh -- the adjoint of one TWA iteration (Appendix B steps
// 1-7) with its branch choices frozen: which collision factors were active
// and which candidate direction each minimizer took.
//
// Forward iteration k (every weight rho0; u = 0 on edges that were not
// active and at fixed nodes):
//   n_e = z^k_node(e) - u^k_e;  x = g(n) per factor
//   z^{k+1}_v = (1 / c_v) sum over the c_v active edges e at v of (x_e + u^k_e)
//   u^{k+1}_e = u^k_e + alpha (x_e - z^{k+1}_v) on active edges at free nodes.
// Given zbar = dL/dz^{k+1} and ubar = dL/du^{k+1}, the adjoint step is
//   zhat_v = zbar_v - alpha sum_e ubar_e,   mbar_v = zhat_v / c_v   (pass 1, 2)
//   xbar_e = mbar_v + alpha ubar_e,          nbar = (dg/dn)^T xbar   (pass 3)
//   dL/dz^k_v = sum_e nbar_e,   dL/du^k_e = ubar_e + mbar_v - nbar_e.
// At fixed nodes z is the start or goal, x is unused and u stays 0.  A
// collision edge's u^{k+1} matters only if the factor is active in both k and
// k+1 (else it is reset or unused), so its adjoint is kept with the iteration
// that wrote it (stamp) and read as 0 unless the stamp is k + 1.  Wall and
// velocity-limit factors are gated the same way and carried alike.
//
// Sums into nodes use FP64 atomics (order-dependent in the last bits only).
#pragma once
#include "twa_adjoint.cuh"
#include "twa_iter.cuh"

namespace {

struct AdjDev {
  int p, eta, ntp, k;
  float rho, alpha;
  const int2* tiles;
  const float* radius;
  const float* cost;        // [p][eta] c_{i,s}
  int nw, nv;               // wall kinds, then velocity-limit kinds (gated segment factors)
  int vo;                   // local planner epoch: no kinetic factor on segment 0
  unsigned vmin_mask;       // velocity kind v is a minimum
  const float4* walls;      // [nw]
  const float* vlim;        // [nv][p][eta]
  // the tape of iteration k
  const float2* z;          // z^k, [p][eta+1]
  const float4* ukin;       // u^k of the kinetic edges, [eta][p]
  const uint32_t* fid;      // collision slots active in iteration k
  const float4* ucl;        // their u^k at the lower break-point: (u_i, u_j)
  const float4* uch;        // ... at the upper break-point
  const unsigned* count;    // how many
  const uint32_t* sidx;     // gated segment factors active in iteration k: (g eta + s) p + i
  const float4* su;         // their u^k (lower, upper)
  const unsigned* scount;   // how many
  // adjoint state
  float4* ubk;              // kinetic u adjoints, [eta][p]: of u^{k+1} in, u^k out
  float4* ubl;              // collision u adjoints by slot (lower, upper)
  float4* ubh;
  int* stamp;               // the iteration whose u adjoint a slot holds
  float4* ubs;              // gated segment factor u adjoints, [(nw + nv) eta p]
  int* sstamp;              // ... and the iteration that wrote them
  const double2* zb_in;     // dL/dz^{k+1}
  double2* zb_out;          // dL/dz^k, accumulated
  double2* S;               // alpha * sum of u adjoints per node
  unsigned* cnt;            // active edges per node
  float2* mbar;             // per node
  double2* g_start;         // [p]
  double2* g_goal;          // [p]
  double* g_r;              // [p]
  double* g_c;              // [p][eta], adjoint of c_{i,s}
};

__device__ __forceinline__ void atomic_add2(double2* a, float2 v) {
  atomicAdd(&a->x, (double)v.x);
  atomicAdd(&a->y, (double)v.y);
}

__device__ __forceinline__ void decode_slot(const AdjDev& A, uint32_t f, int& s, int& i, int& j) {
  const uint32_t row = f >> 5, c = f & 31;
  const uint32_t blk = row >> 5, r = row & 31;
  s = (int)(blk / A.ntp);
  const int2 IJ = A.tiles[blk - (uint32_t)s * A.ntp];
  i = IJ.x * TILE + (int)r;
  j = IJ.y * TILE + (int)c;
}

__device__ __forceinline__ void scatter_edge(const AdjDev& A, int i, int s, float2 ub) {
  const size_t node = (size_t)i * (A.eta + 1) + s;
  atomic_add2(A.S + node, mk(A.alpha * ub.x, A.alpha * ub.y));
  atomicAdd(A.cnt + node, 1u);
}

// Pass 1: alpha * u adjoints and edge counts into the nodes.
__device__ __forceinline__ void bw_scatter_item(const AdjDev& A, unsigned t) {
  const unsigned nkin = (unsigned)(A.eta * A.p);
  const unsigned ncoll = *A.count;
  if (t >= nkin + ncoll) {  // a gated segment factor
    const uint32_t g = A.sidx[t - nkin - ncoll];
    const int i = (int)(g % A.p), s = (int)((g / A.p) % A.eta);
    const float4 ub = (A.sstamp[g] == A.k + 1) ? A.ubs[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (s > 0) scatter_edge(A, i, s, lo2(ub));
    if (s + 1 < A.eta) scatter_edge(A, i, s + 1, hi2(ub));
    return;
  }
  if (t < nkin) {
    const int s = (int)(t / A.p), i = (int)(t - (unsigned)s * A.p);
    if (A.vo && s == 0) return;
    const float4 ub = A.ubk[t];
    if (s > 0) scatter_edge(A, i, s, lo2(ub));
    if (s + 1 < A.eta) scatter_edge(A, i, s + 1, hi2(ub));
    return;
  }
  const uint32_t f = A.fid[t - nkin];
  int s, i, j;
  decode_slot(A, f, s, i, j);
  const bool live = A.stamp[f] == A.k + 1;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 bl = live ? A.ubl[f] : zero, bh = live ? A.ubh[f] : zero;
  if (s > 0) { scatter_edge(A, i, s, lo2(bl)); scatter_edge(A, j, s, hi2(bl)); }
  if (s + 1 < A.eta) { scatter_edge(A, i, s + 1, lo2(bh)); scatter_edge(A, j, s + 1, hi2(bh)); }
}

// Pass 2 per node: mbar at free nodes, start / goal gradients at fixed ones;
// clears the sums and the next adjoint of z.
__device__ __forceinline__ void bw_node(const AdjDev& A, int t) {
  const int E1 = A.eta + 1;
  const int i = t / E1, s = t - i * E1;
  const double2 zb = A.zb_in[t];
  if (s == 0) {
    A.g_start[i].x += zb.x; A.g_start[i].y += zb.y;
  } else if (s == A.eta) {
    A.g_goal[i].x += zb.x; A.g_goal[i].y += zb.y;
  } else {
    const unsigned c = A.cnt[t];
    const double2 S = A.S[t];
    const double inv = c ? 1.0 / (double)c : 0.0;
    A.mbar[t] = mk((float)((zb.x - S.x) * inv), (float)((zb.y - S.y) * inv));
  }
  A.S[t] = make_double2(0.0, 0.0);
  A.cnt[t] = 0u;
  A.zb_out[t] = make_double2(0.0, 0.0);
}

// Per edge of pass 3: xbar, and the u adjoint once nbar is known.
__device__ __forceinline__ float2 edge_xbar(const AdjDev& A, bool fixed, int i, int s, float2 ub,
                                           float2& mb) {
  if (fixed) { mb = mk(0.f, 0.f); return mb; }
  mb = A.mbar[(size_t)i * (A.eta + 1) + s];
  return mk(mb.x + A.alpha * ub.x, mb.y + A.alpha * ub.y);
}
__device__ __forceinline__ float2 edge_ubar(bool fixed, float2 ub, float2 mb, float2 nb) {
  return fixed ? mk(0.f, 0.f) : mk(ub.x + mb.x - nb.x, ub.y + mb.y - nb.y);
}

// Pass 3 for a wall or velocity-limit factor (gated like a collision factor).
__device__ __forceinline__ void bw_seg_item(const AdjDev& A, unsigned w) {
  const int E1 = A.eta + 1;
  const uint32_t g = A.sidx[w];
  const int i = (int)(g % A.p), s = (int)((g / A.p) % A.eta);
  const int kind = (int)(g / ((uint32_t)A.p * A.eta));
  const bool pin_lo = (s == 0), pin_hi = (s == A.eta - 1);
  const float4 u = A.su[w];
  const float2 nl = A.z[(size_t)i * E1 + s] - lo2(u), nh = A.z[(size_t)i * E1 + s + 1] - hi2(u);
  const float4 ub = (A.sstamp[g] == A.k + 1) ? A.ubs[g] : make_float4(0.f, 0.f, 0.f, 0.f);
  float2 ml, mh;
  const float2 xl = edge_xbar(A, pin_lo, i, s, lo2(ub), ml);
  const float2 xh = edge_xbar(A, pin_hi, i, s + 1, hi2(ub), mh);
  float2 bl, bh;
  if (kind < A.nw) {
    const float4 W = A.walls[kind];
    float rb;
    wall_vjp(nl, nh, pin_lo, pin_hi, mk(W.x, W.y), mk(W.z, W.w), A.radius[i], A.rho, xl, xh, bl, bh, rb);
    atomicAdd(A.g_r + i, (double)rb);
  } else {
    const int v = kind - A.nw;
    velocity_vjp(nl, nh, pin_lo, pin_hi, A.vlim[((size_t)v * A.p + i) * A.eta + s], xl, xh, bl, bh);
  }
  atomic_add2(A.zb_out + (size_t)i * E1 + s, bl);
  atomic_add2(A.zb_out + (size_t)i * E1 + s + 1, bh);
  A.ubs[g] = pack(edge_ubar(pin_lo, lo2(ub), ml, bl), edge_ubar(pin_hi, hi2(ub), mh, bh));
  A.sstamp[g] = A.k;
}

// Pass 3: the adjoint of one factor's minimizer.
__device__ __forceinline__ void bw_factor_item(const AdjDev& A, unsigned t) {
  const int E1 = A.eta + 1;
  const unsigned nkin = (unsigned)(A.eta * A.p);
  const unsigned ncoll = *A.count;
  if (t >= nkin + ncoll) { bw_seg_item(A, t - nkin - ncoll); return; }
  if (t < nkin) {
    const int s = (int)(t / A.p), i = (int)(t - (unsigned)s * A.p);
    if (A.vo && s == 0) return;
    const bool pin_lo = (s == 0), pin_hi = (s == A.eta - 1);
    const float4 u = A.ukin[t];
    const float2 nl = A.z[(size_t)i * E1 + s] - lo2(u), nh = A.z[(size_t)i * E1 + s + 1] - hi2(u);
    const float4 ub = A.ubk[t];
    float2 ml, mh;
    const float2 xl = edge_xbar(A, pin_lo, i, s, lo2(ub), ml);
    const float2 xh = edge_xbar(A, pin_hi, i, s + 1, hi2(ub), mh);
    float2 bl, bh;
    float cb;
    energy_vjp(nl, nh, A.rho, pin_lo, pin_hi, A.cost[(size_t)i * A.eta + s], xl, xh, bl, bh, cb);
    atomic_add2(A.zb_out + (size_t)i * E1 + s, bl);
    atomic_add2(A.zb_out + (size_t)i * E1 + s + 1, bh);
    A.ubk[t] = pack(edge_ubar(pin_lo, lo2(ub), ml, bl), edge_ubar(pin_hi, hi2(ub), mh, bh));
    A.g_c[(size_t)i * A.eta + s] += (double)cb;
    return;
  }
  const unsigned w = t - nkin;
  const uint32_t f = A.fid[w];
  int s, i, j;
  decode_slot(A, f, s, i, j);
  const bool pin_lo = (s == 0), pin_hi = (s == A.eta - 1);
  const float4 a = A.ucl[w], b = A.uch[w];
  // n exactly as the forward minimizer pass formed it
  const float2 nil = A.z[(size_t)i * E1 + s] - lo2(a), nih = A.z[(size_t)i * E1 + s + 1] - lo2(b);
  const float2 njl = A.z[(size_t)j * E1 + s] - hi2(a), njh = A.z[(size_t)j * E1 + s + 1] - hi2(b);
  const bool live = A.stamp[f] == A.k + 1;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 bl = live ? A.ubl[f] : zero, bh = live ? A.ubh[f] : zero;
  float2 mil, mjl, mih, mjh;
  const float2 xil = edge_xbar(A, pin_lo, i, s, lo2(bl), mil);
  const float2 xjl = edge_xbar(A, pin_lo, j, s, hi2(bl), mjl);
  const float2 xih = edge_xbar(A, pin_hi, i, s + 1, lo2(bh), mih);
  const float2 xjh = edge_xbar(A, pin_hi, j, s + 1, hi2(bh), mjh);
  float2 nbil, nbih, nbjl, nbjh;
  float Rb;
  coll_vjp(nil, nih, njl, njh, pin_lo, pin_hi, A.radius[i] + A.radius[j], A.rho, xil, xih, xjl,
           xjh, nbil, nbih, nbjl, nbjh, Rb);
  atomic_add2(A.zb_out + (size_t)i * E1 + s, nbil);
  atomic_add2(A.zb_out + (size_t)j * E1 + s, nbjl);
  atomic_add2(A.zb_out + (size_t)i * E1 + s + 1, nbih);
  atomic_add2(A.zb_out + (size_t)j * E1 + s + 1, nbjh);
  atomicAdd(A.g_r + i, (double)Rb);
  atomicAdd(A.g_r + j, (double)Rb);
  A.ubl[f] = pack(edge_ubar(pin_lo, lo2(bl), mil, nbil), edge_ubar(pin_lo, hi2(bl), mjl, nbjl));
  A.ubh[f] = pack(edge_ubar(pin_hi, lo2(bh), mih, nbih), edge_ubar(pin_hi, hi2(bh), mjh, nbjh));
  A.stamp[f] = A.k;
}

}  // namespace

// plan.cu -- GB300 (sm_103a) C ABI of the three-weight ADMM trajectory
// planner (Bento, Derbinsky, Alonso-Mora, Yedidia, NIPS 2013): workspace
// layout, input checks, state reset / import / export, the residual, and the
// per-iteration launch sequence.  The iteration's per-block work lives in
// twa_iter.cuh; one iteration is three kernels on one stream:
//
//   test_kernel      every collision factor: deferred u step, n = z - u,
//                    collision test, activity bits, worklist of active pairs;
//                    in the same launch, the kinetic factors and the wall
//                    tests (worklist of active walls)
//   prox_kernel      the minimizer of every active wall and pair, adding
//                    m = x + u into exact fixed-point consensus sums
//   consensus_kernel z = sum m / count per free break-point
//
// Iterations after the first are replayed from captured CUDA graphs.
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
#include "twa_iter.cuh"
#include "twa_backward.cuh"

namespace {

// Programmatic dependent launch: the three kernels of an iteration are
// launched with programmatic stream serialization, so each one's CTAs can be
// scheduled while the previous kernel drains (every CTA lets its dependents
// launch as soon as it starts); griddepcontrol.wait then holds them until the
// previous kernel has completed and its writes are visible.  Without the
// launch attribute both instructions do nothing.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The single-planner kernels: thin wrappers over the per-block work.
constexpr int TEST_WARPS = 4;
constexpr int TEST_ROWS = TILE / TEST_WARPS;

// Pass 1 is one launch: its first nseg = eta x (agent tiles) blocks take the
// kinetic and wall factors of one (segment, agent tile) each (segment_block,
// dispatched first), the rest the collision blocks.  Both kinds of work
// depend only on z^k, so one launch replaces two streams and their join.
template <bool DENSE>
__global__ void __launch_bounds__(32 * TEST_WARPS, 8) test_kernel(Dev P, int nseg) {
  pdl_begin();
  if ((int)blockIdx.x < nseg) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.res_cur = 0u;
    segment_block<true>(P, blockIdx.x);
    return;
  }
  test_block<DENSE, TEST_ROWS>(P, blockIdx.x - nseg);
}

// Gated state: one warp per tile, lane = row agent (test_tile_rows).  The
// register cap keeps the collision blocks at their own count (48), which
// sets the occupancy; the kinetic and wall blocks spill a little under it.
constexpr int TILES_PER_CTA = 4;  // the batched test pass
constexpr int ROWS_WARPS = 4;     // tiles (warps) per CTA of test_rows_kernel (2 and 8 measured slower)
__global__ void __launch_bounds__(32 * ROWS_WARPS, 40 / ROWS_WARPS) test_rows_kernel(Dev P, int nseg) {
  __shared__ float4 col[ROWS_WARPS][72];
  __shared__ uint32_t nws[ROWS_WARPS][32];
  pdl_begin();
  if (blockIdx.x == 0 && threadIdx.x == 0) *P.res_cur = 0u;
  if ((int)blockIdx.x < nseg) {
    segment_block<true>(P, blockIdx.x);
    return;
  }
  const int warp = threadIdx.x >> 5;
  // the first hcap warps take the tiles listed heavy by the previous
  // iteration; the others go through every tile segment-minor (t -> segment
  // t mod eta, so that a crowded segment spreads over the launch), skipping
  // the listed ones
  const int t = ((int)blockIdx.x - nseg) * ROWS_WARPS + warp;
  int blk;
  bool check_stamp = false;
  if (t < P.hcap) {
    // the list's length and this warp's entry are loaded together (t < hcap
    // keeps the entry in bounds; it is used only below the length)
    const unsigned hc = ld_now(P.hcount_cur);
    const unsigned hb = ld_now(P.heavy_cur + t);
    if (t >= (int)hc) return;  // warp-uniform
    blk = (int)hb;
  } else {
    const int tr = t - P.hcap;
    if (tr >= P.eta * P.ntp) return;  // warp-uniform
    const int s = tr % P.eta;
    if (P.vo && s != 0) return;  // no collision factors on the second segment
    blk = s * P.ntp + tr / P.eta;
    check_stamp = P.hcap != 0;  // skipped there if a heavy warp takes it
  }
  test_tile_rows(P, blk, col[warp], nws[warp], check_stamp);
}

// Worklist items are dealt to warps round-robin (item t to warp t mod W,
// lane t / W mod 32), so that a short list spreads over every SM instead of
// filling the first few warps: each minimizer is a long dependent chain, and
// a warp's time grows with the number of (divergent) items it holds.
__device__ __forceinline__ unsigned long long dealt_first(unsigned long long& stride) {
  const unsigned long long W = (gridDim.x * blockDim.x) >> 5;
  stride = 32ull * W;
  return (unsigned long long)(threadIdx.x & 31) * W + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
}

// Pass 2: every active wall's minimizer on a warp of its own (all lanes
// cooperating), the first warp of each of the first n_wall CTAs, so that
// these long chains sit on different SMs.  The collision minimizers go in
// groups of 32 consecutive worklist entries (pairs of one tile, so of one
// segment: the lanes take the same branches) to the other warps, ordered so
// that consecutive groups land on different CTAs and so spread over the SMs.
// (More active walls than CTAs: walls over all warps, then pairs.)
__global__ void __launch_bounds__(256) prox_kernel(Dev P) {
  pdl_begin();
  const unsigned long long nc = *P.work_count, nwl = *P.wwork_count;
  const unsigned long long wpb = blockDim.x >> 5, G = gridDim.x, b = blockIdx.x;
  const unsigned long long wib = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31;
  unsigned long long v, Wc;  // this warp's place among the collision warps, their number
  // The wall items of this warp: first, first + stride, ... below nwl.  Both
  // dealings go through this one call of the wall minimizer: with two call
  // sites the compiler inlined two copies whose floating-point contractions
  // differed, so the result of a wall factor depended on whether the active
  // walls outnumbered the CTAs (that is, on the GPU's SM count).
  unsigned long long first, stride;
  bool wall_only;
  if (nwl <= G) {
    wall_only = b < nwl && wib == 0;
    first = wall_only ? b : nwl;
    stride = G;
    Wc = G * wpb - nwl;
    v = wib == 0 ? b - nwl : (G - nwl) + (wib - 1) * G + b;
  } else {
    wall_only = false;
    first = b * wpb + wib;
    stride = G * wpb;
    Wc = G * wpb;
    v = wib * G + b;
  }
  for (unsigned long long t = first; t < nwl; t += stride) wall_prox_item_warp(P, P.wwork[t]);
  if (wall_only) return;
  for (unsigned long long t = 32ull * v + lane; t < nc; t += 32ull * Wc) prox_item(P, P.work[t]);
}

__global__ void consensus_kernel(Dev P) {
  pdl_begin();
  const int nfree = (P.eta - 1) * P.p;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *P.work_count_next = 0u;
    *P.wwork_count_next = 0u;
    if (P.hcap) {
      *P.hcount_cur = 0u;  // read by this iteration's pass 1; the next-but-one builds into it
      *P.iter += 1u;
    }
  }
  float dz = 0.f;
  bool bad = false;
  if (t < nfree) consensus_node(P, t, dz, bad);
  consensus_reduce(P, dz, bad);
}

// Fixed-point scale of the consensus sums: the largest power of two with
// 8 (L + 1) x (max incoming edges) x scale <= 2^62, L the largest coordinate
// magnitude of the endpoints and walls.  One block.
// The scale from the largest coordinate magnitude L of endpoints and walls:
// with y = 8 (L + 1) x edges (exact in double: a 27-bit mantissa times an
// integer below 2^17), e = floor(log2(2^62 / y)) = 62 - ceil(log2 y), and
// ceil(log2 y) is read off y's exponent and mantissa bits (no FP64 maths
// library call: a single thread runs this on the update's critical path).
__device__ __forceinline__ void set_fix(const Dev& P, float L) {
  const double edges = 2.0 + 2.0 * (P.p - 1) + 2.0 * (P.nw + P.nv);
  const double bound = 8.0 * ((double)L + 1.0);
  const unsigned long long yb = (unsigned long long)__double_as_longlong(bound * edges);
  const int ex = (int)((yb >> 52) & 0x7ff) - 1023;
  const int clog2 = ex + ((yb & 0xfffffffffffffull) ? 1 : 0);
  int e = 62 - clog2;
  e = e < 8 ? 8 : (e > 60 ? 60 : e);
  float* f = const_cast<float*>(P.fix);
  f[0] = ldexpf(1.f, e);
  f[1] = (float)bound;
}

__device__ __forceinline__ void fix_block(const Dev& P, const float2* start, const float2* goal) {
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
  if (threadIdx.x == 0) set_fix(P, red[0]);
}
__global__ void fix_kernel(Dev P, const float2* start, const float2* goal) {
  fix_block(P, start, goal);
}

// ---------------------------------------------------------------------------
// plan_check: the final feasibility and cost check in FP64 (Eq.
// velo_cost_pair_wise, Eq. basic_opt_prob) on the FP32 break-points z^k.
// Smallest clearances are kept as squared ratios; a non-negative double's bit
// pattern orders like the double, so 64-bit atomicMin takes their minimum.

// Squared distance from the origin to the segment a -> b.
__device__ __forceinline__ double origin_seg_dist2(double ax, double ay, double bx, double by) {
  const double dx = bx - ax, dy = by - ay, dd = dx * dx + dy * dy;
  double t = dd > 0.0 ? -(ax * dx + ay * dy) / dd : 0.0;
  t = fmin(1.0, fmax(0.0, t));
  const double cx = ax + t * dx, cy = ay + t * dy;
  return cx * cx + cy * cy;
}

__device__ __forceinline__ void block_min_u64(unsigned long long v, unsigned long long* out) {
  __shared__ unsigned long long red[32];
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : ~0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w < v ? w : v;
    }
    if (lane == 0 && v != ~0ull) atomicMin(out, v);  // nothing to report: no atomic
  }
}

// One block per (segment s, agent tile pair): min over its pairs i < j of
// dist^2 / (r_i + r_j)^2, dist the smallest distance between the agents
// over the segment (the origin against their relative motion).
__global__ void check_pairs_kernel(Dev P, unsigned long long* out) {
  const int s = blockIdx.x / P.ntp, tp = blockIdx.x - s * P.ntp;
  const int2 IJ = P.tiles[tp];
  const int E1 = P.eta + 1;
  double best = __longlong_as_double(0x7ff0000000000000ll);
  for (int q = threadIdx.x; q < TILE * TILE; q += blockDim.x) {
    const int i = IJ.x * TILE + (q >> 5), j = IJ.y * TILE + (q & 31);
    if (i >= j || j >= P.p) continue;
    const float2 zil = P.z[(size_t)i * E1 + s], zih = P.z[(size_t)i * E1 + s + 1];
    const float2 zjl = P.z[(size_t)j * E1 + s], zjh = P.z[(size_t)j * E1 + s + 1];
    const double ax = (double)zjl.x - (double)zil.x, ay = (double)zjl.y - (double)zil.y;
    const double bx = (double)zjh.x - (double)zih.x, by = (double)zjh.y - (double)zih.y;
    const double R = (double)P.radius[i] + (double)P.radius[j];
    best = fmin(best, origin_seg_dist2(ax, ay, bx, by) / (R * R));
  }
  block_min_u64((unsigned long long)__double_as_longlong(best), out);
}

// Squared distance from point (px, py) to the segment a -> b.
__device__ __forceinline__ double point_seg_dist2(double px, double py, double ax, double ay,
                                                  double bx, double by) {
  return origin_seg_dist2(ax - px, ay - py, bx - px, by - py);
}

// One thread per (wall, segment, agent): dist^2 / r_i^2, dist the distance
// between the agent's segment and the wall segment (0 if they cross).
__global__ void check_walls_kernel(Dev P, int nseg, unsigned long long* out) {
  const int E1 = P.eta + 1;
  double best = __longlong_as_double(0x7ff0000000000000ll);
  const long long n = (long long)P.nw * nseg * P.p;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % P.p);
    const int s = (int)((t / P.p) % nseg);
    const int w = (int)(t / ((long long)P.p * nseg));
    const float4 W = P.walls[w];
    const float2 a = P.z[(size_t)i * E1 + s], b = P.z[(size_t)i * E1 + s + 1];
    const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
    const double cx = W.x, cy = W.y, dx = W.z, dy = W.w;
    const double o1 = (dx - cx) * (ay - cy) - (dy - cy) * (ax - cx);
    const double o2 = (dx - cx) * (by - cy) - (dy - cy) * (bx - cx);
    const double o3 = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    const double o4 = (bx - ax) * (dy - ay) - (by - ay) * (dx - ax);
    double d2;
    if (((o1 > 0.0 && o2 < 0.0) || (o1 < 0.0 && o2 > 0.0)) &&
        ((o3 > 0.0 && o4 < 0.0) || (o3 < 0.0 && o4 > 0.0))) {
      d2 = 0.0;  // the segments cross
    } else {
      d2 = fmin(fmin(point_seg_dist2(ax, ay, cx, cy, dx, dy), point_seg_dist2(bx, by, cx, cy, dx, dy)),
                fmin(point_seg_dist2(cx, cy, ax, ay, bx, by), point_seg_dist2(dx, dy, ax, ay, bx, by)));
    }
    const double r = P.radius[i];
    best = fmin(best, d2 / (r * r));
  }
  block_min_u64((unsigned long long)__double_as_longlong(best), out);
}

// One block: the total kinetic cost sum c_{i,s} |z_i(s+1) - z_i(s)|^2 over
// the kinetic segments (fixed summation order, so the result is
// deterministic), the largest endpoint error |z - start|, |z - goal|, and
// the two clearance minima set to +inf for the kernels that follow.
__global__ void check_cost_kernel(Dev P, const double* ccost, const float2* start, const float2* goal,
                                  int s_lo, int s_hi, double* out) {
  __shared__ double sc[256], se[256];
  const int E1 = P.eta + 1;
  double c = 0.0, e = 0.0;
  for (int t = threadIdx.x; t < P.p * P.eta; t += blockDim.x) {
    const int i = t / P.eta, s = t - i * P.eta;
    if (s >= s_lo && s < s_hi) {
      const float2 a = P.z[(size_t)i * E1 + s], b = P.z[(size_t)i * E1 + s + 1];
      const double dx = (double)b.x - (double)a.x, dy = (double)b.y - (double)a.y;
      c += ccost[t] * (dx * dx + dy * dy);
    }
  }
  for (int i = threadIdx.x; i < P.p; i += blockDim.x) {
    const float2 a = P.z[(size_t)i * E1], b = P.z[(size_t)i * E1 + P.eta];
    e = fmax(e, fmax(fabs((double)a.x - (double)start[i].x), fabs((double)a.y - (double)start[i].y)));
    e = fmax(e, fmax(fabs((double)b.x - (double)goal[i].x), fabs((double)b.y - (double)goal[i].y)));
  }
  sc[threadIdx.x] = c;
  se[threadIdx.x] = e;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sc[threadIdx.x] += sc[threadIdx.x + o];
      se[threadIdx.x] = fmax(se[threadIdx.x], se[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sc[0];
    out[1] = __longlong_as_double(0x7ff0000000000000ll);
    out[2] = __longlong_as_double(0x7ff0000000000000ll);
    out[3] = se[0];
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
  for (int t = gt; t < (P.noenergy ? 0 : P.eta * P.p); t += nth) {
    const int s = t / P.p, i = t - s * P.p;
    if (P.vo && s == 0) continue;  // no kinetic factor on the epoch's motion
    float4 x = P.xkin[t];
    if (s != 0) res = fmaxf(res, maxabs2(lo2(x) - P.z[(size_t)i * E1 + s]));
    if (s != P.eta - 1) res = fmaxf(res, maxabs2(hi2(x) - P.z[(size_t)i * E1 + s + 1]));
  }
  for (int t = gt; t < (P.nw + P.nv) * P.eta * P.p; t += nth) {
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

// New fixed positions after the host check (plan_set_endpoints, large p):
// one block writes the fixed break-points of both z buffers and derives the
// fixed-point scale, which depends on the layout's extent.
__global__ void endpoints_fix_kernel(Dev P, const float2* start, const float2* goal) {
  const size_t E1 = (size_t)P.eta + 1;
  float2* z0 = const_cast<float2*>(P.z);
  for (int i = threadIdx.x; i < P.p; i += blockDim.x) {
    const float2 a = start[i], b = goal[i];
    z0[i * E1] = a; P.z_next[i * E1] = a;
    z0[i * E1 + P.eta] = b; P.z_next[i * E1 + P.eta] = b;
  }
  __syncthreads();
  fix_block(P, start, goal);
}

// A device-checked endpoint update (plan_set_endpoints), two launches.
// Feasibility of the new fixed positions uses the strict test of the host
// check in FP64: two disks closer than r_i + r_j, or a disk closer than r_i
// to a wall segment; a non-finite coordinate fails it before anything else.
// The first violation in the order (non-finite agents, start pairs, goal
// pairs, start-wall, goal-wall; then i; then j or the wall) is kept in key[0]
// as kind << 60 | i << 30 | j (~0 when there is none), and the largest
// coordinate magnitude of the new starts and goals (the layout's extent, for
// the fixed-point scale) in key[1].
// endpoint_stage_kernel, one thread per agent: reads the agent's new start
// and goal from the staging area once (it may sit in pinned host memory, so
// the whole update crosses the link in one coalesced pass), copies them to a
// device shadow and takes the non-finite test and the extent.
// endpoint_update_kernel, launched behind it with programmatic serialization
// (its griddepcontrol.wait makes the shadow visible): one warp takes 8 rows
// of one 32 x 32 agent tile pair of the starts (then of the goals) at a time
// from the shadow, lane c holding column agent c and the row agents coming by
// shuffles; then every thread takes agent-wall tests, grid-stride.  The last
// block to finish (counted in key[2]) writes the verdict (key[0]) to the
// host's word, resets the three key words for the next update and, if key[0]
// is clear, applies the update from the shadow: the new endpoints, the fixed
// break-points of both z buffers and the fixed-point scale.
__device__ __forceinline__ unsigned long long endpoint_key(unsigned kind, unsigned i, unsigned j) {
  return ((unsigned long long)kind << 60) | ((unsigned long long)i << 30) | (unsigned long long)j;
}

constexpr int EP_ROWS = 8;  // rows of a tile pair per warp task

__global__ void __launch_bounds__(256) endpoint_stage_kernel(Dev P, const float2* __restrict__ staged,
                                                             float2* __restrict__ shadow,
                                                             unsigned long long* key) {
  pdl_begin();
  const int p = P.p;
  const int gid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const bool has_e = gid < p;
  const float2 ea = has_e ? staged[gid] : mk(0.f, 0.f), eb = has_e ? staged[p + gid] : mk(0.f, 0.f);
  unsigned long long best = ~0ull;
  float ext = 0.f;
  if (has_e) {
    shadow[gid] = ea;
    shadow[p + gid] = eb;
    if (!(isfinite(ea.x) && isfinite(ea.y) && isfinite(eb.x) && isfinite(eb.y)))
      best = endpoint_key(0, (unsigned)gid, 0);
    ext = fmaxf(maxabs2(ea), maxabs2(eb));
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
    best = w < best ? w : best;
    ext = fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (best != ~0ull) atomicMin(key, best);
    // a non-negative float orders like its bits
    if (ext > 0.f && __float_as_uint(ext) > (unsigned)__ldcg(key + 1))
      atomicMax(key + 1, (unsigned long long)__float_as_uint(ext));
  }
}

__global__ void __launch_bounds__(256) endpoint_update_kernel(Dev P, const float2* __restrict__ shadow,
                                                              int goals, float2* __restrict__ start,
                                                              float2* __restrict__ goal,
                                                              unsigned long long* key,
                                                              unsigned long long* verdict) {
  pdl_begin();
  const int p = P.p, ntp = P.ntp, nw = P.nw;
  const float2* __restrict__ st = shadow;
  const float2* __restrict__ gl = shadow + p;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const long long nwt = (long long)p * nw * (goals ? 2 : 1);
  constexpr int QUARTERS = TILE / EP_ROWS;
  unsigned long long best = ~0ull;
  const int tasks = ntp * (1 + goals) * QUARTERS;
  for (int task = warp; task < tasks; task += nwarps) {
    const int tq = task / QUARTERS, q = task - tq * QUARTERS;
    const int which = tq / ntp;
    const int2 IJ = P.tiles[tq - which * ntp];
    const float2* X = which ? gl : st;
    const int i0 = IJ.x * TILE + q * EP_ROWS, j = IJ.y * TILE + lane;
    const bool rowok = lane < EP_ROWS && i0 + lane < p;
    const float2 xi = rowok ? X[i0 + lane] : mk(0.f, 0.f);
    const float ri = rowok ? P.radius[i0 + lane] : 0.f;
    const float2 xj = j < p ? X[j] : mk(0.f, 0.f);
    const float rj = j < p ? P.radius[j] : 0.f;
#pragma unroll
    for (int r = 0; r < EP_ROWS; ++r) {
      const float xr = __shfl_sync(0xffffffffu, xi.x, r), yr = __shfl_sync(0xffffffffu, xi.y, r);
      const float rr = __shfl_sync(0xffffffffu, ri, r);
      const int i = i0 + r;
      // FP32 screen: pairs farther apart than (1 + 1e-4)(r_i + r_j) cannot
      // fail the FP64 test (FP32 rounding here is below 1e-6 relative)
      const float fx = xj.x - xr, fy = xj.y - yr, fR = rr + rj;
      if (i < j && j < p && fx * fx + fy * fy <= 1.0002f * fR * fR) {
        const double dx = (double)xj.x - (double)xr, dy = (double)xj.y - (double)yr;
        const double R = (double)rr + (double)rj;
        if (dx * dx + dy * dy < R * R) best = min(best, endpoint_key(1 + which, i, j));
      }
    }
  }
  for (long long t = gid; t < nwt; t += nthreads) {
    const int i = (int)(t % p);
    const long long rw = t / p;
    const int w = (int)(rw % nw), which = (int)(rw / nw);
    const float2 x = which ? gl[i] : st[i];
    const float4 W = P.walls[w];
    // FP32 screen: the distance to the segment computed in FP32 is within
    // a few 1e-7 x L of the exact one (L the largest coordinate magnitude
    // involved), so a disk clear of the wall by 1e-4 (1 + L) cannot fail
    // the FP64 test
    {
      const float fdx = W.z - W.x, fdy = W.w - W.y, fpx = x.x - W.x, fpy = x.y - W.y;
      const float fdd = fdx * fdx + fdy * fdy;
      const float ft = fdd > 0.f ? fminf(1.f, fmaxf(0.f, (fpx * fdx + fpy * fdy) / fdd)) : 0.f;
      const float fex = ft * fdx - fpx, fey = ft * fdy - fpy;
      const float Lw = fmaxf(fmaxf(fmaxf(fabsf(W.x), fabsf(W.y)), fmaxf(fabsf(W.z), fabsf(W.w))), maxabs2(x));
      const float rm = P.radius[i] + 1e-4f * (1.f + Lw);
      if (fex * fex + fey * fey > rm * rm) continue;
    }
    const double ax = W.x, ay = W.y, dx = (double)W.z - W.x, dy = (double)W.w - W.y;
    const double dd = dx * dx + dy * dy;
    const double px = (double)x.x - ax, py = (double)x.y - ay;
    const double t01 = dd > 0.0 ? fmin(1.0, fmax(0.0, (px * dx + py * dy) / dd)) : 0.0;
    const double ex = t01 * dx - px, ey = t01 * dy - py;
    const double r = P.radius[i];
    if (ex * ex + ey * ey < r * r) best = min(best, endpoint_key(3 + which, i, w));
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
    best = w < best ? w : best;
  }
  if (lane == 0 && best != ~0ull) atomicMin(key, best);
  // last block done: every block's atomics are ordered before its count
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(key + 2, 1ull) == (unsigned long long)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const unsigned long long k = __ldcg(key);
  const float L0 = __uint_as_float((unsigned)__ldcg(key + 1));
  __syncthreads();  // every thread has read the words before they are reset
  if (threadIdx.x == 0) {  // first, so that the store to the host drains under the copy
    *verdict = k;
    key[0] = ~0ull;
    key[1] = 0ull;
    key[2] = 0ull;
    if (k == ~0ull) {
      float L = L0;
      for (int w = 0; w < nw; ++w) {
        const float4 W = P.walls[w];
        L = fmaxf(L, fmaxf(fmaxf(fabsf(W.x), fabsf(W.y)), fmaxf(fabsf(W.z), fabsf(W.w))));
      }
      set_fix(P, L);
    }
  }
  if (k == ~0ull) {
    const size_t E1 = (size_t)P.eta + 1;
    float2* z0 = const_cast<float2*>(P.z);
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
      const float2 a = __ldcg(shadow + i), b = __ldcg(shadow + p + i);
      start[i] = a; goal[i] = b;
      z0[i * E1] = a; P.z_next[i * E1] = a;
      z0[i * E1 + P.eta] = b; P.z_next[i * E1 + P.eta] = b;
    }
  }
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
    if (P.noenergy || (P.vo && s == 0)) { ul = mk(0.f, 0.f); uh = ul; }  // no kinetic factor here
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
  const int words = (P.nw + P.nv) * P.eta * P.nt;
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

// Velocity kinds (gated segment factors nw .. nw + nv - 1): export u and
// activity; import u (pending x = z^k) and set bits where u != 0.
__global__ void export_vel_kernel(Dev P, int v, float* u_vel, uint8_t* act) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nk = P.eta * P.p, E1 = P.eta + 1;
  if (t >= nk) return;
  const int i = t % P.p, s = t / P.p;
  const size_t g = (size_t)(P.nw + v) * nk + t;
  const size_t ws = (size_t)(P.nw + v) * P.eta + s;
  const bool bprev = (P.wbits[ws * P.nt + i / TILE] >> (i % TILE)) & 1u;
  float4 u4 = P.uwall[g], x4 = P.xwall[g];
  if (!P.dense && !bprev) u4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float dummy = 0.f;
  const float2 ul = finish_u(bprev, s == 0, P.keep, lo2(u4), lo2(x4), P.z[(size_t)i * E1 + s], P.alpha, dummy);
  const float2 uh = finish_u(bprev, s == P.eta - 1, P.keep, hi2(u4), hi2(x4), P.z[(size_t)i * E1 + s + 1], P.alpha, dummy);
  if (u_vel) {
    float* o = u_vel + (size_t)t * 4;
    o[0] = ul.x; o[1] = ul.y; o[2] = uh.x; o[3] = uh.y;
  }
  if (act) act[t] = bprev ? 1 : 0;
}

__global__ void import_vel_kernel(Dev P, int v, const float* u_vel) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nk = P.eta * P.p, E1 = P.eta + 1;
  if (t >= nk) return;
  const int i = t % P.p, s = t / P.p;
  const size_t g = (size_t)(P.nw + v) * nk + t;
  float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
  if (u_vel) u = make_float4(u_vel[4 * (size_t)t], u_vel[4 * (size_t)t + 1], u_vel[4 * (size_t)t + 2], u_vel[4 * (size_t)t + 3]);
  P.uwall[g] = u;
  P.xwall[g] = pack(P.z[(size_t)i * E1 + s], P.z[(size_t)i * E1 + s + 1]);
}

// Back-weight classes of the feasibility problem after an import: rho0 at
// every node some factor sent rho0 to in the last iteration (a set activity
// bit), else 0; every node at the initial state (k = 0, Section 4).
__global__ void wnode_clear_kernel(Dev P, uint8_t value) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < P.p * (P.eta + 1)) P.wnode[t] = value;
}

__global__ void wnode_from_bits_kernel(Dev P) {
  const int E1 = P.eta + 1;
  const size_t nslots = (size_t)P.eta * P.ntp * TILE * TILE;
  const size_t nseg = (size_t)(P.nw + P.nv) * P.eta * P.p;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nslots + nseg;
       t += (size_t)gridDim.x * blockDim.x) {
    if (t < nslots) {
      const size_t row = t / TILE;
      const int lane = (int)(t - row * TILE);
      if (!((P.bits[row] >> lane) & 1u)) continue;
      const size_t blk = row / TILE;
      const int r = (int)(row - blk * TILE);
      const int s = (int)(blk / P.ntp);
      const int2 IJ = P.tiles[blk - (size_t)s * P.ntp];
      const int i = IJ.x * TILE + r, j = IJ.y * TILE + lane;
      P.wnode[(size_t)i * E1 + s] = 1; P.wnode[(size_t)i * E1 + s + 1] = 1;
      P.wnode[(size_t)j * E1 + s] = 1; P.wnode[(size_t)j * E1 + s + 1] = 1;
    } else {
      const size_t g = t - nslots;
      const int i = (int)(g % P.p);
      const size_t ws = g / P.p;
      const int s = (int)(ws % P.eta);
      if ((P.wbits[ws * P.nt + i / TILE] >> (i % TILE)) & 1u) {
        P.wnode[(size_t)i * E1 + s] = 1; P.wnode[(size_t)i * E1 + s + 1] = 1;
      }
    }
  }
}

// Velocity-obstacle epochs (Section 5): x_ref = x(0) + (dest - x(0)) clipped
// to length step; after the solve, x(0) moves a fraction of the way to x.
__global__ void vo_target_kernel(int p, const float2* start, const float2* dest, float step,
                                 float2* goal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  const float2 d = dest[i] - start[i];
  const float L = hypotf(d.x, d.y);
  const float sc = (L > step) ? step / L : 1.f;
  goal[i] = start[i] + sc * d;
}

__global__ void vo_advance_kernel(int p, int eta, const float2* z, const float2* dest, float frac,
                                  float2* start, unsigned* max_dist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float dist = 0.f;
  if (i < p) {
    const float2 x0 = start[i], x1 = z[(size_t)i * (eta + 1) + 1];
    const float2 xn = x0 + frac * (x1 - x0);
    start[i] = xn;
    const float2 d = dest[i] - xn;
    dist = hypotf(d.x, d.y);
  }
  dist = warp_max(dist);
  if ((threadIdx.x & 31) == 0 && dist > 0.f) atomicMax(max_dist, __float_as_uint(dist));
}

// Back-weight classes per node, out (export) or in (import): 2 at the fixed
// ends, else the stored class (rho0 whenever the kinetic factors run).
__global__ void back_weights_kernel(Dev P, uint8_t* out, const uint8_t* in) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int E1 = P.eta + 1;
  if (t >= P.p * E1) return;
  const int s = t % E1;
  const bool fixed = (s == 0 || s == P.eta);
  if (in) {
    if (!fixed) P.wnode[t] = in[t] ? 1 : 0;
  } else {
    out[t] = fixed ? 2 : (P.noenergy ? P.wnode[t] : 1);
  }
}

// New pending kinetic x = z, u = 0 (the kinetic factors switched back on).
__global__ void kinetic_restart_kernel(Dev P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.eta * P.p) return;
  const int s = t / P.p, i = t - s * P.p, E1 = P.eta + 1;
  P.xkin[t] = pack(P.z[(size_t)i * E1 + s], P.z[(size_t)i * E1 + s + 1]);
  P.ukin[t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void fill_kernel(float* a, size_t n, float v) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t] = v;
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

// plan_set_endpoints checks new endpoints on the device up to this many
// agents (an all-pairs test), and with the host grid above it.
constexpr size_t kDeviceEndpointCheck = 8192;

struct Layout {
  size_t z0, z1, start, goal, radius, cost, walls, vlim, wnode, tiles;
  size_t ulo, uhi, xlo, xhi, bits, ukin, xkin, uwall, xwall, wbits, work, wwork, wcount, sched,
      stamps, heavy, accx, accy, accc, fix,
      res, status, count, ccost, chk, ekey, eshadow;
  size_t total;
};

bool sizes_ok(const plan_config* c) {
  if (c->p < 1 || c->eta < 1 || c->n_walls < 0) return false;
  if (c->p > (1 << 16) || c->eta > (1 << 12) || c->n_walls > 4096) return false;
  // pair slots are addressed by 32-bit indices (worklist entries, fid)
  const unsigned long long nt = (c->p + TILE - 1) / TILE, ntp = nt * (nt + 1) / 2;
  if ((unsigned long long)c->eta * ntp * TILE * TILE > 0xffffffffull) return false;
  return true;
}

// Heavy-tile slots at the front of pass 1: an eighth of the tiles.
size_t heavy_cap(size_t ntiles) { return std::max<size_t>(32, ntiles / 8); }

Layout layout_for(const plan_config* c) {
  const size_t p = c->p, eta = c->eta, nw = c->n_walls;
  const size_t nv = ((c->flags & PLAN_VMAX) ? 1 : 0) + ((c->flags & PLAN_VMIN) ? 1 : 0);
  const size_t ng = nw + nv;  // gated segment-factor kinds: walls, then velocity limits
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
  L.vlim = take(nv * p * eta * 4);
  L.wnode = take(p * (eta + 1));
  L.tiles = take(ntp * 8);
  L.ulo = take(slots * 16);
  L.uhi = take(slots * 16);
  L.xlo = take(slots * 16);
  L.xhi = take(slots * 16);
  L.bits = take(eta * ntp * TILE * 4);
  L.ukin = take(eta * p * 16);
  L.xkin = take(eta * p * 16);
  L.uwall = take(ng * eta * p * 16);
  L.xwall = take(ng * eta * p * 16);
  L.wbits = take(ng * eta * nt * 4);
  L.work = take(slots * 4);
  L.wwork = take(nw * eta * p * 4);
  L.wcount = take(4 * 4);  // collision and wall worklist counters, by iteration parity
  L.sched = take(4 * 4);   // iteration number, heavy-tile counts by parity
  L.stamps = take(2 * eta * ntp * 4);
  L.heavy = take(2 * heavy_cap(eta * ntp) * 4);
  L.accx = take(p * (eta + 1) * 8);
  L.accy = take(p * (eta + 1) * 8);
  L.accc = take(p * (eta + 1) * 4);
  L.fix = take(2 * 4);
  L.res = take(4 * 4);
  L.status = take(4);
  L.count = take(16);
  L.ccost = take(p * eta * 8);  // FP64 kinetic coefficients for plan_check
  L.chk = take(4 * 8);          // plan_check results
  L.ekey = take(24);            // plan_set_endpoints: first violation, extent, finished blocks
  // a device copy of the endpoints of a device-checked update, made while
  // they are checked
  L.eshadow = take(p <= kDeviceEndpointCheck ? p * 16 : 0);
  L.total = o;
  return L;
}

bool finite_all(const float* a, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(a[k])) return false;
  return true;
}


// Host-side input check: fixed configurations must be feasible (two disks
// closer than r_i + r_j, or a disk closer than r_i to a wall, make the
// fixed-end minimizers infeasible).  Pairs are found on a uniform grid of
// cells at least max(r_i + r_j) wide: the agents are counting-sorted by cell
// into contiguous arrays, and each agent is compared with the later agents
// of its own cell and with those of four neighbouring cells (every
// neighbouring pair of cells once), so the check is linear in p.  The tests
// only accumulate a flag; the offending pair is looked up again only for the
// error message.  The grid's arrays are kept between calls (EndpointGrid).
struct EndpointGrid {
  std::vector<int> cell, start, fill, order;
  std::vector<double> xs, ys, rs;
};

plan_status check_endpoints(int p, const float* start, const float* goal, const float* radius,
                            int nw, const float* walls, bool goals_fixed = true,
                            EndpointGrid* grid = nullptr) {
  EndpointGrid local;
  EndpointGrid& g = grid ? *grid : local;
  float rmax = 0.f;
  for (int i = 0; i < p; ++i) rmax = std::max(rmax, radius[i]);
  g.cell.resize(p);
  g.order.resize(p);
  g.xs.resize(p);
  g.ys.resize(p);
  g.rs.resize(p);
  // a velocity-obstacle epoch's goal node holds reference points, which the
  // factors never test against each other
  for (int which = 0; which < (goals_fixed ? 2 : 1); ++which) {
    const float* X = which ? goal : start;
    double x0 = X[0], y0 = X[1], x1 = X[0], y1 = X[1];
    for (int i = 1; i < p; ++i) {
      x0 = std::min(x0, (double)X[2 * i]); x1 = std::max(x1, (double)X[2 * i]);
      y0 = std::min(y0, (double)X[2 * i + 1]); y1 = std::max(y1, (double)X[2 * i + 1]);
    }
    // cells at least 2 rmax wide (plus a relative 1e-9, so that rounding in
    // the cell index cannot separate two overlapping disks by two cells), no
    // more than about 4 per agent
    double cw = std::max(2.0 * (double)rmax * (1.0 + 1e-9), 1e-6);
    const double area = std::max(x1 - x0, cw) * std::max(y1 - y0, cw);
    cw = std::max(cw, std::sqrt(area / (4.0 * p + 16.0)));
    const int nx = (int)std::max(1.0, std::floor((x1 - x0) / cw));
    const int ny = (int)std::max(1.0, std::floor((y1 - y0) / cw));
    const double isx = nx / std::max(x1 - x0, 1e-300), isy = ny / std::max(y1 - y0, 1e-300);
    g.start.assign((size_t)nx * ny + 1, 0);
    for (int i = 0; i < p; ++i) {
      const int cx = std::min(nx - 1, (int)((X[2 * i] - x0) * isx));
      const int cy = std::min(ny - 1, (int)((X[2 * i + 1] - y0) * isy));
      g.cell[i] = cy * nx + cx;
      g.start[g.cell[i] + 1] += 1;
    }
    for (size_t c = 0; c < (size_t)nx * ny; ++c) g.start[c + 1] += g.start[c];
    g.fill.assign(g.start.begin() + 1, g.start.end());  // per-cell ends, filled downwards
    for (int i = p - 1; i >= 0; --i) {
      const int u = --g.fill[g.cell[i]];
      g.order[u] = i;
      g.xs[u] = X[2 * i];
      g.ys[u] = X[2 * i + 1];
      g.rs[u] = radius[i];
    }
    // agent u (sorted) against the sorted range [v0, v1)
    auto range_hits = [&](int u, int v0, int v1) {
      bool hit = false;
      for (int v = v0; v < v1; ++v) {
        const double dx = g.xs[v] - g.xs[u], dy = g.ys[v] - g.ys[u], R = g.rs[u] + g.rs[v];
        hit |= dx * dx + dy * dy < R * R;
      }
      return hit;
    };
    static const int nb[4][2] = {{1, 0}, {-1, 1}, {0, 1}, {1, 1}};
    for (int u = 0; u < p; ++u) {
      const int c = g.cell[g.order[u]], cx = c % nx, cy = c / nx;
      bool hit = range_hits(u, u + 1, g.start[c + 1]);
      int culprit_cell = c;
      for (int q = 0; q < 4 && !hit; ++q) {
        const int gx = cx + nb[q][0], gy = cy + nb[q][1];
        if (gx < 0 || gx >= nx || gy >= ny) continue;
        const int d = gy * nx + gx;
        hit = range_hits(u, g.start[d], g.start[d + 1]);
        culprit_cell = d;
      }
      if (hit) {  // find the partner for the message
        const int v0 = culprit_cell == c ? u + 1 : g.start[culprit_cell];
        for (int v = v0; v < g.start[culprit_cell + 1]; ++v) {
          if (range_hits(u, v, v + 1)) {
            const int i = g.order[u], j = g.order[v];
            return fail(PLAN_EINFEASIBLE_INPUT, "%s positions of agents %d and %d overlap",
                        which ? "goal" : "start", std::min(i, j), std::max(i, j));
          }
        }
      }
    }
    for (int w = 0; w < nw; ++w) {
      const float* W = walls + 4 * w;
      const double ax = W[0], ay = W[1], dx = (double)W[2] - W[0], dy = (double)W[3] - W[1];
      const double dd = dx * dx + dy * dy, idd = dd > 0.0 ? 1.0 / dd : 0.0;
      bool hit = false;
      for (int i = 0; i < p; ++i) {
        const double px = (double)X[2 * i] - ax, py = (double)X[2 * i + 1] - ay;
        const double t = std::min(1.0, std::max(0.0, (px * dx + py * dy) * idd));
        const double ex = t * dx - px, ey = t * dy - py;
        hit |= ex * ex + ey * ey < (double)radius[i] * radius[i];
      }
      if (!hit) continue;
      for (int i = 0; i < p; ++i) {
        const double px = (double)X[2 * i] - ax, py = (double)X[2 * i + 1] - ay;
        const double t = std::min(1.0, std::max(0.0, (px * dx + py * dy) * idd));
        const double ex = t * dx - px, ey = t * dy - py;
        if (ex * ex + ey * ey < (double)radius[i] * radius[i])
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
  int nv = 0;             // velocity-limit kinds (PLAN_VMAX, PLAN_VMIN)
  unsigned vmin_mask = 0; // which of them are minima
  bool noenergy = false;  // kinetic factors off (PLAN_NO_ENERGY or plan_set_energy)
  bool vo = false;        // PLAN_VO: one velocity-obstacle epoch
  size_t slots;
  cudaStream_t stream;
  Layout L;
  char* ws;
  bool own_ws;
  int k;
  int cur;  // which z buffer holds z^k
  int prox_grid = 0;  // CTAs of the minimizer pass (resident CTAs per SM x SMs)
  cudaStream_t cap = nullptr;    // private stream for capturing the iteration graphs
  bool profiling = false;        // plan_profile: per-kernel event timing
  cudaEvent_t pev[6] = {};
  cudaEvent_t pend = nullptr;
  cudaGraphExec_t gexec[4] = {};  // captured iterations by (k parity, z buffer)
  cudaGraphExec_t gexec8[4] = {}; // ... and runs of ITERS_PER_GRAPH iterations
  cudaGraphExec_t gexec64[4] = {}; // ... and of ITERS_PER_LONG_GRAPH iterations
  double ptime[4] = {0, 0, 0, 0};
  int pcount = 0;
  unsigned* h_res;  // pinned host words: residual readback (0), endpoint check key (2..3)
  float* h_stage = nullptr;  // pinned staging of new endpoints (plan_set_endpoints)
  cudaGraphExec_t gset = nullptr;  // plan_set_endpoints' device work (fixed pointers)
  cudaEvent_t ep_event = nullptr;  // after the last endpoint update's graph
  bool ep_pending = false;         // an asynchronous endpoint update's verdict not yet read
  std::vector<float> ep_start, ep_goal;  // its endpoints, taken on the host once it passed
  EndpointGrid grid;         // the host check's arrays, kept between calls
  std::vector<float> h_radius;
  std::vector<float> h_walls;
  std::vector<float> h_start, h_goal;
  // differentiation (plan_unroll / plan_backward)
  char* adj = nullptr;           // checkpoints, tape and adjoint state
  size_t adj_bytes = 0;
  int adj_K = -1, adj_C = 0;     // the last unroll
  bool adj_valid = false;        // state unchanged since that unroll
  std::vector<int> ck_cur;       // z buffer holding z at each checkpoint

  template <class T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }

  float rho_at(int kk) const {
    return (kk < cfg.warm_iters) ? cfg.warm_rho : cfg.rho0;
  }
  // first iteration whose kernel arguments no longer change with k (graphs
  // are captured from there): past the warm-up, and past the deferred dual
  // step of its last iteration
  int graph_from() const { return cfg.warm_iters > 0 ? cfg.warm_iters + 1 : 1; }

  Dev dev(int kk) const {
    Dev P{};
    P.p = p; P.eta = eta; P.nw = nw; P.nt = nt; P.ntp = ntp;
    P.nv = nv;
    P.vmin_mask = vmin_mask;
    P.noenergy = noenergy ? 1 : 0;
    P.vo = vo ? 1 : 0;
    P.vlim = at<float>(L.vlim);
    P.wnode = at<uint8_t>(L.wnode);
    P.rho = rho_at(kk);
    // pass 1 of iteration kk finishes the dual step of iteration kk - 1, so
    // the printed step alpha / rho takes the rho of that iteration
    P.alpha = (cfg.flags & PLAN_U_LITERAL) ? cfg.alpha / rho_at(kk > 0 ? kk - 1 : 0) : cfg.alpha;
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
    P.wwork = at<uint32_t>(L.wwork);
    P.wwork_count = at<unsigned>(L.wcount) + 2 + (kk & 1);
    P.wwork_count_next = at<unsigned>(L.wcount) + 2 + ((kk + 1) & 1);
    {
      const size_t cap = heavy_cap((size_t)eta * ntp);
      P.hcap = (int)cap;
      P.iter = at<unsigned>(L.sched);
      P.hcount_cur = at<unsigned>(L.sched) + 1 + (kk & 1);
      P.hcount_next = at<unsigned>(L.sched) + 1 + ((kk + 1) & 1);
      P.heavy_cur = at<uint32_t>(L.heavy) + (kk & 1) * cap;
      P.heavy_next = at<uint32_t>(L.heavy) + ((kk + 1) & 1) * cap;
      const size_t ntiles = (size_t)eta * ntp;
      P.stamp_cur = at<unsigned>(L.stamps) + (kk & 1) * ntiles;
      P.stamp_next = at<unsigned>(L.stamps) + ((kk + 1) & 1) * ntiles;
    }
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
// an asynchronous endpoint update's verdict, read by every call that synchronises
plan_status settle_endpoints(plan_t h);
}  // namespace

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

// A launch with programmatic stream serialization (see pdl_begin).
template <typename... Args>
cudaError_t launch_pdl(void (*kern)(Args...), unsigned grid, unsigned block, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Enqueue the kernels of iteration h->k (no state change on the host).
plan_status enqueue_iteration(plan_t h, cudaStream_t ms) {
  Dev P = h->dev(h->k);
  const unsigned grid = (unsigned)((size_t)h->eta * h->ntp);
  const int nseg = h->eta * h->nt;  // kinetic and wall blocks, ahead of the collision blocks
  const bool prof = h->profiling;
  if (prof) CK(cudaEventRecord(h->pev[0], ms));
  if (P.dense)
    CK(launch_pdl(test_kernel<true>, nseg + grid, 32 * TEST_WARPS, ms, P, nseg));
  else
    CK(launch_pdl(test_rows_kernel, nseg + (P.hcap + grid + ROWS_WARPS - 1) / ROWS_WARPS,
                  32 * ROWS_WARPS, ms, P, nseg));
  if (prof) CK(cudaEventRecord(h->pev[1], ms));
  CK(launch_pdl(prox_kernel, h->prox_grid, 256, ms, P));
  if (prof) CK(cudaEventRecord(h->pev[2], ms));
  // the consensus kernel also clears the next iteration's worklist counter, so
  // it runs even when there is no free break-point (eta = 1)
  const int nfree = (h->eta - 1) * h->p;
  CK(launch_pdl(consensus_kernel, std::max(1, (nfree + 63) / 64), 64, ms, P));
  if (prof) {
    CK(cudaEventRecord(h->pend, ms));
    CK(cudaEventSynchronize(h->pend));
    float t[4];
    CK(cudaEventElapsedTime(&t[0], h->pev[0], h->pev[1]));
    CK(cudaEventElapsedTime(&t[1], h->pev[1], h->pev[2]));
    t[2] = 0.f;  // the kinetic and wall blocks run inside the pass-1 launch
    CK(cudaEventElapsedTime(&t[3], h->pev[2], h->pend));
    for (int q = 0; q < 4; ++q) h->ptime[q] += t[q];
    h->pcount += 1;
  }
  CK(cudaGetLastError());
  return PLAN_OK;
}

// One iteration: replay a captured CUDA graph of the three kernels when one
// fits (past the rho warm-up, not profiling), else launch them directly.
plan_status run_iteration(plan_t h) {
  plan_status st = ensure_prox_grid(h);
  if (st != PLAN_OK) return st;
  const bool graphable = h->cap && !h->profiling && h->k >= h->graph_from();
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

// Runs of ITERS_PER_LONG_GRAPH, then ITERS_PER_GRAPH iterations replayed
// from one graph each (even counts, so a run ends at the parity and z buffer
// it started from): fewer launches for problems small enough that launching
// is the cost, and fewer graph boundaries, where the programmatic-launch
// chain of the kernels starts over, in long runs.
constexpr int ITERS_PER_GRAPH = 8;
constexpr int ITERS_PER_LONG_GRAPH = 64;

plan_status run_graph_runs(plan_t h, int& n, int len, cudaGraphExec_t* execs) {
  while (n >= len && h->cap && !h->profiling && h->k >= h->graph_from()) {
    const int key = ((h->k & 1) << 1) | h->cur;
    if (!execs[key]) {
      const int k0 = h->k, c0 = h->cur;
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
      plan_status cst = PLAN_OK;
      for (int q = 0; q < len && cst == PLAN_OK; ++q) {
        cst = enqueue_iteration(h, h->cap);
        if (h->eta > 1) h->cur ^= 1;
        h->k += 1;
      }
      h->k = k0;
      h->cur = c0;
      cudaError_t e = cudaStreamEndCapture(h->cap, &g);
      if (cst != PLAN_OK) { if (g) cudaGraphDestroy(g); return cst; }
      if (e != cudaSuccess) return fail(PLAN_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&execs[key], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(PLAN_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    CK(cudaGraphLaunch(execs[key], h->stream));
    h->k += len;
    n -= len;
  }
  return PLAN_OK;
}

plan_status run_iterations(plan_t h, int n) {
  plan_status st = ensure_prox_grid(h);
  if (st != PLAN_OK) return st;
  if ((st = run_graph_runs(h, n, ITERS_PER_LONG_GRAPH, h->gexec64)) != PLAN_OK) return st;
  if ((st = run_graph_runs(h, n, ITERS_PER_GRAPH, h->gexec8)) != PLAN_OK) return st;
  for (; n > 0; --n)
    if ((st = run_iteration(h)) != PLAN_OK) return st;
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
  std::vector<double> ccost(p * eta);
  const double norm = (c.flags & (PLAN_COST_UNNORM | PLAN_VO)) ? 1.0 : 1.0 / ((double)p * eta);
  for (size_t i = 0; i < p; ++i)
    for (size_t s = 0; s < eta; ++s) {
      double C = (c.flags & PLAN_COST_PER_SEGMENT) ? cost_w[i * eta + s] : cost_w[i];
      ccost[i * eta + s] = C * norm;
      cost[i * eta + s] = (float)(C * norm);
    }
  std::vector<int2> tiles;
  for (int I = 0; I < h->nt; ++I)
    for (int J = I; J < h->nt; ++J) tiles.push_back(make_int2(I, J));
  CK(cudaMemcpyAsync(h->at<void>(h->L.start), start, p * 8, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.goal), goal, p * 8, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.radius), radius, p * 4, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.cost), cost.data(), p * eta * 4, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.ccost), ccost.data(), p * eta * 8, cudaMemcpyHostToDevice, h->stream));
  if (h->nw)
    CK(cudaMemcpyAsync(h->at<void>(h->L.walls), walls, (size_t)h->nw * 16, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.tiles), tiles.data(), tiles.size() * 8, cudaMemcpyHostToDevice, h->stream));
  // the staging vectors die at return: wait for the copies
  CK(cudaStreamSynchronize(h->stream));
  return PLAN_OK;
}

// Back-weight classes after an import (feasibility problem only).
plan_status derive_wnode(plan_t h) {
  if (!h->noenergy) return PLAN_OK;
  Dev P = h->dev(h->k);
  const int nodes = h->p * (h->eta + 1);
  wnode_clear_kernel<<<(nodes + 255) / 256, 256, 0, h->stream>>>(P, h->k == 0 ? 1 : 0);
  if (h->k > 0) wnode_from_bits_kernel<<<304, 256, 0, h->stream>>>(P);
  CK(cudaGetLastError());
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
  h->adj_valid = false;
  h->k = 0;
  h->cur = 0;
  Dev P = h->dev(0);
  const size_t zbytes = (size_t)h->p * (h->eta + 1) * 8;
  (void)zbytes;
  CK(cudaMemsetAsync(h->at<void>(h->L.bits), 0, (size_t)h->eta * h->ntp * TILE * 4, h->stream));
  const size_t ng = (size_t)h->nw + h->nv;
  if (ng) CK(cudaMemsetAsync(h->at<void>(h->L.wbits), 0, ng * h->eta * h->nt * 4, h->stream));
  CK(cudaMemsetAsync(h->at<void>(h->L.wnode), 1, (size_t)h->p * (h->eta + 1), h->stream));
  if (h->cfg.flags & (PLAN_DENSE_STATE | PLAN_U_KEEP | PLAN_ADMM)) {
    CK(cudaMemsetAsync(h->at<void>(h->L.ulo), 0, h->slots * 16, h->stream));
    CK(cudaMemsetAsync(h->at<void>(h->L.uhi), 0, h->slots * 16, h->stream));
    if (ng) CK(cudaMemsetAsync(h->at<void>(h->L.uwall), 0, ng * h->eta * h->p * 16, h->stream));
  }
  CK(cudaMemsetAsync(h->at<void>(h->L.res), 0, 16, h->stream));
  CK(cudaMemsetAsync(h->at<void>(h->L.wcount), 0, 16, h->stream));
  CK(cudaMemsetAsync(h->at<void>(h->L.sched), 0, 16, h->stream));

  CK(cudaMemsetAsync(h->at<void>(h->L.stamps), 0xff, 2 * (size_t)h->eta * h->ntp * 4, h->stream));
  CK(clear_sums(h));
  CK(cudaMemsetAsync(h->at<void>(h->L.status), 0, 4, h->stream));
  // plan_set_endpoints' words: no violation, extent 0, no fix-up block done
  CK(cudaMemsetAsync(h->at<void>(h->L.ekey), 0xff, 8, h->stream));
  CK(cudaMemsetAsync(h->at<char>(h->L.ekey) + 8, 0, 16, h->stream));
  fix_kernel<<<1, 256, 0, h->stream>>>(P, h->at<float2>(h->L.start), h->at<float2>(h->L.goal));
  const int n = std::max(h->p * (h->eta + 1), h->eta * h->p);
  reset_kernel<<<(n + 255) / 256, 256, 0, h->stream>>>(P, h->at<float2>(h->L.z0), h->at<float2>(h->L.z1),
                                                      h->at<float2>(h->L.start), h->at<float2>(h->L.goal));
  CK(cudaGetLastError());
  return PLAN_OK;
}

}  // extern "C"

namespace {

// Shared by plan_create and the batch: a batch member (member = true) has no
// streams, events or pinned buffer of its own; the batch drives it.
plan_status create_plan(const plan_config* cfg, const float* start, const float* goal,
                        const float* radius, const float* cost_w, const float* walls,
                        void* workspace, size_t workspace_bytes, void* cuda_stream, bool member,
                        plan_t* out) {
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
                         PLAN_DENSE_STATE | PLAN_ADMM | PLAN_NO_ENERGY | PLAN_VMAX | PLAN_VMIN |
                         PLAN_VO | PLAN_U_LITERAL;
  if (cfg->flags & ~known) return fail(PLAN_EINVAL, "unknown flag bits 0x%x", cfg->flags & ~known);
  if ((cfg->flags & PLAN_VO) && (cfg->eta != 2 || (cfg->flags & (PLAN_ADMM | PLAN_NO_ENERGY))))
    return fail(PLAN_EINVAL, "PLAN_VO needs eta = 2 and the kinetic factors, without PLAN_ADMM");
  if ((cfg->flags & PLAN_ADMM) && (cfg->flags & (PLAN_NO_ENERGY | PLAN_VMAX | PLAN_VMIN)))
    return fail(PLAN_EUNSUPPORTED, "standard-ADMM mode runs with the kinetic factors only");
  const size_t p = cfg->p, eta = cfg->eta;
  const size_t ncost = (cfg->flags & PLAN_COST_PER_SEGMENT) ? p * eta : p;
  if (!finite_all(start, 2 * p) || !finite_all(goal, 2 * p) || !finite_all(radius, p) ||
      !finite_all(cost_w, ncost) || (cfg->n_walls && !finite_all(walls, 4 * (size_t)cfg->n_walls)))
    return fail(PLAN_EINVAL, "non-finite input");
  for (size_t i = 0; i < p; ++i)
    if (!(radius[i] > 0.f)) return fail(PLAN_EINVAL, "radius[%zu] must be positive", i);
  for (size_t i = 0; i < ncost; ++i)
    if (cost_w[i] < 0.f) return fail(PLAN_EINVAL, "cost_w[%zu] must be >= 0", i);
  plan_status st = check_endpoints(cfg->p, start, goal, radius, cfg->n_walls, walls,
                                   !(cfg->flags & PLAN_VO));
  if (st != PLAN_OK) return st;

  Layout L = layout_for(cfg);
  plan_s* h = new plan_s();
  h->cfg = *cfg;
  if (h->cfg.check_every < 1) h->cfg.check_every = 1;
  h->p = cfg->p; h->eta = cfg->eta; h->nw = cfg->n_walls;
  h->nv = ((cfg->flags & PLAN_VMAX) ? 1 : 0) + ((cfg->flags & PLAN_VMIN) ? 1 : 0);
  h->vmin_mask = (cfg->flags & PLAN_VMIN) ? (1u << (h->nv - 1)) : 0u;
  h->noenergy = (cfg->flags & PLAN_NO_ENERGY) != 0;
  h->vo = (cfg->flags & PLAN_VO) != 0;
  h->nt = (h->p + TILE - 1) / TILE;
  h->ntp = h->nt * (h->nt + 1) / 2;
  h->slots = (size_t)h->eta * h->ntp * TILE * TILE;
  h->stream = (cudaStream_t)cuda_stream;
  h->L = L;
  h->h_radius.assign(radius, radius + p);
  h->h_start.assign(start, start + 2 * p);
  h->h_goal.assign(goal, goal + 2 * p);
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
  if (!member) {
    cudaError_t e = cudaMallocHost(&h->h_res, 16);
    if (e == cudaSuccess && (size_t)cfg->p <= kDeviceEndpointCheck)
      e = cudaMallocHost(&h->h_stage, (size_t)cfg->p * 16);
    if (e != cudaSuccess) {
      if (h->h_res) cudaFreeHost(h->h_res);
      if (h->own_ws) cudaFree(h->ws);
      delete h;
      return fail(PLAN_ENOMEM, "cudaMallocHost failed: %s", cudaGetErrorString(e));
    }
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
      plan_destroy(h);
      return fail(PLAN_ECUDA, "stream or event creation failed");
    }
  }
  st = upload_inputs(h, start, goal, radius, cost_w, walls);
  // velocity limits start unbinding: maxima +inf, minima 0 (plan_set_velocity_limits)
  for (int v = 0; v < h->nv && st == PLAN_OK; ++v) {
    const size_t n = (size_t)h->p * h->eta;
    fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        h->at<float>(h->L.vlim) + v * n, n, ((h->vmin_mask >> v) & 1u) ? 0.f : INFINITY);
    if (cudaGetLastError() != cudaSuccess) st = fail(PLAN_ECUDA, "fill_kernel launch failed");
  }
  if (st == PLAN_OK) st = plan_reset(h);
  if (st != PLAN_OK) {
    plan_destroy(h);
    return st;
  }
  *out = h;
  return PLAN_OK;
}

}  // namespace

extern "C" {

plan_status plan_create(const plan_config* cfg, const float* start, const float* goal,
                        const float* radius, const float* cost_w, const float* walls,
                        void* workspace, size_t workspace_bytes, void* cuda_stream, plan_t* out) {
  return create_plan(cfg, start, goal, radius, cost_w, walls, workspace, workspace_bytes,
                     cuda_stream, false, out);
}

void plan_destroy(plan_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
  if (h->own_ws && h->ws) cudaFree(h->ws);
  if (h->h_res) cudaFreeHost(h->h_res);
  if (h->h_stage) cudaFreeHost(h->h_stage);
  for (int q = 0; q < 6; ++q)
    if (h->pev[q]) cudaEventDestroy(h->pev[q]);
  for (int q = 0; q < 4; ++q)
    if (h->gexec[q]) cudaGraphExecDestroy(h->gexec[q]);
  for (int q = 0; q < 4; ++q)
    if (h->gexec8[q]) cudaGraphExecDestroy(h->gexec8[q]);
  for (int q = 0; q < 4; ++q)
    if (h->gexec64[q]) cudaGraphExecDestroy(h->gexec64[q]);
  if (h->pend) cudaEventDestroy(h->pend);
  if (h->gset) cudaGraphExecDestroy(h->gset);
  if (h->ep_event) cudaEventDestroy(h->ep_event);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->adj) cudaFree(h->adj);
  delete h;
}

}  // extern "C"

namespace {

// The endpoint update's graph (built on first use): check the staged
// endpoints, apply them if the check passed, hand the verdict back.  The
// kernels read the new endpoints from the pinned staging buffer and write the
// verdict into pinned host memory directly (both are mapped into the
// device's address space), and every pointer is fixed for the plan's life
// (both z buffers get the new fixed ends, whichever is current), so one
// graph serves every call.
plan_status endpoint_graph(plan_t h) {
  if (h->gset) return PLAN_OK;
  const size_t p = h->p;
  // the stage kernel reads the pinned staging area in place, once per
  // agent: for a few tens of KB a copy-engine transfer first costs more than
  // one coalesced pass over the link
  float2* staged = nullptr;
  unsigned long long* verdict = nullptr;
  unsigned long long* hk = reinterpret_cast<unsigned long long*>(h->h_res + 2);
  CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&staged), h->h_stage, 0));
  CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&verdict), hk, 0));
  unsigned long long* key = h->at<unsigned long long>(h->L.ekey);
  const int goals = h->vo ? 0 : 1;
  // one warp per 8 rows of a tile pair (8 warps a block), at most 1,024
  // blocks; enough threads for one agent-wall test each up to that
  const long long tasks = (long long)h->ntp * (1 + goals) * (TILE / EP_ROWS);
  const long long nwall = (long long)p * h->nw * (1 + goals);
  const int blocks = (int)std::min<long long>(std::max<long long>((tasks + 7) / 8, (nwall + 255) / 256), 1024);
  if (!h->ep_event) CK(cudaEventCreateWithFlags(&h->ep_event, cudaEventDisableTiming));
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  float2* shadow = h->at<float2>(h->L.eshadow);
  cudaError_t ce = launch_pdl(endpoint_stage_kernel, (unsigned)((p + 255) / 256), 256u, h->cap, h->dev(h->k),
                              (const float2*)staged, shadow, key);
  if (ce == cudaSuccess)
    ce = launch_pdl(endpoint_update_kernel, (unsigned)blocks, 256u, h->cap, h->dev(h->k), (const float2*)shadow,
                    goals, h->at<float2>(h->L.start), h->at<float2>(h->L.goal), key, verdict);
  cudaError_t e = cudaStreamEndCapture(h->cap, &g);
  if (e == cudaSuccess) e = ce;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gset, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->gset = nullptr;
    return fail(PLAN_ECUDA, "endpoint graph: %s", cudaGetErrorString(e));
  }
  return PLAN_OK;
}

// Enqueue a device-checked endpoint update (p <= kDeviceEndpointCheck):
// stage the endpoints and launch the graph; the verdict is pending until
// settled.
plan_status launch_endpoint_update(plan_t h, const float* start, const float* goal) {
  const size_t p = h->p;
  plan_status st = endpoint_graph(h);
  if (st != PLAN_OK) return st;
  std::memcpy(h->h_stage, start, p * 8);
  std::memcpy(h->h_stage + 2 * p, goal, p * 8);
  CK(cudaGraphLaunch(h->gset, h->stream));
  CK(cudaEventRecord(h->ep_event, h->stream));
  h->ep_start.assign(start, start + 2 * p);
  h->ep_goal.assign(goal, goal + 2 * p);
  h->ep_pending = true;
  h->adj_valid = false;
  return PLAN_OK;
}

// Read a pending endpoint verdict once its graph has run (the caller has
// synchronised, or this waits for the graph): keep the endpoints on the host
// if they passed, else report the violation (the device kept the previous
// endpoints).
plan_status settle_endpoints(plan_t h) {
  if (!h->ep_pending) return PLAN_OK;
  CK(cudaEventSynchronize(h->ep_event));
  h->ep_pending = false;
  const unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(h->h_res + 2);
  if (k == ~0ull) {
    h->h_start.swap(h->ep_start);
    h->h_goal.swap(h->ep_goal);
    return PLAN_OK;
  }
  const unsigned kind = (unsigned)(k >> 60), i = (unsigned)((k >> 30) & 0x3fffffffu),
                 j = (unsigned)(k & 0x3fffffffu);
  if (kind == 0) return fail(PLAN_EINVAL, "non-finite input (the start or goal of agent %u)", i);
  if (kind < 3)
    return fail(PLAN_EINFEASIBLE_INPUT, "%s positions of agents %u and %u overlap",
                kind == 2 ? "goal" : "start", i, j);
  return fail(PLAN_EINFEASIBLE_INPUT, "%s of agent %u is within its radius of wall %u",
              kind == 4 ? "goal" : "start", i, j);
}

}  // namespace

extern "C" {

plan_status plan_set_endpoints(plan_t h, const float* start, const float* goal) {
  if (!h || !start || !goal) return fail(PLAN_EINVAL, "null argument");
  const size_t p = h->p;
  plan_status st = settle_endpoints(h);  // an earlier asynchronous update's verdict
  if (st != PLAN_OK) return st;
  if (!h->h_stage || p > kDeviceEndpointCheck) {
    // the host grid check, then the copies (the device check rejects
    // non-finite coordinates itself)
    if (!finite_all(start, 2 * p) || !finite_all(goal, 2 * p)) return fail(PLAN_EINVAL, "non-finite input");
    st = check_endpoints(h->p, start, goal, h->h_radius.data(), h->nw, h->h_walls.data(), !h->vo,
                         &h->grid);
    if (st != PLAN_OK) return st;
    float2* d_start = h->at<float2>(h->L.start);
    float2* d_goal = h->at<float2>(h->L.goal);
    CK(cudaMemcpyAsync(d_start, start, p * 8, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(d_goal, goal, p * 8, cudaMemcpyHostToDevice, h->stream));
    endpoints_fix_kernel<<<1, 256, 0, h->stream>>>(h->dev(h->k), d_start, d_goal);
    CK(cudaGetLastError());
    // the caller's host buffers may be reused once this returns
    CK(cudaStreamSynchronize(h->stream));
    h->adj_valid = false;
    h->h_start.assign(start, start + 2 * p);
    h->h_goal.assign(goal, goal + 2 * p);
    return PLAN_OK;
  }
  // checked on the device: the whole update is enqueued before the one wait
  st = launch_endpoint_update(h, start, goal);
  if (st != PLAN_OK) return st;
  return settle_endpoints(h);
}

plan_status plan_set_endpoints_async(plan_t h, const float* start, const float* goal) {
  if (!h || !start || !goal) return fail(PLAN_EINVAL, "null argument");
  const size_t p = h->p;
  if (!h->h_stage || p > kDeviceEndpointCheck)
    return fail(PLAN_EUNSUPPORTED, "asynchronous endpoint updates need the device check (p <= %zu)",
                kDeviceEndpointCheck);
  // the previous update must have consumed the staging buffer, and its
  // verdict is read before this one can overwrite it
  plan_status st = settle_endpoints(h);
  if (st != PLAN_OK) return st;
  return launch_endpoint_update(h, start, goal);
}

plan_status plan_iterate(plan_t h, int k_iters, float* max_residual) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  if (k_iters < 0) return fail(PLAN_EINVAL, "k_iters must be >= 0");
  if (k_iters > 0) h->adj_valid = false;
  plan_status st = run_iterations(h, k_iters);
  if (st != PLAN_OK) return st;
  if (max_residual) {
    st = read_residual(h, max_residual);
    return st == PLAN_OK ? settle_endpoints(h) : st;
  }
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
  if (!on_device) {
    CK(cudaStreamSynchronize(h->stream));
    return settle_endpoints(h);
  }
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
  h->adj_valid = false;
  const size_t zbytes = (size_t)h->p * (h->eta + 1) * 8;
  CK(cudaMemcpyAsync(h->at<void>(h->L.z0), z, zbytes, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->at<void>(h->L.z1), z, zbytes, cudaMemcpyDeviceToDevice, h->stream));
  h->cur = 0;
  h->k = k;
  Dev P = h->dev(k);
  if (h->p > 1) import_coll_kernel<<<(unsigned)((h->slots + 255) / 256), 256, 0, h->stream>>>(P, u_coll);
  const int nseg = std::max(h->eta * h->p, h->nw * h->eta * h->p);
  import_seg_kernel<<<(nseg + 255) / 256, 256, 0, h->stream>>>(P, u_kin, u_wall);
  // velocity factors start from u = 0 (plan_import_velocity_state sets them)
  for (int v = 0; v < h->nv; ++v)
    import_vel_kernel<<<(h->eta * h->p + 255) / 256, 256, 0, h->stream>>>(P, v, nullptr);
  if (h->nw + h->nv) {
    const int words = (h->nw + h->nv) * h->eta * h->nt;
    import_wbits_kernel<<<(words * 32 + 255) / 256, 256, 0, h->stream>>>(P);
  }
  plan_status wst = derive_wnode(h);
  if (wst != PLAN_OK) return wst;
  CK(cudaMemsetAsync(h->at<void>(h->L.res), 0, 16, h->stream));
  CK(cudaMemsetAsync(h->at<void>(h->L.wcount), 0, 16, h->stream));
  CK(cudaMemsetAsync(h->at<void>(h->L.sched), 0, 16, h->stream));
  CK(cudaMemsetAsync(h->at<void>(h->L.stamps), 0xff, 2 * (size_t)h->eta * h->ntp * 4, h->stream));
  CK(clear_sums(h));
  CK(cudaMemsetAsync(h->at<void>(h->L.status), 0, 4, h->stream));
  fix_kernel<<<1, 256, 0, h->stream>>>(P, h->at<float2>(h->L.start), h->at<float2>(h->L.goal));
  CK(cudaGetLastError());
  return PLAN_OK;
}

plan_status plan_check(plan_t h, double* total_cost, double* min_pair_clearance,
                       double* min_wall_clearance, double* max_endpoint_error) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  Dev P = h->dev(h->k);
  double* out = h->at<double>(h->L.chk);
  // the local planner's graph: kinetic factor on segment 1, the rest on segment 0
  const int s_lo = h->vo ? 1 : 0;
  const int nseg = h->vo ? 1 : h->eta;
  check_cost_kernel<<<1, 256, 0, h->stream>>>(P, h->at<double>(h->L.ccost), h->at<float2>(h->L.start),
                                              h->at<float2>(h->L.goal), s_lo, h->eta, out);
  if (h->p > 1)
    check_pairs_kernel<<<(unsigned)(nseg * h->ntp), 256, 0, h->stream>>>(
        P, reinterpret_cast<unsigned long long*>(out + 1));
  if (h->nw) {
    const long long n = (long long)h->nw * nseg * h->p;
    check_walls_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, h->stream>>>(
        P, nseg, reinterpret_cast<unsigned long long*>(out + 2));
  }
  CK(cudaGetLastError());
  double v[4];
  CK(cudaMemcpyAsync(v, out, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (total_cost) *total_cost = v[0];
  if (min_pair_clearance) *min_pair_clearance = std::sqrt(v[1]);
  if (min_wall_clearance) *min_wall_clearance = std::sqrt(v[2]);
  if (max_endpoint_error) *max_endpoint_error = v[3];
  return settle_endpoints(h);
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
  return settle_endpoints(h);
}

plan_status plan_profile(plan_t h, int enable, float* ms, int* iterations) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  if (!h->cap) return fail(PLAN_EINVAL, "a batch member cannot be timed on its own");
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

}  // extern "C"

// ---------------------------------------------------------------------------
// Differentiation: K unrolled iterations, checkpoints, and the adjoint pass
// ---------------------------------------------------------------------------
namespace {

__global__ void record_kernel(Dev P, const float2* zk, float2* tz, float4* tukin, uint32_t* tfid,
                              float4* tucl, float4* tuch, unsigned* tcount, uint32_t* tsidx,
                              float4* tsu, unsigned* tscount) {
  pdl_begin();
  const unsigned cnt = *P.work_count;
  const unsigned nz = (unsigned)P.p * (P.eta + 1), nk = (unsigned)P.eta * P.p;
  const unsigned nseg = (unsigned)(P.nw + P.nv) * nk;
  const unsigned n = max(max(max(nz, nk), cnt), nseg);
  if (blockIdx.x == 0 && threadIdx.x == 0) *tcount = cnt;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    if (t < nz) tz[t] = zk[t];
    if (t < nk) tukin[t] = P.ukin[t];
    if (t < cnt) {
      const uint32_t f = P.work[t];
      tfid[t] = f;
      tucl[t] = P.ulo[f];
      tuch[t] = P.uhi[f];
    }
    if (t < nseg) {  // active walls and velocity limits, compacted (tscount zeroed before)
      const unsigned i = t % P.p, ws = t / P.p;
      if ((P.wbits[(size_t)ws * P.nt + i / TILE] >> (i % TILE)) & 1u) {
        const unsigned at = atomicAdd(tscount, 1u);
        tsidx[at] = t;
        tsu[at] = P.uwall[t];
      }
    }
  }
}

// Zeroes n 32-bit counters spaced stride bytes apart (the compaction counter
// of every tape slot of a segment, before its replay).
__global__ void zero_strided_kernel(char* base, size_t stride, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) *reinterpret_cast<unsigned*>(base + i * stride) = 0u;
}

// The adjoint passes run with programmatic dependent launch, like the
// forward ones: each waits (griddepcontrol.wait) for its predecessor's
// writes, but its CTAs are scheduled while the predecessor drains.
__global__ void __launch_bounds__(256) bw_scatter_kernel(AdjDev A) {
  pdl_begin();
  const unsigned n = (unsigned)(A.eta * A.p) + *A.count + *A.scount;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    bw_scatter_item(A, t);
}

__global__ void bw_node_kernel(AdjDev A) {
  pdl_begin();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < A.p * (A.eta + 1)) bw_node(A, t);
}

__global__ void __launch_bounds__(256) bw_factor_kernel(AdjDev A) {
  pdl_begin();
  const unsigned n = (unsigned)(A.eta * A.p) + *A.count + *A.scount;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    bw_factor_item(A, t);
}

__global__ void bw_init_kernel(int n, const float2* dz, double2* zb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) zb[t] = make_double2((double)dz[t].x, (double)dz[t].y);
}

// z^0 is the start at every break-point but the goal node (Section 4); then
// the FP32 outputs.  d_cost: dL/dC_{i,s} = norm dL/dc_{i,s}, summed over s
// when one C_i serves every segment.
__global__ void bw_final_kernel(AdjDev A, const double2* zb0, double norm, int per_segment,
                                float2* d_start, float2* d_goal, float* d_radius, float* d_cost) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.p) return;
  const int E1 = A.eta + 1;
  double2 gs = A.g_start[i];
  for (int s = 0; s < A.eta; ++s) { gs.x += zb0[(size_t)i * E1 + s].x; gs.y += zb0[(size_t)i * E1 + s].y; }
  const double2 zg = zb0[(size_t)i * E1 + A.eta];
  const double2 gg = make_double2(A.g_goal[i].x + zg.x, A.g_goal[i].y + zg.y);
  d_start[i] = mk((float)gs.x, (float)gs.y);
  d_goal[i] = mk((float)gg.x, (float)gg.y);
  d_radius[i] = (float)A.g_r[i];
  if (per_segment) {
    for (int s = 0; s < A.eta; ++s) d_cost[(size_t)i * A.eta + s] = (float)(norm * A.g_c[(size_t)i * A.eta + s]);
  } else {
    double c = 0.0;
    for (int s = 0; s < A.eta; ++s) c += A.g_c[(size_t)i * A.eta + s];
    d_cost[i] = (float)(norm * c);
  }
}

// Device state copied into a checkpoint: everything an iteration reads.
struct Region { size_t off, bytes; };

std::vector<Region> ck_regions(plan_t h) {
  const size_t zb = (size_t)h->p * (h->eta + 1) * 8, kin = (size_t)h->eta * h->p * 16;
  const size_t ng = (size_t)h->nw + h->nv;  // walls and velocity limits
  std::vector<Region> r = {
      {h->L.z0, zb}, {h->L.z1, zb}, {h->L.bits, (size_t)h->eta * h->ntp * TILE * 4},
      {h->L.ulo, h->slots * 16}, {h->L.uhi, h->slots * 16}, {h->L.xlo, h->slots * 16},
      {h->L.xhi, h->slots * 16}, {h->L.ukin, kin}, {h->L.xkin, kin}, {h->L.wcount, 16},
      {h->L.res, 16}, {h->L.status, 4}};
  if (ng) {
    r.push_back({h->L.uwall, ng * kin});
    r.push_back({h->L.xwall, ng * kin});
    r.push_back({h->L.wbits, ng * h->eta * h->nt * 4});
  }
  return r;
}

// Offsets inside the plan's differentiation block.
struct AdjLayout {
  size_t ck_bytes, ck0;
  int nck;
  size_t cap, slot_bytes, tape0;
  size_t t_z, t_ukin, t_count, t_fid, t_ucl, t_uch;  // within one tape slot
  size_t t_scount, t_sidx, t_su, scap;
  size_t ubk, ubl, ubh, stamp, ubs, sstamp, zbA, zbB, S, cnt, mbar, gs, gg, gr, gc;
  size_t total;
};

AdjLayout adj_layout(plan_t h, int K, int C) {
  AdjLayout A{};
  const size_t p = h->p, E1 = h->eta + 1, eta = h->eta;
  A.ck_bytes = 0;
  for (const Region& r : ck_regions(h)) A.ck_bytes += a256(r.bytes);
  A.nck = (K + C - 1) / C + 1;  // segment starts and the final state
  A.cap = std::max<size_t>(1, eta * (p * (p - 1) / 2));
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = a256(o + std::max<size_t>(bytes, 1)); return at; };
  A.t_z = take(p * E1 * 8);
  A.t_ukin = take(eta * p * 16);
  A.t_count = take(4);
  A.t_fid = take(A.cap * 4);
  A.t_ucl = take(A.cap * 16);
  A.t_uch = take(A.cap * 16);
  A.scap = std::max<size_t>(1, (size_t)(h->nw + h->nv) * eta * p);
  A.t_scount = take(4);
  A.t_sidx = take(A.scap * 4);
  A.t_su = take(A.scap * 16);
  A.slot_bytes = o;
  o = 0;
  A.ck0 = take(A.ck_bytes * A.nck);
  A.tape0 = take(A.slot_bytes * C);
  A.ubk = take(eta * p * 16);
  A.ubl = take(h->slots * 16);
  A.ubh = take(h->slots * 16);
  A.stamp = take(h->slots * 4);
  A.ubs = take(A.scap * 16);
  A.sstamp = take(A.scap * 4);
  A.zbA = take(p * E1 * 16);
  A.zbB = take(p * E1 * 16);
  A.S = take(p * E1 * 16);
  A.cnt = take(p * E1 * 4);
  A.mbar = take(p * E1 * 8);
  A.gs = take(p * 16);
  A.gg = take(p * 16);
  A.gr = take(p * 8);
  A.gc = take(p * eta * 8);
  A.total = o;
  return A;
}

plan_status snapshot(plan_t h, const AdjLayout& A, int idx, bool save) {
  char* ck = h->adj + A.ck0 + (size_t)idx * A.ck_bytes;
  for (const Region& r : ck_regions(h)) {
    char* ws = h->ws + r.off;
    CK(cudaMemcpyAsync(save ? ck : ws, save ? ws : ck, r.bytes, cudaMemcpyDeviceToDevice, h->stream));
    ck += a256(r.bytes);
  }
  if (!save) {
    // the pass-1 heavy-tile lists belong to the iteration order that ran, not
    // to the restored state: start over with none (results do not depend on it)
    CK(cudaMemsetAsync(h->at<void>(h->L.sched), 0, 16, h->stream));
    CK(cudaMemsetAsync(h->at<void>(h->L.stamps), 0xff, 2 * (size_t)h->eta * h->ntp * 4, h->stream));
  }
  return PLAN_OK;
}

AdjDev adj_dev(plan_t h, const AdjLayout& A, int slot, int k, char* zb_in, char* zb_out) {
  AdjDev D{};
  D.p = h->p; D.eta = h->eta; D.ntp = h->ntp; D.k = k;
  D.rho = h->cfg.rho0;
  D.alpha = (h->cfg.flags & PLAN_U_LITERAL) ? h->cfg.alpha / h->cfg.rho0 : h->cfg.alpha;
  D.tiles = h->at<int2>(h->L.tiles);
  D.radius = h->at<float>(h->L.radius);
  D.cost = h->at<float>(h->L.cost);
  D.nw = h->nw; D.nv = h->nv; D.vmin_mask = h->vmin_mask;
  D.vo = h->vo ? 1 : 0;
  D.walls = h->at<float4>(h->L.walls);
  D.vlim = h->at<float>(h->L.vlim);
  char* t = h->adj + A.tape0 + (size_t)slot * A.slot_bytes;
  D.z = reinterpret_cast<const float2*>(t + A.t_z);
  D.ukin = reinterpret_cast<const float4*>(t + A.t_ukin);
  D.count = reinterpret_cast<const unsigned*>(t + A.t_count);
  D.fid = reinterpret_cast<const uint32_t*>(t + A.t_fid);
  D.ucl = reinterpret_cast<const float4*>(t + A.t_ucl);
  D.uch = reinterpret_cast<const float4*>(t + A.t_uch);
  D.sidx = reinterpret_cast<const uint32_t*>(t + A.t_sidx);
  D.su = reinterpret_cast<const float4*>(t + A.t_su);
  D.scount = reinterpret_cast<const unsigned*>(t + A.t_scount);
  D.ubs = reinterpret_cast<float4*>(h->adj + A.ubs);
  D.sstamp = reinterpret_cast<int*>(h->adj + A.sstamp);
  D.ubk = reinterpret_cast<float4*>(h->adj + A.ubk);
  D.ubl = reinterpret_cast<float4*>(h->adj + A.ubl);
  D.ubh = reinterpret_cast<float4*>(h->adj + A.ubh);
  D.stamp = reinterpret_cast<int*>(h->adj + A.stamp);
  D.zb_in = reinterpret_cast<const double2*>(zb_in);
  D.zb_out = reinterpret_cast<double2*>(zb_out);
  D.S = reinterpret_cast<double2*>(h->adj + A.S);
  D.cnt = reinterpret_cast<unsigned*>(h->adj + A.cnt);
  D.mbar = reinterpret_cast<float2*>(h->adj + A.mbar);
  D.g_start = reinterpret_cast<double2*>(h->adj + A.gs);
  D.g_goal = reinterpret_cast<double2*>(h->adj + A.gg);
  D.g_r = reinterpret_cast<double*>(h->adj + A.gr);
  D.g_c = reinterpret_cast<double*>(h->adj + A.gc);
  return D;
}

plan_status adj_supported(plan_t h) {
  if (h->cfg.flags & (PLAN_ADMM | PLAN_U_KEEP))
    return fail(PLAN_EUNSUPPORTED, "the adjoint covers TWA with the reset rule only");
  if (h->cfg.warm_iters > 0) return fail(PLAN_EUNSUPPORTED, "the adjoint needs a constant rho0");
  if (h->noenergy)
    return fail(PLAN_EUNSUPPORTED, "the adjoint needs the kinetic factors (not the feasibility "
                                   "problem)");
  return PLAN_OK;
}

}  // namespace

extern "C" {

plan_status plan_set_velocity_limits(plan_t h, const float* vmax, const float* vmin) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  const bool has_max = (h->cfg.flags & PLAN_VMAX) != 0, has_min = (h->cfg.flags & PLAN_VMIN) != 0;
  if ((vmax && !has_max) || (vmin && !has_min))
    return fail(PLAN_EINVAL, "velocity limits need PLAN_VMAX / PLAN_VMIN at plan_create");
  const size_t n = (size_t)h->p * h->eta;
  if (vmax) {
    for (size_t t = 0; t < n; ++t)
      if (!(vmax[t] > 0.f)) return fail(PLAN_EINVAL, "vmax[%zu] must be positive (or +inf)", t);
  }
  if (vmin) {
    for (size_t t = 0; t < n; ++t)
      if (!(vmin[t] >= 0.f) || !std::isfinite(vmin[t])) return fail(PLAN_EINVAL, "vmin[%zu] must be finite and >= 0", t);
  }
  h->adj_valid = false;
  float* lim = h->at<float>(h->L.vlim);
  if (vmax) CK(cudaMemcpyAsync(lim, vmax, n * 4, cudaMemcpyHostToDevice, h->stream));
  if (vmin) CK(cudaMemcpyAsync(lim + (has_max ? n : 0), vmin, n * 4, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PLAN_OK;
}

plan_status plan_export_velocity_state(plan_t h, float* u_vmax, float* u_vmin, uint8_t* act_vmax,
                                       uint8_t* act_vmin) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  const bool has_max = (h->cfg.flags & PLAN_VMAX) != 0, has_min = (h->cfg.flags & PLAN_VMIN) != 0;
  if (((u_vmax || act_vmax) && !has_max) || ((u_vmin || act_vmin) && !has_min))
    return fail(PLAN_EINVAL, "the plan has no such velocity factors");
  Dev P = h->dev(h->k);
  const unsigned grid = (unsigned)((h->eta * h->p + 255) / 256);
  if (has_max && (u_vmax || act_vmax)) export_vel_kernel<<<grid, 256, 0, h->stream>>>(P, 0, u_vmax, act_vmax);
  if (has_min && (u_vmin || act_vmin))
    export_vel_kernel<<<grid, 256, 0, h->stream>>>(P, has_max ? 1 : 0, u_vmin, act_vmin);
  CK(cudaGetLastError());
  return PLAN_OK;
}

plan_status plan_import_velocity_state(plan_t h, const float* u_vmax, const float* u_vmin) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  const bool has_max = (h->cfg.flags & PLAN_VMAX) != 0, has_min = (h->cfg.flags & PLAN_VMIN) != 0;
  if ((u_vmax && !has_max) || (u_vmin && !has_min))
    return fail(PLAN_EINVAL, "the plan has no such velocity factors");
  h->adj_valid = false;
  Dev P = h->dev(h->k);
  const unsigned grid = (unsigned)((h->eta * h->p + 255) / 256);
  if (has_max) import_vel_kernel<<<grid, 256, 0, h->stream>>>(P, 0, u_vmax);
  if (has_min) import_vel_kernel<<<grid, 256, 0, h->stream>>>(P, has_max ? 1 : 0, u_vmin);
  const int words = (h->nw + h->nv) * h->eta * h->nt;
  if (words) import_wbits_kernel<<<(words * 32 + 255) / 256, 256, 0, h->stream>>>(P);
  CK(cudaGetLastError());
  return derive_wnode(h);
}

plan_status plan_export_back_weights(plan_t h, uint8_t* classes) {
  if (!h || !classes) return fail(PLAN_EINVAL, "null argument");
  Dev P = h->dev(h->k);
  const int nodes = h->p * (h->eta + 1);
  back_weights_kernel<<<(nodes + 255) / 256, 256, 0, h->stream>>>(P, classes, nullptr);
  CK(cudaGetLastError());
  return PLAN_OK;
}

plan_status plan_import_back_weights(plan_t h, const uint8_t* classes) {
  if (!h || !classes) return fail(PLAN_EINVAL, "null argument");
  if (!h->noenergy) return fail(PLAN_EINVAL, "back weights are rho0 inside while the kinetic factors run");
  Dev P = h->dev(h->k);
  const int nodes = h->p * (h->eta + 1);
  back_weights_kernel<<<(nodes + 255) / 256, 256, 0, h->stream>>>(P, nullptr, classes);
  CK(cudaGetLastError());
  return PLAN_OK;
}

plan_status plan_get_endpoints(plan_t h, float* start, float* goal) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  if (start) CK(cudaMemcpyAsync(start, h->at<void>(h->L.start), (size_t)h->p * 8, cudaMemcpyDeviceToHost, h->stream));
  if (goal) CK(cudaMemcpyAsync(goal, h->at<void>(h->L.goal), (size_t)h->p * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return settle_endpoints(h);
}

plan_status plan_vo_epoch(plan_t h, const float* dest, float step, float advance, int* iters,
                          float* residual, float* max_dist) {
  if (!h || !dest) return fail(PLAN_EINVAL, "null argument");
  if (!h->vo) return fail(PLAN_EINVAL, "plan_vo_epoch needs a PLAN_VO plan");
  if (!(step > 0.f) || !(advance > 0.f && advance <= 1.f))
    return fail(PLAN_EINVAL, "step must be > 0 and advance in (0, 1]");
  const unsigned g = (unsigned)((h->p + 255) / 256);
  float2* start = h->at<float2>(h->L.start);
  float2* goal = h->at<float2>(h->L.goal);
  vo_target_kernel<<<g, 256, 0, h->stream>>>(h->p, start, reinterpret_cast<const float2*>(dest), step, goal);
  CK(cudaGetLastError());
  plan_status st = plan_reset(h);  // the initial state of Section 4 for this epoch
  if (st != PLAN_OK) return st;
  int it = 0;
  float res = INFINITY;
  const plan_status sst = plan_solve(h, &it, &res);
  if (sst != PLAN_OK && sst != PLAN_ENOTCONV) return sst;
  unsigned* md = h->at<unsigned>(h->L.count);
  CK(cudaMemsetAsync(md, 0, 4, h->stream));
  const float2* z = h->cur ? h->at<float2>(h->L.z1) : h->at<float2>(h->L.z0);
  vo_advance_kernel<<<g, 256, 0, h->stream>>>(h->p, h->eta, z, reinterpret_cast<const float2*>(dest),
                                              advance, start, md);
  CK(cudaGetLastError());
  unsigned mdh = 0;
  CK(cudaMemcpyAsync(h->h_start.data(), start, (size_t)h->p * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_goal.data(), goal, (size_t)h->p * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_res, md, 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  mdh = *h->h_res;
  if (iters) *iters = it;
  if (residual) *residual = res;
  if (max_dist) std::memcpy(max_dist, &mdh, 4);
  h->adj_valid = false;
  return sst;
}

plan_status plan_set_energy(plan_t h, int on) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  if (h->cfg.flags & PLAN_ADMM) return fail(PLAN_EUNSUPPORTED, "standard-ADMM mode keeps the kinetic factors");
  const bool off = (on == 0);
  if (off == h->noenergy) return PLAN_OK;
  h->adj_valid = false;
  // the captured iterations hold the old mode
  for (int q = 0; q < 4; ++q)
    if (h->gexec[q]) { cudaGraphExecDestroy(h->gexec[q]); h->gexec[q] = nullptr; }
  for (int q = 0; q < 4; ++q)
    if (h->gexec8[q]) { cudaGraphExecDestroy(h->gexec8[q]); h->gexec8[q] = nullptr; }
  for (int q = 0; q < 4; ++q)
    if (h->gexec64[q]) { cudaGraphExecDestroy(h->gexec64[q]); h->gexec64[q] = nullptr; }
  h->noenergy = off;
  Dev P = h->dev(h->k);
  if (off) {
    // every node had the kinetic factors' rho0 so far
    const int nodes = h->p * (h->eta + 1);
    wnode_clear_kernel<<<(nodes + 255) / 256, 256, 0, h->stream>>>(P, 1);
  } else {
    kinetic_restart_kernel<<<(h->eta * h->p + 255) / 256, 256, 0, h->stream>>>(P);
  }
  CK(cudaGetLastError());
  return PLAN_OK;
}

plan_status plan_set_params(plan_t h, const float* radius, const float* cost_w) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  {  // new radii are checked against the endpoints on the host: settle them first
    plan_status st = settle_endpoints(h);
    if (st != PLAN_OK) return st;
  }
  const size_t p = h->p, eta = h->eta;
  const size_t ncost = (h->cfg.flags & PLAN_COST_PER_SEGMENT) ? p * eta : p;
  if (radius) {
    if (!finite_all(radius, p)) return fail(PLAN_EINVAL, "non-finite radius");
    for (size_t i = 0; i < p; ++i)
      if (!(radius[i] > 0.f)) return fail(PLAN_EINVAL, "radius[%zu] must be positive", i);
    plan_status st = check_endpoints(h->p, h->h_start.data(), h->h_goal.data(), radius, h->nw,
                                     h->h_walls.data(), !h->vo);
    if (st != PLAN_OK) return st;
  }
  std::vector<float> cost;
  std::vector<double> ccost;
  if (cost_w) {
    if (!finite_all(cost_w, ncost)) return fail(PLAN_EINVAL, "non-finite cost_w");
    for (size_t i = 0; i < ncost; ++i)
      if (cost_w[i] < 0.f) return fail(PLAN_EINVAL, "cost_w[%zu] must be >= 0", i);
    const double norm = (h->cfg.flags & (PLAN_COST_UNNORM | PLAN_VO)) ? 1.0 : 1.0 / ((double)p * eta);
    cost.resize(p * eta);
    ccost.resize(p * eta);
    for (size_t i = 0; i < p; ++i)
      for (size_t s = 0; s < eta; ++s) {
        ccost[i * eta + s] = norm * ((h->cfg.flags & PLAN_COST_PER_SEGMENT) ? cost_w[i * eta + s] : cost_w[i]);
        cost[i * eta + s] = (float)ccost[i * eta + s];
      }
  }
  h->adj_valid = false;
  if (radius) {
    h->h_radius.assign(radius, radius + p);
    CK(cudaMemcpyAsync(h->at<void>(h->L.radius), radius, p * 4, cudaMemcpyHostToDevice, h->stream));
  }
  if (cost_w) {
    CK(cudaMemcpyAsync(h->at<void>(h->L.cost), cost.data(), p * eta * 4, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->at<void>(h->L.ccost), ccost.data(), p * eta * 8, cudaMemcpyHostToDevice, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return PLAN_OK;
}

plan_status plan_unroll(plan_t h, int K, int checkpoint_every) {
  if (!h) return fail(PLAN_EINVAL, "null plan");
  if (K < 0 || checkpoint_every < 0) return fail(PLAN_EINVAL, "K and checkpoint_every must be >= 0");
  plan_status st = adj_supported(h);
  if (st != PLAN_OK) return st;
  int C = checkpoint_every ? checkpoint_every : (int)std::ceil(std::sqrt((double)std::max(K, 1)));
  C = std::max(1, std::min(C, std::max(K, 1)));
  const AdjLayout A = adj_layout(h, K, C);
  if (h->adj_bytes < A.total) {
    if (h->adj) {
      CK(cudaStreamSynchronize(h->stream));
      cudaFree(h->adj);
      h->adj = nullptr;
      h->adj_bytes = 0;
    }
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, A.total);
    if (e != cudaSuccess)
      return fail(PLAN_ENOMEM, "cudaMalloc(%zu) for the adjoint failed: %s", A.total, cudaGetErrorString(e));
    h->adj = static_cast<char*>(mem);
    h->adj_bytes = A.total;
  }
  st = plan_reset(h);
  if (st != PLAN_OK) return st;
  h->ck_cur.assign(A.nck, 0);
  for (int k = 0; k < K; k += C) {
    h->ck_cur[k / C] = h->cur;
    if ((st = snapshot(h, A, k / C, true)) != PLAN_OK) return st;
    if ((st = run_iterations(h, std::min(C, K - k))) != PLAN_OK) return st;
  }
  h->ck_cur[A.nck - 1] = h->cur;
  if ((st = snapshot(h, A, A.nck - 1, true)) != PLAN_OK) return st;
  h->adj_K = K;
  h->adj_C = C;
  h->adj_valid = true;
  return PLAN_OK;
}

plan_status plan_backward(plan_t h, int K, const float* dL_dz, float* d_start, float* d_goal,
                          float* d_radius, float* d_cost_w) {
  if (!h || !dL_dz || !d_start || !d_goal || !d_radius || !d_cost_w)
    return fail(PLAN_EINVAL, "null argument");
  plan_status st = adj_supported(h);
  if (st != PLAN_OK) return st;
  if (!h->adj_valid || K != h->adj_K)
    return fail(PLAN_EINVAL, "plan_backward(K = %d) needs the state left by plan_unroll(K)", K);
  if ((st = ensure_prox_grid(h)) != PLAN_OK) return st;
  const int C = h->adj_C;
  const AdjLayout A = adj_layout(h, K, C);
  const size_t p = h->p, E1 = h->eta + 1, nodes = p * E1;
  // adjoint state: u adjoints 0, no stamps, gradients 0, zbar = dL/dz^K
  CK(cudaMemsetAsync(h->adj + A.ubk, 0, (size_t)h->eta * p * 16, h->stream));
  CK(cudaMemsetAsync(h->adj + A.stamp, 0xff, h->slots * 4, h->stream));
  CK(cudaMemsetAsync(h->adj + A.sstamp, 0xff, A.scap * 4, h->stream));
  CK(cudaMemsetAsync(h->adj + A.S, 0, nodes * 16, h->stream));
  CK(cudaMemsetAsync(h->adj + A.cnt, 0, nodes * 4, h->stream));
  CK(cudaMemsetAsync(h->adj + A.gs, 0, A.gc + p * h->eta * 8 - A.gs, h->stream));
  bw_init_kernel<<<(unsigned)((nodes + 255) / 256), 256, 0, h->stream>>>(
      (int)nodes, reinterpret_cast<const float2*>(dL_dz), reinterpret_cast<double2*>(h->adj + A.zbA));
  CK(cudaGetLastError());
  char* zb_in = h->adj + A.zbA;
  char* zb_out = h->adj + A.zbB;
  const int nseg = A.nck - 1;
  const unsigned node_grid = (unsigned)((nodes + 255) / 256);
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int c0 = seg * C, c1 = std::min(K, c0 + C);
    // recompute the segment from its checkpoint, recording each iteration
    if ((st = snapshot(h, A, seg, false)) != PLAN_OK) return st;
    h->k = c0;
    h->cur = h->ck_cur[seg];
    zero_strided_kernel<<<1, 64, 0, h->stream>>>(h->adj + A.tape0 + A.t_scount, A.slot_bytes, c1 - c0);
    CK(cudaGetLastError());
    for (int k = c0; k < c1; ++k) {
      const float2* zk = h->cur ? h->at<float2>(h->L.z1) : h->at<float2>(h->L.z0);
      if ((st = run_iteration(h)) != PLAN_OK) return st;
      char* t = h->adj + A.tape0 + (size_t)(k - c0) * A.slot_bytes;
      CK(launch_pdl(record_kernel, (unsigned)h->prox_grid, 256u, h->stream, h->dev(k), zk,
                    reinterpret_cast<float2*>(t + A.t_z), reinterpret_cast<float4*>(t + A.t_ukin),
                    reinterpret_cast<uint32_t*>(t + A.t_fid), reinterpret_cast<float4*>(t + A.t_ucl),
                    reinterpret_cast<float4*>(t + A.t_uch), reinterpret_cast<unsigned*>(t + A.t_count),
                    reinterpret_cast<uint32_t*>(t + A.t_sidx), reinterpret_cast<float4*>(t + A.t_su),
                    reinterpret_cast<unsigned*>(t + A.t_scount)));
    }
    // the adjoint steps of the segment, last iteration first
    for (int k = c1 - 1; k >= c0; --k) {
      const AdjDev D = adj_dev(h, A, k - c0, k, zb_in, zb_out);
      CK(launch_pdl(bw_scatter_kernel, (unsigned)h->prox_grid, 256u, h->stream, D));
      CK(launch_pdl(bw_node_kernel, node_grid, 256u, h->stream, D));
      CK(launch_pdl(bw_factor_kernel, (unsigned)h->prox_grid, 256u, h->stream, D));
      CK(cudaGetLastError());
      std::swap(zb_in, zb_out);
    }
  }
  const AdjDev D = adj_dev(h, A, 0, 0, zb_in, zb_out);
  const double norm = (h->cfg.flags & (PLAN_COST_UNNORM | PLAN_VO)) ? 1.0 : 1.0 / ((double)p * h->eta);
  bw_final_kernel<<<(unsigned)((p + 127) / 128), 128, 0, h->stream>>>(
      D, reinterpret_cast<const double2*>(zb_in), norm, (h->cfg.flags & PLAN_COST_PER_SEGMENT) ? 1 : 0,
      reinterpret_cast<float2*>(d_start), reinterpret_cast<float2*>(d_goal), d_radius, d_cost_w);
  CK(cudaGetLastError());
  // leave the plan at iteration K, as plan_unroll did
  if ((st = snapshot(h, A, nseg, false)) != PLAN_OK) return st;
  h->k = K;
  h->cur = h->ck_cur[nseg];
  return PLAN_OK;
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

// A message out of the fixed-point range (status bit 1) was left out of the
// consensus sums: the plan path reports that as a NaN residual
// (PLAN_ENUMERIC); here every entry of z_out becomes NaN instead, so that a
// caller without a residual still sees it.
__global__ void static_poison_kernel(const unsigned* status, float* z_out, int n) {
  if ((*status & 2u) == 0u) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    z_out[t] = __int_as_float(0x7fc00000);
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
  if (!(cfg->rho0 > 0.f) || !std::isfinite(cfg->rho0) || !(cfg->alpha > 0.f) || !std::isfinite(cfg->alpha))
    return fail(PLAN_EINVAL, "rho0 and alpha must be positive");
  if (cfg->warm_iters < 0 || (cfg->warm_iters > 0 && (!(cfg->warm_rho > 0.f) || !std::isfinite(cfg->warm_rho))))
    return fail(PLAN_EINVAL, "warm_rho must be positive when warm_iters > 0");
  if (k < 0) return fail(PLAN_EINVAL, "k must be >= 0");
  if (cfg->flags & (PLAN_NO_ENERGY | PLAN_VMAX | PLAN_VMIN | PLAN_VO))
    return fail(PLAN_EUNSUPPORTED, "plan_iterate_static runs the energy problem without velocity factors");
  const unsigned known = PLAN_U_KEEP | PLAN_COST_UNNORM | PLAN_COST_PER_SEGMENT |
                         PLAN_DENSE_STATE | PLAN_ADMM | PLAN_U_LITERAL;
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
  if (st == PLAN_OK) {
    const int nz = 2 * h.p * (h.eta + 1);
    static_poison_kernel<<<(nz + 255) / 256, 256, 0, h.stream>>>(h.at<unsigned>(L.status), z_out, nz);
    CK(cudaGetLastError());
  }
  return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many independent problems advanced together, one launch per pass
// ---------------------------------------------------------------------------
// Each member is an ordinary plan (its own workspace slice, no streams of its
// own).  Every pass of an iteration is a single launch over the union of all
// members' blocks: a block finds its member by binary search over a prefix
// table of block counts and runs the same per-block code as a single plan,
// on the member's descriptor copied into shared memory.  All members advance
// in lockstep, so the descriptors only depend on the iteration's parity; a
// member that has converged is frozen (its passes do nothing and its z is
// carried over unchanged).  Iterations are replayed from CUDA graphs, and
// three launch-shape knobs are chosen by timing (plan_batch_autotune).

namespace {

__device__ __forceinline__ int find_member(const int* pre, int n, int x) {
  int lo = 0, hi = n - 1;  // largest b with pre[b] <= x (pre is non-decreasing)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <bool DENSE, int TROWS>
__global__ void __launch_bounds__(32 * (TILE / TROWS)) batch_test_kernel(const Dev* tab, const int* pre,
                                                                          int n, const uint8_t* frozen) {
  __shared__ Dev sP;
  __shared__ int sb, sblk;
  if (threadIdx.x == 0) {
    const int b = find_member(pre, n, blockIdx.x);
    sb = b;
    sblk = blockIdx.x - pre[b];
    sP = tab[b];
  }
  __syncthreads();
  if (frozen[sb]) return;
  test_block<DENSE, TROWS>(sP, sblk);
}

// Gated state, one warp per tile (lane = row agent): each warp finds its own
// member, since the 4 tiles of a CTA may belong to different members.
__global__ void __launch_bounds__(32 * TILES_PER_CTA) batch_test_rows_kernel(const Dev* tab, const int* pre,
                                                                         int n, int ntiles,
                                                                         const uint8_t* frozen) {
  __shared__ Dev sP[TILES_PER_CTA];
  __shared__ float4 col[TILES_PER_CTA][72];
  __shared__ uint32_t nws[TILES_PER_CTA][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * TILES_PER_CTA + warp;
  if (t >= ntiles) return;  // warp-uniform
  const int b = find_member(pre, n, t);
  if (frozen[b]) return;
  // the member's descriptor into this warp's shared slot
  const uint32_t* src = reinterpret_cast<const uint32_t*>(tab + b);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sP[warp]);
  for (int w = lane; w < (int)(sizeof(Dev) / 4); w += 32) dst[w] = src[w];
  __syncwarp();
  const int blk = t - pre[b];
  if (blk == 0 && lane == 0) *sP[warp].res_cur = 0u;
  test_tile_rows(sP[warp], blk, col[warp], nws[warp]);
}

__global__ void batch_segment_kernel(const Dev* tab, const int* pre, int n, const uint8_t* frozen) {
  __shared__ Dev sP;
  __shared__ int sb, sblk;
  if (threadIdx.x == 0) {
    const int b = find_member(pre, n, blockIdx.x);
    sb = b;
    sblk = blockIdx.x - pre[b];
    sP = tab[b];
  }
  __syncthreads();
  if (frozen[sb]) return;
  segment_block<false>(sP, sblk);
}

// Exclusive prefix of the members' worklist lengths (frozen members: 0).
__global__ void batch_scan_kernel(const Dev* tab, int n, const uint8_t* frozen, int* pre_work) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  int sum = 0;
  for (int b = t * per; b < min(n, (t + 1) * per); ++b) sum += frozen[b] ? 0 : (int)*tab[b].work_count;
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int q = 0; q < (int)blockDim.x; ++q) { const int v = part[q]; part[q] = acc; acc += v; }
    pre_work[n] = acc;
  }
  __syncthreads();
  int acc = part[t];
  for (int b = t * per; b < min(n, (t + 1) * per); ++b) {
    pre_work[b] = acc;
    acc += frozen[b] ? 0 : (int)*tab[b].work_count;
  }
}

__global__ void __launch_bounds__(256) batch_prox_kernel(const Dev* tab, const int* pre_work, int n) {
  const unsigned long long total = (unsigned long long)pre_work[n];
  unsigned long long stride;
  for (unsigned long long t = dealt_first(stride); t < total; t += stride) {
    const int b = find_member(pre_work, n, (int)t);
    const Dev& P = tab[b];
    prox_item(P, P.work[(int)t - pre_work[b]]);
  }
}

// One thread per free break-point; each member's range is padded to whole
// warps (and at least one warp, which also clears the member's next worklist
// counter), so a warp never spans two members.
__global__ void batch_consensus_kernel(const Dev* tab, const int* pre, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= pre[n]) return;  // whole warps past the end
  const int b = find_member(pre, n, t);
  const Dev& P = tab[b];
  const int tl = t - pre[b];
  if (tl == 0) *P.work_count_next = 0u;
  float dz = 0.f;
  bool bad = false;
  if (tl < (P.eta - 1) * P.p) consensus_node(P, tl, dz, bad);
  consensus_reduce(P, dz, bad);
}

// The residual slot of each member's last iteration, gathered contiguously.
__global__ void batch_gather_res(const Dev* tab, int n, float* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) out[b] = __uint_as_float(*tab[b].res_prev);
}

}  // namespace

struct plan_batch_s {
  int n = 0;
  std::vector<plan_t> m;
  cudaStream_t stream = nullptr, cap = nullptr;
  char* ws = nullptr;
  bool own_ws = false;
  size_t total = 0;
  int k = 0;
  bool dense = false;
  // device tables (in the workspace tail)
  Dev* tab[2] = {nullptr, nullptr};
  int *pre_test = nullptr, *pre_seg = nullptr, *pre_node = nullptr, *pre_work = nullptr;
  uint8_t* frozen = nullptr;
  float* res = nullptr;
  int ntest = 0, nseg = 0, nnode = 0;
  std::vector<uint8_t> h_frozen;
  std::vector<int> conv_iter;
  int warm = 0;  // largest warm-up length among members
  // launch-shape knobs: rows per warp of the test pass, prox CTAs per SM, graph length
  int trows = 8, prox_mult = 2, glen = 8;
  int prox_grid = 0;
  cudaGraphExec_t gexec = nullptr;
  int gexec_trows = 0, gexec_mult = 0, gexec_len = 0;
};

namespace {

size_t batch_tables_bytes(int n) {
  return a256(2 * (size_t)n * sizeof(Dev)) + 4 * a256(((size_t)n + 1) * 4) + a256(n) + a256((size_t)n * 4);
}

plan_status batch_tables(plan_batch_s* B) {
  // descriptors of both parities; members advance together, so their z buffer
  // is the iteration's parity (no flip for eta = 1)
  for (int par = 0; par < 2; ++par) {
    std::vector<Dev> d(B->n);
    for (int b = 0; b < B->n; ++b) {
      plan_t h = B->m[b];
      const int kk = (B->k & ~1) + par;
      h->k = kk;
      h->cur = (h->eta > 1) ? (kk & 1) : 0;
      d[b] = h->dev(kk);
      d[b].hcap = 0;  // the batched test pass keeps its own order
      // the table serves every later iteration of this parity, so the
      // previous iteration's residual slot is always the other one
      d[b].res_prev = h->at<unsigned>(h->L.res) + ((kk + 1) & 1);
    }
    CK(cudaMemcpyAsync(B->tab[par], d.data(), d.size() * sizeof(Dev), cudaMemcpyHostToDevice, B->stream));
  }
  for (int b = 0; b < B->n; ++b) {  // restore the members' own counters
    plan_t h = B->m[b];
    h->k = B->k;
    h->cur = (h->eta > 1) ? (B->k & 1) : 0;
  }
  CK(cudaStreamSynchronize(B->stream));
  return PLAN_OK;
}

template <int TROWS>
void launch_batch_test(plan_batch_s* B, const Dev* tab, cudaStream_t s) {
  constexpr int threads = 32 * (TILE / TROWS);
  if (B->dense) batch_test_kernel<true, TROWS><<<B->ntest, threads, 0, s>>>(tab, B->pre_test, B->n, B->frozen);
  else batch_test_kernel<false, TROWS><<<B->ntest, threads, 0, s>>>(tab, B->pre_test, B->n, B->frozen);
}

plan_status enqueue_batch_iteration(plan_batch_s* B, int parity, cudaStream_t s) {
  const Dev* tab = B->tab[parity];
  if (B->trows == 32 && !B->dense)
    batch_test_rows_kernel<<<(B->ntest + TILES_PER_CTA - 1) / TILES_PER_CTA, 32 * TILES_PER_CTA, 0, s>>>(
        tab, B->pre_test, B->n, B->ntest, B->frozen);
  else if (B->trows == 4) launch_batch_test<4>(B, tab, s);
  else if (B->trows == 16) launch_batch_test<16>(B, tab, s);
  else launch_batch_test<8>(B, tab, s);
  batch_segment_kernel<<<B->nseg, THREADS, 0, s>>>(tab, B->pre_seg, B->n, B->frozen);
  batch_scan_kernel<<<1, 1024, 0, s>>>(tab, B->n, B->frozen, B->pre_work);
  batch_prox_kernel<<<B->prox_grid * B->prox_mult, 256, 0, s>>>(tab, B->pre_work, B->n);
  batch_consensus_kernel<<<(B->nnode + 255) / 256, 256, 0, s>>>(tab, B->pre_node, B->n);
  CK(cudaGetLastError());
  return PLAN_OK;
}

void batch_advance(plan_batch_s* B, int iters) {
  B->k += iters;
  for (plan_t h : B->m) {
    h->k = B->k;
    h->cur = (h->eta > 1) ? (B->k & 1) : 0;
  }
}

// iters iterations: graphs of glen (even) iterations while past every
// member's rho warm-up, direct launches otherwise.
plan_status batch_run(plan_batch_s* B, int iters) {
  while (iters > 0) {
    const bool graphable = B->k >= B->warm && (B->k & 1) == 0 && iters >= B->glen;
    if (graphable) {
      if (!B->gexec || B->gexec_trows != B->trows || B->gexec_mult != B->prox_mult ||
          B->gexec_len != B->glen) {
        if (B->gexec) { cudaGraphExecDestroy(B->gexec); B->gexec = nullptr; }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
        plan_status st = PLAN_OK;
        for (int q = 0; q < B->glen && st == PLAN_OK; ++q) st = enqueue_batch_iteration(B, q & 1, B->cap);
        cudaError_t e = cudaStreamEndCapture(B->cap, &g);
        if (st != PLAN_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return fail(PLAN_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&B->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(PLAN_ECUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e));
        B->gexec_trows = B->trows; B->gexec_mult = B->prox_mult; B->gexec_len = B->glen;
      }
      CK(cudaGraphLaunch(B->gexec, B->stream));
      batch_advance(B, B->glen);
      iters -= B->glen;
    } else {
      if (B->k < B->warm) {  // rho changes with k during the warm-up
        plan_status st = batch_tables(B);
        if (st != PLAN_OK) return st;
      }
      plan_status st = enqueue_batch_iteration(B, B->k & 1, B->stream);
      if (st != PLAN_OK) return st;
      batch_advance(B, 1);
      iters -= 1;
    }
  }
  return PLAN_OK;
}

}  // namespace

extern "C" {

plan_status plan_batch_workspace_size(int n, const plan_config* cfgs, size_t* bytes) {
  if (n < 1 || !cfgs || !bytes) return fail(PLAN_EINVAL, "null argument or n < 1");
  size_t tot = 0;
  for (int b = 0; b < n; ++b) {
    if (!sizes_ok(&cfgs[b])) return fail(PLAN_EINVAL, "member %d: p, eta or n_walls out of range", b);
    tot += a256(layout_for(&cfgs[b]).total);
  }
  *bytes = tot + batch_tables_bytes(n);
  return PLAN_OK;
}

plan_status plan_batch_create(int n, const plan_config* cfgs, const float* const* start,
                              const float* const* goal, const float* const* radius,
                              const float* const* cost_w, const float* const* walls,
                              void* workspace, size_t workspace_bytes, void* cuda_stream,
                              plan_batch_t* out) {
  if (n < 1 || !cfgs || !start || !goal || !radius || !cost_w || !out)
    return fail(PLAN_EINVAL, "null argument or n < 1");
  *out = nullptr;
  const unsigned modes = PLAN_DENSE_STATE | PLAN_U_KEEP | PLAN_ADMM;
  for (int b = 0; b < n; ++b)
    if (cfgs[b].flags & (PLAN_NO_ENERGY | PLAN_VMAX | PLAN_VMIN | PLAN_VO))
      return fail(PLAN_EUNSUPPORTED, "batch members run the energy problem without velocity factors");
  for (int b = 1; b < n; ++b)
    if ((cfgs[b].flags & modes) != (cfgs[0].flags & modes))
      return fail(PLAN_EINVAL, "batch members must share the state-mode flags");
  size_t need = 0;
  plan_status st = plan_batch_workspace_size(n, cfgs, &need);
  if (st != PLAN_OK) return st;
  plan_batch_s* B = new plan_batch_s();
  B->n = n;
  B->stream = (cudaStream_t)cuda_stream;
  B->dense = (cfgs[0].flags & modes) != 0;
  if (workspace) {
    if (workspace_bytes < need) { delete B; return fail(PLAN_ENOMEM, "workspace of %zu bytes, %zu needed", workspace_bytes, need); }
    if (reinterpret_cast<uintptr_t>(workspace) & 255) { delete B; return fail(PLAN_EINVAL, "workspace must be 256-byte aligned"); }
    B->ws = static_cast<char*>(workspace);
  } else {
    void* mem = nullptr;
    if (cudaMalloc(&mem, need) != cudaSuccess) { delete B; return fail(PLAN_ENOMEM, "cudaMalloc(%zu) failed", need); }
    B->ws = static_cast<char*>(mem);
    B->own_ws = true;
  }
  B->total = need;
  size_t off = 0;
  for (int b = 0; b < n; ++b) {
    const size_t sz = a256(layout_for(&cfgs[b]).total);
    plan_t h = nullptr;
    st = create_plan(&cfgs[b], start[b], goal[b], radius[b], cost_w[b], walls ? walls[b] : nullptr,
                     B->ws + off, sz, cuda_stream, true, &h);
    if (st != PLAN_OK) {
      plan_batch_destroy(B);
      char msg[600];
      snprintf(msg, sizeof msg, "member %d: %s", b, g_err.c_str());
      return fail(st, "%s", msg);
    }
    B->m.push_back(h);
    B->warm = std::max(B->warm, h->graph_from());
    off += sz;
  }
  char* t = B->ws + off;
  B->tab[0] = reinterpret_cast<Dev*>(t);
  B->tab[1] = B->tab[0] + n;
  t += a256(2 * (size_t)n * sizeof(Dev));
  B->pre_test = reinterpret_cast<int*>(t); t += a256(((size_t)n + 1) * 4);
  B->pre_seg = reinterpret_cast<int*>(t); t += a256(((size_t)n + 1) * 4);
  B->pre_node = reinterpret_cast<int*>(t); t += a256(((size_t)n + 1) * 4);
  B->pre_work = reinterpret_cast<int*>(t); t += a256(((size_t)n + 1) * 4);
  B->frozen = reinterpret_cast<uint8_t*>(t); t += a256(n);
  B->res = reinterpret_cast<float*>(t);
  std::vector<int> pt(n + 1, 0), ps(n + 1, 0), pn(n + 1, 0);
  for (int b = 0; b < n; ++b) {
    plan_t h = B->m[b];
    pt[b + 1] = pt[b] + h->eta * h->ntp;
    ps[b + 1] = ps[b] + h->eta * h->nt;
    const int nfree = (h->eta - 1) * h->p;
    pn[b + 1] = pn[b] + std::max(32, (nfree + 31) / 32 * 32);
  }
  B->ntest = pt[n]; B->nseg = ps[n]; B->nnode = pn[n];
  B->h_frozen.assign(n, 0);
  B->conv_iter.assign(n, -1);
  cudaError_t e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->pre_test, pt.data(), (n + 1) * 4, cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->pre_seg, ps.data(), (n + 1) * 4, cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->pre_node, pn.data(), (n + 1) * 4, cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->frozen, B->h_frozen.data(), n, cudaMemcpyHostToDevice, B->stream);
  if (e != cudaSuccess) { plan_batch_destroy(B); return fail(PLAN_ECUDA, "batch setup failed: %s", cudaGetErrorString(e)); }
  st = ensure_prox_grid(B->m[0]);
  if (st == PLAN_OK) { B->prox_grid = std::max(1, B->m[0]->prox_grid / 4); st = batch_tables(B); }
  if (st != PLAN_OK) { plan_batch_destroy(B); return st; }
  *out = B;
  return PLAN_OK;
}

plan_status plan_batch_import_state(plan_batch_t B, int member, const float* z, const float* u_coll,
                                    const float* u_kin, const float* u_wall) {
  if (!B || member < 0 || member >= B->n) return fail(PLAN_EINVAL, "null batch or member out of range");
  plan_t h = B->m[member];
  plan_status st = plan_import_state(h, z, u_coll, u_kin, u_wall, B->k);
  if (st != PLAN_OK) return st;
  // the member follows the batch's iteration: its z buffer is the parity's
  h->k = B->k;
  h->cur = (h->eta > 1) ? (B->k & 1) : 0;
  CK(cudaMemsetAsync(B->frozen + member, 0, 1, B->stream));
  CK(cudaStreamSynchronize(B->stream));
  return PLAN_OK;
}

plan_status plan_batch_export_state(plan_batch_t B, int member, float* z, float* u_coll, float* u_kin,
                                    float* u_wall, uint8_t* act_coll, uint8_t* act_wall) {
  if (!B || member < 0 || member >= B->n) return fail(PLAN_EINVAL, "null batch or member out of range");
  plan_status st = plan_export_state(B->m[member], z, u_coll, u_kin, u_wall, act_coll, act_wall, nullptr);
  if (st != PLAN_OK) return st;
  CK(cudaStreamSynchronize(B->stream));
  return PLAN_OK;
}

plan_status plan_batch_iterate(plan_batch_t B, int k_iters) {
  if (!B || k_iters < 0) return fail(PLAN_EINVAL, "bad argument");
  return batch_run(B, k_iters);
}

plan_status plan_batch_solve(plan_batch_t B, int* iters_done, float* residual, int* n_converged) {
  if (!B) return fail(PLAN_EINVAL, "null batch");
  int max_iter = 0, check = 1 << 30;
  for (plan_t h : B->m) { max_iter = std::max(max_iter, h->cfg.max_iter); check = std::min(check, h->cfg.check_every); }
  check = std::max(check, 2);
  if (check & 1) ++check;  // graph chunks are whole pairs of iterations
  std::vector<float> res(B->n, INFINITY);
  int nconv = 0;
  for (int b = 0; b < B->n; ++b) nconv += B->h_frozen[b] ? 1 : 0;
  while (B->k < max_iter && nconv < B->n) {
    const int iters = std::min(check, max_iter - B->k);
    plan_status st = batch_run(B, iters);
    if (st != PLAN_OK) return st;
    // residual of every member's last iteration: the consensus part is in its
    // slot; the primal part needs the next finishing step
    for (int b = 0; b < B->n; ++b) {
      if (B->h_frozen[b]) continue;
      plan_t h = B->m[b];
      Dev P = h->dev(h->k);
      residual_kernel<<<64, 256, 0, B->stream>>>(P);
    }
    batch_gather_res<<<(B->n + 255) / 256, 256, 0, B->stream>>>(B->tab[B->k & 1], B->n, B->res);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(res.data(), B->res, B->n * 4, cudaMemcpyDeviceToHost, B->stream));
    CK(cudaStreamSynchronize(B->stream));
    bool changed = false;
    for (int b = 0; b < B->n; ++b) {
      if (B->h_frozen[b]) continue;
      plan_t h = B->m[b];
      if (!(res[b] == res[b])) return fail(PLAN_ENUMERIC, "member %d: non-finite residual", b);
      if (res[b] < h->cfg.tol || B->k >= h->cfg.max_iter) {
        B->h_frozen[b] = 1;
        if (res[b] < h->cfg.tol) { B->conv_iter[b] = B->k; ++nconv; }
        changed = true;
      }
    }
    if (changed) CK(cudaMemcpyAsync(B->frozen, B->h_frozen.data(), B->n, cudaMemcpyHostToDevice, B->stream));
    int frozen = 0;
    for (int b = 0; b < B->n; ++b) frozen += B->h_frozen[b];
    if (frozen == B->n) break;
  }
  CK(cudaStreamSynchronize(B->stream));
  for (int b = 0; b < B->n; ++b) {
    if (iters_done) iters_done[b] = B->conv_iter[b] >= 0 ? B->conv_iter[b] : B->k;
    if (residual) residual[b] = res[b];
  }
  if (n_converged) *n_converged = nconv;
  return PLAN_OK;
}

plan_status plan_batch_get_trajectory(plan_batch_t B, int member, float* z, int on_device) {
  if (!B || member < 0 || member >= B->n) return fail(PLAN_EINVAL, "bad member index");
  return plan_get_trajectory(B->m[member], z, on_device);
}

plan_status plan_batch_autotune(plan_batch_t B, int iters_per_candidate, int* choice) {
  if (!B || iters_per_candidate < 2) return fail(PLAN_EINVAL, "bad argument");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int tr[4] = {4, 8, 16, 32}, mu[3] = {1, 2, 4}, gl[2] = {2, 8};
  float best = INFINITY;
  int bt = B->trows, bm = B->prox_mult, bg = B->glen;
  if (B->k & 1) { plan_status st = batch_run(B, 1); if (st != PLAN_OK) return st; }
  for (int a = 0; a < (B->dense ? 3 : 4); ++a)
    for (int c = 0; c < 3; ++c)
      for (int g = 0; g < 2; ++g) {
        B->trows = tr[a]; B->prox_mult = mu[c]; B->glen = gl[g];
        const int iters = std::max(iters_per_candidate / gl[g], 1) * gl[g];
        plan_status st = batch_run(B, gl[g]);  // capture outside the timing
        if (st != PLAN_OK) return st;
        CK(cudaEventRecord(e0, B->stream));
        st = batch_run(B, iters);
        if (st != PLAN_OK) return st;
        CK(cudaEventRecord(e1, B->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms / iters < best) { best = ms / iters; bt = tr[a]; bm = mu[c]; bg = gl[g]; }
      }
  B->trows = bt; B->prox_mult = bm; B->glen = bg;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (choice) { choice[0] = bt; choice[1] = bm; choice[2] = bg; }
  return PLAN_OK;
}

plan_status plan_batch_set_shape(plan_batch_t B, int rows_per_warp, int prox_ctas_per_sm,
                                 int iterations_per_graph) {
  if (!B) return fail(PLAN_EINVAL, "null batch");
  if (rows_per_warp != 4 && rows_per_warp != 8 && rows_per_warp != 16 &&
      !(rows_per_warp == 32 && !B->dense))
    return fail(PLAN_EINVAL, "rows_per_warp must be 4, 8, 16 (or 32 with the gated state)");
  if (prox_ctas_per_sm < 1 || prox_ctas_per_sm > 8) return fail(PLAN_EINVAL, "prox_ctas_per_sm must be 1..8");
  if (iterations_per_graph < 2 || (iterations_per_graph & 1))
    return fail(PLAN_EINVAL, "iterations_per_graph must be even and >= 2");
  B->trows = rows_per_warp;
  B->prox_mult = prox_ctas_per_sm;
  B->glen = iterations_per_graph;
  return PLAN_OK;
}

void plan_batch_destroy(plan_batch_t B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream); else cudaDeviceSynchronize();
  for (plan_t h : B->m) plan_destroy(h);
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->own_ws && B->ws) cudaFree(B->ws);
  delete B;
}

}  // extern "C"

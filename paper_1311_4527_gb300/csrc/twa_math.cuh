// twa_math.cuh -- FP32 device minimizers of the planning factors.
//
// Notation of Bento et al., "A message-passing algorithm for multi-agent
// trajectory planning" (NIPS 2013): n_lo / n_hi are the incoming messages of
// the two break-points of a segment, x_* the minimizer outputs.
//
// Collision and wall minimizers (Appendices C, D, I).  A segment [v_lo, v_hi]
// misses an open convex region iff a unit normal n separates them:
// <v_lo,n> >= h(n) and <v_hi,n> >= h(n), h the region's support function.
// For fixed n the cheapest v's are v = a + [h - <a,n>]_+ n, so the minimizer
// is min over directions of
//     E(n) = wl/2 [h - <a,n>]_+^2 + wh/2 [h - <b,n>]_+^2 .
// (Both hinges positive is the paper's tangent-slab configuration, one hinge
// at zero its compressed-spring configuration.)
//
// Disk of radius R at the origin (the collision minimizer through
// Eq. wall_min_goes_to_coll_min).  Let f(n) = wl (R - <a,n>)^2 +
// wh (R - <b,n>)^2 be the both-stretched piece, so E <= f/2 everywhere and
// E = f/2 where both hinges are positive.  Then
//     min E = min( E(n_f), m_a, m_b ),
// n_f the global minimiser of f on the unit circle, m_a the minimum of
// wl/2 [R - <a,n>]_+^2 over the arc <b,n> >= R (where the b hinge is zero)
// and m_b likewise: every piece of the circle is covered, and each of the
// three values is E at some direction.  n_f is a trust-region subproblem:
// with M = wl a a^T + wh b b^T = lambda1 e1 e1^T + lambda2 e2 e2^T and
// S = wl a + wh b, the global minimiser solves (M - mu I) n = R S with
// mu <= lambda1, i.e. t = lambda1 - mu >= 0 is the unique root of the
// decreasing secular function (R s1 / t)^2 + (R s2 / (d + t))^2 = 1,
// d = lambda2 - lambda1 (hard case: s1 = 0 and R |s2| < d gives t = 0).
// m_a / m_b are closed form: the arc point closest in angle to a (or b).
//
// Capsule (wall) regions use the same hinge energy with
// h(n) = max(<xL,n>, <xR,n>) + r, which is the disk energy of one end circle
// on each half-plane of directions.  The global minimum is at one of the two
// kink directions or at a local minimum of one end circle's energy: a local
// minimum of its both-stretched piece (global or local-nonglobal, both from
// the secular equation) or a single-hinge direction.  All are candidates.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace twa {

// Host and device: the same FP32 code is also compiled into a host-side test
// harness (tests/minimizer_harness.cu) that compares it with the FP64 oracle.
// Everything is inlined, and candidate directions are written to fixed
// array slots only (put_dir, unrolled loops), so that the minimizers keep
// their candidates in registers: a call or a dynamically indexed array puts
// them in local memory, whose latency sits on the minimizer's long dependent
// chain.
#define TWA_DEV __host__ __device__ __forceinline__
#define TWA_NOINLINE TWA_DEV
#ifndef TWA_ITER_HOOK
#define TWA_ITER_HOOK(kind)
#endif

TWA_DEV float2 mk(float x, float y) { return make_float2(x, y); }
TWA_DEV float2 operator+(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
TWA_DEV float2 operator-(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }
TWA_DEV float2 operator-(float2 a) { return mk(-a.x, -a.y); }
TWA_DEV float2 operator*(float s, float2 a) { return mk(s * a.x, s * a.y); }
TWA_DEV float dot(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }
TWA_DEV float cross(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }
TWA_DEV float2 perp(float2 a) { return mk(-a.y, a.x); }
TWA_DEV float2 normalized(float2 a) {
#ifdef __CUDA_ARCH__
  // one reciprocal square root (2 ulp) where |a|^2 is a normal float; the
  // directions are unit to a few ulp either way
  const float dd = a.x * a.x + a.y * a.y;
  if (dd > 1e-30f && dd < 1e30f) {
    const float s = rsqrtf(dd);
    return mk(a.x * s, a.y * s);
  }
#endif
  float n = hypotf(a.x, a.y);
  return n > 0.f ? mk(a.x / n, a.y / n) : mk(1.f, 0.f);
}

// Fast division (2 ulp for divisors of normal magnitude; every divisor here
// is a length, a curvature or a secular variable far from the float limits)
// and reciprocal square root, for the secular iterations and the direction
// arithmetic of the minimizers: fewer instructions on their long dependent
// chains.  The host build (test harness) uses the plain operations.
TWA_DEV float fdiv(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
TWA_DEV float frsqrt(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.f / sqrtf(x);
#endif
}

// out[n++] = v with constant indices (up to 4 slots).
TWA_DEV void put_dir(float2* out, int& n, float2 v) {
  if (n == 0) out[0] = v;
  else if (n == 1) out[1] = v;
  else if (n == 2) out[2] = v;
  else out[3] = v;
  ++n;
}

// Angle of a unit vector in [0, 2 pi): the tie-break order of directions.
// Not inlined: it runs only on exact ties, and a copy at every tie-break
// would crowd the minimizers' instruction stream.
__host__ __device__ __noinline__ float angle_of(float2 n) {
  float t = atan2f(n.y, n.x);
  return t < 0.f ? t + 6.283185307179586f : t;
}
// a before b in the tie-break order
__host__ __device__ __noinline__ bool angle_less(float2 a, float2 b) {
  return angle_of(a) < angle_of(b);
}

// Squared distance from the origin to segment [p0, p1].  Interior projections
// use the cross product (absolute error ~ eps |p0|, no cancellation of
// |p0|^2 against the projection).
TWA_DEV float dist2_origin_segment(float2 p0, float2 p1) {
  float2 d = p1 - p0;
  float dd = dot(d, d);
  float t = -dot(p0, d);
  if (t <= 0.f || dd == 0.f) return dot(p0, p0);
  if (t >= dd) return dot(p1, p1);
  float c = cross(p0, d);
  return c * c / dd;
}

TWA_DEV float dist2_point_segment(float2 q, float2 p0, float2 p1) {
  return dist2_origin_segment(p0 - q, p1 - q);
}

// Squared distance between segments [a0, a1] and [b0, b1].
TWA_DEV float dist2_segment_segment(float2 a0, float2 a1, float2 b0, float2 b1) {
  float d1 = cross(a1 - a0, b0 - a0), d2 = cross(a1 - a0, b1 - a0);
  float d3 = cross(b1 - b0, a0 - b0), d4 = cross(b1 - b0, a1 - b0);
  if (((d1 < 0.f && d2 > 0.f) || (d1 > 0.f && d2 < 0.f)) &&
      ((d3 < 0.f && d4 > 0.f) || (d3 > 0.f && d4 < 0.f)))
    return 0.f;
  float m = fminf(dist2_point_segment(a0, b0, b1), dist2_point_segment(a1, b0, b1));
  return fminf(m, fminf(dist2_point_segment(b0, a0, a1), dist2_point_segment(b1, a0, a1)));
}

// Keep the best (lowest E, then smallest angle) candidate direction.  tag
// records which kind of candidate won (read by the adjoint; dead otherwise).
struct Best {
  float2 n;
  float E;
  int tag;
  TWA_DEV void init() { n = mk(1.f, 0.f); E = INFINITY; tag = 0; }
  TWA_DEV void offer(float2 c, float e, int t = 0) {
    if (e < E || (e == E && angle_less(c, n))) { n = c; E = e; tag = t; }
  }
};

// ---------------------------------------------------------------------------
// Energy minimizer (Appendix E, Eq. energy_minimizer_output)
// ---------------------------------------------------------------------------
// pin_lo / pin_hi: that end's incoming weight is infinite (fixed endpoint).
TWA_DEV void energy_prox(float2 n_lo, float2 n_hi, float rho, bool pin_lo, bool pin_hi, float c,
                         float2& x_lo, float2& x_hi) {
  if (pin_lo && pin_hi) { x_lo = n_lo; x_hi = n_hi; return; }
  if (pin_lo) {
    x_lo = n_lo;
    float inv = 1.f / (2.f * c + rho);
    x_hi = mk((rho * n_hi.x + 2.f * c * n_lo.x) * inv, (rho * n_hi.y + 2.f * c * n_lo.y) * inv);
    return;
  }
  if (pin_hi) {
    x_hi = n_hi;
    float inv = 1.f / (2.f * c + rho);
    x_lo = mk((rho * n_lo.x + 2.f * c * n_hi.x) * inv, (rho * n_lo.y + 2.f * c * n_hi.y) * inv);
    return;
  }
  // equal weights rho on both ends
  float inv = 1.f / (4.f * c + rho);
  float2 s = n_lo + n_hi;
  x_lo = mk((rho * n_lo.x + 2.f * c * s.x) * inv, (rho * n_lo.y + 2.f * c * s.y) * inv);
  x_hi = mk((rho * n_hi.x + 2.f * c * s.x) * inv, (rho * n_hi.y + 2.f * c * s.y) * inv);
}

// ---------------------------------------------------------------------------
// Disk of radius R at the origin
// ---------------------------------------------------------------------------
TWA_DEV float hinge_E(float2 a, float2 b, float wl, float wh, float R, float2 n) {
  float ga = fmaxf(R - dot(a, n), 0.f), gb = fmaxf(R - dot(b, n), 0.f);
  return 0.5f * wl * ga * ga + 0.5f * wh * gb * gb;
}

// Global minimiser(s) of f(n) = wl (R - <a,n>)^2 + wh (R - <b,n>)^2 on the
// unit circle.  Writes 1 or 2 directions (2 only for exact ties).
TWA_NOINLINE int trs_global(float2 a, float2 b, float wl, float wh, float R,
                                       float2* out) {
  float m11 = wl * a.x * a.x + wh * b.x * b.x;
  float m22 = wl * a.y * a.y + wh * b.y * b.y;
  float m12 = wl * a.x * a.y + wh * b.x * b.y;
  float2 S = mk(wl * a.x + wh * b.x, wl * a.y + wh * b.y);
  float hd = 0.5f * (m11 - m22);
  float disc = hypotf(hd, m12);
  float d = 2.f * disc;  // lambda2 - lambda1 >= 0
  float2 e2;
  if (disc == 0.f) e2 = mk(1.f, 0.f);
  else if (hd >= 0.f) e2 = normalized(mk(hd + disc, m12));
  else e2 = normalized(mk(m12, disc - hd));
  float2 e1 = perp(e2);
  float s1 = dot(S, e1), s2 = dot(S, e2);
  float Sn = hypotf(s1, s2);
  if (!(Sn > 0.f)) { out[0] = e1; out[1] = -e1; return 2; }
  float A1 = R * fabsf(s1), A2 = R * fabsf(s2);
  if (A1 <= 1e-7f * R * Sn && A2 < d) {  // hard case: t = 0
    float n2 = R * s2 / d;
    float n1 = sqrtf(fmaxf(0.f, 1.f - n2 * n2));
    out[0] = n1 * e1 + n2 * e2;
    out[1] = (-n1) * e1 + n2 * e2;
    return 2;
  }
  // Root of h(t) = phi(t)^{-1/2} - 1 with phi = (A1/t)^2 + (A2/(d+t))^2.
  // 1/|n(t)| is concave and increasing (Moré-Sorensen), so Newton from the
  // left bracket end, where h <= 0, climbs monotonically to the root.
  float lo = fmaxf(fmaxf(A1, R * Sn - d), 0.f), hi = R * Sn;
  if (lo > hi) lo = hi;
  float t = lo > 0.f ? lo : 0.5f * hi;
  for (int it = 0; it < 40; ++it) {
    TWA_ITER_HOOK(0);
    float it_ = fdiv(1.f, t), id = fdiv(1.f, d + t);
    float q1 = A1 * it_, q2 = A2 * id;
    float phi = q1 * q1 + q2 * q2;
    float ip = frsqrt(phi);
    float h = ip - 1.f;
    if (h > 0.f) hi = t; else lo = t;
    if (h == 0.f) break;
    float dh = ip * ip * ip * (q1 * q1 * it_ + q2 * q2 * id);
    float tn = t - fdiv(h, dh);
    if (!(tn > lo && tn < hi)) tn = 0.5f * (lo + hi);
    // FP32 noise in h limits t to ~1e-7 relative; stop at 1e-6
    if (fabsf(tn - t) <= 1e-6f * t || hi - lo <= 1e-6f * hi) { t = tn; break; }
    t = tn;
  }
  float p1 = (t > 0.f) ? fdiv(R * s1, t) : copysignf(INFINITY, s1);
  float p2 = fdiv(R * s2, d + t);
  float n1, n2;
  if (fabsf(p1) <= fabsf(p2)) {
    n1 = p1;
    n2 = copysignf(sqrtf(fmaxf(0.f, 1.f - p1 * p1)), s2);
  } else {
    n2 = p2;
    n1 = copysignf(sqrtf(fmaxf(0.f, 1.f - p2 * p2)), s1);
  }
  out[0] = normalized(n1 * e1 + n2 * e2);
  return 1;
}

// The other stationary points of f: mu in (lambda1, lambda2), where
// t = mu - lambda1 solves (A1/t)^2 + (A2/(d - t))^2 = 1.  The left side is
// convex on (0, d) with its minimum at t_m = d A1^(2/3) / (A1^(2/3) + A2^(2/3)),
// so there are 0 or 2 roots (one is the local-but-not-global minimum); with
// s1 = 0 or s2 = 0 the stationary points at mu = lambda1 or lambda2 are added.
// Writes up to 4 directions; used by the wall minimizer, whose capsule
// restricts each end circle to a half-plane of directions.  part = 0 or 1
// writes only the directions of that part of the sequence (0: the special
// cases or the root left of t_m, 1: the root right of it), for callers that
// split the work over threads; -1 writes all.
TWA_NOINLINE int trs_local(float2 a, float2 b, float wl, float wh, float R, float2* out,
                           int part = -1) {
  float m11 = wl * a.x * a.x + wh * b.x * b.x;
  float m22 = wl * a.y * a.y + wh * b.y * b.y;
  float m12 = wl * a.x * a.y + wh * b.x * b.y;
  float2 S = mk(wl * a.x + wh * b.x, wl * a.y + wh * b.y);
  float hd = 0.5f * (m11 - m22);
  float disc = hypotf(hd, m12);
  float d = 2.f * disc;
  if (!(d > 0.f)) return 0;
  float2 e2 = (hd >= 0.f) ? normalized(mk(hd + disc, m12)) : normalized(mk(m12, disc - hd));
  float2 e1 = perp(e2);
  float s1 = dot(S, e1), s2 = dot(S, e2);
  float A1 = R * fabsf(s1), A2 = R * fabsf(s2);
  int n = 0;
  if (A1 == 0.f && A2 == 0.f) return 0;
  if ((A2 == 0.f || A1 == 0.f) && part == 1) return 0;
  if (A2 == 0.f) {  // hard case at mu = lambda2, and the root t = A1
    if (A1 < d) {
      float n1 = -R * s1 / d;
      float n2 = sqrtf(fmaxf(0.f, 1.f - n1 * n1));
      out[0] = n1 * e1 + n2 * e2;
      out[1] = n1 * e1 + (-n2) * e2;
      out[2] = (s1 > 0.f ? -1.f : 1.f) * e1;
      n = 3;
    }
    return n;
  }
  if (A1 == 0.f) {  // the root t = d - A2
    if (A2 < d) { out[0] = (s2 > 0.f ? 1.f : -1.f) * e2; n = 1; }
    return n;
  }
  float c1 = cbrtf(A1 * A1), c2 = cbrtf(A2 * A2);
  float tm = d * c1 / (c1 + c2);
  float phim = (A1 / tm) * (A1 / tm) + (A2 / (d - tm)) * (A2 / (d - tm));
  if (!(phim <= 1.f)) return 0;
  for (int side = (part == 1) ? 1 : 0; side < ((part == 0) ? 1 : 2); ++side) {
    // h(t) = phi(t)^(-1/2) - 1 is increasing on (0, tm] and decreasing on
    // [tm, d); each root is approached from its pole side, where h <= 0 (at
    // t = A1, resp. t = d - A2), so that the Newton steps move monotonically.
    float lo = side ? tm : 0.f, hi = side ? d : tm;
    float t = side ? fminf(fmaxf(d - A2, tm), d) : fmaxf(fminf(A1, tm), 0.f);
    if (!(t > lo && t < hi)) t = 0.5f * (lo + hi);
    for (int it = 0; it < 40; ++it) {
      TWA_ITER_HOOK(1);
      float it_ = fdiv(1.f, t), id = fdiv(1.f, d - t);
      float q1 = A1 * it_, q2 = A2 * id;
      float phi = q1 * q1 + q2 * q2;
      float ip = frsqrt(phi);
      float h = ip - 1.f;
      bool right = side ? (h < 0.f) : (h > 0.f);  // root lies left of t
      if (right) hi = t; else lo = t;
      if (h == 0.f || hi - lo <= 1e-6f * hi) break;
      float dphi = -2.f * (q1 * q1 * it_) + 2.f * (q2 * q2 * id);
      float dh = -0.5f * ip * ip * ip * dphi;
      float tn = (dh != 0.f) ? t - fdiv(h, dh) : 0.5f * (lo + hi);
      if (!(tn > lo && tn < hi)) tn = 0.5f * (lo + hi);
      const bool done = fabsf(tn - t) <= 1e-6f * fmaxf(t, tn);
      t = tn;
      if (done) break;
    }
    float p1 = fdiv(-R * s1, t), p2 = fdiv(R * s2, d - t);
    float n1, n2;
    if (fabsf(p1) <= fabsf(p2)) { n1 = p1; n2 = copysignf(sqrtf(fmaxf(0.f, 1.f - p1 * p1)), p2); }
    else { n2 = p2; n1 = copysignf(sqrtf(fmaxf(0.f, 1.f - p2 * p2)), p1); }
    put_dir(out, n, normalized(n1 * e1 + n2 * e2));
  }
  return n;
}

// Tangent normals n with <q, n> = R from a point q (|q| >= R).
TWA_DEV void tangent_normals(float2 q, float R, float2& t0, float2& t1) {
  float L2 = dot(q, q);
  float s = sqrtf(fmaxf(L2 - R * R, 0.f));
  float inv = fdiv(1.f, L2);
  float2 pq = perp(q);
  t0 = mk((R * q.x + s * pq.x) * inv, (R * q.y + s * pq.y) * inv);
  t1 = mk((R * q.x - s * pq.x) * inv, (R * q.y - s * pq.y) * inv);
}

// Direction in the arc {n : <q,n> >= R} (|q| >= R) maximising <w, n>.
// tangent: the answer is an end of the arc (<q,n> = R) rather than w / |w|.
TWA_DEV float2 arc_argmax(float2 q, float R, float2 w, bool& tangent) {
  float nw = hypotf(w.x, w.y);
  tangent = false;
  if (nw > 0.f && dot(q, w) >= R * nw) {
    const float inv = fdiv(1.f, nw);
    return mk(w.x * inv, w.y * inv);
  }
  tangent = true;
  float2 t0, t1;
  tangent_normals(q, R, t0, t1);
  float d0 = dot(w, t0), d1 = dot(w, t1);
  if (d0 > d1 || (d0 == d1 && angle_of(t0) <= angle_of(t1))) return normalized(t0);
  return normalized(t1);
}
TWA_DEV float2 arc_argmax(float2 q, float R, float2 w) {
  bool tangent;
  return arc_argmax(q, R, w, tangent);
}

// Kinds of winning direction of the free disk minimizer (Best::tag).
enum DiskTag {
  DISK_DEFAULT = 0,  // the (1, 0) fallback
  DISK_GLOBAL = 1,   // global minimiser n_f of the both-stretched piece f
  DISK_A_INNER = 2,  // a / |a| on the arc where b's hinge is zero
  DISK_A_TANGENT = 3,  // an end of that arc, <b, n> = R
  DISK_B_INNER = 4,  // b / |b| on the arc where a's hinge is zero
  DISK_B_TANGENT = 5   // an end of that arc, <a, n> = R
};

// Separating direction of the free disk minimizer and the kind of candidate
// it came from.
TWA_DEV float2 disk_dir_free(float2 a, float2 b, float wl, float wh, float R, int& tag) {
  Best best;
  best.init();
  best.offer(mk(1.f, 0.f), hinge_E(a, b, wl, wh, R, mk(1.f, 0.f)), DISK_DEFAULT);
  float2 c[2];
  int nc = trs_global(a, b, wl, wh, R, c);
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (k < nc) best.offer(c[k], hinge_E(a, b, wl, wh, R, c[k]), DISK_GLOBAL);
  // side 0: b's hinge can be zero, best a-term on that arc; side 1: the same
  // with a and b exchanged (one copy of the code, run twice)
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    const float2 q = side ? a : b, w = side ? b : a;
    if (dot(q, q) >= R * R) {
      bool tg;
      float2 n = arc_argmax(q, R, w, tg);
      best.offer(n, hinge_E(a, b, wl, wh, R, n),
                 side ? (tg ? DISK_B_TANGENT : DISK_B_INNER) : (tg ? DISK_A_TANGENT : DISK_A_INNER));
    }
  }
  tag = best.tag;
  return best.n;
}

// Collision minimizer core: disk of radius R at the origin, finite equal or
// unequal weights, neither end pinned.  (a, b): targets; (vl, vh): result.
TWA_NOINLINE void disk_prox_free(float2 a, float2 b, float wl, float wh, float R,
                                            float2& vl, float2& vh) {
  int tag;
  float2 n = disk_dir_free(a, b, wl, wh, R, tag);
  vl = a + fmaxf(R - dot(a, n), 0.f) * n;
  vh = b + fmaxf(R - dot(b, n), 0.f) * n;
}

// One end pinned at q (weight infinite): the free end's target is w.  The
// separating direction ranges over the arc {<q,n> >= R}.
TWA_NOINLINE float2 disk_prox_pinned(float2 q, float2 w, float R) {
  float2 n = arc_argmax(q, R, w);
  return w + fmaxf(R - dot(w, n), 0.f) * n;
}

// ---------------------------------------------------------------------------
// Capsule of radius r around the wall segment [c0, c1]
// ---------------------------------------------------------------------------
TWA_DEV float capsule_h(float2 c0, float2 c1, float r, float2 n) {
  return fmaxf(dot(c0, n), dot(c1, n)) + r;
}

TWA_DEV float capsule_E(float2 a, float2 b, float wl, float wh, float2 c0, float2 c1, float r,
                        float2 n) {
  float h = capsule_h(c0, c1, r, n);
  float ga = fmaxf(h - dot(a, n), 0.f), gb = fmaxf(h - dot(b, n), 0.f);
  return 0.5f * wl * ga * ga + 0.5f * wh * gb * gb;
}

// On the half-plane of directions where end circle ci gives the capsule's
// support (<c_ci - c_other, n> >= 0), the energy is that circle's disk
// energy.  Write n = c nu + s e (e the outward wall direction at that end, nu
// its normal, s >= 0) and beta_x, gamma_x for the coordinates of x - c_ci
// along nu and e.  When neither target lies beyond the end (gamma <= 0),
// <x - c_ci, n> <= c beta_x, so the energy is at least
// G(c) = wl/2 [r - c beta_a]_+^2 + wh/2 [r - c beta_b]_+^2, which equals the
// kink energies at c = +-1; with both targets on one side of the wall's line
// (beta_a, beta_b of one sign) G is monotone in c, so nothing in that
// half-plane is below the better kink and the circle's candidates can be
// skipped.  False for a zero-length wall.  The signs are decided in FP32, so
// each coordinate must clear a margin of 1e-6 |e| |x - c_ci| (a few units in
// the last place of the products): a target on the wall's line, on the
// perpendicular through the end or at the end centre keeps the circle's
// candidates (which are then computed exactly) instead of trusting a sign
// that rounding may have flipped.
TWA_DEV bool capsule_end_dominated(float2 a, float2 b, float2 c0, float2 c1, int ci) {
  const float2 e = c1 - c0;
  const float ee = dot(e, e);
  if (!(ee > 0.f)) return false;
  const float2 cc = ci ? c1 : c0;
  const float2 out = ci ? e : -e;
  const float2 nu = perp(e);
  const float2 da = a - cc, db = b - cc;
  const float ta = 1e-6f * sqrtf(ee * dot(da, da)), tb = 1e-6f * sqrtf(ee * dot(db, db));
  const float ga = dot(da, out), gb = dot(db, out);
  const float ba = dot(da, nu), bb = dot(db, nu);
  return ga < -ta && gb < -tb && ((ba > ta && bb > tb) || (ba < -ta && bb < -tb));
}

// Kinds of winning capsule direction (Best::tag): 0 the (1, 0) fallback,
// 1 a kink, and per end circle ci: 2 + 4 ci a stationary point of its
// both-stretched piece (free) or a tangent from the fixed end (pinned),
// 3 + 4 ci the single-hinge direction of the lower (free) / free (pinned)
// end, 4 + 4 ci that of the upper end (free).
TWA_DEV float2 capsule_dir_free(float2 a, float2 b, float wl, float wh, float2 c0, float2 c1,
                                float r, int& tag) {
  Best best;
  best.init();
  best.offer(mk(1.f, 0.f), capsule_E(a, b, wl, wh, c0, c1, r, mk(1.f, 0.f)), 0);
  float2 e = c1 - c0;
  if (e.x != 0.f || e.y != 0.f) {  // kinks: both end circles give the same support
    float2 k0 = normalized(perp(e));
    best.offer(k0, capsule_E(a, b, wl, wh, c0, c1, r, k0), 1);
    best.offer(-k0, capsule_E(a, b, wl, wh, c0, c1, r, -k0), 1);
  }
#pragma unroll 1
  for (int ci = 0; ci < 2; ++ci) {
    if (capsule_end_dominated(a, b, c0, c1, ci)) continue;
    float2 cc = ci ? c1 : c0;
    float2 ac = a - cc, bc = b - cc;
    float2 t[4];
    int nt = trs_global(ac, bc, wl, wh, r, t);
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (k < nt) best.offer(t[k], capsule_E(a, b, wl, wh, c0, c1, r, t[k]), 2 + 4 * ci);
    nt = trs_local(ac, bc, wl, wh, r, t);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < nt) best.offer(t[k], capsule_E(a, b, wl, wh, c0, c1, r, t[k]), 2 + 4 * ci);
    if (dot(ac, ac) > 0.f) {
      float2 n = normalized(ac);
      best.offer(n, capsule_E(a, b, wl, wh, c0, c1, r, n), 3 + 4 * ci);
    }
    if (dot(bc, bc) > 0.f) {
      float2 n = normalized(bc);
      best.offer(n, capsule_E(a, b, wl, wh, c0, c1, r, n), 4 + 4 * ci);
    }
  }
  tag = best.tag;
  return best.n;
}

TWA_NOINLINE void capsule_prox_free(float2 a, float2 b, float wl, float wh, float2 c0,
                                               float2 c1, float r, float2& vl, float2& vh) {
  int tag;
  float2 n = capsule_dir_free(a, b, wl, wh, c0, c1, r, tag);
  float h = capsule_h(c0, c1, r, n);
  vl = a + fmaxf(h - dot(a, n), 0.f) * n;
  vh = b + fmaxf(h - dot(b, n), 0.f) * n;
}

#ifdef __CUDACC__
// capsule_prox_free by a whole warp (every lane calls it with the same
// arguments and gets the same result): the candidate directions of
// capsule_dir_free are shared out over 9 lanes (the fallback and kinks; per
// end circle the global stationary point, the two halves of trs_local and the
// single-hinge directions), each lane keeps its best in the same order, and a
// warp reduction on (E, angle, position in the sequence) picks the candidate
// that the sequential scan keeps.  The secular solves then run side by side
// instead of one after another.
__device__ __forceinline__ void capsule_prox_free_warp(float2 a, float2 b, float wl, float wh,
                                                       float2 c0, float2 c1, float r, float2& vl,
                                                       float2& vh) {
  const int lane = threadIdx.x & 31;
  Best best;
  best.init();
  bool any = false;
  auto offer = [&](float2 c) {
    best.offer(c, capsule_E(a, b, wl, wh, c0, c1, r, c), 0);
    any = true;
  };
  if (lane == 0) {
    offer(mk(1.f, 0.f));
    float2 e = c1 - c0;
    if (e.x != 0.f || e.y != 0.f) {
      float2 k0 = normalized(perp(e));
      offer(k0);
      offer(-k0);
    }
  } else if (lane < 9 && !capsule_end_dominated(a, b, c0, c1, (lane - 1) >> 2)) {
    const int ci = (lane - 1) >> 2, task = (lane - 1) & 3;
    const float2 cc = ci ? c1 : c0;
    const float2 ac = a - cc, bc = b - cc;
    float2 t[4];
    int nt = 0;
    if (task == 0) nt = trs_global(ac, bc, wl, wh, r, t);
    else if (task < 3) nt = trs_local(ac, bc, wl, wh, r, t, task - 1);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < nt) offer(t[k]);
    if (task == 3) {
      if (dot(ac, ac) > 0.f) offer(normalized(ac));
      if (dot(bc, bc) > 0.f) offer(normalized(bc));
    }
  }
  // reduction: lower E, then smaller angle, then the earlier lane (whose
  // candidates come first in the sequential order)
  float E = any ? best.E : INFINITY;
  float2 n = best.n;
  int src = any ? lane : 32;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float E2 = __shfl_xor_sync(0xffffffffu, E, o);
    const float nx = __shfl_xor_sync(0xffffffffu, n.x, o), ny = __shfl_xor_sync(0xffffffffu, n.y, o);
    const int src2 = __shfl_xor_sync(0xffffffffu, src, o);
    bool take;
    if (src2 == 32) take = false;
    else if (src == 32) take = true;
    else if (E2 < E) take = true;
    else if (E2 == E) {
      const float g2 = angle_of(mk(nx, ny)), g = angle_of(n);
      take = g2 < g || (g2 == g && src2 < src);
    } else {
      // NaN energies never win in the sequential scan, and the fallback
      // (lane 0) is always offered first
      take = false;
    }
    if (take) { E = E2; n = mk(nx, ny); src = src2; }
  }
  const float h = capsule_h(c0, c1, r, n);
  vl = a + fmaxf(h - dot(a, n), 0.f) * n;
  vh = b + fmaxf(h - dot(b, n), 0.f) * n;
}
#endif

// One end pinned at q; free end target w.  Candidates: tangent directions
// from q to both end circles, the kinks, and the single-hinge directions;
// only directions that still separate q from the capsule are kept.
// Returns false if no candidate separates q (q inside the capsule).
TWA_DEV bool capsule_dir_pinned(float2 q, float2 w, float2 c0, float2 c1, float r, float2& dir,
                                int& tag) {
  float scale = fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)),
                      fmaxf(fmaxf(fabsf(c0.x), fabsf(c0.y)), fmaxf(fabsf(c1.x), fabsf(c1.y)))) + r;
  float tol = 4e-6f * scale;
  Best best;
  best.init();
  bool any = false;
  // candidates in a fixed order, each kept if it separates q
  auto offer = [&](float2 c, int t) {
    float h = capsule_h(c0, c1, r, c);
    if (dot(q, c) - h >= -tol) {
      float g = fmaxf(h - dot(w, c), 0.f);
      best.offer(c, 0.5f * g * g, t);
      any = true;
    }
  };
#pragma unroll
  for (int ci = 0; ci < 2; ++ci) {
    float2 cc = ci ? c1 : c0;
    float2 qc = q - cc;
    if (dot(qc, qc) >= r * r) {
      float2 t0, t1;
      tangent_normals(qc, r, t0, t1);
      offer(normalized(t0), 2 + 4 * ci);
      offer(normalized(t1), 2 + 4 * ci);
    }
    float2 wc = w - cc;
    if (dot(wc, wc) > 0.f) offer(normalized(wc), 3 + 4 * ci);
  }
  float2 e = c1 - c0;
  if (e.x != 0.f || e.y != 0.f) {
    float2 k0 = normalized(perp(e));
    offer(k0, 1);
    offer(-k0, 1);
  }
  dir = best.n;
  tag = best.tag;
  return any;
}

TWA_NOINLINE bool capsule_prox_pinned(float2 q, float2 w, float2 c0, float2 c1, float r,
                                                 float2& vw) {
  float2 n;
  int tag;
  if (!capsule_dir_pinned(q, w, c0, c1, r, n, tag)) { vw = w; return false; }
  float h = capsule_h(c0, c1, r, n);
  vw = w + fmaxf(h - dot(w, n), 0.f) * n;
  return true;
}

// ---------------------------------------------------------------------------
// Zero incoming weights (the feasibility problem, no kinetic factors)
// ---------------------------------------------------------------------------
// Weight classes of one end: 0 (zero), 1 (rho0), 2 (infinite: fixed end).
// One end's weight -> 0+ with the other finite has a lexicographic limit:
// the weighted end moves out of the region by the least amount (a segment
// shrunk to that point is feasible), then the zero-weight end solves the
// fixed-end problem against it.  Both zero are equal weights.

// Closest point to q outside the open disk of radius R at the origin.
TWA_DEV float2 disk_project_out(float2 q, float R) {
  const float L = hypotf(q.x, q.y);
  if (L >= R) return q;
  if (L > 0.f) return (R / L) * q;
  return mk(R, 0.f);
}

// Closest point to q outside the open capsule of radius r around [c0, c1]; a
// point on the axis leaves along the normal of smallest angle.
TWA_DEV float2 capsule_project_out(float2 q, float2 c0, float2 c1, float r) {
  const float2 e = c1 - c0;
  const float ee = dot(e, e);
  float t = ee > 0.f ? dot(q - c0, e) / ee : 0.f;
  t = fminf(1.f, fmaxf(0.f, t));
  const float2 c = c0 + t * e;
  const float2 d = q - c;
  const float L = hypotf(d.x, d.y);
  if (L >= r) return q;
  if (L > 0.f) return c + (r / L) * d;
  if (!(ee > 0.f)) return c + mk(r, 0.f);
  const float2 n1 = normalized(perp(e));
  return c + r * ((angle_of(n1) < angle_of(-n1)) ? n1 : -n1);
}

// Disk minimizer for weight classes (cl, ch) of the two ends of the relative
// segment (equal finite weights where both are 1).
TWA_DEV void disk_prox_classes(float2 a, float2 b, int cl, int ch, float R, float w, float2& vl,
                               float2& vh) {
  vl = a; vh = b;
  if (cl == 2 && ch == 2) return;
  if (cl == ch) { disk_prox_free(a, b, w, w, R, vl, vh); return; }  // both rho0 or both zero
  // one end fixed (class 2), or one end of zero weight, which first leaves
  // the disk by the least amount and is then held there: either way the other
  // end solves the fixed-end problem (one call site for the four cases)
  const bool lo_fixed = (cl == 2) || (cl == 1 && ch == 0);
  if (cl == 1 && ch == 0) vl = disk_project_out(a, R);
  if (cl == 0 && ch == 1) vh = disk_project_out(b, R);
  const float2 q = lo_fixed ? vl : vh, t = lo_fixed ? b : a;
  const float2 v = disk_prox_pinned(q, t, R);
  if (lo_fixed) vh = v; else vl = v;
}

// Capsule minimizer for weight classes; false if a fixed end lies inside.
TWA_DEV bool capsule_prox_classes(float2 a, float2 b, int cl, int ch, float2 c0, float2 c1, float r,
                                  float w, float2& vl, float2& vh) {
  vl = a; vh = b;
  if (cl == 2 && ch == 2) return true;
  if (cl == ch) { capsule_prox_free(a, b, w, w, c0, c1, r, vl, vh); return true; }  // equal weights
  // as disk_prox_classes: the other end solves the fixed-end problem
  const bool lo_fixed = (cl == 2) || (cl == 1 && ch == 0);
  if (cl == 1 && ch == 0) vl = capsule_project_out(a, c0, c1, r);
  if (cl == 0 && ch == 1) vh = capsule_project_out(b, c0, c1, r);
  return lo_fixed ? capsule_prox_pinned(vl, b, c0, c1, r, vh) : capsule_prox_pinned(vh, a, c0, c1, r, vl);
}

// ---------------------------------------------------------------------------
// Maximum / minimum velocity minimizers (Appendices F and G)
// ---------------------------------------------------------------------------
// |x_lo - x_hi| <= C (is_max) or >= C, from messages that violate it.  With
// equal finite weights the appendix's closed form keeps the midpoint and
// scales x_lo - x_hi to length C along n_lo - n_hi; an infinite weight (or a
// zero weight against a finite one) keeps the other end; both zero are equal
// weights.  Coincident ends (minimum velocity) separate along (1, 0).
TWA_DEV void velocity_prox(float2 n_lo, float2 n_hi, int cl, int ch, float C, float2& x_lo,
                           float2& x_hi) {
  x_lo = n_lo; x_hi = n_hi;
  if (cl == 2 && ch == 2) return;
  const float2 d = n_lo - n_hi;
  const float L = hypotf(d.x, d.y);
  const float2 u = L > 0.f ? (1.f / L) * d : mk(-1.f, 0.f);
  if (cl == 2 || (ch == 0 && cl != 0)) { x_hi = n_lo - C * u; return; }
  if (ch == 2 || (cl == 0 && ch != 0)) { x_lo = n_hi + C * u; return; }
  const float2 m = 0.5f * (n_lo + n_hi);
  x_lo = m + (0.5f * C) * u;
  x_hi = m - (0.5f * C) * u;
}

}  // namespace twa

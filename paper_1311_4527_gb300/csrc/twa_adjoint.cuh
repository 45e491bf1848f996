// twa_adjoint.cuh -- reverse-mode derivatives (vector-Jacobian products) of
// the FP32 minimizers in twa_math.cuh, with the branch each minimizer takes
// held fixed.  Host and device, like twa_math.cuh.
//
// Disk minimizers (Appendix C through the reduction to one relative segment).
// The output of one end is v = w + [R - <w, n>]_+ n, n = (cos phi, sin phi)
// the separating direction and tau = (-sin phi, cos phi).  With n fixed,
//     dv = dw + s (dR - <dw, n> - <w, tau> dphi) n + s g tau dphi,
// s = [g > 0], g = R - <w, n>.  dphi depends on the branch:
//  * a stationary point of an energy E(phi) = sum_v w_v/2 g_v^2 (the global
//    minimiser of the both-stretched piece): E'(phi) = 0 differentiated,
//        dphi = -(dE'/dv . dv + dE'/dR dR) / E'',
//        E'' = sum w_v (<v, tau>^2 + g_v <v, n>),
//        dE'/dv = w_v (<v, tau> n - g_v tau),  dE'/dR = -sum w_v <v, tau>;
//  * the single-hinge direction n = v / |v|: dphi = <tau, dv> / |v|;
//  * an end of an arc, <q, n> = R: dphi = (dR - <dq, n>) / <q, tau>.
// Kinetic minimizer (Appendix E): linear in n, rational in c.
#pragma once
#include "twa_math.cuh"

namespace twa {

// Reverse of v = w + [R - <w, n>]_+ n for fixed n: adds the adjoints of w and
// R and the adjoint of the angle phi of n.
TWA_DEV void end_vjp(float2 w, float2 vbar, float2 n, float R, float2& wbar, float& Rbar,
                     float& phibar) {
  const float g = R - dot(w, n);
  if (g > 0.f) {
    const float2 t = perp(n);
    const float vn = dot(vbar, n);
    wbar = vbar - vn * n;
    Rbar += vn;
    phibar += g * dot(vbar, t) - dot(w, t) * vn;
  } else {
    wbar = vbar;
  }
}

// dphi of a stationary point of sum over {a, b} of w/2 (R - <v, n>)^2.
TWA_DEV void stationary_vjp(float2 a, float2 b, float wl, float wh, float R, float2 n, float phibar,
                            float2& abar, float2& bbar, float& Rbar) {
  const float2 t = perp(n);
  const float an = dot(a, n), bn = dot(b, n), at = dot(a, t), bt = dot(b, t);
  const float ga = R - an, gb = R - bn;
  const float E2 = wl * (at * at + ga * an) + wh * (bt * bt + gb * bn);
  const float scale = wl * (dot(a, a) + R * R) + wh * (dot(b, b) + R * R);
  if (!(E2 > 1e-6f * scale)) return;  // degenerate stationary point: no rotation
  const float k = phibar / E2;
  abar = abar - (k * wl) * (at * n - ga * t);
  bbar = bbar - (k * wh) * (bt * n - gb * t);
  Rbar += k * (wl * at + wh * bt);
}

// n = w / |w|
TWA_DEV void inner_vjp(float2 w, float2 n, float phibar, float2& wbar) {
  const float nw = hypotf(w.x, w.y);
  if (nw > 0.f) wbar = wbar + (phibar / nw) * perp(n);
}

// <q, n> = R
TWA_DEV void tangent_vjp(float2 q, float2 n, float phibar, float2& qbar, float& Rbar) {
  const float qt = dot(q, perp(n));
  if (fabsf(qt) > 1e-6f * hypotf(q.x, q.y)) {
    const float k = phibar / qt;
    Rbar += k;
    qbar = qbar - k * n;
  }
}

// Adjoint of disk_prox_free(a, b, wl, wh, R) -> (vl, vh).
TWA_DEV void disk_free_vjp(float2 a, float2 b, float wl, float wh, float R, float2 vlbar,
                           float2 vhbar, float2& abar, float2& bbar, float& Rbar) {
  int tag;
  const float2 n = disk_dir_free(a, b, wl, wh, R, tag);
  float phib = 0.f;
  Rbar = 0.f;
  end_vjp(a, vlbar, n, R, abar, Rbar, phib);
  end_vjp(b, vhbar, n, R, bbar, Rbar, phib);
  switch (tag) {
    case DISK_GLOBAL: stationary_vjp(a, b, wl, wh, R, n, phib, abar, bbar, Rbar); break;
    case DISK_A_INNER: inner_vjp(a, n, phib, abar); break;
    case DISK_B_INNER: inner_vjp(b, n, phib, bbar); break;
    case DISK_A_TANGENT: tangent_vjp(b, n, phib, bbar, Rbar); break;
    case DISK_B_TANGENT: tangent_vjp(a, n, phib, abar, Rbar); break;
    default: {
      // the (1, 0) fallback wins only where it is itself a minimiser: a
      // stationary point of the hinges that are positive there
      const float ml = (R - dot(a, n) > 0.f) ? wl : 0.f, mh = (R - dot(b, n) > 0.f) ? wh : 0.f;
      stationary_vjp(a, b, ml, mh, R, n, phib, abar, bbar, Rbar);
    }
  }
}

// Adjoint of disk_prox_pinned(q, w, R) -> v (q is the fixed end).
TWA_DEV void disk_pinned_vjp(float2 q, float2 w, float R, float2 vbar, float2& qbar, float2& wbar,
                             float& Rbar) {
  bool tangent;
  const float2 n = arc_argmax(q, R, w, tangent);
  float phib = 0.f;
  Rbar = 0.f;
  qbar = mk(0.f, 0.f);
  end_vjp(w, vbar, n, R, wbar, Rbar, phib);
  if (tangent) tangent_vjp(q, n, phib, qbar, Rbar);
  else inner_vjp(w, n, phib, wbar);
}

// Adjoint of the pair collision minimizer (coll_minimizer in twa_iter.cuh):
// n = (i lo, i hi, j lo, j hi) -> x; xbar = adjoints of x (the caller passes
// 0 at a fixed end, whose x is not used).  Writes nbar and the adjoint of
// R = r_i + r_j.
TWA_DEV void coll_vjp(float2 nil, float2 nih, float2 njl, float2 njh, bool pin_lo, bool pin_hi,
                      float R, float rho, float2 xbil, float2 xbih, float2 xbjl, float2 xbjh,
                      float2& nbil, float2& nbih, float2& nbjl, float2& nbjh, float& Rbar) {
  const float2 cl = njl - nil, ch = njh - nih;
  // x_i = (s - v) / 2, x_j = (s + v) / 2 at a free end; x = n at a fixed one
  const float2 vbl = 0.5f * (xbjl - xbil), sbl = 0.5f * (xbil + xbjl);
  const float2 vbh = 0.5f * (xbjh - xbih), sbh = 0.5f * (xbih + xbjh);
  Rbar = 0.f;
  nbil = xbil; nbjl = xbjl; nbih = xbih; nbjh = xbjh;
  if (pin_lo && pin_hi) return;
  float2 clb, chb;
  if (pin_lo) {
    disk_pinned_vjp(cl, ch, R, vbh, clb, chb, Rbar);
    nbih = sbh - chb; nbjh = sbh + chb;
  } else if (pin_hi) {
    disk_pinned_vjp(ch, cl, R, vbl, chb, clb, Rbar);
    nbil = sbl - clb; nbjl = sbl + clb;
  } else {
    const float w = 0.5f * rho;
    disk_free_vjp(cl, ch, w, w, R, vbl, vbh, clb, chb, Rbar);
    nbil = sbl - clb; nbjl = sbl + clb;
    nbih = sbh - chb; nbjh = sbh + chb;
    return;
  }
  // the fixed end's n enters through the relative vector only
  if (pin_lo) { nbil = nbil - clb; nbjl = nbjl + clb; }
  else { nbih = nbih - chb; nbjh = nbjh + chb; }
}

// Adjoint of energy_prox(n_lo, n_hi, rho, pin_lo, pin_hi, c) -> (x_lo, x_hi);
// cbar is the adjoint of the coefficient c.
TWA_DEV void energy_vjp(float2 n_lo, float2 n_hi, float rho, bool pin_lo, bool pin_hi, float c,
                        float2 xbl, float2 xbh, float2& nbl, float2& nbh, float& cbar) {
  cbar = 0.f;
  if (pin_lo && pin_hi) { nbl = xbl; nbh = xbh; return; }
  if (pin_lo) {
    // x_hi = (rho n_hi + 2 c n_lo) / (2 c + rho)
    const float inv = 1.f / (2.f * c + rho);
    nbl = xbl + (2.f * c * inv) * xbh;
    nbh = (rho * inv) * xbh;
    cbar = 2.f * rho * inv * inv * dot(xbh, n_lo - n_hi);
    return;
  }
  if (pin_hi) {
    const float inv = 1.f / (2.f * c + rho);
    nbh = xbh + (2.f * c * inv) * xbl;
    nbl = (rho * inv) * xbl;
    cbar = 2.f * rho * inv * inv * dot(xbl, n_hi - n_lo);
    return;
  }
  // x_lo = (rho n_lo + 2 c s) / (4 c + rho), x_hi likewise, s = n_lo + n_hi
  const float inv = 1.f / (4.f * c + rho);
  const float2 sb = (2.f * c * inv) * (xbl + xbh);
  nbl = (rho * inv) * xbl + sb;
  nbh = (rho * inv) * xbh + sb;
  cbar = 2.f * rho * inv * inv * dot(xbl - xbh, n_hi - n_lo);
}

// ---------------------------------------------------------------------------
// Walls (Appendix D's capsule) and velocity limits (Appendices F, G)
// ---------------------------------------------------------------------------
// For a fixed direction n the capsule's support is h(n) = <c, n> + r with c
// the end circle that attains the max, so each end's output is the disk's
// with w - c in place of w and R = r; dphi follows the branch as for the
// disk, with the branch's own circle (a kink direction does not move).
TWA_DEV float2 active_circle(float2 c0, float2 c1, float2 n) {
  return dot(c0, n) >= dot(c1, n) ? c0 : c1;
}

// Adjoint of capsule_prox_free (wl = wh = w) -> (vl, vh): abar, bbar, rbar.
TWA_DEV void capsule_free_vjp(float2 a, float2 b, float w, float2 c0, float2 c1, float r,
                              float2 vlbar, float2 vhbar, float2& abar, float2& bbar,
                              float& rbar) {
  int tag;
  const float2 n = capsule_dir_free(a, b, w, w, c0, c1, r, tag);
  const float2 cs = active_circle(c0, c1, n);
  float phib = 0.f;
  rbar = 0.f;
  end_vjp(a - cs, vlbar, n, r, abar, rbar, phib);
  end_vjp(b - cs, vhbar, n, r, bbar, rbar, phib);
  if (tag < 2) return;  // the fallback or a kink: n does not move
  const int ci = (tag - 2) >> 2, kind = (tag - 2) & 3;
  const float2 cc = ci ? c1 : c0;
  if (kind == 0) stationary_vjp(a - cc, b - cc, w, w, r, n, phib, abar, bbar, rbar);
  else if (kind == 1) inner_vjp(a - cc, n, phib, abar);
  else inner_vjp(b - cc, n, phib, bbar);
}

// Adjoint of capsule_prox_pinned(q, w) -> v.
TWA_DEV void capsule_pinned_vjp(float2 q, float2 w, float2 c0, float2 c1, float r, float2 vbar,
                                float2& qbar, float2& wbar, float& rbar) {
  float2 n;
  int tag;
  qbar = mk(0.f, 0.f);
  rbar = 0.f;
  if (!capsule_dir_pinned(q, w, c0, c1, r, n, tag)) { wbar = vbar; return; }
  const float2 cs = active_circle(c0, c1, n);
  float phib = 0.f;
  end_vjp(w - cs, vbar, n, r, wbar, rbar, phib);
  if (tag < 2) return;
  const int ci = (tag - 2) >> 2, kind = (tag - 2) & 3;
  const float2 cc = ci ? c1 : c0;
  if (kind == 0) tangent_vjp(q - cc, n, phib, qbar, rbar);
  else inner_vjp(w - cc, n, phib, wbar);
}

// Adjoint of the wall factor's minimizer for classes 1 (rho0) / 2 (fixed
// end): x = n at a fixed end.  xbar at a fixed end is 0 by the caller.
TWA_DEV void wall_vjp(float2 nl, float2 nh, bool pin_lo, bool pin_hi, float2 c0, float2 c1,
                      float r, float rho, float2 xbl, float2 xbh, float2& nbl, float2& nbh,
                      float& rbar) {
  rbar = 0.f;
  nbl = xbl; nbh = xbh;
  if (pin_lo && pin_hi) return;
  if (pin_lo) {
    float2 qb, wb;
    capsule_pinned_vjp(nl, nh, c0, c1, r, xbh, qb, wb, rbar);
    nbl = nbl + qb; nbh = wb;
  } else if (pin_hi) {
    float2 qb, wb;
    capsule_pinned_vjp(nh, nl, c0, c1, r, xbl, qb, wb, rbar);
    nbh = nbh + qb; nbl = wb;
  } else {
    capsule_free_vjp(nl, nh, 0.5f * rho, c0, c1, r, xbl, xbh, nbl, nbh, rbar);
  }
}

// Adjoint of velocity_prox for classes 1 / 2 (equal finite weights keep the
// midpoint and set x_lo - x_hi = C u, u = (n_lo - n_hi) / L; a fixed end
// stays and the other end is C u from it).
TWA_DEV void velocity_vjp(float2 nl, float2 nh, bool pin_lo, bool pin_hi, float C, float2 xbl,
                          float2 xbh, float2& nbl, float2& nbh) {
  nbl = xbl; nbh = xbh;
  if (pin_lo && pin_hi) return;
  const float2 d = nl - nh;
  const float L = hypotf(d.x, d.y);
  // du = (I - u u^T) dd / L; u is fixed when the ends coincide
  const float2 u = L > 0.f ? (1.f / L) * d : mk(-1.f, 0.f);
  auto proj = [&](float2 g) {  // (I - u u^T) g / L
    if (!(L > 0.f)) return mk(0.f, 0.f);
    const float gu = dot(g, u);
    return (1.f / L) * (g - gu * u);
  };
  if (pin_lo) {  // x_lo = n_lo, x_hi = n_lo - C u
    const float2 pd = (-C) * proj(xbh);
    nbl = xbl + xbh + pd;
    nbh = -1.f * pd;
    return;
  }
  if (pin_hi) {  // x_hi = n_hi, x_lo = n_hi + C u
    const float2 pd = C * proj(xbl);
    nbh = xbh + xbl - pd;
    nbl = pd;
    return;
  }
  const float2 mb = 0.5f * (xbl + xbh);   // d/dn of the midpoint
  const float2 pd = (0.5f * C) * proj(xbl - xbh);
  nbl = mb + pd;
  nbh = mb - pd;
}

}  // namespace twa

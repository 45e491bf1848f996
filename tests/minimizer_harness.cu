// Host build of the CUDA path's FP32 minimizers (csrc/twa_math.cuh) for
// CPU-side tests: the same source the kernels compile, called through a small
// C interface, with counters on the secular-equation iterations.  Test
// infrastructure only; nothing on the product path loads it.
#include <cstdint>

static long long g_iters[2];
__host__ __device__ inline void count_iter(int kind) {
#ifndef __CUDA_ARCH__
  ++g_iters[kind];
#endif
}
#define TWA_ITER_HOOK(kind) count_iter(kind)
#include "twa_math.cuh"
#include "twa_adjoint.cuh"

using namespace twa;

extern "C" {

void h_reset_iters() { g_iters[0] = g_iters[1] = 0; }
long long h_iters(int kind) { return g_iters[kind]; }

// disk of radius R at the origin, neither end pinned
void h_disk_prox_free(const float* a, const float* b, float wl, float wh, float R, float* out) {
  float2 vl, vh;
  disk_prox_free(mk(a[0], a[1]), mk(b[0], b[1]), wl, wh, R, vl, vh);
  out[0] = vl.x; out[1] = vl.y; out[2] = vh.x; out[3] = vh.y;
}

// one end pinned at q; the free end's target is w
void h_disk_prox_pinned(const float* q, const float* w, float R, float* out) {
  float2 v = disk_prox_pinned(mk(q[0], q[1]), mk(w[0], w[1]), R);
  out[0] = v.x; out[1] = v.y;
}

void h_capsule_prox_free(const float* a, const float* b, float wl, float wh, const float* c0,
                         const float* c1, float r, float* out) {
  float2 vl, vh;
  capsule_prox_free(mk(a[0], a[1]), mk(b[0], b[1]), wl, wh, mk(c0[0], c0[1]), mk(c1[0], c1[1]),
                    r, vl, vh);
  out[0] = vl.x; out[1] = vl.y; out[2] = vh.x; out[3] = vh.y;
}

// the capsule minimizer's rule for skipping an end circle's candidates
int h_capsule_end_dominated(const float* a, const float* b, const float* c0, const float* c1,
                            int ci) {
  return capsule_end_dominated(mk(a[0], a[1]), mk(b[0], b[1]), mk(c0[0], c0[1]), mk(c1[0], c1[1]),
                               ci) ? 1 : 0;
}

int h_capsule_prox_pinned(const float* q, const float* w, const float* c0, const float* c1, float r,
                          float* out) {
  float2 v;
  bool ok = capsule_prox_pinned(mk(q[0], q[1]), mk(w[0], w[1]), mk(c0[0], c0[1]),
                                mk(c1[0], c1[1]), r, v);
  out[0] = v.x; out[1] = v.y;
  return ok ? 1 : 0;
}

void h_energy_prox(const float* nl, const float* nh, float rho, int pin_lo, int pin_hi, float c,
                   float* out) {
  float2 xl, xh;
  energy_prox(mk(nl[0], nl[1]), mk(nh[0], nh[1]), rho, pin_lo != 0, pin_hi != 0, c, xl, xh);
  out[0] = xl.x; out[1] = xl.y; out[2] = xh.x; out[3] = xh.y;
}

// Adjoints (twa_adjoint.cuh).  n: 8 floats (i lo, i hi, j lo, j hi); xbar
// likewise; out: nbar (8 floats) then the adjoint of R.
void h_coll_vjp(const float* n, int pin_lo, int pin_hi, float R, float rho, const float* xb,
                float* out) {
  float2 nb[4];
  float Rb;
  coll_vjp(mk(n[0], n[1]), mk(n[2], n[3]), mk(n[4], n[5]), mk(n[6], n[7]), pin_lo != 0,
           pin_hi != 0, R, rho, mk(xb[0], xb[1]), mk(xb[2], xb[3]), mk(xb[4], xb[5]),
           mk(xb[6], xb[7]), nb[0], nb[1], nb[2], nb[3], Rb);
  for (int k = 0; k < 4; ++k) { out[2 * k] = nb[k].x; out[2 * k + 1] = nb[k].y; }
  out[8] = Rb;
}

// out: nbar (4 floats) then the adjoint of c.
void h_energy_vjp(const float* nl, const float* nh, float rho, int pin_lo, int pin_hi, float c,
                  const float* xb, float* out) {
  float2 bl, bh;
  float cb;
  energy_vjp(mk(nl[0], nl[1]), mk(nh[0], nh[1]), rho, pin_lo != 0, pin_hi != 0, c,
             mk(xb[0], xb[1]), mk(xb[2], xb[3]), bl, bh, cb);
  out[0] = bl.x; out[1] = bl.y; out[2] = bh.x; out[3] = bh.y; out[4] = cb;
}

// Wall factor adjoint (classes rho0 / fixed ends): n 4 floats (lo, hi), wall
// 4 floats, xbar 4 floats; out: nbar (4) then the adjoint of r.
void h_wall_vjp(const float* n, int pin_lo, int pin_hi, const float* wall, float r, float rho,
                const float* xb, float* out) {
  float2 bl, bh;
  float rb;
  wall_vjp(mk(n[0], n[1]), mk(n[2], n[3]), pin_lo != 0, pin_hi != 0, mk(wall[0], wall[1]),
           mk(wall[2], wall[3]), r, rho, mk(xb[0], xb[1]), mk(xb[2], xb[3]), bl, bh, rb);
  out[0] = bl.x; out[1] = bl.y; out[2] = bh.x; out[3] = bh.y; out[4] = rb;
}

// Velocity-limit factor adjoint: out nbar (4).
void h_velocity_vjp(const float* n, int pin_lo, int pin_hi, float C, const float* xb, float* out) {
  float2 bl, bh;
  velocity_vjp(mk(n[0], n[1]), mk(n[2], n[3]), pin_lo != 0, pin_hi != 0, C, mk(xb[0], xb[1]),
               mk(xb[2], xb[3]), bl, bh);
  out[0] = bl.x; out[1] = bl.y; out[2] = bh.x; out[3] = bh.y;
}

// Winning candidate kind of the free disk minimizer (DiskTag).
int h_disk_tag(const float* a, const float* b, float wl, float wh, float R) {
  int tag;
  disk_dir_free(mk(a[0], a[1]), mk(b[0], b[1]), wl, wh, R, tag);
  return tag;
}

}  // extern "C"

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

}  // extern "C"

// snap_geom.cuh -- per-slot Cayley-Klein geometry and reverse-slot map,
// computed by the compute_U kernels for their own atom's neighbour slots.
//
// Geometry of a slot (Sec. II-A: the neighbour vector mapped to the
// 3-sphere, with constants from the paper's SNAP reference):
//   theta0 = rfac0 pi (r - rmin0)/(rcut - rmin0), z0 = r cot theta0,
//   r0 = sqrt(r^2 + z0^2), a = (z0 - i z)/r0, b = (y - i x)/r0,
// the cosine switching function f_c, and the derivatives of a, b and f_c
// with respect to r.  r, theta0, a and b are evaluated in FP64; the gradients
// and f_c in the working precision G (they only feed the G recursions, and
// FP64 runs at 1/64 of the FP32 rate).  The neighbour builder gives the two
// slots of a pair exactly opposite vectors, and every operation here is
// odd or even in the vector's sign under round-to-nearest, so the slot (k, i)
// gets exactly conj(a), -b, -grad f_c, -conj(da/dr), db/dr of the slot (i, k).
//
// rev[i][s] is the slot of the opposite pair (k, i, -s) in k's list (the
// force stage gathers dE_k/dr_ki through it instead of scattering with
// atomics); a missing opposite pair raises flags[1].
#pragma once
#include <math.h>

#include "snap_internal.h"

namespace snap {
namespace geo {

__device__ __forceinline__ void sincospi_g(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_g(double x, double* s, double* c) { sincospi(x, s, c); }

// Geometry of slot q into geom[q][0..kGeomStride): a (2), b (2), f_c,
// grad f_c (3), da/dr_d (3 x 2), db/dr_d (3 x 2).
template <typename G>
__device__ void slot_geom(const WorkArgs& a, long q) {
  G* g = reinterpret_cast<G*>(a.geom) + q * kGeomStride;
  const double x = a.rij[3 * q], y = a.rij[3 * q + 1], z = a.rij[3 * q + 2];
  const double r2 = x * x + y * y + z * z;
  const double ir = rsqrt(r2);
  const double r = r2 * ir;
  G v[kGeomStride];
#pragma unroll
  for (int e = 0; e < kGeomStride; ++e) v[e] = G(0);
  if (!(r < a.rcut)) {  // outside the cutoff (caller lists): no contribution
    v[0] = G(1);
#pragma unroll
    for (int e = 0; e < kGeomStride; ++e) g[e] = v[e];
    return;
  }
  // r0 = sqrt(r^2 + z0^2) = r / |sin theta0|, so with sr = |sin theta0| / r
  //   a = z0 / r0 - i z / r0 = sign(sin theta0) cos theta0 - i z sr,
  //   b = (y - i x) / r0     = y sr - i x sr
  // (no division, one reciprocal square root; sr multiplies +-x, +-y, +-z, so
  // the opposite slot still gets exactly conj(a) and -b)
  double st, ct;
  sincospi(a.rfac0 * (r - a.rmin0) * a.inv_span, &st, &ct);
  const double sr = fabs(st) * ir;
  const double ar = st < 0.0 ? -ct : ct, ai = -z * sr;
  const double br = y * sr, bi = -x * sr;
  // z0 = r cot theta0 and 1/r0 for the gradients, in the working precision
  const G gr = G(r), gir = G(ir), gct = G(ct), gst = G(st);
  const G gist = G(1) / gst, gz0 = gr * gct * gist, gir0 = G(sr);
  const G gar = G(ar), gai = G(ai), gbr = G(br), gbi = G(bi);
  const G c = G(a.rfac0 * M_PI * a.inv_span);  // d theta0 / d r
  const G dz0dr = gct * gist - gr * c * gist * gist;
  G fc = G(1), dfcdr = G(0);
  if (a.switchflag && r > a.rmin0) {
    G sw, cw;
    sincospi_g(G((r - a.rmin0) * a.inv_span), &sw, &cw);
    fc = G(0.5) * (cw + G(1));
    dfcdr = G(-0.5 * M_PI * a.inv_span) * sw;
  }
  v[0] = gar;
  v[1] = gai;
  v[2] = gbr;
  v[3] = gbi;
  v[4] = fc;
  const G rv[3] = {G(x), G(y), G(z)};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const G ud = rv[d] * gir;
    const G dz0 = dz0dr * ud;
    const G dr0 = (gr * ud + gz0 * dz0) * gir0;
    v[5 + d] = dfcdr * ud;
    // d a = (d(z0 - i z) - a d r0) / r0 ; d b = (d(y - i x) - b d r0) / r0
    v[8 + 2 * d] = (dz0 - gar * dr0) * gir0;
    v[9 + 2 * d] = ((d == 2 ? G(-1) : G(0)) - gai * dr0) * gir0;
    v[14 + 2 * d] = ((d == 1 ? G(1) : G(0)) - gbr * dr0) * gir0;
    v[15 + 2 * d] = ((d == 0 ? G(-1) : G(0)) - gbi * dr0) * gir0;
  }
#pragma unroll
  for (int e = 0; e < kGeomStride; ++e) g[e] = v[e];
}

// Slot of (k, i, -img) in k's list, or -1.  All of k's slots are read with
// independent loads (no early exit).
__device__ __forceinline__ int slot_rev(const WorkArgs& a, int i, long q) {
  const int k = a.nbr[q];
  const int sx = a.img[3 * q], sy = a.img[3 * q + 1], sz = a.img[3 * q + 2];
  const int ck = min(a.cnt[k], a.K);
  const int* kn = a.nbr + (long)k * a.K;
  int found = -1;
  for (int t0 = 0; t0 < ck; t0 += 8) {
    int nb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) nb[u] = (t0 + u < ck) ? kn[t0 + u] : -1;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (nb[u] == i && found < 0) {
        const long p = (long)k * a.K + t0 + u;
        if (a.img[3 * p] == -sx && a.img[3 * p + 1] == -sy && a.img[3 * p + 2] == -sz) found = t0 + u;
      }
    }
  }
  return found;
}

// Geometry and reverse slot of atom i's slots s = first, first + stride, ...
template <typename G>
__device__ void atom_slots(const WorkArgs& a, int i, int first, int stride) {
  const int cnt = a.cnt[i];
  for (int s = first; s < cnt; s += stride) {
    const long q = (long)i * a.K + s;
    const int r = slot_rev(a, i, q);
    a.rev_out[q] = r;
    if (r < 0) atomicMax(&a.flags[1], 1);
    slot_geom<G>(a, q);
  }
}

}  // namespace geo
}  // namespace snap

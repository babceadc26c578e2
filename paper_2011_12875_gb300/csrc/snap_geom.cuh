// snap_geom.cuh -- per-slot Cayley-Klein geometry (computed where the
// slot's separation is at hand: the fused neighbour build, or the compute_U
// kernels for caller-supplied lists) and the reverse-slot search.
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
// atomics); a missing opposite pair raises flags[1].  The force kernel finds
// it from the pair keys the neighbour build stores (find_rev_key) and keeps
// it for the weighted gather.
#pragma once
#include <math.h>

#include "snap_internal.h"

namespace snap {
namespace geo {

// Geometry of slot q into geom[q][0..kGeomStride): a (2), b (2), f_c,
// grad f_c (3), da/dr_d (3 x 2), db/dr_d (3 x 2).
// With `abf` given, a (2), b (2) and f_c are also written there (the
// compute_U kernel keeps its atom's in shared memory).
//
// FP64 work is kept to what the Cayley-Klein parameters need: r, theta0,
// sin/cos theta0, a and b.  In the mixed path (G = float) everything else --
// f_c and the gradients, which only feed the FP32 recursions -- is computed
// in FP32 from the rounded separation, so an FP64 instruction (1/64 of the
// FP32 rate here, whatever its active lanes) is spent only on those.
template <typename G>
__device__ void pair_geom(const WorkArgs& a, long q, double x, double y, double z, G* abf = nullptr) {
  G* g = reinterpret_cast<G*>(a.geom) + q * kGeomStride;
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
    if (abf)
#pragma unroll
      for (int e = 0; e < 5; ++e) abf[e] = v[e];
    return;
  }
  // r0 = sqrt(r^2 + z0^2) = r / |sin theta0|, so with sr = |sin theta0| / r
  //   a = z0 / r0 - i z / r0 = sign(sin theta0) cos theta0 - i z sr,
  //   b = (y - i x) / r0     = y sr - i x sr
  // (no division, one reciprocal square root; sr multiplies +-x, +-y, +-z, so
  // the opposite slot still gets exactly conj(a) and -b)
  double st, ct;
  sincospi((r - a.rmin0) * a.th_scale, &st, &ct);
  const double sr = fabs(st) * ir;
  const double ar = st < 0.0 ? -ct : ct, ai = -z * sr;
  const double br = y * sr, bi = -x * sr;
  const G gar = G(ar), gai = G(ai), gbr = G(br), gbi = G(bi);
  const G rv[3] = {G(x), G(y), G(z)};
  G gr, gir, gct, gst, c, fc = G(1), dfcdr = G(0);
  if constexpr (sizeof(G) == 4) {
    // the gradient factors in FP32 from the rounded separation
    const float fr2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
    gir = rsqrtf(fr2);
    gr = fr2 * gir;
    sincospif((gr - a.rmin0_f) * a.th_scale_f, &gst, &gct);
    c = a.dth_f;
    if (a.switchflag && gr > a.rmin0_f) {
      float sw, cw;
      sincospif((gr - a.rmin0_f) * a.inv_span_f, &sw, &cw);
      fc = 0.5f * (cw + 1.0f);
      dfcdr = a.dfc_f * sw;
    }
  } else {
    gr = r;
    gir = ir;
    gct = ct;
    gst = st;
    c = M_PI * a.th_scale;  // d theta0 / d r
    if (a.switchflag && r > a.rmin0) {
      double sw, cw;
      sincospi((r - a.rmin0) * a.inv_span, &sw, &cw);
      fc = 0.5 * (cw + 1.0);
      dfcdr = -0.5 * M_PI * a.inv_span * sw;
    }
  }
  // z0 = r cot theta0, 1/r0 = |sin theta0| / r
  const G gist = G(1) / gst, gz0 = gr * gct * gist, gir0 = fabs(gst) * gir;
  const G dz0dr = gct * gist - gr * c * gist * gist;
  v[0] = gar;
  v[1] = gai;
  v[2] = gbr;
  v[3] = gbi;
  v[4] = fc;
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
  if (abf)
#pragma unroll
    for (int e = 0; e < 5; ++e) abf[e] = v[e];
}

// The same for slot q from its stored separation.
template <typename G>
__device__ __forceinline__ void slot_geom(const WorkArgs& a, long q, G* abf = nullptr) {
  pair_geom<G>(a, q, a.rij[3 * q], a.rij[3 * q + 1], a.rij[3 * q + 2], abf);
}

// Slot of (k, i, -img_q) in k's list (k = nbr[q]), or -1.  k's row of the
// table is read with independent loads (16-byte loads when the capacity is a
// multiple of 4, 32 entries a round), and the image of each entry equal to i
// is checked (usually one).
__device__ __forceinline__ int find_rev(const WorkArgs& a, int i, long q, int k) {
  const int K = a.K;
  const int ck = min(a.cnt[k], K);
  const int* kn = a.nbr + (long)k * K;
  const int sx = a.img[3 * q], sy = a.img[3 * q + 1], sz = a.img[3 * q + 2];
  int found = -1;
  for (int t0 = 0; t0 < ck; t0 += 32) {
    int nb[32];
    if ((K & 3) == 0) {
      const int4* row = reinterpret_cast<const int4*>(kn + t0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int4 v = (t0 + 4 * u < ck) ? __ldg(row + u) : make_int4(-1, -1, -1, -1);
        nb[4 * u] = v.x;
        nb[4 * u + 1] = v.y;
        nb[4 * u + 2] = v.z;
        nb[4 * u + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 32; ++u) nb[u] = (t0 + u < ck) ? __ldg(kn + t0 + u) : -1;
    }
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      if (nb[u] == i && t0 + u < ck && found < 0) {
        const long p = (long)k * K + t0 + u;
        if (a.img[3 * p] == -sx && a.img[3 * p + 1] == -sy && a.img[3 * p + 2] == -sz) found = t0 + u;
      }
    }
  }
  return found;
}

// The same from the pair keys (pair_key): with key kq of slot q (k, s) the
// reverse slot is the entry of k's row equal to i * 32 + 26 - (kq & 31), one
// pass of 16-byte loads over the row; a slot without a key (an image shift
// beyond one box) takes find_rev.
__device__ __forceinline__ int find_rev_key(const WorkArgs& a, int i, long q, int k, int kq) {
  const int K = a.K;
  if (kq < 0 || (K & 3) != 0) return find_rev(a, i, q, k);
  const int want = i * 32 + 26 - (kq & 31);
  const int ck = min(a.cnt[k], K);
  const int4* row = reinterpret_cast<const int4*>(a.key + (long)k * K);
  int found = -1;
  for (int t0 = 0; t0 < ck; t0 += 32) {
    int4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (t0 + 4 * u < ck) ? __ldg(row + t0 / 4 + u) : make_int4(-1, -1, -1, -1);
#pragma unroll
    for (int u = 7; u >= 0; --u) {
      const int b = t0 + 4 * u;
      if (v[u].w == want && b + 3 < ck) found = b + 3;
      if (v[u].z == want && b + 2 < ck) found = b + 2;
      if (v[u].y == want && b + 1 < ck) found = b + 1;
      if (v[u].x == want && b < ck) found = b;
    }
    if (found >= 0) break;
  }
  return found;
}

// Geometry of atom i's slots s = first, first + stride, ...
template <typename G>
__device__ void atom_geom(const WorkArgs& a, int i, int first, int stride) {
  const int cnt = a.cnt[i];
  for (int s = first; s < cnt; s += stride) slot_geom<G>(a, (long)i * a.K + s);
}

}  // namespace geo
}  // namespace snap

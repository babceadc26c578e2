// snap_colkernels.cuh -- compute_U and the fused dU + dE/dr kernel with the
// layer recursion held in registers, one lane per half-matrix column.
//
// Eq. (hysphrecur) of arXiv:2011.12875 builds u_t from u_{t-1}; element
// (ma, mb) only reads elements (ma, mb) and (ma-1, mb) of the previous layer,
// so every column mb evolves on its own:
//   u_t[ma][mb] = sqrt((t-ma)/(t-mb)) conj(a) u_{t-1}[ma][mb]
//               - sqrt(ma/(t-mb))     conj(b) u_{t-1}[ma-1][mb].
// Column mb enters the stored half at layer t = 2 mb, from column mb of layer
// t-1, which is the mirror of column mb-1 of that layer:
//   u_{t-1}[m][mb] = (-1)^(m+mb) conj(u_{t-1}[t-1-m][mb-1]).
// Here one lane carries one column of one neighbour pair through all layers
// (twojmax/2 + 1 lanes per pair, several pairs per warp); the layer loop is
// unrolled at compile time, so the column lives in registers and the seed is
// one warp shuffle per element.  This file is included by one translation
// unit per working precision.
#pragma once
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "snap_geom.cuh"
#include "snap_internal.h"
#include "snap_neigh.cuh"

namespace snap {
namespace col {

constexpr unsigned kFull = 0xffffffffu;

template <typename R>
struct __align__(2 * sizeof(R)) c2 {
  R re, im;
};

template <typename R>
__device__ __forceinline__ c2<R> mk(R re, R im) {
  c2<R> c;
  c.re = re;
  c.im = im;
  return c;
}

// sqrt(k) for the small integers of the recursion, folded at compile time.
template <typename R>
__device__ __forceinline__ constexpr R sqrt_int(int k) {
  return k == 0   ? R(0)
         : k == 1 ? R(1)
         : k == 2 ? R(1.4142135623730950488)
         : k == 3 ? R(1.7320508075688772935)
         : k == 4 ? R(2)
         : k == 5 ? R(2.2360679774997896964)
         : k == 6 ? R(2.4494897427831780982)
         : k == 7 ? R(2.6457513110645905905)
         : k == 8 ? R(2.8284271247461900976)
         : k == 9 ? R(3)
         : k == 10 ? R(3.1622776601683793320)
         : k == 11 ? R(3.3166247903553998491)
         : k == 12 ? R(3.4641016151377545871)
         : k == 13 ? R(3.6055512754639892931)
         : k == 14 ? R(3.7416573867739413856)
                   : R(3.8729833462074168852);
}

// Compile-time loop B..E (inclusive): f(std::integral_constant<int, k>).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B <= E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

template <typename R>
__device__ __forceinline__ R shfl_up(R v) {
  return __shfl_up_sync(kFull, v, 1);
}

// Weight of a half-layout element in a full-matrix contraction (see
// snap_kernels.cu): 2 below the middle column, on it 2 / 1 / 0.
__device__ __forceinline__ int hweight(int t, int ma, int mb) {
  if (2 * mb < t) return 2;
  return ma < mb ? 2 : (ma == mb ? 1 : 0);
}

// Lane layout: NC = J2/2 + 1 lanes per pair, P pairs per warp.
template <int J2>
struct Shape {
  static constexpr int NC = J2 / 2 + 1;
  static constexpr int P = 32 / NC;
};

// Replace column mc = t/2 (on the lane with mb == mc) by the mirror of the
// column held one lane below, for layer t-1 (length t).
template <typename R, int T, int N>
__device__ __forceinline__ void seed_column(c2<R> (&v)[N], bool take) {
  constexpr int mc = T / 2;
  c2<R> src[T];
#pragma unroll
  for (int k = 0; k < T; ++k) {
    src[k].re = shfl_up(v[k].re);
    src[k].im = shfl_up(v[k].im);
  }
  if (take) {
#pragma unroll
    for (int m = 0; m < T; ++m) {
      const R s = (((T - 1 - m) + (mc - 1)) & 1) ? R(-1) : R(1);
      v[m] = mk<R>(s * src[T - 1 - m].re, -s * src[T - 1 - m].im);
    }
  }
}

// ------------------------------------------- scaled layer recursion
// With u_t[ma][mb] = S_t(ma, mb) v_t[ma][mb], S_t(ma, mb) =
// sqrt((t - ma)! ma! / (t - mb)!), the recursion of Eq. (hysphrecur) becomes
//   v_t[ma] = conj(a) v_{t-1}[ma] - conj(b) v_{t-1}[ma-1]
// (S_t(ma, mb) = sqrt((t-ma)/(t-mb)) S_{t-1}(ma, mb) = sqrt(ma/(t-mb))
// S_{t-1}(ma-1, mb) absorbs both root factors): 8 real operations an element
// instead of 12.  S splits into sqrt((t - ma)! ma!), a constant of the
// unrolled element, and 1 / sqrt((t - mb)!), one value per lane and layer.
// The mirror that seeds column mc at layer 2 mc - 1 picks up S's ratio
// between the two columns, 1 / sqrt(mc).
__host__ __device__ constexpr double c_fact(int n) { return n <= 1 ? 1.0 : n * c_fact(n - 1); }
__host__ __device__ constexpr double c_sqrt_iter(double x, double y, int k) {
  return k == 0 ? y : c_sqrt_iter(x, 0.5 * (y + x / y), k - 1);
}
// square root of x >= 1 by Newton's iteration from x (64 steps: converged
// for every argument below 2^64)
__host__ __device__ constexpr double c_sqrt(double x) { return x <= 1.0 ? 1.0 : c_sqrt_iter(x, x, 64); }
template <int T, int MA>
__host__ __device__ constexpr double v_scale() { return c_sqrt(c_fact(T - MA) * c_fact(MA)); }

// x * y + z, one rounding (the sums below are written as chains of these:
// a component of a complex multiply-add is two fused operations, where
// x += a*b + c*d would round a product, a fused sum and an addition)
template <typename R>
__device__ __forceinline__ R fm(R x, R y, R z) {
  if constexpr (sizeof(R) == 4) return fmaf(x, y, z);
  else return fma(x, y, z);
}

// One layer of the scaled recursion on a lane's column, in place, ma
// descending; A = conj(a), B = conj(b).  An element is four fused
// multiply-adds a component.
template <typename R, int T, int N>
__device__ __forceinline__ void v_layer(c2<R> (&v)[N], const c2<R> A, const c2<R> B) {
  static_assert(T < N, "column too short");
  c2<R> w = mk<R>(fm(B.im, v[T - 1].im, -(B.re * v[T - 1].re)), fm(-B.im, v[T - 1].re, -(B.re * v[T - 1].im)));
  v[T] = w;
#pragma unroll
  for (int ma = T - 1; ma >= 1; --ma) {
    const c2<R> x = v[ma], y = v[ma - 1];
    w.re = fm(B.im, y.im, fm(-B.re, y.re, fm(-A.im, x.im, A.re * x.re)));
    w.im = fm(-B.im, y.re, fm(-B.re, y.im, fm(A.im, x.re, A.re * x.im)));
    v[ma] = w;
  }
  v[0] = mk<R>(fm(-A.im, v[0].im, A.re * v[0].re), fm(A.im, v[0].re, A.re * v[0].im));
}

// Seed of column T / 2 (lanes with take) for layer T - 1 in the scaled form:
// the mirror of the column one lane below, times 1 / sqrt(T / 2).
template <typename R, int T, int N>
__device__ __forceinline__ void v_seed(c2<R> (&v)[N], bool take) {
  constexpr int mc = T / 2;
  constexpr double qd = 1.0 / c_sqrt(double(mc));
  const R q = R(qd);
  c2<R> src[T];
#pragma unroll
  for (int k = 0; k < T; ++k) {
    src[k].re = shfl_up(v[k].re);
    src[k].im = shfl_up(v[k].im);
  }
  if (take) {
#pragma unroll
    for (int m = 0; m < T; ++m) {
      const R sq = (((T - 1 - m) + (mc - 1)) & 1) ? -q : q;
      v[m] = mk<R>(sq * src[T - 1 - m].re, -sq * src[T - 1 - m].im);
    }
  }
}

// 1 / sqrt((t - mb)!) for t = 0..J2 (0 below mb), once per warp.
template <typename R, int J2>
__device__ __forceinline__ void v_gscale(R (&gs)[J2 + 1], int mb) {
  R f = R(1);
  const R mbr = R(mb);
#pragma unroll
  for (int t = 0; t <= J2; ++t) {
    if (t > mb) f *= R(t) - mbr;
    gs[t] = (t >= mb) ? R(1) / sqrt(f) : R(0);
  }
}

// ------------------------------------------------------------- compute_U
// An atom's pairs are taken in passes of P pairs (a lane per column of a
// pair); f_c u_t of a pass is summed over its pair groups in two steps:
//  * LV levels of shuffles first add the groups g, g + 1, ..., g + 2^LV - 1
//    on the lanes of group g (a multiple of 2^LV), which leaves
//    CPW = ceil(P / 2^LV) partial sums of each element;
//  * those lanes store their partial sums (CPW copies of the half matrix) in
//    the warp's scratch, and after the pass each lane adds the copies of the
//    elements e = lane, lane + 32, ... to the warp's running sum.
// LV is the fewest levels that keep the scratch under 4 KB in FP32 (2J = 8:
// one level, three copies) and none in FP64, whose pipe, not the shuffles'
// latency, bounds that path.  Q warps share an atom (warp q takes passes q,
// q + Q, ...), and the atom's Ulisttot is the sum of the Q running sums plus
// w_self on the diagonal.  Q, LV and P are constants of the instance, so the
// order of every sum is fixed by the slot indices alone.
template <typename R, int J2>
struct UiPlan {
  static constexpr int NC = Shape<J2>::NC, P = Shape<J2>::P;
  static constexpr int HH = half_size(J2);
  static constexpr int kMaxLv = P > 16 ? 5 : P > 8 ? 4 : P > 4 ? 3 : P > 2 ? 2 : P > 1 ? 1 : 0;
  static constexpr int copies(int lv) { return (P + (1 << lv) - 1) >> lv; }
  static constexpr int pick(int lv) {
    return (sizeof(R) == 8 || lv >= kMaxLv || copies(lv) * HH * (int)sizeof(c2<R>) <= 4096) ? lv : pick(lv + 1);
  }
  static constexpr int LV = pick(0);
  static constexpr int CPW = copies(LV);
  static constexpr int Q = (26 + P - 1) / P >= 2 ? 2 : 1;  // warps per atom
  static constexpr int A = Q == 1 ? 2 : 1;                  // atoms per CTA
  static constexpr size_t warp_bytes = sizeof(c2<R>) * (size_t)(CPW + 1) * HH;
};

// Sum of v over the pair groups g, g + 1, ..., g + 2^LV - 1 (on the lanes of
// writer groups; lanes past the warp add nothing).
template <int LV, int NC, typename R>
__device__ __forceinline__ R group_sum(R v, int lane) {
#pragma unroll
  for (int l = 0; l < LV; ++l) {
    const R o = __shfl_down_sync(kFull, v, NC << l);
    if (lane + (NC << l) < 32) v += o;
  }
  return v;
}

// The passes of one warp of an atom (warp wq of its Q): abf = the atom's
// [K][5] (a, b, f_c) in shared memory, scr = the warp's [CPW + 1][H] scratch
// (CPW partial sums of a pass, then the warp's running sum).
template <typename R, int J2>
__device__ __forceinline__ void u_passes(const R* __restrict__ abf, int cnt, int wq, int lane,
                                         c2<R>* __restrict__ scr) {
  using S = Shape<J2>;
  using UP = UiPlan<R, J2>;
  constexpr int NC = S::NC, P = S::P, LV = UP::LV, CPW = UP::CPW, Q = UP::Q, H = UP::HH;
  c2<R>* run = scr + (size_t)CPW * H;
  for (int e = lane; e < H; e += 32) run[e] = mk<R>(0, 0);
  const int g = lane / NC, mb = lane - g * NC;
  const bool grp = g < P;
  const bool writer = grp && (g & ((1 << LV) - 1)) == 0;
  c2<R>* my = scr + (size_t)(writer ? (g >> LV) : 0) * H;
  const int npass = (cnt + P - 1) / P;
  for (int pass = wq; pass < npass; pass += Q) {
    const int s = pass * P + g;
    const bool ok = grp && s < cnt;
    c2<R> ca = mk<R>(1, 0), cb = mk<R>(0, 0);
    R fc = 0;
    if (ok) {
      const R* gm = abf + 5 * s;
      ca = mk<R>(gm[0], -gm[1]);  // conj(a)
      cb = mk<R>(gm[2], -gm[3]);  // conj(b)
      fc = gm[4];
    }
    // the scaled column times f_c (the recursion is linear, so f_c rides
    // along from layer 0); S is applied once, to the atom's sums
    c2<R> v[J2 + 1];
#pragma unroll
    for (int k = 0; k <= J2; ++k) v[k] = mk<R>(0, 0);
    if (mb == 0) v[0] = mk<R>(fc, 0);
    {
      const R v0 = group_sum<LV, NC>(v[0].re, lane);
      if (writer && mb == 0) my[0] = mk<R>(v0, 0);
    }
    static_for<1, J2>([&](auto tc) {
      constexpr int t = decltype(tc)::value;
      if constexpr ((t & 1) == 0) v_seed<R, t>(v, mb == t / 2);
      v_layer<R, t>(v, ca, cb);
      c2<R>* dst = my + half_base(t) + mb * (t + 1);
#pragma unroll
      for (int ma = 0; ma <= t; ++ma) {
        const R vr = group_sum<LV, NC>(v[ma].re, lane);
        const R vi = group_sum<LV, NC>(v[ma].im, lane);
        if (writer && 2 * mb <= t) dst[ma] = mk<R>(vr, vi);
      }
    });
    __syncwarp();
    for (int e = lane; e < H; e += 32) {
      c2<R> v = run[e];
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const c2<R> w = scr[(size_t)c * H + e];
        v.re += w.re;
        v.im += w.im;
      }
      run[e] = v;
    }
    __syncwarp();
  }
}

// Ulisttot of atom i from its Q warps' running sums (ascr = the atom's
// [Q][CPW + 1][H] scratch): their sum in warp order, times S, plus w_self on
// the diagonal; elements e0, e0 + estride, ...
template <typename R, int J2>
__device__ __forceinline__ void u_store(const WorkArgs& a, const c2<R>* __restrict__ ascr, long i, int e0,
                                        int estride) {
  using UP = UiPlan<R, J2>;
  constexpr int CPW = UP::CPW, Q = UP::Q, H = UP::HH;
  c2<R>* Ug = reinterpret_cast<c2<R>*>(a.U);
  for (int e = e0; e < H; e += estride) {
    const c2<R>* rr = ascr + (size_t)CPW * H + e;
    R sr = 0, si = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const c2<R> v = rr[(size_t)q * (CPW + 1) * H];
      sr += v.re;
      si += v.im;
    }
    const R sc = reinterpret_cast<const R*>(a.hscale)[e];
    sr *= sc;
    si *= sc;
    const int p = a.half_tmm[e];
    if (tmm_ma(p) == tmm_mb(p)) sr += (R)a.wself;
    Ug[((i >> 5) * H + e) * 32 + (i & 31)] = mk<R>(sr, si);
  }
}

// Resident CTAs an SM the register allocation is sized for: 16 two-warp CTAs
// (64 registers) in FP32 up to 2J = 8, 8 above and in FP64.
template <typename R, int J2>
constexpr int ui_min_ctas() { return sizeof(R) == 8 ? 8 : (J2 <= 8 ? 16 : 8); }

// compute_U for a neighbour table built elsewhere (caller-supplied lists):
// CTA = A atoms of Q warps; the atom's first warp evaluates the slot
// geometry from the stored separations (dense lanes), then the passes.
template <typename R, int J2>
__global__ void __launch_bounds__(64, ui_min_ctas<R, J2>()) ui_col_kernel(WorkArgs a) {
  using UP = UiPlan<R, J2>;
  constexpr int Q = UP::Q, A = UP::A;
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = a.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int al = warp / Q, wq = warp - al * Q;
  const long i0 = (long)blockIdx.x * A;
  const long i = i0 + al;
  const bool have = i < a.n;  // warp-uniform
  c2<R>* scr = reinterpret_cast<c2<R>*>(smem) + (size_t)warp * (UP::CPW + 1) * UP::HH;
  R* myabf = reinterpret_cast<R*>(smem + (size_t)A * Q * UP::warp_bytes) + (size_t)al * K * 5;
  const int cnt = have ? a.cnt[i] : 0;
  if (have && wq == 0)
    for (int s = lane; s < cnt; s += 32) geo::slot_geom<R>(a, i * K + s, myabf + 5 * s);
  __syncthreads();
  if (have) u_passes<R, J2>(myabf, cnt, wq, lane, scr);
  __syncthreads();
  for (int a2 = 0; a2 < A; ++a2) {
    if (i0 + a2 >= a.n) break;
    u_store<R, J2>(a, reinterpret_cast<const c2<R>*>(smem) + (size_t)a2 * Q * (UP::CPW + 1) * UP::HH, i0 + a2,
                   threadIdx.x, blockDim.x);
  }
}

// ---------------------------------------- neighbour build fused with compute_U
// The neighbour build of snap_neigh.cuh (two atoms a CTA, SPLIT warps each)
// and, in the same CTA, compute_U of those atoms: each stored pair's slot
// geometry is evaluated on the lane that accepts it, from the exact FP64
// separation in its registers (dense lanes, no reload), with a, b and f_c
// kept in shared memory; then the first Q warps of each atom take its
// passes.  One launch and one pass over the pairs instead of two.
template <bool BATCH>
struct NuShape {
  static constexpr int SPLIT = BATCH ? 4 : 2;  // build warps per atom
  static constexpr int NW = 2 * SPLIT;         // warps per CTA (two atoms)
};

template <typename R, int J2, bool BATCH>
__global__ void __launch_bounds__(NuShape<BATCH>::NW * 32) neigh_u_kernel(NeighArgs na, WorkArgs a) {
  using UP = UiPlan<R, J2>;
  constexpr int SPLIT = NuShape<BATCH>::SPLIT, NW = NuShape<BATCH>::NW, Q = UP::Q;
  static_assert(Q <= SPLIT, "an atom's passes run on its build warps");
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = a.K;
  R* abf = reinterpret_cast<R*>(smem + (size_t)2 * Q * UP::warp_bytes);  // [2][K][5]
  nb::neigh_build_cta<BATCH, SPLIT, NW>(na, [&](int al, long i, int slot, long q, double ex, double ey,
                                               double ez) {
    (void)i;
    geo::pair_geom<R>(a, q, ex, ey, ez, abf + ((size_t)al * K + slot) * 5);
  });
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int al = warp / SPLIT, wq = warp - al * SPLIT;
  long i, hi;
  if (BATCH) {
    const int2 m = na.cta_map[blockIdx.x];
    const NeighConf c = na.confs[m.x];
    i = c.start + m.y + al;
    hi = c.start + c.n;
  } else {
    i = (long)blockIdx.x * 2 + al;
    hi = na.n;
  }
  const bool have = i < hi;
  c2<R>* ascr = reinterpret_cast<c2<R>*>(smem) + (size_t)al * Q * (UP::CPW + 1) * UP::HH;
  if (have && wq < Q)
    u_passes<R, J2>(abf + (size_t)al * K * 5, min(na.cnt[i], K), wq, lane,
                    ascr + (size_t)wq * (UP::CPW + 1) * UP::HH);
  __syncthreads();
  if (have) u_store<R, J2>(a, ascr, i, wq * 32 + lane, SPLIT * 32);
}

// ------------------------------------------- tangent of Ulisttot along g
// Forward-mode derivative of Eq. (u) along a displacement field g of the
// atoms: the pair (i, k) moves by delta = g_k - g_i, so
//   dU_t = sum_k d/de [ f_c(r_ik + e delta) u_t(r_ik + e delta) ] at e = 0
//        = sum_k (grad f_c . delta) u_t + f_c (du_t/dr . delta).
// In the scaled form w = f_c v (u = S v): w_t = conj(a) w_{t-1}[ma] -
// conj(b) w_{t-1}[ma-1] from w_0 = f_c, and its tangent
//   dw_t = conj(da) w[ma] + conj(a) dw[ma] - conj(db) w[ma-1] - conj(b) dw[ma-1]
// from dw_0 = grad f_c . delta, so dU_t = S sum_k dw_t (no w_self).  Launch
// shape, reduction and order of the sums as compute_U (UiPlan).
template <typename R, int J2>
__device__ __forceinline__ void du_passes(const R* __restrict__ tg, int cnt, int wq, int lane,
                                          c2<R>* __restrict__ scr) {
  using S = Shape<J2>;
  using UP = UiPlan<R, J2>;
  constexpr int NC = S::NC, P = S::P, LV = UP::LV, CPW = UP::CPW, Q = UP::Q, H = UP::HH;
  c2<R>* run = scr + (size_t)CPW * H;
  for (int e = lane; e < H; e += 32) run[e] = mk<R>(0, 0);
  const int g = lane / NC, mb = lane - g * NC;
  const bool grp = g < P;
  const bool writer = grp && (g & ((1 << LV) - 1)) == 0;
  c2<R>* my = scr + (size_t)(writer ? (g >> LV) : 0) * H;
  const int npass = (cnt + P - 1) / P;
  for (int pass = wq; pass < npass; pass += Q) {
    const int s = pass * P + g;
    const bool ok = grp && s < cnt;
    c2<R> ca = mk<R>(1, 0), cb = mk<R>(0, 0), cda = mk<R>(0, 0), cdb = mk<R>(0, 0);
    R fc = 0, dfc = 0;
    if (ok) {  // [10]: a, b, f_c, d f_c, da, db along delta
      const R* t = tg + 10 * s;
      ca = mk<R>(t[0], -t[1]);
      cb = mk<R>(t[2], -t[3]);
      fc = t[4];
      dfc = t[5];
      cda = mk<R>(t[6], -t[7]);
      cdb = mk<R>(t[8], -t[9]);
    }
    c2<R> w[J2 + 1], dw[J2 + 1];
#pragma unroll
    for (int k = 0; k <= J2; ++k) w[k] = dw[k] = mk<R>(0, 0);
    if (mb == 0) {
      w[0] = mk<R>(fc, 0);
      dw[0] = mk<R>(dfc, 0);
    }
    {
      const R v0 = group_sum<LV, NC>(dw[0].re, lane);
      if (writer && mb == 0) my[0] = mk<R>(v0, 0);
    }
    static_for<1, J2>([&](auto tc) {
      constexpr int t = decltype(tc)::value;
      if constexpr ((t & 1) == 0) {
        v_seed<R, t>(w, mb == t / 2);
        v_seed<R, t>(dw, mb == t / 2);
      }
      // dw first (it reads the old w), then w
#pragma unroll
      for (int ma = t; ma >= 0; --ma) {
        c2<R> y = mk<R>(0, 0);
        if (ma < t) {
          const c2<R> p = w[ma], q = dw[ma];
          y.re = fm(-ca.im, q.im, fm(ca.re, q.re, fm(-cda.im, p.im, fm(cda.re, p.re, y.re))));
          y.im = fm(ca.im, q.re, fm(ca.re, q.im, fm(cda.im, p.re, fm(cda.re, p.im, y.im))));
        }
        if (ma > 0) {
          const c2<R> p = w[ma - 1], q = dw[ma - 1];
          y.re = fm(cb.im, q.im, fm(-cb.re, q.re, fm(cdb.im, p.im, fm(-cdb.re, p.re, y.re))));
          y.im = fm(-cb.im, q.re, fm(-cb.re, q.im, fm(-cdb.im, p.re, fm(-cdb.re, p.im, y.im))));
        }
        dw[ma] = y;
      }
      v_layer<R, t>(w, ca, cb);
      c2<R>* dst = my + half_base(t) + mb * (t + 1);
#pragma unroll
      for (int ma = 0; ma <= t; ++ma) {
        const R vr = group_sum<LV, NC>(dw[ma].re, lane);
        const R vi = group_sum<LV, NC>(dw[ma].im, lane);
        if (writer && 2 * mb <= t) dst[ma] = mk<R>(vr, vi);
      }
    });
    __syncwarp();
    for (int e = lane; e < H; e += 32) {
      c2<R> v = run[e];
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const c2<R> q = scr[(size_t)c * H + e];
        v.re += q.re;
        v.im += q.im;
      }
      run[e] = v;
    }
    __syncwarp();
  }
}

template <typename R, int J2>
__global__ void __launch_bounds__(64, ui_min_ctas<R, J2>()) tan_col_kernel(WorkArgs a, const double* __restrict__ gd,
                                                                         void* dUout) {
  using UP = UiPlan<R, J2>;
  constexpr int Q = UP::Q, A = UP::A, CPW = UP::CPW, H = UP::HH;
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = a.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int al = warp / Q, wq = warp - al * Q;
  const long i0 = (long)blockIdx.x * A;
  const long i = i0 + al;
  const bool have = i < a.n;  // warp-uniform
  c2<R>* scr = reinterpret_cast<c2<R>*>(smem) + (size_t)warp * (CPW + 1) * H;
  R* tg = reinterpret_cast<R*>(smem + (size_t)A * Q * UP::warp_bytes) + (size_t)al * K * 10;
  const int cnt = have ? a.cnt[i] : 0;
  if (have && wq == 0)  // the pair data along delta = g_k - g_i, a lane per slot
    for (int s = lane; s < cnt; s += 32) {
      const long slot = i * K + s;
      const R* gm = reinterpret_cast<const R*>(a.geom) + slot * kGeomStride;
      const int k = a.nbr[slot];
      R dl[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) dl[d] = (R)(gd[3 * (long)k + d] - gd[3 * i + d]);
      R dfc = 0, ar = 0, ai = 0, br = 0, bi = 0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        dfc += dl[d] * gm[5 + d];
        ar += dl[d] * gm[8 + 2 * d];
        ai += dl[d] * gm[9 + 2 * d];
        br += dl[d] * gm[14 + 2 * d];
        bi += dl[d] * gm[15 + 2 * d];
      }
      R* t = tg + 10 * s;
      t[0] = gm[0];
      t[1] = gm[1];
      t[2] = gm[2];
      t[3] = gm[3];
      t[4] = gm[4];
      t[5] = dfc;
      t[6] = ar;
      t[7] = ai;
      t[8] = br;
      t[9] = bi;
    }
  __syncthreads();
  if (have) du_passes<R, J2>(tg, cnt, wq, lane, scr);
  __syncthreads();
  c2<R>* Ug = reinterpret_cast<c2<R>*>(dUout);
  for (int a2 = 0; a2 < A; ++a2) {
    const long ii = i0 + a2;
    if (ii >= a.n) break;
    const c2<R>* rr = reinterpret_cast<const c2<R>*>(smem) + (size_t)a2 * Q * (CPW + 1) * H + (size_t)CPW * H;
    for (int e = threadIdx.x; e < H; e += blockDim.x) {
      R sr = 0, si = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const c2<R> v = rr[(size_t)q * (CPW + 1) * H + e];
        sr += v.re;
        si += v.im;
      }
      const R sc = reinterpret_cast<const R*>(a.hscale)[e];
      Ug[((ii >> 5) * H + e) * 32 + (ii & 31)] = mk<R>(sr * sc, si * sc);
    }
  }
}

template <typename R>
constexpr int de_max_warps() { return sizeof(R) == 4 ? 16 : 8; }

// --------------------------------------- fused dU + dE/dr, reverse mode
// Same lane layout (P pairs a warp, a lane per column); the CTA's atoms have
// their weighted Y_i in shared memory (launch shape below).
// For one pair, S(a, b) = Re sum_t Y_t : conj(u_t) is a real function of the
// Cayley-Klein parameters; its gradient comes from one
// forward pass of the recursion (each lane stores its column of every layer
// in shared memory) and one adjoint pass through the same recursion, with
// the adjoint lambda_t of a column in registers:
//   lambda_{t-1}[m][mb] = Yw_{t-1}[m][mb] + a A - b B,
//   A = sqrt((t-m)/(t-mb)) lambda_t[m][mb],  B = sqrt((m+1)/(t-mb)) lambda_t[m+1][mb],
//   g_a += conj(A) u_{t-1}[m][mb],           g_b -= conj(B) u_{t-1}[m][mb],
// plus, for even t, the part of layer t's column t/2 that read the mirror of
// column t/2-1 (its adjoint comes one lane down by shuffle).  Then
//   dE_i/dr_ik = S grad f_c + f_c (<g_a, da/dr> + <g_b, db/dr>)   (Eq. snapforce2).
template <typename R>
__device__ __forceinline__ R shfl_down(R v) {
  return __shfl_down_sync(kFull, v, 1);
}

// FP32: 128 registers (up to 16 warps a CTA); FP64 may use them all, up to 8
// warps (its FP64 pipe saturates with few warps, and the columns are twice
// the size).
//
// CTA = A consecutive atoms and NW warps (A is a launch parameter, planned
// by launch_de_rev_col_t).  The CTA's pairs, atom after atom, are taken in
// passes of P pairs; warp w takes passes w, w + NW, ...  Every pass but the
// CTA's last is full whatever the atoms' counts, and with A below NW x
// (passes per warp) x P / (pairs per atom) no warp takes more passes than
// planned (the time of a CTA is that of its longest chain of passes).  A
// pair's arithmetic does not depend on its pass or its warp.
//
// QUEUE: a persistent launch over a work queue -- a grid of resident CTAs,
// each taking CTA-sized items (A consecutive atoms) from a device counter
// (flags[6], zeroed with the flags by every evaluation) until they run out;
// an item's arithmetic is that of the CTA it would have been.
template <typename R, int J2, bool QUEUE>
__global__ void __launch_bounds__(de_max_warps<R>() * 32, 1) de_rev_col_kernel(WorkArgs a, int A) {
  using S_ = Shape<J2>;
  constexpr int NC = S_::NC, P = S_::P;
  const int NW = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long item_s;
  const int H = a.H;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long nitems = (a.n + A - 1) / A;
  for (long item = blockIdx.x;;) {
  if (QUEUE) {
    if (threadIdx.x == 0) item_s = atomicAdd(&a.flags[6], 1);
    __syncthreads();
    item = item_s;
    if (item >= nitems) break;
  }
  const long i0 = item * A;  // the CTA's atoms i0 .. i0 + na - 1
  const int na = (int)min((long)A, a.n - i0);
  c2<R>* Ywa = reinterpret_cast<c2<R>*>(smem);                    // [A][H] weighted Y
  c2<R>* ust = Ywa + (size_t)A * H;                              // [NW*P][H] forward columns
  R* red = reinterpret_cast<R*>(ust + (size_t)NW * P * H);       // [NW][32][5]
  int* coff = reinterpret_cast<int*>(red + (size_t)NW * 32 * 5);  // [A+1] first pair of each atom
  const int g = lane / NC, mb = lane - g * NC;
  const bool grp = g < P;
  for (int al = warp; al < na; al += NW) {  // weighted Y of the CTA's atoms
    const long i = i0 + al;
    const c2<R>* Yg = reinterpret_cast<const c2<R>*>(a.Y);
    const long blk = i >> 5;
    const int li = (int)(i & 31);
    c2<R>* Yw = Ywa + (size_t)al * H;
    for (int e = lane; e < H; e += 32) {
      const int p = a.half_tmm[e];
      // the contraction weight times S of the scaled recursion (u = S v)
      const R w = (R)hweight(tmm_t(p), tmm_ma(p), tmm_mb(p)) * reinterpret_cast<const R*>(a.hscale)[e];
      const c2<R> y = Yg[(blk * H + e) * 32 + li];
      Yw[e] = mk<R>(w * y.re, w * y.im);
    }
  }
  if (warp == 0) {  // exclusive offsets of the atoms' pairs (inclusive scan, 32 at a time)
    int carry = 0;
    if (lane == 0) coff[0] = 0;
    for (int b = 0; b < na; b += 32) {
      int c = b + lane < na ? a.cnt[i0 + b + lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, c, o);
        if (lane >= o) c += u;
      }
      if (b + lane < na) coff[b + lane + 1] = carry + c;
      carry += __shfl_sync(kFull, c, 31);
    }
  }
  __syncthreads();
  const int total = coff[na];
  c2<R>* my = ust + (warp * P + (grp ? g : 0)) * H;
  R* myred = red + (warp * 32 + lane) * 5;
  for (int s0 = warp * P; s0 < total; s0 += NW * P) {
    const int f = s0 + g;
    const bool ok = grp && f < total;
    // the pair's atom: the last al with coff[al] <= f (empty atoms skipped)
    const int fk = min(f, total - 1);
    int lo = 0, hi = na - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (coff[mid] <= fk) lo = mid;
      else hi = mid - 1;
    }
    const long i = i0 + lo;
    const c2<R>* Yw = Ywa + (size_t)lo * H;
    const long slot = i * a.K + (ok ? f - coff[lo] : 0);
    const R* gm = reinterpret_cast<const R*>(a.geom) + slot * kGeomStride;
    c2<R> ka = mk<R>(1, 0), kb = mk<R>(0, 0);  // a and b
    if (ok) {
      ka = mk<R>(gm[0], gm[1]);
      kb = mk<R>(gm[2], gm[3]);
    }
    // ---- forward: the scaled columns v, stored per layer
    c2<R> u[J2 + 1];
#pragma unroll
    for (int k = 0; k <= J2; ++k) u[k] = mk<R>(0, 0);
    R Ssum = 0;
    if (mb == 0) {
      u[0] = mk<R>(1, 0);
      Ssum = Yw[0].re;
      if (grp) my[0] = u[0];  // lanes past the last pair group own no storage
    }
    // conj(a), conj(b)
    const c2<R> ca = mk<R>(ka.re, -ka.im), cb = mk<R>(kb.re, -kb.im);
    static_for<1, J2>([&](auto tc) {
      constexpr int t = decltype(tc)::value;
      if constexpr ((t & 1) == 0) v_seed<R, t>(u, mb == t / 2);
      v_layer<R, t>(u, ca, cb);
      if (grp && 2 * mb <= t) {
        c2<R>* dst = my + half_base(t) + mb * (t + 1);
        const c2<R>* yr = Yw + half_base(t) + mb * (t + 1);
#pragma unroll
        for (int ma = 0; ma <= t; ++ma) {
          dst[ma] = u[ma];
          Ssum = fm(yr[ma].im, u[ma].im, fm(yr[ma].re, u[ma].re, Ssum));
        }
      }
    });
    __syncwarp();
    // ---- reverse: adjoint columns
    c2<R> lam[J2 + 1];
#pragma unroll
    for (int k = 0; k <= J2; ++k) lam[k] = mk<R>(0, 0);
    if (2 * mb <= J2) {
      const c2<R>* yr = Yw + half_base(J2) + mb * (J2 + 1);
#pragma unroll
      for (int k = 0; k <= J2; ++k) lam[k] = yr[k];
    }
    c2<R> ga = mk<R>(0, 0), gb = mk<R>(0, 0);
    static_for<1, J2>([&](auto tc) {
      constexpr int t = J2 + 1 - decltype(tc)::value;  // J2 down to 1
      constexpr int tp = t - 1;
      constexpr int mc = t / 2;
      constexpr bool even = (t & 1) == 0;
      c2<R> recv[t + 1];
      if constexpr (even) {
#pragma unroll
        for (int k = 0; k <= t; ++k) {
          recv[k].re = shfl_down(lam[k].re);
          recv[k].im = shfl_down(lam[k].im);
        }
      }
      const bool act = grp && 2 * mb <= tp;
      const bool mir = even && act && (mb == mc - 1);
      const c2<R>* ucol = my + half_base(tp) + (act ? mb * (tp + 1) : 0);
      const c2<R>* yr = Yw + half_base(tp) + (act ? mb * (tp + 1) : 0);
      // the seed's factor 1 / sqrt(mc) (v_seed)
      constexpr double qd = even ? 1.0 / c_sqrt(double(mc)) : 0.0;
      const R qm = R(qd);
#pragma unroll
      for (int m = 0; m <= tp; ++m) {
        const c2<R> uu = act ? ucol[m] : mk<R>(0, 0);
        const c2<R> Av = lam[m];
        const c2<R> Bv = lam[m + 1];
        // g_a += conj(A) u ; g_b -= conj(B) u
        ga.re = fm(Av.im, uu.im, fm(Av.re, uu.re, ga.re));
        ga.im = fm(-Av.im, uu.re, fm(Av.re, uu.im, ga.im));
        gb.re = fm(-Bv.im, uu.im, fm(-Bv.re, uu.re, gb.re));
        gb.im = fm(Bv.im, uu.re, fm(-Bv.re, uu.im, gb.im));
        // new adjoint: Yw + a A - b B
        const c2<R> y = act ? yr[m] : mk<R>(0, 0);
        c2<R> nl;
        nl.re = fm(kb.im, Bv.im, fm(-kb.re, Bv.re, fm(-ka.im, Av.im, fm(ka.re, Av.re, y.re))));
        nl.im = fm(-kb.im, Bv.re, fm(-kb.re, Bv.im, fm(ka.im, Av.re, fm(ka.re, Av.im, y.im))));
        if constexpr (even) {
          if (mir) {
            const int mp = tp - m;
            const R sg = ((m + mc - 1) & 1) ? -qm : qm;
            const c2<R> v = mk<R>(sg * uu.re, -sg * uu.im);
            const c2<R> A2 = recv[mp];
            const c2<R> B2 = recv[mp + 1];
            ga.re = fm(A2.im, v.im, fm(A2.re, v.re, ga.re));
            ga.im = fm(-A2.im, v.re, fm(A2.re, v.im, ga.im));
            gb.re = fm(-B2.im, v.im, fm(-B2.re, v.re, gb.re));
            gb.im = fm(B2.im, v.re, fm(-B2.re, v.im, gb.im));
            const R lr = fm(kb.im, B2.im, fm(-kb.re, B2.re, fm(-ka.im, A2.im, ka.re * A2.re)));
            const R li = fm(-kb.im, B2.re, fm(-kb.re, B2.im, fm(ka.im, A2.re, ka.re * A2.im)));
            nl.re = fm(sg, lr, nl.re);
            nl.im = fm(-sg, li, nl.im);
          }
        }
        lam[m] = nl;
      }
      lam[tp + 1] = mk<R>(0, 0);
    });
    myred[0] = Ssum;
    myred[1] = ga.re;
    myred[2] = ga.im;
    myred[3] = gb.re;
    myred[4] = gb.im;
    __syncwarp();
    if (ok && mb == 0) {
      R q[5] = {0, 0, 0, 0, 0};
      for (int c = 0; c < NC; ++c) {
        const R* p = red + (warp * 32 + lane + c) * 5;
#pragma unroll
        for (int k = 0; k < 5; ++k) q[k] += p[k];
      }
      const R fc = gm[4];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R ds = q[1] * gm[8 + 2 * d] + q[2] * gm[9 + 2 * d] + q[3] * gm[14 + 2 * d] +
                     q[4] * gm[15 + 2 * d];
        a.dedr[slot * 3 + d] = (double)(gm[5 + d] * q[0] + fc * ds);
      }
    }
    __syncwarp();
  }
  if (!QUEUE) break;
  __syncthreads();  // the item's shared memory is reused by the next item
  }
}

template <typename K>
inline cudaError_t col_allow_smem(K kernel, size_t bytes) {
  // the default 48 KB limit covers static and dynamic shared memory together
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (bytes + fa.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Warps (= atoms) per CTA: the tunable, halved until the CTA's shared memory
// (proportional to its warps) fits the 227 KB limit.
inline int col_fit_warps(int nw, size_t per_warp) {
  while (nw > 1 && per_warp * nw > (size_t)227 * 1024) nw >>= 1;
  return nw;
}

template <typename R, int J2>
cudaError_t launch_ui_col_t(const WorkArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  using UP = UiPlan<R, J2>;
  if (a.H != UP::HH) return cudaErrorInvalidValue;
  const size_t smem = (size_t)UP::A * (UP::Q * UP::warp_bytes + sizeof(R) * 5 * (size_t)a.K);
  cudaError_t e = col_allow_smem(ui_col_kernel<R, J2>, smem);
  if (e != cudaSuccess) return e;
  return launch_k(ui_col_kernel<R, J2>, dim3((unsigned)((a.n + UP::A - 1) / UP::A)), dim3(UP::A * UP::Q * 32),
                  smem, s, a);
}

// Fused neighbour build + compute_U: single configuration (ncta = 0: two
// atoms a CTA in order) or a batch (ncta CTAs of na.cta_map).
template <typename R, int J2>
cudaError_t launch_neigh_u_t(const NeighArgs& na, const WorkArgs& a, int ncta, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  using UP = UiPlan<R, J2>;
  if (a.H != UP::HH) return cudaErrorInvalidValue;
  const size_t smem = (size_t)2 * (UP::Q * UP::warp_bytes + sizeof(R) * 5 * (size_t)a.K);
  if (ncta > 0) {
    cudaError_t e = col_allow_smem(neigh_u_kernel<R, J2, true>, smem);
    if (e != cudaSuccess) return e;
    return launch_k(neigh_u_kernel<R, J2, true>, dim3((unsigned)ncta), dim3(NuShape<true>::NW * 32), smem, s, na,
                    a);
  }
  cudaError_t e = col_allow_smem(neigh_u_kernel<R, J2, false>, smem);
  if (e != cudaSuccess) return e;
  return launch_k(neigh_u_kernel<R, J2, false>, dim3((unsigned)((a.n + 1) / 2)), dim3(NuShape<false>::NW * 32),
                  smem, s, na, a);
}

template <typename R, int J2>
cudaError_t launch_tan_col_t(const WorkArgs& a, const double* g, void* dU, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  using UP = UiPlan<R, J2>;
  if (a.H != UP::HH) return cudaErrorInvalidValue;
  const size_t smem = (size_t)UP::A * (UP::Q * UP::warp_bytes + sizeof(R) * 10 * (size_t)a.K);
  cudaError_t e = col_allow_smem(tan_col_kernel<R, J2>, smem);
  if (e != cudaSuccess) return e;
  return launch_k(tan_col_kernel<R, J2>, dim3((unsigned)((a.n + UP::A - 1) / UP::A)), dim3(UP::A * UP::Q * 32),
                  smem, s, a, g, dU);
}

// Launch plan of the fused dE kernel: warps per CTA (NW) and atoms per CTA
// (A) for atoms of `maxcnt` pairs, from the kernel's registers, the shared
// memory of a plan and the SM count.
//  * A plan's cost is (waves of CTAs) x (passes of its longest warp); the
//    search minimises it, ties going to fewer warps in all.
//  * The reference shape is a warp per atom in CTAs of `nw0` warps.  In one or
//    two waves its cost is counted the same way; over more waves its small
//    CTAs even out and it costs about (all passes) / (resident warps).
//  * The searched plan is taken when it costs 3% less than the reference
//    (measured at 2J8 and 2J14 on 2000 atoms, a 64-configuration batch, and
//    16000 atoms at 2J14, where the reference stays ahead).
//  * pipe_bound (FP64, whose pipe runs at 1/64 of the FP32 rate and is busy
//    all the time): the CTAs an SM holds share its pipe, so A is chosen first
//    by ceil(ctas / SMs) x ceil(A x maxcnt / P), the most CTAs an SM takes
//    times a CTA's passes, among the A whose best warp count (the search
//    above) keeps at least 8 warps an SM resident; then the warp count for
//    that A as above.  Measured at 2J8, 2000 atoms: A = 2 1.067 ms, 3 1.138,
//    16 1.151, 8 1.166, 4 1.182, 1 1.194, 6 1.365, 12 1.704 (the model: 63,
//    65, 70, 70, 72, 70, 78, 104).
struct DePlan {
  int nw, A;
  size_t smem;
};
// force_A > 0 (the SNAP_KNOB_DE_ATOMS tunable) restricts the search to CTAs
// of force_A atoms (the best warp count for it) and skips the reference.
inline DePlan de_plan(int n, int maxcnt, int P, size_t per_warp, size_t per_atom, int regs, int nsm,
                      int max_warps, int nw0, int force_A = 0, bool pipe_bound = false);

// The pipe-bound choice of A (see de_plan), then the plan for it.
inline DePlan de_plan_pipe(int n, int maxcnt, int P, size_t per_warp, size_t per_atom, int regs, int nsm,
                           int max_warps, int nw0) {
  const int ralloc = (regs + 7) / 8 * 8;
  DePlan best{0, 0, 0};
  long best_cost = -1;
  for (int A = 1; A <= 64; ++A) {
    const DePlan p = de_plan(n, maxcnt, P, per_warp, per_atom, regs, nsm, max_warps, nw0, A);
    if (p.smem == 0) break;
    const long ctas = (n + A - 1) / A;
    const int cps = std::min({65536 / (ralloc * p.nw * 32), (int)((228 * 1024) / (p.smem + 1024)), 64 / p.nw, 32});
    const long per_sm = (ctas + nsm - 1) / nsm;
    if (std::min<long>(per_sm, cps) * p.nw < 8) continue;  // too few warps to keep the pipe busy
    const long cost = per_sm * (((long)A * maxcnt + P - 1) / P);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = p;
    }
  }
  if (best_cost < 0) return de_plan(n, maxcnt, P, per_warp, per_atom, regs, nsm, max_warps, nw0);
  return best;
}

inline DePlan de_plan(int n, int maxcnt, int P, size_t per_warp, size_t per_atom, int regs, int nsm,
                      int max_warps, int nw0, int force_A, bool pipe_bound) {
  if (pipe_bound && force_A <= 0) return de_plan_pipe(n, maxcnt, P, per_warp, per_atom, regs, nsm, max_warps, nw0);
  const int ralloc = (regs + 7) / 8 * 8;
  auto shape = [&](int nw, int A, size_t* smem, long* waves, long* ppw) -> bool {
    *smem = (size_t)A * per_atom + (size_t)nw * per_warp + sizeof(int) * (A + 1);
    if (*smem > (size_t)227 * 1024) return false;
    const int cps = std::min({65536 / (ralloc * nw * 32), (int)((228 * 1024) / (*smem + 1024)), 64 / nw, 32});
    if (cps < 1) return false;
    const long ctas = (n + A - 1) / A;
    *waves = (ctas + (long)nsm * cps - 1) / ((long)nsm * cps);
    *ppw = ((((long)A * maxcnt + P - 1) / P) + nw - 1) / nw;
    return true;
  };
  DePlan ref{nw0, nw0, 0};
  double ref_cost = 1e300;
  {
    long waves, ppw;
    size_t smem;
    if (shape(nw0, nw0, &smem, &waves, &ppw)) {
      ref.smem = smem;
      const long slots = (long)nsm * std::max(1, (int)std::min<long>(
                                                  {65536L / (ralloc * nw0 * 32), (long)((228 * 1024) / (smem + 1024)),
                                                   64L / nw0, 32L})) * nw0;
      const long per_atom_passes = (maxcnt + P - 1) / P;
      ref_cost = waves <= 2 ? (double)(waves * per_atom_passes)
                            : (double)n * per_atom_passes / (double)slots;
    }
  }
  DePlan best{0, 0, 0};
  long best_cost = -1, best_warps = 0;
  for (int nw = 2; nw <= max_warps; nw *= 2) {
    for (int A = force_A > 0 ? force_A : 1; A <= (force_A > 0 ? force_A : 256); ++A) {
      long waves, ppw;
      size_t smem;
      if (!shape(nw, A, &smem, &waves, &ppw)) break;
      const long cost = waves * ppw;
      const long warps = (long)((n + A - 1) / A) * nw;
      if (best_cost < 0 || cost < best_cost || (cost == best_cost && warps < best_warps)) {
        best_cost = cost;
        best_warps = warps;
        best = DePlan{nw, A, smem};
      }
    }
  }
  if (force_A > 0 && best_cost >= 0) return best;
  if (best_cost < 0 || (ref.smem != 0 && (double)best_cost > 0.97 * ref_cost)) return ref;
  return best;
}

template <typename R, int J2>
cudaError_t launch_de_rev_col_t(const WorkArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  // per warp: forward columns [P][H], lane partials [32][5]; per atom: Yw [H] and its offset
  const size_t per_warp = sizeof(c2<R>) * (size_t)Shape<J2>::P * a.H + sizeof(R) * 32 * 5;
  const size_t per_atom = sizeof(c2<R>) * (size_t)a.H;
  // the kernel's registers and the last plan, per instantiation (the plan
  // search is a few hundred candidate shapes; repeated calls reuse it)
  static std::mutex mu;
  static int regs = 0;
  static long long last_key[4] = {-1, -1, -1, -1};
  static DePlan last_plan{0, 0, 0};
  const int nw0 = std::min(col_fit_warps(a.col_warps, per_warp + per_atom), de_max_warps<R>());
  const int maxcnt = std::max(1, a.de_maxcnt), nsm = std::max(1, a.nsm);
  DePlan p;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (regs == 0) {
      cudaFuncAttributes fa;
      cudaError_t e = cudaFuncGetAttributes(&fa, de_rev_col_kernel<R, J2, false>);
      if (e != cudaSuccess) return e;
      regs = fa.numRegs;
    }
    const long long key[4] = {a.n, ((long long)a.de_atoms << 32) | maxcnt, ((long long)nsm << 32) | nw0, a.H};
    if (std::equal(key, key + 4, last_key)) {
      p = last_plan;
    } else {
      p = de_plan(a.n, maxcnt, Shape<J2>::P, per_warp, per_atom, regs, nsm, de_max_warps<R>(), nw0, a.de_atoms,
                  sizeof(R) == 8);
      std::copy(key, key + 4, last_key);
      last_plan = p;
    }
  }
  if (p.smem == 0) return cudaErrorInvalidConfiguration;  // no plan fits (not reached for 2J <= 14)
  const long nitems = (a.n + p.A - 1) / p.A;
  if (a.persist & 2) {
    // persistent: as many CTAs as stay resident, items from the queue
    auto kq = de_rev_col_kernel<R, J2, true>;
    cudaError_t e = col_allow_smem(kq, p.smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kq, p.nw * 32, p.smem);
    if (e != cudaSuccess) return e;
    const long grid = std::min<long>(nitems, (long)nsm * std::max(1, occ));
    return launch_k(kq, dim3((unsigned)grid), dim3(p.nw * 32), p.smem, s, a, p.A);
  }
  cudaError_t e = col_allow_smem(de_rev_col_kernel<R, J2, false>, p.smem);
  if (e != cudaSuccess) return e;
  return launch_k(de_rev_col_kernel<R, J2, false>, dim3((unsigned)nitems), dim3(p.nw * 32), p.smem, s, a, p.A);
}

}  // namespace col
}  // namespace snap

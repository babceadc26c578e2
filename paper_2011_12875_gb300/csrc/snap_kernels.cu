// snap_kernels.cu -- compute_U, compute_Y, fused dU/dE and the force gather.
//
// Notation follows arXiv:2011.12875: t = 2j, U_t = Ulisttot, Y_t = adjoint
// (Eq. y), dE_i/dr_ik = Re sum_t Y_t : conj(dU_t/dr_ik) (Eq. snapforce2).
// R is the working precision of the recursions: float (mixed) or double.
// Every CTA works on a fixed set of atoms and writes each output once, so the
// results are deterministic; there are no global atomics in the data path.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "snap_geom.cuh"
#include "snap_internal.h"

namespace snap {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename R>
struct __align__(2 * sizeof(R)) cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> mk(R re, R im) {
  cx<R> c;
  c.re = re;
  c.im = im;
  return c;
}
// conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> conj_mul(cx<R> a, cx<R> b) {
  return mk<R>(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// x * y + z with one rounding (complex multiply-adds are written as chains
// of these, two a component)
template <typename R>
__device__ __forceinline__ R fmr(R x, R y, R z) {
  if constexpr (sizeof(R) == 4) return fmaf(x, y, z);
  else return fma(x, y, z);
}

// a * b
template <typename R>
__device__ __forceinline__ cx<R> mul(cx<R> a, cx<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Weight of a half-layout element in a full-matrix contraction M : N* of two
// matrices with the inversion symmetry: 2 for mb < t/2; on the middle column
// (2 mb = t) 2 above the centre, 1 at the centre, 0 below.
__device__ __forceinline__ int half_weight(int t, int ma, int mb) {
  if (2 * mb < t) return 2;
  return ma < mb ? 2 : (ma == mb ? 1 : 0);
}

// Element (m, mb) of layer tp (= t - 1) stored in half layout at `lay`; the
// column mb = (tp+1)/2 past the stored half comes from the inversion symmetry
// u[m][mb] = (-1)^(m+mb) conj(u[tp-m][tp-mb]).
template <typename R>
__device__ __forceinline__ cx<R> prev_elem(const cx<R>* lay, int tp, int m, int mb) {
  if (2 * mb <= tp) return lay[mb * (tp + 1) + m];
  const cx<R> v = lay[(tp - mb) * (tp + 1) + (tp - m)];
  const R s = ((m + mb) & 1) ? R(-1) : R(1);
  return mk<R>(s * v.re, -s * v.im);
}

// The same in the scaled form v = u / S_t(ma, mb) (S_t = sqrt((t-ma)! ma! /
// (t-mb)!)): the mirrored element of the new middle column mb = (tp+1)/2
// also picks up S's ratio between the two columns, 1 / sqrt(mb) (qm).
template <typename R>
__device__ __forceinline__ cx<R> prev_elem_v(const cx<R>* lay, int tp, int m, int mb, R qm) {
  if (2 * mb <= tp) return lay[mb * (tp + 1) + m];
  const cx<R> v = lay[(tp - mb) * (tp + 1) + (tp - m)];
  const R s = ((m + mb) & 1) ? -qm : qm;
  return mk<R>(s * v.re, -s * v.im);
}

// ------------------------------------------------------------- compute_U
// First the atom's slot geometry (snap_geom.cuh), then the recursion.  One
// CTA per atom i, one warp per neighbour pair (lanes over the elements of
// a layer), NW warps per CTA.  u_t of a pair follows the layer recursion
// (Eq. hysphrecur): for mb <= t/2,
//   u_t[ma][mb] = sqrt((t-ma)/(t-mb)) conj(a) u_{t-1}[ma][mb]
//               - sqrt(ma/(t-mb))     conj(b) u_{t-1}[ma-1][mb],
// with only the previous layer kept (double buffer, shared memory), run in the
// scaled form u = S v, v_t[ma] = conj(a) v_{t-1}[ma] - conj(b) v_{t-1}[ma-1]
// (S absorbs both root factors; a multiply and three fused multiply-adds a
// component, with S_t(ma, mb) = sqrt((t-ma)! ma! / (t-mb)!)).  f_c v
// is summed per warp in shared memory, the warps are summed in a fixed order,
// multiplied by S once, and w_self is added on the diagonal (Eq. u).
template <typename R, int NW>
__global__ void __launch_bounds__(NW * 32) ui_kernel(WorkArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int H = a.H, L = a.lmax, J2 = a.twojmax;
  R* root = reinterpret_cast<R*>(smem);
  cx<R>* acc = reinterpret_cast<cx<R>*>(root + kRootDim * kRootDim);
  cx<R>* buf = acc + NW * H;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x;
  const R* rootg = reinterpret_cast<const R*>(a.rootpq);
  for (int e = threadIdx.x; e < kRootDim * kRootDim; e += blockDim.x) root[e] = rootg[e];
  for (int e = threadIdx.x; e < NW * H; e += blockDim.x) acc[e] = mk<R>(0, 0);
  // the atom's slot geometry (snap_geom.cuh)
  geo::atom_geom<R>(a, i, threadIdx.x, blockDim.x);
  __syncthreads();
  cx<R>* myacc = acc + warp * H;
  cx<R>* b0 = buf + warp * 2 * L;
  cx<R>* b1 = b0 + L;
  const int cnt = a.cnt[i];
  for (int s = warp; s < cnt; s += NW) {
    const R* g = reinterpret_cast<const R*>(a.geom) + ((long)i * a.K + s) * kGeomStride;
    const cx<R> ca = mk<R>(g[0], g[1]);
    const cx<R> cb = mk<R>(g[2], g[3]);
    const R fc = g[4];
    cx<R>* cur = b0;
    cx<R>* nxt = b1;
    if (lane == 0) {
      cur[0] = mk<R>(1, 0);
      myacc[0].re += fc;
    }
    __syncwarp();
    for (int t = 1; t <= J2; ++t) {
      const int size = half_layer_size(t), hb = half_base(t);
      const R qm = (t & 1) ? R(0) : root[kRootDim + t / 2];  // 1 / sqrt(t/2): the mirror's ratio
      for (int e = lane; e < size; e += 32) {
        const int mb = e / (t + 1), ma = e - mb * (t + 1);
        cx<R> v = mk<R>(0, 0);
        if (ma < t) {  // + conj(a) v_{t-1}[ma]
          const cx<R> p = prev_elem_v(cur, t - 1, ma, mb, qm);
          v.re = fmr(ca.im, p.im, ca.re * p.re);
          v.im = fmr(-ca.im, p.re, ca.re * p.im);
        }
        if (ma > 0) {  // - conj(b) v_{t-1}[ma-1]
          const cx<R> p = prev_elem_v(cur, t - 1, ma - 1, mb, qm);
          v.re = fmr(-cb.im, p.im, fmr(-cb.re, p.re, v.re));
          v.im = fmr(cb.im, p.re, fmr(-cb.re, p.im, v.im));
        }
        nxt[e] = v;
        myacc[hb + e].re = fmr(fc, v.re, myacc[hb + e].re);
        myacc[hb + e].im = fmr(fc, v.im, myacc[hb + e].im);
      }
      __syncwarp();
      cx<R>* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    __syncwarp();
  }
  __syncthreads();
  cx<R>* Ug = reinterpret_cast<cx<R>*>(a.U);
  const long blk = i >> 5;
  const int li = i & 31;
  for (int e = threadIdx.x; e < H; e += blockDim.x) {
    cx<R> s = acc[e];
    for (int w = 1; w < NW; ++w) {
      s.re += acc[w * H + e].re;
      s.im += acc[w * H + e].im;
    }
    const R sc = reinterpret_cast<const R*>(a.hscale)[e];  // u = S v
    s.re *= sc;
    s.im *= sc;
    const int p = a.half_tmm[e];
    if (tmm_ma(p) == tmm_mb(p)) s.re += (R)a.wself;
    Ug[(blk * H + e) * 32 + li] = s;
  }
}

// ------------------------------------------------------------- compute_Y
// Lanes = 32 consecutive atoms (the paper's warp-of-atoms AoSoA layout,
// Sec. V-B), so every index and coefficient is uniform across the warp.  The
// 32 atoms' Ulisttot (re and im planes, [H][32]) is staged into shared memory
// with one TMA bulk copy per plane.  The contraction of Eq. (z) and the sum of
// Eq. (y) are walked as one list of terms, sorted by output element:
//   Y_t[ma][mb] += coef * U_t1[ma1][mb1] * U_t2[ma2][mb2],
// coef = betaw * C(ma1,ma2) C(mb1,mb2) (with the mirror signs), where a U
// element past the stored half columns is read conjugated from its mirror.
// The terms of an output come grouped by their first factor, so a group
// costs one load and one complex multiply of U_t1 and each term one load and
// two FMAs: Y += U_t1 * sum_k coef_k U_t2,k.  A term record is a word (two
// element offsets, conjugation flags, end-of-group and end-of-output bits)
// and the coefficient.  Each warp owns a contiguous run of outputs, so every
// Y element is accumulated in registers and written once (no atomics).

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded waits.  A wait gives up after kWaitNs of the global timer (or
// kSpinCap polls, whichever comes first), so a copy that never completes
// cannot hang the GPU: the kernel raises an error flag and returns, and the
// call reports SNAP_ERR_TIMEOUT.
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s
constexpr unsigned kSpinCap = 1u << 28;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < kSpinCap; ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Stage `bytes` from global `src` into shared `dst` with one bulk (TMA) copy
// completed on the mbarrier `bar`, issued by thread 0; every thread of the
// CTA waits, bounded.  The outcome is made CTA-uniform.  On a timeout the CTA
// raises flags[3] and waits once more, again bounded, for the copy it issued
// (if that second wait runs out too, the copy may still land in the exiting
// CTA's shared memory).  skip_copy registers the bytes without issuing the
// copy: a test hook under which the wait runs out with nothing in flight.
// `overlap()` runs on every thread while the copy is in flight.
// With src2 given, a second block of `bytes` from src2 lands at dst + off2
// (right after the first when off2 is 0) on the same barrier.
// With src3 given, bytes3 from src3 land at dst + off3, on the same barrier.
template <typename F>
__device__ bool stage_bulk(void* dst, const void* src, unsigned bytes, uint64_t* bar, int* flags,
                           bool skip_copy, F&& overlap, const void* src2 = nullptr, unsigned off2 = 0,
                           const void* src3 = nullptr, unsigned bytes3 = 0, unsigned off3 = 0) {
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (src2 ? 2 * bytes : bytes) + (src3 ? bytes3 : 0u));
    if (!skip_copy) {
      bulk_g2s(dst, src, bytes, bar);
      if (src2) bulk_g2s(static_cast<char*>(dst) + (off2 ? off2 : bytes), src2, bytes, bar);
      if (src3) bulk_g2s(static_cast<char*>(dst) + off3, src3, bytes3, bar);
    }
  }
  overlap();
  const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0, kWaitNs));
  if (!ok) {
    if (threadIdx.x == 0) atomicMax(&flags[3], 1);
    mbar_wait_bounded(bar, 0, kWaitNs / 4);
  }
  return ok;
}

__device__ __forceinline__ float flip_if(float v, unsigned bit) {
  return __int_as_float(__float_as_int(v) ^ (bit << 31));
}
__device__ __forceinline__ double flip_if(double v, unsigned bit) {
  return bit ? -v : v;
}

// v with its sign bit XORed with bit 31 of m
__device__ __forceinline__ float flip_sign(float v, unsigned m) {
  return __int_as_float(__float_as_int(v) ^ (int)m);
}
__device__ __forceinline__ double flip_sign(double v, unsigned m) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)m << 32));
}

template <typename R>
struct YAcc {
  R re, im;  // the output element
  R ar, ai;  // sum of coef * second factor over the current group
};

// Byte offset of a record's second (first) factor from lane 0's element 0:
// elements are 256 B apart for complex float, 512 B for complex double.  PF:
// the FP32 conjugate-plane word, whose top bits are the second factor's
// offset itself (one shift).
template <typename R, bool PF>
__device__ __forceinline__ unsigned y_off2(unsigned w) {
  if constexpr (PF) return w >> 14;
  return (w & 0x3FF00u) << (sizeof(R) == 4 ? 0 : 1);
}
template <typename R, bool PF>
__device__ __forceinline__ unsigned y_off1(unsigned w) {
  if constexpr (PF) return (w & 0x3FFu) << 8;
  return ((w >> 10) & 0x3FF00u) << (sizeof(R) == 4 ? 0 : 1);
}

// Term records of compute_Y read straight from global memory (pulled into
// L1 ahead of use: the stream is read once per CTA).
template <typename R>
struct YRecGlobal {
  static constexpr bool kShared = false;
  const YRec<R>* __restrict__ rec;
  __device__ __forceinline__ void at(int q) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(rec + q + kYRecPrefetch));
  }
  __device__ __forceinline__ const YRec<R>* ptr(int q) const { return rec + q; }
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Term records of compute_Y streamed through a per-warp ring in shared
// memory: chunks of kYChunk records copied by cp.async (16 bytes a lane),
// kYRingChunks of them resident or in flight, and the first kYGroupMax
// records of the chunk in slot 0 mirrored past the ring's end, so that a
// step of up to kYGroupMax records never wraps.  While the warp's steps
// start in chunk c, chunks c and c + 1 are complete (a step may run into
// c + 1) and c + 2, c + 3 are in flight.  A record is then a broadcast
// shared-memory load instead of a global load through the L1 tags.
constexpr int kYChunk = 32;
constexpr int kYRingChunks = 4;
constexpr int kYRingLen = kYChunk * kYRingChunks + kYGroupMax;
static_assert(kYChunk % 2 == 0 && kYGroupMax % 2 == 0 && kYGroupMax <= kYChunk, "16-byte copies");
static_assert(kYChunk * kYRingChunks <= kYRecPad, "ring reads stay in the padding");

// Byte offset of the record rings in compute_Y's dynamic shared memory:
// after the staged plane(s) of complex float and the 16-byte barrier slot.
__host__ __device__ constexpr size_t yi_ring_offset(int H, bool cp) {
  return (size_t)(cp ? 2 : 1) * H * 32 * sizeof(cx<float>) + 16;
}

struct YRecRing {
  static constexpr bool kShared = true;
  YRec<float>* buf;         // [kYRingLen] of this warp
  const YRec<float>* base;  // global record qs (qs even: 16-byte aligned)
  int qs, cross, lane;
  __device__ __forceinline__ void issue(int c) {  // chunk c into slot c % kYRingChunks
    const int slot = (c % kYRingChunks) * kYChunk;
    const YRec<float>* g = base + c * kYChunk;
    if (lane < kYChunk / 2) {
      cp_async16(buf + slot + 2 * lane, g + 2 * lane);
    } else if (slot == 0 && lane < (kYChunk + kYGroupMax) / 2) {
      const int m = lane - kYChunk / 2;
      cp_async16(buf + kYChunk * kYRingChunks + 2 * m, g + 2 * m);
    }
    cp_async_commit();
  }
  __device__ __forceinline__ void init(const YRec<float>* rec, int q0, int ln, YRec<float>* b) {
    buf = b;
    lane = ln;
    qs = q0 & ~1;
    base = rec + qs;
    cross = qs + kYChunk;
#pragma unroll
    for (int c = 0; c < kYRingChunks; ++c) issue(c);
    cp_async_wait<kYRingChunks - 2>();
    __syncwarp();
  }
  // before a step that starts at record q (steps advance by < kYChunk)
  __device__ __forceinline__ void at(int q) {
    if (q >= cross) {
      issue((cross - qs) / kYChunk - 1 + kYRingChunks);  // into the slot just left
      cp_async_wait<kYRingChunks - 2>();
      __syncwarp();
      cross += kYChunk;
    }
  }
  __device__ __forceinline__ const YRec<float>* ptr(int q) const {
    return buf + ((q - qs) & (kYChunk * kYRingChunks - 1));
  }
};

// B consecutive groups of K terms from record q: every record and both
// factors are loaded ahead of the arithmetic (no branch inside), then per
// group acc = sum_k coef_k U2,k and Y += U1 * acc.  `ul` points at lane 0's
// element 0 plus this lane.  CP: the staged block is [2][H][32] with the
// conjugate in its second half (no sign flips).
template <typename R, bool CP, int K, int B, typename Src>
__device__ __forceinline__ void y_groups(Src& src, int q, const char* __restrict__ ul, R& yre, R& yim) {
  src.at(q);
  const YRec<R>* rp = src.ptr(q);
  unsigned w[B * K];
  R c[B * K];
#pragma unroll
  for (int j = 0; j < B * K; ++j) {
    if constexpr (sizeof(R) == 4) {
      const uint2 r = Src::kShared ? *reinterpret_cast<const uint2*>(rp + j)
                                   : __ldg(reinterpret_cast<const uint2*>(rp + j));
      w[j] = r.x;
      c[j] = __uint_as_float(r.y);
    } else {
      const uint4 r = __ldg(reinterpret_cast<const uint4*>(rp + j));
      w[j] = r.x;
      c[j] = (R)__hiloint2double((int)r.w, (int)r.z);
    }
  }
  constexpr bool PF = sizeof(R) == 4 && CP;
  cx<R> u2[B * K], u1[B];
#pragma unroll
  for (int j = 0; j < B * K; ++j) u2[j] = *reinterpret_cast<const cx<R>*>(ul + y_off2<R, PF>(w[j]));
#pragma unroll
  for (int b = 0; b < B; ++b) u1[b] = *reinterpret_cast<const cx<R>*>(ul + y_off1<R, PF>(w[b * K]));
#pragma unroll
  for (int b = 0; b < B; ++b) {
    R ar = R(0), ai = R(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = b * K + k;
      ar += c[j] * u2[j].re;
      ai += c[j] * (CP ? u2[j].im : flip_sign(u2[j].im, w[j] & 0x80000000u));
    }
    const R i1 = CP ? u1[b].im : flip_sign(u1[b].im, (w[b * K] << 1) & 0x80000000u);
    yre = fmr(-i1, ai, fmr(u1[b].re, ar, yre));
    yim = fmr(i1, ar, fmr(u1[b].re, ai, yim));
  }
}

// FP64 path: one term at a time with the group-end and output-end bits of
// the record (FP64 arithmetic, not the integer work around it, bounds that
// path, and this loop keeps its registers low).
template <typename R, bool CP>
__device__ __forceinline__ void y_term(unsigned w, R c, cx<R> u2, const char* __restrict__ ul,
                                       cx<R>* __restrict__ Yg, int lane, int& o, YAcc<R>& y) {
  const R i2 = CP ? u2.im : flip_sign(u2.im, w & 0x80000000u);
  y.ar += c * u2.re;
  y.ai += c * i2;
  if (w & (1u << 28)) {
    const cx<R> u1 = *reinterpret_cast<const cx<R>*>(ul + y_off1<R, false>(w));
    const R i1 = CP ? u1.im : flip_sign(u1.im, (w << 1) & 0x80000000u);
    y.re = fmr(-i1, y.ai, fmr(u1.re, y.ar, y.re));
    y.im = fmr(i1, y.ar, fmr(u1.re, y.ai, y.im));
    y.ar = R(0);
    y.ai = R(0);
    if (w & (1u << 29)) {
      Yg[o * 32 + lane] = mk<R>(y.re, y.im);
      y.re = R(0);
      y.im = R(0);
      ++o;
    }
  }
}

// All groups of K terms of one output (a run of `ng` groups from record q).
template <typename R, bool CP, int K, typename Src>
__device__ __forceinline__ void y_run(Src& src, int& q, int ng, const char* __restrict__ ul, R& yre, R& yim) {
  constexpr int B = K >= 8 ? 1 : 8 / K;  // groups per step: about 8 records
  static_assert(B * K <= kYGroupMax, "a step fits the record ring's mirror");
  for (; ng >= B; ng -= B, q += B * K) y_groups<R, CP, K, B>(src, q, ul, yre, yim);
  for (; ng > 0; --ng, q += K) y_groups<R, CP, K, 1>(src, q, ul, yre, yim);
}

// One warp's outputs [o0, o1): per output its runs of 1-, 2-, ... 8-term
// groups (branch-free bodies of known length).  The records of consecutive
// outputs are consecutive, and the next output's run header is loaded while
// the current one is computed.
template <typename R, bool CP, typename Src>
__device__ __forceinline__ void y_outputs(Src& src, const uint4* __restrict__ runs, int q, int o0, int o1,
                                          const char* __restrict__ ul, cx<R>* __restrict__ Yg, int lane) {
  static_assert(kYGroupMax == 8, "one 16-byte run header per output");
  uint4 h = __ldg(runs + o0);
  for (int o = o0; o < o1; ++o) {
    const uint4 hn = __ldg(runs + min(o + 1, o1 - 1));
    R yre = R(0), yim = R(0);
    y_run<R, CP, 1>(src, q, (int)(h.x & 0xffffu), ul, yre, yim);
    y_run<R, CP, 2>(src, q, (int)(h.x >> 16), ul, yre, yim);
    y_run<R, CP, 3>(src, q, (int)(h.y & 0xffffu), ul, yre, yim);
    y_run<R, CP, 4>(src, q, (int)(h.y >> 16), ul, yre, yim);
    y_run<R, CP, 5>(src, q, (int)(h.z & 0xffffu), ul, yre, yim);
    y_run<R, CP, 6>(src, q, (int)(h.z >> 16), ul, yre, yim);
    y_run<R, CP, 7>(src, q, (int)(h.w & 0xffffu), ul, yre, yim);
    y_run<R, CP, 8>(src, q, (int)(h.w >> 16), ul, yre, yim);
    Yg[o * 32 + lane] = mk<R>(yre, yim);
    h = hn;
  }
}

// One warp's outputs of slice `slice` for the 32-atom block blk, with the
// block's U at `us` (staged in shared memory or in global memory).
template <typename R, bool STAGED, bool CP>
__device__ __forceinline__ void yi_slice(const WorkArgs& a, unsigned char* smem, const cx<R>* us, long blk,
                                         int slice, int warp, int lane) {
  if (slice >= a.nslices) return;
  const int H = a.H;
  const int o0 = a.yslice[slice], o1 = a.yslice[slice + 1];
  if (o0 >= o1) return;
  cx<R>* Yg = reinterpret_cast<cx<R>*>(a.Y) + blk * H * 32;
  const YRec<R>* __restrict__ rec = reinterpret_cast<const YRec<R>*>(a.yrec);
  const char* ul = reinterpret_cast<const char*>(us + lane);
  if constexpr (sizeof(R) == 8) {
    // FP64: the terms of the slice in order, four records per batch
    int q = a.yfirst[o0];
    const int q1 = a.yfirst[o1];
    int o = o0;
    YAcc<R> y;
    y.re = y.im = y.ar = y.ai = R(0);
    for (; q + 4 <= q1; q += 4) {
      uint4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = __ldg(reinterpret_cast<const uint4*>(rec + q + k));
      cx<R> u2[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) u2[k] = *reinterpret_cast<const cx<R>*>(ul + y_off2<R, false>(v[k].x));
#pragma unroll
      for (int k = 0; k < 4; ++k)
        y_term<R, CP>(v[k].x, (R)__hiloint2double((int)v[k].w, (int)v[k].z), u2[k], ul, Yg, lane, o, y);
    }
    for (; q < q1; ++q)
      y_term<R, CP>(rec[q].w, rec[q].c, *reinterpret_cast<const cx<R>*>(ul + y_off2<R, false>(rec[q].w)), ul, Yg,
                    lane, o, y);
  } else {
    // FP32: the records through the warp's ring in shared memory (staged
    // CTAs; the ring sits after the staged planes and their barrier)
    const uint4* runs = reinterpret_cast<const uint4*>(a.yruns);  // 8 u16 counts per output
    const int q0 = a.yfirst[o0];
    if constexpr (STAGED) {
      YRec<float>* rb = reinterpret_cast<YRec<float>*>(smem + yi_ring_offset(H, CP)) + warp * kYRingLen;
      YRecRing src;
      src.init(rec, q0, lane, rb);
      y_outputs<R, CP>(src, runs, q0, o0, o1, ul, Yg, lane);
      cp_async_wait<0>();  // no copy outlives the warp's slice
    } else {
      YRecGlobal<R> src{rec};
      y_outputs<R, CP>(src, runs, q0, o0, o1, ul, Yg, lane);
    }
  }
}

// CTA = one 32-atom block x one ysplit-th of the outputs; U of the block
// staged by a TMA bulk copy.
template <typename R, bool STAGED, bool CP>
__global__ void __launch_bounds__(STAGED ? 1024 : 256, 1) yi_kernel(WorkArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long blk0 = blockIdx.x;
  const int H = a.H;
  const cx<R>* us = reinterpret_cast<const cx<R>*>(a.U) + blk0 * H * 32;
  if (STAGED) {
    cx<R>* su = reinterpret_cast<cx<R>*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(su + (CP ? 2 : 1) * H * 32);
    const unsigned bytes = (unsigned)(H * 32 * sizeof(cx<R>));
    if (!stage_bulk(su, us, bytes, bar, a.flags, a.test_skip_stage != 0, [] {})) return;
    if (CP) {
      for (int e = threadIdx.x; e < H * 32; e += blockDim.x) {
        const cx<R> v = su[e];
        su[H * 32 + e] = mk<R>(v.re, -v.im);
      }
      __syncthreads();
    }
    us = su;
  }
  yi_slice<R, STAGED, CP>(a, smem, us, blk0, blockIdx.y * (blockDim.x >> 5) + warp, warp, lane);
}

// The same work as a persistent launch over a work queue: a grid of resident
// CTAs, each taking (block, split) items from a device counter (flags[5],
// zeroed with the flags by every evaluation) until the items run out, across
// all configurations of a batch.  No CTA waits on another (the counter is the
// only shared state), and an item's arithmetic is that of the CTA it would
// have been, so the results are bit for bit those of yi_kernel.  The staging
// barrier is reused item after item (its phase flips per completed copy).
template <typename R, bool CP>
__global__ void __launch_bounds__(1024, 1) yi_queue_kernel(WorkArgs a, int ysplit) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int item_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int H = a.H;
  const long nitems = (long)((a.n + 31) / 32) * ysplit;
  cx<R>* su = reinterpret_cast<cx<R>*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(su + (CP ? 2 : 1) * H * 32);
  const unsigned bytes = (unsigned)(H * 32 * sizeof(cx<R>));
  if (threadIdx.x == 0) mbar_init(bar, 1);
  unsigned phase = 0;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(&a.flags[5], 1);
    __syncthreads();  // also: every warp is done with the previous block
    const long item = item_s;
    if (item >= nitems) break;
    const long blk = item / ysplit;
    const int part = (int)(item - blk * ysplit);
    if (threadIdx.x == 0) {
      mbar_expect_tx(bar, bytes);
      if (!a.test_skip_stage) bulk_g2s(su, reinterpret_cast<const cx<R>*>(a.U) + blk * H * 32, bytes, bar);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, phase, kWaitNs));
    if (!ok) {
      if (threadIdx.x == 0) atomicMax(&a.flags[3], 1);
      mbar_wait_bounded(bar, phase, kWaitNs / 4);
      return;
    }
    phase ^= 1u;
    if (CP) {
      for (int e = threadIdx.x; e < H * 32; e += blockDim.x) {
        const cx<R> v = su[e];
        su[H * 32 + e] = mk<R>(v.re, -v.im);
      }
      __syncthreads();
    }
    yi_slice<R, true, CP>(a, smem, su, blk, part * (blockDim.x >> 5) + warp, warp, lane);
    __syncthreads();  // item_s is rewritten next
  }
}

// ------------------------------------------- compute_Y, one atom per warp
// The alternative layout to the warp of atoms (the paper compares the two,
// Sec. V-B): warp = one atom, its Ulisttot and conj(Ulisttot) staged in shared
// memory as a [2][H] block, lanes over output elements (dealt to the lanes in
// decreasing term count, snake order, so their loads balance); each lane walks
// its outputs' term records in the same grouped order as yi_kernel.
constexpr int kYaWarps = 8;

template <typename R>
__global__ void __launch_bounds__(kYaWarps * 32) yi_atom_kernel(WorkArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long i = (long)blockIdx.x * kYaWarps + warp;
  if (i >= a.n) return;  // whole warp
  const int H = a.H;
  cx<R>* ua = reinterpret_cast<cx<R>*>(smem) + (size_t)warp * 2 * H;
  const long base = (i >> 5) * (long)H * 32 + (i & 31);
  const cx<R>* Ug = reinterpret_cast<const cx<R>*>(a.U) + base;
  for (int e = lane; e < H; e += 32) {
    const cx<R> v = Ug[(long)e * 32];
    ua[e] = v;
    ua[H + e] = mk<R>(v.re, -v.im);
  }
  __syncwarp();
  cx<R>* Yg = reinterpret_cast<cx<R>*>(a.Y) + base;
  const YRec<R>* __restrict__ rec = reinterpret_cast<const YRec<R>*>(a.yrec);
  const bool pf = yrec_plane_format((int)sizeof(R), H);
  const int m = a.ysched_m;
  for (int k = 0; k < m; ++k) {
    const int o = a.ysched[lane * m + k];
    if (o < 0) break;
    YAcc<R> y;
    y.re = y.im = y.ar = y.ai = R(0);
    const int q1 = a.yfirst[o + 1];
    for (int q = a.yfirst[o]; q < q1; ++q) {
      const unsigned w = rec[q].w;
      const R c = rec[q].c;
      // elements of the factors in the [2][H] block: the staged-conjugate
      // record formats index it directly, the other one sets the sign bits
      const int e2 = pf ? (int)(w >> 22) : (int)((w >> 8) & 1023u) + (int)(w >> 31) * H;
      const cx<R> u2 = ua[e2];
      y.ar += c * u2.re;
      y.ai += c * u2.im;
      if (w & (pf ? (1u << 12) : (1u << 28))) {
        const int e1 = pf ? (int)(w & 1023u) : (int)((w >> 18) & 1023u) + (int)((w >> 30) & 1u) * H;
        const cx<R> u1 = ua[e1];
        y.re = fmr(-u1.im, y.ai, fmr(u1.re, y.ar, y.re));
        y.im = fmr(u1.im, y.ar, fmr(u1.re, y.ai, y.im));
        y.ar = R(0);
        y.ai = R(0);
      }
    }
    Yg[(long)o * 32] = mk<R>(y.re, y.im);
  }
}

// ------------------------------------------------------- bispectrum B_l
// Descriptor output (Sec. II-A, Eq. z): B_l = Re Z^t_{t1t2} : conj(U_t) for
// every canonical component l, 32 atoms a CTA (lanes = atoms; the block's U
// staged in shared memory by a TMA bulk copy, as in compute_Y), and, with
// DERIV, its directional derivative along the tangent dU of Ulisttot
// (Eqs. z and dbidrk): B_l is trilinear in (U_t1, U_t2, conj U_t), so
//   dB_l = Re [ (Z(dU_t1, U_t2) + Z(U_t1, dU_t2)) : conj(U_t) + Z : conj(dU_t) ]
// (dU has the inversion symmetry of U, so the records' conjugation flags hold
// for it too).
// The term list is cut into chunks of whole output groups (never across a
// component).  CTA (block, part) takes the components of its part; its
// warps take the part's chunks in turn, each leaving one partial sum per atom
// (in shared memory, or in a global scratch where the part has too many
// chunks), and the partials of a component are added in chunk order: a fixed
// order, whatever the launch shape, and no warp waits on the largest
// component.
//
// Records (snap_tables.h, bwords): the factors' byte offsets sit in the word
// already scaled to the plane's element stride (one mask each).  Each output
// group is cut into pieces of at most kBGroupMax terms, and a chunk's pieces
// are stored by length, so a chunk is runs of equal-length pieces walked by
// branch-free bodies (records, factors and output elements loaded ahead of
// the arithmetic); a piece's first word holds its output element.  The
// contraction is linear in Z, so each piece is contracted on its own.  CP:
// the staged block is [2][H][32] with the conjugates in its second half (no
// sign flips); with DERIV the tangent's planes follow, [U | conj U | dU |
// conj dU].
template <typename R, bool CP>
__device__ __forceinline__ unsigned b_off1(unsigned w) {
  const unsigned o = CP ? ((w >> 11) & 0x7FF00u) : ((w >> 10) & 0x3FF00u);
  return sizeof(R) == 4 ? o : o << 1;
}
template <typename R, bool CP>
__device__ __forceinline__ unsigned b_off2(unsigned w) {
  const unsigned o = CP ? (w & 0x7FF00u) : (w & 0x3FF00u);
  return sizeof(R) == 4 ? o : o << 1;
}
// byte offset of a piece's output element, from the piece's first word
template <typename R, bool CP>
__device__ __forceinline__ unsigned b_out(unsigned w) {
  const unsigned o = (w & 0xFFu) | (((w >> (CP ? 30 : 28)) & 3u) << 8);
  return o * (unsigned)(32 * sizeof(cx<R>));
}

// one record: from the CTA's staged copy (RS) or through the read-only path
template <typename R, bool RS>
__device__ __forceinline__ void b_load(const YRec<R>* __restrict__ rec, int q, unsigned& w, R& c) {
  if constexpr (RS) {
    if constexpr (sizeof(R) == 4) {
      const uint2 r = *reinterpret_cast<const uint2*>(rec + q);
      w = r.x;
      c = __uint_as_float(r.y);
    } else {
      const uint4 r = *reinterpret_cast<const uint4*>(rec + q);
      w = r.x;
      c = (R)__hiloint2double((int)r.w, (int)r.z);
    }
  } else if constexpr (sizeof(R) == 4) {
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(rec + q));
    w = r.x;
    c = __uint_as_float(r.y);
  } else {
    const uint4 r = __ldg(reinterpret_cast<const uint4*>(rec + q));
    w = r.x;
    c = (R)__hiloint2double((int)r.w, (int)r.z);
  }
}

// G pieces of K terms from record q: per piece Z = sum c u1 u2 (and dZ),
// then acc += Re(Z conj U_o) (DERIV: Re(dZ conj U_o + Z conj dU_o)).
template <typename R, bool CP, bool DERIV, bool RS, int K, int G>
__device__ __forceinline__ void b_pieces(const YRec<R>* __restrict__ rec, int q, const char* __restrict__ ul,
                                         const char* __restrict__ dl, R& acc) {
  constexpr int N = G * K;
  unsigned w[N];
  R c[N];
#pragma unroll
  for (int j = 0; j < N; ++j) b_load<R, RS>(rec, q + j, w[j], c[j]);
  cx<R> u1[N], u2[N], d1[DERIV ? N : 1], d2[DERIV ? N : 1], uo[G], duo[DERIV ? G : 1];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    u1[j] = *reinterpret_cast<const cx<R>*>(ul + b_off1<R, CP>(w[j]));
    u2[j] = *reinterpret_cast<const cx<R>*>(ul + b_off2<R, CP>(w[j]));
    if constexpr (DERIV) {
      d1[j] = *reinterpret_cast<const cx<R>*>(dl + b_off1<R, CP>(w[j]));
      d2[j] = *reinterpret_cast<const cx<R>*>(dl + b_off2<R, CP>(w[j]));
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const unsigned ob = b_out<R, CP>(w[g * K]);
    uo[g] = *reinterpret_cast<const cx<R>*>(ul + ob);
    if constexpr (DERIV) duo[g] = *reinterpret_cast<const cx<R>*>(dl + ob);
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    R zr, zi, dzr = R(0), dzi = R(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int j = g * K + k;
      const unsigned m1 = (w[j] << 1) & 0x80000000u, m2 = w[j] & 0x80000000u;
      const R b1 = CP ? u1[j].im : flip_sign(u1[j].im, m1), b2 = CP ? u2[j].im : flip_sign(u2[j].im, m2);
      // c u1 u2 = (p + i q)(u2.re + i b2), p + i q = c u1
      const R p = c[j] * u1[j].re, qq = c[j] * b1;
      if (k == 0) {
        zr = p * u2[j].re;
        zi = p * b2;
      } else {
        zr = fmr(p, u2[j].re, zr);
        zi = fmr(p, b2, zi);
      }
      zr = fmr(-qq, b2, zr);
      zi = fmr(qq, u2[j].re, zi);
      if constexpr (DERIV) {
        // d(c u1 u2) = c du1 u2 + c u1 du2
        const R db1 = CP ? d1[j].im : flip_sign(d1[j].im, m1), db2 = CP ? d2[j].im : flip_sign(d2[j].im, m2);
        const R dp = c[j] * d1[j].re, dq = c[j] * db1;
        dzr = fmr(dp, u2[j].re, dzr);
        dzr = fmr(-dq, b2, dzr);
        dzr = fmr(p, d2[j].re, dzr);
        dzr = fmr(-qq, db2, dzr);
        dzi = fmr(dp, b2, dzi);
        dzi = fmr(dq, u2[j].re, dzi);
        dzi = fmr(p, db2, dzi);
        dzi = fmr(qq, d2[j].re, dzi);
      }
    }
    if constexpr (DERIV) {
      acc = fmr(uo[g].re, dzr, acc);
      acc = fmr(uo[g].im, dzi, acc);
      acc = fmr(duo[g].re, zr, acc);
      acc = fmr(duo[g].im, zi, acc);
    } else {
      acc = fmr(uo[g].re, zr, acc);
      acc = fmr(uo[g].im, zi, acc);
    }
  }
}

// All ng pieces of K terms from record q (advanced past them): about kStep
// records a body.
template <typename R, bool CP, bool DERIV, bool RS, int K>
__device__ __forceinline__ void b_run(const YRec<R>* __restrict__ rec, int& q, int ng, const char* __restrict__ ul,
                                      const char* __restrict__ dl, R& acc) {
  constexpr int kStep = DERIV ? 4 : 8;
  constexpr int G = K >= kStep ? 1 : kStep / K;
  for (; ng >= G; ng -= G, q += G * K) b_pieces<R, CP, DERIV, RS, K, G>(rec, q, ul, dl, acc);
  for (; ng > 0; --ng, q += K) b_pieces<R, CP, DERIV, RS, K, 1>(rec, q, ul, dl, acc);
}

// gpart: the partial sums' scratch in global memory ([CTA][maxchunks][32]),
// or null for shared memory.  RS: the run's records staged beside the planes
// (rec_bytes of shared memory) by the same bulk copy.
// DS (DERIV): the tangent's block is staged too; without it (two blocks do not
// fit, 2J = 14) U alone is staged and dU is read through L1.
template <typename R, bool STAGED, bool CP, bool DERIV, bool RS, bool DS>
__global__ void __launch_bounds__(kBiThreads, kBiCtasPerSm)
    bi_kernel(WorkArgs a, const cx<R>* __restrict__ dUg, double* __restrict__ out, R* __restrict__ gpart,
              unsigned rec_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  static_assert(STAGED || (!CP && !RS), "the conjugate plane and the records are staged");
  static_assert(!DS || (STAGED && DERIV), "the tangent is staged with U");
  static_assert(!(CP && DERIV && !DS), "the conjugate plane of dU needs dU staged");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long blk = blockIdx.x;
  const int H = a.H;
  const size_t plane = (size_t)H * 32 * sizeof(cx<R>);
  constexpr int NP = (CP ? 2 : 1) * (DS ? 2 : 1);
  const cx<R>* ug = reinterpret_cast<const cx<R>*>(a.U) + blk * H * 32;
  const cx<R>* dg = DERIV ? dUg + blk * H * 32 : nullptr;
  const char* ul = reinterpret_cast<const char*>(ug + lane);
  const char* dl = DERIV ? reinterpret_cast<const char*>(dg + lane) : nullptr;
  const size_t roff = STAGED ? NP * plane + 16 : 0;  // records, then partials
  R* part = gpart ? gpart + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * a.bmaxchunks * 32
                  : reinterpret_cast<R*>(smem + roff + (RS ? rec_bytes : 0u));  // [maxchunks][32]
  const int l0 = a.bpart[blockIdx.y], l1 = a.bpart[blockIdx.y + 1];
  const int c0 = a.bcomp_chunk[l0], c1 = a.bcomp_chunk[l1];
  const YRec<R>* __restrict__ grec = reinterpret_cast<const YRec<R>*>(CP ? a.brec_cp : a.brec);
  // records [qb, q1) of the run; FP32 records start on a 16-byte boundary
  const int qb = RS ? (sizeof(R) == 4 ? a.bchunk_term[c0] & ~1 : a.bchunk_term[c0]) : 0;
  const unsigned rbytes =
      RS ? (unsigned)(((a.bchunk_term[c1] - qb) * sizeof(YRec<R>) + 15) / 16 * 16) : 0u;
  if (STAGED) {
    cx<R>* su = reinterpret_cast<cx<R>*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NP * plane);
    if (!stage_bulk(su, ug, (unsigned)plane, bar, a.flags, a.test_skip_stage != 0, [] {},
                    DS ? reinterpret_cast<const void*>(dg) : nullptr, (unsigned)((CP ? 2 : 1) * plane),
                    RS ? reinterpret_cast<const void*>(grec + qb) : nullptr, rbytes, (unsigned)roff))
      return;
    if (CP) {
      const int he = H * 32;
      for (int e = threadIdx.x; e < he; e += blockDim.x) {
        const cx<R> v = su[e];
        su[he + e] = mk<R>(v.re, -v.im);
        if (DS) {
          const cx<R> d = su[2 * he + e];
          su[3 * he + e] = mk<R>(d.re, -d.im);
        }
      }
      __syncthreads();
    }
    ul = reinterpret_cast<const char*>(su + lane);
    if (DS) dl = ul + (CP ? 2 : 1) * plane;
  }
  const YRec<R>* __restrict__ rec = RS ? reinterpret_cast<const YRec<R>*>(smem + roff) : grec;
  static_assert(kBGroupMax == 8, "one 16-byte run header per chunk");
  const uint4* __restrict__ runs = reinterpret_cast<const uint4*>(a.bchunk_runs);
  for (int ch = c0 + warp; ch < c1; ch += nw) {
    const uint4 h = __ldg(runs + ch);
    int q = a.bchunk_term[ch] - qb;
    R acc = R(0);
    b_run<R, CP, DERIV, RS, 1>(rec, q, (int)(h.x & 0xffffu), ul, dl, acc);
    b_run<R, CP, DERIV, RS, 2>(rec, q, (int)(h.x >> 16), ul, dl, acc);
    b_run<R, CP, DERIV, RS, 3>(rec, q, (int)(h.y & 0xffffu), ul, dl, acc);
    b_run<R, CP, DERIV, RS, 4>(rec, q, (int)(h.y >> 16), ul, dl, acc);
    b_run<R, CP, DERIV, RS, 5>(rec, q, (int)(h.z & 0xffffu), ul, dl, acc);
    b_run<R, CP, DERIV, RS, 6>(rec, q, (int)(h.z >> 16), ul, dl, acc);
    b_run<R, CP, DERIV, RS, 7>(rec, q, (int)(h.w & 0xffffu), ul, dl, acc);
    b_run<R, CP, DERIV, RS, 8>(rec, q, (int)(h.w >> 16), ul, dl, acc);
    part[(ch - c0) * 32 + lane] = acc;
  }
  __syncthreads();
  const long i = blk * 32 + lane;
  for (int l = l0 + warp; l < l1; l += nw) {
    R v = R(0);
    for (int ch = a.bcomp_chunk[l]; ch < a.bcomp_chunk[l + 1]; ++ch) v += part[(ch - c0) * 32 + lane];
    if (i < a.n) out[i * a.ncoeff + l] = (double)v;
  }
}

// ------------------------------------------- weighted force (autograd)
// grad_k = sum_i w_i dE_i/dr_k = -( w_k sum_s dE_k/dr_ks - sum_s w_{k_s} dE_{k_s}/dr_{k_s,k} ),
// gathered through the reverse-slot map like the forces (w = 1 gives -F).
__global__ void __launch_bounds__(256) force_weighted_kernel(WorkArgs a, const double* __restrict__ wt,
                                                             double* __restrict__ grad) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long k = (long)blockIdx.x * 8 + warp;
  if (k >= a.n) return;
  const double wk = wt[k];
  double f[3] = {0, 0, 0};
  const int cnt = a.cnt[k];
  for (int s = lane; s < cnt; s += 32) {
    const long q = k * a.K + s;
    const int j = a.nbr[q];
    const int r = a.rev[q];
    const double* d = a.dedr + q * 3;
    for (int c = 0; c < 3; ++c) f[c] += wk * d[c];
    if (r >= 0) {
      const double wj = wt[j];
      const double* dj = a.dedr + ((long)j * a.K + r) * 3;
      for (int c = 0; c < 3; ++c) f[c] -= wj * dj[c];
    }
  }
  for (int c = 0; c < 3; ++c) f[c] = warp_sum(f[c]);
  if (lane == 0)
    for (int c = 0; c < 3; ++c) grad[3 * k + c] = -f[c];
}

// ------------------------------------------------------ fused dU + dE/dr
// One CTA per atom i with Y_i (weighted by half_weight and by S of the
// scaled recursion u = S v) staged in shared memory; one warp per pair.  For
// a pair, S(a, b) = sum_t Re Y_t : conj(u_t) = sum_t Re (S Y_t) : conj(v_t)
// is a real function of the Cayley-Klein parameters.  Its gradient follows
// from one forward pass of the scaled layer recursion (all layers of v kept
// in shared memory) and one reverse (adjoint) pass through the same
// recursion, so neither dU nor its three Cartesian components is ever
// formed, and neither pass applies a root factor.  Then
//   dE_i/dr_ik = S df_c/dr + f_c (<g_a, da/dr> + <g_b, db/dr>),
// <x, y> = Re(conj(x) y), which is Eq. (snapforce2) for this pair.
template <typename R, int NW>
__global__ void __launch_bounds__(NW * 32) de_kernel(WorkArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int H = a.H, L = a.lmax, J2 = a.twojmax;
  R* root = reinterpret_cast<R*>(smem);
  cx<R>* Yw = reinterpret_cast<cx<R>*>(root + kRootDim * kRootDim);
  cx<R>* ubase = Yw + H;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x;
  const R* rootg = reinterpret_cast<const R*>(a.rootpq);
  for (int e = threadIdx.x; e < kRootDim * kRootDim; e += blockDim.x) root[e] = rootg[e];
  {
    const cx<R>* Yg = reinterpret_cast<const cx<R>*>(a.Y);
    const long blk = i >> 5;
    const int li = i & 31;
    for (int e = threadIdx.x; e < H; e += blockDim.x) {
      const int p = a.half_tmm[e];
      const R w = (R)half_weight(tmm_t(p), tmm_ma(p), tmm_mb(p));
      // the contraction weight times S of the scaled recursion (u = S v)
      const R ws = w * reinterpret_cast<const R*>(a.hscale)[e];
      const cx<R> y = Yg[(blk * H + e) * 32 + li];
      Yw[e] = mk<R>(ws * y.re, ws * y.im);
    }
  }
  __syncthreads();
  cx<R>* ust = ubase + warp * (H + 2 * L);
  cx<R>* lam0 = ust + H;
  cx<R>* lam1 = lam0 + L;
  const int cnt = a.cnt[i];
  for (int s = warp; s < cnt; s += NW) {
    const long slot = (long)i * a.K + s;
    const R* g = reinterpret_cast<const R*>(a.geom) + slot * kGeomStride;
    const cx<R> ca = mk<R>(g[0], g[1]);
    const cx<R> cb = mk<R>(g[2], g[3]);
    // forward: all layers of u (half layout) and S
    R S = 0;
    if (lane == 0) {
      ust[0] = mk<R>(1, 0);
      S = Yw[0].re;
    }
    __syncwarp();
    for (int t = 1; t <= J2; ++t) {
      const int size = half_layer_size(t), hb = half_base(t);
      const cx<R>* pl = ust + half_base(t - 1);
      const R qm = (t & 1) ? R(0) : root[kRootDim + t / 2];  // 1 / sqrt(t/2): the mirror's ratio
      for (int e = lane; e < size; e += 32) {
        const int mb = e / (t + 1), ma = e - mb * (t + 1);
        cx<R> v = mk<R>(0, 0);
        if (ma < t) {  // + conj(a) v_{t-1}[ma]
          const cx<R> p = prev_elem_v(pl, t - 1, ma, mb, qm);
          v.re = fmr(ca.im, p.im, ca.re * p.re);
          v.im = fmr(-ca.im, p.re, ca.re * p.im);
        }
        if (ma > 0) {  // - conj(b) v_{t-1}[ma-1]
          const cx<R> p = prev_elem_v(pl, t - 1, ma - 1, mb, qm);
          v.re = fmr(-cb.im, p.im, fmr(-cb.re, p.re, v.re));
          v.im = fmr(cb.im, p.re, fmr(-cb.re, p.im, v.im));
        }
        ust[hb + e] = v;
        const cx<R> yw = Yw[hb + e];
        S = fmr(yw.im, v.im, fmr(yw.re, v.re, S));
      }
      __syncwarp();
    }
    // reverse: lambda_t = adjoint of layer t, gathered from layer t+1
    {
      const int hb = half_base(J2);
      for (int e = lane; e < half_layer_size(J2); e += 32) lam0[e] = Yw[hb + e];
    }
    __syncwarp();
    cx<R> ga = mk<R>(0, 0), gb = mk<R>(0, 0);
    cx<R>* lt = lam0;
    cx<R>* ln = lam1;
    for (int t = J2; t >= 1; --t) {
      const int tp = t - 1;
      const int sizep = half_layer_size(tp), hbp = half_base(tp);
      const bool mirror = ((t & 1) == 0);
      const int mc = t >> 1;  // the column of layer t that reads a mirrored column
      const R qmc = mirror ? root[kRootDim + mc] : R(0);  // 1 / sqrt(mc)
      for (int e = lane; e < sizep; e += 32) {
        const int mb = e / (tp + 1), m = e - mb * (tp + 1);
        const cx<R> u = ust[hbp + e];
        // v_{t-1}[m][mb] feeds v_t[m][mb] (a-term) and v_t[m+1][mb] (b-term)
        const cx<R> A = lt[mb * (t + 1) + m];
        const cx<R> B = lt[mb * (t + 1) + m + 1];
        // g_a += conj(A) u ; g_b -= conj(B) u ; new adjoint Yw + a A - b B
        ga.re = fmr(A.im, u.im, fmr(A.re, u.re, ga.re));
        ga.im = fmr(-A.im, u.re, fmr(A.re, u.im, ga.im));
        gb.re = fmr(-B.im, u.im, fmr(-B.re, u.re, gb.re));
        gb.im = fmr(B.im, u.re, fmr(-B.re, u.im, gb.im));
        const cx<R> yw = Yw[hbp + e];
        cx<R> nl;
        nl.re = fmr(cb.im, B.im, fmr(-cb.re, B.re, fmr(-ca.im, A.im, fmr(ca.re, A.re, yw.re))));
        nl.im = fmr(-cb.im, B.re, fmr(-cb.re, B.im, fmr(ca.im, A.re, fmr(ca.re, A.im, yw.im))));
        if (mirror && mb == mc - 1) {
          // v_t column mc reads sig qm conj(v_{t-1}[m][mc-1]) at row mp = tp - m
          const int mp = tp - m;
          const R sig = ((m + mc - 1) & 1) ? -qmc : qmc;
          const cx<R> v = mk<R>(sig * u.re, -sig * u.im);
          const cx<R> A2 = lt[mc * (t + 1) + mp];
          const cx<R> B2 = lt[mc * (t + 1) + mp + 1];
          ga.re = fmr(A2.im, v.im, fmr(A2.re, v.re, ga.re));
          ga.im = fmr(-A2.im, v.re, fmr(A2.re, v.im, ga.im));
          gb.re = fmr(-B2.im, v.im, fmr(-B2.re, v.re, gb.re));
          gb.im = fmr(B2.im, v.re, fmr(-B2.re, v.im, gb.im));
          const R lr = fmr(cb.im, B2.im, fmr(-cb.re, B2.re, fmr(-ca.im, A2.im, ca.re * A2.re)));
          const R li = fmr(-cb.im, B2.re, fmr(-cb.re, B2.im, fmr(ca.im, A2.re, ca.re * A2.im)));
          nl.re = fmr(sig, lr, nl.re);
          nl.im = fmr(-sig, li, nl.im);
        }
        ln[e] = nl;
      }
      __syncwarp();
      cx<R>* tmp = lt;
      lt = ln;
      ln = tmp;
    }
    S = warp_sum(S);
    ga.re = warp_sum(ga.re);
    ga.im = warp_sum(ga.im);
    gb.re = warp_sum(gb.re);
    gb.im = warp_sum(gb.im);
    // lanes 0..2: component d of dE_i/dr_ik in the working precision; the
    // per-atom force and virial sums over pairs are FP64 (force_kernel)
    if (lane < 3) {
      const int d = lane;
      const R ds = ga.re * g[8 + 2 * d] + ga.im * g[9 + 2 * d] + gb.re * g[14 + 2 * d] +
                   gb.im * g[15 + 2 * d];
      a.dedr[slot * 3 + d] = (double)(g[5 + d] * S + g[4] * ds);
    }
    __syncwarp();
  }
}

// --------------------------------------------- energy, forces and virial
// CTA = kFAtoms consecutive atoms, kFThreads threads (a warp per two atoms).
// FP64 runs at 1/64 of the FP32 rate on this part and a warp FP64
// instruction costs the same whatever its active lanes, so the FP64 sums are
// short trees on full warps instead of long chains on a few threads:
//  * energy: E_i - beta_0 is a cubic form in U, so by Euler's relation
//    E_i = beta_0 + (1/3) Re sum_t Y_t : conj(U_t) (full matrices; half layout
//    with half_weight).  kFSlices slices per atom take every kFSlices-th
//    element in the working precision (lanes over atoms: the U and Y reads
//    are coalesced); the slices are added in FP64 by a fixed tree;
//  * forces: lane l of an atom's kFLanes takes slots l, l + kFLanes, ...: it
//    forms g = dE_i/dr_ik - dE_k/dr_ki (the second term through the
//    reverse-slot map, no atomics), adds its g in slot order and accumulates
//    the virial products -dE_i/dr_ik,a r_ik,b; the lane sums are then added
//    by a fixed butterfly;
//  * virial: W_ab is reduced per CTA by the same kind of tree and the last
//    CTA to finish adds the CTA partials in a fixed order (batch mode: per
//    atom, reduced per configuration afterwards).
// Every sum has an order fixed by the slot and element indices alone, so the
// per-atom results do not depend on launch shape or batching.
constexpr int kFAtoms = 8;
constexpr int kFThreads = 128;
constexpr int kFWarps = kFThreads / 32;
constexpr int kFSlices = kFThreads / kFAtoms;  // energy slices per atom
constexpr int kFLanes = 16;                    // lanes per atom in the force sums
static_assert(kFWarps * 32 / kFLanes == kFAtoms, "a warp per two atoms");

// Sum of x[0..N) over each aligned group of G lanes (N <= G, both powers of
// two).  A level with mask m first halves the components a lane carries (the
// lane with bit m clear keeps the lower half and receives its partner's
// lower half), so N components take N - 1 + log2(G / N) additions instead of
// N log2(G).  Returns the total of component (lane mod G) / (G / N).
template <int N, int G>
__device__ __forceinline__ double tree_sum(double (&x)[N], int lane) {
  static_assert(N >= 1 && N <= G && G <= 32 && (N & (N - 1)) == 0 && (G & (G - 1)) == 0, "");
  int n = N;
#pragma unroll
  for (int m = G / 2; m >= 1; m >>= 1) {
    if (n > 1) {
      const bool up = lane & m;
      const int h = n / 2;
#pragma unroll
      for (int j = 0; j < N / 2; ++j) {
        if (j < h) {
          const double send = up ? x[j] : x[j + h];
          const double keep = up ? x[j + h] : x[j];
          x[j] = keep + __shfl_xor_sync(kFull, send, m);
        }
      }
      n = h;
    } else {
      x[0] += __shfl_xor_sync(kFull, x[0], m);
    }
  }
  return x[0];
}

inline size_t force_smem(int, bool) { return 0; }

template <typename R>
__global__ void __launch_bounds__(kFThreads) force_kernel(WorkArgs a) {
  __shared__ double ew[kFWarps][kFAtoms];  // energy: per warp, per atom
  __shared__ double wv[kFWarps][8];        // virial: per warp, per component
  __shared__ bool last;
  const int K = a.K, H = a.H;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long i0 = (long)blockIdx.x * kFAtoms;
  const int na = (int)min((long)kFAtoms, a.n - i0);
  // forces: lanes 16h .. 16h + 15 of warp w take atom 2w + h.  The first
  // pass's slot loads go out before the count and the energy loads (every
  // slot below K is in bounds; those at or past the count are discarded).
  const int l = lane % kFLanes;
  const int ai = 2 * w + lane / kFLanes;
  const bool have = ai < na;
  const long i = i0 + ai;
  bool ok[2];
  int rv[2], kn[2], ky[2];
  double d[2][3], r[2][3], dk[2][3];
  auto load_slots = [&](int s0) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int s = s0 + u * kFLanes + l;
      rv[u] = -1;
      kn[u] = 0;
      ky[u] = -1;
#pragma unroll
      for (int c = 0; c < 3; ++c) d[u][c] = r[u][c] = dk[u][c] = 0.0;
      if (have && s < K) {
        const long q = i * K + s;
        kn[u] = a.nbr[q];
        ky[u] = a.key[q];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          d[u][c] = a.dedr[q * 3 + c];
          r[u][c] = a.rij[q * 3 + c];
        }
      }
    }
  };
  const int cnt_raw = have ? a.cnt[i] : 0;
  load_slots(0);
  // energy partials: lane = atom (8) x slice (4) of the warp's 4 slices
  if (a.energy) {
    const int ae = lane % kFAtoms, sl = (kFSlices / kFWarps) * w + lane / kFAtoms;
    R e = R(0);
    if (ae < na) {
      const long ie = i0 + ae;
      const long blk = ie >> 5;
      const int li = (int)(ie & 31);
      const cx<R>* Ug = reinterpret_cast<const cx<R>*>(a.U) + blk * H * 32 + li;
      const cx<R>* Yg = reinterpret_cast<const cx<R>*>(a.Y) + blk * H * 32 + li;
#pragma unroll 8
      for (int el = sl; el < H; el += kFSlices) {
        const int p = __ldg(a.half_tmm + el);
        const R w8 = (R)half_weight(tmm_t(p), tmm_ma(p), tmm_mb(p));
        const cx<R> u = Ug[el * 32], y = Yg[el * 32];
        e += w8 * (y.re * u.re + y.im * u.im);
      }
    }
    double de = (double)e;
    de += __shfl_xor_sync(kFull, de, 8);
    de += __shfl_xor_sync(kFull, de, 16);
    if (lane < kFAtoms) ew[w][lane] = de;
  }
  const int cnt = min(cnt_raw, K);
  double f[4] = {0.0, 0.0, 0.0, 0.0};
  double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int s0 = 0; s0 < cnt; s0 += 2 * kFLanes) {
    // two slots per pass: the reverse slot (a pass over the neighbour's row
    // of pair keys, kept for the weighted gather) after the first-level
    // loads, then its dE/dr
    if (s0 > 0) load_slots(s0);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      ok[u] = s0 + u * kFLanes + l < cnt;
      if (ok[u]) {
        const long q = i * K + s0 + u * kFLanes + l;
        rv[u] = geo::find_rev_key(a, (int)i, q, kn[u], ky[u]);
        a.rev_out[q] = rv[u];
        if (rv[u] < 0) atomicMax(&a.flags[1], 1);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (ok[u] && rv[u] >= 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) dk[u][c] = a.dedr[((long)kn[u] * K + rv[u]) * 3 + c];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!ok[u]) continue;
#pragma unroll
      for (int c = 0; c < 3; ++c) f[c] += d[u][c] - dk[u][c];
      v[0] = fma(-d[u][0], r[u][0], v[0]);
      v[1] = fma(-d[u][1], r[u][1], v[1]);
      v[2] = fma(-d[u][2], r[u][2], v[2]);
      v[3] = fma(-d[u][0], r[u][1], v[3]);
      v[4] = fma(-d[u][0], r[u][2], v[4]);
      v[5] = fma(-d[u][1], r[u][2], v[5]);
    }
  }
  const double fsum = tree_sum<4, kFLanes>(f, lane);  // component l / 4
  if (have && l % 4 == 0 && l / 4 < 3) a.forces[3 * i + l / 4] = fsum;
  if (a.vatom) {  // batch mode: per-atom virial, reduced per configuration later
    const double vs = tree_sum<8, kFLanes>(v, lane);  // component l / 2
    if (have && l % 2 == 0 && l / 2 < 6) a.vatom[6 * i + l / 2] = vs;
  } else if (a.virial) {
    const double vs = tree_sum<8, 32>(v, lane);  // component lane / 4
    if (lane % 4 == 0) wv[w][lane / 4] = vs;
  }
  __syncthreads();
  if (a.energy && tid < na) {
    const double e = (ew[0][tid] + ew[1][tid]) + (ew[2][tid] + ew[3][tid]);
    a.energy[i0 + tid] = a.beta0 + e * (1.0 / 3.0);
  }
  const bool vir = !a.vatom && a.virial;
  if (!vir && !a.hflags) return;
  const int cta = blockIdx.x, ncta = gridDim.x;
  if (vir && tid < 6) a.vpart[6 * cta + tid] = (wv[0][tid] + wv[1][tid]) + (wv[2][tid] + wv[3][tid]);
  __syncthreads();
  // the fence after the barrier makes every write and flag update of this
  // CTA (the reverse-slot check's included) visible before its count
  if (tid == 0) {
    __threadfence();
    last = (atomicAdd(&a.flags[4], 1) == ncta - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (a.hflags) {
    // the evaluation's end: the status words to the host-mapped copy and all
    // flags zeroed for the next evaluation (no other CTA touches them now)
    __syncthreads();  // every thread of this CTA is past its own flag reads
    if (tid < 8) {
      const int v = __ldcg(a.flags + tid);
      if (tid < 4) a.hflags[tid] = v;
      a.flags[tid] = 0;
    }
  }
  if (!vir) return;
  // last CTA: thread t adds the CTA partials t, t + kFThreads, ... in order
  // (loads issued four at a time), then the same trees: a fixed order, so
  // the virial is deterministic
  double x[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b0 = tid; b0 < ncta; b0 += 4 * kFThreads) {
    double y[4][6];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int b = b0 + k * kFThreads;
#pragma unroll
      for (int c = 0; c < 6; ++c) y[k][c] = b < ncta ? __ldcg(a.vpart + 6 * b + c) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 6; ++c) x[c] += y[k][c];
  }
  const double xs = tree_sum<8, 32>(x, lane);
  if (lane % 4 == 0) wv[w][lane / 4] = xs;
  __syncthreads();
  if (tid < 6) a.virial[tid] = (wv[0][tid] + wv[1][tid]) + (wv[2][tid] + wv[3][tid]);
}

constexpr int kUiWarps = 4;
constexpr int kDeWarps = 4;

template <typename R>
size_t ui_smem(int H, int L) {
  return sizeof(R) * kRootDim * kRootDim + sizeof(cx<R>) * (size_t)kUiWarps * (H + 2 * L);
}
template <typename R>
size_t de_smem(int H, int L) {
  return sizeof(R) * kRootDim * kRootDim + sizeof(cx<R>) * (H + (size_t)kDeWarps * (H + 2 * L));
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  // the default 48 KB limit covers static and dynamic shared memory together
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (bytes + fa.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace


template <typename R>
cudaError_t launch_ui(const WorkArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const size_t sm = ui_smem<R>(a.H, a.lmax);
  cudaError_t e = allow_smem(ui_kernel<R, kUiWarps>, sm);
  if (e != cudaSuccess) return e;
  return launch_k(ui_kernel<R, kUiWarps>, dim3(a.n), dim3(kUiWarps * 32), sm, s, a);
}

template <typename R, bool STAGED, bool CP>
cudaError_t yi_occupancy(const YiGeometry& g, int* ctas) {
  cudaError_t e = STAGED ? allow_smem(yi_kernel<R, STAGED, CP>, g.smem) : cudaSuccess;
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, yi_kernel<R, STAGED, CP>, g.threads, g.smem);
}


YiGeometry yi_geometry(int rsize, int H, int n, int nsm, int waves) {
  YiGeometry g;
  g.nblk = (n + 31) / 32;
  const size_t block = (size_t)2 * H * 32 * rsize;  // one staged [H][32] complex block
  g.staged = block + 16 <= 200 * 1024;
  g.conjplane = yi_conjplane(rsize, H);
  g.smem = g.staged ? (g.conjplane ? 2 : 1) * block + 16 : 0;
  g.threads = (g.smem > 100 * 1024) ? 1024 : (g.smem > 60 * 1024 ? 512 : 256);
  // FP32 staged CTAs: a term-record ring per warp after the planes
  if (g.staged && rsize == 4) g.smem += (size_t)(g.threads / 32) * kYRingLen * sizeof(YRec<float>);
  int cps = 2048 / g.threads;
  if (g.staged) cps = std::max(1, std::min(cps, (int)((227 * 1024) / g.smem)));
  // the instance's real residency (registers can limit it further), queried
  // once per (precision, H)
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> occ_cache;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = occ_cache.find({rsize, H});
    if (it != occ_cache.end()) {
      occ = it->second;
    } else {
      cudaError_t oe;
      if (rsize == 4)
        oe = g.staged ? (g.conjplane ? yi_occupancy<float, true, true>(g, &occ)
                                     : yi_occupancy<float, true, false>(g, &occ))
                      : yi_occupancy<float, false, false>(g, &occ);
      else
        oe = g.staged ? (g.conjplane ? yi_occupancy<double, true, true>(g, &occ)
                                     : yi_occupancy<double, true, false>(g, &occ))
                      : yi_occupancy<double, false, false>(g, &occ);
      if (oe != cudaSuccess) {
        cudaGetLastError();
        occ = 0;
      } else {
        occ_cache[{rsize, H}] = occ;
      }
    }
  }
  if (occ > 0) cps = std::min(cps, occ);
  // Split each CTA's outputs into ysplit CTAs.  CTAs of one launch take about
  // equal time, so the launch lasts ceil(CTAs / resident) CTA lifetimes;
  // pick the split that minimises
  //   ceil(nblk ysplit / resident) (1 / ysplit + c),
  // c = the fixed per-CTA cost (staging U) relative to a whole block's terms,
  // taken as 0.02 / waves (the tunable: more waves, finer splits), and a
  // tenth of that without staging.  Staged FP64 keeps its pipe busy all the
  // time, so the CTAs an SM holds share it: there the count is the most CTAs
  // an SM takes, ceil(nblk ysplit / SMs), instead of the waves (2J8, 2000
  // atoms: 405 against 426 us).  Unstaged (2J14) it reads U through L1 and
  // wants the warps of the finer split (11.06 against 9.33 ms by the SM count).
  const long resident = (long)nsm * cps;
  const long per = (rsize == 8 && g.staged) ? (long)nsm : resident;
  const double c = (g.staged ? 0.02 : 0.002) / std::max(1, waves);
  double best = 1e300;
  g.ysplit = 1;
  for (int ys = 1; ys <= 64; ++ys) {
    const long w = ((long)g.nblk * ys + per - 1) / per;
    const double t = (double)w * (1.0 / ys + c);
    if (t < best - 1e-12) {
      best = t;
      g.ysplit = ys;
    }
  }
  g.nslices = g.ysplit * (g.threads / 32);
  return g;
}

template <typename R>
cudaError_t launch_yi(const WorkArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (a.yi_layout == 1) {
    const size_t sm = sizeof(cx<R>) * 2 * (size_t)a.H * kYaWarps;
    cudaError_t e = allow_smem(yi_atom_kernel<R>, sm);
    if (e != cudaSuccess) return e;
    return launch_k(yi_atom_kernel<R>, dim3((unsigned)((a.n + kYaWarps - 1) / kYaWarps)),
                    dim3(kYaWarps * 32), sm, s, a);
  }
  const YiGeometry g = yi_geometry(sizeof(R), a.H, a.n, a.nsm, a.yi_waves);
  if (g.nslices != a.nslices) return cudaErrorInvalidValue;
  if ((a.persist & 1) && g.staged) {
    // persistent: as many CTAs as stay resident, (block, split) items from the queue
    auto kq = g.conjplane ? yi_queue_kernel<R, true> : yi_queue_kernel<R, false>;
    cudaError_t e = allow_smem(kq, g.smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kq, g.threads, g.smem);
    if (e != cudaSuccess) return e;
    const long nitems = (long)g.nblk * g.ysplit;
    const long grid = std::min<long>(nitems, (long)a.nsm * std::max(1, occ));
    return launch_k(kq, dim3((unsigned)grid), dim3(g.threads), g.smem, s, a, g.ysplit);
  }
  dim3 grid(g.nblk, g.ysplit);
  if (g.staged && g.conjplane) {
    cudaError_t e = allow_smem(yi_kernel<R, true, true>, g.smem);
    if (e != cudaSuccess) return e;
    return launch_k(yi_kernel<R, true, true>, grid, dim3(g.threads), g.smem, s, a);
  }
  if (g.staged) {
    cudaError_t e = allow_smem(yi_kernel<R, true, false>, g.smem);
    if (e != cudaSuccess) return e;
    return launch_k(yi_kernel<R, true, false>, grid, dim3(g.threads), g.smem, s, a);
  }
  return launch_k(yi_kernel<R, false, false>, grid, dim3(g.threads), 0, s, a);
}

template <typename R>
cudaError_t launch_de(const WorkArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const size_t sm = de_smem<R>(a.H, a.lmax);
  cudaError_t e = allow_smem(de_kernel<R, kDeWarps>, sm);
  if (e != cudaSuccess) return e;
  return launch_k(de_kernel<R, kDeWarps>, dim3(a.n), dim3(kDeWarps * 32), sm, s, a);
}

template <typename R>
cudaError_t launch_force(const WorkArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const size_t sm = force_smem(a.K, a.vatom != nullptr);
  cudaError_t e = allow_smem(force_kernel<R>, sm);
  if (e != cudaSuccess) return e;
  return launch_k(force_kernel<R>, dim3((unsigned)((a.n + kFAtoms - 1) / kFAtoms)), dim3(kFThreads), sm, s, a);
}

// Bispectrum (dU == nullptr) or its derivative along dU into out [N][N_B]:
// grid (32-atom blocks, component runs a.nbparts), 8 warps a CTA.
BiPlan bi_plan(int rsize, int H, bool deriv, int maxchunks, int maxterms, int layout, bool have_cp) {
  BiPlan p;
  const size_t plane = (size_t)H * 32 * 2 * rsize;
  const size_t np = deriv ? 2 : 1;
  const size_t part = (size_t)maxchunks * 32 * rsize;
  p.staged = plane + 16 <= kBiSmemMax;              // U's block
  p.ds = deriv && np * plane + 16 <= kBiSmemMax;    // and the tangent's beside it
  const size_t ns = p.ds ? 2 : 1;                    // staged blocks
  // the conjugate plane when asked for, or (planned) when two CTAs still fit an SM
  p.cp = p.staged && (!deriv || p.ds) && have_cp && layout != 1 && 2 * ns * plane + 16 <= kBiSmemMax &&
         (layout == 2 || 2 * ns * plane + 16 + part <= kBiSmemPair);
  const size_t planes = p.staged ? (p.cp ? 2 : 1) * ns * plane + 16 : 0;
  p.gpart = planes + part > kBiSmemMax;
  const size_t base = planes + (p.gpart ? 0 : part);
  // a run's records (one more for the 16-byte-aligned start of FP32 records)
  // when they fit without losing the second CTA of an SM
  const size_t rec = (((size_t)maxterms + 1) * (rsize == 4 ? 8 : 16) + 15) / 16 * 16;
  p.rs = p.staged && base + rec <= (base <= kBiSmemPair ? kBiSmemPair : kBiSmemMax);
  p.rec_bytes = p.rs ? rec : 0;
  p.smem = base + p.rec_bytes;
  return p;
}

bool bi_plane_fits(int rsize, int H) { return 2 * (size_t)H * 32 * 2 * rsize + 16 <= kBiSmemMax; }

template <typename R, bool DERIV>
cudaError_t launch_bi_t(const WorkArgs& a, const void* dU, double* out, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const long nblk = (a.n + 31) / 32;
  const BiPlan p = bi_plan((int)sizeof(R), a.H, DERIV, a.bmaxchunks, a.bmaxterms, a.bi_layout, a.brec_cp != nullptr);
  R* gpart = p.gpart ? reinterpret_cast<R*>(a.bscratch) : nullptr;
  if (p.gpart && !gpart) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)nblk, (unsigned)a.nbparts);
  const cx<R>* d = reinterpret_cast<const cx<R>*>(dU);
  const unsigned rb = (unsigned)p.rec_bytes;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = allow_smem(kern, p.smem);
    if (e != cudaSuccess) return e;
    return launch_k(kern, grid, dim3(kBiThreads), p.smem, s, a, d, out, gpart, rb);
  };
  if (!p.staged) return go(bi_kernel<R, false, false, DERIV, false, false>);
  if (DERIV && !p.ds)  // U staged, dU through L1
    return p.rs ? go(bi_kernel<R, true, false, DERIV, true, false>) : go(bi_kernel<R, true, false, DERIV, false, false>);
  if (p.cp)
    return p.rs ? go(bi_kernel<R, true, true, DERIV, true, DERIV>) : go(bi_kernel<R, true, true, DERIV, false, DERIV>);
  return p.rs ? go(bi_kernel<R, true, false, DERIV, true, DERIV>) : go(bi_kernel<R, true, false, DERIV, false, DERIV>);
}

template <typename R>
cudaError_t launch_bi(const WorkArgs& a, cudaStream_t s) {
  return launch_bi_t<R, false>(a, nullptr, a.B, s);
}
template cudaError_t launch_bi<float>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_bi<double>(const WorkArgs&, cudaStream_t);

template <typename R>
cudaError_t launch_dbi(const WorkArgs& a, const void* dU, double* dB, cudaStream_t s) {
  return launch_bi_t<R, true>(a, dU, dB, s);
}
template cudaError_t launch_dbi<float>(const WorkArgs&, const void*, double*, cudaStream_t);
template cudaError_t launch_dbi<double>(const WorkArgs&, const void*, double*, cudaStream_t);

cudaError_t launch_force_weighted(const WorkArgs& a, const double* w, double* grad, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  return launch_k(force_weighted_kernel, dim3((a.n + 7) / 8), dim3(256), 0, s, a, w, grad);
}

// End of an evaluation: the status words (flags 0-3) go to the host-mapped
// copy, and every flag, counters included, is zeroed for the next
// evaluation (the kernels before it in the stream have completed).
__global__ void flags_out_kernel(int* __restrict__ flags, int* __restrict__ hflags) {
  const int t = threadIdx.x;
  if (t < 8) {
    const int v = flags[t];
    if (t < 4) hflags[t] = v;
    flags[t] = 0;
  }
}

cudaError_t launch_flags_out(int* flags, int* hflags, cudaStream_t s) {
  return launch_k(flags_out_kernel, dim3(1), dim3(32), 0, s, flags, hflags);
}

// Per-configuration virial: one CTA per configuration sums its atoms in a
// fixed order (strided partial sums, then a tree).
__global__ void __launch_bounds__(256) virial_conf_kernel(const double* __restrict__ vatom,
                                                          const NeighConf* __restrict__ confs,
                                                          double* __restrict__ virial) {
  __shared__ double red[256];
  const NeighConf c = confs[blockIdx.x];
  for (int k = 0; k < 6; ++k) {
    double t = 0.0;
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) t += vatom[6 * (long)(c.start + i) + k];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) virial[6 * blockIdx.x + k] = red[0];
    __syncthreads();
  }
}

cudaError_t launch_virial_conf(const double* vatom, const NeighConf* confs, int nconf, double* virial,
                               cudaStream_t s) {
  if (nconf <= 0) return cudaSuccess;
  return launch_k(virial_conf_kernel, dim3(nconf), dim3(256), 0, s, vatom, confs, virial);
}

template cudaError_t launch_ui<float>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_ui<double>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_yi<float>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_yi<double>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_de<float>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_de<double>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_force<float>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_force<double>(const WorkArgs&, cudaStream_t);

// ------------------------------------------------- FMA throughput probe
// Peak FMA rate of the working precision, for the roofline denominators:
// every thread runs kProbeChains independent multiply-add chains (enough to
// cover the pipeline latency) for `iters` rounds.  The chains' operands come
// from the arguments, and the sums are stored only under a condition the host
// never meets, so nothing is folded away.
constexpr int kProbeChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, R b, R c, R* sink) {
  R x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = R(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], b, c);
  }
  R t = R(0);
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) t += x[k];
  if (t == R(-12345.0)) sink[threadIdx.x] = t;
}

template <typename R>
cudaError_t fma_probe(int nsm, int iters, double* flops, float* ms, R* sink, cudaStream_t s) {
  const int blocks = nsm * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  // warm-up launch, then the timed one
  e = launch_k(fma_probe_kernel<R>, dim3(blocks), dim3(threads), 0, s, iters / 8, R(0.999), R(1e-3), sink);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch_k(fma_probe_kernel<R>, dim3(blocks), dim3(threads), 0, s, iters, R(0.999), R(1e-3), sink);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *flops = 2.0 * kProbeChains * 4 * (double)iters * blocks * threads;
  return e;
}
template cudaError_t fma_probe<float>(int, int, double*, float*, float*, cudaStream_t);
template cudaError_t fma_probe<double>(int, int, double*, float*, double*, cudaStream_t);

}  // namespace snap

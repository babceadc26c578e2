// snap_neigh.cuh -- device code of the neighbour build (build_neighborlist,
// arXiv:2011.12875 Sec. II-B and Listing 2), shared by the plain build
// kernels (snap_neigh.cu) and the fused neighbour + compute_U kernel
// (snap_colkernels.cuh).
//
// For every atom i: every atom k and periodic image s with
// |r_k + s L - r_i| < R_cut, into a fixed-capacity [N][K] table with exact
// FP64 separations.  SPLIT warps per centre atom each scan one contiguous
// part of the candidate range: lanes test 32 atoms k at a time in FP32 with a
// margin (all images in range) and the survivors are appended, in a fixed
// order (32-block, image, lane), to the part's candidate list in shared
// memory.  Then one warp per atom checks the parts' lists, concatenated in
// order, exactly in FP64 32 candidates at a time (FP64 runs at 1/64 of the
// FP32 rate, so it is spent once per atom, on dense lanes) and appends the
// accepted pairs with a ballot: the list is deterministic and identical to a
// sequential scan of all candidates, whatever SPLIT.
#pragma once
#include <math.h>

#include "snap_internal.h"

namespace snap {
namespace nb {

constexpr unsigned kFull = 0xffffffffu;

// Exact FP64 separation r_k + s L - r_i, computed so that the pairs (i,k,s)
// and (k,i,-s) get exactly opposite vectors (the list is then symmetric even
// at the cutoff).  No contraction into FMA: __d*_rn intrinsics.
__device__ __forceinline__ double sep1(int i, int k, double xi, double xk, int s, double L) {
  if (i < k) return __dsub_rn(__dadd_rn(xk, __dmul_rn((double)s, L)), xi);
  if (i > k) return -__dsub_rn(__dadd_rn(xi, __dmul_rn((double)(-s), L)), xk);
  return __dmul_rn((double)s, L);
}

// The same for |s| <= 1, where s L is exactly 0 or +-L: a select instead of
// the int -> double conversion and the multiply (both on the FP64 pipe).
__device__ __forceinline__ double sep1_near(int i, int k, double xi, double xk, int s, double L) {
  const double sl = s == 0 ? 0.0 : (s > 0 ? L : -L);
  if (i < k) return __dsub_rn(__dadd_rn(xk, sl), xi);
  if (i > k) return -__dsub_rn(__dadd_rn(xi, -sl), xk);
  return sl;
}

__device__ __forceinline__ double norm2(double x, double y, double z) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}

constexpr int kCandCap = 128;  // candidates per part (more: reported as overflow)

constexpr int kSure = 1 << 24;  // candidate flag: certainly within rcut

__device__ __forceinline__ int pack_img(int x, int y, int z) {
  return (x + 128) | ((y + 128) << 8) | ((z + 128) << 16);
}

// The build of one CTA's atoms (the body of the neighbour-build kernels).
// on_pair(al, i, slot, q, ex, ey, ez) is called, on the lane that writes
// it, for every pair stored in the table (al = the atom's index within the
// CTA, i its index, q = i * K + slot, ex..ez = the exact FP64 separation);
// the fused neighbour + compute_U kernel evaluates the slot geometry there.
template <bool BATCH, int SPLIT, int NW, typename OnPair>
__device__ __forceinline__ void neigh_build_cta(const NeighArgs& a, OnPair&& on_pair) {
  constexpr int kAtoms = NW / SPLIT;
  __shared__ int cand_j[NW][kCandCap];
  __shared__ int cand_s[NW][kCandCap];
  __shared__ int ncands[NW];
  __shared__ int cmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int part = warp % SPLIT, ai = warp / SPLIT;
  const unsigned lt = (1u << lane) - 1u;
  // candidate range [j_lo, j_hi), box and image range of this CTA's atoms
  int j_lo = 0, j_hi = a.n, i = blockIdx.x * kAtoms + ai;
  int Sx = a.Sx, Sy = a.Sy, Sz = a.Sz;
  double Ldx = a.Lx, Ldy = a.Ly, Ldz = a.Lz;
  if (BATCH) {
    const int2 m = a.cta_map[blockIdx.x];
    const NeighConf c = a.confs[m.x];
    j_lo = c.start;
    j_hi = c.start + c.n;
    i = c.start + m.y + ai;
    Ldx = c.L[0];
    Ldy = c.L[1];
    Ldz = c.L[2];
    Sx = c.S[0];
    Sy = c.S[1];
    Sz = c.S[2];
  }
  if (threadIdx.x == 0) cmax = 0;
  __syncthreads();  // before any warp's atomicMax on cmax
  const bool NEAREST = (Sx == 0 && Sy == 0 && Sz == 0);
  const bool active = i < j_hi;
  // this warp's part of the candidate range, in 32-blocks [b0, b1)
  const int nblk32 = (j_hi - j_lo + 31) / 32;
  const int per = (nblk32 + SPLIT - 1) / SPLIT;
  const int b0 = min(nblk32, per * part), b1 = min(nblk32, per * (part + 1));
  const int c1 = min(j_hi, j_lo + 32 * b1);
  int* cj = cand_j[warp];
  int* cs = cand_s[warp];
  int ncand = 0;  // candidates of this part (warp-uniform, may pass kCandCap)
  float4 pi4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (active) pi4 = a.pos4[i];
  const float Lx = (float)Ldx, Ly = (float)Ldy, Lz = (float)Ldz;
  const float iLx = 1.f / Lx, iLy = 1.f / Ly, iLz = 1.f / Lz;
  const float rcf = (float)a.rcut + 1e-2f;
  const float rc2f = rcf * rcf;
  // below rcut - 0.01 A in FP32 the pair is certainly within rcut
  const float rsf = fmaxf((float)a.rcut - 1e-2f, 0.f);
  const float rs2f = rsf * rsf;
  auto push = [&](bool c, int j, int pk) {
    const unsigned m = __ballot_sync(kFull, c);
    if (c) {
      const int p = ncand + __popc(m & lt);
      if (p < kCandCap) {
        cj[p] = j;
        cs[p] = pk;
      }
    }
    ncand += __popc(m);
  };
  // Far tiles are skipped: their minimum-image distance bound passes
  // rcut + 0.02 A, so they hold no candidate of the rcut + 0.01 A test and the
  // list is the same (single configuration, nearest image; tiles start at 0).
  // Each lane tests one of the next 32 tiles, and the warp scans the tiles
  // that pass, in order.
  const bool cull = !BATCH && NEAREST && a.tiles != nullptr;
  const float rcull2 = ((float)a.rcut + 2e-2f) * ((float)a.rcut + 2e-2f);
  if (active) {
    for (int bb = b0; bb < b1; bb += 32) {
      bool near = bb + lane < b1;
      if (cull && near) {
        const float4 tc = __ldg(a.tiles + 2 * (bb + lane)), th = __ldg(a.tiles + 2 * (bb + lane) + 1);
        float ex = tc.x - pi4.x, ey = tc.y - pi4.y, ez = tc.z - pi4.z;
        ex = fmaxf(fabsf(ex - Lx * rintf(ex * iLx)) - th.x, 0.f);
        ey = fmaxf(fabsf(ey - Ly * rintf(ey * iLy)) - th.y, 0.f);
        ez = fmaxf(fabsf(ez - Lz * rintf(ez * iLz)) - th.z, 0.f);
        near = ex * ex + ey * ey + ez * ez <= rcull2;
      }
      for (unsigned tm = __ballot_sync(kFull, near); tm; tm &= tm - 1) {
        const int j0 = j_lo + 32 * (bb + __ffs(tm) - 1);
        const int j = j0 + lane;
        const bool valid = j < c1;
        const float4 pj = valid ? __ldg(a.pos4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float dx0 = pj.x - pi4.x, dy0 = pj.y - pi4.y, dz0 = pj.z - pi4.z;
        // nearest-image shift counts, kept in float (int <-> float conversions
        // run on a slow pipe and are only done for the rare candidates)
        const float nxf = -rintf(dx0 * iLx), nyf = -rintf(dy0 * iLy), nzf = -rintf(dz0 * iLz);
        const float bx = dx0 + nxf * Lx, by = dy0 + nyf * Ly, bz = dz0 + nzf * Lz;
        if (NEAREST) {
          // box > 2 (rcut + margin) in every direction: only the nearest image
          const float d2 = bx * bx + by * by + bz * bz;
          const bool c = valid && (d2 < rc2f) && (j != i);
          push(c, j, c ? pack_img((int)nxf, (int)nyf, (int)nzf) | (d2 < rs2f ? kSure : 0) : 0);
          continue;
        }
        float sxf = -(float)Sx;
        for (int sx = -Sx; sx <= Sx; ++sx, sxf += 1.f) {
          float syf = -(float)Sy;
          for (int sy = -Sy; sy <= Sy; ++sy, syf += 1.f) {
            float szf = -(float)Sz;
            for (int sz = -Sz; sz <= Sz; ++sz, szf += 1.f) {
              const float fx = bx + sxf * Lx, fy = by + syf * Ly, fz = bz + szf * Lz;
              const float d2 = fx * fx + fy * fy + fz * fz;
              bool c = valid && (d2 < rc2f);
              int ix = 0, iy = 0, iz = 0;
              if (c) {
                ix = (int)(nxf + sxf);
                iy = (int)(nyf + syf);
                iz = (int)(nzf + szf);
                c = !((j == i) && ix == 0 && iy == 0 && iz == 0);
              }
              push(c, j, c ? pack_img(ix, iy, iz) | (d2 < rs2f ? kSure : 0) : 0);
            }
          }
        }
      }
    }
  }
  if (lane == 0) ncands[warp] = ncand;
  if (SPLIT > 1) __syncthreads();
  else __syncwarp();
  if (active && part == 0) {
    // exact FP64 check of the concatenated candidate lists
    int off[SPLIT + 1];
    off[0] = 0;
    bool over = false;
    for (int p = 0; p < SPLIT; ++p) {
      const int c = ncands[warp + p];
      over |= c > kCandCap;
      off[p + 1] = off[p] + min(c, kCandCap);
    }
    const double xi = a.pos[3 * i], yi = a.pos[3 * i + 1], zi = a.pos[3 * i + 2];
    const double rc2 = a.rcut * a.rcut;
    int count = 0;
    for (int e0 = 0; e0 < off[SPLIT]; e0 += 32) {
      const int e = e0 + lane;
      const bool have = e < off[SPLIT];
      double ex = 0, ey = 0, ez = 0;
      int j = 0, ix = 0, iy = 0, iz = 0, pk = 0;
      if (have) {
        int p = 0;
        while (e >= off[p + 1]) ++p;
        j = cand_j[warp + p][e - off[p]];
        pk = cand_s[warp + p][e - off[p]];
        ix = (pk & 0xff) - 128;
        iy = ((pk >> 8) & 0xff) - 128;
        iz = ((pk >> 16) & 0xff) - 128;
      }
      // FP64 is spent only where needed, decided for the whole warp: the
      // select shift when every image is within one box, the exact distance
      // test unless every candidate is certainly inside
      // (both votes are taken by all 32 lanes, outside any branch)
      const bool all_near =
          __all_sync(kFull, !have || (abs(ix) <= 1 && abs(iy) <= 1 && abs(iz) <= 1));
      const bool sure = have && (pk & kSure);
      const bool all_sure = __all_sync(kFull, !have || sure);
      if (have) {
        const double xj = a.pos[3 * j], yj = a.pos[3 * j + 1], zj = a.pos[3 * j + 2];
        if (all_near) {
          ex = sep1_near(i, j, xi, xj, ix, Ldx);
          ey = sep1_near(i, j, yi, yj, iy, Ldy);
          ez = sep1_near(i, j, zi, zj, iz, Ldz);
        } else {
          ex = sep1(i, j, xi, xj, ix, Ldx);
          ey = sep1(i, j, yi, yj, iy, Ldy);
          ez = sep1(i, j, zi, zj, iz, Ldz);
        }
      }
      bool in = sure;
      if (!all_sure) in = have && (sure || norm2(ex, ey, ez) < rc2);
      const unsigned m = __ballot_sync(kFull, in);
      if (in) {
        const int slot = count + __popc(m & lt);
        if (slot < a.K) {
          const long q = (long)i * a.K + slot;
          a.nbr[q] = j;
          a.img[3 * q] = (signed char)ix;
          a.img[3 * q + 1] = (signed char)iy;
          a.img[3 * q + 2] = (signed char)iz;
          a.rij[3 * q] = ex;
          a.rij[3 * q + 1] = ey;
          a.rij[3 * q + 2] = ez;
          if (a.key) a.key[q] = pair_key(j, ix, iy, iz, a.n);
          on_pair(ai, (long)i, slot, q, ex, ey, ez);
        }
      }
      count += __popc(m);
    }
    // a part with more candidates than it can hold is reported as a list
    // overflow (the caller sees a count above any capacity)
    if (over) count = max(count, 1 << 20);
    if (lane == 0) {
      a.cnt[i] = min(count, a.K);
      atomicMax(&cmax, count);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&a.flags[0], cmax);
}


}  // namespace nb
}  // namespace snap

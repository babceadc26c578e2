// snap_neigh.cu -- neighbour list.
//
// The neighbour list is the build_neighborlist stage of the SNAP algorithm
// (arXiv:2011.12875, Sec. II-B and Listing 2): for every atom i, every atom k
// and periodic image s with |r_k + s L - r_i| < R_cut.  Here it is built on
// the device into a fixed-capacity [N][K] table with exact FP64 separations
// (the slot geometry and reverse-slot map are derived from it in
// snap_geom.cuh).
#include <math.h>

#include "snap_internal.h"

namespace snap {

namespace {

constexpr int kNbWarps = 8;        // warps per CTA of the batch build
constexpr int kNbWarpsSingle = 2;  // warps (= atoms) per CTA of a single configuration: small
                                   // CTAs spread the one-warp atoms evenly over the SMs
// Warps per centre atom: a batch build scans every block of its
// configuration, so four warps share the scan; a single-configuration build
// skips far tiles and one warp per atom suffices.
constexpr int kNbSplitBatch = 4;
static_assert(kNbWarps / kNbSplitBatch == kNeighAtomsPerCta, "batch CTA map and kernel disagree");
constexpr unsigned kFull = 0xffffffffu;

// FP32 positions, (when `tiles` is given) the bounding box of every tile of
// 32 consecutive atoms as an FP32 centre and half extent, padded by 1e-4 A for
// rounding, and (when `copy` is given) a device copy of the FP64 positions,
// for positions read from mapped host memory.  Blocks are whole warps, one
// tile per warp.
__global__ void pos4_kernel(int n, const double* __restrict__ pos, float4* __restrict__ pos4,
                            float4* __restrict__ tiles, double* __restrict__ copy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool ok = i < n;
  float x = 0.f, y = 0.f, z = 0.f;
  if (ok) {
    const double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    if (copy) {
      copy[3 * i] = px;
      copy[3 * i + 1] = py;
      copy[3 * i + 2] = pz;
    }
    x = (float)px;
    y = (float)py;
    z = (float)pz;
    pos4[i] = make_float4(x, y, z, 0.f);
  }
  if (!tiles) return;  // uniform over the grid
  float lx = ok ? x : INFINITY, ly = ok ? y : INFINITY, lz = ok ? z : INFINITY;
  float hx = ok ? x : -INFINITY, hy = ok ? y : -INFINITY, hz = ok ? z : -INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lx = fminf(lx, __shfl_xor_sync(kFull, lx, o));
    ly = fminf(ly, __shfl_xor_sync(kFull, ly, o));
    lz = fminf(lz, __shfl_xor_sync(kFull, lz, o));
    hx = fmaxf(hx, __shfl_xor_sync(kFull, hx, o));
    hy = fmaxf(hy, __shfl_xor_sync(kFull, hy, o));
    hz = fmaxf(hz, __shfl_xor_sync(kFull, hz, o));
  }
  if (lane == 0 && ok) {
    const int t = i >> 5;
    tiles[2 * t] = make_float4(0.5f * (lx + hx), 0.5f * (ly + hy), 0.5f * (lz + hz), 0.f);
    tiles[2 * t + 1] = make_float4(0.5f * (hx - lx) + 1e-4f, 0.5f * (hy - ly) + 1e-4f, 0.5f * (hz - lz) + 1e-4f, 0.f);
  }
}

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

// SPLIT warps per centre atom i, each scanning one contiguous part of the
// candidate range: lanes test 32 atoms k at a time in FP32 with a margin (all
// images in range) and the survivors are appended, in a fixed order
// (32-block, image, lane), to the part's candidate list in shared memory.
// Then one warp per atom checks the parts' lists, concatenated in order,
// exactly in FP64 32 candidates at a time (FP64 runs at 1/64 of the FP32 rate,
// so it is spent once per atom, on dense lanes) and appends the accepted
// pairs with a ballot: the list is deterministic and identical to a
// sequential scan of all candidates.
constexpr int kCandCap = 128;  // candidates per part (more: reported as overflow)

constexpr int kSure = 1 << 24;  // candidate flag: certainly within rcut

__device__ __forceinline__ int pack_img(int x, int y, int z) {
  return (x + 128) | ((y + 128) << 8) | ((z + 128) << 16);
}

template <bool BATCH, int SPLIT, int NW>
__global__ void __launch_bounds__(NW * 32) neigh_build_kernel(NeighArgs a) {
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

// Caller-supplied list -> internal [N][K] tables with exact separations.
__global__ void neigh_ingest_kernel(int n, int K, const double* __restrict__ pos, double Lx,
                                    double Ly, double Lz, const int* __restrict__ ucnt,
                                    const int* __restrict__ uidx, const signed char* __restrict__ uimg,
                                    int ucap, int* cnt, int* nbr, signed char* img, double* rij,
                                    int* flags) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)n * K) return;
  const int i = (int)(q / K), s = (int)(q - (long)i * K);
  int c = ucnt[i];
  if (s == 0) {
    if (c < 0 || c > ucap) atomicMax(&flags[2], 1);
    atomicMax(&flags[0], c);
    cnt[i] = min(max(c, 0), K);
  }
  if (s >= min(c, K)) return;
  const long u = (long)i * ucap + s;
  const int k = uidx[u];
  if (k < 0 || k >= n) {
    atomicMax(&flags[2], 1);
    nbr[q] = i;
    img[3 * q] = img[3 * q + 1] = img[3 * q + 2] = 0;
    rij[3 * q] = rij[3 * q + 1] = rij[3 * q + 2] = 1e30;  // beyond rcut: ignored
    return;
  }
  const int ix = uimg[3 * u], iy = uimg[3 * u + 1], iz = uimg[3 * u + 2];
  nbr[q] = k;
  img[3 * q] = (signed char)ix;
  img[3 * q + 1] = (signed char)iy;
  img[3 * q + 2] = (signed char)iz;
  rij[3 * q] = sep1(i, k, pos[3 * i], pos[3 * k], ix, Lx);
  rij[3 * q + 1] = sep1(i, k, pos[3 * i + 1], pos[3 * k + 1], iy, Ly);
  rij[3 * q + 2] = sep1(i, k, pos[3 * i + 2], pos[3 * k + 2], iz, Lz);
}

inline int blocks_for(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_pos4(int n, const double* pos, float4* pos4, cudaStream_t s, float4* tiles,
                        double* copy) {
  if (n <= 0) return cudaSuccess;
  return launch_k(pos4_kernel, dim3(blocks_for(n, 256)), dim3(256), 0, s, n, pos, pos4, tiles, copy);
}

cudaError_t launch_neigh_build(const NeighArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  return launch_k(neigh_build_kernel<false, 1, kNbWarpsSingle>, dim3(blocks_for(a.n, kNbWarpsSingle)),
                  dim3(kNbWarpsSingle * 32), 0, s, a);
}

cudaError_t launch_neigh_build_batch(const NeighArgs& a, int ncta, cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  return launch_k(neigh_build_kernel<true, kNbSplitBatch, kNbWarps>, dim3(ncta), dim3(kNbWarps * 32), 0, s, a);
}

cudaError_t launch_neigh_ingest(int n, int K, const double* pos, double Lx, double Ly,
                                double Lz, const int* ucnt, const int* uidx,
                                const signed char* uimg, int ucap, int* cnt, int* nbr,
                                signed char* img, double* rij, int* flags, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return launch_k(neigh_ingest_kernel, dim3(blocks_for((long)n * K, 256)), dim3(256), 0, s, n, K, pos, Lx, Ly, Lz, ucnt, uidx, uimg, ucap, cnt, nbr, img, rij, flags);
}


}  // namespace snap

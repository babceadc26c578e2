// snap_neigh.cu -- neighbour list, reverse-slot map and per-slot FP64
// Cayley-Klein geometry.
//
// The neighbour list is the build_neighborlist stage of the SNAP algorithm
// (arXiv:2011.12875, Sec. II-B and Listing 2): for every atom i, every atom k
// and periodic image s with |r_k + s L - r_i| < R_cut.  Here it is built on
// the device into a fixed-capacity [N][K] table.  The reverse-slot map lets
// the force stage gather dE_k/dr_ki instead of scattering with atomics.
#include <math.h>

#include "snap_internal.h"

namespace snap {

namespace {

constexpr int kNbWarps = 8;   // centre atoms per CTA (one warp each)
constexpr int kNbTile = 256;  // candidate atoms staged per shared-memory tile
constexpr unsigned kFull = 0xffffffffu;

__global__ void pos4_kernel(int n, const double* __restrict__ pos, float4* __restrict__ pos4) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pos4[i] = make_float4((float)pos[3 * i], (float)pos[3 * i + 1], (float)pos[3 * i + 2], 0.f);
}

// Exact FP64 separation r_k + s L - r_i, computed so that the pairs (i,k,s)
// and (k,i,-s) get exactly opposite vectors (the list is then symmetric even
// at the cutoff).  No contraction into FMA: __d*_rn intrinsics.
__device__ __forceinline__ double sep1(int i, int k, double xi, double xk, int s, double L) {
  if (i < k) return __dsub_rn(__dadd_rn(xk, __dmul_rn((double)s, L)), xi);
  if (i > k) return -__dsub_rn(__dadd_rn(xi, __dmul_rn((double)(-s), L)), xk);
  return __dmul_rn((double)s, L);
}

__device__ __forceinline__ double norm2(double x, double y, double z) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}

// One warp per centre atom i.  Lanes first test 32 atoms k at a time in
// FP32 with a margin (all images in range); the survivors are appended, in a
// fixed order (tile, image, lane), to a per-warp candidate list in shared
// memory.  Every 32 candidates, the list is checked exactly in FP64 with all
// lanes busy, and accepted pairs are appended to the output with a ballot, so
// the list is deterministic and FP64 work is spent only on real candidates.
constexpr int kCandCap = 64;

__device__ __forceinline__ int pack_img(int x, int y, int z) {
  return (x + 128) | ((y + 128) << 8) | ((z + 128) << 16);
}

__device__ __forceinline__ void exact_batch(const NeighArgs& a, double Lx, double Ly, double Lz, int i,
                                            double xi, double yi, double zi, double rc2, const int* cj,
                                            const int* cs, int nb, int lane, int& count) {
  bool in = false;
  double ex = 0, ey = 0, ez = 0;
  int j = 0, ix = 0, iy = 0, iz = 0;
  if (lane < nb) {
    j = cj[lane];
    const int pk = cs[lane];
    ix = (pk & 0xff) - 128;
    iy = ((pk >> 8) & 0xff) - 128;
    iz = ((pk >> 16) & 0xff) - 128;
    ex = sep1(i, j, xi, a.pos[3 * j], ix, Lx);
    ey = sep1(i, j, yi, a.pos[3 * j + 1], iy, Ly);
    ez = sep1(i, j, zi, a.pos[3 * j + 2], iz, Lz);
    in = norm2(ex, ey, ez) < rc2;
  }
  const unsigned m = __ballot_sync(kFull, in);
  if (in) {
    const int slot = count + __popc(m & ((1u << lane) - 1u));
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

template <bool BATCH>
__global__ void __launch_bounds__(kNbWarps * 32) neigh_build_kernel(NeighArgs a) {
  __shared__ float4 tile[kNbTile];
  __shared__ int cand_j[kNbWarps][kCandCap];
  __shared__ int cand_s[kNbWarps][kCandCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // candidate range [j_lo, j_hi), box and image range of this CTA's atoms
  int j_lo = 0, j_hi = a.n, i = blockIdx.x * kNbWarps + warp;
  int Sx = a.Sx, Sy = a.Sy, Sz = a.Sz;
  double Ldx = a.Lx, Ldy = a.Ly, Ldz = a.Lz;
  if (BATCH) {
    const int2 m = a.cta_map[blockIdx.x];
    const NeighConf c = a.confs[m.x];
    j_lo = c.start;
    j_hi = c.start + c.n;
    i = c.start + m.y + warp;
    Ldx = c.L[0];
    Ldy = c.L[1];
    Ldz = c.L[2];
    Sx = c.S[0];
    Sy = c.S[1];
    Sz = c.S[2];
  }
  const bool NEAREST = (Sx == 0 && Sy == 0 && Sz == 0);
  const bool active = i < j_hi;
  int* cj = cand_j[warp];
  int* cs = cand_s[warp];
  float4 pi4 = make_float4(0.f, 0.f, 0.f, 0.f);
  double xi = 0, yi = 0, zi = 0;
  if (active) {
    pi4 = a.pos4[i];
    xi = a.pos[3 * i];
    yi = a.pos[3 * i + 1];
    zi = a.pos[3 * i + 2];
  }
  const float Lx = (float)Ldx, Ly = (float)Ldy, Lz = (float)Ldz;
  const float iLx = 1.f / Lx, iLy = 1.f / Ly, iLz = 1.f / Lz;
  const float rcf = (float)a.rcut + 1e-2f;
  const float rc2f = rcf * rcf;
  const double rc2 = a.rcut * a.rcut;
  const unsigned lt = (1u << lane) - 1u;
  int count = 0;  // accepted pairs (warp-uniform)
  int ncand = 0;  // pending candidates (warp-uniform)
  for (int j0 = j_lo; j0 < j_hi; j0 += kNbTile) {
    __syncthreads();
    for (int q = threadIdx.x; q < kNbTile; q += blockDim.x)
      tile[q] = (j0 + q < j_hi) ? a.pos4[j0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    if (!active) continue;
    const int jn = min(kNbTile, j_hi - j0);
    for (int jj = 0; jj < jn; jj += 32) {
      const int j = j0 + jj + lane;
      const bool valid = (jj + lane) < jn;
      const float4 pj = tile[jj + lane];
      const float dx0 = pj.x - pi4.x, dy0 = pj.y - pi4.y, dz0 = pj.z - pi4.z;
      // nearest-image shift counts, kept in float (int <-> float conversions
      // run on a slow pipe and are only done for the rare candidates)
      const float nxf = -rintf(dx0 * iLx), nyf = -rintf(dy0 * iLy), nzf = -rintf(dz0 * iLz);
      const float bx = dx0 + nxf * Lx, by = dy0 + nyf * Ly, bz = dz0 + nzf * Lz;
      if (NEAREST) {
        // box > 2 (rcut + margin) in every direction: only the nearest image
        bool c = valid && (bx * bx + by * by + bz * bz < rc2f) && (j != i);
        const unsigned m = __ballot_sync(kFull, c);
        if (m) {
          if (c) {
            const int pos = ncand + __popc(m & lt);
            cj[pos] = j;
            cs[pos] = pack_img((int)nxf, (int)nyf, (int)nzf);
          }
          ncand += __popc(m);
          if (ncand >= 32) {
            __syncwarp();
            exact_batch(a, Ldx, Ldy, Ldz, i, xi, yi, zi, rc2, cj, cs, 32, lane, count);
            __syncwarp();
            const int rest = ncand - 32;
            int mj = 0, ms = 0;
            if (lane < rest) {
              mj = cj[32 + lane];
              ms = cs[32 + lane];
            }
            __syncwarp();
            if (lane < rest) {
              cj[lane] = mj;
              cs[lane] = ms;
            }
            ncand = rest;
            __syncwarp();
          }
        }
        continue;
      }
      float sxf = -(float)Sx;
      for (int sx = -Sx; sx <= Sx; ++sx, sxf += 1.f) {
        float syf = -(float)Sy;
        for (int sy = -Sy; sy <= Sy; ++sy, syf += 1.f) {
          float szf = -(float)Sz;
          for (int sz = -Sz; sz <= Sz; ++sz, szf += 1.f) {
            const float fx = bx + sxf * Lx, fy = by + syf * Ly, fz = bz + szf * Lz;
            bool c = valid && (fx * fx + fy * fy + fz * fz < rc2f);
            int ix = 0, iy = 0, iz = 0;
            if (c) {
              ix = (int)(nxf + sxf);
              iy = (int)(nyf + syf);
              iz = (int)(nzf + szf);
              c = !((j == i) && ix == 0 && iy == 0 && iz == 0);
            }
            const unsigned m = __ballot_sync(kFull, c);
            if (c) {
              const int pos = ncand + __popc(m & lt);
              cj[pos] = j;
              cs[pos] = pack_img(ix, iy, iz);
            }
            ncand += __popc(m);
            if (ncand >= 32) {
              __syncwarp();
              exact_batch(a, Ldx, Ldy, Ldz, i, xi, yi, zi, rc2, cj, cs, 32, lane, count);
              __syncwarp();
              const int rest = ncand - 32;
              int mj = 0, ms = 0;
              if (lane < rest) {
                mj = cj[32 + lane];
                ms = cs[32 + lane];
              }
              __syncwarp();
              if (lane < rest) {
                cj[lane] = mj;
                cs[lane] = ms;
              }
              ncand = rest;
              __syncwarp();
            }
          }
        }
      }
    }
  }
  __shared__ int cmax;
  if (threadIdx.x == 0) cmax = 0;
  __syncthreads();
  if (active) {
    __syncwarp();
    if (ncand > 0) exact_batch(a, Ldx, Ldy, Ldz, i, xi, yi, zi, rc2, cj, cs, ncand, lane, count);
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

// Reverse-slot map and FP64 Cayley-Klein geometry, once per unordered pair.
//
// rev[i][s] is the slot of the opposite pair (k, i, -s) in k's list (the
// force gather reads dE_k/dr_ki through it).  The geometry of a slot
// (Sec. II-A: the neighbour vector mapped to the 3-sphere, with constants
// from the paper's SNAP reference): theta0 = rfac0 pi (r - rmin0)/(rcut -
// rmin0), z0 = r cot theta0, r0 = sqrt(r^2 + z0^2), a = (z0 - i z)/r0,
// b = (y - i x)/r0, the cosine switching function f_c, and the derivatives
// of a, b and f_c with respect to r.  For the opposite vector -r the same
// quantities are a' = conj(a), b' = -b, grad f_c' = -grad f_c,
// da'/dr = -conj(da/dr), db'/dr = db/dr, exactly, so only one slot of each
// pair is evaluated (in FP64) and both are written (in the working
// precision G).  A CTA collects the canonical slots of kPairAtoms atoms in
// shared memory first, so the FP64 work runs on dense lanes.
constexpr int kPairAtoms = 2;
constexpr int kPairThreads = 64;

template <typename G>
__device__ void write_geom(G* g, G* gm, double ar, double ai, double br, double bi, double fc,
                           const double* dfc, const double* da, const double* db) {
  G v[kGeomStride];
  v[0] = G(ar);
  v[1] = G(ai);
  v[2] = G(br);
  v[3] = G(bi);
  v[4] = G(fc);
  for (int d = 0; d < 3; ++d) {
    v[5 + d] = G(dfc[d]);
    v[8 + 2 * d] = G(da[2 * d]);
    v[9 + 2 * d] = G(da[2 * d + 1]);
    v[14 + 2 * d] = G(db[2 * d]);
    v[15 + 2 * d] = G(db[2 * d + 1]);
  }
  for (int e = 0; e < kGeomStride; ++e) g[e] = v[e];
  if (!gm) return;
  // opposite vector: a -> conj(a), b -> -b, grad f_c -> -grad f_c,
  // da -> -conj(da), db -> db (negation is exact in any precision)
  gm[0] = v[0];
  gm[1] = -v[1];
  gm[2] = -v[2];
  gm[3] = -v[3];
  gm[4] = v[4];
  for (int d = 0; d < 3; ++d) {
    gm[5 + d] = -v[5 + d];
    gm[8 + 2 * d] = -v[8 + 2 * d];
    gm[9 + 2 * d] = v[9 + 2 * d];
    gm[14 + 2 * d] = v[14 + 2 * d];
    gm[15 + 2 * d] = v[15 + 2 * d];
  }
}

template <typename G>
__global__ void __launch_bounds__(kPairThreads) pairs_kernel(WorkArgs a, int* rev) {
  __shared__ long qs[kPairAtoms * kMaxNeighCap];
  __shared__ long qm[kPairAtoms * kMaxNeighCap];
  __shared__ int ncanon;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) ncanon = 0;
  __syncthreads();
  constexpr int per_warp = kPairAtoms / (kPairThreads / 32);
  for (int aa = 0; aa < per_warp; ++aa) {
    const int i = blockIdx.x * kPairAtoms + warp * per_warp + aa;
    if (i >= a.n) break;
    const int cnt = a.cnt[i];
    for (int s0 = 0; s0 < cnt; s0 += 32) {
      const int s = s0 + lane;
      bool canon = false;
      long q = 0, q2 = -1;
      if (s < cnt) {
        q = (long)i * a.K + s;
        const int k = a.nbr[q];
        const int sx = a.img[3 * q], sy = a.img[3 * q + 1], sz = a.img[3 * q + 2];
        const int ck = a.cnt[k];
        int found = -1;
        // all of k's slots are read with independent loads (no early exit)
        const int* kn = a.nbr + (long)k * a.K;
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
        rev[q] = found;
        if (found < 0) atomicMax(&a.flags[1], 1);
        const bool pos = sx > 0 || (sx == 0 && (sy > 0 || (sy == 0 && sz > 0)));
        canon = found < 0 || i < k || (i == k && pos);
        if (found >= 0) q2 = (long)k * a.K + found;
      }
      const unsigned m = __ballot_sync(0xffffffffu, canon);
      int base = 0;
      if (lane == 0) base = atomicAdd(&ncanon, __popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (canon) {
        const int p = base + __popc(m & lt);
        qs[p] = q;
        qm[p] = q2;
      }
    }
  }
  __syncthreads();
  const int nc = ncanon;
  for (int p = threadIdx.x; p < nc; p += blockDim.x) {
    const long q = qs[p], q2 = qm[p];
    G* g = reinterpret_cast<G*>(a.geom) + q * kGeomStride;
    G* gm = q2 >= 0 ? reinterpret_cast<G*>(a.geom) + q2 * kGeomStride : nullptr;
    const double x = a.rij[3 * q], y = a.rij[3 * q + 1], z = a.rij[3 * q + 2];
    const double r2 = x * x + y * y + z * z;
    const double ir = rsqrt(r2);
    const double r = r2 * ir;
    double dfc[3] = {0, 0, 0}, da[6] = {0, 0, 0, 0, 0, 0}, db[6] = {0, 0, 0, 0, 0, 0};
    if (!(r < a.rcut)) {  // outside the cutoff (caller lists): no contribution
      write_geom(g, gm, 1.0, 0.0, 0.0, 0.0, 0.0, dfc, da, db);
      continue;
    }
    const double c = a.rfac0 * M_PI * a.inv_span;  // d theta0 / d r
    double st, ct;
    sincospi(a.rfac0 * (r - a.rmin0) * a.inv_span, &st, &ct);
    const double ist = 1.0 / st;
    const double z0 = r * ct * ist;
    const double dz0dr = ct * ist - r * c * ist * ist;
    const double ir0 = rsqrt(r2 + z0 * z0);
    const double ar = z0 * ir0, ai = -z * ir0;
    const double br = y * ir0, bi = -x * ir0;
    double fc = 1.0, dfcdr = 0.0;
    if (a.switchflag && r > a.rmin0) {
      double sw, cw;
      sincospi((r - a.rmin0) * a.inv_span, &sw, &cw);
      fc = 0.5 * (cw + 1.0);
      dfcdr = -0.5 * M_PI * a.inv_span * sw;
    }
    const double rv[3] = {x, y, z};
    for (int d = 0; d < 3; ++d) {
      const double ud = rv[d] * ir;
      dfc[d] = dfcdr * ud;
      const double dz0 = dz0dr * ud;
      const double dr0 = (r * ud + z0 * dz0) * ir0;
      // d a = (d(z0 - i z) - a d r0) / r0 ; d b = (d(y - i x) - b d r0) / r0
      da[2 * d] = (dz0 - ar * dr0) * ir0;
      da[2 * d + 1] = ((d == 2 ? -1.0 : 0.0) - ai * dr0) * ir0;
      db[2 * d] = ((d == 1 ? 1.0 : 0.0) - br * dr0) * ir0;
      db[2 * d + 1] = ((d == 0 ? -1.0 : 0.0) - bi * dr0) * ir0;
    }
    write_geom(g, gm, ar, ai, br, bi, fc, dfc, da, db);
  }
}

inline int blocks_for(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_pos4(int n, const double* pos, float4* pos4, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  pos4_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, pos, pos4);
  return cudaGetLastError();
}

cudaError_t launch_neigh_build(const NeighArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  neigh_build_kernel<false><<<blocks_for(a.n, kNbWarps), kNbWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_neigh_build_batch(const NeighArgs& a, int ncta, cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  neigh_build_kernel<true><<<ncta, kNbWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_neigh_ingest(int n, int K, const double* pos, double Lx, double Ly,
                                double Lz, const int* ucnt, const int* uidx,
                                const signed char* uimg, int ucap, int* cnt, int* nbr,
                                signed char* img, double* rij, int* flags, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  neigh_ingest_kernel<<<blocks_for((long)n * K, 256), 256, 0, s>>>(
      n, K, pos, Lx, Ly, Lz, ucnt, uidx, uimg, ucap, cnt, nbr, img, rij, flags);
  return cudaGetLastError();
}

template <typename G>
cudaError_t launch_pairs(const WorkArgs& a, int* rev, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  pairs_kernel<G><<<blocks_for(a.n, kPairAtoms), kPairThreads, 0, s>>>(a, rev);
  return cudaGetLastError();
}
template cudaError_t launch_pairs<float>(const WorkArgs&, int*, cudaStream_t);
template cudaError_t launch_pairs<double>(const WorkArgs&, int*, cudaStream_t);

}  // namespace snap

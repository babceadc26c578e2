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

constexpr int kNbWarps = 8;                       // warps per CTA
constexpr int kNbSplit = 4;                       // warps per centre atom
constexpr int kNbAtoms = kNbWarps / kNbSplit;     // centre atoms per CTA
static_assert(kNbAtoms == kNeighAtomsPerCta, "batch CTA map and kernel disagree");
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

// kNbSplit warps per centre atom i, each scanning one contiguous part of the
// candidate range: lanes test 32 atoms k at a time in FP32 with a margin (all
// images in range) and the survivors are appended, in a fixed order
// (32-block, image, lane), to the part's candidate list in shared memory.
// Then one warp per atom checks the parts' lists, concatenated in order,
// exactly in FP64 32 candidates at a time (FP64 runs at 1/64 of the FP32 rate,
// so it is spent once per atom, on dense lanes) and appends the accepted
// pairs with a ballot: the list is deterministic and identical to a
// sequential scan of all candidates.
constexpr int kCandCap = 128;  // candidates per part (more: reported as overflow)

__device__ __forceinline__ int pack_img(int x, int y, int z) {
  return (x + 128) | ((y + 128) << 8) | ((z + 128) << 16);
}

template <bool BATCH>
__global__ void __launch_bounds__(kNbWarps * 32) neigh_build_kernel(NeighArgs a) {
  __shared__ int cand_j[kNbWarps][kCandCap];
  __shared__ int cand_s[kNbWarps][kCandCap];
  __shared__ int ncands[kNbWarps];
  __shared__ int cmax;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int part = warp % kNbSplit, ai = warp / kNbSplit;
  const unsigned lt = (1u << lane) - 1u;
  // candidate range [j_lo, j_hi), box and image range of this CTA's atoms
  int j_lo = 0, j_hi = a.n, i = blockIdx.x * kNbAtoms + ai;
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
  const bool NEAREST = (Sx == 0 && Sy == 0 && Sz == 0);
  const bool active = i < j_hi;
  // this warp's part of the candidate range, in 32-blocks
  const int nblk32 = (j_hi - j_lo + 31) / 32;
  const int per = (nblk32 + kNbSplit - 1) / kNbSplit;
  const int c0 = j_lo + 32 * min(nblk32, per * part);
  const int c1 = min(j_hi, j_lo + 32 * min(nblk32, per * (part + 1)));
  int* cj = cand_j[warp];
  int* cs = cand_s[warp];
  int ncand = 0;  // candidates of this part (warp-uniform, may pass kCandCap)
  float4 pi4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (active) pi4 = a.pos4[i];
  const float Lx = (float)Ldx, Ly = (float)Ldy, Lz = (float)Ldz;
  const float iLx = 1.f / Lx, iLy = 1.f / Ly, iLz = 1.f / Lz;
  const float rcf = (float)a.rcut + 1e-2f;
  const float rc2f = rcf * rcf;
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
  if (active) {
    for (int j0 = c0; j0 < c1; j0 += 32) {
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
        const bool c = valid && (bx * bx + by * by + bz * bz < rc2f) && (j != i);
        push(c, j, c ? pack_img((int)nxf, (int)nyf, (int)nzf) : 0);
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
            push(c, j, c ? pack_img(ix, iy, iz) : 0);
          }
        }
      }
    }
  }
  if (lane == 0) ncands[warp] = ncand;
  __syncthreads();
  if (active && part == 0) {
    // exact FP64 check of the concatenated candidate lists
    int off[kNbSplit + 1];
    off[0] = 0;
    bool over = false;
    for (int p = 0; p < kNbSplit; ++p) {
      const int c = ncands[warp + p];
      over |= c > kCandCap;
      off[p + 1] = off[p] + min(c, kCandCap);
    }
    const double xi = a.pos[3 * i], yi = a.pos[3 * i + 1], zi = a.pos[3 * i + 2];
    const double rc2 = a.rcut * a.rcut;
    int count = 0;
    for (int e0 = 0; e0 < off[kNbSplit]; e0 += 32) {
      const int e = e0 + lane;
      bool in = false;
      double ex = 0, ey = 0, ez = 0;
      int j = 0, ix = 0, iy = 0, iz = 0;
      if (e < off[kNbSplit]) {
        int p = 0;
        while (e >= off[p + 1]) ++p;
        j = cand_j[warp + p][e - off[p]];
        const int pk = cand_s[warp + p][e - off[p]];
        ix = (pk & 0xff) - 128;
        iy = ((pk >> 8) & 0xff) - 128;
        iz = ((pk >> 16) & 0xff) - 128;
        ex = sep1(i, j, xi, a.pos[3 * j], ix, Ldx);
        ey = sep1(i, j, yi, a.pos[3 * j + 1], iy, Ldy);
        ez = sep1(i, j, zi, a.pos[3 * j + 2], iz, Ldz);
        in = norm2(ex, ey, ez) < rc2;
      }
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

__device__ __forceinline__ void sincospi_g(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_g(double x, double* s, double* c) { sincospi(x, s, c); }

template <typename G>
__device__ void write_geom(G* g, G* gm, double ar, double ai, double br, double bi, G fc,
                           const G* dfc, const G* da, const G* db) {
  G v[kGeomStride];
  v[0] = G(ar);
  v[1] = G(ai);
  v[2] = G(br);
  v[3] = G(bi);
  v[4] = fc;
  for (int d = 0; d < 3; ++d) {
    v[5 + d] = dfc[d];
    v[8 + 2 * d] = da[2 * d];
    v[9 + 2 * d] = da[2 * d + 1];
    v[14 + 2 * d] = db[2 * d];
    v[15 + 2 * d] = db[2 * d + 1];
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
    G dfc[3] = {0, 0, 0}, da[6] = {0, 0, 0, 0, 0, 0}, db[6] = {0, 0, 0, 0, 0, 0};
    if (!(r < a.rcut)) {  // outside the cutoff (caller lists): no contribution
      write_geom(g, gm, 1.0, 0.0, 0.0, 0.0, G(0), dfc, da, db);
      continue;
    }
    // The Cayley-Klein parameters in FP64 (Sec. II-A): theta0, z0 = r cot theta0,
    // r0 = sqrt(r^2 + z0^2), a = (z0 - i z) / r0, b = (y - i x) / r0.
    double st, ct;
    sincospi(a.rfac0 * (r - a.rmin0) * a.inv_span, &st, &ct);
    const double ist = 1.0 / st;
    const double z0 = r * ct * ist;
    const double ir0 = rsqrt(r2 + z0 * z0);
    const double ar = z0 * ir0, ai = -z * ir0;
    const double br = y * ir0, bi = -x * ir0;
    // Their gradients and the switching function in the working precision G
    // (they only feed the G recursions): FP64 runs at 1/64 of the FP32 rate.
    const G gr = G(r), gir = G(ir), gz0 = G(z0), gir0 = G(ir0), gist = G(ist), gct = G(ct);
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
    const G rv[3] = {G(x), G(y), G(z)};
    for (int d = 0; d < 3; ++d) {
      const G ud = rv[d] * gir;
      dfc[d] = dfcdr * ud;
      const G dz0 = dz0dr * ud;
      const G dr0 = (gr * ud + gz0 * dz0) * gir0;
      // d a = (d(z0 - i z) - a d r0) / r0 ; d b = (d(y - i x) - b d r0) / r0
      da[2 * d] = (dz0 - gar * dr0) * gir0;
      da[2 * d + 1] = ((d == 2 ? G(-1) : G(0)) - gai * dr0) * gir0;
      db[2 * d] = ((d == 1 ? G(1) : G(0)) - gbr * dr0) * gir0;
      db[2 * d + 1] = ((d == 0 ? G(-1) : G(0)) - gbi * dr0) * gir0;
    }
    write_geom(g, gm, ar, ai, br, bi, fc, dfc, da, db);
  }
}

inline int blocks_for(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_pos4(int n, const double* pos, float4* pos4, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return launch_k(pos4_kernel, dim3(blocks_for(n, 256)), dim3(256), 0, s, n, pos, pos4);
}

cudaError_t launch_neigh_build(const NeighArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  return launch_k(neigh_build_kernel<false>, dim3(blocks_for(a.n, kNbAtoms)), dim3(kNbWarps * 32), 0, s, a);
}

cudaError_t launch_neigh_build_batch(const NeighArgs& a, int ncta, cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  return launch_k(neigh_build_kernel<true>, dim3(ncta), dim3(kNbWarps * 32), 0, s, a);
}

cudaError_t launch_neigh_ingest(int n, int K, const double* pos, double Lx, double Ly,
                                double Lz, const int* ucnt, const int* uidx,
                                const signed char* uimg, int ucap, int* cnt, int* nbr,
                                signed char* img, double* rij, int* flags, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return launch_k(neigh_ingest_kernel, dim3(blocks_for((long)n * K, 256)), dim3(256), 0, s, n, K, pos, Lx, Ly, Lz, ucnt, uidx, uimg, ucap, cnt, nbr, img, rij, flags);
}

template <typename G>
cudaError_t launch_pairs(const WorkArgs& a, int* rev, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  return launch_k(pairs_kernel<G>, dim3(blocks_for(a.n, kPairAtoms)), dim3(kPairThreads), 0, s, a, rev);
}
template cudaError_t launch_pairs<float>(const WorkArgs&, int*, cudaStream_t);
template cudaError_t launch_pairs<double>(const WorkArgs&, int*, cudaStream_t);

}  // namespace snap

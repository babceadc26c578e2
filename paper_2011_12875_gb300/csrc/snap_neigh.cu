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

__device__ __forceinline__ void exact_batch(const NeighArgs& a, int i, double xi, double yi,
                                            double zi, double rc2, const int* cj, const int* cs,
                                            int nb, int lane, int& count) {
  bool in = false;
  double ex = 0, ey = 0, ez = 0;
  int j = 0, ix = 0, iy = 0, iz = 0;
  if (lane < nb) {
    j = cj[lane];
    const int pk = cs[lane];
    ix = (pk & 0xff) - 128;
    iy = ((pk >> 8) & 0xff) - 128;
    iz = ((pk >> 16) & 0xff) - 128;
    ex = sep1(i, j, xi, a.pos[3 * j], ix, a.Lx);
    ey = sep1(i, j, yi, a.pos[3 * j + 1], iy, a.Ly);
    ez = sep1(i, j, zi, a.pos[3 * j + 2], iz, a.Lz);
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

__global__ void __launch_bounds__(kNbWarps * 32) neigh_build_kernel(NeighArgs a) {
  __shared__ float4 tile[kNbTile];
  __shared__ int cand_j[kNbWarps][kCandCap];
  __shared__ int cand_s[kNbWarps][kCandCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kNbWarps + warp;
  const bool active = i < a.n;
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
  const float Lx = (float)a.Lx, Ly = (float)a.Ly, Lz = (float)a.Lz;
  const float iLx = 1.f / Lx, iLy = 1.f / Ly, iLz = 1.f / Lz;
  const float rcf = (float)a.rcut + 1e-2f;
  const float rc2f = rcf * rcf;
  const double rc2 = a.rcut * a.rcut;
  const unsigned lt = (1u << lane) - 1u;
  int count = 0;  // accepted pairs (warp-uniform)
  int ncand = 0;  // pending candidates (warp-uniform)
  for (int j0 = 0; j0 < a.n; j0 += kNbTile) {
    __syncthreads();
    for (int q = threadIdx.x; q < kNbTile; q += blockDim.x)
      tile[q] = (j0 + q < a.n) ? a.pos4[j0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    if (!active) continue;
    const int jn = min(kNbTile, a.n - j0);
    for (int jj = 0; jj < jn; jj += 32) {
      const int j = j0 + jj + lane;
      const bool valid = (jj + lane) < jn;
      const float4 pj = tile[jj + lane];
      const float dx0 = pj.x - pi4.x, dy0 = pj.y - pi4.y, dz0 = pj.z - pi4.z;
      const int nx = -(int)rintf(dx0 * iLx), ny = -(int)rintf(dy0 * iLy), nz = -(int)rintf(dz0 * iLz);
      for (int sx = -a.Sx; sx <= a.Sx; ++sx)
        for (int sy = -a.Sy; sy <= a.Sy; ++sy)
          for (int sz = -a.Sz; sz <= a.Sz; ++sz) {
            const int ix = nx + sx, iy = ny + sy, iz = nz + sz;
            const float fx = dx0 + (float)ix * Lx, fy = dy0 + (float)iy * Ly, fz = dz0 + (float)iz * Lz;
            const bool self = (j == i) && ix == 0 && iy == 0 && iz == 0;
            const bool c = valid && !self && (fx * fx + fy * fy + fz * fz < rc2f);
            const unsigned m = __ballot_sync(kFull, c);
            if (c) {
              const int pos = ncand + __popc(m & lt);
              cj[pos] = j;
              cs[pos] = pack_img(ix, iy, iz);
            }
            ncand += __popc(m);
            if (ncand >= 32) {
              __syncwarp();
              exact_batch(a, i, xi, yi, zi, rc2, cj, cs, 32, lane, count);
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
  if (active) {
    __syncwarp();
    if (ncand > 0) exact_batch(a, i, xi, yi, zi, rc2, cj, cs, ncand, lane, count);
    if (lane == 0) {
      a.cnt[i] = min(count, a.K);
      atomicMax(&a.flags[0], count);
    }
  }
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

// rev[i][s] = slot s' of k = nbr[i][s] whose entry is (i, -img).
__global__ void rev_kernel(WorkArgs a, int* rev) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)a.n * a.K) return;
  const int i = (int)(q / a.K), s = (int)(q - (long)i * a.K);
  if (s >= a.cnt[i]) return;
  const int k = a.nbr[q];
  const int ix = -a.img[3 * q], iy = -a.img[3 * q + 1], iz = -a.img[3 * q + 2];
  const int ck = a.cnt[k];
  int found = -1;
  for (int t = 0; t < ck; ++t) {
    const long p = (long)k * a.K + t;
    if (a.nbr[p] == i && a.img[3 * p] == ix && a.img[3 * p + 1] == iy && a.img[3 * p + 2] == iz) {
      found = t;
      break;
    }
  }
  rev[q] = found;
  if (found < 0) atomicMax(&a.flags[1], 1);
}

// Per-slot Cayley-Klein parameters and derivatives, FP64 (Sec. II-A: the
// neighbour vector mapped to the 3-sphere; constants from the paper's SNAP
// reference): theta0 = rfac0 pi (r - rmin0)/(rcut - rmin0), z0 = r cot theta0,
// r0 = sqrt(r^2 + z0^2), a = (z0 - i z)/r0, b = (y - i x)/r0, and the
// cosine switching function f_c.
template <typename G>
__global__ void geom_kernel(WorkArgs a) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)a.n * a.K) return;
  const int i = (int)(q / a.K), s = (int)(q - (long)i * a.K);
  if (s >= a.cnt[i]) return;
  const double x = a.rij[3 * q], y = a.rij[3 * q + 1], z = a.rij[3 * q + 2];
  // arithmetic in FP64; the result is stored in the working precision G
  G* g = reinterpret_cast<G*>(a.geom) + q * kGeomStride;
  const double r2 = x * x + y * y + z * z;
  const double r = sqrt(r2);
  if (!(r < a.rcut)) {
    for (int e = 0; e < kGeomStride; ++e) g[e] = G(0);
    g[0] = G(1);
    return;
  }
  const double span = a.rcut - a.rmin0;
  const double c = a.rfac0 * M_PI / span;  // d theta0 / d r
  const double theta0 = c * (r - a.rmin0);
  double st, ct;
  sincos(theta0, &st, &ct);
  const double ist = 1.0 / st;
  const double z0 = r * ct * ist;
  const double dz0dr = ct * ist - r * c * ist * ist;
  const double r0 = sqrt(r2 + z0 * z0);
  const double ir0 = 1.0 / r0;
  const double ar = z0 * ir0, ai = -z * ir0;
  const double br = y * ir0, bi = -x * ir0;
  g[0] = G(ar);
  g[1] = G(ai);
  g[2] = G(br);
  g[3] = G(bi);
  double fc = 1.0, dfcdr = 0.0;
  if (a.switchflag && r > a.rmin0) {
    const double w = M_PI * (r - a.rmin0) / span;
    double sw, cw;
    sincos(w, &sw, &cw);
    fc = 0.5 * (cw + 1.0);
    dfcdr = -0.5 * M_PI / span * sw;
  }
  g[4] = G(fc);
  const double rv[3] = {x, y, z};
  const double ir = 1.0 / r;
  for (int d = 0; d < 3; ++d) {
    const double ud = rv[d] * ir;
    g[5 + d] = G(dfcdr * ud);
    const double dz0 = dz0dr * ud;
    const double dr0 = (r * ud + z0 * dz0) * ir0;
    // d a = (d(z0 - i z) - a d r0) / r0 ; d b = (d(y - i x) - b d r0) / r0
    g[8 + 2 * d] = G((dz0 - ar * dr0) * ir0);
    g[9 + 2 * d] = G(((d == 2 ? -1.0 : 0.0) - ai * dr0) * ir0);
    g[14 + 2 * d] = G(((d == 1 ? 1.0 : 0.0) - br * dr0) * ir0);
    g[15 + 2 * d] = G(((d == 0 ? -1.0 : 0.0) - bi * dr0) * ir0);
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
  neigh_build_kernel<<<blocks_for(a.n, kNbWarps), kNbWarps * 32, 0, s>>>(a);
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

cudaError_t launch_rev(const WorkArgs& a, int* rev, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  rev_kernel<<<blocks_for((long)a.n * a.K, 256), 256, 0, s>>>(a, rev);
  return cudaGetLastError();
}

template <typename G>
cudaError_t launch_geom(const WorkArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  geom_kernel<G><<<blocks_for((long)a.n * a.K, 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_geom<float>(const WorkArgs&, cudaStream_t);
template cudaError_t launch_geom<double>(const WorkArgs&, cudaStream_t);

}  // namespace snap

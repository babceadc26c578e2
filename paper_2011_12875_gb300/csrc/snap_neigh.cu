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
#include "snap_neigh.cuh"

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

template <bool BATCH, int SPLIT, int NW>
__global__ void __launch_bounds__(NW * 32) neigh_build_kernel(NeighArgs a) {
  nb::neigh_build_cta<BATCH, SPLIT, NW>(a, [](int, long, int, long, double, double, double) {});
}

// Caller-supplied list -> internal [N][K] tables with exact separations.
__global__ void neigh_ingest_kernel(int n, int K, const double* __restrict__ pos, double Lx,
                                    double Ly, double Lz, const int* __restrict__ ucnt,
                                    const int* __restrict__ uidx, const signed char* __restrict__ uimg,
                                    int ucap, int* cnt, int* nbr, signed char* img, double* rij,
                                    int* key, int* flags) {
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
    key[q] = -1;
    return;
  }
  const int ix = uimg[3 * u], iy = uimg[3 * u + 1], iz = uimg[3 * u + 2];
  nbr[q] = k;
  img[3 * q] = (signed char)ix;
  img[3 * q + 1] = (signed char)iy;
  img[3 * q + 2] = (signed char)iz;
  rij[3 * q] = nb::sep1(i, k, pos[3 * i], pos[3 * k], ix, Lx);
  rij[3 * q + 1] = nb::sep1(i, k, pos[3 * i + 1], pos[3 * k + 1], iy, Ly);
  rij[3 * q + 2] = nb::sep1(i, k, pos[3 * i + 2], pos[3 * k + 2], iz, Lz);
  key[q] = pair_key(k, ix, iy, iz, n);
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
                                signed char* img, double* rij, int* key, int* flags, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return launch_k(neigh_ingest_kernel, dim3(blocks_for((long)n * K, 256)), dim3(256), 0, s, n, K, pos, Lx, Ly,
                  Lz, ucnt, uidx, uimg, ucap, cnt, nbr, img, rij, key, flags);
}


}  // namespace snap

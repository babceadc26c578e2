// snap_internal.h -- device-side layouts and launcher prototypes shared by the
// library's translation units (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace snap {

// Kernel launch with the configuration as arguments (one place to change how
// the library launches).
#ifdef __CUDACC__
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args... args) {
  kernel<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
  return cudaGetLastError();
}
#endif

constexpr int kMaxTwoJ = 14;
constexpr int kYGroupMax = 8;  // longest compute_Y term group (longer ones are cut)
constexpr int kBChunk = 96;    // bispectrum terms a warp takes at a time (whole groups)
constexpr int kBMaxChunks = 1024;  // chunks are lengthened past this count
constexpr int kBGroupMax = 8;      // longest bispectrum term piece (longer groups are cut)
constexpr int kYRecPad = 256;  // zero records after the compute_Y term list (read-ahead)
constexpr int kYRecPrefetch = 64;  // compute_Y's L1 prefetch distance without the record ring
constexpr int kMaxNeighCap = 64;
constexpr int kRootDim = 16;     // rootpq table is kRootDim x kRootDim
constexpr int kGeomStride = 20;  // doubles per neighbour slot, see PairGeom

// Half-matrix layout (Sec. V-A: u_j only needs floor(j)+1 of its columns):
// layer t = 2j holds columns mb = 0..t/2, each column ma = 0..t.
__host__ __device__ constexpr int half_layer_size(int t) { return (t + 1) * (t / 2 + 1); }
__host__ __device__ constexpr int half_base(int t) {
  int n = 0;
  for (int s = 0; s < t; ++s) n += half_layer_size(s);
  return n;
}
__host__ __device__ constexpr int half_size(int twojmax) { return half_base(twojmax + 1); }

// Packed (t, ma, mb) of a half-layout element.
__host__ __device__ constexpr int pack_tmm(int t, int ma, int mb) { return t | (ma << 8) | (mb << 16); }
__host__ __device__ constexpr int tmm_t(int p) { return p & 0xff; }
__host__ __device__ constexpr int tmm_ma(int p) { return (p >> 8) & 0xff; }
__host__ __device__ constexpr int tmm_mb(int p) { return (p >> 16) & 0xff; }

// compute_Y term record: w = index of U_t1 element (10 bits) | index of the
// U_t2 element << 10 | conj U_t1 << 20 | conj U_t2 << 21 | last term of the
// output << 22; c = coefficient in the working precision.
template <typename R>
struct YRec;
template <>
struct __align__(8) YRec<float> {
  unsigned w;
  float c;
};
template <>
struct __align__(16) YRec<double> {
  unsigned w, pad;
  double c;
};

// Per neighbour slot geometry (Cayley-Klein parameters, Sec. II-A), computed
// in FP64 and stored in the working precision R:
//  [0..1] a, [2..3] b, [4] f_c, [5..7] d f_c / d r_d,
//  [8..13] d a / d r_d (re, im per d), [14..19] d b / d r_d.
// A slot with r >= rcut has f_c = 0 and zero derivatives.

// One configuration of a batch: atoms [start, start + n), box L, image
// shifts S enumerated beyond the nearest image.
struct NeighConf {
  int start, n;
  double L[3];
  int S[3];
};

// Image shifts the device neighbour build enumerates beyond the nearest
// image, per axis: none when the box is longer than 2 (rcut + 0.05 A), else
// ceil(rcut / L) + 1.  The build loops over (2 Sx + 1)(2 Sy + 1)(2 Sz + 1)
// images for every 32 candidates and stores shifts as signed bytes, so a box
// that needs more than kMaxImageLoop images in all, or more than kMaxImageShift
// along one axis, is refused (false): such a box holds more images of a
// single atom within rcut than any neighbour capacity.  rcut and the box
// lengths must be finite and positive.
constexpr int kMaxImageLoop = 4096;
constexpr int kMaxImageShift = 100;
inline bool image_shifts(const double* L, double rcut, int S[3]) {
  if (!(rcut > 0.0 && rcut < 1e30)) return false;
  long loop = 1;
  for (int d = 0; d < 3; ++d) {
    if (!(L[d] > 0.0 && L[d] < 1e300)) return false;
    const double q = rcut / L[d];
    if (!(q < (double)kMaxImageShift)) return false;
    S[d] = (L[d] > 2.0 * (rcut + 0.05)) ? 0 : (int)std::ceil(q) + 1;
    if (S[d] > kMaxImageShift) return false;
    loop *= 2L * S[d] + 1;
  }
  return loop <= kMaxImageLoop;
}

// centre atoms per CTA of the device neighbour build
constexpr int kNeighAtomsPerCta = 2;

struct NeighArgs {
  int n, K;
  // batch mode: confs != nullptr; CTA b builds atoms
  // cta_map[b].y + 0..kNeighAtomsPerCta-1 of configuration cta_map[b].x
  const NeighConf* confs;
  const int2* cta_map;
  const double* pos;     // [n][3]
  const float4* pos4;    // [n] FP32 copy for the coarse test
  // [ceil(n/32)][2]: FP32 centre and half extent of each 32-atom tile, for
  // skipping far tiles in the single-configuration build; nullptr: no skipping
  const float4* tiles = nullptr;
  double Lx, Ly, Lz;
  int Sx, Sy, Sz;        // image shifts enumerated beyond the nearest image
  double rcut;
  int* cnt;
  int* nbr;
  signed char* img;
  double* rij;
  int* key;  // [n][K] pair_key of every stored slot, or nullptr
  int* flags;
};

// Search key of a stored pair (k, image s): k * 32 + the image's code
// (s_d + 1 in base 3) when every |s_d| <= 1 (and the atoms index below 2^26),
// else -1.  The opposite pair (i, -s) has code 26 - code, so the force gather
// finds the reverse slot with one pass over k's row of keys.
__host__ __device__ constexpr int pair_key(int k, int ix, int iy, int iz, long n) {
  return (ix >= -1 && ix <= 1 && iy >= -1 && iy <= 1 && iz >= -1 && iz <= 1 && n < (1L << 26))
             ? k * 32 + (ix + 1) * 9 + (iy + 1) * 3 + (iz + 1)
             : -1;
}

struct WorkArgs {
  int n, K, twojmax, H, lmax;
  double rcut, rfac0, rmin0, wself, beta0;
  double inv_span;  // 1 / (rcut - rmin0)
  double th_scale;  // rfac0 / (rcut - rmin0): theta0 / pi = th_scale (r - rmin0)
  // FP32 copies for the mixed path's slot gradients (no FP64 work per slot):
  // th_scale, d theta0 / d r = pi th_scale, 1 / (rcut - rmin0), rmin0 and
  // the switching derivative's factor -pi / (2 (rcut - rmin0))
  float th_scale_f, dth_f, inv_span_f, rmin0_f, dfc_f;
  int switchflag;
  const int* cnt;
  const int* nbr;
  const signed char* img;
  const int* rev;
  int* rev_out;  // the same table, written by the force kernel
  const int* key;  // [N][K] pair_key of every slot
  double* rij;
  void* geom;  // R [N][K][kGeomStride]: Cayley-Klein geometry in the working precision
  // Ulisttot and Y: complex (re, im interleaved), AoSoA [ceil(N/32)][H][32]
  void* U;
  void* Y;
  double* dedr;
  double* vatom;   // per-atom virial [N][6] (batch mode) or nullptr
  double* energy;
  double* forces;
  double* vpart;
  double* virial;
  int* flags;
  // non-null on the kernel that ends an evaluation (the force kernel): its
  // last CTA writes flags[0..3] to this host-mapped copy and zeroes the flags
  int* hflags;
  const int* half_tmm;
  const void* yrec;       // compute_Y term records (see snap_tables.cpp)
  const int* yfirst;      // [H+1] first term of each output element
  const void* yruns;      // [H][kYGroupMax] u16: groups of 1..kYGroupMax terms per output
  const int* yslice;
  int nslices;
  int yi_layout;          // 0: warp of 32 atoms (AoSoA), 1: warp per atom
  const int* ysched;      // [32][ysched_m] outputs of each lane (warp-per-atom layout)
  int ysched_m;
  int nsm;
  int col_warps;  // warps per CTA of the column-chain kernels (tunable)
  int de_maxcnt;  // neighbour count the fused dE launch is planned for (last seen maximum, else K)
  int yi_waves;   // compute_Y waves per SM (tunable)
  int persist;    // tunable: bit 0 persistent compute_Y, bit 1 persistent fused dE (work queues)
  int de_atoms;   // tunable: atoms per fused dE CTA (0: planned)
  int test_skip_stage;  // test hook: TMA staging registers its bytes but issues no copy
  // bispectrum output
  int ncoeff;
  const void* brec;       // YRec<R> records of the bispectrum terms (sign-flip words)
  const void* brec_cp;    // the same records in the conjugate-plane words (null: unused)
  const int* bchunk_term;   // chunks of the bispectrum term list (snap_tables.h)
  const void* bchunk_runs;  // [nchunks][kBGroupMax] u16: pieces of 1, 2, ... terms of every chunk
  const int* bcomp_chunk;
  int bi_layout;            // tunable: 0 planned, 1 sign flips, 2 conjugate plane
  void* bscratch;           // partial sums of the bispectrum chunks when shared memory is short
  const int* bpart;         // [nbparts+1] first component of each CTA's run
  int nbparts, bmaxchunks, bmaxterms;  // runs, most chunks and most terms of one run
  double* B;              // [N][ncoeff]
  const void* rootpq;
  const void* hscale;  // R [H]: S_t(ma, mb) of the scaled recursion (u = S v)
};

// Launchers (snap_neigh.cu)
cudaError_t launch_pos4(int n, const double* pos, float4* pos4, cudaStream_t s, float4* tiles = nullptr,
                        double* copy = nullptr);
cudaError_t launch_neigh_build(const NeighArgs& a, cudaStream_t s);
// batch: one launch over all configurations (ncta CTAs)
cudaError_t launch_neigh_build_batch(const NeighArgs& a, int ncta, cudaStream_t s);
cudaError_t launch_neigh_ingest(int n, int K, const double* pos, double Lx, double Ly,
                                double Lz, const int* ucnt, const int* uidx,
                                const signed char* uimg, int ucap, int* cnt, int* nbr,
                                signed char* img, double* rij, int* key, int* flags, cudaStream_t s);
// reverse-slot map + geometry in the working precision G (one kernel)

// Launchers (snap_kernels.cu), R = float (mixed) or double (FP64)
template <typename R> cudaError_t launch_ui(const WorkArgs& a, cudaStream_t s);
template <typename R> cudaError_t launch_yi(const WorkArgs& a, cudaStream_t s);

// Launch shape of compute_Y for N atoms: grid (nblk, ysplit), `threads` per
// CTA, nslices = ysplit * warps per CTA work slices per 32-atom block; the
// block's Ulisttot is staged in `smem` bytes of shared memory when it fits.
struct YiGeometry {
  int nblk, ysplit, threads, nslices;
  size_t smem;
  bool staged;
  bool conjplane;  // a conjugated copy of the block is staged too (records index it)
};
// Whether compute_Y stages U and its conjugate (records in the 2H-index format).
__host__ __device__ inline bool yi_conjplane(int rsize, int H) {
  return (size_t)4 * H * 32 * rsize + 16 <= 100 * 1024;
}
// compute_Y term record word.  FP32 with the conjugate plane: bits 14-31 the
// byte offset of the second factor's [32] lanes (element times 256, the
// element over the 2H plane), bits 0-9 the first factor's element, bit 12
// ends a group, bit 13 an output.  Otherwise: bits 8-17 the second factor's
// element, 18-27 the first's, bit 28 ends a group, 29 an output, 30 / 31
// conjugate the first / second factor (no conjugation bits with the plane).
__host__ __device__ inline bool yrec_plane_format(int rsize, int H) {
  return rsize == 4 && yi_conjplane(rsize, H);
}
YiGeometry yi_geometry(int rsize, int H, int n, int nsm, int waves);

// End of an evaluation: flags[0..3] into the host-mapped status words
// (device pointer hflags), all eight flags zeroed.
cudaError_t launch_flags_out(int* flags, int* hflags, cudaStream_t s);

// Per-configuration virial: sum of vatom over each configuration's atoms.
cudaError_t launch_virial_conf(const double* vatom, const NeighConf* confs, int nconf, double* virial,
                               cudaStream_t s);
template <typename R> cudaError_t launch_de(const WorkArgs& a, cudaStream_t s);
template <typename R> cudaError_t launch_force(const WorkArgs& a, cudaStream_t s);
template <typename R> cudaError_t launch_bi(const WorkArgs& a, cudaStream_t s);

// Launch plan of the bispectrum kernels (B and dB) for the precision's size
// (4 or 8 bytes), H, and the most chunks and terms of a CTA's run: the
// block's planes staged (U's, and dU's when both fit) or read from global memory, the conjugate plane or
// sign flips, the run's term records staged or read through L1 (rs), the
// partial sums in shared memory or in the global scratch (gpart, then CTAs x
// maxchunks x 32 x rsize bytes), and the dynamic shared memory.  Layout:
// [planes][barrier, 16 B][records, rec_bytes][partials].
constexpr int kBiThreads = 512;
constexpr int kBiCtasPerSm = 2;  // register budget of the kernels (64 a thread)
constexpr size_t kBiSmemMax = 200 * 1024;   // one CTA an SM
constexpr size_t kBiSmemPair = 112 * 1024;  // two CTAs an SM
struct BiPlan {
  bool staged, ds, cp, rs, gpart;  // ds: the tangent's block staged beside U (dB)
  size_t smem, rec_bytes;
};
BiPlan bi_plan(int rsize, int H, bool deriv, int maxchunks, int maxterms, int layout, bool have_cp);
// whether the conjugate-plane records can ever be used for this size and H
bool bi_plane_fits(int rsize, int H);

// Register column-chain kernels (snap_col_*.cu), for 1 <= twojmax <= 14;
// cudaErrorInvalidValue when no instance exists for the precision/2J.
template <typename R> cudaError_t launch_ui_col(const WorkArgs& a, cudaStream_t s);
template <typename R> cudaError_t launch_de_col(const WorkArgs& a, cudaStream_t s);
// Neighbour build fused with compute_U (FP32: 1 <= twojmax <= 14; FP64: up
// to 8): one configuration (ncta = 0) or a batch of ncta CTAs (na.confs).
template <typename R>
cudaError_t launch_neigh_u(const NeighArgs& na, const WorkArgs& a, int ncta, cudaStream_t s);
// Tangent of Ulisttot along the displacement field g ([N][3], device); 0..14.
template <typename R>
cudaError_t launch_tan_col(const WorkArgs& a, const double* g, void* dU, cudaStream_t s);

// d B_l along the tangent dU (snap_kernels.cu) and the weighted force gather.
template <typename R> cudaError_t launch_dbi(const WorkArgs& a, const void* dU, double* dB, cudaStream_t s);
cudaError_t launch_force_weighted(const WorkArgs& a, const double* w, double* grad, cudaStream_t s);

// FMA throughput probe (synchronous): flops and milliseconds of one timed launch
template <typename R>
cudaError_t fma_probe(int nsm, int iters, double* flops, float* ms, R* sink, cudaStream_t s);

}  // namespace snap

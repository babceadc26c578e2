// snap_api.cu -- the C ABI declared in include/snap_gb300.h: context, tables,
// workspace and the per-call launch sequence (arXiv:2011.12875, Listing 5:
// build_neighborlist, compute_U, compute_Y, compute_dU + compute_dE fused,
// update_forces).
#include <cmath>
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "snap_gb300.h"
#include "snap_internal.h"
#include "snap_tables.h"

using snap::HostTables;

// A captured single-configuration evaluation, replayed while the same call
// repeats (same sizes, box, buffers, tunables and workspace).  A key is
// captured the second time it is seen in a row, so one-off calls never pay
// for capture and instantiation.
struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned long long> key;   // of exec
  std::vector<unsigned long long> seen;  // key of the previous uncaptured call
  snap::WorkArgs args;                   // host-side state of the captured call
  int launches = 0, n = 0, K = 0;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key.clear();
    seen.clear();
  }
};

struct snap_ctx {
  int twojmax = 0;
  double rcut = 0, rfac0 = 0, rmin0 = 0, wself = 1.0;
  int switchflag = 1;
  int precision = SNAP_FP64;
  int nsm = 152;
  HostTables tab;
  std::vector<double> beta;
  int K = 32;
  int col_warps = 4;  // tunables (snap_set_tuning / snap_autotune)
  int yi_waves = 2;
  int yi_layout = 0;
  int test_skip_stage = 0;  // snap_test_stage_timeout
  int persist = 0;          // SNAP_KNOB_PERSIST
  int de_atoms = 0;         // SNAP_KNOB_DE_ATOMS
  int last_nmax = 0;
  int seen_nmax = 0;  // largest neighbour count seen: the fused dE launch is planned for it
  int last_n = 0, last_K = 0;
  std::string err;

  // device tables
  int* d_half_tmm = nullptr;
  void* d_yrec = nullptr;
  int* d_yfirst = nullptr;
  unsigned short* d_yruns = nullptr;
  void* d_brec = nullptr;
  void* d_brec_cp = nullptr;
  void* d_bscratch = nullptr;  // chunk partials of the bispectrum kernels (when shared memory is short)
  size_t bscratch_cap = 0;
  int bi_layout = 0;           // knob: 0 planned, 1 sign flips, 2 conjugate plane
  int* d_bchunk_term = nullptr;
  unsigned short* d_bchunk_runs = nullptr;
  int* d_bcomp_chunk = nullptr;
  // bispectrum component runs by run count: device table and most chunks a run
  struct BPart {
    int* d;         // [runs + 1] first component of each run
    int maxchunks;  // most chunks of one run
    int maxterms;   // most terms of one run
  };
  std::map<int, BPart> bpart_cache;
  int nbparts = 0;
  void* d_root = nullptr;
  void* d_hscale = nullptr;
  int* d_yslice = nullptr;
  int* d_ysched = nullptr;  // lane schedule of the warp-per-atom compute_Y
  int ysched_m = 0;
  int nslices = -1;
  std::map<int, int*> yslice_cache;  // compute_Y slice tables by slice count

  // workspace
  long cap_nk = 0;
  int cap_n = 0;
  float4* d_pos4 = nullptr;
  float4* d_tiles = nullptr;  // bounding boxes of 32-atom tiles
  int* d_cnt = nullptr;
  int* d_nbr = nullptr;
  signed char* d_img = nullptr;
  double* d_rij = nullptr;
  int* d_rev = nullptr;
  int* d_key = nullptr;  // pair keys of the neighbour table (reverse-slot search)
  double* d_geom = nullptr;
  double* d_dedr = nullptr;
  void* d_U = nullptr;  // complex AoSoA [ceil(N/32)][H][32]
  void* d_Y = nullptr;
  void* d_dU = nullptr;  // tangent of U (bispectrum derivative)
  long long generation = 0;  // number of evaluations enqueued
  snap::WorkArgs last_args;   // arguments of the last evaluation (weighted gather)
  bool have_last = false;
  double* d_vpart = nullptr;
  // device status words and counters, zeroed at the end of every evaluation
  // (flags_out_kernel), which also writes the status words to h_flags,
  // pinned and mapped (d_hflags: its device address)
  int* d_flags = nullptr;
  int* h_flags = nullptr;
  int* d_hflags = nullptr;
  bool flags_dirty = false;  // an evaluation was begun and not closed: zero before the next

  // per-stage profiling
  bool prof_on = false;
  std::vector<std::vector<cudaEvent_t>> prof_pending, prof_free;
  double prof_ms[SNAP_NSTAGES] = {0};
  long long prof_calls[SNAP_NSTAGES] = {0};
  int launches = 0;

  // batches of configurations
  std::vector<int> bat_n;
  std::vector<double> bat_box;
  snap::NeighConf* d_confs = nullptr;
  int2* d_ctamap = nullptr;
  int bat_ncta = 0, bat_nconf = 0, bat_total = 0;
  double* d_vatom = nullptr;
  int cap_vatom = 0;
  // captured CUDA graph of the last batch (shape and pointers baked in)
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* g_key[4] = {nullptr, nullptr, nullptr, nullptr};
  long long g_ws = -1;  // workspace generation the batch graph was captured with
  int g_demax = -1;     // neighbour count its fused dE launch was planned for
  // bumped whenever a device buffer that a captured graph refers to moves
  long long ws_gen = 0;
  // single-configuration graphs (snap_compute*, snap_compute_host)
  GraphSlot gdev, ghost;

  // buffers of snap_compute_host
  int cap_host = 0;
  double* d_hpos = nullptr;
  double* d_hE = nullptr;
  double* d_hF = nullptr;
  double* d_hW = nullptr;

  size_t rsize() const { return precision == SNAP_MIXED ? sizeof(float) : sizeof(double); }
};

namespace {

std::string g_create_error;

int fail(snap_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define SNAP_CUDA(ctx, expr)                                                            \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, SNAP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Convert doubles to the working precision and upload (allocating if needed).
int upload_r(snap_ctx* c, void** dst, const std::vector<double>& v) {
  const size_t n = v.size() ? v.size() : 1;
  if (!*dst) SNAP_CUDA(c, cudaMalloc(dst, n * c->rsize()));
  if (c->precision == SNAP_MIXED) {
    std::vector<float> f(v.begin(), v.end());
    if (f.empty()) f.push_back(0.f);
    SNAP_CUDA(c, cudaMemcpy(*dst, f.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  } else {
    std::vector<double> d(v);
    if (d.empty()) d.push_back(0.0);
    SNAP_CUDA(c, cudaMemcpy(*dst, d.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  }
  return SNAP_OK;
}

template <typename T>
int upload(snap_ctx* c, T** dst, const std::vector<T>& v) {
  const size_t n = v.size() ? v.size() : 1;
  dfree(*dst);
  SNAP_CUDA(c, cudaMalloc((void**)dst, n * sizeof(T)));
  if (!v.empty()) SNAP_CUDA(c, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SNAP_OK;
}

// Overwrite an existing table of the same size in place (its address, which
// captured graphs hold, stays valid); allocate it the first time.
template <typename T>
int upload_inplace(snap_ctx* c, T** dst, const std::vector<T>& v) {
  if (!*dst) return upload(c, dst, v);
  if (!v.empty()) SNAP_CUDA(c, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SNAP_OK;
}

// compute_Y term records (index word + coefficient in the working precision)
int upload_yrec(snap_ctx* c) {
  const std::vector<double> coef = c->tab.term_coef(c->beta.data());
  const size_t n = c->tab.terms.size();
  // Kernel word (the formats are described with yrec_plane_format): the
  // element offsets in units of 256 B (one element's [32] lanes of complex
  // float; the FP64 kernel doubles them), the group-end and output-end bits
  // and, without a staged conjugate plane, the conjugation flags (the sign
  // bit of the factor's imaginary part).  With the plane the elements run
  // over 2H (element + H for a conjugated read).
  const bool cp = snap::yi_conjplane((int)c->rsize(), c->tab.H);
  const bool pf = snap::yrec_plane_format((int)c->rsize(), c->tab.H);
  const unsigned H = (unsigned)c->tab.H;
  if ((cp ? 2 * H : H) > 1024u) return fail(c, SNAP_ERR_ARG, "compute_Y element index exceeds 10 bits");
  auto word = [&](unsigned w) -> unsigned {
    unsigned e1 = w & 1023u, e2 = (w >> 10) & 1023u;
    unsigned c1 = (w >> 20) & 1u, c2 = (w >> 21) & 1u;
    const unsigned ge = (w >> 23) & 1u, oe = (w >> 22) & 1u;
    if (cp) {
      e1 += c1 * H;
      e2 += c2 * H;
      c1 = c2 = 0;
    }
    if (pf) return (e2 << 22) | e1 | (ge << 12) | (oe << 13);
    return (e2 << 8) | (e1 << 18) | (ge << 28) | (oe << 29) | (c1 << 30) | (c2 << 31);
  };
  // kYRecPad zero records past the end: compute_Y reads up to that far ahead
  if (c->precision == SNAP_MIXED) {
    std::vector<snap::YRec<float>> r(n + snap::kYRecPad);
    for (size_t k = 0; k < n; ++k) {
      r[k].w = word(c->tab.terms[k]);
      r[k].c = (float)coef[k];
    }
    return upload_inplace(c, reinterpret_cast<snap::YRec<float>**>(&c->d_yrec), r);
  }
  std::vector<snap::YRec<double>> r(n + snap::kYRecPad);
  for (size_t k = 0; k < n; ++k) {
    r[k].w = word(c->tab.terms[k]);
    r[k].pad = 0;
    r[k].c = coef[k];
  }
  return upload_inplace(c, reinterpret_cast<snap::YRec<double>**>(&c->d_yrec), r);
}

// bispectrum term records (coefficients do not depend on beta), in both
// word layouts; the conjugate-plane records only where the doubled plane of
// one 32-atom block can be staged (snap_kernels.cu decides per launch)
template <typename R>
int upload_brec_t(snap_ctx* c, const std::vector<unsigned>& w, void** dst) {
  // two zero records of padding: a run's staged copy may round its end up to
  // 16 bytes
  std::vector<snap::YRec<R>> r(w.size() + 2);
  std::memset(r.data(), 0, r.size() * sizeof(r[0]));
  for (size_t k = 0; k < w.size(); ++k) {
    r[k].w = w[k];
    r[k].c = (R)c->tab.bdev_coef[k];
  }
  return upload(c, reinterpret_cast<snap::YRec<R>**>(dst), r);
}

int upload_brec(snap_ctx* c) {
  const bool mixed = c->precision == SNAP_MIXED;
  for (int cp = 0; cp < 2; ++cp) {
    if (cp && !snap::bi_plane_fits((int)c->rsize(), c->tab.H)) break;
    const std::vector<unsigned> w = c->tab.bwords(cp != 0);
    if (w.size() != c->tab.bdev.size()) return fail(c, SNAP_ERR_ARG, "bispectrum tables: element out of range");
    void** dst = cp ? &c->d_brec_cp : &c->d_brec;
    const int rc = mixed ? upload_brec_t<float>(c, w, dst) : upload_brec_t<double>(c, w, dst);
    if (rc) return rc;
  }
  return SNAP_OK;
}

void free_workspace(snap_ctx* c) {
  dfree(c->d_pos4);
  dfree(c->d_tiles);
  dfree(c->d_cnt);
  dfree(c->d_nbr);
  dfree(c->d_img);
  dfree(c->d_rij);
  dfree(c->d_rev);
  dfree(c->d_key);
  dfree(c->d_geom);
  dfree(c->d_dedr);
  dfree(c->d_U);
  dfree(c->d_Y);
  dfree(c->d_dU);
  dfree(c->d_vpart);
  c->cap_nk = 0;
  c->cap_n = 0;
}

int ensure_workspace(snap_ctx* c, int n, int K) {
  const long nk = (long)n * K;
  if (n <= c->cap_n && nk <= c->cap_nk) return SNAP_OK;
  cudaDeviceSynchronize();
  free_workspace(c);
  const int ncap = std::max(n, 1);
  const long nkcap = std::max(nk, 1L);
  const long nblk = (ncap + 31) / 32;
  const size_t uy = (size_t)nblk * 32 * c->tab.H * 2 * c->rsize();
  SNAP_CUDA(c, cudaMalloc(&c->d_pos4, sizeof(float4) * ncap));
  SNAP_CUDA(c, cudaMalloc(&c->d_tiles, sizeof(float4) * 2 * ((ncap + 31) / 32)));
  SNAP_CUDA(c, cudaMalloc(&c->d_cnt, sizeof(int) * ncap));
  SNAP_CUDA(c, cudaMalloc(&c->d_nbr, sizeof(int) * nkcap));
  SNAP_CUDA(c, cudaMalloc(&c->d_img, 3 * nkcap));
  SNAP_CUDA(c, cudaMalloc(&c->d_rij, sizeof(double) * 3 * nkcap));
  SNAP_CUDA(c, cudaMalloc(&c->d_rev, sizeof(int) * nkcap));
  SNAP_CUDA(c, cudaMalloc(&c->d_key, sizeof(int) * nkcap));
  SNAP_CUDA(c, cudaMalloc(&c->d_geom, sizeof(double) * snap::kGeomStride * nkcap));
  SNAP_CUDA(c, cudaMalloc(&c->d_dedr, sizeof(double) * 3 * nkcap));
  SNAP_CUDA(c, cudaMalloc(&c->d_U, uy));
  SNAP_CUDA(c, cudaMalloc(&c->d_Y, uy));
  SNAP_CUDA(c, cudaMalloc(&c->d_dU, uy));
  // lanes past the last atom read zeros in compute_Y
  SNAP_CUDA(c, cudaMemset(c->d_U, 0, uy));
  // one virial partial per force CTA (at least one atom each)
  SNAP_CUDA(c, cudaMalloc(&c->d_vpart, sizeof(double) * 6 * (ncap + 1)));
  c->cap_n = ncap;
  c->cap_nk = nkcap;
  c->ws_gen += 1;
  return SNAP_OK;
}

int ensure_slices(snap_ctx* c, int n) {
  const snap::YiGeometry g = snap::yi_geometry((int)c->rsize(), c->tab.H, n, c->nsm, c->yi_waves);
  if (g.nslices == c->nslices) return SNAP_OK;
  auto it = c->yslice_cache.find(g.nslices);
  if (it == c->yslice_cache.end()) {
    int* d = nullptr;
    int rc = upload(c, &d, c->tab.slices(g.nslices));
    if (rc) return rc;
    it = c->yslice_cache.emplace(g.nslices, d).first;
  }
  c->d_yslice = it->second;
  c->nslices = g.nslices;
  c->ws_gen += 1;
  return SNAP_OK;
}

int ensure_flags(snap_ctx* c) {
  if (c->d_flags) return SNAP_OK;
  SNAP_CUDA(c, cudaMalloc(&c->d_flags, 8 * sizeof(int)));
  SNAP_CUDA(c, cudaMemset(c->d_flags, 0, 8 * sizeof(int)));
  SNAP_CUDA(c, cudaHostAlloc(reinterpret_cast<void**>(&c->h_flags), 8 * sizeof(int), cudaHostAllocMapped));
  std::memset(c->h_flags, 0, 8 * sizeof(int));
  SNAP_CUDA(c, cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->d_hflags), c->h_flags, 0));
  return SNAP_OK;
}

// Begin an evaluation on stream s: the flags are zero unless the previous
// evaluation did not reach its end (a launch failed), then they are zeroed.
cudaError_t open_flags(snap_ctx* c, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (c->flags_dirty) e = cudaMemsetAsync(c->d_flags, 0, 8 * sizeof(int), s);
  c->flags_dirty = true;
  return e;
}
// End it: the status words to the host (read after the stream's work), the
// flags zeroed, by one small kernel rather than a copy and a memset (each a
// copy-engine operation on the step's critical path).
cudaError_t close_flags(snap_ctx* c, cudaStream_t s) {
  cudaError_t e = snap::launch_flags_out(c->d_flags, c->d_hflags, s);
  if (e == cudaSuccess) {
    c->flags_dirty = false;
    c->launches += 1;
  }
  return e;
}

// Component runs of the bispectrum kernels (B, or dB with deriv) for n
// atoms, and the global scratch of the chunk partials when a run has more
// than shared memory holds.  CTAs = 32-atom blocks x runs; the CTAs an SM
// runs share its issue slots, so the time goes as the most CTAs an SM takes
// times a CTA's share of a block (1/runs) plus its fixed cost (staging the
// block, about kBiCtaCost of a block's work): the run count minimises
// ceil(blocks x runs / SMs) x (1 / runs + kBiCtaCost), at most one run per
// component.
int ensure_bparts(snap_ctx* c, long n, bool deriv) {
  const long nblk = std::max(1L, (n + 31) / 32);
  const int rs = (int)c->rsize();
  const bool have_cp = c->d_brec_cp != nullptr;
  constexpr double kBiCtaCost = 0.02;
  int parts = 1;
  double best = 1e300;
  for (int p = 1; p <= std::min(64, c->tab.ncoeff); ++p) {
    const double cost = (double)((nblk * p + c->nsm - 1) / c->nsm) * (1.0 / p + kBiCtaCost);
    if (cost < best * (1.0 - 1e-9)) {
      best = cost;
      parts = p;
    }
  }
  if (parts != c->nbparts) {
    auto it = c->bpart_cache.find(parts);
    if (it == c->bpart_cache.end()) {
      int mx = 0, mt = 0;
      const std::vector<int> b = c->tab.bparts(parts, &mx, &mt);
      int* d = nullptr;
      int rc = upload(c, &d, b);
      if (rc) return rc;
      it = c->bpart_cache.emplace(parts, snap_ctx::BPart{d, mx, mt}).first;
    }
    c->nbparts = parts;
    c->ws_gen += 1;
  }
  const snap_ctx::BPart& bp = c->bpart_cache.at(parts);
  const int mx = bp.maxchunks;
  const snap::BiPlan p = snap::bi_plan(rs, c->tab.H, deriv, mx, bp.maxterms, c->bi_layout, have_cp);
  if (p.gpart) {
    const size_t bytes = (size_t)nblk * parts * mx * 32 * rs;
    if (bytes > c->bscratch_cap) {
      cudaDeviceSynchronize();
      dfree(c->d_bscratch);
      c->bscratch_cap = 0;
      SNAP_CUDA(c, cudaMalloc(&c->d_bscratch, bytes));
      c->bscratch_cap = bytes;
      c->ws_gen += 1;
    }
  }
  return SNAP_OK;
}

bool box_ok(const double* box) {
  if (!box) return false;
  for (int d = 0; d < 3; ++d)
    if (!(std::isfinite(box[d]) && box[d] > 0.0)) return false;
  return true;
}

// A box the device neighbour build can enumerate (snap::image_shifts): each
// length finite and > 0, and not so short against rcut that the image loop
// would run away.  SNAP_OK or SNAP_ERR_BOX with the reason.
int check_box(snap_ctx* c, const double* box) {
  if (!box_ok(box)) return fail(c, SNAP_ERR_BOX, "box lengths must be finite and > 0");
  int S[3];
  if (!snap::image_shifts(box, c->rcut, S))
    return fail(c, SNAP_ERR_BOX, "box too short for rcut: the neighbour build would enumerate more than " +
                                     std::to_string(snap::kMaxImageLoop) + " periodic images per atom (or shifts beyond " +
                                     std::to_string(snap::kMaxImageShift) + " along one axis)");
  return SNAP_OK;
}

// Kernel arguments for n atoms with capacity K (workspace and tables).
// Neighbour count the fused dE launch is planned for: the largest count the
// context has seen (monotone, so a captured graph is re-captured at most a
// few times as it grows), else the capacity.
int de_maxcnt(const snap_ctx* c, int K) { return (c->seen_nmax > 0 && c->seen_nmax <= K) ? c->seen_nmax : K; }

snap::WorkArgs make_args(snap_ctx* c, int n, int K) {
  snap::WorkArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.K = K;
  a.twojmax = c->twojmax;
  a.H = c->tab.H;
  a.lmax = c->tab.lmax;
  a.rcut = c->rcut;
  a.rfac0 = c->rfac0;
  a.rmin0 = c->rmin0;
  a.inv_span = 1.0 / (c->rcut - c->rmin0);
  a.th_scale = c->rfac0 * a.inv_span;
  a.th_scale_f = (float)a.th_scale;
  a.dth_f = (float)(M_PI * a.th_scale);
  a.inv_span_f = (float)a.inv_span;
  a.rmin0_f = (float)c->rmin0;
  a.dfc_f = (float)(-0.5 * M_PI * a.inv_span);
  a.wself = c->wself;
  a.beta0 = c->beta[0];
  a.switchflag = c->switchflag;
  a.cnt = c->d_cnt;
  a.nbr = c->d_nbr;
  a.img = c->d_img;
  a.rev = c->d_rev;
  a.rev_out = c->d_rev;
  a.key = c->d_key;
  a.rij = c->d_rij;
  a.geom = c->d_geom;
  a.U = c->d_U;
  a.Y = c->d_Y;
  a.dedr = c->d_dedr;
  a.vpart = c->d_vpart;
  a.flags = c->d_flags;
  a.half_tmm = c->d_half_tmm;
  a.yrec = c->d_yrec;
  a.yfirst = c->d_yfirst;
  a.yruns = c->d_yruns;
  a.yslice = c->d_yslice;
  a.yi_layout = c->yi_layout;
  a.ysched = c->d_ysched;
  a.ysched_m = c->ysched_m;
  a.nslices = c->nslices;
  a.nsm = c->nsm;
  a.col_warps = c->col_warps;
  a.de_maxcnt = de_maxcnt(c, K);
  a.yi_waves = c->yi_waves;
  a.test_skip_stage = c->test_skip_stage;
  a.persist = c->persist;
  a.de_atoms = c->de_atoms;
  a.ncoeff = c->tab.ncoeff;
  a.brec = c->d_brec;
  a.brec_cp = c->d_brec_cp;
  a.bchunk_term = c->d_bchunk_term;
  a.bchunk_runs = c->d_bchunk_runs;
  a.bcomp_chunk = c->d_bcomp_chunk;
  a.bi_layout = c->bi_layout;
  a.bscratch = c->d_bscratch;
  a.nbparts = c->nbparts;
  if (c->nbparts > 0) {
    const auto& bp = c->bpart_cache.at(c->nbparts);
    a.bpart = bp.d;
    a.bmaxchunks = bp.maxchunks;
    a.bmaxterms = bp.maxterms;
  }
  a.rootpq = c->d_root;
  a.hscale = c->d_hscale;
  return a;
}

// Enqueue the whole evaluation on stream s (no synchronisation).
// mode 0: energy, forces, virial; mode 1: bispectrum components into B;
// mode 2: derivative of the bispectrum along the displacement field g into B.
// pos_stage: positions are in mapped host memory; the position kernel copies
// them there (device) and the neighbour build reads the copy.
int enqueue(snap_ctx* c, int n, const double* pos, const double* box, const int* ucnt,
            const int* uidx, const signed char* uimg, int ucap, double* energy, double* forces,
            double* virial, cudaStream_t s, int mode = 0, double* B = nullptr,
            const double* g = nullptr, double* pos_stage = nullptr) {
  const bool user = (ucnt || uidx || uimg);
  if (user && (!ucnt || !uidx || !uimg || ucap < 1 || ucap > snap::kMaxNeighCap))
    return fail(c, SNAP_ERR_ARG, "neighbour list: cnt, idx and img must all be given with 1 <= cap <= 64");
  const int K = user ? ucap : c->K;
  int rc = ensure_workspace(c, n, K);
  if (!rc) rc = ensure_flags(c);
  if (rc) return rc;
  rc = ensure_slices(c, n);
  if (!rc && mode != 0) rc = ensure_bparts(c, n, mode == 2);
  if (rc) return rc;
  SNAP_CUDA(c, open_flags(c, s));
  std::vector<cudaEvent_t> ev;
  if (c->prof_on && mode == 0) {
    if (!c->prof_free.empty()) {
      ev = c->prof_free.back();
      c->prof_free.pop_back();
    } else {
      ev.resize(SNAP_NSTAGES + 1);
      for (auto& e : ev) SNAP_CUDA(c, cudaEventCreate(&e));
    }
  }
  int stage = 0;
  auto mark = [&]() -> cudaError_t {
    if (ev.empty()) return cudaSuccess;
    return cudaEventRecord(ev[stage++], s);
  };
  c->launches = 0;
  SNAP_CUDA(c, mark());

  snap::WorkArgs a = make_args(c, n, K);
  a.energy = energy;
  a.forces = forces;
  a.virial = virial;
  a.B = B;
  const bool mixed = c->precision == SNAP_MIXED;
  // register column-chain kernels: FP32 for 2J >= 1; FP64 up to 2J = 8 (above,
  // the FP64 columns need all 255 registers and the occupancy loss costs more
  // than the layout gains: fused dE 6.1 vs 4.6 ms at 2J = 14, 2000 atoms)
  const bool colk = c->twojmax >= 1 && (mixed || c->twojmax <= 8);
  auto launch_u = [&]() -> cudaError_t {
    return colk ? (mixed ? snap::launch_ui_col<float>(a, s) : snap::launch_ui_col<double>(a, s))
                : (mixed ? snap::launch_ui<float>(a, s) : snap::launch_ui<double>(a, s));
  };
  if (user) {
    SNAP_CUDA(c, snap::launch_neigh_ingest(n, K, pos, box[0], box[1], box[2], ucnt, uidx, uimg, ucap,
                                           c->d_cnt, c->d_nbr, c->d_img, c->d_rij, c->d_key, c->d_flags, s));
    c->launches += 1;
    SNAP_CUDA(c, mark());
    SNAP_CUDA(c, launch_u());
    c->launches += 1;
  } else {
    snap::NeighArgs na;
    std::memset(&na, 0, sizeof(na));
    na.n = n;
    na.K = K;
    na.pos = pos;
    na.pos4 = c->d_pos4;
    na.tiles = c->d_tiles;
    na.Lx = box[0];
    na.Ly = box[1];
    na.Lz = box[2];
    int S[3];
    if (!snap::image_shifts(box, c->rcut, S)) return check_box(c, box);
    na.Sx = S[0];
    na.Sy = S[1];
    na.Sz = S[2];
    na.rcut = c->rcut;
    na.cnt = c->d_cnt;
    na.nbr = c->d_nbr;
    na.img = c->d_img;
    na.rij = c->d_rij;
    na.key = c->d_key;
    na.flags = c->d_flags;
    SNAP_CUDA(c, snap::launch_pos4(n, pos, c->d_pos4, s, c->d_tiles, pos_stage));
    if (pos_stage) na.pos = pos_stage;
    c->launches += 1;
    SNAP_CUDA(c, mark());
    if (colk) {
      // the neighbour build fused with compute_U
      SNAP_CUDA(c, mixed ? snap::launch_neigh_u<float>(na, a, 0, s) : snap::launch_neigh_u<double>(na, a, 0, s));
      c->launches += 1;
    } else {
      SNAP_CUDA(c, snap::launch_neigh_build(na, s));
      SNAP_CUDA(c, launch_u());
      c->launches += 2;
    }
  }
  SNAP_CUDA(c, mark());
  c->generation += 1;
  c->last_args = a;
  c->have_last = (mode == 0);
  if (mode == 1 || mode == 2) {
    if (mode == 1) {
      SNAP_CUDA(c, mixed ? snap::launch_bi<float>(a, s) : snap::launch_bi<double>(a, s));
      c->launches += 1;
    } else {
      SNAP_CUDA(c, mixed ? snap::launch_tan_col<float>(a, g, c->d_dU, s)
                         : snap::launch_tan_col<double>(a, g, c->d_dU, s));
      SNAP_CUDA(c, mixed ? snap::launch_dbi<float>(a, c->d_dU, B, s)
                         : snap::launch_dbi<double>(a, c->d_dU, B, s));
      c->launches += 2;
    }
    SNAP_CUDA(c, close_flags(c, s));
    c->last_n = n;
    c->last_K = K;
    return SNAP_OK;
  }
  SNAP_CUDA(c, mixed ? snap::launch_yi<float>(a, s) : snap::launch_yi<double>(a, s));
  SNAP_CUDA(c, mark());
  SNAP_CUDA(c, colk ? (mixed ? snap::launch_de_col<float>(a, s) : snap::launch_de_col<double>(a, s))
                    : (mixed ? snap::launch_de<float>(a, s) : snap::launch_de<double>(a, s)));
  SNAP_CUDA(c, mark());
  a.hflags = c->d_hflags;  // the force kernel ends the evaluation
  SNAP_CUDA(c, mixed ? snap::launch_force<float>(a, s) : snap::launch_force<double>(a, s));
  c->flags_dirty = false;
  SNAP_CUDA(c, mark());
  c->launches += 3;
  if (!ev.empty()) c->prof_pending.push_back(ev);
  c->last_n = n;
  c->last_K = K;
  return SNAP_OK;
}

// ---------------------------------------------------------------- batches
// Shape of a batch: per-configuration atom ranges, boxes and image ranges,
// and the CTA -> (configuration, first atom) map of the batched neighbour
// build (kNeighAtomsPerCta atoms of one configuration per CTA).  Uploaded
// when it changes.
int prepare_batch(snap_ctx* c, int nconf, const int* natoms, const double* boxes) {
  bool same = (nconf == c->bat_nconf) && (int)c->bat_n.size() == nconf;
  for (int k = 0; same && k < nconf; ++k)
    same = c->bat_n[k] == natoms[k] && c->bat_box[3 * k] == boxes[3 * k] &&
           c->bat_box[3 * k + 1] == boxes[3 * k + 1] && c->bat_box[3 * k + 2] == boxes[3 * k + 2];
  if (!same) {
    std::vector<snap::NeighConf> confs(nconf);
    std::vector<int2> map;
    int start = 0;
    for (int k = 0; k < nconf; ++k) {
      snap::NeighConf& f = confs[k];
      f.start = start;
      f.n = natoms[k];
      for (int d = 0; d < 3; ++d) f.L[d] = boxes[3 * k + d];
      if (!snap::image_shifts(f.L, c->rcut, f.S)) return check_box(c, f.L);
      for (int o = 0; o < f.n; o += snap::kNeighAtomsPerCta) map.push_back(make_int2(k, o));
      start += f.n;
    }
    int rc = upload(c, &c->d_confs, confs);
    if (!rc) rc = upload(c, &c->d_ctamap, map);
    if (rc) return rc;
    c->bat_n.assign(natoms, natoms + nconf);
    c->bat_box.assign(boxes, boxes + 3 * nconf);
    c->bat_nconf = nconf;
    c->bat_total = start;
    c->bat_ncta = (int)map.size();
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
  }
  const int n = c->bat_total;
  int rc = ensure_workspace(c, n, c->K);
  if (!rc) rc = ensure_flags(c);
  if (rc) return rc;
  const int old_slices = c->nslices;
  rc = ensure_slices(c, n);
  if (rc) return rc;
  if (c->nslices != old_slices && c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  if (n > c->cap_vatom) {
    cudaDeviceSynchronize();
    dfree(c->d_vatom);
    SNAP_CUDA(c, cudaMalloc(&c->d_vatom, sizeof(double) * 6 * (size_t)std::max(n, 1)));
    c->cap_vatom = n;
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
  }
  c->last_n = n;
  c->last_K = c->K;
  return SNAP_OK;
}

// The launch sequence of a prepared batch: asynchronous, allocates nothing
// (so it can be captured into a CUDA graph).
int launch_batch(snap_ctx* c, const double* pos, double* energy, double* forces, double* virial,
                 cudaStream_t s) {
  const int n = c->bat_total;
  SNAP_CUDA(c, open_flags(c, s));
  snap::NeighArgs na;
  std::memset(&na, 0, sizeof(na));
  na.n = n;
  na.K = c->K;
  na.confs = c->d_confs;
  na.cta_map = c->d_ctamap;
  na.pos = pos;
  na.pos4 = c->d_pos4;
  na.rcut = c->rcut;
  na.cnt = c->d_cnt;
  na.nbr = c->d_nbr;
  na.img = c->d_img;
  na.rij = c->d_rij;
  na.key = c->d_key;
  na.flags = c->d_flags;
  snap::WorkArgs a = make_args(c, n, c->K);
  a.energy = energy;
  a.forces = forces;
  a.virial = virial;
  a.vatom = c->d_vatom;
  const bool mixed = c->precision == SNAP_MIXED;
  const bool colk = c->twojmax >= 1 && (mixed || c->twojmax <= 8);
  SNAP_CUDA(c, snap::launch_pos4(n, pos, c->d_pos4, s));
  int nl = 1;
  if (colk) {
    SNAP_CUDA(c, mixed ? snap::launch_neigh_u<float>(na, a, c->bat_ncta, s)
                       : snap::launch_neigh_u<double>(na, a, c->bat_ncta, s));
    nl += 1;
  } else {
    SNAP_CUDA(c, snap::launch_neigh_build_batch(na, c->bat_ncta, s));
    SNAP_CUDA(c, mixed ? snap::launch_ui<float>(a, s) : snap::launch_ui<double>(a, s));
    nl += 2;
  }
  SNAP_CUDA(c, mixed ? snap::launch_yi<float>(a, s) : snap::launch_yi<double>(a, s));
  SNAP_CUDA(c, colk ? (mixed ? snap::launch_de_col<float>(a, s) : snap::launch_de_col<double>(a, s))
                    : (mixed ? snap::launch_de<float>(a, s) : snap::launch_de<double>(a, s)));
  a.hflags = c->d_hflags;  // the force kernel ends the evaluation (the virial sums use no flag)
  SNAP_CUDA(c, mixed ? snap::launch_force<float>(a, s) : snap::launch_force<double>(a, s));
  c->flags_dirty = false;
  a.hflags = nullptr;
  if (virial) SNAP_CUDA(c, snap::launch_virial_conf(c->d_vatom, c->d_confs, c->bat_nconf, virial, s));
  c->launches = nl + 3 + (virial ? 1 : 0);
  c->generation += 1;
  c->last_args = a;
  c->have_last = true;
  return SNAP_OK;
}

// The derivative of the bispectrum of a prepared batch along g (mode 2 of
// enqueue over the concatenated configurations): asynchronous, allocates
// nothing.
int launch_batch_deriv(snap_ctx* c, const double* pos, const double* g, double* dB, cudaStream_t s) {
  const int n = c->bat_total;
  SNAP_CUDA(c, open_flags(c, s));
  snap::NeighArgs na;
  std::memset(&na, 0, sizeof(na));
  na.n = n;
  na.K = c->K;
  na.confs = c->d_confs;
  na.cta_map = c->d_ctamap;
  na.pos = pos;
  na.pos4 = c->d_pos4;
  na.rcut = c->rcut;
  na.cnt = c->d_cnt;
  na.nbr = c->d_nbr;
  na.img = c->d_img;
  na.rij = c->d_rij;
  na.key = c->d_key;
  na.flags = c->d_flags;
  snap::WorkArgs a = make_args(c, n, c->K);
  const bool mixed = c->precision == SNAP_MIXED;
  const bool colk = c->twojmax >= 1 && (mixed || c->twojmax <= 8);
  SNAP_CUDA(c, snap::launch_pos4(n, pos, c->d_pos4, s));
  int nl = 1;
  if (colk) {
    SNAP_CUDA(c, mixed ? snap::launch_neigh_u<float>(na, a, c->bat_ncta, s)
                       : snap::launch_neigh_u<double>(na, a, c->bat_ncta, s));
    nl += 1;
  } else {
    SNAP_CUDA(c, snap::launch_neigh_build_batch(na, c->bat_ncta, s));
    SNAP_CUDA(c, mixed ? snap::launch_ui<float>(a, s) : snap::launch_ui<double>(a, s));
    nl += 2;
  }
  SNAP_CUDA(c, mixed ? snap::launch_tan_col<float>(a, g, c->d_dU, s) : snap::launch_tan_col<double>(a, g, c->d_dU, s));
  SNAP_CUDA(c, mixed ? snap::launch_dbi<float>(a, c->d_dU, dB, s) : snap::launch_dbi<double>(a, c->d_dU, dB, s));
  SNAP_CUDA(c, close_flags(c, s));
  c->launches = nl + 2 + 1;  // + the flags kernel
  c->generation += 1;
  c->have_last = false;
  return SNAP_OK;
}

int check_flags(snap_ctx* c) {
  c->last_nmax = c->h_flags[0];
  c->seen_nmax = std::max(c->seen_nmax, c->last_nmax);
  if (c->h_flags[3]) return fail(c, SNAP_ERR_TIMEOUT, "a bounded device wait (TMA staging) gave up");
  if (c->h_flags[2]) return fail(c, SNAP_ERR_ARG, "neighbour list: count outside 0..cap or index outside 0..N-1");
  if (c->h_flags[0] > c->last_K)
    return fail(c, SNAP_ERR_NEIGH_OVERFLOW,
                "an atom has " + std::to_string(c->h_flags[0]) + " neighbours, capacity is " +
                    std::to_string(c->last_K));
  if (c->h_flags[1]) return fail(c, SNAP_ERR_NEIGH_ASYM, "neighbour list is not symmetric (missing reverse pair)");
  return SNAP_OK;
}

unsigned long long key_bits(double x) {
  unsigned long long u;
  std::memcpy(&u, &x, sizeof(u));
  return u;
}
unsigned long long key_ptr(const void* p) { return (unsigned long long)(uintptr_t)p; }

bool pinned_or_null(const void* p) {
  if (!p) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// Replay the slot's graph if the key matches; run directly the first time a
// key is seen; capture (on the context's capture stream) and replay the
// second time in a row.  run(stream) enqueues the whole evaluation and sets
// the host-side state of the call (generation, last arguments and sizes).
template <typename F>
int graph_run(snap_ctx* c, GraphSlot& g, const std::vector<unsigned long long>& key, cudaStream_t s,
              F&& run) {
  if (!(g.exec && g.key == key)) {
    if (g.seen != key) {
      g.seen = key;
      return run(s);
    }
    g.reset();
    if (!c->gstream) SNAP_CUDA(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    const long long gen0 = c->generation;
    SNAP_CUDA(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    const int rc = run(c->gstream);
    cudaError_t e = cudaStreamEndCapture(c->gstream, &graph);
    c->generation = gen0;  // capturing evaluated nothing
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(c, SNAP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return fail(c, SNAP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    g.key = key;
    g.args = c->last_args;
    g.n = c->last_n;
    g.K = c->last_K;
    g.launches = c->launches;
  }
  SNAP_CUDA(c, cudaGraphLaunch(g.exec, s));
  c->generation += 1;
  c->last_args = g.args;
  c->have_last = true;
  c->last_n = g.n;
  c->last_K = g.K;
  c->launches = g.launches;
  return SNAP_OK;
}

// One energy + force evaluation on device buffers, through a cached CUDA
// graph when the same call repeats (not while stage profiling is on).
int compute_dev(snap_ctx* c, int n, const double* pos, const double* box, const int* ucnt,
                const int* uidx, const signed char* uimg, int ucap, double* energy, double* forces,
                double* virial, cudaStream_t s) {
  const bool user = (ucnt || uidx || uimg);
  auto run = [&](cudaStream_t st) {
    return enqueue(c, n, pos, box, ucnt, uidx, uimg, ucap, energy, forces, virial, st);
  };
  if (c->prof_on || (user && (!ucnt || !uidx || !uimg || ucap < 1 || ucap > snap::kMaxNeighCap))) return run(s);
  // every buffer exists before a capture (no allocation inside one)
  const int K = user ? ucap : c->K;
  int rc = ensure_workspace(c, n, K);
  if (!rc) rc = ensure_flags(c);
  if (!rc) rc = ensure_slices(c, n);
  if (rc) return rc;
  const std::vector<unsigned long long> key = {
      1, (unsigned long long)c->ws_gen, (unsigned long long)n, (unsigned long long)K,
      (unsigned long long)c->col_warps, (unsigned long long)c->yi_waves,
      (unsigned long long)c->yi_layout | ((unsigned long long)c->persist << 8) |
          ((unsigned long long)c->de_atoms << 16),
      key_bits(box[0]), key_bits(box[1]), key_bits(box[2]), key_ptr(pos), key_ptr(energy), key_ptr(forces),
      key_ptr(virial), key_ptr(ucnt), key_ptr(uidx), key_ptr(uimg), (unsigned long long)ucap,
      (unsigned long long)de_maxcnt(c, K)};
  return graph_run(c, c->gdev, key, s, run);
}

}  // namespace

extern "C" {

int snap_num_coeff(int twojmax) { return snap::count_coeff(twojmax); }

int snap_half_size(int twojmax) {
  if (twojmax < 0 || twojmax > snap::kMaxTwoJ) return -1;
  return snap::half_size(twojmax);
}

int snap_half_index(int twojmax, int t, int ma, int mb) {
  if (twojmax < 0 || twojmax > snap::kMaxTwoJ || t < 0 || t > twojmax || ma < 0 || ma > t || mb < 0 ||
      2 * mb > t)
    return -1;
  return snap::half_base(t) + mb * (t + 1) + ma;
}

int snap_yi_host(int twojmax, int precision, const double* beta, const double* u, double* y) {
  if (twojmax < 0 || twojmax > snap::kMaxTwoJ || (precision != SNAP_FP64 && precision != SNAP_MIXED) ||
      !beta || !u || !y)
    return SNAP_ERR_ARG;
  snap::HostTables tab;
  tab.build(twojmax, precision == SNAP_MIXED);
  const std::vector<double> coef = tab.term_coef(beta);
  auto fac = [&](unsigned idx, unsigned conj, double& re, double& im) {
    re = u[2 * idx];
    im = conj ? -u[2 * idx + 1] : u[2 * idx + 1];
  };
  for (int o = 0; o < tab.H; ++o) {
    double yr = 0.0, yi = 0.0;
    for (int k = tab.term_out_first[o]; k < tab.term_out_first[o + 1]; ++k) {
      const unsigned w = tab.terms[k];
      double ar, ai, br, bi;
      fac(w & 1023u, (w >> 20) & 1u, ar, ai);
      fac((w >> 10) & 1023u, (w >> 21) & 1u, br, bi);
      yr += coef[k] * (ar * br - ai * bi);
      yi += coef[k] * (ar * bi + ai * br);
    }
    y[2 * o] = yr;
    y[2 * o + 1] = yi;
  }
  return SNAP_OK;
}

int snap_bi_host(int twojmax, int layout, const double* u, double* b) {
  if (twojmax < 0 || twojmax > snap::kMaxTwoJ || (layout != 0 && layout != 1) || !u || !b) return SNAP_ERR_ARG;
  snap::HostTables tab;
  tab.build(twojmax);
  const bool cp = layout == 1;
  const std::vector<unsigned> words = tab.bwords(cp);
  if (words.size() != tab.bdev.size()) return SNAP_ERR_ARG;
  const int H = tab.H;
  // factor x of the word: an element, conjugated past H (cp) or by its flag
  auto fac = [&](unsigned x, unsigned conj, double& re, double& im) {
    if (cp && x >= (unsigned)H) {
      x -= (unsigned)H;
      conj = 1;
    }
    re = u[2 * x];
    im = conj ? -u[2 * x + 1] : u[2 * x + 1];
  };
  for (int l = 0; l < tab.ncoeff; ++l) {
    double v = 0.0;
    for (int ch = tab.bcomp_chunk[l]; ch < tab.bcomp_chunk[l + 1]; ++ch) {
      // the chunk's runs of pieces of 1, 2, ... kBGroupMax terms, in order
      int q = tab.bchunk_term[ch];
      double acc = 0.0;
      for (int len = 1; len <= snap::kBGroupMax; ++len) {
        for (int n = tab.bchunk_runs[(size_t)ch * snap::kBGroupMax + len - 1]; n > 0; --n) {
          const unsigned w0 = words[q];
          const unsigned o = (w0 & 0xFFu) | (((w0 >> (cp ? 30 : 28)) & 3u) << 8);
          double zr = 0.0, zi = 0.0;
          for (int k = 0; k < len; ++k, ++q) {
            const unsigned w = words[q];
            const unsigned x1 = cp ? (w >> 19) & 0x7FFu : (w >> 18) & 0x3FFu;
            const unsigned x2 = cp ? (w >> 8) & 0x7FFu : (w >> 8) & 0x3FFu;
            double ar, ai, br, bi;
            fac(x1, cp ? 0u : (w >> 30) & 1u, ar, ai);
            fac(x2, cp ? 0u : (w >> 31) & 1u, br, bi);
            const double c = tab.bdev_coef[q];
            zr += c * (ar * br - ai * bi);
            zi += c * (ar * bi + ai * br);
          }
          acc += u[2 * o] * zr + u[2 * o + 1] * zi;  // Re(Z conj U_o)
        }
      }
      if (q != tab.bchunk_term[ch + 1]) return SNAP_ERR_ARG;  // runs must cover the chunk
      v += acc;
    }
    b[l] = v;
  }
  return SNAP_OK;
}

int snap_create(int twojmax, double rcut, double rfac0, double rmin0, int switchflag,
                const double* beta, int precision, snap_ctx** out) {
  if (!out) {
    g_create_error = "out is NULL";
    return SNAP_ERR_ARG;
  }
  *out = nullptr;
  if (twojmax < 0 || twojmax > snap::kMaxTwoJ) {
    g_create_error = "twojmax must be in 0..14";
    return SNAP_ERR_ARG;
  }
  if (!(std::isfinite(rcut) && std::isfinite(rmin0) && rmin0 >= 0.0 && rcut > rmin0)) {
    g_create_error = "need 0 <= rmin0 < rcut";
    return SNAP_ERR_ARG;
  }
  if (!(rfac0 > 0.0 && rfac0 <= 1.0)) {
    g_create_error = "rfac0 must be in (0, 1]";
    return SNAP_ERR_ARG;
  }
  if (switchflag != 0 && switchflag != 1) {
    g_create_error = "switchflag must be 0 or 1";
    return SNAP_ERR_ARG;
  }
  if (precision != SNAP_FP64 && precision != SNAP_MIXED) {
    g_create_error = "precision must be SNAP_FP64 or SNAP_MIXED";
    return SNAP_ERR_ARG;
  }
  if (!beta) {
    g_create_error = "beta is NULL";
    return SNAP_ERR_ARG;
  }
  snap_ctx* c = new (std::nothrow) snap_ctx;
  if (!c) {
    g_create_error = "out of host memory";
    return SNAP_ERR_NOMEM;
  }
  c->twojmax = twojmax;
  c->rcut = rcut;
  c->rfac0 = rfac0;
  c->rmin0 = rmin0;
  c->switchflag = switchflag;
  c->precision = precision;
  c->tab.build(twojmax, precision == SNAP_MIXED);
  c->beta.assign(beta, beta + 1 + c->tab.ncoeff);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA: ") + cudaGetErrorString(e);
    delete c;
    return SNAP_ERR_CUDA;
  }
  int rc = upload(c, &c->d_half_tmm, c->tab.half_tmm);
  if (!rc) rc = upload(c, &c->d_yfirst, c->tab.term_out_first);
  if (!rc) rc = upload(c, &c->d_yruns, c->tab.term_runs);
  if (!rc) rc = upload(c, &c->d_ysched, c->tab.lane_outputs(32, &c->ysched_m));
  if (!rc) rc = upload_r(c, &c->d_root, c->tab.rootpq);
  if (!rc) rc = upload_r(c, &c->d_hscale, c->tab.half_scale);
  if (!rc) rc = upload_yrec(c);
  if (!rc) rc = upload_brec(c);
  if (!rc) rc = upload(c, &c->d_bchunk_term, c->tab.bchunk_term);
  if (!rc) rc = upload(c, &c->d_bchunk_runs, c->tab.bchunk_runs);
  if (!rc) rc = upload(c, &c->d_bcomp_chunk, c->tab.bcomp_chunk);
  if (rc) {
    g_create_error = c->err;
    snap_destroy(c);
    return rc;
  }
  *out = c;
  return SNAP_OK;
}

int snap_set_beta(snap_ctx* c, const double* beta) {
  if (!c || !beta) return fail(c, SNAP_ERR_ARG, "NULL argument");
  cudaDeviceSynchronize();
  c->beta.assign(beta, beta + 1 + c->tab.ncoeff);
  // beta_0 is a kernel argument: captured graphs hold the old value
  c->gdev.reset();
  c->ghost.reset();
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return upload_yrec(c);
}

int snap_set_neigh_cap(snap_ctx* c, int cap) {
  if (!c) return SNAP_ERR_ARG;
  if (cap < 1 || cap > snap::kMaxNeighCap) return fail(c, SNAP_ERR_ARG, "capacity must be in 1..64");
  c->K = cap;
  return SNAP_OK;
}

int snap_neigh_max(const snap_ctx* c) { return c ? c->last_nmax : -1; }

int snap_compute(snap_ctx* c, int natoms, const double* pos, const double* box, const int* nbr_cnt,
                 const int* nbr_idx, const signed char* nbr_img, int nbr_cap, double* energy,
                 double* forces, double* virial, void* stream) {
  if (!c) return SNAP_ERR_ARG;
  if (natoms < 0) return fail(c, SNAP_ERR_ARG, "natoms < 0");
  if (int rb = check_box(c, box)) return rb;
  cudaStream_t s = (cudaStream_t)stream;
  if (natoms == 0) {
    if (virial) SNAP_CUDA(c, cudaMemsetAsync(virial, 0, 6 * sizeof(double), s));
    return SNAP_OK;
  }
  if (!pos || !forces) return fail(c, SNAP_ERR_ARG, "pos and forces are required");
  int rc = compute_dev(c, natoms, pos, box, nbr_cnt, nbr_idx, nbr_img, nbr_cap, energy, forces, virial, s);
  if (rc) return rc;
  SNAP_CUDA(c, cudaStreamSynchronize(s));
  return check_flags(c);
}

int snap_compute_async(snap_ctx* c, int natoms, const double* pos, const double* box,
                       const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                       int nbr_cap, double* energy, double* forces, double* virial, void* stream) {
  if (!c) return SNAP_ERR_ARG;
  if (natoms < 0) return fail(c, SNAP_ERR_ARG, "natoms < 0");
  if (int rb = check_box(c, box)) return rb;
  cudaStream_t s = (cudaStream_t)stream;
  if (natoms == 0) {
    if (virial) SNAP_CUDA(c, cudaMemsetAsync(virial, 0, 6 * sizeof(double), s));
    return SNAP_OK;
  }
  if (!pos || !forces) return fail(c, SNAP_ERR_ARG, "pos and forces are required");
  return compute_dev(c, natoms, pos, box, nbr_cnt, nbr_idx, nbr_img, nbr_cap, energy, forces, virial, s);
}

int snap_sync(snap_ctx* c, void* stream) {
  if (!c) return SNAP_ERR_ARG;
  SNAP_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
  if (!c->h_flags || c->last_n == 0) return SNAP_OK;
  return check_flags(c);
}

int snap_profile(snap_ctx* c, int enable) {
  if (!c) return SNAP_ERR_ARG;
  double ms[SNAP_NSTAGES];
  long long calls[SNAP_NSTAGES];
  snap_profile_read(c, ms, calls, SNAP_NSTAGES);  // drain pending events
  for (int k = 0; k < SNAP_NSTAGES; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_calls[k] = 0;
  }
  c->prof_on = enable != 0;
  return SNAP_OK;
}

int snap_profile_read(snap_ctx* c, double* ms, long long* calls, int nstages) {
  if (!c) return SNAP_ERR_ARG;
  for (auto& ev : c->prof_pending) {
    SNAP_CUDA(c, cudaEventSynchronize(ev[SNAP_NSTAGES]));
    for (int k = 0; k < SNAP_NSTAGES; ++k) {
      float t = 0.f;
      SNAP_CUDA(c, cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
      c->prof_ms[k] += t;
      c->prof_calls[k] += 1;
    }
    c->prof_free.push_back(ev);
  }
  c->prof_pending.clear();
  for (int k = 0; k < std::min(nstages, SNAP_NSTAGES); ++k) {
    if (ms) ms[k] = c->prof_ms[k];
    if (calls) calls[k] = c->prof_calls[k];
  }
  return SNAP_NSTAGES;
}

const char* snap_stage_name(int stage) {
  static const char* names[SNAP_NSTAGES] = {"neighbor_prep", "neighbor_compute_ui",
                                            "compute_yi", "fused_dE", "energy_force_virial"};
  return (stage >= 0 && stage < SNAP_NSTAGES) ? names[stage] : "";
}

int snap_launches_per_call(const snap_ctx* c) { return c ? c->launches : -1; }

namespace {
int bispectrum_enqueue(snap_ctx* c, int natoms, const double* pos, const double* box, const int* nbr_cnt,
                       const int* nbr_idx, const signed char* nbr_img, int nbr_cap, double* B, cudaStream_t s) {
  if (!c) return SNAP_ERR_ARG;
  if (natoms < 0) return fail(c, SNAP_ERR_ARG, "natoms < 0");
  if (int rb = check_box(c, box)) return rb;
  if (natoms == 0) return SNAP_OK;
  if (!pos || !B) return fail(c, SNAP_ERR_ARG, "pos and B are required");
  return enqueue(c, natoms, pos, box, nbr_cnt, nbr_idx, nbr_img, nbr_cap, nullptr, nullptr, nullptr, s, 1, B);
}
}  // namespace

int snap_compute_bispectrum(snap_ctx* c, int natoms, const double* pos, const double* box,
                            const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                            int nbr_cap, double* B, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int rc = bispectrum_enqueue(c, natoms, pos, box, nbr_cnt, nbr_idx, nbr_img, nbr_cap, B, s);
  if (rc || natoms == 0) return rc;
  SNAP_CUDA(c, cudaStreamSynchronize(s));
  return check_flags(c);
}

int snap_compute_bispectrum_async(snap_ctx* c, int natoms, const double* pos, const double* box,
                                  const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                                  int nbr_cap, double* B, void* stream) {
  return bispectrum_enqueue(c, natoms, pos, box, nbr_cnt, nbr_idx, nbr_img, nbr_cap, B, (cudaStream_t)stream);
}

int snap_bispectrum_deriv(snap_ctx* c, int natoms, const double* pos, const double* box,
                          const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                          int nbr_cap, const double* g, double* dB, void* stream) {
  if (!c) return SNAP_ERR_ARG;
  if (natoms < 0) return fail(c, SNAP_ERR_ARG, "natoms < 0");
  if (int rb = check_box(c, box)) return rb;
  if (natoms == 0) return SNAP_OK;
  if (!pos || !g || !dB) return fail(c, SNAP_ERR_ARG, "pos, g and dB are required");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = enqueue(c, natoms, pos, box, nbr_cnt, nbr_idx, nbr_img, nbr_cap, nullptr, nullptr, nullptr, s,
                   2, dB, g);
  if (rc) return rc;
  SNAP_CUDA(c, cudaStreamSynchronize(s));
  return check_flags(c);
}

int snap_force_weighted(snap_ctx* c, const double* weight, double* grad, void* stream) {
  if (!c) return SNAP_ERR_ARG;
  if (!c->have_last) return fail(c, SNAP_ERR_ARG, "no energy/force evaluation to differentiate");
  if (!weight || !grad) return fail(c, SNAP_ERR_ARG, "weight and grad are required");
  if (c->last_n == 0) return SNAP_OK;
  SNAP_CUDA(c, snap::launch_force_weighted(c->last_args, weight, grad, (cudaStream_t)stream));
  return SNAP_OK;
}

long long snap_generation(const snap_ctx* c) { return c ? c->generation : -1; }

int snap_compute_batch(snap_ctx* c, int nconf, const int* natoms, const double* boxes,
                       const double* pos, double* energy, double* forces, double* virial,
                       int use_graph, void* stream) {
  if (!c) return SNAP_ERR_ARG;
  if (nconf < 0 || (nconf > 0 && (!natoms || !boxes))) return fail(c, SNAP_ERR_ARG, "bad batch description");
  long total = 0;
  for (int k = 0; k < nconf; ++k) {
    if (natoms[k] < 0) return fail(c, SNAP_ERR_ARG, "natoms < 0");
    if (int rb = check_box(c, boxes + 3 * k)) return rb;
    total += natoms[k];
  }
  if (total > (1L << 30)) return fail(c, SNAP_ERR_ARG, "batch too large");
  if (total == 0) return SNAP_OK;
  if (!pos || !forces) return fail(c, SNAP_ERR_ARG, "pos and forces are required");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = prepare_batch(c, nconf, natoms, boxes);
  if (rc) return rc;
  if (!use_graph) return launch_batch(c, pos, energy, forces, virial, s);
  const void* key[4] = {pos, energy, forces, virial};
  const int demax = de_maxcnt(c, c->K);
  const bool same = c->gexec && std::equal(key, key + 4, c->g_key) && c->g_ws == c->ws_gen && c->g_demax == demax;
  if (!same) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    if (!c->gstream) SNAP_CUDA(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    SNAP_CUDA(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    rc = launch_batch(c, pos, energy, forces, virial, c->gstream);
    cudaError_t e = cudaStreamEndCapture(c->gstream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(c, SNAP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->gexec = nullptr;
      return fail(c, SNAP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    std::copy(key, key + 4, c->g_key);
    c->g_ws = c->ws_gen;
    c->g_demax = demax;
  }
  SNAP_CUDA(c, cudaGraphLaunch(c->gexec, s));
  c->generation += 1;
  return SNAP_OK;
}

int snap_bispectrum_deriv_batch(snap_ctx* c, int nconf, const int* natoms, const double* boxes,
                                const double* pos, const double* g, double* dB, void* stream) {
  if (!c) return SNAP_ERR_ARG;
  if (nconf < 0 || (nconf > 0 && (!natoms || !boxes))) return fail(c, SNAP_ERR_ARG, "bad batch description");
  long total = 0;
  for (int k = 0; k < nconf; ++k) {
    if (natoms[k] < 0) return fail(c, SNAP_ERR_ARG, "natoms < 0");
    if (int rb = check_box(c, boxes + 3 * k)) return rb;
    total += natoms[k];
  }
  if (total > (1L << 30)) return fail(c, SNAP_ERR_ARG, "batch too large");
  if (total == 0) return SNAP_OK;
  if (!pos || !g || !dB) return fail(c, SNAP_ERR_ARG, "pos, g and dB are required");
  int rc = prepare_batch(c, nconf, natoms, boxes);
  if (!rc) rc = ensure_bparts(c, c->bat_total, true);
  if (rc) return rc;
  return launch_batch_deriv(c, pos, g, dB, (cudaStream_t)stream);
}

int snap_set_tuning(snap_ctx* c, int col_warps, int yi_waves, int yi_layout) {
  if (!c) return SNAP_ERR_ARG;
  if (col_warps != 2 && col_warps != 4 && col_warps != 8)
    return fail(c, SNAP_ERR_ARG, "col_warps must be 2, 4 or 8");
  if (yi_waves < 1 || yi_waves > 8) return fail(c, SNAP_ERR_ARG, "yi_waves must be in 1..8");
  if (yi_layout != 0 && yi_layout != 1) return fail(c, SNAP_ERR_ARG, "yi_layout must be 0 or 1");
  if (c->col_warps != col_warps || c->yi_waves != yi_waves || c->yi_layout != yi_layout) {
    c->col_warps = col_warps;
    c->yi_waves = yi_waves;
    c->yi_layout = yi_layout;
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
  }
  return SNAP_OK;
}

int snap_set_knob(snap_ctx* c, int knob, int value) {
  if (!c) return SNAP_ERR_ARG;
  switch (knob) {
    case SNAP_KNOB_COL_WARPS: return snap_set_tuning(c, value, c->yi_waves, c->yi_layout);
    case SNAP_KNOB_YI_WAVES: return snap_set_tuning(c, c->col_warps, value, c->yi_layout);
    case SNAP_KNOB_YI_LAYOUT: return snap_set_tuning(c, c->col_warps, c->yi_waves, value);
    case SNAP_KNOB_PERSIST:
    case SNAP_KNOB_DE_ATOMS: {
      int& slot = knob == SNAP_KNOB_PERSIST ? c->persist : c->de_atoms;
      if (knob == SNAP_KNOB_PERSIST && (value < 0 || value > 3))
        return fail(c, SNAP_ERR_ARG, "persist must be in 0..3");
      if (knob == SNAP_KNOB_DE_ATOMS && (value < 0 || value > 256))
        return fail(c, SNAP_ERR_ARG, "de_atoms must be in 0..256");
      if (slot != value) {
        slot = value;
        c->gdev.reset();
        c->ghost.reset();
        if (c->gexec) {
          cudaGraphExecDestroy(c->gexec);
          c->gexec = nullptr;
        }
      }
      return SNAP_OK;
    }
    case SNAP_KNOB_BI_LAYOUT:
      if (value < 0 || value > 2) return fail(c, SNAP_ERR_ARG, "bi_layout must be in 0..2");
      if (c->bi_layout != value) {
        c->bi_layout = value;
        c->nbparts = 0;  // re-plan the runs and the scratch
      }
      return SNAP_OK;
    default: return fail(c, SNAP_ERR_ARG, "unknown knob");
  }
}

int snap_get_knob(const snap_ctx* c, int knob, int* value) {
  if (!c || !value) return SNAP_ERR_ARG;
  switch (knob) {
    case SNAP_KNOB_COL_WARPS: *value = c->col_warps; return SNAP_OK;
    case SNAP_KNOB_YI_WAVES: *value = c->yi_waves; return SNAP_OK;
    case SNAP_KNOB_YI_LAYOUT: *value = c->yi_layout; return SNAP_OK;
    case SNAP_KNOB_PERSIST: *value = c->persist; return SNAP_OK;
    case SNAP_KNOB_DE_ATOMS: *value = c->de_atoms; return SNAP_OK;
    case SNAP_KNOB_BI_LAYOUT: *value = c->bi_layout; return SNAP_OK;
    default: return SNAP_ERR_ARG;
  }
}

int snap_test_stage_timeout(snap_ctx* c, int on) {
  if (!c) return SNAP_ERR_ARG;
  if (on != 0 && on != 1) return fail(c, SNAP_ERR_ARG, "on must be 0 or 1");
  if (c->test_skip_stage != on) {
    c->test_skip_stage = on;
    // the flag is a kernel argument: captured graphs hold the old value
    c->gdev.reset();
    c->ghost.reset();
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
  }
  return SNAP_OK;
}

int snap_get_tuning(const snap_ctx* c, int* col_warps, int* yi_waves, int* yi_layout) {
  if (!c) return SNAP_ERR_ARG;
  if (col_warps) *col_warps = c->col_warps;
  if (yi_waves) *yi_waves = c->yi_waves;
  if (yi_layout) *yi_layout = c->yi_layout;
  return SNAP_OK;
}

int snap_autotune(snap_ctx* c, int nconf, const int* natoms, const double* boxes, const double* pos,
                  double* energy, double* forces, double* virial, int reps, double* best_ms,
                  void* stream) {
  if (!c) return SNAP_ERR_ARG;
  if (reps < 1) reps = 5;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  SNAP_CUDA(c, cudaEventCreate(&e0));
  SNAP_CUDA(c, cudaEventCreate(&e1));
  // median milliseconds of the batch at the context's current knobs
  auto measure = [&](double* out) -> int {
    std::vector<float> ms;
    for (int it = 0; it < reps + 2; ++it) {
      cudaEventRecord(e0, s);
      const int r = snap_compute_batch(c, nconf, natoms, boxes, pos, energy, forces, virial, 0, stream);
      cudaEventRecord(e1, s);
      if (r) return r;
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (it >= 2) ms.push_back(t);
    }
    std::sort(ms.begin(), ms.end());
    *out = ms[ms.size() / 2];
    return SNAP_OK;
  };
  const int cw[3] = {2, 4, 8};
  const int yw[3] = {1, 2, 4};
  double best = 1e300;
  int bc = c->col_warps, by = c->yi_waves, bl = c->yi_layout, bp = c->persist;
  int rc = snap_set_knob(c, SNAP_KNOB_PERSIST, 0);
  // 1. launch shapes: col_warps x (yi_waves of the warp-of-atoms compute_Y,
  //    or the warp-per-atom compute_Y, which has no split), one-shot grids
  for (int a = 0; a < 3 && !rc; ++a)
    for (int b = 0; b < 4 && !rc; ++b) {
      const int lay = b == 3 ? 1 : 0;
      const int wav = b == 3 ? c->yi_waves : yw[b];
      rc = snap_set_tuning(c, cw[a], wav, lay);
      double med = 0.0;
      if (!rc) rc = measure(&med);
      if (!rc && med < best) {
        best = med;
        bc = cw[a];
        by = wav;
        bl = lay;
        bp = 0;
      }
    }
  // 2. at the best shape, the persistent work-queue launches of compute_Y
  //    and the fused dE (alone and together)
  if (!rc) rc = snap_set_tuning(c, bc, by, bl);
  for (int p = 1; p <= 3 && !rc; ++p) {
    rc = snap_set_knob(c, SNAP_KNOB_PERSIST, p);
    double med = 0.0;
    if (!rc) rc = measure(&med);
    if (!rc && med < best) {
      best = med;
      bp = p;
    }
  }
  // 3. at the best of those, the fused dE kernel's atoms per CTA (the pass
  //    count of a warp follows from it): planned, or 2, 4, ... 32
  int bd = 0;
  if (!rc) rc = snap_set_knob(c, SNAP_KNOB_PERSIST, bp);
  for (int d = 2; d <= 32 && !rc; d *= 2) {
    rc = snap_set_knob(c, SNAP_KNOB_DE_ATOMS, d);
    double med = 0.0;
    if (!rc) rc = measure(&med);
    if (!rc && med < best) {
      best = med;
      bd = d;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = snap_set_tuning(c, bc, by, bl);
  if (!rc) rc = snap_set_knob(c, SNAP_KNOB_PERSIST, bp);
  if (!rc) rc = snap_set_knob(c, SNAP_KNOB_DE_ATOMS, bd);
  if (best_ms) *best_ms = best;
  SNAP_CUDA(c, cudaStreamSynchronize(s));
  return rc ? rc : check_flags(c);
}

int snap_compute_host(snap_ctx* c, int natoms, const double* pos_host, const double* box,
                      double* energy_host, double* forces_host, double* virial_host, void* stream) {
  if (!c) return SNAP_ERR_ARG;
  if (natoms < 0) return fail(c, SNAP_ERR_ARG, "natoms < 0");
  if (int rb = check_box(c, box)) return rb;
  if (natoms == 0) {
    if (virial_host) std::memset(virial_host, 0, 6 * sizeof(double));
    return SNAP_OK;
  }
  if (!pos_host || !forces_host) return fail(c, SNAP_ERR_ARG, "pos and forces are required");
  cudaStream_t s = (cudaStream_t)stream;
  if (natoms > c->cap_host) {
    cudaDeviceSynchronize();
    dfree(c->d_hpos);
    dfree(c->d_hE);
    dfree(c->d_hF);
    dfree(c->d_hW);
    SNAP_CUDA(c, cudaMalloc(&c->d_hpos, sizeof(double) * 3 * natoms));
    SNAP_CUDA(c, cudaMalloc(&c->d_hE, sizeof(double) * natoms));
    SNAP_CUDA(c, cudaMalloc(&c->d_hF, sizeof(double) * 3 * natoms));
    SNAP_CUDA(c, cudaMalloc(&c->d_hW, sizeof(double) * 6));
    c->cap_host = natoms;
  }
  auto run = [&](cudaStream_t st) -> int {
    SNAP_CUDA(c, cudaMemcpyAsync(c->d_hpos, pos_host, sizeof(double) * 3 * natoms, cudaMemcpyHostToDevice, st));
    int rc = enqueue(c, natoms, c->d_hpos, box, nullptr, nullptr, nullptr, 0, energy_host ? c->d_hE : nullptr,
                     c->d_hF, virial_host ? c->d_hW : nullptr, st);
    if (rc) return rc;
    if (energy_host)
      SNAP_CUDA(c, cudaMemcpyAsync(energy_host, c->d_hE, sizeof(double) * natoms, cudaMemcpyDeviceToHost, st));
    SNAP_CUDA(c, cudaMemcpyAsync(forces_host, c->d_hF, sizeof(double) * 3 * natoms, cudaMemcpyDeviceToHost, st));
    if (virial_host)
      SNAP_CUDA(c, cudaMemcpyAsync(virial_host, c->d_hW, sizeof(double) * 6, cudaMemcpyDeviceToHost, st));
    return SNAP_OK;
  };
  // With pinned (hence device-mapped) host buffers the kernels read the
  // positions and write the results through the mapping: the position kernel
  // stages the positions in device memory as it reads them, the force kernel
  // writes energies, forces and virial straight to the caller's buffers.
  const double* mpos = nullptr;
  double *mE = nullptr, *mF = nullptr, *mW = nullptr;
  auto mapped = [&]() -> bool {
    auto dev = [](const void* h, void** d) {
      if (!h) return true;
      if (cudaHostGetDevicePointer(d, const_cast<void*>(h), 0) == cudaSuccess) return true;
      cudaGetLastError();
      return false;
    };
    return dev(pos_host, (void**)&mpos) && dev(energy_host, (void**)&mE) && dev(forces_host, (void**)&mF) &&
           dev(virial_host, (void**)&mW);
  };
  auto run_mapped = [&](cudaStream_t st) -> int {
    return enqueue(c, natoms, mpos, box, nullptr, nullptr, nullptr, 0, mE, mF, mW, st, 0, nullptr, nullptr,
                   c->d_hpos);
  };
  int rc = SNAP_OK;
  if (c->prof_on) {
    rc = run(s);
  } else {
    // every buffer exists before a capture (no allocation inside one)
    rc = ensure_workspace(c, natoms, c->K);
    if (!rc) rc = ensure_flags(c);
    if (!rc) rc = ensure_slices(c, natoms);
    if (rc) return rc;
    const std::vector<unsigned long long> key = {
        2, (unsigned long long)c->ws_gen, (unsigned long long)natoms, (unsigned long long)c->K,
        (unsigned long long)c->col_warps, (unsigned long long)c->yi_waves,
        (unsigned long long)c->yi_layout | ((unsigned long long)c->persist << 8) |
            ((unsigned long long)c->de_atoms << 16),
        key_bits(box[0]), key_bits(box[1]), key_bits(box[2]), key_ptr(pos_host), key_ptr(energy_host),
        key_ptr(forces_host), key_ptr(virial_host), key_ptr(c->d_hpos),
        (unsigned long long)de_maxcnt(c, c->K)};
    // pageable host memory is neither mapped nor capturable: plain copies (a
    // key that matches the captured graph was checked when it was captured)
    const bool replay = c->ghost.exec && c->ghost.key == key;
    if (replay ||
        (pinned_or_null(pos_host) && pinned_or_null(energy_host) && pinned_or_null(forces_host) &&
         pinned_or_null(virial_host) && mapped()))
      rc = graph_run(c, c->ghost, key, s, run_mapped);
    else
      rc = run(s);
  }
  if (rc) return rc;
  SNAP_CUDA(c, cudaStreamSynchronize(s));
  return check_flags(c);
}

long long snap_get_buffer(snap_ctx* c, int which, void* dst, size_t bytes) {
  if (!c) return SNAP_ERR_ARG;
  const long n = c->last_n, K = c->last_K, H = c->tab.H;
  if (n == 0) return 0;
  SNAP_CUDA(c, cudaDeviceSynchronize());
  auto copy = [&](const void* src, size_t size) -> long long {
    if (dst) {
      const cudaError_t e = cudaMemcpy(dst, src, std::min(size, bytes), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return fail(c, SNAP_ERR_CUDA, cudaGetErrorString(e));
    }
    return (long long)size;
  };
  switch (which) {
    case SNAP_BUF_NBR_CNT: return copy(c->d_cnt, sizeof(int) * n);
    case SNAP_BUF_NBR_IDX: return copy(c->d_nbr, sizeof(int) * n * K);
    case SNAP_BUF_NBR_IMG: return copy(c->d_img, 3 * n * K);
    case SNAP_BUF_NBR_REV: return copy(c->d_rev, sizeof(int) * n * K);
    case SNAP_BUF_RIJ: return copy(c->d_rij, sizeof(double) * 3 * n * K);
    case SNAP_BUF_DEDR: return copy(c->d_dedr, sizeof(double) * 3 * n * K);
    case SNAP_BUF_ULISTTOT:
    case SNAP_BUF_YLIST: {
      const size_t size = sizeof(double) * 2 * n * H;
      if (!dst) return (long long)size;
      const long nblk = (n + 31) / 32;
      const size_t cnt = (size_t)nblk * 32 * H * 2;
      const void* src = which == SNAP_BUF_ULISTTOT ? c->d_U : c->d_Y;
      std::vector<double> hv(cnt);
      if (c->precision == SNAP_MIXED) {
        std::vector<float> f(cnt);
        SNAP_CUDA(c, cudaMemcpy(f.data(), src, cnt * sizeof(float), cudaMemcpyDeviceToHost));
        hv.assign(f.begin(), f.end());
      } else {
        SNAP_CUDA(c, cudaMemcpy(hv.data(), src, cnt * sizeof(double), cudaMemcpyDeviceToHost));
      }
      std::vector<double> out(2 * n * H);
      for (long i = 0; i < n; ++i)
        for (long e = 0; e < H; ++e) {
          const size_t q = ((size_t)(i >> 5) * H + e) * 32 + (i & 31);
          out[2 * (i * H + e)] = hv[2 * q];
          out[2 * (i * H + e) + 1] = hv[2 * q + 1];
        }
      if (which == SNAP_BUF_YLIST) {
        // compute_Y leaves the middle column below its centre (2 mb = t,
        // ma > mb) at zero: no contraction reads it.  Fill it from the
        // inversion symmetry Y[ma][mb] = (-1)^(ma+mb) conj(Y[t-ma][t-mb]).
        for (int t = 0; t <= c->tab.twojmax; t += 2) {
          const int mb = t / 2;
          for (int ma = mb + 1; ma <= t; ++ma) {
            const long e = snap_half_index(c->tab.twojmax, t, ma, mb);
            const long m = snap_half_index(c->tab.twojmax, t, t - ma, mb);
            const double sg = ((ma + mb) & 1) ? -1.0 : 1.0;
            for (long i = 0; i < n; ++i) {
              out[2 * (i * H + e)] = sg * out[2 * (i * H + m)];
              out[2 * (i * H + e) + 1] = -sg * out[2 * (i * H + m) + 1];
            }
          }
        }
      }
      std::memcpy(dst, out.data(), std::min(size, bytes));
      return (long long)size;
    }
    default: return fail(c, SNAP_ERR_ARG, "unknown buffer");
  }
}

int snap_destroy(snap_ctx* c) {
  if (!c) return SNAP_OK;
  cudaDeviceSynchronize();
  free_workspace(c);
  dfree(c->d_half_tmm);
  dfree(c->d_yrec);
  dfree(c->d_yfirst);
  dfree(c->d_yruns);
  dfree(c->d_ysched);
  dfree(c->d_brec);
  dfree(c->d_brec_cp);
  dfree(c->d_bscratch);
  dfree(c->d_bchunk_term);
  dfree(c->d_bchunk_runs);
  dfree(c->d_bcomp_chunk);
  for (auto& kv : c->bpart_cache) cudaFree(kv.second.d);
  c->bpart_cache.clear();
  dfree(c->d_root);
  dfree(c->d_hscale);
  for (auto& kv : c->yslice_cache) cudaFree(kv.second);
  c->yslice_cache.clear();
  c->d_yslice = nullptr;
  dfree(c->d_flags);
  dfree(c->d_hpos);
  dfree(c->d_hE);
  dfree(c->d_hF);
  dfree(c->d_hW);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  dfree(c->d_confs);
  dfree(c->d_ctamap);
  dfree(c->d_vatom);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gdev.reset();
  c->ghost.reset();
  if (c->gstream) cudaStreamDestroy(c->gstream);
  for (auto* pool : {&c->prof_pending, &c->prof_free})
    for (auto& ev : *pool)
      for (auto e : ev) cudaEventDestroy(e);
  delete c;
  return SNAP_OK;
}

int snap_probe_fma(int precision, int iters, double* tflops, void* stream) {
  if ((precision != SNAP_FP64 && precision != SNAP_MIXED) || iters < 8 || iters > (1 << 24) || !tflops)
    return SNAP_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SNAP_ERR_CUDA;
  void* sink = nullptr;
  if (cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) return SNAP_ERR_NOMEM;
  double flops = 0.0;
  float ms = 0.f;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = precision == SNAP_MIXED
                            ? snap::fma_probe<float>(nsm, iters, &flops, &ms, (float*)sink, s)
                            : snap::fma_probe<double>(nsm, iters, &flops, &ms, (double*)sink, s);
  cudaFree(sink);
  if (e != cudaSuccess || !(ms > 0.f)) return SNAP_ERR_CUDA;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SNAP_OK;
}

const char* snap_last_error(const snap_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

/*
 * snap_gb300.h -- C ABI of the GB300 (sm_103a) SNAP energy + force library.
 *
 * The library computes, for a periodic orthorhombic configuration of atoms of
 * one species, the SNAP per-atom energies, the forces and the virial with the
 * adjoint formulation of Gayatri et al., "Rapid Exploration of Optimization
 * Strategies on Advanced Architectures using TestSNAP and LAMMPS"
 * (arXiv:2011.12875):
 *
 *   neighbour list            (Sec. II-B, build_neighborlist)
 *   U_j = sum_k f_c u_j       (Sec. II-A Eq. u; Sec. V-A Eq. hysphrecur)
 *   Y_j = sum beta Z^j_{j1j2} (Sec. III Eq. y)
 *   dE_i/dr_ik = Y : conj(dU/dr)  (Sec. III Eq. snapforce2; fused dU + dE)
 *   E_i = beta_0 + sum beta_l B_l          (Sec. II-A Eq. snapatomenergy)
 *   F, virial from dE_i/dr_ik (Sec. III, dElist and update_forces)
 *
 * Conventions shared by all calls:
 *  - Status: every call returns 0 (SNAP_OK) or a negative snap_status; the
 *    message is in snap_last_error(ctx).  No call aborts, traps or prints.
 *  - Memory: all array arguments are owned by the caller.  Unless a call
 *    says "host", pointers are CUDA device pointers on the current device.
 *    The context owns its coefficient tables and a device workspace that
 *    grows with the largest system seen; it is released by snap_destroy.
 *  - Streams: work is enqueued on the caller's cudaStream_t (passed as
 *    void*; NULL = legacy default stream).
 *  - Units: lengths in Angstrom; energies in the units of beta.
 *  - One context must not be used from two host threads at once.
 */
#ifndef SNAP_GB300_H
#define SNAP_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snap_ctx snap_ctx;

/* Working precision of the U, Y and dU recursions.  SNAP_FP64: everything
 * in FP64.  SNAP_MIXED: the three recursions run in FP32; the Cayley-Klein
 * parameters and the per-atom energy, force and virial accumulations stay
 * in FP64. */
enum snap_precision { SNAP_FP64 = 0, SNAP_MIXED = 1 };

enum snap_status {
  SNAP_OK = 0,
  SNAP_ERR_ARG = -1,            /* invalid argument (message says which) */
  SNAP_ERR_NEIGH_OVERFLOW = -2, /* an atom has more neighbours than the capacity */
  SNAP_ERR_BOX = -3,            /* box length <= 0 or not finite, or too short against rcut */
  SNAP_ERR_CUDA = -4,           /* a CUDA call failed (message has the CUDA error) */
  SNAP_ERR_TIMEOUT = -5,        /* a bounded device wait gave up */
  SNAP_ERR_NOMEM = -6,          /* device or host allocation failed */
  SNAP_ERR_NEIGH_ASYM = -7      /* a given neighbour list is not symmetric */
};

/* Number of bispectrum components N_B for 0 <= 2j2 <= 2j1 <= 2j <= twojmax
 * (Sec. II-A): 55 at twojmax 8, 204 at 14.  Returns -1 for twojmax outside
 * 0..14. */
int snap_num_coeff(int twojmax);

/* Create a context.
 *   twojmax    : 2J, 0..14 (Sec. II-C: 2J8 and 2J14 are the paper's sizes)
 *   rcut       : cutoff radius R_cut (> rmin0)
 *   rfac0      : in (0, 1]; theta0 = rfac0*pi*(r - rmin0)/(rcut - rmin0)
 *   rmin0      : >= 0, start of the switching region
 *   switchflag : 1 = cosine switching f_c on [rmin0, rcut), 0 = f_c = 1
 *   beta       : host, 1 + N_B doubles: beta_0, then beta_l in canonical
 *                order (2j1 outer, 2j2 <= 2j1, 2j from 2j1-2j2 in steps of
 *                2 up to min(twojmax, 2j1+2j2), keeping 2j >= 2j1)
 *   precision  : SNAP_FP64 or SNAP_MIXED
 *   out        : receives the new context (NULL on failure)
 * Uploads the index, Clebsch-Gordan and coefficient tables to the current
 * device (synchronous). */
int snap_create(int twojmax, double rcut, double rfac0, double rmin0, int switchflag,
                const double* beta, int precision, snap_ctx** out);

/* Replace beta (host, 1 + N_B doubles); used by fitting loops.  Synchronous
 * with respect to the host; later snap_compute calls see the new values. */
int snap_set_beta(snap_ctx* ctx, const double* beta);

/* Capacity K of the device-built neighbour list (slots per atom, 1..64,
 * default 32).  Counts above K make snap_compute return
 * SNAP_ERR_NEIGH_OVERFLOW; snap_neigh_max() then reports the count needed. */
int snap_set_neigh_cap(snap_ctx* ctx, int cap);

/* Largest neighbour count seen by the last snap_compute (device builder). */
int snap_neigh_max(const snap_ctx* ctx);

/* Energy, forces and virial of one configuration.
 *   natoms  : N >= 0 (N = 0 returns at once)
 *   pos     : device, [N][3] doubles (x, y, z).  Any position is accepted (no
 *             wrapping into the box is needed), but the device neighbour builder
 *             pre-screens pairs in FP32 with a 0.01 A margin, so |coordinates|
 *             should stay below about 1e4 A.
 *   box     : HOST, 3 doubles: orthorhombic box lengths, periodic in x, y, z,
 *             finite and > 0.  A box so short against rcut that the device
 *             neighbour build would enumerate more than 4096 periodic images
 *             per atom (or shifts beyond 100 along one axis) returns
 *             SNAP_ERR_BOX before anything is launched (such a box holds more
 *             images of one atom within rcut than any neighbour capacity).
 *   nbr_cnt, nbr_idx, nbr_img, nbr_cap :
 *             all NULL/0 -> the library builds the list on the device
 *             (every k, image s with |r_k + s L - r_i| < rcut, k != i or
 *             s != 0).  Otherwise a caller list on the device: nbr_cnt [N]
 *             ints, nbr_idx [N][nbr_cap] ints, nbr_img [N][nbr_cap][3]
 *             signed chars (image shift s, r_ik = r_k + s L - r_i).  The
 *             list must be full (both (i,k,s) and (k,i,-s)); pairs with
 *             r >= rcut are ignored.
 *   energy  : device, [N] doubles per-atom energy E_i, or NULL
 *   forces  : device, [N][3] doubles F_i = -dE/dr_i (required)
 *   virial  : device, 6 doubles W_xx, W_yy, W_zz, W_xy, W_xz, W_yz with
 *             W_ab = -sum_{i,k} (dE_i/dr_ik)_a (r_ik)_b, or NULL
 *   stream  : cudaStream_t (void*)
 * Returns after the stream has finished the call (the status needs the
 * neighbour-overflow flag).  Results are deterministic for a given input. */
int snap_compute(snap_ctx* ctx, int natoms, const double* pos, const double* box,
                 const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                 int nbr_cap, double* energy, double* forces, double* virial,
                 void* stream);

/* snap_compute without the final wait: enqueues the whole evaluation on
 * the stream and returns.  Argument errors are returned at once; errors
 * found on the device (neighbour overflow, asymmetric list) are returned by
 * the next snap_sync.  The first call for a given N and capacity allocates
 * the workspace, so that call must not happen inside a CUDA graph capture;
 * later calls with the same sizes allocate nothing and may be captured.
 * The output buffers must stay valid until the stream reaches them. */
int snap_compute_async(snap_ctx* ctx, int natoms, const double* pos, const double* box,
                       const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                       int nbr_cap, double* energy, double* forces, double* virial,
                       void* stream);

/* Wait for `stream` and return the device status of the last
 * snap_compute_async on ctx (SNAP_OK, SNAP_ERR_NEIGH_OVERFLOW, ...). */
int snap_sync(snap_ctx* ctx, void* stream);

/* Per-stage timing with CUDA events recorded on the compute stream.
 * snap_profile(ctx, 1) starts (and zeroes) the totals, 0 stops.
 * snap_profile_read waits for the recorded events and fills, for each of
 * min(nstages, SNAP_NSTAGES) stages, the total milliseconds and the number of
 * calls timed; it returns SNAP_NSTAGES.  snap_stage_name(k) names stage k.
 * snap_launches_per_call(ctx) is the number of kernels the last compute
 * launched. */
#define SNAP_NSTAGES 5
int snap_profile(snap_ctx* ctx, int enable);
int snap_profile_read(snap_ctx* ctx, double* ms, long long* calls, int nstages);
const char* snap_stage_name(int stage);
int snap_launches_per_call(const snap_ctx* ctx);

/* Bispectrum components of every atom, the SNAP descriptors used to fit
 * beta (Sec. II-A, Eq. z): B[i][l] = Re sum over the full (2j+1)^2 matrix of
 * Z^j_{j1j2} : conj(U_j) for the canonical (2j1, 2j2, 2j) of component l
 * (order as for beta, without beta_0).  Arguments as snap_compute; B is a
 * device array [N][N_B] of doubles (computed in the context's working
 * precision).  Returns after the stream has finished. */
int snap_compute_bispectrum(snap_ctx* ctx, int natoms, const double* pos, const double* box,
                            const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                            int nbr_cap, double* B, void* stream);

/* snap_compute_bispectrum without the final wait, as snap_compute_async:
 * argument errors at once, device-side errors from the next snap_sync; the
 * first call for a given N and capacity allocates (not inside a capture). */
int snap_compute_bispectrum_async(snap_ctx* ctx, int natoms, const double* pos, const double* box,
                                  const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                                  int nbr_cap, double* B, void* stream);

/* Derivative of every atom's bispectrum along a displacement field g of the
 * atoms (forward mode, dB/dr is never stored):
 *   dB[i][l] = sum_k g_k . dB_l(i)/dr_k      (Sec. II-A, Eqs. z and dbidrk)
 * g: device [N][3] doubles; dB: device [N][N_B] doubles.  Since
 * F_k = -sum_i sum_l beta_l dB_l(i)/dr_k, the force-matching gradient is
 * d(sum_k g_k . F_k)/d(beta_l) = -sum_i dB[i][l].  Other arguments as
 * snap_compute.  Returns after the stream has finished. */
int snap_bispectrum_deriv(snap_ctx* ctx, int natoms, const double* pos, const double* box,
                          const int* nbr_cnt, const int* nbr_idx, const signed char* nbr_img,
                          int nbr_cap, const double* g, double* dB, void* stream);

/* Gradient of sum_i w_i E_i with respect to the positions, for the atoms,
 * neighbour lists and dE_i/dr_ik of the last snap_compute /
 * snap_compute_async on ctx (the adjoint backward of the per-atom energies):
 *   grad[k] = sum_i w_i dE_i/dr_k,   w: device [N], grad: device [N][3].
 * w = 1 gives -forces.  Enqueued on stream; returns SNAP_ERR_ARG if ctx has
 * no energy evaluation. */
int snap_force_weighted(snap_ctx* ctx, const double* weight, double* grad, void* stream);

/* Number of evaluations enqueued on ctx so far (lets a caller check that the
 * buffers used by snap_force_weighted are still those of its evaluation). */
long long snap_generation(const snap_ctx* ctx);

/* Many independent configurations in one evaluation: their atoms are
 * concatenated and every stage runs once over all of them (one launch per
 * stage), or, with use_graph != 0, as one CUDA graph captured on the first
 * call for this batch shape and these buffers and replayed afterwards.
 *   nconf   : number of configurations
 *   natoms  : HOST [nconf] atom counts (configuration k owns atoms
 *             start_k .. start_k + natoms[k] - 1, start_k = sum of earlier counts)
 *   boxes   : HOST [nconf][3] orthorhombic box lengths
 *   pos     : device [sum natoms][3]; energy device [sum natoms] or NULL;
 *             forces device [sum natoms][3]; virial device [nconf][6] or NULL
 * Asynchronous like snap_compute_async (status of the device-side checks
 * from snap_sync).  Results equal those of one snap_compute per
 * configuration (virial up to summation order). */
int snap_compute_batch(snap_ctx* ctx, int nconf, const int* natoms, const double* boxes,
                       const double* pos, double* energy, double* forces, double* virial,
                       int use_graph, void* stream);

/* snap_bispectrum_deriv for a batch of independent configurations (layout
 * as snap_compute_batch): dB[i][l] = sum_k g_k . dB_l(i)/dr_k for every atom
 * of every configuration (Sec. II-A, Eqs. z and dbidrk), one launch per
 * stage over all of them.  g: device [sum natoms][3]; dB: device
 * [sum natoms][N_B].  Asynchronous like snap_compute_batch (device-side
 * status from snap_sync).  The force-matching gradient of configuration k
 * is d(sum g . F)/d(beta_l) = -sum of dB over its atoms. */
int snap_bispectrum_deriv_batch(snap_ctx* ctx, int nconf, const int* natoms, const double* boxes,
                                const double* pos, const double* g, double* dB, void* stream);

/* Launch-shape tunables:
 *  col_warps (2, 4 or 8): warps per CTA of the register column-chain kernels
 *    (compute_U takes half of it, at least 2); each warp computes one atom,
 *    so this is atoms per CTA (halved where the CTA's shared memory would
 *    pass 227 KB).  The fused dE kernel plans its own CTA shape (atoms and
 *    warps per CTA) from the system size and the largest neighbour count
 *    seen, and falls back to this shape when the plan gains nothing;
 *  yi_waves (1..8): fineness of the compute_Y split; the slices per 32-atom
 *    block minimise ceil(CTAs / resident CTAs) * (1/slices + 0.02/yi_waves);
 *  yi_layout: 0 = compute_Y with a warp of 32 atoms (lanes = atoms, the
 *    block's Ulisttot staged by TMA; the paper's AoSoA layout, Sec. V-B),
 *    1 = a warp per atom (its Ulisttot staged in shared memory, lanes over
 *    output elements), the layout the paper compares it with.
 * col_warps and yi_waves change no result bit; yi_layout changes the
 * compute_Y kernel and may change rounding.  snap_autotune times every
 * combination of col_warps in {2, 4, 8} with yi_waves in {1, 2, 4} (layout 0)
 * or layout 1 on the given batch (reps timed calls each, CUDA events on
 * `stream`), then the persistent launches (SNAP_KNOB_PERSIST 1..3) at the
 * fastest shape, then the fused dE kernel's atoms per CTA (SNAP_KNOB_DE_ATOMS
 * 2, 4, ..., 32), keeps the fastest setting, and reports its median time in
 * *best_ms.  Synchronous. */
int snap_set_tuning(snap_ctx* ctx, int col_warps, int yi_waves, int yi_layout);

/* The same tunables one at a time, plus SNAP_KNOB_PERSIST (0..3, default
 * 0): bit 0 runs compute_Y, bit 1 the fused dE kernel, as a persistent
 * launch over a work queue -- a grid of as many CTAs as stay resident, each
 * taking items (a 32-atom block and output slice for compute_Y, a CTA's
 * atoms for the fused dE) from a device counter until none are left, across
 * all configurations of a batch (the paper's stage-per-kernel refactor,
 * Listing 2, with one launch per stage over many configurations).  No CTA
 * waits on another, and an item computes what the CTA it replaces would, so
 * the knob changes no result bit.  snap_autotune also searches it (after the
 * launch shapes, at the best shape).  SNAP_ERR_ARG for an unknown knob or
 * value. */
enum snap_knob {
  SNAP_KNOB_COL_WARPS = 0,
  SNAP_KNOB_YI_WAVES = 1,
  SNAP_KNOB_YI_LAYOUT = 2,
  SNAP_KNOB_PERSIST = 3,
  /* atoms per CTA of the fused dE kernel (0..256, default 0 = planned from
   * the system size and the largest neighbour count seen); with a value the
   * warp count is the best one for it.  A warp's pass count (neighbours per
   * warp) follows.  Changes no result bit. */
  SNAP_KNOB_DE_ATOMS = 4,
  /* word layout of the bispectrum kernels (B and dB): 0 (default) planned,
   * 1 sign flips on a single staged plane, 2 the conjugate plane staged
   * beside U where it fits (else as 1).  Not searched by snap_autotune (it
   * times the energy path).  The conjugate is the same value either way, so
   * the knob changes no result bit. */
  SNAP_KNOB_BI_LAYOUT = 5
};
int snap_set_knob(snap_ctx* ctx, int knob, int value);
int snap_get_knob(const snap_ctx* ctx, int knob, int* value);
int snap_get_tuning(const snap_ctx* ctx, int* col_warps, int* yi_waves, int* yi_layout);
int snap_autotune(snap_ctx* ctx, int nconf, const int* natoms, const double* boxes,
                  const double* pos, double* energy, double* forces, double* virial, int reps,
                  double* best_ms, void* stream);

/* Same as snap_compute with HOST buffers and the device neighbour builder:
 * copies pos to the device, computes, and copies energy (may be NULL),
 * forces and virial (may be NULL) back, all on the given stream.  The host
 * buffers should be pinned for full copy bandwidth. */
int snap_compute_host(snap_ctx* ctx, int natoms, const double* pos_host,
                      const double* box, double* energy_host, double* forces_host,
                      double* virial_host, void* stream);

/* Internal buffers of the last snap_compute, copied to HOST memory for
 * inspection and parity tests.  Returns the number of bytes the buffer
 * holds (copying min(bytes, that) when dst != NULL), or a negative status.
 * Layouts (N atoms, K = capacity, H = half-matrix size, see below):
 *   SNAP_BUF_NBR_CNT : int [N]
 *   SNAP_BUF_NBR_IDX : int [N][K]
 *   SNAP_BUF_NBR_IMG : signed char [N][K][3]
 *   SNAP_BUF_NBR_REV : int [N][K]   slot of the reverse pair in k's list
 *   SNAP_BUF_RIJ     : double [N][K][3]
 *   SNAP_BUF_ULISTTOT: double [N][H][2] (re, im) in half layout
 *   SNAP_BUF_YLIST   : double [N][H][2] (re, im) in half layout
 *   SNAP_BUF_DEDR    : double [N][K][3]  dE_i/dr_ik per slot
 * Half layout: for t = 2j = 0..twojmax, the columns mb = 0..floor(t/2) of
 * the (t+1)x(t+1) matrix, each column ma = 0..t; element (t, ma, mb) at
 * snap_half_index(twojmax, t, ma, mb).  The other columns follow from
 * M[t-ma][t-mb] = (-1)^(ma+mb) conj(M[ma][mb]).  On the device, Y below the
 * centre of the middle column (2 mb = t, ma > mb) is left at zero (no
 * contraction reads it); SNAP_BUF_YLIST fills it in from that symmetry. */
enum snap_buffer {
  SNAP_BUF_NBR_CNT = 0,
  SNAP_BUF_NBR_IDX = 1,
  SNAP_BUF_NBR_IMG = 2,
  SNAP_BUF_NBR_REV = 3,
  SNAP_BUF_RIJ = 4,
  SNAP_BUF_ULISTTOT = 5,
  SNAP_BUF_YLIST = 6,
  SNAP_BUF_DEDR = 7
};
long long snap_get_buffer(snap_ctx* ctx, int which, void* dst_host, size_t bytes);

/* Index of element (t, ma, mb), mb <= t/2, in the half layout; -1 if out of
 * range.  snap_half_size(twojmax) is H (155 at 8, 652 at 14). */
int snap_half_index(int twojmax, int t, int ma, int mb);
int snap_half_size(int twojmax);

/* Test hook for the timeout path (Sec. V-B's staged compute_Y has no such
 * path in the paper; the library adds one because its staging waits are
 * bounded).  With on = 1 every TMA staging step of compute_Y and of the
 * bispectrum kernels registers its bytes on its mbarrier but issues no copy,
 * so its bounded wait (1 s of the GPU's global timer) runs out with nothing in
 * flight: the kernel raises an error flag and returns, and the call returns
 * SNAP_ERR_TIMEOUT.  on = 0 (the default) restores normal operation; the
 * context stays usable.  Returns SNAP_ERR_ARG for on outside {0, 1}. */
int snap_test_stage_timeout(snap_ctx* ctx, int on);

/* compute_Y's term list for one atom, evaluated on the host in FP64 from the
 * same tables the device walks (Sec. III, Eq. y: Y = sum over the Y triples
 * of beta~ C C U_t1 U_t2, with the list's exact reductions: the two terms of
 * a t1 == t2 triple with swapped factors kept as one, the factors of each
 * output grouped, and the outputs below the centre of the middle column,
 * 2 mb = t with ma > mb, left at zero).  No GPU work: a check of the tables.
 *   precision: SNAP_FP64 or SNAP_MIXED (the table variant of that path)
 *   beta:      double [snap_num_coeff(twojmax) + 1], beta_0 first
 *   u:         double [H][2] (re, im), Ulisttot of the atom in half layout
 *   y:         double [H][2] out, Y in half layout
 * Returns SNAP_OK, or SNAP_ERR_ARG for a twojmax outside 0..14, an unknown
 * precision or a NULL pointer. */
int snap_yi_host(int twojmax, int precision, const double* beta, const double* u, double* y);

/* The bispectrum kernels' term records for one atom, walked on the host in
 * FP64 exactly as the device walks them (Sec. II-A, Eq. z: B_l = Re of the
 * triple product Z^t_{t1t2} : conj(U_t), each output element's terms summed
 * and contracted with conj(U_t) at the element, over the half layout with
 * the mirrored elements' weights folded into the coefficients, chunk
 * partials added in chunk order).  No GPU work: a check of the record words.
 *   layout: 0 the sign-flip words, 1 the conjugate-plane words
 *   u:      double [H][2] (re, im), Ulisttot of the atom in half layout (it
 *           must have the inversion symmetry of a physical Ulisttot)
 *   b:      double [snap_num_coeff(twojmax)] out
 * Returns SNAP_OK, or SNAP_ERR_ARG for a twojmax outside 0..14, a layout
 * other than 0 or 1 or a NULL pointer. */
int snap_bi_host(int twojmax, int layout, const double* u, double* b);

/* Neighbour list for callers that cannot call cudaMalloc.  Such callers
 * include host programs that hand the GPU's memory to their own allocator or
 * pool (reserved up front, so there may be no room outside it, and libraries
 * must not take memory the pool counts on), and callers on a latency-critical
 * path, where cudaMalloc may synchronise the device and stall other streams.
 * The paper has no counterpart: this is a deployment variant of the device
 * builder used by snap_compute, and it builds the same list (same order).
 * It allocates nothing: its scratch is a fixed 1 MiB device array inside the
 * library, held by every GPU that loads the library until the process exits.
 *   natoms  : 0..65536 (more returns SNAP_ERR_ARG)
 *   pos     : device, [natoms][3] doubles
 *   box     : HOST, 3 box lengths (periodic, orthorhombic), finite and > 0;
 *             SNAP_ERR_BOX also for a box so short against rcut that the
 *             build would enumerate more than 4096 periodic images per atom
 *             (or shifts beyond 100 along one axis)
 *   rcut    : cutoff, finite and > 0 (else SNAP_ERR_ARG)
 *   cap     : slots per atom, 1..64
 *   cnt, nbr, img, rij : device outputs, [natoms], [natoms][cap],
 *             [natoms][cap][3] signed char image shifts, [natoms][cap][3]
 *             doubles r_k + s L - r_i; counts above cap are truncated
 *   max_count : device, 1 int, receives the largest count (a value above cap
 *             means the list overflowed), or NULL
 *   stream  : cudaStream_t (void*); the call only enqueues work.
 * Set-up: the first valid call on a device (natoms = 0 included) looks up the
 * device address of the scratch array, so make it before any stream capture.
 * All calls share the one array and each call clears its counters; calls
 * that may overlap on the GPU (different streams, or several host threads)
 * race and must be serialised by the caller. */
int snap_neighbors_noalloc(int natoms, const double* pos, const double* box, double rcut,
                           int cap, int* cnt, int* nbr, signed char* img, double* rij,
                           int* max_count, void* stream);

/* Measured peak fused multiply-add rate of the current device in the
 * working precision of `precision` (SNAP_MIXED: FP32, SNAP_FP64: FP64), the
 * denominator against which the library's kernels, which use no tensor cores,
 * are compared (Sec. II-C, Table 1 of the paper states SNAP speeds as a
 * fraction of the nominal peak FLOP rate the same way).  Every thread of 8 CTAs per SM runs 8 independent FMA chains for
 * `iters` rounds of 4 (8 <= iters <= 2^24); one untimed and one timed launch
 * on `stream`, CUDA events.  *tflops receives 2 x FMAs / seconds / 1e12.
 * Synchronous; allocates and frees a 2 KB buffer.  SNAP_ERR_ARG for a bad
 * precision, iters or NULL tflops. */
int snap_probe_fma(int precision, int iters, double* tflops, void* stream);

/* Release the context and its device memory. */
int snap_destroy(snap_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); with ctx == NULL the
 * message of the last failed snap_create. */
const char* snap_last_error(const snap_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SNAP_GB300_H */

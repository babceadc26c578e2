/*
 * snap_oracle.c -- plain, slow FP64 reference for the SNAP energy/force path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product path never does.  It shares no
 * code, table or helper with the CUDA library.
 *
 * It follows the definitions of Gayatri et al., "Rapid Exploration of
 * Optimization Strategies on Advanced Architectures using TestSNAP and LAMMPS"
 * (arXiv:2011.12875), Sec. II-A, with full (2j+1)x(2j+1) matrices and no
 * storage or symmetry tricks:
 *
 *   Eq. (u)       U_j = w_self*I + sum_k f_c(r_ik) u_j(r_ik)
 *   Eq. (z)       Z^j_{j1j2} = U_j1 (x)^j_{j1j2} U_j2,  B_{j1j2j} = Z : U_j^*
 *   Eq. (snapatomenergy)  E_i = beta_0 + sum_l beta_l B_l
 *   Eq. (y)       Y_j = dE_i/dU_j  (the adjoint of B with respect to U)
 *   Eq. (snapforce2)      dE_i/dr_ik = sum_j Re[ Y_j : conj(dU_j/dr_ik) ]
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *  - u_j is the spin-j representation of the SU(2) element with Cayley-Klein
 *    parameters a = (z0 - i z)/r0, b = (y - i x)/r0, z0 = r cot(theta0),
 *    r0 = sqrt(r^2 + z0^2), theta0 = rfac0*pi*(r - rmin0)/(rcut - rmin0)
 *    (the 3-ball -> S^3 map the paper takes from its Ref. [Thompson2015]).
 *  - u_j is built by the layer recursion of Sec. V-A (Eq. hysphrecur): every
 *    element of u_j is a combination of two adjacent elements of u_{j-1/2}.
 *  - f_c(r) = (cos(pi (r-rmin0)/(rcut-rmin0)) + 1)/2 on [rmin0, rcut), 1 below
 *    rmin0, 0 from rcut on; switchflag = 0 gives f_c = 1.
 *  - Self contribution w_self = 1 on the diagonal of every U_j; neighbour
 *    weight 1 (single species); no constant subtracted from B.
 *  - Y is the gradient of E_i with respect to the entries of the U_j treated as
 *    independent complex numbers: Y = dE/dRe(U) + i dE/dIm(U).  The oracle
 *    obtains it from the product rule applied to the triple products of
 *    Eq. (z); no weighting factors are assumed.
 *
 * Index conventions (oracle-only): j is carried as t = 2j (0..twojmax);
 * matrix indices ma, mb run over 0..t and stand for m = ma - t/2.  A full
 * matrix block for layer t is stored row-major [ma][mb] at offset
 * sum_{t'<t} (t'+1)^2.  Complex numbers are C99 double complex.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Enumeration of the bispectrum components (Sec. II-A: 0<=2j2<=2j1<=2j<=2J,
 * j in |j1-j2| .. j1+j2).  Canonical order: t1 outer, t2 <= t1, then t from
 * t1-t2 upward in steps of 2, keeping only t >= t1.                    */

int orc_ncoeff(int twojmax) {
  int n = 0;
  for (int t1 = 0; t1 <= twojmax; ++t1)
    for (int t2 = 0; t2 <= t1; ++t2)
      for (int t = t1 - t2; t <= t1 + t2 && t <= twojmax; t += 2)
        if (t >= t1) ++n;
  return n;
}

void orc_triples(int twojmax, int* out) {
  int n = 0;
  for (int t1 = 0; t1 <= twojmax; ++t1)
    for (int t2 = 0; t2 <= t1; ++t2)
      for (int t = t1 - t2; t <= t1 + t2 && t <= twojmax; t += 2)
        if (t >= t1) {
          out[3 * n + 0] = t1;
          out[3 * n + 1] = t2;
          out[3 * n + 2] = t;
          ++n;
        }
}

int orc_full_size(int twojmax) {
  int n = 0;
  for (int t = 0; t <= twojmax; ++t) n += (t + 1) * (t + 1);
  return n;
}

static int full_base(int t) {
  int n = 0;
  for (int s = 0; s < t; ++s) n += (s + 1) * (s + 1);
  return n;
}

/* ------------------------------------------------------------------ */
/* Clebsch-Gordan coefficient <j1 m1 j2 m2 | j m> by Racah's closed form.
 * Arguments are doubled: t1 = 2 j1, m1x2 = 2 m1, etc.                  */

static double fact(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= (double)k;
  return f;
}

double orc_cg(int t1, int m1x2, int t2, int m2x2, int t, int mx2) {
  if (m1x2 + m2x2 != mx2) return 0.0;
  if (t < abs(t1 - t2) || t > t1 + t2 || ((t1 + t2 + t) & 1)) return 0.0;
  if (abs(m1x2) > t1 || abs(m2x2) > t2 || abs(mx2) > t) return 0.0;
  if (((t1 + m1x2) & 1) || ((t2 + m2x2) & 1) || ((t + mx2) & 1)) return 0.0;
  /* integer quantities j1+j2-j, j1-m1, ... */
  const int a = (t1 + t2 - t) / 2;  /* j1 + j2 - j */
  const int b = (t1 - t2 + t) / 2;  /* j1 - j2 + j */
  const int c = (-t1 + t2 + t) / 2; /* -j1 + j2 + j */
  const int s = (t1 + t2 + t) / 2;  /* j1 + j2 + j */
  const int j1pm1 = (t1 + m1x2) / 2, j1mm1 = (t1 - m1x2) / 2;
  const int j2pm2 = (t2 + m2x2) / 2, j2mm2 = (t2 - m2x2) / 2;
  const int jpm = (t + mx2) / 2, jmm = (t - mx2) / 2;
  double pre = sqrt((double)(t + 1) * fact(a) * fact(b) * fact(c) / fact(s + 1));
  pre *= sqrt(fact(jpm) * fact(jmm) * fact(j1pm1) * fact(j1mm1) * fact(j2pm2) *
              fact(j2mm2));
  double sum = 0.0;
  for (int k = 0; k <= s; ++k) {
    const int d1 = a - k;                  /* j1 + j2 - j - k */
    const int d2 = j1mm1 - k;              /* j1 - m1 - k */
    const int d3 = j2pm2 - k;              /* j2 + m2 - k */
    const int d4 = (t - t2 + m1x2) / 2 + k; /* j - j2 + m1 + k */
    const int d5 = (t - t1 - m2x2) / 2 + k; /* j - j1 - m2 + k */
    if (d1 < 0 || d2 < 0 || d3 < 0 || d4 < 0 || d5 < 0) continue;
    const double term =
        1.0 / (fact(k) * fact(d1) * fact(d2) * fact(d3) * fact(d4) * fact(d5));
    sum += (k & 1) ? -term : term;
  }
  return pre * sum;
}

/* ------------------------------------------------------------------ */
/* Cayley-Klein parameters of one neighbour vector and their derivatives. */

typedef struct {
  cplx a, b;        /* Cayley-Klein parameters */
  cplx da[3], db[3];/* d a / d r_d, d b / d r_d */
  double fc;        /* switching function */
  double dfc[3];    /* d f_c / d r_d */
} pair_geom;

static void ck_params(double x, double y, double z, double rcut, double rfac0,
                      double rmin0, int switchflag, pair_geom* g) {
  const double rv[3] = {x, y, z};
  const double r = sqrt(x * x + y * y + z * z);
  const double span = rcut - rmin0;
  const double theta0 = rfac0 * M_PI * (r - rmin0) / span;
  const double dtheta0 = rfac0 * M_PI / span; /* d theta0 / d r */
  const double z0 = r * cos(theta0) / sin(theta0);
  /* d z0 / d r = cot(theta0) - r * dtheta0 / sin^2(theta0) */
  const double dz0 = cos(theta0) / sin(theta0) -
                     r * dtheta0 / (sin(theta0) * sin(theta0));
  const double r0 = sqrt(r * r + z0 * z0);
  g->a = (z0 - I * z) / r0;
  g->b = (y - I * x) / r0;
  for (int d = 0; d < 3; ++d) {
    const double ud = rv[d] / r;            /* d r / d r_d */
    const double dz0d = dz0 * ud;           /* d z0 / d r_d */
    const double dr0d = (r * ud + z0 * dz0d) / r0;
    /* d/d r_d of (z0 - i z) and of (y - i x) */
    const cplx dnum_a = dz0d - I * (d == 2 ? 1.0 : 0.0);
    const cplx dnum_b = (d == 1 ? 1.0 : 0.0) - I * (d == 0 ? 1.0 : 0.0);
    g->da[d] = dnum_a / r0 - g->a * dr0d / r0;
    g->db[d] = dnum_b / r0 - g->b * dr0d / r0;
  }
  double fc = 1.0, dfc_dr = 0.0;
  if (switchflag) {
    if (r >= rcut) {
      fc = 0.0;
      dfc_dr = 0.0;
    } else if (r > rmin0) {
      const double w = M_PI * (r - rmin0) / span;
      fc = 0.5 * (cos(w) + 1.0);
      dfc_dr = -0.5 * M_PI / span * sin(w);
    }
  }
  g->fc = fc;
  for (int d = 0; d < 3; ++d) g->dfc[d] = dfc_dr * rv[d] / r;
}

/* ------------------------------------------------------------------ */
/* Hyperspherical harmonics of one neighbour: u_t for t = 0..twojmax, full
 * matrices, by the layer recursion (Eq. hysphrecur):
 *   u_t[ma][mb] = sqrt((t-ma)/(t-mb)) conj(a) u_{t-1}[ma][mb]
 *               - sqrt(ma/(t-mb))     conj(b) u_{t-1}[ma-1][mb],  mb < t,
 * and the last column from the inversion symmetry
 *   u_t[t-ma][t-mb] = (-1)^(ma+mb) conj(u_t[ma][mb]).
 * With du != NULL it also differentiates the recursion along the three
 * Cartesian directions (du has 3 blocks of the full size).             */

static void ulist_one(int twojmax, const pair_geom* g, cplx* u, cplx* du) {
  const int nfull = orc_full_size(twojmax);
  memset(u, 0, sizeof(cplx) * nfull);
  if (du) memset(du, 0, sizeof(cplx) * 3 * nfull);
  u[0] = 1.0;
  const cplx ca = conj(g->a), cb = conj(g->b);
  for (int t = 1; t <= twojmax; ++t) {
    const int bt = full_base(t), bp = full_base(t - 1);
    for (int mb = 0; mb < t; ++mb) {
      for (int ma = 0; ma <= t; ++ma) {
        cplx v = 0.0;
        if (ma < t) v += sqrt((double)(t - ma) / (t - mb)) * ca * u[bp + ma * t + mb];
        if (ma > 0) v -= sqrt((double)ma / (t - mb)) * cb * u[bp + (ma - 1) * t + mb];
        u[bt + ma * (t + 1) + mb] = v;
        if (du) {
          for (int d = 0; d < 3; ++d) {
            cplx* dd = du + d * nfull;
            const cplx cda = conj(g->da[d]), cdb = conj(g->db[d]);
            cplx w = 0.0;
            if (ma < t)
              w += sqrt((double)(t - ma) / (t - mb)) *
                   (cda * u[bp + ma * t + mb] + ca * dd[bp + ma * t + mb]);
            if (ma > 0)
              w -= sqrt((double)ma / (t - mb)) *
                   (cdb * u[bp + (ma - 1) * t + mb] + cb * dd[bp + (ma - 1) * t + mb]);
            dd[bt + ma * (t + 1) + mb] = w;
          }
        }
      }
    }
    /* last column mb = t from column 0: u[ma][t] = (-1)^(t-ma) conj(u[t-ma][0]) */
    for (int ma = 0; ma <= t; ++ma) {
      const double sgn = ((t - ma) & 1) ? -1.0 : 1.0;
      u[bt + ma * (t + 1) + t] = sgn * conj(u[bt + (t - ma) * (t + 1) + 0]);
      if (du)
        for (int d = 0; d < 3; ++d) {
          cplx* dd = du + d * nfull;
          dd[bt + ma * (t + 1) + t] = sgn * conj(dd[bt + (t - ma) * (t + 1) + 0]);
        }
    }
  }
}

/* Exported for the pins: u_t (and du_t/dr) of a single neighbour vector.
 * u_out: 2*nfull doubles (re, im interleaved); du_out: 3*2*nfull or NULL. */
void orc_ulist_pair(int twojmax, double x, double y, double z, double rcut,
                    double rfac0, double rmin0, int switchflag, double* u_out,
                    double* du_out, double* geom_out) {
  pair_geom g;
  ck_params(x, y, z, rcut, rfac0, rmin0, switchflag, &g);
  const int nfull = orc_full_size(twojmax);
  cplx* u = (cplx*)malloc(sizeof(cplx) * nfull);
  cplx* du = du_out ? (cplx*)malloc(sizeof(cplx) * 3 * nfull) : NULL;
  ulist_one(twojmax, &g, u, du);
  memcpy(u_out, u, sizeof(cplx) * nfull);
  if (du_out) memcpy(du_out, du, sizeof(cplx) * 3 * nfull);
  if (geom_out) {
    /* a, b, fc, dfc[3], da[3], db[3] as re/im pairs */
    geom_out[0] = creal(g.a); geom_out[1] = cimag(g.a);
    geom_out[2] = creal(g.b); geom_out[3] = cimag(g.b);
    geom_out[4] = g.fc;
    for (int d = 0; d < 3; ++d) geom_out[5 + d] = g.dfc[d];
    for (int d = 0; d < 3; ++d) {
      geom_out[8 + 2 * d] = creal(g.da[d]); geom_out[9 + 2 * d] = cimag(g.da[d]);
      geom_out[14 + 2 * d] = creal(g.db[d]); geom_out[15 + 2 * d] = cimag(g.db[d]);
    }
  }
  free(u);
  free(du);
}

/* ------------------------------------------------------------------ */
/* Neighbour list by brute force over all atoms and all periodic images
 * (orthorhombic box, periodic in x, y, z).  Pair (i, k, s) is kept when
 * |r_k + s*L - r_i| < rcut and (k != i or s != 0).  Pairs come out grouped
 * by i.  Returns the number of pairs, or -(needed) when maxpairs is short. */

int orc_build_neighbors(int n, const double* pos, const double* box, double rcut,
                        int maxpairs, int* pi, int* pk, int* pimg, double* rij) {
  int S[3];
  for (int d = 0; d < 3; ++d) S[d] = (int)ceil(rcut / box[d]) + 1;
  int np = 0;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k)
      for (int sx = -S[0]; sx <= S[0]; ++sx)
        for (int sy = -S[1]; sy <= S[1]; ++sy)
          for (int sz = -S[2]; sz <= S[2]; ++sz) {
            if (k == i && sx == 0 && sy == 0 && sz == 0) continue;
            const double dx = pos[3 * k + 0] + sx * box[0] - pos[3 * i + 0];
            const double dy = pos[3 * k + 1] + sy * box[1] - pos[3 * i + 1];
            const double dz = pos[3 * k + 2] + sz * box[2] - pos[3 * i + 2];
            if (dx * dx + dy * dy + dz * dz < rcut * rcut) {
              if (np < maxpairs) {
                pi[np] = i;
                pk[np] = k;
                pimg[3 * np + 0] = sx;
                pimg[3 * np + 1] = sy;
                pimg[3 * np + 2] = sz;
                rij[3 * np + 0] = dx;
                rij[3 * np + 1] = dy;
                rij[3 * np + 2] = dz;
              }
              ++np;
            }
          }
  return np <= maxpairs ? np : -np;
}

/* ------------------------------------------------------------------ */
/* Per-atom quantities: Ulisttot, B, E and Y.                           */

typedef struct {
  int twojmax, nfull, ncoeff;
  double rcut, rfac0, rmin0, wself;
  int switchflag;
  const double* beta; /* beta0, beta_1..beta_ncoeff */
  int* triples;
} orc_params;

/* U_t = wself*I + sum over the atom's neighbours of f_c u_t (Eq. u). */
static void ulisttot_atom(const orc_params* p, int npair_i, const double* rij_i,
                          cplx* utot) {
  const int nfull = p->nfull;
  memset(utot, 0, sizeof(cplx) * nfull);
  for (int t = 0; t <= p->twojmax; ++t) {
    const int bt = full_base(t);
    for (int ma = 0; ma <= t; ++ma) utot[bt + ma * (t + 1) + ma] = p->wself;
  }
  cplx* u = (cplx*)malloc(sizeof(cplx) * nfull);
  for (int q = 0; q < npair_i; ++q) {
    pair_geom g;
    ck_params(rij_i[3 * q], rij_i[3 * q + 1], rij_i[3 * q + 2], p->rcut, p->rfac0,
              p->rmin0, p->switchflag, &g);
    ulist_one(p->twojmax, &g, u, NULL);
    for (int e = 0; e < nfull; ++e) utot[e] += g.fc * u[e];
  }
  free(u);
}

/* For one canonical triple (t1, t2, t) visit every term
 *   c * U_t1[ma1][mb1] * U_t2[ma2][mb2] * conj(U_t[ma][mb]),
 *   c = <j1 m1 j2 m2|j m> <j1 m1' j2 m2'|j m'>, m = m1 + m2, m' = m1' + m2',
 * accumulating B = Re(sum), and, if Y != NULL, the product-rule gradient
 * scaled by beta_l into Y.                                             */
static double triple_product(const orc_params* p, int t1, int t2, int t,
                             const cplx* U, double beta_l, cplx* Y) {
  (void)p;
  const int b1 = full_base(t1), b2 = full_base(t2), b3 = full_base(t);
  /* cg[x1][x2] = <j1 m1 j2 m2 | j m1+m2>, m1 = x1 - t1/2, m2 = x2 - t2/2 */
  double* cg = (double*)malloc(sizeof(double) * (t1 + 1) * (t2 + 1));
  for (int x1 = 0; x1 <= t1; ++x1)
    for (int x2 = 0; x2 <= t2; ++x2) {
      const int m1 = 2 * x1 - t1, m2 = 2 * x2 - t2;
      cg[x1 * (t2 + 1) + x2] = orc_cg(t1, m1, t2, m2, t, m1 + m2);
    }
  double B = 0.0;
  for (int ma1 = 0; ma1 <= t1; ++ma1)
    for (int ma2 = 0; ma2 <= t2; ++ma2) {
      const int m = (2 * ma1 - t1) + (2 * ma2 - t2);
      if (m < -t || m > t) continue;
      const int ma = (m + t) / 2;
      const double ca = cg[ma1 * (t2 + 1) + ma2];
      if (ca == 0.0) continue;
      for (int mb1 = 0; mb1 <= t1; ++mb1)
        for (int mb2 = 0; mb2 <= t2; ++mb2) {
          const int nn = (2 * mb1 - t1) + (2 * mb2 - t2);
          if (nn < -t || nn > t) continue;
          const int mb = (nn + t) / 2;
          const double cb = cg[mb1 * (t2 + 1) + mb2];
          if (cb == 0.0) continue;
          const double c = ca * cb;
          const cplx u1 = U[b1 + ma1 * (t1 + 1) + mb1];
          const cplx u2 = U[b2 + ma2 * (t2 + 1) + mb2];
          const cplx u3 = U[b3 + ma * (t + 1) + mb];
          B += creal(c * u1 * u2 * conj(u3));
          if (Y) {
            Y[b3 + ma * (t + 1) + mb] += beta_l * c * u1 * u2;
            Y[b1 + ma1 * (t1 + 1) + mb1] += beta_l * c * conj(u2) * u3;
            Y[b2 + ma2 * (t2 + 1) + mb2] += beta_l * c * conj(u1) * u3;
          }
        }
    }
  free(cg);
  return B;
}

/* E_i = beta_0 + sum_l beta_l B_l (Eq. snapatomenergy) and, optionally,
 * the bispectrum B[l] and the adjoint Y = dE_i/dU (Eq. y).             */
static double energy_atom(const orc_params* p, const cplx* U, double* B, cplx* Y) {
  if (Y) memset(Y, 0, sizeof(cplx) * p->nfull);
  double E = p->beta[0];
  for (int l = 0; l < p->ncoeff; ++l) {
    const int* tr = p->triples + 3 * l;
    const double bl = triple_product(p, tr[0], tr[1], tr[2], U, p->beta[1 + l], Y);
    if (B) B[l] = bl;
    E += p->beta[1 + l] * bl;
  }
  return E;
}

/* dE_i/dr_ik for one neighbour (Eq. snapforce2):
 *   sum_t sum_{ma,mb} Re[ conj(Y_t) * d(f_c u_t)/dr ]                   */
static void dedr_pair(const orc_params* p, const double* r, const cplx* Y,
                      double* out) {
  const int nfull = p->nfull;
  pair_geom g;
  ck_params(r[0], r[1], r[2], p->rcut, p->rfac0, p->rmin0, p->switchflag, &g);
  cplx* u = (cplx*)malloc(sizeof(cplx) * nfull);
  cplx* du = (cplx*)malloc(sizeof(cplx) * 3 * nfull);
  ulist_one(p->twojmax, &g, u, du);
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
    for (int e = 0; e < nfull; ++e) {
      const cplx dU = g.dfc[d] * u[e] + g.fc * du[d * nfull + e];
      s += creal(conj(Y[e]) * dU);
    }
    out[d] = s;
  }
  free(u);
  free(du);
}

/* ------------------------------------------------------------------ */
/* Whole evaluation.  The pair list (pi, pk, rij) must be grouped by pi.
 * need[i] != 0 selects the centre atoms whose E, B, U, Y and whose pairs'
 * dedr are computed (need == NULL: all atoms).  F and W are filled only
 * when need == NULL.  Outputs may be NULL.  Returns 0, or -1 on bad input.
 *   beta : 1 + ncoeff doubles (beta_0 first)
 *   Uout, Yout : n * nfull complex (re, im interleaved)
 *   Bout : n * ncoeff;  dedr : npairs * 3;  F : n * 3;
 *   W : 6 (xx, yy, zz, xy, xz, yz), W_ab = -sum_pairs dedr_a r_b       */

int orc_compute(int twojmax, double rcut, double rfac0, double rmin0,
                int switchflag, double wself, const double* beta, int n,
                int npairs, const int* pi, const int* pk, const double* rij,
                const unsigned char* need, double* E, double* Bout,
                double* Uout, double* Yout, double* dedr, double* F, double* W) {
  (void)pk;
  if (twojmax < 0 || n < 0 || npairs < 0) return -1;
  orc_params p;
  p.twojmax = twojmax;
  p.nfull = orc_full_size(twojmax);
  p.ncoeff = orc_ncoeff(twojmax);
  p.rcut = rcut;
  p.rfac0 = rfac0;
  p.rmin0 = rmin0;
  p.switchflag = switchflag;
  p.wself = wself;
  p.beta = beta;
  p.triples = (int*)malloc(sizeof(int) * 3 * (p.ncoeff > 0 ? p.ncoeff : 1));
  orc_triples(twojmax, p.triples);

  /* first pair of every atom (pairs grouped by centre atom) */
  int* first = (int*)malloc(sizeof(int) * (n + 1));
  int* count = (int*)calloc(n > 0 ? n : 1, sizeof(int));
  for (int q = 0; q < npairs; ++q) {
    if (pi[q] < 0 || pi[q] >= n) { free(first); free(count); free(p.triples); return -1; }
    if (q > 0 && pi[q] < pi[q - 1]) { free(first); free(count); free(p.triples); return -1; }
    count[pi[q]]++;
  }
  first[0] = 0;
  for (int i = 0; i < n; ++i) first[i + 1] = first[i] + count[i];

  const int nfull = p.nfull;
  cplx* Yall = (cplx*)calloc((size_t)(n > 0 ? n : 1) * nfull, sizeof(cplx));

#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; ++i) {
    if (need && !need[i]) continue;
    cplx* U = (cplx*)malloc(sizeof(cplx) * nfull);
    cplx* Y = Yall + (size_t)i * nfull;
    ulisttot_atom(&p, count[i], rij + 3 * (size_t)first[i], U);
    const double Ei = energy_atom(&p, U, Bout ? Bout + (size_t)i * p.ncoeff : NULL, Y);
    if (E) E[i] = Ei;
    if (Uout) memcpy(Uout + 2 * (size_t)i * nfull, U, sizeof(cplx) * nfull);
    if (Yout) memcpy(Yout + 2 * (size_t)i * nfull, Y, sizeof(cplx) * nfull);
    free(U);
  }

#pragma omp parallel for schedule(dynamic, 16)
  for (int q = 0; q < npairs; ++q) {
    const int i = pi[q];
    if (need && !need[i]) continue;
    double o[3];
    dedr_pair(&p, rij + 3 * (size_t)q, Yall + (size_t)i * nfull, o);
    if (dedr) for (int d = 0; d < 3; ++d) dedr[3 * (size_t)q + d] = o[d];
  }

  if (!need && (F || W)) {
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    double w[6] = {0, 0, 0, 0, 0, 0};
    double* o = (double*)malloc(sizeof(double) * 3 * (size_t)(npairs > 0 ? npairs : 1));
    if (dedr) memcpy(o, dedr, sizeof(double) * 3 * (size_t)npairs);
    else
      for (int q = 0; q < npairs; ++q)
        dedr_pair(&p, rij + 3 * (size_t)q, Yall + (size_t)pi[q] * nfull, o + 3 * (size_t)q);
    for (int q = 0; q < npairs; ++q) {
      const double* g = o + 3 * (size_t)q;
      const double* r = rij + 3 * (size_t)q;
      if (F)
        for (int d = 0; d < 3; ++d) {
          F[3 * (size_t)pi[q] + d] += g[d]; /* -dE_i/dr_i  = +dE_i/dr_ik */
          F[3 * (size_t)pk[q] + d] -= g[d]; /* -dE_i/dr_k  = -dE_i/dr_ik */
        }
      w[0] -= g[0] * r[0];
      w[1] -= g[1] * r[1];
      w[2] -= g[2] * r[2];
      w[3] -= g[0] * r[1];
      w[4] -= g[0] * r[2];
      w[5] -= g[1] * r[2];
    }
    if (W) memcpy(W, w, sizeof(w));
    free(o);
  }

  free(Yall);
  free(first);
  free(count);
  free(p.triples);
  return 0;
}

/* Energy of a single atom from an explicit U (full matrices, re/im
 * interleaved); used by the pins to differentiate E with respect to U. */
double orc_energy_from_u(int twojmax, const double* beta, const double* Uin,
                         double* Yout) {
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.twojmax = twojmax;
  p.nfull = orc_full_size(twojmax);
  p.ncoeff = orc_ncoeff(twojmax);
  p.beta = beta;
  p.triples = (int*)malloc(sizeof(int) * 3 * (p.ncoeff > 0 ? p.ncoeff : 1));
  orc_triples(twojmax, p.triples);
  cplx* U = (cplx*)malloc(sizeof(cplx) * p.nfull);
  memcpy(U, Uin, sizeof(cplx) * p.nfull);
  cplx* Y = Yout ? (cplx*)malloc(sizeof(cplx) * p.nfull) : NULL;
  const double E = energy_atom(&p, U, NULL, Y);
  if (Yout) memcpy(Yout, Y, sizeof(cplx) * p.nfull);
  free(Y);
  free(U);
  free(p.triples);
  return E;
}

/* ------------------------------------------------------------------ */
/* Floating-point work of the oracle's own (unreduced) evaluation of one
 * step, counted by walking the loops of ulist_one, ulisttot_atom,
 * triple_product and dedr_pair with the same bounds and the same
 * zero-coefficient skips, without their arithmetic.  Convention: a real add
 * or multiply is 1, a real-by-complex scale 2, a complex add 2, a complex
 * multiply 6; a square root or a division is 1; sign changes and
 * conjugations are free.
 *   out[0]: compute_U of one neighbour pair (recursion, f_c u added to U)
 *   out[1]: B and the product-rule Y of one atom (every canonical triple)
 *   out[2]: dU and dE/dr of one neighbour pair (recursion with its three
 *           Cartesian derivatives, then the contraction with Y)
 * The per-atom energy, forces and virial sums are not counted.        */
void orc_flops(int twojmax, double* out) {
  double u_pair = 0.0, y_atom = 0.0, de_pair = 0.0;
  /* ulist_one: a term is sqrt of a ratio (2), its scale of conj(a) (2),
   * the complex product (6) and the accumulation (2); with du, per
   * direction two complex products and their sum (14), the scale (2) and
   * the accumulation (2) */
  double terms = 0.0;
  for (int t = 1; t <= twojmax; ++t)
    for (int mb = 0; mb < t; ++mb)
      for (int ma = 0; ma <= t; ++ma) terms += (ma < t) + (ma > 0);
  const int nfull = orc_full_size(twojmax);
  u_pair = 12.0 * terms + 4.0 * nfull;             /* + f_c u added to U_tot */
  de_pair = 12.0 * terms + 3.0 * 18.0 * terms +     /* u and du */
            3.0 * 10.0 * nfull;                     /* dU (6) and Re conj(Y) dU (4) */
  /* triple_product: per nonzero term c = ca cb (1), c u1 (2), (c u1) u2
   * (6), times conj(u3) (6), real part added (1); the Y update of u3:
   * beta c (1), its scale of u1 u2 (2 + 6), accumulation (2); of u1 and of
   * u2: a complex product (6), the scale (2), accumulation (2) each */
  for (int t1 = 0; t1 <= twojmax; ++t1)
    for (int t2 = 0; t2 <= t1; ++t2)
      for (int t = t1 - t2; t <= t1 + t2 && t <= twojmax; t += 2) {
        if (t < t1) continue;
        for (int ma1 = 0; ma1 <= t1; ++ma1)
          for (int ma2 = 0; ma2 <= t2; ++ma2) {
            const int m = (2 * ma1 - t1) + (2 * ma2 - t2);
            if (m < -t || m > t) continue;
            if (orc_cg(t1, 2 * ma1 - t1, t2, 2 * ma2 - t2, t, m) == 0.0) continue;
            for (int mb1 = 0; mb1 <= t1; ++mb1)
              for (int mb2 = 0; mb2 <= t2; ++mb2) {
                const int nn = (2 * mb1 - t1) + (2 * mb2 - t2);
                if (nn < -t || nn > t) continue;
                if (orc_cg(t1, 2 * mb1 - t1, t2, 2 * mb2 - t2, t, nn) == 0.0) continue;
                y_atom += 16.0 + 11.0 + 2.0 * 10.0;
              }
          }
      }
  out[0] = u_pair;
  out[1] = y_atom;
  out[2] = de_pair;
}

// snap_tables.cpp -- host-side index and coefficient tables of the library.
//
//  * bispectrum enumeration 0 <= 2j2 <= 2j1 <= 2j <= 2J (arXiv:2011.12875,
//    Sec. II-A) in canonical order, and the (t1 >= t2, t) triples of the
//    adjoint Y (Sec. III, Eq. y);
//  * Clebsch-Gordan coefficients, obtained here from Wigner 3j symbols
//    (Racah's sum for the 3j symbol, long double);
//  * the weighted beta of every Y triple, and the Y work list sorted by
//    output element with its balanced split into warp slices.
#include "snap_tables.h"

#include <algorithm>
#include <cmath>
#include <map>

namespace snap {

namespace {

long double lfact(int n) {
  long double f = 1.0L;
  for (int k = 2; k <= n; ++k) f *= (long double)k;
  return f;
}

// Wigner 3j symbol (j1 j2 j3; m1 m2 m3) with doubled arguments.
long double wigner3j(int tj1, int tj2, int tj3, int tm1, int tm2, int tm3) {
  if (tm1 + tm2 + tm3 != 0) return 0.0L;
  if (tj3 < std::abs(tj1 - tj2) || tj3 > tj1 + tj2 || ((tj1 + tj2 + tj3) & 1)) return 0.0L;
  if (std::abs(tm1) > tj1 || std::abs(tm2) > tj2 || std::abs(tm3) > tj3) return 0.0L;
  // integer combinations
  const int j1pj2mj3 = (tj1 + tj2 - tj3) / 2;
  const int j1mj2pj3 = (tj1 - tj2 + tj3) / 2;
  const int mj1pj2pj3 = (-tj1 + tj2 + tj3) / 2;
  const int jsum1 = (tj1 + tj2 + tj3) / 2 + 1;
  const long double tri = lfact(j1pj2mj3) * lfact(j1mj2pj3) * lfact(mj1pj2pj3) / lfact(jsum1);
  const long double mf = lfact((tj1 + tm1) / 2) * lfact((tj1 - tm1) / 2) * lfact((tj2 + tm2) / 2) *
                         lfact((tj2 - tm2) / 2) * lfact((tj3 + tm3) / 2) * lfact((tj3 - tm3) / 2);
  // k runs where all of these are >= 0
  const int x1 = (tj3 - tj2 + tm1) / 2;  // j3 - j2 + m1 + k
  const int x2 = (tj3 - tj1 - tm2) / 2;  // j3 - j1 - m2 + k
  const int y1 = j1pj2mj3;               // j1 + j2 - j3 - k
  const int y2 = (tj1 - tm1) / 2;        // j1 - m1 - k
  const int y3 = (tj2 + tm2) / 2;        // j2 + m2 - k
  const int kmin = std::max(0, std::max(-x1, -x2));
  const int kmax = std::min(y1, std::min(y2, y3));
  long double sum = 0.0L;
  for (int k = kmin; k <= kmax; ++k) {
    const long double den =
        lfact(k) * lfact(x1 + k) * lfact(x2 + k) * lfact(y1 - k) * lfact(y2 - k) * lfact(y3 - k);
    sum += ((k & 1) ? -1.0L : 1.0L) / den;
  }
  // overall phase (-1)^(j1 - j2 - m3)
  const int ph = (tj1 - tj2 - tm3) / 2;
  const long double sign = (ph & 1) ? -1.0L : 1.0L;
  return sign * std::sqrt(tri) * std::sqrt(mf) * sum;
}

}  // namespace

// <j1 m1 j2 m2 | j m> = (-1)^(j1 - j2 + m) sqrt(2j+1) (j1 j2 j; m1 m2 -m)
double clebsch_gordan(int tj1, int tm1, int tj2, int tm2, int tj, int tm) {
  if (tm1 + tm2 != tm) return 0.0;
  const long double w = wigner3j(tj1, tj2, tj, tm1, tm2, -tm);
  const int ph = (tj1 - tj2 + tm) / 2;
  const long double s = (ph & 1) ? -1.0L : 1.0L;
  return (double)(s * std::sqrt((long double)(tj + 1)) * w);
}

int count_coeff(int twojmax) {
  if (twojmax < 0 || twojmax > kMaxTwoJ) return -1;
  int n = 0;
  for (int t1 = 0; t1 <= twojmax; ++t1)
    for (int t2 = 0; t2 <= t1; ++t2)
      for (int t = t1 - t2; t <= std::min(twojmax, t1 + t2); t += 2)
        if (t >= t1) ++n;
  return n;
}

void HostTables::build(int J2) {
  twojmax = J2;
  H = half_size(J2);
  lmax = half_layer_size(J2);
  half_tmm.clear();
  for (int t = 0; t <= J2; ++t)
    for (int mb = 0; 2 * mb <= t; ++mb)
      for (int ma = 0; ma <= t; ++ma) half_tmm.push_back(pack_tmm(t, ma, mb));

  // canonical bispectrum index
  std::map<long, int> bidx;
  ncoeff = 0;
  for (int t1 = 0; t1 <= J2; ++t1)
    for (int t2 = 0; t2 <= t1; ++t2)
      for (int t = t1 - t2; t <= std::min(J2, t1 + t2); t += 2)
        if (t >= t1) bidx[(long)t1 * 10000 + t2 * 100 + t] = ncoeff++;
  auto idx_of = [&](int a, int b, int c) { return bidx.at((long)a * 10000 + b * 100 + c); };

  // Y triples (t1 >= t2, any t) with their CG blocks and beta weights.
  ztrip.clear();
  cg.clear();
  for (int t1 = 0; t1 <= J2; ++t1)
    for (int t2 = 0; t2 <= t1; ++t2)
      for (int t = t1 - t2; t <= std::min(J2, t1 + t2); t += 2) {
        ZTrip z;
        z.t1 = t1;
        z.t2 = t2;
        z.t = t;
        z.cg_off = (int)cg.size();
        for (int x1 = 0; x1 <= t1; ++x1)
          for (int x2 = 0; x2 <= t2; ++x2) {
            const int m1 = 2 * x1 - t1, m2 = 2 * x2 - t2;
            cg.push_back(std::abs(m1 + m2) <= t ? clebsch_gordan(t1, m1, t2, m2, t, m1 + m2) : 0.0);
          }
        // The derivative of E_i = sum_l beta_l B_l with respect to U_t collects,
        // for every component l whose sorted triple contains t, the Z matrix
        // built from the other two U's.  Moving the conjugate of a triple
        // product from U_t to a U of larger rank scales it by
        // (t_big + 1)/(t + 1); coinciding ranks count once per occurrence.
        if (t >= t1) {  // t is the largest rank: component (t1, t2, t)
          z.bidx = idx_of(t1, t2, t);
          z.fac = (t1 == t) ? ((t2 == t) ? 3.0 : 2.0) : 1.0;
        } else if (t >= t2) {  // t1 > t >= t2: component (t, t2, t1)
          z.bidx = idx_of(t, t2, t1);
          z.fac = ((t2 == t) ? 2.0 : 1.0) * (double)(t1 + 1) / (double)(t + 1);
        } else {  // t < t2 <= t1: component (t2, t, t1)
          z.bidx = idx_of(t2, t, t1);
          z.fac = (double)(t1 + 1) / (double)(t + 1);
        }
        ztrip.push_back(z);
      }

  // Padded Clebsch-Gordan blocks for compute_Y: rows x1 = 0..t1, columns
  // x2 = -kYiRW .. t2 + kYiRW (zeros outside 0..t2), so the kernel reads the
  // coefficients of kYiRW consecutive outputs without bounds checks.
  cgpad.clear();
  for (ZTrip& z : ztrip) {
    z.cgpad_off = (int)cgpad.size();
    const int w2 = z.t2 + 1 + 2 * kYiRW;
    for (int x1 = 0; x1 <= z.t1; ++x1)
      for (int c = 0; c < w2; ++c) {
        const int x2 = c - kYiRW;
        cgpad.push_back((x2 >= 0 && x2 <= z.t2) ? cg[z.cg_off + x1 * (z.t2 + 1) + x2] : 0.0);
      }
  }

  // Work list: for every triple and every half column mb <= t/2, groups of
  // kYiRW consecutive rows ma0..ma0+kYiRW-1, sorted by output group (stable in
  // triple order), so all contributions to one group are adjacent.
  jobs.clear();
  cost.clear();
  struct Tmp {
    int out, trip, ma0, mb, nr;
  };
  std::vector<Tmp> tmp;
  for (int q = 0; q < (int)ztrip.size(); ++q) {
    const ZTrip& z = ztrip[q];
    for (int mb = 0; 2 * mb <= z.t; ++mb)
      for (int ma0 = 0; ma0 <= z.t; ma0 += kYiRW)
        tmp.push_back({half_base(z.t) + mb * (z.t + 1) + ma0, q, ma0, mb,
                       std::min(kYiRW, z.t + 1 - ma0)});
  }
  std::stable_sort(tmp.begin(), tmp.end(), [](const Tmp& x, const Tmp& y) { return x.out < y.out; });
  for (const Tmp& w : tmp) {
    const ZTrip& z = ztrip[w.trip];
    YJob j;
    j.x = z.t1 | (z.t2 << 4) | (z.t << 8) | (w.ma0 << 12) | (w.mb << 16) | (w.nr << 20);
    j.y = half_base(z.t1) | (half_base(z.t2) << 16);
    j.z = z.cgpad_off;
    j.w = w.trip | (w.out << 16);
    jobs.push_back(j);
    const int dl = (z.t1 + z.t2 - z.t) / 2;
    const int na = std::min(z.t1, w.ma0 + w.nr - 1 + dl) - std::max(0, w.ma0 + dl - z.t2) + 1;
    const int nb = std::min(z.t1, w.mb + dl) - std::max(0, w.mb + dl - z.t2) + 1;
    cost.push_back(std::max(nb, 0) * (std::max(na, 0) * kYiRW + 8) + 16);
  }

  rootpq.assign(kRootDim * kRootDim, 0.0);
  for (int p = 0; p < kRootDim; ++p)
    for (int q = 1; q < kRootDim; ++q) rootpq[p * kRootDim + q] = std::sqrt((double)p / (double)q);
}

std::vector<double> HostTables::beta_weights(const double* beta) const {
  std::vector<double> w(ztrip.size());
  for (size_t q = 0; q < ztrip.size(); ++q) w[q] = ztrip[q].fac * beta[1 + ztrip[q].bidx];
  return w;
}

std::vector<int> HostTables::slices(int nslices) const {
  // contiguous runs of work items, cut only between output elements, with
  // about equal total cost
  long total = 0;
  for (int c : cost) total += c;
  std::vector<int> b;
  b.push_back(0);
  long acc = 0;
  int k = 1;
  const int n = (int)jobs.size();
  for (int q = 0; q < n; ++q) {
    acc += cost[q];
    const bool boundary = (q + 1 == n) || ((jobs[q + 1].w >> 16) != (jobs[q].w >> 16));
    if (boundary && k < nslices && acc * nslices >= total * k) {
      b.push_back(q + 1);
      ++k;
    }
  }
  while ((int)b.size() < nslices + 1) b.push_back(n);
  b[nslices] = n;
  return b;
}

}  // namespace snap

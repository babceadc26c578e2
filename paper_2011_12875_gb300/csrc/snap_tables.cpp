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
#include <array>
#include <cmath>
#include <map>
#include <unordered_map>

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

namespace {

// Factor order of the terms [first, end) of one output.  A term's product is
// symmetric in its two factors, and compute_Y groups the terms of an output
// by their first factor (Y += U[e1] * sum_k c_k U[e2,k]), so fewer distinct
// first factors mean fewer groups.  Choosing them is a vertex cover of the
// graph whose vertices are the stored elements (index, conjugation) and
// whose edges are the terms; the greedy cover takes, again and again, the
// element with the most terms not yet covered (ties: the larger element) and
// makes it the first factor of those terms.
void orient_by_cover(std::vector<unsigned>& terms, size_t first) {
  const size_t n = terms.size() - first;
  if (n < 2) return;
  auto e1 = [](unsigned w) { return (w & 1023u) << 1 | ((w >> 20) & 1u); };
  auto e2 = [](unsigned w) { return ((w >> 10) & 1023u) << 1 | ((w >> 21) & 1u); };
  std::unordered_map<unsigned, std::vector<size_t>> inc;  // element -> its terms
  for (size_t k = first; k < terms.size(); ++k) {
    const unsigned a = e1(terms[k]), b = e2(terms[k]);
    inc[a].push_back(k);
    if (b != a) inc[b].push_back(k);
  }
  std::unordered_map<unsigned, int> deg;
  std::vector<std::pair<int, unsigned>> heap;  // (uncovered terms, element)
  for (const auto& kv : inc) {
    deg[kv.first] = (int)kv.second.size();
    heap.push_back({(int)kv.second.size(), kv.first});
  }
  std::make_heap(heap.begin(), heap.end());
  std::vector<char> covered(n, 0);
  while (!heap.empty()) {
    std::pop_heap(heap.begin(), heap.end());
    const auto top = heap.back();
    heap.pop_back();
    const unsigned v = top.second;
    if (top.first != deg[v]) {  // stale entry: push the current count back
      if (deg[v] > 0) {
        heap.push_back({deg[v], v});
        std::push_heap(heap.begin(), heap.end());
      }
      continue;
    }
    if (top.first == 0) break;
    for (size_t k : inc[v]) {
      if (covered[k - first]) continue;
      covered[k - first] = 1;
      unsigned& w = terms[k];
      const unsigned a = e1(w), b = e2(w);
      if (a != v) {  // v is the second factor: swap the two factors
        w = ((w >> 10) & 1023u) | ((w & 1023u) << 10) | (((w >> 21) & 1u) << 20) |
            (((w >> 20) & 1u) << 21) | (w & ~((1u << 22) - 1));
      }
      const unsigned o = (a == v) ? b : a;
      if (o != v) --deg[o];
    }
    deg[v] = 0;
  }
}

}  // namespace

void HostTables::build(int J2, bool size_runs) {
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

  // compute_Y term list.  For every half-layout output element (t, ma, mb)
  // of Y, in output order, every nonzero term of every triple (t1 >= t2)
  // with output rank t:
  //   Y_t[ma][mb] += betaw * C(ma1, ma2) C(mb1, mb2) U_t1[ma1][mb1] U_t2[ma2][mb2],
  // ma2 = ma + d - ma1, mb2 = mb + d - mb1, d = (t1+t2-t)/2.  An element of U
  // past the stored half columns is (-1)^(ma+mb) conj of its mirror, so each
  // term stores the two half-layout indices, two conjugation flags, and a
  // coefficient with the signs, the CG product and betaw folded in.
  terms.clear();
  term_cg.clear();
  term_trip.clear();
  term_out_first.clear();
  term_runs.clear();
  auto half_elem = [&](int tt, int xa, int xb, int& idx, int& conj, double& sgn) {
    if (2 * xb <= tt) {
      idx = half_base(tt) + xb * (tt + 1) + xa;
      conj = 0;
      sgn = 1.0;
    } else {
      idx = half_base(tt) + (tt - xb) * (tt + 1) + (tt - xa);
      conj = 1;
      sgn = ((xa + xb) & 1) ? -1.0 : 1.0;
    }
  };
  // triples grouped by output rank
  std::vector<std::vector<int>> by_t(J2 + 1);
  std::unordered_map<unsigned long long, size_t> same_layer;  // (triple, word) -> term
  for (int q = 0; q < (int)ztrip.size(); ++q) by_t[ztrip[q].t].push_back(q);
  for (int t = 0; t <= J2; ++t)
    for (int mb = 0; 2 * mb <= t; ++mb)
      for (int ma = 0; ma <= t; ++ma) {
        const size_t first = terms.size();
        same_layer.clear();
        // Below the centre of the middle column (2 mb = t, ma > mb) Y is the
        // mirror of the element above it, and the contractions that read Y
        // (energy, dE/dr) give it weight 0: one zero term there (Y = 0), and
        // the host export fills in the mirror.
        const bool mirrored = 2 * mb == t && ma > mb;
        for (int q : by_t[t]) {
          if (mirrored) break;
          const ZTrip& z = ztrip[q];
          const int dl = (z.t1 + z.t2 - t) / 2;
          for (int mb1 = std::max(0, mb + dl - z.t2); mb1 <= std::min(z.t1, mb + dl); ++mb1) {
            const int mb2 = mb + dl - mb1;
            const double cb = cg[z.cg_off + mb1 * (z.t2 + 1) + mb2];
            if (cb == 0.0) continue;
            for (int ma1 = std::max(0, ma + dl - z.t2); ma1 <= std::min(z.t1, ma + dl); ++ma1) {
              const int ma2 = ma + dl - ma1;
              const double ca = cg[z.cg_off + ma1 * (z.t2 + 1) + ma2];
              if (ca == 0.0) continue;
              int i1, c1, i2, c2;
              double s1, s2;
              half_elem(z.t1, ma1, mb1, i1, c1, s1);
              half_elem(z.t2, ma2, mb2, i2, c2, s2);
              // t1 == t2: the term with the factors swapped, (ma2, mb2) as
              // the first, has the same coefficient and the same product, so
              // the two are kept as one term, the stored element with the
              // lower (index, conjugation) first, with the summed coefficient
              if (z.t1 == z.t2 && (i2 < i1 || (i2 == i1 && c2 < c1))) {
                std::swap(i1, i2);
                std::swap(c1, c2);
              }
              const unsigned w = (unsigned)i1 | ((unsigned)i2 << 10) | ((unsigned)c1 << 20) |
                                 ((unsigned)c2 << 21);
              const double cgp = ca * cb * s1 * s2;
              if (z.t1 == z.t2) {
                const auto ins = same_layer.emplace(((unsigned long long)q << 32) | w, terms.size());
                if (!ins.second) {
                  term_cg[ins.first->second] += cgp;
                  continue;
                }
              }
              terms.push_back(w);
              term_cg.push_back(cgp);
              term_trip.push_back(q);
            }
          }
        }
        {  // drop merged terms whose coefficients cancelled exactly
          size_t o = first;
          for (size_t k = first; k < terms.size(); ++k)
            if (term_cg[k] != 0.0) {
              terms[o] = terms[k];
              term_cg[o] = term_cg[k];
              term_trip[o] = term_trip[k];
              ++o;
            }
          terms.resize(o);
          term_cg.resize(o);
          term_trip.resize(o);
        }
        if (mirrored) {
          terms.push_back(0u);
          term_cg.push_back(0.0);
          term_trip.push_back(by_t[t].front());
        }
        orient_by_cover(terms, first);
        // Group the output's terms by their first factor (index and
        // conjugation flag, stable): compute_Y then forms
        //   Y += U_t1[..] * sum_k coef_k U_t2,k[..]
        // once per group.  Groups longer than kYGroupMax are cut into chunks,
        // and with size_runs the chunks are ordered by length (stable), so an
        // output is a run of 1-term groups, then of 2-term groups, ...;
        // term_runs counts them.  Without it the groups keep the order of
        // their first factor.  Bit 23 ends a group, bit 22 the output; every output has at
        // least one term: the term of the (t, 0, t) triple, whose
        // Clebsch-Gordan product is 1, or the zero term of a mirrored output.
        const size_t cnt = terms.size() - first;
        std::array<unsigned short, kYGroupMax> runs{};
        if (cnt > 0) {
          std::vector<size_t> ord(cnt);
          for (size_t k = 0; k < cnt; ++k) ord[k] = k;
          auto key = [&](size_t k) { return terms[first + k] & ((1023u) | (1u << 20)); };
          std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return key(x) < key(y); });
          std::vector<unsigned> tw(cnt);
          std::vector<double> tc(cnt);
          std::vector<int> tq(cnt);
          for (size_t k = 0; k < cnt; ++k) {
            tw[k] = terms[first + ord[k]];
            tc[k] = term_cg[first + ord[k]];
            tq[k] = term_trip[first + ord[k]];
          }
          const unsigned kmask = 1023u | (1u << 20);
          struct Chunk {
            size_t b, n;
          };
          std::vector<Chunk> ch;
          for (size_t k = 0; k < cnt;) {
            size_t e = k + 1;
            while (e < cnt && (tw[e] & kmask) == (tw[k] & kmask)) ++e;
            for (size_t b = k; b < e; b += kYGroupMax) ch.push_back({b, std::min<size_t>(kYGroupMax, e - b)});
            k = e;
          }
          if (size_runs)
            std::stable_sort(ch.begin(), ch.end(), [](const Chunk& x, const Chunk& y) { return x.n < y.n; });
          size_t pos = first;
          for (const Chunk& c : ch) {
            runs[c.n - 1] += 1;
            for (size_t j = 0; j < c.n; ++j, ++pos) {
              terms[pos] = tw[c.b + j] | (j + 1 == c.n ? (1u << 23) : 0u);
              term_cg[pos] = tc[c.b + j];
              term_trip[pos] = tq[c.b + j];
            }
          }
          terms.back() |= (1u << 22);
        }
        term_runs.insert(term_runs.end(), runs.begin(), runs.end());
        term_out_first.push_back((int)first);
      }
  term_out_first.push_back((int)terms.size());

  // Bispectrum term list (descriptor output, Eq. z): for every canonical
  // component l = (t1 >= t2, t >= t1), for every half-layout element (t, ma,
  // mb) with a nonzero half weight w,
  //   B_l += Re( conj(U_t[ma][mb]) * w * sum C(ma1,ma2) C(mb1,mb2) U_t1 U_t2 ),
  // so B_l = Re Z^t_{t1t2} : conj(U_t) over the full matrix.  The records
  // use the compute_Y format with w folded into the coefficient; bit 22 ends
  // an output element, bit 23 ends a component; bout holds the U_t element
  // index of every output group in order.
  bterms.clear();
  bterm_coef.clear();
  bout.clear();
  bcomp_first.clear();
  bgroup_first.clear();
  for (int q = 0; q < (int)ztrip.size(); ++q) {
    const ZTrip& z = ztrip[q];
    if (z.t < z.t1) continue;  // canonical components only
    bcomp_first.push_back((int)bterms.size());
    bgroup_first.push_back((int)bout.size());
    const int t = z.t, dl = (z.t1 + z.t2 - t) / 2;
    for (int mb = 0; 2 * mb <= t; ++mb)
      for (int ma = 0; ma <= t; ++ma) {
        const int wgt = (2 * mb < t) ? 2 : (ma < mb ? 2 : (ma == mb ? 1 : 0));
        if (wgt == 0) continue;
        const size_t first = bterms.size();
        for (int mb1 = std::max(0, mb + dl - z.t2); mb1 <= std::min(z.t1, mb + dl); ++mb1) {
          const int mb2 = mb + dl - mb1;
          const double cb = cg[z.cg_off + mb1 * (z.t2 + 1) + mb2];
          if (cb == 0.0) continue;
          for (int ma1 = std::max(0, ma + dl - z.t2); ma1 <= std::min(z.t1, ma + dl); ++ma1) {
            const int ma2 = ma + dl - ma1;
            const double ca = cg[z.cg_off + ma1 * (z.t2 + 1) + ma2];
            if (ca == 0.0) continue;
            int i1, c1, i2, c2;
            double s1, s2;
            half_elem(z.t1, ma1, mb1, i1, c1, s1);
            half_elem(z.t2, ma2, mb2, i2, c2, s2);
            bterms.push_back((unsigned)i1 | ((unsigned)i2 << 10) | ((unsigned)c1 << 20) |
                             ((unsigned)c2 << 21));
            bterm_coef.push_back(wgt * ca * cb * s1 * s2);
          }
        }
        if (bterms.size() > first) {
          bterms.back() |= (1u << 22);
          bout.push_back(half_base(t) + mb * (t + 1) + ma);
        }
      }
    bterms.back() |= (1u << 23);
  }
  bcomp_first.push_back((int)bterms.size());
  bgroup_first.push_back((int)bout.size());
  // chunks of whole groups, about kBChunk terms (more at large 2J, so that
  // there are at most about kBMaxChunks), within components
  const int chunk_len = std::max<int>(kBChunk, (int)((bterms.size() + kBMaxChunks - 1) / kBMaxChunks));
  bchunk_term.clear();
  bchunk_group.clear();
  bcomp_chunk.clear();
  for (int l = 0; l < ncoeff; ++l) {
    bcomp_chunk.push_back((int)bchunk_term.size());
    int q = bcomp_first[l], gq = bgroup_first[l];
    bchunk_term.push_back(q);
    bchunk_group.push_back(gq);
    int inchunk = 0;
    for (; q < bcomp_first[l + 1]; ++q) {
      ++inchunk;
      if (bterms[q] & (1u << 22)) {  // a group ends here
        ++gq;
        if (inchunk >= chunk_len && q + 1 < bcomp_first[l + 1]) {
          bchunk_term.push_back(q + 1);
          bchunk_group.push_back(gq);
          inchunk = 0;
        }
      }
    }
  }
  bcomp_chunk.push_back((int)bchunk_term.size());
  bchunk_term.push_back((int)bterms.size());
  bchunk_group.push_back((int)bout.size());
  // device order: every chunk's groups cut into pieces of at most kBGroupMax
  // terms (a group of n terms into ceil(n / kBGroupMax) pieces whose lengths
  // differ by at most one), pieces ordered by length, stably
  const int nchunks = (int)bchunk_term.size() - 1;
  bdev.assign(bterms.size(), 0u);
  bdev_coef.assign(bterms.size(), 0.0);
  bdev_o.assign(bterms.size(), -1);
  bchunk_runs.assign((size_t)nchunks * kBGroupMax, 0);
  struct Piece {
    int first, len, o;
  };
  std::vector<Piece> pieces;
  for (int ch = 0; ch < nchunks; ++ch) {
    pieces.clear();
    int g = bchunk_group[ch], gfirst = bchunk_term[ch];
    for (int q = bchunk_term[ch]; q < bchunk_term[ch + 1]; ++q) {
      if (!(bterms[q] & (1u << 22))) continue;
      const int n = q + 1 - gfirst, np = (n + kBGroupMax - 1) / kBGroupMax;
      for (int k = 0, at = gfirst; k < np; ++k) {
        const int len = n / np + (k < n % np ? 1 : 0);
        pieces.push_back({at, len, bout[g]});
        at += len;
      }
      gfirst = q + 1;
      ++g;
    }
    std::stable_sort(pieces.begin(), pieces.end(), [](const Piece& x, const Piece& y) { return x.len < y.len; });
    int at = bchunk_term[ch];
    for (const Piece& pc : pieces) {
      bchunk_runs[(size_t)ch * kBGroupMax + pc.len - 1] += 1;
      for (int k = 0; k < pc.len; ++k, ++at) {
        bdev[at] = bterms[pc.first + k] & 0x3FFFFFu;
        bdev_coef[at] = bterm_coef[pc.first + k];
        bdev_o[at] = k == 0 ? pc.o : -1;
      }
    }
  }

  half_scale.assign(H, 0.0);
  for (int e = 0; e < H; ++e) {
    const int t = tmm_t(half_tmm[e]), ma = tmm_ma(half_tmm[e]), mb = tmm_mb(half_tmm[e]);
    long double f = 1.0L;
    for (int k = 2; k <= t - ma; ++k) f *= k;
    for (int k = 2; k <= ma; ++k) f *= k;
    for (int k = 2; k <= t - mb; ++k) f /= k;
    half_scale[e] = (double)std::sqrt(f);
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

std::vector<double> HostTables::term_coef(const double* beta) const {
  const std::vector<double> bw = beta_weights(beta);
  std::vector<double> c(terms.size());
  for (size_t k = 0; k < terms.size(); ++k) c[k] = term_cg[k] * bw[term_trip[k]];
  return c;
}

std::vector<int> HostTables::bslices(int nslices) const {
  // contiguous runs of components with about equal term counts
  const long total = (long)bterms.size();
  std::vector<int> b(1, 0);
  int k = 1;
  for (int l = 0; l < ncoeff; ++l) {
    if (k < nslices && (long)bcomp_first[l + 1] * nslices >= total * k) {
      b.push_back(l + 1);
      ++k;
    }
  }
  while ((int)b.size() < nslices + 1) b.push_back(ncoeff);
  b[nslices] = ncoeff;
  return b;
}

std::vector<int> HostTables::bparts(int nparts, int* maxchunks, int* maxterms) const {
  const std::vector<int> b = bslices(nparts);
  int mx = 0, mt = 0;
  for (int k = 0; k < nparts; ++k) {
    const int c0 = bcomp_chunk[b[k]], c1 = bcomp_chunk[b[k + 1]];
    mx = std::max(mx, c1 - c0);
    mt = std::max(mt, bchunk_term[c1] - bchunk_term[c0]);
  }
  *maxchunks = mx;
  *maxterms = mt;
  return b;
}

std::vector<int> HostTables::lane_outputs(int lanes, int* m) const {
  std::vector<int> ord(H);
  for (int o = 0; o < H; ++o) ord[o] = o;
  auto nterm = [&](int o) { return term_out_first[o + 1] - term_out_first[o]; };
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return nterm(x) > nterm(y); });
  const int mm = (H + lanes - 1) / lanes;
  std::vector<int> t((size_t)lanes * mm, -1);
  for (int k = 0; k < H; ++k) {
    const int round = k / lanes, pos = k % lanes;
    const int lane = (round & 1) ? lanes - 1 - pos : pos;
    t[(size_t)lane * mm + round] = ord[k];
  }
  *m = mm;
  return t;
}

std::vector<int> HostTables::slices(int nslices) const {
  // nslices contiguous runs of output elements with about equal term counts;
  // entry k is the first output of run k (entry nslices = H)
  const long total = (long)terms.size();
  std::vector<int> b(1, 0);
  int k = 1;
  for (int o = 0; o < H; ++o) {
    const long done = term_out_first[o + 1];
    if (k < nslices && done * nslices >= total * k) {
      b.push_back(o + 1);
      ++k;
    }
  }
  while ((int)b.size() < nslices + 1) b.push_back(H);
  b[nslices] = H;
  return b;
}

std::vector<unsigned> HostTables::bwords(bool cp) const {
  std::vector<unsigned> w(bdev.size(), 0u);
  for (size_t q = 0; q < bdev.size(); ++q) {
    const unsigned t = bdev[q];
    const unsigned i1 = t & 1023u, i2 = (t >> 10) & 1023u, c1 = (t >> 20) & 1u, c2 = (t >> 21) & 1u;
    unsigned x = cp ? (((i2 + c2 * (unsigned)H) << 8) | ((i1 + c1 * (unsigned)H) << 19))
                    : ((i2 << 8) | (i1 << 18) | (c1 << 30) | (c2 << 31));
    if (bdev_o[q] >= 0) {
      const unsigned o = (unsigned)bdev_o[q];
      if (o > 1023u) return {};  // not reached for 2J <= 14 (H = 652)
      x |= (o & 0xFFu) | ((o >> 8) << (cp ? 30 : 28));
    }
    w[q] = x;
  }
  return w;
}

}  // namespace snap

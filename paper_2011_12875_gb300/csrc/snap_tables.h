// snap_tables.h -- host-side tables of the library (see snap_tables.cpp).
#pragma once
#include <vector>

#include "snap_internal.h"

namespace snap {

struct ZTrip {
  int t1, t2, t;  // Y triple: Z^t_{t1 t2} with t1 >= t2
  int cg_off;     // offset of its cg[x1][x2] block
  int bidx;       // canonical bispectrum component it belongs to
  double fac;     // multiplicity / rank factor of the derivative
};

struct HostTables {
  int twojmax = 0, H = 0, lmax = 0, ncoeff = 0;
  std::vector<int> half_tmm;
  std::vector<ZTrip> ztrip;
  std::vector<double> cg;
  // compute_Y terms: packed indices/flags, CG product with signs, triple
  std::vector<unsigned> terms;
  std::vector<double> term_cg;
  std::vector<int> term_trip;
  std::vector<int> term_out_first;  // [H+1] first term of every output
  // [H][kYGroupMax]: number of groups of 1, 2, ... kYGroupMax terms of each
  // output (they follow one another in that order)
  std::vector<unsigned short> term_runs;
  // bispectrum terms (records as above, coefficient without beta), the U
  // element of each output group, and the first term of each component
  std::vector<unsigned> bterms;
  std::vector<double> bterm_coef;
  std::vector<int> bout;
  std::vector<int> bcomp_first;
  std::vector<int> bgroup_first;  // [ncoeff+1] first output group of each component
  // the bispectrum term list cut into chunks of whole output groups (about
  // kBChunk terms, never across a component): first term and first group of
  // every chunk (+1 end entry each) and the first chunk of every component
  std::vector<int> bchunk_term, bchunk_group, bcomp_chunk;
  // The device order of the bispectrum terms: within every chunk each output
  // group cut into pieces of at most kBGroupMax terms (near-equal lengths),
  // the pieces ordered by length (stably), so that the device walks runs of
  // equal-length pieces with branch-free bodies.  Chunks keep their term
  // ranges.  bdev: the table words (as bterms, without the end bits);
  // bdev_coef: their coefficients; bdev_o: the U element of each term's
  // piece, -1 on all but a piece's first term; bchunk_runs [nchunks]
  // [kBGroupMax]: the number of pieces of 1, 2, ... terms of every chunk.
  std::vector<unsigned> bdev;
  std::vector<double> bdev_coef;
  std::vector<int> bdev_o;
  std::vector<unsigned short> bchunk_runs;
  std::vector<double> rootpq;
  // [H]: S_t(ma, mb) = sqrt((t - ma)! ma! / (t - mb)!) of every half-layout
  // element, the factor between the scaled recursion's v and u
  std::vector<double> half_scale;

  // size_runs: order each output's term groups by length (the run layout of
  // the FP32 compute_Y); otherwise by first factor
  void build(int twojmax, bool size_runs = true);
  std::vector<double> beta_weights(const double* beta) const;
  std::vector<double> term_coef(const double* beta) const;
  std::vector<int> slices(int nslices) const;
  // outputs dealt to `lanes` lanes in decreasing term count, snake order:
  // [lanes][m] output indices, -1 past a lane's last; m returned in *m
  std::vector<int> lane_outputs(int lanes, int* m) const;
  std::vector<int> bslices(int nslices) const;
  // nparts contiguous runs of components with about equal term counts (entry
  // k = first component of run k, entry nparts = ncoeff); *maxchunks = the
  // most chunks of one run
  // and *maxterms = the most terms of one run
  std::vector<int> bparts(int nparts, int* maxchunks, int* maxterms) const;
  // The bispectrum records' words as the device reads them (one per term of
  // the device order):
  //   cp = false (factors' stored elements, imaginary parts flipped by flag):
  //     bits 8-17 second factor, 18-27 first factor, 30 conjugate the first
  //     factor, 31 conjugate the second; a piece's U element in bits 0-7
  //     (low) and 28-29 (high) of its first word
  //   cp = true (factors in a [2][H] plane, conjugates in the second half):
  //     bits 8-18 second factor, 19-29 first factor; the piece's U element in
  //     bits 0-7 and 30-31 of its first word
  // Empty if an element does not fit in 10 bits.
  std::vector<unsigned> bwords(bool cp) const;
};

double clebsch_gordan(int tj1, int tm1, int tj2, int tm2, int tj, int tm);
int count_coeff(int twojmax);

}  // namespace snap

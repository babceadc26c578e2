// snap_col_f64.cu -- register column-chain kernels in FP64 working
// precision, one instance per 2J: compute_U, the reverse-mode fused dE and
// the tangent of Ulisttot along a displacement field.
#include "snap_colkernels.cuh"

namespace snap {

template <>
cudaError_t launch_ui_col<double>(const WorkArgs& a, cudaStream_t s) {
  switch (a.twojmax) {
#define SNAP_CASE(J) \
  case J: return col::launch_ui_col_t<double, J>(a, s);
    SNAP_CASE(1) SNAP_CASE(2) SNAP_CASE(3) SNAP_CASE(4) SNAP_CASE(5) SNAP_CASE(6) SNAP_CASE(7)
    SNAP_CASE(8) SNAP_CASE(9) SNAP_CASE(10) SNAP_CASE(11) SNAP_CASE(12) SNAP_CASE(13) SNAP_CASE(14)
#undef SNAP_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_de_col<double>(const WorkArgs& a, cudaStream_t s) {
  switch (a.twojmax) {
#define SNAP_CASE(J) \
  case J: return col::launch_de_rev_col_t<double, J>(a, s);
    SNAP_CASE(1) SNAP_CASE(2) SNAP_CASE(3) SNAP_CASE(4) SNAP_CASE(5) SNAP_CASE(6) SNAP_CASE(7)
    SNAP_CASE(8) SNAP_CASE(9) SNAP_CASE(10) SNAP_CASE(11) SNAP_CASE(12) SNAP_CASE(13) SNAP_CASE(14)
#undef SNAP_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_tan_col<double>(const WorkArgs& a, const double* g, void* dU, cudaStream_t s) {
  switch (a.twojmax) {
#define SNAP_CASE(J) \
  case J: return col::launch_tan_col_t<double, J>(a, g, dU, s);
    SNAP_CASE(0) SNAP_CASE(1) SNAP_CASE(2) SNAP_CASE(3) SNAP_CASE(4) SNAP_CASE(5) SNAP_CASE(6)
    SNAP_CASE(7) SNAP_CASE(8) SNAP_CASE(9) SNAP_CASE(10) SNAP_CASE(11) SNAP_CASE(12) SNAP_CASE(13)
    SNAP_CASE(14)
#undef SNAP_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_neigh_u<double>(const NeighArgs& na, const WorkArgs& a, int ncta, cudaStream_t s) {
  switch (a.twojmax) {
#define SNAP_CASE(J) \
  case J: return col::launch_neigh_u_t<double, J>(na, a, ncta, s);
    SNAP_CASE(1) SNAP_CASE(2) SNAP_CASE(3) SNAP_CASE(4) SNAP_CASE(5) SNAP_CASE(6) SNAP_CASE(7) SNAP_CASE(8)
#undef SNAP_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace snap

// Instantiations of the register-resident solver for the Eikonal family (the
// two- and ten-dimensional problems of Section 6.1; other d run in the
// coordinate-parallel kernel).
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_eikonal(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 2: return launch_warp_shape<T, FamEikonal, 2, false>(a, c, s);
    case 10: return launch_warp_shape<T, FamEikonal, 10, false>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_eikonal<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_eikonal<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

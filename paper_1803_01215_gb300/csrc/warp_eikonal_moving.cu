// Instantiations of the register-resident solver for the eikonal family with a
// moving bump (Section 6.1's state-and-time-dependent example, d = 2, and the
// 10-dimensional slice), backward Euler.
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_eikonal_moving(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 2: return launch_warp_shape<T, FamEikonalMoving, 2, false>(a, c, s);
    case 10: return launch_warp_shape<T, FamEikonalMoving, 10, false>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_eikonal_moving<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_eikonal_moving<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

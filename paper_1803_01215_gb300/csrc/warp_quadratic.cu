// Instantiations of the register-resident solver for the Quadratic family.
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_quadratic(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 1: return launch_warp_shape<T, FamQuadratic, 1, false>(a, c, s);
    case 2: return launch_warp_shape<T, FamQuadratic, 2, false>(a, c, s);
    case 3: return launch_warp_shape<T, FamQuadratic, 3, false>(a, c, s);
    case 4: return launch_warp_shape<T, FamQuadratic, 4, false>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_quadratic<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_quadratic<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

// Hopf-form (Algorithm 2) instantiations of the register-resident solver for the Quadratic family.
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_quadratic_hopf(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 1: return launch_warp_shape<T, FamQuadratic, 1, true>(a, c, s);
    case 2: return launch_warp_shape<T, FamQuadratic, 2, true>(a, c, s);
    case 3: return launch_warp_shape<T, FamQuadratic, 3, true>(a, c, s);
    case 4: return launch_warp_shape<T, FamQuadratic, 4, true>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_quadratic_hopf<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_quadratic_hopf<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

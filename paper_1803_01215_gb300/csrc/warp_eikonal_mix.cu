// Instantiations of the register-resident solver for the Eikonal family,
// forward-Euler and trapezoid schemes.
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_eikonal_mix(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 2: return launch_warp_shape<T, FamEikonal, 2, false, true>(a, c, s);
    case 10: return launch_warp_shape<T, FamEikonal, 10, false, true>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_eikonal_mix<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_eikonal_mix<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

// Instantiations of the register-resident solver for the TanhDrift family.
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_tanh(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 2: return launch_warp_shape<T, FamTanhDrift, 2, false>(a, c, s);
    case 4: return launch_warp_shape<T, FamTanhDrift, 4, false>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_tanh<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_tanh<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

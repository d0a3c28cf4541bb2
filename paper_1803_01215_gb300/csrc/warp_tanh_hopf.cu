// Hopf-form (Algorithm 2) instantiations of the register-resident solver for the TanhDrift family.
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_tanh_hopf(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 2: return launch_warp_shape<T, FamTanhDrift, 2, true>(a, c, s);
    case 4: return launch_warp_shape<T, FamTanhDrift, 4, true>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_tanh_hopf<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_tanh_hopf<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

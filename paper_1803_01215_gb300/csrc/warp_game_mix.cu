// Instantiations of the register-resident solver for the difference-of-norms
// game, forward-Euler and trapezoid schemes.
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_game_mix(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 2: return launch_warp_shape<T, FamGame, 2, false, true>(a, c, s);
    case 7: return launch_warp_shape<T, FamGame, 7, false, true>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_game_mix<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_game_mix<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

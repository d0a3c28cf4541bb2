// Instantiations of the register-resident solver for the difference-of-norms
// game of Section 6.2 (its two- and seven-dimensional cases).
#include "warp_solver.cuh"

namespace hj {

template <typename T>
hj_status launch_warp_game(const SolveArgs<T>& a, WarpConfig c, cudaStream_t s) {
  switch (a.d) {
    case 2: return launch_warp_shape<T, FamGame, 2, false>(a, c, s);
    case 7: return launch_warp_shape<T, FamGame, 7, false>(a, c, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_game<float>(const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_game<double>(const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

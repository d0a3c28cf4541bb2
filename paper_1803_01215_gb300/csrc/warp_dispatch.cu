// Launch-shape selection for the register-resident solver.
#include "hj_internal.cuh"

namespace hj {

namespace {
bool warp_family_has(int family, int d) {
  switch (family) {
    case HJ_FAMILY_QUADRATIC: return d >= 1 && d <= 4;
    case HJ_FAMILY_QUADCOPTER: return d == 12;
    case HJ_FAMILY_TANH_DRIFT: return d == 2 || d == 4;
    case HJ_FAMILY_EIKONAL: return d == 2 || d == 10;
    case HJ_FAMILY_GAME_NORMS: return d == 2 || d == 7;
    default: return false;
  }
}
}  // namespace

bool warp_config_available(int family, int d, WarpConfig c, bool fp64) {
  if (!warp_family_has(family, d)) return false;
  if (c.half) return c.G == 1 && c.NPL == 1 && d <= 16;
  if (c.G != 1 && c.G != 2 && c.G != 4 && c.G != 8) return false;
  return fp64 ? c.NPL == 1 : (c.NPL == 1 || c.NPL == 2);
}

// One time node per lane and as many warps as N needs, except for H = |p|^2/2,
// whose node update is so short that two nodes per lane (half the exchanges
// and barriers per node) win: at N = 64 (FP32, 2048-4096 points) one node per
// lane over two warps ran 1.26x (quadcopter), 1.46x (tanh drift, d = 4) and
// 1.47x (eikonal, d = 2) faster than two nodes per lane in one warp, and 0.87x
// for the quadratic family.
// Half a warp per point for the eikonal family and the game at 8 < N <= 16
// (FP32, 3721-5329 points): 1.12-1.33x faster at N = 10 and 15 (eikonal d = 10,
// the game d = 2 and 7), 0.95x for the eikonal d = 2 at N = 10 (1.06x with the
// trapezoid scheme); 0.85x for the quadcopter at N = 16 and 0.97x for the game
// d = 2 at N = 5, which keep a whole warp.
WarpConfig default_warp_config(int family, int d, int Nmax, bool fp64) {
  if (!warp_family_has(family, d) || Nmax < 1 || Nmax > kMaxN) return WarpConfig{0, 0};
  if ((family == HJ_FAMILY_EIKONAL || family == HJ_FAMILY_GAME_NORMS) && Nmax > 8 &&
      Nmax <= 16 && d <= 16)
    return WarpConfig{1, 1, 1};
  if (!fp64 && family == HJ_FAMILY_QUADRATIC) {
    if (Nmax <= 32) return WarpConfig{1, 1};
    if (Nmax <= 64) return WarpConfig{1, 2};
    if (Nmax <= 128) return WarpConfig{2, 2};
    return WarpConfig{4, 2};
  }
  int G = 1;
  while (32 * G < Nmax) G *= 2;
  return WarpConfig{G, 1};
}

template <typename T>
hj_status launch_warp_solver(int family, const SolveArgs<T>& a, WarpConfig cfg, cudaStream_t s) {
  if (!warp_config_available(family, a.d, cfg, sizeof(T) == 8)) return HJ_ERR_UNSUPPORTED;
  if (a.N > warp_config_lanes(cfg) * cfg.NPL) return HJ_ERR_UNSUPPORTED;
  const bool hopf = a.formulation == HJ_FORM_HOPF;
  if (a.scheme != HJ_SCHEME_BE) {                 // forward Euler, trapezoid (Lax form)
    if (hopf) return HJ_ERR_UNSUPPORTED;
    switch (family) {
      case HJ_FAMILY_QUADCOPTER: return launch_warp_quadcopter_mix<T>(a, cfg, s);
      case HJ_FAMILY_TANH_DRIFT: return launch_warp_tanh_mix<T>(a, cfg, s);
      case HJ_FAMILY_EIKONAL: return launch_warp_eikonal_mix<T>(a, cfg, s);
      case HJ_FAMILY_GAME_NORMS: return launch_warp_game_mix<T>(a, cfg, s);
      default: return HJ_ERR_UNSUPPORTED;
    }
  }
  switch (family) {
    case HJ_FAMILY_QUADRATIC:
      return hopf ? launch_warp_quadratic_hopf<T>(a, cfg, s) : launch_warp_quadratic<T>(a, cfg, s);
    case HJ_FAMILY_QUADCOPTER:
      return hopf ? launch_warp_quadcopter_hopf<T>(a, cfg, s) : launch_warp_quadcopter<T>(a, cfg, s);
    case HJ_FAMILY_TANH_DRIFT:
      return hopf ? launch_warp_tanh_hopf<T>(a, cfg, s) : launch_warp_tanh<T>(a, cfg, s);
    case HJ_FAMILY_EIKONAL:
      if (hopf) return HJ_ERR_UNSUPPORTED;
      return a.eik_moving ? launch_warp_eikonal_moving<T>(a, cfg, s) : launch_warp_eikonal<T>(a, cfg, s);
    case HJ_FAMILY_GAME_NORMS:
      return hopf ? HJ_ERR_UNSUPPORTED : launch_warp_game<T>(a, cfg, s);
    default: return HJ_ERR_UNSUPPORTED;
  }
}

template hj_status launch_warp_solver<float>(int, const SolveArgs<float>&, WarpConfig, cudaStream_t);
template hj_status launch_warp_solver<double>(int, const SolveArgs<double>&, WarpConfig, cudaStream_t);

}  // namespace hj

// Residual of the discrete characteristic equations at given trajectories.
//
// At a saddle of Eq. (disclaxBE) the Lagrangian is stationary in every x_j and
// p_j, which gives the discrete form of x' = H_p, p' = -H_x with p(0) = grad g
// (Section 4):
//   r1_j = x_j - x_{j-1} - delta grad_p H(x_j, p_j, s_j)     j = 1..N
//   r2   = p_1 - grad g(x_0)
//   r3_j = p_{j+1} - p_j + delta grad_x H(x_j, p_j, s_j)     j = 1..N-1
// This kernel evaluates max(|r1|, |r2|, |r3|) per point in FP64 from the
// trajectories in either iterate type, for the families and dimensions beyond
// the register-resident solver's (which kkt_node.cu serves one thread per node):
// tanh drift and H = |p|^2/2 at larger d, the eikonal family at any other d.
// It serves hj_kkt_residual and the kkt output of hj_solve_batch.
//
// One CTA per point (grid-stride over points); the CTA walks the nodes
// j = 1..N, its threads over coordinates, with the node's x_j and p_j staged in
// shared memory in FP64 for the products (tanh drift) and sums (eikonal).  For
// the negative eikonal equation the equations are taken in the solver's
// variables (costate -p, initial data -g), whose residuals have the magnitudes
// of phi's own; where the eikonal H = c|p| is not differentiable (p_j = 0), r1_j
// is the distance of x_j - x_{j-1} to the ball of radius delta c(x_j).
#include <cuda_runtime.h>

#include <cmath>

#include "hj_internal.cuh"
#include "hjpdhg.h"
#include "problem.cuh"

namespace hj {

namespace {

constexpr int kKktThreads = 128;

struct KktArgs {
  int64_t B;
  int32_t N, d, family;
  const double* t;
  const double* W2;       // [d]
  const double* c;        // [d]
  const double* A;        // tanh drift [d][d] row-major
  const double* At;       // its transpose
  double qc_m, qc_ah, qc_gz, qc_eps;
  double sign;            // -1: negative eikonal equation (the solver's variables)
  double c0, c1, c2;      // eikonal speed
  const double* xb;       // [d]
  const double* vb;       // [d] or null
  double* kkt;            // [B]
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum<double>(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();                               // red free from any earlier use
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max_nan(v, __shfl_xor_sync(kFull, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max_nan(m, red[w]);
  return m;
}

// thrust direction a(psi, theta, phi) and J[3 r + k] = d a_r / d (psi, theta, phi)_k
__device__ void qc_thrust(double psi, double th, double ph, double (&a)[3], double (&J)[9]) {
  double sps, cps, sth, cth, sph, cph;
  sincos(psi, &sps, &cps);
  sincos(th, &sth, &cth);
  sincos(ph, &sph, &cph);
  const double cc = cph * cps, cs = cph * sps, sc = sph * cps, ss = sph * sps;
  a[0] = ss + cc * sth;
  a[1] = -sc + cs * sth;
  a[2] = cth * cph;
  J[0] = sc - cs * sth;  J[1] = cc * cth;    J[2] = cs - sc * sth;
  J[3] = ss + cc * sth;  J[4] = cs * cth;    J[5] = -cc - ss * sth;
  J[6] = 0.0;            J[7] = -sth * cph;  J[8] = -cth * sph;
}

template <typename T>
__global__ void __launch_bounds__(kKktThreads)
kkt_kernel(const KktArgs k, const T* __restrict__ X, const T* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int d = k.d, N = k.N;
  double* xs = reinterpret_cast<double*>(smem);   // x_j        [d]
  double* qs = xs + d;                            // p_j        [d] (solver's sign)
  double* ws = qs + d;                            // tanh drift: (1 - a^2) p_j  [d]
  double* red = ws + d;                           // [kKktThreads / 32]
  for (int64_t b = blockIdx.x; b < k.B; b += gridDim.x) {
    const T* xb_ = X + (size_t)b * (N + 1) * d;
    const T* pb_ = P + (size_t)b * (N + 1) * d;
    const double delta = k.t[b] / N;
    double r = 0.0;
    // r2 = p_1 - grad g(x_0)
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
      const double w2 = k.sign * k.W2[i];
      r = max_nan(r, fabs(k.sign * (double)pb_[d + i] - w2 * ((double)xb_[i] - k.c[i])));
    }
    for (int j = 1; j <= N; ++j) {
      const double sj = j * delta;
      __syncthreads();                            // the previous node's xs, qs, ws are read
      for (int i = threadIdx.x; i < d; i += blockDim.x) {
        xs[i] = (double)xb_[(size_t)j * d + i];
        qs[i] = k.sign * (double)pb_[(size_t)j * d + i];
      }
      __syncthreads();
      // family-specific node scalars
      double ec = 0.0, egf = 0.0, qn = 0.0, dn = 0.0;   // eikonal: c, -2 c1 c2 e, |p|, |dx|
      if (k.family == HJ_FAMILY_EIKONAL) {
        double r2 = 0.0, q2 = 0.0, d2 = 0.0;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
          const double cb = k.xb[i] + (k.vb ? sj * k.vb[i] : 0.0);
          const double y = xs[i] - cb, dx = xs[i] - (double)xb_[(size_t)(j - 1) * d + i];
          r2 += y * y;
          q2 += qs[i] * qs[i];
          d2 += dx * dx;
        }
        r2 = block_sum(r2, red);
        q2 = block_sum(q2, red);
        d2 = block_sum(d2, red);
        const double e = exp(-k.c2 * r2);
        ec = k.c0 + k.c1 * e;
        egf = -2.0 * k.c1 * k.c2 * e;
        qn = sqrt(q2);
        dn = sqrt(d2);
      } else if (k.family == HJ_FAMILY_TANH_DRIFT) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
          double y = 0.0;
          for (int m = 0; m < d; ++m) y += k.A[(size_t)i * d + m] * xs[m];
          const double av = tanh(y);
          const double dx = xs[i] - (double)xb_[(size_t)(j - 1) * d + i];
          r = max_nan(r, fabs(dx - delta * (av + qs[i])));
          ws[i] = (1.0 - av * av) * qs[i];
        }
        __syncthreads();
      }
      double qa[3], qJ[9], u0 = 0.0;
      if (k.family == HJ_FAMILY_QUADCOPTER && (int)threadIdx.x < d) {
        qc_thrust(xs[3], xs[4], xs[5], qa, qJ);
        u0 = (qa[0] * qs[6] + qa[1] * qs[7] + qa[2] * qs[8]) / k.qc_m;
      }
      for (int i = threadIdx.x; i < d; i += blockDim.x) {
        const double xl = (double)xb_[(size_t)(j - 1) * d + i];
        const double dx = xs[i] - xl;
        double gx = 0.0;
        switch (k.family) {
          case HJ_FAMILY_QUADRATIC:
            r = max_nan(r, fabs(dx - delta * qs[i]));
            break;
          case HJ_FAMILY_QUADCOPTER: {
            double gp;
            if (i < 6) gp = xs[6 + i];
            else if (i < 9) gp = k.qc_ah * qa[i - 6] - (i == 8 ? k.qc_gz : 0.0) + qa[i - 6] * u0 / k.qc_m;
            else gp = qs[i];
            gp += k.qc_eps * qs[i];
            r = max_nan(r, fabs(dx - delta * gp));
            if (i >= 3 && i < 6)
              gx = (k.qc_ah + u0 / k.qc_m) * (qJ[i - 3] * qs[6] + qJ[i] * qs[7] + qJ[i + 3] * qs[8]);
            else if (i >= 6)
              gx = qs[i - 6];
            break;
          }
          case HJ_FAMILY_TANH_DRIFT: {            // r1 done above
            for (int m = 0; m < d; ++m) gx += k.At[(size_t)i * d + m] * ws[m];
            break;
          }
          case HJ_FAMILY_EIKONAL: {
            const double r1 = qn > 0.0 ? dx - delta * ec * qs[i] / qn
                                       : dx * fmax(0.0, 1.0 - delta * ec / (dn > 0.0 ? dn : 1.0));
            r = max_nan(r, fabs(r1));
            const double cb = k.xb[i] + (k.vb ? sj * k.vb[i] : 0.0);
            gx = qn * egf * (xs[i] - cb);
            break;
          }
          default:
            break;
        }
        if (j < N) {
          const double qr = k.sign * (double)pb_[(size_t)(j + 1) * d + i];
          r = max_nan(r, fabs(qr - qs[i] + delta * gx));
        }
      }
    }
    r = block_max(r, red);
    if (threadIdx.x == 0) k.kkt[b] = r;
  }
}

}  // namespace

// Families the residual is defined for here (the control families and the
// eikonal family; the game has two players' equations and is not covered).
bool kkt_family_supported(int family) {
  return family == HJ_FAMILY_QUADRATIC || family == HJ_FAMILY_QUADCOPTER ||
         family == HJ_FAMILY_TANH_DRIFT || family == HJ_FAMILY_EIKONAL;
}

hj_status launch_kkt(const hj_problem_s* p, int64_t B, int32_t N, bool fp64, const double* t,
                     const void* traj_x, const void* traj_p, double* kkt, cudaStream_t s) {
  if (!kkt_family_supported(p->family)) return HJ_ERR_UNSUPPORTED;
  if (B == 0) return HJ_OK;
  {
    const hj_status r =
        fp64 ? launch_kkt_nodes<double>(p, B, N, t, static_cast<const double*>(traj_x),
                                        static_cast<const double*>(traj_p), kkt, s)
             : launch_kkt_nodes<float>(p, B, N, t, static_cast<const float*>(traj_x),
                                       static_cast<const float*>(traj_p), kkt, s);
    if (r != HJ_ERR_UNSUPPORTED) return r;
  }
  KktArgs k{};
  k.B = B; k.N = N; k.d = p->d; k.family = p->family; k.t = t;
  k.W2 = p->W2; k.c = p->c; k.A = p->Ad; k.At = p->Atd;
  k.qc_m = p->qc[0]; k.qc_ah = p->qc[1]; k.qc_gz = p->qc[2]; k.qc_eps = p->qc[3];
  k.sign = (p->family == HJ_FAMILY_EIKONAL && p->eik[0] < 0) ? -1.0 : 1.0;
  k.c0 = p->eik[1]; k.c1 = p->eik[2]; k.c2 = p->eik[3];
  k.xb = p->xbd; k.vb = p->eik_moving ? p->vbd : nullptr;
  k.kkt = kkt;
  const size_t smem = (3 * (size_t)p->d + kKktThreads / 32) * sizeof(double);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HJ_ERR_CUDA;
  const int64_t cap = (int64_t)nsm * 16;
  const int grid = (int)(B < cap ? B : cap);
  if (fp64) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kkt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return HJ_ERR_CUDA;
    kkt_kernel<double><<<grid, kKktThreads, smem, s>>>(k, static_cast<const double*>(traj_x),
                                                       static_cast<const double*>(traj_p));
  } else {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kkt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return HJ_ERR_CUDA;
    kkt_kernel<float><<<grid, kKktThreads, smem, s>>>(k, static_cast<const float*>(traj_x),
                                                      static_cast<const float*>(traj_p));
  }
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

}  // namespace hj

extern "C" hj_status hj_kkt_residual(hj_problem prob, int64_t B, const double* t, int32_t N,
                                     int32_t precision, const void* traj_x, const void* traj_p,
                                     double* kkt, void* stream) {
  if (prob == nullptr || B < 0 || N < 1 || N > hj::kMaxN) return HJ_ERR_INVALID_ARG;
  if (precision != HJ_PREC_FP32 && precision != HJ_PREC_FP64) return HJ_ERR_INVALID_ARG;
  if (!hj::kkt_family_supported(prob->family)) return HJ_ERR_UNSUPPORTED;
  if (B == 0) return HJ_OK;
  if (t == nullptr || traj_x == nullptr || traj_p == nullptr || kkt == nullptr)
    return HJ_ERR_INVALID_ARG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return HJ_ERR_CUDA;
  if (cur != prob->device) return HJ_ERR_INVALID_ARG;
  return hj::launch_kkt(prob, B, N, precision == HJ_PREC_FP64, t, traj_x, traj_p, kkt,
                        reinterpret_cast<cudaStream_t>(stream));
}

// Gradient of L = sum_b w_b V_b with respect to the cost weights W, the cost
// centre c, the dynamics parameters and the query points, evaluated at solved
// trajectories.
//
// At a saddle (x*, p*) of the Lagrangian of Eq. (disclaxBE),
//   V(theta) = g(x_0; W, c) + sum_j <p_j, x_j - x_{j-1}> - delta sum_j H(x_j, p_j; theta),
// the stationarity conditions make every total derivative equal the partial
// one (envelope theorem), so with e = x_0 - c:
//   dV/dW_i     = W_i e_i^2              dV/dc_i = -W_i^2 e_i
//   dV/dtheta   = -delta sum_{j=1}^N dH/dtheta(x_j, p_j)
//   dV/dx_q     = p_N - delta grad_x H(x_N, p_N)        (x_N = x_q is pinned)
// Per-node arithmetic runs in the trajectory's type; every sum over nodes,
// points and the batch is accumulated in FP64.
// Eikonal family (V = s V_int, V_int the positive equation's value for the
// data s g, returned p = s p_int): H = c(x_j - s_j v_b)|p_j|, so with
// e_j = exp(-c2 r_j^2), r_j = |x_j - x_b - s_j v_b| and a_j = 2 c1 c2 e_j |p_j|,
//   dV/d(c0, c1, c2) = -s delta sum_j |p_j| (1, e_j, -c1 r_j^2 e_j),
//   dV/dx_b = -s delta sum_j a_j (x_j - x_b - s_j v_b),   dV/dv_b: the same times s_j,
//   dV/dx_q = p_N + s delta a_N (x_N - x_b - t v_b);
// W and c keep the formulas above (the sign enters g and V alike).
#include <cuda_runtime.h>

#include "families.cuh"
#include "hj_internal.cuh"
#include "hjpdhg.h"

namespace hj {

template <typename T>
__device__ __forceinline__ void qc_dir(T psi, T th, T ph, T (&a)[3], T (&J)[9]) {
  FamQuadcopter<T, 12>::template thrust<T>(psi, th, ph, a, J);
}

// family 0: quadratic, 1: quadcopter, 2: tanh drift, 3: eikonal
template <typename T, int FAM>
__global__ void __launch_bounds__(256) value_grad_kernel(const GradArgs<T> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int d = g.d, N = g.N, nthr = blockDim.x, tid = threadIdx.x;
  double* acc_W = reinterpret_cast<double*>(smem_raw);     // [d]
  double* acc_c = acc_W + d;                               // [d]
  double* acc_dyn = acc_c + d;                             // [n_dyn]
  T* sA = reinterpret_cast<T*>(acc_dyn + g.n_dyn);         // tanh drift: [d][d]
  T* su = sA + (FAM == 2 ? d * d : 0);                     // tanh drift: [d]
  T* sx = su + (FAM == 2 ? d : 0);                         // tanh drift: [d]
  double* nodeA = reinterpret_cast<double*>(acc_dyn + g.n_dyn);   // eikonal: [N + 1] a_j
  for (int e = tid; e < 2 * d + g.n_dyn; e += nthr) acc_W[e] = 0.0;
  if (FAM == 2)
    for (int e = tid; e < d * d; e += nthr) sA[e] = g.A[e];
  __syncthreads();

  constexpr int kPairs = 64;            // tanh drift: (i, k) pairs per thread, d*d <= 64 * 256
  for (int64_t b = blockIdx.x; b < g.B; b += gridDim.x) {
    const double wb = g.w[b];
    const double delta = g.t[b] / N;
    const T* X = g.X + (size_t)b * (N + 1) * d;
    const T* P = g.P + (size_t)b * (N + 1) * d;
    for (int i = tid; i < d; i += nthr) {
      const double e = (double)X[i] - g.c[i];
      acc_W[i] += wb * g.W[i] * e * e;
      acc_c[i] += -wb * g.W2[i] * e;
    }
    if (FAM == 0) {
      if (g.dxq != nullptr)
        for (int i = tid; i < d; i += nthr) g.dxq[b * d + i] = wb * (double)P[(size_t)N * d + i];
    } else if (FAM == 1) {
      // dH/d(m, a_h, g_z, eps) per node, summed over nodes in FP64
      double s_m = 0.0, s_ah = 0.0, s_gz = 0.0, s_eps = 0.0;
      const T minv = T(1.0 / g.qc_m);
      for (int j = 1 + tid; j <= N; j += nthr) {
        const T* x = X + (size_t)j * d;
        const T* p = P + (size_t)j * d;
        T a[3], J[9];
        qc_dir<T>(x[3], x[4], x[5], a, J);
        const T s = a[0] * p[6] + a[1] * p[7] + a[2] * p[8];
        const T u0 = s * minv;
        T pp = T(0);
        for (int k = 0; k < 12; ++k) pp += p[k] * p[k];
        s_m += -(double)(u0 * u0 * minv);
        s_ah += (double)s;
        s_gz += -(double)p[8];
        s_eps += 0.5 * (double)pp;
      }
      s_m = warp_sum<double>(s_m); s_ah = warp_sum<double>(s_ah);
      s_gz = warp_sum<double>(s_gz); s_eps = warp_sum<double>(s_eps);
      if ((tid & 31) == 0) {
        atomicAdd(&acc_dyn[0], -wb * delta * s_m);
        atomicAdd(&acc_dyn[1], -wb * delta * s_ah);
        atomicAdd(&acc_dyn[2], -wb * delta * s_gz);
        atomicAdd(&acc_dyn[3], -wb * delta * s_eps);
      }
      if (g.dxq != nullptr && tid == 0) {
        const T* x = X + (size_t)N * d;
        const T* p = P + (size_t)N * d;
        T a[3], J[9];
        qc_dir<T>(x[3], x[4], x[5], a, J);
        const T u0 = (a[0] * p[6] + a[1] * p[7] + a[2] * p[8]) * minv;
        const T coef = T(g.qc_ah) + u0 * minv;
        double gx[12];
        for (int k = 0; k < 3; ++k) gx[k] = 0.0;
        for (int k = 0; k < 3; ++k)
          gx[3 + k] = (double)(coef * (J[k] * p[6] + J[3 + k] * p[7] + J[6 + k] * p[8]));
        for (int k = 0; k < 3; ++k) gx[6 + k] = (double)p[k];
        for (int k = 0; k < 3; ++k) gx[9 + k] = (double)p[3 + k];
        for (int k = 0; k < 12; ++k) g.dxq[b * d + k] = wb * ((double)p[k] - delta * gx[k]);
      }
    } else if (FAM == 3) {
      // node scalars |p_j|, e_j, r_j^2 (threads over nodes), then the x_b and v_b
      // sums (threads over coordinates)
      const double sgn = g.cost_sign, c1 = g.eik_c1, c2 = g.eik_c2;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int j = 1 + tid; j <= N; j += nthr) {
        const double sj = j * delta;
        double r2 = 0.0, n2 = 0.0;
        for (int k = 0; k < d; ++k) {
          const double ctr = g.xb64[k] + (g.vb64 ? sj * g.vb64[k] : 0.0);
          const double y = (double)X[(size_t)j * d + k] - ctr;
          const double pk = (double)P[(size_t)j * d + k];
          r2 += y * y;
          n2 += pk * pk;
        }
        const double e = exp(-c2 * r2), np = sqrt(n2);
        s0 += np;
        s1 += np * e;
        s2 += -c1 * r2 * e * np;
        nodeA[j] = 2.0 * c1 * c2 * e * np;
      }
      s0 = warp_sum<double>(s0); s1 = warp_sum<double>(s1); s2 = warp_sum<double>(s2);
      if ((tid & 31) == 0) {
        atomicAdd(&acc_dyn[1], -sgn * wb * delta * s0);
        atomicAdd(&acc_dyn[2], -sgn * wb * delta * s1);
        atomicAdd(&acc_dyn[3], -sgn * wb * delta * s2);
      }
      __syncthreads();
      for (int k = tid; k < d; k += nthr) {
        double sb = 0.0, sv = 0.0;
        for (int j = 1; j <= N; ++j) {
          const double sj = j * delta;
          const double ctr = g.xb64[k] + (g.vb64 ? sj * g.vb64[k] : 0.0);
          const double term = nodeA[j] * ((double)X[(size_t)j * d + k] - ctr);
          sb += term;
          sv += term * sj;
        }
        acc_dyn[4 + k] += -sgn * wb * delta * sb;
        if (g.vb64) acc_dyn[4 + d + k] += -sgn * wb * delta * sv;
        if (g.dxq != nullptr) {
          const double ctr = g.xb64[k] + (g.vb64 ? N * delta * g.vb64[k] : 0.0);
          g.dxq[b * d + k] = wb * ((double)P[(size_t)N * d + k] +
                                   sgn * delta * nodeA[N] * ((double)X[(size_t)N * d + k] - ctr));
        }
      }
      __syncthreads();                             // nodeA is rewritten for the next point
    } else {
      // dH/dA_ik = u_i x_k with u = p * (1 - tanh(A x)^2); node sums in T, point sum in FP64
      T part[kPairs];
#pragma unroll
      for (int q = 0; q < kPairs; ++q) part[q] = T(0);
      for (int j = 1; j <= N; ++j) {
        __syncthreads();
        for (int i = tid; i < d; i += nthr) sx[i] = X[(size_t)j * d + i];
        __syncthreads();
        for (int i = tid; i < d; i += nthr) {
          T y = T(0);
          for (int k = 0; k < d; ++k) y += sA[i * d + k] * sx[k];
          const T th = tanh(y);
          su[i] = P[(size_t)j * d + i] * (T(1) - th * th);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPairs; ++q) {
          const int e = tid + q * nthr;
          if (e < d * d) part[q] += su[e / d] * sx[e % d];
        }
        if (j == N && g.dxq != nullptr) {
          // dV/dx_q = p_N - delta A^T u_N
          for (int k = tid; k < d; k += nthr) {
            T s = T(0);
            for (int i = 0; i < d; ++i) s += sA[i * d + k] * su[i];
            g.dxq[b * d + k] = wb * ((double)P[(size_t)N * d + k] - delta * (double)s);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kPairs; ++q) {
        const int e = tid + q * nthr;
        if (e < d * d) acc_dyn[e] += -wb * delta * (double)part[q];
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < d; i += nthr) {
    atomicAdd(&g.dW[i], acc_W[i]);
    atomicAdd(&g.dc[i], acc_c[i]);
  }
  for (int e = tid; e < g.n_dyn; e += nthr) atomicAdd(&g.ddyn[e], acc_dyn[e]);
}

template <typename T>
hj_status launch_value_grad(int family, const GradArgs<T>& g, cudaStream_t s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HJ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HJ_ERR_CUDA;
  const size_t smem = (size_t)(2 * g.d + g.n_dyn) * sizeof(double) +
                      (family == HJ_FAMILY_TANH_DRIFT ? (size_t)(g.d * g.d + 2 * g.d) * sizeof(T) : 0) +
                      (family == HJ_FAMILY_EIKONAL ? (size_t)(g.N + 1) * sizeof(double) : 0);
  if (smem > 227u * 1024u) return HJ_ERR_UNSUPPORTED;
  const int64_t grid64 = g.B < (int64_t)nsm * 2 ? g.B : (int64_t)nsm * 2;
  const int grid = (int)(grid64 > 0 ? grid64 : 1);
  const int threads = family == HJ_FAMILY_TANH_DRIFT ? 256 : 64;
  cudaError_t e = cudaSuccess;
  switch (family) {
    case HJ_FAMILY_QUADRATIC:
      value_grad_kernel<T, 0><<<grid, threads, smem, s>>>(g);
      break;
    case HJ_FAMILY_QUADCOPTER:
      value_grad_kernel<T, 1><<<grid, threads, smem, s>>>(g);
      break;
    case HJ_FAMILY_TANH_DRIFT:
      if (g.d * g.d > 64 * 256) return HJ_ERR_UNSUPPORTED;
      e = cudaFuncSetAttribute(value_grad_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return HJ_ERR_CUDA;
      value_grad_kernel<T, 2><<<grid, threads, smem, s>>>(g);
      break;
    case HJ_FAMILY_EIKONAL:
      e = cudaFuncSetAttribute(value_grad_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return HJ_ERR_CUDA;
      value_grad_kernel<T, 3><<<grid, threads, smem, s>>>(g);
      break;
    default:
      return HJ_ERR_UNSUPPORTED;
  }
  return cudaGetLastError() == cudaSuccess ? HJ_OK : HJ_ERR_CUDA;
}

template hj_status launch_value_grad<float>(int, const GradArgs<float>&, cudaStream_t);
template hj_status launch_value_grad<double>(int, const GradArgs<double>&, cudaStream_t);

}  // namespace hj

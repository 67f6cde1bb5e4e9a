// Linear spatiotemporal theory of the paper (Eq. 5) marched on the GPU, batched over transverse
// modes: the procedure behind the paper's Fig. 1e growth curves.  See include/qsa.h
// (qsa_eq5_march) for the contract.
//
// Per mode, Eq. 5 reads (d_xi^2 + 1) d_tau^2 psi = Gamma^2 psi.  With zero data ahead of the
// beam front (xi < 0), d_tau^2 psi = V[psi] = Gamma^2 int_0^xi sin(xi - xi') psi(xi') dxi', and
// sin(xi - xi') = sin xi cos xi' - cos xi sin xi' turns the integral into two prefix sums:
//   V_i = Gamma^2 (sin xi_i A_i - cos xi_i B_i),  A_i = int_0^xi_i cos psi,  B_i = int_0^xi_i sin psi
// (trapezoid rule on the uniform grid xi_i = i dxi).  The state (psi, d_tau psi) advances by
// classical RK4 in tau.
//
// Layout: one block of 256 threads per mode; thread t owns the EPT consecutive grid points
// t EPT .. t EPT + EPT - 1 in registers (FP64), so a prefix sum is a per-thread serial sum plus
// one block-wide exclusive scan of the thread totals (warp shuffles, then one warp over the
// warp totals).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/qsa.h"

namespace qsa {
void set_global_error(const std::string& msg);
}

namespace {

constexpr int kEq5Threads = 256;
constexpr int kEq5Points = 8;  // grid points per thread: n_xi <= 256 x 8 = QSA_EQ5_MAX_XI
static_assert(kEq5Threads * kEq5Points == QSA_EQ5_MAX_XI, "grid capacity");

struct D2 {
  double a, b;
};

__device__ __forceinline__ D2 shfl_up2(D2 v, int o) {
  return D2{__shfl_up_sync(0xffffffffu, v.a, o), __shfl_up_sync(0xffffffffu, v.b, o)};
}

// Exclusive block scan of (a, b) over the threads in index order; scratch >= 2 * 8 doubles.
__device__ D2 block_exclusive_scan(D2 v, double* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  D2 inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const D2 u = shfl_up2(inc, o);
    if (lane >= o) {
      inc.a += u.a;
      inc.b += u.b;
    }
  }
  __syncthreads();  // scratch of the previous call is no longer read
  if (lane == 31) {
    scratch[2 * w] = inc.a;
    scratch[2 * w + 1] = inc.b;
  }
  __syncthreads();
  if (w == 0) {
    D2 t = lane < nw ? D2{scratch[2 * lane], scratch[2 * lane + 1]} : D2{0.0, 0.0};
    for (int o = 1; o < 32; o <<= 1) {
      const D2 u = shfl_up2(t, o);
      if (lane >= o) {
        t.a += u.a;
        t.b += u.b;
      }
    }
    if (lane < nw) {  // exclusive prefix of the warp totals
      scratch[2 * lane] = t.a - scratch[2 * lane];
      scratch[2 * lane + 1] = t.b - scratch[2 * lane + 1];
    }
  }
  __syncthreads();
  return D2{scratch[2 * w] + inc.a - v.a, scratch[2 * w + 1] + inc.b - v.b};
}

// V[y] on the thread's points (see the file comment); y0sh receives y at xi = 0 (cos 0 = 1,
// sin 0 = 0) from thread 0.  Consecutive calls must alternate between two y0sh slots: a slot
// is rewritten only after the next call's barriers, when every thread has read it.
template <int EPT>
__device__ void eval_V(const double (&y)[EPT], const double (&c)[EPT], const double (&s)[EPT],
                       int i0, int n, double dxi, double g2, double* scratch, double* y0sh,
                       double (&V)[EPT]) {
  double ga[EPT], gb[EPT];
  D2 tot{0.0, 0.0};
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const bool in = i0 + e < n;
    tot.a += in ? c[e] * y[e] : 0.0;
    tot.b += in ? s[e] * y[e] : 0.0;
    ga[e] = tot.a;  // inclusive prefix within the thread
    gb[e] = tot.b;
  }
  if (threadIdx.x == 0) *y0sh = y[0];
  const D2 off = block_exclusive_scan(tot, scratch);  // its barriers publish *y0sh
  const double g0 = *y0sh;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    // trapezoid: int_0^xi_i f = dxi (sum_{m<=i} f_m - (f_0 + f_i) / 2), f = cos psi, sin psi
    const double A = dxi * (off.a + ga[e] - 0.5 * (g0 + c[e] * y[e]));
    const double B = dxi * (off.b + gb[e] - 0.5 * (0.0 + s[e] * y[e]));
    V[e] = g2 * (s[e] * A - c[e] * B);
  }
}

template <int EPT>
__global__ void __launch_bounds__(kEq5Threads) eq5_kernel(int n, double dxi,
                                                          const double* __restrict__ gamma,
                                                          const double* __restrict__ psi0,
                                                          const double* __restrict__ dpsi0,
                                                          double h, int n_tau, int every,
                                                          double* __restrict__ out, int nm) {
  __shared__ double scratch[2 * 32];
  __shared__ double y0sh[2];
  const int m = blockIdx.x;
  const int i0 = threadIdx.x * EPT;
  const double g2 = gamma[m] * gamma[m];
  double c[EPT], s[EPT], y[EPT], v[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = i0 + e;
    const bool in = i < n;
    sincos((double)i * dxi, &s[e], &c[e]);
    y[e] = in ? psi0[(size_t)m * n + i] : 0.0;
    v[e] = in ? dpsi0[(size_t)m * n + i] : 0.0;
  }
  int call = 0;
  for (int step = 1; step <= n_tau; ++step) {
    double ap[EPT], av[EPT], t[EPT], K[EPT];
    // stage 1: k1p = v, k1v = V(y)
    eval_V<EPT>(y, c, s, i0, n, dxi, g2, scratch, &y0sh[(call++) & 1], K);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      ap[e] = v[e];
      av[e] = K[e];
      t[e] = y[e] + 0.5 * h * v[e];  // y + h/2 k1p
    }
    // stage 2: k2p = v + h/2 k1v, k2v = V(y + h/2 k1p)
    double kp[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) kp[e] = v[e] + 0.5 * h * K[e];
    eval_V<EPT>(t, c, s, i0, n, dxi, g2, scratch, &y0sh[(call++) & 1], K);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      ap[e] += 2.0 * kp[e];
      av[e] += 2.0 * K[e];
      t[e] = y[e] + 0.5 * h * kp[e];  // y + h/2 k2p
      kp[e] = v[e] + 0.5 * h * K[e];  // k3p
    }
    // stage 3: k3v = V(y + h/2 k2p)
    eval_V<EPT>(t, c, s, i0, n, dxi, g2, scratch, &y0sh[(call++) & 1], K);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      ap[e] += 2.0 * kp[e];
      av[e] += 2.0 * K[e];
      t[e] = y[e] + h * kp[e];  // y + h k3p
      kp[e] = v[e] + h * K[e];  // k4p
    }
    // stage 4: k4v = V(y + h k3p)
    eval_V<EPT>(t, c, s, i0, n, dxi, g2, scratch, &y0sh[(call++) & 1], K);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      ap[e] += kp[e];
      av[e] += K[e];
      y[e] += h / 6.0 * ap[e];
      v[e] += h / 6.0 * av[e];
    }
    if (step % every == 0) {
      double* o = out + ((size_t)(step / every - 1) * nm + m) * n;
#pragma unroll
      for (int e = 0; e < EPT; ++e)
        if (i0 + e < n) o[i0 + e] = y[e];
    }
  }
}

int fail(int code, const std::string& msg) {
  qsa::set_global_error("qsa_eq5_march: " + msg);
  return code;
}

}  // namespace

extern "C" int qsa_eq5_march(int32_t n_modes, int32_t n_xi, double dxi, const double* gamma,
                             const double* psi0, const double* dpsi0, double tau_end,
                             int32_t n_tau, int32_t n_out, double* psi_out, void* stream) {
  if (n_modes < 1 || n_xi < 2 || n_xi > QSA_EQ5_MAX_XI)
    return fail(QSA_ERR_ARG, "need n_modes >= 1 and 2 <= n_xi <= 2048");
  if (!(dxi > 0) || !(tau_end >= 0) || n_tau < 1 || n_out < 1 || n_tau % n_out != 0)
    return fail(QSA_ERR_ARG, "need dxi > 0, tau_end >= 0, n_tau >= 1, n_out | n_tau");
  if (!gamma || !psi0 || !dpsi0 || !psi_out) return fail(QSA_ERR_ARG, "NULL array");
  for (int m = 0; m < n_modes; ++m)
    if (!(gamma[m] >= 0)) return fail(QSA_ERR_ARG, "Gamma must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nm = (size_t)n_modes, nx = (size_t)n_xi;
  double *dg = nullptr, *dp = nullptr, *dv = nullptr, *dout = nullptr;
  auto release = [&]() {
    if (dg) cudaFreeAsync(dg, st);
    if (dp) cudaFreeAsync(dp, st);
    if (dv) cudaFreeAsync(dv, st);
    if (dout) cudaFreeAsync(dout, st);
    cudaStreamSynchronize(st);
  };
  auto cuda_err = [&](cudaError_t e, const char* what) {
    release();
    return fail(QSA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaMallocAsync((void**)&dg, nm * sizeof(double), st)) != cudaSuccess ||
      (e = cudaMallocAsync((void**)&dp, nm * nx * sizeof(double), st)) != cudaSuccess ||
      (e = cudaMallocAsync((void**)&dv, nm * nx * sizeof(double), st)) != cudaSuccess ||
      (e = cudaMallocAsync((void**)&dout, (size_t)n_out * nm * nx * sizeof(double), st)) !=
          cudaSuccess)
    return cuda_err(e, "allocation");
  if ((e = cudaMemcpyAsync(dg, gamma, nm * sizeof(double), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(dp, psi0, nm * nx * sizeof(double), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(dv, dpsi0, nm * nx * sizeof(double), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess)
    return cuda_err(e, "copy in");
  const double h = tau_end / n_tau;
  const int every = n_tau / n_out;
  eq5_kernel<kEq5Points><<<n_modes, kEq5Threads, 0, st>>>(n_xi, dxi, dg, dp, dv, h, n_tau,
                                                           every, dout, n_modes);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "launch");
  if ((e = cudaMemcpyAsync(psi_out, dout, (size_t)n_out * nm * nx * sizeof(double),
                           cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_err(e, "copy out");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_err(e, "kernel");
  release();
  return QSA_OK;
}

// Spectral helpers of the learned subgrid-stress closure (standalone kernels on
// caller-owned device arrays; spectral arrays use the public layout
// (c, N, N, N/2+1) [c][kx][ky][kz], kx and ky in FFT order):
//   box filter of width 2 pi/Nc + truncation to |k_i| < Nc/2 of an Nc^3 grid,
//   velocity gradients i k_j u_hat_i, pointwise products u_i u_j, the stress
//   tau_ij = filter(u_i u_j) - ubar_i ubar_j and its force -i k_j tau_hat_ij.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/dns.h"
#include "dns_internal.h"
#include "fft_core.cuh"

namespace dns {
void set_error_message(const char* msg);
}

namespace {

using dns::cx;
using dns::mk;

constexpr int SGS_THREADS = 256;

__device__ __forceinline__ int fftk(int i, int N) { return i < N / 2 ? i : i - N; }
__device__ __forceinline__ double sincd(double x) { return fabs(x) < 1e-12 ? 1.0 : sin(x) / x; }

template <typename T>
__global__ void k_filter_truncate(const cx<T>* __restrict__ fine, int Nf, cx<T>* __restrict__ coarse, int Nc,
                                  double scale, double half_width) {
  const int M1c = Nc / 2 + 1, M1f = Nf / 2 + 1;
  const size_t per = (size_t)Nc * Nc * M1c;
  for (size_t i = blockIdx.x * (size_t)SGS_THREADS + threadIdx.x; i < 3 * per; i += (size_t)gridDim.x * SGS_THREADS) {
    const int c = (int)(i / per);
    const size_t r = i % per;
    const int kz = (int)(r % M1c), b = (int)((r / M1c) % Nc), a = (int)(r / ((size_t)M1c * Nc));
    const int kx = fftk(a, Nc), ky = fftk(b, Nc);
    cx<T> v = mk((T)0, (T)0);
    if (2 * abs(kx) < Nc && 2 * abs(ky) < Nc && 2 * kz < Nc) {
      const double g = sincd(kx * half_width) * sincd(ky * half_width) * sincd(kz * half_width) * scale;
      const int af = (kx + Nf) % Nf, bf = (ky + Nf) % Nf;
      const cx<T> u = fine[((size_t)c * Nf * Nf + (size_t)af * Nf + bf) * M1f + kz];
      v = mk((T)(g * (double)u.x), (T)(g * (double)u.y));
    }
    coarse[i] = v;
  }
}

template <typename T>
__global__ void k_gradient(const cx<T>* __restrict__ uh, int N, cx<T>* __restrict__ g9) {
  const int M1 = N / 2 + 1;
  const size_t per = (size_t)N * N * M1;
  for (size_t i = blockIdx.x * (size_t)SGS_THREADS + threadIdx.x; i < per; i += (size_t)gridDim.x * SGS_THREADS) {
    const int kz = (int)(i % M1), b = (int)((i / M1) % N), a = (int)(i / ((size_t)M1 * N));
    const T k[3] = {(T)fftk(a, N), (T)fftk(b, N), (T)kz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cx<T> u = uh[c * per + i];
#pragma unroll
      for (int j = 0; j < 3; ++j) g9[(3 * c + j) * per + i] = mk(-k[j] * u.y, k[j] * u.x);  // i k_j u
    }
  }
}

template <typename T>
__global__ void k_stress_force(const cx<T>* __restrict__ th, int N, cx<T>* __restrict__ f3) {
  const int M1 = N / 2 + 1;
  const size_t per = (size_t)N * N * M1;
  // (i, j) -> stress component: 00 0, 11 1, 22 2, 01 3, 02 4, 12 5
  const int idx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  for (size_t i = blockIdx.x * (size_t)SGS_THREADS + threadIdx.x; i < per; i += (size_t)gridDim.x * SGS_THREADS) {
    const int kz = (int)(i % M1), b = (int)((i / M1) % N), a = (int)(i / ((size_t)M1 * N));
    const T k[3] = {(T)fftk(a, N), (T)fftk(b, N), (T)kz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T re = 0, im = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const cx<T> t = th[idx[c][j] * per + i];
        re += k[j] * t.y;  // -i k t = k t.y - i k t.x
        im -= k[j] * t.x;
      }
      f3[c * per + i] = mk(re, im);
    }
  }
}

template <typename T>
__global__ void k_products(const T* __restrict__ u3, size_t n3, T* __restrict__ p6) {
  for (size_t i = blockIdx.x * (size_t)SGS_THREADS + threadIdx.x; i < n3; i += (size_t)gridDim.x * SGS_THREADS) {
    const T a = u3[i], b = u3[n3 + i], c = u3[2 * n3 + i];
    p6[i] = a * a;
    p6[n3 + i] = b * b;
    p6[2 * n3 + i] = c * c;
    p6[3 * n3 + i] = a * b;
    p6[4 * n3 + i] = a * c;
    p6[5 * n3 + i] = b * c;
  }
}

template <typename T>
__global__ void k_sub_products(T* __restrict__ tau6, const T* __restrict__ ub3, size_t n3) {
  for (size_t i = blockIdx.x * (size_t)SGS_THREADS + threadIdx.x; i < n3; i += (size_t)gridDim.x * SGS_THREADS) {
    const T a = ub3[i], b = ub3[n3 + i], c = ub3[2 * n3 + i];
    tau6[i] -= a * a;
    tau6[n3 + i] -= b * b;
    tau6[2 * n3 + i] -= c * c;
    tau6[3 * n3 + i] -= a * b;
    tau6[4 * n3 + i] -= a * c;
    tau6[5 * n3 + i] -= b * c;
  }
}

int grid_for(size_t n) {
  size_t b = (n + SGS_THREADS - 1) / SGS_THREADS;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

int bad(const char* msg) {
  dns::set_error_message(msg);
  return DNS_ERR_ARG;
}

int launched(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    dns::set_error_message(where);
    return DNS_ERR_CUDA;
  }
  return DNS_OK;
}

bool ok_n(int N) { return N >= 2 && N % 2 == 0 && N <= 4096; }

// ---------------------------------------------------------------------------
// The same gradient and force on the solver's internal spectral layout
// [c][kz][ky][kx] (kz < N/2, kx and ky in FFT order), used by the closure the
// solver evaluates inside its step (dns_set_closure). The arithmetic of every
// mode is that of k_gradient and k_stress_force.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_grad_internal(const cx<T>* __restrict__ U, int N, int comp, cx<T>* __restrict__ G3) {
  const size_t per = (size_t)(N / 2) * N * N;
  for (size_t i = blockIdx.x * (size_t)SGS_THREADS + threadIdx.x; i < per; i += (size_t)gridDim.x * SGS_THREADS) {
    const int kx = (int)(i % N), ky = (int)((i / N) % N), kz = (int)(i / ((size_t)N * N));
    const T k[3] = {(T)fftk(kx, N), (T)fftk(ky, N), (T)kz};
    const cx<T> u = U[comp * per + i];
#pragma unroll
    for (int j = 0; j < 3; ++j) G3[j * per + i] = mk(-k[j] * u.y, k[j] * u.x);  // i k_j u
  }
}

template <typename T>
__global__ void k_force_internal(const cx<T>* __restrict__ th, int N, cx<T>* __restrict__ f3) {
  const size_t per = (size_t)(N / 2) * N * N;
  const int idx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  for (size_t i = blockIdx.x * (size_t)SGS_THREADS + threadIdx.x; i < per; i += (size_t)gridDim.x * SGS_THREADS) {
    const int kx = (int)(i % N), ky = (int)((i / N) % N), kz = (int)(i / ((size_t)N * N));
    const T k[3] = {(T)fftk(kx, N), (T)fftk(ky, N), (T)kz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T re = 0, im = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const cx<T> t = th[idx[c][j] * per + i];
        re += k[j] * t.y;  // -i k t = k t.y - i k t.x
        im -= k[j] * t.x;
      }
      f3[c * per + i] = mk(re, im);
    }
  }
}

__global__ void k_fill_f32(float* __restrict__ p, size_t n, float v) {
  for (size_t i = blockIdx.x * (size_t)SGS_THREADS + threadIdx.x; i < n; i += (size_t)gridDim.x * SGS_THREADS) p[i] = v;
}

}  // namespace

namespace dns {

cudaError_t closure_gradient(const void* U, int N, int comp, void* G3, int dtype, cudaStream_t st) {
  const size_t n = (size_t)(N / 2) * N * N;
  if (dtype == DNS_F32)
    k_grad_internal<float><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<float>*)U, N, comp, (cx<float>*)G3);
  else
    k_grad_internal<double><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<double>*)U, N, comp, (cx<double>*)G3);
  return cudaGetLastError();
}

cudaError_t closure_force(const void* S6, int N, void* F3, int dtype, cudaStream_t st) {
  const size_t n = (size_t)(N / 2) * N * N;
  if (dtype == DNS_F32)
    k_force_internal<float><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<float>*)S6, N, (cx<float>*)F3);
  else
    k_force_internal<double><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<double>*)S6, N, (cx<double>*)F3);
  return cudaGetLastError();
}

cudaError_t fill_f32(float* p, size_t n, float v, cudaStream_t st) {
  k_fill_f32<<<grid_for(n), SGS_THREADS, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

}  // namespace dns

extern "C" {

int dns_spectral_filter(const void* fine, int Nf, void* coarse, int Nc, int dtype, void* stream) {
  if (!fine || !coarse || !ok_n(Nf) || !ok_n(Nc) || Nc > Nf || (dtype != DNS_F32 && dtype != DNS_F64))
    return bad("dns_spectral_filter: bad arguments (need device arrays, even Nc <= Nf)");
  const double scale = std::pow((double)Nc / (double)Nf, 3.0), hw = 3.14159265358979323846 / Nc;
  const size_t n = 3ull * Nc * Nc * (Nc / 2 + 1);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == DNS_F32)
    k_filter_truncate<float><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<float>*)fine, Nf, (cx<float>*)coarse, Nc,
                                                                  scale, hw);
  else
    k_filter_truncate<double><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<double>*)fine, Nf, (cx<double>*)coarse,
                                                                   Nc, scale, hw);
  return launched("dns_spectral_filter: launch failed");
}

int dns_spectral_gradient(const void* uhat3, int N, void* grad9, int dtype, void* stream) {
  if (!uhat3 || !grad9 || !ok_n(N) || (dtype != DNS_F32 && dtype != DNS_F64))
    return bad("dns_spectral_gradient: bad arguments");
  const size_t n = (size_t)N * N * (N / 2 + 1);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == DNS_F32)
    k_gradient<float><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<float>*)uhat3, N, (cx<float>*)grad9);
  else
    k_gradient<double><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<double>*)uhat3, N, (cx<double>*)grad9);
  return launched("dns_spectral_gradient: launch failed");
}

int dns_stress_force(const void* tauhat6, int N, void* force3, int dtype, void* stream) {
  if (!tauhat6 || !force3 || !ok_n(N) || (dtype != DNS_F32 && dtype != DNS_F64))
    return bad("dns_stress_force: bad arguments");
  const size_t n = (size_t)N * N * (N / 2 + 1);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == DNS_F32)
    k_stress_force<float><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<float>*)tauhat6, N, (cx<float>*)force3);
  else
    k_stress_force<double><<<grid_for(n), SGS_THREADS, 0, st>>>((const cx<double>*)tauhat6, N, (cx<double>*)force3);
  return launched("dns_stress_force: launch failed");
}

int dns_pointwise_products(const void* u3, int N, void* prod6, int dtype, void* stream) {
  if (!u3 || !prod6 || !ok_n(N) || (dtype != DNS_F32 && dtype != DNS_F64))
    return bad("dns_pointwise_products: bad arguments");
  const size_t n3 = (size_t)N * N * N;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == DNS_F32)
    k_products<float><<<grid_for(n3), SGS_THREADS, 0, st>>>((const float*)u3, n3, (float*)prod6);
  else
    k_products<double><<<grid_for(n3), SGS_THREADS, 0, st>>>((const double*)u3, n3, (double*)prod6);
  return launched("dns_pointwise_products: launch failed");
}

int dns_subtract_products(void* tau6, const void* ubar3, int N, int dtype, void* stream) {
  if (!tau6 || !ubar3 || !ok_n(N) || (dtype != DNS_F32 && dtype != DNS_F64))
    return bad("dns_subtract_products: bad arguments");
  const size_t n3 = (size_t)N * N * N;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == DNS_F32)
    k_sub_products<float><<<grid_for(n3), SGS_THREADS, 0, st>>>((float*)tau6, (const float*)ubar3, n3);
  else
    k_sub_products<double><<<grid_for(n3), SGS_THREADS, 0, st>>>((double*)tau6, (const double*)ubar3, n3);
  return launched("dns_subtract_products: launch failed");
}

}  // extern "C"

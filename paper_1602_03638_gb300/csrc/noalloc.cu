// dns_spectral_sums_noalloc: the energy / dissipation / helicity / enstrophy
// sums of dns_diagnostics for a caller-supplied spectral field, computed
// without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// entirely owned by another allocator (for example a framework's caching pool
// that has reserved the whole device), or a time-critical loop that must not
// take the device-wide synchronisation a cudaMalloc/cudaFree can imply. The
// regular diagnostics path needs a handle, whose creation allocates. This entry
// point needs none: the per-block partial sums live in a fixed file-scope device
// array, sized for NOALLOC_BLOCKS blocks (32 KB), that every GPU which loads
// the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/dns.h"
#include "fft_core.cuh"

namespace dns {
void set_error_message(const char* msg);
}

namespace {

constexpr int NOALLOC_BLOCKS = 1024;   // partial-sum slots in the fixed array
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_N = 2048;    // largest grid accepted
constexpr int NOALLOC_MAX_DEVICES = 64;

}  // namespace

// Fixed scratch: 4 FP64 partial sums per block. In host code this name is only a
// host-side stand-in; kernels get the device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_sums_scratch[NOALLOC_BLOCKS * 4];

namespace {

// Same sums as the handle's diagnostics kernel, but over the public layout
// (3, N, N, N/2+1) [c][kx][ky][kz]; weight 1 at kz = 0 and kz = N/2, else 2.
template <typename T>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_sums_paper_layout(const dns::cx<T>* __restrict__ uh, int N, double* __restrict__ partials) {
  const int M1 = N / 2 + 1;
  const size_t fs = (size_t)N * N * M1;
  double se = 0, sz = 0, sh = 0, bad = 0;
  for (size_t i = (size_t)blockIdx.x * NOALLOC_THREADS + threadIdx.x; i < fs;
       i += (size_t)gridDim.x * NOALLOC_THREADS) {
    const int kzi = (int)(i % M1);
    const int kyi = (int)((i / M1) % N);
    const int kxi = (int)(i / ((size_t)M1 * N));
    const double kx = kxi < N / 2 ? kxi : kxi - N;
    const double ky = kyi < N / 2 ? kyi : kyi - N;
    const double kz = kzi;
    const double w = (kzi == 0 || kzi == N / 2) ? 1.0 : 2.0;
    const dns::cx<T> a0 = uh[i], a1 = uh[fs + i], a2 = uh[2 * fs + i];
    const double u0r = a0.x, u0i = a0.y, u1r = a1.x, u1i = a1.y, u2r = a2.x, u2i = a2.y;
    const double t0r = ky * u2r - kz * u1r, t0i = ky * u2i - kz * u1i;
    const double t1r = kz * u0r - kx * u2r, t1i = kz * u0i - kx * u2i;
    const double t2r = kx * u1r - ky * u0r, t2i = kx * u1i - ky * u0i;
    const double w0r = -t0i, w0i = t0r, w1r = -t1i, w1i = t1r, w2r = -t2i, w2i = t2r;
    const double uu = u0r * u0r + u0i * u0i + u1r * u1r + u1i * u1i + u2r * u2r + u2i * u2i;
    const double ww = w0r * w0r + w0i * w0i + w1r * w1r + w1i * w1i + w2r * w2r + w2i * w2i;
    const double uw = u0r * w0r + u0i * w0i + u1r * w1r + u1i * w1i + u2r * w2r + u2i * w2i;
    se += w * uu;
    sz += w * ww;
    sh += w * uw;
    if (!isfinite(uu)) bad += 1.0;
  }
  __shared__ double red[4][NOALLOC_THREADS / 32];
  double v[4] = {se, sz, sh, bad};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int w = 0; w < NOALLOC_THREADS / 32; ++w) t += red[threadIdx.x][w];
    partials[blockIdx.x * 4 + threadIdx.x] = t;  // every slot is rewritten on every call
  }
}

__global__ void k_sums_finish(const double* __restrict__ partials, int nblocks, double nu, double n6,
                              double* __restrict__ out) {
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[b * 4 + threadIdx.x];
    switch (threadIdx.x) {
      case 0: out[0] = 0.5 * t / n6; break;  // energy
      case 1:
        out[1] = nu * t / n6;                 // dissipation
        out[3] = 0.5 * t / n6;                // enstrophy
        break;
      case 2: out[2] = t / n6; break;        // helicity
      default: out[4] = t; break;            // non-finite mode count
    }
  }
}

std::mutex g_setup_mutex;
void* g_scratch_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the fixed array for the current device (looked up once per device).
int scratch_for_current_device(void** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return -1;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return -2;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sums_scratch);
    if (e != cudaSuccess || !p) return -3;
    g_scratch_ptr[dev] = p;
  }
  *ptr = g_scratch_ptr[dev];
  return 0;
}

int noalloc_fail(int code, const char* msg) {
  dns::set_error_message(msg);
  return code;
}

}  // namespace

extern "C" int dns_spectral_sums_noalloc(const void* uhat, int N, int dtype, double nu, double* out,
                                         void* stream) {
  if (!uhat || !out) return noalloc_fail(DNS_ERR_ARG, "dns_spectral_sums_noalloc: uhat or out is NULL");
  if ((uintptr_t)uhat % 16 || (uintptr_t)out % 8)
    return noalloc_fail(DNS_ERR_ARG, "dns_spectral_sums_noalloc: uhat must be 16-byte and out 8-byte aligned");
  if (dtype != DNS_F32 && dtype != DNS_F64)
    return noalloc_fail(DNS_ERR_ARG, "dns_spectral_sums_noalloc: dtype must be DNS_F32 or DNS_F64");
  if (N < 2 || N % 2)
    return noalloc_fail(DNS_ERR_ARG, "dns_spectral_sums_noalloc: N must be even and >= 2");
  if (N > NOALLOC_MAX_N) {
    char msg[160];
    snprintf(msg, sizeof(msg), "dns_spectral_sums_noalloc: N = %d exceeds the maximum %d of the fixed scratch path",
             N, NOALLOC_MAX_N);
    return noalloc_fail(DNS_ERR_ARG, msg);
  }
  if (!(nu >= 0.0) || !std::isfinite(nu))
    return noalloc_fail(DNS_ERR_ARG, "dns_spectral_sums_noalloc: nu must be finite and >= 0");
  void* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != 0)
    return noalloc_fail(DNS_ERR_CUDA, "dns_spectral_sums_noalloc: no device address for the fixed scratch array");
  cudaStream_t st = (cudaStream_t)stream;
  double* partials = static_cast<double*>(scratch);
  if (dtype == DNS_F32)
    k_sums_paper_layout<float><<<NOALLOC_BLOCKS, NOALLOC_THREADS, 0, st>>>(
        static_cast<const dns::cx<float>*>(uhat), N, partials);
  else
    k_sums_paper_layout<double><<<NOALLOC_BLOCKS, NOALLOC_THREADS, 0, st>>>(
        static_cast<const dns::cx<double>*>(uhat), N, partials);
  const double n = (double)N;
  k_sums_finish<<<1, 32, 0, st>>>(partials, NOALLOC_BLOCKS, nu, n * n * n * n * n * n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(DNS_ERR_CUDA, cudaGetErrorString(e));
  return DNS_OK;
}

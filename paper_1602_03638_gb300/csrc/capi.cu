// C ABI of the solver (include/dns.h): handle life cycle, state transfer,
// RK4 stepping through a captured CUDA graph, diagnostics, and the small
// non-templated kernels (layout transposes, final diagnostic sum).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dns.h"
#include "dns_internal.h"
#include "fft_core.cuh"
#include "instances.h"

namespace dns {

#define DNS_DECL(T, tag, N) const DnsOps* dns_ops_##tag##_##N();
DNS_INSTANCES(DNS_DECL)
#undef DNS_DECL
#define DNS_DECL3(T, tag, NX, NY, NZ) const DnsOps* dns_ops_##tag##_##NX##x##NY##x##NZ();
DNS_BOX_INSTANCES(DNS_DECL3)
#undef DNS_DECL3

const DnsOps* find_ops(int dtype, int N) {
#define DNS_FIND(T, tag, NN) \
  if (N == NN && dtype == (sizeof(T) == 4 ? 0 : 1)) return dns_ops_##tag##_##NN();
  DNS_INSTANCES(DNS_FIND)
#undef DNS_FIND
  return nullptr;
}

const DnsOps* find_ops3(int dtype, int Nx, int Ny, int Nz) {
  if (Nx == Ny && Ny == Nz) return find_ops(dtype, Nx);
#define DNS_FIND3(T, tag, NX, NY, NZ) \
  if (Nx == NX && Ny == NY && Nz == NZ && dtype == (sizeof(T) == 4 ? 0 : 1)) return dns_ops_##tag##_##NX##x##NY##x##NZ();
  DNS_BOX_INSTANCES(DNS_FIND3)
#undef DNS_FIND3
  return nullptr;
}

__global__ void k_diag_final(double* partials, int nblocks) {
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[b * 4 + threadIdx.x];
    partials[nblocks * 4 + threadIdx.x] = t;
  }
}

// The row flag of the state U (3 fields of M x Ny rows of Nx values, internal layout):
// bit 0 is set if a row (kz, ky) outside the 2/3 box (3 kz >= k3z or 3 |ky| >= k3y) holds a
// nonzero value, bit 1 if a row inside it does at a column with 3 |kx| >= k3x (NaN counts as
// nonzero, -0 as zero); the bits are only set here (the caller clears the flag).
template <typename T>
__global__ void k_rows_outside(const cx<T>* __restrict__ U, int Nx, int Ny, int M, int k3x, int k3y, int k3z,
                               int* flag) {
  const size_t rows = (size_t)3 * M * Ny;
  for (size_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int ky = (int)(r % Ny), kz = (int)((r / Ny) % M);
    const int kf = ky < Ny / 2 ? ky : ky - Ny;
    const bool inside = 3 * kz < k3z && 3 * (kf < 0 ? -kf : kf) < k3y;  // the same for the whole block
    const cx<T>* p = U + r * Nx;
    int nz = 0;
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) {
      const int kx = j < Nx / 2 ? j : j - Nx;
      if (!inside || 3 * (kx < 0 ? -kx : kx) >= k3x) nz |= (p[j].x != (T)0) | (p[j].y != (T)0);
    }
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(flag, inside ? 2 : 1);
  }
}

// Paper order P[c][kx][ky][kz'] (kz' <= Nz/2)  <->  internal O[c][kz][ky][kx] (kz < Nz/2).
// grid = (ceil(Nx/32), ceil(kzcount/32), 3*Ny), block = (32, 8)
template <typename T>
__global__ void k_paper_to_internal(const cx<T>* __restrict__ P, cx<T>* __restrict__ O, int Nx, int Ny, int Nz) {
  __shared__ cx<T> tile[32][33];
  const int M = Nz / 2;
  const int c = blockIdx.z / Ny, ky = blockIdx.z % Ny;
  const int kx0 = blockIdx.x * 32, kz0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int kx = kx0 + i, kz = kz0 + threadIdx.x;
    if (kx < Nx && kz < M) tile[i][threadIdx.x] = P[(((size_t)c * Nx + kx) * Ny + ky) * (M + 1) + kz];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int kz = kz0 + i, kx = kx0 + threadIdx.x;
    if (kx < Nx && kz < M) {
      cx<T> v = tile[threadIdx.x][i];
      if (kx == Nx / 2 || ky == Ny / 2) v = mk((T)0, (T)0);
      O[(((size_t)c * M + kz) * Ny + ky) * Nx + kx] = v;
    }
  }
}

template <typename T>
__global__ void k_internal_to_paper(const cx<T>* __restrict__ O, cx<T>* __restrict__ P, int Nx, int Ny, int Nz) {
  __shared__ cx<T> tile[32][33];
  const int M = Nz / 2;
  const int c = blockIdx.z / Ny, ky = blockIdx.z % Ny;
  const int kx0 = blockIdx.x * 32, kz0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int kz = kz0 + i, kx = kx0 + threadIdx.x;
    if (kx < Nx && kz < M) tile[i][threadIdx.x] = O[(((size_t)c * M + kz) * Ny + ky) * Nx + kx];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int kx = kx0 + i, kz = kz0 + threadIdx.x;
    if (kx < Nx && kz <= M) {
      const cx<T> v = kz < M ? tile[threadIdx.x][i] : mk((T)0, (T)0);
      P[(((size_t)c * Nx + kx) * Ny + ky) * (M + 1) + kz] = v;
    }
  }
}

// FP64 FMA throughput probe: FMA_PROBE_CHAINS independent dependent-FMA chains
// per thread, x <- x * a + b, so that the FP64 pipe, not latency, sets the rate.
constexpr int FMA_PROBE_CHAINS = 8;
constexpr int FMA_PROBE_THREADS = 256;
__global__ void __launch_bounds__(FMA_PROBE_THREADS) k_fp64_fma_probe(double* sink, int iters, double a, double b) {
  double x[FMA_PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < FMA_PROBE_CHAINS; ++i) x[i] = 1e-3 * threadIdx.x + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < FMA_PROBE_CHAINS; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < FMA_PROBE_CHAINS; ++i) s += x[i];
  if (s == -1.0) *sink = s;  // never true: keeps the chains live
}

}  // namespace dns

using namespace dns;

namespace {

thread_local std::string g_err = "no error";
std::atomic<int> g_fail_after{0};

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(DNS_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define DNS_CUDA(call, where)                         \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

// Explicit Runge-Kutta schemes, each in one of two two-register forms.
// Form 0, the Appendix driver's: stage s evaluates dU_s on its stage state, stage
// s + 1 starts from u0 + b_s dt dU_s, and the new state is u0 + sum_s a_s dt dU_s.
// Form 1, Williamson's 2N low-storage form: stage s does dU <- a_s dU + dt RHS(u),
// u <- u + b_s dU (a_0 multiplies a zero register and is ignored).
// Index 0 is the classical RK4 of the Appendix (the default), 1 forward Euler (the
// integrator loop of Sec. 3.1), 2 and 3 the two-stage Heun and midpoint rules, 4
// Williamson's three-stage third-order 2N scheme, 5 the five-stage fourth-order 2N
// scheme of Carpenter & Kennedy (1994). Sec. 3.1 notes that other integrators may
// be added; dns_set_rk_tableau takes any scheme of either form.
const double kTwoPi = 6.283185307179586476925286766559;

constexpr int RK_MAX_STAGES = 8;
struct RkScheme {
  int form;    // 0: Appendix two-register form, 1: Williamson 2N form
  int stages;  // 1 .. RK_MAX_STAGES
  double a[RK_MAX_STAGES];
  double b[RK_MAX_STAGES];
};
const RkScheme RK_SCHEMES[6] = {
    {0, 4, {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}, {0.5, 0.5, 1.0}},
    {0, 1, {1.0}, {0.0}},
    {0, 2, {0.5, 0.5}, {1.0}},
    {0, 2, {0.0, 1.0}, {0.5}},
    {1, 3, {0.0, -5.0 / 9.0, -153.0 / 128.0}, {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0}},
    {1, 5,
     {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
      -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0},
     {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0, 1720146321549.0 / 2090206949498.0,
      3134564353537.0 / 4481467310338.0, 2277821191437.0 / 14882151754819.0}},
};
constexpr int RK_BUILTIN = 6;

bool same_scheme(const RkScheme& x, const RkScheme& y) {
  if (x.form != y.form || x.stages != y.stages) return false;
  for (int i = 0; i < x.stages; ++i)
    if (x.a[i] != y.a[i] || x.b[i] != y.b[i]) return false;
  return true;
}

// exp(-2 pi i t / N) in FP64 with exact quadrant/octant symmetry.
void twiddle(long t, long N, double* re, double* im) {
  t %= N;
  const long q = (4 * t) / N;
  const long r = 4 * t - q * N;  // angle = q pi/2 + (pi/2) r/N, 0 <= r < N
  const double pi = 3.14159265358979323846;
  double c, s;
  if (2 * r <= N) {
    const double phi = pi * (double)r / (2.0 * (double)N);
    c = std::cos(phi);
    s = std::sin(phi);
  } else {
    const double phi = pi * (double)(N - r) / (2.0 * (double)N);
    c = std::sin(phi);
    s = std::cos(phi);
  }
  double C, S;
  switch (q & 3) {
    case 0: C = c; S = s; break;
    case 1: C = -s; S = c; break;
    case 2: C = -c; S = -s; break;
    default: C = s; S = -c; break;
  }
  *re = C;
  *im = -S;
}

}  // namespace

namespace dns {
// Lets other translation units of the library report through dns_last_error().
void set_error_message(const char* msg) { g_err = msg; }
}  // namespace dns

struct dns_handle {
  int N = 0;  // points along x (and along y and z on a cubic grid)
  int Ny = 0, Nz = 0;  // points along y and z
  int dtype = 0;
  int variant = 0;
  int integrator = 0;  // index into RK_SCHEMES, -1 for a scheme set by dns_set_rk_tableau
  RkScheme rk = RK_SCHEMES[0];
  double L[3] = {kTwoPi, kTwoPi, kTwoPi};  // box lengths along x, y, z
  int ytile[2] = {0, 0};  // y-pass tile widths of the stage (inverse, forward); 0 = default
  int ztile = 0;          // z-pass tile width of the stage; 0 = default
  int plan = 0;  // radix plan variant per pass of the stage's line transforms (option "fft_plan", bits PLAN_*)
  int use_graph = 1;
  double nu = 0.0, dt = 0.0, t = 0.0;
  const DnsOps* ops = nullptr;
  int device = 0;
  cudaStream_t own_stream = nullptr, stream = nullptr, cap_stream = nullptr;
  void* U = nullptr;
  void* U1 = nullptr;
  void* US = nullptr;
  void* W = nullptr;
  void* D = nullptr;
  void* F = nullptr;  // optional force, internal layout
  bool has_force = false;
  // learned closure evaluated at the start of every step (dns_set_closure): the network
  // (borrowed), the filter width, and scratch (cubic grids): features (10 x N^3 floats), stress
  // (6 x N^3 floats), 6 spectral fields, 3 spectral work fields, the force (3 fields)
  dns_mlp* closure = nullptr;
  double closure_delta = 0.0;
  void* CX = nullptr;
  void* CT = nullptr;
  void* CS = nullptr;  // 9 spectral fields: the gradients of u_0, u_1, u_2, then 6 stress fields
  void* CW = nullptr;  // 9 work fields of the three gradient transforms
  void* FC = nullptr;
  // side streams and fork/join events of the closure's independent transforms
  cudaStream_t cl_side[2] = {nullptr, nullptr};
  cudaEvent_t cl_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  void* tw = nullptr;
  double* diag = nullptr;
  size_t bytes = 0;
  size_t fs = 0;  // complex values per field
  bool w_valid = false;
  int prune_rows = 1;  // option "prune_rows": skip the rows outside the 2/3 box where the state vanishes
  int support = PRUNE_BOX;  // where the state vanishes (PRUNE_*), from the last check (the zero state: everywhere)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_dirty = true;
  unsigned epoch = 0;  // bumped whenever a captured step of this handle goes stale
};

namespace {

int dev_alloc(dns_handle* h, void** p, size_t bytes, const char* what) {
  int n = g_fail_after.load();
  if (n > 0) {
    if (n == 1) {
      g_fail_after.store(0);
      return fail(DNS_ERR_OOM, "allocation of %s (%zu bytes) failed (injected)", what, bytes);
    }
    g_fail_after.store(n - 1);
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(DNS_ERR_OOM, "cudaMalloc of %s (%zu bytes) failed: %s", what, bytes, cudaGetErrorString(e));
  }
  h->bytes += bytes;
  return DNS_OK;
}

void release(dns_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  void* bufs[] = {h->U, h->U1, h->US, h->W, h->D, h->F, h->tw, h->diag, h->CX, h->CT, h->CS, h->CW, h->FC};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (cudaEvent_t ev : h->cl_ev)
    if (ev) cudaEventDestroy(ev);
  for (cudaStream_t cs : h->cl_side)
    if (cs) cudaStreamDestroy(cs);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
}

// Scratch word of the row check (check_rows) in the diagnostics block, past the results and max|div|.
int* row_flag(const dns_handle* h) { return reinterpret_cast<int*>(h->diag + DIAG_BLOCKS * 4 + 6); }

PassArgs base_args(const dns_handle* h) {
  PassArgs a;
  a.U = h->U;
  a.U1 = h->U1;
  a.US = h->US;
  a.W = h->W;
  a.D = h->D;
  a.tw = h->tw;
  a.F = h->has_force ? h->F : (h->closure ? h->FC : nullptr);
  a.nu = h->nu;
  a.kmax3 = h->N + 2 * h->variant;
  a.kmax3y = h->Ny + 2 * h->variant;
  a.kmax3z = h->Nz + 2 * h->variant;
  for (int i = 0; i < 3; ++i) a.ks[i] = kTwoPi / h->L[i];  // exactly 1 on the 2 pi box
  a.ytile[0] = h->ytile[0];
  a.ytile[1] = h->ytile[1];
  a.ztile = h->ztile;
  a.plan = h->plan;
  a.partials = h->diag;
  a.maxbits = reinterpret_cast<unsigned long long*>(h->diag + DIAG_BLOCKS * 4 + 4);
  if (h->prune_rows) a.prune = h->support;
  return a;
}

// Where the state now in U vanishes (h->support, PRUNE_*): the row flag, bit 0 unless U
// vanishes on every row (kz, ky) outside the handle's 2/3 box, bit 1 unless it also vanishes
// at the columns |kx| >= N/3 of the rows inside, computed on the handle's stream and read
// back (synchronises). A change re-captures the step graph.
cudaError_t check_rows(dns_handle* h) {
  int* flag = row_flag(h);
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) return e;
  const int k3x = h->N + 2 * h->variant, k3y = h->Ny + 2 * h->variant, k3z = h->Nz + 2 * h->variant;
  const int M = h->Nz / 2, blocks = 1024;
  if (h->dtype == DNS_F32)
    k_rows_outside<float><<<blocks, 256, 0, h->stream>>>((const cx<float>*)h->U, h->N, h->Ny, M, k3x, k3y, k3z, flag);
  else
    k_rows_outside<double><<<blocks, 256, 0, h->stream>>>((const cx<double>*)h->U, h->N, h->Ny, M, k3x, k3y, k3z,
                                                          flag);
  int f = 3;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  const int support = (f & 1) ? PRUNE_NONE : ((f & 2) ? PRUNE_ROWS : PRUNE_BOX);
  if (support != h->support) {
    h->support = support;
    h->graph_dirty = true;
    ++h->epoch;
  }
  return cudaSuccess;
}

int rk_stages(const dns_handle* h) { return h->rk.stages; }

// Brings W into the form the stage launches expect: the x-inverse of u and omega.
cudaError_t prime_work(dns_handle* h, cudaStream_t st) {
  PassArgs a = base_args(h);
  return h->ops->x_inverse_curl(a, 0, st);
}

// stage s of the handle's scheme: its coefficients times dt and the index of the last stage
void set_stage(const dns_handle* h, int s, PassArgs& a) {
  const RkScheme& r = h->rk;
  a.stage = s;
  a.last = r.stages - 1;
  if (r.form == 1) {  // 2N: the coefficients as given, dt separately
    a.lsrk = 1;
    a.cA = s > 0 ? r.a[s] : 0.0;
    a.cB = r.b[s];
    a.cC = h->dt;
  } else {
    a.lsrk = 0;
    a.cA = r.a[s] * h->dt;
    a.cB = s < r.stages - 1 ? r.b[s] * h->dt : 0.0;
    a.cC = 0.0;
  }
}

// The closure force of the current state into FC (dns_set_closure): velocity
// gradients i k_j u_hat_i -> 9 inverse transforms -> features; the network -> the 6
// stress components -> 2 x 3 forward transforms -> f_i = -i k_j tau_hat_ij. FP32
// handles on the 2 pi box; everything on the stream, no host synchronisation. The
// three gradient transforms and the two stress transforms are independent: they run
// on the stream and two side streams (fork and join through events, also inside a
// captured graph), each with its own scratch, so that their short launches overlap.
cudaError_t closure_eval(dns_handle* h, cudaStream_t st) {
  const int N = h->N;
  const size_t P = (size_t)N * N * N, cb = h->ops->elem_bytes, fb = h->fs * cb;
  PassArgs a = base_args(h);
  cudaStream_t sc[3] = {st, h->cl_side[0], h->cl_side[1]};
  cudaError_t e = cudaEventRecord(h->cl_ev[0], st);
  for (int c = 1; c < 3 && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(sc[c], h->cl_ev[0], 0);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
    PassArgs g = a;
    g.U = (char*)h->CS + 3 * c * fb;
    g.W = (char*)h->CW + 3 * c * fb;
    g.out = (float*)h->CX + 3 * c * P;
    e = closure_gradient(h->U, N, c, g.U, h->dtype, sc[c]);
    if (e == cudaSuccess) e = h->ops->inverse3d(g, sc[c]);
  }
  for (int c = 1; c < 3 && e == cudaSuccess; ++c) {
    e = cudaEventRecord(h->cl_ev[c], sc[c]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->cl_ev[c], 0);
  }
  if (e == cudaSuccess) e = mlp_forward_async(h->closure, (const float*)h->CX, (float*)h->CT, (int)P, st);
  if (e == cudaSuccess) e = cudaEventRecord(h->cl_ev[3], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sc[1], h->cl_ev[3], 0);
  for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
    PassArgs f = a;
    f.in = (const float*)h->CT + 3 * r * P;
    f.U = (char*)h->CS + 3 * r * fb;
    e = h->ops->forward3d(f, sc[r]);
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->cl_ev[4], sc[1]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->cl_ev[4], 0);
  if (e == cudaSuccess) e = closure_force(h->CS, N, h->FC, h->dtype, st);
  return e;
}

cudaError_t enqueue_step(dns_handle* h, cudaStream_t st) {
  if (h->closure) {
    cudaError_t e = closure_eval(h, st);
    if (e != cudaSuccess) return e;
  }
  PassArgs a = base_args(h);
  for (int s = 0; s < rk_stages(h); ++s) {
    set_stage(h, s, a);
    cudaError_t e = h->ops->rk_stage(a, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int check_handle(const dns_handle* h) {
  if (!h || !h->ops) return fail(DNS_ERR_ARG, "invalid handle");
  return DNS_OK;
}

int use_device(const dns_handle* h) {
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return DNS_OK;
}

size_t phys_bytes(const dns_handle* h) { return (size_t)3 * h->N * h->Ny * h->Nz * (h->dtype ? 8 : 4); }
size_t paper_spec_bytes(const dns_handle* h) {
  return (size_t)3 * h->N * h->Ny * (h->Nz / 2 + 1) * h->ops->elem_bytes;
}

cudaError_t launch_transpose(dns_handle* h, const void* src, void* dst, bool to_internal) {
  const int Nx = h->N, Ny = h->Ny, Nz = h->Nz, M = Nz / 2;
  dim3 block(32, 8);
  dim3 grid((Nx + 31) / 32, ((to_internal ? M : M + 1) + 31) / 32, 3 * Ny);
  if (h->dtype == 0) {
    if (to_internal)
      k_paper_to_internal<float><<<grid, block, 0, h->stream>>>((const cx<float>*)src, (cx<float>*)dst, Nx, Ny, Nz);
    else
      k_internal_to_paper<float><<<grid, block, 0, h->stream>>>((const cx<float>*)src, (cx<float>*)dst, Nx, Ny, Nz);
  } else {
    if (to_internal)
      k_paper_to_internal<double><<<grid, block, 0, h->stream>>>((const cx<double>*)src, (cx<double>*)dst, Nx, Ny, Nz);
    else
      k_internal_to_paper<double><<<grid, block, 0, h->stream>>>((const cx<double>*)src, (cx<double>*)dst, Nx, Ny, Nz);
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int dns_create(int N, double nu, double dt, int dtype, dns_handle** out) {
  return dns_create3(N, N, N, nu, dt, dtype, out);
}

int dns_create3(int Nx, int Ny, int Nz, double nu, double dt, int dtype, dns_handle** out) {
  if (!out) return fail(DNS_ERR_ARG, "dns_create: out is NULL");
  *out = nullptr;
  if (dtype != DNS_F32 && dtype != DNS_F64) return fail(DNS_ERR_ARG, "dns_create: dtype %d is not DNS_F32/DNS_F64", dtype);
  if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(DNS_ERR_ARG, "dns_create: nu must be finite and >= 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DNS_ERR_ARG, "dns_create: dt must be finite and > 0");
  const DnsOps* ops = find_ops3(dtype, Nx, Ny, Nz);
  if (!ops) {
    if (Nx == Ny && Ny == Nz) return fail(DNS_ERR_ARG, "dns_create: N = %d is not a supported grid size", Nx);
    return fail(DNS_ERR_ARG, "dns_create3: %d x %d x %d is not a compiled grid", Nx, Ny, Nz);
  }
  const int N = Nx;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(DNS_ERR_UNSUPPORTED, "dns_create: no CUDA device (%s)", cudaGetErrorString(e));
  }
  int dev = 0;
  DNS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  cudaDeviceProp prop;
  DNS_CUDA(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(DNS_ERR_UNSUPPORTED, "dns_create: device %d is sm_%d%d; this library is built for sm_103a", dev,
                prop.major, prop.minor);

  dns_handle* h = new dns_handle();
  h->N = N;
  h->Ny = Ny;
  h->Nz = Nz;
  h->plan = ops->default_plan;
  h->dtype = dtype;
  h->nu = nu;
  h->dt = dt;
  h->ops = ops;
  h->device = dev;
  const int M = Nz / 2;
  h->fs = (size_t)M * Ny * N;
  const size_t cb = ops->elem_bytes;
  int rc = DNS_OK;
  cudaError_t ce = ops->prepare();
  if (ce != cudaSuccess) rc = cuda_fail(ce, "kernel attribute set-up");
  if (rc == DNS_OK) {
    ce = cudaStreamCreate(&h->own_stream);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "cudaStreamCreate");
    h->stream = h->own_stream;
  }
  if (rc == DNS_OK) rc = dev_alloc(h, &h->U, 3 * h->fs * cb, "state U");
  if (rc == DNS_OK) rc = dev_alloc(h, &h->U1, 3 * h->fs * cb, "RK4 accumulator");
  if (rc == DNS_OK) rc = dev_alloc(h, &h->US, 3 * h->fs * cb, "RK4 stage state");
  if (rc == DNS_OK) rc = dev_alloc(h, &h->W, (6 * h->fs + (size_t)3 * N * Ny) * cb, "work fields");
  if (rc == DNS_OK) rc = dev_alloc(h, &h->D, h->fs * cb, "divergence field");
  const int TW = ops->TW;  // exp(-2 pi i t / TW): N on a cubic grid, else a common multiple of the counts
  if (rc == DNS_OK) rc = dev_alloc(h, &h->tw, (size_t)TW * cb, "twiddles");
  if (rc == DNS_OK) rc = dev_alloc(h, (void**)&h->diag, (DIAG_BLOCKS * 4 + 8) * sizeof(double), "diagnostics");
  if (rc == DNS_OK) {
    std::vector<double> t64(2 * TW);
    for (int t = 0; t < TW; ++t) twiddle(t, TW, &t64[2 * t], &t64[2 * t + 1]);
    if (dtype == DNS_F32) {
      std::vector<float> t32(2 * TW);
      for (int i = 0; i < 2 * TW; ++i) t32[i] = (float)t64[i];
      ce = cudaMemcpy(h->tw, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
    } else {
      ce = cudaMemcpy(h->tw, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess) ce = cudaMemset(h->U, 0, 3 * h->fs * cb);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "dns_create initialisation");
  }
  if (rc != DNS_OK) {
    std::string msg = g_err;
    release(h);
    delete h;
    g_err = msg;
    return rc;
  }
  *out = h;
  return DNS_OK;
}

int dns_destroy(dns_handle* h) {
  if (!h) return DNS_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  release(h);
  delete h;
  return DNS_OK;
}

int dns_set_stream(dns_handle* h, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  return DNS_OK;
}

int dns_set_option(dns_handle* h, const char* key, double value) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!key) return fail(DNS_ERR_ARG, "dns_set_option: key is NULL");
  if (!strcmp(key, "dealias_variant")) {
    if (value != 0.0 && value != 1.0) return fail(DNS_ERR_ARG, "dealias_variant must be 0 or 1");
    h->variant = (int)value;
    if ((rc = use_device(h))) return rc;
    DNS_CUDA(check_rows(h), "dealias_variant row check");  // the box changed
  } else if (!strcmp(key, "prune_rows")) {
    if (value != 0.0 && value != 1.0) return fail(DNS_ERR_ARG, "prune_rows must be 0 or 1");
    h->prune_rows = (int)value;
  } else if (!strcmp(key, "integrator")) {
    if (!(value >= 0.0 && value < RK_BUILTIN) || value != std::floor(value))
      return fail(DNS_ERR_ARG,
                  "integrator must be 0 (RK4), 1 (Euler), 2 (Heun), 3 (midpoint), 4 (Williamson 2N RK3) "
                  "or 5 (Carpenter-Kennedy 2N RK4)");
    h->integrator = (int)value;
    h->rk = RK_SCHEMES[h->integrator];
  } else if (!strcmp(key, "Lx") || !strcmp(key, "Ly") || !strcmp(key, "Lz")) {
    if (!(value > 0.0) || !std::isfinite(value)) return fail(DNS_ERR_ARG, "%s must be finite and > 0", key);
    h->L[key[1] - 'x'] = value;
  } else if (!strcmp(key, "y_tile_inverse") || !strcmp(key, "y_tile_forward")) {
    int tiles[8];
    const int n = h->ops->y_tiles(tiles, 8);
    bool ok = value == 0.0;
    for (int i = 0; i < n; ++i) ok = ok || value == (double)tiles[i];
    if (!ok) return fail(DNS_ERR_ARG, "%s: %g is not a tile width of this grid", key, value);
    h->ytile[key[7] == 'i' ? 0 : 1] = (int)value;
  } else if (!strcmp(key, "z_tile")) {
    int tiles[8];
    const int n = h->ops->z_tiles(tiles, 8);
    bool ok = value == 0.0;
    for (int i = 0; i < n; ++i) ok = ok || value == (double)tiles[i];
    if (!ok) return fail(DNS_ERR_ARG, "z_tile: %g is not a tile width of this grid", value);
    h->ztile = (int)value;
  } else if (!strcmp(key, "fft_plan")) {
    const int masks = h->ops->plans > 1 ? 1 << PLAN_BITS : 1;
    if (!(value >= 0.0 && value < masks) || value != std::floor(value))
      return fail(DNS_ERR_ARG, "fft_plan: %g is not a plan mask of this grid (0 .. %d)", value, masks - 1);
    h->plan = (int)value;
  } else if (!strcmp(key, "use_graph")) {
    if (value != 0.0 && value != 1.0) return fail(DNS_ERR_ARG, "use_graph must be 0 or 1");
    h->use_graph = (int)value;
  } else if (!strcmp(key, "nu")) {
    if (!(value >= 0.0) || !std::isfinite(value)) return fail(DNS_ERR_ARG, "nu must be finite and >= 0");
    h->nu = value;
  } else if (!strcmp(key, "dt")) {
    if (!(value > 0.0) || !std::isfinite(value)) return fail(DNS_ERR_ARG, "dt must be finite and > 0");
    h->dt = value;
  } else if (!strcmp(key, "time")) {
    if (!std::isfinite(value)) return fail(DNS_ERR_ARG, "time must be finite");
    h->t = value;
    return DNS_OK;
  } else {
    return fail(DNS_ERR_ARG, "dns_set_option: unknown key '%s'", key);
  }
  h->graph_dirty = true;
  ++h->epoch;
  h->w_valid = false;  // the x-inverse in W does not depend on these, but keep it simple
  return DNS_OK;
}

int dns_get_option(const dns_handle* h, const char* key, double* value) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!key || !value) return fail(DNS_ERR_ARG, "dns_get_option: key or value is NULL");
  if (!strcmp(key, "dealias_variant")) *value = h->variant;
  else if (!strcmp(key, "integrator")) *value = h->integrator;
  else if (!strcmp(key, "Lx") || !strcmp(key, "Ly") || !strcmp(key, "Lz")) *value = h->L[key[1] - 'x'];
  else if (!strcmp(key, "y_tile_inverse")) *value = h->ytile[0];
  else if (!strcmp(key, "y_tile_forward")) *value = h->ytile[1];
  else if (!strcmp(key, "z_tile")) *value = h->ztile;
  else if (!strcmp(key, "fft_plan")) *value = h->plan;
  else if (!strcmp(key, "use_graph")) *value = h->use_graph;
  else if (!strcmp(key, "nu")) *value = h->nu;
  else if (!strcmp(key, "dt")) *value = h->dt;
  else if (!strcmp(key, "time")) *value = h->t;
  else if (!strcmp(key, "Nx")) *value = h->N;
  else if (!strcmp(key, "Ny")) *value = h->Ny;
  else if (!strcmp(key, "Nz")) *value = h->Nz;
  else if (!strcmp(key, "prune_rows")) *value = h->prune_rows;
  else if (!strcmp(key, "rows_vanish")) *value = h->support >= PRUNE_ROWS ? 1.0 : 0.0;
  else if (!strcmp(key, "box_vanish")) *value = h->support == PRUNE_BOX ? 1.0 : 0.0; else return fail(DNS_ERR_ARG, "dns_get_option: unknown key '%s'", key);
  return DNS_OK;
}

int dns_set_rk_tableau(dns_handle* h, int form, int stages, const double* a, const double* b) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (form != 0 && form != 1) return fail(DNS_ERR_ARG, "dns_set_rk_tableau: form must be 0 or 1");
  if (stages < 1 || stages > RK_MAX_STAGES)
    return fail(DNS_ERR_ARG, "dns_set_rk_tableau: stages must be in 1 .. %d", RK_MAX_STAGES);
  const int nb = form == 0 ? stages - 1 : stages;
  if (!a || (nb > 0 && !b)) return fail(DNS_ERR_ARG, "dns_set_rk_tableau: coefficient array is NULL");
  RkScheme r{};
  r.form = form;
  r.stages = stages;
  for (int i = 0; i < stages; ++i) {
    r.a[i] = (form == 1 && i == 0) ? 0.0 : a[i];
    if (!std::isfinite(a[i])) return fail(DNS_ERR_ARG, "dns_set_rk_tableau: a[%d] is not finite", i);
  }
  for (int i = 0; i < nb; ++i) {
    if (!std::isfinite(b[i])) return fail(DNS_ERR_ARG, "dns_set_rk_tableau: b[%d] is not finite", i);
    r.b[i] = b[i];
  }
  h->rk = r;
  h->integrator = -1;
  for (int k = 0; k < RK_BUILTIN; ++k)
    if (same_scheme(r, RK_SCHEMES[k])) h->integrator = k;
  h->graph_dirty = true;
  ++h->epoch;
  h->w_valid = false;
  return DNS_OK;
}

}  // extern "C"

namespace {

// ---- tune cache: the tuners' choices kept in a text file across runs ----
// One entry per line, later lines win:
//   tiles <device> <Nx> <Ny> <Nz> <f32|f64> <y_inverse> <y_forward> <z> <plan>
//   ensemble <device> <f32|f64> <N:count,...> <max_batch> <streams>
std::mutex g_tc_mu;
std::string g_tc_path;

std::string tc_device(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string n = p.name;
  for (char& c : n)
    if (c == ' ' || c == '\t') c = '_';
  return n.empty() ? std::string("unknown") : n;
}

// values of the last line whose leading tokens equal `key`, or false
bool tc_find(const std::vector<std::string>& key, std::vector<long>& vals, size_t nvals) {
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (g_tc_path.empty()) return false;
  FILE* f = fopen(g_tc_path.c_str(), "r");
  if (!f) return false;
  bool found = false;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    std::vector<std::string> tok;
    for (char* t = strtok(line, " \t\r\n"); t; t = strtok(nullptr, " \t\r\n")) tok.push_back(t);
    if (tok.size() != key.size() + nvals || !std::equal(key.begin(), key.end(), tok.begin())) continue;
    std::vector<long> v;
    bool ok = true;
    for (size_t i = key.size(); i < tok.size() && ok; ++i) {
      char* end = nullptr;
      v.push_back(strtol(tok[i].c_str(), &end, 10));
      ok = end && *end == '\0';
    }
    if (ok) {
      vals = v;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tc_put(const std::vector<std::string>& key, const std::vector<long>& vals) {
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (g_tc_path.empty()) return;
  FILE* f = fopen(g_tc_path.c_str(), "a");
  if (!f) return;
  for (const std::string& k : key) fprintf(f, "%s ", k.c_str());
  for (size_t i = 0; i < vals.size(); ++i) fprintf(f, i + 1 < vals.size() ? "%ld " : "%ld\n", vals[i]);
  fclose(f);
}

std::vector<std::string> tc_tiles_key(const std::string& device, int Nx, int Ny, int Nz, int dtype) {
  return {"tiles", device, std::to_string(Nx), std::to_string(Ny), std::to_string(Nz), dtype ? "f64" : "f32"};
}

bool offered(int v, const int* cand, int n) {
  for (int i = 0; i < n; ++i)
    if (cand[i] == v) return true;
  return false;
}

}  // namespace

extern "C" {

int dns_set_tune_cache(const char* path) {
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (!path || !*path) {
    g_tc_path.clear();
    return DNS_OK;
  }
  FILE* f = fopen(path, "a");
  if (!f) return fail(DNS_ERR_ARG, "dns_set_tune_cache: cannot open '%s' for appending", path);
  fclose(f);
  g_tc_path = path;
  return DNS_OK;
}

int dns_tune_cache_lookup(const char* device, int Nx, int Ny, int Nz, int dtype, int* y_inverse, int* y_forward,
                          int* z, int* plan) {
  if (!device || !y_inverse || !y_forward || !z || !plan)
    return fail(DNS_ERR_ARG, "dns_tune_cache_lookup: NULL argument");
  std::vector<long> v;
  if (!tc_find(tc_tiles_key(device, Nx, Ny, Nz, dtype), v, 4)) return 0;
  *y_inverse = (int)v[0];
  *y_forward = (int)v[1];
  *z = (int)v[2];
  *plan = (int)v[3];
  return 1;
}

int dns_tune_tiles(dns_handle* h, int steps, int* y_inverse, int* y_forward, int* z) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (steps < 1 || !y_inverse || !y_forward || !z) return fail(DNS_ERR_ARG, "dns_tune_tiles: bad arguments");
  if ((rc = use_device(h))) return rc;
  // candidates per knob (the default first): y-inverse width, y-forward width, z width,
  // and the radix plan variant (0, 1) of each pass
  int ycand[9] = {0}, zcand[9] = {0};
  const int ny = 1 + h->ops->y_tiles(ycand + 1, 8);
  const int nz = 1 + h->ops->z_tiles(zcand + 1, 8);
  const int np = h->ops->plans;
  if (ny == 1 && nz == 1 && np == 1) {  // this grid offers the defaults only
    *y_inverse = h->ytile[0];
    *y_forward = h->ytile[1];
    *z = h->ztile;
    return DNS_OK;
  }
  // a choice stored in the tune cache for this device and grid is applied without timing
  const std::vector<std::string> tkey = tc_tiles_key(tc_device(h->device), h->N, h->Ny, h->Nz, h->dtype);
  std::vector<long> cached;
  if (tc_find(tkey, cached, 4) && offered((int)cached[0], ycand, ny) && offered((int)cached[1], ycand, ny) &&
      offered((int)cached[2], zcand, nz) && cached[3] >= 0 && cached[3] < (np > 1 ? 1 << PLAN_BITS : 1)) {
    h->ytile[0] = (int)cached[0];
    h->ytile[1] = (int)cached[1];
    h->ztile = (int)cached[2];
    h->plan = (int)cached[3];
    h->graph_dirty = true;
    ++h->epoch;
    h->w_valid = false;
    *y_inverse = h->ytile[0];
    *y_forward = h->ytile[1];
    *z = h->ztile;
    return DNS_OK;
  }
  const size_t bytes = 3 * h->fs * h->ops->elem_bytes;
  void* save = nullptr;
  if ((rc = dev_alloc(h, &save, bytes, "tuning copy of the state"))) return rc;
  const double t0 = h->t;
  const int keep[4] = {h->ytile[0], h->ytile[1], h->ztile, h->plan};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMemcpyAsync(save, h->U, bytes, cudaMemcpyDeviceToDevice, h->stream);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err != cudaSuccess) rc = cuda_fail(err, "dns_tune_tiles set-up");
  auto apply = [&](const int* v) {
    h->ytile[0] = v[0];
    h->ytile[1] = v[1];
    h->ztile = v[2];
    h->plan = v[3];
    h->graph_dirty = true;
  };
  // each candidate starts from the saved state: capture and one warm-up step, then
  // three timings of `steps` steps exactly as dns_step runs them; *ms = their median,
  // *spread = their range
  auto timed = [&](const int* v, float* ms, float* spread) -> int {
    apply(v);
    cudaError_t ce = cudaMemcpyAsync(h->U, save, bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "dns_tune_tiles copy");
    h->w_valid = false;
    int r = dns_step(h, 1);
    if (r) return r;
    float t[3];
    for (int k = 0; k < 3; ++k) {
      if ((ce = cudaEventRecord(e0, h->stream)) != cudaSuccess) return cuda_fail(ce, "dns_tune_tiles event");
      if ((r = dns_step(h, steps))) return r;
      if ((ce = cudaEventRecord(e1, h->stream)) == cudaSuccess) ce = cudaEventSynchronize(e1);
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t[k], e0, e1);
      if (ce != cudaSuccess) return cuda_fail(ce, "dns_tune_tiles timing");
    }
    std::sort(t, t + 3);
    *ms = t[1];
    *spread = t[2] - t[0];
    return DNS_OK;
  };
  // one knob at a time, the others kept: the radix plan of the x-, y-inverse, z- and
  // y-forward passes (with the widths the handle has), the y-inverse width, the
  // y-forward width, then the z width, each with
  // the best values found before it. The first candidate is the default; another
  // replaces the one kept so far only if its median beats that one's median by more
  // than that one's spread (differences inside the timing noise keep the earlier choice).
  int best_v[4] = {keep[0], keep[1], keep[2], h->ops->default_plan};
  // which < 3: a tile width; which = 3 + b: the plan bit b
  auto pick = [&](int n, const int* cand, int which) {
    float best = 0.f, best_spread = 0.f, ms = 0.f, spread = 0.f;
    auto with = [&](int* v, int c) {
      if (which < 3) v[which] = cand[c];
      else v[3] = (v[3] & ~(1 << (which - 3))) | (cand[c] << (which - 3));
    };
    for (int c = 0; c < n && !rc; ++c) {
      int v[4] = {best_v[0], best_v[1], best_v[2], best_v[3]};
      with(v, c);
      if ((rc = timed(v, &ms, &spread))) return;
      if (c == 0 || ms < best - best_spread) {
        best = ms;
        best_spread = spread;
        with(best_v, c);
      }
    }
  };
  if (np > 1)
    for (int b : {PLAN_X, PLAN_YI, PLAN_Z, PLAN_YF}) {
      const int d = (h->ops->default_plan >> b) & 1;  // the default's bit first
      const int bits[2] = {d, 1 - d};
      pick(np, bits, 3 + b);
    }
  pick(ny, ycand, 0);
  pick(ny, ycand, 1);
  pick(nz, zcand, 2);
  // the state and time as before; the fastest values kept
  err = cudaMemcpyAsync(h->U, save, bytes, cudaMemcpyDeviceToDevice, h->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(save);
  h->bytes -= bytes;
  h->t = t0;
  h->w_valid = false;
  apply(rc ? keep : best_v);
  ++h->epoch;
  if (!rc && err != cudaSuccess) rc = cuda_fail(err, "dns_tune_tiles restore");
  if (!rc) tc_put(tkey, {best_v[0], best_v[1], best_v[2], best_v[3]});
  *y_inverse = h->ytile[0];
  *y_forward = h->ytile[1];
  *z = h->ztile;
  return rc;
}

int dns_tile_widths(int N, int dtype, int which, int* widths, int max) {
  if (!widths || max < 1 || (which != 0 && which != 1)) return fail(DNS_ERR_ARG, "dns_tile_widths: bad arguments");
  const DnsOps* ops = find_ops(dtype, N);
  if (!ops) return fail(DNS_ERR_ARG, "dns_tile_widths: N = %d, dtype %d is not compiled", N, dtype);
  return which == 0 ? ops->y_tiles(widths, max) : ops->z_tiles(widths, max);
}

int dns_set_state(dns_handle* h, const void* u, int on_device) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!u) return fail(DNS_ERR_ARG, "dns_set_state: u is NULL");
  if ((rc = use_device(h))) return rc;
  PassArgs a = base_args(h);
  if (on_device) {
    if ((uintptr_t)u % 16) return fail(DNS_ERR_ARG, "dns_set_state: device pointer must be 16-byte aligned");
    a.in = u;
  } else {
    DNS_CUDA(cudaMemcpyAsync(h->W, u, phys_bytes(h), cudaMemcpyHostToDevice, h->stream), "dns_set_state copy");
    a.in = h->W;
  }
  DNS_CUDA(h->ops->forward3d(a, h->stream), "dns_set_state transform");
  DNS_CUDA(check_rows(h), "dns_set_state row check");
  h->w_valid = false;
  h->t = 0.0;
  return DNS_OK;
}

int dns_set_state_spectral(dns_handle* h, const void* uhat, int on_device) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!uhat) return fail(DNS_ERR_ARG, "dns_set_state_spectral: uhat is NULL");
  if ((rc = use_device(h))) return rc;
  const void* src = uhat;
  if (on_device) {
    if ((uintptr_t)uhat % 16) return fail(DNS_ERR_ARG, "dns_set_state_spectral: device pointer must be 16-byte aligned");
  } else {
    DNS_CUDA(cudaMemcpyAsync(h->W, uhat, paper_spec_bytes(h), cudaMemcpyHostToDevice, h->stream),
             "dns_set_state_spectral copy");
    src = h->W;
  }
  DNS_CUDA(launch_transpose(h, src, h->U, true), "dns_set_state_spectral transpose");
  DNS_CUDA(check_rows(h), "dns_set_state_spectral row check");
  h->w_valid = false;
  h->t = 0.0;
  return DNS_OK;
}

int dns_step(dns_handle* h, int n) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (n < 0) return fail(DNS_ERR_ARG, "dns_step: n = %d < 0", n);
  if (n == 0) return DNS_OK;
  if ((rc = use_device(h))) return rc;
  if (!h->w_valid) {
    DNS_CUDA(prime_work(h, h->stream), "dns_step initial transform");
    h->w_valid = true;
  }
  if (h->use_graph) {
    if (h->graph_dirty || !h->gexec) {
      if (h->gexec) cudaGraphExecDestroy(h->gexec);
      if (h->graph) cudaGraphDestroy(h->graph);
      h->gexec = nullptr;
      h->graph = nullptr;
      DNS_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
      cudaError_t e = enqueue_step(h, h->cap_stream);
      cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &h->graph);
      if (e != cudaSuccess) return cuda_fail(e, "graph capture");
      if (e2 != cudaSuccess) return cuda_fail(e2, "graph capture end");
      DNS_CUDA(cudaGraphInstantiate(&h->gexec, h->graph, 0), "graph instantiate");
      h->graph_dirty = false;
    }
    for (int i = 0; i < n; ++i) DNS_CUDA(cudaGraphLaunch(h->gexec, h->stream), "graph launch");
  } else {
    for (int i = 0; i < n; ++i) DNS_CUDA(enqueue_step(h, h->stream), "dns_step");
  }
  h->t += n * h->dt;
  return DNS_OK;
}

int dns_get_state(dns_handle* h, void* u, int on_device) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!u) return fail(DNS_ERR_ARG, "dns_get_state: u is NULL");
  if ((rc = use_device(h))) return rc;
  if (on_device && (uintptr_t)u % 16) return fail(DNS_ERR_ARG, "dns_get_state: device pointer must be 16-byte aligned");
  PassArgs a = base_args(h);
  void* dst = on_device ? u : (void*)((char*)h->W + 3 * h->fs * h->ops->elem_bytes);
  a.out = dst;
  DNS_CUDA(h->ops->inverse3d(a, h->stream), "dns_get_state transform");
  if (!on_device)
    DNS_CUDA(cudaMemcpyAsync(u, dst, phys_bytes(h), cudaMemcpyDeviceToHost, h->stream), "dns_get_state copy");
  DNS_CUDA(cudaStreamSynchronize(h->stream), "dns_get_state");
  h->w_valid = false;
  return DNS_OK;
}

int dns_get_state_spectral(dns_handle* h, void* uhat, int on_device) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!uhat) return fail(DNS_ERR_ARG, "dns_get_state_spectral: uhat is NULL");
  if ((rc = use_device(h))) return rc;
  if (on_device && (uintptr_t)uhat % 16)
    return fail(DNS_ERR_ARG, "dns_get_state_spectral: device pointer must be 16-byte aligned");
  void* dst = on_device ? uhat : (void*)((char*)h->W + 3 * h->fs * h->ops->elem_bytes);
  DNS_CUDA(launch_transpose(h, h->U, dst, false), "dns_get_state_spectral transpose");
  if (!on_device) {
    DNS_CUDA(cudaMemcpyAsync(uhat, dst, paper_spec_bytes(h), cudaMemcpyDeviceToHost, h->stream),
             "dns_get_state_spectral copy");
    h->w_valid = false;
  }
  DNS_CUDA(cudaStreamSynchronize(h->stream), "dns_get_state_spectral");
  return DNS_OK;
}

int dns_rhs(dns_handle* h, void* duhat, int on_device) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!duhat) return fail(DNS_ERR_ARG, "dns_rhs: duhat is NULL");
  if ((rc = use_device(h))) return rc;
  if (on_device && (uintptr_t)duhat % 16) return fail(DNS_ERR_ARG, "dns_rhs: device pointer must be 16-byte aligned");
  if (h->closure) DNS_CUDA(closure_eval(h, h->stream), "dns_rhs closure");
  PassArgs a = base_args(h);
  a.out = h->W;  // dU overwrites the forward-transformed product in place
  DNS_CUDA(h->ops->rhs(a, h->stream), "dns_rhs");
  void* dst = on_device ? duhat : (void*)((char*)h->W + 3 * h->fs * h->ops->elem_bytes);
  DNS_CUDA(launch_transpose(h, h->W, dst, false), "dns_rhs transpose");
  if (!on_device)
    DNS_CUDA(cudaMemcpyAsync(duhat, dst, paper_spec_bytes(h), cudaMemcpyDeviceToHost, h->stream), "dns_rhs copy");
  DNS_CUDA(cudaStreamSynchronize(h->stream), "dns_rhs");
  h->w_valid = false;
  return DNS_OK;
}

int dns_diagnostics(dns_handle* h, dns_diag* out) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!out) return fail(DNS_ERR_ARG, "dns_diagnostics: out is NULL");
  if ((rc = use_device(h))) return rc;
  PassArgs a = base_args(h);
  DNS_CUDA(h->ops->diag(a, h->stream), "dns_diagnostics");
  double r[5];
  DNS_CUDA(cudaMemcpyAsync(r, h->diag + DIAG_BLOCKS * 4, sizeof(r), cudaMemcpyDeviceToHost, h->stream),
           "dns_diagnostics copy");
  DNS_CUDA(cudaStreamSynchronize(h->stream), "dns_diagnostics");
  const double n3 = (double)h->N * (double)h->Ny * (double)h->Nz;
  const double n6 = n3 * n3;
  unsigned long long bits;
  memcpy(&bits, &r[4], sizeof(bits));
  double mdiv;
  memcpy(&mdiv, &bits, sizeof(mdiv));
  out->t = h->t;
  out->energy = 0.5 * r[0] / n6;
  out->dissipation = h->nu * r[1] / n6;
  out->max_div = mdiv;
  out->helicity = r[2] / n6;
  out->enstrophy = 0.5 * r[1] / n6;
  if (r[3] != 0.0 || !std::isfinite(out->energy))
    return fail(DNS_ERR_NONFINITE, "dns_diagnostics: %g non-finite modes in the state", r[3]);
  return DNS_OK;
}

int dns_transform_r2c(dns_handle* h, const void* phys3, void* spec3) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!phys3 || !spec3 || (uintptr_t)phys3 % 16 || (uintptr_t)spec3 % 16)
    return fail(DNS_ERR_ARG, "dns_transform_r2c: device pointers must be non-NULL and 16-byte aligned");
  if ((rc = use_device(h))) return rc;
  PassArgs a = base_args(h);
  a.in = phys3;
  a.U = h->US;  // scratch: the stage state is rebuilt by every step
  DNS_CUDA(h->ops->forward3d(a, h->stream), "dns_transform_r2c");
  DNS_CUDA(launch_transpose(h, h->US, spec3, false), "dns_transform_r2c layout");
  return DNS_OK;
}

int dns_transform_c2r(dns_handle* h, const void* spec3, void* phys3) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!phys3 || !spec3 || (uintptr_t)phys3 % 16 || (uintptr_t)spec3 % 16)
    return fail(DNS_ERR_ARG, "dns_transform_c2r: device pointers must be non-NULL and 16-byte aligned");
  if ((rc = use_device(h))) return rc;
  DNS_CUDA(launch_transpose(h, spec3, h->US, true), "dns_transform_c2r layout");
  PassArgs a = base_args(h);
  a.U = h->US;
  a.out = phys3;
  DNS_CUDA(h->ops->inverse3d(a, h->stream), "dns_transform_c2r");
  h->w_valid = false;
  return DNS_OK;
}

int dns_set_forcing(dns_handle* h, const void* f3, int on_device) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (f3 && h->closure) return fail(DNS_ERR_ARG, "dns_set_forcing: a closure is attached (dns_set_closure)");
  if ((rc = use_device(h))) return rc;
  if (!f3) {
    if (h->has_force) {
      h->graph_dirty = true;
      ++h->epoch;
    }
    h->has_force = false;
    return DNS_OK;
  }
  if (!h->F && (rc = dev_alloc(h, &h->F, 3 * h->fs * h->ops->elem_bytes, "force"))) return rc;
  const void* src = f3;
  if (on_device) {
    if ((uintptr_t)f3 % 16) return fail(DNS_ERR_ARG, "dns_set_forcing: device pointer must be 16-byte aligned");
  } else {
    void* stage = (char*)h->W + 3 * h->fs * h->ops->elem_bytes;
    DNS_CUDA(cudaMemcpyAsync(stage, f3, paper_spec_bytes(h), cudaMemcpyHostToDevice, h->stream), "dns_set_forcing copy");
    DNS_CUDA(cudaStreamSynchronize(h->stream), "dns_set_forcing");
    src = stage;
    h->w_valid = false;
  }
  DNS_CUDA(launch_transpose(h, src, h->F, true), "dns_set_forcing layout");
  if (!h->has_force) {
    h->graph_dirty = true;
    ++h->epoch;
  }
  h->has_force = true;
  return DNS_OK;
}

int dns_set_closure(dns_handle* h, dns_mlp* net, double delta) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!net) {
    if (h->closure) {
      h->closure = nullptr;
      h->graph_dirty = true;
      ++h->epoch;
    }
    return DNS_OK;
  }
  if (h->dtype != DNS_F32) return fail(DNS_ERR_UNSUPPORTED, "dns_set_closure: the closure runs on FP32 handles");
  if (h->Ny != h->N || h->Nz != h->N)
    return fail(DNS_ERR_UNSUPPORTED, "dns_set_closure: the closure runs on cubic grids");
  for (int i = 0; i < 3; ++i)
    if (h->L[i] != kTwoPi) return fail(DNS_ERR_UNSUPPORTED, "dns_set_closure: the closure assumes the 2 pi box");
  if (h->has_force) return fail(DNS_ERR_ARG, "dns_set_closure: a force is set (dns_set_forcing)");
  if (!(delta > 0.0) || !std::isfinite(delta)) return fail(DNS_ERR_ARG, "dns_set_closure: delta must be finite and > 0");
  if (net == h->closure && delta == h->closure_delta) return DNS_OK;  // already attached: the graph stays
  if ((rc = use_device(h))) return rc;
  const size_t P = (size_t)h->N * h->N * h->N, cb = h->ops->elem_bytes;
  if (!h->CX) {
    if ((rc = dev_alloc(h, &h->CX, 10 * P * sizeof(float), "closure features"))) return rc;
    if ((rc = dev_alloc(h, &h->CT, 6 * P * sizeof(float), "closure stress"))) return rc;
    if ((rc = dev_alloc(h, &h->CS, 9 * h->fs * cb, "closure spectral fields"))) return rc;
    if ((rc = dev_alloc(h, &h->CW, 9 * h->fs * cb, "closure work fields"))) return rc;
    if ((rc = dev_alloc(h, &h->FC, 3 * h->fs * cb, "closure force"))) return rc;
    for (cudaStream_t& cs : h->cl_side)
      DNS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "dns_set_closure streams");
    for (cudaEvent_t& ev : h->cl_ev)
      DNS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "dns_set_closure events");
  }
  DNS_CUDA(fill_f32((float*)h->CX + 9 * P, P, (float)delta, h->stream), "dns_set_closure");
  h->closure = net;
  h->closure_delta = delta;
  h->graph_dirty = true;
  ++h->epoch;
  return DNS_OK;
}

int dns_profile_steps(dns_handle* h, int n, double* ms, int* launches, int nclass) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (n < 1 || !ms || !launches || nclass < 4) return fail(DNS_ERR_ARG, "dns_profile_steps: bad arguments");
  if ((rc = use_device(h))) return rc;
  if (!h->w_valid) {
    DNS_CUDA(prime_work(h, h->stream), "dns_profile_steps initial transform");
    h->w_valid = true;
  }
  const int parts = 4;
  const int nk = parts * rk_stages(h) * n;
  std::vector<cudaEvent_t> ev(nk + 1);
  for (auto& e : ev) DNS_CUDA(cudaEventCreate(&e), "cudaEventCreate");
  PassArgs a = base_args(h);
  cudaError_t err = cudaEventRecord(ev[0], h->stream);
  int k = 0;
  for (int i = 0; i < n && err == cudaSuccess; ++i) {
    for (int s = 0; s < rk_stages(h) && err == cudaSuccess; ++s) {
      set_stage(h, s, a);
      for (int p = 0; p < parts && err == cudaSuccess; ++p) {
        err = h->ops->rk_stage_part(a, p, h->stream);
        if (err == cudaSuccess) err = cudaEventRecord(ev[++k], h->stream);
      }
    }
  }
  if (err == cudaSuccess) err = cudaEventSynchronize(ev[k]);
  for (int c = 0; c < nclass; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
  }
  for (int j = 1; j <= k && err == cudaSuccess; ++j) {
    float t = 0.f;
    err = cudaEventElapsedTime(&t, ev[j - 1], ev[j]);
    ms[(j - 1) % parts] += t;
    launches[(j - 1) % parts] += 1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) return cuda_fail(err, "dns_profile_steps");
  h->t += n * h->dt;
  return DNS_OK;
}

size_t dns_device_bytes(const dns_handle* h) { return h ? h->bytes : 0; }

const char* dns_last_error(const dns_handle* h) {
  (void)h;
  return g_err.c_str();
}

int dns_measure_fp64_peak(double* tflops) {
  if (!tflops) return fail(DNS_ERR_ARG, "dns_measure_fp64_peak: tflops is NULL");
  int dev = 0, sms = 0;
  DNS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  DNS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  const int blocks = 4 * sms, iters = 8192;
  double* sink = nullptr;
  DNS_CUDA(cudaMalloc(&sink, sizeof(double)), "dns_measure_fp64_peak sink");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t ce = cudaEventCreate(&t0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&t1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && ce == cudaSuccess; ++rep) {  // first launch warms up
    ce = cudaEventRecord(t0, 0);
    k_fp64_fma_probe<<<blocks, FMA_PROBE_THREADS>>>(sink, iters, 0.9999999, 1e-9);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaEventRecord(t1, 0);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(t1);
    float f = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&f, t0, t1);
    if (ce == cudaSuccess && rep > 0 && f < best) best = f;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(sink);
  if (ce != cudaSuccess) return cuda_fail(ce, "dns_measure_fp64_peak");
  const double flops = 2.0 * FMA_PROBE_CHAINS * (double)iters * blocks * FMA_PROBE_THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return DNS_OK;
}

int dns_debug_fail_alloc_after(int n) {
  if (n < 0) return fail(DNS_ERR_ARG, "dns_debug_fail_alloc_after: n < 0");
  g_fail_after.store(n);
  return DNS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Ensembles: many independent handles (any mix of grid sizes) advanced by one
// CUDA graph per step whose member chains are parallel branches over K streams.
// ---------------------------------------------------------------------------
constexpr int kEnsembleWholeGroups = 1 << 30;  // batch size meaning "whole group"

struct dns_ensemble {
  std::vector<dns_handle*> m;
  cudaStream_t main = nullptr;
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int streams = 0;  // per-member schedule: graph branches (0 = one per member)
  int batch = kEnsembleWholeGroups;  // members per batched launch (0 = per-member schedule)
  bool dirty = true;
  std::vector<unsigned> epochs;  // the members' epochs at the last capture
};

namespace {

// A unit of the step graph: one member stepped by its own kernels, or a batch
// of members of equal (N, precision, dealias rule, integrator) stepped by shared
// launches (their stage arguments at hargs + offset, one array of `count` per
// stage, copied into the kernels' parameters at capture).
struct EnsUnit {
  int first = 0;   // single member index, or -1 for a batch
  std::vector<int> members;
  size_t offset = 0;
};

void ens_free_graph(dns_ensemble* e) {
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  if (e->graph) cudaGraphDestroy(e->graph);
  e->gexec = nullptr;
  e->graph = nullptr;
}

// Work units of the current schedule: batches of at most e->batch members
// (batch > 0) for every batchable (N, dtype, kmax3) group, singles otherwise.
std::vector<EnsUnit> ens_units(const dns_ensemble* e) {
  std::vector<EnsUnit> units;
  const int n = (int)e->m.size();
  std::vector<bool> done(n, false);
  if (e->batch > 0) {
    for (int i = 0; i < n; ++i) {
      const dns_handle* h = e->m[i];
      if (done[i] || !h->ops->rk_stage_batch || h->closure) continue;
      std::vector<int> group;
      for (int j = i; j < n; ++j) {
        const dns_handle* g = e->m[j];
        if (!done[j] && !g->closure && g->ops == h->ops && g->variant == h->variant && g->plan == h->plan &&
            same_scheme(g->rk, h->rk)) {
          group.push_back(j);
          done[j] = true;
        }
      }
      const size_t per = (size_t)std::min(e->batch, BATCH_MAX_COUNT);
      for (size_t o = 0; o < group.size(); o += per) {
        EnsUnit u;
        u.first = -1;
        const size_t end = std::min(group.size(), o + per);
        u.members.assign(group.begin() + o, group.begin() + end);
        if (u.members.size() == 1) u.first = u.members[0];
        units.push_back(u);
      }
    }
  }
  for (int i = 0; i < n; ++i)
    if (!done[i]) {
      EnsUnit u;
      u.first = i;
      u.members.push_back(i);
      units.push_back(u);
    }
  return units;
}

int ens_capture(dns_ensemble* e, int K) {
  ens_free_graph(e);
  std::vector<EnsUnit> units = ens_units(e);
  // stage arguments of the batched units, uploaded once per capture
  std::vector<PassArgs> hargs;
  for (EnsUnit& u : units) {
    if (u.first >= 0) continue;
    u.offset = hargs.size();
    for (int s = 0; s < rk_stages(e->m[u.members[0]]); ++s)
      for (int i : u.members) {
        const dns_handle* h = e->m[i];
        PassArgs a = base_args(h);
        set_stage(h, s, a);
        hargs.push_back(a);
      }
  }
  const int nu = (int)units.size();
  if (K < 1 || K > nu) K = nu;
  while ((int)e->aux.size() < K) {
    cudaStream_t st;
    DNS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "ensemble stream");
    e->aux.push_back(st);
    cudaEvent_t ev;
    DNS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "ensemble event");
    e->join.push_back(ev);
  }
  DNS_CUDA(cudaStreamBeginCapture(e->main, cudaStreamCaptureModeThreadLocal), "ensemble capture begin");
  cudaError_t err = cudaEventRecord(e->fork, e->main);
  for (int k = 0; k < K && err == cudaSuccess; ++k) err = cudaStreamWaitEvent(e->aux[k], e->fork, 0);
  for (int u = 0; u < nu && err == cudaSuccess; ++u) {
    const EnsUnit& un = units[u];
    cudaStream_t st = e->aux[u % K];
    if (un.first >= 0) {
      err = enqueue_step(e->m[un.first], st);
    } else {
      const dns_handle* h = e->m[un.members[0]];
      const int cnt = (int)un.members.size();
      for (int s = 0; s < rk_stages(h) && err == cudaSuccess; ++s)
        err = h->ops->rk_stage_batch(hargs.data() + un.offset + (size_t)s * cnt, cnt, h->N + 2 * h->variant, st);
    }
  }
  for (int k = 0; k < K && err == cudaSuccess; ++k) {
    err = cudaEventRecord(e->join[k], e->aux[k]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(e->main, e->join[k], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(e->main, &g);
  if (err != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(err, "ensemble capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "ensemble capture end");
  e->graph = g;
  DNS_CUDA(cudaGraphInstantiate(&e->gexec, e->graph, 0), "ensemble graph instantiate");
  e->dirty = false;
  e->epochs.clear();
  for (const dns_handle* h : e->m) e->epochs.push_back(h->epoch);
  return DNS_OK;
}

int ens_prepare_members(dns_ensemble* e) {
  for (dns_handle* h : e->m) {
    if (!h->w_valid) {
      DNS_CUDA(prime_work(h, e->main), "ensemble initial transform");
      h->w_valid = true;
    }
  }
  // re-capture only when a member's options or forcing changed since the last capture
  if (e->epochs.size() != e->m.size()) e->dirty = true;
  for (size_t i = 0; i < e->m.size() && !e->dirty; ++i)
    if (e->epochs[i] != e->m[i]->epoch) e->dirty = true;
  return DNS_OK;
}

}  // namespace

extern "C" {

int dns_ensemble_create(int count, const int* N, const double* nu, const double* dt, int dtype, dns_ensemble** out) {
  if (!out) return fail(DNS_ERR_ARG, "dns_ensemble_create: out is NULL");
  *out = nullptr;
  if (count < 1 || !N || !nu || !dt) return fail(DNS_ERR_ARG, "dns_ensemble_create: need count >= 1 and N, nu, dt arrays");
  dns_ensemble* e = new dns_ensemble();
  int rc = DNS_OK;
  for (int i = 0; i < count && rc == DNS_OK; ++i) {
    dns_handle* h = nullptr;
    rc = dns_create(N[i], nu[i], dt[i], dtype, &h);
    if (rc == DNS_OK) e->m.push_back(h);
  }
  if (rc == DNS_OK) {
    cudaError_t ce = cudaStreamCreate(&e->main);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "dns_ensemble_create");
  }
  if (rc != DNS_OK) {
    std::string msg = g_err;
    dns_ensemble_destroy(e);
    g_err = msg;
    return rc;
  }
  for (dns_handle* h : e->m) h->stream = e->main;  // members are ordered on the ensemble's stream
  *out = e;
  return DNS_OK;
}

int dns_ensemble_destroy(dns_ensemble* e) {
  if (!e) return DNS_OK;
  if (e->main) cudaStreamSynchronize(e->main);
  ens_free_graph(e);
  for (dns_handle* h : e->m) {
    h->stream = h->own_stream;
    dns_destroy(h);
  }
  for (cudaStream_t st : e->aux) cudaStreamDestroy(st);
  for (cudaEvent_t ev : e->join) cudaEventDestroy(ev);
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->main) cudaStreamDestroy(e->main);
  delete e;
  return DNS_OK;
}

int dns_ensemble_size(const dns_ensemble* e) { return e ? (int)e->m.size() : 0; }

int dns_ensemble_member(dns_ensemble* e, int i, dns_handle** member) {
  if (!e || !member || i < 0 || i >= (int)e->m.size()) return fail(DNS_ERR_ARG, "dns_ensemble_member: bad index");
  *member = e->m[i];
  return DNS_OK;
}

int dns_ensemble_set_streams(dns_ensemble* e, int streams) {
  if (!e || streams < 0) return fail(DNS_ERR_ARG, "dns_ensemble_set_streams: bad arguments");
  e->streams = streams;
  e->dirty = true;
  return DNS_OK;
}

int dns_ensemble_set_batching(dns_ensemble* e, int max_batch) {
  if (!e || max_batch < 0) return fail(DNS_ERR_ARG, "dns_ensemble_set_batching: bad arguments");
  e->batch = max_batch;
  e->dirty = true;
  return DNS_OK;
}

int dns_ensemble_batching(const dns_ensemble* e) { return e ? e->batch : 0; }

int dns_ensemble_step(dns_ensemble* e, int n) {
  if (!e) return fail(DNS_ERR_ARG, "dns_ensemble_step: ensemble is NULL");
  if (n < 0) return fail(DNS_ERR_ARG, "dns_ensemble_step: n = %d < 0", n);
  if (n == 0) return DNS_OK;
  int rc = ens_prepare_members(e);
  if (rc) return rc;
  if (e->dirty || !e->gexec) {
    if ((rc = ens_capture(e, e->streams))) return rc;
  }
  for (int i = 0; i < n; ++i) DNS_CUDA(cudaGraphLaunch(e->gexec, e->main), "ensemble graph launch");
  for (dns_handle* h : e->m) h->t += n * h->dt;
  return DNS_OK;
}

int dns_ensemble_tune(dns_ensemble* e, int* best_streams) {
  if (!e) return fail(DNS_ERR_ARG, "dns_ensemble_tune: ensemble is NULL");
  // schedule, radix plans and y- and z-pass tile widths per size class: tuned on one
  // member (its state is kept), applied to every member of the class
  int rc = DNS_OK;
  std::vector<const DnsOps*> done_ops;
  std::vector<std::array<int, 4>> done_tiles;  // y-inverse, y-forward, z widths, radix plan
  for (dns_handle* h : e->m) {
    size_t k = 0;
    while (k < done_ops.size() && done_ops[k] != h->ops) ++k;
    if (k == done_ops.size()) {
      int ti = 0, tf = 0, tz = 0;
      if ((rc = dns_tune_tiles(h, 5, &ti, &tf, &tz))) return rc;
      done_ops.push_back(h->ops);
      done_tiles.push_back({ti, tf, tz, h->plan});
    } else if (h->ytile[0] != done_tiles[k][0] || h->ytile[1] != done_tiles[k][1] || h->ztile != done_tiles[k][2] ||
               h->plan != done_tiles[k][3]) {
      h->ytile[0] = done_tiles[k][0];
      h->ytile[1] = done_tiles[k][1];
      h->ztile = done_tiles[k][2];
      h->plan = done_tiles[k][3];
      h->graph_dirty = true;
      ++h->epoch;
      h->w_valid = false;
    }
  }
  rc = ens_prepare_members(e);
  if (rc) return rc;
  const int n = (int)e->m.size();
  // the schedule stored in the tune cache for this device, precision and member sizes
  std::map<int, int> census;
  for (dns_handle* h : e->m) ++census[h->N];
  std::string sizes;
  for (const auto& kv : census) sizes += (sizes.empty() ? "" : ",") + std::to_string(kv.first) + ":" + std::to_string(kv.second);
  const std::vector<std::string> ekey = {"ensemble", tc_device(e->m[0]->device), e->m[0]->dtype ? "f64" : "f32", sizes};
  std::vector<long> cached;
  if (tc_find(ekey, cached, 2) && cached[0] >= 0 && cached[1] >= 0 && cached[1] <= n) {
    e->batch = (int)cached[0];
    e->streams = (int)cached[1];
    e->dirty = true;
    if (best_streams) *best_streams = e->streams;
    return DNS_OK;
  }
  // candidate schedules: batched launches (whole groups, then smaller batches,
  // one graph branch per unit) and per-member launches over 1 .. n branches
  struct Cand {
    int batch, streams;
  };
  std::vector<Cand> cand = {{kEnsembleWholeGroups, 0}, {8, 0}};
  for (int k = 1; k < 2 * n; k *= 4) cand.push_back({0, k < n ? k : n});
  float best = 1e30f;
  Cand pick = cand[0];
  cudaEvent_t t0, t1;
  DNS_CUDA(cudaEventCreate(&t0), "tune event");
  DNS_CUDA(cudaEventCreate(&t1), "tune event");
  int taken = 0;
  for (const Cand& c : cand) {
    e->batch = c.batch;
    e->streams = c.streams;
    if ((rc = ens_capture(e, c.streams))) break;
    cudaError_t ce = cudaGraphLaunch(e->gexec, e->main);  // warm-up
    if (ce == cudaSuccess) ce = cudaEventRecord(t0, e->main);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(e->gexec, e->main);
    if (ce == cudaSuccess) ce = cudaEventRecord(t1, e->main);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(t1);
    if (ce != cudaSuccess) {
      rc = cuda_fail(ce, "dns_ensemble_tune");
      break;
    }
    taken += 2;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  for (dns_handle* h : e->m) h->t += taken * h->dt;
  if (rc) return rc;
  e->batch = pick.batch;
  e->streams = pick.streams;
  e->dirty = true;
  tc_put(ekey, {pick.batch, pick.streams});
  if (best_streams) *best_streams = pick.streams;
  return DNS_OK;
}

int dns_ensemble_streams(const dns_ensemble* e) { return e ? e->streams : 0; }

int dns_ensemble_synchronize(dns_ensemble* e) {
  if (!e) return fail(DNS_ERR_ARG, "dns_ensemble_synchronize: ensemble is NULL");
  DNS_CUDA(cudaStreamSynchronize(e->main), "dns_ensemble_synchronize");
  return DNS_OK;
}

int dns_ensemble_time_steps(dns_ensemble* e, int n, double* ms) {
  if (!e || n < 1 || !ms) return fail(DNS_ERR_ARG, "dns_ensemble_time_steps: bad arguments");
  int rc = ens_prepare_members(e);
  if (rc) return rc;
  if (e->dirty || !e->gexec) {
    if ((rc = ens_capture(e, e->streams))) return rc;
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t ce = cudaEventCreate(&t0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&t1);
  if (ce == cudaSuccess) ce = cudaEventRecord(t0, e->main);
  for (int i = 0; i < n && ce == cudaSuccess; ++i) ce = cudaGraphLaunch(e->gexec, e->main);
  if (ce == cudaSuccess) ce = cudaEventRecord(t1, e->main);
  if (ce == cudaSuccess) ce = cudaEventSynchronize(t1);
  float f = 0.f;
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&f, t0, t1);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (ce != cudaSuccess) return cuda_fail(ce, "dns_ensemble_time_steps");
  for (dns_handle* h : e->m) h->t += n * h->dt;
  *ms = f;
  return DNS_OK;
}

}  // extern "C"

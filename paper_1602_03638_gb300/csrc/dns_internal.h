// Host-side interface between the C-ABI layer and the per-(dtype, N)
// kernel instantiations. One DnsOps table exists for every supported grid
// size and precision; each entry enqueues kernels on the given stream and
// returns the launch status.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

struct dns_mlp;

namespace dns {

// Network forward on the given stream (mlp.cu): tau (6 x P) from features X (10 x P).
cudaError_t mlp_forward_async(::dns_mlp* net, const float* X, float* Y, int P, cudaStream_t st);

// Device buffers and scalars shared by all passes. Complex arrays use the
// internal spectral layout [component][kz][ky][kx] with kz < Nz/2 (the
// Nyquist plane kz = Nz/2 is identically zero and not stored).
struct PassArgs {
  void* U = nullptr;   // state u_hat at the start of the RK4 step (3 fields)
  void* U1 = nullptr;  // RK4 accumulator (3 fields)
  void* US = nullptr;  // RK4 stage state (3 fields)
  void* W = nullptr;   // work: 6 fields, transforms in flight
  void* D = nullptr;   // work: 1 field, divergence diagnostic
  const void* tw = nullptr;  // exp(-2 pi i t / TW), t < TW (TW = N on a cubic grid)
  const void* F = nullptr;   // optional force (3 fields, internal layout) added to N_hat
  double nu = 0.0;
  double cA = 0.0;  // a_s * dt
  double cB = 0.0;  // b_s * dt
  // low-storage 2N stage (Williamson): dU <- cA dU + cC RHS; u <- u + cB dU, with
  // cA = A_s, cB = B_s, cC = dt; U holds u and U1 holds dU
  int lsrk = 0;
  double cC = 0.0;
  int stage = 0;    // stage of the step, 0..last
  int last = 3;     // the step's final stage (it writes the new state); 3 for RK4
  int kmax3 = 0;    // a mode is kept by the 2/3 rule iff 3|k_i| < kmax3 (along x; all
                    // directions on a cubic grid)
  int kmax3y = 0, kmax3z = 0;  // the same along y and z (read where the counts differ)
  double ks[3] = {1.0, 1.0, 1.0};  // 2 pi / L along x, y, z: the wavenumber of index 1
  // FP32 copies of nu, cA, cB and ks for the FP32 kernels (filled when a kernel is
  // launched), so that they need no double-to-float conversion per thread
  float f_nu = 0.f, f_cA = 0.f, f_cB = 0.f, f_cC = 0.f;
  float f_ks[3] = {1.f, 1.f, 1.f};
  int ytile[2] = {0, 0};  // y-pass tile widths of the stage launches (inverse, forward); 0 = default
  int ztile = 0;          // z-pass tile width of the stage launches; 0 = default
  int plan = 0;           // radix plan variant per pass of the stage launches: bit PLAN_* set = AltPlan
  // Support of the state (PRUNE_*): PRUNE_ROWS when it vanishes on every row (kz, ky)
  // outside the 2/3 box, PRUNE_BOX when it also vanishes at |kx| >= N/3 on the rows inside.
  // The RK stage keeps such zeros (no nonlinear term there, the viscous term is
  // proportional to u_hat), so the stage's passes skip them: the x-stage and x inverse
  // leave the rows outside unwritten (and with PRUNE_BOX read and write the kept columns
  // only), the y-inverse transforms only the planes kz < kc and reads the rows outside the
  // box as zeros, the z-pass reads only kz < kc. The results are those of the full
  // transforms (the skipped terms are zeros).
  int prune = 0;
  const void* in = nullptr;  // physical input (3,Nx,Ny,Nz) for set_state
  void* out = nullptr;       // physical output (3,Nx,Ny,Nz) / RHS output
  double* partials = nullptr;          // diagnostics block partials
  unsigned long long* maxbits = nullptr;  // diagnostics max|div| (bits of a double)
};

struct DnsOps {
  int N;
  int dtype;  // 0 = FP32, 1 = FP64
  size_t elem_bytes;  // bytes of one complex value
  cudaError_t (*prepare)();  // one-time kernel attribute set-up
  // u_hat (state in a.US if from_stage else a.U) -> W[0..5] = x-inverse of (u, omega) / N^3
  cudaError_t (*x_inverse_curl)(const PassArgs& a, int from_stage, cudaStream_t s);
  // one RK4 stage on W (holding the x-inverse of the stage state); leaves
  // W holding the x-inverse of the next stage state
  cudaError_t (*rk_stage)(const PassArgs& a, cudaStream_t s);
  // the same stage one kernel at a time: part 0 y-inverse, 1 z-pass,
  // 2 y-forward, 3 x-stage (for per-kernel timing)
  cudaError_t (*rk_stage_part)(const PassArgs& a, int part, cudaStream_t s);
  // dU = RHS(U) in internal layout, written to a.out (3 fields)
  cudaError_t (*rhs)(const PassArgs& a, cudaStream_t s);
  // a.in (physical, device) -> U (spectral, Nyquist zeroed)
  cudaError_t (*forward3d)(const PassArgs& a, cudaStream_t s);
  // U -> a.out (physical, device); uses W[0..2] as scratch
  cudaError_t (*inverse3d)(const PassArgs& a, cudaStream_t s);
  // FP64 sums over U into a.partials (DIAG_BLOCKS x 4) and max|div u| into a.maxbits
  cudaError_t (*diag)(const PassArgs& a, cudaStream_t s);
  // rk_stage for `count` <= BATCH_MAX_COUNT independent members at once (same
  // N, precision and kmax3), their arguments in A[count]: one launch per pass,
  // the arguments travelling as kernel parameters. nullptr where one member
  // already fills the GPU (N > BATCH_MAX_N).
  cudaError_t (*rk_stage_batch)(const PassArgs* A, int count, int kmax3, cudaStream_t s);
  // tile widths (x columns per block) the stage's y-passes offer besides the
  // default, written to tiles[0..count); returns count (<= max)
  int (*y_tiles)(int* tiles, int max);
  // the same for the z-pass
  int (*z_tiles)(int* tiles, int max);
  int NY, NZ;  // points along y and z (N is the count along x)
  int TW;      // length of the twiddle table exp(-2 pi i t / TW) (a multiple of N, NY, NZ)
  int plans;   // radix plan variants the stage launches offer (1: the default only, 2: AltPlan too)
  int default_plan;  // the plan mask a new handle starts with
};

// values of PassArgs::prune
constexpr int PRUNE_NONE = 0, PRUNE_ROWS = 1, PRUNE_BOX = 2;

// bits of PassArgs::plan: the radix plan variant of each pass of a stage
constexpr int PLAN_X = 0, PLAN_YI = 1, PLAN_Z = 2, PLAN_YF = 3, PLAN_BITS = 4;

constexpr int BATCH_MAX_N = 128;
constexpr int BATCH_MAX_COUNT = 32;
struct BatchArgs {  // by-value kernel parameter (constant bank) of the batched passes
  PassArgs a[BATCH_MAX_COUNT];
};
static_assert(sizeof(BatchArgs) <= 32764, "kernel parameters are limited to 32764 bytes");

constexpr int DIAG_BLOCKS = 592;  // 4 x 148..152 SMs: one wave of 4 blocks per SM

// Lookup of the instantiation for (dtype, N) or (dtype, Nx, Ny, Nz); nullptr if unsupported.
const DnsOps* find_ops(int dtype, int N);
const DnsOps* find_ops3(int dtype, int Nx, int Ny, int Nz);

// Closure helpers on the internal layout (sgs.cu): G3 = i k_j u_hat_comp (j = 0..2),
// F3 = -i k_j tau_hat_ij from the 6 stress components (00 11 22 01 02 12); fill of a
// float array.
cudaError_t closure_gradient(const void* U, int N, int comp, void* G3, int dtype, cudaStream_t st);
cudaError_t closure_force(const void* S6, int N, void* F3, int dtype, cudaStream_t st);
cudaError_t fill_f32(float* p, size_t n, float v, cudaStream_t st);

}  // namespace dns

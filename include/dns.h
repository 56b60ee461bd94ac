/*
 * C ABI of the GB300 pseudo-spectral Navier-Stokes solver.
 *
 * The library advances the Galerkin ODE of Eq. NSfinal (Mortensen &
 * Langtangen, arXiv 1602.03638, Sec. 2)
 *
 *     d u_hat/dt = P[ mask * F(u x omega) ] - nu |k|^2 u_hat,
 *     P(v) = v - k (k.v)/|k|^2,   omega_hat = i k x u_hat,
 *
 * on the triply periodic box [0, 2 pi]^3 with N^3 points (Eq. realmesh),
 * using the classical RK4 driver of the paper's Appendix and the 2/3-rule
 * dealiasing of Sec. 3.1. Every step of the path runs in the library's own
 * CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Every function returns an int status: DNS_OK (0) or a negative dns_status.
 *   No function aborts the process. dns_last_error() gives a message.
 * - Precision: DNS_F32 (float / complex float) or DNS_F64 (double / complex
 *   double); all array arguments use the handle's precision.
 * - Physical arrays: real, shape (3, N, N, N), C order, x slowest
 *   (u[c][i][j][k] = u_c(2 pi i/N, 2 pi j/N, 2 pi k/N)).
 * - Spectral arrays: interleaved complex, shape (3, N, N, N/2+1), C order
 *   [c][kx][ky][kz] as in Sec. 3.1: kx, ky in FFT order (0..N/2-1, -N/2..-1),
 *   kz = 0..N/2. Transforms are unnormalised forward (e^{-ik.x}) and
 *   1/N^3-normalised inverse.
 * - The state never carries Nyquist modes: on input every mode with
 *   |kx| = N/2, |ky| = N/2 or kz = N/2 is set to zero, and the method keeps
 *   them zero (they lie outside the dealiasing box).
 * - Pointers: `on_device` = 1 means a CUDA device pointer (16-byte aligned,
 *   e.g. a torch tensor's data_ptr()); 0 means host memory (pinned host
 *   memory gives the fastest copies). The caller owns every buffer it
 *   passes; the library copies in and out and keeps no reference.
 * - Streams: work is enqueued on the handle's stream (dns_set_stream);
 *   dns_step returns after enqueueing, and kernel errors surface at the next
 *   call that synchronises (dns_get_state*, dns_diagnostics, dns_rhs).
 * - Supported N: 8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 512, 1024.
 * - Grids with other point counts per direction (dns_create3): the shapes above
 *   become (3, Nx, Ny, Nz) and (3, Nx, Ny, Nz/2+1), kx in the FFT order of Nx, ky
 *   of Ny, kz = 0..Nz/2; the inverse carries 1/(Nx Ny Nz) and the Nyquist modes
 *   are |kx| = Nx/2, |ky| = Ny/2, kz = Nz/2. Compiled: 32 x 16 x 24,
 *   24 x 48 x 16 and 1024 x 512 x 256 in both precisions.
 */
#ifndef DNS_GB300_H
#define DNS_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dns_handle dns_handle;

typedef enum { DNS_F32 = 0, DNS_F64 = 1 } dns_dtype;

typedef enum {
  DNS_OK = 0,
  DNS_ERR_ARG = -1,         /* invalid argument (N, dtype, pointer, option, ...) */
  DNS_ERR_OOM = -2,         /* device allocation failed */
  DNS_ERR_CUDA = -3,        /* a CUDA call or kernel failed */
  DNS_ERR_NONFINITE = -4,   /* the state holds NaN or Inf */
  DNS_ERR_TIMEOUT = -5,     /* a bounded device wait gave up (1 s): the tensor-core MLP kernels */
  DNS_ERR_UNSUPPORTED = -6  /* no usable sm_103 device, or N not instantiated */
} dns_status;

/* Diagnostics, all computed in FP64 on the device (Appendix energy; the
 * workshop quantities named in Sec. 4 "Verification"):
 *   t           simulated time (number of steps taken times dt)
 *   energy      E   = 1/2 <|u|^2>            (grid mean, Appendix reduce)
 *   dissipation eps = nu <|omega|^2>
 *   max_div     max over the mesh of |div u| = |F^{-1}(i k . u_hat)|
 *   helicity    H   = <u . omega>
 *   enstrophy   Z   = 1/2 <|omega|^2>
 * E, eps, H, Z use the spectral (Parseval) sums over the half spectrum. */
typedef struct {
  double t, energy, dissipation, max_div, helicity, enstrophy;
} dns_diag;

/* Creates a solver for an N^3 grid with viscosity nu and time step dt in the
 * given precision; allocates 16 complex component-volumes of N^2 (N/2) values
 * on the current CUDA device (state, RK4 base/accumulator/stage, 6+1 work
 * fields). Sec. 3.1 (mesh, wavenumbers, arrays) and the Appendix constants.
 * Errors: DNS_ERR_ARG (N unsupported, nu < 0, dt <= 0, dtype, out NULL),
 * DNS_ERR_UNSUPPORTED (no compute capability 10.3 device), DNS_ERR_OOM. */
int dns_create(int N, double nu, double dt, int dtype, dns_handle** out);

/* Creates a solver for a grid of Nx x Ny x Nz points (x, y, z), the Sec. 2
 * footnote's other numbers of points per direction: x_i = Lx i / Nx and so on
 * (Eq. realmesh per direction), wavenumbers in the FFT order of each count
 * (Sec. 3.1), the 2/3 rule |k_i| < N_i/3 per direction (2/3 (N_i/2+1) with
 * "dealias_variant" 1), the inverse transform normalised by 1/(Nx Ny Nz).
 * Array shapes and errors as for dns_create; Nx = Ny = Nz is the same as
 * dns_create(Nx, ...). The other counts run the generic passes: the options
 * "fft_plan", "y_tile_*" and "z_tile" offer only their defaults, and
 * dns_set_closure and ensembles take cubic grids only. dns_get_option reads
 * the counts back as "Nx", "Ny", "Nz" (on any handle).
 * Errors: DNS_ERR_ARG (the shape is not compiled, see the list above), as for
 * dns_create otherwise. */
int dns_create3(int Nx, int Ny, int Nz, double nu, double dt, int dtype, dns_handle** out);

/* Frees everything the handle owns. NULL is accepted. */
int dns_destroy(dns_handle* h);

/* Stream for all subsequent work (a cudaStream_t; NULL = the handle's own
 * stream, created at dns_create). */
int dns_set_stream(dns_handle* h, void* stream);

/* Options:
 *   "dealias_variant"  0: keep |k_i| < N/3 (Sec. 3.1 text, default)
 *                      1: keep |k_i| < 2/3 (N/2+1) (the Appendix script)
 *   "integrator"       explicit Runge-Kutta scheme of dns_step; 0 - 3 in the
 *                      two-register form of the Appendix driver (stage s + 1
 *                      starts from u0 + b_s dt dU_s, the new state is
 *                      u0 + sum_s a_s dt dU_s), 4 - 5 in Williamson's 2N
 *                      low-storage form (see dns_set_rk_tableau):
 *                      0: classical RK4, a = 1/6,1/3,1/3,1/6, b = 1/2,1/2,1
 *                         (Appendix, default)
 *                      1: forward Euler, a = 1 (the integrator loop of Sec. 3.1)
 *                      2: Heun, a = 1/2,1/2, b = 1
 *                      3: midpoint, a = 0,1, b = 1/2
 *                      4: Williamson's 3-stage 3rd-order 2N scheme
 *                         (A = 0, -5/9, -153/128; B = 1/3, 15/16, 8/15)
 *                      5: Carpenter & Kennedy's 5-stage 4th-order 2N scheme
 *                      dns_get_option reports -1 after dns_set_rk_tableau set a
 *                      scheme that is none of these
 *   "Lx", "Ly", "Lz"   box lengths (default 2 pi each): the mesh spacing along x is
 *                      Lx / N and the wavenumber of index l is 2 pi l / Lx (Sec. 2
 *                      footnote, Sec. 3.1: other box sizes by scaling). The 2/3
 *                      rule acts on the indices; the SGS helpers assume 2 pi.
 *   "y_tile_inverse", "y_tile_forward"
 *                      x columns per block of the stage's inverse and forward
 *                      y-passes: 0 (default) or a width the grid offers (4, 8, 16,
 *                      32 as far as they divide N and fit 256-byte rows; N <= 128
 *                      only). The arithmetic of every column is the same, so the
 *                      results do not depend on it; see dns_tune_tiles.
 *   "z_tile"           x columns per block of the generic z-pass of the small
 *                      grids: 0 (default) or an offered width (4 .. 32); results
 *                      independent of it, see dns_tune_tiles.
 *   "fft_plan"         radix schedule of the line transforms of each pass of a stage,
 *                      N <= 128 only: a bit mask, bit 0 the x-stage (and the x inverse
 *                      before the first stage), bit 1 the y-inverse, bit 2 the z-pass,
 *                      bit 3 the y-forward; a clear bit keeps the default schedule
 *                      (radix-8/16 passes, radix 3 last), a set bit takes radix 3 first,
 *                      then radix-4 passes (one radix-8 pass for odd powers of two).
 *                      The same transforms with another rounding order: results agree
 *                      to round-off, not bit for bit; dns_tune_tiles picks the bits by
 *                      timing. 0 .. 15; only 0 on the other grids. A new handle starts with
 *                      the mask measured fastest per grid size and precision on GB300
 *                      (dns_get_option reads it).
 *   "use_graph"        1: dns_step replays a captured CUDA graph (default)
 *   "prune_rows"       1 (default): where the state vanishes on every row (kz, ky)
 *                      outside the 2/3 box (checked on the device, and read back, by
 *                      dns_set_state, dns_set_state_spectral and a change of
 *                      "dealias_variant", which therefore synchronise the stream), the
 *                      stage's passes skip those rows: the RK stage keeps them zero
 *                      (no nonlinear term there, a viscous term proportional to u_hat;
 *                      Eq. NSfinal), so their transforms are transforms of zeros. The
 *                      x-stage and the x inverse leave them alone, the y-inverse
 *                      transforms only the planes kz < Nz/3 and reads the other rows as
 *                      zeros, the z-pass reads only kz < Nz/3; where the state also
 *                      vanishes at |kx| >= Nx/3, the x-stage reads and writes its rows at
 *                      the kept columns only. The results equal the full transforms bit
 *                      for bit (exact zeros of either sign); the RK registers and work
 *                      fields of the skipped rows are left unwritten. 0: the full
 *                      transforms whatever the state.
 *   "nu", "dt"         change the viscosity / time step
 *   "time"             set the simulated time reported by dns_diagnostics
 * Errors: DNS_ERR_ARG for an unknown key or a value out of range. */
int dns_set_option(dns_handle* h, const char* key, double value);

/* The current value of an option of dns_set_option ("time" included), or of the
 * read-only keys, in *value: the grid counts "Nx", "Ny", "Nz"; "rows_vanish" 1 if the
 * state vanishes on every row (kz, ky) outside the 2/3 box, else 0, and "box_vanish" 1 if
 * it vanishes at every mode outside the box (what "prune_rows" uses, as checked by the
 * last dns_set_state* or change of "dealias_variant").
 * Errors: DNS_ERR_ARG for an unknown key or a NULL pointer. */
int dns_get_option(const dns_handle* h, const char* key, double* value);

/* A user-supplied explicit Runge-Kutta scheme for dns_step (Sec. 3.1: "more
 * advanced integrators may be easily added"), in one of two two-register forms:
 *   form 0 (the Appendix driver's): stages >= 1 weights a[0..stages-1] and
 *     offsets b[0..stages-2]; stage s evaluates dU_s = RHS(stage state), stage
 *     s + 1 starts from u0 + b_s dt dU_s, the new state is u0 + sum a_s dt dU_s
 *     (Butcher tableaux whose only non-zero entries are A[s+1][s] = b_s);
 *   form 1 (Williamson's 2N low-storage form): A = a[0..stages-1], B =
 *     b[0..stages-1]; stage s does dU <- A_s dU + dt RHS(u), u <- u + B_s dU
 *     (a[0] multiplies a zero register and is ignored).
 * 1 <= stages <= 8; coefficients must be finite. The arrays are copied. Each
 * stage costs the same four passes; the step reads and writes the same state
 * arrays as the built-in schemes. Errors: DNS_ERR_ARG. */
int dns_set_rk_tableau(dns_handle* h, int form, int stages, const double* a, const double* b);

/* Schedule tuner: times dns_step with both radix plans of each pass ("fft_plan" bits,
 * N <= 128) and every tile width the grid offers for the y-inverse, the y-forward and the
 * z-pass (N <= 128; defaults included), one knob at a time (the plan bits, then the widths)
 * with the best values found before it, three timings of `steps` graph replays each
 * after a capture and a warm-up step; a candidate replaces the one kept so far
 * (starting from the default) only if its median time beats that one's median by
 * more than that one's spread (max - min); the kept widths are written to
 * *y_inverse, *y_forward, *z (0 = default), the kept plan is the handle's "fft_plan".
 * Every candidate starts from the same state, and the state and time
 * are restored at the end; the results of later steps do not depend on the widths
 * (the plan changes their rounding only). Allocates and frees one state copy (3
 * fields). Synchronises. Errors: DNS_ERR_ARG (steps < 1, NULL outputs),
 * DNS_ERR_OOM, DNS_ERR_CUDA. */
int dns_tune_tiles(dns_handle* h, int steps, int* y_inverse, int* y_forward, int* z);

/* Tune cache (no counterpart in the paper; the tuners' choices kept across runs):
 * with a path set, dns_tune_tiles first looks for a stored choice for the handle's
 * device (its name), grid counts and precision and applies it without timing (the
 * state is untouched); otherwise it tunes and appends its choice. dns_ensemble_tune
 * does the same for its schedule, keyed by device, precision and the members' sizes
 * with their counts (a stored schedule is applied without advancing the members;
 * the size classes' plans and widths come from the tiles entries). The file is plain
 * text, one entry per line, the last matching line wins:
 *   tiles <device> <Nx> <Ny> <Nz> <f32|f64> <y_inverse> <y_forward> <z> <fft_plan>
 *   ensemble <device> <f32|f64> <N:count,...> <max_batch> <streams>
 * with blanks in the device name written as '_'; a stored value the grid does not
 * offer makes the tuner time again. Process-wide; NULL or "" turns it off (the
 * default). Errors: DNS_ERR_ARG if the file cannot be opened for appending. */
int dns_set_tune_cache(const char* path);

/* The stored tiles entry of the tune cache for (device, Nx, Ny, Nz, dtype): returns 1
 * and writes the widths and the plan mask when found, 0 when not (or no cache is set),
 * DNS_ERR_ARG for a NULL argument. Host only; needs no device. */
int dns_tune_cache_lookup(const char* device, int Nx, int Ny, int Nz, int dtype, int* y_inverse, int* y_forward,
                          int* z, int* plan);

/* The tile widths a grid offers the tuner besides the default: which = 0 the
 * y-passes ("y_tile_inverse", "y_tile_forward"), 1 the z-pass ("z_tile"), for
 * the compiled grid (N, dtype). Writes up to `max` widths to `widths` and returns
 * their count (0: the grid offers the defaults only), or DNS_ERR_ARG. Needs no
 * device. The paper has no counterpart. */
int dns_tile_widths(int N, int dtype, int which, int* widths, int max);

/* State from a physical velocity field u (3,N,N,N): u_hat = F(u) with the
 * Nyquist modes zeroed (Eq. iffteq forward transform; no projection).
 * Resets the time to 0. Checks where the state vanishes (option "prune_rows") and
 * synchronises the stream. */
int dns_set_state(dns_handle* h, const void* u, int on_device);

/* State from spectral coefficients (3,N,N,N/2+1), complex, paper order;
 * Nyquist modes are zeroed. Resets the time to 0. Checks where the state vanishes
 * (option "prune_rows") and synchronises the stream. */
int dns_set_state_spectral(dns_handle* h, const void* uhat, int on_device);

/* Enqueues n >= 0 steps of Eq. NSfinal with the handle's integrator (default
 * the classical RK4 of the Appendix: a = 1/6,1/3,1/3,1/6, b = 1/2,1/2,1).
 * Asynchronous. */
int dns_step(dns_handle* h, int n);

/* Physical velocity u = F^{-1}(u_hat), (3,N,N,N). Synchronises the stream. */
int dns_get_state(dns_handle* h, void* u, int on_device);

/* Spectral state (3,N,N,N/2+1) complex, paper order (kz = N/2 plane = 0).
 * Synchronises the stream. */
int dns_get_state_spectral(dns_handle* h, void* uhat, int on_device);

/* One evaluation of the right-hand side of Eq. NSfinal at the current state,
 * written as (3,N,N,N/2+1) complex in paper order (computeRHS of Sec. 3.1).
 * Does not change the state. Synchronises the stream. */
int dns_rhs(dns_handle* h, void* duhat, int on_device);

/* FP64 diagnostics of the current state (see dns_diag). Synchronises.
 * Returns DNS_ERR_NONFINITE (with *out filled) if any NaN/Inf is present. */
int dns_diagnostics(dns_handle* h, dns_diag* out);

/* Measurement aid: advances n >= 1 steps exactly like dns_step but
 * launches the kernels one by one (no graph) with a CUDA event after each,
 * and returns per kernel class the summed device time in ms[c] and the
 * launch count in launches[c]: c = 0 y-inverse, 1 z-pass (c2r, u x omega, r2c),
 * 2 y-forward, 3 x-stage (forward x, mask, projection, viscous term, stage update,
 * next inverse x). nclass must be >= 4. Synchronises. */
int dns_profile_steps(dns_handle* h, int n, double* ms, int* launches, int nclass);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (2 flops per
 * FMA): independent chains of dependent FMAs on 4 blocks of 256 threads per SM,
 * best of three CUDA-event-timed launches after one warm-up. The denominator of
 * the FP64 form's arithmetic roofline (its step is bound by FP64 arithmetic, not
 * HBM). Allocates 8 bytes; synchronous. The paper has no counterpart. */
int dns_measure_fp64_peak(double* tflops);

/* Bytes of device memory the handle owns. */
size_t dns_device_bytes(const dns_handle* h);

/* Message of the last failed call on this thread (h may be NULL). Never NULL. */
const char* dns_last_error(const dns_handle* h);

/* Energy, dissipation, helicity and enstrophy of a caller-supplied spectral
 * velocity field, computed without allocating any device memory. (The paper
 * has no counterpart: this is a library service.)
 *
 * For callers that cannot call cudaMalloc -- a process whose device memory is
 * entirely owned by another allocator (e.g. a framework's caching pool that has
 * reserved the device), or a time-critical loop that must not take the
 * device-wide synchronisation of cudaMalloc/cudaFree. No handle is needed.
 *
 *   uhat   device pointer, 16-byte aligned: (3, N, N, N/2+1) complex in the
 *          public spectral layout, precision `dtype` (DNS_F32 / DNS_F64)
 *   N      even, 2 <= N <= 2048 (larger N is rejected with DNS_ERR_ARG)
 *   nu     viscosity used for the dissipation
 *   out    device pointer to 5 doubles, 8-byte aligned: energy, dissipation,
 *          helicity, enstrophy (same definitions and FP64 sums as
 *          dns_diagnostics on the [0, 2 pi]^3 box), then the number of
 *          non-finite modes. The wavenumber of index k is k: for a field of a
 *          handle whose box lengths were changed (options "Lx", "Ly", "Lz"),
 *          dns_diagnostics scales each index by 2 pi / L and the vorticity sums
 *          (dissipation, helicity, enstrophy) differ from these
 *   stream cudaStream_t the two kernels are enqueued on (NULL = legacy default)
 *
 * Asynchronous: returns after enqueueing; read `out` after synchronising.
 * Partial sums go to a fixed 32 KB array inside the library that every GPU
 * loading the library holds until exit; every call overwrites all of it before
 * reading it. Calls that overlap on the GPU (e.g. on two streams at once) share
 * that array and race: serialise them. The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it for the life
 * of the process; make that first call before any stream capture, and do not
 * call this entry point after a cudaDeviceReset of that device in the same
 * process (the kept address would be stale). Calls no cudaMalloc, cudaFree or
 * other allocating routine. */
int dns_spectral_sums_noalloc(const void* uhat, int N, int dtype, double nu, double* out, void* stream);

/* ---- Ensembles (many independent runs of mixed grid sizes) ------------------
 * An ensemble owns `count` handles created as by dns_create(N[i], nu[i], dt[i],
 * dtype). dns_ensemble_step(e, n) advances every member by n steps of its
 * integrator (RK4 unless set on the member's handle; Sec. 3, Appendix driver);
 * each step is one launch of a CUDA graph.
 * Schedule: with batching on (default), members of equal N (N <= 128),
 * precision, dealias option, radix plan and integrator are advanced together, one kernel launch per
 * pass for up to min(max_batch, 32) members (their pointers and RK
 * coefficients passed as kernel parameters); every batch, and every member that is not batched, is
 * a parallel branch of the graph. With batching off (max_batch = 0) every
 * member runs its own kernels and the members are spread over `streams`
 * branches (0 = one branch per member). dns_ensemble_tune first tunes the
 * radix plan and tile widths of each grid size class on one of its members
 * (dns_tune_tiles, "fft_plan" and the y- and z-pass widths; that member's state is
 * kept) and gives every member of the class the plan and widths found (batched
 * launches use the widths where the batch's members agree), then times a set of
 * schedules (batched, and per-member over 1 .. count branches) on the actual
 * members and keeps the fastest; it ADVANCES every member by 2 steps per
 * schedule tried (the count is returned in the members' time, dns_diag.t) and
 * writes the chosen branch count of the per-member schedule (0 when batched).
 * Members are ordinary handles for every other call (set_state, get_state,
 * diagnostics, ...) and all run on the ensemble's stream; do not destroy them
 * or change their stream. Results are identical to stepping each member alone
 * (the batched kernels run the same per-member arithmetic). Errors:
 * DNS_ERR_ARG for bad arguments, DNS_ERR_CUDA/OOM from capture or launch. */
typedef struct dns_ensemble dns_ensemble;
int dns_ensemble_create(int count, const int* N, const double* nu, const double* dt, int dtype, dns_ensemble** out);
int dns_ensemble_destroy(dns_ensemble* e);
int dns_ensemble_size(const dns_ensemble* e);
int dns_ensemble_member(dns_ensemble* e, int i, dns_handle** member);
int dns_ensemble_set_streams(dns_ensemble* e, int streams); /* 0 = one branch per member */
int dns_ensemble_streams(const dns_ensemble* e);            /* branch count (0 = per member) */
int dns_ensemble_set_batching(dns_ensemble* e, int max_batch); /* 0 = off; else members per launch */
int dns_ensemble_batching(const dns_ensemble* e);              /* current max_batch (0 = off) */
int dns_ensemble_tune(dns_ensemble* e, int* best_streams);  /* advances the members, see above */
int dns_ensemble_step(dns_ensemble* e, int n);              /* asynchronous */
int dns_ensemble_synchronize(dns_ensemble* e);
/* n ensemble steps timed on the device: CUDA events recorded on the ensemble's
 * stream around the n graph launches; synchronises and writes the elapsed
 * milliseconds to *ms. Advances every member by n steps like dns_ensemble_step. */
int dns_ensemble_time_steps(dns_ensemble* e, int n, double* ms);

/* ---- Transforms and forcing on a handle ---------------------------------------
 * dns_transform_r2c: F of 3 physical fields (3,N,N,N) (device) into the public
 *   spectral layout (3,N,N,N/2+1) (device), Nyquist modes zeroed; does not touch
 *   the state. dns_transform_c2r: the inverse (1/N^3 included, the c2r reading
 *   of include/dns.h's header). Both are asynchronous on the handle's stream and
 *   use the handle's work buffers (Eqs. fft/ifft, Sec. 2).
 * dns_set_forcing: a spectral force f (3,N,N,N/2+1), public layout, added to
 *   the nonlinear term before the 2/3 mask and the projection at every stage of
 *   every following step (used by the learned closure, -i k_j tau_hat_ij); the
 *   library keeps its own copy; f = NULL removes the force. Host input is copied
 *   synchronously; device input is read on the handle's stream. */
int dns_transform_r2c(dns_handle* h, const void* phys3, void* spec3);
int dns_transform_c2r(dns_handle* h, const void* spec3, void* phys3);
int dns_set_forcing(dns_handle* h, const void* f3, int on_device);

/* ---- Learned subgrid-stress closure: spectral helpers ------------------------
 * Standalone kernels on caller-owned device arrays, enqueued on `stream`
 * (a cudaStream_t, NULL = legacy default); spectral arrays in the public layout.
 * The paper has no closure model; these serve the closure chosen for the
 * coarse-grid runs (box filter of width 2 pi/Nc, gradient features, SGS stress
 * tau_ij = filter(u_i u_j) - ubar_i ubar_j, components 00 11 22 01 02 12).
 *   dns_spectral_filter:   coarse(3,Nc..) = (Nc/Nf)^3 prod_i sinc(k_i pi/Nc) fine(3,Nf..)
 *                          for |k_i| < Nc/2, zero elsewhere (Nc <= Nf, both even)
 *   dns_spectral_gradient: grad9[3 i + j] = i k_j uhat_i        (9 spectral fields)
 *   dns_stress_force:      force3[i] = -i sum_j k_j tauhat[ij]  (6 -> 3 spectral fields)
 *   dns_pointwise_products: prod6 = (u0u0, u1u1, u2u2, u0u1, u0u2, u1u2)  (physical)
 *   dns_subtract_products:  tau6 -= products of ubar3 (same order)        (physical) */
int dns_spectral_filter(const void* fine, int Nf, void* coarse, int Nc, int dtype, void* stream);
int dns_spectral_gradient(const void* uhat3, int N, void* grad9, int dtype, void* stream);
int dns_stress_force(const void* tauhat6, int N, void* force3, int dtype, void* stream);
int dns_pointwise_products(const void* u3, int N, void* prod6, int dtype, void* stream);
int dns_subtract_products(void* tau6, const void* ubar3, int N, int dtype, void* stream);

/* ---- Learned subgrid-stress closure: the pointwise network -------------------
 * 10 inputs (9 resolved velocity gradients + filter width) -> 64 SiLU -> 64 SiLU
 * -> 6 stress components, BF16 tensor-core products with FP32 accumulation and
 * FP32 master weights. Parameter vector (dns_mlp_param_count() = 5286 floats):
 * in_shift[10] in_scale[10] W1[10][64] b1[64] W2[64][64] b2[64] W3[64][6] b3[6]
 * out_scale[6] out_shift[6]; inputs are standardised as (x - in_shift) *
 * in_scale and tau = y * out_scale + out_shift. Arrays are planar FP32 device
 * arrays: X[f * P + p] (10 x P), tau[c * P + p] (6 x P). Training minimises the
 * mean squared error of the standardised stress with Adam (beta 0.9, 0.999,
 * eps 1e-8) on W1..b3; the normalisation entries are fixed. */
typedef struct dns_mlp dns_mlp;
int dns_mlp_param_count(void);
int dns_mlp_create(dns_mlp** out);
int dns_mlp_destroy(dns_mlp* net);
int dns_mlp_set_params(dns_mlp* net, const float* host_params, int count); /* resets Adam */
int dns_mlp_get_params(dns_mlp* net, float* host_params, int count);
int dns_mlp_forward(dns_mlp* net, const float* X, float* tau, int P, void* stream);
/* Sets the normalisation entries from data: in_shift = mean and in_scale = 1 /
 * std of each feature row of X (scale 1 where std <= 1e-12), out_shift = mean
 * and out_scale = std of each stress row of T (1 where std <= 1e-30); std is the
 * unbiased (P - 1) standard deviation, both sums in FP64 in a device kernel.
 * X (10 x P) and T (6 x P) device arrays, P >= 2; asynchronous on `stream`. */
int dns_mlp_set_normalisation(dns_mlp* net, const float* X, const float* T, int P, void* stream);
/* loss and the gradient of every parameter (zeros for the normalisation entries), synchronous */
int dns_mlp_loss_grad(dns_mlp* net, const float* X, const float* T, int P, float* grad_host, float* loss_host,
                      void* stream);
/* one Adam step on the full batch; loss_host (may be NULL) receives the loss before the update */
int dns_mlp_train_step(dns_mlp* net, const float* X, const float* T, int P, double lr, float* loss_host,
                       void* stream);

/* Attaches the network as a subgrid-stress closure of the handle's run (no
 * counterpart in the paper: the learned closure of the coarse-grid runs). From
 * the next step on, every dns_step (and dns_rhs) first evaluates, on the
 * handle's stream and inside its captured graph, with no host synchronisation:
 * the resolved velocity gradients A_ij = F^{-1}(i k_j u_hat_i) (9 inverse
 * transforms) and the filter width `delta` as the 10 features of every grid
 * point, the network's stress tau (6 components), its forward transforms, and
 * the force f_i = -i k_j tau_hat_ij, which is added to the nonlinear term before
 * the 2/3 mask and the projection in every stage of the step (held over the
 * step, as the force of dns_set_forcing). `net` is borrowed: keep it alive and
 * attached only while the handle steps (parameter changes by training between
 * steps are seen by the next step); net = NULL detaches. FP32 handles of cubic
 * grids on the 2 pi box only (DNS_ERR_UNSUPPORTED otherwise); not together with
 * dns_set_forcing (DNS_ERR_ARG). Allocates its scratch (10 + 6 floats per grid
 * point and 21 spectral fields) and two side streams on the first attach: the three
 * gradient transforms and the two stress transforms are independent and run
 * concurrently (forked from and joined back into the handle's stream). */
int dns_set_closure(dns_handle* h, dns_mlp* net, double delta);

/* Test hook for allocation-failure handling: the n-th device allocation made
 * by the library from now on (n >= 1) reports DNS_ERR_OOM without touching
 * the device; n = 0 disables the hook. */
int dns_debug_fail_alloc_after(int n);


#ifdef __cplusplus
}
#endif

#endif /* DNS_GB300_H */

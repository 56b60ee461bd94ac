// Fused kernels of one RK4 right-hand-side evaluation and its stage update,
// templated on the precision T and the grid size N (N = 2^a or 3*2^a). The
// generic passes also take per-direction point counts (Sec. 2 footnote): N is
// then the count along x, NY and NZ those along y and z (defaults N).
//
// Per RK4 stage (Eq. NSfinal with the Appendix's RK4 driver) the state goes
// through four passes over HBM:
//   y-inverse  : complex inverse transform along y of the 6 fields u, omega
//   z-pass     : c2r along z of the 6 fields, u x omega in registers/shared
//                memory (Eq. curl_convection), r2c along z of the 3 products;
//                only kz < N/3 is written (the rest is removed by the 2/3 mask)
//   y-forward  : forward transform along y, only |ky| < N/3 rows written
//   x-stage    : forward transform along x, dealias mask, projection
//                N - k (k.N)/|k|^2, viscous term -nu |k|^2 u, RK4 axpy, then
//                curl i k x u of the new stage state and the inverse transform
//                along x of u and omega for the next stage (the paper's slab
//                transposes become the change of pass direction).
// Physical fields never leave the z-pass. Spectral arrays use the layout
// [component][kz][ky][kx], kz < N/2, kx and ky in FFT order.
#pragma once

#include <type_traits>

#include "dns_internal.h"
#include "fft_core.cuh"

namespace dns {

constexpr int XP_THREADS = 192;  // 6 warps: one per line of a row (u, omega)
constexpr int YP_THREADS = 256;
constexpr int ZP_THREADS = 256;
constexpr int DG_THREADS = 256;

constexpr int pow2_part(int n) {
  int r = 1;
  while (n % (r * 2) == 0) r *= 2;
  return r;
}
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int odd_ld(int lines) { return (lines % 2) ? lines : lines + 1; }
constexpr int igcd(int a, int b) { return b == 0 ? a : igcd(b, a % b); }
constexpr int ilcm(int a, int b) { return a / igcd(a, b) * b; }

// Grid of N x NY x NZ points (x, y, z); the spectral fields hold kz < NZ/2.
template <typename T, int N, int NY = N, int NZ = N>
struct Geometry {
  static constexpr int M = NZ / 2;
  static constexpr size_t FS = (size_t)M * NY * N;  // complex values per field
  // length of the twiddle table exp(-2 pi i t / TW): every line length divides it
  static constexpr int TW = ilcm(ilcm(N, NY), NZ);
  static constexpr int CB = (int)sizeof(cx<T>);
  // x-pass: one row (fixed kz, ky) per block, 6 padded line buffers. The
  // stage update (XPRE, where it fits in 100 KB) uses 3 padded lines (the
  // nonlinear term, then u) and 9 unpadded rows that receive the stage's state
  // rows by cp.async (then omega in rows 0-2 and the padded work lines of the
  // omega transforms over rows 3-8).
  // Where 6 padded lines and the 9 rows fit in 64 KB (XWIDE), omega keeps
  // its own 3 padded lines instead (faster at N = 512 FP32).
  static constexpr int XLS = padded_len(N);
  static constexpr bool XWIDE = (size_t)((6 * XLS + 1) / 2 * 2 + 9 * N) * CB <= 64 * 1024;
  static constexpr int XST = ((XWIDE ? 6 : 3) * XLS + 1) / 2 * 2;  // 16-byte aligned start of the state rows
  static constexpr bool XPRE = (size_t)(XST + 9 * N) * CB <= 100 * 1024;
  static constexpr size_t XSMEM = (size_t)6 * XLS * CB;
  static constexpr size_t XSMEM_ST = XPRE ? (size_t)(XST + 9 * N) * CB : XSMEM;  // XM_STAGE, XM_RHS
  // z-pass: ZTX adjacent x at fixed y, 6 fields of M values each, <= 112 KB
  // (two blocks per SM); rows narrower than one 32-byte sector may use up to 200 KB.
  static constexpr size_t zbytes(int t) { return (size_t)padded_len(M) * odd_ld(6 * t) * CB; }
  static constexpr int ztx() {
    int t = cmin(16, pow2_part(N));
    while (t > 1 && zbytes(t) > 112 * 1024 && !(t * CB <= 32 && zbytes(t) <= 200 * 1024)) t /= 2;
    return t;
  }
  static constexpr int ZTX = ztx();
  // Minimum resident blocks per SM for the register cap: lines longer than 4 KB
  // hold 32+ registers of data per lane in the warp FFT, so allow more registers.
  static constexpr int LINE_BYTES = N * CB;
  static constexpr int XMIN = LINE_BYTES > 4096 ? 2 : 4;
  static constexpr int ZMIN = (M * CB > 4096) ? 1 : 2;
  static constexpr int ZLD = odd_ld(6 * ZTX);
  static constexpr size_t ZSMEM = zbytes(ZTX);
};

// Tile of the y-pass by direction. The inverse pass (6 full fields) takes 128-byte
// rows in FP32 up to N = 512 with 8 warps looping over its 16 columns (3 blocks per
// SM); the forward pass (3 fields, pruned) takes 64-byte rows, one warp per column, 4
// blocks per SM (both measured at 512^3). FP64 keeps 128-byte rows up to N = 512,
// 64-byte rows above.
// TXO > 0 replaces the tile width (a tuned schedule of the small grids).
// NY: the line length (points along y) where it differs from N (the x extent).
template <typename T, int N, int INV, int TXO = 0, int NY = N>
struct YCfg {
  static constexpr int CB = (int)sizeof(cx<T>);
  static constexpr int TX = TXO > 0 ? TXO : cmin(((INV || CB == 16) && NY <= 512 ? 128 : 64) / CB, pow2_part(N));
  static constexpr int THREADS = cmin(32 * TX, 256);
  static constexpr int LD = odd_ld(TX);
  static constexpr size_t SMEM = (size_t)padded_len(NY) * LD * CB;
  static constexpr int MINB = (CB == 8 && NY <= 512) ? (INV ? 3 : 4) : 2;
};

__device__ __forceinline__ int kfreq(int i, int N) { return i < N / 2 ? i : i - N; }

// the launch parameters with their FP32 copies filled in
inline PassArgs f32args(PassArgs a) {
  a.f_nu = (float)a.nu;
  a.f_cA = (float)a.cA;
  a.f_cB = (float)a.cB;
  a.f_cC = (float)a.cC;
  for (int i = 0; i < 3; ++i) a.f_ks[i] = (float)a.ks[i];
  return a;
}
// a launch parameter in the kernel's precision: the FP32 copy or the FP64 value
template <typename T>
__device__ __forceinline__ T par(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}
__device__ __forceinline__ bool kept(int k, int kmax3) { return 3 * (k < 0 ? -k : k) < kmax3; }
// The support of the stage's state (PassArgs::prune): rows_vanish, it vanishes on every
// row (kz, ky) outside the 2/3 box; box_vanish, at every mode outside the box.
__device__ __forceinline__ bool rows_vanish(const PassArgs& a) { return a.prune >= PRUNE_ROWS; }
__device__ __forceinline__ bool box_vanish(const PassArgs& a) { return a.prune == PRUNE_BOX; }

// XM_STAGE2N: the stage update of Williamson's 2N low-storage form (a mode of its
// own, so that the two-register stage update compiles without its branch)
enum XMode { XM_INV_CURL = 0, XM_STAGE = 1, XM_RHS = 2, XM_FWD_STORE = 3, XM_INV_PLAIN = 4, XM_INV_DIV = 5, XM_STAGE2N = 6 };
enum ZMode { ZM_CROSS = 0, ZM_STORE = 1, ZM_LOAD = 2, ZM_MAXABS = 3 };

// Writes conj(u/N^3) and conj(i k x u / N^3) of one mode into the 6 line
// buffers (stride LS) at padded position pos (conjugated because the following
// x transform is an inverse one).
template <typename T>
__device__ __forceinline__ void put_curl_lines(cx<T>* s, int pos, int LS, cx<T> u0, cx<T> u1, cx<T> u2, T kx, T ky,
                                               T kz, T sc) {
  u0 = scal(u0, sc);
  u1 = scal(u1, sc);
  u2 = scal(u2, sc);
  // omega_hat = i k x u_hat
  const cx<T> w0 = mul_pi(mk(ky * u2.x - kz * u1.x, ky * u2.y - kz * u1.y));
  const cx<T> w1 = mul_pi(mk(kz * u0.x - kx * u2.x, kz * u0.y - kx * u2.y));
  const cx<T> w2 = mul_pi(mk(kx * u1.x - ky * u0.x, kx * u1.y - ky * u0.y));
  cx<T>* p = s + pos;
  p[0 * LS] = conjg(u0);
  p[1 * LS] = conjg(u1);
  p[2 * LS] = conjg(u2);
  p[3 * LS] = conjg(w0);
  p[4 * LS] = conjg(w1);
  p[5 * LS] = conjg(w2);
}

// Global store of one complex value of the RK state.
template <typename T>
__device__ __forceinline__ void st_state(cx<T>* p, cx<T> v) {
  *p = v;
}

// Global store of a forward-transformed state row with the Nyquist modes zeroed.
template <typename T>
struct GStoreNyquistFree {
  cx<T>* g;
  int N;
  bool zero_row;
  __device__ __forceinline__ cx<T>* at(int p) const { return g + p; }
  static constexpr int off(int d) { return d; }
  __device__ __forceinline__ void store(cx<T>* q, int p, cx<T> v) const {
    *q = (zero_row || p == N / 2) ? mk((T)0, (T)0) : v;
  }
};

// R of the rows |ky| <= R kept by the 2/3 rule 3|ky| < k3y on a line of NY points (R < NY/2)
template <int NY>
__host__ __device__ constexpr int xpass_kept_ky(int k3y) {
  return (k3y - 1) / 3 < NY / 2 - 1 ? (k3y - 1) / 3 : NY / 2 - 1;
}
// x-stage launches of a pruned state cover only the rows inside the box (compact grid) up to
// rows of 512 points; the 1024-point rows keep the full grid with early returns (measured on
// GB300: 0.861 -> 0.848 ms per launch at 512^3 and a 3 % shorter ensemble step, but 8.46 ->
// 8.81 ms at 1024^3)
template <int N>
constexpr bool xpass_compact_ok() { return N <= 512; }

// ---------------------------------------------------------------------------
// x-pass: one block owns one row (kz, ky) of length N; warp f transforms line f.
// ---------------------------------------------------------------------------
// NY, NZ: points along y and z where they differ from N (rows kz * NY + ky).
// V: radix plan variant of the line transforms (SmemPlanV).
// compact: the grid covers only the rows inside the 2/3 box (xpass_rows_kept blocks, block bx
// taking row kz = bx / (2R + 1), |ky| <= R), the launch of a state that vanishes outside it.
template <typename T, int N, int MODE, int NY = N, int NZ = N, int V = 0>
__device__ __forceinline__ void xpass_body(const PassArgs a, const int bx, const bool compact = false) {
  constexpr int NT = XP_THREADS;  // one warp per line of u and omega
  constexpr bool STAGE = MODE == XM_STAGE || MODE == XM_STAGE2N;  // a stage update (either form)
  using G = Geometry<T, N, NY, NZ>;
  constexpr int LS = G::XLS;
  constexpr size_t FS = G::FS;
  constexpr int TW = G::TW;
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
  cx<T>* U = reinterpret_cast<cx<T>*>(a.U);
  cx<T>* U1 = reinterpret_cast<cx<T>*>(a.U1);
  cx<T>* US = reinterpret_cast<cx<T>*>(a.US);
  cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // rows outside the 2/3 box carry no nonlinear term (each direction's cut-off from its
  // own point count); where the state vanishes on them, the stage leaves them zero and
  // neither the update nor the x inverse has anything to do there
  const int k3y = NY == N ? a.kmax3 : a.kmax3y, k3z = NZ == N ? a.kmax3 : a.kmax3z;
  int row = bx;  // row = kz * NY + ky
  if (compact) {
    const int R = xpass_kept_ky<NY>(k3y), w = 2 * R + 1, t = bx % w;
    row = (bx / w) * NY + (t <= R ? t : NY - w + t);
  }
  const int kz = row / NY, ky = row % NY;
  const size_t rb = (size_t)row * N;
  const T sc = (T)(1.0 / ((double)N * (double)NY * (double)NZ));
  // wavenumbers of the row and of column j: integer index times 2 pi / L (1 on the 2 pi box)
  const T ksx = par<T>(a.ks[0], a.f_ks[0]);
  const T kzv = (T)kz * par<T>(a.ks[2], a.f_ks[2]), kyv = (T)kfreq(ky, NY) * par<T>(a.ks[1], a.f_ks[1]);
  const bool row_kept = (3 * kz < k3z) && kept(kfreq(ky, NY), k3y);
  if constexpr (STAGE || MODE == XM_INV_CURL) {
    if (!row_kept && rows_vanish(a)) return;
  }

  if constexpr (STAGE || MODE == XM_RHS) {
    // rows outside the box: skip their forward transform
    const T nu = par<T>(a.nu, a.f_nu), cA = par<T>(a.cA, a.f_cA), cB = par<T>(a.cB, a.f_cB);
    const int stage = a.stage, last = a.last;
    // Williamson 2N stages keep the stage state in U (updated in place) and dU in U1
    constexpr bool lsrk = MODE == XM_STAGE2N;
    const cx<T>* Sst = (stage == 0 || lsrk) ? U : US;
    // state rows read by the update: stage state (all stages), accumulator
    // (stages after the first), step-start state (the stages between first and
    // last of the two-register form)
    const bool need1 = STAGE && stage > 0, need0 = STAGE && stage > 0 && stage < last && !lsrk;
    cx<T>* const st = s + G::XST;  // XPRE: rows [Sst 0..2][U1 0..2][U 0..2], N values each
    // a state that vanishes at every mode outside the box (box_vanish) keeps vanishing at
    // the columns |kx| >= N/3 of this row too: its rows are read and written at the kept
    // columns only, the others give u = omega = 0
    const bool xbox = STAGE && box_vanish(a);
    if constexpr (G::XPRE) {
      if (row_kept) {
        for (int e = threadIdx.x; e < 3 * N; e += NT) {
          const int f = e / N, j = e % N;
          cp_async<sizeof(cx<T>)>(s + f * LS + padp(j), W + f * FS + rb + j);
        }
      }
      cp_async_commit();
      constexpr int PK = 16 / (int)sizeof(cx<T>);  // complex values per 16-byte copy
      auto fetch_rows = [&](const cx<T>* src, cx<T>* dst) {
        for (int e = threadIdx.x; e < 3 * N / PK; e += NT) {
          const int f = (e * PK) / N, j = (e * PK) % N;
          // the columns outside the box are one contiguous range: a copy none of whose
          // columns is kept has both ends outside
          if (xbox && !kept(kfreq(j, N), a.kmax3) && !kept(kfreq(j + PK - 1, N), a.kmax3)) continue;
          cp_async<16>(dst + f * N + j, src + f * FS + rb + j);
        }
      };
      fetch_rows(Sst, st);
      if (need1) fetch_rows(U1, st + 3 * N);
      if (need0) fetch_rows(U, st + 6 * N);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      if (row_kept && warp < 3) {
        const SLine<T, 1> line{s + warp * LS};
        warp_fft<T, N, TW, V>(line, line, line, tw, lane);
      }
      cp_async_wait<0>();
    } else {
      if (row_kept && warp < 3) {
        const SLine<T, 1> line{s + warp * LS};
        warp_fft<T, N, TW, V>(GLoad<T, false>{W + warp * FS + rb}, line, line, tw, lane);
      }
    }
    __syncthreads();
    // state values of component c at column j: staged rows or global memory
    auto ld_s = [&](int c, int j) -> cx<T> { return G::XPRE ? st[c * N + j] : Sst[c * FS + rb + j]; };
    auto ld_1 = [&](int c, int j) -> cx<T> { return G::XPRE ? st[(3 + c) * N + j] : U1[c * FS + rb + j]; };
    auto ld_0 = [&](int c, int j) -> cx<T> { return G::XPRE ? st[(6 + c) * N + j] : U[c * FS + rb + j]; };
    // the column loop, with the wavenumber kx = index * 2 pi / Lx; on the 2 pi box the
    // index itself, exactly as without a box option
    auto columns = [&](auto scaled) {
      constexpr bool SCALED = decltype(scaled)::value;
      for (int j = threadIdx.x; j < N; j += NT) {
        const int kxi = kfreq(j, N);
        const T kx = SCALED ? (T)kxi * ksx : (T)kxi;
        const int pj = padp(j);
        cx<T> n0 = mk((T)0, (T)0), n1 = n0, n2 = n0;
        if (row_kept && kept(kxi, a.kmax3)) {
          n0 = s[0 * LS + pj];
          n1 = s[1 * LS + pj];
          n2 = s[2 * LS + pj];
          if (a.F) {  // external force (learned closure), masked like the nonlinear term
            const cx<T>* F = reinterpret_cast<const cx<T>*>(a.F);
            n0 = n0 + F[rb + j];
            n1 = n1 + F[FS + rb + j];
            n2 = n2 + F[2 * FS + rb + j];
          }
        }
        const T k2 = kx * kx + kyv * kyv + kzv * kzv;
        const T ik2 = k2 > (T)0 ? (T)1 / k2 : (T)0;
        // P = (k . N_hat) / |k|^2   (Eq. mod_pressure without the factor i)
        const cx<T> p = mk((kx * n0.x + kyv * n1.x + kzv * n2.x) * ik2, (kx * n0.y + kyv * n1.y + kzv * n2.y) * ik2);
        const size_t gi = rb + j;
        const bool xin = !xbox || kept(kxi, a.kmax3);
        const cx<T> zero = mk((T)0, (T)0);
        const cx<T> u0 = xin ? ld_s(0, j) : zero, u1 = xin ? ld_s(1, j) : zero, u2 = xin ? ld_s(2, j) : zero;
        const T nk2 = nu * k2;
        // dU = N_hat - k P - nu |k|^2 u_hat   (Eq. NSfinal)
        const cx<T> d0 = mk(n0.x - kx * p.x - nk2 * u0.x, n0.y - kx * p.y - nk2 * u0.y);
        const cx<T> d1 = mk(n1.x - kyv * p.x - nk2 * u1.x, n1.y - kyv * p.y - nk2 * u1.y);
        const cx<T> d2 = mk(n2.x - kzv * p.x - nk2 * u2.x, n2.y - kzv * p.y - nk2 * u2.y);
        if constexpr (MODE == XM_RHS) {
          cx<T>* out = reinterpret_cast<cx<T>*>(a.out);
          out[gi] = d0;
          out[FS + gi] = d1;
          out[2 * FS + gi] = d2;
        } else {
          cx<T> v0 = zero, v1 = zero, v2 = zero;
          if (!xin) {
            // outside the box: the state stays zero there and is not written
          } else if constexpr (lsrk) {  // 2N stage: dU <- A_s dU + dt RHS, u <- u + B_s dU
            const T cC = par<T>(a.cC, a.f_cC);
            cx<T> e0 = scal(d0, cC), e1 = scal(d1, cC), e2 = scal(d2, cC);
            if (stage > 0) {
              e0 = e0 + scal(ld_1(0, j), cA);
              e1 = e1 + scal(ld_1(1, j), cA);
              e2 = e2 + scal(ld_1(2, j), cA);
            }
            if (stage < last) {
              st_state(U1 + gi, e0);
              st_state(U1 + FS + gi, e1);
              st_state(U1 + 2 * FS + gi, e2);
            }
            v0 = u0 + scal(e0, cB);
            v1 = u1 + scal(e1, cB);
            v2 = u2 + scal(e2, cB);
            st_state(U + gi, v0);
            st_state(U + FS + gi, v1);
            st_state(U + 2 * FS + gi, v2);
          } else if (stage == 0 && last == 0) {  // one-stage step (forward Euler): u += a_0 dt dU
            v0 = u0 + scal(d0, cA);
            v1 = u1 + scal(d1, cA);
            v2 = u2 + scal(d2, cA);
            st_state(U + gi, v0);
            st_state(U + FS + gi, v1);
            st_state(U + 2 * FS + gi, v2);
          } else if (stage == 0) {
            st_state(U1 + gi, u0 + scal(d0, cA));
            st_state(U1 + FS + gi, u1 + scal(d1, cA));
            st_state(U1 + 2 * FS + gi, u2 + scal(d2, cA));
            v0 = u0 + scal(d0, cB);
            v1 = u1 + scal(d1, cB);
            v2 = u2 + scal(d2, cB);
            st_state(US + gi, v0);
            st_state(US + FS + gi, v1);
            st_state(US + 2 * FS + gi, v2);
          } else if (stage < last) {
            const cx<T> b0 = ld_0(0, j), b1 = ld_0(1, j), b2 = ld_0(2, j);
            st_state(U1 + gi, ld_1(0, j) + scal(d0, cA));
            st_state(U1 + FS + gi, ld_1(1, j) + scal(d1, cA));
            st_state(U1 + 2 * FS + gi, ld_1(2, j) + scal(d2, cA));
            v0 = b0 + scal(d0, cB);
            v1 = b1 + scal(d1, cB);
            v2 = b2 + scal(d2, cB);
            st_state(US + gi, v0);
            st_state(US + FS + gi, v1);
            st_state(US + 2 * FS + gi, v2);
          } else {
            v0 = ld_1(0, j) + scal(d0, cA);
            v1 = ld_1(1, j) + scal(d1, cA);
            v2 = ld_1(2, j) + scal(d2, cA);
            st_state(U + gi, v0);
            st_state(U + FS + gi, v1);
            st_state(U + 2 * FS + gi, v2);
          }
          if constexpr (G::XPRE && !G::XWIDE) {
            // u into lines 0-2 (padded, where this thread read N_hat), omega into
            // state rows 0-2 (unpadded, where this thread read the stage state)
            const cx<T> s0 = scal(v0, sc), s1 = scal(v1, sc), s2 = scal(v2, sc);
            s[0 * LS + pj] = conjg(s0);
            s[1 * LS + pj] = conjg(s1);
            s[2 * LS + pj] = conjg(s2);
            st[0 * N + j] = conjg(mul_pi(mk(kyv * s2.x - kzv * s1.x, kyv * s2.y - kzv * s1.y)));
            st[1 * N + j] = conjg(mul_pi(mk(kzv * s0.x - kx * s2.x, kzv * s0.y - kx * s2.y)));
            st[2 * N + j] = conjg(mul_pi(mk(kx * s1.x - kyv * s0.x, kx * s1.y - kyv * s0.y)));
          } else {
            put_curl_lines<T>(s, pj, LS, v0, v1, v2, kx, kyv, kzv, sc);
          }
        }
      }
    };
    if (ksx == (T)1)
      columns(std::false_type{});
    else
      columns(std::true_type{});
    if constexpr (STAGE) {
      __syncthreads();
      if constexpr (G::XPRE && !G::XWIDE) {
        if (warp < 3) {
          const SLine<T, 1> line{s + warp * LS};
          warp_fft<T, N, TW, V>(line, line, GStore<T, true>{W + warp * FS + rb}, tw, lane);
        } else {  // omega: from its unpadded row, through a padded work line over rows 3-8
          const int c = warp - 3;
          const SLine<T, 1> work{st + 3 * N + c * LS};
          warp_fft<T, N, TW, V>(SRow<T>{st + c * N}, work, GStore<T, true>{W + warp * FS + rb}, tw, lane);
        }
      } else {
        const SLine<T, 1> line{s + warp * LS};
        warp_fft<T, N, TW, V>(line, line, GStore<T, true>{W + warp * FS + rb}, tw, lane);
      }
    }
  } else if constexpr (MODE == XM_FWD_STORE) {
    if (warp < 3) {
      const SLine<T, 1> line{s + warp * LS};
      warp_fft<T, N, TW, V>(GLoad<T, false>{U + warp * FS + rb}, line,
                        GStoreNyquistFree<T>{U + warp * FS + rb, N, ky == NY / 2}, tw, lane);
    }
  } else {
    // inverse x transform of u and omega (XM_INV_CURL), of u alone
    // (XM_INV_PLAIN) or of i k . u (XM_INV_DIV), all scaled by 1/N^3
    constexpr int NF = (MODE == XM_INV_CURL) ? 6 : (MODE == XM_INV_PLAIN ? 3 : 1);
    const bool xbox = MODE == XM_INV_CURL && box_vanish(a);  // columns |kx| >= N/3 hold zeros
    for (int j = threadIdx.x; j < N; j += NT) {
      const size_t gi = rb + j;
      const int pj = padp(j);
      const bool xin = !xbox || kept(kfreq(j, N), a.kmax3);
      const cx<T> zero = mk((T)0, (T)0);
      const cx<T> u0 = xin ? U[gi] : zero, u1 = xin ? U[FS + gi] : zero, u2 = xin ? U[2 * FS + gi] : zero;
      const T kx = (T)kfreq(j, N) * ksx;
      if constexpr (MODE == XM_INV_CURL) {
        put_curl_lines<T>(s, pj, LS, u0, u1, u2, kx, kyv, kzv, sc);
      } else if constexpr (MODE == XM_INV_PLAIN) {
        s[0 * LS + pj] = conjg(scal(u0, sc));
        s[1 * LS + pj] = conjg(scal(u1, sc));
        s[2 * LS + pj] = conjg(scal(u2, sc));
      } else {
        const cx<T> d = mul_pi(mk(kx * u0.x + kyv * u1.x + kzv * u2.x, kx * u0.y + kyv * u1.y + kzv * u2.y));
        s[pj] = conjg(scal(d, sc));
      }
    }
    __syncthreads();
    cx<T>* dst = (MODE == XM_INV_DIV) ? reinterpret_cast<cx<T>*>(a.D) : W;
    if (warp < NF) {
      const SLine<T, 1> line{s + warp * LS};
      warp_fft<T, N, TW, V>(line, line, GStore<T, true>{dst + warp * FS + rb}, tw, lane);
    }
  }
}

template <typename T, int N, int MODE, int NY = N, int NZ = N, int V = 0>
__global__ void __launch_bounds__(XP_THREADS, (Geometry<T, N, NY, NZ>::XMIN)) k_xpass(PassArgs a) {
  constexpr bool CAN = (MODE == XM_STAGE || MODE == XM_STAGE2N || MODE == XM_INV_CURL) && xpass_compact_ok<N>();
  xpass_body<T, N, MODE, NY, NZ, V>(a, blockIdx.x, CAN && a.prune >= PRUNE_ROWS);
}

// Batched form (ensembles): member blockIdx.y, its arguments in B.a[blockIdx.y].
template <typename T, int N, int MODE, int V = 0>
__global__ void __launch_bounds__(XP_THREADS, (Geometry<T, N>::XMIN)) k_xpass_b(const __grid_constant__ BatchArgs B) {
  xpass_body<T, N, MODE, N, N, V>(B.a[blockIdx.y], blockIdx.x);
}

// ---------------------------------------------------------------------------
// y-pass: one block owns TX adjacent columns (fixed field and kz) of length N;
// the tile is loaded with coalesced rows, each warp transforms whole columns.
// INV: conj-in/conj-out (inverse DFT). PRUNE: store only rows with |ky| < N/3.
// grid = (N / TX, number of kz planes, number of fields); TX etc. from YCfg
// ---------------------------------------------------------------------------
// Row walked by tile element group r of the y-pass. With 8-byte values in
// 8-wide rows (row stride 9 in shared memory) a warp covers 4 rows; rows y and
// y + 1 in one half-warp share banks, rows y and y + 8 do not, so the walk takes
// rows in the order 0, 8, 1, 9, 2, 10, ... within each block of 16 (a
// permutation of 0 .. N-1 only when N is a multiple of 16; otherwise the rows
// are walked in order).
template <typename T, int TX, int N>
__device__ __forceinline__ int ywalk_row(int r) {
  if constexpr (sizeof(cx<T>) == 8 && TX == 8 && N % 16 == 0) {
    const int t = r & 15, u = t >> 2, q = t & 3;
    return (r & ~15) | (2 * u + (q >> 1) + (q & 1) * 8);
  } else {
    return r;
  }
}

// Fill of a y tile (TX columns of L rows, row stride `stride` in global memory) whose rows
// outside the 2/3 box are zeros: the kept rows |ky| <= R (R = (kmax3 - 1) / 3, rows 0 .. R
// and L - R .. L - 1) by cp.async (in the bank-friendly walk order where it permutes the
// rows), the rows R + 1 .. L - R - 1 between them as zeros.
template <typename T, int L, int TX, int LD, int NT>
__device__ __noinline__ void ytile_fill_kept(cx<T>* s, const cx<T>* __restrict__ base, int stride, int kmax3) {
  int R = (kmax3 - 1) / 3;
  if (R > L / 2 - 1) R = L / 2 - 1;
  const int lo = R + 1, gap = L - 2 * R - 1;  // kept rows [0, lo) and [lo + gap, L)
  if constexpr (sizeof(cx<T>) == 8 && TX == 8 && L % 16 == 0) {
#pragma unroll 8
    for (int e = threadIdx.x; e < TX * L; e += NT) {
      const int x = e % TX, y = ywalk_row<T, TX, L>(e / TX);
      if (y < lo || y >= lo + gap) cp_async<sizeof(cx<T>)>(s + padp(y) * LD + x, base + (size_t)y * stride + x);
    }
  } else {
#pragma unroll 8
    for (int e = threadIdx.x; e < TX * (L - gap); e += NT) {
      const int x = e % TX, r = e / TX, y = r < lo ? r : r + gap;
      cp_async<sizeof(cx<T>)>(s + padp(y) * LD + x, base + (size_t)y * stride + x);
    }
  }
#pragma unroll 4
  for (int e = threadIdx.x; e < TX * gap; e += NT) {
    const int x = e % TX, y = lo + e / TX;
    s[padp(y) * LD + x] = mk((T)0, (T)0);
  }
}

// One y tile: TX adjacent columns starting at `base` (field, kz plane and first
// column already applied), transformed along y in place. NT: threads of the block.
// vanish (inverse only): the rows with |ky| >= N/3 are zeros, not read.
template <typename T, int N, int INV, int PRUNE, int TXO, int NT, int V = 0>
__device__ __forceinline__ void ypass_tile(cx<T>* __restrict__ base, const cx<T>* __restrict__ tw, int kmax3,
                                           bool vanish = false) {
  using Y = YCfg<T, N, INV, TXO>;
  constexpr int TX = Y::TX;
  constexpr int LD = Y::LD;
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the whole tile in flight at once (cp.async, no register staging); the
  // inverse's conjugation is applied when the first pass reads it
  if (INV && vanish) {
    ytile_fill_kept<T, N, TX, LD, NT>(s, base, N, kmax3);
  } else {
#pragma unroll 8
    for (int e = threadIdx.x; e < TX * N; e += NT) {
      const int x = e % TX, y = ywalk_row<T, TX, N>(e / TX);
      cp_async<sizeof(cx<T>)>(s + padp(y) * LD + x, base + (size_t)y * N + x);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll 1
  for (int c = warp; c < TX; c += NT / 32) {  // warps loop over the columns
    const SLine<T, LD> line{s + c};
    if constexpr (INV) warp_fft<T, N, N, V>(SLineConj<T, LD>{s + c}, line, line, tw, lane);
    else warp_fft<T, N, N, V>(line, line, line, tw, lane);
  }
  __syncthreads();
#pragma unroll 8
  for (int e = threadIdx.x; e < TX * N; e += NT) {
    const int x = e % TX, y = ywalk_row<T, TX, N>(e / TX);
    if (PRUNE && !kept(kfreq(y, N), kmax3)) continue;
    const cx<T> v = s[padp(y) * LD + x];
    base[(size_t)y * N + x] = INV ? conjg(v) : v;
  }
}

// NY, NZ: points along y and z where they differ from N (N: the x extent, the
// row stride of the tile's columns).
// PR (inverse of a stage whose state vanishes outside the 2/3 box): the grid covers the
// planes kz < kc only (the others hold zeros that the z-pass does not read) and the rows
// with |ky| >= NY/3 (kmax3) are read as zeros.
template <typename T, int N, int INV, int PRUNE, int TXO = 0, int NY = N, int NZ = N, int V = 0, int PR = 0>
__global__ void __launch_bounds__(YCfg<T, N, INV, TXO, NY>::THREADS, (YCfg<T, N, INV, TXO, NY>::MINB))
    k_ypass(cx<T>* __restrict__ F, const cx<T>* __restrict__ tw, int kmax3) {
  using G = Geometry<T, N, NY, NZ>;
  using Y = YCfg<T, N, INV, TXO, NY>;
  constexpr int TX = Y::TX;
  constexpr int LD = Y::LD;
  constexpr int NT = Y::THREADS;  // warps loop over the columns
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cx<T>* base = F + blockIdx.z * G::FS + (size_t)blockIdx.y * NY * N + blockIdx.x * TX;
  // the whole tile in flight at once (cp.async, no register staging); the
  // inverse's conjugation is applied when the first pass reads it
  if constexpr (INV && PR) {
    ytile_fill_kept<T, NY, TX, LD, NT>(s, base, N, kmax3);
  } else {
#pragma unroll 8
    for (int e = threadIdx.x; e < TX * NY; e += NT) {
      const int x = e % TX, y = ywalk_row<T, TX, NY>(e / TX);
      cp_async<sizeof(cx<T>)>(s + padp(y) * LD + x, base + (size_t)y * N + x);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll 1
  for (int c = warp; c < TX; c += NT / 32) {
    const SLine<T, LD> line{s + c};
    if constexpr (INV) warp_fft<T, NY, G::TW, V>(SLineConj<T, LD>{s + c}, line, line, tw, lane);
    else warp_fft<T, NY, G::TW, V>(line, line, line, tw, lane);
  }
  __syncthreads();
#pragma unroll 8
  for (int e = threadIdx.x; e < TX * NY; e += NT) {
    const int x = e % TX, y = ywalk_row<T, TX, NY>(e / TX);
    if (PRUNE && !kept(kfreq(y, NY), kmax3)) continue;
    const cx<T> v = s[padp(y) * LD + x];
    base[(size_t)y * N + x] = INV ? conjg(v) : v;
  }
}

// Batched form on the members' work arrays (ensembles): blockIdx.z = member *
// fields + field; otherwise the same steps as k_ypass (TXO: a tuned tile width).
template <typename T, int N, int INV, int PRUNE, int TXO = 0, int V = 0>
__global__ void __launch_bounds__(YCfg<T, N, INV, TXO>::THREADS, (YCfg<T, N, INV, TXO>::MINB))
    k_ypass_b(const __grid_constant__ BatchArgs B, int fields) {
  using G = Geometry<T, N>;
  using Y = YCfg<T, N, INV, TXO>;
  const PassArgs& a = B.a[blockIdx.z / fields];
  const bool vanish = INV && rows_vanish(a);  // the member's planes kz >= kc are not transformed
  if (vanish && 3 * (int)blockIdx.y >= a.kmax3) return;
  cx<T>* base = reinterpret_cast<cx<T>*>(a.W) + (blockIdx.z % fields) * G::FS + (size_t)blockIdx.y * N * N +
                blockIdx.x * Y::TX;
  ypass_tile<T, N, INV, PRUNE, TXO, Y::THREADS, V>(base, reinterpret_cast<const cx<T>*>(a.tw), a.kmax3, vanish);
}

// ---------------------------------------------------------------------------
// z-pass: one block owns ZTX adjacent x at fixed y; lines run along kz / z.
// Real transforms of length N use one complex DFT of length M = N/2 on
// z_n = x_{2n} + i x_{2n+1} with the usual pre/post-processing of the pairs
// (k, M-k); the imaginary part of the kz = 0 coefficient is ignored and the
// kz = N/2 coefficient is zero (it is not stored).
// ---------------------------------------------------------------------------
// NY, NZ: points along y and z where they differ from N (lines of NZ points at the
// NX x NY positions; physical arrays (3, N, NY, NZ)).
template <typename T, int N, int MODE, int TXO = 0, int NY = N, int NZ = N, int V = 0>
__device__ __forceinline__ void zpass_body(const PassArgs a, const int bx, const int by) {
  using G = Geometry<T, N, NY, NZ>;
  constexpr int M = G::M;
  constexpr int TW = G::TW, TS = TW / NZ;  // exp(-2 pi i k / NZ) = tw[k * TS]
  constexpr int TX = TXO > 0 ? TXO : G::ZTX;  // TXO: a tuned tile width of the small grids
  constexpr int LD = odd_ld(6 * TX);
  constexpr size_t FS = G::FS;
  constexpr int NF = (MODE == ZM_CROSS) ? 6 : (MODE == ZM_MAXABS ? 1 : 3);
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x0 = bx * TX;
  const int y = by;

  if constexpr (MODE == ZM_LOAD) {
    // physical lines (x0 + x, y, :) of the 3 components, packed in pairs
    // (the whole tile in flight at once by cp.async, no register staging)
    const cx<T>* in = reinterpret_cast<const cx<T>*>(a.in);
    for (int e = threadIdx.x; e < 3 * TX * M; e += ZP_THREADS) {
      const int n = e % M, x = (e / M) % TX, c = e / (M * TX);
      cp_async<sizeof(cx<T>)>(s + padp(n) * LD + c * TX + x, in + ((size_t)(c * N + x0 + x) * NY + y) * M + n);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
  } else {
    const cx<T>* src = reinterpret_cast<const cx<T>*>(MODE == ZM_MAXABS ? a.D : a.W);
    // a stage whose state vanishes outside the 2/3 box: the planes kz >= kc hold zeros
    // (the y-inverse left them alone) and are filled with zeros instead of read
    int klim = M;
    if constexpr (MODE == ZM_CROSS) {
      if (rows_vanish(a)) {
        klim = ((NZ == N ? a.kmax3 : a.kmax3z) + 2) / 3;
        if (klim > M) klim = M;
      }
    }
    if (klim < M) {  // the walk of the full fill (compile-time divisors), planes past klim as zeros
      for (int e = threadIdx.x; e < NF * TX * M; e += ZP_THREADS) {
        const int x = e % TX, k = (e / TX) % M, f = e / (TX * M);
        if (k < klim)
          cp_async<sizeof(cx<T>)>(s + padp(k) * LD + f * TX + x, src + f * FS + ((size_t)k * NY + y) * N + x0 + x);
        else
          s[padp(k) * LD + f * TX + x] = mk((T)0, (T)0);
      }
    } else {
      for (int e = threadIdx.x; e < NF * TX * M; e += ZP_THREADS) {
        const int x = e % TX, k = (e / TX) % M, f = e / (TX * M);
        cp_async<sizeof(cx<T>)>(s + padp(k) * LD + f * TX + x, src + f * FS + ((size_t)k * NY + y) * N + x0 + x);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // c2r pre-processing: Z'_k = (X_k + conj X_{M-k}) + i e^{+2 pi i k/N} (X_k - conj X_{M-k}),
    // stored conjugated so that a forward DFT gives the inverse one.
    constexpr int NL = NF * TX;
    for (int e = threadIdx.x; e < NL * (M / 2 + 1); e += ZP_THREADS) {
      const int l = e % NL, k = e / NL;
      if (k == 0) {
        const T r0 = s[l].x;  // Im X_0 ignored, X_M = 0
        s[l] = mk(r0, -r0);
      } else {
        cx<T>* pk = s + padp(k) * LD + l;
        cx<T>* pm = s + padp(M - k) * LD + l;
        const cx<T> xk = *pk, xm = *pm;
        const cx<T> wk = ldro(tw + k * TS);  // exp(-2 pi i k / NZ)
        const cx<T> A = xk + conjg(xm), B = xk - conjg(xm);
        *pk = conjg(A + mul_pi(cmul(conjg(wk), B)));
        if (k != M - k) {
          // partner M-k: e^{+2 pi i (M-k)/N} = -wk
          const cx<T> A2 = xm + conjg(xk), B2 = xm - conjg(xk);
          *pm = conjg(A2 - mul_pi(cmul(wk, B2)));
        }
      }
    }
    __syncthreads();
    constexpr int GL = LinesPerWarp<M, V>::value <= TX ? LinesPerWarp<M, V>::value : TX;  // lines per warp
#pragma unroll 1
    for (int l = warp * GL; l < NL; l += (ZP_THREADS / 32) * GL) warp_fft_lines<T, M, TW, GL, LD, V>(s + l, tw, lane);
    __syncthreads();
    // now conj(s) = x_{2n} + i x_{2n+1} (physical values, unnormalised c2r)
  }

  if constexpr (MODE == ZM_CROSS) {
    for (int e = threadIdx.x; e < TX * M; e += ZP_THREADS) {
      const int x = e % TX, n = e / TX;
      cx<T>* p = s + padp(n) * LD + x;
      const cx<T> u0 = conjg(p[0 * TX]), u1 = conjg(p[1 * TX]), u2 = conjg(p[2 * TX]);
      const cx<T> w0 = conjg(p[3 * TX]), w1 = conjg(p[4 * TX]), w2 = conjg(p[5 * TX]);
      // u x omega on both packed points (real and imaginary parts)
      p[0 * TX] = mk(u1.x * w2.x - u2.x * w1.x, u1.y * w2.y - u2.y * w1.y);
      p[1 * TX] = mk(u2.x * w0.x - u0.x * w2.x, u2.y * w0.y - u0.y * w2.y);
      p[2 * TX] = mk(u0.x * w1.x - u1.x * w0.x, u0.y * w1.y - u1.y * w0.y);
    }
    __syncthreads();
  }

  if constexpr (MODE == ZM_CROSS || MODE == ZM_LOAD) {
    constexpr int GL = LinesPerWarp<M, V>::value <= TX ? LinesPerWarp<M, V>::value : TX;
#pragma unroll 1
    for (int l = warp * GL; l < 3 * TX; l += (ZP_THREADS / 32) * GL) warp_fft_lines<T, M, TW, GL, LD, V>(s + l, tw, lane);
    __syncthreads();
    // r2c post-processing: X_k = 1/2 [(Z_k + conj Z_{M-k}) - i e^{-2 pi i k/N} (Z_k - conj Z_{M-k})]
    cx<T>* dst = reinterpret_cast<cx<T>*>(MODE == ZM_CROSS ? a.W : a.U);
    int kc = M;
    if (MODE == ZM_CROSS) {
      kc = ((NZ == N ? a.kmax3 : a.kmax3z) + 2) / 3;
      if (kc > M) kc = M;
    }
    // the walk over (product, k < kc, x) with kc a compile-time constant where it is the
    // default rule's (or M), so that its divisions are multiplications
    auto post = [&](auto kcc) {
      constexpr int KC = decltype(kcc)::value;  // 0: kc known at run time only
      const int kk = KC > 0 ? KC : kc;
      for (int e = threadIdx.x; e < 3 * TX * kk; e += ZP_THREADS) {
        const int x = e % TX, k = (e / TX) % kk, c = e / (TX * kk);
        const int l = c * TX + x;
        const cx<T> zk = s[padp(k) * LD + l], zm = s[padp((M - k) % M) * LD + l];
        const cx<T> wk = ldro(tw + k * TS);
        const cx<T> A = zk + conjg(zm), B = zk - conjg(zm);
        dst[c * FS + ((size_t)k * NY + y) * N + x0 + x] = scal(A + mul_mi(cmul(wk, B)), (T)0.5);
      }
    };
    constexpr int KC0 = (NZ + 2) / 3 < M ? (NZ + 2) / 3 : M;  // kc of the rule 3|k| < NZ
    if (kc == M)
      post(std::integral_constant<int, M>{});
    else if (kc == KC0)
      post(std::integral_constant<int, KC0>{});
    else
      post(std::integral_constant<int, 0>{});
  } else if constexpr (MODE == ZM_STORE) {
    cx<T>* out = reinterpret_cast<cx<T>*>(a.out);
    for (int e = threadIdx.x; e < 3 * TX * M; e += ZP_THREADS) {
      const int n = e % M, x = (e / M) % TX, c = e / (M * TX);
      out[((size_t)(c * N + x0 + x) * NY + y) * M + n] = conjg(s[padp(n) * LD + c * TX + x]);
    }
  } else if constexpr (MODE == ZM_MAXABS) {
    double m = 0.0;
    for (int e = threadIdx.x; e < TX * M; e += ZP_THREADS) {
      const int x = e % TX, n = e / TX;
      const cx<T> v = s[padp(n) * LD + x];
      m = fmax(m, fmax(fabs((double)v.x), fabs((double)v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double red[ZP_THREADS / 32];
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < ZP_THREADS / 32; ++w) m = fmax(m, red[w]);
      // non-negative doubles order like their bit patterns
      atomicMax(a.maxbits, (unsigned long long)__double_as_longlong(m));
    }
  }
}

template <typename T, int N, int MODE, int TXO = 0, int NY = N, int NZ = N, int V = 0>
__global__ void __launch_bounds__(ZP_THREADS, (Geometry<T, N, NY, NZ>::ZMIN)) k_zpass(PassArgs a) {
  zpass_body<T, N, MODE, TXO, NY, NZ, V>(a, blockIdx.x, blockIdx.y);
}

// Batched form (ensembles): member blockIdx.z (TXO: a tuned tile width).
template <typename T, int N, int MODE, int TXO = 0, int V = 0>
__global__ void __launch_bounds__(ZP_THREADS, (Geometry<T, N>::ZMIN)) k_zpass_b(const __grid_constant__ BatchArgs B) {
  zpass_body<T, N, MODE, TXO, N, N, V>(B.a[blockIdx.z], blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// z-pass of the right-hand side with register-resident columns (M = N/2 a
// multiple of 32, M >= 128): a block owns ZTX adjacent x at fixed y and has one
// warp per x. After a coalesced load of the 6 fields, each warp on its own
// column: c2r of u (pre-processing fused into the first pass; physical values
// parked in the column's own lines), c2r of omega one component at a time
// with the cross product accumulated incrementally, r2c of each finished
// component with the post-processing done through lane shuffles. Only the load
// and the store need block barriers.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ cx<T> pmul(cx<T> a, cx<T> b) { return mk(a.x * b.x, a.y * b.y); }

template <typename T, int N>
struct ZCross {
  static constexpr int M = N / 2;
  static constexpr int V = M / 32;
  static constexpr bool enabled = (M % 32 == 0) && (M >= 128) && CanonPlan<M>::valid();
};

// Twiddles the z-cross warps reuse for every line: the canonical-FFT bases
// and exp(-2 pi i lane / N); exp(-2 pi i k / N) for k = lane + 32 m is then
// tl * tw[32 m] (a broadcast load).
template <typename T, int N>
struct ZTw {
  CanonTw<T, N / 2, N> fft;
  cx<T> tl;
  __device__ __forceinline__ void load(const cx<T>* __restrict__ tw, int lane) {
    fft.load(tw, lane);
    tl = ldro(tw + lane);
  }
  __device__ __forceinline__ cx<T> wk(const cx<T>* __restrict__ tw, int m) const {
    if constexpr (sizeof(T) == 4) return m == 0 ? tl : cmul(tl, ldro(tw + 32 * m));
    else return ldro(tw + (threadIdx.x & 31) + 32 * m);
  }
};

// c2r of one column line (element k at ln[padp(k) * LD]) into canonical
// physical pairs v[m] = x_{2n} + i x_{2n+1}, n = lane + 32 m. The pre-processing
// Z'_k = (X_k + conj X_{M-k}) + i e^{+2 pi i k/N} (X_k - conj X_{M-k}) is fused
// into the load (stored conjugated: a forward DFT then gives the inverse one).
template <typename T, int N, int LD = Geometry<T, N>::ZLD>
__device__ __forceinline__ void zc_c2r(cx<T> (&v)[N / 64], cx<T>* ln, const ZTw<T, N>& zt,
                                       const cx<T>* __restrict__ tw, int lane) {
  constexpr int M = N / 2, V = M / 32;
  const cx<T>* pa = ln + padp(lane) * LD;            // X_k, k = lane + 32 m
  const cx<T>* pb = ln + padp((32 - lane) & 31) * LD;  // X_{M-k} for lane > 0
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const cx<T> xk = pa[34 * m * LD];
    cx<T> xm;
    if (lane != 0) xm = pb[34 * (V - 1 - m) * LD];
    else xm = (m == 0) ? mk((T)0, (T)0) : ln[34 * (V - m) * LD];
    cx<T> z;
    if (lane == 0 && m == 0) {
      z = mk(xk.x, xk.x);  // Im X_0 ignored, X_M = 0
    } else {
      const cx<T> wk = zt.wk(tw, m);
      const cx<T> A = xk + conjg(xm), B = xk - conjg(xm);
      z = A + mul_pi(cmul(conjg(wk), B));
    }
    v[m] = conjg(z);
  }
  __syncwarp();
  warp_fft_canon<T, M, N, LD>(v, ln, zt.fft, tw, lane);
#pragma unroll
  for (int m = 0; m < V; ++m) v[m] = conjg(v[m]);
}

// r2c of canonical physical pairs c, then X_k for k < kc written into line out:
// X_k = 1/2 [(Z_k + conj Z_{M-k}) - i e^{-2 pi i k/N} (Z_k - conj Z_{M-k})],
// the partner Z_{M-k} coming from lane 32 - lane (lane 0 holds both).
template <typename T, int N, int LD = Geometry<T, N>::ZLD>
__device__ __forceinline__ void zc_r2c(cx<T> (&c)[N / 64], cx<T>* scratch, cx<T>* out, int kc, const ZTw<T, N>& zt,
                                       const cx<T>* __restrict__ tw, int lane) {
  constexpr int M = N / 2, V = M / 32;
  warp_fft_canon<T, M, N, LD>(c, scratch, zt.fft, tw, lane);
  const int partner = (32 - lane) & 31;
  cx<T>* po = out + padp(lane) * LD;
#pragma unroll
  for (int m = 0; m < V; ++m) {
    cx<T> zo;
    zo.x = __shfl_sync(0xffffffffu, c[V - 1 - m].x, partner);
    zo.y = __shfl_sync(0xffffffffu, c[V - 1 - m].y, partner);
    if (lane == 0) zo = c[(V - m) % V];
    const cx<T> wk = zt.wk(tw, m);
    const cx<T> A = c[m] + conjg(zo), B = c[m] - conjg(zo);
    if (lane + 32 * m < kc) po[34 * m * LD] = scal(A + mul_mi(cmul(wk, B)), (T)0.5);
  }
}

// Warps per z-cross block: 6 ZTX c2r lines and 3 ZTX r2c lines split evenly
// (4 and 2 per warp).
template <typename T, int N>
struct ZCrossWarps {  // at most 12, so that two blocks share an SM and overlap load and transform
  static constexpr int full = (3 * Geometry<T, N>::ZTX) / 2 >= 1 ? (3 * Geometry<T, N>::ZTX) / 2 : 1;
  static constexpr int value = full > 12 ? 12 : full;
};

// Tile element walk for the z-cross block (load, cross product, store): one
// warp instruction covers kz = 16 g + (ZTX/2) kq + c for kq = lane / ZTX and
// x = lane % ZTX, which touches every shared-memory bank pair exactly twice
// with the odd row stride ZLD, while each global access reads whole 32-byte
// sectors of ZTX contiguous x.
template <typename T, int N>
struct ZWalk {
  static constexpr int TX = Geometry<T, N>::ZTX;
  static constexpr int S = TX / 2 > 0 ? TX / 2 : 1;  // values of c
  static constexpr int G16 = (N / 2) / 16;           // values of g
  static constexpr int ITEMS = G16 * S;              // per field
};

template <typename T, int N>
__global__ void __launch_bounds__(32 * ZCrossWarps<T, N>::value, (ZCrossWarps<T, N>::value > 16 ? 1 : 2)) k_zcross(PassArgs a) {
  using G = Geometry<T, N>;
  using ZW = ZWalk<T, N>;
  constexpr int M = G::M, TX = G::ZTX, LD = G::ZLD, V = M / 32;
  constexpr int NW = ZCrossWarps<T, N>::value;
  constexpr size_t FS = G::FS;
  static_assert(32 % TX == 0 && (M % 16) == 0, "z-cross tile walk");
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
  cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x0 = blockIdx.x * TX, y = blockIdx.y;
  int kc = (a.kmax3 + 2) / 3;
  if (kc > M) kc = M;
  const int tx = lane % TX, kq = lane / TX;
  // lane part of the walk: k = 16 g + S kq + c  ->  padp(k) = 17 g + S kq + c
  const cx<T>* gl = W + ((size_t)(ZW::S * kq) * N + y) * N + x0 + tx;
  cx<T>* sl = s + (ZW::S * kq) * LD + tx;

  if (rows_vanish(a)) {  // planes kz >= kc of a state that vanishes outside the 2/3 box: zeros
    for (int it = w; it < 6 * ZW::ITEMS; it += NW) {
      const int f = it / ZW::ITEMS, r = it % ZW::ITEMS, g = r / ZW::S, c = r % ZW::S;
      sl[(17 * g + c) * LD + f * TX] =
          16 * g + ZW::S * kq + c < kc ? gl[f * FS + (size_t)(16 * g + c) * N * N] : mk((T)0, (T)0);
    }
  } else {
    for (int it = w; it < 6 * ZW::ITEMS; it += NW) {
      const int f = it / ZW::ITEMS, r = it % ZW::ITEMS, g = r / ZW::S, c = r % ZW::S;
      sl[(17 * g + c) * LD + f * TX] = gl[f * FS + (size_t)(16 * g + c) * N * N];
    }
  }
  ZTw<T, N> zt;
  zt.load(tw, lane);
  __syncthreads();
  // c2r of the 6 TX lines (u and omega of each column); physical pairs are
  // written back into the same line at canonical positions
  cx<T> v[V];
#pragma unroll 1
  for (int l = w; l < 6 * TX; l += NW) {
    cx<T>* ln = s + l;
    zc_c2r<T, N>(v, ln, zt, tw, lane);
    cx<T>* pa = ln + padp(lane) * LD;
#pragma unroll
    for (int m = 0; m < V; ++m) pa[34 * m * LD] = v[m];
  }
  __syncthreads();
  // u x omega at every point, into the u lines
  for (int it = w; it < ZW::ITEMS; it += NW) {
    const int g = it / ZW::S, c = it % ZW::S;
    cx<T>* p = sl + (17 * g + c) * LD;
    const cx<T> u0 = p[0 * TX], u1 = p[1 * TX], u2 = p[2 * TX];
    const cx<T> w0 = p[3 * TX], w1 = p[4 * TX], w2 = p[5 * TX];
    p[0 * TX] = mk(u1.x * w2.x - u2.x * w1.x, u1.y * w2.y - u2.y * w1.y);
    p[1 * TX] = mk(u2.x * w0.x - u0.x * w2.x, u2.y * w0.y - u0.y * w2.y);
    p[2 * TX] = mk(u0.x * w1.x - u1.x * w0.x, u0.y * w1.y - u1.y * w0.y);
  }
  __syncthreads();
  // r2c of the 3 TX product lines, X_k (k < kc) written back into the line
#pragma unroll 1
  for (int l = w; l < 3 * TX; l += NW) {
    cx<T>* ln = s + l;
    const cx<T>* pa = ln + padp(lane) * LD;
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = pa[34 * m * LD];
    __syncwarp();
    zc_r2c<T, N>(v, ln, ln, kc, zt, tw, lane);
  }
  __syncthreads();
  cx<T>* gd = W + ((size_t)(ZW::S * kq) * N + y) * N + x0 + tx;
  for (int it = w; it < 3 * ZW::ITEMS; it += NW) {
    const int f = it / ZW::ITEMS, r = it % ZW::ITEMS, g = r / ZW::S, c = r % ZW::S;
    if (16 * g + ZW::S * kq + c < kc) gd[f * FS + (size_t)(16 * g + c) * N * N] = sl[(17 * g + c) * LD + f * TX];
  }
}

// ---------------------------------------------------------------------------
// Half-warp 256-point FFT of the N = 512 z-pass (lines of M = 256 values): each
// line belongs to one half-warp, lane h holding positions h + 16 m (m < 16),
// and the 256-point DFT is two radix-16 passes with a single shared-memory
// exchange whose stores (17 h + r) and loads (h + 17 m) are free of bank
// conflicts.
// ---------------------------------------------------------------------------
// Leaner per-lane twiddles for the FP32 pipelined z-pass: the second-pass powers
// p2[r] as in HwTw, and exp(-2 pi i (h + 16 m) / 512) formed on use as
// tl * exp(-2 pi i m / 32) with the second factor a compile-time constant.
struct HwTwL {
  cx<float> p2[16];
  cx<float> tl;
  // ts: stride into a twiddle table longer than the real line's own (1 on its own table)
  __device__ __forceinline__ void init(const cx<float>* __restrict__ tw, int h, int ts = 1) {
    twiddle_powers<16>(ldro(tw + 2 * h * ts), p2);
    tl = ldro(tw + h * ts);
  }
  __device__ __forceinline__ cx<float> wk(const cx<float>* __restrict__, int, int m) const {
    constexpr float c[16][2] = {
        {1.0f, -0.0f},
        {0.9807852804032304f, -0.19509032201612825f},
        {0.9238795325112867f, -0.3826834323650898f},
        {0.8314696123025452f, -0.5555702330196022f},
        {0.7071067811865476f, -0.7071067811865475f},
        {0.5555702330196023f, -0.8314696123025452f},
        {0.38268343236508984f, -0.9238795325112867f},
        {0.19509032201612833f, -0.9807852804032304f},
        {0.0f, -1.0f},
        {-0.1950903220161282f, -0.9807852804032304f},
        {-0.3826834323650897f, -0.9238795325112867f},
        {-0.555570233019602f, -0.8314696123025455f},
        {-0.7071067811865475f, -0.7071067811865476f},
        {-0.8314696123025453f, -0.5555702330196022f},
        {-0.9238795325112867f, -0.3826834323650899f},
        {-0.9807852804032304f, -0.1950903220161286f}
    };
    return m == 0 ? tl : cmul(tl, mk(c[m][0], c[m][1]));
  }
};

template <typename T, int TWN, int ES, class HT>
__device__ __forceinline__ void hw_fft256(cx<T> (&v)[16], cx<T>* ln, const HT& ht, const cx<T>* __restrict__ tw,
                                          int h) {
  dft16(v);
  cx<T>* q = ln + 17 * h * ES;
#pragma unroll
  for (int r = 0; r < 16; ++r) q[r * ES] = v[r];
  __syncwarp();
  const cx<T>* rb = ln + h * ES;
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = rb[17 * m * ES];
  __syncwarp();
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], ht.p2[r]);
  } else {
    constexpr int C = TWN / 256;
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], ldro(tw + h * r * C));
  }
  dft16(v);
}

// ---------------------------------------------------------------------------
// Pipelined z-pass for N = 512: one persistent block per SM walks tiles of
// 128-byte rows (16 adjacent x in FP32, 8 in FP64) at fixed y. The whole tile
// (6 fields x 256 kz) sits in shared memory and arrives by cp.async straight
// into the padded layout; the next tile's omega fields are fetched while the
// products are transformed and stored, its u fields while the omega lines are
// transformed, so HBM traffic overlaps the shared-memory-bound transforms.
// Line transforms, cross product and walks are those of k_zcross16. FP32 only:
// the FP64 form (8 x per row) would spill and keeps k_zcross16.
// ---------------------------------------------------------------------------
template <typename T>
struct Z16P {
  static constexpr int M = 256;
  static constexpr int TX = 128 / (int)sizeof(cx<T>);  // 128-byte rows
  static constexpr int LD = odd_ld(6 * TX);
  static constexpr int NW = 24;                        // warps per block
  static constexpr int ITEMS = (M / 32) * TX;          // walk items per field
  static constexpr size_t SMEM = (size_t)padded_len(M) * LD * sizeof(cx<T>);
};

template <typename T, int N>
__global__ void __launch_bounds__(32 * Z16P<T>::NW, 1) k_zcross16p(PassArgs a) {
  using P = Z16P<T>;
  constexpr int M = P::M, TX = P::TX, LD = P::LD, NW = P::NW, ITEMS = P::ITEMS;
  constexpr size_t FS = Geometry<T, N>::FS;
  constexpr int XT = N / TX, NT = XT * N;  // tiles: x-tiles times y
  static_assert(N == 512 && (TX == 8 || TX == 16), "k_zcross16p is the N = 512 z-pass");
  static_assert((3 * ITEMS) % NW == 0, "z tile load split");
    extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
  cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = lane & 15, half = lane >> 4;
  int kc = (a.kmax3 + 2) / 3;
  if (kc > M) kc = M;
  const int tx = lane % TX, kq = lane / TX;
  // lane part of the walk kz = 32 g + TX kq + c: padp(kz) = 34 g + padp(TX kq) + c
  cx<T>* const sl = s + padp(TX * kq) * LD + tx;
  const size_t lane_g = ((size_t)(TX * kq) * N) * N + tx;

  // asynchronous fetch of fields f0 .. f0+2 of tile t into their lines. Warp w takes the
  // 16 consecutive walk items 16 w + j: with ITEMS = 8 TX = 128 its field (w / 8) and row
  // group g = w % 8 are fixed and j is the row offset c, so the addresses are a per-warp
  // base plus j times a constant stride.
  static_assert(TX == 16 && ITEMS == 128 && 3 * ITEMS == 16 * NW, "z tile chunking");
  auto fetch = [&](int t, int f0) {
    // a stage whose state vanishes outside the 2/3 box: the planes kz >= kc hold zeros (the
    // y-inverse left them alone) and are filled with zeros instead of read
    const int f = f0 + w / 8, g = w % 8;
    const cx<T>* gl = W + lane_g + (size_t)(t / XT) * N + (t % XT) * TX + (size_t)f * FS + (size_t)(32 * g) * N * N;
    cx<T>* sd = sl + 34 * g * LD + f * TX;
    if (rows_vanish(a)) {
      const int nv = kc - (32 * g + TX * kq);  // rows of this lane's chunk below kc
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j < nv) cp_async<sizeof(cx<T>)>(sd + j * LD, gl + (size_t)j * N * N);
        else sd[j * LD] = mk((T)0, (T)0);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) cp_async<sizeof(cx<T>)>(sd + j * LD, gl + (size_t)j * N * N);
    }
  };
  // c2r of the TX lines of fields f0 .. f0+2, two lines per warp at a time
  HwTwL ht;
  ht.init(tw, h);
  // partner X_{M-k} of k = h + 16 m sits at padded row padp(M - k) = pb0 + 17 (15 - m)
  // with pb0 = 16 - h for h > 0 and 17 for h = 0 (k = 0 has no partner: X_M = 0)
  const int pb0 = (h == 0) ? 17 : 16 - h;
  // The inputs of modes k and M - k come from one pair (X_k, X_{M-k}): with
  // A = X_k + conj X_{M-k}, B = X_k - conj X_{M-k} and P = i conj(w_k) B,
  // z_k = A + P and z_{M-k} = conj(A - P). Lane h forms the pairs of its slots
  // m < 8 (k = h + 16 m); the mirror M - k = (16 - h) + 16 (15 - m) is slot
  // 15 - m of lane 16 - h, which receives it by a shuffle. Lane 0 pairs its slots
  // m and 16 - m, takes the self-paired k = M/2 at m = 0 and forms k = 0 apart.
  auto c2r_lines = [&](int f0) {
    cx<T> v[16];
#pragma unroll 1
    for (int l = f0 * TX + 2 * w + half; l < (f0 + 3) * TX; l += 2 * NW) {
      cx<T>* ln = s + l;
      const cx<T>* pa = ln + h * LD;
      const cx<T>* pb = ln + pb0 * LD;
      const cx<T> x0 = ln[0];
      cx<T> zq[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        cx<T> xk, xm, wk;
        if (m == 0) {
          const cx<T>* ph = ln + padp(M / 2) * LD;
          xk = (h == 0) ? *ph : pa[0];
          xm = (h == 0) ? xk : pb[17 * 15 * LD];
          wk = (h == 0) ? mk((T)0, (T)-1) : ht.wk(tw, h, 0);  // w_{M/2} = -i
        } else {
          xk = pa[17 * m * LD];
          xm = pb[17 * (15 - m) * LD];
          wk = ht.wk(tw, h, m);
        }
        const cx<T> A = xk + conjg(xm), B = xk - conjg(xm);
        const cx<T> P = mul_pi(cmul(conjg(wk), B));
        v[m] = conjg(A + P);
        zq[m] = A - P;  // conj of z_{M-k}
      }
      const int src = (16 - h) & 15;
#pragma unroll
      for (int q = 8; q < 16; ++q) {
        v[q].x = __shfl_sync(0xffffffffu, zq[15 - q].x, src, 16);
        v[q].y = __shfl_sync(0xffffffffu, zq[15 - q].y, src, 16);
      }
      if (h == 0) {
        v[8] = v[0];
#pragma unroll
        for (int q = 9; q < 16; ++q) v[q] = zq[16 - q];
        v[0] = mk(x0.x, -x0.x);  // z_0 = (1 + i) Re X_0: Im X_0 ignored, X_M = 0
      }
      __syncwarp();
      hw_fft256<T, N, LD>(v, ln, ht, tw, h);
      cx<T>* pw = ln + h * LD;
#pragma unroll
      for (int m = 0; m < 16; ++m) pw[17 * m * LD] = conjg(v[m]);
    }
  };

  int t = blockIdx.x;
  if (t < NT) fetch(t, 3);
  cp_async_commit();
  if (t < NT) fetch(t, 0);
  cp_async_commit();
#pragma unroll 1
  for (; t < NT; t += gridDim.x) {
    const int x0 = (t % XT) * TX, y = t / XT, tn = t + gridDim.x;
    cp_async_wait<1>();  // omega fields of tile t
    __syncthreads();
    c2r_lines(3);
    cp_async_wait<0>();  // u fields of tile t
    __syncthreads();
    c2r_lines(0);
    __syncthreads();
    // u x omega at every point, into the u lines
    for (int it = w; it < ITEMS; it += NW) {
      const int g = it / TX, c = it % TX;
      cx<T>* p = sl + (34 * g + c) * LD;
      const cx<T> u0 = p[0 * TX], u1 = p[1 * TX], u2 = p[2 * TX];
      const cx<T> w0 = p[3 * TX], w1v = p[4 * TX], w2 = p[5 * TX];
      p[0 * TX] = mk(u1.x * w2.x - u2.x * w1v.x, u1.y * w2.y - u2.y * w1v.y);
      p[1 * TX] = mk(u2.x * w0.x - u0.x * w2.x, u2.y * w0.y - u0.y * w2.y);
      p[2 * TX] = mk(u0.x * w1v.x - u1.x * w0.x, u0.y * w1v.y - u1.y * w0.y);
    }
    __syncthreads();
    if (tn < NT) fetch(tn, 3);  // the omega lines are free
    cp_async_commit();
    // r2c of the 3 TX product lines; X_k (k < kc) back into the line
    {
      cx<T> v[16];
#pragma unroll 1
      for (int l = 2 * w + half; l < 3 * TX; l += 2 * NW) {
        cx<T>* ln = s + l;
        const cx<T>* pa = ln + h * LD;
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = pa[17 * m * LD];
        __syncwarp();
        hw_fft256<T, N, LD>(v, ln, ht, tw, h);
        cx<T>* po = ln + h * LD;
        const int partner = (16 - h) & 15;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          if (16 * m >= kc) break;  // slots m and above hold modes past the 2/3 cut
          cx<T> zo;
          zo.x = __shfl_sync(0xffffffffu, v[15 - m].x, partner, 16);
          zo.y = __shfl_sync(0xffffffffu, v[15 - m].y, partner, 16);
          if (h == 0) zo = v[(16 - m) & 15];
          const cx<T> wk = ht.wk(tw, h, m);
          const cx<T> A = v[m] + conjg(zo), B = v[m] - conjg(zo);
          if (h + 16 * m < kc) po[17 * m * LD] = scal(A + mul_mi(cmul(wk, B)), (T)0.5);
        }
      }
    }
    __syncthreads();
    {  // the same chunks as the fetch: field w / 8, rows 32 (w % 8) + TX kq + j
      const int f = w / 8, g = w % 8, k0 = 32 * g + TX * kq;
      cx<T>* gd = W + lane_g + (size_t)y * N + x0 + (size_t)f * FS + (size_t)(32 * g) * N * N;
      const cx<T>* sd = sl + 34 * g * LD + f * TX;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (k0 + j < kc) gd[(size_t)j * N * N] = sd[j * LD];
    }
    __syncthreads();  // the u lines have been read out
    if (tn < NT) fetch(tn, 0);
    cp_async_commit();
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Half-warp 512-point FFT for the N = 1024 z-pass (FP32). Lane h of a half-warp
// holds v[m] = x[h + 16 m], m < 32. With k = k1 + 32 k2: a 32-point DFT over m in
// each lane gives Y[h][k1]; after the twiddle exp(-2 pi i h k1 / 512) one
// shared-memory exchange (stores at 33 h + k1, loads at 33 h + h' and
// 33 h + h' + 16: conflict-free for any odd element stride) gives lane h' the
// 16-point columns k1 = h' and h' + 16, whose DFTs over h leave
// v[j] = X[h' + 16 j] in the lane: the input layout again.
// ---------------------------------------------------------------------------
struct HwTw32 {
  cx<float> p[16];  // w^r, w = exp(-2 pi i h / 512), r < 16
  cx<float> q[16];  // w^(16 + r)
  cx<float> tl;     // exp(-2 pi i h / 1024)
  __device__ __forceinline__ void init(const cx<float>* __restrict__ tw, int h) {
    twiddle_powers<16>(ldro(tw + 2 * h), p);
    p[0] = mk(1.f, 0.f);
    const cx<float> w16 = cmul(p[8], p[8]);
#pragma unroll
    for (int r = 0; r < 16; ++r) q[r] = r == 0 ? w16 : cmul(w16, p[r]);
    tl = ldro(tw + h);
  }
  // exp(-2 pi i (h + 16 m) / 1024) = tl * exp(-2 pi i m / 64)
  __device__ __forceinline__ cx<float> wk(int m) const {
    constexpr float c[32][2] = {
      {1.0f, 0.0f},
      {0.9951847266721969f, -0.0980171403295606f},
      {0.9807852804032304f, -0.19509032201612825f},
      {0.9569403357322088f, -0.29028467725446233f},
      {0.9238795325112867f, -0.3826834323650898f},
      {0.881921264348355f, -0.47139673682599764f},
      {0.8314696123025452f, -0.5555702330196022f},
      {0.773010453362737f, -0.6343932841636455f},
      {0.7071067811865476f, -0.7071067811865475f},
      {0.6343932841636455f, -0.773010453362737f},
      {0.5555702330196023f, -0.8314696123025452f},
      {0.4713967368259978f, -0.8819212643483549f},
      {0.38268343236508984f, -0.9238795325112867f},
      {0.29028467725446233f, -0.9569403357322089f},
      {0.19509032201612833f, -0.9807852804032304f},
      {0.09801714032956077f, -0.9951847266721968f},
      {0.0f, -1.0f},
      {-0.09801714032956065f, -0.9951847266721969f},
      {-0.1950903220161282f, -0.9807852804032304f},
      {-0.29028467725446216f, -0.9569403357322089f},
      {-0.3826834323650897f, -0.9238795325112867f},
      {-0.4713967368259977f, -0.881921264348355f},
      {-0.555570233019602f, -0.8314696123025455f},
      {-0.6343932841636454f, -0.7730104533627371f},
      {-0.7071067811865475f, -0.7071067811865476f},
      {-0.773010453362737f, -0.6343932841636455f},
      {-0.8314696123025453f, -0.5555702330196022f},
      {-0.8819212643483549f, -0.47139673682599786f},
      {-0.9238795325112867f, -0.3826834323650899f},
      {-0.9569403357322088f, -0.2902846772544624f},
      {-0.9807852804032304f, -0.1950903220161286f},
      {-0.9951847266721968f, -0.09801714032956083f}};
    return m == 0 ? tl : cmul(tl, mk(c[m][0], c[m][1]));
  }
};

template <int ES>
__device__ __forceinline__ void hw_fft512(cx<float> (&v)[32], cx<float>* ln, const HwTw32& ht, int h) {
  dft32(v);
#pragma unroll
  for (int k = 1; k < 32; ++k) v[k] = cmul(v[k], k < 16 ? ht.p[k] : ht.q[k - 16]);
  cx<float>* q = ln + 33 * h * ES;
#pragma unroll
  for (int k = 0; k < 32; ++k) q[k * ES] = v[k];
  __syncwarp();
  cx<float> a[16], b[16];
  const cx<float>* rb = ln + h * ES;
#pragma unroll
  for (int g = 0; g < 16; ++g) {
    a[g] = rb[33 * g * ES];
    b[g] = rb[(33 * g + 16) * ES];
  }
  __syncwarp();
  dft16(a);
  dft16(b);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    v[2 * k2] = a[k2];
    v[2 * k2 + 1] = b[k2];
  }
}

// Pipelined z-pass for N = 1024, FP32, with half-warp lines: the schedule of
// k_zcross16p (persistent block, whole tile in shared memory, next tile's omega
// fields fetched during the product transforms, its u fields during the omega
// transforms) on tiles of 8 adjacent x (64-byte rows) and 512-value lines.
template <typename T>
struct Z32P {
  static constexpr int M = 512;
  static constexpr int TX = 64 / (int)sizeof(cx<T>);
  static constexpr int LD = odd_ld(6 * TX);
  static constexpr int NW = 12;
  static constexpr int ITEMS = (M / 32) * TX;
  static constexpr size_t SMEM = (size_t)padded_len(M) * LD * sizeof(cx<T>);
};

template <typename T, int N>
__global__ void __launch_bounds__(32 * Z32P<T>::NW, 1) k_zcross32p(PassArgs a) {
  using P = Z32P<T>;
  using G = Geometry<T, N>;
  constexpr int M = P::M, TX = P::TX, LD = P::LD, NW = P::NW, ITEMS = P::ITEMS;
  constexpr size_t FS = G::FS;
  constexpr int XT = N / TX, NT = XT * N;
  static_assert(N == 1024 && sizeof(T) == 4 && TX == 8, "k_zcross32p is the FP32 N = 1024 z-pass");
  static_assert((3 * ITEMS) % NW == 0 && (3 * TX) % (2 * NW) == 0, "z tile split");
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
  cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = lane & 15, half = lane >> 4;
  int kc = (a.kmax3 + 2) / 3;
  if (kc > M) kc = M;
  const int tx = lane % TX, kq = lane / TX;
  // walk kz = 32 g + TX kq + c: padp(kz) = 34 g + padp(TX kq) + c
  cx<T>* const sl = s + padp(TX * kq) * LD + tx;
  const size_t lane_g = ((size_t)(TX * kq) * N) * N + tx;
  // warp w takes the 32 consecutive walk items 32 w + j (j = 8 a + b): field f0 + w / 4, row
  // group g = 4 (w % 4) + a, row offset c = b, so the addresses are a per-warp base plus
  // compile-time offsets
  static_assert(TX == 8 && ITEMS == 128 && 3 * ITEMS == 32 * NW, "z tile chunking");
  auto fetch = [&](int t, int f0) {
    // planes kz >= kc of a stage whose state vanishes outside the 2/3 box: zeros, not read
    const int f = f0 + w / 4, q = w % 4;
    const cx<T>* gl = W + lane_g + (size_t)(t / XT) * N + (t % XT) * TX + (size_t)f * FS + (size_t)(128 * q) * N * N;
    cx<T>* sd = sl + 136 * q * LD + f * TX;
    if (rows_vanish(a)) {
      const int nv = kc - (128 * q + TX * kq);  // this lane's rows below kc: 32 (j / 8) + j % 8 < nv
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (32 * (j / 8) + j % 8 < nv)
          cp_async<sizeof(cx<T>)>(sd + (34 * (j / 8) + j % 8) * LD, gl + (size_t)(32 * (j / 8) + j % 8) * N * N);
        else
          sd[(34 * (j / 8) + j % 8) * LD] = mk((T)0, (T)0);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        cp_async<sizeof(cx<T>)>(sd + (34 * (j / 8) + j % 8) * LD, gl + (size_t)(32 * (j / 8) + j % 8) * N * N);
    }
  };
  HwTw32 ht;
  ht.init(tw, h);
  // partner X_{M-k} of k = h + 16 m at padded row pb0 + 17 (31 - m), pb0 = 16 - h (h > 0), 17 (h = 0)
  const int pb0 = (h == 0) ? 17 : 16 - h;
  auto c2r_lines = [&](int f0) {
    cx<T> v[32];
#pragma unroll 1
    for (int l = f0 * TX + 2 * w + half; l < (f0 + 3) * TX; l += 2 * NW) {
      cx<T>* ln = s + l;
      const cx<T>* pa = ln + h * LD;
      const cx<T>* pb = ln + pb0 * LD;
      const cx<T> x0 = ln[0];
      // modes k = h + 16 m (m < 16) and M - k = (16 - h) + 16 (31 - m) from one pair:
      // z_k = A + P, z_{M-k} = conj(A - P), the mirror going to slot 31 - m of lane
      // 16 - h; lane 0 pairs its slots m and 32 - m and takes k = M/2 at m = 0
      cx<T> zq[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        cx<T> xk, xm, wk;
        if (m == 0) {
          const cx<T>* ph = ln + padp(M / 2) * LD;
          xk = (h == 0) ? *ph : pa[0];
          xm = (h == 0) ? xk : pb[17 * 31 * LD];
          wk = (h == 0) ? mk((T)0, (T)-1) : ht.wk(0);  // w_{M/2} = -i
        } else {
          xk = pa[17 * m * LD];
          xm = pb[17 * (31 - m) * LD];
          wk = ht.wk(m);
        }
        const cx<T> A = xk + conjg(xm), B = xk - conjg(xm);
        const cx<T> P = mul_pi(cmul(conjg(wk), B));
        v[m] = conjg(A + P);
        zq[m] = A - P;  // conj of z_{M-k}
      }
      const int src = (16 - h) & 15;
#pragma unroll
      for (int q = 16; q < 32; ++q) {
        v[q].x = __shfl_sync(0xffffffffu, zq[31 - q].x, src, 16);
        v[q].y = __shfl_sync(0xffffffffu, zq[31 - q].y, src, 16);
      }
      if (h == 0) {
        v[16] = v[0];
#pragma unroll
        for (int q = 17; q < 32; ++q) v[q] = zq[32 - q];
        v[0] = mk(x0.x, -x0.x);  // z_0 = (1 + i) Re X_0: Im X_0 ignored, X_M = 0
      }
      __syncwarp();
      hw_fft512<LD>(v, ln, ht, h);
      cx<T>* pw = ln + h * LD;
#pragma unroll
      for (int m = 0; m < 32; ++m) pw[17 * m * LD] = conjg(v[m]);
    }
  };

  int t = blockIdx.x;
  if (t < NT) fetch(t, 3);
  cp_async_commit();
  if (t < NT) fetch(t, 0);
  cp_async_commit();
#pragma unroll 1
  for (; t < NT; t += gridDim.x) {
    const int x0 = (t % XT) * TX, y = t / XT, tn = t + gridDim.x;
    cp_async_wait<1>();  // omega fields of tile t
    __syncthreads();
    c2r_lines(3);
    cp_async_wait<0>();  // u fields of tile t
    __syncthreads();
    c2r_lines(0);
    __syncthreads();
    for (int it = w; it < ITEMS; it += NW) {
      const int g = it / TX, c = it % TX;
      cx<T>* p = sl + (34 * g + c) * LD;
      const cx<T> u0 = p[0 * TX], u1 = p[1 * TX], u2 = p[2 * TX];
      const cx<T> w0 = p[3 * TX], w1v = p[4 * TX], w2 = p[5 * TX];
      p[0 * TX] = mk(u1.x * w2.x - u2.x * w1v.x, u1.y * w2.y - u2.y * w1v.y);
      p[1 * TX] = mk(u2.x * w0.x - u0.x * w2.x, u2.y * w0.y - u0.y * w2.y);
      p[2 * TX] = mk(u0.x * w1v.x - u1.x * w0.x, u0.y * w1v.y - u1.y * w0.y);
    }
    __syncthreads();
    if (tn < NT) fetch(tn, 3);  // the omega lines are free
    cp_async_commit();
    {
      cx<T> v[32];
#pragma unroll 1
      for (int l = 2 * w + half; l < 3 * TX; l += 2 * NW) {
        cx<T>* ln = s + l;
        const cx<T>* pa = ln + h * LD;
#pragma unroll
        for (int m = 0; m < 32; ++m) v[m] = pa[17 * m * LD];
        __syncwarp();
        hw_fft512<LD>(v, ln, ht, h);
        cx<T>* po = ln + h * LD;
        const int partner = (16 - h) & 15;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
          if (16 * m >= kc) break;  // slots m and above hold modes past the 2/3 cut
          cx<T> zo;
          zo.x = __shfl_sync(0xffffffffu, v[31 - m].x, partner, 16);
          zo.y = __shfl_sync(0xffffffffu, v[31 - m].y, partner, 16);
          if (h == 0) zo = v[(32 - m) & 31];
          const cx<T> wk = ht.wk(m);
          const cx<T> A = v[m] + conjg(zo), B = v[m] - conjg(zo);
          if (h + 16 * m < kc) po[17 * m * LD] = scal(A + mul_mi(cmul(wk, B)), (T)0.5);
        }
      }
    }
    __syncthreads();
    {  // the same chunks as the fetch: field w / 4, rows 128 (w % 4) + 32 a + TX kq + b
      const int f = w / 4, q = w % 4, k0 = 128 * q + TX * kq;
      cx<T>* gd = W + lane_g + (size_t)y * N + x0 + (size_t)f * FS + (size_t)(128 * q) * N * N;
      const cx<T>* sd = sl + 136 * q * LD + f * TX;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (k0 + 32 * (j / 8) + j % 8 < kc) gd[(size_t)(32 * (j / 8) + j % 8) * N * N] = sd[(34 * (j / 8) + j % 8) * LD];
    }
    __syncthreads();  // the u lines have been read out
    if (tn < NT) fetch(tn, 0);
    cp_async_commit();
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Quarter-warp 128-point FFT for the N = 256 z-pass (FP32): lane h < 8 of a
// quarter-warp holds v[m] = x[h + 8 m], m < 16; a 16-point DFT in each lane, the
// twiddle exp(-2 pi i h k1 / 128), one exchange through positions 17 h + k1 and two
// 8-point DFTs per lane leave v[j] = X[h + 8 j] in the lane. The two quarter-warps of
// a half-warp work on lines l and l + 8, whose banks are disjoint. The twiddles are
// those of the 256-point half-warp transform (HwTwL) on the N = 256 table.
// ---------------------------------------------------------------------------
template <int ES>
__device__ __forceinline__ void qw_fft128(cx<float> (&v)[16], cx<float>* ln, const HwTwL& qt, int h) {
  dft16(v);
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], qt.p2[k]);
  cx<float>* q = ln + 17 * h * ES;
#pragma unroll
  for (int k = 0; k < 16; ++k) q[k * ES] = v[k];
  __syncwarp();
  cx<float> a[8], b[8];
  const cx<float>* rb = ln + h * ES;
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    a[g] = rb[17 * g * ES];
    b[g] = rb[(17 * g + 8) * ES];
  }
  __syncwarp();
  dft8(a);
  dft8(b);
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) {
    v[2 * k2] = a[k2];
    v[2 * k2 + 1] = b[k2];
  }
}

template <typename T>
struct Z8Q {
  static constexpr int M = 128;
  static constexpr int TX = 128 / (int)sizeof(cx<T>);  // 128-byte rows
  static constexpr int LD = odd_ld(6 * TX);
  static constexpr int NW = 12;
  static constexpr int ITEMS = (M / 32) * TX;
  static constexpr size_t SMEM = (size_t)padded_len(M) * LD * sizeof(cx<T>);
};

// z-pass for N = 256, FP32: one tile (16 adjacent x at fixed y, 6 fields of 128
// values) per block, fetched whole by cp.async, two blocks per SM; each warp
// transforms four lines at once as quarter-warps (lines b, b + 8, b + 1, b + 9).
// NY, NZ: counts along y and z where they differ from N (NZ = 256; N a multiple of 16).
template <typename T, int N, int NY = N, int NZ = N>
__global__ void __launch_bounds__(32 * Z8Q<T>::NW, 2) k_zcross8q(PassArgs a) {
  using P = Z8Q<T>;
  using G = Geometry<T, N, NY, NZ>;
  constexpr int M = P::M, TX = P::TX, LD = P::LD, NW = P::NW, ITEMS = P::ITEMS;
  constexpr size_t FS = G::FS;
  constexpr size_t PL = (size_t)NY * N;  // one kz plane
  static_assert(NZ == 256 && N % TX == 0 && sizeof(T) == 4 && TX == 16, "k_zcross8q is the FP32 256-point z-pass");
  static_assert((6 * ITEMS) % NW == 0, "z tile split");
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
  cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h = lane & 7, qw = lane >> 3;
  const int x0 = blockIdx.x * TX, y = blockIdx.y;
  int kc = ((NZ == N ? a.kmax3 : a.kmax3z) + 2) / 3;
  if (kc > M) kc = M;
  const int tx = lane % TX, kq = lane / TX;
  // walk kz = 32 g + TX kq + c: padp(kz) = 34 g + padp(TX kq) + c
  cx<T>* const sl = s + padp(TX * kq) * LD + tx;
  const cx<T>* gl = W + ((size_t)(TX * kq) * NY + y) * N + x0 + tx;
  // warp w takes the 32 consecutive walk items 32 w + j (j = 16 a + b): field w / 2, row group
  // g = 2 (w % 2) + a, row offset c = b: a per-warp base plus compile-time offsets
  static_assert(TX == 16 && ITEMS == 64 && 6 * ITEMS == 32 * NW && 3 * ITEMS == 16 * NW, "z tile chunking");
  {
    const int f = w / 2, q = w % 2;
    const cx<T>* gf = gl + (size_t)f * FS + (size_t)(64 * q) * PL;
    cx<T>* sd = sl + 68 * q * LD + f * TX;
    if (rows_vanish(a)) {  // planes kz >= kc of a state that vanishes outside the 2/3 box: zeros
      const int nv = kc - (64 * q + TX * kq);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (32 * (j / 16) + j % 16 < nv)
          cp_async<sizeof(cx<T>)>(sd + (34 * (j / 16) + j % 16) * LD, gf + (size_t)(32 * (j / 16) + j % 16) * PL);
        else
          sd[(34 * (j / 16) + j % 16) * LD] = mk((T)0, (T)0);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        cp_async<sizeof(cx<T>)>(sd + (34 * (j / 16) + j % 16) * LD, gf + (size_t)(32 * (j / 16) + j % 16) * PL);
    }
  }
  cp_async_commit();
  HwTwL qt;  // w = exp(-2 pi i h / 128), tl = exp(-2 pi i h / 256)
  qt.init(tw, h, G::TW / NZ);
  // quarter-warp line of group gi (groups of 4 lines b, b + 8, b + 1, b + 9 with b = 16 f + 2 i)
  auto line_of = [&](int gi) { return 16 * (gi >> 2) + 2 * (gi & 3) + (qw & 1) * 8 + (qw >> 1); };
  cp_async_wait<0>();
  __syncthreads();
  {
    cx<T> v[16];
#pragma unroll 1
    for (int gi = w; gi < 6 * 4; gi += NW) {  // c2r of the 96 lines
      cx<T>* ln = s + line_of(gi);
      const cx<T> x0 = ln[0];
      // modes k = h + 8 m (m < 8) and M - k = (8 - h) + 8 (15 - m) from one pair:
      // z_k = A + P, z_{M-k} = conj(A - P), the mirror going to slot 15 - m of lane
      // 8 - h; lane 0 pairs its slots m and 16 - m and takes k = M/2 at m = 0
      cx<T> zq[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int k = (m == 0 && h == 0) ? M / 2 : h + 8 * m;
        const cx<T> xk = ln[padp(k) * LD];
        const cx<T> xm = (m == 0 && h == 0) ? xk : ln[padp(M - k) * LD];
        const cx<T> wk = (m == 0 && h == 0) ? mk((T)0, (T)-1) : qt.wk(tw, h, m);  // w_{M/2} = -i
        const cx<T> A = xk + conjg(xm), B = xk - conjg(xm);
        const cx<T> P = mul_pi(cmul(conjg(wk), B));
        v[m] = conjg(A + P);
        zq[m] = A - P;  // conj of z_{M-k}
      }
      const int src = (8 - h) & 7;
#pragma unroll
      for (int q = 8; q < 16; ++q) {
        v[q].x = __shfl_sync(0xffffffffu, zq[15 - q].x, src, 8);
        v[q].y = __shfl_sync(0xffffffffu, zq[15 - q].y, src, 8);
      }
      if (h == 0) {
        v[8] = v[0];
#pragma unroll
        for (int q = 9; q < 16; ++q) v[q] = zq[16 - q];
        v[0] = mk(x0.x, -x0.x);  // z_0 = (1 + i) Re X_0: Im X_0 ignored, X_M = 0
      }
      __syncwarp();
      qw_fft128<LD>(v, ln, qt, h);
#pragma unroll
      for (int m = 0; m < 16; ++m) ln[padp(h + 8 * m) * LD] = conjg(v[m]);
    }
  }
  __syncthreads();
  for (int it = w; it < ITEMS; it += NW) {
    const int g = it / TX, c = it % TX;
    cx<T>* p = sl + (34 * g + c) * LD;
    const cx<T> u0 = p[0 * TX], u1 = p[1 * TX], u2 = p[2 * TX];
    const cx<T> w0 = p[3 * TX], w1v = p[4 * TX], w2 = p[5 * TX];
    p[0 * TX] = mk(u1.x * w2.x - u2.x * w1v.x, u1.y * w2.y - u2.y * w1v.y);
    p[1 * TX] = mk(u2.x * w0.x - u0.x * w2.x, u2.y * w0.y - u0.y * w2.y);
    p[2 * TX] = mk(u0.x * w1v.x - u1.x * w0.x, u0.y * w1v.y - u1.y * w0.y);
  }
  __syncthreads();
  {
    cx<T> v[16];
    const int partner = (8 - h) & 7;
#pragma unroll 1
    for (int gi = w; gi < 3 * 4; gi += NW) {  // r2c of the 48 product lines
      cx<T>* ln = s + line_of(gi);
#pragma unroll
      for (int m = 0; m < 16; ++m) v[m] = ln[padp(h + 8 * m) * LD];
      __syncwarp();
      qw_fft128<LD>(v, ln, qt, h);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        if (8 * m >= kc) break;  // slots m and above hold modes past the 2/3 cut
        cx<T> zo;
        zo.x = __shfl_sync(0xffffffffu, v[15 - m].x, partner, 8);
        zo.y = __shfl_sync(0xffffffffu, v[15 - m].y, partner, 8);
        if (h == 0) zo = v[(16 - m) & 15];
        const cx<T> wk = qt.wk(tw, h, m);
        const cx<T> A = v[m] + conjg(zo), B = v[m] - conjg(zo);
        if (h + 8 * m < kc) ln[padp(h + 8 * m) * LD] = scal(A + mul_mi(cmul(wk, B)), (T)0.5);
      }
    }
  }
  __syncthreads();
  {  // warp w stores items 16 w + j: field w / 4, rows 32 (w % 4) + TX kq + j
    const int f = w / 4, g = w % 4, k0 = 32 * g + TX * kq;
    cx<T>* gd = W + ((size_t)(TX * kq) * NY + y) * N + x0 + tx + (size_t)f * FS + (size_t)(32 * g) * PL;
    const cx<T>* sd = sl + 34 * g * LD + f * TX;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (k0 + j < kc) gd[(size_t)j * PL] = sd[j * LD];
  }
}

// ---------------------------------------------------------------------------
// FP64 spectral sums for the diagnostics (Parseval): per block
//   sum w|u|^2, sum w|omega|^2, sum w Re(conj(u).omega), count of non-finite,
// w = 1 at kz = 0 and 2 otherwise (half spectrum; kz = N/2 is zero).
// ---------------------------------------------------------------------------
template <typename T, int N, int NY = N, int NZ = N>
__global__ void __launch_bounds__(DG_THREADS) k_diag(PassArgs a) {
  using G = Geometry<T, N, NY, NZ>;
  constexpr size_t FS = G::FS;
  const cx<T>* U = reinterpret_cast<const cx<T>*>(a.U);
  double se = 0, sz = 0, sh = 0, bad = 0;
  for (size_t i = (size_t)blockIdx.x * DG_THREADS + threadIdx.x; i < FS; i += (size_t)gridDim.x * DG_THREADS) {
    const int kxi = (int)(i % N), kyi = (int)((i / N) % NY), kzi = (int)(i / ((size_t)N * NY));
    const double kx = kfreq(kxi, N) * a.ks[0], ky = kfreq(kyi, NY) * a.ks[1], kz = kzi * a.ks[2];
    const double w = kzi == 0 ? 1.0 : 2.0;
    const cx<T> a0 = U[i], a1 = U[FS + i], a2 = U[2 * FS + i];
    const double u0r = a0.x, u0i = a0.y, u1r = a1.x, u1i = a1.y, u2r = a2.x, u2i = a2.y;
    // omega = i (k x u): real part = -(k x u).imag, imag part = (k x u).real
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
  __shared__ double red[4][DG_THREADS / 32];
  double v[4] = {se, sz, sh, bad};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int w = 0; w < DG_THREADS / 32; ++w) t += red[threadIdx.x][w];
    a.partials[blockIdx.x * 4 + threadIdx.x] = t;
  }
}

// Fixed-order final sum of the block partials into partials[DIAG_BLOCKS*4 + q].
__global__ void k_diag_final(double* partials, int nblocks);

// ---------------------------------------------------------------------------
// Host launchers for one (T, N).
// ---------------------------------------------------------------------------
// Number of SMs of the current device (persistent kernels launch one block each).
inline int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      n = 148;
  }
  return n;
}

// NY, NZ: points along y and z where they differ from N (a non-cubic grid runs the
// generic passes only: no tuned tile widths, specialised z-passes or batched
// ensembles).
template <typename T, int N, int NY = N, int NZ = N>
struct SolverImpl {
  using G = Geometry<T, N, NY, NZ>;
  static constexpr int M = G::M;
  static constexpr bool ISO = NY == N && NZ == N;
  static constexpr int ROWS = M * NY;  // x-pass rows (kz, ky)
  static constexpr bool BATCHED = ISO && N <= BATCH_MAX_N && !ZCross<T, N>::enabled;
  // non-cubic grids with 256-point FP32 z-lines use the quarter-warp z-pass of 256^3
  static constexpr bool Z8_BOX = !ISO && NZ == 256 && sizeof(T) == 4 && N % 16 == 0;
  // each direction's 2/3 cut-off (3|k_i| < kmax3 of that direction)
  static int k3y(const PassArgs& a) { return NY == N ? a.kmax3 : a.kmax3y; }
  static int k3z(const PassArgs& a) { return NZ == N ? a.kmax3 : a.kmax3z; }

  template <class K>
  static cudaError_t smem_attr(K k, size_t bytes) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }

  // y-pass tile widths offered to a tuner besides the default (grids of the
  // ensembles only, to bound the number of instantiations)
  static constexpr bool ytile_ok(int t) {
    return ISO && N <= BATCH_MAX_N && t >= 4 && t <= 32 && pow2_part(N) % t == 0 && t * (int)sizeof(cx<T>) <= 256;
  }
  // radix plan variants of the stage's line transforms offered to the tuner (SmemPlanV /
  // LinePlanV: 0 the default schedule, 1 AltPlan); the ensemble grids only. PassArgs::plan
  // holds one bit per pass: PLAN_X (x-stage and x inverse), PLAN_YI (y-inverse),
  // PLAN_Z (z-pass), PLAN_YF (y-forward).
  static constexpr int PLANS = (ISO && N <= BATCH_MAX_N) ? 2 : 1;
  // The handle's initial plan mask: AltPlan in the passes where it measured faster on
  // GB300 (per-pass CUDA-event times of both schedules, 100 graph-replayed steps; FP64
  // passes whose default has a radix-16 pass or radix-8 passes only run about twice as
  // fast with radix 4). dns_tune_tiles re-measures on the machine at hand.
  static constexpr int default_plan() {
    if constexpr (PLANS == 1) {
      return 0;
    } else if constexpr (sizeof(T) == 8) {
      constexpr int XYY = (1 << PLAN_X) | (1 << PLAN_YI) | (1 << PLAN_YF);
      return (N == 16 || N == 48 || N == 64 || N == 128) ? XYY : 0;
    } else {
      switch (N) {
        case 48: return (1 << PLAN_X) | (1 << PLAN_YF);
        case 64: return (1 << PLAN_X) | (1 << PLAN_YI);
        case 128: return (1 << PLAN_X) | (1 << PLAN_YI) | (1 << PLAN_YF);
        default: return 0;
      }
    }
  }
  static int bit(int plan, int b) { return (plan >> b) & 1; }
  // f(std::integral_constant<int, V>) with the variant V = plan (0 where not offered)
  template <class F>
  static void with_plan(int plan, F&& f) {
    if constexpr (PLANS > 1) {
      if (plan == 1) return f(std::integral_constant<int, 1>{});
    }
    f(std::integral_constant<int, 0>{});
  }

  template <int TXO, int V>
  static void tile_attr_v(cudaError_t& e) {
    if (e == cudaSuccess) e = smem_attr(k_ypass<T, N, 1, 0, TXO, N, N, V>, YCfg<T, N, 1, TXO>::SMEM);
    if (e == cudaSuccess) e = smem_attr(k_ypass<T, N, 1, 0, TXO, N, N, V, 1>, YCfg<T, N, 1, TXO>::SMEM);
    if (e == cudaSuccess) e = smem_attr(k_ypass<T, N, 0, 1, TXO, N, N, V>, YCfg<T, N, 0, TXO>::SMEM);
    if constexpr (!ZCross<T, N>::enabled) {
      if (e == cudaSuccess) e = smem_attr(k_ypass_b<T, N, 1, 0, TXO, V>, YCfg<T, N, 1, TXO>::SMEM);
      if (e == cudaSuccess) e = smem_attr(k_ypass_b<T, N, 0, 1, TXO, V>, YCfg<T, N, 0, TXO>::SMEM);
    }
  }
  template <int TXO>
  static void tile_attr(cudaError_t& e) {
    if constexpr (ytile_ok(TXO)) {
      tile_attr_v<TXO, 0>(e);
      if constexpr (PLANS > 1) tile_attr_v<TXO, 1>(e);
    }
  }
  static int y_tiles(int* tiles, int max) {
    int n = 0;
    for (int t = 4; t <= 32; t *= 2)
      if (ytile_ok(t) && n < max) tiles[n++] = t;
    return n;
  }
  // z-pass tile widths offered besides the default (the generic z-pass of the small grids)
  static constexpr bool ztile_ok(int t) {
    return ISO && N <= BATCH_MAX_N && !ZCross<T, N>::enabled && t >= 4 && t <= 32 && pow2_part(N) % t == 0 &&
           G::zbytes(t) <= 112 * 1024;
  }
  template <int TXO>
  static void ztile_attr(cudaError_t& e) {
    if constexpr (ztile_ok(TXO)) {
      if (e == cudaSuccess) e = smem_attr(k_zpass<T, N, ZM_CROSS, TXO>, G::zbytes(TXO));
      if (e == cudaSuccess) e = smem_attr(k_zpass_b<T, N, ZM_CROSS, TXO>, G::zbytes(TXO));
      if constexpr (PLANS > 1) {
        if (e == cudaSuccess) e = smem_attr(k_zpass<T, N, ZM_CROSS, TXO, N, N, 1>, G::zbytes(TXO));
        if (e == cudaSuccess) e = smem_attr(k_zpass_b<T, N, ZM_CROSS, TXO, 1>, G::zbytes(TXO));
      }
    }
  }
  static int z_tiles(int* tiles, int max) {
    int n = 0;
    for (int t = 4; t <= 32; t *= 2)
      if (ztile_ok(t) && n < max) tiles[n++] = t;
    return n;
  }
  template <int TXO, int V = 0>
  static void z_go(const PassArgs& a, cudaStream_t st) {
    constexpr int TX = TXO > 0 ? TXO : G::ZTX;
    k_zpass<T, N, ZM_CROSS, TXO, NY, NZ, V><<<dim3(N / TX, NY), ZP_THREADS, G::zbytes(TX), st>>>(a);
  }
  // PR: the y-inverse of a stage whose state vanishes outside the 2/3 box (k_ypass)
  template <int INV, int PRUNE, int TXO, int V = 0, int PR = 0>
  static void y_go(cx<T>* F, const cx<T>* tw, int kmax3, int planes, int fields, cudaStream_t st) {
    using Y = YCfg<T, N, INV, TXO, NY>;
    k_ypass<T, N, INV, PRUNE, TXO, NY, NZ, V, PR><<<dim3(N / Y::TX, planes, fields), Y::THREADS, Y::SMEM, st>>>(F, tw, kmax3);
  }
  // the stage's y-pass with tile width `tile` (0, or a width not offered: the default) and
  // radix plan variant `plan`; pr (inverse only): the pruned form PR = 1
  template <int INV, int PRUNE>
  static void y_stage(int tile, int plan, cx<T>* F, const cx<T>* tw, int kmax3, int planes, int fields,
                      cudaStream_t st, bool pr = false) {
    with_plan(plan, [&](auto v) {
      constexpr int V = decltype(v)::value;
      auto go = [&](auto t) {
        constexpr int TXO = decltype(t)::value;
        if constexpr (INV) {
          if (pr) return y_go<INV, PRUNE, TXO, V, 1>(F, tw, kmax3, planes, fields, st);
        }
        y_go<INV, PRUNE, TXO, V, 0>(F, tw, kmax3, planes, fields, st);
      };
      if constexpr (ISO && N <= BATCH_MAX_N) {
        if constexpr (ytile_ok(4)) if (tile == 4) return go(std::integral_constant<int, 4>{});
        if constexpr (ytile_ok(8)) if (tile == 8) return go(std::integral_constant<int, 8>{});
        if constexpr (ytile_ok(16)) if (tile == 16) return go(std::integral_constant<int, 16>{});
        if constexpr (ytile_ok(32)) if (tile == 32) return go(std::integral_constant<int, 32>{});
      }
      go(std::integral_constant<int, 0>{});
    });
  }

  static cudaError_t prepare() {
    cudaError_t e = cudaSuccess;
    tile_attr<4>(e);
    tile_attr<8>(e);
    tile_attr<16>(e);
    tile_attr<32>(e);
    ztile_attr<4>(e);
    ztile_attr<8>(e);
    ztile_attr<16>(e);
    ztile_attr<32>(e);
#define DNS_ATTR(kern, bytes) \
  if (e == cudaSuccess) e = smem_attr(kern, bytes)
    DNS_ATTR((k_xpass<T, N, XM_INV_CURL, NY, NZ>), G::XSMEM);
    DNS_ATTR((k_xpass<T, N, XM_STAGE, NY, NZ>), G::XSMEM_ST);
    DNS_ATTR((k_xpass<T, N, XM_STAGE2N, NY, NZ>), G::XSMEM_ST);
    DNS_ATTR((k_xpass<T, N, XM_RHS, NY, NZ>), G::XSMEM_ST);
    DNS_ATTR((k_xpass<T, N, XM_FWD_STORE, NY, NZ>), G::XSMEM);
    DNS_ATTR((k_xpass<T, N, XM_INV_PLAIN, NY, NZ>), G::XSMEM);
    DNS_ATTR((k_xpass<T, N, XM_INV_DIV, NY, NZ>), G::XSMEM);
    DNS_ATTR((k_ypass<T, N, 1, 0, 0, NY, NZ>), (YCfg<T, N, 1, 0, NY>::SMEM));
    DNS_ATTR((k_ypass<T, N, 1, 0, 0, NY, NZ, 0, 1>), (YCfg<T, N, 1, 0, NY>::SMEM));
    DNS_ATTR((k_ypass<T, N, 0, 1, 0, NY, NZ>), (YCfg<T, N, 0, 0, NY>::SMEM));
    DNS_ATTR((k_ypass<T, N, 0, 0, 0, NY, NZ>), (YCfg<T, N, 0, 0, NY>::SMEM));
    DNS_ATTR((k_zpass<T, N, ZM_CROSS, 0, NY, NZ>), G::ZSMEM);
    if constexpr (PLANS > 1) {
      DNS_ATTR((k_xpass<T, N, XM_INV_CURL, N, N, 1>), G::XSMEM);
      DNS_ATTR((k_xpass<T, N, XM_STAGE, N, N, 1>), G::XSMEM_ST);
      DNS_ATTR((k_xpass<T, N, XM_STAGE2N, N, N, 1>), G::XSMEM_ST);
      DNS_ATTR((k_xpass<T, N, XM_RHS, N, N, 1>), G::XSMEM_ST);
      DNS_ATTR((k_ypass<T, N, 1, 0, 0, N, N, 1>), (YCfg<T, N, 1, 0>::SMEM));
      DNS_ATTR((k_ypass<T, N, 1, 0, 0, N, N, 1, 1>), (YCfg<T, N, 1, 0>::SMEM));
      DNS_ATTR((k_ypass<T, N, 0, 1, 0, N, N, 1>), (YCfg<T, N, 0, 0>::SMEM));
      DNS_ATTR((k_zpass<T, N, ZM_CROSS, 0, N, N, 1>), G::ZSMEM);
    }
    if constexpr (ISO && ZCross<T, N>::enabled) DNS_ATTR((k_zcross<T, N>), G::ZSMEM);
    if constexpr (ISO && N == 512 && sizeof(T) == 4) DNS_ATTR((k_zcross16p<T, N>), Z16P<T>::SMEM);
    if constexpr (ISO && N == 1024 && sizeof(T) == 4) DNS_ATTR((k_zcross32p<T, N>), Z32P<T>::SMEM);
    if constexpr (ISO && N == 256 && sizeof(T) == 4) DNS_ATTR((k_zcross8q<T, N>), Z8Q<T>::SMEM);
    if constexpr (Z8_BOX) DNS_ATTR((k_zcross8q<T, N, NY, NZ>), Z8Q<T>::SMEM);
    DNS_ATTR((k_zpass<T, N, ZM_STORE, 0, NY, NZ>), G::ZSMEM);
    DNS_ATTR((k_zpass<T, N, ZM_LOAD, 0, NY, NZ>), G::ZSMEM);
    DNS_ATTR((k_zpass<T, N, ZM_MAXABS, 0, NY, NZ>), G::ZSMEM);
    if constexpr (BATCHED) {
      DNS_ATTR((k_ypass_b<T, N, 1, 0>), (YCfg<T, N, 1>::SMEM));
      DNS_ATTR((k_zpass_b<T, N, ZM_CROSS>), G::ZSMEM);
      DNS_ATTR((k_ypass_b<T, N, 0, 1>), (YCfg<T, N, 0>::SMEM));
      DNS_ATTR((k_xpass_b<T, N, XM_STAGE>), G::XSMEM_ST);
      DNS_ATTR((k_xpass_b<T, N, XM_STAGE2N>), G::XSMEM_ST);
      if constexpr (PLANS > 1) {
        DNS_ATTR((k_ypass_b<T, N, 1, 0, 0, 1>), (YCfg<T, N, 1>::SMEM));
        DNS_ATTR((k_zpass_b<T, N, ZM_CROSS, 0, 1>), G::ZSMEM);
        DNS_ATTR((k_ypass_b<T, N, 0, 1, 0, 1>), (YCfg<T, N, 0>::SMEM));
        DNS_ATTR((k_xpass_b<T, N, XM_STAGE, 1>), G::XSMEM_ST);
        DNS_ATTR((k_xpass_b<T, N, XM_STAGE2N, 1>), G::XSMEM_ST);
      }
    }
#undef DNS_ATTR
    return e;
  }

  static void z_cross(const PassArgs& a, cudaStream_t st) {
    if constexpr (Z8_BOX)
      k_zcross8q<T, N, NY, NZ><<<dim3(N / Z8Q<T>::TX, NY), 32 * Z8Q<T>::NW, Z8Q<T>::SMEM, st>>>(a);
    else if constexpr (!ISO)
      z_go<0>(a, st);
    else if constexpr (N == 512 && sizeof(T) == 4)
      k_zcross16p<T, N><<<num_sms(), 32 * Z16P<T>::NW, Z16P<T>::SMEM, st>>>(a);
    else if constexpr (N == 512)  // FP64: the generic z-pass, measured faster than a half-warp
      z_go<0>(a, st);             // radix-16 kernel (38.2 against 41.2 ms per launch)
    else if constexpr (N == 1024 && sizeof(T) == 4)
      k_zcross32p<T, N><<<num_sms(), 32 * Z32P<T>::NW, Z32P<T>::SMEM, st>>>(a);
    else if constexpr (N == 256 && sizeof(T) == 4)
      k_zcross8q<T, N><<<dim3(N / Z8Q<T>::TX, N), 32 * Z8Q<T>::NW, Z8Q<T>::SMEM, st>>>(a);
    else if constexpr (ZCross<T, N>::enabled)
      k_zcross<T, N><<<dim3(N / G::ZTX, N), 32 * ZCrossWarps<T, N>::value, G::ZSMEM, st>>>(a);
    else {
      with_plan(bit(a.plan, PLAN_Z), [&](auto v) {
        constexpr int V = decltype(v)::value;
        if constexpr (ztile_ok(4)) if (a.ztile == 4) return z_go<4, V>(a, st);
        if constexpr (ztile_ok(8)) if (a.ztile == 8) return z_go<8, V>(a, st);
        if constexpr (ztile_ok(16)) if (a.ztile == 16) return z_go<16, V>(a, st);
        if constexpr (ztile_ok(32)) if (a.ztile == 32) return z_go<32, V>(a, st);
        z_go<0, V>(a, st);
      });
    }
  }

  // shared memory of a stage-update launch: with the wide layout only the rows
  // the stage reads are allocated (3 in the first stage, 6 in the last, 9 in the
  // stages between), so the lighter stages keep more blocks per SM
  static size_t xsmem_stage(int stage, int last) {
    if constexpr (G::XPRE && G::XWIDE) {
      const int rows = stage == 0 ? 3 : (stage == last ? 6 : 9);
      return (size_t)(G::XST + rows * N) * sizeof(cx<T>);
    } else {
      return G::XSMEM_ST;
    }
  }

  static int kc_of(int kmax3) {
    int kc = (kmax3 + 2) / 3;
    return kc > M ? M : kc;
  }

  // blocks of an x-stage or x-inverse launch: every row, or with a pruned state only the
  // kc_z x (2R + 1) rows inside the 2/3 box (the kernel maps them, xpass_body; N <= 512)
  static int x_rows(const PassArgs& a) {
    return xpass_compact_ok<N>() && a.prune >= PRUNE_ROWS ? kc_of(k3z(a)) * (2 * xpass_kept_ky<NY>(k3y(a)) + 1)
                                                           : ROWS;
  }

  static cudaError_t x_inverse_curl(const PassArgs& a0, int from_stage, cudaStream_t st) {
    PassArgs a = a0;
    if (from_stage) a.U = a.US;
    with_plan(bit(a.plan, PLAN_X), [&](auto v) {
      k_xpass<T, N, XM_INV_CURL, NY, NZ, decltype(v)::value><<<x_rows(a), XP_THREADS, G::XSMEM, st>>>(f32args(a));
    });
    return cudaGetLastError();
  }

  // the stage's y-inverse of the 6 fields (a pruned state: the planes kz < kc only)
  static void y_inverse(const PassArgs& a, cudaStream_t st) {
    const bool pr = a.prune >= PRUNE_ROWS;
    y_stage<1, 0>(a.ytile[0], bit(a.plan, PLAN_YI), reinterpret_cast<cx<T>*>(a.W),
                  reinterpret_cast<const cx<T>*>(a.tw), k3y(a), pr ? kc_of(k3z(a)) : M, 6, st, pr);
  }

  static void rhs_front(const PassArgs& a, cudaStream_t st) {
    cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
    const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
    y_inverse(a, st);
    z_cross(a, st);
    y_stage<0, 1>(a.ytile[1], bit(a.plan, PLAN_YF), W, tw, k3y(a), kc_of(k3z(a)), 3, st);
  }

  // the x-stage launch of a stage, in the form of the stage's scheme
  static void x_stage(const PassArgs& a, cudaStream_t st) {
    with_plan(bit(a.plan, PLAN_X), [&](auto v) {
      constexpr int V = decltype(v)::value;
      if (a.lsrk)
        k_xpass<T, N, XM_STAGE2N, NY, NZ, V><<<x_rows(a), XP_THREADS, xsmem_stage(a.stage, a.last), st>>>(f32args(a));
      else
        k_xpass<T, N, XM_STAGE, NY, NZ, V><<<x_rows(a), XP_THREADS, xsmem_stage(a.stage, a.last), st>>>(f32args(a));
    });
  }

  static cudaError_t rk_stage(const PassArgs& a, cudaStream_t st) {
    rhs_front(a, st);
    x_stage(a, st);
    return cudaGetLastError();
  }

  static cudaError_t rk_stage_part(const PassArgs& a, int part, cudaStream_t st) {
    cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
    const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
    switch (part) {
      case 0: y_inverse(a, st); break;
      case 1: z_cross(a, st); break;
      case 2: y_stage<0, 1>(a.ytile[1], bit(a.plan, PLAN_YF), W, tw, k3y(a), kc_of(k3z(a)), 3, st); break;
      default: x_stage(a, st); break;
    }
    return cudaGetLastError();
  }

  // batched passes with tile width TXO (0: default) and plan variant V
  template <int INV, int PRUNE, int TXO, int V>
  static void yb_go(const BatchArgs& B, int count, int planes, int fields, cudaStream_t st) {
    using Y = YCfg<T, N, INV, TXO>;
    k_ypass_b<T, N, INV, PRUNE, TXO, V><<<dim3(N / Y::TX, planes, fields * count), Y::THREADS, Y::SMEM, st>>>(B, fields);
  }
  template <int INV, int PRUNE, int V>
  static void yb_stage(int tile, const BatchArgs& B, int count, int planes, int fields, cudaStream_t st) {
    if constexpr (ISO && N <= BATCH_MAX_N) {
      if constexpr (ytile_ok(4)) if (tile == 4) return yb_go<INV, PRUNE, 4, V>(B, count, planes, fields, st);
      if constexpr (ytile_ok(8)) if (tile == 8) return yb_go<INV, PRUNE, 8, V>(B, count, planes, fields, st);
      if constexpr (ytile_ok(16)) if (tile == 16) return yb_go<INV, PRUNE, 16, V>(B, count, planes, fields, st);
      if constexpr (ytile_ok(32)) if (tile == 32) return yb_go<INV, PRUNE, 32, V>(B, count, planes, fields, st);
    }
    yb_go<INV, PRUNE, 0, V>(B, count, planes, fields, st);
  }
  template <int TXO, int V>
  static void zb_go(const BatchArgs& B, int count, cudaStream_t st) {
    constexpr int TX = TXO > 0 ? TXO : G::ZTX;
    k_zpass_b<T, N, ZM_CROSS, TXO, V><<<dim3(N / TX, N, count), ZP_THREADS, G::zbytes(TX), st>>>(B);
  }
  template <int V>
  static void zb_stage(int tile, const BatchArgs& B, int count, cudaStream_t st) {
    if constexpr (ztile_ok(4)) if (tile == 4) return zb_go<4, V>(B, count, st);
    if constexpr (ztile_ok(8)) if (tile == 8) return zb_go<8, V>(B, count, st);
    if constexpr (ztile_ok(16)) if (tile == 16) return zb_go<16, V>(B, count, st);
    if constexpr (ztile_ok(32)) if (tile == 32) return zb_go<32, V>(B, count, st);
    zb_go<0, V>(B, count, st);
  }

  // one batched stage; the members share one radix plan (the ensemble groups them by it)
  static cudaError_t rk_stage_batch(const PassArgs* A, int count, int kmax3, cudaStream_t st) {
    if constexpr (BATCHED && N != 512 && N != 1024) {
      if (count < 1 || count > BATCH_MAX_COUNT) return cudaErrorInvalidValue;
      for (int i = 1; i < count; ++i)
        if (A[i].plan != A[0].plan) return cudaErrorInvalidValue;
      BatchArgs B;
      for (int i = 0; i < count; ++i) B.a[i] = f32args(A[i]);
      // the members' tile widths where they agree (a size class tuned together), else the defaults
      int yi = A[0].ytile[0], yf = A[0].ytile[1], zt = A[0].ztile;
      for (int i = 1; i < count; ++i) {
        if (A[i].ytile[0] != yi) yi = 0;
        if (A[i].ytile[1] != yf) yf = 0;
        if (A[i].ztile != zt) zt = 0;
      }
      const int plan = A[0].plan;
      with_plan(bit(plan, PLAN_YI), [&](auto v) { yb_stage<1, 0, decltype(v)::value>(yi, B, count, M, 6, st); });
      with_plan(bit(plan, PLAN_Z), [&](auto v) { zb_stage<decltype(v)::value>(zt, B, count, st); });
      with_plan(bit(plan, PLAN_YF),
                [&](auto v) { yb_stage<0, 1, decltype(v)::value>(yf, B, count, kc_of(kmax3), 3, st); });
      with_plan(bit(plan, PLAN_X), [&](auto v) {
        constexpr int V = decltype(v)::value;
        if (A[0].lsrk)
          k_xpass_b<T, N, XM_STAGE2N, V><<<dim3(M * N, count), XP_THREADS, xsmem_stage(A[0].stage, A[0].last), st>>>(B);
        else
          k_xpass_b<T, N, XM_STAGE, V><<<dim3(M * N, count), XP_THREADS, xsmem_stage(A[0].stage, A[0].last), st>>>(B);
      });
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }

  static cudaError_t rhs(const PassArgs& a, cudaStream_t st) {
    cudaError_t e = x_inverse_curl(a, 0, st);
    if (e != cudaSuccess) return e;
    rhs_front(a, st);
    PassArgs b = a;
    b.stage = 0;
    with_plan(bit(b.plan, PLAN_X), [&](auto v) {
      k_xpass<T, N, XM_RHS, NY, NZ, decltype(v)::value><<<ROWS, XP_THREADS, xsmem_stage(0, 3), st>>>(f32args(b));
    });
    return cudaGetLastError();
  }

  static cudaError_t forward3d(const PassArgs& a, cudaStream_t st) {
    using Y = YCfg<T, N, 0, 0, NY>;
    k_zpass<T, N, ZM_LOAD, 0, NY, NZ><<<dim3(N / G::ZTX, NY), ZP_THREADS, G::ZSMEM, st>>>(a);
    k_ypass<T, N, 0, 0, 0, NY, NZ><<<dim3(N / Y::TX, M, 3), Y::THREADS, Y::SMEM, st>>>(
        reinterpret_cast<cx<T>*>(a.U), reinterpret_cast<const cx<T>*>(a.tw), k3y(a));
    k_xpass<T, N, XM_FWD_STORE, NY, NZ><<<ROWS, XP_THREADS, G::XSMEM, st>>>(f32args(a));
    return cudaGetLastError();
  }

  static cudaError_t inverse3d(const PassArgs& a, cudaStream_t st) {
    using Y = YCfg<T, N, 1, 0, NY>;
    k_xpass<T, N, XM_INV_PLAIN, NY, NZ><<<ROWS, XP_THREADS, G::XSMEM, st>>>(f32args(a));
    k_ypass<T, N, 1, 0, 0, NY, NZ><<<dim3(N / Y::TX, M, 3), Y::THREADS, Y::SMEM, st>>>(
        reinterpret_cast<cx<T>*>(a.W), reinterpret_cast<const cx<T>*>(a.tw), k3y(a));
    k_zpass<T, N, ZM_STORE, 0, NY, NZ><<<dim3(N / G::ZTX, NY), ZP_THREADS, G::ZSMEM, st>>>(a);
    return cudaGetLastError();
  }

  static cudaError_t diag(const PassArgs& a, cudaStream_t st) {
    using Y = YCfg<T, N, 1, 0, NY>;
    k_diag<T, N, NY, NZ><<<DIAG_BLOCKS, DG_THREADS, 0, st>>>(a);
    k_diag_final<<<1, 32, 0, st>>>(a.partials, DIAG_BLOCKS);
    k_xpass<T, N, XM_INV_DIV, NY, NZ><<<ROWS, XP_THREADS, G::XSMEM, st>>>(f32args(a));
    k_ypass<T, N, 1, 0, 0, NY, NZ><<<dim3(N / Y::TX, M, 1), Y::THREADS, Y::SMEM, st>>>(
        reinterpret_cast<cx<T>*>(a.D), reinterpret_cast<const cx<T>*>(a.tw), k3y(a));
    cudaMemsetAsync(a.maxbits, 0, sizeof(unsigned long long), st);
    k_zpass<T, N, ZM_MAXABS, 0, NY, NZ><<<dim3(N / G::ZTX, NY), ZP_THREADS, G::ZSMEM, st>>>(a);
    return cudaGetLastError();
  }

  static const DnsOps* ops() {
    static const DnsOps o = {N,         sizeof(T) == 4 ? 0 : 1, sizeof(cx<T>), &prepare,   &x_inverse_curl,
                             &rk_stage, &rk_stage_part,        &rhs,          &forward3d, &inverse3d,
                             &diag,     BATCHED ? &rk_stage_batch : nullptr, &y_tiles, &z_tiles,
                             NY,        NZ,                    G::TW,         PLANS,      default_plan()};
    return &o;
  }
};

}  // namespace dns

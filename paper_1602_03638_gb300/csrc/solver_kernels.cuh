// Fused kernels of one RK4 right-hand-side evaluation and its stage update,
// templated on the precision T and the grid size N (N = 2^a or 3*2^a).
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

#include "dns_internal.h"
#include "fft_core.cuh"

namespace dns {

constexpr int XP_THREADS = 256;
constexpr int YP_THREADS = 256;
constexpr int ZP_THREADS = 256;
constexpr int DG_THREADS = 256;

constexpr int pow2_floor(int x) {
  int r = 1;
  while (r * 2 <= x) r *= 2;
  return r;
}
constexpr int pow2_part(int n) {
  int r = 1;
  while (n % (r * 2) == 0) r *= 2;
  return r;
}
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int odd_ld(int lines) { return (lines % 2) ? lines : lines + 1; }

template <typename T, int N>
struct Geometry {
  static constexpr int M = N / 2;
  static constexpr size_t FS = (size_t)M * N * N;  // complex values per field
  static constexpr int CB = (int)sizeof(cx<T>);
  // x-pass: XROWS rows (fixed kz, consecutive ky) per block, <= ~64 KB smem.
  static constexpr int XROWS = cmin(cmin(pow2_floor(cmax(1, (64 * 1024) / (6 * N * CB))), 16), pow2_part(N));
  static constexpr int XLD = odd_ld(6 * XROWS);
  static constexpr size_t XSMEM = (size_t)N * XLD * CB;
  // y-pass: YTX adjacent columns (128-byte rows).
  static constexpr int YTX = cmin(128 / CB, pow2_part(N));
  static constexpr int YLD = odd_ld(YTX);
  static constexpr size_t YSMEM = (size_t)N * YLD * CB;
  // z-pass: ZTX adjacent x at fixed y, 6 fields of M values each, <= ~112 KB.
  static constexpr int zfit(int t) { return (size_t)M * odd_ld(6 * t) * CB <= 112 * 1024 ? 1 : 0; }
  static constexpr int ztx() {
    int t = cmin(16, pow2_part(N));
    while (t > 1 && !zfit(t)) t /= 2;
    return t;
  }
  static constexpr int ZTX = ztx();
  static constexpr int ZLD = odd_ld(6 * ZTX);
  static constexpr size_t ZSMEM = (size_t)M * ZLD * CB;
};

__device__ __forceinline__ int kfreq(int i, int N) { return i < N / 2 ? i : i - N; }
__device__ __forceinline__ bool kept(int k, int kmax3) { return 3 * (k < 0 ? -k : k) < kmax3; }

enum XMode { XM_INV_CURL = 0, XM_STAGE = 1, XM_RHS = 2, XM_FWD_STORE = 3, XM_INV_PLAIN = 4, XM_INV_DIV = 5 };
enum ZMode { ZM_CROSS = 0, ZM_STORE = 1, ZM_LOAD = 2, ZM_MAXABS = 3 };

// Writes conj(u/N^3) and conj(i k x u / N^3) into the 6 lines of one mode
// (conjugated because the following x transform is an inverse one).
template <typename T, int R, int LD>
__device__ __forceinline__ void put_curl_lines(cx<T>* s, int j, int q, cx<T> u0, cx<T> u1, cx<T> u2,
                                               T kx, T ky, T kz, T sc) {
  u0 = scal(u0, sc);
  u1 = scal(u1, sc);
  u2 = scal(u2, sc);
  // omega_hat = i k x u_hat
  cx<T> w0 = mul_pi(mk(ky * u2.x - kz * u1.x, ky * u2.y - kz * u1.y));
  cx<T> w1 = mul_pi(mk(kz * u0.x - kx * u2.x, kz * u0.y - kx * u2.y));
  cx<T> w2 = mul_pi(mk(kx * u1.x - ky * u0.x, kx * u1.y - ky * u0.y));
  cx<T>* p = s + j * LD + q;
  p[0 * R] = conjg(u0);
  p[1 * R] = conjg(u1);
  p[2 * R] = conjg(u2);
  p[3 * R] = conjg(w0);
  p[4 * R] = conjg(w1);
  p[5 * R] = conjg(w2);
}

// ---------------------------------------------------------------------------
// x-pass: one block owns XROWS rows (kz fixed, consecutive ky) of length N.
// ---------------------------------------------------------------------------
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(XP_THREADS) k_xpass(PassArgs a) {
  using G = Geometry<T, N>;
  constexpr int R = G::XROWS;
  constexpr int LD = G::XLD;
  constexpr size_t FS = G::FS;
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
  cx<T>* U = reinterpret_cast<cx<T>*>(a.U);
  cx<T>* U1 = reinterpret_cast<cx<T>*>(a.U1);
  cx<T>* US = reinterpret_cast<cx<T>*>(a.US);
  cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
  const int row0 = blockIdx.x * R;  // row r = kz * N + ky
  const int kz = row0 / N;
  const T sc = (T)(1.0 / ((double)N * (double)N * (double)N));
  const T kzv = (T)kz;

  if constexpr (MODE == XM_STAGE || MODE == XM_RHS) {
    const bool kz_kept = 3 * kz < a.kmax3;
    if (kz_kept) {
      for (int e = threadIdx.x; e < 3 * R * N; e += XP_THREADS) {
        const int j = e % N, cq = e / N, q = cq % R, c = cq / R;
        const int ky = (row0 + q) % N;
        cx<T> v = mk((T)0, (T)0);
        if (kept(kfreq(ky, N), a.kmax3)) v = W[c * FS + (size_t)(row0 + q) * N + j];
        s[j * LD + c * R + q] = v;
      }
      __syncthreads();
      fft_lines<T, N, XP_THREADS, LD, N, ChunkLines<N, XP_THREADS, 3 * R>::value>(s, 3 * R, tw);
    }
    const T nu = (T)a.nu, cA = (T)a.cA, cB = (T)a.cB;
    const int stage = a.stage;
    const cx<T>* Sst = (stage == 0) ? U : US;
    for (int e = threadIdx.x; e < R * N; e += XP_THREADS) {
      const int j = e % N, q = e / N;
      const int r = row0 + q, ky = r % N;
      const int kxi = kfreq(j, N), kyi = kfreq(ky, N);
      const T kx = (T)kxi, kyv = (T)kyi;
      cx<T> n0 = mk((T)0, (T)0), n1 = n0, n2 = n0;
      if (kz_kept && kept(kxi, a.kmax3) && kept(kyi, a.kmax3)) {
        n0 = s[j * LD + 0 * R + q];
        n1 = s[j * LD + 1 * R + q];
        n2 = s[j * LD + 2 * R + q];
      }
      const T k2 = kx * kx + kyv * kyv + kzv * kzv;
      const T ik2 = k2 > (T)0 ? (T)1 / k2 : (T)0;
      // P = (k . N_hat) / |k|^2   (Eq. mod_pressure without the factor i)
      const cx<T> p = mk((kx * n0.x + kyv * n1.x + kzv * n2.x) * ik2, (kx * n0.y + kyv * n1.y + kzv * n2.y) * ik2);
      const size_t gi = (size_t)r * N + j;
      const cx<T> u0 = Sst[gi], u1 = Sst[FS + gi], u2 = Sst[2 * FS + gi];
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
        cx<T> v0, v1, v2;
        if (stage == 0) {
          U1[gi] = u0 + scal(d0, cA);
          U1[FS + gi] = u1 + scal(d1, cA);
          U1[2 * FS + gi] = u2 + scal(d2, cA);
          v0 = u0 + scal(d0, cB);
          v1 = u1 + scal(d1, cB);
          v2 = u2 + scal(d2, cB);
          US[gi] = v0;
          US[FS + gi] = v1;
          US[2 * FS + gi] = v2;
        } else if (stage < 3) {
          const cx<T> b0 = U[gi], b1 = U[FS + gi], b2 = U[2 * FS + gi];
          U1[gi] = U1[gi] + scal(d0, cA);
          U1[FS + gi] = U1[FS + gi] + scal(d1, cA);
          U1[2 * FS + gi] = U1[2 * FS + gi] + scal(d2, cA);
          v0 = b0 + scal(d0, cB);
          v1 = b1 + scal(d1, cB);
          v2 = b2 + scal(d2, cB);
          US[gi] = v0;
          US[FS + gi] = v1;
          US[2 * FS + gi] = v2;
        } else {
          v0 = U1[gi] + scal(d0, cA);
          v1 = U1[FS + gi] + scal(d1, cA);
          v2 = U1[2 * FS + gi] + scal(d2, cA);
          U[gi] = v0;
          U[FS + gi] = v1;
          U[2 * FS + gi] = v2;
        }
        put_curl_lines<T, R, LD>(s, j, q, v0, v1, v2, kx, kyv, kzv, sc);
      }
    }
    if constexpr (MODE == XM_STAGE) {
      __syncthreads();
      fft_lines<T, N, XP_THREADS, LD, N, ChunkLines<N, XP_THREADS, 6 * R>::value>(s, 6 * R, tw);
      for (int e = threadIdx.x; e < 6 * R * N; e += XP_THREADS) {
        const int j = e % N, fq = e / N, q = fq % R, f = fq / R;
        W[f * FS + (size_t)(row0 + q) * N + j] = conjg(s[j * LD + f * R + q]);
      }
    }
  } else if constexpr (MODE == XM_FWD_STORE) {
    for (int e = threadIdx.x; e < 3 * R * N; e += XP_THREADS) {
      const int j = e % N, cq = e / N, q = cq % R, c = cq / R;
      s[j * LD + c * R + q] = U[c * FS + (size_t)(row0 + q) * N + j];
    }
    __syncthreads();
    fft_lines<T, N, XP_THREADS, LD, N, ChunkLines<N, XP_THREADS, 3 * R>::value>(s, 3 * R, tw);
    for (int e = threadIdx.x; e < 3 * R * N; e += XP_THREADS) {
      const int j = e % N, cq = e / N, q = cq % R, c = cq / R;
      const int ky = (row0 + q) % N;
      cx<T> v = s[j * LD + c * R + q];
      if (j == N / 2 || ky == N / 2) v = mk((T)0, (T)0);  // Nyquist modes are not part of the state
      U[c * FS + (size_t)(row0 + q) * N + j] = v;
    }
  } else {
    // inverse x transform of u and omega (XM_INV_CURL), of u alone
    // (XM_INV_PLAIN) or of i k . u (XM_INV_DIV), all scaled by 1/N^3
    constexpr int NF = (MODE == XM_INV_CURL) ? 6 : (MODE == XM_INV_PLAIN ? 3 : 1);
    for (int e = threadIdx.x; e < R * N; e += XP_THREADS) {
      const int j = e % N, q = e / N;
      const int r = row0 + q, ky = r % N;
      const size_t gi = (size_t)r * N + j;
      const cx<T> u0 = U[gi], u1 = U[FS + gi], u2 = U[2 * FS + gi];
      const T kx = (T)kfreq(j, N), kyv = (T)kfreq(ky, N);
      if constexpr (MODE == XM_INV_CURL) {
        put_curl_lines<T, R, LD>(s, j, q, u0, u1, u2, kx, kyv, kzv, sc);
      } else if constexpr (MODE == XM_INV_PLAIN) {
        s[j * LD + 0 * R + q] = conjg(scal(u0, sc));
        s[j * LD + 1 * R + q] = conjg(scal(u1, sc));
        s[j * LD + 2 * R + q] = conjg(scal(u2, sc));
      } else {
        const cx<T> d = mul_pi(mk(kx * u0.x + kyv * u1.x + kzv * u2.x, kx * u0.y + kyv * u1.y + kzv * u2.y));
        s[j * LD + q] = conjg(scal(d, sc));
      }
    }
    __syncthreads();
    fft_lines<T, N, XP_THREADS, LD, N, ChunkLines<N, XP_THREADS, NF * R>::value>(s, NF * R, tw);
    cx<T>* dst = (MODE == XM_INV_DIV) ? reinterpret_cast<cx<T>*>(a.D) : W;
    for (int e = threadIdx.x; e < NF * R * N; e += XP_THREADS) {
      const int j = e % N, fq = e / N, q = fq % R, f = fq / R;
      dst[f * FS + (size_t)(row0 + q) * N + j] = conjg(s[j * LD + f * R + q]);
    }
  }
}

// ---------------------------------------------------------------------------
// y-pass: one block owns YTX adjacent columns (fixed field and kz) of length N.
// INV: conj-in/conj-out (inverse DFT). PRUNE: store only rows with |ky| < N/3.
// grid = (N / YTX, number of kz planes, number of fields)
// ---------------------------------------------------------------------------
template <typename T, int N, int INV, int PRUNE>
__global__ void __launch_bounds__(YP_THREADS) k_ypass(cx<T>* __restrict__ F, const cx<T>* __restrict__ tw, int kmax3) {
  using G = Geometry<T, N>;
  constexpr int TX = G::YTX;
  constexpr int LD = G::YLD;
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* base = F + blockIdx.z * G::FS + (size_t)blockIdx.y * N * N + blockIdx.x * TX;
  for (int e = threadIdx.x; e < TX * N; e += YP_THREADS) {
    const int x = e % TX, y = e / TX;
    const cx<T> v = base[(size_t)y * N + x];
    s[y * LD + x] = INV ? conjg(v) : v;
  }
  __syncthreads();
  fft_lines<T, N, YP_THREADS, LD, N, ChunkLines<N, YP_THREADS, TX>::value>(s, TX, tw);
  for (int e = threadIdx.x; e < TX * N; e += YP_THREADS) {
    const int x = e % TX, y = e / TX;
    if (PRUNE && !kept(kfreq(y, N), kmax3)) continue;
    const cx<T> v = s[y * LD + x];
    base[(size_t)y * N + x] = INV ? conjg(v) : v;
  }
}

// ---------------------------------------------------------------------------
// z-pass: one block owns ZTX adjacent x at fixed y; lines run along kz / z.
// Real transforms of length N use one complex DFT of length M = N/2 on
// z_n = x_{2n} + i x_{2n+1} with the usual pre/post-processing of the pairs
// (k, M-k); the imaginary part of the kz = 0 coefficient is ignored and the
// kz = N/2 coefficient is zero (it is not stored).
// ---------------------------------------------------------------------------
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(ZP_THREADS) k_zpass(PassArgs a) {
  using G = Geometry<T, N>;
  constexpr int M = G::M;
  constexpr int TX = G::ZTX;
  constexpr int LD = G::ZLD;
  constexpr size_t FS = G::FS;
  constexpr int NF = (MODE == ZM_CROSS) ? 6 : (MODE == ZM_MAXABS ? 1 : 3);
  extern __shared__ unsigned char smraw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smraw);
  const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
  const int x0 = blockIdx.x * TX;
  const int y = blockIdx.y;

  if constexpr (MODE == ZM_LOAD) {
    // physical lines (x0 + x, y, :) of the 3 components, packed in pairs
    const cx<T>* in = reinterpret_cast<const cx<T>*>(a.in);
    for (int e = threadIdx.x; e < 3 * TX * M; e += ZP_THREADS) {
      const int n = e % M, x = (e / M) % TX, c = e / (M * TX);
      s[n * LD + c * TX + x] = in[((size_t)(c * N + x0 + x) * N + y) * M + n];
    }
    __syncthreads();
  } else {
    const cx<T>* src = reinterpret_cast<const cx<T>*>(MODE == ZM_MAXABS ? a.D : a.W);
    for (int e = threadIdx.x; e < NF * TX * M; e += ZP_THREADS) {
      const int x = e % TX, k = (e / TX) % M, f = e / (TX * M);
      s[k * LD + f * TX + x] = src[f * FS + ((size_t)k * N + y) * N + x0 + x];
    }
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
        const cx<T> xk = s[k * LD + l], xm = s[(M - k) * LD + l];
        const cx<T> wk = ldro(tw + k);  // exp(-2 pi i k / N)
        const cx<T> A = xk + conjg(xm), B = xk - conjg(xm);
        const cx<T> zk = A + mul_pi(cmul(conjg(wk), B));
        s[k * LD + l] = conjg(zk);
        if (k != M - k) {
          // partner M-k: e^{+2 pi i (M-k)/N} = -wk
          const cx<T> A2 = xm + conjg(xk), B2 = xm - conjg(xk);
          const cx<T> zm = A2 - mul_pi(cmul(wk, B2));
          s[(M - k) * LD + l] = conjg(zm);
        }
      }
    }
    __syncthreads();
    fft_lines<T, M, ZP_THREADS, LD, N, ChunkLines<M, ZP_THREADS, NL>::value>(s, NL, tw);
    // now conj(s) = x_{2n} + i x_{2n+1} (physical values, unnormalised c2r)
  }

  if constexpr (MODE == ZM_CROSS) {
    for (int e = threadIdx.x; e < TX * M; e += ZP_THREADS) {
      const int x = e % TX, n = e / TX;
      cx<T>* p = s + n * LD + x;
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
    fft_lines<T, M, ZP_THREADS, LD, N, ChunkLines<M, ZP_THREADS, 3 * TX>::value>(s, 3 * TX, tw);
    // r2c post-processing: X_k = 1/2 [(Z_k + conj Z_{M-k}) - i e^{-2 pi i k/N} (Z_k - conj Z_{M-k})]
    cx<T>* dst = reinterpret_cast<cx<T>*>(MODE == ZM_CROSS ? a.W : a.U);
    int kc = M;
    if (MODE == ZM_CROSS) {
      kc = (a.kmax3 + 2) / 3;
      if (kc > M) kc = M;
    }
    for (int e = threadIdx.x; e < 3 * TX * kc; e += ZP_THREADS) {
      const int x = e % TX, k = (e / TX) % kc, c = e / (TX * kc);
      const int l = c * TX + x;
      const cx<T> zk = s[k * LD + l], zm = s[((M - k) % M) * LD + l];
      const cx<T> wk = ldro(tw + k);
      const cx<T> A = zk + conjg(zm), B = zk - conjg(zm);
      const cx<T> X = scal(A + mul_mi(cmul(wk, B)), (T)0.5);
      dst[c * FS + ((size_t)k * N + y) * N + x0 + x] = X;
    }
  } else if constexpr (MODE == ZM_STORE) {
    cx<T>* out = reinterpret_cast<cx<T>*>(a.out);
    for (int e = threadIdx.x; e < 3 * TX * M; e += ZP_THREADS) {
      const int n = e % M, x = (e / M) % TX, c = e / (M * TX);
      out[((size_t)(c * N + x0 + x) * N + y) * M + n] = conjg(s[n * LD + c * TX + x]);
    }
  } else if constexpr (MODE == ZM_MAXABS) {
    double m = 0.0;
    for (int e = threadIdx.x; e < TX * M; e += ZP_THREADS) {
      const int x = e % TX, n = e / TX;
      const cx<T> v = s[n * LD + x];
      const double ax = fabs((double)v.x), ay = fabs((double)v.y);
      m = fmax(m, fmax(ax, ay));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double red[ZP_THREADS / 32];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < ZP_THREADS / 32; ++w) m = fmax(m, red[w]);
      // non-negative doubles order like their bit patterns
      atomicMax(a.maxbits, (unsigned long long)__double_as_longlong(m));
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 spectral sums for the diagnostics (Parseval): per block
//   sum w|u|^2, sum w|omega|^2, sum w Re(conj(u).omega), count of non-finite,
// w = 1 at kz = 0 and 2 otherwise (half spectrum; kz = N/2 is zero).
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(DG_THREADS) k_diag(PassArgs a) {
  using G = Geometry<T, N>;
  constexpr size_t FS = G::FS;
  const cx<T>* U = reinterpret_cast<const cx<T>*>(a.U);
  double se = 0, sz = 0, sh = 0, bad = 0;
  for (size_t i = (size_t)blockIdx.x * DG_THREADS + threadIdx.x; i < FS; i += (size_t)gridDim.x * DG_THREADS) {
    const int kxi = (int)(i % N), kyi = (int)((i / N) % N), kzi = (int)(i / ((size_t)N * N));
    const double kx = kfreq(kxi, N), ky = kfreq(kyi, N), kz = kzi;
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
template <typename T, int N>
struct SolverImpl {
  using G = Geometry<T, N>;
  static constexpr int M = G::M;

  template <class K>
  static cudaError_t smem_attr(K k, size_t bytes) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }

  static cudaError_t prepare() {
    cudaError_t e = cudaSuccess;
#define DNS_ATTR(kern, bytes) \
  if (e == cudaSuccess) e = smem_attr(kern, bytes)
    DNS_ATTR((k_xpass<T, N, XM_INV_CURL>), G::XSMEM);
    DNS_ATTR((k_xpass<T, N, XM_STAGE>), G::XSMEM);
    DNS_ATTR((k_xpass<T, N, XM_RHS>), G::XSMEM);
    DNS_ATTR((k_xpass<T, N, XM_FWD_STORE>), G::XSMEM);
    DNS_ATTR((k_xpass<T, N, XM_INV_PLAIN>), G::XSMEM);
    DNS_ATTR((k_xpass<T, N, XM_INV_DIV>), G::XSMEM);
    DNS_ATTR((k_ypass<T, N, 1, 0>), G::YSMEM);
    DNS_ATTR((k_ypass<T, N, 0, 1>), G::YSMEM);
    DNS_ATTR((k_ypass<T, N, 0, 0>), G::YSMEM);
    DNS_ATTR((k_zpass<T, N, ZM_CROSS>), G::ZSMEM);
    DNS_ATTR((k_zpass<T, N, ZM_STORE>), G::ZSMEM);
    DNS_ATTR((k_zpass<T, N, ZM_LOAD>), G::ZSMEM);
    DNS_ATTR((k_zpass<T, N, ZM_MAXABS>), G::ZSMEM);
#undef DNS_ATTR
    return e;
  }

  static int kc_of(int kmax3) {
    int kc = (kmax3 + 2) / 3;
    return kc > M ? M : kc;
  }

  static cudaError_t x_inverse_curl(const PassArgs& a0, int from_stage, cudaStream_t st) {
    PassArgs a = a0;
    if (from_stage) a.U = a.US;
    k_xpass<T, N, XM_INV_CURL><<<M * N / G::XROWS, XP_THREADS, G::XSMEM, st>>>(a);
    return cudaGetLastError();
  }

  static void rhs_front(const PassArgs& a, cudaStream_t st) {
    cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
    const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
    k_ypass<T, N, 1, 0><<<dim3(N / G::YTX, M, 6), YP_THREADS, G::YSMEM, st>>>(W, tw, a.kmax3);
    k_zpass<T, N, ZM_CROSS><<<dim3(N / G::ZTX, N), ZP_THREADS, G::ZSMEM, st>>>(a);
    k_ypass<T, N, 0, 1><<<dim3(N / G::YTX, kc_of(a.kmax3), 3), YP_THREADS, G::YSMEM, st>>>(W, tw, a.kmax3);
  }

  static cudaError_t rk_stage(const PassArgs& a, cudaStream_t st) {
    rhs_front(a, st);
    k_xpass<T, N, XM_STAGE><<<M * N / G::XROWS, XP_THREADS, G::XSMEM, st>>>(a);
    return cudaGetLastError();
  }

  static cudaError_t rk_stage_part(const PassArgs& a, int part, cudaStream_t st) {
    cx<T>* W = reinterpret_cast<cx<T>*>(a.W);
    const cx<T>* tw = reinterpret_cast<const cx<T>*>(a.tw);
    switch (part) {
      case 0: k_ypass<T, N, 1, 0><<<dim3(N / G::YTX, M, 6), YP_THREADS, G::YSMEM, st>>>(W, tw, a.kmax3); break;
      case 1: k_zpass<T, N, ZM_CROSS><<<dim3(N / G::ZTX, N), ZP_THREADS, G::ZSMEM, st>>>(a); break;
      case 2: k_ypass<T, N, 0, 1><<<dim3(N / G::YTX, kc_of(a.kmax3), 3), YP_THREADS, G::YSMEM, st>>>(W, tw, a.kmax3); break;
      default: k_xpass<T, N, XM_STAGE><<<M * N / G::XROWS, XP_THREADS, G::XSMEM, st>>>(a); break;
    }
    return cudaGetLastError();
  }

  static cudaError_t rhs(const PassArgs& a, cudaStream_t st) {
    cudaError_t e = x_inverse_curl(a, 0, st);
    if (e != cudaSuccess) return e;
    rhs_front(a, st);
    PassArgs b = a;
    b.stage = 0;
    k_xpass<T, N, XM_RHS><<<M * N / G::XROWS, XP_THREADS, G::XSMEM, st>>>(b);
    return cudaGetLastError();
  }

  static cudaError_t forward3d(const PassArgs& a, cudaStream_t st) {
    k_zpass<T, N, ZM_LOAD><<<dim3(N / G::ZTX, N), ZP_THREADS, G::ZSMEM, st>>>(a);
    k_ypass<T, N, 0, 0><<<dim3(N / G::YTX, M, 3), YP_THREADS, G::YSMEM, st>>>(
        reinterpret_cast<cx<T>*>(a.U), reinterpret_cast<const cx<T>*>(a.tw), a.kmax3);
    k_xpass<T, N, XM_FWD_STORE><<<M * N / G::XROWS, XP_THREADS, G::XSMEM, st>>>(a);
    return cudaGetLastError();
  }

  static cudaError_t inverse3d(const PassArgs& a, cudaStream_t st) {
    k_xpass<T, N, XM_INV_PLAIN><<<M * N / G::XROWS, XP_THREADS, G::XSMEM, st>>>(a);
    k_ypass<T, N, 1, 0><<<dim3(N / G::YTX, M, 3), YP_THREADS, G::YSMEM, st>>>(
        reinterpret_cast<cx<T>*>(a.W), reinterpret_cast<const cx<T>*>(a.tw), a.kmax3);
    k_zpass<T, N, ZM_STORE><<<dim3(N / G::ZTX, N), ZP_THREADS, G::ZSMEM, st>>>(a);
    return cudaGetLastError();
  }

  static cudaError_t diag(const PassArgs& a, cudaStream_t st) {
    k_diag<T, N><<<DIAG_BLOCKS, DG_THREADS, 0, st>>>(a);
    k_diag_final<<<1, 32, 0, st>>>(a.partials, DIAG_BLOCKS);
    k_xpass<T, N, XM_INV_DIV><<<M * N / G::XROWS, XP_THREADS, G::XSMEM, st>>>(a);
    k_ypass<T, N, 1, 0><<<dim3(N / G::YTX, M, 1), YP_THREADS, G::YSMEM, st>>>(
        reinterpret_cast<cx<T>*>(a.D), reinterpret_cast<const cx<T>*>(a.tw), a.kmax3);
    cudaMemsetAsync(a.maxbits, 0, sizeof(unsigned long long), st);
    k_zpass<T, N, ZM_MAXABS><<<dim3(N / G::ZTX, N), ZP_THREADS, G::ZSMEM, st>>>(a);
    return cudaGetLastError();
  }

  static const DnsOps* ops() {
    static const DnsOps o = {N,        sizeof(T) == 4 ? 0 : 1, sizeof(cx<T>), &prepare,   &x_inverse_curl,
                             &rk_stage, &rk_stage_part,        &rhs,          &forward3d, &inverse3d,
                             &diag};
    return &o;
  }
};

}  // namespace dns

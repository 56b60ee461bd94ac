// Complex arithmetic, small-radix DFT butterflies and a shared-memory Stockham
// FFT engine for the batched 1D transforms of the pseudo-spectral solver.
//
// The 3D transforms of Eqs. fft/ifft (Sec. 2) are compositions of 1D
// transforms along z (real), y and x (complex). Every 1D transform here is a
// forward DFT  X_k = sum_j x_j exp(-2 pi i j k / L)  computed by a mixed-radix
// (16/8/4/2 and 3) Stockham autosort: natural order in and out, one pass per
// radix, each thread holding one radix-R butterfly in registers per pass.
// Inverse transforms use conj(DFT(conj(x))), folded into the callers' loads
// and stores. Twiddles come from a table of exp(-2 pi i t / TWN), t < TWN,
// generated on the host in FP64 (rounded to T for the FP32 form).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dns {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cx<T> conjg(cx<T> a) { return mk(a.x, -a.y); }
template <typename T>
__device__ __forceinline__ cx<T> scal(cx<T> a, T s) { return mk(a.x * s, a.y * s); }
// a * (-i)
template <typename T>
__device__ __forceinline__ cx<T> mul_mi(cx<T> a) { return mk(a.y, -a.x); }
// a * (+i)
template <typename T>
__device__ __forceinline__ cx<T> mul_pi(cx<T> a) { return mk(-a.y, a.x); }

// Read-only cached load of one complex value (twiddle tables).
__device__ __forceinline__ cx<float> ldro(const cx<float>* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mk(v.x, v.y);
}
__device__ __forceinline__ cx<double> ldro(const cx<double>* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mk(v.x, v.y);
}

// ---------------------------------------------------------------------------
// Forward DFT butterflies of size 2, 3, 4, 8, 16 (in place, natural order).
// Constants are the exact values cos/sin of pi/4, pi/8 and sqrt(3)/2.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void dft2(cx<T>* v) {
  cx<T> a = v[0];
  v[0] = a + v[1];
  v[1] = a - v[1];
}

template <typename T>
__device__ __forceinline__ void dft3(cx<T>* v) {
  const T h3 = (T)0.86602540378443864676;  // sqrt(3)/2
  cx<T> t = v[1] + v[2];
  cx<T> m = mk(v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y);
  cx<T> d = v[1] - v[2];
  cx<T> dd = mk(d.y * h3, -d.x * h3);  // (b - c) * (-i sqrt(3)/2)
  v[0] = v[0] + t;
  v[1] = m + dd;
  v[2] = m - dd;
}

template <typename T>
__device__ __forceinline__ void dft4(cx<T>* v) {
  cx<T> t0 = v[0] + v[2], t1 = v[0] - v[2];
  cx<T> t2 = v[1] + v[3], t3 = mul_mi(v[1] - v[3]);
  v[0] = t0 + t2;
  v[2] = t0 - t2;
  v[1] = t1 + t3;
  v[3] = t1 - t3;
}

template <typename T>
__device__ __forceinline__ void dft8(cx<T>* v) {
  const T h = (T)0.70710678118654752440;
  cx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e);
  dft4(o);
  o[1] = mk((o[1].x + o[1].y) * h, (o[1].y - o[1].x) * h);  // * exp(-i pi/4)
  o[2] = mul_mi(o[2]);                                     // * exp(-i pi/2)
  o[3] = mk((o[3].y - o[3].x) * h, -(o[3].x + o[3].y) * h); // * exp(-3i pi/4)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = e[k] + o[k];
    v[k + 4] = e[k] - o[k];
  }
}

template <typename T>
__device__ __forceinline__ void dft16(cx<T>* v) {
  const T c1 = (T)0.92387953251128675613;  // cos(pi/8)
  const T s1 = (T)0.38268343236508977173;  // sin(pi/8)
  const T h = (T)0.70710678118654752440;
  cx<T> e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    e[k] = v[2 * k];
    o[k] = v[2 * k + 1];
  }
  dft8(e);
  dft8(o);
  // o[k] *= exp(-i pi k / 8)
  o[1] = cmul(o[1], mk(c1, -s1));
  o[2] = mk((o[2].x + o[2].y) * h, (o[2].y - o[2].x) * h);
  o[3] = cmul(o[3], mk(s1, -c1));
  o[4] = mul_mi(o[4]);
  o[5] = cmul(o[5], mk(-s1, -c1));
  o[6] = mk((o[6].y - o[6].x) * h, -(o[6].x + o[6].y) * h);
  o[7] = cmul(o[7], mk(-c1, -s1));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = e[k] + o[k];
    v[k + 8] = e[k] - o[k];
  }
}

template <int R, typename T>
__device__ __forceinline__ void dft(cx<T>* v) {
  if constexpr (R == 2) dft2(v);
  else if constexpr (R == 3) dft3(v);
  else if constexpr (R == 4) dft4(v);
  else if constexpr (R == 8) dft8(v);
  else if constexpr (R == 16) dft16(v);
  else static_assert(R == 2, "unsupported radix");
}

// ---------------------------------------------------------------------------
// Radix schedule for a length L = 2^a * 3^b (b <= 1): the power-of-two part is
// split into ceil(a/4) passes of radix <= 16, as evenly as possible (larger
// radices first); a radix-3 pass comes last.
// ---------------------------------------------------------------------------
constexpr int ilog2c(int x) {
  int r = 0;
  while (x > 1) { x >>= 1; ++r; }
  return r;
}

template <int L>
struct FFTPlan {
  static constexpr int three = (L % 3 == 0) ? 1 : 0;
  static constexpr int p2 = three ? L / 3 : L;
  static constexpr int a = ilog2c(p2);
  static constexpr int np2 = (a + 3) / 4;
  static constexpr int npass = np2 + three;
  static_assert((1 << a) == p2 && (p2 % 3) != 0, "FFT length must be 2^a or 3*2^a");
  static constexpr int radix(int p) {
    if (p >= np2) return 3;
    int rem = a;
    for (int q = 0; q < p; ++q) rem -= (rem + (np2 - q) - 1) / (np2 - q);
    return 1 << ((rem + (np2 - p) - 1) / (np2 - p));
  }
  static constexpr int ns(int p) {
    int r = 1;
    for (int q = 0; q < p; ++q) r *= radix(q);
    return r;
  }
};

// One Stockham pass over NL lines (runtime count nl <= NL) of length L held in
// shared memory; element j of line l sits at s[j * LD + l]. Butterflies are
// assigned line-fastest so that neighbouring threads touch neighbouring words.
// All reads of a pass finish (barrier) before any thread writes.
template <typename T, int L, int NL, int THREADS, int LD, int TWN, int P>
__device__ __forceinline__ void fft_pass(cx<T>* __restrict__ s, int nl, const cx<T>* __restrict__ tw) {
  using PL = FFTPlan<L>;
  constexpr int R = PL::radix(P);
  constexpr int NS = PL::ns(P);
  constexpr int NB = NL * (L / R);
  constexpr int BPT = (NB + THREADS - 1) / THREADS;
  cx<T> v[BPT][R];
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = threadIdx.x + i * THREADS;
    const int l = b % NL, j = b / NL;
    if ((NB % THREADS == 0 || b < NB) && l < nl) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = s[(j + r * (L / R)) * LD + l];
      if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], ldro(tw + k * r * (TWN / (NS * R))));
      }
      dft<R>(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int b = threadIdx.x + i * THREADS;
    const int l = b % NL, j = b / NL;
    if ((NB % THREADS == 0 || b < NB) && l < nl) {
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) s[(base + r * NS) * LD + l] = v[i][r];
    }
  }
  __syncthreads();
  if constexpr (P + 1 < PL::npass) fft_pass<T, L, NL, THREADS, LD, TWN, P + 1>(s, nl, tw);
}

// Forward DFT of `lines` lines (elements at s[j*LD + l]), processed in chunks
// of at most CH lines so that each thread holds a bounded number of values.
// Caller must have synchronised after filling s; returns synchronised.
template <typename T, int L, int THREADS, int LD, int TWN, int CH>
__device__ __forceinline__ void fft_lines(cx<T>* __restrict__ s, int lines, const cx<T>* __restrict__ tw) {
  for (int l0 = 0; l0 < lines; l0 += CH) {
    const int nl = (lines - l0) < CH ? (lines - l0) : CH;
    fft_pass<T, L, CH, THREADS, LD, TWN, 0>(s + l0, nl, tw);
  }
}

// Lines per chunk so that each thread holds about 16 complex values per pass.
template <int L, int THREADS, int LINES>
struct ChunkLines {
  static constexpr int raw = (16 * THREADS) / L;
  static constexpr int c1 = raw < 1 ? 1 : raw;
  static constexpr int value = c1 > LINES ? LINES : c1;
};

}  // namespace dns

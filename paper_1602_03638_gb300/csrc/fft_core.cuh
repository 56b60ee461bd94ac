// Complex arithmetic, small-radix DFT butterflies and a shared-memory Stockham
// FFT engine for the batched 1D transforms of the pseudo-spectral solver.
//
// The 3D transforms of Eqs. fft/ifft (Sec. 2) are compositions of 1D
// transforms along z (real), y and x (complex). Every 1D transform here is a
// forward DFT  X_k = sum_j x_j exp(-2 pi i j k / L)  computed by one warp with
// a mixed-radix (8, then 16/4/2, then 3) Stockham autosort: natural order in
// and out, one pass per radix, each lane holding its butterflies in registers
// and exchanging through a shared-memory line between passes (warp barriers
// only). The first pass may read and the last pass may write global memory
// directly. Inverse transforms use conj(DFT(conj(x))), folded into the
// callers' loads and stores. Twiddles come from a table of
// exp(-2 pi i t / TWN), t < TWN, generated on the host in FP64 (rounded to T
// for the FP32 form).
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

// 32-point DFT in place: two 16-point DFTs of the even and odd elements
// combined with exp(-2 pi i k / 32) (exact constants).
template <typename T>
__device__ __forceinline__ void dft32(cx<T>* v) {
  constexpr double c32[16][2] = {
      {1.0, 0.0},
      {0.9807852804032304, -0.19509032201612825},
      {0.9238795325112867, -0.3826834323650898},
      {0.8314696123025452, -0.5555702330196022},
      {0.7071067811865476, -0.7071067811865475},
      {0.5555702330196023, -0.8314696123025452},
      {0.38268343236508984, -0.9238795325112867},
      {0.19509032201612833, -0.9807852804032304},
      {0.0, -1.0},
      {-0.1950903220161282, -0.9807852804032304},
      {-0.3826834323650897, -0.9238795325112867},
      {-0.555570233019602, -0.8314696123025455},
      {-0.7071067811865475, -0.7071067811865476},
      {-0.8314696123025453, -0.5555702330196022},
      {-0.9238795325112867, -0.3826834323650899},
      {-0.9807852804032304, -0.1950903220161286}};
  cx<T> e[16], o[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    e[k] = v[2 * k];
    o[k] = v[2 * k + 1];
  }
  dft16(e);
  dft16(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    cx<T> t;
    if (k == 0) t = o[0];
    else if (k == 8) t = mul_mi(o[8]);
    else t = cmul(o[k], mk((T)c32[k][0], (T)c32[k][1]));
    v[k] = e[k] + t;
    v[k + 16] = e[k] - t;
  }
}

template <int R, typename T>
__device__ __forceinline__ void dft(cx<T>* v) {
  if constexpr (R == 2) dft2(v);
  else if constexpr (R == 3) dft3(v);
  else if constexpr (R == 4) dft4(v);
  else if constexpr (R == 8) dft8(v);
  else if constexpr (R == 16) dft16(v);
  else if constexpr (R == 32) dft32(v);
  else static_assert(R == 2, "unsupported radix");
}

// Powers w^1..w^(R-1) of one twiddle w = exp(-2 pi i k / (NS R)) loaded from the
// FP64-generated table: one table load per butterfly instead of R-1 scattered
// loads, the rest formed by a multiplication tree at most 4 products deep
// (FP32 form; the FP64 form loads every power).
template <int R, typename T>
__device__ __forceinline__ void twiddle_powers(cx<T> w1, cx<T>* w) {
  w[1] = w1;
  if constexpr (R > 2) w[2] = cmul(w1, w1);
  if constexpr (R > 3) w[3] = cmul(w[2], w1);
  if constexpr (R > 4) {
    w[4] = cmul(w[2], w[2]);
    w[5] = cmul(w[4], w1);
    w[6] = cmul(w[3], w[3]);
    w[7] = cmul(w[4], w[3]);
  }
  if constexpr (R > 8) {
    w[8] = cmul(w[4], w[4]);
#pragma unroll
    for (int r = 9; r < R; ++r) w[r] = cmul(w[8], w[r - 8]);
  }
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, sm_80+): used to prefetch
// the next tile while the current one is transformed.
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// ---------------------------------------------------------------------------
// Shared-memory line layout: element p sits at padded position p + p/16. With
// this padding both the contiguous accesses (j + r*L/R over lanes j) and the
// stride-R Stockham stores of every pass used here touch each bank pair at
// most twice per warp (the minimum for 8-byte words).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int padp(int p) { return p + (p >> 4); }
__host__ __device__ constexpr int padded_len(int L) { return L + L / 16 + 1; }

constexpr int ilog2c(int x) {
  int r = 0;
  while (x > 1) { x >>= 1; ++r; }
  return r;
}

// Radix schedule of the warp FFT for L = 2^a or 3 * 2^a: radix-8 passes, the
// remaining factor 2 or 4 as one radix-16 or radix-4 pass, then radix 3.
template <int L>
struct WarpPlan {
  static constexpr int three = (L % 3 == 0) ? 1 : 0;
  static constexpr int p2 = three ? L / 3 : L;
  static constexpr int a = ilog2c(p2);
  static_assert((1 << a) == p2 && (p2 % 3) != 0, "FFT length must be 2^a or 3*2^a");
  static constexpr int n8 = a / 3, rem = a % 3;
  // list of power-of-two radices
  static constexpr int np2 = (rem == 0) ? n8 : (rem == 1 ? (n8 >= 1 ? n8 : 1) : n8 + 1);
  static constexpr int npass = np2 + three;
  static constexpr int radix(int p) {
    if (p >= np2) return 3;
    if (rem == 0) return 8;
    if (rem == 1) return (n8 == 0) ? 2 : (p == np2 - 1 ? 16 : 8);
    return p == np2 - 1 ? 4 : 8;
  }
  static constexpr int ns(int p) {
    int r = 1;
    for (int q = 0; q < p; ++q) r *= radix(q);
    return r;
  }
};

// Radix schedule of the shared-memory warp FFT (warp_fft). For 8-byte values
// and 512- or 1024-point lines the schedules (16, 16, 2) and (16, 16, 4) replace
// the radix-8 ones: with the padded line layout (element stride 1 or any odd
// stride) their reads and Stockham writes hit distinct banks in every pass,
// while the radix-8 schedules' second-pass writes conflict two-way, and they
// need slightly fewer operations per point. Other cases use WarpPlan.
template <int L, int CB>
struct SmemPlan : WarpPlan<L> {};
template <int L, int R0, int R1, int R2>
struct FixedPlan3 {
  static constexpr int npass = 3;
  static constexpr int radix(int p) { return p == 0 ? R0 : (p == 1 ? R1 : R2); }
  static constexpr int ns(int p) {
    int r = 1;
    for (int q = 0; q < p; ++q) r *= radix(q);
    return r;
  }
  static_assert(R0 * R1 * R2 == L, "plan covers the line");
};
template <>
struct SmemPlan<512, 8> : FixedPlan3<512, 16, 16, 2> {};
template <>
struct SmemPlan<1024, 8> : FixedPlan3<1024, 16, 16, 4> {};

// Alternative radix schedule (plan variant 1, offered to the tile tuner of the small
// grids): radix 3 first where L has the factor 3, then radix-4 passes, and one radix-8
// pass last when the power-of-two exponent is odd (radix 2 when it is 1). More passes
// of smaller radix than WarpPlan: more butterflies per pass (lanes busy), fewer
// registers, one more exchange through shared memory.
template <int L>
struct AltPlan {
  static constexpr int three = (L % 3 == 0) ? 1 : 0;
  static constexpr int p2 = three ? L / 3 : L;
  static constexpr int a = ilog2c(p2);
  static_assert((1 << a) == p2 && (p2 % 3) != 0 && a >= 1, "FFT length must be 2^a or 3*2^a");
  static constexpr int odd_r = (a % 2) ? (a == 1 ? 2 : 8) : 0;  // the last power-of-two radix
  static constexpr int n4 = (a % 2) ? (a == 1 ? 0 : (a - 3) / 2) : a / 2;
  static constexpr int npass = three + n4 + (odd_r ? 1 : 0);
  static constexpr int radix(int p) { return (three && p == 0) ? 3 : (p - three < n4 ? 4 : odd_r); }
  static constexpr int ns(int p) {
    int r = 1;
    for (int q = 0; q < p; ++q) r *= radix(q);
    return r;
  }
};

// The plan of variant V: 0 = the default schedule, 1 = AltPlan.
template <int L, int CB, int V>
struct SmemPlanV : SmemPlan<L, CB> {};
template <int L, int CB>
struct SmemPlanV<L, CB, 1> : AltPlan<L> {};
template <int L, int V>
struct LinePlanV : WarpPlan<L> {};
template <int L>
struct LinePlanV<L, 1> : AltPlan<L> {};

template <int L>
struct IsPow2 {
  static constexpr bool value = L > 0 && (L & (L - 1)) == 0;
};

// Access policies for the warp FFT. at(p) gives the address of position p;
// for power-of-two plans every pass touches positions base + d with
// padp(base + d) = padp(base) + padp(d), so off(d) is a compile-time offset.
template <typename T, int ES>
struct SLine {  // a line in shared memory at padded positions, element stride ES
  cx<T>* s;
  __device__ __forceinline__ cx<T>* at(int p) const { return s + padp(p) * ES; }
  static constexpr int off(int d) { return padp(d) * ES; }
  __device__ __forceinline__ cx<T> load(const cx<T>* q) const { return *q; }
  __device__ __forceinline__ void store(cx<T>* q, int, cx<T> v) const { *q = v; }
};
template <typename T, int ES>
struct SLineConj {  // shared-memory line read conjugated (inverse DFT of staged data)
  cx<T>* s;
  __device__ __forceinline__ cx<T>* at(int p) const { return s + padp(p) * ES; }
  static constexpr int off(int d) { return padp(d) * ES; }
  __device__ __forceinline__ cx<T> load(const cx<T>* q) const { return conjg(*q); }
};
template <typename T>
struct SRow {  // unpadded contiguous line in shared memory (read only)
  const cx<T>* s;
  __device__ __forceinline__ const cx<T>* at(int p) const { return s + p; }
  static constexpr int off(int d) { return d; }
  __device__ __forceinline__ cx<T> load(const cx<T>* q) const { return *q; }
};
template <typename T, bool CONJ>
struct GLoad {  // contiguous line in global memory
  const cx<T>* g;
  __device__ __forceinline__ const cx<T>* at(int p) const { return g + p; }
  static constexpr int off(int d) { return d; }
  __device__ __forceinline__ cx<T> load(const cx<T>* q) const {
    const cx<T> v = *q;
    return CONJ ? conjg(v) : v;
  }
};
template <typename T, bool CONJ>
struct GStore {
  cx<T>* g;
  __device__ __forceinline__ cx<T>* at(int p) const { return g + p; }
  static constexpr int off(int d) { return d; }
  __device__ __forceinline__ void store(cx<T>* q, int, cx<T> v) const { *q = CONJ ? conjg(v) : v; }
};

template <typename T, int L, int TWN, int P, int V, class Src, class Work, class Dst>
__device__ __forceinline__ void warp_fft_pass(const Src& src, const Work& work, const Dst& dst,
                                              const cx<T>* __restrict__ tw, int lane) {
  using PL = SmemPlanV<L, (int)sizeof(cx<T>), V>;
  constexpr int R = PL::radix(P);
  constexpr int NS = PL::ns(P);
  constexpr int NB = L / R;
  constexpr int BPL = (NB + 31) / 32;
  constexpr bool FIRST = (P == 0);
  constexpr bool LAST = (P + 1 == PL::npass);
  constexpr bool FAST = IsPow2<L>::value;
  constexpr int TWC = TWN / (NS * R);
  cx<T> v[BPL][R];
#pragma unroll
  for (int b = 0; b < BPL; ++b) {
    const int j = lane + 32 * b;
    if (NB % 32 == 0 || j < NB) {
      if constexpr (FIRST) {
        if constexpr (FAST) {
          const auto q = src.at(j);
#pragma unroll
          for (int r = 0; r < R; ++r) v[b][r] = src.load(q + Src::off(r * NB));
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) v[b][r] = src.load(src.at(j + r * NB));
        }
      } else {
        if constexpr (FAST) {
          const auto q = work.at(j);
#pragma unroll
          for (int r = 0; r < R; ++r) v[b][r] = work.load(q + Work::off(r * NB));
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) v[b][r] = work.load(work.at(j + r * NB));
        }
      }
      if constexpr (NS > 1) {
        if constexpr (sizeof(T) == 4) {
          cx<T> w[R];
          twiddle_powers<R>(ldro(tw + (j % NS) * TWC), w);
#pragma unroll
          for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
        } else {  // FP64 multiplies are scarcer than loads: read every power
          const int kc = (j % NS) * TWC;
#pragma unroll
          for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], ldro(tw + r * kc));
        }
      }
      dft<R>(v[b]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int b = 0; b < BPL; ++b) {
    const int j = lane + 32 * b;
    if (NB % 32 == 0 || j < NB) {
      const int base = (j / NS) * NS * R + (j % NS);
      if constexpr (LAST) {
        if constexpr (FAST) {
          const auto q = dst.at(base);
#pragma unroll
          for (int r = 0; r < R; ++r) dst.store(q + Dst::off(r * NS), base + r * NS, v[b][r]);
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) dst.store(dst.at(base + r * NS), base + r * NS, v[b][r]);
        }
      } else {
        if constexpr (FAST) {
          const auto q = work.at(base);
#pragma unroll
          for (int r = 0; r < R; ++r) work.store(q + Work::off(r * NS), base + r * NS, v[b][r]);
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) work.store(work.at(base + r * NS), base + r * NS, v[b][r]);
        }
      }
    }
  }
  __syncwarp();
  if constexpr (!LAST) warp_fft_pass<T, L, TWN, P + 1, V>(src, work, dst, tw, lane);
}

// Forward DFT of one line of length L by one warp: reads through `src`, uses
// the shared-memory line `work` between passes, writes through `dst` (which may
// alias `work` or `src`: every pass reads all its values before writing).
// V: the radix plan variant (SmemPlanV).
template <typename T, int L, int TWN, int V = 0, class Src, class Work, class Dst>
__device__ __forceinline__ void warp_fft(const Src& src, const Work& work, const Dst& dst,
                                         const cx<T>* __restrict__ tw, int lane) {
  warp_fft_pass<T, L, TWN, 0, V>(src, work, dst, tw, lane);
}

// ---------------------------------------------------------------------------
// Several short lines per warp: G lines at s0 + g (g < G), element p of every
// line at padded position padp(p) * LD, transformed in place. The butterflies
// of all G lines of a pass are spread over the lanes (virtual butterfly
// g * NB + j), so short lines whose passes have fewer butterflies than lanes
// still keep the warp busy. Same radix plan and twiddles as warp_fft.
// ---------------------------------------------------------------------------
template <int L, int V = 0>
struct LinesPerWarp {  // largest power of two G with G * (butterflies of pass 0) <= 32, at most 16
  static constexpr int nb0 = L / LinePlanV<L, V>::radix(0);
  static constexpr int value = nb0 >= 32 ? 1 : (nb0 >= 16 ? 2 : (nb0 >= 8 ? 4 : (nb0 >= 4 ? 8 : 16)));
};

template <typename T, int L, int TWN, int G, int LD, int P, int V>
__device__ __forceinline__ void warp_fft_lines_pass(cx<T>* s0, const cx<T>* __restrict__ tw, int lane) {
  using PL = LinePlanV<L, V>;
  constexpr int R = PL::radix(P);
  constexpr int NS = PL::ns(P);
  constexpr int NB = L / R;
  constexpr int TOT = G * NB;
  constexpr int BPL = (TOT + 31) / 32;
  constexpr bool LAST = (P + 1 == PL::npass);
  constexpr int TWC = TWN / (NS * R);
  cx<T> v[BPL][R];
#pragma unroll
  for (int b = 0; b < BPL; ++b) {
    const int vj = lane + 32 * b;
    if (TOT % 32 == 0 || vj < TOT) {
      const int g = vj / NB, j = vj % NB;
      const cx<T>* ln = s0 + g;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = ln[padp(j + r * NB) * LD];
      if constexpr (NS > 1) {
        if constexpr (sizeof(T) == 4) {
          cx<T> w[R];
          twiddle_powers<R>(ldro(tw + (j % NS) * TWC), w);
#pragma unroll
          for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
        } else {
          const int kc = (j % NS) * TWC;
#pragma unroll
          for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], ldro(tw + r * kc));
        }
      }
      dft<R>(v[b]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int b = 0; b < BPL; ++b) {
    const int vj = lane + 32 * b;
    if (TOT % 32 == 0 || vj < TOT) {
      const int g = vj / NB, j = vj % NB;
      cx<T>* ln = s0 + g;
      const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) ln[padp(base + r * NS) * LD] = v[b][r];
    }
  }
  __syncwarp();
  if constexpr (!LAST) warp_fft_lines_pass<T, L, TWN, G, LD, P + 1, V>(s0, tw, lane);
}

// Forward DFT, in place, of the G lines s0 + g (see above) by one warp (V: plan variant).
template <typename T, int L, int TWN, int G, int LD, int V = 0>
__device__ __forceinline__ void warp_fft_lines(cx<T>* s0, const cx<T>* __restrict__ tw, int lane) {
  warp_fft_lines_pass<T, L, TWN, G, LD, 0, V>(s0, tw, lane);
}

// ---------------------------------------------------------------------------
// Register-resident warp FFT ("canonical" layout): lane l holds positions
// l + 32 m, m < L/32, in v[m]. Every pass reads its butterfly inputs from the
// lane's own registers (positions j + r L/R with j = l + 32 b); the Stockham
// outputs go through the shared-memory line `ln` (padded positions, element
// stride es) and are read back canonically; the last pass's outputs are
// already canonical and stay in registers. Needs L/R >= 32 in every pass.
// ---------------------------------------------------------------------------
template <int L>
struct CanonPlan {
  static constexpr int npass = (L == 128) ? 4 : WarpPlan<L>::npass;
  static constexpr int radix(int p) { return (L == 128) ? (p < 3 ? 4 : 2) : WarpPlan<L>::radix(p); }
  static constexpr int ns(int p) {
    int r = 1;
    for (int q = 0; q < p; ++q) r *= radix(q);
    return r;
  }
  static constexpr bool valid() {
    if (L % 32) return false;
    for (int p = 0; p < npass; ++p)
      if ((L / radix(p)) % 32) return false;
    return true;
  }
};

// Per-lane twiddle bases of the canonical FFT, loaded once per kernel: for
// every pass P >= 1 and butterfly slot b, w1 = exp(-2 pi i ((l + 32 b) mod NS) / (NS R)).
template <typename T, int L, int TWN>
struct CanonTw {
  using PL = CanonPlan<L>;
  static constexpr int off(int P) {
    int o = 0;
    for (int q = 1; q < P; ++q) o += (L / PL::radix(q)) / 32;
    return o;
  }
  static constexpr int count() { return off(PL::npass) > 0 ? off(PL::npass) : 1; }
  cx<T> w[count()];
  __device__ __forceinline__ void load(const cx<T>* __restrict__ tw, int lane) {
    load_pass<1>(tw, lane);
  }
  template <int P>
  __device__ __forceinline__ void load_pass(const cx<T>* __restrict__ tw, int lane) {
    if constexpr (P < PL::npass) {
      constexpr int R = PL::radix(P), NS = PL::ns(P), BPL = (L / R) / 32, TWC = TWN / (NS * R);
#pragma unroll
      for (int b = 0; b < BPL; ++b) w[off(P) + b] = ldro(tw + ((lane + 32 * b) % NS) * TWC);
      load_pass<P + 1>(tw, lane);
    }
  }
};

template <typename T, int L, int TWN, int ES, int P>
__device__ __forceinline__ void warp_fft_canon_pass(cx<T> (&v)[L / 32], cx<T>* ln, const CanonTw<T, L, TWN>& ctw,
                                                    const cx<T>* __restrict__ tw, int lane) {
  using PL = CanonPlan<L>;
  constexpr int R = PL::radix(P);
  constexpr int NS = PL::ns(P);
  constexpr int NB = L / R;
  constexpr int BPL = NB / 32;
  constexpr bool LAST = (P + 1 == PL::npass);
  constexpr int TWC = TWN / (NS * R);
  static_assert(NB % 32 == 0, "canonical warp FFT needs L/R >= 32");
  static_assert(IsPow2<L>::value, "canonical warp FFT needs a power-of-two length");
  cx<T> u[BPL][R];
#pragma unroll
  for (int b = 0; b < BPL; ++b) {
#pragma unroll
    for (int r = 0; r < R; ++r) u[b][r] = v[b + r * BPL];
    if constexpr (NS > 1) {
      if constexpr (sizeof(T) == 4) {
        cx<T> w[R];
        twiddle_powers<R>(ctw.w[CanonTw<T, L, TWN>::off(P) + b], w);
#pragma unroll
        for (int r = 1; r < R; ++r) u[b][r] = cmul(u[b][r], w[r]);
      } else {
        const int kc = ((lane + 32 * b) % NS) * TWC;
#pragma unroll
        for (int r = 1; r < R; ++r) u[b][r] = cmul(u[b][r], ldro(tw + r * kc));
      }
    }
    dft<R>(u[b]);
  }
  if constexpr (LAST) {
    // outputs j + r NS with NS = NB: canonical index b + r BPL
#pragma unroll
    for (int b = 0; b < BPL; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) v[b + r * BPL] = u[b][r];
  } else {
#pragma unroll
    for (int b = 0; b < BPL; ++b) {
      const int j = lane + 32 * b;
      cx<T>* q = ln + padp((j / NS) * NS * R + (j % NS)) * ES;
#pragma unroll
      for (int r = 0; r < R; ++r) q[padp(r * NS) * ES] = u[b][r];
    }
    __syncwarp();
    const cx<T>* rb = ln + padp(lane) * ES;
#pragma unroll
    for (int m = 0; m < L / 32; ++m) v[m] = rb[34 * m * ES];
    __syncwarp();
    warp_fft_canon_pass<T, L, TWN, ES, P + 1>(v, ln, ctw, tw, lane);
  }
}

// Forward DFT of the canonical register array v (length L) by one warp, using
// the shared-memory line ln (L padded positions, element stride ES) for the
// exchanges. The caller must have finished reading ln (and __syncwarp'ed).
template <typename T, int L, int TWN, int ES>
__device__ __forceinline__ void warp_fft_canon(cx<T> (&v)[L / 32], cx<T>* ln, const CanonTw<T, L, TWN>& ctw,
                                               const cx<T>* __restrict__ tw, int lane) {
  warp_fft_canon_pass<T, L, TWN, ES, 0>(v, ln, ctw, tw, lane);
}

}  // namespace dns

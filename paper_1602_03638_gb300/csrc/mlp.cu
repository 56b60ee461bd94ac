// Pointwise subgrid-stress network 10 -> 64 (SiLU) -> 64 (SiLU) -> 6 on BF16
// tensor cores with FP32 accumulation: inference on the 5th-generation tensor
// cores (tcgen05.mma, accumulators in TMEM, k_mlp_tc), training (forward +
// backward with the weight-gradient products also on the tensor cores, WMMA
// m16n16k16 fragments, k_mlp<1>) and Adam on FP32 master weights.
//
// Parameter vector (floats), in this order:
//   in_shift[10] in_scale[10] W1[10][64] b1[64] W2[64][64] b2[64] W3[64][6]
//   b3[6] out_scale[6] out_shift[6]                                  (5286 values)
// Inputs are standardised as (x - in_shift) * in_scale; the network output y
// is the standardised stress, tau = y * out_scale + out_shift. The training
// loss is the mean over points and components of (y - (t - out_shift) /
// out_scale)^2. Feature and stress arrays are planar: X[f * P + p], T[c * P + p].
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/dns.h"
#include "dns_internal.h"

namespace dns {
void set_error_message(const char* msg);
}

using namespace nvcuda;

namespace {

constexpr int NIN = 10, NH = 64, NOUT = 6;
constexpr int O_INSH = 0, O_INSC = 10, O_W1 = 20, O_B1 = 660, O_W2 = 724, O_B2 = 4820, O_W3 = 4884, O_B3 = 5268,
              O_OUTSC = 5274, O_OUTSH = 5280, NPARAM = 5286;
constexpr int TRAIN_BEGIN = O_W1, TRAIN_END = O_OUTSC;  // trainable range [W1 .. b3]
constexpr int WARPS = 4, THREADS = 32 * WARPS;
// packed BF16 weights: W1p[16][64] (rows >= 10 zero), W2[64][64], W3p[64][16] (cols >= 6 zero)
constexpr int PW1 = 0, PW2 = 16 * 64, PW3 = PW2 + 64 * 64, NPACK = PW3 + 64 * 16;

typedef __nv_bfloat16 bf;

// per-warp shared-memory work area (bytes, all offsets multiples of 32)
constexpr int A0_B = 16 * 16 * 2, Z1_B = 16 * 64 * 4, H_B = 16 * 64 * 2, Y_B = 16 * 16 * 4, DY_B = 16 * 16 * 2,
              G_B = 16 * 64 * 4, T_B = 16 * 16 * 4;
constexpr int OFF_A0 = 0, OFF_Z1 = OFF_A0 + A0_B, OFF_H1 = OFF_Z1 + Z1_B, OFF_Z2 = OFF_H1 + H_B, OFF_H2 = OFF_Z2 + Z1_B,
              OFF_Y = OFF_H2 + H_B, OFF_DY = OFF_Y + Y_B, OFF_G = OFF_DY + DY_B, OFF_DZ2 = OFF_G + G_B,
              OFF_DZ1 = OFF_DZ2 + H_B, OFF_T = OFF_DZ1 + H_B, WARP_B = OFF_T + T_B;
// block area: packed weights, then FP32 gradient accumulators (trainable range) and the loss
constexpr int BLK_W_B = NPACK * 2, BLK_G = TRAIN_END - TRAIN_BEGIN;
constexpr int SMEM_B = BLK_W_B + WARPS * WARP_B + (BLK_G + 8) * 4;


// SiLU and its derivative with the fast exponential and division intrinsics (their
// relative error, ~1e-6, is far below the BF16 rounding the activations then take)
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = __fdividef(1.f, 1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

__global__ void k_pack(const float* __restrict__ p, bf* __restrict__ w) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < NPACK; i += blockDim.x * gridDim.x) {
    float v = 0.f;
    if (i < PW2) {
      const int k = i / 64, n = i % 64;
      v = k < NIN ? p[O_W1 + k * 64 + n] : 0.f;
    } else if (i < PW3) {
      v = p[O_W2 + (i - PW2)];
    } else {
      const int k = (i - PW3) / 16, n = (i - PW3) % 16;
      v = n < NOUT ? p[O_W3 + k * NOUT + n] : 0.f;
    }
    w[i] = __float2bfloat16(v);
  }
}

typedef wmma::fragment<wmma::matrix_a, 16, 16, 16, bf, wmma::row_major> FragA;
typedef wmma::fragment<wmma::matrix_a, 16, 16, 16, bf, wmma::col_major> FragAT;
typedef wmma::fragment<wmma::matrix_b, 16, 16, 16, bf, wmma::row_major> FragB;
typedef wmma::fragment<wmma::matrix_b, 16, 16, 16, bf, wmma::col_major> FragBT;
typedef wmma::fragment<wmma::accumulator, 16, 16, 16, float> FragC;

// Adds a 16x16 FP32 tile (row-major in `tile`) into acc[(r0 + r) * ld + c0 + c] (shared atomics).
__device__ __forceinline__ void add_tile(float* acc, int ld, int r0, int c0, int rmax, int cmax, const float* tile,
                                         int lane) {
  for (int e = lane; e < 256; e += 32) {
    const int r = e >> 4, c = e & 15;
    if (r0 + r < rmax && c0 + c < cmax) atomicAdd(&acc[(r0 + r) * ld + c0 + c], tile[e]);
  }
}

// TRAIN = 0: Y = network(X). TRAIN = 1: accumulate the loss and the gradients
// of the trainable parameters into gsum (global, FP32) for targets T.
template <int TRAIN>
__global__ void __launch_bounds__(THREADS) k_mlp(const float* __restrict__ prm, const bf* __restrict__ wpack,
                                                  const float* __restrict__ X, int P, float* __restrict__ Y,
                                                  const float* __restrict__ T, float* __restrict__ gsum) {
  extern __shared__ __align__(128) unsigned char sm[];
  bf* sw = reinterpret_cast<bf*>(sm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wb = sm + BLK_W_B + warp * WARP_B;
  bf* A0 = reinterpret_cast<bf*>(wb + OFF_A0);
  float* Z1 = reinterpret_cast<float*>(wb + OFF_Z1);
  bf* H1 = reinterpret_cast<bf*>(wb + OFF_H1);
  float* Z2 = reinterpret_cast<float*>(wb + OFF_Z2);
  bf* H2 = reinterpret_cast<bf*>(wb + OFF_H2);
  float* Yt = reinterpret_cast<float*>(wb + OFF_Y);
  bf* DY = reinterpret_cast<bf*>(wb + OFF_DY);
  float* G = reinterpret_cast<float*>(wb + OFF_G);
  bf* DZ2 = reinterpret_cast<bf*>(wb + OFF_DZ2);
  bf* DZ1 = reinterpret_cast<bf*>(wb + OFF_DZ1);
  float* TT = reinterpret_cast<float*>(wb + OFF_T);
  float* acc = reinterpret_cast<float*>(sm + BLK_W_B + WARPS * WARP_B);  // [BLK_G] + loss

  static_assert(NPACK % 8 == 0, "16-byte weight staging");
  for (int i = threadIdx.x; i < NPACK / 8; i += THREADS)
    reinterpret_cast<uint4*>(sw)[i] = reinterpret_cast<const uint4*>(wpack)[i];
  if (TRAIN)
    for (int i = threadIdx.x; i < BLK_G + 8; i += THREADS) acc[i] = 0.f;
  __syncthreads();
  const bf* W1p = sw + PW1;
  const bf* W2s = sw + PW2;
  const bf* W3p = sw + PW3;
  float* gW1 = acc + (O_W1 - TRAIN_BEGIN);
  float* gb1 = acc + (O_B1 - TRAIN_BEGIN);
  float* gW2 = acc + (O_W2 - TRAIN_BEGIN);
  float* gb2 = acc + (O_B2 - TRAIN_BEGIN);
  float* gW3 = acc + (O_W3 - TRAIN_BEGIN);
  float* gb3 = acc + (O_B3 - TRAIN_BEGIN);
  float* gloss = acc + BLK_G;

  const int ntiles = (P + 15) / 16;
  for (int tile = blockIdx.x * WARPS + warp; tile < ntiles; tile += gridDim.x * WARPS) {
    const int p0 = tile * 16;
    // standardised inputs, BF16, features 10..15 zero
    for (int e = lane; e < 256; e += 32) {
      const int pt = e & 15, f = e >> 4;
      float v = 0.f;
      if (f < NIN && p0 + pt < P) v = (X[(size_t)f * P + p0 + pt] - prm[O_INSH + f]) * prm[O_INSC + f];
      A0[pt * 16 + f] = __float2bfloat16(v);
    }
    __syncwarp();
    FragA fa;
    FragB fb;
    FragC fc;
    // layer 1: Z1 = A0 W1p (16 x 64)
    wmma::load_matrix_sync(fa, A0, 16);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      wmma::fill_fragment(fc, 0.f);
      wmma::load_matrix_sync(fb, W1p + nt * 16, 64);
      wmma::mma_sync(fc, fa, fb, fc);
      wmma::store_matrix_sync(Z1 + nt * 16, fc, 64, wmma::mem_row_major);
    }
    __syncwarp();
    for (int e = lane; e < 1024; e += 32) {
      const float z = Z1[e] + prm[O_B1 + (e & 63)];
      if (TRAIN) Z1[e] = z;  // the backward pass reads the pre-activation
      H1[e] = __float2bfloat16(silu(z));
    }
    __syncwarp();
    // layer 2: Z2 = H1 W2 (16 x 64)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      wmma::fill_fragment(fc, 0.f);
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        wmma::load_matrix_sync(fa, H1 + kt * 16, 64);
        wmma::load_matrix_sync(fb, W2s + kt * 16 * 64 + nt * 16, 64);
        wmma::mma_sync(fc, fa, fb, fc);
      }
      wmma::store_matrix_sync(Z2 + nt * 16, fc, 64, wmma::mem_row_major);
    }
    __syncwarp();
    for (int e = lane; e < 1024; e += 32) {
      const float z = Z2[e] + prm[O_B2 + (e & 63)];
      if (TRAIN) Z2[e] = z;
      H2[e] = __float2bfloat16(silu(z));
    }
    __syncwarp();
    // layer 3: Y = H2 W3p (16 x 16, columns >= 6 zero)
    wmma::fill_fragment(fc, 0.f);
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      wmma::load_matrix_sync(fa, H2 + kt * 16, 64);
      wmma::load_matrix_sync(fb, W3p + kt * 16 * 16, 16);
      wmma::mma_sync(fc, fa, fb, fc);
    }
    wmma::store_matrix_sync(Yt, fc, 16, wmma::mem_row_major);
    __syncwarp();
    if (!TRAIN) {
      for (int e = lane; e < 16 * NOUT; e += 32) {
        const int pt = e & 15, c = e >> 4;
        if (p0 + pt < P) {
          const float y = Yt[pt * 16 + c] + prm[O_B3 + c];
          Y[(size_t)c * P + p0 + pt] = y * prm[O_OUTSC + c] + prm[O_OUTSH + c];
        }
      }
      continue;
    }
    // ---- training: dY = 2 (y - t_n) / (P * 6)
    float lsum = 0.f;
    const float inv = 2.f / ((float)P * (float)NOUT);
    for (int e = lane; e < 256; e += 32) {
      const int pt = e >> 4, c = e & 15;
      float d = 0.f;
      if (c < NOUT && p0 + pt < P) {
        const float tn = (T[(size_t)c * P + p0 + pt] - prm[O_OUTSH + c]) / prm[O_OUTSC + c];
        const float dd = Yt[e] + prm[O_B3 + c] - tn;
        lsum += dd * dd;
        d = inv * dd;
      }
      Yt[e] = d;  // FP32 dY
      DY[e] = __float2bfloat16(d);
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) atomicAdd(gloss, lsum);
    __syncwarp();
    if (lane < NOUT) {
      float s = 0.f;
      for (int pt = 0; pt < 16; ++pt) s += Yt[pt * 16 + lane];
      atomicAdd(&gb3[lane], s);
    }
    // dH2 = dY W3^T (W3p read as a column-major B); dZ2 = dH2 * silu'(Z2)
    wmma::load_matrix_sync(fa, DY, 16);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      FragBT fbt;
      wmma::fill_fragment(fc, 0.f);
      wmma::load_matrix_sync(fbt, W3p + nt * 16 * 16, 16);
      wmma::mma_sync(fc, fa, fbt, fc);
      wmma::store_matrix_sync(G + nt * 16, fc, 64, wmma::mem_row_major);
    }
    __syncwarp();
    for (int e = lane; e < 1024; e += 32) {
      const float g = G[e] * dsilu(Z2[e]);
      G[e] = g;
      DZ2[e] = __float2bfloat16(g);
    }
    __syncwarp();
    for (int n = lane; n < 64; n += 32) {
      float s = 0.f;
      for (int pt = 0; pt < 16; ++pt) s += G[pt * 64 + n];
      atomicAdd(&gb2[n], s);
    }
    // dH1 = dZ2 W2^T (into G, free again); dZ1 = dH1 * silu'(Z1)
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      wmma::fill_fragment(fc, 0.f);
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        FragBT fbt;
        wmma::load_matrix_sync(fa, DZ2 + kt * 16, 64);
        wmma::load_matrix_sync(fbt, W2s + nt * 16 * 64 + kt * 16, 64);
        wmma::mma_sync(fc, fa, fbt, fc);
      }
      wmma::store_matrix_sync(G + nt * 16, fc, 64, wmma::mem_row_major);
    }
    __syncwarp();
    for (int e = lane; e < 1024; e += 32) {
      const float g = G[e] * dsilu(Z1[e]);
      G[e] = g;
      DZ1[e] = __float2bfloat16(g);
    }
    __syncwarp();
    for (int n = lane; n < 64; n += 32) {
      float s = 0.f;
      for (int pt = 0; pt < 16; ++pt) s += G[pt * 64 + n];
      atomicAdd(&gb1[n], s);
    }
    // weight gradients (sums over the 16 points of the tile) on the tensor cores
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {  // gW3 += H2^T dY
      FragAT fat;
      wmma::fill_fragment(fc, 0.f);
      wmma::load_matrix_sync(fat, H2 + mt * 16, 64);
      wmma::load_matrix_sync(fb, DY, 16);
      wmma::mma_sync(fc, fat, fb, fc);
      wmma::store_matrix_sync(TT, fc, 16, wmma::mem_row_major);
      __syncwarp();
      add_tile(gW3, NOUT, mt * 16, 0, NH, NOUT, TT, lane);
      __syncwarp();
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {  // gW2 += H1^T dZ2
      FragAT fat;
      wmma::load_matrix_sync(fat, H1 + mt * 16, 64);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        wmma::fill_fragment(fc, 0.f);
        wmma::load_matrix_sync(fb, DZ2 + nt * 16, 64);
        wmma::mma_sync(fc, fat, fb, fc);
        wmma::store_matrix_sync(TT, fc, 16, wmma::mem_row_major);
        __syncwarp();
        add_tile(gW2, NH, mt * 16, nt * 16, NH, NH, TT, lane);
        __syncwarp();
      }
    }
    {  // gW1 += A0^T dZ1 (feature rows >= 10 are padding)
      FragAT fat;
      wmma::load_matrix_sync(fat, A0, 16);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        wmma::fill_fragment(fc, 0.f);
        wmma::load_matrix_sync(fb, DZ1 + nt * 16, 64);
        wmma::mma_sync(fc, fat, fb, fc);
        wmma::store_matrix_sync(TT, fc, 16, wmma::mem_row_major);
        __syncwarp();
        add_tile(gW1, NH, 0, nt * 16, NIN, NH, TT, lane);
        __syncwarp();
      }
    }
  }
  if (TRAIN) {
    __syncthreads();
    for (int i = threadIdx.x; i < BLK_G; i += THREADS) atomicAdd(&gsum[TRAIN_BEGIN + i], acc[i]);
    if (threadIdx.x == 0) atomicAdd(&gsum[NPARAM], gloss[0]);
  }
}

// ---------------------------------------------------------------------------
// Inference on the 5th-generation tensor cores (tcgen05, sm_100-class): tiles of
// 128 points, one TMEM lane (one thread of the 4 warps) per point. Operands are
// BF16 in shared memory in the K-major layout without swizzle: 8 x 8 core
// matrices of 128 contiguous bytes (row r of a core matrix at 16 r bytes), core
// matrices adjacent along K 128 bytes apart (the leading-dimension offset) and
// row groups of 8 rows K/8 * 128 bytes apart (the stride offset). One thread
// issues the MMAs of a layer (K = 16 per instruction, FP32 accumulation in TMEM)
// and commits them to an mbarrier; then every thread reads its row of the
// accumulator (tcgen05.ld), adds the bias, applies SiLU and writes the BF16 row
// of the next layer's A operand.
//   layer 1: D1 (TMEM columns 0..63)   = X (128 x 16) . W1 (16 x 64)
//   layer 2: D2 (TMEM columns 64..127) = H1 (128 x 64) . W2 (64 x 64)
//   layer 3: D3 (TMEM columns 0..15)   = H2 (128 x 64) . W3 (64 x 16, columns >= 6 zero)
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_THREADS = 128, TC_TMEM_COLS = 128;
// shared memory: A operands X (4 KB), H1, H2 (16 KB each); B operands W1^T (64 x 16, 2 KB),
// W2^T (64 x 64, 8 KB), W3^T (16 x 64, 2 KB); then the mbarrier and the TMEM address
constexpr int TC_X = 0, TC_H1 = TC_X + 128 * 16 * 2, TC_H2 = TC_H1 + 128 * 64 * 2, TC_W1 = TC_H2 + 128 * 64 * 2,
              TC_W2 = TC_W1 + 64 * 16 * 2, TC_W3 = TC_W2 + 64 * 64 * 2, TC_BAR = TC_W3 + 16 * 64 * 2,
              TC_SMEM = TC_BAR + 16;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;  // 1 s bound on every mbarrier wait

// byte offset of element (r, k) of a K-major operand with K columns in the core-matrix layout
__device__ __forceinline__ int tc_off(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// shared-memory matrix descriptor: start address, leading (K) and stride (row-group)
// byte offsets, the fixed version bits 46-47 = 1, no swizzle
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((saddr & 0x3FFFF) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
         ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr unsigned tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(unsigned dt, unsigned long long ad, unsigned long long bd, unsigned idesc,
                                       int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}
// waits for the phase `parity` of the mbarrier; false if it did not complete within TC_WAIT_NS
__device__ __forceinline__ bool tc_wait(unsigned bar, unsigned parity) {
  unsigned long long t0 = 0;
  for (int it = 0;; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (it == 0) t0 = t;
    else if (t - t0 > TC_WAIT_NS) return false;
  }
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// bias + SiLU of this thread's 64 accumulator columns at TMEM column c0, written as the
// thread's BF16 row of a K = 64 A operand at `dst`
__device__ __forceinline__ void tc_hidden(unsigned trow, int c0, const float* __restrict__ bias, unsigned char* dst,
                                          int row) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float v[16];
    tc_ld16(trow + c0 + 16 * q, v);
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // two 8-element core-matrix rows of 16 bytes
      __align__(16) bf o[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) o[i] = __float2bfloat16(silu(v[8 * h + i] + bias[16 * q + 8 * h + i]));
      *reinterpret_cast<uint4*>(dst + tc_off(row, 16 * q + 8 * h, 64)) = *reinterpret_cast<const uint4*>(o);
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS) k_mlp_tc(const float* __restrict__ prm, const bf* __restrict__ wpack,
                                                       const float* __restrict__ X, int P, float* __restrict__ Y,
                                                       int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ unsigned s_taddr;
  __shared__ float s_b[2 * NH + 16];  // b1, b2, b3
  const int t = threadIdx.x, warp = t >> 5;
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(tsm);
  const unsigned bar = sbase + TC_BAR;
  // B operands from the packed weights: W^T rows n, columns k
  for (int i = t; i < 64 * 16; i += TC_THREADS) {  // W1^T (64 x 16): W1p[k][n]
    const int n = i >> 4, k = i & 15;
    *reinterpret_cast<bf*>(tsm + TC_W1 + tc_off(n, k, 16)) = wpack[PW1 + k * 64 + n];
  }
  for (int i = t; i < 64 * 64; i += TC_THREADS) {  // W2^T (64 x 64): W2[k][n]
    const int n = i >> 6, k = i & 63;
    *reinterpret_cast<bf*>(tsm + TC_W2 + tc_off(n, k, 64)) = wpack[PW2 + k * 64 + n];
  }
  for (int i = t; i < 16 * 64; i += TC_THREADS) {  // W3^T (16 x 64): W3p[k][n]
    const int n = i >> 6, k = i & 63;
    *reinterpret_cast<bf*>(tsm + TC_W3 + tc_off(n, k, 64)) = wpack[PW3 + k * 16 + n];
  }
  for (int i = t; i < 2 * NH + 16; i += TC_THREADS)
    s_b[i] = i < NH ? prm[O_B1 + i] : (i < 2 * NH ? prm[O_B2 + i - NH] : (i - 2 * NH < NOUT ? prm[O_B3 + i - 2 * NH] : 0.f));
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(&s_taddr)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = s_taddr;
  const unsigned trow = tmem + ((unsigned)(32 * warp) << 16);  // this warp's 32 lanes
  const unsigned long long dW1 = tc_desc(sbase + TC_W1, 128, 2 * 128);
  const unsigned long long dW2 = tc_desc(sbase + TC_W2, 128, 8 * 128);
  const unsigned long long dW3 = tc_desc(sbase + TC_W3, 128, 8 * 128);
  const unsigned long long dX = tc_desc(sbase + TC_X, 128, 2 * 128);
  const unsigned long long dH1 = tc_desc(sbase + TC_H1, 128, 8 * 128);
  const unsigned long long dH2 = tc_desc(sbase + TC_H2, 128, 8 * 128);
  constexpr unsigned ID64 = tc_idesc(128, 64), ID16 = tc_idesc(128, 16);
  constexpr unsigned long long KSTEP = (2 * 128) >> 4;  // descriptor start address step of K = 16
  unsigned phase = 0;
  bool ok = true;
  const int ntiles = (P + TC_M - 1) / TC_M;
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int p = tile * TC_M + t;
    {  // A operand of layer 1: the standardised features of point p, BF16, features >= 10 zero
      __align__(16) bf o[16];
#pragma unroll
      for (int f = 0; f < 16; ++f) {
        float v = 0.f;
        if (f < NIN && p < P) v = (X[(size_t)f * P + p] - prm[O_INSH + f]) * prm[O_INSC + f];
        o[f] = __float2bfloat16(v);
      }
      *reinterpret_cast<uint4*>(tsm + TC_X + tc_off(t, 0, 16)) = *reinterpret_cast<const uint4*>(o);
      *reinterpret_cast<uint4*>(tsm + TC_X + tc_off(t, 8, 16)) = *reinterpret_cast<const uint4*>(o + 8);
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      tc_mma(tmem, dX, dW1, ID64, 0);
      tc_commit(bar);
    }
    // every thread takes the same barriers whatever its waits returned; the block leaves
    // the loop together at the end of the tile (__syncthreads_and)
    ok = tc_wait(bar, phase) && ok;
    phase ^= 1;
    tc_fence_after();
    tc_hidden(trow, 0, s_b, tsm + TC_H1, t);
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) tc_mma(tmem + 64, dH1 + kk * KSTEP, dW2 + kk * KSTEP, ID64, kk);
      tc_commit(bar);
    }
    ok = tc_wait(bar, phase) && ok;
    phase ^= 1;
    tc_fence_after();
    tc_hidden(trow, 64, s_b + NH, tsm + TC_H2, t);
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) tc_mma(tmem, dH2 + kk * KSTEP, dW3 + kk * KSTEP, ID16, kk);
      tc_commit(bar);
    }
    ok = tc_wait(bar, phase) && ok;
    phase ^= 1;
    tc_fence_after();
    {
      float v[16];
      tc_ld16(trow, v);
      if (p < P) {
#pragma unroll
        for (int c = 0; c < NOUT; ++c) Y[(size_t)c * P + p] = (v[c] + s_b[2 * NH + c]) * prm[O_OUTSC + c] + prm[O_OUTSH + c];
      }
    }
    tc_fence_before();
    ok = __syncthreads_and(ok);  // shared operands and TMEM columns are free for the next tile
    tc_fence_after();
  }
  if (!ok && t == 0) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

// Adam on the trainable range; moments m, v; step t >= 1; clears the gradient sums.
__global__ void k_adam(float* __restrict__ prm, float* __restrict__ gsum, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = TRAIN_BEGIN + threadIdx.x + blockIdx.x * blockDim.x; i < TRAIN_END; i += blockDim.x * gridDim.x) {
    const float g = gsum[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    prm[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    gsum[i] = 0.f;
  }
}

}  // namespace

struct dns_mlp {
  float* prm = nullptr;   // NPARAM (device)
  float* gsum = nullptr;  // NPARAM + 1 (device): gradient sums and the loss sum
  float* m = nullptr;
  float* v = nullptr;
  bf* pack = nullptr;  // NPACK (device)
  int* err = nullptr;  // device flag: a tensor-core wait of the inference kernel gave up
  int t = 0;           // Adam steps taken
};

namespace {

int mlp_fail(int code, const char* msg) {
  dns::set_error_message(msg);
  return code;
}

#define MLP_CUDA(call, where)                      \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return mlp_fail(DNS_ERR_CUDA, where); \
  } while (0)

// inference grid: four blocks per SM (4 x 128 TMEM columns fill an SM's 512), each block
// walking several 128-point tiles
int mlp_blocks_tc(int P) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 148;
  }
  const int tiles = (P + TC_M - 1) / TC_M;
  return tiles < 4 * sms ? (tiles < 1 ? 1 : tiles) : 4 * sms;
}

int mlp_blocks(int P) {
  int tiles = (P + 15) / 16;
  int b = (tiles + WARPS - 1) / WARPS;
  return b > 2048 ? 2048 : (b < 1 ? 1 : b);
}

int mlp_run_grad(dns_mlp* net, const float* X, const float* T, int P, cudaStream_t st) {
  MLP_CUDA(cudaMemsetAsync(net->gsum, 0, (NPARAM + 1) * sizeof(float), st), "dns_mlp: clear gradients");
  k_mlp<1><<<mlp_blocks(P), THREADS, SMEM_B, st>>>(net->prm, net->pack, X, P, nullptr, T, net->gsum);
  MLP_CUDA(cudaGetLastError(), "dns_mlp: training kernel launch");
  return DNS_OK;
}

// Mean and unbiased standard deviation of each feature row of X (10 x P) and each
// stress row of T (6 x P), in FP64, written into the normalisation entries of the
// parameter vector: in_shift = mean, in_scale = 1/std (1 where std <= 1e-12),
// out_scale = std (1 where std <= 1e-30), out_shift = mean. One block per row.
constexpr int NORM_THREADS = 256;
__global__ void __launch_bounds__(NORM_THREADS) k_norm(float* __restrict__ prm, const float* __restrict__ X,
                                                       const float* __restrict__ T, int P) {
  const int r = blockIdx.x;
  const float* row = r < NIN ? X + (size_t)r * P : T + (size_t)(r - NIN) * P;
  __shared__ double red[NORM_THREADS / 32];
  __shared__ double s_mean;
  auto block_sum = [&](double v) -> double {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < NORM_THREADS / 32; ++w) t += red[w];
    return t;
  };
  double s = 0.0;
  for (int i = threadIdx.x; i < P; i += NORM_THREADS) s += (double)row[i];
  const double tot = block_sum(s);
  if (threadIdx.x == 0) s_mean = tot / (double)P;
  __syncthreads();
  const double mean = s_mean;
  double q = 0.0;
  for (int i = threadIdx.x; i < P; i += NORM_THREADS) {
    const double d = (double)row[i] - mean;
    q += d * d;
  }
  const double ss = block_sum(q);
  if (threadIdx.x == 0) {
    const double sd = P > 1 ? sqrt(ss / (double)(P - 1)) : 0.0;
    if (r < NIN) {
      prm[O_INSH + r] = (float)mean;
      prm[O_INSC + r] = sd > 1e-12 ? (float)(1.0 / sd) : 1.f;
    } else {
      prm[O_OUTSC + r - NIN] = sd > 1e-30 ? (float)sd : 1.f;
      prm[O_OUTSH + r - NIN] = (float)mean;
    }
  }
}

// Reports (and clears) a tensor-core wait of the inference kernel that gave up; synchronises.
int mlp_check_err(dns_mlp* n, const char* where) {
  int err = 0;
  MLP_CUDA(cudaMemcpy(&err, n->err, sizeof(int), cudaMemcpyDeviceToHost), where);
  if (!err) return DNS_OK;
  MLP_CUDA(cudaMemset(n->err, 0, sizeof(int)), where);
  return mlp_fail(DNS_ERR_TIMEOUT, "dns_mlp: an inference kernel's tensor-core wait gave up after 1 s; its output is not valid");
}

}  // namespace

namespace dns {
cudaError_t mlp_forward_async(::dns_mlp* n, const float* X, float* Y, int P, cudaStream_t st) {
  k_mlp_tc<<<mlp_blocks_tc(P), TC_THREADS, TC_SMEM, st>>>(n->prm, n->pack, X, P, Y, n->err);
  return cudaGetLastError();
}
}  // namespace dns

extern "C" {

int dns_mlp_set_normalisation(dns_mlp* n, const float* X, const float* T, int P, void* stream) {
  if (!n || !X || !T || P < 2) return mlp_fail(DNS_ERR_ARG, "dns_mlp_set_normalisation: bad arguments");
  k_norm<<<NIN + NOUT, NORM_THREADS, 0, (cudaStream_t)stream>>>(n->prm, X, T, P);
  MLP_CUDA(cudaGetLastError(), "dns_mlp_set_normalisation launch");
  return DNS_OK;
}

int dns_mlp_param_count(void) { return NPARAM; }

int dns_mlp_create(dns_mlp** out) {
  if (!out) return mlp_fail(DNS_ERR_ARG, "dns_mlp_create: out is NULL");
  *out = nullptr;
  dns_mlp* n = new dns_mlp();
  cudaError_t e = cudaMalloc(&n->prm, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->gsum, (NPARAM + 1) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->m, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->v, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->pack, NPACK * sizeof(bf));
  if (e == cudaSuccess) e = cudaMalloc(&n->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->prm, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->gsum, 0, (NPARAM + 1) * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_B);
  if (e != cudaSuccess) {
    dns_mlp_destroy(n);
    cudaGetLastError();
    return mlp_fail(e == cudaErrorMemoryAllocation ? DNS_ERR_OOM : DNS_ERR_CUDA, "dns_mlp_create: device set-up failed");
  }
  *out = n;
  return DNS_OK;
}

int dns_mlp_destroy(dns_mlp* n) {
  if (!n) return DNS_OK;
  cudaFree(n->prm);
  cudaFree(n->gsum);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->pack);
  cudaFree(n->err);
  delete n;
  return DNS_OK;
}

int dns_mlp_set_params(dns_mlp* n, const float* host, int count) {
  if (!n || !host || count != NPARAM) return mlp_fail(DNS_ERR_ARG, "dns_mlp_set_params: need 5286 host floats");
  MLP_CUDA(cudaMemcpy(n->prm, host, NPARAM * sizeof(float), cudaMemcpyHostToDevice), "dns_mlp_set_params copy");
  MLP_CUDA(cudaMemset(n->m, 0, NPARAM * sizeof(float)), "dns_mlp_set_params");
  MLP_CUDA(cudaMemset(n->v, 0, NPARAM * sizeof(float)), "dns_mlp_set_params");
  n->t = 0;
  k_pack<<<16, 256>>>(n->prm, n->pack);
  MLP_CUDA(cudaGetLastError(), "dns_mlp_set_params pack");
  MLP_CUDA(cudaDeviceSynchronize(), "dns_mlp_set_params");
  return DNS_OK;
}

int dns_mlp_get_params(dns_mlp* n, float* host, int count) {
  if (!n || !host || count != NPARAM) return mlp_fail(DNS_ERR_ARG, "dns_mlp_get_params: need 5286 host floats");
  MLP_CUDA(cudaDeviceSynchronize(), "dns_mlp_get_params");
  MLP_CUDA(cudaMemcpy(host, n->prm, NPARAM * sizeof(float), cudaMemcpyDeviceToHost), "dns_mlp_get_params copy");
  return mlp_check_err(n, "dns_mlp_get_params");
}

int dns_mlp_forward(dns_mlp* n, const float* X, float* Y, int P, void* stream) {
  if (!n || !X || !Y || P < 1) return mlp_fail(DNS_ERR_ARG, "dns_mlp_forward: bad arguments");
  k_mlp_tc<<<mlp_blocks_tc(P), TC_THREADS, TC_SMEM, (cudaStream_t)stream>>>(n->prm, n->pack, X, P, Y, n->err);
  MLP_CUDA(cudaGetLastError(), "dns_mlp_forward launch");
  return DNS_OK;
}

int dns_mlp_loss_grad(dns_mlp* n, const float* X, const float* T, int P, float* grad_host, float* loss_host,
                      void* stream) {
  if (!n || !X || !T || P < 1) return mlp_fail(DNS_ERR_ARG, "dns_mlp_loss_grad: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_run_grad(n, X, T, P, st);
  if (rc) return rc;
  std::vector<float> g(NPARAM + 1);
  MLP_CUDA(cudaMemcpyAsync(g.data(), n->gsum, (NPARAM + 1) * sizeof(float), cudaMemcpyDeviceToHost, st),
           "dns_mlp_loss_grad copy");
  MLP_CUDA(cudaStreamSynchronize(st), "dns_mlp_loss_grad");
  if (grad_host) memcpy(grad_host, g.data(), NPARAM * sizeof(float));
  if (loss_host) *loss_host = g[NPARAM] / ((float)P * (float)NOUT);
  MLP_CUDA(cudaMemsetAsync(n->gsum, 0, (NPARAM + 1) * sizeof(float), st), "dns_mlp_loss_grad clear");
  return DNS_OK;
}

int dns_mlp_train_step(dns_mlp* n, const float* X, const float* T, int P, double lr, float* loss_host, void* stream) {
  if (!n || !X || !T || P < 1 || !(lr > 0.0)) return mlp_fail(DNS_ERR_ARG, "dns_mlp_train_step: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_run_grad(n, X, T, P, st);
  if (rc) return rc;
  float lsum = 0.f;
  if (loss_host) MLP_CUDA(cudaMemcpyAsync(&lsum, n->gsum + NPARAM, sizeof(float), cudaMemcpyDeviceToHost, st),
                          "dns_mlp_train_step loss copy");
  n->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->t), c2 = 1.f - std::pow(b2, (float)n->t);
  k_adam<<<8, 256, 0, st>>>(n->prm, n->gsum, n->m, n->v, (float)lr, b1, b2, 1e-8f, c1, c2);
  k_pack<<<16, 256, 0, st>>>(n->prm, n->pack);
  MLP_CUDA(cudaGetLastError(), "dns_mlp_train_step update");
  if (loss_host) {
    MLP_CUDA(cudaStreamSynchronize(st), "dns_mlp_train_step");
    *loss_host = lsum / ((float)P * (float)NOUT);
  }
  return DNS_OK;
}

}  // extern "C"

// Device side of the learned Voigt surrogate (not part of the paper): a 2-64-64-64-1 SiLU
// network that predicts t = ln(K(x, y) / K0(x, y)) from u1 = ln y and
// u2 = ln(1 + |x| / (1 + y)), with the baseline
//   K0 = exp(-x^2) / (1 + 2y/sqrt(pi)) + y / (sqrt(pi) (x^2 + y^2 + 1)),
// so that K = K0 exp(t).
//
// Inference is warp-collective: the 32 lanes of a converged warp evaluate 32 (x, y)
// pairs at once. Layer 1 (2 -> 64) runs in FP32 and is written straight into the BF16 A
// fragments of mma.sync m16n8k16; layers 2 and 3 (64 -> 64) run on the tensor cores with
// BF16 operands and FP32 accumulation, chained through registers; layer 3's activations
// stay in FP32 for the output dot product, which each quad of lanes reduces with shuffles.
//
// The guard decides where the surrogate may stand in for the plain FP32 Voigt: a bit per
// cell of the (|x|, y) plane, set by k_mlp_guard only for cells inside the region where
// the plain evaluation takes its costly branch and where the surrogate agreed with the
// plain evaluation to within the error budget at every sample point of the cell.
#pragma once
#include <cuda_bf16.h>

#include <cstring>

#include "marfa_internal.cuh"
#include "voigt.cuh"

namespace marfa {

__device__ __forceinline__ float mlp_silu_acc(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// z sigmoid(z) with sigmoid(z) = (1 + tanh(z/2)) / 2; used where the result is rounded
// to BF16 right after.
__device__ __forceinline__ float mlp_silu_bf(float z) {
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(0.5f * z));
  return 0.5f * z * (1.0f + th);
}

__device__ __forceinline__ float mlp_baseline_fast(float x, float y) {
  const float kSp = 1.7724538509055159f;
  const float x2 = x * x;
  return __fdividef(__expf(-x2), fmaf(2.0f / kSp, y, 1.0f)) +
         __fdividef(y, kSp * (x2 + fmaf(y, y, 1.0f)));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One 64 -> 64 layer for 32 samples: in = A fragments [2 m-tiles][4 k-tiles][4 regs],
// W rows [out][kWStride] in BF16, bias FP32. Accumulators start at the bias; the
// callback f(nt, d) consumes n-tile nt (columns 8nt + 2t, +1; rows g, g + 8).
template <class F>
__device__ __forceinline__ void mlp_layer(const uint32_t (&in)[2][4][4], const uint16_t* W,
                                          const float* b, int lane, F&& f) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float d[2][4];
    const float bl = b[8 * nt + 2 * t], bh = b[8 * nt + 2 * t + 1];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      d[mt][0] = bl; d[mt][1] = bh; d[mt][2] = bl; d[mt][3] = bh;
    }
    const uint16_t* wr = W + (8 * nt + g) * kWStride + 2 * t;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr + 16 * kt);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 16 * kt + 8);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) mma16816(d[mt], in[mt][kt], b0, b1);
    }
    f(nt, d);
  }
}

// Surrogate K(x, y) for the 32 lanes of a converged warp, one input per lane.
static __device__ __noinline__ float mlp_warp_K(const MlpWeights& S, float x, float y) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const float ax = fabsf(x);
  const float u1 = __logf(y);
  const float u2 = __logf(1.0f + __fdividef(ax, 1.0f + y));
  // the inputs of A-fragment rows g and g + 8 of m-tile mt: samples 16 mt + g (+ 8)
  float su1[2][2], su2[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      su1[mt][r] = __shfl_sync(0xffffffffu, u1, 16 * mt + g + 8 * r);
      su2[mt][r] = __shfl_sync(0xffffffffu, u2, 16 * mt + g + 8 * r);
    }
  // layer 1 into A fragments: k-tile kt holds hidden units 16kt + 2t + {0, 1} (regs 0, 1)
  // and 16kt + 8 + 2t + {0, 1} (regs 2, 3); reg parity picks row g or g + 8.
  uint32_t a1[2][4][4];
#pragma unroll
  for (int kt = 0; kt < 4; ++kt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int c0 = 16 * kt + 8 * half + 2 * t;
      const float w00 = S.w1[2 * c0], w01 = S.w1[2 * c0 + 1], bb0 = S.b1[c0];
      const float w10 = S.w1[2 * c0 + 2], w11 = S.w1[2 * c0 + 3], bb1 = S.b1[c0 + 1];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const float z0 = fmaf(w00, su1[mt][r], fmaf(w01, su2[mt][r], bb0));
          const float z1 = fmaf(w10, su1[mt][r], fmaf(w11, su2[mt][r], bb1));
          a1[mt][kt][2 * half + r] = pack_bf16(mlp_silu_bf(z0), mlp_silu_bf(z1));
        }
    }
  // layer 2: the outputs of n-tile nt are k-tile nt / 2, half nt % 2 of layer 3's input
  uint32_t a2[2][4][4];
  mlp_layer(a1, S.w2, S.b2, lane, [&](int nt, float (&d)[2][4]) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      a2[mt][nt >> 1][(nt & 1) ? 2 : 0] = pack_bf16(mlp_silu_bf(d[mt][0]), mlp_silu_bf(d[mt][1]));
      a2[mt][nt >> 1][(nt & 1) ? 3 : 1] = pack_bf16(mlp_silu_bf(d[mt][2]), mlp_silu_bf(d[mt][3]));
    }
  });
  // layer 3 and the output layer: per-lane partial dot products with W4 in FP32
  float part[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  mlp_layer(a2, S.w3, S.b3, lane, [&](int nt, float (&d)[2][4]) {
    const float wl = S.w4[8 * nt + 2 * t], wh = S.w4[8 * nt + 2 * t + 1];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      part[mt][0] = fmaf(wl, mlp_silu_acc(d[mt][0]), fmaf(wh, mlp_silu_acc(d[mt][1]), part[mt][0]));
      part[mt][1] = fmaf(wl, mlp_silu_acc(d[mt][2]), fmaf(wh, mlp_silu_acc(d[mt][3]), part[mt][1]));
    }
  });
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      part[mt][r] += __shfl_xor_sync(0xffffffffu, part[mt][r], 1);
      part[mt][r] += __shfl_xor_sync(0xffffffffu, part[mt][r], 2);
    }
  // sample s = 16 mt + 8 r + gg sits in part[mt][r] of lanes 4gg .. 4gg + 3
  const int smt = lane >> 4, sr = (lane >> 3) & 1, sg = lane & 7;
  float tv = 0.0f;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const float v = __shfl_sync(0xffffffffu, part[mt][r], 4 * sg);
      if (mt == smt && r == sr) tv = v;
    }
  tv += S.b4;
  return mlp_baseline_fast(x, y) * __expf(tv);
}

// Copy the weights and guard bits into shared memory (whole block; caller syncs).
__device__ __forceinline__ void mlp_load_smem(MlpWeights& S, const MlpWeights* __restrict__ src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(&S);
  for (int i = threadIdx.x; i < (int)(sizeof(MlpWeights) / 16); i += blockDim.x) d[i] = __ldg(s + i);
}

// Guard cell of (x, y): |x| in steps of 1/8 up to 12; y by binary exponent and the two
// leading mantissa bits (y in [2^e (1 + k/4), 2^e (1 + (k+1)/4)), e in [-14, 3]).
// Returns -1 outside the guarded domain.
__host__ __device__ __forceinline__ int mlp_guard_cell(float x, float y) {
  const float ax = fabsf(x);
  if (!(ax < 12.0f) || !(y >= 6.103515625e-05f) || !(y < 16.0f)) return -1;
#ifdef __CUDA_ARCH__
  const uint32_t bits = __float_as_uint(y);
#else
  uint32_t bits;
  memcpy(&bits, &y, 4);
#endif
  const int e = (int)(bits >> 23) - 127;
  const int iy = (e + 14) * 4 + (int)((bits >> 21) & 3u);
  const int ix = (int)(ax * 8.0f);
  return iy * kGuardNx + ix;
}

__device__ __forceinline__ bool mlp_guard(const MlpWeights& S, float x, float y) {
  const int c = mlp_guard_cell(x, y);
  return c >= 0 && ((S.guard[c >> 5] >> (c & 31)) & 1u);
}

// The Voigt K for a converged warp: the surrogate for the lanes whose (x, y) passes the
// guard (when any does), the plain FP32 evaluation for the other active lanes, 0 for
// inactive lanes. n_mlp counts this lane's surrogate evaluations.
template <bool SMEM>
__device__ __forceinline__ float voigt_K_coll(float x, float y, bool active, const float* tab,
                                              const MlpWeights& S, int64_t& n_mlp) {
  const bool use = active && mlp_guard(S, x, y);
  float k = 0.0f;
  if (__ballot_sync(0xffffffffu, use)) {
    const float km = mlp_warp_K(S, use ? x : 0.0f, use ? y : 1.0f);
    if (use) k = km;
  }
  if (active && !use) k = voigt_K<SMEM>(x, y, tab);
  n_mlp += use ? 1 : 0;
  return k;
}

}  // namespace marfa

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

// One 64 -> 64 layer for one m-tile of 16 samples: in = A fragments [4 k-tiles][4 regs],
// W rows [out][kWStride] in BF16, bias FP32. Accumulators start at the bias; the
// callback f(nt, d) consumes n-tile nt (columns 8nt + 2t, +1 of rows g, g + 8).
template <class F>
__device__ __forceinline__ void mlp_layer(const uint32_t (&in)[4][4], const uint16_t* W, const float* b,
                                          int lane, F&& f) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bl = b[8 * nt + 2 * t], bh = b[8 * nt + 2 * t + 1];
    float d[4] = {bl, bh, bl, bh};
    const uint16_t* wr = W + (8 * nt + g) * kWStride + 2 * t;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr + 16 * kt);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 16 * kt + 8);
      mma16816(d, in[kt], b0, b1);
    }
    f(nt, d);
  }
}

// Surrogate K(x, y) for the 32 lanes of a converged warp, one input per lane. The two
// m-tiles (samples 0-15 and 16-31) go through the network one after the other, which
// keeps a tile's activations (16 + 16 registers) the only large live state.
static __device__ __noinline__ float mlp_warp_K(const MlpWeights& S, float x, float y) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const float ax = fabsf(x);
  const float u1 = __logf(y);
  const float u2 = __logf(1.0f + __fdividef(ax, 1.0f + y));
  float tv = 0.0f;
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    // inputs of A-fragment rows g and g + 8: samples 16 mt + g (+ 8)
    const float p0 = __shfl_sync(0xffffffffu, u1, 16 * mt + g), q0 = __shfl_sync(0xffffffffu, u2, 16 * mt + g);
    const float p1 = __shfl_sync(0xffffffffu, u1, 16 * mt + g + 8), q1 = __shfl_sync(0xffffffffu, u2, 16 * mt + g + 8);
    // layer 1 into A fragments: k-tile kt holds hidden units 16kt + 2t + {0, 1} (regs 0, 1)
    // and 16kt + 8 + 2t + {0, 1} (regs 2, 3); reg parity picks row g or g + 8
    uint32_t a1[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int c0 = 16 * kt + 8 * half + 2 * t;
        const float w00 = S.w1[2 * c0], w01 = S.w1[2 * c0 + 1], bb0 = S.b1[c0];
        const float w10 = S.w1[2 * c0 + 2], w11 = S.w1[2 * c0 + 3], bb1 = S.b1[c0 + 1];
        a1[kt][2 * half] = pack_bf16(mlp_silu_bf(fmaf(w00, p0, fmaf(w01, q0, bb0))),
                                     mlp_silu_bf(fmaf(w10, p0, fmaf(w11, q0, bb1))));
        a1[kt][2 * half + 1] = pack_bf16(mlp_silu_bf(fmaf(w00, p1, fmaf(w01, q1, bb0))),
                                         mlp_silu_bf(fmaf(w10, p1, fmaf(w11, q1, bb1))));
      }
    // layer 2: the outputs of n-tile nt are k-tile nt / 2, half nt % 2 of layer 3's input
    uint32_t a2[4][4];
    mlp_layer(a1, S.w2, S.b2, lane, [&](int nt, float (&d)[4]) {
      a2[nt >> 1][(nt & 1) ? 2 : 0] = pack_bf16(mlp_silu_bf(d[0]), mlp_silu_bf(d[1]));
      a2[nt >> 1][(nt & 1) ? 3 : 1] = pack_bf16(mlp_silu_bf(d[2]), mlp_silu_bf(d[3]));
    });
    // layer 3 and the output layer: per-lane partial dot products with W4 in FP32
    float part0 = 0.0f, part1 = 0.0f;
    mlp_layer(a2, S.w3, S.b3, lane, [&](int nt, float (&d)[4]) {
      const float wl = S.w4[8 * nt + 2 * t], wh = S.w4[8 * nt + 2 * t + 1];
      part0 = fmaf(wl, mlp_silu_acc(d[0]), fmaf(wh, mlp_silu_acc(d[1]), part0));
      part1 = fmaf(wl, mlp_silu_acc(d[2]), fmaf(wh, mlp_silu_acc(d[3]), part1));
    });
    part0 += __shfl_xor_sync(0xffffffffu, part0, 1);
    part0 += __shfl_xor_sync(0xffffffffu, part0, 2);
    part1 += __shfl_xor_sync(0xffffffffu, part1, 1);
    part1 += __shfl_xor_sync(0xffffffffu, part1, 2);
    // sample 16 mt + 8 r + gg sits in part_r of lanes 4gg .. 4gg + 3
    const float v0 = __shfl_sync(0xffffffffu, part0, 4 * (lane & 7));
    const float v1 = __shfl_sync(0xffffffffu, part1, 4 * (lane & 7));
    if ((lane >> 4) == mt) tv = ((lane >> 3) & 1) ? v1 : v0;
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

// ------------------------------------------------------------------ per-warp queue
// The profile kernels do not call the network where an evaluation passes the guard:
// they push (x, y, weight, tag) into their warp's queue in shared memory and go on with
// the plain evaluations. When the queue is nearly full, and wherever the kernel needs
// the results, the warp flushes it: the network runs on full batches of 32 entries, and
// each lane then applies the results of its own entries, in queue order, through the
// kernel's callback (weight x K, tag says where it goes). All calls are warp-collective.
constexpr int kQCap = 256;
struct SurrQueue {
  float x[kQCap], y[kQCap], w[kQCap], r[kQCap];
  uint16_t tag[kQCap];
  uint8_t owner[kQCap];
};

// owner: the lane that applies the result (default: the pushing lane).
__device__ __forceinline__ void q_push(SurrQueue& Q, int& n, bool want, float x, float y, float w,
                                       int tag, int owner = -1) {
  const int lane = threadIdx.x & 31;
  const unsigned b = __ballot_sync(0xffffffffu, want);
  if (want) {
    const int pos = n + __popc(b & ((1u << lane) - 1u));
    Q.x[pos] = x;
    Q.y[pos] = y;
    Q.w[pos] = w;
    Q.tag[pos] = (uint16_t)tag;
    Q.owner[pos] = (uint8_t)(owner < 0 ? lane : owner);
  }
  n += __popc(b);
}

template <class Apply>
__device__ __forceinline__ void q_flush(SurrQueue& Q, int& n, const MlpWeights& S, Apply&& apply) {
  if (n == 0) return;  // n is warp-uniform
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int b = 0; b < n; b += 32) {
    const int i = b + lane;
    const bool act = i < n;
    const float k = mlp_warp_K(S, act ? Q.x[i] : 0.0f, act ? Q.y[i] : 1.0f);
    if (act) Q.r[i] = k * Q.w[i];
  }
  __syncwarp();
  for (int i = 0; i < n; ++i)
    if (Q.owner[i] == lane) apply((int)Q.tag[i], Q.r[i]);
  __syncwarp();
  n = 0;
}

// The queue of the calling warp, in a surrogate block of shared memory laid out as the
// weights followed by one queue per warp.
__device__ __forceinline__ SurrQueue& warp_queue(unsigned char* dsm) {
  return reinterpret_cast<SurrQueue*>(dsm + sizeof(MlpWeights))[threadIdx.x >> 5];
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

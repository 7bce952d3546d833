// FP32 Voigt function K(x, y) = Re w(x + iy) (Eq. (8) of arXiv 2411.03418) for the
// profile kernels, with a relative error of about 1e-6 over the whole (x, y >= 0)
// plane. The paper's own Humlicek/Kuntz variant (Appendix C) is accurate to 1 % only;
// this one is built from:
//   y < 1, |x| < 12    exact split w = exp(-z^2) + (2i/sqrt(pi)) F(z), F the complex
//                Dawson function, K = exp(y^2-x^2) cos(2xy) - (2/sqrt(pi)) y Psi,
//                Psi(x, y^2) = Im F / y from a table of bivariate polynomials (the
//                Gaussian term is below 4e-19 and dropped for |x| >= 6.5); below
//                y = 1/4 a second table of low degree in y^2 (6 x 4 terms per cell
//                instead of 9 x 9) serves the narrow lines;
//   |z| < 4.5, y >= 1  K from a table of bivariate polynomials;
//   elsewhere   asymptotic series of w (Abramowitz & Stegun 7.1.23),
//                w ~ i/(sqrt(pi) z) sum_n (2n-1)!!/(2 z^2)^n, truncated by |z|
//                (2 terms for |z| >= 100, 6 for |z| >= 8 (or 3 for |z| >= 22.5 where
//                the caller asks for it), 15 for |z| >= 4.5).
// The tables come from gen_voigt_tables.py (mpmath, 30 digits).
#pragma once
#include <cuda_runtime.h>

#define MARFA_VOIGT_QUAL static __device__ const __align__(16)
#include "voigt_tables.inc"
#undef MARFA_VOIGT_QUAL

namespace marfa {

constexpr float kInvSqrtPi = 0.56418958354775628f;  // 1/sqrt(pi)
constexpr float kTwoOverSqrtPi = 1.1283791670955126f;

// exp(y^2 - x^2) cos(2xy), with the exponent carried to about one extra word so
// that the Gaussian core keeps its relative accuracy out to |x| ~ 4.5. The cosine is
// the hardware approximation (absolute error about 4e-7 for |2xy| <= pi, growing
// slowly beyond): where cos(2xy) is small or its argument large, the Gaussian term is
// small against K (y < 1 here, and the term is dropped for |x| >= 6.5).
__device__ __forceinline__ float gauss_term(float x, float y) {
  float xx = x * x;
  float xl = fmaf(x, x, -xx);
  float yy = y * y;
  float yl = fmaf(y, y, -yy);
  float a = yy - xx;
  float bb = a - yy;                      // TwoSum(yy, -xx)
  float e = (yy - (a - bb)) + (-xx - bb);
  float d = e + yl - xl;
  return expf(a) * (1.0f + d) * __cosf(2.0f * x * y);
}

// Re of the asymptotic series with N+1 terms, in real arithmetic on u = 1/z, v = u^2.
template <int N>
__device__ __forceinline__ float voigt_asym(float x, float y) {
  float r2 = fmaf(x, x, y * y);
  float inv = __fdividef(1.0f, r2);  // r2 >= 20.25: 2 ulp
  float ur = x * inv, ui = -y * inv;
  float vr = ur * ur - ui * ui, vi = 2.0f * ur * ui;
  // c_n = (2n-1)!!/2^n
  float c[N + 1];
  c[0] = 1.0f;
#pragma unroll
  for (int n = 1; n <= N; ++n) c[n] = c[n - 1] * (0.5f * (2 * n - 1));
  float sr = c[N], si = 0.0f;
#pragma unroll
  for (int n = N - 1; n >= 0; --n) {
    float tr = fmaf(sr, vr, -si * vi) + c[n];
    float ti = fmaf(sr, vi, si * vr);
    sr = tr;
    si = ti;
  }
  // w ~ (i/sqrt(pi)) u S  ->  Re w = -Im(u S)/sqrt(pi)
  return -(ui * sr + ur * si) * kInvSqrtPi;
}

// One bivariate cell; tab is the coefficient table, either the global copy (read
// through the read-only cache) or a copy a kernel placed in shared memory (SMEM). Cells
// are padded to an even number of floats (81 -> 82); the shared copy is read as float2
// (vector loads through the read-only cache cost the global readers registers, and
// float4 reads of these 81-term cells make the finest-grid kernels spill).
constexpr int kVoigtCellFloats = (VOIGT_DEG + 1) * (VOIGT_DEG + 1);
constexpr int kVoigtCellStride = VOIGT_CELL_STRIDE;
static_assert(kVoigtCellStride % 2 == 0 && kVoigtCellStride >= kVoigtCellFloats, "cell padding");

template <bool SMEM, bool VEC = false>
__device__ __forceinline__ float voigt_cell(const float* tab, int cell, float u, float v) {
  if (!SMEM && !VEC) {  // global copy: scalar loads through the read-only cache
    const float* c = tab + cell * kVoigtCellStride;
    float acc = 0.0f;
#pragma unroll
    for (int p = VOIGT_DEG; p >= 0; --p) {
      float r = 0.0f;
#pragma unroll
      for (int q = VOIGT_DEG; q >= 0; --q) r = fmaf(r, v, __ldg(c + p * (VOIGT_DEG + 1) + q));
      acc = fmaf(acc, u, r);
    }
    return acc;
  }
  if (!SMEM) {  // global copy, VEC: float2 loads through the read-only cache
    const float2* c2 = reinterpret_cast<const float2*>(tab + cell * kVoigtCellStride);
    float acc = 0.0f, r = 0.0f;
#pragma unroll
    for (int i = kVoigtCellStride / 2 - 1; i >= 0; --i) {
      const float2 t = __ldg(c2 + i);
#pragma unroll
      for (int h = 1; h >= 0; --h) {
        const int k = 2 * i + h;
        if (k >= kVoigtCellFloats) continue;
        r = fmaf(r, v, h ? t.y : t.x);
        if (k % (VOIGT_DEG + 1) == 0) {  // q = 0: row p done
          acc = fmaf(acc, u, r);
          r = 0.0f;
        }
      }
    }
    return acc;
  }
  const float2* c2 = reinterpret_cast<const float2*>(tab + cell * kVoigtCellStride);
  float acc = 0.0f, r = 0.0f;
  // coefficient k = p (DEG + 1) + q of u^p v^q, taken from k = 80 down to 0, two at a time
#pragma unroll
  for (int i = kVoigtCellStride / 2 - 1; i >= 0; --i) {
    const float2 t = c2[i];
#pragma unroll
    for (int h = 1; h >= 0; --h) {
      const int k = 2 * i + h;
      if (k >= kVoigtCellFloats) continue;
      r = fmaf(r, v, h ? t.y : t.x);
      if (k % (VOIGT_DEG + 1) == 0) {  // q = 0: row p done
        acc = fmaf(acc, u, r);
        r = 0.0f;
      }
    }
  }
  return acc;
}

// A kernel's shared copy pads each small-y cell from 24 to 28 floats: every cell starts
// on a 16-byte boundary (one float4 per row), and consecutive cells lie 28 banks apart,
// so the cells that the eight lanes of one 128-bit load phase read (one lane group's
// neighbouring nodes: up to eight consecutive cells) fall on disjoint banks.
constexpr int kVoigtSmallCellSmem = 28;

// One small-y cell (degree VOIGT_SMALL_DX in u, VOIGT_SMALL_DV = 3 in v: one row of four
// coefficients per power of u, read from a shared copy as one float4).
template <bool SMEM, bool VEC = false>
__device__ __forceinline__ float voigt_cell_small(const float* tab, int cell, float u, float v) {
  static_assert(VOIGT_SMALL_DV == 3, "four coefficients per row");
  if (!SMEM && !VEC) {  // global copy: scalar loads through the read-only cache
    const float* c = tab + cell * (VOIGT_SMALL_DX + 1) * 4;
    float acc = 0.0f;
#pragma unroll
    for (int p = VOIGT_SMALL_DX; p >= 0; --p) {
      float r = 0.0f;
#pragma unroll
      for (int q = 3; q >= 0; --q) r = fmaf(r, v, __ldg(c + p * 4 + q));
      acc = fmaf(acc, u, r);
    }
    return acc;
  }
  if (!SMEM) {  // global copy, VEC: one float4 per row through the read-only cache
    const float4* c4 = reinterpret_cast<const float4*>(tab + cell * (VOIGT_SMALL_DX + 1) * 4);
    float acc = 0.0f;
#pragma unroll
    for (int p = VOIGT_SMALL_DX; p >= 0; --p) {
      const float4 t = __ldg(c4 + p);
      acc = fmaf(acc, u, fmaf(fmaf(fmaf(t.w, v, t.z), v, t.y), v, t.x));
    }
    return acc;
  }
  const float4* c4 = reinterpret_cast<const float4*>(tab + cell * kVoigtSmallCellSmem);
  float acc = 0.0f;
#pragma unroll
  for (int p = VOIGT_SMALL_DX; p >= 0; --p) {
    const float4 t = c4[p];
    acc = fmaf(acc, u, fmaf(fmaf(fmaf(t.w, v, t.z), v, t.y), v, t.x));
  }
  return acc;
}

// Floats of the large table in a kernel's shared copy; the small-y table follows it.
constexpr int kVoigtBigSmem = VOIGT_NCELL * kVoigtCellStride;

// Far-wing form (|z| >= 100): two terms of the series, K = y/(sqrt(pi) r^2) (1 + (3x^2 - y^2)/(2 r^4)).
__device__ __forceinline__ float voigt_far(float x, float y) {
  float x2 = x * x, y2 = y * y;
  float inv = __fdividef(1.0f, x2 + y2);  // x2 + y2 >= 1e4: 2 ulp
  float t = (3.0f * x2 - y2) * inv * inv * 0.5f;
  return y * kInvSqrtPi * inv * (1.0f + t);
}

// Everything but the far wing. The Dawson-table branch covers the whole near wing of
// narrow lines (y < 1, |x| < 12) so that one line's nodes on the fine grids take a
// single code path.
template <bool SMEM, bool VEC = false>
__device__ __forceinline__ float voigt_near_body(float ax, float y, const float* tab) {
  if (y < 0.25f && ax < 12.0f) {
    const int ci = min((int)(ax * 4.0f), VOIGT_SMALL_NX - 1);
    const float u = (ax - (0.25f * ci + 0.125f)) * 8.0f;
    const float v = fmaf(32.0f * y, y, -1.0f);
    const float ps = voigt_cell_small<SMEM, VEC>(SMEM ? tab + kVoigtBigSmem : kVoigtSmall, ci, u, v);
    const float gt = ax < 6.5f ? gauss_term(ax, y) : 0.0f;
    return gt - kTwoOverSqrtPi * y * ps;
  }
  if (y < 1.0f && ax < 12.0f) {
    int ci = min((int)(ax * 2.0f), VOIGT_NPSI - 1);
    float u = (ax - (0.5f * ci + 0.25f)) * 4.0f;
    float v = 2.0f * y * y - 1.0f;
    float ps = voigt_cell<SMEM, VEC>(tab, ci, u, v);
    float gt = ax < 6.5f ? gauss_term(ax, y) : 0.0f;
    return gt - kTwoOverSqrtPi * y * ps;
  }
  float r2 = fmaf(ax, ax, y * y);
  if (r2 >= 64.0f) return voigt_asym<5>(ax, y);
  if (r2 >= 20.25f) return voigt_asym<14>(ax, y);  // here y >= 1
  int ix = min((int)(ax * (1.0f / 0.9f)), 4);
  int iy = min((int)((y - 1.0f) * (1.0f / 1.75f)), 1);
  float u = (ax - (0.9f * ix + 0.45f)) * (1.0f / 0.45f);
  float v = (y - (1.0f + 1.75f * iy + 0.875f)) * (1.0f / 0.875f);
  return voigt_cell<SMEM, VEC>(tab, VOIGT_NPSI + ix * 2 + iy, u, v);
}

// The same out of line, so that callers with several evaluation sites stay small.
template <bool SMEM>
__device__ __noinline__ float voigt_K_near(float ax, float y, const float* tab) {
  return voigt_near_body<SMEM>(ax, y, tab);
}

// MID3: evaluate 22.5 <= |z| < 100 inline with three terms of the series (the first
// omitted term is below 7 (15/8) / |z|^6 < 1e-7 relative, also for Re w near the real
// axis) instead of the six terms of voigt_K_near; it pays where most evaluations lie in
// the mid wing (grids 2..8) and costs registers and branches elsewhere. INL: the near
// wing inline (one evaluation site in the caller's loop) instead of a call.
// VEC (global tables only): vector loads of the cells, for a caller with the registers
// to spare (they raise the register count of most kernels).
template <bool SMEM, bool MID3 = false, bool INL = false, bool VEC = false>
__device__ __forceinline__ float voigt_K(float x, float y, const float* tab) {
  float ax = fabsf(x);
  float r2 = fmaf(ax, ax, y * y);
  if (r2 >= 1.0e4f) return voigt_far(ax, y);
  if (MID3 && r2 >= 506.25f) return voigt_asym<2>(ax, y);
  return INL ? voigt_near_body<SMEM, VEC>(ax, y, tab) : voigt_K_near<SMEM>(ax, y, tab);
}

__device__ __forceinline__ float voigt_K(float x, float y) { return voigt_K<false>(x, y, kVoigtCells); }

// K(x, y) as the paper's Appendix C computes it, in FP32 like the paper's code: the
// Lorentz wing y / (sqrt(pi) (x^2 + y^2)) beyond |x| = 15; in region 4 (y < 0.02,
// 1 < |x| < 5.5) the asymptote exp(-x^2) + y / (sqrt(pi) x^2) (1 + 3 / (2 x^2)); elsewhere
// Re of Humlicek's (1982) rational approximation of w in t = y - i|x| for the region
// |x| + y falls in (I: >= 15, II: >= 5.5, III: below). Accurate to Humlicek's 1e-4 in
// regions I-III, about 1 % in the Lorentz wing and the rest of Humlicek's region IV, and
// several per cent in region 4 (the paper's choices).
__device__ __forceinline__ float voigt_K_paper(float x, float y) {
  const float ax = fabsf(x);
  if (ax > 15.0f) return y * kInvSqrtPi / fmaf(ax, ax, y * y);
  if (y < 0.02f && ax > 1.0f && ax < 5.5f) {
    const float ix2 = 1.0f / (ax * ax);
    return expf(-ax * ax) + y * kInvSqrtPi * ix2 * fmaf(1.5f, ix2, 1.0f);
  }
  const float tr = y, ti = -ax;  // t = y - i|x|
  auto mul = [](float& ar, float& ai, float br, float bi) {
    const float r = ar * br - ai * bi;
    ai = ar * bi + ai * br;
    ar = r;
  };
  float nr, ni, dr, di;  // w = (nr + i ni) / (dr + i di)
  const float s = ax + y;
  if (s >= 5.5f) {
    float ur = tr, ui = ti;  // u = t^2
    mul(ur, ui, tr, ti);
    if (s >= 15.0f) {  // region I: 0.5641896 t / (0.5 + u)
      nr = 0.5641896f * tr;
      ni = 0.5641896f * ti;
      dr = 0.5f + ur;
      di = ui;
    } else {  // region II: t (1.410474 + 0.5641896 u) / (0.75 + u (3 + u))
      nr = 1.410474f + 0.5641896f * ur;
      ni = 0.5641896f * ui;
      mul(nr, ni, tr, ti);
      dr = 3.0f + ur;
      di = ui;
      mul(dr, di, ur, ui);
      dr += 0.75f;
    }
  } else {  // region III: quartic over quintic in t
    nr = 0.5642236f * tr;
    ni = 0.5642236f * ti;
    nr += 3.778987f;
    mul(nr, ni, tr, ti);
    nr += 11.96482f;
    mul(nr, ni, tr, ti);
    nr += 20.20933f;
    mul(nr, ni, tr, ti);
    nr += 16.4955f;
    dr = tr + 6.699398f;
    di = ti;
    mul(dr, di, tr, ti);
    dr += 21.69274f;
    mul(dr, di, tr, ti);
    dr += 39.27121f;
    mul(dr, di, tr, ti);
    dr += 38.82363f;
    mul(dr, di, tr, ti);
    dr += 16.4955f;
  }
  return __fdividef(fmaf(nr, dr, ni * di), fmaf(dr, dr, di * di));
}

// The same out of line, for the generic shape switch (keeps its callers' registers).
static __device__ __noinline__ float voigt_K_paper_call(float x, float y) { return voigt_K_paper(x, y); }

// Cost class of one voigt_K evaluation, for operation counts: 0 the far-wing two-term
// series, 1 the 6- or 15-term asymptotic series, 2 a 9 x 9 polynomial cell (Dawson or K
// table), 3 a small-y cell.
__device__ __forceinline__ int voigt_class(float x, float y) {
  const float ax = fabsf(x);
  const float r2 = fmaf(ax, ax, y * y);
  if (r2 >= 1.0e4f) return 0;
  if (y < 0.25f && ax < 12.0f) return 3;
  if (y < 1.0f && ax < 12.0f) return 2;
  return r2 >= 20.25f ? 1 : 2;
}

constexpr int kVoigtSmallFloats = VOIGT_SMALL_NX * (VOIGT_SMALL_DX + 1) * (VOIGT_SMALL_DV + 1);
constexpr int kVoigtTableFloats = kVoigtBigSmem + VOIGT_SMALL_NX * kVoigtSmallCellSmem;  // shared copy
static_assert(kVoigtSmallCellSmem % 4 == 0 && kVoigtSmallCellSmem >= (VOIGT_SMALL_DX + 1) * 4, "small cell padding");
static_assert(kVoigtBigSmem % 4 == 0, "the small-y table starts on a 16-byte boundary");

// Copy both coefficient tables into shared memory (all threads of the block take part:
// warp w copies cells w, w + nwarps, ..., lane by lane, in the global layout; then the
// small-y cells, each padded to kVoigtSmallCellSmem floats). dst: 16-byte aligned.
__device__ __forceinline__ void voigt_table_to_smem(float* dst) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int cell = threadIdx.x >> 5; cell < VOIGT_NCELL; cell += nw) {
    const float* src = kVoigtCells + cell * kVoigtCellStride;
    float* d = dst + cell * kVoigtCellStride;
#pragma unroll
    for (int k = lane; k < kVoigtCellStride; k += 32) d[k] = src[k];
  }
  constexpr int cf = (VOIGT_SMALL_DX + 1) * 4;  // floats of a small-y cell
  for (int i = threadIdx.x; i < VOIGT_SMALL_NX * kVoigtSmallCellSmem; i += blockDim.x) {
    const int cell = i / kVoigtSmallCellSmem, k = i - cell * kVoigtSmallCellSmem;
    dst[kVoigtBigSmem + i] = k < cf ? kVoigtSmall[cell * cf + k] : 0.0f;
  }
}

}  // namespace marfa

// Kernels of libmarfa: per-level line preparation, the coarse-grid (G1..G10) panel
// sums and the finest-grid sum with the fused interpolation cascade (Sec. 2.4 of
// arXiv 2411.03418).
//
// Partition (which grid sums which part of a line's profile), in exact fixed point:
// grid g (1..10) accepts panel m of a line (the closed interval [m P, (m+1) P],
// P = 2 h_g, nodes at 0, h_g, 2 h_g) when the whole panel lies within the cut-off,
// it is at least R_w h_g from the line centre or h_g <= W / R_c (g >= g*), and, with
// the chi-factor on, no Eq. (10) breakpoint lies in it. Grid g owns the panel when it
// accepts it and grid g-1 does not accept the parent panel; the finest grid owns a
// node within the cut-off whose G10 panel is not accepted. Each grid sums the
// profile at the three nodes of each owned panel into panel-local values L, M, R;
// the finest-grid pass adds, at every node, its own sum and the quadratic through
// the L, M, R of the panel containing the node on each coarse grid.
#include <cstdio>

#include "marfa_internal.cuh"
#include "voigt.cuh"

namespace marfa {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  float y = v - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Sum of a compensated pair over the 32 lanes of a warp; every lane gets the same
// result (the butterfly's pairwise TwoSum is symmetric in its operands).
__device__ __forceinline__ float warp_sum_comp(float s, float c) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    float t = s + s2;
    float bp = t - s;
    float e = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = (c + c2) + e;
  }
  return s + c;
}

// first line index whose key is >= K
__device__ __forceinline__ int64_t lower_idx(const ReqDev& R, int64_t K) {
  int64_t b = (K - R.key_base) >> R.bshift;
  if (K <= R.key_base) return 0;
  if (b >= R.nbuck) return R.n_lines;
  int64_t i = R.bfirst[b];
  while (i < R.n_lines && __ldg(R.key + i) < K) ++i;
  return i;
}
// first line index whose key is > K
__device__ __forceinline__ int64_t upper_idx(const ReqDev& R, int64_t K) {
  if (K < R.key_base) return 0;
  int64_t b = (K - R.key_base) >> R.bshift;
  if (b >= R.nbuck) return R.n_lines;
  int64_t i = R.bfirst[b];
  while (i < R.n_lines && __ldg(R.key + i) <= K) ++i;
  return i;
}

// Index ranges of the lines whose centre c may lie in one of up to 9 position bands,
// merged into disjoint ranges so that every line is visited once.
struct Bands {
  int64_t lo[9], hi[9];
  int n;
  __device__ __forceinline__ void add(const ReqDev& R, const LevelDev& L, int64_t clo, int64_t chi) {
    int64_t a = lower_idx(R, clo - L.smax);
    int64_t b = upper_idx(R, chi - L.smin);
    if (a < b) {
      lo[n] = a;
      hi[n] = b;
      ++n;
    }
  }
  __device__ __forceinline__ void merge() {
    for (int i = 1; i < n; ++i) {  // insertion sort by lo
      int64_t a = lo[i], b = hi[i];
      int j = i - 1;
      while (j >= 0 && lo[j] > a) {
        lo[j + 1] = lo[j];
        hi[j + 1] = hi[j];
        --j;
      }
      lo[j + 1] = a;
      hi[j + 1] = b;
    }
    int m = 0;
    for (int i = 0; i < n; ++i) {
      if (m > 0 && lo[i] <= hi[m - 1]) {
        hi[m - 1] = max(hi[m - 1], hi[i]);
      } else {
        lo[m] = lo[i];
        hi[m] = hi[i];
        ++m;
      }
    }
    n = m;
  }
};

__device__ __constant__ int64_t kChiBreakFx[3] = {3LL << kFixBits, 150LL << kFixBits,
                                                  300LL << kFixBits};

// Bits i = 0..nb-1 stand for panels base + i; set those in the closed interval [a, b].
__device__ __forceinline__ uint32_t rmask(int64_t a, int64_t b, int64_t base, int nb) {
  int64_t lo = a - base;
  int64_t hi = b - base;
  if (lo < 0) lo = 0;
  if (hi > nb - 1) hi = nb - 1;
  if (lo > hi) return 0u;
  return ((2u << (int)hi) - 1u) & (0xffffffffu << (int)lo);
}

// Panels of grid g accepted for a line, over panels [base, base + nb). With child set,
// the accepted panels of grid g are mapped to their two children on grid g + 1 and
// base/nb refer to grid g + 1.
__device__ __forceinline__ uint32_t accept_mask(int g, int64_t c, int gst, bool chi,
                                                int64_t cut, int R_w, int64_t base, int nb,
                                                bool child) {
  const int s = panel_shift(g);
  const int64_t k = child ? 1 : 0, f = child ? 2 : 1;  // panel a of grid g -> children [2a, 2a+1]
  int64_t s_lo = cl_sh(c - cut, s), s_hi = fl_sh(c + cut, s) - 1;
  uint32_t m = rmask(s_lo * f, s_hi * f + k, base, nb);
  if (!m) return 0u;
  if (gst > g) {
    int64_t R = (int64_t)R_w * step_fx(g);
    int64_t gl = fl_sh(c - R, s), gh = cl_sh(c + R, s) - 1;
    m &= ~rmask(gl * f, gh * f + k, base, nb);
  }
  if (chi) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      int64_t B = kChiBreakFx[b];
      int64_t s1 = c - B, s2 = c + B;
      m &= ~rmask((cl_sh(s1, s) - 1) * f, fl_sh(s1, s) * f + k, base, nb);
      m &= ~rmask((cl_sh(s2, s) - 1) * f, fl_sh(s2, s) * f + k, base, nb);
    }
  }
  return m;
}

// Panels of grid g (1..10) owned by a line over [base, base + nb).
__device__ __forceinline__ uint32_t owned_mask(int g, int64_t c, int gst, bool chi, int64_t cut,
                                               int R_w, int64_t base, int nb) {
  uint32_t m = accept_mask(g, c, gst, chi, cut, R_w, base, nb, false);
  if (g > 1 && m) m &= ~accept_mask(g - 1, c, gst, chi, cut, R_w, base, nb, true);
  return m;
}

__device__ __forceinline__ int clamp32(int64_t v) {
  return (int)max(min(v, (int64_t)(1 << 30)), (int64_t)-(1 << 30));
}

// chi-factor piece thresholds in node units relative to position X0, node spacing 2^sh.
struct ChiThr {
  int r3, r150, r300, l3, l150, l300;
  __device__ __forceinline__ void init(int64_t c, int64_t X0, int sh) {
    r3 = clamp32(cl_sh(c + kChiBreakFx[0] - X0, sh));
    r150 = clamp32(fl_sh(c + kChiBreakFx[1] - X0, sh));
    r300 = clamp32(fl_sh(c + kChiBreakFx[2] - X0, sh));
    l3 = clamp32(fl_sh(c - kChiBreakFx[0] - X0, sh));
    l150 = clamp32(cl_sh(c - kChiBreakFx[1] - X0, sh));
    l300 = clamp32(cl_sh(c - kChiBreakFx[2] - X0, sh));
  }
  // Eq. (10): 1 below 3 cm^-1; 1.084 e^{-0.027|d|} on [3, 150]; 0.208 e^{-0.016|d|} on
  // (150, 300]; 0.025 e^{-0.009|d|} above 300. Branch chosen on the exact node index.
  __device__ __forceinline__ float value(int j, float absd) const {
    int b = (j >= r3) + (j > r150) + (j > r300) + (j <= l3) + (j < l150) + (j < l300);
    if (b == 0) return 1.0f;
    const float C = b == 1 ? 1.084f : (b == 2 ? 0.208f : 0.025f);
    const float r = b == 1 ? 0.027f : (b == 2 ? 0.016f : 0.009f);
    return C * expf(-r * absd);
  }
};

__device__ __forceinline__ float shape_f(int shape, float x, float y) {
  switch (shape) {
    case kShapeVoigt: return voigt_K(x, y);
    case kShapeLorentz: return 1.0f / fmaf(x, x, 1.0f);
    case kShapeDoppler: return expf(-x * x);
    case kShapeConst: return 1.0f;
    default: return fmaf(x, fmaf(x, 0.0625f, 0.25f), 1.0f);  // kShapeQuad
  }
}

// ------------------------------------------------------------------ K1: level prep
__global__ void __launch_bounds__(256) k_level_prep(PrepArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lev = blockIdx.y;
  if (i >= a.n) return;
  const LevelDev L = a.lev[lev];
  const int s = a.species[i];
  const LevelSpeciesDev LS = a.ls[(int64_t)lev * a.n_species + s];
  const double nu0 = a.nu0[i];
  const float S296 = a.S296[i], ga = a.ga[i], gs = a.gs[i], E = a.E[i], na = a.na[i],
              da = a.da[i];
  const int64_t o = (int64_t)lev * a.n + i;

  // centre: rint((nu0 + delta p) 2^43), FP64, no contraction (identical on the host)
  const double nt = __dadd_rn(nu0, __dmul_rn((double)da, L.p));
  a.c[o] = __double2ll_rn(__dmul_rn(nt, kFix));

  // widths and intensity in FP32 (Sec. 2.2)
  const float gL = exp2f(na * L.log2_ratio) * fmaf(ga, L.pf - LS.ps, gs * LS.ps);
  const float aD = (float)nu0 * LS.ad;
  const float arg = E * L.kb_hi;
  const float err = fmaf(E, L.kb_hi, -arg) + E * L.kb_lo;
  const float boltz = expf(arg) * (1.0f + err);
  const float nuf = (float)nu0;
  const float stim = expm1f(-nuf * L.c2_T) / expm1f(-nuf * L.c2_Tref);
  const float S = S296 * LS.F * boltz * stim;

  float amp, sx, y = 0.0f, W;
  const float kSqrtLn2 = 0.83255461115769776f, kSqrtLn2Pi = 0.46971863934982566f;
  switch (a.shape) {
    case kShapeLorentz:
      amp = S * 0.31830988618379067f / gL;
      sx = 1.0f / gL;
      W = gL;
      break;
    case kShapeDoppler:
      amp = S * kSqrtLn2Pi / aD;
      sx = kSqrtLn2 / aD;
      W = aD;
      break;
    default:
      amp = (a.shape == kShapeVoigt) ? S * kSqrtLn2Pi / aD : (a.shape == kShapeConst ? 1.0f : S);
      sx = (a.shape == kShapeVoigt) ? kSqrtLn2 / aD : 1.0f;
      y = kSqrtLn2 * gL / aD;
      W = fmaf(0.5346f, gL, sqrtf(fmaf(0.2166f * gL, gL, aD * aD)));
      if (a.shape != kShapeVoigt) y = 0.0f;
  }
  // g*: coarsest grid with h_g <= W / R_c. Decided in FP32 unless W lies within 1e-5
  // of a threshold, then in FP64 with the operations in the same order as the FP64
  // reference so that both sides take the same integer decision.
  bool near = false;
#pragma unroll
  for (int g = 1; g <= kNGrid; ++g) {
    float thr = ldexpf((float)a.R_c, 1 - g);
    near |= fabsf(W - thr) <= 1e-5f * thr;
  }
  int gs_ = kNGrid + 1;
  if (!near) {
    for (int g = kNGrid; g >= 1; --g)
      if (W >= ldexpf((float)a.R_c, 1 - g)) gs_ = g;
  } else {
    const double gL64 = __dmul_rn(pow(L.ratio, (double)na),
                                  __dadd_rn(__dmul_rn((double)ga, __dsub_rn(L.p, LS.ps_d)),
                                            __dmul_rn((double)gs, LS.ps_d)));
    const double aD64 = __dmul_rn(__ddiv_rn(nu0, 2.99792458e8), LS.sqrtv);
    double W64;
    if (a.shape == kShapeLorentz)
      W64 = gL64;
    else if (a.shape == kShapeDoppler)
      W64 = aD64;
    else
      W64 = __dadd_rn(__dmul_rn(0.5346, gL64),
                      __dsqrt_rn(__dadd_rn(__dmul_rn(__dmul_rn(0.2166, gL64), gL64),
                                           __dmul_rn(aD64, aD64))));
    for (int g = kNGrid; g >= 1; --g)
      if (W64 >= ldexp((double)a.R_c, 1 - g)) gs_ = g;
  }
  a.amp[o] = amp;
  a.sx[o] = sx;
  a.yv[o] = y;
  a.gstar[o] = (int8_t)gs_;
  a.flags[o] = (uint8_t)(LS.chi ? 1 : 0);
}

void launch_level_prep(const PrepArgs& a, int n_levels, cudaStream_t st) {
  dim3 grid((unsigned)((a.n + 255) / 256), (unsigned)n_levels);
  k_level_prep<<<grid, 256, 0, st>>>(a);
}

// ------------------------------------------------------------------ coarse grids
// One warp = a block of kPairs node pairs (even node 2m and odd node 2m+1 for
// m = mb .. mb+kPairs-1) of grid g. Even node 2m carries slot L of panel m and slot R
// of panel m-1, odd node 2m+1 slot M of panel m. The lanes stride over the lines whose
// centres can own a panel of the block; each lane evaluates its line at the block's
// nodes it owns; the lane sums are combined across the warp at the end.
template <bool COUNT>
__global__ void __launch_bounds__(kCoarseWarps * 32)
    k_coarse(const ReqDev* __restrict__ reqs, const CoarseItem* __restrict__ items,
             int64_t* __restrict__ counts) {
  const CoarseItem it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = it.grid;
  const int lev = it.level;
  const int64_t m_first = R.m_first[g];
  const int64_t m_last = m_first + R.npan[g] - 1;
  const int64_t mb = m_first + ((int64_t)it.block0 + warp) * kPairs;
  if (mb > m_last + 1) return;  // whole warp leaves together

  const LevelDev L = R.lev[lev];
  const int s = panel_shift(g);
  const int64_t cut = R.cut_fx;
  const int64_t base = mb - 1;  // mask bit i <-> panel mb - 1 + i
  const int nb = kPairs + 1;
  uint32_t win = rmask(m_first, m_last, base, nb);

  // candidate bands for the centres
  Bands bd;
  bd.n = 0;
  if (g == 1) {
    bd.add(R, L, (base << s) - cut, ((base + nb) << s) + cut);
  } else {
    const int64_t P = int64_t(1) << s;
    const int64_t A = (base >> 1) << (s + 1);
    const int64_t B = (((base + nb - 1) >> 1) + 1) << (s + 1);
    const int64_t Rg1 = (int64_t)R.R_w * step_fx(g - 1);
    bd.add(R, L, A - Rg1 - P, B + Rg1 + P);
    bd.add(R, L, A - cut - P, B - cut + P);
    bd.add(R, L, A + cut - P, B + cut + P);
    if (R.chi_req) {
      for (int b = 0; b < 3; ++b) {
        const int64_t Bk = kChiBreakFx[b];
        if (Bk > cut + (B - A) + P) break;
        bd.add(R, L, A - Bk - P, B - Bk + P);
        bd.add(R, L, A + Bk - P, B + Bk + P);
      }
    }
    bd.merge();
  }

  float sL[kPairs], cL[kPairs], sR[kPairs], cR[kPairs], sM[kPairs], cM[kPairs];
#pragma unroll
  for (int j = 0; j < kPairs; ++j) sL[j] = cL[j] = sR[j] = cR[j] = sM[j] = cM[j] = 0.0f;
  int64_t nev = 0;

  const int64_t lo_off = (int64_t)lev * R.n_lines;
  const int64_t X0 = mb << s;            // position of node 2 mb
  const float to_h = ldexpf(1.0f, 1 - s);  // fixed units -> units of h_g
  const float hg = ldexpf(1.0f, 1 - g);
  const bool physical = R.shape < kShapeConst;

  for (int r = 0; r < bd.n; ++r) {
    for (int64_t i = bd.lo[r] + lane; i < bd.hi[r]; i += 32) {
      const int64_t c = __ldg(R.c + lo_off + i);
      const int gst = __ldg(R.gstar + lo_off + i);
      const bool chi = __ldg(R.flags + lo_off + i) & 1;
      uint32_t own = owned_mask(g, c, gst, chi, cut, R.R_w, base, nb) & win;
      if (!own) continue;
      const float amp = __ldg(R.amp + lo_off + i);
      const float hs = __ldg(R.sx + lo_off + i) * hg;
      const float y = __ldg(R.yv + lo_off + i);
      const float t0 = __ll2float_rn(X0 - c) * to_h;
      ChiThr ct;
      const bool use_chi = chi && physical;
      if (use_chi) ct.init(c, X0, s - 1);
#pragma unroll
      for (int j = 0; j < 2 * kPairs; ++j) {
        const int p = j >> 1;
        const bool oA = (own >> (p + 1)) & 1u;         // L (even) or M (odd) of panel mb+p
        const bool oR = !(j & 1) && ((own >> p) & 1u);  // R of panel mb+p-1 (even only)
        if (!(oA || oR)) continue;
        const float t = t0 + (float)j;
        float v = amp * shape_f(R.shape, t * hs, y);
        if (use_chi) v *= ct.value(j, fabsf(t) * hg);
        if (j & 1) {
          kahan_add(sM[p], cM[p], v);
        } else {
          if (oA) kahan_add(sL[p], cL[p], v);
          if (oR) kahan_add(sR[p], cR[p], v);
        }
        if (COUNT) ++nev;
      }
    }
  }

  float* base_ptr = R.slots + (int64_t)lev * R.slots_per_level + R.slot_off[g];
  const int64_t np = R.npan[g];
#pragma unroll
  for (int j = 0; j < kPairs; ++j) {
    const float vL = warp_sum_comp(sL[j], cL[j]);
    const float vM = warp_sum_comp(sM[j], cM[j]);
    const float vR = warp_sum_comp(sR[j], cR[j]);
    if (lane == j) {
      const int64_t m = mb + j;
      if (m <= m_last) {
        base_ptr[m - m_first] = vL;
        base_ptr[np + (m - m_first)] = vM;
      }
      if (m - 1 >= m_first && m - 1 <= m_last) base_ptr[2 * np + (m - 1 - m_first)] = vR;
    }
  }
  if (COUNT) {
#pragma unroll
    for (int o = 16; o; o >>= 1) nev += __shfl_xor_sync(0xffffffffu, nev, o);
    if (lane == 0) counts[(int64_t)blockIdx.x * kCoarseWarps + warp] = nev;
  }
}

void launch_coarse(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts,
                   cudaStream_t st) {
  if (n_items <= 0) return;
  if (counts)
    k_coarse<true><<<n_items, kCoarseWarps * 32, 0, st>>>(reqs, items, counts);
  else
    k_coarse<false><<<n_items, kCoarseWarps * 32, 0, st>>>(reqs, items, counts);
}

// ------------------------------------------------------------------ finest grid + cascade
// Each thread owns 4 consecutive finest nodes (one G10 panel), sums the lines that the
// finest grid owns there, adds the quadratic interpolants of the ten coarse grids and
// the CTA writes its 1024 outputs with aligned vector stores.
template <bool COUNT>
__global__ void __launch_bounds__(kFineThreads)
    k_fine(const ReqDev* __restrict__ reqs, const FineItem* __restrict__ items,
           int64_t* __restrict__ counts) {
  __shared__ float tile[kFineTile];
  __shared__ int64_t red[kFineThreads / 32];
  const FineItem it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const int lev = it.level;
  const int tid = threadIdx.x;
  const int64_t k0 = it.k0 + (int64_t)kFinePerThread * tid;
  uint32_t valid = 0;
#pragma unroll
  for (int q = 0; q < kFinePerThread; ++q)
    if (k0 + q >= R.k_lo && k0 + q <= R.k_hi) valid |= 1u << q;

  float acc[kFinePerThread], cmp[kFinePerThread];
#pragma unroll
  for (int q = 0; q < kFinePerThread; ++q) acc[q] = cmp[q] = 0.0f;
  int64_t nev = 0;

  if (valid) {
    const LevelDev L = R.lev[lev];
    const int64_t cut = R.cut_fx;
    const int64_t X0 = k0 << kFineShift;
    const int64_t X3 = (k0 + kFinePerThread - 1) << kFineShift;
    const int64_t P10 = int64_t(1) << panel_shift(kNGrid);
    const int64_t R10 = (int64_t)R.R_w * step_fx(kNGrid);
    Bands bd;
    bd.n = 0;
    bd.add(R, L, X0 - R10 - P10, X3 + R10 + P10);
    bd.add(R, L, X0 - cut - P10, X3 - cut + P10);
    bd.add(R, L, X0 + cut - P10, X3 + cut + P10);
    if (R.chi_req) {
      for (int b = 0; b < 3; ++b) {
        const int64_t Bk = kChiBreakFx[b];
        if (Bk > cut + 2 * P10) break;
        bd.add(R, L, X0 - Bk - P10, X3 - Bk + P10);
        bd.add(R, L, X0 + Bk - P10, X3 + Bk + P10);
      }
    }
    bd.merge();
    const int64_t p10 = k0 >> 3;  // the G10 panel of the four nodes
    const int64_t lo_off = (int64_t)lev * R.n_lines;
    const float to_h = ldexpf(1.0f, -kFineShift);
    const float h11 = ldexpf(1.0f, -kFineBits);
    const bool physical = R.shape < kShapeConst;
    for (int r = 0; r < bd.n; ++r) {
      for (int64_t i = bd.lo[r]; i < bd.hi[r]; ++i) {
        const int64_t c = __ldg(R.c + lo_off + i);
        const int gst = __ldg(R.gstar + lo_off + i);
        const bool chi = __ldg(R.flags + lo_off + i) & 1;
        if (accept_mask(kNGrid, c, gst, chi, cut, R.R_w, p10, 1, false)) continue;
        uint32_t own = 0;
#pragma unroll
        for (int q = 0; q < kFinePerThread; ++q) {
          const int64_t d = X0 + ((int64_t)q << kFineShift) - c;
          if ((d < 0 ? -d : d) <= cut) own |= 1u << q;
        }
        own &= valid;
        if (!own) continue;
        const float amp = __ldg(R.amp + lo_off + i);
        const float hs = __ldg(R.sx + lo_off + i) * h11;
        const float y = __ldg(R.yv + lo_off + i);
        const float t0 = __ll2float_rn(X0 - c) * to_h;
        ChiThr ct;
        const bool use_chi = chi && physical;
        if (use_chi) ct.init(c, X0, kFineShift);
#pragma unroll
        for (int q = 0; q < kFinePerThread; ++q) {
          if (!((own >> q) & 1u)) continue;
          const float t = t0 + (float)q;
          float v = amp * shape_f(R.shape, t * hs, y);
          if (use_chi) v *= ct.value(q, fabsf(t) * h11);
          kahan_add(acc[q], cmp[q], v);
          if (COUNT) ++nev;
        }
      }
    }
    // cascade: quadratic through the panel-local L, M, R of every coarse grid
    const float* sl = R.slots + (int64_t)lev * R.slots_per_level;
    float out[kFinePerThread];
#pragma unroll
    for (int q = 0; q < kFinePerThread; ++q) out[q] = acc[q] + cmp[q];
#pragma unroll
    for (int g = 1; g <= kNGrid; ++g) {
      const int sh = 13 - g;  // finest nodes per panel of grid g: 2^(13-g)
      const int64_t m = k0 >> sh;
      const int64_t idx = m - R.m_first[g];
      const int64_t np = R.npan[g];
      const float* gp = sl + R.slot_off[g];
      const float vL = __ldg(gp + idx), vM = __ldg(gp + np + idx), vR = __ldg(gp + 2 * np + idx);
      const int off0 = (int)(k0 - (m << sh));
      const float inv_h = ldexpf(1.0f, 1 - sh);
#pragma unroll
      for (int q = 0; q < kFinePerThread; ++q) {
        const float t = (float)(off0 + q) * inv_h;  // position in steps of h_g, [0, 2)
        const float w0 = (t - 1.0f) * (t - 2.0f) * 0.5f;
        const float w1 = t * (2.0f - t);
        const float w2 = t * (t - 1.0f) * 0.5f;
        out[q] += fmaf(vL, w0, fmaf(vM, w1, vR * w2));
      }
    }
#pragma unroll
    for (int q = 0; q < kFinePerThread; ++q) tile[kFinePerThread * tid + q] = out[q] * R.out_scale;
  }
  __syncthreads();
  // write the valid part [a, b] of the tile
  const int64_t a = max(it.k0, R.k_lo), b = min(it.k0 + kFineTile - 1, R.k_hi);
  if (a <= b) {
    float* row = R.out + (int64_t)lev * R.npts;
    const int64_t i0 = a - R.k_lo;           // first output index
    const int n = (int)(b - a + 1);
    const int t0 = (int)(a - it.k0);         // its position in the tile
    float* dst = row + i0;
    // elements before the first 16-byte boundary
    int head = (int)((16 - ((uintptr_t)dst & 15)) & 15) / 4;
    if (head > n) head = n;
    if (tid < head) dst[tid] = tile[t0 + tid];
    const int nv = (n - head) / 4;
    float4* d4 = reinterpret_cast<float4*>(dst + head);
    for (int v = tid; v < nv; v += kFineThreads) {
      const int e = t0 + head + 4 * v;
      d4[v] = make_float4(tile[e], tile[e + 1], tile[e + 2], tile[e + 3]);
    }
    const int done = head + 4 * nv;
    if (tid < n - done) dst[done + tid] = tile[t0 + done + tid];
  }
  if (COUNT) {
#pragma unroll
    for (int o = 16; o; o >>= 1) nev += __shfl_xor_sync(0xffffffffu, nev, o);
    if ((tid & 31) == 0) red[tid >> 5] = nev;
    __syncthreads();
    if (tid == 0) {
      int64_t t = 0;
      for (int w = 0; w < kFineThreads / 32; ++w) t += red[w];
      counts[blockIdx.x] = t;
    }
  }
}

void launch_fine(const ReqDev* reqs, const FineItem* items, int n_items, int64_t* counts,
                 cudaStream_t st) {
  if (n_items <= 0) return;
  if (counts)
    k_fine<true><<<n_items, kFineThreads, 0, st>>>(reqs, items, counts);
  else
    k_fine<false><<<n_items, kFineThreads, 0, st>>>(reqs, items, counts);
}

// ------------------------------------------------------------------ diagnostics
__global__ void k_diag_voigt(const float* x, const float* y, float* out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = voigt_K(x[i], y[i]);
}

void launch_diag_voigt(const float* x, const float* y, float* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  k_diag_voigt<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, out, n);
}

__global__ void k_diag_owned(const ReqDev* __restrict__ req, int lev, int grid, int64_t first,
                             int count, uint8_t* out) {
  const ReqDev& R = *req;
  const int64_t line = blockIdx.x;
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= count || line >= R.n_lines) return;
  const int64_t o = (int64_t)lev * R.n_lines + line;
  const int64_t c = R.c[o];
  const int gst = R.gstar[o];
  const bool chi = R.flags[o] & 1;
  uint8_t v;
  if (grid <= kNGrid) {
    v = owned_mask(grid, c, gst, chi, R.cut_fx, R.R_w, first + i, 1) & 1u;
  } else {
    const int64_t k = first + i;
    const int64_t d = (k << kFineShift) - c;
    const bool within = (d < 0 ? -d : d) <= R.cut_fx;
    v = within && !accept_mask(kNGrid, c, gst, chi, R.cut_fx, R.R_w, k >> 3, 1, false);
  }
  out[line * (int64_t)count + i] = v;
}

void launch_diag_owned(const ReqDev* req, int64_t n_lines, int level, int grid, int64_t first,
                       int count, uint8_t* out, cudaStream_t st) {
  if (count <= 0 || n_lines <= 0) return;
  dim3 gr((unsigned)n_lines, (unsigned)((count + 127) / 128));
  k_diag_owned<<<gr, 128, 0, st>>>(req, level, grid, first, count, out);
}

}  // namespace marfa

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
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "marfa_internal.cuh"
#include "ownership.cuh"
#include "mlp.cuh"
#include "voigt.cuh"

namespace marfa {

// ------------------------------------------------------------------ device-side checks
#ifdef MARFA_DEBUG
static __device__ unsigned g_marfa_status = 0;
__device__ bool marfa_dcheck_fail(unsigned code) {
  atomicCAS(&g_marfa_status, 0u, code);
  return false;
}
#endif

int device_check_status(unsigned* code, bool clear) {
  *code = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return -3;  // MARFA_E_CUDA
#ifdef MARFA_DEBUG
  if (cudaMemcpyFromSymbol(code, g_marfa_status, sizeof(unsigned)) != cudaSuccess) return -3;
  if (clear && *code) {
    const unsigned zero = 0;
    if (cudaMemcpyToSymbol(g_marfa_status, &zero, sizeof(unsigned)) != cudaSuccess) return -3;
  }
#else
  (void)clear;
#endif
  return 0;
}

// The probe of the checks: a store at index i of a 32-entry shared array, made only when
// i is in range (in a MARFA_DEBUG build an index out of range records code 901).
__global__ void k_diag_check(int i, int* sink) {
  __shared__ int a[32];
  a[threadIdx.x] = 0;
  __syncwarp();
  if (i >= 0 && i < 32 && MARFA_DCHECK(true, 901)) a[i] = 1;
  else (void)MARFA_DCHECK(false, 901);
  __syncwarp();
  if (a[threadIdx.x] && sink) *sink = 1;
}

void launch_diag_check(int i, cudaStream_t st) { k_diag_check<<<1, 32, 0, st>>>(i, nullptr); }

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
// merged into disjoint ranges so that every line is visited once. The 2 n boundary
// lookups run in parallel, one per lane of a converged warp.
struct Bands {
  int64_t lo[9], hi[9];
  int n;
  // zone z: lines with c in [zlo[z], zhi[z]] (fixed point); the shift bounds of the
  // level turn the centre range into a conservative key range.
  __device__ __forceinline__ void lookup(const ReqDev& R, const LevelDev& L, const int64_t* zlo,
                                         const int64_t* zhi, int nz) {
    const int lane = threadIdx.x & 31;
    int64_t v = 0;
    if (lane < 2 * nz) {
      const int z = lane >> 1;
      v = (lane & 1) ? upper_idx(R, zhi[z] - L.smin) : lower_idx(R, zlo[z] - L.smax);
    }
    n = 0;
    for (int z = 0; z < nz; ++z) {
      const int64_t a = __shfl_sync(0xffffffffu, v, 2 * z);
      const int64_t b = __shfl_sync(0xffffffffu, v, 2 * z + 1);
      if (a < b) {
        lo[n] = a;
        hi[n] = b;
        ++n;
      }
    }
    merge();
#ifdef MARFA_DEBUG
    for (int r = 0; r < n; ++r)
      if (!MARFA_DCHECK(lo[r] >= 0 && lo[r] <= hi[r] && hi[r] <= R.n_lines, 401)) n = 0;
#endif
  }
  // All candidates of the bands as one sequence 0 .. total-1, so that a loop over them
  // by a block or a warp leaves idle lanes only in its last round.
  __device__ __forceinline__ int64_t total() const {
    int64_t t = 0;
    for (int r = 0; r < n; ++r) t += hi[r] - lo[r];
    return t;
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


// Maps increasing positions t of the flattened candidate sequence of a Bands to line
// indices (each thread walks forward through the bands).
struct BandCursor {
  int r = 0;
  int64_t start = 0;  // position of band r's first line in the sequence
  __device__ __forceinline__ int64_t line(const Bands& bd, int64_t t) {
    while (t - start >= bd.hi[r] - bd.lo[r]) {
      start += bd.hi[r] - bd.lo[r];
      ++r;
    }
    return bd.lo[r] + (t - start);
  }
};

// The same walk over bands copied to shared memory (the CTA's copy, sb): the current
// band's bounds stay in registers and only a band change reads shared memory, so the
// per-candidate walk makes no local-memory access.
struct SharedBandCursor {
  int r = 0;
  int64_t start = 0, blo = 0, blen = 0;
  __device__ __forceinline__ void init(const int64_t* sb_lo, const int64_t* sb_hi, int n) {
    if (n > 0) {
      blo = sb_lo[0];
      blen = sb_hi[0] - sb_lo[0];
    }
  }
  __device__ __forceinline__ int64_t line(const int64_t* sb_lo, const int64_t* sb_hi, int64_t t) {
    while (t - start >= blen) {
      start += blen;
      ++r;
      blo = sb_lo[r];
      blen = sb_hi[r] - sb_lo[r];
    }
    return blo + (t - start);
  }
};

// Position zones where a line centre must lie for the line to own something in the
// span [A, B]: within Rc of it (centre), at the cut-off distance (edges) or at a chi
// breakpoint distance (kinks), each widened by the margin P.
__device__ __forceinline__ int make_zones(int64_t A, int64_t B, int64_t Rc, int64_t cut, int64_t P,
                                          bool chi, int64_t* zlo, int64_t* zhi) {
  int nz = 0;
  zlo[nz] = A - Rc - P; zhi[nz] = B + Rc + P; ++nz;
  zlo[nz] = A - cut - P; zhi[nz] = B - cut + P; ++nz;
  zlo[nz] = A + cut - P; zhi[nz] = B + cut + P; ++nz;
  if (chi) {
    for (int b = 0; b < 3; ++b) {
      const int64_t Bk = chi_break_fx(b);
      if (Bk > cut + (B - A) + P) break;
      zlo[nz] = A - Bk - P; zhi[nz] = B - Bk + P; ++nz;
      zlo[nz] = A + Bk - P; zhi[nz] = B + Bk + P; ++nz;
    }
  }
  return nz;
}

// A node index relative to a tile, clamped to int16 (comparisons with indices 0..4095 keep
// their outcome).
__device__ __forceinline__ int16_t clamp_node16(int v) { return (int16_t)max(min(v, 4096), -4096); }

// Lowest and highest set bit of a non-zero panel mask.
__device__ __forceinline__ int mask_lowest(uint32_t m) { return __ffs((int)m) - 1; }
__device__ __forceinline__ int mask_lowest(uint64_t m) { return __ffsll((long long)m) - 1; }
__device__ __forceinline__ int mask_highest(uint32_t m) { return 31 - __clz((int)m); }
__device__ __forceinline__ int mask_highest(uint64_t m) { return 63 - __clzll((long long)m); }

__device__ __forceinline__ int clamp32(int64_t v) {
  return (int)max(min(v, (int64_t)(1 << 30)), (int64_t)-(1 << 30));
}

// chi-factor piece thresholds in node units relative to position X0, node spacing 2^sh.
struct ChiThr {
  int r3, r150, r300, l3, l150, l300;
  bool near = false;  // only r3 and l3 can be crossed (set by init)
  // cut: the request's cut-off. The nodes a line contributes to lie within its cut-off
  // (an owned panel lies wholly inside it); when the cut-off stays short of the 150 cm^-1
  // breakpoint (by a margin of 8 cm^-1), the two outer thresholds on each side are never
  // crossed and are set out of reach instead of computed.
  __device__ __forceinline__ void init(int64_t c, int64_t X0, int sh, int64_t cut) {
    r3 = clamp32(cl_sh(c + chi_break_fx(0) - X0, sh));
    l3 = clamp32(fl_sh(c - chi_break_fx(0) - X0, sh));
    near = cut + (int64_t(8) << kFixBits) <= chi_break_fx(1);
    if (near) {
      r150 = r300 = 1 << 30;
      l150 = l300 = -(1 << 30);
      return;
    }
    r150 = clamp32(fl_sh(c + chi_break_fx(1) - X0, sh));
    r300 = clamp32(fl_sh(c + chi_break_fx(2) - X0, sh));
    l150 = clamp32(cl_sh(c - chi_break_fx(1) - X0, sh));
    l300 = clamp32(cl_sh(c - chi_break_fx(2) - X0, sh));
  }
  __device__ __forceinline__ int branch(int j) const {
    if (near) return (j >= r3) + (j <= l3);
    return (j >= r3) + (j > r150) + (j > r300) + (j <= l3) + (j < l150) + (j < l300);
  }
  // The branch is the same at every node of [ja, jb] (it changes only at j = r3,
  // r150 + 1, r300 + 1, l3 + 1, l150, l300).
  __device__ __forceinline__ bool uniform(int ja, int jb) const {
    auto in = [&](int t) { return t > ja && t <= jb; };
    if (near) return !(in(r3) || in(l3 + 1));
    return !(in(r3) || in(r150 + 1) || in(r300 + 1) || in(l3 + 1) || in(l150) || in(l300));
  }
  // Eq. (10): 1 below 3 cm^-1; 1.084 e^{-0.027|d|} on [3, 150]; 0.208 e^{-0.016|d|} on
  // (150, 300]; 0.025 e^{-0.009|d|} above 300. Branch chosen on the exact node index.
  __device__ __forceinline__ float value(int j, float absd) const {
    int b = branch(j);
    if (b == 0) return 1.0f;
    const float C = b == 1 ? 1.084f : (b == 2 ? 0.208f : 0.025f);
    const float r = b == 1 ? 0.027f : (b == 2 ? 0.016f : 0.009f);
    return C * __expf(-r * absd);
  }
  // The same without a branch (the exponential always taken, 1 selected where the branch
  // is 0): cheaper where the lanes of a warp fall on both sides of a breakpoint.
  __device__ __forceinline__ float value_sel(int j, float absd) const {
    const int b = branch(j);
    const float C = b == 1 ? 1.084f : (b == 2 ? 0.208f : 0.025f);
    const float r = b == 1 ? 0.027f : (b == 2 ? 0.016f : 0.009f);
    const float e = C * __expf(-r * absd);
    return b == 0 ? 1.0f : e;
  }
};

// chi-factor along the nodes ja, ja + 1, ... of one line when its branch is the same at
// all of them (ChiThr::uniform): chi(ja) once, and a constant ratio per node step
// (e^{-r h} on the side right of the centre, e^{+r h} on the left), so that node ja + k
// costs one exp2 (at(k)); lr = log2 of the ratio, 0 where chi = 1.
struct ChiRun {
  float v = 1.0f, ratio = 1.0f, lr = 0.0f;  // chi at node ja, ratio per node step
  __device__ __forceinline__ void init(const ChiThr& ct, int ja, float absd_a, int sh) {
    const int b = ct.branch(ja);
    if (b == 0) {
      v = 1.0f;
      ratio = 1.0f;
      lr = 0.0f;
      return;
    }
    const float C = b == 1 ? 1.084f : (b == 2 ? 0.208f : 0.025f);
    const float r = b == 1 ? 0.027f : (b == 2 ? 0.016f : 0.009f);
    v = C * __expf(-r * absd_a);
    const float h = ldexpf(1.0f, sh - kFixBits);  // node step, cm^-1
    const float rh = (ja >= ct.r3 ? -r : r) * h;
    ratio = __expf(rh);
    lr = rh * 1.4426950408889634f;
  }
  // chi at node ja + k
  __device__ __forceinline__ float at(int k) const { return lr != 0.0f ? v * exp2f(lr * (float)k) : v; }
};

// Position of the nodes of a line relative to its centre: with rel = X0 - c (fixed
// point) and node spacing 2^sh units, node j sits at (j + q + phi) steps, q integer,
// phi in [0, 1). Then x_j = ((j + q) + phi) * hs with hs = sx * step is formed as
// fma(j + q, hs, phi * hs): j + q is exact in FP32 and only one rounding remains.
// Both conversions stay in 32 bits (64-bit integer conversions run on the FP64 pipe):
// q is a node count below 2^31 (tiles lie within the cut-off, <= 1000 cm^-1, of a
// candidate line), and phi is taken from the top 31 bits of the remainder (sh >= 32),
// rounded to FP32 (error <= 2^-25 + 2^-31 of a step).
struct NodeX {
  float qf, hs, phs, phi;
  __device__ __forceinline__ void init(int64_t rel, int sh, float sx) {
    const int64_t q = fl_sh(rel, sh);
    phi = __int2float_rn((int)((rel - (q << sh)) >> (sh - 31))) * 0x1p-31f;
    qf = __int2float_rn((int)q);
    hs = sx * ldexpf(1.0f, sh - kFixBits);
    phs = phi * hs;
  }
  __device__ __forceinline__ float x(float jf) const { return fmaf(jf + qf, hs, phs); }
  // |nu - nu~0| in cm^-1 at node j
  __device__ __forceinline__ float absd(float jf, int sh) const {
    return fabsf((jf + qf) + phi) * ldexpf(1.0f, sh - kFixBits);
  }
};

// ------------------------------------------------------------------ line shapes
// The paper lets a user redirect the line shape to any function (its procedure-pointer
// hook, Sec. 2.2). Here every shape is g(x, y) in the shape's own scaled variable x (the
// level preparation sets the amplitude and the x scale per shape): Lorentz 1/(1 + x^2),
// Voigt K(x, y), Doppler exp(-x^2), the paper's fast Voigt, and the user's shape. The
// user's shape g(x) is given as n samples over [0, x_max] (symmetric in x), linear
// between samples and g(x_max) (x_max / x)^2 beyond, on the Lorentz scaling
// x = (nu - nu~0) / gamma_L with the Lorentz amplitude S / (pi gamma_L) (the Lorentz
// itself is g = 1/(1 + x^2)). The kernels evaluate K inline and reach the other shapes
// through shape_f, a switch over direct calls: a table of device function pointers
// would serve as well, but an indirect call site makes ptxas budget the kernel for any
// target (grid 1's kernel went from 80 to 177 registers, a third of its occupancy).
__device__ float g_user_tab[kUserShapeMax];
__device__ int g_user_n = 0;
__device__ float g_user_xmax = 1.0f, g_user_scale = 1.0f;  // scale = (n - 1) / x_max

static __device__ __noinline__ float shape_user(float x) {
  const float ax = fabsf(x);
  const int n = g_user_n;
  if (ax >= g_user_xmax) {
    const float r = g_user_xmax / ax;
    return g_user_tab[n - 1] * r * r;
  }
  const float t = ax * g_user_scale;
  const int i = min((int)t, n - 2);
  const float f = t - (float)i;
  return fmaf(f, g_user_tab[i + 1] - g_user_tab[i], g_user_tab[i]);
}

__device__ __forceinline__ float shape_f(int shape, float x, float y) {
  switch (shape) {
    case kShapeVoigt: return voigt_K(x, y);
    case kShapeVoigtPaper: return voigt_K_paper_call(x, y);
    case kShapeLorentz: return 1.0f / fmaf(x, x, 1.0f);
    case kShapeDoppler: return expf(-x * x);
    case kShapeUser: return shape_user(x);
    case kShapeConst: return 1.0f;
    case kShapeQuart: return fmaf(x, fmaf(x, fmaf(x, fmaf(x, 0.00390625f, 0.015625f), 0.0625f), 0.25f), 1.0f);
    default: return fmaf(x, fmaf(x, 0.0625f, 0.25f), 1.0f);  // kShapeQuad
  }
}

int set_user_shape(const float* g, int n, float x_max) {
  const float scale = (float)(n - 1) / x_max;
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(g_user_tab, g, sizeof(float) * n)) ||
      (e = cudaMemcpyToSymbol(g_user_n, &n, sizeof(int))) ||
      (e = cudaMemcpyToSymbol(g_user_xmax, &x_max, sizeof(float))) ||
      (e = cudaMemcpyToSymbol(g_user_scale, &scale, sizeof(float))))
    return (int)e;
  return 0;
}

// Per-CTA evaluation counts, kCountFields per block: all profile evaluations, those the
// surrogate took, and the plain Voigt evaluations in 9 x 9 polynomial cells (cost class
// 2), in the asymptotic series (class 1) and in small-y cells (class 3).
template <int NW>
__device__ __forceinline__ void block_counts(int64_t nev, int64_t nmlp, int64_t nnear, int64_t nmid,
                                             int64_t nsmall, int64_t (*red)[NW], int64_t* counts) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t v[kCountFields] = {nev, nmlp, nnear, nmid, nsmall};
#pragma unroll
  for (int i = 0; i < kCountFields; ++i) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if (lane == 0) red[i][warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < kCountFields) {
    int64_t t = 0;
    for (int w = 0; w < NW; ++w) t += red[threadIdx.x][w];
    counts[kCountFields * (int64_t)blockIdx.x + threadIdx.x] = t;
  }
}

// One counted evaluation at (x, y) (COUNT variants only).
template <bool COUNT>
__device__ __forceinline__ void count_eval(bool voigt, float x, float y, int64_t& nev, int64_t& nnear,
                                           int64_t& nmid, int64_t& nsmall) {
  if (!COUNT) return;
  ++nev;
  if (voigt) {
    const int c = voigt_class(x, y);
    nnear += c == 2 ? 1 : 0;
    nmid += c == 1 ? 1 : 0;
    nsmall += c == 3 ? 1 : 0;
  }
}

// Raise a kernel's dynamic shared-memory limit to `bytes` once per kernel, device and size.
static void dyn_smem_optin(const void* k, size_t bytes) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, bool> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(k, dev, bytes);
  if (done.count(key)) return;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  done[key] = true;
}

// Launch with `bytes` of dynamic shared memory.
template <class... KA, class... A>
static void launch_dyn(void (*k)(KA...), int n_items, int threads, size_t bytes, cudaStream_t st,
                       A... args) {
  dyn_smem_optin(reinterpret_cast<const void*>(k), bytes);
  k<<<n_items, threads, bytes, st>>>(args...);
}

// Dynamic shared memory of the surrogate part: the network weights and one queue per warp.
constexpr size_t surr_bytes(int threads) {
  return sizeof(MlpWeights) + (size_t)(threads / 32) * sizeof(SurrQueue);
}

// Launch a surrogate-capable kernel with the network weights and one queue per warp in
// dynamic shared memory.
template <class... KA, class... A>
static void launch_surr(void (*k)(KA...), int n_items, int threads, cudaStream_t st, A... args) {
  launch_dyn(k, n_items, threads, surr_bytes(threads), st, args...);
}

// ------------------------------------------------------------------ K1: level prep
// The per-(level, line) data of line i at level lev.
// rint(t 2^43) (round half to even) for a finite double t, from its bits: |t| 2^43 =
// m 2^(e - 9) with m the 53-bit significand and e the unbiased exponent, so the product
// is exact and only a right shift rounds. Equal to __double2ll_rn(t * 2^43) for every
// finite t with |t| 2^43 < 2^62, without instructions of the FP64 pipe.
__device__ __forceinline__ int64_t fix43_rint(double t) {
  const uint64_t b = (uint64_t)__double_as_longlong(t);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero or subnormal: |t| 2^43 < 2^-979
  const uint64_t m = (b & ((uint64_t(1) << 52) - 1)) | (uint64_t(1) << 52);
  const int sh = ex - 1023 - 9;
  uint64_t q = 0;
  if (sh >= 0) {
    q = m << sh;
  } else if (sh >= -53) {
    const int k = -sh;
    q = m >> k;
    const uint64_t r = m & ((uint64_t(1) << k) - 1), half = uint64_t(1) << (k - 1);
    q += (r > half || (r == half && (q & 1))) ? 1 : 0;
  }  // else |t| 2^43 < 1/2
  return (b >> 63) ? -(int64_t)q : (int64_t)q;
}

__device__ __forceinline__ void level_prep_pair(const PrepArgs& a, int64_t i, int lev) {
  const LevelDev L = a.lev[lev];
  const int s = a.species[i];
  const LevelSpeciesDev LS = a.ls[(int64_t)lev * a.n_species + s];
  const double nu0 = a.nu0[i];
  const float S296 = a.S296[i], ga = a.ga[i], gs = a.gs[i], E = a.E[i], na = a.na[i],
              da = a.da[i];
  const int64_t o = (int64_t)lev * a.n + i;

  // centre: rint((nu0 + delta p) 2^43), FP64, no contraction (identical on the host);
  // the scaling by 2^43 and the rounding to an integer from the bits of the sum
  const double nt = __dadd_rn(nu0, __dmul_rn((double)da, L.p));
  a.c[o] = fix43_rint(nt);

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
    case kShapeUser:  // the user's shape on the Lorentz scaling
      amp = S * 0.31830988618379067f / gL;
      sx = 1.0f / gL;
      W = gL;
      break;
    case kShapeDoppler:
      amp = S * kSqrtLn2Pi / aD;
      sx = kSqrtLn2 / aD;
      W = aD;
      break;
    default: {
      const bool vgt = a.shape == kShapeVoigt || a.shape == kShapeVoigtPaper;
      amp = vgt ? S * kSqrtLn2Pi / aD : (a.shape == kShapeConst ? 1.0f : S);
      sx = vgt ? kSqrtLn2 / aD : 1.0f;
      y = kSqrtLn2 * gL / aD;
      W = fmaf(0.5346f, gL, sqrtf(fmaf(0.2166f * gL, gL, aD * aD)));
      if (!vgt) y = 0.0f;
    }
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
    if (a.shape == kShapeLorentz || a.shape == kShapeUser)
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

__global__ void __launch_bounds__(256) k_level_prep(PrepArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) level_prep_pair(a, i, blockIdx.y);
}

// All requests of a batch in one launch: block b belongs to the last request r with
// first[r] <= b, whose blocks run over its levels (outer) and 256-line chunks (inner).
__global__ void __launch_bounds__(256) k_level_prep_batch(const PrepArgs* __restrict__ args,
                                                          const int64_t* __restrict__ first, int n_req) {
  const int64_t b = blockIdx.x;
  int lo = 0, hi = n_req - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const PrepArgs a = args[lo];
  const int64_t local = b - first[lo], nb = (a.n + 255) / 256;
  const int lev = (int)(local / nb);
  const int64_t i = (local - lev * nb) * 256 + threadIdx.x;
  if (i < a.n) level_prep_pair(a, i, lev);
}

void launch_level_prep(const PrepArgs& a, int n_levels, cudaStream_t st) {
  dim3 grid((unsigned)((a.n + 255) / 256), (unsigned)n_levels);
  k_level_prep<<<grid, 256, 0, st>>>(a);
}

void launch_level_prep_batch(const PrepArgs* args, const int64_t* first, int n_req, int64_t blocks,
                             cudaStream_t st) {
  if (n_req <= 0 || blocks <= 0) return;
  k_level_prep_batch<<<(unsigned)blocks, 256, 0, st>>>(args, first, n_req);
}

// ------------------------------------------------------------------ grid 1
// Grid 1 (1 cm^-1 step) carries the long cut-off tails of every line and most of the
// profile evaluations. A CTA owns kG1Pairs consecutive node pairs of one level: lane p
// of every warp holds pair p (even node 2m, odd node 2m+1; a tile the window covers only
// in part may fold four lines onto the lanes instead, see k_g1), and the 8 warps split the
// candidate lines, which are staged in shared memory and read by broadcast. For a line
// whose tile nodes are all in the far Voigt wing (|z| >= 100) the profile is the two-term
// series y/(sqrt(pi) r^2)(1 + (3x^2 - y^2)/(2 r^4)), and the chi-factor of branch 1 is a
// per-line factor times a per-node constant exp(-0.027 |j|); other lines take the exact path.
__device__ __noinline__ float2 g1_exact_pair(const ReqDev& R, int64_t o, int64_t X0, int j0,
                                            bool need0, bool need1, int& n_near, int& n_mid,
                                            int& n_small) {
  const int sh = panel_shift(1) - 1;
  const int64_t c = __ldg(R.c + o);
  const float amp = __ldg(R.amp + o), sx = __ldg(R.sx + o), y = __ldg(R.yv + o);
  const bool use_chi = (__ldg(R.flags + o) & 1) && R.shape < kShapeConst;
  NodeX nx;
  nx.init(X0 - c, sh, sx);
  ChiThr ct;
  if (use_chi) ct.init(c, X0, sh, R.cut_fx);
  float v[2] = {0.0f, 0.0f};
  for (int q = 0; q < 2; ++q) {
    if (!(q ? need1 : need0)) continue;
    const int j = j0 + q;
    const float jf = (float)j, xv = nx.x(jf);
    const bool voigt = R.shape == kShapeVoigt;
    float f = amp * (voigt ? voigt_K(xv, y) : shape_f(R.shape, xv, y));
    if (use_chi) f *= ct.value(j, nx.absd(jf, sh));
    v[q] = f;
    const int cl = voigt ? voigt_class(xv, y) : 0;
    n_near += cl == 2 ? 1 : 0;
    n_mid += cl == 1 ? 1 : 0;
    n_small += cl == 3 ? 1 : 0;
  }
  return make_float2(v[0], v[1]);
}

// The exact-path nodes j0, j0 + 1 of a grid-1 line for the surrogate variant: x at both
// nodes, y, and the weights amp * chi.
struct G1Nodes {
  float x0, x1, y, w0, w1;
};
__device__ __noinline__ G1Nodes g1_exact_nodes(const ReqDev& R, int64_t o, int64_t X0, int j0) {
  const int sh = panel_shift(1) - 1;
  const int64_t c = __ldg(R.c + o);
  const float amp = __ldg(R.amp + o), sx = __ldg(R.sx + o);
  const bool use_chi = (__ldg(R.flags + o) & 1) && R.shape < kShapeConst;
  NodeX nx;
  nx.init(X0 - c, sh, sx);
  G1Nodes r;
  r.y = __ldg(R.yv + o);
  r.x0 = nx.x((float)j0);
  r.x1 = nx.x((float)(j0 + 1));
  r.w0 = r.w1 = amp;
  if (use_chi) {
    ChiThr ct;
    ct.init(c, X0, sh, R.cut_fx);
    r.w0 = amp * ct.value(j0, nx.absd((float)j0, sh));
    r.w1 = amp * ct.value(j0 + 1, nx.absd((float)(j0 + 1), sh));
  }
  return r;
}

__device__ __forceinline__ void comp_merge(float& s, float& c, float s2, float c2) {
  const float t = s + s2;
  const float bp = t - s;
  const float e = (s - (t - bp)) + (s2 - bp);
  s = t;
  c = (c + c2) + e;
}

// WIDE: 0 the paper's 3-point partition, 1 the 5-point variant, 2 either, per request
// (counting and surrogate variants).
template <bool COUNT, bool SURR, int WIDE>
__global__ void __launch_bounds__(kG1Warps * 32)
    k_g1(const ReqDev* __restrict__ reqs, const G1Item* __restrict__ items,
         int64_t* __restrict__ counts) {
  extern __shared__ __align__(16) unsigned char dsm[];  // surrogate weights and queues (SURR only)
  MlpWeights& S = *reinterpret_cast<MlpWeights*>(dsm);
  __shared__ float4 sA[kG1Batch];               // q, sx, phi*sx, y^2
  __shared__ float4 sB[kG1Batch];               // a_centre, a_left, a_right, -y^2/2
  __shared__ unsigned long long sM[kG1Batch];   // owned panels m0-1 .. m0+31
  __shared__ int4 sC[kG1Batch];                 // j_left3, j_right3, exact-path flag, -
  __shared__ float sRed[kG1Warps][8][32];
  __shared__ int64_t sCnt[kCountFields][kG1Warps];
  const G1Item it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const bool wide = WIDE == 2 ? R.wide != 0 : WIDE == 1;  // 5-point partition
  const bool use_mlp = SURR && R.mlp != nullptr;  // block-uniform
  if (use_mlp) mlp_load_smem(S, R.mlp);  // made visible by the first barrier below
  const int lev = it.level;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = panel_shift(1);  // panel 2 cm^-1 = 2^44 units; nodes every 2^43
  const int64_t m_first = R.m_first[1], m_last = m_first + R.npan[1] - 1;
  const int64_t m0 = it.m0, base = m0 - 1;
  const int nb = kG1Pairs + 1;
  const uint64_t win = rmask<uint64_t>(m_first, m_last, base, nb);
  const uint64_t full_tile = (2ull << (nb - 1)) - 1ull;  // all nb panels (tile inside the window)
  const int64_t X0 = m0 << s;  // node 2 m0
  const int64_t cut = R.cut_fx;
  const LevelDev L = R.lev[lev];
  Bands bd;
  {
    const int64_t Pw = wide ? (int64_t(1) << (s + 1)) : 0;  // a four-step panel may overhang the tile
    const int64_t zlo = (base << s) - cut - Pw, zhi = ((m0 + kG1Pairs) << s) + cut + Pw;
    bd.lookup(R, L, &zlo, &zhi, 1);
  }
  // this CTA's share of the candidate lines
  const int64_t c_lo = bd.n ? bd.lo[0] : 0, c_n = bd.n ? bd.hi[0] - c_lo : 0;
  const int64_t i_lo = c_lo + c_n * it.part / R.g1_split, i_hi = c_lo + c_n * (it.part + 1) / R.g1_split;
  const int64_t off = (int64_t)lev * R.n_lines;
  const bool voigt = R.shape == kShapeVoigt;
  const bool physical = R.shape < kShapeConst;

  // Lane mapping. Normally lane = pair and a warp takes one staged line at a time. A tile
  // of which the window covers at most 8 pairs, pw0 .. pw1 (the other lanes would idle),
  // takes 4 lines at a time instead: lane = (line slot lane / 8, pair pw0 + lane % 8); the
  // four slots' sums are merged before the per-warp reduction.
  const int64_t bw0 = max(m_first - base, (int64_t)0), bw1 = min(m_last - base, (int64_t)(nb - 1));
  const int pw0 = (int)max(bw0 - 1, (int64_t)0), pw1 = (int)min(bw1, (int64_t)(kG1Pairs - 1));
  const bool narrow = !use_mlp && pw1 - pw0 < 8;  // block-uniform
  float eS = 0.f, eC = 0.f, lS = 0.f, lC = 0.f, rS = 0.f, rC = 0.f, mS = 0.f, mC = 0.f;
  int64_t nev = 0, nmlp = 0, nnear = 0, nmid = 0, nsmall = 0;
  if (use_mlp) __syncthreads();
  int qn = 0;  // entries in this warp's surrogate queue (warp-uniform)

  // the sums over the candidate lines, compiled once for each lane mapping
  auto sum_lines = [&](auto narrow_tag) {
    constexpr bool NARROW = decltype(narrow_tag)::value;
    constexpr int n_slot = NARROW ? 4 : 1;
    const int slot = NARROW ? lane >> 3 : 0;
    const int p = NARROW ? pw0 + (lane & 7) : lane, j0 = 2 * p;
    const float f0 = (float)j0, f1 = (float)(j0 + 1);
    const float rR0 = expf(-0.027f * f0), rR1 = expf(-0.027f * f1);
    const float rL0 = expf(0.027f * f0), rL1 = expf(0.027f * f1);
    for (int64_t b0 = i_lo; b0 < i_hi; b0 += kG1Batch) {
      const int nbat = (int)min((int64_t)kG1Batch, i_hi - b0);
      __syncthreads();
      for (int k = tid; k < nbat; k += kG1Warps * 32) {
        const int64_t o = off + b0 + k;
        const int64_t c = __ldg(R.c + o);
        const int gst = __ldg(R.gstar + o);
        const bool chi = __ldg(R.flags + o) & 1;
        // acceptance panels: two steps of grid 1, or four in the 5-point variant
        const uint64_t msk = accept_mask_s<uint64_t>(1, c, gst, chi, cut, R.R_w, base, nb, s + wide, s) & win;
        const float amp = __ldg(R.amp + o), sx = __ldg(R.sx + o), y = __ldg(R.yv + o);
        NodeX nx;
        nx.init(X0 - c, s - 1, sx);
        // distance from the centre to the nearest node of the owned panels (bit b <-> panel
        // base + b, nodes 2(base + b) .. 2(base + b) + 2): the owned panels nearest to c
        // below and above it bound it from below
        int64_t dn = 0;
        if (msk) {
          const int64_t pc = fl_sh(c, s) - base;  // panel holding c, relative to base
          const uint64_t below = pc <= 0 ? 0ull : (pc >= nb ? msk : msk & ((1ull << pc) - 1ull));
          const uint64_t above = pc < 0 ? msk : (pc >= nb - 1 ? 0ull : msk & ~((2ull << pc) - 1ull));
          const bool inside = pc >= 0 && pc < nb && ((msk >> pc) & 1ull);
          int64_t d1 = INT64_MAX, d2 = INT64_MAX;
          if (below) d1 = c - ((base + (63 - __clzll((long long)below)) + 1) << s);  // end of that panel
          if (above) d2 = ((base + (__ffsll((long long)above) - 1)) << s) - c;       // start of that panel
          dn = inside ? 0 : min(d1, d2);
        }
        // dn < 2^62: its top 31 bits suffice for the far-wing test (32-bit conversion)
        const bool far = voigt && (__int2float_rn((int)(dn >> 31)) * ldexpf(1.0f, 31 - kFixBits) * sx >= 100.0f ||
                                   y >= 100.0f);
        int jL = -(1 << 30), jR = 1 << 30;
        bool exact = !far;
        const float aC = amp * y * kInvSqrtPi;
        float aL = aC, aR = aC;
        if (chi && physical) {
          jR = clamp32(cl_sh(c + chi_break_fx(0) - X0, s - 1));
          jL = clamp32(fl_sh(c - chi_break_fx(0) - X0, s - 1));
          if (cut > chi_break_fx(1)) {  // owned nodes may lie beyond 150 cm^-1 (branches 2, 3)
            const int jR150 = clamp32(fl_sh(c + chi_break_fx(1) - X0, s - 1));
            const int jL150 = clamp32(cl_sh(c - chi_break_fx(1) - X0, s - 1));
            if (jR150 < 2 * kG1Pairs - 1 || jL150 > 0) exact = true;
          }
          const float d0 = (nx.qf + nx.phi);  // offset of node 0 from the centre, cm^-1
          aR = aC * 1.084f * expf(-0.027f * d0);
          aL = aC * 1.084f * expf(0.027f * d0);
        }
        // fast-path flags: bit 0 exact path; bit 1 the line owns every panel of the tile;
        // bits 2-3 the chi side of all evaluated nodes (1 left, 2 right, 0 centre/mixed)
        int fl = exact ? 1 : 0;
        if (jL >= 2 * kG1Pairs - 1) fl |= 4;        // every node at d <= -3
        else if (jR <= 0) fl |= 8;                  // every node at d >= 3
        const bool one_side = !(chi && physical) || (fl & 12);
        if (msk == full_tile && one_side) fl |= 2;
        sA[k] = make_float4(nx.qf, nx.hs, nx.phs, y * y);
        sB[k] = make_float4(aC, aL, aR, -0.5f * y * y);
        sM[k] = msk;
        sC[k] = make_int4(jL, jR, fl, 0);
      }
      __syncthreads();
      float pe = 0.f, pl = 0.f, pr = 0.f, pm = 0.f;
      // surrogate results: tag bit 0 odd node; bits 1, 2 the even node's L and R slots
      auto g1_apply = [&](int tag, float v) {
        if (tag & 1) pm += v;
        else if ((tag & 6) == 6) pe += v;
        else if (tag & 2) pl += v;
        else pr += v;
      };
      for (int k = warp * n_slot + slot; k < nbat; k += kG1Warps * n_slot) {
        const int4 C = sC[k];
        if ((C.z & 3) == 2) {
          // the line owns the whole tile through the far wing, on one chi side or with no chi
          const float4 a = sA[k], b = sB[k];
          const bool right = C.z & 8, left = C.z & 4;
          const float a0 = right ? b.z * rR0 : (left ? b.y * rL0 : b.x);
          const float a1 = right ? b.z * rR1 : (left ? b.y * rL1 : b.x);
          const float x0 = fmaf(f0 + a.x, a.y, a.z), x02 = x0 * x0;
          const float i0 = __fdividef(1.0f, x02 + a.w);
          const float x1 = fmaf(f1 + a.x, a.y, a.z), x12 = x1 * x1;
          const float i1 = __fdividef(1.0f, x12 + a.w);
          pe += a0 * i0 * fmaf(fmaf(1.5f, x02, b.w), i0 * i0, 1.0f);
          pm += a1 * i1 * fmaf(fmaf(1.5f, x12, b.w), i1 * i1, 1.0f);
          if (COUNT) nev += 2;
          continue;
        }
        const uint64_t msk = sM[k];
        const bool bL = (msk >> (p + 1)) & 1ull;  // panel m0+p: L of node 2m, M of node 2m+1
        const bool bR = (msk >> p) & 1ull;        // panel m0+p-1: R of node 2m
        if (SURR && use_mlp && (C.z & 1)) {  // exact path, warp-uniform: every lane takes part
          if (qn > kQCap - 64) q_flush(warp_queue(dsm), qn, S, g1_apply);
          const G1Nodes nd = g1_exact_nodes(R, off + b0 + k, X0, j0);
          const bool a0 = bL || bR, a1 = bL;
          const bool u0 = a0 && mlp_guard(S, nd.x0, nd.y), u1 = a1 && mlp_guard(S, nd.x1, nd.y);
          q_push(warp_queue(dsm), qn, u0, nd.x0, nd.y, nd.w0, (bL ? 2 : 0) | (bR ? 4 : 0));
          q_push(warp_queue(dsm), qn, u1, nd.x1, nd.y, nd.w1, 1);
          if (a0 && !u0) g1_apply((bL ? 2 : 0) | (bR ? 4 : 0), nd.w0 * voigt_K(nd.x0, nd.y));
          if (a1 && !u1) g1_apply(1, nd.w1 * voigt_K(nd.x1, nd.y));
          if (a0) count_eval<COUNT>(true, nd.x0, nd.y, nev, nnear, nmid, nsmall);
          if (a1) count_eval<COUNT>(true, nd.x1, nd.y, nev, nnear, nmid, nsmall);
          if (COUNT) nmlp += (u0 ? 1 : 0) + (u1 ? 1 : 0);
          continue;
        }
        if (!(C.z & 1)) {
          // far wing, without branches: every lane evaluates both nodes and each sum
          // takes a value only where the panels own the node (adding zero elsewhere
          // leaves the sums as they were)
          const float4 a = sA[k], b = sB[k];
          const float x0 = fmaf(f0 + a.x, a.y, a.z), x02 = x0 * x0;
          const float i0 = __fdividef(1.0f, x02 + a.w);
          const float s0 = fmaf(fmaf(1.5f, x02, b.w), i0 * i0, 1.0f);
          const float am0 = j0 >= C.y ? b.z * rR0 : (j0 <= C.x ? b.y * rL0 : b.x);
          const float v0 = am0 * i0 * s0;
          const float x1 = fmaf(f1 + a.x, a.y, a.z), x12 = x1 * x1;
          const float i1 = __fdividef(1.0f, x12 + a.w);
          const float s1 = fmaf(fmaf(1.5f, x12, b.w), i1 * i1, 1.0f);
          const float am1 = j0 + 1 >= C.y ? b.z * rR1 : (j0 + 1 <= C.x ? b.y * rL1 : b.x);
          const float v1 = am1 * i1 * s1;
          pe += (bL && bR) ? v0 : 0.0f;
          pl += (bL && !bR) ? v0 : 0.0f;
          pr += (!bL && bR) ? v0 : 0.0f;
          pm += bL ? v1 : 0.0f;
          if (COUNT) nev += (bL || bR ? 1 : 0) + (bL ? 1 : 0);
          continue;
        }
        if (!(bL || bR)) continue;
        float v0, v1;
        {
          int nn = 0, nm = 0, ns = 0;
          const float2 v = g1_exact_pair(R, off + b0 + k, X0, j0, true, bL, nn, nm, ns);
          v0 = v.x;
          v1 = v.y;
          if (COUNT) {
            nnear += nn;
            nmid += nm;
            nsmall += ns;
          }
        }
        if (bL && bR) pe += v0; else if (bL) pl += v0; else pr += v0;
        pm += v1;
        if (COUNT) nev += 1 + (bL ? 1 : 0);
      }
      if (SURR && use_mlp) q_flush(warp_queue(dsm), qn, S, g1_apply);
      kahan_add(eS, eC, pe);
      kahan_add(lS, lC, pl);
      kahan_add(rS, rC, pr);
      kahan_add(mS, mC, pm);
    }
  };
  if (narrow)
    sum_lines(std::true_type{});
  else
    sum_lines(std::false_type{});
  const int slot = narrow ? lane >> 3 : 0;
  const int p = narrow ? pw0 + (lane & 7) : lane;
  if (narrow) {
    // merge the four line slots of each pair (slots 0 + 1 and 2 + 3, then the two), and
    // leave the pairs' sums at their own lanes
#pragma unroll
    for (int d = 8; d <= 16; d <<= 1) {
      float o0 = __shfl_xor_sync(0xffffffffu, eS, d), o1 = __shfl_xor_sync(0xffffffffu, eC, d);
      comp_merge(eS, eC, o0, o1);
      o0 = __shfl_xor_sync(0xffffffffu, lS, d), o1 = __shfl_xor_sync(0xffffffffu, lC, d);
      comp_merge(lS, lC, o0, o1);
      o0 = __shfl_xor_sync(0xffffffffu, rS, d), o1 = __shfl_xor_sync(0xffffffffu, rC, d);
      comp_merge(rS, rC, o0, o1);
      o0 = __shfl_xor_sync(0xffffffffu, mS, d), o1 = __shfl_xor_sync(0xffffffffu, mC, d);
      comp_merge(mS, mC, o0, o1);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) sRed[warp][q][lane] = 0.0f;
    __syncwarp();
    if (slot == 0 && p <= pw1) {
      sRed[warp][0][p] = eS; sRed[warp][1][p] = eC;
      sRed[warp][2][p] = lS; sRed[warp][3][p] = lC;
      sRed[warp][4][p] = rS; sRed[warp][5][p] = rC;
      sRed[warp][6][p] = mS; sRed[warp][7][p] = mC;
    }
  } else {
    sRed[warp][0][lane] = eS; sRed[warp][1][lane] = eC;
    sRed[warp][2][lane] = lS; sRed[warp][3][lane] = lC;
    sRed[warp][4][lane] = rS; sRed[warp][5][lane] = rC;
    sRed[warp][6][lane] = mS; sRed[warp][7][lane] = mC;
  }
  __syncthreads();
  if (warp == 0) {
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = sRed[0][q][lane];
    for (int w = 1; w < kG1Warps; ++w) {
      comp_merge(a[0], a[1], sRed[w][0][lane], sRed[w][1][lane]);
      comp_merge(a[2], a[3], sRed[w][2][lane], sRed[w][3][lane]);
      comp_merge(a[4], a[5], sRed[w][4][lane], sRed[w][5][lane]);
      comp_merge(a[6], a[7], sRed[w][6][lane], sRed[w][7][lane]);
    }
    float ls = a[0], lc = a[1], rs = a[0], rc = a[1];
    comp_merge(ls, lc, a[2], a[3]);
    comp_merge(rs, rc, a[4], a[5]);
    const int64_t np = R.npan[1];
    float* gp = R.slots + (int64_t)lev * R.slots_per_level + R.slot_off[1] + 3 * np * it.part;
    const int64_t m = m0 + lane;  // this lane's pair
    if (m <= m_last && MARFA_DCHECK(m >= m_first, 301)) {
      gp[m - m_first] = ls + lc;
      gp[np + (m - m_first)] = a[6] + a[7];
    }
    if (m - 1 >= m_first && m - 1 <= m_last) gp[2 * np + (m - 1 - m_first)] = rs + rc;
  }
  if (COUNT) block_counts<kG1Warps>(nev, nmlp, nnear, nmid, nsmall, sCnt, counts);
}

void launch_g1(const ReqDev* reqs, const G1Item* items, int n_items, int64_t* counts, bool surr,
               bool wide, cudaStream_t st) {
  if (n_items <= 0) return;
  if (surr) {
    if (counts)
      launch_surr(k_g1<true, true, 2>, n_items, kG1Warps * 32, st, reqs, items, counts);
    else
      launch_surr(k_g1<false, true, 2>, n_items, kG1Warps * 32, st, reqs, items, counts);
  } else if (counts) {
    k_g1<true, false, 2><<<n_items, kG1Warps * 32, 0, st>>>(reqs, items, counts);
  } else if (wide) {
    k_g1<false, false, 1><<<n_items, kG1Warps * 32, 0, st>>>(reqs, items, counts);
  } else {
    k_g1<false, false, 0><<<n_items, kG1Warps * 32, 0, st>>>(reqs, items, counts);
  }
}

// ------------------------------------------------------------------ grids 2..10, line-major
// A CTA owns PAIRS (16 or 32) consecutive node pairs of grid g of one level. Each thread takes
// one candidate line at a time, forms the exact mask of the panels the line owns in
// the tile, evaluates the profile at the nodes of those panels only, and adds the
// values into lane-private shared-memory slots (acc[pair][lane]); the slots are summed
// over lanes and warps in a fixed order at the end.
// Register budgets: 72 for the plain 16-pair variant (seven CTAs per SM), 128 for the
// plain 32-pair one (four, as its 48 KB of slots allow), 168 with the surrogate.
template <bool COUNT, bool SURR, int PAIRS, int WIDE>
__global__ void __launch_bounds__(kLWarps * 32, SURR ? 3 : (PAIRS == 16 ? 7 : 4))
    k_coarse_lm(const ReqDev* __restrict__ reqs, const CoarseItem* __restrict__ items,
             int64_t* __restrict__ counts) {
  extern __shared__ __align__(16) unsigned char dsm[];  // surrogate weights (SURR only)
  MlpWeights& S = *reinterpret_cast<MlpWeights*>(dsm);
  __shared__ float accL[kLWarps][PAIRS][32];
  __shared__ float accM[kLWarps][PAIRS][32];
  __shared__ float accR[kLWarps][PAIRS][32];
  __shared__ int64_t sCnt[kCountFields][kLWarps];
  const CoarseItem it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const bool wide = WIDE == 2 ? R.wide != 0 : WIDE == 1;  // 5-point partition
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = it.grid;
  const int lev = it.level;
  const int64_t m_first = R.m_first[g];
  const int64_t m_last = m_first + R.npan[g] - 1;
  const int64_t m0 = it.m0;
  const int s = panel_shift(g);
  const int64_t cut = R.cut_fx;
  const int64_t base = m0 - 1;  // mask bit b <-> panel m0 - 1 + b
  const int nb = PAIRS + 1;
  // panel masks of PAIRS + 1 bits: 32-bit words for 16 pairs
  using MT = typename std::conditional<(PAIRS < 32), uint32_t, uint64_t>::type;
  const MT win = rmask<MT>(m_first, m_last, base, nb);
  PanelFrame fr;  // 32-bit ownership where the offsets are whole panels
  fr.init(g, base, nb, cut, R.R_w);
  if (wide) fr.ok = false;
  for (int p = 0; p < PAIRS; ++p) {
    accL[warp][p][lane] = 0.0f;
    accM[warp][p][lane] = 0.0f;
    accR[warp][p][lane] = 0.0f;
  }
  const LevelDev L = R.lev[lev];
  Bands bd;
  bd.n = 0;
  {
    // the span of the parent grid's panels over the tile's panels inside the window,
    // widened by one of them
    const int64_t pa = max(base, m_first), pb = min(base + nb - 1, m_last);
    const int al = wide ? s + 2 : s + 1;  // parent panels: two (four) steps of grid g - 1
    const int64_t P = int64_t(1) << (wide ? s + 2 : s);
    const int64_t A = fl_sh(pa << s, al) << al;
    const int64_t B = (fl_sh(pb << s, al) + 1) << al;
    int64_t zlo[9], zhi[9];
    const int nz = make_zones(A, B, (int64_t)R.R_w * step_fx(g - 1), cut, P, R.chi_req, zlo, zhi);
    if (pa <= pb) bd.lookup(R, L, zlo, zhi, nz);
  }
  // the bands in shared memory for the candidate walk (every warp looked them up alike)
  __shared__ int64_t sb_lo[9], sb_hi[9];
  if (tid < bd.n) {
    sb_lo[tid] = bd.lo[tid];
    sb_hi[tid] = bd.hi[tid];
  }
  __syncthreads();
  const int64_t lo_off = (int64_t)lev * R.n_lines;
  const int64_t X0 = m0 << s;  // position of node 2 m0 (j = 0)
  const int64_t xa_t = base << s, xb_t = (base + nb) << s;  // span of the mask's panels
  const int64_t P_t = int64_t(1) << (wide ? s + 2 : s);  // one parent panel (5-point: four steps of g - 1)
  const bool physical = R.shape < kShapeConst;
  const bool voigt = R.shape == kShapeVoigt;
  int64_t nev = 0, nmlp = 0, nnear = 0, nmid = 0, nsmall = 0;
  const bool use_mlp = SURR && R.mlp != nullptr;  // block-uniform
  if (use_mlp) {
    mlp_load_smem(S, R.mlp);
    __syncthreads();
  }
  int qn = 0;  // entries in this warp's surrogate queue (warp-uniform)
  // surrogate results: tag bits 0-4 pair, 5 L slot, 6 R slot, 7 odd node (M slot)
  auto lm_apply = [&](int tag, float v) {
    const int p = tag & 31;
    if (tag & 128) {
      accM[warp][p][lane] += v;
    } else {
      if (tag & 32) accL[warp][p][lane] += v;
      if (tag & 64) accR[warp][p][lane] += v;
    }
  };
  __syncwarp();
  const int64_t n_cand = bd.total();
  SharedBandCursor cur;
  cur.init(sb_lo, sb_hi, bd.n);
  {
    for (int64_t t0 = 0; t0 < n_cand; t0 += kLWarps * 32) {  // block-uniform
      const bool valid = t0 + tid < n_cand;
      const int64_t i = valid ? cur.line(sb_lo, sb_hi, t0 + tid) : 0;
      if (SURR && use_mlp) {
        // all lanes step through the union of their pair ranges together; evaluations
        // that pass the guard go to the warp's queue
        MT own = 0;
        int64_t c = 0;
        bool chi = false;
        if (valid) {
          c = __ldg(R.c + lo_off + i);
          const int gst = __ldg(R.gstar + lo_off + i);
          chi = __ldg(R.flags + lo_off + i) & 1;
          own = owned_any<MT>(wide, g, c, gst, chi, cut, R.R_w, base, nb) & win;
        }
        float amp = 0.0f, y = 1.0f;
        NodeX nx;
        nx.qf = nx.hs = nx.phs = nx.phi = 0.0f;
        ChiThr ct;
        const bool use_chi = own && chi && physical;
        int pa = 1 << 20, pb = -1;
        if (own) {
          amp = __ldg(R.amp + lo_off + i);
          y = __ldg(R.yv + lo_off + i);
          nx.init(X0 - c, s - 1, __ldg(R.sx + lo_off + i));
          if (use_chi) ct.init(c, X0, s - 1, R.cut_fx);
          pa = max(mask_lowest(own) - 1, 0);
          pb = min(mask_highest(own), PAIRS - 1);
        }
        const int qa = __reduce_min_sync(0xffffffffu, pa), qb = __reduce_max_sync(0xffffffffu, pb);
        for (int p = qa; p <= qb; ++p) {
          if (qn > kQCap - 64) q_flush(warp_queue(dsm), qn, S, lm_apply);
          const bool bR = (own >> p) & MT(1), bL = (own >> (p + 1)) & MT(1);
          const bool ae = bR || bL, ao = bL;
          const float jf = (float)(2 * p);
          const float xe = nx.x(jf), xo = nx.x(jf + 1.0f);
          const bool ue = ae && mlp_guard(S, xe, y), uo = ao && mlp_guard(S, xo, y);
          const float ce = (use_chi && ae) ? ct.value(2 * p, nx.absd(jf, s - 1)) : 1.0f;
          const float co = (use_chi && ao) ? ct.value(2 * p + 1, nx.absd(jf + 1.0f, s - 1)) : 1.0f;
          const int te = p | (bL ? 32 : 0) | (bR ? 64 : 0), to = p | 128;
          q_push(warp_queue(dsm), qn, ue, xe, y, amp * ce, te);
          q_push(warp_queue(dsm), qn, uo, xo, y, amp * co, to);
          if (ae && !ue) {
            float v = amp * voigt_K(xe, y);
            if (use_chi) v *= ce;
            lm_apply(te, v);
          }
          if (ao && !uo) {
            float w = amp * voigt_K(xo, y);
            if (use_chi) w *= co;
            lm_apply(to, w);
          }
          if (ae) count_eval<COUNT>(true, xe, y, nev, nnear, nmid, nsmall);
          if (ao) count_eval<COUNT>(true, xo, y, nev, nnear, nmid, nsmall);
          if (COUNT) nmlp += (ue ? 1 : 0) + (uo ? 1 : 0);
        }
        continue;
      }
      if (!valid) continue;
      const int64_t c = __ldg(R.c + lo_off + i);
      const int gst = __ldg(R.gstar + lo_off + i);
      const bool chi = __ldg(R.flags + lo_off + i) & 1;
      // the line's data with its position (consecutive lines across the threads:
      // coalesced), so that a candidate costs one round trip to memory
      const float amp = __ldg(R.amp + lo_off + i);
      const float sx = __ldg(R.sx + lo_off + i);
      const float y = __ldg(R.yv + lo_off + i);
      MT own;
      if (fr.ok) {
        const PanelPos pp = fr.pos(c);
        if (owns_nothing_frame(fr, pp, g, gst, chi)) continue;
        own = accept_frame<MT>(fr, pp, g, gst, chi) & win;
        if (own) own &= ~accept_parent_frame<MT>(fr, pp, g, gst, chi);
      } else {
        if (owns_nothing(g, c, gst, chi, cut, xa_t, xb_t, P_t)) continue;
        own = owned_any<MT>(wide, g, c, gst, chi, cut, R.R_w, base, nb) & win;
      }
      if (!own) continue;
      NodeX nx;
      nx.init(X0 - c, s - 1, sx);
      ChiThr ct;
      const bool use_chi = chi && physical;
      if (use_chi) ct.init(c, X0, s - 1, R.cut_fx);
      // pair p uses bits p (R slot of node 2p) and p + 1 (L of node 2p, M of node 2p+1)
      const int pa = max(mask_lowest(own) - 1, 0);
      const int pb = min(mask_highest(own), PAIRS - 1);
      // a chi branch common to all nodes 2pa .. 2pb + 1: one exponential per line
      const bool run = use_chi && ct.uniform(2 * pa, 2 * pb + 1);
      ChiRun cr;
      if (run) cr.init(ct, 2 * pa, nx.absd((float)(2 * pa), s - 1), s - 1);
      if (PAIRS == 16) {
        // 16 pairs: every pair of pa..pb, chi by a running product (cheaper than exp2 here)
        const float r2 = run ? cr.ratio * cr.ratio : 1.0f;
        for (int p = pa; p <= pb; ++p, cr.v *= r2) {
          const bool bR = (own >> p) & MT(1), bL = (own >> (p + 1)) & MT(1);
          if (!(bR || bL)) continue;
          const float jf = (float)(2 * p);
          const float xv = nx.x(jf);
          float v = amp * (voigt ? voigt_K<false, true>(xv, y, kVoigtCells) : shape_f(R.shape, xv, y));
          if (use_chi) v *= run ? cr.v : ct.value(2 * p, nx.absd(jf, s - 1));
          if (!MARFA_DCHECK(p >= 0 && p < PAIRS, 106)) continue;
          if (bL) accL[warp][p][lane] += v;
          if (bR) accR[warp][p][lane] += v;
          count_eval<COUNT>(voigt, xv, y, nev, nnear, nmid, nsmall);
          if (bL) {
            const float xw = nx.x(jf + 1.0f);
            float w = amp * (voigt ? voigt_K<false, true>(xw, y, kVoigtCells) : shape_f(R.shape, xw, y));
            if (use_chi) w *= run ? cr.v * cr.ratio : ct.value(2 * p + 1, nx.absd(jf + 1.0f, s - 1));
            accM[warp][p][lane] += w;
            count_eval<COUNT>(voigt, xw, y, nev, nnear, nmid, nsmall);
          }
        }
      } else {
        // 32 pairs: the touched pairs only (not the gap inside a line's ring)
        for (uint32_t tm = (uint32_t)(own | (own >> 1)); tm; tm &= tm - 1) {
          const int p = __ffs((int)tm) - 1;
          const bool bR = (own >> p) & MT(1), bL = (own >> (p + 1)) & MT(1);
          const float cv = run ? cr.at(2 * (p - pa)) : 1.0f;
          const float jf = (float)(2 * p);
          const float xv = nx.x(jf);
          float v = amp * (voigt ? voigt_K<false, true>(xv, y, kVoigtCells) : shape_f(R.shape, xv, y));
          if (use_chi) v *= run ? cv : ct.value(2 * p, nx.absd(jf, s - 1));
          if (!MARFA_DCHECK(p >= 0 && p < PAIRS, 106)) continue;
          if (bL) accL[warp][p][lane] += v;
          if (bR) accR[warp][p][lane] += v;
          count_eval<COUNT>(voigt, xv, y, nev, nnear, nmid, nsmall);
          if (bL) {
            const float xw = nx.x(jf + 1.0f);
            float w = amp * (voigt ? voigt_K<false, true>(xw, y, kVoigtCells) : shape_f(R.shape, xw, y));
            if (use_chi) w *= run ? cv * cr.ratio : ct.value(2 * p + 1, nx.absd(jf + 1.0f, s - 1));
            accM[warp][p][lane] += w;
            count_eval<COUNT>(voigt, xw, y, nev, nnear, nmid, nsmall);
          }
        }
      }
    }
  }
  if (SURR && use_mlp) q_flush(warp_queue(dsm), qn, S, lm_apply);
  __syncthreads();
  // thread t < 3 PAIRS sums slot (t / PAIRS, pair t % PAIRS) over warps and lanes
  if (tid < 3 * PAIRS) {
    const int kind = tid / PAIRS, p = tid % PAIRS;
    float (*acc)[PAIRS][32] = kind == 0 ? accL : (kind == 1 ? accM : accR);
    // one compensated sum per warp's lanes, interleaved (independent chains), then the
    // warps' sums merged in warp order
    float sw[kLWarps], cw[kLWarps];
#pragma unroll
    for (int w = 0; w < kLWarps; ++w) sw[w] = cw[w] = 0.0f;
    for (int l = 0; l < 32; ++l)
#pragma unroll
      for (int w = 0; w < kLWarps; ++w) kahan_add(sw[w], cw[w], acc[w][p][(l + p) & 31]);
    float sum = sw[0], cmp = cw[0];
#pragma unroll
    for (int w = 1; w < kLWarps; ++w) comp_merge(sum, cmp, sw[w], cw[w]);
    const float v = sum + cmp;
    float* gp = R.slots + (int64_t)lev * R.slots_per_level + R.slot_off[g];
    const int64_t np = R.npan[g];
    const int64_t m = m0 + p;
    if (kind == 0 && m <= m_last && MARFA_DCHECK(m >= m_first, 105)) gp[m - m_first] = v;
    if (kind == 1 && m <= m_last) gp[np + (m - m_first)] = v;
    if (kind == 2 && m - 1 >= m_first && m - 1 <= m_last) gp[2 * np + (m - 1 - m_first)] = v;
  }
  if (COUNT) block_counts<kLWarps>(nev, nmlp, nnear, nmid, nsmall, sCnt, counts);
}

void launch_coarse_lm(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts,
                      bool surr, int pairs, bool wide, cudaStream_t st) {
  if (n_items <= 0) return;
  const int T = kLWarps * 32;
  if (pairs == 16) {
    if (surr) {
      if (counts)
        launch_surr(k_coarse_lm<true, true, 16, 2>, n_items, T, st, reqs, items, counts);
      else
        launch_surr(k_coarse_lm<false, true, 16, 2>, n_items, T, st, reqs, items, counts);
    } else if (counts) {
      k_coarse_lm<true, false, 16, 2><<<n_items, T, 0, st>>>(reqs, items, counts);
    } else if (wide) {
      k_coarse_lm<false, false, 16, 1><<<n_items, T, 0, st>>>(reqs, items, counts);
    } else {
      k_coarse_lm<false, false, 16, 0><<<n_items, T, 0, st>>>(reqs, items, counts);
    }
    return;
  }
  if (surr) {
    if (counts)
      launch_surr(k_coarse_lm<true, true, 32, 2>, n_items, T, st, reqs, items, counts);
    else
      launch_surr(k_coarse_lm<false, true, 32, 2>, n_items, T, st, reqs, items, counts);
  } else if (counts) {
    k_coarse_lm<true, false, 32, 2><<<n_items, T, 0, st>>>(reqs, items, counts);
  } else if (wide) {
    k_coarse_lm<false, false, 32, 1><<<n_items, T, 0, st>>>(reqs, items, counts);
  } else {
    k_coarse_lm<false, false, 32, 0><<<n_items, T, 0, st>>>(reqs, items, counts);
  }
}

// 32 x 32 bit-matrix transpose across a warp: lane t holds row t; returns column `lane`
// (bit t = bit lane of row t). Five stages swap the off-diagonal blocks of width 16, 8,
// 4, 2 and 1 between lanes t and t ^ j.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  constexpr uint32_t kM[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int j = 16 >> k;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~kM[k]) | ((y & ~kM[k]) >> j)) : ((x & kM[k]) | ((y & kM[k]) << j));
  }
  return x;
}

// ------------------------------------------------------------------ grids 2..10
// Warp w of a CTA owns kCPairs consecutive node pairs of grid g of one level (lane p
// holds pair p: even node 2m, odd node 2m+1). The warp takes 32 candidate lines at a
// time, one per lane. Phase 1: each lane forms the exact mask of the panels its line
// owns in the tile and evaluates the profile at the nodes of those panels, into a
// per-warp shared buffer (row = line). Phase 2: each lane adds, for its own pair, the
// buffered values of the lines owning its panels into compensated register sums.
// At most 80 registers a thread in the plain variants (168 with the surrogate): with the
// Voigt tables read through the read-only cache (no shared copy), six CTAs fit on an SM.
template <bool COUNT, bool SURR, int WIDE>
__global__ void __launch_bounds__(kCWarps * 32, SURR ? 3 : 6)
    k_coarse(const ReqDev* __restrict__ reqs, const CoarseItem* __restrict__ items,
             int64_t* __restrict__ counts) {
  extern __shared__ __align__(16) unsigned char dsm[];  // surrogate weights and queues (SURR only)
  MlpWeights& S = *reinterpret_cast<MlpWeights*>(dsm);
  __shared__ float bufE[kCWarps][32][kCPairs + 1];  // value at node 2p of staged line t
  __shared__ float bufO[kCWarps][32][kCPairs + 1];  // value at node 2p + 1
  __shared__ unsigned long long smsk[kCWarps][32];
  __shared__ int64_t sCnt[kCountFields][kCWarps];
  const CoarseItem it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const bool wide = WIDE == 2 ? R.wide != 0 : WIDE == 1;  // 5-point partition
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = it.grid;
  const int lev = it.level;
  const int64_t m_first = R.m_first[g];
  const int64_t m_last = m_first + R.npan[g] - 1;
  const int64_t m0 = it.m0 + (int64_t)kCPairs * warp;  // this warp's first pair
  int64_t nev = 0, nmlp = 0, nnear = 0, nmid = 0, nsmall = 0;
  const bool use_mlp = SURR && R.mlp != nullptr;  // block-uniform
  if (use_mlp) mlp_load_smem(S, R.mlp);
  __syncthreads();
  if (m0 <= m_last + 1) {  // warp-uniform
    const int s = panel_shift(g);
    const int64_t cut = R.cut_fx;
    const int64_t base = m0 - 1;  // mask bit b <-> panel m0 - 1 + b
    const int nb = kCPairs + 1;
    const uint64_t win = rmask<uint64_t>(m_first, m_last, base, nb);
    PanelFrame fr;  // 32-bit ownership where the offsets are whole panels
    fr.init(g, base, nb, cut, R.R_w);
    if (wide) fr.ok = false;
    const LevelDev L = R.lev[lev];
    Bands bd;
    bd.n = 0;
    {
      // the span of the parent grid's panels over the tile's panels inside the window,
      // widened by one of them
      const int64_t pa = max(base, m_first), pb = min(base + nb - 1, m_last);
      const int al = wide ? s + 2 : s + 1;  // parent panels: two (four) steps of grid g - 1
      const int64_t P = int64_t(1) << (wide ? s + 2 : s);
      const int64_t A = fl_sh(pa << s, al) << al;
      const int64_t B = (fl_sh(pb << s, al) + 1) << al;
      int64_t zlo[9], zhi[9];
      const int nz = make_zones(A, B, (int64_t)R.R_w * step_fx(g - 1), cut, P, R.chi_req, zlo, zhi);
      if (pa <= pb) bd.lookup(R, L, zlo, zhi, nz);
    }
    const int64_t lo_off = (int64_t)lev * R.n_lines;
    const int64_t X0 = m0 << s;  // position of node 2 m0 (j = 0)
    const int64_t xa_t = base << s, xb_t = (base + nb) << s;  // span of the mask's panels
    const int64_t P_t = int64_t(1) << (wide ? s + 2 : s);  // one parent panel (5-point: four steps of g - 1)
    const bool physical = R.shape < kShapeConst;
    const bool voigt = R.shape == kShapeVoigt;
    const int p = lane;
    float (*bE)[kCPairs + 1] = bufE[warp];
    float (*bO)[kCPairs + 1] = bufO[warp];
    unsigned long long* mk = smsk[warp];
    int qn = 0;  // entries in this warp's surrogate queue (warp-uniform)
    float sL = 0.f, cL = 0.f, sR = 0.f, cR = 0.f, sM = 0.f, cM = 0.f;
    // surrogate results, applied by the lane of the pair they belong to (the queue owner):
    // tag bits 0-4 pair, 5 L slot, 6 R slot (even node), 7 M slot (odd node)
    auto tp_apply = [&](int tag, float v) {
      if (tag & 128) {
        kahan_add(sM, cM, v);
      } else {
        if (tag & 32) kahan_add(sL, cL, v);
        if (tag & 64) kahan_add(sR, cR, v);
      }
    };
    const int64_t n_cand = bd.total();
    BandCursor cur;
    {
      for (int64_t t0 = 0; t0 < n_cand; t0 += 32) {  // warp-uniform
        const bool valid = t0 + lane < n_cand;
        const int64_t i = valid ? cur.line(bd, t0 + lane) : 0;
        uint64_t own = 0;
        int64_t c = 0;
        bool chi = false;
        if (valid) {
          c = __ldg(R.c + lo_off + i);
          const int gst = __ldg(R.gstar + lo_off + i);
          chi = __ldg(R.flags + lo_off + i) & 1;
          if (fr.ok) {
            const PanelPos pp = fr.pos(c);
            if (!owns_nothing_frame(fr, pp, g, gst, chi)) {
              own = accept_frame<uint64_t>(fr, pp, g, gst, chi) & win;
              if (own) own &= ~accept_parent_frame<uint64_t>(fr, pp, g, gst, chi);
            }
          } else if (!owns_nothing(g, c, gst, chi, cut, xa_t, xb_t, P_t)) {
            own = owned_any<uint64_t>(wide, g, c, gst, chi, cut, R.R_w, base, nb) & win;
          }
        }
        const uint32_t any = __ballot_sync(0xffffffffu, own != 0);
        if (!any) continue;
        // phase 1: this lane's line at the nodes of its owned panels
        if (SURR && use_mlp) {
          // all lanes step through the union of their pair ranges together; evaluations
          // that pass the guard go to the warp's queue, flushed before phase 2
          float amp = 0.0f, y = 1.0f;
          NodeX nx;
          nx.qf = nx.hs = nx.phs = nx.phi = 0.0f;
          ChiThr ct;
          const bool use_chi = own && chi && physical;
          int pa = 1 << 20, pb = -1;
          if (own) {
            amp = __ldg(R.amp + lo_off + i);
            y = __ldg(R.yv + lo_off + i);
            nx.init(X0 - c, s - 1, __ldg(R.sx + lo_off + i));
            if (use_chi) ct.init(c, X0, s - 1, R.cut_fx);
            pa = max(__ffsll((long long)own) - 2, 0);
            pb = min(63 - __clzll((long long)own), kCPairs - 1);
          }
          const int qa = __reduce_min_sync(0xffffffffu, pa), qb = __reduce_max_sync(0xffffffffu, pb);
          for (int q = qa; q <= qb; ++q) {
            if (qn > kQCap - 64) q_flush(warp_queue(dsm), qn, S, tp_apply);
            const bool bR = (own >> q) & 1ull, bL = (own >> (q + 1)) & 1ull;
            const bool ae = bR || bL, ao = bL;
            const float jf = (float)(2 * q);
            const float xv = nx.x(jf), xw = nx.x(jf + 1.0f);
            const bool ue = ae && mlp_guard(S, xv, y), uo = ao && mlp_guard(S, xw, y);
            const float ce = (use_chi && ae) ? ct.value(2 * q, nx.absd(jf, s - 1)) : 1.0f;
            const float co = (use_chi && ao) ? ct.value(2 * q + 1, nx.absd(jf + 1.0f, s - 1)) : 1.0f;
            // deferred values go straight to the pair's lane; the buffer gets 0 there
            q_push(warp_queue(dsm), qn, ue, xv, y, amp * ce, q | (bL ? 32 : 0) | (bR ? 64 : 0), q);
            q_push(warp_queue(dsm), qn, uo, xw, y, amp * co, q | 128, q);
            if (ae) {
              float v = 0.0f;
              if (!ue) {
                v = amp * voigt_K(xv, y);
                if (use_chi) v *= ce;
              }
              if (MARFA_DCHECK(q >= 0 && q < kCPairs, 101)) bE[lane][q] = v;
            }
            if (ao) {
              float w = 0.0f;
              if (!uo) {
                w = amp * voigt_K(xw, y);
                if (use_chi) w *= co;
              }
              if (MARFA_DCHECK(q >= 0 && q < kCPairs, 101)) bO[lane][q] = w;
            }
            if (ae) count_eval<COUNT>(true, xv, y, nev, nnear, nmid, nsmall);
            if (ao) count_eval<COUNT>(true, xw, y, nev, nnear, nmid, nsmall);
            if (COUNT) nmlp += (ue ? 1 : 0) + (uo ? 1 : 0);
          }
        } else if (own) {
          const float amp = __ldg(R.amp + lo_off + i);
          const float sx = __ldg(R.sx + lo_off + i);
          const float y = __ldg(R.yv + lo_off + i);
          NodeX nx;
          nx.init(X0 - c, s - 1, sx);
          ChiThr ct;
          const bool use_chi = chi && physical;
          if (use_chi) ct.init(c, X0, s - 1, R.cut_fx);
          const int pa = max(__ffsll((long long)own) - 2, 0);
          const int pb = min(63 - __clzll((long long)own), kCPairs - 1);
          // a chi branch common to all nodes 2pa .. 2pb + 1: one exponential per line
          const bool run = use_chi && ct.uniform(2 * pa, 2 * pb + 1);
          ChiRun cr;
          if (run) cr.init(ct, 2 * pa, nx.absd((float)(2 * pa), s - 1), s - 1);
          // the touched pairs only (not the gap inside a line's ring)
          for (uint32_t tm = (uint32_t)(own | (own >> 1)); tm; tm &= tm - 1) {
            const int q = __ffs((int)tm) - 1;
            const bool bL = (own >> (q + 1)) & 1ull;
            const float cv = run ? cr.at(2 * (q - pa)) : 1.0f;
            const float jf = (float)(2 * q);
            const float xv = nx.x(jf);
            float v = amp * (voigt ? voigt_K<false, false, true>(xv, y, kVoigtCells) : shape_f(R.shape, xv, y));
            if (use_chi) v *= run ? cv : ct.value(2 * q, nx.absd(jf, s - 1));
            if (MARFA_DCHECK(q >= 0 && q < kCPairs, 101)) bE[lane][q] = v;
            count_eval<COUNT>(voigt, xv, y, nev, nnear, nmid, nsmall);
            if (bL) {
              const float xw = nx.x(jf + 1.0f);
              float w = amp * (voigt ? voigt_K<false, false, true>(xw, y, kVoigtCells) : shape_f(R.shape, xw, y));
              if (use_chi) w *= run ? cv * cr.ratio : ct.value(2 * q + 1, nx.absd(jf + 1.0f, s - 1));
              if (MARFA_DCHECK(q >= 0 && q < kCPairs, 101)) bO[lane][q] = w;
              count_eval<COUNT>(voigt, xw, y, nev, nnear, nmid, nsmall);
            }
          }
        }
        mk[lane] = own;
        __syncwarp();
        // phase 2: the staged lines owning panel m0+p-1 (bit p) or m0+p (bit p+1): bit t
        // of lane p's mask = bit p of lane t's (own | own >> 1), a 32 x 32 bit transpose
        uint32_t mine = warp_transpose32((uint32_t)(own | (own >> 1)), lane);
        while (mine) {
          const int t = __ffs(mine) - 1;
          mine &= mine - 1;
          const uint64_t m2 = mk[t];
          const float v0 = bE[t][p];
          if ((m2 >> (p + 1)) & 1ull) {
            kahan_add(sL, cL, v0);
            kahan_add(sM, cM, bO[t][p]);
          }
          if ((m2 >> p) & 1ull) kahan_add(sR, cR, v0);
        }
        __syncwarp();
      }
    }
    if (SURR && use_mlp) q_flush(warp_queue(dsm), qn, S, tp_apply);  // warp-uniform
    float* gp = R.slots + (int64_t)lev * R.slots_per_level + R.slot_off[g];
    const int64_t np = R.npan[g];
    const int64_t m = m0 + p;
    if (m <= m_last && MARFA_DCHECK(m >= m_first, 104)) {
      gp[m - m_first] = sL + cL;
      gp[np + (m - m_first)] = sM + cM;
    }
    if (m - 1 >= m_first && m - 1 <= m_last) gp[2 * np + (m - 1 - m_first)] = sR + cR;
  }
  if (COUNT) block_counts<kCWarps>(nev, nmlp, nnear, nmid, nsmall, sCnt, counts);
}

void launch_coarse(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts,
                   bool surr, bool wide, cudaStream_t st) {
  if (n_items <= 0) return;
  const int T = kCWarps * 32;
  if (surr) {
    if (counts)
      launch_surr(k_coarse<true, true, 2>, n_items, T, st, reqs, items, counts);
    else
      launch_surr(k_coarse<false, true, 2>, n_items, T, st, reqs, items, counts);
  } else if (counts) {
    k_coarse<true, false, 2><<<n_items, T, 0, st>>>(reqs, items, counts);
  } else if (wide) {
    k_coarse<false, false, 1><<<n_items, T, 0, st>>>(reqs, items, counts);
  } else {
    k_coarse<false, false, 0><<<n_items, T, 0, st>>>(reqs, items, counts);
  }
}

// ------------------------------------------------------------------ grids 2..10 by mechanism
// Where a line's centre region, cut-off edges and chi breakpoints act on disjoint panels
// of grid g (mech_ok), its owned panels are the union of closed forms (ownership.cuh).
// Each warp (32 node pairs of grid g, as in k_coarse) then takes its candidates in
// separate passes, one per mechanism, each over the lines whose centre, edge or
// breakpoint position falls near the tile: the centre pass gives a line its ring (or
// core) as at most two runs of panels, an edge pass at most one panel, a breakpoint
// pass at most two. A pass decides ownership with a few shifts instead of the general
// masks, and the lanes of one pass carry similar work (a ring, or one panel's three
// nodes). The chi-factor is 1 in the centre region (it lies inside the first breakpoint),
// one branch of Eq. (10) along an edge panel, and decided per node near a breakpoint.
// Values go through the per-line buffers and phase 2 of k_coarse (pair sums in line
// order within a pass, passes in a fixed order): results are deterministic.
// MERGED: one pass over the merged position zones of all mechanisms instead of one pass
// per mechanism (fewer band lookups and rounds; a candidate's panels are then the union
// of its mechanisms' closed forms, and the chi-factor of a run of panels is 1 when the
// run lies in the centre region, else decided per node).
template <bool COUNT, bool MERGED>
__global__ void __launch_bounds__(kCWarps * 32, 6)
    k_coarse_mech(const ReqDev* __restrict__ reqs, const CoarseItem* __restrict__ items,
                  int64_t* __restrict__ counts) {
  __shared__ float bufE[kCWarps][32][kCPairs + 1];
  __shared__ float bufO[kCWarps][32][kCPairs + 1];
  __shared__ unsigned long long smsk[kCWarps][32];
  __shared__ int64_t sCnt[kCountFields][kCWarps];
  const CoarseItem it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = it.grid;
  const int lev = it.level;
  const int64_t m_first = R.m_first[g];
  const int64_t m_last = m_first + R.npan[g] - 1;
  const int64_t m0 = it.m0 + (int64_t)kCPairs * warp;
  int64_t nev = 0, nnear = 0, nmid = 0, nsmall = 0;
  if (m0 <= m_last + 1) {  // warp-uniform
    const int s = panel_shift(g);
    const int64_t P = int64_t(1) << s;
    const int64_t cut = R.cut_fx;
    const int64_t base = m0 - 1;
    const int nb = kCPairs + 1;
    const uint64_t win = rmask<uint64_t>(m_first, m_last, base, nb);
    const int64_t xa = base << s, xb = (base + nb) << s;  // span of the mask's panels
    const int64_t X0 = m0 << s;                            // node j = 0
    const int64_t R2 = (int64_t)R.R_w * step_fx(g - 1);
    const LevelDev L = R.lev[lev];
    const int64_t lo_off = (int64_t)lev * R.n_lines;
    const bool physical = R.shape < kShapeConst;
    const bool voigt = R.shape == kShapeVoigt;
    const float hnode = ldexpf(1.0f, s - 1 - kFixBits);
    // chi branch along the cut-off edges (no breakpoint lies within two panels of it)
    const int eb = (cut >= chi_break_fx(0)) + (cut > chi_break_fx(1)) + (cut > chi_break_fx(2));
    const float eC = eb == 1 ? 1.084f : (eb == 2 ? 0.208f : 0.025f);
    const float er = eb == 1 ? 0.027f : (eb == 2 ? 0.016f : 0.009f);
    int nB = 0;
    if (R.chi_req)
      for (int b = 0; b < 3 && chi_break_fx(b) <= cut; ++b) nB = b + 1;
    const int npass = MERGED ? 1 : 3 + 2 * nB;
    // the centre region ends before the first breakpoint's region begins (mech_ok)
    const float centre_end = 3.0f - 4.0f * ldexpf(1.0f, s - 1 - kFixBits);
    float (*bE)[kCPairs + 1] = bufE[warp];
    float (*bO)[kCPairs + 1] = bufO[warp];
    unsigned long long* mk = smsk[warp];
    const int p = lane;
    float sL = 0.f, sR = 0.f, sM = 0.f;
    // pass 0 centre; 1, 2 the right and left cut-off edges; then the right and left
    // positions of each breakpoint. The mechanism sits at c + off; positions of c + off
    // within reach of the tile can give panels of it.
    auto pass_off = [&](int q) {
      return q == 0 ? (int64_t)0
           : q == 1 ? cut
           : q == 2 ? -cut
           : ((q & 1) ? chi_break_fx((q - 3) >> 1) : -chi_break_fx((q - 3) >> 1));
    };
    // every pass's candidate range at once (lane 2q: the first line of pass q, lane
    // 2q + 1: its end), so that the lookups' global loads overlap
    int64_t range_v = 0;
    if (!MERGED && lane < 2 * npass) {
      const int q = lane >> 1;
      const int64_t off = pass_off(q), reach = q == 0 ? R2 + 2 * P : 2 * P;
      range_v = (lane & 1) ? upper_idx(R, xb + reach - off - L.smin) : lower_idx(R, xa - reach - off - L.smax);
    }
    for (int pass = 0; pass < npass; ++pass) {  // warp-uniform
      const int64_t off = pass_off(pass);
      // a pass per mechanism: one range of candidates (first line r_lo), kept in
      // registers; merged: the bands of all mechanisms
      Bands bd;
      bd.n = 0;
      int64_t r_lo = 0, r_n = 0;
      if (!MERGED) {
        r_lo = __shfl_sync(0xffffffffu, range_v, 2 * pass);
        r_n = max(__shfl_sync(0xffffffffu, range_v, 2 * pass + 1) - r_lo, (int64_t)0);
      } else {
        int64_t zlo[9], zhi[9];
        int nz = 0;
        zlo[nz] = xa - R2 - 2 * P; zhi[nz] = xb + R2 + 2 * P; ++nz;
        zlo[nz] = xa - 2 * P - cut; zhi[nz] = xb + 2 * P - cut; ++nz;
        zlo[nz] = xa - 2 * P + cut; zhi[nz] = xb + 2 * P + cut; ++nz;
        for (int b = 0; b < nB; ++b) {
          const int64_t B = chi_break_fx(b);
          zlo[nz] = xa - 2 * P - B; zhi[nz] = xb + 2 * P - B; ++nz;
          zlo[nz] = xa - 2 * P + B; zhi[nz] = xb + 2 * P + B; ++nz;
        }
        bd.lookup(R, L, zlo, zhi, nz);
      }
      const int64_t n_cand = MERGED ? bd.total() : r_n;
      BandCursor cur;
      for (int64_t t0 = 0; t0 < n_cand; t0 += 32) {  // warp-uniform
        const bool valid = t0 + lane < n_cand;
        const int64_t i = valid ? (MERGED ? cur.line(bd, t0 + lane) : r_lo + t0 + lane) : 0;
        uint64_t own = 0;
        int64_t c = 0;
        bool chi = false;
        float amp_p = 0.0f, sx_p = 1.0f, y_p = 0.0f;
        if (valid && MERGED) {
          c = __ldg(R.c + lo_off + i);
          const int gst = __ldg(R.gstar + lo_off + i);
          chi = __ldg(R.flags + lo_off + i) & 1;
          if (gst >= g) {
            int64_t a1, b1, a2, b2;
            mech_centre(g, c, gst, R.R_w, a1, b1, a2, b2);
            own = rmask<uint64_t>(a1, b1, base, nb) | rmask<uint64_t>(a2, b2, base, nb);
          }
          int64_t q = mech_edge_right(g, c + cut);
          if (q != -1) own |= rmask<uint64_t>(q, q, base, nb);
          q = mech_edge_left(g, c - cut);
          if (q != -1) own |= rmask<uint64_t>(q, q, base, nb);
          if (chi)
            for (int b = 0; b < nB; ++b) {
              int64_t q0, q1;
              mech_kink(g, c + chi_break_fx(b), q0, q1);
              if (q0 != -1) own |= rmask<uint64_t>(q0, q0, base, nb);
              if (q1 != -1) own |= rmask<uint64_t>(q1, q1, base, nb);
              mech_kink(g, c - chi_break_fx(b), q0, q1);
              if (q0 != -1) own |= rmask<uint64_t>(q0, q0, base, nb);
              if (q1 != -1) own |= rmask<uint64_t>(q1, q1, base, nb);
            }
          own &= win;
        } else if (valid) {
          c = __ldg(R.c + lo_off + i);
          // the evaluation's line data with the candidate's (one round trip)
          amp_p = __ldg(R.amp + lo_off + i);
          sx_p = __ldg(R.sx + lo_off + i);
          y_p = __ldg(R.yv + lo_off + i);
          if (pass == 0) {
            const int gst = __ldg(R.gstar + lo_off + i);
            if (gst >= g) {
              int64_t a1, b1, a2, b2;
              mech_centre(g, c, gst, R.R_w, a1, b1, a2, b2);
              own = (rmask<uint64_t>(a1, b1, base, nb) | rmask<uint64_t>(a2, b2, base, nb)) & win;
            }
          } else if (pass <= 2) {
            const int64_t q = pass == 1 ? mech_edge_right(g, c + cut) : mech_edge_left(g, c - cut);
            if (q != -1) own = rmask<uint64_t>(q, q, base, nb) & win;
            chi = __ldg(R.flags + lo_off + i) & 1;
          } else {
            chi = __ldg(R.flags + lo_off + i) & 1;
            if (chi) {
              int64_t q0, q1;
              mech_kink(g, c + off, q0, q1);
              if (q0 != -1) own |= rmask<uint64_t>(q0, q0, base, nb);
              if (q1 != -1) own |= rmask<uint64_t>(q1, q1, base, nb);
              own &= win;
            }
          }
        }
        const uint32_t tev = (uint32_t)(own | (own >> 1));
        if (!__ballot_sync(0xffffffffu, tev != 0)) continue;
        if (tev) {
          const float amp = MERGED ? __ldg(R.amp + lo_off + i) : amp_p;
          const float sx = MERGED ? __ldg(R.sx + lo_off + i) : sx_p;
          const float y = MERGED ? __ldg(R.yv + lo_off + i) : y_p;
          NodeX nx;
          nx.init(X0 - c, s - 1, sx);
          const bool use_chi = chi && physical;
          ChiThr ct;
          if (use_chi && MERGED) ct.init(c, X0, s - 1, R.cut_fx);
          // a breakpoint pass: near the lane's nodes the chi branch changes only at this
          // breakpoint (kb, on the right of the centre when kr), so one threshold of
          // ChiThr decides it (the same index and rounding)
          const int kb = (pass - 3) >> 1;
          const bool kr = pass & 1;
          int kthr = 0;
          if (!MERGED && use_chi && pass > 2) {
            const int64_t rel = c + (kr ? chi_break_fx(kb) : -chi_break_fx(kb)) - X0;
            kthr = clamp32((kr == (kb == 0)) ? cl_sh(rel, s - 1) : fl_sh(rel, s - 1));
          }
          // runs of owned panels: bits [ba, be] give nodes [2 ba - 2, 2 be] of the tile
          for (uint64_t rest = own; rest;) {
            const int ba = __ffsll((long long)rest) - 1;
            const uint64_t above = ~rest & (~0ull << ba);
            const int be = above ? __ffsll((long long)above) - 2 : 63;
            rest &= be >= 63 ? 0ull : (~0ull << (be + 1));
            const int ja = max(2 * ba - 2, 0), jb = min(2 * be, 2 * kCPairs - 1);
            // merged: a run in the centre region has chi = 1, any other run takes the
            // general per-node rule (an edge run or a breakpoint run)
            const bool run_chi = MERGED && use_chi && nx.absd((float)ja, s - 1) >= centre_end;
            for (int j = ja; j <= jb; ++j) {
              const float jf = (float)j;
              const float xv = nx.x(jf);
              float v = amp * (voigt ? voigt_K<false, false, true, true>(xv, y, kVoigtCells) : shape_f(R.shape, xv, y));
              if (MERGED) {
                if (run_chi) v *= ct.value(j, nx.absd(jf, s - 1));
              } else if (use_chi) {
                if (pass > 2) {
                  const bool beyond = kr ? (kb == 0 ? j >= kthr : j > kthr) : (kb == 0 ? j <= kthr : j < kthr);
                  const int br = kb + (beyond ? 1 : 0);
                  const float C = br == 1 ? 1.084f : (br == 2 ? 0.208f : 0.025f);
                  const float r = br == 1 ? 0.027f : (br == 2 ? 0.016f : 0.009f);
                  const float e = C * __expf(-r * nx.absd(jf, s - 1));
                  v *= br == 0 ? 1.0f : e;
                }
                else if (pass > 0 && eb > 0)
                  v *= eC * __expf(-er * nx.absd(jf, s - 1));
              }
              if (!MARFA_DCHECK(j >= 0 && j < 2 * kCPairs, 102)) continue;
              if (j & 1) bO[lane][j >> 1] = v;
              else bE[lane][j >> 1] = v;
              count_eval<COUNT>(voigt, xv, y, nev, nnear, nmid, nsmall);
            }
          }
        }
        mk[lane] = own;
        __syncwarp();
        uint32_t mine = warp_transpose32(tev, lane);
        // plain FP32 sums: a pair of grids 8..10 gathers a few dozen values at most, so
        // that the rounding error stays below 4e-6 relative
        while (mine) {
          const int t = __ffs(mine) - 1;
          mine &= mine - 1;
          const uint64_t m2 = mk[t];
          const float v0 = bE[t][p];
          if ((m2 >> (p + 1)) & 1ull) {
            sL += v0;
            sM += bO[t][p];
          }
          if ((m2 >> p) & 1ull) sR += v0;
        }
        __syncwarp();
      }
    }
    float* gp = R.slots + (int64_t)lev * R.slots_per_level + R.slot_off[g];
    const int64_t np = R.npan[g];
    const int64_t m = m0 + p;
    if (m <= m_last && MARFA_DCHECK(m >= m_first, 104)) {
      gp[m - m_first] = sL;
      gp[np + (m - m_first)] = sM;
    }
    if (m - 1 >= m_first && m - 1 <= m_last) gp[2 * np + (m - 1 - m_first)] = sR;
  }
  if (COUNT) block_counts<kCWarps>(nev, 0, nnear, nmid, nsmall, sCnt, counts);
}

void launch_coarse_mech(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts, bool merged,
                        cudaStream_t st) {
  if (n_items <= 0) return;
  const int T = kCWarps * 32;
  if (merged) {
    if (counts)
      k_coarse_mech<true, true><<<n_items, T, 0, st>>>(reqs, items, counts);
    else
      k_coarse_mech<false, true><<<n_items, T, 0, st>>>(reqs, items, counts);
  } else if (counts) {
    k_coarse_mech<true, false><<<n_items, T, 0, st>>>(reqs, items, counts);
  } else {
    k_coarse_mech<false, false><<<n_items, T, 0, st>>>(reqs, items, counts);
  }
}

// ------------------------------------------------------------------ grids 2..10, flattened
// The two-phase tiles (warp = 32 node pairs of grid g, 32 staged candidate lines per
// round) with phase 1 spread evenly over the lanes. Each owned node of a staged line is
// one entry (line, node); the round's entries are grouped by the branch of the Voigt
// function their node falls in (far wing, 6-term series, 15-term series, small-y
// cell, 9 x 9 cell; found per line from the node ranges between the branches'
// |x| boundaries), and the warp walks the grouped list 32 entries at a time, so that a
// line owning twenty nodes no longer holds 31 lanes idle and the lanes of a step take
// one branch. Values land in the per-line buffers of the two-phase kernel and phase 2
// sums them per pair in line order, as there: results are deterministic.
struct __align__(16) JobLine {
  float qf, hs, phs, amp;   // NodeX of the line relative to the tile's node 0, amplitude
  float y, phi, cv, clr;    // Voigt y; chi run: chi(j) = cv 2^(clr (j - cja))
  int16_t mode, cja;        // chi: 0 none, 1 run, 2 by thresholds
  int16_t r3, r150, r300, l3, l150, l300;  // ChiThr relative to node 0, clamped
};

// Pairs p of a 32-pair tile whose even node 2p (odd: 2p + 1) satisfies |j + o| hs >= T,
// j the node index, o = q + phi the centre's offset: j >= ceil(T / hs - o) or
// j <= floor(-T / hs - o).
__device__ __forceinline__ void far_side_pairs(float T, float hs, float o, uint32_t& ev, uint32_t& od) {
  const float tr = fminf(fmaxf(T / hs - o, -1.0e6f), 1.0e6f);
  const float tl = fminf(fmaxf(-T / hs - o, -1.0e6f), 1.0e6f);
  const int jr = (int)ceilf(tr), jl = (int)floorf(tl);
  // even: 2p >= jr <=> p >= ceil(jr / 2); 2p <= jl <=> p <= floor(jl / 2)
  const int er = (jr + 1) >> 1, el = jl >> 1;
  // odd: 2p + 1 >= jr <=> p >= ceil((jr - 1) / 2) = jr >> 1; 2p + 1 <= jl <=> p <= floor((jl - 1) / 2)
  const int orr = jr >> 1, ol = (jl - 1) >> 1;
  ev = rmask_rel<uint32_t>(er, 31, 32) | rmask_rel<uint32_t>(0, el, 32);
  od = rmask_rel<uint32_t>(orr, 31, 32) | rmask_rel<uint32_t>(0, ol, 32);
}

template <bool COUNT, int WIDE>
__global__ void __launch_bounds__(kCWarps * 32)
    k_coarse_jobs(const ReqDev* __restrict__ reqs, const CoarseItem* __restrict__ items,
                  int64_t* __restrict__ counts) {
  constexpr int kEntCap = 512;  // entries of a round evaluated per chunk
  __shared__ float bufE[kCWarps][32][kCPairs + 1];
  __shared__ float bufO[kCWarps][32][kCPairs + 1];
  __shared__ unsigned long long smsk[kCWarps][32];
  __shared__ JobLine sJL[kCWarps][32];
  __shared__ uint16_t sEnt[kCWarps][kEntCap];
  __shared__ int64_t sCnt[kCountFields][kCWarps];
  const CoarseItem it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const bool wide = WIDE == 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = it.grid;
  const int lev = it.level;
  const int64_t m_first = R.m_first[g];
  const int64_t m_last = m_first + R.npan[g] - 1;
  const int64_t m0 = it.m0 + (int64_t)kCPairs * warp;
  int64_t nev = 0, nnear = 0, nmid = 0, nsmall = 0;
  if (m0 <= m_last + 1) {  // warp-uniform
    const int s = panel_shift(g);
    const int64_t cut = R.cut_fx;
    const int64_t base = m0 - 1;
    const int nb = kCPairs + 1;
    const uint64_t win = rmask<uint64_t>(m_first, m_last, base, nb);
    PanelFrame fr;
    fr.init(g, base, nb, cut, R.R_w);
    if (wide) fr.ok = false;
    const LevelDev L = R.lev[lev];
    Bands bd;
    bd.n = 0;
    {
      const int64_t pa = max(base, m_first), pb = min(base + nb - 1, m_last);
      const int al = wide ? s + 2 : s + 1;
      const int64_t P = int64_t(1) << (wide ? s + 2 : s);
      const int64_t A = fl_sh(pa << s, al) << al;
      const int64_t B = (fl_sh(pb << s, al) + 1) << al;
      int64_t zlo[9], zhi[9];
      const int nz = make_zones(A, B, (int64_t)R.R_w * step_fx(g - 1), cut, P, R.chi_req, zlo, zhi);
      if (pa <= pb) bd.lookup(R, L, zlo, zhi, nz);
    }
    const int64_t lo_off = (int64_t)lev * R.n_lines;
    const int64_t X0 = m0 << s;
    const int64_t xa_t = base << s, xb_t = (base + nb) << s;
    const int64_t P_t = int64_t(1) << (wide ? s + 2 : s);
    const bool physical = R.shape < kShapeConst;
    const bool voigt = R.shape == kShapeVoigt;
    const int p = lane;
    float (*bE)[kCPairs + 1] = bufE[warp];
    float (*bO)[kCPairs + 1] = bufO[warp];
    unsigned long long* mk = smsk[warp];
    JobLine* jl = sJL[warp];
    uint16_t* ent = sEnt[warp];
    const float hnode = ldexpf(1.0f, s - 1 - kFixBits);  // node step, cm^-1
    float sL = 0.f, cL = 0.f, sR = 0.f, cR = 0.f, sM = 0.f, cM = 0.f;
    const int64_t n_cand = bd.total();
    BandCursor cur;
    for (int64_t t0 = 0; t0 < n_cand; t0 += 32) {  // warp-uniform
      const bool valid = t0 + lane < n_cand;
      const int64_t i = valid ? cur.line(bd, t0 + lane) : 0;
      uint64_t own = 0;
      int64_t c = 0;
      bool chi = false;
      if (valid) {
        c = __ldg(R.c + lo_off + i);
        const int gst = __ldg(R.gstar + lo_off + i);
        chi = __ldg(R.flags + lo_off + i) & 1;
        if (fr.ok) {
          const PanelPos pp = fr.pos(c);
          if (!owns_nothing_frame(fr, pp, g, gst, chi)) {
            own = accept_frame<uint64_t>(fr, pp, g, gst, chi) & win;
            if (own) own &= ~accept_parent_frame<uint64_t>(fr, pp, g, gst, chi);
          }
        } else if (!owns_nothing(g, c, gst, chi, cut, xa_t, xb_t, P_t)) {
          own = owned_any<uint64_t>(wide, g, c, gst, chi, cut, R.R_w, base, nb) & win;
        }
      }
      if (!__ballot_sync(0xffffffffu, own != 0)) continue;
      // even nodes 2p of the touched pairs, odd nodes 2p + 1 of the owned panels m0 + p
      const uint32_t tev = (uint32_t)(own | (own >> 1)), tod = (uint32_t)(own >> 1);
      // per branch (0 far, 1 6-term, 2 15-term, 3 small-y cell, 4 9 x 9 cell) the nodes
      uint32_t ce0 = 0, ce1 = 0, ce2 = 0, ce3 = 0, ce4 = 0, co0 = 0, co1 = 0, co2 = 0, co3 = 0, co4 = 0;
      if (own) {
        const float amp = __ldg(R.amp + lo_off + i);
        const float sx = __ldg(R.sx + lo_off + i);
        const float y = __ldg(R.yv + lo_off + i);
        NodeX nx;
        nx.init(X0 - c, s - 1, sx);
        JobLine J;
        J.qf = nx.qf; J.hs = nx.hs; J.phs = nx.phs; J.amp = amp;
        J.y = y; J.phi = nx.phi; J.cv = 1.0f; J.clr = 0.0f;
        J.mode = 0; J.cja = 0;
        J.r3 = J.r150 = J.r300 = J.l3 = J.l150 = J.l300 = 0;
        if (chi && physical) {
          ChiThr ct;
          ct.init(c, X0, s - 1, R.cut_fx);
          const int ja = max(__ffsll((long long)own) - 2, 0) * 2;
          const int jb = min(63 - __clzll((long long)own), kCPairs - 1) * 2 + 1;
          if (ct.uniform(ja, jb)) {
            ChiRun cr;
            cr.init(ct, ja, nx.absd((float)ja, s - 1), s - 1);
            J.mode = 1; J.cja = (int16_t)ja; J.cv = cr.v; J.clr = cr.lr;
          } else {
            J.mode = 2;
            J.r3 = clamp_node16(ct.r3); J.r150 = clamp_node16(ct.r150); J.r300 = clamp_node16(ct.r300);
            J.l3 = clamp_node16(ct.l3); J.l150 = clamp_node16(ct.l150); J.l300 = clamp_node16(ct.l300);
          }
        }
        jl[lane] = J;
        if (voigt) {
          // |x| boundaries T1 <= T2 <= T3 of the branches: below T1 a cell (small-y for
          // y < 1/4), T1..T2 the 15-term series (empty for y < 1), T2..T3 the 6-term
          // series, from T3 on the far wing
          const float y2 = y * y;
          const float T3 = sqrtf(fmaxf(1.0e4f - y2, 0.0f));
          const bool narrow = y < 1.0f;
          const float T1 = narrow ? 12.0f : sqrtf(fmaxf(20.25f - y2, 0.0f));
          const float T2 = narrow ? 12.0f : sqrtf(fmaxf(64.0f - y2, 0.0f));
          const float o = nx.qf + nx.phi;
          uint32_t e1, o1, e2, o2, e3, o3;
          far_side_pairs(T1, nx.hs, o, e1, o1);
          far_side_pairs(T2, nx.hs, o, e2, o2);
          far_side_pairs(T3, nx.hs, o, e3, o3);
          ce0 = tev & e3;       co0 = tod & o3;
          ce1 = tev & e2 & ~e3; co1 = tod & o2 & ~o3;
          ce2 = tev & e1 & ~e2; co2 = tod & o1 & ~o2;
          const uint32_t le = tev & ~e1, lo = tod & ~o1;
          const bool small = y < 0.25f;
          ce3 = small ? le : 0u; co3 = small ? lo : 0u;
          ce4 = small ? 0u : le; co4 = small ? 0u : lo;
        } else {
          ce0 = tev;
          co0 = tod;
        }
      }
      mk[lane] = own;
      // entries grouped by branch, each group in line (lane) order: inclusive scans of
      // the five counts, two 16-bit fields per word
      const int n0 = __popc(ce0) + __popc(co0), n1 = __popc(ce1) + __popc(co1), n2 = __popc(ce2) + __popc(co2),
                n3 = __popc(ce3) + __popc(co3), n4 = __popc(ce4) + __popc(co4);
      int a01 = n0 | (n1 << 16), a23 = n2 | (n3 << 16), a4 = n4;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v01 = __shfl_up_sync(0xffffffffu, a01, o);
        const int v23 = __shfl_up_sync(0xffffffffu, a23, o);
        const int v4 = __shfl_up_sync(0xffffffffu, a4, o);
        if (lane >= o) {
          a01 += v01;
          a23 += v23;
          a4 += v4;
        }
      }
      const int t01 = __shfl_sync(0xffffffffu, a01, 31), t23 = __shfl_sync(0xffffffffu, a23, 31);
      const int t4 = __shfl_sync(0xffffffffu, a4, 31);
      // this lane's first entry in each group
      const int b0 = (a01 & 0xffff) - n0;
      const int b1 = (t01 & 0xffff) + (a01 >> 16) - n1;
      const int b2 = (t01 & 0xffff) + (t01 >> 16) + (a23 & 0xffff) - n2;
      const int b3 = (t01 & 0xffff) + (t01 >> 16) + (t23 & 0xffff) + (a23 >> 16) - n3;
      const int b4 = (t01 & 0xffff) + (t01 >> 16) + (t23 & 0xffff) + (t23 >> 16) + a4 - n4;
      const int total = (t01 & 0xffff) + (t01 >> 16) + (t23 & 0xffff) + (t23 >> 16) + t4;
      // the list in chunks of kEntCap entries: each lane writes its entries that fall in
      // the chunk, then the warp evaluates the chunk, 32 entries per step
      for (int c0 = 0; c0 < total; c0 += kEntCap) {  // warp-uniform
        const int c1 = c0 + kEntCap;
        auto put = [&](int w, uint32_t me, uint32_t mo) {
          for (uint32_t m = me; m; m &= m - 1, ++w)
            if (w >= c0 && w < c1) ent[w - c0] = (uint16_t)((lane << 6) | (2 * (__ffs(m) - 1)));
          for (uint32_t m = mo; m; m &= m - 1, ++w)
            if (w >= c0 && w < c1) ent[w - c0] = (uint16_t)((lane << 6) | (2 * (__ffs(m) - 1) + 1));
        };
        put(b0, ce0, co0);
        put(b1, ce1, co1);
        put(b2, ce2, co2);
        put(b3, ce3, co3);
        put(b4, ce4, co4);
        __syncwarp();
        const int nc = min(total - c0, kEntCap);
#pragma unroll 1
        for (int e0 = 0; e0 < nc; e0 += 32) {  // warp-uniform
          const int e = e0 + lane;
          if (e >= nc) continue;
          const int en = ent[e];
          const int li = en >> 6, j = en & 63;
          const JobLine J = jl[li];
          const float jf = (float)j;
          const float xv = fmaf(jf + J.qf, J.hs, J.phs);
          float v = J.amp * (voigt ? voigt_K<false, false, true>(xv, J.y, kVoigtCells) : shape_f(R.shape, xv, J.y));
          if (J.mode == 1) {
            v *= J.clr != 0.0f ? J.cv * exp2f(J.clr * (float)(j - J.cja)) : J.cv;
          } else if (J.mode == 2) {
            const ChiThr ct{J.r3, J.r150, J.r300, J.l3, J.l150, J.l300};
            v *= ct.value(j, fabsf((jf + J.qf) + J.phi) * hnode);
          }
          if (!MARFA_DCHECK(li < 32 && j < 2 * kCPairs, 103)) continue;
          if (j & 1) bO[li][j >> 1] = v;
          else bE[li][j >> 1] = v;
          count_eval<COUNT>(voigt, xv, J.y, nev, nnear, nmid, nsmall);
        }
        __syncwarp();
      }
      // phase 2 (as in k_coarse): the staged lines owning pair p's panels, in line order
      uint32_t mine = warp_transpose32(tev, lane);
      while (mine) {
        const int t = __ffs(mine) - 1;
        mine &= mine - 1;
        const uint64_t m2 = mk[t];
        const float v0 = bE[t][p];
        if ((m2 >> (p + 1)) & 1ull) {
          kahan_add(sL, cL, v0);
          kahan_add(sM, cM, bO[t][p]);
        }
        if ((m2 >> p) & 1ull) kahan_add(sR, cR, v0);
      }
      __syncwarp();
    }
    float* gp = R.slots + (int64_t)lev * R.slots_per_level + R.slot_off[g];
    const int64_t np = R.npan[g];
    const int64_t m = m0 + p;
    if (m <= m_last && MARFA_DCHECK(m >= m_first, 104)) {
      gp[m - m_first] = sL + cL;
      gp[np + (m - m_first)] = sM + cM;
    }
    if (m - 1 >= m_first && m - 1 <= m_last) gp[2 * np + (m - 1 - m_first)] = sR + cR;
  }
  if (COUNT) block_counts<kCWarps>(nev, 0, nnear, nmid, nsmall, sCnt, counts);
}

void launch_coarse_jobs(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts, bool wide,
                        cudaStream_t st) {
  if (n_items <= 0) return;
  const int T = kCWarps * 32;
  if (counts) {
    if (wide)
      k_coarse_jobs<true, 1><<<n_items, T, 0, st>>>(reqs, items, counts);
    else
      k_coarse_jobs<true, 0><<<n_items, T, 0, st>>>(reqs, items, counts);
  } else if (wide) {
    k_coarse_jobs<false, 1><<<n_items, T, 0, st>>>(reqs, items, counts);
  } else {
    k_coarse_jobs<false, 0><<<n_items, T, 0, st>>>(reqs, items, counts);
  }
}

// ------------------------------------------------------------------ finest grid + cascade
// A CTA owns 1024 consecutive finest nodes of one level; warp w owns 128 of them
// (16 G10 panels of 8 nodes). Each warp loads 32 candidate lines at a time; the loading
// lane works out which of the warp's G10 panels the line leaves to the finest grid (not
// accepted on G10) and the node range within the cut-off, and stages them in shared
// memory. The warp then sums the staged lines over its nodes in four passes: in pass s
// the lane group gi = lane / 8 takes panel 4 s + gi and lane node 32 s + lane, and each
// group steps through the staged lines owning its panel in line order, so the eight
// lanes of a group evaluate one line at eight neighbouring nodes (one code path of the
// profile per group). Per-node compensated sums live in shared memory. Finally each node
// adds the quadratic interpolants of the ten coarse grids, and the CTA writes its
// outputs with aligned vector stores.
struct __align__(16) FineLine {
  int klo, khi;        // nodes of the warp in the cut-off
  float amp, y;
  float qf, hs, phs, phi;  // NodeX of the line relative to the warp's first node
};
struct __align__(16) FineChi {
  int r3, r150, r300, l3, l150, l300;  // ChiThr relative to the warp's first node
  int on, pad;                          // chi-factor applies
};

// The 3-point cascade at the four nodes k0 + q of a thread: the quadratic through
// (0, vL), (1, vM), (2, vR) of a coarse grid's panel, in t (steps of h_g from the
// panel's left node), is vL + t (c1 + t c2); the nodes sit at t0 + q dt, so it is
// a + q (b + q c) there, and the ten grids' a, b, c add up. Only for threads with a
// node inside the window (the slots exist there).
struct Cascade3 {
  float a, b, c;
};

__device__ __forceinline__ Cascade3 cascade3(const ReqDev& R, int lev, int64_t k0) {
  Cascade3 r{0.0f, 0.0f, 0.0f};
  const float* sl = R.slots + (int64_t)lev * R.slots_per_level;
#pragma unroll
  for (int g = 1; g <= kNGrid; ++g) {
    const int sh = 13 - g;  // finest nodes per panel of grid g: 2^(13-g)
    const int64_t np = R.npan[g];
    const float* gp = sl + R.slot_off[g];
    const int64_t m = k0 >> sh;
    const int64_t idx = m - R.m_first[g];
    float vL = __ldg(gp + idx), vM = __ldg(gp + np + idx), vR = __ldg(gp + 2 * np + idx);
    if (g == 1) {  // the g1_split partial copies of grid 1, summed in part order
#pragma unroll
      for (int part = 1; part < kG1Split; ++part)
        if (part < R.g1_split) {  // loads issued together, not one round trip per part
          const float* gq = gp + 3 * np * part;
          vL += __ldg(gq + idx);
          vM += __ldg(gq + np + idx);
          vR += __ldg(gq + 2 * np + idx);
        }
    }
    const float c1 = 0.5f * fmaf(-3.0f, vL, fmaf(4.0f, vM, -vR));
    const float c2 = 0.5f * fmaf(-2.0f, vM, vL + vR);
    const float dt = ldexpf(1.0f, 1 - sh);
    const float t0 = (float)(int)(k0 - (m << sh)) * dt;
    r.a += fmaf(t0, fmaf(t0, c2, c1), vL);
    r.b += dt * fmaf(2.0f * t0, c2, c1);
    r.c += (dt * dt) * c2;
  }
  return r;
}

// Whether any of the thread's nodes k0 .. k0 + 3 lies inside the window.
__device__ __forceinline__ bool fine_lane_valid(const ReqDev& R, int64_t k0) {
  return k0 + kFinePerThread - 1 >= R.k_lo && k0 <= R.k_hi;
}

// The finest-grid epilogue shared by the finest-grid kernels: node k0 + q of this thread
// holds out[q] (its finest-grid sum); add the quadratic (quartic: 5-point variant)
// through the panel-local slots of every coarse grid, scale, and write the CTA's tile
// [it.k0, it.k0 + kFineTile) of level lev to the output with aligned vector stores.
// Every thread of the CTA calls it (it ends with a CTA barrier and the stores). pre: the
// 3-point cascade when the caller computed it already (cascade3), else null.
__device__ __forceinline__ void fine_cascade_store(const ReqDev& R, const FineItem& it, int lev, bool wide,
                                                   int64_t k0, float (&out)[kFinePerThread], float* tile,
                                                   const Cascade3* pre = nullptr) {
  const int tid = threadIdx.x;
  if (fine_lane_valid(R, k0)) {
    if (!wide) {
      const Cascade3 cc = pre ? *pre : cascade3(R, lev, k0);
#pragma unroll
      for (int q = 0; q < kFinePerThread; ++q) out[q] += fmaf((float)q, fmaf((float)q, cc.c, cc.b), cc.a);
    } else {
      // 5-point: the four-step panel M4 is two-step panels 2 M4, 2 M4 + 1 (m_first is
      // even); its nodes are L, M, R of the first and M, R of the second
      const float* sl = R.slots + (int64_t)lev * R.slots_per_level;
#pragma unroll
      for (int g = 1; g <= kNGrid; ++g) {
        const int sh = 13 - g;  // finest nodes per panel of grid g: 2^(13-g)
        const int64_t np = R.npan[g];
        const float* gp = sl + R.slot_off[g];
        const int64_t M4 = k0 >> (sh + 1);
        const int64_t i0 = 2 * M4 - R.m_first[g];
        float v0 = __ldg(gp + i0), v1 = __ldg(gp + np + i0), v2 = __ldg(gp + 2 * np + i0);
        float v3 = __ldg(gp + np + i0 + 1), v4 = __ldg(gp + 2 * np + i0 + 1);
        if (g == 1) {  // the g1_split partial copies of grid 1, summed in part order
          for (int part = 1; part < R.g1_split; ++part) {
            const float* gq = gp + 3 * np * part;
            v0 += __ldg(gq + i0);
            v1 += __ldg(gq + np + i0);
            v2 += __ldg(gq + 2 * np + i0);
            v3 += __ldg(gq + np + i0 + 1);
            v4 += __ldg(gq + 2 * np + i0 + 1);
          }
        }
        const int off0 = (int)(k0 - (M4 << (sh + 1)));
        const float inv_h = ldexpf(1.0f, 1 - sh);
#pragma unroll
        for (int q = 0; q < kFinePerThread; ++q) {
          const float t = (float)(off0 + q) * inv_h;  // position in steps of h_g, [0, 4)
          const float d1 = t - 1.0f, d2 = t - 2.0f, d3 = t - 3.0f, d4 = t - 4.0f;
          // quartic Lagrange weights of the nodes 0..4
          const float w0 = (d1 * d2) * (d3 * d4) * (1.0f / 24.0f);
          const float w1 = -(t * d2) * (d3 * d4) * (1.0f / 6.0f);
          const float w2 = (t * d1) * (d3 * d4) * 0.25f;
          const float w3 = -(t * d1) * (d2 * d4) * (1.0f / 6.0f);
          const float w4 = (t * d1) * (d2 * d3) * (1.0f / 24.0f);
          out[q] += fmaf(v0, w0, fmaf(v1, w1, fmaf(v2, w2, fmaf(v3, w3, v4 * w4))));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kFinePerThread; ++q) tile[kFinePerThread * tid + q] = out[q] * R.out_scale;
  }
  __syncthreads();
  // write the valid part [a, b] of the tile
  const int64_t a = max(it.k0, R.k_lo), b = min(it.k0 + kFineTile - 1, R.k_hi);
  if (a <= b && MARFA_DCHECK(a - R.k_lo >= 0 && b - R.k_lo < R.npts, 203)) {
    float* row = R.out + (int64_t)lev * R.npts;
    const int64_t i0 = a - R.k_lo;           // first output index
    const int n = (int)(b - a + 1);
    const int t0 = (int)(a - it.k0);         // its position in the tile
    float* dst = row + i0;
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
}

template <bool COUNT, bool SURR, int WIDE>
__global__ void __launch_bounds__(kFineThreads)
    k_fine(const ReqDev* __restrict__ reqs, const FineItem* __restrict__ items,
           int64_t* __restrict__ counts) {
  constexpr int NW = kFineThreads / 32;
  constexpr int kWarpNodes = kFinePerThread * 32;  // nodes of a warp
  extern __shared__ __align__(16) unsigned char dsm[];  // surrogate weights (SURR only)
  MlpWeights& S = *reinterpret_cast<MlpWeights*>(dsm);
  __shared__ float tile[kFineTile];
  __shared__ __align__(16) float stab[kVoigtTableFloats];
  __shared__ FineLine sL[NW][32];  // staged lines, one per lane of each warp
  __shared__ FineChi sC[NW][32];
  __shared__ __align__(16) float sAcc[NW][kWarpNodes], sCmp[NW][kWarpNodes];
  __shared__ int64_t red[kCountFields][NW];
  const FineItem it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const bool wide = WIDE == 2 ? R.wide != 0 : WIDE == 1;  // 5-point partition
  const int lev = it.level;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool use_mlp = SURR && R.mlp != nullptr;  // block-uniform
  voigt_table_to_smem(stab);
  if (use_mlp) mlp_load_smem(S, R.mlp);
#pragma unroll
  for (int q = 0; q < kFinePerThread; ++q) sAcc[warp][32 * q + lane] = sCmp[warp][32 * q + lane] = 0.0f;
  const int64_t kw = it.k0 + (int64_t)kWarpNodes * warp;  // first node of the warp
  const int64_t k0 = kw + kFinePerThread * lane;           // first node of the lane's output
  const int64_t cut = R.cut_fx;
  const LevelDev L = R.lev[lev];
  const int wlo = (int)max(R.k_lo - kw, (int64_t)0);
  const int whi = (int)min(R.k_hi - kw, (int64_t)(kWarpNodes - 1));
  const int64_t Xa = kw << kFineShift;  // position of the warp's first node
  // the warp's candidate bands, looked up before the barrier (global loads only), so
  // that their latency overlaps the table copy
  Bands bd;
  bd.n = 0;
  if (wlo <= whi) {  // warp-uniform
    // the span of the warp's nodes inside the window
    const int64_t P10 = int64_t(1) << panel_shift(kNGrid);
    int64_t zlo[9], zhi[9];
    const int nz = make_zones((kw + wlo) << kFineShift, (kw + whi) << kFineShift, (int64_t)R.R_w * step_fx(kNGrid),
                              cut, wide ? P10 << 1 : P10, R.chi_req, zlo, zhi);
    bd.lookup(R, L, zlo, zhi, nz);
  }
  __syncthreads();
  int64_t nev = 0, nmlp = 0, nnear = 0, nmid = 0, nsmall = 0;
  int qn = 0;  // entries in this warp's surrogate queue (warp-uniform)
  // surrogate results: the tag is the warp node
  auto fine_apply = [&](int tag, float v) { kahan_add(sAcc[warp][tag], sCmp[warp][tag], v); };
  if (wlo <= whi) {  // warp-uniform
    const int64_t pbase = kw >> 3;  // first G10 panel of the warp
    const int64_t lo_off = (int64_t)lev * R.n_lines;
    const bool physical = R.shape < kShapeConst;
    const bool voigt = R.shape == kShapeVoigt;
    const int gi = lane >> 3;  // lane group
    const int64_t n_cand = bd.total();
    BandCursor cur;
    for (int64_t t0 = 0; t0 < n_cand; t0 += 32) {  // warp-uniform
      const bool valid = t0 + lane < n_cand;
      const int64_t i = valid ? cur.line(bd, t0 + lane) : 0;
      uint32_t pm = 0;
      int klo = 0, khi = -1;
      int64_t c = 0;
      bool chi = false;
      if (valid) {
        c = __ldg(R.c + lo_off + i);
        const int gst = __ldg(R.gstar + lo_off + i);
        chi = __ldg(R.flags + lo_off + i) & 1;
        klo = (int)max(cl_sh(c - cut, kFineShift) - kw, (int64_t)wlo);
        khi = (int)min(fl_sh(c + cut, kFineShift) - kw, (int64_t)whi);
        if (klo <= khi) {
          const int s10 = panel_shift(kNGrid);  // acceptance panels of grid 10: two (four) steps
          pm = ~accept_mask_s<uint32_t>(kNGrid, c, gst, chi, cut, R.R_w, pbase, 16, s10 + wide, s10) &
               rmask<uint32_t>(klo >> 3, khi >> 3, 0, 16);
        }
      }
      if (!__ballot_sync(0xffffffffu, pm != 0)) continue;
      __syncwarp();
      if (pm) {
        NodeX nx;
        nx.init(Xa - c, kFineShift, __ldg(R.sx + lo_off + i));
        FineLine fl;
        fl.klo = klo;
        fl.khi = khi;
        fl.amp = __ldg(R.amp + lo_off + i);
        fl.y = __ldg(R.yv + lo_off + i);
        fl.qf = nx.qf;
        fl.hs = nx.hs;
        fl.phs = nx.phs;
        fl.phi = nx.phi;
        sL[warp][lane] = fl;
        FineChi fc;
        fc.on = chi && physical;
        if (fc.on) {
          ChiThr ct;
          ct.init(c, Xa, kFineShift, R.cut_fx);
          fc.r3 = ct.r3; fc.r150 = ct.r150; fc.r300 = ct.r300;
          fc.l3 = ct.l3; fc.l150 = ct.l150; fc.l300 = ct.l300;
          // within 3 cm^-1 of the centre at all its nodes of the warp: chi = 1 exactly
          if (ct.uniform(klo, khi) && ct.branch(klo) == 0) fc.on = 0;
        }
        sC[warp][lane] = fc;
      }
      __syncwarp();
      // lane q < 16: the staged lines owning panel q (a 32 x 32 bit transpose of the masks)
      const uint32_t pcol = warp_transpose32(pm, lane);
#pragma unroll 1
      for (int s = 0; s < kFinePerThread; ++s) {
        // the staged lines owning this group's panel 4 s + gi
        uint32_t mine = __shfl_sync(0xffffffffu, pcol, 4 * s + gi);
        if (!__any_sync(0xffffffffu, mine != 0)) continue;
        const int j = 32 * s + lane;
        const float jf = (float)j;
        if (SURR && use_mlp) {
          // groups step together; evaluations that pass the guard go to the warp's queue
          while (__any_sync(0xffffffffu, mine != 0)) {
            if (qn > kQCap - 32) q_flush(warp_queue(dsm), qn, S, fine_apply);
            int e = -1;
            if (mine) {
              e = __ffs(mine) - 1;
              mine &= mine - 1;
            }
            const FineLine fl = sL[warp][e < 0 ? 0 : e];
            const bool act = e >= 0 && j >= fl.klo && j <= fl.khi;
            const float y = act ? fl.y : 1.0f;
            const float xv = fmaf(jf + fl.qf, fl.hs, fl.phs);
            const bool use = act && mlp_guard(S, xv, y);
            float cv = 1.0f;
            if (act && sC[warp][e].on) {
              const FineChi fc = sC[warp][e];
              const ChiThr ct{fc.r3, fc.r150, fc.r300, fc.l3, fc.l150, fc.l300};
              cv = ct.value(j, fabsf((jf + fl.qf) + fl.phi) * ldexpf(1.0f, -kFineBits));
            }
            q_push(warp_queue(dsm), qn, use, xv, y, fl.amp * cv, j);
            if (act && !use) {
              float v = fl.amp * voigt_K<true>(xv, y, stab);
              v *= cv;
              kahan_add(sAcc[warp][j], sCmp[warp][j], v);
            }
            if (act) count_eval<COUNT>(true, xv, y, nev, nnear, nmid, nsmall);
            if (COUNT && use) ++nmlp;
          }
        } else {
          float a = sAcc[warp][j], cp = sCmp[warp][j];
          while (mine) {  // uniform within a group
            const int e = __ffs(mine) - 1;
            mine &= mine - 1;
            const FineLine fl = sL[warp][e];
            if (j < fl.klo || j > fl.khi) continue;
            const float xv = fmaf(jf + fl.qf, fl.hs, fl.phs);
            float v = fl.amp * (voigt ? voigt_K<true, false, true>(xv, fl.y, stab) : shape_f(R.shape, xv, fl.y));
            if (sC[warp][e].on) {
              const FineChi fc = sC[warp][e];
              const ChiThr ct{fc.r3, fc.r150, fc.r300, fc.l3, fc.l150, fc.l300};
              v *= ct.value(j, fabsf((jf + fl.qf) + fl.phi) * ldexpf(1.0f, -kFineBits));
            }
            kahan_add(a, cp, v);
            count_eval<COUNT>(voigt, xv, fl.y, nev, nnear, nmid, nsmall);
          }
          sAcc[warp][j] = a;
          sCmp[warp][j] = cp;
        }
      }
      __syncwarp();
    }
  }
  if (SURR && use_mlp) q_flush(warp_queue(dsm), qn, S, fine_apply);  // warp-uniform
  __syncwarp();
  {
    float out[kFinePerThread];
#pragma unroll
    for (int q = 0; q < kFinePerThread; ++q)
      out[q] = sAcc[warp][kFinePerThread * lane + q] + sCmp[warp][kFinePerThread * lane + q];
    fine_cascade_store(R, it, lev, wide, k0, out, tile);
  }
  if (COUNT) block_counts<NW>(nev, nmlp, nnear, nmid, nsmall, red, counts);
}

// The finest grid with flattened jobs. The tiles, candidate bands and staged lines are
// those of k_fine; what differs is how a warp spreads the evaluations over its lanes.
// A job is one staged line on one of the warp's 16 G10 panels (eight nodes, one per
// lane of an 8-lane group). The round's jobs form one list, far-wing jobs first (the
// two-term series, at the panel's centre |z| >= 100), then the others, each part in line
// order, so that the four groups of a warp step mostly evaluate the same line on
// neighbouring panels (one branch of the Voigt function) and no group waits for another
// group's longer list. Group gi of a step adds into its own accumulator row (plain FP32;
// the four rows of a node are merged with TwoSum in the epilogue), so the order of every
// sum is fixed by the job list: results are deterministic.
struct __align__(16) FineChi16 {
  int16_t r3, r150, r300, l3, l150, l300;  // ChiThr relative to the warp's first node, clamped
  int16_t on, pad;
};

// MECH (1 or 2): where the centre region, cut-off edges and chi breakpoints lie apart
// (mech_fine_ok), a candidate's nodes come in closed form (mech_fine_*). With MECH = 1
// the candidates come in one pass per mechanism: the centre pass takes the lines with
// g* = 11 (chi = 1 there: the region lies inside the first breakpoint), the edge and
// breakpoint passes the lines whose edge or breakpoint falls near the warp's nodes. With
// MECH = 2 the centre pass is followed by one pass over the merged ranges of all edges
// and breakpoints (fewer rounds of staging); a candidate's nodes in the warp then come
// from one mechanism (mech_fine_merge_ok: they lie more than a warp's span apart).
template <bool COUNT, int WIDE, int MECH>
__global__ void __launch_bounds__(kFineThreads, 4)
    k_fine_jobs(const ReqDev* __restrict__ reqs, const FineItem* __restrict__ items,
                int64_t* __restrict__ counts) {
  constexpr int NW = kFineThreads / 32;
  constexpr int kWarpNodes = kFinePerThread * 32;  // 128 nodes = 16 G10 panels
  __shared__ __align__(16) float stab[kVoigtTableFloats];
  __shared__ FineLine sL[NW][32];
  __shared__ FineChi16 sC[NW][32];
  // per job group gi a row over the CTA's nodes (dynamic shared memory, kFineJobsDyn
  // bytes); row 0 doubles as the output tile (a lane reads its four nodes of every row
  // before it overwrites them in row 0)
  extern __shared__ __align__(16) unsigned char dsm[];
  float (*sAcc)[NW * kWarpNodes] = reinterpret_cast<float (*)[NW * kWarpNodes]>(dsm);
  __shared__ uint16_t sJob[NW][32 * 16];
  __shared__ int64_t red[kCountFields][NW];
  const FineItem it = items[blockIdx.x];
  const ReqDev& R = reqs[it.req];
  const bool wide = WIDE == 1;
  const int lev = it.level;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  voigt_table_to_smem(stab);
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int q = 0; q < kFinePerThread; ++q) sAcc[g][kWarpNodes * warp + 32 * q + lane] = 0.0f;
  const int64_t kw = it.k0 + (int64_t)kWarpNodes * warp;  // first node of the warp
  const int64_t k0 = kw + kFinePerThread * lane;           // first node of the lane's output
  const int64_t cut = R.cut_fx;
  const LevelDev L = R.lev[lev];
  const int wlo = (int)max(R.k_lo - kw, (int64_t)0);
  const int whi = (int)min(R.k_hi - kw, (int64_t)(kWarpNodes - 1));
  const int64_t Xa = kw << kFineShift;
  const int64_t P10 = int64_t(1) << panel_shift(kNGrid);
  Bands bd;
  bd.n = 0;
  if (MECH == 0 && wlo <= whi) {
    int64_t zlo[9], zhi[9];
    const int nz = make_zones((kw + wlo) << kFineShift, (kw + whi) << kFineShift, (int64_t)R.R_w * step_fx(kNGrid),
                              cut, wide ? P10 << 1 : P10, R.chi_req, zlo, zhi);
    bd.lookup(R, L, zlo, zhi, nz);
  }
  // the coarse grids' cascade (3-point), loaded now so that its latency overlaps the
  // summation instead of the end of the CTA
  Cascade3 cc{0.0f, 0.0f, 0.0f};
  if (!wide && fine_lane_valid(R, k0)) cc = cascade3(R, lev, k0);
  __syncthreads();
  int64_t nev = 0, nnear = 0, nmid = 0, nsmall = 0;
  int nB = 0;
  if (MECH && R.chi_req)
    for (int b = 0; b < 3 && chi_break_fx(b) <= cut; ++b) nB = b + 1;
  const int nmech = 3 + 2 * nB;  // centre, two cut-off edges, two per breakpoint
  const int npass = MECH == 1 ? nmech : (MECH == 2 ? 2 : 1);
  // the mechanism of pass q sits at c + off(q) (MECH only)
  auto pass_off = [&](int q) {
    return q == 0 ? (int64_t)0
         : q == 1 ? cut
         : q == 2 ? -cut
         : ((q & 1) ? chi_break_fx((q - 3) >> 1) : -chi_break_fx((q - 3) >> 1));
  };
  // MECH: every mechanism's candidate range at once (lane 2q: first line, 2q + 1: end)
  int64_t range_v = 0;
  if (MECH && wlo <= whi && lane < 2 * nmech) {
    const int q = lane >> 1;
    const int64_t off = pass_off(q);
    const int64_t reach = (q == 0 ? (int64_t)R.R_w * step_fx(kNGrid) : 0) + P10 + 1;
    range_v = (lane & 1) ? upper_idx(R, ((kw + whi) << kFineShift) + reach - off - L.smin)
                         : lower_idx(R, ((kw + wlo) << kFineShift) - reach - off - L.smax);
  }
  for (int pass = 0; pass < npass && wlo <= whi; ++pass) {  // warp-uniform
    const int64_t off = pass_off(pass);
    // one mechanism: one range of candidates (first line r_lo) kept in registers;
    // otherwise the bands
    const bool one_range = MECH == 1 || (MECH == 2 && pass == 0);
    int64_t r_lo = 0, r_n = 0;
    if (one_range) {
      r_lo = __shfl_sync(0xffffffffu, range_v, 2 * pass);
      r_n = max(__shfl_sync(0xffffffffu, range_v, 2 * pass + 1) - r_lo, (int64_t)0);
    } else if (MECH == 2) {  // the edges' and breakpoints' ranges, merged
      bd.n = 0;
      for (int q = 1; q < nmech; ++q) {
        const int64_t a = __shfl_sync(0xffffffffu, range_v, 2 * q);
        const int64_t b = __shfl_sync(0xffffffffu, range_v, 2 * q + 1);
        if (a < b) {
          bd.lo[bd.n] = a;
          bd.hi[bd.n] = b;
          ++bd.n;
        }
      }
      bd.merge();
    }
    const int64_t pbase = kw >> 3;
    // MECH = 1: the chi branch along an edge (eb), and the breakpoint of a breakpoint
    // pass (kb, on the right of the centre when kr)
    const int eb = (cut >= chi_break_fx(0)) + (cut > chi_break_fx(1)) + (cut > chi_break_fx(2));
    const float eC = eb == 1 ? 1.084f : (eb == 2 ? 0.208f : 0.025f);
    const float er = eb == 1 ? 0.027f : (eb == 2 ? 0.016f : 0.009f);
    const int kb = (pass - 3) >> 1;
    const bool kr = pass & 1;
    const int64_t lo_off = (int64_t)lev * R.n_lines;
    const bool physical = R.shape < kShapeConst;
    const bool voigt = R.shape == kShapeVoigt;
    const int gi = lane >> 3, t8 = lane & 7;
    const int64_t n_cand = one_range ? r_n : bd.total();
    BandCursor cur;
    uint16_t* jobs = sJob[warp];
    for (int64_t t0 = 0; t0 < n_cand; t0 += 32) {  // warp-uniform
      const bool valid = t0 + lane < n_cand;
      const int64_t i = valid ? (one_range ? r_lo + t0 + lane : cur.line(bd, t0 + lane)) : 0;
      // the line's data with its position (consecutive lines: coalesced), so that a
      // candidate costs one round trip to memory
      float amp_p = 0.0f, sx_p = 0.0f, y_p = 0.0f;
      if (valid) {
        amp_p = __ldg(R.amp + lo_off + i);
        sx_p = __ldg(R.sx + lo_off + i);
        y_p = __ldg(R.yv + lo_off + i);
      }
      uint32_t pm = 0;
      int klo = 0, khi = -1;
      int64_t c = 0;
      bool chi = false;
      if (valid && MECH == 2 && pass == 1) {
        c = __ldg(R.c + lo_off + i);
        chi = __ldg(R.flags + lo_off + i) & 1;
        const int64_t lo = kw + wlo, hi = kw + whi;
        int64_t a = 1, b = 0, a2, b2;
        int found = 0;
        auto take = [&](int64_t x, int64_t y) {
          x = max(x, lo);
          y = min(y, hi);
          if (x <= y) {
            a = x;
            b = y;
            ++found;
          }
        };
        mech_fine_edge_right(c + cut, a2, b2);
        take(a2, b2);
        mech_fine_edge_left(c - cut, a2, b2);
        take(a2, b2);
        if (chi)
          for (int q = 0; q < nB; ++q) {
            mech_fine_kink(c + chi_break_fx(q), a2, b2);
            take(a2, b2);
            mech_fine_kink(c - chi_break_fx(q), a2, b2);
            take(a2, b2);
          }
        if (found && MARFA_DCHECK(found == 1, 204)) {
          klo = (int)(a - kw);
          khi = (int)(b - kw);
          pm = rmask<uint32_t>(klo >> 3, khi >> 3, 0, 16);
        }
      } else if (valid && MECH) {  // one mechanism: pass 0 the centre
        c = __ldg(R.c + lo_off + i);
        int64_t a = 1, b = 0;
        if (pass == 0) {
          mech_fine_centre(c, __ldg(R.gstar + lo_off + i), R.R_w, a, b);
        } else {
          chi = __ldg(R.flags + lo_off + i) & 1;
          if (pass == 1) mech_fine_edge_right(c + cut, a, b);
          else if (pass == 2) mech_fine_edge_left(c - cut, a, b);
          else if (chi) mech_fine_kink(c + off, a, b);
        }
        klo = (int)max(min(a - kw, (int64_t)kWarpNodes), (int64_t)wlo);
        khi = (int)min(max(b - kw, (int64_t)-1), (int64_t)whi);
        if (klo <= khi) pm = rmask<uint32_t>(klo >> 3, khi >> 3, 0, 16);
      } else if (valid) {
        c = __ldg(R.c + lo_off + i);
        const int gst = __ldg(R.gstar + lo_off + i);
        chi = __ldg(R.flags + lo_off + i) & 1;
        klo = (int)max(cl_sh(c - cut, kFineShift) - kw, (int64_t)wlo);
        khi = (int)min(fl_sh(c + cut, kFineShift) - kw, (int64_t)whi);
        if (klo <= khi) {
          const int s10 = panel_shift(kNGrid);
          pm = ~accept_mask_s<uint32_t>(kNGrid, c, gst, chi, cut, R.R_w, pbase, 16, s10 + wide, s10) &
               rmask<uint32_t>(klo >> 3, khi >> 3, 0, 16);
        }
      }
      if (!__ballot_sync(0xffffffffu, pm != 0)) continue;
      __syncwarp();  // the previous round's jobs are done with the staged lines
      uint32_t far = 0;
      if (pm) {
        NodeX nx;
        nx.init(Xa - c, kFineShift, sx_p);
        FineLine fl;
        fl.klo = klo;
        fl.khi = khi;
        fl.amp = amp_p;
        fl.y = y_p;
        fl.qf = nx.qf;
        fl.hs = nx.hs;
        fl.phs = nx.phs;
        fl.phi = nx.phi;
        sL[warp][lane] = fl;
        FineChi16 fc{};  // thresholds 0 where chi is off (read, then not used)
        fc.on = chi && physical && !(MECH && pass == 0);
        fc.pad = 0;
        if (fc.on && MECH == 1 && pass <= 2) {
          fc.on = eb > 0;  // a cut-off edge: one branch of Eq. (10) at all its nodes
        } else if (fc.on && MECH == 1) {
          // a breakpoint: the branch changes only at its own threshold near these nodes
          const int64_t rel = c + (kr ? chi_break_fx(kb) : -chi_break_fx(kb)) - Xa;
          fc.r3 = clamp_node16(clamp32((kr == (kb == 0)) ? cl_sh(rel, kFineShift) : fl_sh(rel, kFineShift)));
        } else if (fc.on) {
          ChiThr ct;
          ct.init(c, Xa, kFineShift, R.cut_fx);
          fc.r3 = clamp_node16(ct.r3); fc.r150 = clamp_node16(ct.r150); fc.r300 = clamp_node16(ct.r300);
          fc.l3 = clamp_node16(ct.l3); fc.l150 = clamp_node16(ct.l150); fc.l300 = clamp_node16(ct.l300);
          if (ct.uniform(klo, khi) && ct.branch(klo) == 0) fc.on = 0;
        }
        sC[warp][lane] = fc;
        if (voigt && MECH == 1) {
          // by mechanism: a core (g* = 11, within R_w h_10 of the centre) lies in the near
          // wing, an edge or a breakpoint in the far wing (the order of the job list only)
          far = pass == 0 ? 0u : pm;
        } else if (voigt) {
          // panels whose centre node lies in the far wing |z| >= 100: |j + q + phi| hs >= X
          // (the order of the job list only: approximate square root and division)
          const float X2 = fmaxf(1.0e4f - fl.y * fl.y, 1.0e-30f);
          const float t = fminf(__fdividef(X2 * rsqrtf(X2), fl.hs), 1.0e6f);
          const float off = 3.5f + nx.qf + nx.phi;  // centre node of panel p is 8 p + 3.5
          const int pr = (int)ceilf(fmaxf((t - off) * 0.125f, -1.0f));    // first far panel right of c
          const int pl = (int)floorf(fminf((-t - off) * 0.125f, 17.0f));  // last far panel left of c
          far = (rmask<uint32_t>(pr, 15, 0, 16) | rmask<uint32_t>(0, pl, 0, 16)) & pm;
        }
      }
      // job list: far jobs, then the rest, each in line order (lane order, then panel)
      const int nf = __popc(far), nn = __popc(pm & ~far);
      int pre = nf | (nn << 16);  // inclusive scan of both counts at once
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
      }
      const int tot = __shfl_sync(0xffffffffu, pre, 31);
      const int F = tot & 0xffff, J = F + (tot >> 16);
      int pf = (pre & 0xffff) - nf, pn = F + (pre >> 16) - nn;
      for (uint32_t m = far; m; m &= m - 1)
        if (MARFA_DCHECK(pf < 32 * 16, 201)) jobs[pf++] = (uint16_t)((lane << 4) | (__ffs(m) - 1));
      for (uint32_t m = pm & ~far; m; m &= m - 1)
        if (MARFA_DCHECK(pn < 32 * 16, 201)) jobs[pn++] = (uint16_t)((lane << 4) | (__ffs(m) - 1));
      __syncwarp();
      float* acc = &sAcc[gi][kWarpNodes * warp];
#pragma unroll 1
      for (int e0 = 0; e0 < J; e0 += 4) {  // warp-uniform
        const int e = e0 + gi;
        if (e >= J) continue;
        const int job = jobs[e];
        const int li = job >> 4;
        const int jn = 8 * (job & 15) + t8;
        const FineLine fl = sL[warp][li];
        // a lane outside the line's nodes evaluates its group's nearest node (the same
        // branch of the Voigt function: no divergence) and adds zero to its own node
        const bool inr = jn >= fl.klo && jn <= fl.khi;
        const int j = min(max(jn, fl.klo), fl.khi);
        const float jf = (float)j;
        const float xv = fmaf(jf + fl.qf, fl.hs, fl.phs);
        float v = fl.amp * (voigt ? voigt_K<true, false, true>(xv, fl.y, stab) : shape_f(R.shape, xv, fl.y));
        if (!(MECH && pass == 0)) {  // chi = 1 in the centre region
          // the chi factor by select (the groups of a step take different lines)
          const FineChi16 fc = sC[warp][li];
          const float absd = fabsf((jf + fl.qf) + fl.phi) * ldexpf(1.0f, -kFineBits);
          float cv;
          if (MECH == 1 && pass <= 2) {  // an edge: its one branch
            cv = eC * __expf(-er * absd);
          } else if (MECH == 1) {  // a breakpoint: the branch from its threshold (in r3)
            const int kthr = fc.r3;
            const bool beyond = kr ? (kb == 0 ? j >= kthr : j > kthr) : (kb == 0 ? j <= kthr : j < kthr);
            const int br = kb + (beyond ? 1 : 0);
            const float C = br == 1 ? 1.084f : (br == 2 ? 0.208f : 0.025f);
            const float r = br == 1 ? 0.027f : (br == 2 ? 0.016f : 0.009f);
            const float e = C * __expf(-r * absd);
            cv = br == 0 ? 1.0f : e;
          } else {
            const ChiThr ct{fc.r3, fc.r150, fc.r300, fc.l3, fc.l150, fc.l300};
            cv = ct.value_sel(j, absd);
          }
          v *= fc.on ? cv : 1.0f;
        }
        if (MARFA_DCHECK(jn >= 0 && jn < kWarpNodes, 202)) acc[jn] += inr ? v : 0.0f;
        if (inr) count_eval<COUNT>(voigt, xv, fl.y, nev, nnear, nmid, nsmall);
      }
      __syncwarp();
    }
  }
  __syncwarp();
  float out[kFinePerThread];
#pragma unroll
  for (int q = 0; q < kFinePerThread; ++q) {
    const int n = kFinePerThread * tid + q;
    float s_ = sAcc[0][n], c_ = 0.0f;
    comp_merge(s_, c_, sAcc[1][n], 0.0f);
    comp_merge(s_, c_, sAcc[2][n], 0.0f);
    comp_merge(s_, c_, sAcc[3][n], 0.0f);
    out[q] = s_ + c_;
  }
  fine_cascade_store(R, it, lev, wide, k0, out, sAcc[0], &cc);
  if (COUNT) block_counts<NW>(nev, 0, nnear, nmid, nsmall, red, counts);
}

constexpr size_t kFineJobsDyn = sizeof(float) * 4 * kFineTile;

void launch_fine_jobs(const ReqDev* reqs, const FineItem* items, int n_items, int64_t* counts, bool wide,
                      int mech, cudaStream_t st) {
  if (n_items <= 0) return;
  const size_t B = kFineJobsDyn;
  if (mech == 1) {  // 3-point only
    if (counts)
      launch_dyn(k_fine_jobs<true, 0, 1>, n_items, kFineThreads, B, st, reqs, items, counts);
    else
      launch_dyn(k_fine_jobs<false, 0, 1>, n_items, kFineThreads, B, st, reqs, items, counts);
  } else if (mech == 2) {
    if (counts)
      launch_dyn(k_fine_jobs<true, 0, 2>, n_items, kFineThreads, B, st, reqs, items, counts);
    else
      launch_dyn(k_fine_jobs<false, 0, 2>, n_items, kFineThreads, B, st, reqs, items, counts);
  } else if (counts) {
    if (wide)
      launch_dyn(k_fine_jobs<true, 1, 0>, n_items, kFineThreads, B, st, reqs, items, counts);
    else
      launch_dyn(k_fine_jobs<true, 0, 0>, n_items, kFineThreads, B, st, reqs, items, counts);
  } else if (wide) {
    launch_dyn(k_fine_jobs<false, 1, 0>, n_items, kFineThreads, B, st, reqs, items, counts);
  } else {
    launch_dyn(k_fine_jobs<false, 0, 0>, n_items, kFineThreads, B, st, reqs, items, counts);
  }
}

void launch_fine(const ReqDev* reqs, const FineItem* items, int n_items, int64_t* counts, bool surr,
                 bool wide, cudaStream_t st) {
  if (n_items <= 0) return;
  if (surr) {
    if (counts)
      launch_surr(k_fine<true, true, 2>, n_items, kFineThreads, st, reqs, items, counts);
    else
      launch_surr(k_fine<false, true, 2>, n_items, kFineThreads, st, reqs, items, counts);
  } else if (counts) {
    k_fine<true, false, 2><<<n_items, kFineThreads, 0, st>>>(reqs, items, counts);
  } else if (wide) {
    k_fine<false, false, 1><<<n_items, kFineThreads, 0, st>>>(reqs, items, counts);
  } else {
    k_fine<false, false, 0><<<n_items, kFineThreads, 0, st>>>(reqs, items, counts);
  }
}

// ------------------------------------------------------------------ work lists
// One CTA per descriptor writes its items (see ExpandDesc): the work lists of a call are
// made on the device from a few descriptors per request instead of being built on the
// host and copied.
__global__ void __launch_bounds__(256) k_expand_items(const ExpandDesc* __restrict__ ds) {
  const ExpandDesc d = ds[blockIdx.x];
  const int64_t per_level = d.tiles * d.split, count = per_level * d.n_levels;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
    const int l = (int)(i / per_level);
    const int64_t r = i - (int64_t)l * per_level;
    const int64_t t = r / d.split;
    const int part = (int)(r - t * d.split);
    const int64_t pos = d.base + t * d.step;
    if (d.kind == 1)
      static_cast<G1Item*>(d.dst)[i] = G1Item{d.req, l, pos, part, 0};
    else if (d.kind <= kNGrid)
      static_cast<CoarseItem*>(d.dst)[i] = CoarseItem{d.req, l, d.kind, 0, pos};
    else
      static_cast<FineItem*>(d.dst)[i] = FineItem{d.req, l, pos};
  }
}

void launch_expand_items(const ExpandDesc* d, int n, cudaStream_t st) {
  if (n > 0) k_expand_items<<<n, 256, 0, st>>>(d);
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

__global__ void k_diag_shape(int shape, const float* x, const float* y, float* out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = shape_f(shape, x[i], y[i]);
}

void launch_diag_shape(int shape, const float* x, const float* y, float* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  k_diag_shape<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(shape, x, y, out, n);
}

// Issue-rate probes for the roofline denominators: every thread runs kPipeChains
// independent dependency chains of one instruction kind. PIPE 0: FP32 FMA; 1: MUFU
// ex2.approx; 2: MUFU rcp.approx; 3: MUFU cos.approx (__cosf). The chains stay in range
// (FMA: a fixed point near 1e-3; ex2 of -a: (0, 1]; rcp of 1 + a: [1/2, 1]; cos of a:
// [cos 1, 1]), and their sum is stored so that none is dropped.
constexpr int kPipeChains = 8;

template <int PIPE>
__global__ void __launch_bounds__(256) k_diag_pipe(float* out, int iters) {
  float a[kPipeChains];
#pragma unroll
  for (int k = 0; k < kPipeChains; ++k) a[k] = 1e-3f * (float)((threadIdx.x + k) & 7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kPipeChains; ++k) {
      if (PIPE == 0) {
        a[k] = fmaf(a[k], 0.999f, 1e-6f);
      } else if (PIPE == 1) {
        float r;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-a[k]));
        a[k] = r;
      } else if (PIPE == 2) {
        float r;
        asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + a[k]));
        a[k] = r;
      } else {
        a[k] = __cosf(a[k]);
      }
    }
  }
  float t = 0.0f;
#pragma unroll
  for (int k = 0; k < kPipeChains; ++k) t += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

int64_t launch_diag_pipe(int pipe, float* out, int blocks, int iters, cudaStream_t st) {
  switch (pipe) {
    case 0: k_diag_pipe<0><<<blocks, 256, 0, st>>>(out, iters); break;
    case 1: k_diag_pipe<1><<<blocks, 256, 0, st>>>(out, iters); break;
    case 2: k_diag_pipe<2><<<blocks, 256, 0, st>>>(out, iters); break;
    default: k_diag_pipe<3><<<blocks, 256, 0, st>>>(out, iters); break;
  }
  return (int64_t)blocks * 256 * iters * kPipeChains;  // instructions of the probed kind
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
    const int sg = panel_shift(grid);
    v = grid == 1 ? accept_mask_s<uint32_t>(1, c, gst, chi, R.cut_fx, R.R_w, first + i, 1, sg + R.wide, sg) & 1u
                  : owned_any<uint32_t>(R.wide, grid, c, gst, chi, R.cut_fx, R.R_w, first + i, 1) & 1u;
  } else {
    const int64_t k = first + i;
    const int64_t d = (k << kFineShift) - c;
    const bool within = (d < 0 ? -d : d) <= R.cut_fx;
    const int s10 = panel_shift(kNGrid);
    v = within && !accept_mask_s<uint32_t>(kNGrid, c, gst, chi, R.cut_fx, R.R_w, k >> 3, 1, s10 + R.wide, s10);
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

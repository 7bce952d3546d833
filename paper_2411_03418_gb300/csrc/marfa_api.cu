// Host runtime of libmarfa: the C-ABI declared in include/marfa.h. It validates the
// arguments, prepares line lists (Appendix B records -> sorted per-field device arrays
// with a bucket index over the centres), builds the per-level tables and the work
// lists of the coarse and finest-grid kernels, runs them on the caller's stream and
// writes PT-table files (Appendix A).
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/marfa.h"
#include "marfa_internal.cuh"

using namespace marfa;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? MARFA_E_NOMEM : MARFA_E_CUDA,         \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                        \
    }                                                                                     \
  } while (0)

extern "C" const char* marfa_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ physical constants
static const double kTref = 296.0;
static const double kC2 = 1.438776877;     // cm K
static const double kKB = 1.380649e-23;    // J/K
static const double kNA = 6.02214076e23;   // 1/mol
static const double kC = 2.99792458e8;     // m/s
static const double kAtm = 101325.0;       // Pa
static const double kSigmaScale = 18446744073709551616.0;  // 2^64: keeps sigma sums normal

// ------------------------------------------------------------------ device memory
// Stream-ordered allocations from the device's default pool, kept cached between calls.
static int dev_alloc(void** p, size_t bytes, cudaStream_t st) {
  static std::mutex mu;
  static bool pool_set[64] = {false};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && !pool_set[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      pool_set[dev] = true;
    }
  }
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  CK(cudaMallocAsync(p, bytes, st));
  return MARFA_OK;
}

// ------------------------------------------------------------------ kernel timing
// Optional event pairs around each launch (marfa_diag_kernel_timing).
namespace {
struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<TimedLaunch> g_tl;
}  // namespace

static cudaEvent_t timing_begin(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (!g_timing) return nullptr;
  cudaEvent_t a = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
  cudaEventRecord(a, st);
  return a;
}

static void timing_end(cudaEvent_t a, int kind, cudaStream_t st) {
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  cudaEvent_t b = nullptr;
  if (cudaEventCreate(&b) != cudaSuccess) return;
  cudaEventRecord(b, st);
  g_tl.push_back(TimedLaunch{kind, a, b});
}

extern "C" int marfa_diag_kernel_timing(int32_t enable, double* ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_tmu);
  double t[kNGrid + 2] = {0};
  int64_t c[kNGrid + 2] = {0};
  for (auto& x : g_tl) {
    float f = 0;
    if (cudaEventSynchronize(x.b) == cudaSuccess && cudaEventElapsedTime(&f, x.a, x.b) == cudaSuccess) {
      t[x.kind] += f;
      c[x.kind] += 1;
    }
    cudaEventDestroy(x.a);
    cudaEventDestroy(x.b);
  }
  g_tl.clear();
  g_timing = enable != 0;
  if (ms) std::copy(t, t + kNGrid + 2, ms);
  if (launches) std::copy(c, c + kNGrid + 2, launches);
  return MARFA_OK;
}

// ------------------------------------------------------------------ prepared lines
struct marfa_lines {
  int device = 0;
  int64_t n = 0;
  std::vector<marfa_species_t> species;
  std::vector<int64_t> perm;  // prepared index of input line i
  double delta_min = 0, delta_max = 0;
  int64_t key_base = 0;
  int32_t bshift = 0, nbuck = 0;
  int64_t* key = nullptr;
  double* nu0 = nullptr;
  float *S296 = nullptr, *ga = nullptr, *gs = nullptr, *E = nullptr, *na = nullptr, *da = nullptr;
  int16_t* sp = nullptr;
  int32_t* bfirst = nullptr;
  void* block = nullptr;  // single device allocation holding all arrays
};

extern "C" void marfa_free_lines(marfa_lines_t* L) {
  if (!L) return;
  if (L->block) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(L->device);
    cudaFree(L->block);
    cudaSetDevice(cur);
  }
  delete L;
}

static int64_t rint_fix(double v) { return (int64_t)std::nearbyint(v * kFix); }

extern "C" int marfa_prepare_lines(const marfa_line_t* lines, int64_t n, const marfa_species_t* sp,
                                   int32_t n_sp, marfa_lines_t** out) {
  if (!out) return fail(MARFA_E_INVAL, "out is NULL");
  *out = nullptr;
  if (!lines || n < 1) return fail(MARFA_E_INVAL, "need at least one line");
  if (n > (int64_t)1 << 31) return fail(MARFA_E_INVAL, "at most 2^31 lines");
  if (!sp || n_sp < 1 || n_sp > 32767) return fail(MARFA_E_INVAL, "need 1..32767 species");
  std::unordered_map<int32_t, int> code;
  for (int s = 0; s < n_sp; ++s) {
    if (code.count(sp[s].mol_iso)) return fail(MARFA_E_INVAL, "duplicate species %d", sp[s].mol_iso);
    if (!(sp[s].mass_amu > 0) || !std::isfinite(sp[s].mass_amu) || !std::isfinite(sp[s].q_exp))
      return fail(MARFA_E_INVAL, "species %d: mass must be > 0 and q finite", sp[s].mol_iso);
    code[sp[s].mol_iso] = s;
  }
  std::vector<int64_t> order(n);
  for (int64_t i = 0; i < n; ++i) {
    const marfa_line_t& l = lines[i];
    if (!std::isfinite(l.nu0) || l.nu0 < 0 || l.nu0 > 1e5)
      return fail(MARFA_E_INVAL, "line %lld: nu0 must be in [0, 1e5]", (long long)i);
    if (!code.count(l.mol_iso))
      return fail(MARFA_E_INVAL, "line %lld: unknown species %d", (long long)i, l.mol_iso);
    if (!std::isfinite(l.S296) || !std::isfinite(l.gamma_air) || !std::isfinite(l.gamma_self) ||
        !std::isfinite(l.E_lower) || !std::isfinite(l.n_air) || !std::isfinite(l.delta_air))
      return fail(MARFA_E_INVAL, "line %lld: non-finite parameter", (long long)i);
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t a, int64_t b) { return lines[a].nu0 < lines[b].nu0; });

  marfa_lines_t* L = new (std::nothrow) marfa_lines_t();
  if (!L) return fail(MARFA_E_NOMEM, "host allocation failed");
  cudaGetDevice(&L->device);
  L->n = n;
  L->species.assign(sp, sp + n_sp);
  L->perm.assign(n, 0);
  std::vector<int64_t> key(n);
  std::vector<double> nu0(n);
  std::vector<float> S(n), ga(n), gs(n), E(n), na(n), da(n);
  std::vector<int16_t> spi(n);
  double dmin = 1e300, dmax = -1e300;
  for (int64_t j = 0; j < n; ++j) {
    const marfa_line_t& l = lines[order[j]];
    L->perm[order[j]] = j;
    nu0[j] = l.nu0;
    key[j] = rint_fix(l.nu0);
    S[j] = l.S296;
    ga[j] = l.gamma_air;
    gs[j] = l.gamma_self;
    E[j] = l.E_lower;
    na[j] = l.n_air;
    da[j] = l.delta_air;
    spi[j] = (int16_t)code[l.mol_iso];
    dmin = std::min(dmin, (double)l.delta_air);
    dmax = std::max(dmax, (double)l.delta_air);
  }
  L->delta_min = dmin;
  L->delta_max = dmax;
  // bucket index: about one line per two buckets on average, at most 2^26 buckets
  const int64_t span = std::max<int64_t>(key[n - 1] - key[0], 1);
  int bs = 20;
  while (bs < 50 && (((int64_t)1 << (bs + 1)) * 2 * n <= span || (span >> bs) > ((int64_t)1 << 26))) ++bs;
  L->bshift = bs;
  L->key_base = (key[0] >> bs) << bs;
  const int64_t nb64 = ((key[n - 1] - L->key_base) >> bs) + 1;
  if (nb64 > (int64_t)1 << 30) {
    delete L;
    return fail(MARFA_E_INVAL, "line list too sparse for the bucket index");
  }
  L->nbuck = (int32_t)nb64;
  std::vector<int32_t> bfirst(L->nbuck + 1);
  {
    int64_t i = 0;
    for (int64_t b = 0; b <= L->nbuck; ++b) {
      const int64_t K = L->key_base + (b << bs);
      while (i < n && key[i] < K) ++i;
      bfirst[b] = (int32_t)i;
    }
  }
  // one device block for all arrays (256-byte aligned sub-arrays)
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t sz_key = al(8 * n), sz_nu = al(8 * n), sz_f = al(4 * n), sz_sp = al(2 * n),
               sz_b = al(4 * (L->nbuck + 1));
  const size_t total = sz_key + sz_nu + 6 * sz_f + sz_sp + sz_b;
  cudaError_t e = cudaMalloc(&L->block, total);
  if (e != cudaSuccess) {
    L->block = nullptr;
    delete L;
    return fail(MARFA_E_NOMEM, "cudaMalloc(%zu) failed: %s", total, cudaGetErrorString(e));
  }
  char* p = (char*)L->block;
  L->key = (int64_t*)p; p += sz_key;
  L->nu0 = (double*)p; p += sz_nu;
  L->S296 = (float*)p; p += sz_f;
  L->ga = (float*)p; p += sz_f;
  L->gs = (float*)p; p += sz_f;
  L->E = (float*)p; p += sz_f;
  L->na = (float*)p; p += sz_f;
  L->da = (float*)p; p += sz_f;
  L->sp = (int16_t*)p; p += sz_sp;
  L->bfirst = (int32_t*)p;
  struct Cp { void* d; const void* h; size_t b; } cps[] = {
      {L->key, key.data(), 8 * (size_t)n}, {L->nu0, nu0.data(), 8 * (size_t)n},
      {L->S296, S.data(), 4 * (size_t)n},  {L->ga, ga.data(), 4 * (size_t)n},
      {L->gs, gs.data(), 4 * (size_t)n},   {L->E, E.data(), 4 * (size_t)n},
      {L->na, na.data(), 4 * (size_t)n},   {L->da, da.data(), 4 * (size_t)n},
      {L->sp, spi.data(), 2 * (size_t)n},  {L->bfirst, bfirst.data(), 4 * bfirst.size()}};
  for (auto& c : cps) {
    e = cudaMemcpy(c.d, c.h, c.b, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      marfa_free_lines(L);
      return fail(MARFA_E_CUDA, "cudaMemcpy failed: %s", cudaGetErrorString(e));
    }
  }
  *out = L;
  return MARFA_OK;
}

extern "C" int64_t marfa_num_points(double nu_lo, double nu_hi) {
  if (!std::isfinite(nu_lo) || !std::isfinite(nu_hi) || nu_lo < 0 || nu_hi < 0 || nu_hi > 1e5)
    return MARFA_E_INVAL;
  const int64_t k_lo = (int64_t)std::ceil(nu_lo * 2048.0);
  const int64_t k_hi = (int64_t)std::floor(nu_hi * 2048.0);
  return k_hi >= k_lo ? k_hi - k_lo + 1 : 0;
}

// ------------------------------------------------------------------ request plans
struct Plan {
  const marfa_lines_t* lines = nullptr;
  marfa_request_t rq{};
  int32_t n_levels = 0;
  std::vector<LevelDev> lev;
  std::vector<LevelSpeciesDev> ls;
  ReqDev rd{};
  int64_t npts = 0;
  std::vector<G1Item> g1;
  std::vector<CoarseItem> coarse;
  std::vector<FineItem> fine;
  // device buffers
  void* dbuf = nullptr;       // per-level line data + slots + tables
  float* dout = nullptr;      // output (own buffer when the caller's is on the host)
  bool own_out = false;
  float* user_out = nullptr;
};

static int validate_request(const marfa_request_t* rq, int64_t* npts) {
  if (!rq) return fail(MARFA_E_INVAL, "request is NULL");
  const int64_t np = marfa_num_points(rq->nu_lo, rq->nu_hi);
  if (np < 0) return fail(MARFA_E_INVAL, "window bounds must be finite, >= 0 and <= 1e5");
  if (!(rq->nu_lo <= rq->nu_hi)) return fail(MARFA_E_INVAL, "nu_lo must be <= nu_hi");
  if (np == 0) return fail(MARFA_E_INVAL, "window holds no 2^-11 grid point");
  if (np > 0x7fffffff) return fail(MARFA_E_INVAL, "window too wide (more than 2^31 points)");
  if (!std::isfinite(rq->cutoff) || !(rq->cutoff > 0) || rq->cutoff > 1000)
    return fail(MARFA_E_INVAL, "cut-off must be in (0, 1000] cm^-1");
  const int s = rq->shape;
  if (!(s == MARFA_SHAPE_LORENTZ || s == MARFA_SHAPE_VOIGT || s == MARFA_SHAPE_DOPPLER ||
        s == MARFA_SHAPE_TEST_CONST || s == MARFA_SHAPE_TEST_QUAD))
    return fail(MARFA_E_INVAL, "unknown shape %d", s);
  if (rq->chi != MARFA_CHI_NONE && rq->chi != MARFA_CHI_TONKOV)
    return fail(MARFA_E_INVAL, "unknown chi %d", rq->chi);
  if (rq->units < MARFA_UNITS_SIGMA || rq->units > MARFA_UNITS_K_KM1)
    return fail(MARFA_E_INVAL, "unknown units %d", rq->units);
  if (rq->surrogate != 0) return fail(MARFA_E_INVAL, "surrogate must be 0");
  if (rq->R_w < 1 || rq->R_w > 64 || rq->R_c < 1 || rq->R_c > 64)
    return fail(MARFA_E_INVAL, "R_w and R_c must be in 1..64");
  *npts = np;
  return MARFA_OK;
}

static int build_plan(Plan& P, const marfa_lines_t* L, const marfa_level_t* levels,
                      const double* vmr, int32_t n_levels, const marfa_request_t* rq, int req_idx) {
  if (!L) return fail(MARFA_E_INVAL, "lines is NULL");
  int r = validate_request(rq, &P.npts);
  if (r) return r;
  if (n_levels < 1 || n_levels > 65535 || !levels || !vmr)
    return fail(MARFA_E_INVAL, "need 1..65535 levels with their vmr");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != L->device) return fail(MARFA_E_INVAL, "lines were prepared on device %d", L->device);
  const int ns = (int)L->species.size();
  for (int l = 0; l < n_levels; ++l) {
    const double T = levels[l].T_K, p = levels[l].p_atm;
    if (!std::isfinite(T) || !(T > 0) || !std::isfinite(p) || !(p > 0))
      return fail(MARFA_E_INVAL, "level %d: T and p must be finite and > 0", l);
    for (int s = 0; s < ns; ++s) {
      const double v = vmr[(int64_t)l * ns + s];
      if (!std::isfinite(v) || v < 0 || v > 1)
        return fail(MARFA_E_INVAL, "level %d: vmr must be in [0, 1]", l);
    }
  }
  P.lines = L;
  P.rq = *rq;
  P.n_levels = n_levels;
  const bool physical = rq->shape < MARFA_SHAPE_TEST_CONST;
  P.lev.resize(n_levels);
  P.ls.resize((size_t)n_levels * ns);
  const double scale = rq->units == MARFA_UNITS_SIGMA ? kSigmaScale : 1.0;
  for (int l = 0; l < n_levels; ++l) {
    const double T = levels[l].T_K, p = levels[l].p_atm;
    LevelDev& d = P.lev[l];
    d.T = T;
    d.p = p;
    d.ratio = kTref / T;
    // c - key = rint((nu0 + delta p) 2^43) - rint(nu0 2^43): within delta p 2^43 plus
    // the rounding of the FP64 sum (ulp(1e5)/2 < 2^8 units) and of both rint
    d.smin = (int64_t)std::floor(L->delta_min * p * kFix) - 1024;
    d.smax = (int64_t)std::ceil(L->delta_max * p * kFix) + 1024;
    d.pf = (float)p;
    d.log2_ratio = (float)std::log2(kTref / T);
    const double kb = -kC2 * (1.0 / T - 1.0 / kTref);
    d.kb_hi = (float)kb;
    d.kb_lo = (float)(kb - (double)d.kb_hi);
    d.c2_T = (float)(kC2 / T);
    d.c2_Tref = (float)(kC2 / kTref);
    for (int s = 0; s < ns; ++s) {
      const marfa_species_t& sp = L->species[s];
      const double v = vmr[(int64_t)l * ns + s];
      LevelSpeciesDev& q = P.ls[(size_t)l * ns + s];
      q.ps_d = v * p;
      q.ps = (float)q.ps_d;
      q.sqrtv = std::sqrt(2.0 * kNA * kKB * T * std::log(2.0) / (sp.mass_amu * 1e-3));
      q.ad = (float)(q.sqrtv / kC);
      double F = std::pow(kTref / T, sp.q_exp) * scale;  // Q(296)/Q(T)
      if (rq->units != MARFA_UNITS_SIGMA) F *= v * p * kAtm / (kKB * T) * 1e-6;
      if (rq->units == MARFA_UNITS_K_KM1) F *= 1e5;
      q.F = (float)F;
      q.chi = (rq->chi == MARFA_CHI_TONKOV && sp.chi_enabled) ? 1 : 0;
    }
  }
  ReqDev& R = P.rd;
  R.n_lines = L->n;
  R.key = L->key;
  R.key_base = L->key_base;
  R.bshift = L->bshift;
  R.nbuck = L->nbuck;
  R.bfirst = L->bfirst;
  R.n_levels = n_levels;
  R.k_lo = (int64_t)std::ceil(rq->nu_lo * 2048.0);
  R.k_hi = (int64_t)std::floor(rq->nu_hi * 2048.0);
  const int64_t X_lo = R.k_lo << kFineShift, X_hi = R.k_hi << kFineShift;
  int64_t off = 0;
  R.m_first[0] = R.npan[0] = R.slot_off[0] = 0;
  for (int g = 1; g <= kNGrid; ++g) {
    const int s = panel_shift(g);
    R.m_first[g] = X_lo >> s;
    R.npan[g] = (X_hi >> s) - R.m_first[g] + 1;
    R.slot_off[g] = off;
    off += 3 * R.npan[g];
  }
  R.slots_per_level = off;
  R.cut_fx = (int64_t)std::nearbyint(rq->cutoff * kFix);
  R.R_w = rq->R_w;
  R.shape = rq->shape;
  R.chi_req = rq->chi == MARFA_CHI_TONKOV ? 1 : 0;
  R.out_scale = (float)(1.0 / scale);
  R.npts = P.npts;
  (void)physical;
  // work lists: grid 1 in tiles of kG1Pairs pairs; grids 2..10 from coarse to fine
  for (int l = 0; l < n_levels; ++l)
    for (int64_t m0 = R.m_first[1]; m0 <= R.m_first[1] + R.npan[1]; m0 += kG1Pairs)
      P.g1.push_back(G1Item{req_idx, l, m0});
  for (int g = 2; g <= kNGrid; ++g)
    for (int l = 0; l < n_levels; ++l)
      for (int64_t m0 = R.m_first[g]; m0 <= R.m_first[g] + R.npan[g];
           m0 += g <= kLastLM ? (int64_t)kLPairs : (int64_t)kCPairs * kCWarps)
        P.coarse.push_back(CoarseItem{req_idx, l, g, 0, m0});
  const int64_t kb0 = R.k_lo & ~(int64_t)7;  // tiles start on a G10 panel
  for (int l = 0; l < n_levels; ++l)
    for (int64_t k0 = kb0; k0 <= R.k_hi; k0 += kFineTile) P.fine.push_back(FineItem{req_idx, l, k0});
  return MARFA_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Allocate the per-request device buffers of a plan and run the level preparation.
static int upload_and_prep(Plan& P, float* k_out, cudaStream_t st) {
  const marfa_lines_t* L = P.lines;
  const int64_t n = L->n, nl = P.n_levels;
  const int ns = (int)L->species.size();
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t pairs = (size_t)(n * nl);
  const size_t sz_c = al(8 * pairs), sz_f = al(4 * pairs), sz_b = al(pairs);
  const size_t sz_slots = al(4 * (size_t)P.rd.slots_per_level * nl);
  const size_t sz_lev = al(sizeof(LevelDev) * nl), sz_ls = al(sizeof(LevelSpeciesDev) * nl * ns);
  const size_t total = sz_c + 3 * sz_f + 2 * sz_b + sz_slots + sz_lev + sz_ls;
  int r = dev_alloc(&P.dbuf, total, st);
  if (r) return r;
  char* p = (char*)P.dbuf;
  ReqDev& R = P.rd;
  int64_t* c = (int64_t*)p; p += sz_c;
  float* amp = (float*)p; p += sz_f;
  float* sx = (float*)p; p += sz_f;
  float* yv = (float*)p; p += sz_f;
  int8_t* gst = (int8_t*)p; p += sz_b;
  uint8_t* fl = (uint8_t*)p; p += sz_b;
  R.slots = (float*)p; p += sz_slots;
  LevelDev* dlev = (LevelDev*)p; p += sz_lev;
  LevelSpeciesDev* dls = (LevelSpeciesDev*)p;
  R.c = c; R.amp = amp; R.sx = sx; R.yv = yv; R.gstar = gst; R.flags = fl; R.lev = dlev;
  CK(cudaMemcpyAsync(dlev, P.lev.data(), sizeof(LevelDev) * nl, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dls, P.ls.data(), sizeof(LevelSpeciesDev) * nl * ns, cudaMemcpyHostToDevice, st));
  P.user_out = k_out;
  if (k_out && is_device_ptr(k_out)) {
    P.dout = k_out;
    P.own_out = false;
  } else {
    r = dev_alloc((void**)&P.dout, 4 * (size_t)P.npts * nl, st);
    if (r) return r;
    P.own_out = true;
  }
  R.out = P.dout;
  PrepArgs a;
  a.n = n;
  a.nu0 = L->nu0; a.S296 = L->S296; a.ga = L->ga; a.gs = L->gs; a.E = L->E; a.na = L->na; a.da = L->da;
  a.species = L->sp;
  a.n_species = ns;
  a.lev = dlev;
  a.ls = dls;
  a.shape = P.rq.shape;
  a.R_c = P.rq.R_c;
  a.c = c; a.amp = amp; a.sx = sx; a.yv = yv; a.gstar = gst; a.flags = fl;
  cudaEvent_t ev = timing_begin(st);
  launch_level_prep(a, (int)nl, st);
  timing_end(ev, 0, st);
  CK(cudaGetLastError());
  return MARFA_OK;
}

static void release(Plan& P, cudaStream_t st) {
  if (P.dbuf) cudaFreeAsync(P.dbuf, st);
  if (P.own_out && P.dout) cudaFreeAsync(P.dout, st);
  P.dbuf = nullptr;
  P.dout = nullptr;
}

// Run the coarse and finest-grid kernels for a set of prepared plans.
static int run_plans(std::vector<Plan>& plans, cudaStream_t st, std::vector<int64_t>* coarse_counts,
                     std::vector<int64_t>* fine_counts) {
  std::vector<ReqDev> rds;
  std::vector<G1Item> gi;
  std::vector<CoarseItem> ci;
  std::vector<FineItem> fi;
  for (auto& P : plans) rds.push_back(P.rd);
  for (auto& P : plans) gi.insert(gi.end(), P.g1.begin(), P.g1.end());
  // interleave the coarse lists grid by grid so that the heaviest CTAs start first
  for (int g = 1; g <= kNGrid; ++g)
    for (auto& P : plans)
      for (auto& it : P.coarse)
        if (it.grid == g) ci.push_back(it);
  for (auto& P : plans) fi.insert(fi.end(), P.fine.begin(), P.fine.end());
  if (gi.size() > 0x7fffffffu || ci.size() > 0x7fffffffu || fi.size() > 0x7fffffffu)
    return fail(MARFA_E_INVAL, "too much work in one call");
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t sz_r = al(sizeof(ReqDev) * rds.size()), sz_gi = al(sizeof(G1Item) * gi.size()),
               sz_ci = al(sizeof(CoarseItem) * ci.size()), sz_fi = al(sizeof(FineItem) * fi.size());
  const bool count = coarse_counts != nullptr;
  const size_t sz_gc = count ? al(8 * gi.size()) : 0;
  const size_t sz_cc = count ? al(8 * ci.size()) : 0, sz_fc = count ? al(8 * fi.size()) : 0;
  void* buf = nullptr;
  int r = dev_alloc(&buf, sz_r + sz_gi + sz_ci + sz_fi + sz_gc + sz_cc + sz_fc, st);
  if (r) return r;
  char* p = (char*)buf;
  ReqDev* drd = (ReqDev*)p; p += sz_r;
  G1Item* dgi = (G1Item*)p; p += sz_gi;
  CoarseItem* dci = (CoarseItem*)p; p += sz_ci;
  FineItem* dfi = (FineItem*)p; p += sz_fi;
  int64_t* dgc = count ? (int64_t*)p : nullptr; p += sz_gc;
  int64_t* dcc = count ? (int64_t*)p : nullptr; p += sz_cc;
  int64_t* dfc = count ? (int64_t*)p : nullptr;
  auto done = [&](int code) {
    cudaFreeAsync(buf, st);
    return code;
  };
  cudaError_t e;
  if ((e = cudaMemcpyAsync(drd, rds.data(), sizeof(ReqDev) * rds.size(), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(dgi, gi.data(), sizeof(G1Item) * gi.size(), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(dci, ci.data(), sizeof(CoarseItem) * ci.size(), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(dfi, fi.data(), sizeof(FineItem) * fi.size(), cudaMemcpyHostToDevice, st)))
    return done(fail(MARFA_E_CUDA, "upload of work lists failed: %s", cudaGetErrorString(e)));
  if (count && ((e = cudaMemsetAsync(dgc, 0, sz_gc, st)) || (e = cudaMemsetAsync(dcc, 0, sz_cc, st)) ||
                (e = cudaMemsetAsync(dfc, 0, sz_fc, st))))
    return done(fail(MARFA_E_CUDA, "count buffers: %s", cudaGetErrorString(e)));
  cudaEvent_t ev = timing_begin(st);
  launch_g1(drd, dgi, (int)gi.size(), dgc, st);
  timing_end(ev, 1, st);
  if ((e = cudaGetLastError())) return done(fail(MARFA_E_CUDA, "grid-1 kernel: %s", cudaGetErrorString(e)));
  {
    size_t k = 0;
    for (int g = 2; g <= kNGrid; ++g) {  // ci is ordered by grid
      size_t k1 = k;
      while (k1 < ci.size() && ci[k1].grid == g) ++k1;
      ev = timing_begin(st);
      if (g <= kLastLM)
        launch_coarse_lm(drd, dci + k, (int)(k1 - k), dcc ? dcc + k : nullptr, st);
      else
        launch_coarse(drd, dci + k, (int)(k1 - k), dcc ? dcc + k : nullptr, st);
      timing_end(ev, g, st);
      k = k1;
    }
  }
  ev = timing_begin(st);
  launch_fine(drd, dfi, (int)fi.size(), dfc, st);
  timing_end(ev, kNGrid + 1, st);
  if ((e = cudaGetLastError())) return done(fail(MARFA_E_CUDA, "fine kernel: %s", cudaGetErrorString(e)));
  if (count) {
    std::vector<int64_t> hg(gi.size()), hc(ci.size()), hf(fi.size());
    if ((e = cudaMemcpyAsync(hg.data(), dgc, 8 * hg.size(), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(hc.data(), dcc, 8 * hc.size(), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(hf.data(), dfc, 8 * hf.size(), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
      return done(fail(MARFA_E_CUDA, "count read-back failed: %s", cudaGetErrorString(e)));
    // per (plan, level, grid)
    for (size_t q = 0; q < plans.size(); ++q) {
      coarse_counts[q].assign((size_t)plans[q].n_levels * 11, 0);
    }
    for (size_t k = 0; k < gi.size(); ++k) coarse_counts[gi[k].req][(size_t)gi[k].level * 11] += hg[k];
    for (size_t k = 0; k < ci.size(); ++k)
      coarse_counts[ci[k].req][(size_t)ci[k].level * 11 + ci[k].grid - 1] += hc[k];
    for (size_t k = 0; k < fi.size(); ++k)
      coarse_counts[fi[k].req][(size_t)fi[k].level * 11 + 10] += hf[k];
    (void)fine_counts;
  }
  return done(MARFA_OK);
}

static int finish_outputs(std::vector<Plan>& plans, cudaStream_t st) {
  bool any_host = false;
  for (auto& P : plans) {
    if (P.own_out && P.user_out) {
      CK(cudaMemcpyAsync(P.user_out, P.dout, 4 * (size_t)P.npts * P.n_levels, cudaMemcpyDeviceToHost, st));
      any_host = true;
    }
  }
  for (auto& P : plans) release(P, st);
  if (any_host) CK(cudaStreamSynchronize(st));
  return MARFA_OK;
}

static int absorption_impl(int32_t n_req, const marfa_lines_t* const* lines,
                           const marfa_level_t* const* levels, const double* const* vmr,
                           const int32_t* n_levels, const marfa_request_t* rq, float* const* k_out,
                           cudaStream_t st, std::vector<int64_t>* counts) {
  if (n_req < 1 || !lines || !levels || !vmr || !n_levels || !rq || !k_out)
    return fail(MARFA_E_INVAL, "bad batch arguments");
  std::vector<Plan> plans(n_req);
  for (int q = 0; q < n_req; ++q) {
    if (!k_out[q]) return fail(MARFA_E_INVAL, "k_out[%d] is NULL", q);
    int r = build_plan(plans[q], lines[q], levels[q], vmr[q], n_levels[q], &rq[q], q);
    if (r) return r;
  }
  for (int q = 0; q < n_req; ++q) {
    int r = upload_and_prep(plans[q], k_out[q], st);
    if (r) {
      for (auto& P : plans) release(P, st);
      return r;
    }
  }
  int r = run_plans(plans, st, counts, nullptr);
  if (r) {
    for (auto& P : plans) release(P, st);
    return r;
  }
  return finish_outputs(plans, st);
}

extern "C" int marfa_absorption(const marfa_lines_t* lines, const marfa_level_t* levels,
                                const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                                float* k_out, void* stream) {
  float* outs[1] = {k_out};
  return absorption_impl(1, &lines, &levels, &vmr, &n_levels, rq, outs, (cudaStream_t)stream, nullptr);
}

extern "C" int marfa_absorption_batch(int32_t n_req, const marfa_lines_t* const* lines,
                                      const marfa_level_t* const* levels, const double* const* vmr,
                                      const int32_t* n_levels, const marfa_request_t* rq,
                                      float* const* k_out, void* stream) {
  return absorption_impl(n_req, lines, levels, vmr, n_levels, rq, k_out, (cudaStream_t)stream, nullptr);
}

// ------------------------------------------------------------------ PT-table (Appendix A)
extern "C" int marfa_write_pt_table(const char* dir, int32_t level_number, double nu_lo,
                                    double nu_hi, const float* k, int64_t npts) {
  const int64_t NT = 20481;
  if (!dir || !k) return fail(MARFA_E_INVAL, "dir and k must not be NULL");
  if (level_number < 0) return fail(MARFA_E_INVAL, "level number must be >= 0");
  if (!std::isfinite(nu_lo) || !std::isfinite(nu_hi) || nu_lo < 10 || nu_hi <= nu_lo ||
      std::fmod(nu_lo, 10.0) != 0 || std::fmod(nu_hi, 10.0) != 0 || nu_hi > 1e5)
    return fail(MARFA_E_INVAL, "window must be multiples of 10 with 10 <= nu_lo < nu_hi <= 1e5");
  if (npts != marfa_num_points(nu_lo, nu_hi))
    return fail(MARFA_E_INVAL, "npts must be %lld", (long long)marfa_num_points(nu_lo, nu_hi));
  char name[32];
  snprintf(name, sizeof name, "%d", level_number);
  std::string fn = name;
  while (fn.size() < 3) fn += '_';
  std::string path = std::string(dir) + "/" + fn + ".ptbin";
  int fd = open(path.c_str(), O_WRONLY | O_CREAT, 0644);
  if (fd < 0) return fail(MARFA_E_IO, "cannot open %s: %s", path.c_str(), strerror(errno));
  const int64_t r0 = (int64_t)(nu_lo / 10.0), r1 = (int64_t)(nu_hi / 10.0);
  for (int64_t rr = r0; rr < r1; ++rr) {
    const float* src = k + (rr - r0) * (NT - 1);
    const off_t off = (off_t)(rr - 1) * NT * 4;
    const char* b = (const char*)src;
    size_t left = (size_t)NT * 4;
    off_t o = off;
    while (left) {
      ssize_t w = pwrite(fd, b, left, o);
      if (w <= 0) {
        int er = errno;
        close(fd);
        return fail(MARFA_E_IO, "write to %s failed: %s", path.c_str(), strerror(er));
      }
      left -= (size_t)w;
      b += w;
      o += w;
    }
  }
  if (close(fd) != 0) return fail(MARFA_E_IO, "close of %s failed: %s", path.c_str(), strerror(errno));
  return MARFA_OK;
}

// ------------------------------------------------------------------ absorption without allocation
// Callers that cannot allocate device memory (a host model that has handed all free
// device memory to its own pool, so that cudaMalloc fails or fragments it, or a
// pipeline that must not let an allocation or a free synchronise the device while
// other streams run) use marfa_absorption_noalloc. Its scratch is this file-scope
// array: every GPU that loads the library holds it until the process exits.
static constexpr size_t kNoAllocBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, looked up once per device with that device
// current (in host code the symbol is only a host-side stand-in).
static int noalloc_scratch(char** out) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(MARFA_E_INVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(MARFA_E_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    addr[dev] = ptr;
  }
  *out = (char*)addr[dev];
  return MARFA_OK;
}

extern "C" int marfa_absorption_noalloc(const marfa_lines_t* lines, const marfa_level_t* levels,
                                        const double* vmr, int32_t n_levels,
                                        const marfa_request_t* rq, float* k_out, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Plan P;
  int r = build_plan(P, lines, levels, vmr, n_levels, rq, 0);
  if (r) return r;
  if (!k_out || !is_device_ptr(k_out))
    return fail(MARFA_E_INVAL, "k_out must be device memory for marfa_absorption_noalloc");
  const marfa_lines_t* L = P.lines;
  const int64_t n = L->n, nl = P.n_levels;
  const int ns = (int)L->species.size();
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t pairs = (size_t)(n * nl);
  const size_t sz_c = al(8 * pairs), sz_f = al(4 * pairs), sz_b = al(pairs);
  const size_t sz_slots = al(4 * (size_t)P.rd.slots_per_level * nl);
  const size_t sz_lev = al(sizeof(LevelDev) * nl), sz_ls = al(sizeof(LevelSpeciesDev) * nl * ns);
  const size_t sz_r = al(sizeof(ReqDev)), sz_gi = al(sizeof(G1Item) * P.g1.size()),
               sz_ci = al(sizeof(CoarseItem) * P.coarse.size()), sz_fi = al(sizeof(FineItem) * P.fine.size());
  const size_t total = sz_c + 3 * sz_f + 2 * sz_b + sz_slots + sz_lev + sz_ls + sz_r + sz_gi + sz_ci + sz_fi;
  if (total > kNoAllocBytes)
    return fail(MARFA_E_INVAL, "request needs %zu bytes of scratch; marfa_absorption_noalloc holds %zu",
                total, kNoAllocBytes);
  char* p = nullptr;
  r = noalloc_scratch(&p);
  if (r) return r;
  ReqDev& R = P.rd;
  int64_t* c = (int64_t*)p; p += sz_c;
  float* amp = (float*)p; p += sz_f;
  float* sx = (float*)p; p += sz_f;
  float* yv = (float*)p; p += sz_f;
  int8_t* gst = (int8_t*)p; p += sz_b;
  uint8_t* fl = (uint8_t*)p; p += sz_b;
  R.slots = (float*)p; p += sz_slots;
  LevelDev* dlev = (LevelDev*)p; p += sz_lev;
  LevelSpeciesDev* dls = (LevelSpeciesDev*)p; p += sz_ls;
  ReqDev* drd = (ReqDev*)p; p += sz_r;
  G1Item* dgi = (G1Item*)p; p += sz_gi;
  CoarseItem* dci = (CoarseItem*)p; p += sz_ci;
  FineItem* dfi = (FineItem*)p;
  R.c = c; R.amp = amp; R.sx = sx; R.yv = yv; R.gstar = gst; R.flags = fl; R.lev = dlev;
  R.out = k_out;
  CK(cudaMemcpyAsync(dlev, P.lev.data(), sizeof(LevelDev) * nl, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dls, P.ls.data(), sizeof(LevelSpeciesDev) * nl * ns, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(drd, &R, sizeof(ReqDev), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dgi, P.g1.data(), sizeof(G1Item) * P.g1.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dci, P.coarse.data(), sizeof(CoarseItem) * P.coarse.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dfi, P.fine.data(), sizeof(FineItem) * P.fine.size(), cudaMemcpyHostToDevice, st));
  PrepArgs a;
  a.n = n;
  a.nu0 = L->nu0; a.S296 = L->S296; a.ga = L->ga; a.gs = L->gs; a.E = L->E; a.na = L->na; a.da = L->da;
  a.species = L->sp;
  a.n_species = ns;
  a.lev = dlev;
  a.ls = dls;
  a.shape = P.rq.shape;
  a.R_c = P.rq.R_c;
  a.c = c; a.amp = amp; a.sx = sx; a.yv = yv; a.gstar = gst; a.flags = fl;
  // Every slot and per-level value is written by these kernels before it is read, so
  // nothing left in the scratch by an earlier call needs clearing.
  launch_level_prep(a, (int)nl, st);
  launch_g1(drd, dgi, (int)P.g1.size(), nullptr, st);
  size_t k = 0;
  for (int g = 2; g <= kNGrid; ++g) {  // P.coarse is ordered by grid
    size_t k1 = k;
    while (k1 < P.coarse.size() && P.coarse[k1].grid == g) ++k1;
    if (g <= kLastLM)
      launch_coarse_lm(drd, dci + k, (int)(k1 - k), nullptr, st);
    else
      launch_coarse(drd, dci + k, (int)(k1 - k), nullptr, st);
    k = k1;
  }
  launch_fine(drd, dfi, (int)P.fine.size(), nullptr, st);
  CK(cudaGetLastError());
  return MARFA_OK;
}

// ------------------------------------------------------------------ diagnostics
extern "C" int marfa_diag_voigt(const float* x, const float* y, float* out, int64_t n) {
  if (n < 0 || (n > 0 && (!x || !y || !out))) return fail(MARFA_E_INVAL, "bad arguments");
  if (n == 0) return MARFA_OK;
  float *dx, *dy, *dz;
  CK(cudaMalloc(&dx, 12 * (size_t)n));
  dy = dx + n;
  dz = dy + n;
  cudaError_t e;
  if ((e = cudaMemcpy(dx, x, 4 * n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(dy, y, 4 * n, cudaMemcpyHostToDevice))) {
    cudaFree(dx);
    return fail(MARFA_E_CUDA, "copy failed: %s", cudaGetErrorString(e));
  }
  launch_diag_voigt(dx, dy, dz, n, 0);
  e = cudaMemcpy(out, dz, 4 * n, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  if (e) return fail(MARFA_E_CUDA, "voigt kernel: %s", cudaGetErrorString(e));
  return MARFA_OK;
}

extern "C" int marfa_diag_level_lines(const marfa_lines_t* lines, const marfa_level_t* levels,
                                      const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                                      int64_t* c_out, int8_t* gstar_out, int64_t* perm) {
  Plan P;
  int r = build_plan(P, lines, levels, vmr, n_levels, rq, 0);
  if (r) return r;
  r = upload_and_prep(P, nullptr, 0);
  if (r) {
    release(P, 0);
    return r;
  }
  const size_t pairs = (size_t)lines->n * n_levels;
  cudaError_t e;
  if ((c_out && (e = cudaMemcpy(c_out, P.rd.c, 8 * pairs, cudaMemcpyDeviceToHost))) ||
      (gstar_out && (e = cudaMemcpy(gstar_out, P.rd.gstar, pairs, cudaMemcpyDeviceToHost)))) {
    release(P, 0);
    return fail(MARFA_E_CUDA, "read-back failed: %s", cudaGetErrorString(e));
  }
  if (perm) std::copy(lines->perm.begin(), lines->perm.end(), perm);
  release(P, 0);
  CK(cudaDeviceSynchronize());
  return MARFA_OK;
}

extern "C" int marfa_diag_owned(const marfa_lines_t* lines, const marfa_level_t* levels,
                                const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                                int32_t level, int32_t grid, int64_t first, int32_t count,
                                uint8_t* out) {
  if (!out || count < 1 || grid < 1 || grid > 11 || level < 0 || level >= n_levels)
    return fail(MARFA_E_INVAL, "bad diag_owned arguments");
  Plan P;
  int r = build_plan(P, lines, levels, vmr, n_levels, rq, 0);
  if (r) return r;
  r = upload_and_prep(P, nullptr, 0);
  if (r) {
    release(P, 0);
    return r;
  }
  ReqDev* drd = nullptr;
  uint8_t* dout = nullptr;
  const size_t bytes = (size_t)lines->n * count;
  cudaError_t e;
  if ((e = cudaMalloc(&drd, sizeof(ReqDev))) || (e = cudaMalloc(&dout, bytes)) ||
      (e = cudaMemcpy(drd, &P.rd, sizeof(ReqDev), cudaMemcpyHostToDevice))) {
    cudaFree(drd);
    cudaFree(dout);
    release(P, 0);
    return fail(MARFA_E_CUDA, "diag setup failed: %s", cudaGetErrorString(e));
  }
  launch_diag_owned(drd, lines->n, level, grid, first, count, dout, 0);
  e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
  cudaFree(drd);
  cudaFree(dout);
  release(P, 0);
  if (e) return fail(MARFA_E_CUDA, "diag_owned kernel: %s", cudaGetErrorString(e));
  CK(cudaDeviceSynchronize());
  return MARFA_OK;
}

extern "C" int marfa_diag_absorption_counted(const marfa_lines_t* lines, const marfa_level_t* levels,
                                             const double* vmr, int32_t n_levels,
                                             const marfa_request_t* rq, float* k_out, int64_t* counts) {
  if (!counts) return fail(MARFA_E_INVAL, "counts is NULL");
  std::vector<int64_t> cc[1];
  float* outs[1] = {k_out};
  int r = absorption_impl(1, &lines, &levels, &vmr, &n_levels, rq, outs, 0, cc);
  if (r) return r;
  std::copy(cc[0].begin(), cc[0].end(), counts);
  CK(cudaDeviceSynchronize());
  return MARFA_OK;
}

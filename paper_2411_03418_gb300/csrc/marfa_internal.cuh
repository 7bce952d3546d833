// Internal layouts shared by the host runtime (marfa_api.cu), the profile kernels
// (marfa_kernels.cu) and the surrogate kernels (marfa_mlp.cu) of libmarfa. Not part of
// the C-ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace marfa {

// Positions are int64 fixed point in units of 2^-43 cm^-1, so line centres, grid
// nodes, panel ends, cut-offs and chi-factor breakpoints compare exactly.
constexpr int kFixBits = 43;
constexpr double kFix = 8796093022208.0;  // 2^43
constexpr int kFineBits = 11;             // finest step 2^-11 = 10/20480 cm^-1 (Sec. 2.4)
constexpr int kFineShift = kFixBits - kFineBits;  // 32
constexpr int kNGrid = 10;                // coarse grids G1..G10, h_g = 2^(1-g) cm^-1

// A panel of grid g spans two steps, 2 h_g = 2^(2-g) cm^-1 = 2^(45-g) units.
__host__ __device__ constexpr int panel_shift(int g) { return kFixBits + 2 - g; }
__host__ __device__ constexpr int64_t step_fx(int g) { return int64_t(1) << (kFixBits + 1 - g); }

__host__ __device__ __forceinline__ int64_t fl_sh(int64_t a, int s) { return a >> s; }
__host__ __device__ __forceinline__ int64_t cl_sh(int64_t a, int s) { return -((-a) >> s); }

constexpr int kShapeLorentz = 0, kShapeVoigt = 1, kShapeDoppler = 2, kShapeVoigtPaper = 3, kShapeUser = 4,
              kShapeConst = 100, kShapeQuad = 101, kShapeQuart = 102;
constexpr int kUserShapeMax = 4096;  // samples of a user-defined shape

// Per level (host-computed in double precision).
struct LevelDev {
  double T, p;
  double ratio;        // 296 / T, for the FP64 width (fallback of the g* decision)
  int64_t smin, smax;  // bounds of c - key over all lines, fixed point (conservative)
  float pf;            // p as float
  float log2_ratio;    // log2(296 / T)
  float kb_hi, kb_lo;  // -c2 (1/T - 1/296) as a float pair (Boltzmann factor exponent)
  float c2_T, c2_Tref; // c2 / T, c2 / 296
};

// Per (level, species).
struct LevelSpeciesDev {
  double ps_d;    // vmr p (partial pressure, atm)
  double sqrtv;   // sqrt(2 N_A k_B T ln2 / (M 1e-3)) (m/s), alpha_D = nu0/c * sqrtv
  float ps;       // vmr p
  float F;        // [n_s] Q(296)/Q(T) * internal scale: multiplies S296
  float ad;       // alpha_D / nu0
  int32_t chi;    // chi-factor applies (request chi on, species flag, physical shape)
};

// ------------------------------------------------------------------ Voigt surrogate
// The 2-64-64-64-1 SiLU network (not part of the paper). Training parameters are FP32,
// packed W1[64][2], b1, W2[64][64], b2, W3[64][64], b3, W4[64], b4 (W row-major
// [out][in]); inference weights keep W2 and W3 in BF16 with rows padded to kWStride.
constexpr int kMlpH = 64;
constexpr int kMlpParams = 8577;
constexpr int kMlpOffW1 = 0, kMlpOffB1 = 128, kMlpOffW2 = 192, kMlpOffB2 = 4288,
              kMlpOffW3 = 4352, kMlpOffB3 = 8448, kMlpOffW4 = 8512, kMlpOffB4 = 8576;
constexpr int kWStride = 72;  // BF16 row stride: conflict-free B-fragment loads
// Guard cells: |x| in [0, 12) by 1/8; y by binary exponent e in [-14, 3] and the two
// leading mantissa bits.
constexpr int kGuardNx = 96, kGuardNy = 72;
constexpr int kGuardWords = kGuardNx * kGuardNy / 32;

struct __align__(16) MlpWeights {
  float w1[2 * kMlpH];
  float b1[kMlpH], b2[kMlpH], b3[kMlpH], w4[kMlpH];
  float b4, pad[3];
  uint16_t w2[kMlpH * kWStride];  // BF16 bits
  uint16_t w3[kMlpH * kWStride];
  uint32_t guard[kGuardWords];    // bit c: surrogate allowed in guard cell c
};
static_assert(sizeof(MlpWeights) % 16 == 0, "MlpWeights is copied in 16-byte words");

// One request as the kernels see it.
struct ReqDev {
  // prepared lines (sorted by nu0)
  int64_t n_lines;
  const int64_t* key;       // rint(nu0 2^43)
  int64_t key_base;         // bucket index over the keys
  int32_t bshift;
  int32_t nbuck;
  const int32_t* bfirst;    // [nbuck + 1] first line with key >= key_base + b 2^bshift
  // per-level line data [n_levels][n_lines]
  const int64_t* c;         // shifted centre, fixed point
  const float* amp;         // amplitude (shape normalisation, S(T), [n], internal scale)
  const float* sx;          // x per cm^-1
  const float* yv;          // Voigt y
  const int8_t* gstar;      // coarsest grid resolving the core (11 = finest)
  const uint8_t* flags;     // bit 0: chi-factor on
  int32_t n_levels;
  const LevelDev* lev;      // [n_levels]
  // window and grids
  int64_t k_lo, k_hi;       // finest node indices of the window
  int64_t m_first[kNGrid + 1];  // per grid 1..10: first panel of the window
  int64_t npan[kNGrid + 1];     // per grid: panels of the window
  int64_t slot_off[kNGrid + 1]; // per grid: offset of its L|M|R arrays in a level's slots
                                // (grid 1: room for kG1Split copies, [part][L|M|R][npan])
  int64_t slots_per_level;
  float* slots;             // [n_levels][slots_per_level]
  int64_t cut_fx;           // cut-off, fixed point
  int32_t R_w;
  int32_t wide;             // 5-point variant: ownership on panels of four steps, quartic cascade
  int32_t shape;
  int32_t chi_req;          // request asks for the chi-factor
  int32_t mech;             // bit g (2..10): mech_ok on grid g; bit 11: mech_fine_ok; bit 12:
                            // mech_fine_merge_ok (3-point only)
  int32_t g1_split;         // CTAs sharing a grid-1 tile's candidate lines (1..kG1Split)
  const MlpWeights* mlp;    // surrogate weights and guard, null for the plain path
  float out_scale;          // inverse internal scale
  float* out;               // [n_levels][npts]
  int64_t npts;
};

// One CTA of the kernel of grids 2..10: kCWarps tiles of kCPairs consecutive node pairs
// of one grid.
struct CoarseItem {
  int32_t req, level, grid, pad;
  int64_t m0;  // first pair
};
// One CTA of the finest-grid kernel: 1024 finest nodes of one level.
struct FineItem {
  int32_t req, level;
  int64_t k0;  // first node of the tile (multiple of 4)
};

// One CTA of the G1 kernel: kG1Pairs consecutive node pairs of grid 1 of one level, and
// part `part` of the request's g1_split equal shares of the tile's candidate lines.
struct G1Item {
  int32_t req, level;
  int64_t m0;  // first pair
  int32_t part, pad;
};

// The work items of one (request, kind) for the device to write (launch_expand_items):
// n_levels x tiles x split items, level-major, then tile, then part, the same order as
// the host loops would write them. kind 1: G1Item (m0 = base + tile step, part);
// 2..10: CoarseItem of that grid (m0 = base + tile step); 11: FineItem (k0 = base +
// tile step).
struct ExpandDesc {
  int32_t kind, req, n_levels, split;
  int64_t base, step, tiles;
  void* dst;  // the first item
};
void launch_expand_items(const ExpandDesc* d, int n, cudaStream_t st);

constexpr int kG1Pairs = 32;         // node pairs per G1 tile (one per lane)
constexpr int kG1Split = 6;          // at most this many CTAs share one G1 tile's candidate
                                     // lines (ReqDev::g1_split, tuned); each writes its own
                                     // copy of the tile's slots
constexpr int kG1Warps = 8;          // warps of a G1 CTA, each takes every 8th staged line
constexpr int kG1Batch = 512;        // lines staged in shared memory at a time
constexpr int kLPairs = 32;          // node pairs per CTA of the line-major kernel (or 16)
constexpr int kLWarps = 4;
constexpr int kCPairs = 32;          // node pairs per warp tile of the two-phase kernel
constexpr int kCWarps = 4;           // warps (tiles) of a grids-2..10 CTA
constexpr int kFineThreads = 256;
constexpr int kFinePerThread = 4;
constexpr int kFineTile = kFineThreads * kFinePerThread;
constexpr int kFineWarpNodes = kFinePerThread * 32;  // finest nodes of one warp

struct PrepArgs {
  int64_t n;
  const double* nu0;
  const float *S296, *ga, *gs, *E, *na, *da;
  const int16_t* species;
  int32_t n_species;
  const LevelDev* lev;
  const LevelSpeciesDev* ls;   // [n_levels][n_species]
  int32_t shape, R_c;
  int64_t* c;
  float *amp, *sx, *yv;
  int8_t* gstar;
  uint8_t* flags;
};

// ------------------------------------------------------------------ device-side checks
// In a MARFA_DEBUG build, MARFA_DCHECK(cond, code) is cond, and when cond is false it also
// records code in the library's device status word (the first failure wins); callers
// skip the guarded access when it is false, so a failed check never faults. In an
// ordinary build it is `true` and costs nothing. Codes: 1xx grids 2..10, 2xx the finest
// grid, 3xx grid 1, 4xx candidate bands, 9xx the diagnostic probe.
#ifdef MARFA_DEBUG
__device__ bool marfa_dcheck_fail(unsigned code);
#define MARFA_DCHECK(cond, code) ((cond) || marfa_dcheck_fail(code))
#else
#define MARFA_DCHECK(cond, code) true
#endif
// The status word (0: no check failed), optionally cleared; MARFA_OK in ordinary builds
// (always 0). Synchronises the current device.
int device_check_status(unsigned* code, bool clear);
constexpr bool kDebugBuild =
#ifdef MARFA_DEBUG
    true;
#else
    false;
#endif
// launches the diagnostic probe: a guarded store at index i of a 32-entry array
void launch_diag_check(int i, cudaStream_t st);
// the user-defined shape of the current device: g(x) at n samples over [0, x_max]
// (marfa_kernels.cu); MARFA_OK or a CUDA error code
int set_user_shape(const float* g, int n, float x_max);

// kernels (marfa_kernels.cu). With surr set, the surrogate-capable variants run (requests
// with mlp != null use the surrogate under its guard). counts, when given, selects the
// counting variants and receives kCountFields entries per item: all profile evaluations,
// those the surrogate took, and the plain Voigt evaluations in 9 x 9 polynomial cells,
// in the asymptotic series and in small-y cells (voigt_class 2, 1 and 3).
constexpr int kCountFields = 5;
void launch_level_prep(const PrepArgs& a, int n_levels, cudaStream_t st);
// every request's level preparation in one launch: args[n_req] (device), first[n_req + 1]
// (device) the prefix sums of the requests' blocks, ceil(n / 256) x n_levels each
void launch_level_prep_batch(const PrepArgs* args, const int64_t* first, int n_req, int64_t blocks,
                             cudaStream_t st);
// wide: every request of the launch uses the 5-point partition (the plain kernels are
// compiled for one partition; the counting and surrogate variants read it per request).
void launch_g1(const ReqDev* reqs, const G1Item* items, int n_items, int64_t* counts, bool surr,
               bool wide, cudaStream_t st);
void launch_coarse(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts,
                   bool surr, bool wide, cudaStream_t st);
void launch_coarse_lm(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts,
                      bool surr, int pairs, bool wide, cudaStream_t st);
void launch_fine(const ReqDev* reqs, const FineItem* items, int n_items, int64_t* counts, bool surr,
                 bool wide, cudaStream_t st);
// The flattened variants (plain path only): grids 2..10 over the two-phase tiles with
// phase 1 spread evenly over the lanes and grouped by Voigt branch (k_coarse_jobs), and
// the finest grid with (line, G10 panel) jobs spread evenly over 8-lane groups
// (k_fine_jobs).
// Grids 2..10 and the finest grid with ownership by mechanism (centre, cut-off edges,
// chi breakpoints in separate candidate passes, closed forms of ownership.cuh); only for
// requests whose mech bit of the grid is set (3-point, plain path).
void launch_coarse_mech(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts, bool merged,
                        cudaStream_t st);
void launch_coarse_jobs(const ReqDev* reqs, const CoarseItem* items, int n_items, int64_t* counts, bool wide,
                        cudaStream_t st);
// mech: 0 general ownership, 1 closed forms in one pass per mechanism, 2 closed forms
// in one merged pass (1, 2: 3-point requests with the mech bit of the finest grid)
void launch_fine_jobs(const ReqDev* reqs, const FineItem* items, int n_items, int64_t* counts, bool wide,
                      int mech, cudaStream_t st);
void launch_diag_voigt(const float* x, const float* y, float* out, int64_t n, cudaStream_t st);
void launch_diag_shape(int shape, const float* x, const float* y, float* out, int64_t n, cudaStream_t st);
// instructions issued by one probe launch (out: blocks x 256 floats)
int64_t launch_diag_pipe(int pipe, float* out, int blocks, int iters, cudaStream_t st);
void launch_diag_owned(const ReqDev* req, int64_t n_lines, int level, int grid, int64_t first,
                       int count, uint8_t* out, cudaStream_t st);


// surrogate kernels (marfa_mlp.cu)
void launch_mlp_fwd_bwd(const float* params, const float* x, const float* y, const float* t,
                        int64_t n, int64_t first, int nblk, float inv_batch, bool qat, float* part,
                        float* loss_part, cudaStream_t st);
int mlp_train_tile();
void launch_mlp_reduce(const float* part, int nblk, float* grad, cudaStream_t st);
void launch_mlp_loss_sum(const float* lp, int n, float inv, float* out, cudaStream_t st);
void launch_mlp_adam(float* p, const float* g, float* m, float* v, float lr, float b1t, float b2t,
                     cudaStream_t st);
void launch_mlp_pack(const float* p, MlpWeights* out, cudaStream_t st);
void launch_mlp_guard(MlpWeights* w, float budget, int samples, float* cell_err, cudaStream_t st);
void launch_mlp_eval(const MlpWeights* w, const float* x, const float* y, float* out, int64_t n,
                     bool guarded, cudaStream_t st);

}  // namespace marfa

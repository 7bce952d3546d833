/*
 * marfa.h — C-ABI of the GB300 line-by-line absorption library (libmarfa).
 *
 * The library computes, for every pressure–temperature level of a request, the
 * absorption coefficient k(nu) (or the cross-section sigma(nu)) of a line list on the
 * 2^-11 cm^-1 output grid, following arXiv 2411.03418:
 *   Sec. 2.1, Eqs. (2)-(3)  k(nu; p, T) = n(p, T) sum_j S_j(T) f_j(nu - nu~0_j)
 *   Sec. 2.2, Eqs. (4)-(8)  Lorentz, Gauss and Voigt line shapes, Voigt K(x, y)
 *   Sec. 2.3, Eqs. (9)-(10) Tonkov chi-factor of the line wings
 *   Sec. 2.4                the eleven-grid scheme: line centres on the finest grid,
 *                           wings on grids of steps 2^(1-g) cm^-1 (g = 1..10),
 *                           quadratic 3-point interpolation back onto the finest grid
 *   Appendix A              PT-table files, Appendix B  36-byte line records.
 *
 * Conventions for every call:
 *   - return 0 (MARFA_OK) on success or a negative MARFA_E_* code; nothing is thrown or
 *     aborted across the ABI; marfa_last_error() gives a message (thread-local);
 *   - inputs are copied by the library; outputs are owned by the caller;
 *   - all device work runs on the current CUDA device;
 *   - pointers documented as "host or device" are classified with
 *     cudaPointerGetAttributes; host outputs are filled before the call returns.
 */
#ifndef MARFA_H
#define MARFA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MARFA_OK 0
#define MARFA_E_INVAL (-1)    /* an argument is out of range or inconsistent          */
#define MARFA_E_NOMEM (-2)    /* a device or host allocation failed                    */
#define MARFA_E_CUDA (-3)     /* a CUDA runtime call or a kernel launch failed          */
#define MARFA_E_IO (-4)       /* a PT-table file could not be written                  */
#define MARFA_E_INTERNAL (-5) /* a device-side consistency check failed (bug)           */

/* line shapes (Sec. 2.2); the TEST shapes exist to pin the grid bookkeeping:
 * TEST_CONST adds exactly 1 per line within the cut-off (k counts lines),
 * TEST_QUAD adds S(T)[n](1 + d/4 + d^2/16), d = nu - nu~0 in cm^-1, which the 3-point
 * interpolation reproduces exactly. Neither applies the chi-factor. */
enum {
  MARFA_SHAPE_LORENTZ = 0,    /* Eq. (4)                                      */
  MARFA_SHAPE_VOIGT = 1,      /* Eqs. (7)-(8), the default of the paper        */
  MARFA_SHAPE_DOPPLER = 2,    /* Eq. (5)                                      */
  MARFA_SHAPE_TEST_CONST = 100,
  MARFA_SHAPE_TEST_QUAD = 101
};
enum { MARFA_CHI_NONE = 0, MARFA_CHI_TONKOV = 1 };          /* Eq. (10)          */
enum { MARFA_UNITS_SIGMA = 0,   /* cm^2/molecule, Eq. (3)                      */
       MARFA_UNITS_K_CM1 = 1,   /* cm^-1, Eq. (2) with n in molecules/cm^3      */
       MARFA_UNITS_K_KM1 = 2 }; /* km^-1                                        */

/* Appendix B database record: 36 bytes, no padding, little-endian. */
#pragma pack(push, 1)
typedef struct {
  double nu0;          /* transition wavenumber, cm^-1 (vacuum)                    */
  float S296;          /* intensity at 296 K, cm/molecule                           */
  float gamma_air;     /* air-broadened HWHM at 296 K, cm^-1/atm                     */
  float gamma_self;    /* self-broadened HWHM at 296 K, cm^-1/atm                    */
  float E_lower;       /* lower-state energy E'', cm^-1                              */
  float n_air;         /* temperature exponent of the widths                          */
  int32_t mol_iso;     /* jointMolIso: selects an entry of the species table         */
  float delta_air;     /* pressure shift at 296 K, cm^-1/atm                          */
} marfa_line_t;
#pragma pack(pop)

/* One per jointMolIso code. Q(T)/Q(296) = (T/296)^q_exp stands in for the TIPS table
 * (Sec. 4.2.2); chi_enabled marks molecules the chi-factor applies to (Sec. 2.3). */
typedef struct {
  int32_t mol_iso;
  int32_t chi_enabled;
  double mass_amu;     /* molar mass, g/mol (Sec. 4.2.3)                            */
  double q_exp;
} marfa_species_t;

typedef struct {
  double T_K;          /* temperature, K (> 0)                                      */
  double p_atm;        /* pressure, atm (> 0)                                        */
} marfa_level_t;

typedef struct {
  double nu_lo, nu_hi; /* window, cm^-1: outputs at k 2^-11 with nu_lo <= k 2^-11 <= nu_hi */
  double cutoff;       /* lines contribute where |nu - nu~0| <= cutoff, cm^-1 (0 < cutoff <= 1000) */
  int32_t shape;       /* MARFA_SHAPE_*                                              */
  int32_t chi;         /* MARFA_CHI_*                                                */
  int32_t units;       /* MARFA_UNITS_*                                              */
  int32_t surrogate;   /* must be 0: the learned Voigt is not part of this library   */
  int32_t R_w;         /* wing distance, in steps of a grid, below which that grid
                          refines (1..64; 8 is the default preset)                    */
  int32_t R_c;         /* a grid resolves a core when its step <= W / R_c (1..64)      */
} marfa_request_t;

/* Opaque prepared line list, resident on the device it was prepared on. */
typedef struct marfa_lines marfa_lines_t;

/*
 * Copy n_lines Appendix-B records (host pointer) to the current device, sorted by nu0
 * (stable: ties keep input order), split into per-field arrays, together with the
 * species table (n_species entries, host pointer; every mol_iso of a line must appear
 * exactly once). *out receives a handle owned by the library; free it with
 * marfa_free_lines. Errors: MARFA_E_INVAL (n_lines < 1, non-finite or negative nu0,
 * unknown species, duplicate species), MARFA_E_NOMEM, MARFA_E_CUDA.
 */
int marfa_prepare_lines(const marfa_line_t* lines, int64_t n_lines,
                        const marfa_species_t* species, int32_t n_species,
                        marfa_lines_t** out);

/* Release a handle from marfa_prepare_lines (NULL is ignored). */
void marfa_free_lines(marfa_lines_t* lines);

/* Number of output points of a window: #{k : nu_lo <= k 2^-11 <= nu_hi}; 0 if empty,
 * negative (MARFA_E_INVAL) for non-finite or negative bounds. */
int64_t marfa_num_points(double nu_lo, double nu_hi);

/*
 * Absorption of one request at n_levels levels (Sec. 2.1-2.4).
 *   levels : host, [n_levels] T and p;
 *   vmr    : host, [n_levels][n_species] volume mixing ratios in species-table order
 *            (partial pressure vmr*p, number density vmr*p/(k_B T));
 *   k_out  : host or device, [n_levels][npts] float32 row-major, npts =
 *            marfa_num_points(nu_lo, nu_hi); caller-owned;
 *   stream : cudaStream_t to run on (NULL = legacy default stream). With a device
 *            k_out the call is asynchronous on that stream; with a host k_out it
 *            returns after the copy back.
 * The line list must cover [nu_lo - cutoff, nu_hi + cutoff] for the sum to be complete;
 * lines outside cannot contribute. The value at a given nu does not depend on the
 * window or on other requests. Errors: MARFA_E_INVAL (window, cut-off, R_w/R_c, enum
 * values, T/p/vmr not finite and positive/non-negative, surrogate != 0, more than
 * 2^31 points), MARFA_E_NOMEM, MARFA_E_CUDA.
 */
int marfa_absorption(const marfa_lines_t* lines, const marfa_level_t* levels,
                     const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                     float* k_out, void* stream);

/*
 * n_req independent requests in one pass: request r uses lines[r], levels[r],
 * vmr[r], n_levels[r], rq[r] and writes k_out[r] (host or device), with the same
 * meaning as marfa_absorption. All work of all requests goes into the same kernel
 * launches. Results are identical to n_req separate marfa_absorption calls.
 */
int marfa_absorption_batch(int32_t n_req, const marfa_lines_t* const* lines,
                           const marfa_level_t* const* levels, const double* const* vmr,
                           const int32_t* n_levels, const marfa_request_t* rq,
                           float* const* k_out, void* stream);

/*
 * Appendix A PT-table: write k (host, npts float32 values at k 2^-11 over
 * [nu_lo, nu_hi]) into <dir>/<level_number padded with '_' to 3 chars>.ptbin as
 * direct-access records of 20481 float32 (little-endian) each; record r (1-based,
 * r = int(nu/10)) covers [10 r, 10 r + 10] and sits at byte offset
 * (r - 1) * 20481 * 4. nu_lo and nu_hi must be multiples of 10 with nu_lo < nu_hi and
 * npts must equal marfa_num_points(nu_lo, nu_hi). Records outside the window are left
 * as they are in an existing file (zero in a new one). Errors: MARFA_E_INVAL, MARFA_E_IO.
 */
int marfa_write_pt_table(const char* dir, int32_t level_number, double nu_lo,
                         double nu_hi, const float* k, int64_t npts);

/*
 * marfa_absorption without any device allocation, for callers that cannot allocate
 * device memory: a host model that has given all free device memory to its own pool
 * (so cudaMalloc would fail or fragment it), or a pipeline that must not let an
 * allocation or a free synchronise the device while its other streams run. The paper
 * has no counterpart of this call; it computes the same k(nu) as marfa_absorption.
 *   - Scratch: a file-scope __device__ array of 32 MiB (MARFA_NOALLOC_SCRATCH_BYTES)
 *     that every GPU loading the library holds until the process exits. A request
 *     whose per-level line data, grid slots and work lists exceed it is rejected with
 *     MARFA_E_INVAL (for example: one level of 200,000 lines on a 1000 cm^-1 window
 *     fits; sixty such levels do not).
 *   - k_out must be device memory ([n_levels][npts] float32); host outputs are
 *     rejected with MARFA_E_INVAL. lines comes from marfa_prepare_lines.
 *   - The first call on a device looks up the scratch's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before
 *     any stream capture.
 *   - Every call reuses the same scratch and leaves its contents there; the kernels
 *     write every value they read, so nothing needs clearing between calls. Calls
 *     whose work overlaps on the GPU (other streams, other host threads) race on the
 *     scratch: serialise them.
 *   - Asynchronous on stream (NULL = legacy default stream); the copies of the level
 *     tables and work lists come from pageable host memory into the scratch.
 */
#define MARFA_NOALLOC_SCRATCH_BYTES (32u << 20)
int marfa_absorption_noalloc(const marfa_lines_t* lines, const marfa_level_t* levels,
                             const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                             float* k_out, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* marfa_last_error(void);

/* ---------------------------------------------------------------- diagnostics
 * Entry points used by the parity tests; same conventions as above.
 */

/* FP32 Voigt function K(x, y) of Eq. (8) as the kernels evaluate it, at n points
 * (x, y host arrays, out host array; y > 0). */
int marfa_diag_voigt(const float* x, const float* y, float* out, int64_t n);

/* Per-level line data the kernels use: centre c = rint((nu0 + delta p) 2^43) (int64)
 * and g* (the coarsest grid 1..10 resolving the core, 11 = finest), per level and per
 * line in prepared (sorted) order; outputs host arrays [n_levels][n_lines]. The
 * prepared order of input line i is perm[i] (host, [n_lines], may be NULL). */
int marfa_diag_level_lines(const marfa_lines_t* lines, const marfa_level_t* levels,
                           const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                           int64_t* c_out, int8_t* gstar_out, int64_t* perm);

/* Ownership as the kernels decide it, for one level and one grid g (1..10: panels
 * [first, first + count) of width 2^(2-g) cm^-1; 11: finest nodes [first, first + count)),
 * for every line in prepared order: out[line * count + i] = 1 if that grid sums the line
 * there, else 0 (host array [n_lines][count]). */
int marfa_diag_owned(const marfa_lines_t* lines, const marfa_level_t* levels,
                     const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                     int32_t level, int32_t grid, int64_t first, int32_t count,
                     uint8_t* out);

/* marfa_absorption that also counts the distinct (line, node) profile evaluations per
 * level and grid: counts host array [n_levels][11] (grids 1..10, then the finest). */
int marfa_diag_absorption_counted(const marfa_lines_t* lines, const marfa_level_t* levels,
                                  const double* vmr, int32_t n_levels,
                                  const marfa_request_t* rq, float* k_out, int64_t* counts);

/* Per-kernel device time: enable = 1 clears the totals and starts recording CUDA events
 * around every kernel launch of this library (on the launch stream); enable = 0 stops,
 * waits for the recorded events and writes, for the twelve kernel launches of a call
 * (0 level preparation, g = 1..10 the sums on grid g, 11 finest grid + cascade), the
 * summed milliseconds to ms[12] and the launch counts to launches[12] (host arrays,
 * may be NULL). */
int marfa_diag_kernel_timing(int32_t enable, double* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* MARFA_H */

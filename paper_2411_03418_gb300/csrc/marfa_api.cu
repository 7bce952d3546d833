// Host runtime of libmarfa: the C-ABI declared in include/marfa.h. It validates the
// arguments, prepares line lists (Appendix B records -> sorted per-field device arrays
// with a bucket index over the centres), builds the per-level tables and the work
// lists of the coarse and finest-grid kernels, runs them on the caller's stream and
// writes PT-table files (Appendix A).
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <cerrno>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/marfa.h"
#include "marfa_internal.cuh"
#include "ownership.cuh"

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

// MARFA_DEBUG builds: after a call's kernels, the device-side checks' status word (the
// call waits for the device); a failed check is reported as MARFA_E_INTERNAL and cleared.
static int debug_checks() {
  if (!kDebugBuild) return 0;
  unsigned code = 0;
  if (marfa::device_check_status(&code, true)) return fail(MARFA_E_CUDA, "device synchronisation failed");
  if (code) return fail(MARFA_E_INTERNAL, "device-side check %u failed", code);
  return 0;
}

// ------------------------------------------------------------------ physical constants
static const double kTref = 296.0;
static const double kC2 = 1.438776877;     // cm K
static const double kKB = 1.380649e-23;    // J/K
static const double kNA = 6.02214076e23;   // 1/mol
static const double kC = 2.99792458e8;     // m/s
static const double kAtm = 101325.0;       // Pa
static const double kSigmaScale = 18446744073709551616.0;  // 2^64: keeps sigma sums normal

// ------------------------------------------------------------------ allocation-failure injection
// For tests of the error paths: armed with n >= 1, the n-th allocation from then on
// fails as if the memory were exhausted (device allocations of dev_alloc, the line
// list's device block, host staging buffer and object, plan objects, the surrogate's
// buffers), and the injector disarms itself. MARFA_FAIL_ALLOC=n in the environment arms
// it when the library loads; marfa_diag_fail_alloc re-arms it.
static std::atomic<int64_t> g_fail_left{-1};  // allocations to let through before the failure; < 0: off
static int64_t fail_alloc_env() {
  const char* v = std::getenv("MARFA_FAIL_ALLOC");
  const long long n = v ? std::atoll(v) : 0;
  return n >= 1 ? n - 1 : -1;
}
static const bool g_fail_env_read = (g_fail_left.store(fail_alloc_env()), true);

// True when this allocation is the one to fail.
static bool alloc_fails() {
  int64_t v = g_fail_left.load();
  while (v >= 0)
    if (g_fail_left.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}

extern "C" int marfa_diag_fail_alloc(int64_t nth, int64_t* left) {
  (void)g_fail_env_read;
  if (left) *left = g_fail_left.load() >= 0 ? g_fail_left.load() + 1 : 0;
  if (nth < 0) return fail(MARFA_E_INVAL, "nth must be >= 0 (0: off)");
  g_fail_left.store(nth >= 1 ? nth - 1 : -1);
  return MARFA_OK;
}

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
  if (alloc_fails()) return fail(MARFA_E_NOMEM, "device allocation of %zu bytes failed (injected)", bytes);
  CK(cudaMallocAsync(p, bytes, st));
  return MARFA_OK;
}

extern "C" int marfa_diag_device_memory(int64_t* pool_used, int64_t* device_free) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceSynchronize());
  if (pool_used) {
    cudaMemPool_t pool;
    uint64_t used = 0;
    CK(cudaDeviceGetDefaultMemPool(&pool, dev));
    CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    *pool_used = (int64_t)used;
  }
  if (device_free) {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    *device_free = (int64_t)fr;
  }
  return MARFA_OK;
}

// ------------------------------------------------------------------ absorption without allocation
// The scratch of marfa_absorption_noalloc (declared here, where marfa_prepare_lines can
// reach it; the entry point itself is at the end of the file).
static constexpr size_t kNoAllocBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch on the current device (in host code the symbol is
// only a host-side stand-in). Looked up on every call, so that a context torn down and
// made again by the host application never leaves a stale address behind. The first
// lookup on a device loads the module holding the array, which commits its 32 MiB:
// marfa_prepare_lines makes that lookup, so the memory is taken by a call that
// allocates anyway, before any marfa_absorption_noalloc on that device.
static int noalloc_scratch(char** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return fail(e == cudaErrorMemoryAllocation ? MARFA_E_NOMEM : MARFA_E_CUDA,
                "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
  *out = (char*)ptr;
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
    cudaDeviceSynchronize();  // every use of the list, on any stream, has finished
    cudaFreeAsync(L->block, 0);  // back to the device's pool
    cudaSetDevice(cur);
  }
  delete L;
}

// ---------------------------------------------------------------- host line preparation
// The host work of marfa_prepare_lines (validation, fixed-point keys, the stable sort by
// nu0, the sorted arrays and the bucket index) runs over contiguous chunks on up to
// kHostThreads threads; every result, errors included, is independent of their number.
constexpr int kHostThreads = 16;

// Persistent host threads for those chunked loops (starting and joining 15 threads costs
// about as much as one loop over 200k lines). The pool starts on first use, and again in a
// child process after fork (which inherits no threads); it runs one job at a time and is
// never torn down: its threads sleep on a condition variable until the process ends.
class HostPool {
 public:
  // the pool of this process, or nullptr if it cannot be made (then loops run serially)
  static HostPool* get() {
    static std::mutex create_mu;
    static HostPool* pool = nullptr;
    std::lock_guard<std::mutex> g(create_mu);
    if (!pool || pool->pid_ != getpid()) pool = new (std::nothrow) HostPool();
    return pool;
  }
  int size() const { return 1 + nworkers_; }
  // f(t) for t in [0, nt), nt <= size(); t = 0 runs on the calling thread. f must not throw.
  void run(int nt, const std::function<void(int)>& f) {
    std::lock_guard<std::mutex> job(job_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &f;
      want_ = nt;
      pending_ = nt - 1;
      ++gen_;
    }
    cv_start_.notify_all();
    f(0);
    std::unique_lock<std::mutex> lk(mu_);
    cv_done_.wait(lk, [&] { return pending_ == 0; });
  }

 private:
  HostPool() : pid_(getpid()) {
    const unsigned hc = std::thread::hardware_concurrency();
    const int nw = (int)std::min<unsigned>(hc ? hc : 1, kHostThreads) - 1;
    for (int i = 1; i <= nw; ++i) {
      try {
        std::thread([this, i] { loop(i); }).detach();
      } catch (...) {
        break;
      }
      nworkers_ = i;
    }
  }
  void loop(int id) {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_start_.wait(lk, [&] { return gen_ != seen; });
      seen = gen_;
      if (id >= want_) continue;  // not part of this job
      const std::function<void(int)>* f = fn_;
      lk.unlock();
      (*f)(id);
      lk.lock();
      if (--pending_ == 0) cv_done_.notify_one();
    }
  }
  const pid_t pid_;
  int nworkers_ = 0;
  std::mutex job_mu_, mu_;
  std::condition_variable cv_start_, cv_done_;
  const std::function<void(int)>* fn_ = nullptr;
  uint64_t gen_ = 0;
  int want_ = 0, pending_ = 0;
};

static thread_local bool t_serial_loops = false;  // set on a thread that runs one job of a batch
static int host_threads(int64_t work, int64_t min_per_thread) {
  if (t_serial_loops) return 1;
  const HostPool* pool = HostPool::get();
  const int64_t nt = std::min<int64_t>(pool ? pool->size() : 1, std::max<int64_t>(1, work / min_per_thread));
  return (int)nt;
}

// f(lo, hi, t) on the nt contiguous chunks of [0, n), chunk t on pool thread t (chunk 0 on
// the calling thread); nt comes from host_threads. f must not throw.
template <class F>
static void par_chunks(int nt, int64_t n, const F& f) {
  HostPool* pool = nt > 1 ? HostPool::get() : nullptr;
  if (!pool || nt > pool->size()) {
    for (int t = 0; t < nt; ++t) f(n * t / nt, n * (t + 1) / nt, t);
    return;
  }
  pool->run(nt, [&](int t) { f(n * t / nt, n * (t + 1) / nt, t); });
}

// mol_iso -> species code: open addressing over a power-of-two table (read-only once built,
// so the threads share it)
struct SpeciesIndex {
  std::vector<int32_t> iso;
  std::vector<int16_t> code;  // -1 = empty slot
  int lg = 0;
  uint32_t slot(int32_t m) const { return ((uint32_t)m * 2654435761u) >> (32 - lg); }
  // returns false if m is already present
  bool insert(int32_t m, int16_t c) {
    const uint32_t mask = (1u << lg) - 1;
    for (uint32_t h = slot(m);; h = (h + 1) & mask) {
      if (code[h] < 0) {
        iso[h] = m;
        code[h] = c;
        return true;
      }
      if (iso[h] == m) return false;
    }
  }
  int find(int32_t m) const {
    const uint32_t mask = (1u << lg) - 1;
    for (uint32_t h = slot(m);; h = (h + 1) & mask) {
      if (code[h] < 0) return -1;
      if (iso[h] == m) return code[h];
    }
  }
  void init(int n_sp) {
    lg = 2;
    while ((1 << lg) < 2 * n_sp) ++lg;
    iso.assign((size_t)1 << lg, 0);
    code.assign((size_t)1 << lg, (int16_t)-1);
  }
};

static int64_t rint_fix(double v) { return (int64_t)std::nearbyint(v * kFix); }

// Sorts idx[0..m) (line indices in input order, fixed-point keys key[]) stably by nu0: a
// counting pass on the leading bits of the keys, which are monotone in nu0 (about one line
// per bucket), then each bucket stably by nu0 itself (insertion sort; a library stable sort
// for the rare crowded bucket). tmp and start are scratch.
static void sort_run(const marfa_line_t* lines, const int64_t* key, int64_t* idx, int64_t m,
                     std::vector<int64_t>& tmp, std::vector<int64_t>& start) {
  auto less = [&](int64_t x, int64_t y) { return lines[x].nu0 < lines[y].nu0; };
  auto insertion = [&](int64_t* a, int64_t len) {
    for (int64_t i = 1; i < len; ++i) {
      const int64_t v = a[i];
      int64_t j = i - 1;
      while (j >= 0 && less(v, a[j])) {
        a[j + 1] = a[j];
        --j;
      }
      a[j + 1] = v;
    }
  };
  if (m <= 32) {
    insertion(idx, m);
    return;
  }
  int64_t kmin = INT64_MAX, kmax = INT64_MIN;
  for (int64_t i = 0; i < m; ++i) {
    kmin = std::min(kmin, key[idx[i]]);
    kmax = std::max(kmax, key[idx[i]]);
  }
  const uint64_t span = (uint64_t)(kmax - kmin);
  int bits = 0;
  while (bits < 64 && (span >> bits)) ++bits;
  int kb = 1;
  while (kb < 24 && ((int64_t)1 << kb) < m) ++kb;
  const int shift = bits > kb ? bits - kb : 0;
  const int64_t nbk = (int64_t)(span >> shift) + 1;
  start.assign(nbk + 1, 0);
  tmp.resize(m);
  for (int64_t i = 0; i < m; ++i) ++start[((uint64_t)(key[idx[i]] - kmin) >> shift) + 1];
  for (int64_t b = 0; b < nbk; ++b) start[b + 1] += start[b];
  for (int64_t i = 0; i < m; ++i) tmp[start[(uint64_t)(key[idx[i]] - kmin) >> shift]++] = idx[i];
  // start[b] now holds the end of bucket b
  int64_t a0 = 0;
  for (int64_t b = 0; b < nbk; ++b) {
    const int64_t a1 = start[b];
    if (a1 - a0 > 32)
      std::stable_sort(tmp.begin() + a0, tmp.begin() + a1, less);
    else if (a1 - a0 > 1)
      insertion(tmp.data() + a0, a1 - a0);
    a0 = a1;
  }
  std::copy(tmp.begin(), tmp.begin() + m, idx);
}

// order = the line indices src[0..n) (the identity 0..n-1 when src is NULL) stably sorted
// by nu0 (what std::stable_sort gives): a counting pass on the leading bits of key - kmin,
// each thread over its chunk of the input in order, splits the lines into coarse buckets;
// a bucket holding more than its share of the lines is split again the same way (once),
// and the threads then take the remaining buckets one at a time and sort each with
// sort_run. Returns false if scratch memory ran out.
static bool split_sort(const marfa_line_t* lines, const int64_t* key, const int64_t* src, int64_t n,
                       int64_t kmin, int64_t kmax, int64_t* order, bool top) {
  const uint64_t span = (uint64_t)(kmax - kmin);
  int bits = 0;
  while (bits < 64 && (span >> bits)) ++bits;
  int cb = 1;
  while (cb < 12 && ((int64_t)64 << cb) < n) ++cb;
  const int shift = bits > cb ? bits - cb : 0;
  const int64_t C = (int64_t)(span >> shift) + 1;
  const int nt = host_threads(n, 16384);
  std::vector<int64_t> hist;
  try {
    hist.assign((size_t)nt * C, 0);
  } catch (...) {
    return false;
  }
  auto line = [&](int64_t i) { return src ? src[i] : i; };
  auto coarse = [&](int64_t i) { return (int64_t)((uint64_t)(key[line(i)] - kmin) >> shift); };
  par_chunks(nt, n, [&](int64_t lo, int64_t hi, int t) {
    int64_t* h = hist.data() + (size_t)t * C;
    for (int64_t i = lo; i < hi; ++i) ++h[coarse(i)];
  });
  std::vector<int64_t> bstart(C + 1);
  int64_t run = 0;
  for (int64_t c = 0; c < C; ++c) {
    bstart[c] = run;
    for (int t = 0; t < nt; ++t) {
      const int64_t k = hist[(size_t)t * C + c];
      hist[(size_t)t * C + c] = run;
      run += k;
    }
  }
  bstart[C] = run;
  par_chunks(nt, n, [&](int64_t lo, int64_t hi, int t) {
    int64_t* pos = hist.data() + (size_t)t * C;
    for (int64_t i = lo; i < hi; ++i) order[pos[coarse(i)]++] = line(i);
  });
  // crowded buckets (a dense band in a wide key range): split again on all threads
  std::vector<char> done(C, 0);
  if (top && nt > 1) {
    const int64_t big = std::max<int64_t>(2 * n / nt, 1 << 15);
    for (int64_t c = 0; c < C; ++c) {
      const int64_t m = bstart[c + 1] - bstart[c];
      if (m <= big) continue;
      std::vector<int64_t> sub;
      try {
        sub.assign(order + bstart[c], order + bstart[c + 1]);
      } catch (...) {
        return false;
      }
      int64_t lo = INT64_MAX, hi = INT64_MIN;
      for (const int64_t i : sub) {
        lo = std::min(lo, key[i]);
        hi = std::max(hi, key[i]);
      }
      if (!split_sort(lines, key, sub.data(), m, lo, hi, order + bstart[c], false)) return false;
      done[c] = 1;
    }
  }
  std::atomic<int64_t> next{0};
  std::atomic<bool> oom{false};
  par_chunks(nt, nt, [&](int64_t, int64_t, int) {
    try {
      std::vector<int64_t> tmp, start;
      for (int64_t c; (c = next.fetch_add(1)) < C;)
        if (!done[c] && bstart[c + 1] - bstart[c] > 1)
          sort_run(lines, key, order + bstart[c], bstart[c + 1] - bstart[c], tmp, start);
    } catch (...) {
      oom = true;
    }
  });
  return !oom;
}

static bool sort_by_nu0(const marfa_line_t* lines, const int64_t* key, int64_t n, int64_t kmin,
                        int64_t kmax, int64_t* order) {
  return split_sort(lines, key, nullptr, n, kmin, kmax, order, true);
}

// what the validation of one chunk of lines found
struct ChunkScan {
  int64_t bad = INT64_MAX;  // first invalid line of the chunk
  int why = 0;              // 1 nu0 out of range, 2 unknown species, 3 non-finite parameter
  int32_t iso = 0;          // the unknown species
  bool sorted = true;       // the chunk is ordered by nu0
  int64_t kmin = INT64_MAX, kmax = INT64_MIN;
  double dmin = 1e300, dmax = -1e300;
};

// A line list prepared on the host: the list object (no device block yet) and the host
// staging block in the device block's layout, with the offsets of its sub-arrays.
struct StagedLines {
  marfa_lines_t* L = nullptr;
  std::unique_ptr<unsigned char[]> hb;
  size_t total = 0;
  size_t o_key = 0, o_nu = 0, o_S = 0, o_ga = 0, o_gs = 0, o_E = 0, o_na = 0, o_da = 0, o_sp = 0, o_b = 0;
};

// Validation, order, per-field arrays and bucket index of one line list, on the host
// (App. B records; the ordering and keys of the header's marfa_prepare_lines).
static int prepare_host(const marfa_line_t* lines, int64_t n, const marfa_species_t* sp, int32_t n_sp,
                        StagedLines& out) {
  if (!lines || n < 1) return fail(MARFA_E_INVAL, "need at least one line");
  if (n > (int64_t)1 << 31) return fail(MARFA_E_INVAL, "at most 2^31 lines");
  if (!sp || n_sp < 1 || n_sp > 32767) return fail(MARFA_E_INVAL, "need 1..32767 species");
  SpeciesIndex code;
  std::vector<int16_t> code_of;
  std::vector<int64_t> keyin, order;
  try {
    code.init(n_sp);
    code_of.resize(n);
    keyin.resize(n);
  } catch (...) {
    return fail(MARFA_E_NOMEM, "host allocation failed");
  }
  for (int s = 0; s < n_sp; ++s) {
    if (!code.insert(sp[s].mol_iso, (int16_t)s)) return fail(MARFA_E_INVAL, "duplicate species %d", sp[s].mol_iso);
    if (!(sp[s].mass_amu > 0) || !std::isfinite(sp[s].mass_amu) || !std::isfinite(sp[s].q_exp))
      return fail(MARFA_E_INVAL, "species %d: mass must be > 0 and q finite", sp[s].mol_iso);
  }
  // validate, resolve species codes (looked up once per run of equal species), take the
  // fixed-point keys and check whether the lines already come ordered by nu0 (line lists
  // usually do); each chunk stops at its first invalid line, and the first over all chunks
  // is the one reported
  const int nt = host_threads(n, 8192);
  std::vector<ChunkScan> scan(nt);
  par_chunks(nt, n, [&](int64_t lo, int64_t hi, int t) {
    ChunkScan& S = scan[t];
    int32_t last_iso = 0;
    int last_code = -1;
    for (int64_t i = lo; i < hi; ++i) {
      const marfa_line_t& l = lines[i];
      if (!std::isfinite(l.nu0) || l.nu0 < 0 || l.nu0 > 1e5) {
        S.bad = i, S.why = 1;
        return;
      }
      if (last_code < 0 || l.mol_iso != last_iso) {
        last_code = code.find(l.mol_iso);
        if (last_code < 0) {
          S.bad = i, S.why = 2, S.iso = l.mol_iso;
          return;
        }
        last_iso = l.mol_iso;
      }
      code_of[i] = (int16_t)last_code;
      if (!std::isfinite(l.S296) || !std::isfinite(l.gamma_air) || !std::isfinite(l.gamma_self) ||
          !std::isfinite(l.E_lower) || !std::isfinite(l.n_air) || !std::isfinite(l.delta_air)) {
        S.bad = i, S.why = 3;
        return;
      }
      if (i > 0 && l.nu0 < lines[i - 1].nu0) S.sorted = false;
      const int64_t k = rint_fix(l.nu0);
      keyin[i] = k;
      S.kmin = std::min(S.kmin, k);
      S.kmax = std::max(S.kmax, k);
      S.dmin = std::min(S.dmin, (double)l.delta_air);
      S.dmax = std::max(S.dmax, (double)l.delta_air);
    }
  });
  bool sorted = true;
  int64_t key_first = INT64_MAX, key_last = INT64_MIN;
  double dmin = 1e300, dmax = -1e300;
  for (const ChunkScan& S : scan) {
    if (S.why == 1) return fail(MARFA_E_INVAL, "line %lld: nu0 must be in [0, 1e5]", (long long)S.bad);
    if (S.why == 2) return fail(MARFA_E_INVAL, "line %lld: unknown species %d", (long long)S.bad, S.iso);
    if (S.why == 3) return fail(MARFA_E_INVAL, "line %lld: non-finite parameter", (long long)S.bad);
    sorted = sorted && S.sorted;
    key_first = std::min(key_first, S.kmin);
    key_last = std::max(key_last, S.kmax);
    dmin = std::min(dmin, S.dmin);
    dmax = std::max(dmax, S.dmax);
  }
  if (!sorted) {
    try {
      order.resize(n);
    } catch (...) {
      return fail(MARFA_E_NOMEM, "host allocation failed");
    }
    if (!sort_by_nu0(lines, keyin.data(), n, key_first, key_last, order.data()))
      return fail(MARFA_E_NOMEM, "host allocation failed");
  }
  auto src = [&](int64_t j) { return sorted ? j : order[j]; };

  marfa_lines_t* L = alloc_fails() ? nullptr : new (std::nothrow) marfa_lines_t();
  if (!L) return fail(MARFA_E_NOMEM, "host allocation failed");
  L->n = n;
  // bucket index over the sorted keys: about one line per two buckets on average, at
  // most 2^26 buckets
  const int64_t span = std::max<int64_t>(key_last - key_first, 1);
  int bs = 20;
  while (bs < 50 && (((int64_t)1 << (bs + 1)) * 2 * n <= span || (span >> bs) > ((int64_t)1 << 26))) ++bs;
  L->bshift = bs;
  L->key_base = (key_first >> bs) << bs;
  const int64_t nb64 = ((key_last - L->key_base) >> bs) + 1;
  if (nb64 > (int64_t)1 << 30) {
    delete L;
    return fail(MARFA_E_INVAL, "line list too sparse for the bucket index");
  }
  L->nbuck = (int32_t)nb64;
  // one device block for all arrays (256-byte aligned sub-arrays), filled in a host
  // staging block of the same layout and copied at once
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t sz_key = al(8 * n), sz_nu = al(8 * n), sz_f = al(4 * n), sz_sp = al(2 * n),
               sz_b = al(4 * (L->nbuck + 1));
  const size_t total = sz_key + sz_nu + 6 * sz_f + sz_sp + sz_b;
  std::unique_ptr<unsigned char[]> hb;
  try {
    L->species.assign(sp, sp + n_sp);
    L->perm.resize(n);
    if (alloc_fails()) throw std::bad_alloc();
    hb.reset(new unsigned char[total]);
  } catch (...) {
    delete L;
    return fail(MARFA_E_NOMEM, "host allocation failed");
  }
  size_t off = 0;
  // a sub-array of `used` bytes in a slot of sz bytes; the padding is zeroed
  auto carve = [&](size_t sz, size_t used) {
    const size_t o = off;
    off += sz;
    std::memset(hb.get() + o + used, 0, sz - used);
    return o;
  };
  const size_t o_key = carve(sz_key, 8 * n), o_nu = carve(sz_nu, 8 * n), o_S = carve(sz_f, 4 * n),
               o_ga = carve(sz_f, 4 * n), o_gs = carve(sz_f, 4 * n), o_E = carve(sz_f, 4 * n),
               o_na = carve(sz_f, 4 * n), o_da = carve(sz_f, 4 * n), o_sp = carve(sz_sp, 2 * n),
               o_b = carve(sz_b, 4 * ((size_t)L->nbuck + 1));
  int64_t* key = (int64_t*)(hb.get() + o_key);
  double* nu0 = (double*)(hb.get() + o_nu);
  float *S = (float*)(hb.get() + o_S), *ga = (float*)(hb.get() + o_ga), *gs = (float*)(hb.get() + o_gs),
        *E = (float*)(hb.get() + o_E), *na = (float*)(hb.get() + o_na), *da = (float*)(hb.get() + o_da);
  int16_t* spi = (int16_t*)(hb.get() + o_sp);
  int32_t* bfirst = (int32_t*)(hb.get() + o_b);
  int64_t* perm = L->perm.data();
  par_chunks(host_threads(n, 8192), n, [&](int64_t lo, int64_t hi, int) {
    for (int64_t j = lo; j < hi; ++j) {
      const int64_t i = src(j);
      const marfa_line_t& l = lines[i];
      perm[i] = j;
      nu0[j] = l.nu0;
      key[j] = keyin[i];
      S[j] = l.S296;
      ga[j] = l.gamma_air;
      gs[j] = l.gamma_self;
      E[j] = l.E_lower;
      na[j] = l.n_air;
      da[j] = l.delta_air;
      spi[j] = code_of[i];
    }
  });
  L->delta_min = dmin;
  L->delta_max = dmax;
  // bfirst[b] = the first sorted line whose key is >= the start of bucket b
  par_chunks(host_threads(L->nbuck + 1, 16384), L->nbuck + 1, [&](int64_t b0, int64_t b1, int) {
    int64_t i = std::lower_bound(key, key + n, L->key_base + (b0 << bs)) - key;
    for (int64_t b = b0; b < b1; ++b) {
      const int64_t K = L->key_base + (b << bs);
      while (i < n && key[i] < K) ++i;
      bfirst[b] = (int32_t)i;
    }
  });
  out.L = L;
  out.hb = std::move(hb);
  out.total = total;
  out.o_key = o_key, out.o_nu = o_nu, out.o_S = o_S, out.o_ga = o_ga, out.o_gs = o_gs;
  out.o_E = o_E, out.o_na = o_na, out.o_da = o_da, out.o_sp = o_sp, out.o_b = o_b;
  return MARFA_OK;
}

// The device block of a staged list from the stream-ordered pool, filled by one copy on
// the legacy default stream (a plain cudaMalloc per list costs more than the copy for the
// small lists of a batch of requests); the caller synchronises that stream.
static int upload_staged(StagedLines& st) {
  marfa_lines_t* L = st.L;
  CK(cudaGetDevice(&L->device));  // the calling thread's device
  if (const int ra = dev_alloc(&L->block, st.total, 0)) {
    L->block = nullptr;
    return ra;
  }
  char* p = (char*)L->block;
  L->key = (int64_t*)(p + st.o_key);
  L->nu0 = (double*)(p + st.o_nu);
  L->S296 = (float*)(p + st.o_S);
  L->ga = (float*)(p + st.o_ga);
  L->gs = (float*)(p + st.o_gs);
  L->E = (float*)(p + st.o_E);
  L->na = (float*)(p + st.o_na);
  L->da = (float*)(p + st.o_da);
  L->sp = (int16_t*)(p + st.o_sp);
  L->bfirst = (int32_t*)(p + st.o_b);
  CK(cudaMemcpyAsync(L->block, st.hb.get(), st.total, cudaMemcpyHostToDevice, 0));
  return MARFA_OK;
}

extern "C" int marfa_prepare_lines(const marfa_line_t* lines, int64_t n, const marfa_species_t* sp,
                                   int32_t n_sp, marfa_lines_t** out) {
  if (!out) return fail(MARFA_E_INVAL, "out is NULL");
  *out = nullptr;
  StagedLines st;
  int r = prepare_host(lines, n, sp, n_sp, st);
  if (r) return r;
  r = upload_staged(st);
  if (!r && cudaStreamSynchronize(0) != cudaSuccess) r = fail(MARFA_E_CUDA, "copying the line list failed");
  // commit marfa_absorption_noalloc's scratch on this device now (see noalloc_scratch)
  char* scratch = nullptr;
  if (!r) r = noalloc_scratch(&scratch);
  if (r) {
    marfa_free_lines(st.L);
    return r;
  }
  *out = st.L;
  return MARFA_OK;
}

// Several line lists at once: the host stages run in parallel on the host pool (one list
// per thread, each list's own loops serial), then the device blocks are filled in order
// on the legacy default stream and synchronised once.
extern "C" int marfa_prepare_lines_batch(int32_t n_req, const marfa_line_t* const* lines, const int64_t* n,
                                         const marfa_species_t* const* sp, const int32_t* n_sp,
                                         marfa_lines_t** out) {
  if (!out || !lines || !n || !sp || !n_sp || n_req < 1) return fail(MARFA_E_INVAL, "bad batch arguments");
  for (int32_t q = 0; q < n_req; ++q) out[q] = nullptr;
  std::vector<StagedLines> st;
  std::vector<int> rc;
  std::vector<std::string> msg;
  try {
    st.resize(n_req);
    rc.assign(n_req, 0);
    msg.resize(n_req);
  } catch (...) {
    return fail(MARFA_E_NOMEM, "host allocation failed");
  }
  std::atomic<int32_t> next{0};
  const int nt = (int)std::min<int64_t>(host_threads((int64_t)n_req << 20, 1 << 20), n_req);
  par_chunks(nt, nt, [&](int64_t, int64_t, int) {
    const bool was = t_serial_loops;
    t_serial_loops = true;
    for (int32_t q; (q = next.fetch_add(1)) < n_req;) {
      rc[q] = prepare_host(lines[q], n[q], sp[q], n_sp[q], st[q]);
      if (rc[q]) msg[q] = g_err;
    }
    t_serial_loops = was;
  });
  int r = MARFA_OK;
  for (int32_t q = 0; q < n_req && !r; ++q)
    if (rc[q]) r = fail(rc[q], "request %d: %s", q, msg[q].c_str());
  for (int32_t q = 0; q < n_req && !r; ++q) {
    r = upload_staged(st[q]);
    if (r) r = fail(r, "request %d: %s", q, g_err.c_str());
  }
  if (!r && cudaStreamSynchronize(0) != cudaSuccess) r = fail(MARFA_E_CUDA, "copying the line lists failed");
  char* scratch = nullptr;
  if (!r) r = noalloc_scratch(&scratch);
  if (r) {
    for (auto& x : st) marfa_free_lines(x.L);
    return r;
  }
  for (int32_t q = 0; q < n_req; ++q) out[q] = st[q].L;
  return MARFA_OK;
}

extern "C" int marfa_diag_line_order(const marfa_line_t* lines, int64_t n, int64_t* order) {
  if (!lines || !order || n < 1 || n > (int64_t)1 << 31) return fail(MARFA_E_INVAL, "bad arguments");
  std::vector<int64_t> key;
  try {
    key.resize(n);
  } catch (...) {
    return fail(MARFA_E_NOMEM, "host allocation failed");
  }
  int64_t kmin = INT64_MAX, kmax = INT64_MIN;
  bool sorted = true;
  for (int64_t i = 0; i < n; ++i) {
    const double v = lines[i].nu0;
    if (!std::isfinite(v) || v < 0 || v > 1e5)
      return fail(MARFA_E_INVAL, "line %lld: nu0 must be in [0, 1e5]", (long long)i);
    key[i] = rint_fix(v);
    kmin = std::min(kmin, key[i]);
    kmax = std::max(kmax, key[i]);
    if (i > 0 && v < lines[i - 1].nu0) sorted = false;
  }
  if (sorted) {
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    return MARFA_OK;
  }
  if (!sort_by_nu0(lines, key.data(), n, kmin, kmax, order)) return fail(MARFA_E_NOMEM, "host allocation failed");
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
// Size classes of a batch's requests, tuned apart: windows up to 16 cm^-1 (narrow) and
// wider ones. Per class: the grid-1 split (entry 1 of a choice row), the kernel variant of
// grids 2..10 (entries 2..10) and of the finest grid (entry 11).
constexpr int kNClasses = 2;
constexpr int64_t kNarrowPts = 16 * 2048 + 1;
constexpr int kG1Splits[4] = {1, 2, 3, 6};
// The grid-1 split of calls without tuning, per size class: what the autotuner chooses on
// the uneven batch for its narrow requests (2) and on the Venus window (6).
constexpr int kG1DefaultSplit[2] = {2, 6};

struct Plan {
  const marfa_lines_t* lines = nullptr;
  marfa_request_t rq{};
  int32_t n_levels = 0;
  std::vector<LevelDev> lev;
  std::vector<LevelSpeciesDev> ls;
  ReqDev rd{};
  int64_t npts = 0;
  int req_idx = 0;
  int cls = 0;                // size class: 0 narrow window, 1 wide (kernel choices per class)
  PrepArgs prep{};            // level-preparation launch, filled by upload()
  // device buffers
  void* dbuf = nullptr;       // per-level line data + slots + tables
  float* dout = nullptr;      // output (own buffer when the caller's is on the host)
  bool own_out = false;
  bool host_direct = false;  // dout is the device view of a page-locked host k_out
  float* user_out = nullptr;
};

// ------------------------------------------------------------------ surrogate state
// The loaded surrogate: inference weights and guard on one device.
static std::mutex g_surr_mu;
static int g_surr_dev = -1;
static MlpWeights* g_surr_w = nullptr;

static int surrogate_for_current_device(const MlpWeights** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_surr_mu);
  if (!g_surr_w) return fail(MARFA_E_INVAL, "surrogate requested but none is loaded (marfa_surrogate_load)");
  if (g_surr_dev != dev)
    return fail(MARFA_E_INVAL, "the surrogate is loaded on device %d, not on the current device %d",
                g_surr_dev, dev);
  *out = g_surr_w;
  return MARFA_OK;
}

// ------------------------------------------------------------------ user-defined shape
// The devices on which marfa_shape_user_set has put a table.
static std::mutex g_user_mu;
static uint64_t g_user_devs = 0;
static bool user_shape_set_here() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lk(g_user_mu);
  return (g_user_devs >> dev) & 1;
}

extern "C" int marfa_shape_user_set(const float* g, int32_t n, double x_max) {
  if (!g || n < 2 || n > kUserShapeMax) return fail(MARFA_E_INVAL, "need 2..%d samples", kUserShapeMax);
  if (!std::isfinite(x_max) || !(x_max > 0) || x_max > 1e6) return fail(MARFA_E_INVAL, "x_max must be in (0, 1e6]");
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(g[i]) || g[i] < 0) return fail(MARFA_E_INVAL, "sample %d is negative or not finite", i);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(MARFA_E_INVAL, "device %d out of range", dev);
  const int e = set_user_shape(g, n, (float)x_max);
  if (e) return fail(MARFA_E_CUDA, "user shape upload: %s", cudaGetErrorString((cudaError_t)e));
  CK(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_user_mu);
  g_user_devs |= uint64_t(1) << dev;
  return MARFA_OK;
}

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
        s == MARFA_SHAPE_VOIGT_PAPER || s == MARFA_SHAPE_USER || s == MARFA_SHAPE_TEST_CONST ||
        s == MARFA_SHAPE_TEST_QUAD || s == MARFA_SHAPE_TEST_QUART))
    return fail(MARFA_E_INVAL, "unknown shape %d", s);
  if (s == MARFA_SHAPE_USER && !user_shape_set_here())
    return fail(MARFA_E_INVAL, "shape USER requested but no user shape is set on this device (marfa_shape_user_set)");
  if (rq->chi != MARFA_CHI_NONE && rq->chi != MARFA_CHI_TONKOV)
    return fail(MARFA_E_INVAL, "unknown chi %d", rq->chi);
  if (rq->units < MARFA_UNITS_SIGMA || rq->units > MARFA_UNITS_K_KM1)
    return fail(MARFA_E_INVAL, "unknown units %d", rq->units);
  if (rq->surrogate != 0 && rq->surrogate != 1) return fail(MARFA_E_INVAL, "surrogate must be 0 or 1");
  if (rq->surrogate && rq->shape != MARFA_SHAPE_VOIGT)
    return fail(MARFA_E_INVAL, "the surrogate stands in for the Voigt profile only");
  if (rq->R_w < 1 || rq->R_w > 64 || rq->R_c < 1 || rq->R_c > 64)
    return fail(MARFA_E_INVAL, "R_w and R_c must be in 1..64");
  if (rq->stencil != 0 && rq->stencil != 3 && rq->stencil != 5)
    return fail(MARFA_E_INVAL, "stencil must be 3 or 5 (0: 3)");
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
  R.wide = rq->stencil == 5 ? 1 : 0;
  for (int g = 1; g <= kNGrid; ++g) {
    const int s = panel_shift(g);
    if (R.wide) {  // whole four-step panels: both halves of every panel the window touches
      R.m_first[g] = (X_lo >> (s + 1)) << 1;
      R.npan[g] = (((X_hi >> (s + 1)) << 1) + 1) - R.m_first[g] + 1;
    } else {
      R.m_first[g] = X_lo >> s;
      R.npan[g] = (X_hi >> s) - R.m_first[g] + 1;
    }
    R.slot_off[g] = off;
    off += 3 * R.npan[g] * (g == 1 ? kG1Split : 1);
  }
  R.slots_per_level = off;
  R.cut_fx = (int64_t)std::nearbyint(rq->cutoff * kFix);
  R.R_w = rq->R_w;
  R.shape = rq->shape;
  R.chi_req = rq->chi == MARFA_CHI_TONKOV ? 1 : 0;
  R.mech = 0;
  if (!R.wide) {
    for (int g = 2; g <= kNGrid; ++g)
      if (mech_ok(g, R.cut_fx, R.R_w, R.chi_req != 0)) R.mech |= 1 << g;
    if (mech_fine_ok(R.cut_fx, R.R_w, R.chi_req != 0)) R.mech |= 1 << (kNGrid + 1);
    if (mech_fine_merge_ok(R.cut_fx, R.R_w, R.chi_req != 0, (int64_t)kFineWarpNodes << kFineShift))
      R.mech |= 1 << (kNGrid + 2);
  }
  R.mlp = nullptr;
  if (rq->surrogate) {
    r = surrogate_for_current_device(&R.mlp);
    if (r) return r;
  }
  R.out_scale = (float)(1.0 / scale);
  R.npts = P.npts;
  R.g1_split = kG1Split;
  P.cls = P.npts <= kNarrowPts ? 0 : 1;
  (void)physical;
  P.req_idx = req_idx;
  return MARFA_OK;
}

// The work items of a plan: grid 1 in tiles of kG1Pairs pairs (each in `split` parts),
// grids 2..10 in tiles of their kernel variant's pairs (variant_pairs), the finest grid in
// tiles of kFineTile nodes starting on a G10 panel; every level, level-major. Each kind
// as an ExpandDesc (base, step, tiles per level), written by the device or, for the
// no-alloc path and the counting runs, by expand_on_host.
static int64_t variant_pairs(int v);
static ExpandDesc plan_desc(const Plan& P, int kind, int v_or_split) {
  const ReqDev& R = P.rd;
  ExpandDesc d{};
  d.kind = kind;
  d.req = P.req_idx;
  d.n_levels = P.n_levels;
  d.split = kind == 1 ? v_or_split : 1;
  if (kind == 1) {
    d.base = R.m_first[1];
    d.step = kG1Pairs;
    d.tiles = R.npan[1] / kG1Pairs + 1;
  } else if (kind <= kNGrid) {
    d.base = R.m_first[kind];
    d.step = variant_pairs(v_or_split);
    d.tiles = R.npan[kind] / d.step + 1;
  } else {
    d.base = R.k_lo & ~(int64_t)7;
    d.step = kFineTile;
    d.tiles = (R.k_hi - d.base) / kFineTile + 1;
  }
  return d;
}
static int64_t desc_count(const ExpandDesc& d) { return d.tiles * d.split * d.n_levels; }
template <class Item>
static void expand_on_host(const ExpandDesc& d, std::vector<Item>& out) {
  for (int l = 0; l < d.n_levels; ++l)
    for (int64_t t = 0; t < d.tiles; ++t)
      for (int part = 0; part < d.split; ++part) {
        const int64_t pos = d.base + t * d.step;
        if constexpr (std::is_same<Item, G1Item>::value)
          out.push_back(G1Item{d.req, l, pos, part, 0});
        else if constexpr (std::is_same<Item, CoarseItem>::value)
          out.push_back(CoarseItem{d.req, l, d.kind, 0, pos});
        else
          out.push_back(FineItem{d.req, l, pos});
      }
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory (cudaHostAlloc / cudaHostRegister, mapped
// into the device's address space), or null for any other memory.
static void* pinned_host_view(void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Kernel variants of grids 2..10: 0 = line-major (k_coarse_lm, kLPairs node pairs per
// CTA), 1 = two-phase (k_coarse, kCWarps x kCPairs node pairs per CTA), 2 = line-major
// with 16 node pairs per CTA (half the shared memory, narrower tiles), 3 = flattened
// (k_coarse_jobs: the two-phase tiles with phase 1 spread evenly over the lanes and
// grouped by Voigt branch), 4 = by mechanism (k_coarse_mech: the two-phase tiles with
// closed-form ownership, one candidate pass per mechanism, where every request of the
// launch has its mech bit for the grid; otherwise the launch takes variant 1), 5 = the
// same in one merged pass. Finest grid (kind kFineKind): 0 = k_fine (an 8-lane group per
// G10 panel), 1 = k_fine_jobs ((line, panel) jobs spread evenly over the groups), 2 = the
// same with closed-form ownership, one pass per mechanism (mech bit of every request;
// otherwise variant 1), 3 = the same with a centre pass and one merged pass over the
// edges and breakpoints (merge bit of every request; otherwise variant 2).
// Surrogate-capable launches always take variant 1 on grids 2..10 (when 3 is chosen)
// and k_fine. Calls without tuning take the process-wide defaults (marfa_diag_variants).
constexpr int kNVariants = 6;
constexpr int kFineKind = kNGrid + 1;
constexpr int kNFineVariants = 4;
// Defaults measured on the Venus workload (line-major over 16 pairs on grids 2..7, the
// mechanism kernel on 8..10, flattened jobs by mechanism, a pass per mechanism, on the
// finest grid).
static std::atomic<int> g_default_variant[kNGrid + 2] = {{-1}, {-1}, {2}, {2}, {2}, {2}, {2}, {2}, {4}, {4}, {4}, {2}};
static int default_variant(int g) { return g_default_variant[g].load(std::memory_order_relaxed); }
static int64_t variant_pairs(int v) {
  return v == 0 ? (int64_t)kLPairs : (v == 2 ? (int64_t)16 : (int64_t)kCPairs * kCWarps);
}

static void coarse_items(const Plan& P, int g, int v, std::vector<CoarseItem>& out) {
  const ReqDev& R = P.rd;
  for (int l = 0; l < P.n_levels; ++l)
    for (int64_t m0 = R.m_first[g]; m0 <= R.m_first[g] + R.npan[g]; m0 += variant_pairs(v))
      out.push_back(CoarseItem{P.req_idx, l, g, 0, m0});
}

static void launch_prep(const Plan& P, cudaStream_t st, bool timed) {
  cudaEvent_t ev = timed ? timing_begin(st) : nullptr;
  launch_level_prep(P.prep, (int)P.n_levels, st);
  timing_end(ev, 0, st);
}

static int upload(Plan& P, float* k_out, cudaStream_t st);

// Allocate the per-request device buffers of a plan and run the level preparation.
static int upload_and_prep(Plan& P, float* k_out, cudaStream_t st) {
  int r = upload(P, k_out, st);
  if (r) return r;
  launch_prep(P, st, true);
  CK(cudaGetLastError());
  return MARFA_OK;
}

// Allocate the per-request device buffers of a plan and copy its level tables.
static int upload(Plan& P, float* k_out, cudaStream_t st) {
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
  void* pinned = k_out && !is_device_ptr(k_out) ? pinned_host_view(k_out) : nullptr;
  if (k_out && is_device_ptr(k_out)) {
    P.dout = k_out;
    P.own_out = false;
  } else if (pinned) {
    // the finest-grid kernel stores the result straight into the page-locked host
    // buffer (no device buffer, no copy back); the call still returns when it is there
    P.dout = (float*)pinned;
    P.own_out = false;
    P.host_direct = true;
  } else {
    r = dev_alloc((void**)&P.dout, 4 * (size_t)P.npts * nl, st);
    if (r) return r;
    P.own_out = true;
  }
  R.out = P.dout;
  PrepArgs& a = P.prep;
  a.n = n;
  a.nu0 = L->nu0; a.S296 = L->S296; a.ga = L->ga; a.gs = L->gs; a.E = L->E; a.na = L->na; a.da = L->da;
  a.species = L->sp;
  a.n_species = ns;
  a.lev = dlev;
  a.ls = dls;
  a.shape = P.rq.shape;
  a.R_c = P.rq.R_c;
  a.c = c; a.amp = amp; a.sx = sx; a.yv = yv; a.gstar = gst; a.flags = fl;
  return MARFA_OK;
}

static void release(Plan& P, cudaStream_t st) {
  if (P.dbuf) cudaFreeAsync(P.dbuf, st);
  if (P.own_out && P.dout) cudaFreeAsync(P.dout, st);
  P.dbuf = nullptr;
  P.dout = nullptr;
}

// Run the coarse and finest-grid kernels for a set of prepared plans.
// ------------------------------------------------------------------ work sets
// All launches of a set of prepared requests: the work lists of every kernel (grid 1,
// grids 2..10 with their kernel variants, finest grid) and their device copies.
struct WorkSet {
  std::vector<ReqDev> rds;
  // items of each kind (1 grid 1, 2..10 grids, 11 finest), class 0 first then class 1:
  // kind k's class-c items are first[k][c] .. first[k][c + 1] - 1
  size_t n_gi = 0, n_ci[kNGrid + 1] = {}, n_fi = 0;  // items of grid 1, grids 2..10, the finest
  std::vector<ExpandDesc> desc;  // the items, written on the device (launch_expand_items)
  // host copies of the items, made for counting runs only (read_counts)
  std::vector<G1Item> gi;
  std::vector<CoarseItem> ci[kNGrid + 1];  // grids 2..10
  std::vector<FineItem> fi;
  size_t first[kNGrid + 2][kNClasses + 1] = {};
  int tune[kNClasses][kNGrid + 2] = {};    // per class: [1] grid-1 split, [2..10] variants, [11] finest
  bool surr = false;                       // some request uses the surrogate
  bool wide = false;                       // the requests use the 5-point partition
  bool surr_grid[kNGrid + 2] = {false};    // surrogate-capable kernels for grid 1..10, 11 finest
  size_t cw = 8 * kCountFields;            // count bytes per item
  void* buf = nullptr;
  ReqDev* drd = nullptr;
  G1Item* dgi = nullptr;
  CoarseItem* dci[kNGrid + 1] = {nullptr};
  FineItem* dfi = nullptr;
  int64_t* dgc = nullptr;
  int64_t* dcc[kNGrid + 1] = {nullptr};
  int64_t* dfc = nullptr;
  // every request's level preparation as one launch: the requests' arguments and the
  // prefix sums of their blocks
  std::vector<PrepArgs> prep;
  std::vector<int64_t> prep_first;
  PrepArgs* dprep = nullptr;
  int64_t* dprep_first = nullptr;
};

static void free_work(WorkSet& W, cudaStream_t st) {
  if (W.buf) cudaFreeAsync(W.buf, st);
  W.buf = nullptr;
}

// Build the work lists of plans with the kernel choices tune[class] (NULL: the defaults
// for every class: grid-1 split kG1DefaultSplit), allocate their device copies (plus
// count buffers when count) and upload.
static int build_work(std::vector<Plan>& plans, const int (*tune)[kNGrid + 2], bool count, WorkSet& W,
                      cudaStream_t st) {
  for (int c = 0; c < kNClasses; ++c)
    for (int k = 1; k <= kNGrid + 1; ++k)
      W.tune[c][k] = tune ? tune[c][k] : (k == 1 ? kG1DefaultSplit[c] : default_variant(k));
  for (auto& P : plans) {
    W.rds.push_back(P.rd);
    W.rds.back().g1_split = W.tune[P.cls][1];
  }
  for (auto& R : W.rds) W.surr = W.surr || R.mlp != nullptr;
  W.wide = !W.rds.empty() && W.rds[0].wide != 0;
  for (auto& R : W.rds)
    if ((R.wide != 0) != W.wide)
      return fail(MARFA_E_INVAL, "the requests of one call or plan must share one stencil");
  for (int g = 1; g <= kNGrid + 1; ++g) W.surr_grid[g] = W.surr;
  // items in order: class, then request, then kind; kind k's class-c items are
  // first[k][c] .. first[k][c + 1] - 1
  size_t at[kNGrid + 2] = {};
  for (int c = 0; c < kNClasses; ++c) {
    for (int k = 1; k <= kNGrid + 1; ++k) W.first[k][c] = at[k];
    for (auto& P : plans) {
      if (P.cls != c) continue;
      for (int k = 1; k <= kNGrid + 1; ++k) {
        ExpandDesc d = plan_desc(P, k, k == kNGrid + 1 ? 0 : W.tune[c][k]);
        d.dst = reinterpret_cast<void*>(at[k]);  // the item index for now; a pointer below
        at[k] += (size_t)desc_count(d);
        if (desc_count(d) > 0) W.desc.push_back(d);
        if (count) {
          if (k == 1) expand_on_host(d, W.gi);
          else if (k <= kNGrid) expand_on_host(d, W.ci[k]);
          else expand_on_host(d, W.fi);
        }
      }
    }
  }
  for (int k = 1; k <= kNGrid + 1; ++k) W.first[k][kNClasses] = at[k];
  W.n_gi = at[1];
  for (int g = 2; g <= kNGrid; ++g) W.n_ci[g] = at[g];
  W.n_fi = at[kNGrid + 1];
  W.prep_first.push_back(0);
  for (auto& P : plans) {
    W.prep.push_back(P.prep);
    W.prep_first.push_back(W.prep_first.back() + (P.prep.n + 255) / 256 * P.n_levels);
  }
  if (W.prep_first.back() > 0x7fffffff) return fail(MARFA_E_INVAL, "too many (level, line) pairs in one call");
  size_t total_items = W.n_gi + W.n_fi;
  for (int g = 2; g <= kNGrid; ++g) total_items += W.n_ci[g];
  if (W.n_gi > 0x7fffffffu || W.n_fi > 0x7fffffffu || total_items > ((size_t)1 << 34) ||
      W.desc.size() > 0x7fffffffu)
    return fail(MARFA_E_INVAL, "too much work in one call");
  for (int g = 2; g <= kNGrid; ++g)
    if (W.n_ci[g] > 0x7fffffffu) return fail(MARFA_E_INVAL, "too much work in one call");
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t cw = count ? W.cw : 0;
  size_t sz = al(sizeof(ReqDev) * W.rds.size()) + al(sizeof(G1Item) * W.n_gi) + al(sizeof(FineItem) * W.n_fi) +
              al(cw * W.n_gi) + al(cw * W.n_fi) + al(sizeof(ExpandDesc) * W.desc.size());
  for (int g = 2; g <= kNGrid; ++g) sz += al(sizeof(CoarseItem) * W.n_ci[g]) + al(cw * W.n_ci[g]);
  sz += al(sizeof(PrepArgs) * W.prep.size()) + al(sizeof(int64_t) * W.prep_first.size());
  int r = dev_alloc(&W.buf, sz, st);
  if (r) return r;
  char* p = (char*)W.buf;
  auto take = [&](size_t b) {
    char* q = p;
    p += al(b);
    return q;
  };
  W.drd = (ReqDev*)take(sizeof(ReqDev) * W.rds.size());
  W.dgi = (G1Item*)take(sizeof(G1Item) * W.n_gi);
  W.dfi = (FineItem*)take(sizeof(FineItem) * W.n_fi);
  for (int g = 2; g <= kNGrid; ++g) W.dci[g] = (CoarseItem*)take(sizeof(CoarseItem) * W.n_ci[g]);
  W.dprep = (PrepArgs*)take(sizeof(PrepArgs) * W.prep.size());
  W.dprep_first = (int64_t*)take(sizeof(int64_t) * W.prep_first.size());
  ExpandDesc* ddesc = (ExpandDesc*)take(sizeof(ExpandDesc) * W.desc.size());
  if (count) {
    W.dgc = (int64_t*)take(cw * W.n_gi);
    W.dfc = (int64_t*)take(cw * W.n_fi);
    for (int g = 2; g <= kNGrid; ++g) W.dcc[g] = (int64_t*)take(cw * W.n_ci[g]);
  }
  for (auto& d : W.desc) {  // item index -> device address of the kind's array
    const size_t i = reinterpret_cast<size_t>(d.dst);
    d.dst = d.kind == 1 ? (void*)(W.dgi + i) : (d.kind <= kNGrid ? (void*)(W.dci[d.kind] + i) : (void*)(W.dfi + i));
  }
  cudaError_t e = cudaSuccess;
  auto up = [&](void* d, const void* h, size_t b) {
    if (!e && b) e = cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, st);
  };
  up(W.drd, W.rds.data(), sizeof(ReqDev) * W.rds.size());
  up(ddesc, W.desc.data(), sizeof(ExpandDesc) * W.desc.size());
  up(W.dprep, W.prep.data(), sizeof(PrepArgs) * W.prep.size());
  up(W.dprep_first, W.prep_first.data(), sizeof(int64_t) * W.prep_first.size());
  if (!e) {
    launch_expand_items(ddesc, (int)W.desc.size(), st);
    e = cudaGetLastError();
  }
  if (!e && count) {
    e = cudaMemsetAsync(W.dgc, 0, cw * W.n_gi, st);
    if (!e) e = cudaMemsetAsync(W.dfc, 0, cw * W.n_fi, st);
    for (int g = 2; g <= kNGrid && !e; ++g) e = cudaMemsetAsync(W.dcc[g], 0, cw * W.n_ci[g], st);
  }
  if (e) {
    free_work(W, st);
    return fail(MARFA_E_CUDA, "upload of work lists failed: %s", cudaGetErrorString(e));
  }
  return MARFA_OK;
}

// Grid g (2..10) of a work set, the items of class c, with that class's kernel variant.
static void launch_grid(const WorkSet& W, int g, int c, cudaStream_t st) {
  const size_t f0 = W.first[g][c];
  const int n = (int)(W.first[g][c + 1] - f0);
  if (n <= 0) return;
  const int v = W.tune[c][g];
  const CoarseItem* items = W.dci[g] + f0;
  int64_t* counts = W.dcc[g] ? W.dcc[g] + f0 * kCountFields : nullptr;
  bool mech = (v == 4 || v == 5) && !W.surr_grid[g] && !W.wide;
  for (const auto& R : W.rds) mech = mech && ((R.mech >> g) & 1);
  if (mech)
    launch_coarse_mech(W.drd, items, n, counts, v == 5, st);
  else if (v == 3 && !W.surr_grid[g])
    launch_coarse_jobs(W.drd, items, n, counts, W.wide, st);
  else if (v == 1 || v >= 3)
    launch_coarse(W.drd, items, n, counts, W.surr_grid[g], W.wide, st);
  else
    launch_coarse_lm(W.drd, items, n, counts, W.surr_grid[g], v == 2 ? 16 : kLPairs, W.wide, st);
}
static void launch_grid(const WorkSet& W, int g, cudaStream_t st) {
  for (int c = 0; c < kNClasses; ++c) launch_grid(W, g, c, st);
}

// The finest grid + cascade of a work set, the items of class c, with that class's variant.
static void launch_finest(const WorkSet& W, int c, cudaStream_t st) {
  const size_t f0 = W.first[kNGrid + 1][c];
  const int n = (int)(W.first[kNGrid + 1][c + 1] - f0);
  if (n <= 0) return;
  const int v = W.tune[c][kFineKind];
  const FineItem* items = W.dfi + f0;
  int64_t* counts = W.dfc ? W.dfc + f0 * kCountFields : nullptr;
  bool mech = v >= 2 && !W.wide, merge = v == 3;
  for (const auto& R : W.rds) {
    mech = mech && ((R.mech >> (kNGrid + 1)) & 1);
    merge = merge && ((R.mech >> (kNGrid + 2)) & 1);
  }
  if (v >= 1 && !W.surr_grid[kNGrid + 1])
    launch_fine_jobs(W.drd, items, n, counts, W.wide, mech ? (merge ? 2 : 1) : 0, st);
  else
    launch_fine(W.drd, items, n, counts, W.surr_grid[kNGrid + 1], W.wide, st);
}
static void launch_finest(const WorkSet& W, cudaStream_t st) {
  for (int c = 0; c < kNClasses; ++c) launch_finest(W, c, st);
}

// Grid 1 of a work set, the items of class c (their requests' g1_split parts).
static void launch_grid1(const WorkSet& W, int c, cudaStream_t st) {
  const size_t f0 = W.first[1][c];
  const int n = (int)(W.first[1][c + 1] - f0);
  if (n <= 0) return;
  launch_g1(W.drd, W.dgi + f0, n, W.dgc ? W.dgc + f0 * kCountFields : nullptr, W.surr_grid[1], W.wide, st);
}
static void launch_grid1(const WorkSet& W, cudaStream_t st) {
  for (int c = 0; c < kNClasses; ++c) launch_grid1(W, c, st);
}

// Every summation launch of a work set: grid 1, grids 2..10, finest grid + cascade.
static int launch_work(const WorkSet& W, cudaStream_t st, bool timed) {
  cudaEvent_t ev = timed ? timing_begin(st) : nullptr;
  launch_grid1(W, st);
  timing_end(ev, 1, st);
  cudaError_t e;
  if ((e = cudaGetLastError())) return fail(MARFA_E_CUDA, "grid-1 kernel: %s", cudaGetErrorString(e));
  for (int g = 2; g <= kNGrid; ++g) {
    ev = timed ? timing_begin(st) : nullptr;
    launch_grid(W, g, st);
    timing_end(ev, g, st);
  }
  if ((e = cudaGetLastError())) return fail(MARFA_E_CUDA, "coarse-grid kernel: %s", cudaGetErrorString(e));
  ev = timed ? timing_begin(st) : nullptr;
  launch_finest(W, st);
  timing_end(ev, kNGrid + 1, st);
  if ((e = cudaGetLastError())) return fail(MARFA_E_CUDA, "fine kernel: %s", cudaGetErrorString(e));
  return MARFA_OK;
}

// Read the count buffers of a work set (synchronises st): counts[q] receives, per level
// of plan q and per grid (1..10, then the finest), kCountFields numbers: all profile
// evaluations, those the surrogate took, plain Voigt evaluations in 9 x 9 polynomial
// cells, in the asymptotic series and in small-y cells ([n_levels][11][kCountFields]).
static int read_counts(const WorkSet& W, std::vector<Plan>& plans, cudaStream_t st,
                       std::vector<int64_t>* counts) {
  constexpr int F = kCountFields;
  std::vector<int64_t> hg(W.gi.size() * F), hf(W.fi.size() * F), hc[kNGrid + 1];
  cudaError_t e = cudaSuccess;
  auto down = [&](void* h, const void* d, size_t b) {
    if (!e && b) e = cudaMemcpyAsync(h, d, b, cudaMemcpyDeviceToHost, st);
  };
  down(hg.data(), W.dgc, 8 * hg.size());
  down(hf.data(), W.dfc, 8 * hf.size());
  for (int g = 2; g <= kNGrid; ++g) {
    hc[g].resize(W.ci[g].size() * F);
    down(hc[g].data(), W.dcc[g], 8 * hc[g].size());
  }
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return fail(MARFA_E_CUDA, "count read-back failed: %s", cudaGetErrorString(e));
  for (size_t q = 0; q < plans.size(); ++q) counts[q].assign((size_t)plans[q].n_levels * 11 * F, 0);
  auto add = [&](int req, int level, int slot, const int64_t* v) {
    int64_t* d = &counts[req][((size_t)level * 11 + slot) * F];
    for (int i = 0; i < F; ++i) d[i] += v[i];
  };
  for (size_t k = 0; k < W.gi.size(); ++k) add(W.gi[k].req, W.gi[k].level, 0, &hg[k * F]);
  for (int g = 2; g <= kNGrid; ++g)
    for (size_t k = 0; k < W.ci[g].size(); ++k) add(W.ci[g][k].req, W.ci[g][k].level, g - 1, &hc[g][k * F]);
  for (size_t k = 0; k < W.fi.size(); ++k) add(W.fi[k].req, W.fi[k].level, 10, &hf[k * F]);
  return MARFA_OK;
}

// Run the summation kernels for a set of prepared plans (default kernel variants);
// counts (optional) as in read_counts.
static int run_plans(std::vector<Plan>& plans, cudaStream_t st, std::vector<int64_t>* counts) {
  WorkSet W;
  int r = build_work(plans, nullptr, counts != nullptr, W, st);
  if (r) return r;
  // the level preparation: one launch for all requests of a batch (each alone would fill
  // the GPU poorly), the request's own for one
  if (plans.size() > 1) {
    cudaEvent_t ev = timing_begin(st);
    launch_level_prep_batch(W.dprep, W.dprep_first, (int)plans.size(), W.prep_first.back(), st);
    timing_end(ev, 0, st);
  } else {
    launch_prep(plans[0], st, true);
  }
  r = launch_work(W, st, true);
  if (!r && counts) r = read_counts(W, plans, st, counts);
  free_work(W, st);
  return r;
}

static int finish_outputs(std::vector<Plan>& plans, cudaStream_t st) {
  bool any_host = false;
  for (auto& P : plans) {
    if (P.own_out && P.user_out) {
      CK(cudaMemcpyAsync(P.user_out, P.dout, 4 * (size_t)P.npts * P.n_levels, cudaMemcpyDeviceToHost, st));
      any_host = true;
    }
    if (P.host_direct) any_host = true;
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
    int r = upload(plans[q], k_out[q], st);
    if (r) {
      for (auto& P : plans) release(P, st);
      return r;
    }
  }
  int r = run_plans(plans, st, counts);
  if (r) {
    for (auto& P : plans) release(P, st);
    return r;
  }
  r = finish_outputs(plans, st);
  return r ? r : debug_checks();
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

// ------------------------------------------------------------------ captured plans
// A batch of requests prepared once and captured as one CUDA graph: level preparation
// of every request, then grid 1, grids 2..10 and the finest grid over all requests.
// Event-record nodes around each kernel kind give per-kernel times of the last replay.
constexpr int kKinds = kNGrid + 2;
constexpr int kSide = 4;  // capture streams of the parallel coarse-grid branches

struct marfa_plan {
  int device = 0;
  std::vector<Plan> plans;
  WorkSet W;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[2 * kKinds] = {nullptr};
  // per class: the autotuner's time per launch of each variant ([1]: of each grid-1
  // split, kG1Splits order), -1 where not timed
  float tune_ms[kNClasses][kNGrid + 2][kNVariants] = {};
  bool tuned = false;
  MlpWeights* mlp = nullptr;  // the plan's own copy of the surrogate (if any request uses it)
  bool serial = false;        // capture the coarse grids one after the other
  cudaStream_t side[kSide] = {nullptr};
  cudaEvent_t fork = nullptr, join[kSide] = {nullptr};
};

extern "C" void marfa_plan_destroy(marfa_plan_t* X) {
  if (!X) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(X->device);
  cudaDeviceSynchronize();
  if (X->exec) cudaGraphExecDestroy(X->exec);
  if (X->graph) cudaGraphDestroy(X->graph);
  for (auto& e : X->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : X->join)
    if (e) cudaEventDestroy(e);
  if (X->fork) cudaEventDestroy(X->fork);
  for (auto& s : X->side)
    if (s) cudaStreamDestroy(s);
  free_work(X->W, 0);
  for (auto& P : X->plans) release(P, 0);
  if (X->mlp) cudaFreeAsync(X->mlp, 0);
  cudaDeviceSynchronize();
  cudaSetDevice(cur);
  delete X;
}

// Time, for each size class present, each grid-1 split and each kernel variant of grids
// 2..10 and of the finest grid on the class's own work (two timed launches after one
// warm-up each) and keep the fastest: chosen[class][kind] as WorkSet::tune.
static int plan_autotune(marfa_plan_t* X, cudaStream_t st, int (*chosen)[kNGrid + 2]) {
  constexpr int NS = 4;  // grid-1 splits tried (kG1Splits)
  WorkSet A[kNVariants], B[NS];
  int all[kNClasses][kNGrid + 2];
  bool present[kNClasses] = {false, false};
  for (auto& P : X->plans) present[P.cls] = true;
  int r = MARFA_OK;
  for (int v = 0; v < kNVariants && !r; ++v) {
    for (int c = 0; c < kNClasses; ++c) {
      for (int g = 2; g <= kNGrid; ++g) all[c][g] = v;
      all[c][1] = kG1Split;
      all[c][kFineKind] = v < kNFineVariants ? v : 0;
    }
    r = build_work(X->plans, all, false, A[v], st);
  }
  for (int k = 0; k < NS && !r; ++k) {
    for (int c = 0; c < kNClasses; ++c) {
      for (int g = 2; g <= kNGrid + 1; ++g) all[c][g] = default_variant(g);
      all[c][1] = kG1Splits[k];
    }
    r = build_work(X->plans, all, false, B[k], st);
  }
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaSuccess;
  if (!r && ((e = cudaEventCreate(&a)) || (e = cudaEventCreate(&b))))
    r = fail(MARFA_E_CUDA, "autotune events: %s", cudaGetErrorString(e));
  for (int c = 0; c < kNClasses; ++c)
    for (int g = 0; g <= kNGrid + 1; ++g)
      for (int v = 0; v < kNVariants; ++v) X->tune_ms[c][g][v] = -1.0f;
  auto time3 = [&](const std::function<void()>& launch, float* out) {
    launch();
    cudaEventRecord(a, st);
    launch();
    launch();
    cudaEventRecord(b, st);
    float ms = 0;
    if ((e = cudaEventSynchronize(b)) || (e = cudaEventElapsedTime(&ms, a, b)))
      return fail(MARFA_E_CUDA, "autotune: %s", cudaGetErrorString(e));
    *out = 0.5f * ms;
    return MARFA_OK;
  };
  auto best_of = [](const float* t, int n) {
    int best = 0;
    for (int v = 1; v < n; ++v)
      if (t[v] < t[best]) best = v;
    return best;
  };
  for (int c = 0; c < kNClasses && !r; ++c) {
    if (!present[c]) {
      for (int k = 1; k <= kNGrid + 1; ++k) chosen[c][k] = k == 1 ? kG1DefaultSplit[c] : default_variant(k);
      continue;
    }
    for (int k = 0; k < NS && !r; ++k) r = time3([&] { launch_grid1(B[k], c, st); }, &X->tune_ms[c][1][k]);
    if (!r) chosen[c][1] = kG1Splits[best_of(X->tune_ms[c][1], NS)];
    for (int g = 2; g <= kNGrid && !r; ++g) {
      for (int v = 0; v < kNVariants && !r; ++v)
        r = time3([&] { launch_grid(A[v], g, c, st); }, &X->tune_ms[c][g][v]);
      if (!r) chosen[c][g] = best_of(X->tune_ms[c][g], kNVariants);
    }
    // the finest grid reads the coarse grids' slots (already filled by the runs above)
    for (int v = 0; v < kNFineVariants && !r; ++v)
      r = time3([&] { launch_finest(A[v], c, st); }, &X->tune_ms[c][kFineKind][v]);
    if (!r) chosen[c][kFineKind] = best_of(X->tune_ms[c][kFineKind], kNFineVariants);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  for (int v = 0; v < kNVariants; ++v) free_work(A[v], st);
  for (int k = 0; k < NS; ++k) free_work(B[k], st);
  X->tuned = !r;
  return r;
}

static int plan_launch_all(marfa_plan_t* X, cudaStream_t st, bool capture) {
  auto rec = [&](int k, cudaStream_t s) {
    if (capture) cudaEventRecordWithFlags(X->ev[k], s, cudaEventRecordExternal);
  };
  const bool branches = capture && !X->serial;
  rec(0, st);
  const WorkSet& W = X->W;
  if (X->plans.size() > 1)  // one launch for all requests (each alone would fill the GPU poorly)
    launch_level_prep_batch(W.dprep, W.dprep_first, (int)X->plans.size(), W.prep_first.back(), st);
  else
    for (auto& P : X->plans) launch_prep(P, st, false);
  rec(1, st);
  // grid g runs on branch stream br[g] (capture) or on st
  cudaStream_t br[kNGrid + 1];
  for (int g = 1; g <= kNGrid; ++g) br[g] = branches ? X->side[(g == 1 ? 0 : 1 + (kNGrid - g)) % kSide] : st;
  if (branches) {
    cudaEventRecord(X->fork, st);
    for (int i = 0; i < kSide; ++i) cudaStreamWaitEvent(X->side[i], X->fork, 0);
  }
  rec(2, br[1]);
  launch_grid1(W, br[1]);
  rec(3, br[1]);
  for (int g = kNGrid; g >= 2; --g) {  // the finer grids carry more work: start them first
    rec(2 * g, br[g]);
    launch_grid(W, g, br[g]);
    rec(2 * g + 1, br[g]);
  }
  if (branches)
    for (int i = 0; i < kSide; ++i) {
      cudaEventRecord(X->join[i], X->side[i]);
      cudaStreamWaitEvent(st, X->join[i], 0);
    }
  rec(2 * (kNGrid + 1), st);
  launch_finest(W, st);
  rec(2 * (kNGrid + 1) + 1, st);
  cudaError_t e = cudaGetLastError();
  if (e) return fail(MARFA_E_CUDA, "plan launches: %s", cudaGetErrorString(e));
  return MARFA_OK;
}

extern "C" int marfa_plan_create(int32_t n_req, const marfa_lines_t* const* lines,
                                 const marfa_level_t* const* levels, const double* const* vmr,
                                 const int32_t* n_levels, const marfa_request_t* rq, float* const* k_out,
                                 int32_t flags, void* stream, marfa_plan_t** out) {
  const bool autotune = flags & MARFA_PLAN_AUTOTUNE;
  if (!out) return fail(MARFA_E_INVAL, "out is NULL");
  *out = nullptr;
  if (flags & ~(MARFA_PLAN_AUTOTUNE | MARFA_PLAN_SERIAL)) return fail(MARFA_E_INVAL, "unknown plan flags");
  if (n_req < 1 || !lines || !levels || !vmr || !n_levels || !rq || !k_out)
    return fail(MARFA_E_INVAL, "bad batch arguments");
  for (int q = 0; q < n_req; ++q)
    if (!k_out[q] || !is_device_ptr(k_out[q]))
      return fail(MARFA_E_INVAL, "k_out[%d] must be device memory for a captured plan", q);
  cudaStream_t st = (cudaStream_t)stream;
  marfa_plan_t* X = alloc_fails() ? nullptr : new (std::nothrow) marfa_plan_t();
  if (!X) return fail(MARFA_E_NOMEM, "host allocation failed");
  cudaGetDevice(&X->device);
  X->serial = flags & MARFA_PLAN_SERIAL;
  X->plans.resize(n_req);
  int r = MARFA_OK;
  for (int q = 0; q < n_req && !r; ++q) r = build_plan(X->plans[q], lines[q], levels[q], vmr[q], n_levels[q], &rq[q], q);
  for (int q = 0; q < n_req && !r; ++q) r = upload(X->plans[q], k_out[q], st);
  // requests with the surrogate use the plan's own copy of its weights and guard, so that
  // the plan does not depend on what is loaded later
  const MlpWeights* src = nullptr;
  for (auto& P : X->plans)
    if (P.rd.mlp) src = P.rd.mlp;
  if (!r && src) {
    r = dev_alloc((void**)&X->mlp, sizeof(MlpWeights), st);
    cudaError_t e2;
    if (!r && (e2 = cudaMemcpyAsync(X->mlp, src, sizeof(MlpWeights), cudaMemcpyDeviceToDevice, st)))
      r = fail(MARFA_E_CUDA, "surrogate copy: %s", cudaGetErrorString(e2));
    for (auto& P : X->plans)
      if (P.rd.mlp) P.rd.mlp = X->mlp;
  }
  int chosen[kNClasses][kNGrid + 2];
  for (int c = 0; c < kNClasses; ++c)
    for (int g = 0; g <= kNGrid + 1; ++g) chosen[c][g] = g == 1 ? kG1DefaultSplit[c] : default_variant(g);
  if (!r && autotune) {
    for (auto& P : X->plans) launch_prep(P, st, false);
    r = plan_autotune(X, st, chosen);
  }
  if (!r) r = build_work(X->plans, chosen, false, X->W, st);
  // with the surrogate: one counted run; grids where its guard never holds for this batch
  // take the plain kernels (same results, without the network's registers and shared
  // memory)
  if (!r && X->W.surr) {
    WorkSet C;
    r = build_work(X->plans, chosen, true, C, st);
    if (!r) {
      for (auto& P : X->plans) launch_prep(P, st, false);
      r = launch_work(C, st, false);
    }
    std::vector<std::vector<int64_t>> cnt(X->plans.size());
    if (!r) r = read_counts(C, X->plans, st, cnt.data());
    if (!r) {
      int64_t per_grid[kNGrid + 2] = {0};
      for (auto& v : cnt)
        for (size_t i = 0; i < v.size() / kCountFields; ++i) per_grid[1 + i % 11] += v[kCountFields * i + 1];
      for (int g = 1; g <= kNGrid + 1; ++g) X->W.surr_grid[g] = per_grid[g] > 0;
    }
    free_work(C, st);
  }
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 * kKinds && !r; ++k)
    if ((e = cudaEventCreate(&X->ev[k]))) r = fail(MARFA_E_CUDA, "plan events: %s", cudaGetErrorString(e));
  if (!r && (e = cudaEventCreateWithFlags(&X->fork, cudaEventDisableTiming)))
    r = fail(MARFA_E_CUDA, "plan events: %s", cudaGetErrorString(e));
  for (int i = 0; i < kSide && !r; ++i)
    if ((e = cudaEventCreateWithFlags(&X->join[i], cudaEventDisableTiming)) ||
        (e = cudaStreamCreateWithFlags(&X->side[i], cudaStreamNonBlocking)))
      r = fail(MARFA_E_CUDA, "plan streams: %s", cudaGetErrorString(e));
  // one ordinary run first: checks every launch outside capture and leaves the output valid
  if (!r) r = plan_launch_all(X, st, false);
  if (!r && (e = cudaStreamSynchronize(st))) r = fail(MARFA_E_CUDA, "plan run: %s", cudaGetErrorString(e));
  if (!r) r = debug_checks();
  cudaStream_t cs = nullptr;
  if (!r && (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)))
    r = fail(MARFA_E_CUDA, "capture stream: %s", cudaGetErrorString(e));
  if (!r) {
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal))) {
      r = fail(MARFA_E_CUDA, "begin capture: %s", cudaGetErrorString(e));
    } else {
      const int r2 = plan_launch_all(X, cs, true);
      e = cudaStreamEndCapture(cs, &X->graph);
      if (r2) r = r2;
      else if (e) r = fail(MARFA_E_CUDA, "end capture: %s", cudaGetErrorString(e));
      else if ((e = cudaGraphInstantiate(&X->exec, X->graph, 0)))
        r = fail(MARFA_E_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
    }
  }
  if (cs) cudaStreamDestroy(cs);
  if (r) {
    marfa_plan_destroy(X);
    return r;
  }
  *out = X;
  return MARFA_OK;
}

extern "C" int marfa_plan_execute(marfa_plan_t* X, void* stream) {
  if (!X || !X->exec) return fail(MARFA_E_INVAL, "plan is NULL");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != X->device) return fail(MARFA_E_INVAL, "plan belongs to device %d, current is %d", X->device, dev);
  CK(cudaGraphLaunch(X->exec, (cudaStream_t)stream));
  return debug_checks();
}

extern "C" int marfa_plan_info(const marfa_plan_t* X, int32_t* variant, float* tune_ms, double* kernel_ms) {
  if (!X) return fail(MARFA_E_INVAL, "plan is NULL");
  const int c = X->plans.empty() ? 0 : X->plans[0].cls;  // the class of request 0
  if (variant)
    for (int g = 1; g <= kFineKind; ++g) variant[g - 1] = g == 1 ? -1 : X->W.tune[c][g];
  if (tune_ms)
    for (int g = 1; g <= kFineKind; ++g)
      for (int v = 0; v < kNVariants; ++v)
        tune_ms[kNVariants * (g - 1) + v] = (X->tuned && g > 1) ? X->tune_ms[c][g][v] : -1.0f;
  if (kernel_ms) {
    for (int k = 0; k < kKinds; ++k) {
      float ms = 0;
      cudaError_t e;
      if ((e = cudaEventSynchronize(X->ev[2 * k + 1])) ||
          (e = cudaEventElapsedTime(&ms, X->ev[2 * k], X->ev[2 * k + 1]))) {
        cudaGetLastError();  // not a sticky error: clear it for later calls
        return fail(MARFA_E_CUDA, "plan kernel times: %s", cudaGetErrorString(e));
      }
      kernel_ms[k] = ms;
    }
  }
  return MARFA_OK;
}

extern "C" int marfa_plan_classes(const marfa_plan_t* X, int32_t* req_class, int32_t* choice, float* tune_ms) {
  if (!X) return fail(MARFA_E_INVAL, "plan is NULL");
  bool present[kNClasses] = {false, false};
  for (size_t q = 0; q < X->plans.size(); ++q) {
    present[X->plans[q].cls] = true;
    if (req_class) req_class[q] = X->plans[q].cls;
  }
  for (int c = 0; c < kNClasses; ++c) {
    if (choice)
      for (int g = 1; g <= kFineKind; ++g) choice[c * kFineKind + g - 1] = present[c] ? X->W.tune[c][g] : -1;
    if (tune_ms)
      for (int g = 1; g <= kFineKind; ++g)
        for (int v = 0; v < kNVariants; ++v)
          tune_ms[(c * kFineKind + g - 1) * kNVariants + v] = (X->tuned && present[c]) ? X->tune_ms[c][g][v] : -1.0f;
  }
  return MARFA_OK;
}

extern "C" int marfa_diag_variants(const int32_t* set, int32_t* get) {
  if (set) {
    for (int g = 2; g <= kFineKind; ++g) {
      const int v = set[g - 1];
      const int nv = g == kFineKind ? kNFineVariants : kNVariants;
      if (v < 0 || v >= nv) return fail(MARFA_E_INVAL, "variant %d of kind %d out of range", v, g);
    }
    for (int g = 2; g <= kFineKind; ++g) g_default_variant[g].store(set[g - 1], std::memory_order_relaxed);
  }
  if (get)
    for (int g = 1; g <= kFineKind; ++g) get[g - 1] = g == 1 ? -1 : default_variant(g);
  return MARFA_OK;
}

// ------------------------------------------------------------------ PT-table (Appendix A)
// One fixed-width numeric field of a .par record: columns [c0, c0 + w) (0-based), blank-
// padded; false when it is empty or not a number.
static bool par_field(const char* rec, int c0, int w, double* v) {
  char buf[32];
  int n = 0;
  for (int i = 0; i < w; ++i) {
    const char ch = rec[c0 + i];
    if (ch != ' ') buf[n++] = ch;
  }
  buf[n] = 0;
  if (n == 0) return false;
  char* end = nullptr;
  *v = std::strtod(buf, &end);
  return end == buf + n && std::isfinite(*v);
}

extern "C" int marfa_read_par(const char* text, int64_t len, marfa_line_t* out, int64_t cap,
                              int64_t* n_out) {
  if (!text || len < 0 || !n_out || cap < 0 || (cap > 0 && !out))
    return fail(MARFA_E_INVAL, "bad arguments");
  // pass 1 counts and checks the records, pass 2 writes them
  for (int pass = 0; pass < 2; ++pass) {
    int64_t n = 0, line_no = 0;
    for (int64_t pos = 0; pos < len;) {
      int64_t end = pos;
      while (end < len && text[end] != '\n') ++end;
      const int64_t next = end + 1;
      int64_t e = end;
      if (e > pos && text[e - 1] == '\r') --e;
      ++line_no;
      bool blank = true;
      for (int64_t i = pos; i < e && blank; ++i) blank = text[i] == ' ' || text[i] == '\t';
      if (!blank) {
        if (e - pos < 67) return fail(MARFA_E_INVAL, "line %lld: shorter than 67 columns", (long long)line_no);
        const char* rec = text + pos;
        double mol, nu, S, ga, gs, E, na, da;
        const char ic = rec[2];
        int iso = -1;
        if (ic >= '1' && ic <= '9') iso = ic - '0';
        else if (ic == '0') iso = 10;
        else if (ic >= 'A' && ic <= 'Z') iso = 11 + (ic - 'A');
        if (!par_field(rec, 0, 2, &mol) || mol < 1 || mol > 999 || mol != std::floor(mol) || iso < 0 ||
            !par_field(rec, 3, 12, &nu) || !par_field(rec, 15, 10, &S) || !par_field(rec, 35, 5, &ga) ||
            !par_field(rec, 40, 5, &gs) || !par_field(rec, 45, 10, &E) || !par_field(rec, 55, 4, &na) ||
            !par_field(rec, 59, 8, &da))
          return fail(MARFA_E_INVAL, "line %lld: malformed .par record", (long long)line_no);
        if (pass == 1) {
          marfa_line_t& L = out[n];
          L.nu0 = nu;
          L.S296 = (float)S;
          L.gamma_air = (float)ga;
          L.gamma_self = (float)gs;
          L.E_lower = (float)E;
          L.n_air = (float)na;
          L.mol_iso = 100 * (int32_t)mol + iso;
          L.delta_air = (float)da;
        }
        ++n;
      }
      pos = next;
    }
    if (pass == 0) {
      *n_out = n;
      if (cap == 0 && !out) return MARFA_OK;
      if (cap < n) return fail(MARFA_E_INVAL, "room for %lld records, the text holds %lld", (long long)cap,
                               (long long)n);
    }
  }
  return MARFA_OK;
}

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
// other streams run) use marfa_absorption_noalloc. Its scratch is g_noalloc_scratch:
// every GPU on which marfa_prepare_lines has run holds it until the process exits.
extern "C" int marfa_absorption_noalloc(const marfa_lines_t* lines, const marfa_level_t* levels,
                                        const double* vmr, int32_t n_levels,
                                        const marfa_request_t* rq, float* k_out, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  // The level tables and work lists are copied from this call's own host memory, which
  // is gone when it returns: a stream in capture would record copies of freed memory.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(MARFA_E_INVAL, "marfa_absorption_noalloc refuses a stream in capture (use marfa_plan_* for graphs)");
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
  int var[kNGrid + 2];  // the default kernel variants, read once
  for (int g = 0; g <= kNGrid + 1; ++g) var[g] = default_variant(g);
  std::vector<CoarseItem> coarse;  // grids 2..10 in order
  for (int g = 2; g <= kNGrid; ++g) coarse_items(P, g, var[g], coarse);
  std::vector<G1Item> g1items;  // grid 1 with kG1Split parts (R.g1_split), the finest grid
  std::vector<FineItem> fine;
  expand_on_host(plan_desc(P, 1, kG1Split), g1items);
  expand_on_host(plan_desc(P, kNGrid + 1, 0), fine);
  const size_t sz_r = al(sizeof(ReqDev)), sz_gi = al(sizeof(G1Item) * g1items.size()),
               sz_ci = al(sizeof(CoarseItem) * coarse.size()), sz_fi = al(sizeof(FineItem) * fine.size());
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
  CK(cudaMemcpyAsync(dgi, g1items.data(), sizeof(G1Item) * g1items.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dci, coarse.data(), sizeof(CoarseItem) * coarse.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dfi, fine.data(), sizeof(FineItem) * fine.size(), cudaMemcpyHostToDevice, st));
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
  const bool surr = R.mlp != nullptr;
  const bool wide = P.rd.wide != 0;
  launch_g1(drd, dgi, (int)g1items.size(), nullptr, surr, wide, st);
  size_t k = 0;
  for (int g = 2; g <= kNGrid; ++g) {  // coarse is ordered by grid
    size_t k1 = k;
    while (k1 < coarse.size() && coarse[k1].grid == g) ++k1;
    const int v = var[g];
    if ((v == 4 || v == 5) && !surr && !wide && ((R.mech >> g) & 1))
      launch_coarse_mech(drd, dci + k, (int)(k1 - k), nullptr, v == 5, st);
    else if (v == 3 && !surr)
      launch_coarse_jobs(drd, dci + k, (int)(k1 - k), nullptr, wide, st);
    else if (v == 1 || v >= 3)
      launch_coarse(drd, dci + k, (int)(k1 - k), nullptr, surr, wide, st);
    else
      launch_coarse_lm(drd, dci + k, (int)(k1 - k), nullptr, surr, v == 2 ? 16 : kLPairs, wide, st);
    k = k1;
  }
  if (var[kFineKind] >= 1 && !surr) {
    const bool mech = var[kFineKind] >= 2 && !wide && ((R.mech >> (kNGrid + 1)) & 1);
    const bool merge = var[kFineKind] == 3 && ((R.mech >> (kNGrid + 2)) & 1);
    launch_fine_jobs(drd, dfi, (int)fine.size(), nullptr, wide, mech ? (merge ? 2 : 1) : 0, st);
  }
  else
    launch_fine(drd, dfi, (int)fine.size(), nullptr, surr, wide, st);
  CK(cudaGetLastError());
  return debug_checks();
}

extern "C" int marfa_diag_check(int32_t index, int32_t* debug_build) {
  if (debug_build) *debug_build = kDebugBuild ? 1 : 0;
  launch_diag_check(index, 0);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  return debug_checks();
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

extern "C" int marfa_diag_pipe_rate(int32_t pipe, double* ops_per_s) {
  if (pipe < 0 || pipe > 3 || !ops_per_s) return fail(MARFA_E_INVAL, "pipe must be 0..3 and ops_per_s non-NULL");
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * nsm;  // 2048 threads on every SM
  const int iters = pipe == 0 ? 8192 : 1024;
  const int reps = 5;
  float* out = nullptr;
  CK(cudaMalloc(&out, (size_t)blocks * 256 * sizeof(float)));
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (!e) e = cudaEventCreate(&ev[1]);
  int64_t n = 0;
  float ms = 0.0f;
  if (!e) {
    launch_diag_pipe(pipe, out, blocks, iters, 0);  // warm-up
    e = cudaEventRecord(ev[0], 0);
    for (int r = 0; r < reps && !e; ++r) n += launch_diag_pipe(pipe, out, blocks, iters, 0);
    if (!e) e = cudaEventRecord(ev[1], 0);
    if (!e) e = cudaEventSynchronize(ev[1]);
    if (!e) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (!e) e = cudaGetLastError();
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  cudaFree(out);
  if (e) return fail(MARFA_E_CUDA, "pipe probe: %s", cudaGetErrorString(e));
  if (!(ms > 0.0f)) return fail(MARFA_E_CUDA, "pipe probe: no elapsed time");
  *ops_per_s = (double)n / (ms * 1e-3);
  return MARFA_OK;
}

extern "C" int marfa_diag_shape(int32_t shape, const float* x, const float* y, float* out, int64_t n) {
  if (!(shape == MARFA_SHAPE_LORENTZ || shape == MARFA_SHAPE_VOIGT || shape == MARFA_SHAPE_DOPPLER ||
        shape == MARFA_SHAPE_VOIGT_PAPER || shape == MARFA_SHAPE_USER || shape == MARFA_SHAPE_TEST_CONST ||
        shape == MARFA_SHAPE_TEST_QUAD || shape == MARFA_SHAPE_TEST_QUART))
    return fail(MARFA_E_INVAL, "unknown shape %d", shape);
  if (shape == MARFA_SHAPE_USER && !user_shape_set_here())
    return fail(MARFA_E_INVAL, "no user shape is set on this device");
  if (n < 0 || (n > 0 && (!x || !y || !out))) return fail(MARFA_E_INVAL, "bad arguments");
  if (n == 0) return MARFA_OK;
  float* dx;
  CK(cudaMalloc(&dx, 12 * (size_t)n));
  float *dy = dx + n, *dz = dy + n;
  cudaError_t e;
  if ((e = cudaMemcpy(dx, x, 4 * n, cudaMemcpyHostToDevice)) || (e = cudaMemcpy(dy, y, 4 * n, cudaMemcpyHostToDevice))) {
    cudaFree(dx);
    return fail(MARFA_E_CUDA, "copy failed: %s", cudaGetErrorString(e));
  }
  launch_diag_shape(shape, dx, dy, dz, n, 0);
  e = cudaMemcpy(out, dz, 4 * n, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  if (e) return fail(MARFA_E_CUDA, "shape kernel: %s", cudaGetErrorString(e));
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

extern "C" int marfa_diag_absorption_counts(const marfa_lines_t* lines, const marfa_level_t* levels,
                                            const double* vmr, int32_t n_levels, const marfa_request_t* rq,
                                            float* k_out, int64_t* counts) {
  if (!counts) return fail(MARFA_E_INVAL, "counts is NULL");
  std::vector<int64_t> cc[1];
  float* outs[1] = {k_out};
  int r = absorption_impl(1, &lines, &levels, &vmr, &n_levels, rq, outs, 0, cc);
  if (r) return r;
  std::copy(cc[0].begin(), cc[0].end(), counts);
  CK(cudaDeviceSynchronize());
  return MARFA_OK;
}

extern "C" int marfa_diag_absorption_counted(const marfa_lines_t* lines, const marfa_level_t* levels,
                                             const double* vmr, int32_t n_levels,
                                             const marfa_request_t* rq, float* k_out, int64_t* counts) {
  if (!counts) return fail(MARFA_E_INVAL, "counts is NULL");
  if (n_levels < 1 || n_levels > 65535) return fail(MARFA_E_INVAL, "need 1..65535 levels");
  std::vector<int64_t> c5((size_t)n_levels * 11 * kCountFields);
  int r = marfa_diag_absorption_counts(lines, levels, vmr, n_levels, rq, k_out, c5.data());
  if (r) return r;
  for (size_t i = 0; i < (size_t)n_levels * 11; ++i) counts[i] = c5[kCountFields * i];
  return MARFA_OK;
}

extern "C" int marfa_diag_absorption_counted_surrogate(const marfa_lines_t* lines,
                                                       const marfa_level_t* levels, const double* vmr,
                                                       int32_t n_levels, const marfa_request_t* rq,
                                                       float* k_out, int64_t* counts,
                                                       int64_t* surrogate_counts) {
  if (!counts || !surrogate_counts) return fail(MARFA_E_INVAL, "counts is NULL");
  if (n_levels < 1 || n_levels > 65535) return fail(MARFA_E_INVAL, "need 1..65535 levels");
  std::vector<int64_t> c5((size_t)n_levels * 11 * kCountFields);
  int r = marfa_diag_absorption_counts(lines, levels, vmr, n_levels, rq, k_out, c5.data());
  if (r) return r;
  for (size_t i = 0; i < (size_t)n_levels * 11; ++i) {
    counts[i] = c5[kCountFields * i];
    surrogate_counts[i] = c5[kCountFields * i + 1];
  }
  return MARFA_OK;
}

// ------------------------------------------------------------------ surrogate: training
namespace {
// Device buffers of one training or gradient call, freed on every exit path.
struct MlpBufs {
  float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *part = nullptr, *lp = nullptr;
  float *x = nullptr, *y = nullptr, *t = nullptr, *loss = nullptr;
  ~MlpBufs() {
    for (float* q : {p, m, v, g, part, lp, x, y, t, loss})
      if (q) cudaFree(q);
  }
};
}  // namespace

static int mlp_check_samples(const float* x, const float* y, const float* t, int64_t n) {
  if (!x || !y || !t || n < 1) return fail(MARFA_E_INVAL, "need n >= 1 samples (x, y, t)");
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i]) || !(y[i] > 0) || !std::isfinite(y[i]) || !std::isfinite(t[i]))
      return fail(MARFA_E_INVAL, "sample %lld: x, t must be finite and y finite and > 0", (long long)i);
  return MARFA_OK;
}

static int mlp_upload(MlpBufs& B, const float* params, const float* x, const float* y, const float* t,
                      int64_t n, int max_batch) {
  const int tile = mlp_train_tile();
  const int nblk = (max_batch + tile - 1) / tile;
  cudaError_t e;
  if ((e = cudaMalloc(&B.p, 4 * kMlpParams)) || (e = cudaMalloc(&B.m, 4 * kMlpParams)) ||
      (e = cudaMalloc(&B.v, 4 * kMlpParams)) || (e = cudaMalloc(&B.g, 4 * kMlpParams)) ||
      (e = cudaMalloc(&B.part, 4 * (size_t)nblk * kMlpParams)) ||
      (e = cudaMalloc(&B.lp, 4 * (size_t)nblk * tile)) || (e = cudaMalloc(&B.x, 4 * (size_t)n)) ||
      (e = cudaMalloc(&B.y, 4 * (size_t)n)) || (e = cudaMalloc(&B.t, 4 * (size_t)n)))
    return fail(MARFA_E_NOMEM, "surrogate training buffers: %s", cudaGetErrorString(e));
  if ((e = cudaMemcpy(B.p, params, 4 * kMlpParams, cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(B.m, 0, 4 * kMlpParams)) || (e = cudaMemset(B.v, 0, 4 * kMlpParams)) ||
      (e = cudaMemcpy(B.x, x, 4 * (size_t)n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(B.y, y, 4 * (size_t)n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(B.t, t, 4 * (size_t)n, cudaMemcpyHostToDevice)))
    return fail(MARFA_E_CUDA, "surrogate upload: %s", cudaGetErrorString(e));
  return MARFA_OK;
}

extern "C" int marfa_mlp_loss_grad(const float* params, const float* x, const float* y, const float* t,
                                   int64_t n, int32_t qat, double* loss, float* grad) {
  if (!params || !loss || !grad) return fail(MARFA_E_INVAL, "params, loss and grad must not be NULL");
  if (n > MARFA_MLP_MAX_BATCH) return fail(MARFA_E_INVAL, "at most %d samples", MARFA_MLP_MAX_BATCH);
  int r = mlp_check_samples(x, y, t, n);
  if (r) return r;
  MlpBufs B;
  r = mlp_upload(B, params, x, y, t, n, (int)n);
  if (r) return r;
  const int tile = mlp_train_tile();
  const int nblk = (int)((n + tile - 1) / tile);
  launch_mlp_fwd_bwd(B.p, B.x, B.y, B.t, n, 0, nblk, (float)(1.0 / (double)n), qat != 0, B.part, B.lp, 0);
  launch_mlp_reduce(B.part, nblk, B.g, 0);
  CK(cudaGetLastError());
  std::vector<float> lp((size_t)nblk * tile);
  cudaError_t e;
  if ((e = cudaMemcpy(grad, B.g, 4 * kMlpParams, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(lp.data(), B.lp, 4 * lp.size(), cudaMemcpyDeviceToHost)))
    return fail(MARFA_E_CUDA, "surrogate gradient: %s", cudaGetErrorString(e));
  double sum = 0.0;
  for (int64_t i = 0; i < n; ++i) sum += lp[(size_t)i];
  *loss = sum / (double)n;
  return MARFA_OK;
}

extern "C" int marfa_mlp_train(float* params, const float* x, const float* y, const float* t, int64_t n,
                               const marfa_mlp_train_t* cfg, float* loss_curve) {
  if (!params || !cfg) return fail(MARFA_E_INVAL, "params and cfg must not be NULL");
  if (cfg->steps < 1 || cfg->batch < 1 || cfg->batch > MARFA_MLP_MAX_BATCH)
    return fail(MARFA_E_INVAL, "need steps >= 1 and 1 <= batch <= %d", MARFA_MLP_MAX_BATCH);
  if (!(cfg->lr0 > 0) || !(cfg->lr1 > 0) || !std::isfinite(cfg->lr0) || !std::isfinite(cfg->lr1))
    return fail(MARFA_E_INVAL, "learning rates must be finite and > 0");
  for (int i = 0; i < kMlpParams; ++i)
    if (!std::isfinite(params[i])) return fail(MARFA_E_INVAL, "parameter %d is not finite", i);
  int r = mlp_check_samples(x, y, t, n);
  if (r) return r;
  MlpBufs B;
  r = mlp_upload(B, params, x, y, t, n, cfg->batch);
  if (r) return r;
  cudaError_t e;
  if ((e = cudaMalloc(&B.loss, 4 * (size_t)cfg->steps)))
    return fail(MARFA_E_NOMEM, "loss curve: %s", cudaGetErrorString(e));
  const int tile = mlp_train_tile();
  const double kPi = 3.14159265358979323846;
  double b1t = 1.0, b2t = 1.0;
  int64_t first = 0;
  for (int k = 0; k < cfg->steps; ++k) {
    const int64_t nb = std::min<int64_t>(cfg->batch, n - first);
    const int nblk = (int)((nb + tile - 1) / tile);
    const double lr = cfg->lr1 + 0.5 * (cfg->lr0 - cfg->lr1) * (1.0 + std::cos(kPi * k / cfg->steps));
    b1t *= 0.9;
    b2t *= 0.999;
    launch_mlp_fwd_bwd(B.p, B.x, B.y, B.t, first + nb, first, nblk, (float)(1.0 / (double)nb), cfg->qat != 0,
                       B.part, B.lp, 0);
    launch_mlp_reduce(B.part, nblk, B.g, 0);
    launch_mlp_adam(B.p, B.g, B.m, B.v, (float)lr, (float)b1t, (float)b2t, 0);
    launch_mlp_loss_sum(B.lp, nblk * tile, (float)(1.0 / (double)nb), B.loss + k, 0);
    first += nb;
    if (first >= n) first = 0;
  }
  CK(cudaGetLastError());
  if ((e = cudaMemcpy(params, B.p, 4 * kMlpParams, cudaMemcpyDeviceToHost)) ||
      (loss_curve && (e = cudaMemcpy(loss_curve, B.loss, 4 * (size_t)cfg->steps, cudaMemcpyDeviceToHost))))
    return fail(MARFA_E_CUDA, "surrogate training: %s", cudaGetErrorString(e));
  return MARFA_OK;
}

// ------------------------------------------------------------------ surrogate: inference
extern "C" int marfa_surrogate_load(const float* params, float budget, int32_t samples,
                                    int32_t* cells_on, float* cell_err) {
  if (!params) return fail(MARFA_E_INVAL, "params must not be NULL");
  if (!(budget > 0) || !(budget < 1)) return fail(MARFA_E_INVAL, "budget must be in (0, 1)");
  if (samples < 2 || samples > 64) return fail(MARFA_E_INVAL, "samples must be in 2..64");
  for (int i = 0; i < kMlpParams; ++i)
    if (!std::isfinite(params[i])) return fail(MARFA_E_INVAL, "parameter %d is not finite", i);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_surr_mu);
  if (g_surr_w) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g_surr_dev);
    cudaFree(g_surr_w);
    cudaSetDevice(cur);
    g_surr_w = nullptr;
    g_surr_dev = -1;
  }
  MlpWeights* w = nullptr;
  float *dp = nullptr, *derr = nullptr;
  const int cells = kGuardNx * kGuardNy;
  cudaError_t e;
  if ((e = alloc_fails() ? cudaErrorMemoryAllocation : cudaMalloc(&w, sizeof(MlpWeights))) ||
      (e = cudaMalloc(&dp, 4 * kMlpParams)) || (e = cudaMalloc(&derr, 4 * cells))) {
    cudaFree(w);
    cudaFree(dp);
    cudaFree(derr);
    return fail(MARFA_E_NOMEM, "surrogate weights: %s", cudaGetErrorString(e));
  }
  std::vector<uint32_t> bits(kGuardWords);
  std::vector<float> err(cells);
  if (!(e = cudaMemcpy(dp, params, 4 * kMlpParams, cudaMemcpyHostToDevice))) {
    launch_mlp_pack(dp, w, 0);
    launch_mlp_guard(w, budget, samples, derr, 0);
    if (!(e = cudaGetLastError()) &&
        !(e = cudaMemcpy(bits.data(), (const char*)w + offsetof(MlpWeights, guard), 4 * kGuardWords,
                         cudaMemcpyDeviceToHost)))
      e = cudaMemcpy(err.data(), derr, 4 * cells, cudaMemcpyDeviceToHost);
  }
  cudaFree(dp);
  cudaFree(derr);
  if (e) {
    cudaFree(w);
    return fail(MARFA_E_CUDA, "surrogate load: %s", cudaGetErrorString(e));
  }
  int on = 0;
  for (uint32_t b : bits) on += __builtin_popcount(b);
  if (cells_on) *cells_on = on;
  if (cell_err) std::copy(err.begin(), err.end(), cell_err);
  g_surr_w = w;
  g_surr_dev = dev;
  return MARFA_OK;
}

extern "C" int marfa_surrogate_unload(void) {
  std::lock_guard<std::mutex> lk(g_surr_mu);
  if (g_surr_w) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g_surr_dev);
    cudaError_t e = cudaFree(g_surr_w);
    cudaSetDevice(cur);
    g_surr_w = nullptr;
    g_surr_dev = -1;
    if (e) return fail(MARFA_E_CUDA, "surrogate unload: %s", cudaGetErrorString(e));
  }
  return MARFA_OK;
}

extern "C" int marfa_surrogate_eval(const float* x, const float* y, float* out, int64_t n, int32_t guarded) {
  if (n < 0 || (n > 0 && (!x || !y || !out))) return fail(MARFA_E_INVAL, "bad arguments");
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i]) || !(y[i] > 0) || !std::isfinite(y[i]))
      return fail(MARFA_E_INVAL, "point %lld: x must be finite and y finite and > 0", (long long)i);
  const MlpWeights* w = nullptr;
  int r = surrogate_for_current_device(&w);
  if (r) return r;
  if (n == 0) return MARFA_OK;
  float* d = nullptr;
  CK(cudaMalloc(&d, 12 * (size_t)n));
  cudaError_t e;
  if (!(e = cudaMemcpy(d, x, 4 * (size_t)n, cudaMemcpyHostToDevice)) &&
      !(e = cudaMemcpy(d + n, y, 4 * (size_t)n, cudaMemcpyHostToDevice))) {
    launch_mlp_eval(w, d, d + n, d + 2 * n, n, guarded != 0, 0);
    if (!(e = cudaGetLastError())) e = cudaMemcpy(out, d + 2 * n, 4 * (size_t)n, cudaMemcpyDeviceToHost);
  }
  cudaFree(d);
  if (e) return fail(MARFA_E_CUDA, "surrogate eval: %s", cudaGetErrorString(e));
  return MARFA_OK;
}

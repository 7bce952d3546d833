// Host check of the two forms of panel ownership in csrc/ownership.cuh: wherever the
// 32-bit panel frame applies (PanelFrame::ok) its masks must equal those of the 64-bit
// fixed-point form, bit for bit. Built and run by tests/test_ownership_cpu.py; prints
// "cases <n> frames_ok <k> mismatches <m>" and exits 1 on any mismatch.
#include <cstdint>
#include <cstdio>
#include "ownership.cuh"

using namespace marfa;

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static int64_t uniform(int64_t lo, int64_t hi) { return lo + (int64_t)(next_u64() % (uint64_t)(hi - lo + 1)); }

template <typename MT>
static long check(int g, int64_t base, int nb, int64_t cut, int R_w, int64_t c, int gst, bool chi, bool& ok) {
  PanelFrame F;
  F.init(g, base, nb, cut, R_w);
  ok = F.ok;
  if (!F.ok) return 0;
  const PanelPos p = F.pos(c);
  long bad = 0;
  const MT a64 = accept_mask<MT>(g, c, gst, chi, cut, R_w, base, nb, false);
  const MT a32 = accept_frame<MT>(F, p, g, gst, chi);
  const MT b64 = accept_mask<MT>(g - 1, c, gst, chi, cut, R_w, base, nb, true);
  const MT b32 = accept_parent_frame<MT>(F, p, g, gst, chi);
  const int s = panel_shift(g);
  const bool n64 = owns_nothing(g, c, gst, chi, cut, base << s, (base + nb) << s, int64_t(1) << s);
  const bool n32 = owns_nothing_frame(F, p, g, gst, chi);
  if (a64 != a32) ++bad;
  if (b64 != b32) ++bad;
  if (n64 != n32) ++bad;
  if (bad && bad < 1000000)
    fprintf(stderr, "g %d base %lld nb %d cut %lld R_w %d c %lld gst %d chi %d: %llx/%llx %llx/%llx %d/%d\n", g,
            (long long)base, nb, (long long)cut, R_w, (long long)c, gst, (int)chi, (unsigned long long)a64,
            (unsigned long long)a32, (unsigned long long)b64, (unsigned long long)b32, (int)n64, (int)n32);
  return bad;
}

int main() {
  const int64_t one = int64_t(1) << kFixBits;  // 1 cm^-1
  const int64_t cuts[] = {25 * one, 125 * one, 5 * one / 2, 125 * one + one / 3, 400 * one};
  const int Rws[] = {8, 6, 4, 2, 7};
  long cases = 0, okc = 0, bad = 0;
  for (int rep = 0; rep < 400000; ++rep) {
    const int g = (int)uniform(2, 10);
    const int s = panel_shift(g);
    const int64_t P = int64_t(1) << s;
    const int64_t cut = cuts[uniform(0, 4)];
    const int R_w = Rws[uniform(0, 4)];
    const int kind = (int)uniform(0, 2);
    const int nb = kind == 0 ? 17 : (kind == 1 ? 33 : 16);
    // tile near 500..3000 cm^-1, either parity of base
    const int64_t base = fl_sh(uniform(500, 3000) * one, s) + uniform(-3, 3);
    // centre: near the tile, or at a cut-off / breakpoint / core distance from its ends
    const int64_t span = (int64_t)nb * P;
    int64_t off;
    switch ((int)uniform(0, 4)) {
      case 0: off = uniform(-4 * P, span + 4 * P); break;
      case 1: off = (uniform(0, 1) ? -cut : cut) + uniform(-3, nb + 3) * P; break;
      case 2: off = (uniform(0, 1) ? -1 : 1) * chi_break_fx((int)uniform(0, 2)) + uniform(-3, nb + 3) * P; break;
      case 3: off = uniform(-R_w - 2, nb + R_w + 2) * (P / 2); break;
      default: off = uniform(-cut - 2 * span, cut + 2 * span); break;
    }
    // land exactly on a panel end (and one unit beside it) often
    const int jit = (int)uniform(0, 3);
    if (jit == 0) off = (off >> s) << s;
    if (jit == 1) off = ((off >> s) << s) + (uniform(0, 1) ? 1 : -1);
    const int64_t c = (base << s) + off;
    const int gst = (int)uniform(1, 11);
    const bool chi = uniform(0, 1) != 0;
    bool ok = false;
    if (nb > 32)
      bad += check<uint64_t>(g, base, nb, cut, R_w, c, gst, chi, ok);
    else
      bad += check<uint32_t>(g, base, nb, cut, R_w, c, gst, chi, ok);
    ++cases;
    okc += ok;
  }
  printf("cases %ld frames_ok %ld mismatches %ld\n", cases, okc, bad);
  return bad ? 1 : 0;
}

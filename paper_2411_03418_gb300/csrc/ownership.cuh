// Exact panel ownership of a line on the coarse grids (rule R2 of Sec. 2.4 as read in
// the oracle): which panels of grid g a line's profile is accumulated on, from its
// fixed-point centre c, its core grid g*, the cut-off and the chi-factor breakpoints.
// Host and device code, so that tests can compare the two forms on the CPU.
//
// Two forms give identical masks:
//  * accept_mask / owns_nothing work on 64-bit fixed-point positions;
//  * the PanelFrame forms work on 32-bit panel indices relative to the tile. They hold
//    when the cut-off, R_w h_g, R_w h_(g-1) and the breakpoints within the cut-off are
//    whole panels of grids g and g - 1 (PanelFrame::ok; true for whole-cm^-1 cut-offs,
//    even R_w and g >= 3): then floor((c + o) / P) = floor(c / P) + o / P and
//    ceil((c + o) / P) = floor(c / P) + o / P + [c not a multiple of P].
#pragma once
#include <cstdint>
#include "marfa_internal.cuh"

#define MARFA_HD __host__ __device__ __forceinline__

namespace marfa {

// chi-factor breakpoints of Eq. (10): 3, 150 and 300 cm^-1, fixed point
MARFA_HD constexpr int64_t chi_break_fx(int b) {
  return b == 0 ? (int64_t(3) << kFixBits) : (b == 1 ? (int64_t(150) << kFixBits) : (int64_t(300) << kFixBits));
}

// Bits i = 0..nb-1 stand for panels base + i; set those in the closed interval [a, b].
template <typename MT>
MARFA_HD MT rmask(int64_t a, int64_t b, int64_t base, int nb) {
  int64_t lo = a - base;
  int64_t hi = b - base;
  if (lo < 0) lo = 0;
  if (hi > nb - 1) hi = nb - 1;
  if (lo > hi) return MT(0);
  return ((MT(2) << (int)hi) - MT(1)) & (~MT(0) << (int)lo);
}

// The same with a and b already relative to base.
template <typename MT>
MARFA_HD MT rmask_rel(int lo, int hi, int nb) {
  if (lo < 0) lo = 0;
  if (hi > nb - 1) hi = nb - 1;
  if (lo > hi) return MT(0);
  return ((MT(2) << hi) - MT(1)) & (~MT(0) << lo);
}

// Panels of grid g accepted for a line: the acceptance panels are 2^s fixed-point units
// wide (s = panel_shift(g): two steps of grid g; one more for the 5-point variant's four
// steps), and each is mapped onto the mask bits, panels of 2^sb units (sb <= s) over
// [base, base + nb): acceptance panel a covers bits a f .. a f + f - 1, f = 2^(s - sb).
template <typename MT>
MARFA_HD MT accept_mask_s(int g, int64_t c, int gst, bool chi, int64_t cut, int R_w, int64_t base, int nb,
                          int s, int sb) {
  const int64_t f = int64_t(1) << (s - sb), k = f - 1;
  int64_t s_lo = cl_sh(c - cut, s), s_hi = fl_sh(c + cut, s) - 1;
  MT m = rmask<MT>(s_lo * f, s_hi * f + k, base, nb);
  if (!m) return MT(0);
  // the span covered by the mask bits, in fixed point
  const int64_t xa = base << sb, xb = (base + nb) << sb;
  const int64_t P = int64_t(1) << s;  // acceptance panel width: a gap or kink panel lies
                                      // within one panel width of c +- R or c +- B
  if (gst > g) {
    const int64_t R = (int64_t)R_w * step_fx(g);
    if (c + R + P >= xa && c - R - P <= xb) {
      int64_t gl = fl_sh(c - R, s), gh = cl_sh(c + R, s) - 1;
      m &= ~rmask<MT>(gl * f, gh * f + k, base, nb);
    }
  }
  if (chi) {
    // a panel holding a breakpoint beyond the cut-off already fails the support test
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int64_t B = chi_break_fx(b);
      if (B > cut) break;
      const int64_t s1 = c - B, s2 = c + B;
      if (s1 >= xa - P && s1 <= xb + P)
        m &= ~rmask<MT>((cl_sh(s1, s) - 1) * f, fl_sh(s1, s) * f + k, base, nb);
      if (s2 >= xa - P && s2 <= xb + P)
        m &= ~rmask<MT>((cl_sh(s2, s) - 1) * f, fl_sh(s2, s) * f + k, base, nb);
    }
  }
  return m;
}

// Panels of grid g accepted for a line, over panels [base, base + nb). With child set,
// the accepted panels of grid g are mapped to their two children on grid g + 1 and
// base/nb refer to grid g + 1.
template <typename MT>
MARFA_HD MT accept_mask(int g, int64_t c, int gst, bool chi, int64_t cut, int R_w, int64_t base, int nb,
                        bool child) {
  const int s = panel_shift(g);
  return accept_mask_s<MT>(g, c, gst, chi, cut, R_w, base, nb, s, child ? s - 1 : s);
}

// Panels of grid g (2..10) a line owns over the two-step panels [base, base + nb): the
// panels grid g accepts and its parent grid does not; wide selects the 5-point variant
// (acceptance on four-step panels). One code path for both: the shifts are arguments.
template <typename MT>
MARFA_HD MT owned_any(bool wide, int g, int64_t c, int gst, bool chi, int64_t cut, int R_w, int64_t base,
                      int nb) {
  const int sb = panel_shift(g), w = wide ? 1 : 0;
  MT m = accept_mask_s<MT>(g, c, gst, chi, cut, R_w, base, nb, sb + w, sb);
  if (m) m &= ~accept_mask_s<MT>(g - 1, c, gst, chi, cut, R_w, base, nb, sb + 1 + w, sb);
  return m;
}

// Quick rejection for grids 2..10: with its core on a coarser grid (gst < g) a line
// owns panels of grid g only where the parent panel holds its cut-off edge or a chi
// breakpoint, i.e. within one panel width P of the child; if no edge or breakpoint lies
// within P of the span [xa, xb] of the tile's panels, the line owns nothing there.
MARFA_HD bool owns_nothing(int g, int64_t c, int gst, bool chi, int64_t cut, int64_t xa, int64_t xb,
                           int64_t P) {
  if (gst >= g) return false;
  const int64_t lo = xa - P, hi = xb + P;
  if ((c - cut >= lo && c - cut <= hi) || (c + cut >= lo && c + cut <= hi)) return false;
  if (chi) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int64_t B = chi_break_fx(b);
      if (B > cut) break;
      if ((c - B >= lo && c - B <= hi) || (c + B >= lo && c + B <= hi)) return false;
    }
  }
  return true;
}

// ------------------------------------------------------------------ 32-bit panel frame
// A line centre against a tile's panel frame: q0 = floor(c / P) - base and r0 = [P does
// not divide c] for the panels P of grid g; q1, r1 the same for the parent grid's
// panels 2P, relative to floor(base / 2).
struct PanelPos {
  int q0, r0, q1, r1;
};

// The tile's panels base .. base + nb - 1 of grid g (2..10) and the offsets in whole
// panels; ok = false when an offset is not a whole panel (use the 64-bit form then).
struct PanelFrame {
  int s;            // panel shift of grid g
  int64_t base;
  int nb;
  int e;            // base - 2 floor(base / 2)
  int cut0, cut1;   // cut-off in panels of grid g, of grid g - 1
  int R0, R1;       // R_w h_g in panels of grid g, R_w h_(g-1) in panels of grid g - 1
  int nB;           // breakpoints within the cut-off
  int B0[3], B1[3]; // those breakpoints in panels of grid g, of grid g - 1
  bool ok;

  MARFA_HD void init(int g, int64_t base_, int nb_, int64_t cut, int R_w) {
    s = panel_shift(g);
    base = base_;
    nb = nb_;
    e = (int)(base - 2 * fl_sh(base, 1));
    const int64_t P = int64_t(1) << s, P1 = P << 1;
    const int64_t Rg = (int64_t)R_w * step_fx(g), Rg1 = (int64_t)R_w * step_fx(g - 1);
    ok = g >= 2 && cut >= 0 && cut % P1 == 0 && Rg % P == 0 && Rg1 % P1 == 0 &&
         (cut >> s) < (int64_t(1) << 24) && (Rg1 >> s) < (int64_t(1) << 24);
    cut0 = (int)(cut >> s);
    cut1 = (int)(cut >> (s + 1));
    R0 = (int)(Rg >> s);
    R1 = (int)(Rg1 >> (s + 1));
    nB = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int64_t B = chi_break_fx(b);
      B0[b] = B1[b] = 0;
      if (B > cut) continue;
      if (B % P1 != 0) ok = false;
      B0[b] = (int)(B >> s);
      B1[b] = (int)(B >> (s + 1));
      nB = b + 1;
    }
  }
  // c must lie within 2^30 panels of the tile
  MARFA_HD PanelPos pos(int64_t c) const {
    PanelPos p;
    p.q0 = (int)(fl_sh(c, s) - base);
    p.r0 = (c & ((int64_t(1) << s) - 1)) != 0;
    p.q1 = (int)(fl_sh(c, s + 1) - fl_sh(base, 1));
    p.r1 = (c & ((int64_t(1) << (s + 1)) - 1)) != 0;
    return p;
  }
};

// accept_mask(g, ...) over the frame's panels, from the frame (ok) and the line's PanelPos.
template <typename MT>
MARFA_HD MT accept_frame(const PanelFrame& F, const PanelPos& p, int g, int gst, bool chi) {
  MT m = rmask_rel<MT>(p.q0 - F.cut0 + p.r0, p.q0 + F.cut0 - 1, F.nb);
  if (!m) return MT(0);
  if (gst > g && p.q0 + F.R0 + 1 >= 0 && p.q0 + p.r0 - F.R0 - 1 <= F.nb)
    m &= ~rmask_rel<MT>(p.q0 - F.R0, p.q0 + F.R0 + p.r0 - 1, F.nb);
  if (chi) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b >= F.nB) break;
      const int a1 = p.q0 - F.B0[b], a2 = p.q0 + F.B0[b];
      if (a1 >= -1 && a1 + p.r0 <= F.nb + 1) m &= ~rmask_rel<MT>(a1 + p.r0 - 1, a1, F.nb);
      if (a2 >= -1 && a2 + p.r0 <= F.nb + 1) m &= ~rmask_rel<MT>(a2 + p.r0 - 1, a2, F.nb);
    }
  }
  return m;
}

// accept_mask(g - 1, ..., child = true) over the frame's panels of grid g.
template <typename MT>
MARFA_HD MT accept_parent_frame(const PanelFrame& F, const PanelPos& p, int g, int gst, bool chi) {
  // parent panel a (relative to floor(base / 2)) -> children 2a - e, 2a + 1 - e
  MT m = rmask_rel<MT>(2 * (p.q1 - F.cut1 + p.r1) - F.e, 2 * (p.q1 + F.cut1 - 1) + 1 - F.e, F.nb);
  if (!m) return MT(0);
  if (gst > g - 1 && p.q0 + 2 * F.R1 + 2 >= 0 && p.q0 + p.r0 - 2 * F.R1 - 2 <= F.nb)
    m &= ~rmask_rel<MT>(2 * (p.q1 - F.R1) - F.e, 2 * (p.q1 + F.R1 + p.r1 - 1) + 1 - F.e, F.nb);
  if (chi) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b >= F.nB) break;
      const int c1 = p.q0 - F.B0[b], c2 = p.q0 + F.B0[b];  // in panels of grid g
      if (c1 >= -2 && c1 + p.r0 <= F.nb + 2) {
        const int a = p.q1 - F.B1[b];
        m &= ~rmask_rel<MT>(2 * (a + p.r1 - 1) - F.e, 2 * a + 1 - F.e, F.nb);
      }
      if (c2 >= -2 && c2 + p.r0 <= F.nb + 2) {
        const int a = p.q1 + F.B1[b];
        m &= ~rmask_rel<MT>(2 * (a + p.r1 - 1) - F.e, 2 * a + 1 - F.e, F.nb);
      }
    }
  }
  return m;
}

// owns_nothing(g, ...) for the frame's span (xa = base P, xb = (base + nb) P).
MARFA_HD bool owns_nothing_frame(const PanelFrame& F, const PanelPos& p, int g, int gst, bool chi) {
  if (gst >= g) return false;
  auto near = [&](int a) { return a >= -1 && a + p.r0 <= F.nb + 1; };
  if (near(p.q0 - F.cut0) || near(p.q0 + F.cut0)) return false;
  if (chi) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
      if (b < F.nB && (near(p.q0 - F.B0[b]) || near(p.q0 + F.B0[b]))) return false;
  }
  return true;
}

// ------------------------------------------------------------------ ownership by mechanism
// Away from each other, the three things that decide a line's panels on grid g act
// separately: the centre (grid g carries the ring d_near(Q) >= R_w h_g of a line whose
// core is finer, or the whole core when g* = g), each cut-off edge (the grid carries the
// panel inside the cut-off whose parent straddles it) and each chi breakpoint (the
// grid carries the children of a parent holding the breakpoint that do not hold it
// themselves). mech_ok tells when they are far enough apart on grid g (3-point
// partition) that the owned panels are exactly the union of the closed forms below and
// no node belongs to panels of two mechanisms (so that each node is evaluated once):
// the centre's panels lie within R_w h_(g-1) + 4 h_g of the centre (their parents are
// nearer than R_w h_(g-1)), a breakpoint's and an edge's within the one parent (4 h_g)
// holding it; so an applicable breakpoint B (B <= cut-off) needs B >= R_w h_(g-1) + 8 h_g
// and B + 8 h_g < cut-off, consecutive breakpoints more than 8 h_g apart, and without
// breakpoints the cut-off needs to exceed R_w h_(g-1) + 8 h_g.
// The finest grid has the same structure with the G10 panels (mech_fine_ok).
MARFA_HD bool mech_ok(int g, int64_t cut, int R_w, bool chi_req) {
  const int64_t h8 = step_fx(g) << 3, R2 = (int64_t)R_w * step_fx(g - 1);
  if (!(R2 + h8 < cut)) return false;
  if (chi_req) {
    int64_t prev = -h8;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int64_t B = chi_break_fx(b);
      if (B > cut) break;
      if (!(B >= R2 + h8 && B + h8 < cut && B - prev > h8)) return false;
      prev = B;
    }
  }
  return true;
}

// Finest grid: the centre's nodes lie within R_w h_10 + P of the centre (P the G10 panel
// width), a breakpoint's within P of it, an edge's within P inside it.
MARFA_HD bool mech_fine_ok(int64_t cut, int R_w, bool chi_req) {
  const int64_t P = int64_t(1) << panel_shift(kNGrid), R = (int64_t)R_w * step_fx(kNGrid);
  if (!(R + 2 * P < cut)) return false;
  if (chi_req) {
    int64_t prev = -2 * P;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int64_t B = chi_break_fx(b);
      if (B > cut) break;
      if (!(B >= R + 2 * P && B + 2 * P < cut && B - prev > 2 * P)) return false;
      prev = B;
    }
  }
  return true;
}

// The finest grid's merged pass takes every cut-off edge and chi breakpoint of a line in
// one pass and gives a candidate the nodes of one mechanism in a span of `span` units
// (a warp's nodes): that needs the edge and the applicable breakpoints on one side of
// the centre to lie more than the span plus two G10 panels apart (mech_fine_ok alone
// allows two G10 panels).
MARFA_HD bool mech_fine_merge_ok(int64_t cut, int R_w, bool chi_req, int64_t span) {
  if (!mech_fine_ok(cut, R_w, chi_req)) return false;
  if (!chi_req) return true;
  const int64_t gap = span + (int64_t(2) << panel_shift(kNGrid));
  int64_t prev = -1;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int64_t B = chi_break_fx(b);
    if (B > cut) break;
    if (cut - B <= gap || (prev >= 0 && B - prev <= gap)) return false;
    prev = B;
  }
  return true;
}

// The centre's panels of grid g (absolute indices): [a1, b1] left of the centre and
// [a2, b2] right of it (either may be empty: a > b); with gst == g the two ranges
// join into the core [a1, b2] (b1 = a2 - 1); with gst < g none.
MARFA_HD void mech_centre(int g, int64_t c, int gst, int R_w, int64_t& a1, int64_t& b1, int64_t& a2, int64_t& b2) {
  const int s = panel_shift(g);
  const int64_t R = (int64_t)R_w * step_fx(g), R2 = (int64_t)R_w * step_fx(g - 1);
  const int64_t lo = fl_sh(c - R2, s + 1) << 1, hi = ((cl_sh(c + R2, s + 1) - 1) << 1) + 1;
  if (gst < g) {
    a1 = a2 = 1;
    b1 = b2 = 0;
  } else if (gst == g) {
    a1 = lo;
    b2 = hi;
    a2 = hi + 1;
    b1 = hi;
  } else {
    a1 = lo;
    b1 = min(hi, fl_sh(c - R, s) - 1);
    a2 = max(lo, cl_sh(c + R, s));
    b2 = hi;
  }
}

// The panel of grid g a cut-off edge gives (-1: none; a negative panel lies outside
// every window): right edge E = c + cut-off, left edge E = c - cut-off.
MARFA_HD int64_t mech_edge_right(int g, int64_t E) {
  const int64_t t = fl_sh(E, panel_shift(g));
  return (t & 1) ? t - 1 : -1;
}
MARFA_HD int64_t mech_edge_left(int g, int64_t E) {
  const int64_t u = cl_sh(E, panel_shift(g));
  return (u & 1) ? u : -1;
}

// The panels of grid g a breakpoint at position K gives: q[0], q[1] (-1: none).
MARFA_HD void mech_kink(int g, int64_t K, int64_t& q0, int64_t& q1) {
  const int s = panel_shift(g);
  const int64_t n = fl_sh(K, s + 1), r = K - (n << (s + 1)), P = int64_t(1) << s;
  q0 = q1 = -1;
  if (r == 0) {
    q0 = 2 * n - 2;
    q1 = 2 * n + 1;
  } else if (r < P) {
    q0 = 2 * n + 1;
  } else if (r > P) {
    q0 = 2 * n;
  }
}

// Finest-grid nodes (absolute indices, inclusive ranges; a > b empty) of each mechanism.
MARFA_HD void mech_fine_centre(int64_t c, int gst, int R_w, int64_t& a, int64_t& b) {
  const int s10 = panel_shift(kNGrid);
  const int64_t R = (int64_t)R_w * step_fx(kNGrid);
  if (gst <= kNGrid) {
    a = 1;
    b = 0;
    return;
  }
  a = fl_sh(c - R, s10) << 3;
  b = ((cl_sh(c + R, s10) - 1) << 3) + 7;
}
MARFA_HD void mech_fine_edge_right(int64_t E, int64_t& a, int64_t& b) {
  a = fl_sh(E, panel_shift(kNGrid)) << 3;
  b = fl_sh(E, kFineShift);
}
MARFA_HD void mech_fine_edge_left(int64_t E, int64_t& a, int64_t& b) {
  a = cl_sh(E, kFineShift);
  b = ((cl_sh(E, panel_shift(kNGrid)) - 1) << 3) + 7;
}
MARFA_HD void mech_fine_kink(int64_t K, int64_t& a, int64_t& b) {
  const int s10 = panel_shift(kNGrid);
  const int64_t p = fl_sh(K, s10);
  b = (p << 3) + 7;
  a = (K == (p << s10)) ? (p - 1) << 3 : p << 3;
}

}  // namespace marfa

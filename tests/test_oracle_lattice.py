"""Pins of the oracle's lattice constants, equilibrium and mode basis.

Every value is fixed by the paper (Sec. 2 lattice and Eq. e.LB2; Sec. 4 Table 1)
or by an exact algebraic identity, not by re-reading the oracle's own code.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [c.strip() for c in line.split("|")]


def test_lattice_vectors_from_paper_formulas(oracle):
    """Sec. 2: e_i from the printed cos/sin formulas, omega_i as printed."""
    e, w, opp = oracle.lattice()
    env = {"cos": math.cos, "sin": math.sin, "sqrt": math.sqrt, "pi": math.pi}
    for i, expr, wi in _rows("d2q9_lattice.txt"):
        ex, ey = eval(expr, env)  # noqa: S307 - fixture text written from the paper
        assert (round(ex), round(ey)) == tuple(e[int(i)])
        assert abs(ex - round(ex)) < 1e-12 and abs(ey - round(ey)) < 1e-12
        assert w[int(i)] == pytest.approx(float(Fraction(wi)), abs=0, rel=1e-15)
    for i in range(9):
        assert tuple(e[opp[i]]) == (-e[i][0], -e[i][1])


def test_lattice_isotropy(oracle):
    """Weights give sum w = 1, zero first and third moments, second moment c_s^2 delta
    and the isotropic fourth moment c_s^4 (dd + dd + dd) that e.LB2 relies on."""
    e, w, _ = oracle.lattice()
    e = e.astype(float)
    cs2 = 1.0 / 3.0
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs(w @ e).max() < 1e-16
    M2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(M2, cs2 * np.eye(2), atol=1e-16, rtol=0)
    M3 = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    assert np.abs(M3).max() < 1e-16
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(2)
    iso = cs2 * cs2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-16, rtol=0)


def test_table1_basis_as_printed(oracle):
    """Table 1: e_ki evaluated from the printed expressions, chi_ki = e_ki / sqrt(w_k)."""
    e, w, _ = oracle.lattice()
    chi, wk = oracle.basis()
    for k, expr, wk_txt in _rows("table1_basis.txt"):
        k = int(k)
        assert wk[k] == pytest.approx(float(Fraction(wk_txt)), rel=1e-15)
        for i in range(9):
            ex, ey = float(e[i][0]), float(e[i][1])
            eki = eval(expr, {"ex": ex, "ey": ey, "e2": ex * ex + ey * ey})  # noqa: S307
            assert chi[k, i] * math.sqrt(wk[k]) == pytest.approx(eki, abs=1e-14)


def test_table1_lengths_match_caption_definition(oracle):
    """Table 1 caption: w_k = sum_i omega_i e_ki^2, exactly, in rationals."""
    e, w, _ = oracle.lattice()
    wts = [Fraction(4, 9)] + [Fraction(1, 9)] * 4 + [Fraction(1, 36)] * 4
    for k, expr, wk_txt in _rows("table1_basis.txt"):
        s = Fraction(0)
        for i in range(9):
            ex, ey = int(e[i][0]), int(e[i][1])
            eki = eval(expr, {"ex": Fraction(ex), "ey": Fraction(ey),  # noqa: S307
                              "e2": Fraction(ex * ex + ey * ey)})
            s += wts[i] * eki * eki
        assert s == Fraction(wk_txt)


def test_basis_orthonormal_both_ways(oracle):
    """Sec. 4: sum_i omega_i chi_ki chi_li = delta_kl and sum_k omega_i chi_ki chi_ki' = delta_ii'."""
    _, w, _ = oracle.lattice()
    chi, _ = oracle.basis()
    assert np.allclose(chi @ np.diag(w) @ chi.T, np.eye(9), atol=1e-14, rtol=0)
    assert np.allclose(np.diag(w) @ chi.T @ chi, np.eye(9), atol=1e-14, rtol=0)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.003, 0.05, -0.02), (0.97, -0.11, 0.07)])
def test_equilibrium_moments(oracle, rho, ux, uy):
    """Eq. e.LB2 on D2Q9 reproduces rho, rho u and rho c_s^2 I + rho u u exactly."""
    e, _, _ = oracle.lattice()
    e = e.astype(float)
    f = oracle.feq(rho, ux, uy)
    u = np.array([ux, uy])
    assert f.sum() == pytest.approx(rho, abs=1e-15)
    assert np.allclose(f @ e, rho * u, atol=1e-16, rtol=0)
    Pi = np.einsum("i,ia,ib->ab", f, e, e)
    assert np.allclose(Pi, rho / 3.0 * np.eye(2) + rho * np.outer(u, u), atol=1e-15, rtol=0)

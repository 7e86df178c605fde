"""Pins of the oracle's spherical-harmonic basis (the colour model of the
rasterizer the paper uses, Sec. 3.3 "Implementation": SH up to degree 3)
against closed forms and a library routine, so that a sign flip or a
permutation of m within a band -- which orthonormality and homogeneity
cannot see -- fails here.

The basis is the real form of the complex harmonics Y_l^m that carry the
Condon-Shortley phase (-1)^m, taken as
    m > 0:  sqrt(2) Re Y_l^m,   m = 0:  Y_l^0,   m < 0:  sqrt(2) Im Y_l^|m|,
with coefficient k = l^2 + l + m, the order and signs of the original 3DGS
renderer (e.g. Y_{1,-1} = -sqrt(3/(4 pi)) y, Y_{1,1} = -sqrt(3/(4 pi)) x).
"""
import math

import numpy as np
import pytest

import oracle

scipy_special = pytest.importorskip("scipy.special")

AXES = {"+x": (1, 0, 0), "-x": (-1, 0, 0), "+y": (0, 1, 0), "-y": (0, -1, 0), "+z": (0, 0, 1), "-z": (0, 0, -1)}
OBLIQUE = [(1.0, 1.0, 1.0), (0.3, -0.8, 0.52)]


def _library_real_sh(l, m, d):
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    Y = complex(scipy_special.sph_harm_y(l, abs(m), theta, phi))
    if m > 0:
        return math.sqrt(2.0) * Y.real
    if m < 0:
        return math.sqrt(2.0) * Y.imag
    return Y.real


def test_library_carries_the_condon_shortley_phase():
    # Y_1^1 = -(1/2) sqrt(3/(2 pi)) sin(theta) e^{i phi}: negative real part at +x
    Y = complex(scipy_special.sph_harm_y(1, 1, math.pi / 2, 0.0))
    assert Y.real == pytest.approx(-0.5 * math.sqrt(3.0 / (2.0 * math.pi)), rel=1e-12)


@pytest.mark.parametrize("name", list(AXES) + ["oblique0", "oblique1"])
def test_every_coefficient_equals_the_library_real_form(name):
    d = AXES[name] if name in AXES else OBLIQUE[int(name[-1])]
    d = np.asarray(d, dtype=np.float64) / np.linalg.norm(d)
    Y = oracle.sh_eval(3, d)[0]
    for l in range(4):
        for m in range(-l, l + 1):
            assert Y[l * l + l + m] == pytest.approx(_library_real_sh(l, m, d), abs=1e-13), (l, m)


def test_random_directions_match_the_library():
    rng = np.random.default_rng(11)
    for _ in range(40):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y = oracle.sh_eval(3, d)[0]
        ref = [_library_real_sh(l, m, d) for l in range(4) for m in range(-l, l + 1)]
        np.testing.assert_allclose(Y, ref, atol=1e-13)


def test_axis_values_closed_form():
    """Values at the axes written out from the Legendre functions:
    on +-z only m = 0 survives, Y_l0 = (+-1)^l sqrt((2l+1)/(4 pi));
    on +x / +y the degree-1 functions are -sqrt(3/(4 pi)) (x and y carry the
    phase), and the degree-2 ones at +x are Y_22 = sqrt(15/pi)/4,
    Y_20 = -sqrt(5/pi)/4, at +y Y_22 = -sqrt(15/pi)/4; the degree-3 ones at
    +x are Y_33 = -sqrt(35/(2 pi))/4, Y_31 = sqrt(21/(2 pi))/4."""
    pi = math.pi
    exp = {
        "+z": {(l, 0): math.sqrt((2 * l + 1) / (4 * pi)) for l in range(4)},
        "-z": {(l, 0): (-1) ** l * math.sqrt((2 * l + 1) / (4 * pi)) for l in range(4)},
        "+x": {(0, 0): 0.5 / math.sqrt(pi), (1, 1): -math.sqrt(3 / (4 * pi)), (2, 2): math.sqrt(15 / pi) / 4,
               (2, 0): -math.sqrt(5 / pi) / 4, (3, 3): -math.sqrt(35 / (2 * pi)) / 4,
               (3, 1): math.sqrt(21 / (2 * pi)) / 4},
        "+y": {(0, 0): 0.5 / math.sqrt(pi), (1, -1): -math.sqrt(3 / (4 * pi)), (2, 2): -math.sqrt(15 / pi) / 4,
               (2, 0): -math.sqrt(5 / pi) / 4, (3, -3): math.sqrt(35 / (2 * pi)) / 4,
               (3, -1): math.sqrt(21 / (2 * pi)) / 4},
    }
    for name, vals in exp.items():
        Y = oracle.sh_eval(3, AXES[name])[0]
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(vals.get((l, m), 0.0), abs=1e-14), (name, l, m)

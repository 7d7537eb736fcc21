"""The host-side logic of the complex-plane strategy in libeigdc (CPU, no GPU).

The library's enclosing circle and line draws (Sec. 3.3: random angle, offset
within half the radius, the perpendicular line of the 2-step rule, the
recentering circle) are compared with the oracle on the same regions and
Philox counters.  Both are host code, so this parity runs without a GPU.
"""
import numpy as np
import pytest

from oracle import cplane
from oracle.cplane import Region, enclosing_circle, draw_line, SHRINK


@pytest.fixture(scope="module")
def eigdc():
    from paper_1011_3077_gb300 import build, eigdc as mod
    build.build()
    mod.lib()
    return mod


def _random_region(rng):
    c = complex(*rng.uniform(-2, 2, 2))
    R = rng.uniform(0.1, 3.0)
    anchor = c + 0.3 * R * np.exp(2j * np.pi * rng.uniform())
    hps = []
    for _ in range(int(rng.integers(0, 5))):
        w = np.exp(2j * np.pi * rng.uniform())
        t = (np.conj(w) * c).real + R * rng.uniform(-0.5, 0.5)
        hps.append((w, t) if (np.conj(w) * anchor).real >= t else (-w, -t))
    return c, R, hps


def test_enclosing_circle_matches_the_oracle(eigdc):
    rng = np.random.default_rng(101)
    for _ in range(300):
        c, R, hps = _random_region(rng)
        m_lib, r_lib = eigdc.cplane_enclosing_circle(c, R, hps)
        m_or, r_or = enclosing_circle(Region(c, R, hps))
        assert abs(r_lib - r_or) <= 1e-13 * R
        assert abs(m_lib - m_or) <= 1e-13 * (R + abs(c))


def test_enclosing_circle_closed_forms(eigdc):
    m, r = eigdc.cplane_enclosing_circle(0, 1.0, [(1, -0.5), (-1j, -0.5)])
    assert abs(r - SHRINK) < 1e-15 and abs(r - np.sin(5 * np.pi / 12)) < 1e-15
    m, r = eigdc.cplane_enclosing_circle(0, 2.0, [(1, 0.0), (-1j, 0.0)])
    assert abs(r - np.sqrt(2.0)) < 1e-14 and abs(m - (1 - 1j)) < 1e-14
    m, r = eigdc.cplane_enclosing_circle(1 + 1j, 1.0, [])
    assert m == 1 + 1j and r == 1.0


@pytest.mark.parametrize("seed", [0, 7, 2 ** 40 + 3])
def test_draw_line_matches_the_oracle(eigdc, seed):
    rng = np.random.default_rng(seed % 1000)
    for attempt in range(40):
        node = int(rng.integers(1, 2 ** 62))
        c = complex(*rng.uniform(-1, 1, 2))
        R = float(rng.uniform(0.1, 4.0))
        perp = None if attempt % 3 else np.exp(2j * np.pi * rng.uniform())
        w_lib, t_lib = eigdc.cplane_draw_line(seed, node, attempt, c, R, perp)
        w_or, t_or = draw_line(Region(c, R), seed, node, attempt, perp)
        assert abs(w_lib - w_or) < 1e-15
        assert abs(t_lib - t_or) < 1e-14 * (1 + R + abs(c))
        assert abs(abs(w_lib) - 1.0) < 1e-15
        # the line lies at most R/2 from the centre
        assert abs(t_lib - (np.conj(w_lib) * c).real) <= 0.5 * R


def test_host_helpers_reject_bad_arguments(eigdc):
    with pytest.raises(eigdc.EigError):
        eigdc.cplane_enclosing_circle(0, -1.0, [])
    with pytest.raises(eigdc.EigError):
        eigdc.cplane_draw_line(0, 1, 0, 0, -2.0)

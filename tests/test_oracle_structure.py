"""Pins for the oracle structure functions (Sec. 3.5, strfunc-def / strfunc-verif): closed forms
of a single velocity mode, brute force on a tiny grid, the Wiener-Khinchin identity for p = 2,
the periodic symmetry, and the large-separation limit the paper uses as its check."""
import math

import numpy as np
import pytest

from inputs import grid_coords, random_psi
from oracle import structure as SF
from oracle import scheme as S


def _p(n):
    return S.params_from_dx_ratio(n, 1.5, 0.01)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_velocity_of_a_phase_wave_is_exact(axis):
    """psi = A(x) exp(i a cos(k x_j)) with an amplitude A that varies along another axis has
    v_j = -2 alpha a k sin(k x_j) whatever A is (band-limited to round-off for a small a), the
    other components 0."""
    n, a, k = 32, 0.15, 2
    p = _p(n)
    c = grid_coords(n)[axis]
    amp = 0.6 * (1 + 0.3 * np.cos(grid_coords(n)[(axis + 1) % 3]))
    v = SF.velocity(amp * np.exp(1j * a * np.cos(k * c)), p)
    want = -2 * p.alpha * a * k * np.sin(k * c)
    for j in range(3):
        assert np.max(np.abs(v[j] - (want if j == axis else 0.0))) < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_single_mode_closed_forms(axis):
    """v_j = A sin(k x_j): v(x + r) - v(x) = 2 A sin(k r / 2) cos(k x + k r / 2), so
    S^1 = S^3 = 0, S^2 = A^2 (1 - cos k r), S^4 = 6 A^4 sin^4(k r / 2); along the two other
    axes the field does not change and every S^p is 0."""
    n, A, k = 24, 0.7, 3
    c = grid_coords(n)[axis]
    v = [np.zeros((n, n, n)) for _ in range(3)]
    v[axis] = A * np.sin(k * c)
    r = SF.separations(n)
    s2 = SF.structure_function(v, 2)
    s4 = SF.structure_function(v, 4)
    s1 = SF.structure_function(v, 1)
    s3 = SF.structure_function(v, 3)
    assert np.max(np.abs(s2[axis] - A * A * (1 - np.cos(k * r)))) < 1e-14
    assert np.max(np.abs(s4[axis] - 6 * A ** 4 * np.sin(k * r / 2) ** 4)) < 1e-14
    assert np.max(np.abs(s1[axis])) < 1e-15 and np.max(np.abs(s3[axis])) < 1e-15
    for j in range(3):
        if j != axis:
            assert np.max(np.abs(s2[j])) == 0.0


def test_brute_force_on_a_tiny_grid():
    """Explicit loops over the points of a 6^3 grid with a random field, for odd and even
    orders (an odd order fixes the direction of the shift)."""
    n = 6
    rng = np.random.default_rng(3)
    v = [rng.standard_normal((n, n, n)) for _ in range(3)]
    for order in (1, 2, 3):
        got = SF.structure_function(v, order)
        for j in range(3):
            for s in range(n // 2 + 1):
                tot = 0.0
                for z in range(n):
                    for y in range(n):
                        for x in range(n):
                            q = [x, y, z]
                            q[j] = (q[j] + s) % n
                            tot += (v[j][q[2], q[1], q[0]] - v[j][z, y, x]) ** order
                assert got[j, s] == pytest.approx(tot / n ** 3, abs=1e-13)


def test_second_order_by_wiener_khinchin():
    """S^2_j(r) = 2 <v_j^2> - 2 C_j(r), with the autocorrelation C_j(r) = <v_j(x) v_j(x + r e_j)>
    computed from the power spectrum along axis j (numpy's FFT: an independent route)."""
    n = 16
    p = _p(n)
    v = SF.velocity(random_psi(n, 7, amp_jitter=0.2), p)
    got = SF.structure_function(v, 2)
    for j, ax in enumerate((2, 1, 0)):
        f = np.fft.fft(v[j], axis=ax)
        corr = np.real(np.fft.ifft(np.abs(f) ** 2, axis=ax))          # sum_x v(x) v(x + s)
        c = np.mean(np.moveaxis(corr, ax, 0).reshape(n, -1), axis=1)[: n // 2 + 1] / n
        want = 2 * np.mean(v[j] ** 2) - 2 * c
        assert np.max(np.abs(got[j] - want)) < 1e-12 * np.max(np.abs(want))


def test_periodic_symmetry_and_zero_shift():
    """S^p(0) = 0, and the shift by N - s gives (-1)^p S^p(s): checked with the full range of
    shifts written out for the odd order."""
    n = 12
    p = _p(n)
    v = SF.velocity(random_psi(n, 9, amp_jitter=0.2), p)
    for order in (2, 3):
        got = SF.structure_function(v, order)
        assert np.all(got[:, 0] == 0.0)
        for j, ax in enumerate((2, 1, 0)):
            for s in range(1, n // 2 + 1):
                back = float(np.mean((np.roll(v[j], -(n - s), axis=ax) - v[j]) ** order))
                assert back == pytest.approx((-1) ** order * got[j, s], abs=1e-12)


def test_large_separation_limit():
    """strfunc-verif: for a field whose velocity decorrelates over a short distance, S^2 at half
    the box approaches 2 <v_x^2> (here a sum of random modes of wavenumber 5 to 8 with random
    phases: at r = pi the mode correlations cos(k pi) alternate and largely cancel)."""
    n = 32
    X, Y, Z = grid_coords(n)
    rng = np.random.default_rng(11)
    vx = np.zeros((n, n, n))
    for _ in range(40):
        k = rng.integers(5, 9, size=3) * rng.choice([-1, 1], size=3)
        vx += math.cos(rng.uniform(0, 2 * math.pi)) * np.cos(k[0] * X + k[1] * Y + k[2] * Z + rng.uniform(0, 6.3))
    v = [vx, np.zeros_like(vx), np.zeros_like(vx)]
    s2 = SF.structure_function(v, 2)
    assert s2[0, -1] == pytest.approx(2 * np.mean(vx ** 2), rel=0.35)
    # and exactly: S^2(pi) = 2 <v^2> - 2 sum over modes of their power times cos(k_x pi)
    f = np.fft.fftn(vx) / n ** 3
    kx = np.fft.fftfreq(n, 1.0 / n)[None, None, :]
    want = 2 * np.sum(np.abs(f) ** 2 * (1 - np.cos(kx * math.pi)))
    assert s2[0, -1] == pytest.approx(want, rel=1e-12)

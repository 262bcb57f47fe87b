"""Pins for the oracle random stream and initial conditions (Sec. 5.3, 5.4)."""
import math

import numpy as np
import pytest

from oracle import fft, initial as I, rng
from oracle import scheme as S


def _splitmix64_sequential(state, count):
    """SplitMix64 written as the published stateful generator (independent of the counter form)."""
    out = []
    mask = (1 << 64) - 1
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_counter_form_matches_stateful_generator():
    seq = _splitmix64_sequential(0, 16)
    got = [int(v) for v in rng.splitmix64(np.arange(16, dtype=np.uint64))]
    assert got == seq
    # published first output of SplitMix64 started from state 0
    assert seq[0] == 0xE220A8397B1DCDAF
    # seed s reads positions s * 2^40 + i: a stateful generator that already made s * 2^40 draws
    seq7 = _splitmix64_sequential(((7 << 40) * 0x9E3779B97F4A7C15) & ((1 << 64) - 1), 3)
    assert [int(v) for v in rng.splitmix64(rng.positions(7, np.arange(3)))] == seq7


def test_uniform_and_normal_draws():
    v = rng.splitmix64(np.arange(200000, dtype=np.uint64))
    u = rng.uniform01(v)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 3e-3
    assert rng.uniform01_open0(np.uint64(0)) == 2.0 ** -53
    g = I.white_noise(40, 3).ravel()
    assert abs(g.mean()) < 5e-3 and abs(g.var() - 1.0) < 1e-2


def test_srp_spectral_properties():
    n, k0 = 24, 4.0
    th = I.srp_theta(n, 0, k0)
    assert abs(math.sqrt(np.mean(th ** 2)) - math.pi) < 1e-12
    assert abs(np.mean(th)) < 1e-12
    # theta_k = c * F(w)_k * exp(-|k|^2/k0^2) for k != 0 with one real constant c (numpy.fft)
    k = np.fft.fftfreq(n, 1.0 / n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    th_hat = np.fft.fftn(th)
    model = np.fft.fftn(I.white_noise(n, 0)) * np.exp(-k2 / k0 ** 2)
    model[0, 0, 0] = 0.0
    c = np.real(th_hat[0, 0, 1] / model[0, 0, 1])
    assert c > 0 and np.max(np.abs(th_hat - c * model)) < 1e-12 * np.max(np.abs(th_hat))
    psi = I.srp_spectral(n, 0, k0)
    assert np.max(np.abs(np.abs(psi) - 1.0)) < 1e-14
    # different seeds differ, same seed repeats
    assert np.array_equal(th, I.srp_theta(n, 0, k0))
    assert np.max(np.abs(th - I.srp_theta(n, 1, k0))) > 0.1


def test_periodic_spline_matches_scipy():
    """The A, B, C, D spline of Sec. 5.3 equals the textbook periodic cubic spline."""
    from scipy.interpolate import CubicSpline
    rs = np.random.default_rng(4)
    nr, ns = 5, 7
    yc = rs.uniform(-1, 1, nr)
    fine = I._spline_fill(yc[None, :], ns)[0]
    xs = np.arange(nr + 1) * ns
    cs = CubicSpline(xs, np.append(yc, yc[0]), bc_type="periodic")
    assert np.max(np.abs(fine - cs(np.arange(nr * ns)))) < 1e-12
    assert np.max(np.abs(fine[::ns] - yc)) < 1e-15


def test_srp_spline_field():
    n, nr, K = 16, 4, 8 * math.pi
    th = I.srp_spline_theta(n, 2, K, nr)
    ns = n // nr
    idx = np.arange(nr ** 3, dtype=np.uint64)
    lat = (K * (2.0 * rng.uniform01(rng.splitmix64(rng.positions(2, idx))) - 1.0)).reshape(nr, nr, nr)
    assert np.max(np.abs(th[::ns, ::ns, ::ns] - lat)) < 1e-12       # passes through the lattice
    assert np.abs(lat).max() <= K
    # the tensor-product spline: interpolating along z first gives the same field
    from scipy.interpolate import CubicSpline
    xs = np.arange(nr + 1) * ns
    t = lat
    for ax in (2, 1, 0):
        t = np.moveaxis(t, ax, -1)
        cs = CubicSpline(xs, np.concatenate([t, t[..., :1]], axis=-1), axis=-1, bc_type="periodic")
        t = np.moveaxis(cs(np.arange(n)), -1, ax)
    assert np.max(np.abs(t - th)) < 1e-10


def test_rvr_ring_draws():
    R, c, nv = I.rvr_rings(0, 40, 0.2, 0.6)
    assert R.min() >= 0.2 and R.max() < 0.6
    assert c.min() >= 0 and c.max() < 2 * math.pi
    assert np.max(np.abs(np.linalg.norm(nv, axis=1) - 1.0)) < 1e-14


def test_rvr_tanh_core_and_winding():
    """One ring: |psi| vanishes on the core circle and the phase winds by 2 pi around it."""
    xi = 0.05
    R = np.array([0.6])
    c = np.array([[3.0, 2.5, 3.5]])
    nv = np.array([[0.0, 0.6, 0.8]])
    e1 = np.array([1.0, 0.0, 0.0])                    # in-plane unit vector (orthogonal to nv)
    core = c[0] + R[0] * e1
    assert abs(I.rvr_tanh_points(core[None, :], xi, R, c, nv)[0]) < 1e-12
    t = np.linspace(0, 2 * math.pi, 65)
    loop = core + 0.5 * xi * (np.cos(t)[:, None] * e1 + np.sin(t)[:, None] * nv[0])
    ph = np.angle(I.rvr_tanh_points(loop, xi, R, c, nv))
    winding = np.sum(np.angle(np.exp(1j * np.diff(ph)))) / (2 * math.pi)
    assert abs(abs(winding) - 1.0) < 1e-9
    far = c[0] + np.array([1.5, 0.0, 0.0])
    assert abs(abs(I.rvr_tanh_points(far[None, :], xi, R, c, nv)[0]) - 1.0) < 1e-10


def test_pade_profile_asymptotics():
    """f^2 ~ a1 (r/xi)^2 at small r, and the large-r solution of the vortex equation
    f^2 = 1 - xi^2/r^2 + ... fixes b1 - a1 = a2."""
    assert abs(I.PADE_B1 - I.PADE_A1 - I.PADE_A2) < 1e-15
    xi = 0.1
    assert abs(I.pade_profile(1e-4 * xi, xi) ** 2 / 1e-8 - I.PADE_A1) < 1e-6
    r = 1e3 * xi
    assert abs((1.0 - I.pade_profile(r, xi) ** 2) * (r / xi) ** 2 - 1.0) < 1e-3
    # the residual of -alpha/r (r f')' + alpha f / r^2 + beta (f^2 - 1) f decays at least like
    # (r/xi)^-3 at large r (its leading terms cancel); a wrong coefficient leaves an (r/xi)^-2 residual
    alpha = 0.1
    beta = alpha / xi ** 2

    def res(eta):
        r, h = eta * xi, 1e-3 * xi
        f = lambda x: I.pade_profile(x, xi)
        fp = (f(r + h) - f(r - h)) / (2 * h)
        fpp = (f(r + h) - 2 * f(r) + f(r - h)) / h ** 2
        return abs(-alpha * (fpp + fp / r) + alpha * f(r) / r ** 2 + beta * (f(r) ** 2 - 1) * f(r))

    assert math.log2(res(10.0) / res(20.0)) > 2.8 and math.log2(res(5.0) / res(10.0)) > 2.8
    assert res(10.0) < 0.2 * beta / 100.0


def test_rvr_pade_building_blocks():
    n = 16
    xi = 0.2
    X = S.wavenumbers_deriv(n)
    pts = I.grid_points(n)
    base = I.vortex_ring_pair_periodised(pts[..., 0], pts[..., 1], pts[..., 2], 0.5 * math.pi, math.pi, xi)
    # spectral shift by a whole number of cells is an exact roll: moved(x) = base(x + X)
    shift = 4 * 2 * math.pi / n          # an even number of cells: the Nyquist phase is 1 too
    moved = fft.ifft3(np.exp(1j * X[None, None, :] * shift) * fft.fft3(base))
    assert np.max(np.abs(moved - np.roll(base, -4, axis=2))) < 1e-10
    psi = I.rvr_pade(n, 5, xi, 2)
    assert psi.shape == (n, n, n) and np.isfinite(psi).all()
    assert np.max(np.abs(psi)) < 1.05


# ---- the composite of the paper's ring-pair field (Sec. 5.4: eq-one-vortex-ring, eq-Pade,
# psiRP, psiRVR), checked piece by piece with explicit shifts and axis orders

def _pair(x, y, z, xi=0.1):
    return I.vortex_ring_pair_periodised(x, y, z, 0.5 * math.pi, math.pi, xi)


def test_ring_pair_cores_and_windings():
    """The pair psi_VR(z - d/2) psi_VR*(z + d/2) (R = pi/2, d = pi) vanishes on its two core circles
    r = R at z = pi + d/2 and z = pi - d/2, and its phase winds by +1 around the first and by -1
    around the second (the conjugate); the mirror images, nonzero there, change neither."""
    R, d, xi = 0.5 * math.pi, math.pi, 0.1
    t = np.linspace(0.0, 2.0 * math.pi, 129)
    for zc, wind in ((math.pi + 0.5 * d, 1.0), (math.pi - 0.5 * d, -1.0)):
        for phi in (0.0, 1.1, 2.5):                   # three points of each core circle
            cx, cy = math.pi + R * math.cos(phi), math.pi + R * math.sin(phi)
            assert abs(_pair(np.array(cx), np.array(cy), np.array(zc))) < 1e-12
            eps = 0.3 * xi                             # loop in the (r, z) half-plane
            rr = R + eps * np.cos(t)
            ph = np.angle(_pair(math.pi + rr * math.cos(phi), math.pi + rr * math.sin(phi), zc + eps * np.sin(t)))
            w = np.sum(np.angle(np.exp(1j * np.diff(ph)))) / (2.0 * math.pi)
            assert abs(w - wind) < 1e-9, (zc, phi, w)
    # between the rings and far from them there is no core
    assert abs(_pair(np.array(math.pi), np.array(math.pi), np.array(math.pi))) > 0.5


def test_ring_pair_mirror_images_are_paired_about_the_faces():
    """With the images at -x and 2L - x (L = 2 pi) in each direction the periodised pair keeps the
    pair's reflection symmetry x -> 2 pi - x in every coordinate (the conjugated image at -x maps
    onto the one at 4 pi - x), so its values on opposite faces agree; one image alone, or images
    at -x and 2L + x, break it.  The normal derivative is not continuous across the faces: the
    field is only approximately periodic."""
    rng = np.random.default_rng(0)
    x, y, z = rng.uniform(0.0, 2.0 * math.pi, (3, 400))
    f = _pair(x, y, z)
    L2 = 2.0 * math.pi
    assert np.max(np.abs(_pair(L2 - x, y, z) - f)) < 1e-13
    assert np.max(np.abs(_pair(x, L2 - y, z) - f)) < 1e-13
    assert np.max(np.abs(_pair(x, y, L2 - z) - f)) < 1e-13
    zero = np.zeros_like(y)
    assert np.max(np.abs(_pair(zero, y, z) - _pair(zero + L2, y, z))) < 1e-13
    assert np.max(np.abs(_pair(y, z, zero) - _pair(y, z, zero + L2))) < 1e-13
    # a mistake in the image pairing is visible
    R, d, xi = 0.5 * math.pi, math.pi, 0.1
    g = lambda a, b, c: I.vortex_ring_pair(a, b, c, R, d, xi)
    wrong = lambda a, b, c: _pair(a, b, c) * np.conj(g(2 * 2 * math.pi - a, b, c)) / np.conj(g(2 * 2 * math.pi + a, b, c))
    assert np.max(np.abs(wrong(L2 - x, y, z) - wrong(x, y, z))) > 1e-3


def test_rvr_pade_whole_cell_shift_is_a_roll():
    """A translation by an even number of cells in each direction is an exact roll of the pair
    (moved(x) = base(x + X)); the Nyquist-zeroed shift phase is then the exact one."""
    n, xi = 16, 0.2
    dx = 2.0 * math.pi / n
    base = I.rvr_pade_from(n, xi, [(0.0, 0.0, 0.0)], [0])
    moved = I.rvr_pade_from(n, xi, [(2 * dx, 4 * dx, 6 * dx)], [0])
    assert np.max(np.abs(moved - np.roll(base, (-6, -4, -2), axis=(0, 1, 2)))) < 1e-10
    pts = I.grid_points(n)
    direct = _pair(pts[..., 0], pts[..., 1], pts[..., 2], xi)
    assert np.max(np.abs(base - direct)) < 1e-12


def test_rvr_pade_axis_orders_are_transposes():
    """psiRVR's six orders psi(x_s0, x_s1, x_s2): order s is the transpose of the identity-ordered
    field that sends the field's axis c to the coordinate s_c -- one transpose matches, and the
    rings, perpendicular to the pair's own z, end up perpendicular to coordinate s_2."""
    n, xi = 16, 0.2
    dx = 2.0 * math.pi / n
    X = (2 * dx, 4 * dx, 6 * dx)                     # breaks the pair's x <-> y symmetry
    ident = I.rvr_pade_from(n, xi, [X], [0])
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    for o, s in enumerate(I.AXIS_ORDERS):
        f = I.rvr_pade_from(n, xi, [X], [o])
        hits = [A for A in perms if np.max(np.abs(f - np.transpose(ident, A))) < 1e-12]
        assert len(hits) == 1, (s, hits)
        A = hits[0]
        # array axis 2 - c holds coordinate c; the field's coordinate c comes from s_c
        for c in range(3):
            assert A[2 - s[c]] == 2 - c, (s, A)
        # a core point of the first ring: pair coordinates (pi + R, pi, pi + d/2) before the shift
        q = [0, 0, 0]
        for c, v in enumerate((math.pi + 0.5 * math.pi, math.pi, 1.5 * math.pi)):
            q[s[c]] = int(round((v - X[c]) / dx)) % n   # grid index along coordinate s_c
        assert abs(f[q[2], q[1], q[0]]) < 1e-10, s


def test_rvr_pade_is_the_product_of_its_pairs():
    n, xi = 16, 0.2
    shifts, orders = [(0.3, 1.7, 4.1), (5.0, 2.2, 0.9)], [4, 1]
    both = I.rvr_pade_from(n, xi, shifts, orders)
    one = I.rvr_pade_from(n, xi, shifts[:1], orders[:1])
    two = I.rvr_pade_from(n, xi, shifts[1:], orders[1:])
    assert np.max(np.abs(both - one * two)) < 1e-13
    s, o = I.rvr_pade_draws(7, 3)
    assert np.max(np.abs(I.rvr_pade(n, 7, xi, 3) - I.rvr_pade_from(n, xi, s, o))) == 0.0
    assert all(0.0 <= v < 2.0 * math.pi for X in s for v in X) and all(0 <= v < 6 for v in o)

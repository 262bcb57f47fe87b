"""Oracle initial conditions: smoothed random phase (SRP) and random vortex rings (RVR).

Test infrastructure only (see ``oracle/__init__``).

Four generators, all returning complex128 arrays indexed [z, y, x]:

srp_spectral   psi = exp(i theta) (Sec. 5.3, SRP_Init) with theta a Gaussian random field whose
               Fourier amplitudes are filtered by exp(-|k|^2/k0^2), mean removed, scaled to RMS
               theta_rms.  White noise: Box-Muller normals from the counter stream of ``rng``,
               point i (linear index (z N + y) N + x) using stream positions 2i and 2i+1.
srp_spline     the paper's construction (Sec. 5.3): theta uniform in [-K, K] on an N_r^3 lattice
               at N_s (i, j, k), N_s = N/N_r, then periodic uniform cubic-spline interpolation
               along x, then y, then z.  Lattice point (i, j, k) draws stream position
               (k N_r + j) N_r + i.  The tridiagonal system of the paper relates second
               derivatives at neighbouring lattice nodes N_s (i_r - 1), N_s i_r, N_s (i_r + 1).
rvr_tanh       product over rings of tanh(s / (sqrt(2) xi)) exp(i atan2(z', rho' - R)), with s the
               distance to the ring's core circle, computed with the minimum-image displacement;
               radius uniform in [rmin, rmax], centre uniform in the box, normal uniform on the
               sphere.  Ring j draws stream positions 8j .. 8j+7 (R, centre x/y/z, two
               Box-Muller pairs for the normal's three Gaussian components).
rvr_pade       the paper's construction (Sec. 5.4): Pade vortex-ring profile, ring pair
               psi_VR(z - d/2) psi_VR*(z + d/2), the six conjugate mirror images, spectral
               translation by a uniform random X, one of six axis orders, product over N_V pairs.
               Pair p draws stream positions 4p .. 4p+3 (X, Y, Z, permutation).
"""
import math

import numpy as np

from . import fft, rng
from .scheme import wavenumbers, wavenumbers_deriv


def _normals(seed, pos_a, pos_b):
    a = rng.splitmix64(rng.positions(seed, pos_a))
    b = rng.splitmix64(rng.positions(seed, pos_b))
    r = np.sqrt(-2.0 * np.log(rng.uniform01_open0(a)))
    t = 2.0 * math.pi * rng.uniform01(b)
    return r * np.cos(t), r * np.sin(t)


def white_noise(n, seed):
    i = np.arange(n ** 3, dtype=np.uint64)
    g, _ = _normals(seed, 2 * i, 2 * i + 1)
    return g.reshape(n, n, n)


def srp_theta(n, seed, k0, theta_rms=math.pi):
    w = white_noise(n, seed)
    k = wavenumbers(n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    th = fft.fft3(w) * np.exp(-k2 / (k0 * k0))
    th[0, 0, 0] = 0.0
    theta = np.real(fft.ifft3(th))
    return theta * (theta_rms / math.sqrt(float(np.mean(theta ** 2))))


def srp_spectral(n, seed, k0, theta_rms=math.pi):
    return np.exp(1j * srp_theta(n, seed, k0, theta_rms))


# ---------------- SRP, paper variant (spline) ----------------

def _spline_second_derivatives(yc, ns):
    """Solve the periodic system M_{r-1} + 4 M_r + M_{r+1} = 6 (y_{r-1} - 2 y_r + y_{r+1}) / ns^2
    along the last axis (nodes spaced ns fine-grid points apart)."""
    nr = yc.shape[-1]
    A = np.zeros((nr, nr))
    for r in range(nr):
        A[r, r] += 4.0
        A[r, (r - 1) % nr] += 1.0
        A[r, (r + 1) % nr] += 1.0
    rhs = 6.0 * (np.roll(yc, 1, -1) - 2.0 * yc + np.roll(yc, -1, -1)) / ns ** 2
    return np.linalg.solve(A, rhs.reshape(-1, nr).T).T.reshape(yc.shape)


def _spline_fill(yc, ns):
    """Periodic uniform cubic spline through nodes yc[..., r] at fine index ns*r; returns the
    fine samples (length nr*ns) on the last axis, with the A, B, C, D weights of Sec. 5.3."""
    nr = yc.shape[-1]
    M = _spline_second_derivatives(yc, ns)
    out = np.empty(yc.shape[:-1] + (nr * ns,))
    for r in range(nr):
        y0, y1 = yc[..., r], yc[..., (r + 1) % nr]
        m0, m1 = M[..., r], M[..., (r + 1) % nr]
        for s in range(ns):
            A = (ns - s) / ns
            B = s / ns
            C = (A ** 3 - A) * ns ** 2 / 6.0
            D = (B ** 3 - B) * ns ** 2 / 6.0
            out[..., ns * r + s] = A * y0 + B * y1 + C * m0 + D * m1
    return out


def srp_spline_theta(n, seed, K, nr):
    if n % nr:
        raise ValueError("N must be a multiple of N_r")
    ns = n // nr
    idx = np.arange(nr ** 3, dtype=np.uint64)
    u = rng.uniform01(rng.splitmix64(rng.positions(seed, idx)))
    lat = (K * (2.0 * u - 1.0)).reshape(nr, nr, nr)          # [k_r, j_r, i_r]
    t = _spline_fill(lat, ns)                                  # along x: [k_r, j_r, x]
    t = np.moveaxis(_spline_fill(np.moveaxis(t, 1, -1), ns), -1, 1)   # along y: [k_r, y, x]
    t = np.moveaxis(_spline_fill(np.moveaxis(t, 0, -1), ns), -1, 0)   # along z: [z, y, x]
    return t


def srp_spline(n, seed, K, nr):
    return np.exp(1j * srp_spline_theta(n, seed, K, nr))


# ---------------- RVR, configuration variant (tanh rings) ----------------

def rvr_rings(seed, count, rmin, rmax):
    """Ring parameters (R, centre[3], unit normal[3]) drawn from the counter stream."""
    j = np.arange(count, dtype=np.uint64)
    u = [rng.uniform01(rng.splitmix64(rng.positions(seed, 8 * j + c))) for c in range(4)]
    R = rmin + (rmax - rmin) * u[0]
    centre = 2.0 * math.pi * np.stack([u[1], u[2], u[3]], axis=1)
    g0, g1 = _normals(seed, 8 * j + 4, 8 * j + 5)
    g2, _ = _normals(seed, 8 * j + 6, 8 * j + 7)
    nv = np.stack([g0, g1, g2], axis=1)
    nv /= np.linalg.norm(nv, axis=1, keepdims=True)
    return R, centre, nv


def rvr_tanh_points(pts, xi, R, centre, nv):
    """psi at the points pts[..., 3] = (x, y, z) as the product of the ring factors."""
    psi = np.ones(pts.shape[:-1], dtype=np.complex128)
    two_pi = 2.0 * math.pi
    for j in range(len(R)):
        d = pts - centre[j]
        d = d - two_pi * np.floor((d + math.pi) / two_pi)        # minimum image in [-pi, pi)
        zp = d @ nv[j]
        perp = d - zp[..., None] * nv[j]
        rp = np.sqrt(np.sum(perp ** 2, axis=-1))
        s = np.sqrt((rp - R[j]) ** 2 + zp ** 2)
        psi *= np.tanh(s / (math.sqrt(2.0) * xi)) * np.exp(1j * np.arctan2(zp, rp - R[j]))
    return psi


def grid_points(n):
    x = 2.0 * math.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def rvr_tanh(n, seed, xi, count, rmin, rmax):
    R, c, nv = rvr_rings(seed, count, rmin, rmax)
    return rvr_tanh_points(grid_points(n), xi, R, c, nv)


# ---------------- RVR, paper variant (Pade vortex-ring pairs) ----------------

PADE_A1 = (73.0 + 3.0 * math.sqrt(201.0)) / 352.0
PADE_A2 = (6.0 + math.sqrt(201.0)) / 528.0
PADE_B1 = (21.0 + math.sqrt(201.0)) / 96.0


def pade_profile(r, xi):
    """f(r) of eq-Pade with the coefficients of eq-Pade-coefficient."""
    e2 = (r / xi) ** 2
    return np.sqrt((PADE_A1 * e2 + PADE_A2 * e2 ** 2) / (1.0 + PADE_B1 * e2 + PADE_A2 * e2 ** 2))


def vortex_ring(x, y, z, R, xi):
    """psi_VR of eq-one-vortex-ring, centred at (pi, pi, pi), winding +1 (phase atan2(z~, r - R))."""
    xt, yt, zt = x - math.pi, y - math.pi, z - math.pi
    r = np.sqrt(xt ** 2 + yt ** 2)
    return pade_profile(np.sqrt((r - R) ** 2 + zt ** 2), xi) * np.exp(1j * np.arctan2(zt, r - R))


def vortex_ring_pair(x, y, z, R, d, xi):
    return vortex_ring(x, y, z - 0.5 * d, R, xi) * np.conj(vortex_ring(x, y, z + 0.5 * d, R, xi))


def vortex_ring_pair_periodised(x, y, z, R, d, xi):
    """eq psiRP: the pair times the conjugates of its six mirror images (L = 2 pi)."""
    L = 2.0 * math.pi
    f = lambda a, b, c: vortex_ring_pair(a, b, c, R, d, xi)
    return (f(x, y, z)
            * np.conj(f(2 * L - x, y, z)) * np.conj(f(-x, y, z))
            * np.conj(f(x, 2 * L - y, z)) * np.conj(f(x, -y, z))
            * np.conj(f(x, y, 2 * L - z)) * np.conj(f(x, y, -z)))


AXIS_ORDERS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def rvr_pade_draws(seed, npairs):
    """The random part of rvr_pade: per pair a translation X = 2 pi (u0, u1, u2) and an axis order
    index floor(6 u3), pair p using stream positions 4p .. 4p+3."""
    shifts, orders = [], []
    for pidx in range(npairs):
        u = [float(rng.uniform01(rng.splitmix64(rng.positions(seed, 4 * pidx + c)))) for c in range(4)]
        shifts.append((2.0 * math.pi * u[0], 2.0 * math.pi * u[1], 2.0 * math.pi * u[2]))
        orders.append(min(int(6.0 * u[3]), 5))
    return shifts, orders


def rvr_pade_from(n, xi, shifts, orders, R=0.5 * math.pi, d=math.pi):
    """Product over pairs p of the periodised pair translated by shifts[p] = (X, Y, Z) (spectral
    shift with the Nyquist-zeroed wavenumbers: moved(x) = base(x + X)) and read in the axis order
    AXIS_ORDERS[orders[p]] = s: the factor at the point (x0, x1, x2) is moved(x_s0, x_s1, x_s2)."""
    pts = grid_points(n)
    base = vortex_ring_pair_periodised(pts[..., 0], pts[..., 1], pts[..., 2], R, d, xi)
    bh = fft.fft3(base)
    kd = wavenumbers_deriv(n)
    idx = np.arange(n)
    I = np.meshgrid(idx, idx, idx, indexing="ij")          # [iz, iy, ix]
    coords = (I[2], I[1], I[0])                            # (x index, y index, z index)
    psi = np.ones((n, n, n), dtype=np.complex128)
    for X, o in zip(shifts, orders):
        shift = np.exp(1j * (kd[None, None, :] * X[0] + kd[None, :, None] * X[1] + kd[:, None, None] * X[2]))
        moved = fft.ifft3(shift * bh)                      # moved(x) = base(x + X)
        order = AXIS_ORDERS[o]
        a = [coords[order[0]], coords[order[1]], coords[order[2]]]
        psi *= moved[a[2], a[1], a[0]]                     # value of moved at (a0, a1, a2)
    return psi


def rvr_pade(n, seed, xi, npairs, R=0.5 * math.pi, d=math.pi):
    shifts, orders = rvr_pade_draws(seed, npairs)
    return rvr_pade_from(n, xi, shifts, orders, R, d)

"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

The paper prints no worked numerical example (its figures did not survive), so
the oracle is pinned by:

* P1  Eq. tlLapl1 (two-link form) equals Eq. tlLapl2 (single links twice).
* P2  the free field U = 1 (Sec. 2, Fig. 1a): the exact Fourier multiplier
      (1 - (sigma/n) sum_i sin^2 k_i)^n, the exact multinomial expansion in
      rational arithmetic, the conserved sum and the per-axis variance 2 sigma,
      and the lowest mode k = (pi/2, pi/2, pi/2) with eigenvalue -3 of Lap_two.
* P3  gauge covariance under random SU(3) transformations (Sec. 2).
* P4  Hermiticity <phi, Delta psi> = <Delta phi, psi>, the spectrum of
      Delta inside [-12, 0] and the norm bound of the smearing.
* P5  taste/sublattice decoupling (Sec. 2: the operator preserves taste) and
      time-slice decoupling: exact zeros, untouched slices bitwise equal.
* P6  n = 0 and sigma = 0 are the identity; linearity; a batch equals
      separate smears.
* P7  SU(3) closure of W (W W^dag = 1, det W = 1).
* P7b staggered phases on the spatial links leave W unchanged bitwise.
* P8  dense brute force on tiny lattices, and block structure over the 8
      sublattices.
"""

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2301_05518_gb300 import synth
from helpers import rel_l2, sublattice_mask

pytestmark = pytest.mark.filterwarnings("ignore")


def _gauge(dims, seed, kind="near", eps=0.3, nd=4):
    if kind == "near":
        return synth.gauge_near_unit(dims, eps, seed, nd=nd).numpy()
    if kind == "haar":
        return synth.gauge_haar(dims, seed, nd=nd).numpy()
    return synth.gauge_unit(dims, nd=nd).numpy()


def _gauss(dims, nvec, seed, t=None):
    return synth.gaussian_vectors(dims, nvec, seed, t=t).numpy()


# --------------------------------------------------------------------------- P1
@pytest.mark.parametrize("dims,kind", [((4, 4, 4, 2), "near"), ((6, 6, 6, 2), "haar"),
                                        ((8, 8, 8, 16), "near"), ((2, 4, 6, 1), "haar"),
                                        ((2, 2, 2, 2), "haar")])
def test_p1_fused_equals_unfused(dims, kind):
    U = _gauge(dims, 11, kind)
    psi = _gauss(dims, 2, 12)
    W = oracle.twolink(U)
    for v in range(2):
        a = oracle.apply_lap(W, psi[v])
        b = oracle.apply_lap_unfused(U, psi[v])
        assert rel_l2(a, b) < 1e-14
    s1 = oracle.smear(W, psi, 4, 1.0)
    s2 = oracle.smear_unfused(U, psi, 4, 1.0)
    assert rel_l2(s1, s2) < 1e-14


# --------------------------------------------------------------------------- P2
def _fourier_smear(psi5, n, sigma):
    """Exact free-field smear through the plane-wave multiplier."""
    Lt, Lz, Ly, Lx, _ = psi5.shape
    kz = 2 * np.pi * np.arange(Lz) / Lz
    ky = 2 * np.pi * np.arange(Ly) / Ly
    kx = 2 * np.pi * np.arange(Lx) / Lx
    s2 = (np.sin(kz)[:, None, None] ** 2 + np.sin(ky)[None, :, None] ** 2
          + np.sin(kx)[None, None, :] ** 2)
    mult = (1.0 - (sigma / n) * s2) ** n
    f = np.fft.fftn(psi5, axes=(1, 2, 3))
    return np.fft.ifftn(f * mult[None, :, :, :, None], axes=(1, 2, 3))


@pytest.mark.parametrize("dims,n,sigma", [((8, 8, 8, 2), 10, 2.0), ((12, 8, 16, 1), 7, 1.3),
                                          ((6, 10, 4, 3), 3, 0.9)])
def test_p2_free_field_fourier(dims, n, sigma):
    U = _gauge(dims, 0, "unit")
    W = oracle.twolink(U)
    pt = synth.point_sources(dims, [(0, 0, 0, 0)], [0]).numpy()[0]
    g = _gauss(dims, 1, 3)[0]
    for psi in (pt, g):
        got = oracle.smear(W, psi, n, sigma)
        want = _fourier_smear(psi, n, sigma)
        assert rel_l2(got, want) < 1e-13


def _coef(j, m, half):
    """Coefficient of offset m (sublattice units, mod half) in (S + 1/S - 2)^j delta."""
    tot = 0
    for mm in range(-j, j + 1):
        if (mm - m) % half == 0:
            tot += (-1) ** ((j + mm) % 2) * math.comb(2 * j, j + mm)
    return tot


def test_p2_free_field_multinomial_exact():
    """(1 + a(Dx+Dy+Dz))^n delta expanded with integer binomials, a = sigma/(4n)."""
    L, n = 8, 5
    sigma = Fraction(3, 2)
    a = sigma / (4 * n)
    dims = (L, L, L, 1)
    W = oracle.twolink(_gauge(dims, 0, "unit"))
    psi = synth.point_sources(dims, [(0, 0, 0, 0)], [0]).numpy()[0]
    got = oracle.smear(W, psi, n, float(sigma))
    half = L // 2
    want = np.zeros((L, L, L))
    for mz, my, mx in itertools.product(range(half), repeat=3):
        val = Fraction(0)
        for jx in range(n + 1):
            for jy in range(n + 1 - jx):
                for jz in range(n + 1 - jx - jy):
                    j0 = n - jx - jy - jz
                    mult = math.factorial(n) // (math.factorial(j0) * math.factorial(jx)
                                                 * math.factorial(jy) * math.factorial(jz))
                    c = _coef(jx, mx, half) * _coef(jy, my, half) * _coef(jz, mz, half)
                    if c:
                        val += mult * a ** (jx + jy + jz) * c
        want[2 * mz, 2 * my, 2 * mx] = float(val)
    assert np.abs(got[0, ..., 1:]).max() == 0.0
    assert np.abs(got[0, ..., 0].imag).max() == 0.0
    assert np.abs(got[0, ..., 0].real - want).max() < 1e-15 * max(1.0, np.abs(want).max()) * 10


def test_p2_free_field_moments():
    """Sum conserved; per-axis second moment = 2 sigma; |x|^2 moment = 6 sigma (no wrap)."""
    L, n, sigma = 24, 5, 2.5
    dims = (L, L, L, 1)
    W = oracle.twolink(_gauge(dims, 0, "unit"))
    psi = synth.point_sources(dims, [(0, 0, 0, 0)], [0]).numpy()[0]
    out = oracle.smear(W, psi, n, sigma)[0, ..., 0].real
    assert abs(out.sum() - 1.0) < 1e-13
    off = np.where(np.arange(L) < L // 2, np.arange(L), np.arange(L) - L)
    z, y, x = np.meshgrid(off, off, off, indexing="ij")
    for c in (x, y, z):
        assert abs((c ** 2 * out).sum() - 2 * sigma) < 1e-12
        assert abs((c * out).sum()) < 1e-13
    assert abs(((x ** 2 + y ** 2 + z ** 2) * out).sum() - 6 * sigma) < 1e-12


def test_p2_lowest_mode():
    """U = 1, L divisible by 4: k = (pi/2, pi/2, pi/2) has Delta = -12 (Lap_two = -3)."""
    L = 8
    dims = (L, L, L, 1)
    W = oracle.twolink(_gauge(dims, 0, "unit"))
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    psi = np.zeros((1, L, L, L, 3), dtype=np.complex128)
    psi[0, ..., 1] = np.exp(0.5j * np.pi * (x + y + z))
    got = oracle.apply_lap(W, psi)
    assert rel_l2(got, -12.0 * psi) < 1e-14


def test_p2_two_site_extent_is_identity_on_free_field():
    """L = 2: x +- 2 = x, so on U = 1 each hop pair cancels the -2 and Delta = 0."""
    dims = (2, 2, 2, 2)
    W = oracle.twolink(_gauge(dims, 0, "unit"))
    psi = _gauss(dims, 1, 4)[0]
    assert np.abs(oracle.apply_lap(W, psi)).max() < 1e-14 * np.abs(psi).max()
    out = oracle.smear(W, psi, 5, 3.0)
    assert rel_l2(out, psi) < 1e-15


# --------------------------------------------------------------------------- P3
def _shift(a, axis, d):
    """a[x + d along axis] at x (periodic)."""
    return np.roll(a, -d, axis=axis)


@pytest.mark.parametrize("dims", [(4, 4, 4, 2), (6, 4, 8, 1)])
def test_p3_gauge_covariance(dims):
    U = _gauge(dims, 21, "haar", nd=3)
    G = synth.gauge_transform_haar(dims, 22).numpy()
    psi = _gauss(dims, 1, 23)[0]
    Ug = np.empty_like(U)
    for i, ax in enumerate((3, 2, 1)):  # x, y, z axes of [t, z, y, x]
        Gp = _shift(G, ax, 1)
        Ug[..., i, :, :] = G @ U[..., i, :, :] @ np.conj(np.swapaxes(Gp, -1, -2))
    psig = np.einsum("...ij,...j->...i", G, psi)
    W, Wg = oracle.twolink(U), oracle.twolink(Ug)
    # W transforms as G(x) W_i(x) G(x + 2i)^dag
    for i, ax in enumerate((3, 2, 1)):
        G2 = _shift(G, ax, 2)
        want = G @ W[..., i, :, :] @ np.conj(np.swapaxes(G2, -1, -2))
        assert rel_l2(Wg[..., i, :, :], want) < 1e-14
    a = oracle.smear(Wg, psig, 6, 2.0)
    b = np.einsum("...ij,...j->...i", G, oracle.smear(W, psi, 6, 2.0))
    assert rel_l2(a, b) < 1e-13


# --------------------------------------------------------------------------- P4
@pytest.mark.parametrize("dims,kind", [((4, 4, 4, 2), "haar"), ((6, 6, 2, 1), "near"),
                                        ((2, 2, 2, 1), "haar")])
def test_p4_hermitian_and_spectrum(dims, kind):
    U = _gauge(dims, 31, kind)
    W = oracle.twolink(U)
    phi, psi = _gauss(dims, 2, 32)
    dphi, dpsi = oracle.apply_lap(W, phi), oracle.apply_lap(W, psi)
    lhs = np.vdot(phi, dpsi)
    rhs = np.vdot(dphi, psi)
    assert abs(lhs - rhs) < 1e-14 * np.linalg.norm(phi) * np.linalg.norm(dpsi)
    q = np.vdot(psi, dpsi)
    nn = np.vdot(psi, psi).real
    assert abs(q.imag) < 1e-12 * nn
    assert -12.0 * nn - 1e-12 <= q.real <= 1e-12
    # (1 + (sigma/n) Lap_two) has spectrum in [1 - 3 sigma/n, 1]: contraction for sigma/n <= 2/3
    out = oracle.smear(W, psi, 8, 8 * 0.6)
    assert np.linalg.norm(out) <= np.linalg.norm(psi) * (1 + 1e-14)


# --------------------------------------------------------------------------- P5
@pytest.mark.parametrize("c", [0, 3, 5, 7])
def test_p5_sublattice_and_slice_decoupling(c):
    dims = (6, 4, 8, 3)
    t0 = 1
    W = oracle.twolink(_gauge(dims, 41, "haar"))
    psi = _gauss(dims, 1, 42)[0]
    mask = sublattice_mask(dims, c)
    src = psi.copy()
    src[t0][~mask] = 0.0
    out = oracle.smear(W, src, 7, 2.0, t0=t0)
    assert np.all(out[t0][~mask] == 0.0)
    assert np.abs(out[t0][mask]).max() > 0
    for t in range(dims[3]):
        if t != t0:
            assert np.array_equal(out[t], src[t])
    # A full-lattice smear restricted to one slice leaves the others bitwise alone.
    out2 = oracle.smear(W, psi, 3, 1.0, t0=t0)
    for t in range(dims[3]):
        if t != t0:
            assert np.array_equal(out2[t], psi[t])


# --------------------------------------------------------------------------- P6
def test_p6_trivial_cases_and_linearity():
    dims = (4, 6, 4, 2)
    W = oracle.twolink(_gauge(dims, 51, "near"))
    psi = _gauss(dims, 3, 52)
    assert np.array_equal(oracle.smear(W, psi, 0, 2.0), psi)
    assert np.array_equal(oracle.smear(W, psi, 5, 0.0), psi)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    lhs = oracle.smear(W, a * psi[0] + b * psi[1], 5, 2.0)
    rhs = a * oracle.smear(W, psi[0], 5, 2.0) + b * oracle.smear(W, psi[1], 5, 2.0)
    assert rel_l2(lhs, rhs) < 1e-14
    batch = oracle.smear(W, psi, 5, 2.0, t0=1)
    for v in range(3):
        assert np.array_equal(batch[v], oracle.smear(W, psi[v], 5, 2.0, t0=1))


# --------------------------------------------------------------------------- P7
@pytest.mark.parametrize("kind", ["near", "haar"])
def test_p7_su3_closure_of_twolink(kind):
    dims = (4, 4, 6, 2)
    W = oracle.twolink(_gauge(dims, 61, kind))
    eye = np.eye(3)
    WWd = W @ np.conj(np.swapaxes(W, -1, -2))
    assert np.abs(WWd - eye).max() < 1e-14
    assert np.abs(np.linalg.det(W) - 1).max() < 1e-14


def test_p7b_staggered_phases_leave_twolink_unchanged():
    """eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y) do not depend on x_mu, so they cancel."""
    dims = (4, 6, 4, 2)
    U = _gauge(dims, 71, "haar")
    Lx, Ly, Lz, Lt = dims
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    eta = [np.ones_like(x), (-1.0) ** x, (-1.0) ** (x + y)]
    Ue = U.copy()
    for mu in range(3):
        Ue[:, :, :, :, mu] *= eta[mu][None, :, :, :, None, None]
    assert not np.array_equal(U, Ue)
    assert np.array_equal(oracle.twolink(U), oracle.twolink(Ue))


# --------------------------------------------------------------------------- P8
def _dense_delta(U, dims):
    """Dense 3V x 3V matrix of Delta from Eq. tlLapl2, built site by site."""
    Lx, Ly, Lz, _ = dims
    V = Lx * Ly * Lz

    def idx(x, y, z):
        return (z % Lz) * Ly * Lx + (y % Ly) * Lx + (x % Lx)

    M = np.zeros((3 * V, 3 * V), dtype=np.complex128)
    for z, y, x in itertools.product(range(Lz), range(Ly), range(Lx)):
        s = idx(x, y, z)
        M[3 * s:3 * s + 3, 3 * s:3 * s + 3] -= 6 * np.eye(3)
        for mu in range(3):
            e = [0, 0, 0]
            e[mu] = 1
            p1 = (x + e[0], y + e[1], z + e[2])
            p2 = (x + 2 * e[0], y + 2 * e[1], z + 2 * e[2])
            m1 = (x - e[0], y - e[1], z - e[2])
            m2 = (x - 2 * e[0], y - 2 * e[1], z - 2 * e[2])
            u = lambda p: U[0, p[2] % Lz, p[1] % Ly, p[0] % Lx, mu]
            f = idx(*p2)
            b = idx(*m2)
            M[3 * s:3 * s + 3, 3 * f:3 * f + 3] += u((x, y, z)) @ u(p1)
            M[3 * s:3 * s + 3, 3 * b:3 * b + 3] += u(m1).conj().T @ u(m2).conj().T
    return M


@pytest.mark.parametrize("dims", [(2, 2, 2, 1), (4, 4, 4, 1), (4, 2, 6, 1)])
def test_p8_dense_bruteforce(dims):
    U = _gauge(dims, 81, "haar")
    W = oracle.twolink(U)
    psi = _gauss(dims, 1, 82)[0]
    n, sigma = 4, 1.7
    M = _dense_delta(U, dims)
    step = np.eye(M.shape[0]) + (sigma / (4 * n)) * M
    want = np.linalg.matrix_power(step, n) @ psi.reshape(-1)
    got = oracle.smear(W, psi, n, sigma)
    assert rel_l2(got.reshape(-1), want) < 1e-14
    # block structure: no matrix element joins different sublattices
    Lx, Ly, Lz, _ = dims
    sub = np.array([(x & 1) | ((y & 1) << 1) | ((z & 1) << 2)
                    for z in range(Lz) for y in range(Ly) for x in range(Lx)])
    sub3 = np.repeat(sub, 3)
    cross = sub3[:, None] != sub3[None, :]
    assert np.abs(M[cross]).max() == 0.0


def test_generator_reproducible_by_slice():
    """The input generators draw each slice from its own seed (needed for big lattices)."""
    dims = (4, 4, 4, 3)
    U = synth.gauge_near_unit(dims, 0.2, 5)
    U1 = synth.gauge_near_unit((4, 4, 4, 1), 0.2, 5)
    assert torch.equal(U[0], U1[0])



# --------------------------------------------------------------------------- one-link (Eq. 2-4)
@pytest.mark.parametrize("dims,n,alpha", [((8, 8, 8, 2), 6, 0.1), ((6, 10, 4, 1), 4, -0.05)])
def test_onelink_free_field_fourier(dims, n, alpha):
    """U = 1: a plane wave picks up (1 + alpha sum_mu 2 cos k_mu)^n."""
    U = _gauge(dims, 0, "unit")
    psi = _gauss(dims, 1, 91)[0]
    got = oracle.smear_onelink(U, psi, n, alpha)
    Lt, Lz, Ly, Lx, _ = psi.shape
    kz = 2 * np.pi * np.arange(Lz) / Lz
    ky = 2 * np.pi * np.arange(Ly) / Ly
    kx = 2 * np.pi * np.arange(Lx) / Lx
    c = (2 * np.cos(kz)[:, None, None] + 2 * np.cos(ky)[None, :, None] + 2 * np.cos(kx)[None, None, :])
    want = np.fft.ifftn(np.fft.fftn(psi, axes=(1, 2, 3)) * ((1 + alpha * c) ** n)[None, :, :, :, None],
                        axes=(1, 2, 3))
    assert rel_l2(got, want) < 1e-13


def test_onelink_hermitian_and_covariant():
    dims = (4, 6, 4, 2)
    U = _gauge(dims, 92, "haar", nd=3)
    phi, psi = _gauss(dims, 2, 93)
    hphi, hpsi = oracle.apply_hop(U, phi), oracle.apply_hop(U, psi)
    assert abs(np.vdot(phi, hpsi) - np.vdot(hphi, psi)) < 1e-14 * np.linalg.norm(phi) * np.linalg.norm(hpsi)
    G = synth.gauge_transform_haar(dims, 94).numpy()
    Ug = np.empty_like(U)
    for i, ax in enumerate((3, 2, 1)):
        Ug[..., i, :, :] = G @ U[..., i, :, :] @ np.conj(np.swapaxes(np.roll(G, -1, axis=ax), -1, -2))
    a = oracle.smear_onelink(Ug, np.einsum("...ij,...j->...i", G, psi), 5, 0.12)
    b = np.einsum("...ij,...j->...i", G, oracle.smear_onelink(U, psi, 5, 0.12))
    assert rel_l2(a, b) < 1e-13


def test_onelink_laplacian_rewrite():
    """Sec. 2: C(1 + alpha H)^n = C' (1 + alpha' Lap)^n, C' = C(1+6 alpha)^n, alpha' = alpha/(1+6 alpha).

    The right side is built from the one-link Laplacian Lap = H - 6 applied step by step.
    """
    dims = (4, 4, 6, 1)
    U = _gauge(dims, 95, "near")
    psi = _gauss(dims, 1, 96)[0]
    n, alpha = 5, 0.08
    lhs = oracle.smear_onelink(U, psi, n, alpha)
    ap = alpha / (1 + 6 * alpha)
    x = psi.copy()
    for _ in range(n):
        x = x + ap * (oracle.apply_hop(U, x) - 6 * x)
    assert rel_l2(lhs, (1 + 6 * alpha) ** n * x) < 1e-13


def test_twolink_is_the_straight_part_of_h_squared():
    """Sec. 2: the two-link hops are the straight two-step paths of the one-link hops.

    Each single hop (one direction, one sign) is written out here with numpy
    (roll + einsum).  Applying the same hop twice and summing over the six
    (direction, sign) pairs gives the straight +-2 mu paths, which must equal the
    oracle's (Delta + 6) psi (Eq. tlLapl1 / Eq. tlLapl2).  The sum of the six
    single hops must equal the oracle's H psi (Eq. 2).
    """
    dims = (6, 6, 6, 1)
    U = _gauge(dims, 97, "haar", nd=3)
    psi = _gauss(dims, 1, 98)[0]
    W = oracle.twolink(U)
    two = oracle.apply_lap(W, psi) + 6 * psi
    # straight two-step paths from single hops: forward-forward and backward-backward per direction
    def hop_dir(vec, mu, sign):
        out = np.zeros_like(vec)
        ax = (3, 2, 1)[mu]
        if sign > 0:
            out = np.einsum("...ij,...j->...i", U[..., mu, :, :], np.roll(vec, -1, axis=ax))
        else:
            Um = np.roll(U[..., mu, :, :], 1, axis=ax)
            out = np.einsum("...ji,...j->...i", np.conj(Um), np.roll(vec, 1, axis=ax))
        return out
    straight = sum(hop_dir(hop_dir(psi, mu, s), mu, s) for mu in range(3) for s in (1, -1))
    assert rel_l2(two, straight) < 1e-14
    # and the full one-link H is the sum of the six single hops
    h = sum(hop_dir(psi, mu, s) for mu in range(3) for s in (1, -1))
    assert rel_l2(oracle.apply_hop(U, psi), h) < 1e-14


# --------------------------------------------------------------------------- APE
# Gauge-smeared links (Sec. 2, the remark after Eq. tlSmear): APE smearing with
# the spatial staples and projection onto SU(3).
def _svd_su3(M):
    """Independent projection: unitary polar factor from numpy's SVD, det phase removed."""
    u, _, vh = np.linalg.svd(M)
    W = u @ vh
    ph = np.exp(-1j * np.angle(np.linalg.det(W)) / 3)
    return W * ph[..., None, None]


def test_ape_projection_is_the_polar_factor():
    rng = np.random.default_rng(51)
    M = rng.normal(size=(40, 3, 3)) + 1j * rng.normal(size=(40, 3, 3))
    P = oracle.su3_project(M)
    assert np.abs(P - _svd_su3(M)).max() < 1e-12
    # a positive multiple of an SU(3) matrix projects back onto it
    S = _gauge((2, 2, 2, 1), 52, "haar", nd=3)[0, 0, 0, 0]
    assert np.abs(oracle.su3_project(2.5 * S) - S).max() < 1e-13


def test_ape_identity_cases():
    dims = (4, 4, 4, 2)
    U = _gauge(dims, 53, "haar", nd=4)
    assert np.abs(oracle.ape_smear(U, 0.0, 3) - U[..., :3, :, :]).max() < 1e-13
    assert np.array_equal(oracle.ape_smear(U, 0.7, 0), U[..., :3, :, :])
    one = synth.gauge_unit(dims, nd=3).numpy()
    assert np.abs(oracle.ape_smear(one, 0.6, 4) - one).max() < 1e-14


def test_ape_pure_gauge_is_invariant():
    """U_mu(x) = G(x) G(x+mu)^dag has unit plaquettes: every staple equals the link."""
    dims = (4, 6, 4, 2)
    G = synth.gauge_transform_haar(dims, 54).numpy()
    U = np.empty(G.shape[:4] + (3, 3, 3), dtype=np.complex128)
    for i, ax in enumerate((3, 2, 1)):
        U[..., i, :, :] = G @ np.conj(np.swapaxes(_shift(G, ax, 1), -1, -2))
    assert np.abs(oracle.ape_smear(U, 0.6, 3) - U).max() < 1e-12


def test_ape_gauge_covariance():
    dims = (4, 4, 6, 2)
    U = _gauge(dims, 55, "haar", nd=3)
    G = synth.gauge_transform_haar(dims, 56).numpy()

    def transform(A):
        out = np.empty_like(A)
        for i, ax in enumerate((3, 2, 1)):
            out[..., i, :, :] = G @ A[..., i, :, :] @ np.conj(np.swapaxes(_shift(G, ax, 1), -1, -2))
        return out

    a = oracle.ape_smear(transform(U), 0.45, 2)
    b = transform(oracle.ape_smear(U, 0.45, 2))
    assert np.abs(a - b).max() < 1e-12


def test_ape_single_excited_link():
    """All links 1 except U_x at the origin = R: the staples that contain R are
    known by hand, and their projections are taken with numpy's SVD."""
    dims = (4, 4, 4, 1)
    U = synth.gauge_unit(dims, nd=3).numpy().copy()
    R = _gauge((2, 2, 2, 1), 57, "haar", nd=3)[0, 0, 0, 0, 0]
    U[0, 0, 0, 0, 0] = R  # [t, z, y, x, mu]
    a = 0.4
    out = oracle.ape_smear(U, a, 1)
    I = np.eye(3)
    expect = {
        # link (x, y, z, mu): V before projection
        (0, 0, 0, 0): (1 - a) * R + a * I,                      # its own staples are all 1
        (0, 0, 0, 1): (1 - a) * I + a / 4 * (R + 3 * I),        # forward nu = x staple: R 1 1^dag
        (1, 0, 0, 1): (1 - a) * I + a / 4 * (R.conj().T + 3 * I),  # backward nu = x staple: R^dag 1 1
        (0, 1, 0, 0): (1 - a) * I + a / 4 * (R + 3 * I),        # backward nu = y staple: 1^dag R 1
        (0, 3, 0, 0): (1 - a) * I + a / 4 * (R + 3 * I),        # forward nu = y staple: 1 R 1^dag
        (0, 0, 1, 0): (1 - a) * I + a / 4 * (R + 3 * I),        # backward nu = z staple
        (2, 2, 2, 0): I,                                        # far from the origin
    }
    for (x, y, z, mu), V in expect.items():
        assert np.abs(out[0, z, y, x, mu] - _svd_su3(V)).max() < 1e-13, (x, y, z, mu)


def test_ape_output_is_su3():
    U = _gauge((4, 4, 4, 2), 58, "haar", nd=4)
    A = oracle.ape_smear(U, 0.5, 3)
    assert np.abs(A @ np.conj(np.swapaxes(A, -1, -2)) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(A) - 1).max() < 1e-13


# --------------------------------------------------------------------------- input recipe
# The seeded stand-ins for the paper's configurations and sources (Sec. 3-4, 6).
@pytest.mark.parametrize("kind", ["near", "haar"])
def test_inputs_links_are_su3(kind):
    U = _gauge((4, 6, 4, 2), 81, kind, eps=0.3, nd=4)
    eye = np.eye(3)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - eye).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_inputs_haar_links_have_the_haar_trace_moments():
    """Haar measure on SU(3): E[tr U] = 0, E[|tr U|^2] = 1 (the fundamental
    representation is irreducible) and E[(tr U)^3] = 1 (3 x 3 x 3 holds the
    trivial representation once, the determinant; on U(3) this would be 0).
    65,536 links; the standard errors are about 0.004, 0.004 and 0.01."""
    U = _gauge((16, 16, 16, 4), 84, "haar", nd=4).reshape(-1, 3, 3)
    tr = np.trace(U, axis1=-2, axis2=-1)
    assert abs(tr.mean()) < 0.02
    assert abs((np.abs(tr) ** 2).mean() - 1) < 0.02
    assert abs((tr ** 3).mean() - 1) < 0.06


def test_inputs_near_unit_links_scale_with_eps():
    """exp(i eps H) with unit-variance Gell-Mann coefficients: |U - 1| grows like eps."""
    d1 = np.abs(_gauge((4, 4, 4, 1), 82, "near", eps=0.05) - np.eye(3)).mean()
    d2 = np.abs(_gauge((4, 4, 4, 1), 82, "near", eps=0.10) - np.eye(3)).mean()
    assert 1.8 < d2 / d1 < 2.2


def test_inputs_corner_walls():
    """24 vectors = 3 colours x 8 corners on slice 0; each one sublattice, unit colour vector."""
    dims = (6, 4, 8, 3)
    src = synth.corner_wall_sources(dims).numpy()
    assert src.shape == (24,) + (3, 8, 4, 6, 3)
    for c in range(8):
        for a in range(3):
            v = src[3 * c + a]
            assert np.array_equal(v[1:], np.zeros_like(v[1:]))  # only t = 0
            mask = sublattice_mask(dims, c)                     # sites of corner c on a slice
            assert np.array_equal(v[0][..., a] != 0, mask)
            assert np.all(v[0][mask][:, a] == 1) and np.all(np.delete(v[0][mask], a, axis=-1) == 0)
    assert src.sum() == 3 * dims[0] * dims[1] * dims[2]  # every site of slice 0 once per colour


def test_inputs_gaussian_vectors_moments():
    x = synth.gaussian_vectors((8, 8, 8, 2), 4, 83).numpy()
    assert abs(x.real.mean()) < 0.02 and abs(x.imag.mean()) < 0.02
    assert abs(x.real.var() - 1) < 0.03 and abs(x.imag.var() - 1) < 0.03
    only = synth.gaussian_vectors((8, 8, 8, 3), 2, 83, t=1).numpy()
    assert np.count_nonzero(only[:, 0]) == 0 and np.count_nonzero(only[:, 2]) == 0

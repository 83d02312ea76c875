"""Pins of the oracle's Wilson-Dirac operator (Eqs. (3)-(7)) to closed forms and invariants."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import wilson as W
from oracle import spectrum
from paper_2608_03515_b300 import fixtures as fx


def random_links(Nt, Nx, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))


def free_momentum_operator(m0, pt, px):
    """Momentum-space form of Eq. (3) at U = 1, derived by hand:
    a plane wave e^{i p.n} u is mapped to e^{i p.n} D(p) u with
    D(p) = (m0 + sum_mu (1 - cos p_mu)) I + i sum_mu sigma_mu sin p_mu,
    sigma_0 attached to the t momentum and sigma_1 to the x momentum."""
    s0 = np.array([[0, 1], [1, 0]], dtype=complex)
    s1 = np.array([[0, -1j], [1j, 0]], dtype=complex)
    return ((m0 + (1 - np.cos(pt)) + (1 - np.cos(px))) * np.eye(2)
            + 1j * (s0 * np.sin(pt) + s1 * np.sin(px)))


@pytest.mark.parametrize("Nt,Nx", [(8, 8), (6, 10)])
def test_free_field_spectrum_closed_form(Nt, Nx):
    m0 = 0.3
    U = np.ones((2, Nt, Nx), dtype=complex)
    lam = np.linalg.eigvals(W.dirac_matrix(U, m0).toarray())
    expect = []
    for kt in range(Nt):
        pt = np.pi * (2 * kt + 1) / Nt            # antiperiodic in t (Eq. (7))
        for kx in range(Nx):
            px = 2 * np.pi * kx / Nx              # periodic in x
            re = m0 + (1 - np.cos(pt)) + (1 - np.cos(px))
            im = np.sqrt(np.sin(pt) ** 2 + np.sin(px) ** 2)
            expect += [re + 1j * im, re - 1j * im]
    key = lambda z: (round(z.real, 9), round(z.imag, 9))
    a = np.array(sorted(lam, key=key))
    b = np.array(sorted(expect, key=key))
    assert np.max(np.abs(a - b)) < 1e-12


def test_free_field_plane_waves_fix_the_spin_structure():
    """D acting on plane waves equals the momentum-space matrix: fixes which
    Pauli matrix goes with which direction and the sign of each hop."""
    Nt, Nx, m0 = 6, 8, -0.2
    U = np.ones((2, Nt, Nx), dtype=complex)
    t = np.arange(Nt)[:, None]
    x = np.arange(Nx)[None, :]
    rng = np.random.Generator(np.random.PCG64(5))
    for kt, kx in [(0, 0), (1, 3), (2, 5), (5, 7)]:
        pt = np.pi * (2 * kt + 1) / Nt
        px = 2 * np.pi * kx / Nx
        u = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        phase = np.exp(1j * (pt * t + px * x))
        psi = np.stack([u[0] * phase, u[1] * phase])
        got = W.apply_dirac(U, m0, psi)
        Du = free_momentum_operator(m0, pt, px) @ u
        want = np.stack([Du[0] * phase, Du[1] * phase])
        assert np.max(np.abs(got - want)) < 1e-13
        got_sparse = W.from_flat(W.dirac_matrix(U, m0) @ W.to_flat(psi), Nt, Nx)
        assert np.max(np.abs(got_sparse - want)) < 1e-13


def test_sigma3_hermiticity_and_conjugate_pairs():
    U = random_links(6, 8, 1)
    D = W.dirac_matrix(U, 0.1)
    S = W.sigma3_full(48)
    assert abs(S @ D @ S - D.conj().T).max() == 0.0        # Eq. (6), exact
    lam = np.linalg.eigvals(D.toarray())
    # eigenvalues come in complex-conjugate pairs
    for z in lam:
        assert np.min(np.abs(lam - np.conj(z))) < 1e-10


def test_gauge_covariance():
    Nt, Nx = 8, 6
    U = random_links(Nt, Nx, 2)
    rng = np.random.Generator(np.random.PCG64(3))
    omega = np.exp(1j * rng.uniform(-np.pi, np.pi, size=(Nt, Nx)))
    U2 = W.gauge_transform_links(U, omega)
    D1 = W.dirac_matrix(U, 0.05)
    D2 = W.dirac_matrix(U2, 0.05)
    Om = sp.diags(np.repeat(omega.reshape(-1), 2))
    assert abs(D2 - Om @ D1 @ Om.conj().T).max() < 1e-14


def test_matrix_free_equals_sparse_and_k_formulation():
    Nt, Nx = 8, 8
    U = random_links(Nt, Nx, 4)
    D = W.dirac_matrix(U, 0.2)
    psi = fx.gaussian_rhs(1, Nt, Nx, 9)[0]
    a = W.apply_dirac(U, 0.2, psi)
    b = W.from_flat(D @ W.to_flat(psi), Nt, Nx)
    assert np.max(np.abs(a - b)) < 1e-14
    # K-formulation (Sec. 4.2): the real 2n system has the same solution
    K = W.k_formulation(D)
    f = W.to_flat(psi)
    fr = np.empty(2 * f.size)
    fr[0::2], fr[1::2] = f.real, f.imag
    ur = spla.spsolve(K.tocsc(), fr)
    u = spla.spsolve(D.tocsc(), f)
    assert np.max(np.abs((ur[0::2] + 1j * ur[1::2]) - u)) < 1e-12 * np.max(np.abs(u))


def test_boundary_signs_by_translation():
    """Eq. (7): shifting a field by one step in t across the boundary flips its
    sign.  With uniform links, D commutes with the antiperiodic translation."""
    Nt, Nx = 6, 4
    U = np.ones((2, Nt, Nx), dtype=complex)
    psi = fx.gaussian_rhs(1, Nt, Nx, 11)[0]

    def shift_t(f):
        g = np.roll(f, -1, axis=1)
        g[:, Nt - 1, :] *= -1.0          # psi(N_t - 1 + 1) = -psi(0)
        return g

    lhs = W.apply_dirac(U, 0.1, shift_t(psi))
    rhs = shift_t(W.apply_dirac(U, 0.1, psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-14


@pytest.mark.parametrize("Nt,Nx", [(8, 8), (48, 48)])
def test_free_field_critical_mass(Nt, Nx):
    """At U = 1 the smallest real part of the spectrum at m0 = 0 is 1 - cos(pi/N_t)."""
    U = np.ones((2, Nt, Nx), dtype=complex)
    mc = spectrum.critical_mass(U)
    assert abs(mc - (-(1 - np.cos(np.pi / Nt)))) < 1e-8


@pytest.mark.parametrize("L,beta,seed", [(32, 3.0, 0), (40, 6.0, 2)])
def test_arnoldi_critical_mass_matches_dense(L, beta, seed):
    U = fx.links_from_angles(fx.metropolis_u1(L, L, beta, 200, seed))
    assert abs(spectrum.critical_mass(U, dense=False) - spectrum.critical_mass(U, dense=True)) < 1e-6


def test_arnoldi_critical_mass_matches_dense_at_64():
    """The Arnoldi route that tabulates the fields of 128^2 and more, against
    all eigenvalues of the dense 8192 x 8192 operator of two 64^2 fields (the
    benchmark coupling and the weak coupling of the 1024^2 workload), at both
    tolerances it is used with (tests/golden/make_mcrit_dense.py)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mcrit_dense.json")
    table = json.load(open(path))
    assert len(table) >= 1
    for key, e in table.items():
        assert e["m_crit"] < 0.0
        for tol, mc in e["arpack"].items():
            assert abs(mc - e["m_crit"]) < 1e-9, (key, tol, mc, e["m_crit"])

"""Checks of the synthetic input generators (quenched U(1) Metropolis, Gaussian RHS)."""
import numpy as np
import pytest
import scipy.special as ss

from paper_2608_03515_b300 import fixtures as fx


def total_action(theta, beta):
    return beta * np.sum(1.0 - np.cos(fx.plaquette_angles(theta)))


def test_local_staples_match_global_action_difference():
    """The two-plaquette local action used by the update equals the change of the total action."""
    rng = np.random.Generator(np.random.PCG64(40))
    theta = rng.uniform(-np.pi, np.pi, size=(2, 6, 8))
    beta = 1.7
    for mu in (0, 1):
        A, B = fx._local_angles_mu0(theta) if mu == 0 else fx._local_angles_mu1(theta)
        for (t, x) in [(0, 0), (5, 7), (2, 3)]:
            d = 0.37
            th2 = theta.copy()
            th2[mu, t, x] += d
            old, new = theta[mu, t, x], th2[mu, t, x]
            if mu == 0:
                loc = lambda v: -np.cos(v + A[t, x]) - np.cos(B[t, x] - v)
            else:
                loc = lambda v: -np.cos(A[t, x] - v) - np.cos(v + B[t, x])
            dS_loc = beta * (loc(new) - loc(old))
            dS_glob = total_action(th2, beta) - total_action(theta, beta)
            assert abs(dS_loc - dS_glob) < 1e-12


@pytest.mark.parametrize("beta", [3.0, 6.0])
def test_mean_plaquette_matches_exact_2d_u1(beta):
    """2D U(1), plaquette action: <cos theta_P> = I_1(beta) / I_0(beta) (infinite volume)."""
    theta, hist = fx.metropolis_u1(32, 32, beta, 600, 0, return_history=True)
    meas = hist[200:]
    exact = ss.iv(1, beta) / ss.iv(0, beta)
    # error from blocks of 40 sweeps (autocorrelation-safe), then 4 sigma + small bias allowance
    blocks = meas[: len(meas) // 40 * 40].reshape(-1, 40).mean(axis=1)
    sigma = blocks.std(ddof=1) / np.sqrt(len(blocks))
    assert abs(meas.mean() - exact) < 4 * sigma + 2e-3


def test_generators_are_seeded_and_shaped():
    a = fx.metropolis_u1(8, 8, 2.0, 20, 3)
    b = fx.metropolis_u1(8, 8, 2.0, 20, 3)
    assert a.shape == (2, 8, 8) and np.array_equal(a, b)
    U = fx.links_from_angles(a)
    assert np.allclose(np.abs(U), 1.0)
    psi = fx.gaussian_rhs(3, 8, 4, 1)
    assert psi.shape == (3, 2, 8, 4) and psi.dtype == np.complex128
    assert np.array_equal(psi, fx.gaussian_rhs(3, 8, 4, 1))

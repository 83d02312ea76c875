"""Pins of the oracle's FGMRES and of the whole preconditioned solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import amg, krylov
from oracle import wilson as W
from paper_2608_03515_b300 import fixtures as fx


def random_links(Nt, Nx, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(1j * rng.uniform(-np.pi, np.pi, size=(2, Nt, Nx)))


def test_identity_preconditioner_reproduces_gmres():
    """M = I: flexible GMRES is plain restarted GMRES; compare with scipy's GMRES."""
    Nt = Nx = 8
    D = W.dirac_matrix(random_links(Nt, Nx, 30), 0.4)
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 31)[0])
    res = krylov.fgmres(lambda v: D @ v, lambda v: v, b, 10, 1e-10, 2000)
    assert res.converged and res.true_relres <= 1e-10
    hist = []
    x, info = spla.gmres(D, b, restart=10, rtol=1e-10, atol=0.0, maxiter=200,
                         callback=lambda pr: hist.append(pr), callback_type="pr_norm")
    assert info == 0
    # same Krylov spaces: same number of inner steps to reach the tolerance (+-1 for
    # the different stopping bookkeeping) and the same solution
    assert abs(len(hist) - res.iterations) <= 1
    xs = np.linalg.solve(D.toarray(), b)
    assert np.linalg.norm(res.x - xs) <= 1e-8 * np.linalg.norm(xs)
    # first restart cycle: relative residual estimates coincide with scipy's
    k = min(9, len(hist))
    assert np.allclose(res.estimates[:k], hist[:k], rtol=1e-6)


def test_exact_preconditioner_converges_in_one_step():
    Nt = Nx = 8
    D = W.dirac_matrix(random_links(Nt, Nx, 32), 0.1)
    Dd = D.toarray()
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 33)[0])
    res = krylov.fgmres(lambda v: D @ v, lambda v: np.linalg.solve(Dd, v), b, 30, 1e-10, 100)
    assert res.iterations == 1 and res.converged


def test_residual_estimate_non_increasing_within_cycle():
    Nt = Nx = 16
    D = W.dirac_matrix(random_links(Nt, Nx, 34), 0.05)
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 35)[0])
    m = 20
    res = krylov.fgmres(lambda v: D @ v, lambda v: v, b, m, 1e-10, 400)
    est = np.array(res.estimates)
    for start in range(0, len(est), m):
        cyc = est[start:start + m]
        assert np.all(np.diff(cyc) <= 1e-14)


@pytest.mark.parametrize("aggs", [[2], [4], [2, 2]])
def test_amg_preconditioned_solve_matches_dense_lu(aggs):
    Nt = Nx = 8
    D = W.dirac_matrix(random_links(Nt, Nx, 36), 0.1)
    levels = amg.build_hierarchy(D, Nt, Nx, aggs)
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 37)[0])
    res = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 500)
    xs = np.linalg.solve(D.toarray(), b)
    assert res.converged and res.true_relres <= 1e-10
    assert np.linalg.norm(res.x - xs) <= 1e-9 * np.linalg.norm(xs)
    # the preconditioner helps: fewer steps than plain GMRES
    plain = krylov.fgmres(lambda v: D @ v, lambda v: v, b, 30, 1e-10, 2000)
    assert res.iterations < plain.iterations


def test_cgnr_equals_cg_on_the_normal_equations_and_solves_the_system():
    """CGNR's iterates are those of CG applied to D^H D x = D^H b: after k steps
    they equal the minimiser of ||b - D x|| over the Krylov space
    K_k(D^H D, D^H b), which a dense least-squares solve in that space gives;
    run to the tolerance, the solution matches the dense solve of D x = b, and
    D^H taken as sigma_3 D sigma_3 (Eq. (6)) gives the same iterates."""
    Nt = Nx = 8
    D = W.dirac_matrix(random_links(Nt, Nx, 35), 0.3)
    Dd = D.toarray()
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 36)[0])
    AH = lambda v: D.conj().T @ v
    for k in (1, 3, 6):
        res = krylov.cgnr(lambda v: D @ v, AH, b, 1e-300, k)
        assert res.iterations == k
        # dense Krylov basis of D^H D from D^H b, orthonormalised, then least squares
        N = Dd.conj().T @ Dd
        Kb = [Dd.conj().T @ b]
        for _ in range(k - 1):
            Kb.append(N @ Kb[-1])
        Q, _ = np.linalg.qr(np.stack(Kb, axis=1))
        y, *_ = np.linalg.lstsq(Dd @ Q, b, rcond=None)
        xk = Q @ y
        assert np.linalg.norm(res.x - xk) <= 1e-8 * np.linalg.norm(xk)
    res = krylov.cgnr(lambda v: D @ v, AH, b, 1e-10, 5000)
    assert res.converged and res.true_relres <= 1e-10
    xs = np.linalg.solve(Dd, b)
    assert np.linalg.norm(res.x - xs) <= 1e-7 * np.linalg.norm(xs)
    s3 = W.sigma3_full(Nt * Nx)
    res3 = krylov.cgnr(lambda v: D @ v, lambda v: s3 @ (D @ (s3 @ v)), b, 1e-10, 5000)
    assert res3.iterations == res.iterations
    assert np.linalg.norm(res3.x - res.x) <= 1e-10 * np.linalg.norm(res.x)


def test_classical_gram_schmidt_with_second_pass_pins():
    """gs="cgs2" (the GPU's default variant): with M = I it is GMRES like the
    modified form (same Krylov spaces, so the same solution and step count as
    scipy's GMRES); its second pass runs exactly when the first pass removed
    more than 1 - 1/sqrt(2) of ||w||; with the V-cycle it takes the modified
    form's step count on a Wilson problem."""
    Nt = Nx = 8
    D = W.dirac_matrix(random_links(Nt, Nx, 40), 0.4)
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 41)[0])
    r_m = krylov.fgmres(lambda v: D @ v, lambda v: v, b, 10, 1e-10, 2000)
    r_c = krylov.fgmres(lambda v: D @ v, lambda v: v, b, 10, 1e-10, 2000, gs="cgs2")
    assert r_c.converged and r_c.true_relres <= 1e-10
    assert r_c.iterations == r_m.iterations
    assert np.allclose(r_c.estimates, r_m.estimates, rtol=1e-8)
    xs = np.linalg.solve(D.toarray(), b)
    assert np.linalg.norm(r_c.x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert r_m.second_passes == 0
    # the criterion: an operator that maps v to (1 - eps) v + eps u leaves
    # about eps of w after projecting out v (second pass), the identity plus a
    # large orthogonal part leaves most of it (no second pass)
    n = 6
    e = np.eye(n, dtype=complex)
    for eps, want in ((1e-3, 1), (0.9, 0)):
        A = (1 - eps) * np.eye(n) + eps * np.roll(np.eye(n), 1, axis=0)
        res = krylov.fgmres(lambda v: A @ v, lambda v: v, e[0], 1, 1e-300, 1, gs="cgs2")
        assert res.second_passes == want, (eps, res.second_passes)
    with pytest.raises(ValueError):
        krylov.fgmres(lambda v: v, lambda v: v, e[0], 1, 1e-10, 1, gs="cgs1")
    # preconditioned by the V-cycle on a 16^2 Wilson problem: same step count
    Nt = Nx = 16
    D = W.dirac_matrix(random_links(Nt, Nx, 42), 0.05)
    levels = amg.build_hierarchy(D, Nt, Nx, [2, 2])
    b = W.to_flat(fx.gaussian_rhs(1, Nt, Nx, 43)[0])
    m1 = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 500)
    c1 = krylov.fgmres(lambda v: D @ v, lambda r: amg.vcycle(levels, r), b, 30, 1e-10, 500, gs="cgs2")
    assert m1.converged and c1.converged
    assert c1.iterations == m1.iterations
    assert np.linalg.norm(c1.x - m1.x) <= 1e-8 * np.linalg.norm(m1.x)

"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module draws the inputs of a Dirac solve and nothing else: quenched U(1)
gauge fields and Gaussian right-hand sides.  It holds none of the solver's
arithmetic (no Wilson operator, no interpolation, no Krylov step), so that the
oracle and the CUDA library receive identical inputs while sharing no code.

Lattice conventions (Sec. "Schwinger Model"): sites n = (n_t, n_x) with
0 <= n_t < N_t, 0 <= n_x < N_x; direction mu = 0 is t, mu = 1 is x.  A gauge
field is stored as link angles theta[mu, t, x] (float64) with
U_mu(n) = exp(i * theta[mu, n]).  The paper generates its fields with a
two-flavour HMC whose configurations are not public; the stand-in here is a
quenched Metropolis chain for the plaquette action, with the same lattice
shapes and random U(1) phases.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "plaquette_angles",
    "metropolis_u1",
    "links_from_angles",
    "gaussian_rhs",
    "field_seed_for",
]


def plaquette_angles(theta: np.ndarray) -> np.ndarray:
    """theta_P(n) = theta_0(n) + theta_1(n+0) - theta_0(n+1) - theta_1(n) (periodic links)."""
    th0, th1 = theta[0], theta[1]
    return th0 + np.roll(th1, -1, axis=0) - np.roll(th0, -1, axis=1) - th1


def _local_angles_mu0(theta):
    """For each t-link theta_0(n): the two plaquettes that contain it, written as
    theta_P = theta_0(n) + A(n) and theta_P' = B(n) - theta_0(n)."""
    th0, th1 = theta[0], theta[1]
    # plaquette P(n): th0(n) + th1(n+t) - th0(n+x) - th1(n)
    A = np.roll(th1, -1, axis=0) - np.roll(th0, -1, axis=1) - th1
    # plaquette P(n - x): th0(n-x) + th1(n-x+t) - th0(n) - th1(n-x)
    B = np.roll(th0, 1, axis=1) + np.roll(np.roll(th1, -1, axis=0), 1, axis=1) - np.roll(th1, 1, axis=1)
    return A, B


def _local_angles_mu1(theta):
    """Same for each x-link theta_1(n): theta_P = C(n) - theta_1(n) (plaquette P(n)) and
    theta_P' = theta_1(n) + E(n) (plaquette P(n - t))."""
    th0, th1 = theta[0], theta[1]
    # P(n): th0(n) + th1(n+t) - th0(n+x) - th1(n)
    C = th0 + np.roll(th1, -1, axis=0) - np.roll(th0, -1, axis=1)
    # P(n - t): th0(n-t) + th1(n) - th0(n-t+x) - th1(n-t)
    E = np.roll(th0, 1, axis=0) - np.roll(np.roll(th0, 1, axis=0), -1, axis=1) - np.roll(th1, 1, axis=0)
    return C, E


def metropolis_u1(Nt: int, Nx: int, beta: float, sweeps: int, seed: int,
                  return_history: bool = False):
    """Quenched U(1) gauge field from a Metropolis chain for S = beta * sum_P (1 - cos theta_P).

    Cold start (theta = 0); proposal theta' = theta + U(-eps, eps) with
    eps = min(pi, 2/sqrt(beta)); one hit per link; checkerboard order per sweep:
    t-links on even x, t-links on odd x, x-links on even t, x-links on odd t
    (links of one direction interact only with links of the same direction
    one step away across a shared plaquette, so each half set is independent).
    Random numbers: numpy PCG64(seed); per half update one full [Nt, Nx] array of
    proposals and one of uniforms, in that order.

    Returns theta[2, Nt, Nx] (float64, wrapped to (-pi, pi]); with
    return_history also the mean plaquette cos after every sweep.
    """
    if Nt % 2 or Nx % 2:
        raise ValueError("checkerboard Metropolis needs even Nt and Nx")
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = min(np.pi, 2.0 / np.sqrt(beta))
    theta = np.zeros((2, Nt, Nx))
    tt, xx = np.meshgrid(np.arange(Nt), np.arange(Nx), indexing="ij")
    hist = []
    for _ in range(sweeps):
        for mu in (0, 1):
            parity_coord = xx if mu == 0 else tt
            for par in (0, 1):
                mask = (parity_coord % 2) == par
                prop = rng.uniform(-eps, eps, size=(Nt, Nx))
                u = rng.uniform(0.0, 1.0, size=(Nt, Nx))
                old = theta[mu]
                new = old + prop
                if mu == 0:
                    A, B = _local_angles_mu0(theta)
                    s_old = -np.cos(old + A) - np.cos(B - old)
                    s_new = -np.cos(new + A) - np.cos(B - new)
                else:
                    C, E = _local_angles_mu1(theta)
                    s_old = -np.cos(C - old) - np.cos(old + E)
                    s_new = -np.cos(C - new) - np.cos(new + E)
                dS = beta * (s_new - s_old)
                accept = mask & (u < np.exp(-np.maximum(dS, 0.0)))
                theta[mu] = np.where(accept, new, old)
        if return_history:
            hist.append(float(np.mean(np.cos(plaquette_angles(theta)))))
    theta = np.angle(np.exp(1j * theta))
    if return_history:
        return theta, np.array(hist)
    return theta


def links_from_angles(theta: np.ndarray) -> np.ndarray:
    """U[mu, t, x] = exp(i theta) as complex128, the layout the library takes."""
    return np.exp(1j * theta).astype(np.complex128)


def gaussian_rhs(R: int, Nt: int, Nx: int, seed: int) -> np.ndarray:
    """psi[R, 2, Nt, Nx] complex128 with Re, Im iid N(0, 1), drawn Re-then-Im
    per element in [R][spin][t][x] order from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(size=(R, 2, Nt, Nx, 2))
    return (z[..., 0] + 1j * z[..., 1]).astype(np.complex128)


def gaussian_rhs_device(Nt: int, Nx: int, seed: int, device):
    """One right-hand side [2, Nt, Nx] complex128 drawn on the device (torch's
    Philox generator seeded with `seed`; Re, Im iid N(0, 1)) -- for request
    streams too large to draw on the host."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    z = torch.randn(2, 2, Nt, Nx, dtype=torch.float64, device=device, generator=g)
    return torch.complex(z[0], z[1]).contiguous()


def field_seed_for(k: int) -> int:
    """Seed of resident field k in the serving mix (fields 0..7 use seeds 10..17)."""
    return 10 + int(k)

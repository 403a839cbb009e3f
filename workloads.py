"""Workload descriptions and seeded synthetic inputs.

This module holds no arithmetic of the method: it only names the parameter
sets of the five workloads and draws the random numbers they need, so that
the CUDA path (through ``paper_2608_20657_b300``) and the FP64 oracle
(``oracle``) receive identical inputs.  Each side turns a description into
its own bath decomposition and its own initial unique variables.

Energies are in units of a reference energy 1.0 (hbar = 1).  ``gsn`` is the
collective coupling g*sqrt(N); ``detuning`` is eps_x - omega_cav; ``kappa``
the photon population decay rate.

Workloads
  w1  N=2, m=1 (high-T Drude-Lorentz), L=3, cavity start, dt 0.05 x 2000.
  w2  N=10, m=2 (Drude-Lorentz + 1 Matsubara), L=6, bright start,
      dt 0.02 x 5000.
  w3  N=100, m=2, L=8, detuning 0.02, gsn 0.1, lambda 0.02, kappa 0.01,
      upper-polariton start, dt 0.02 x 20000.
  w4  512 independent instances, seed 2608: N ~ U{2..64}, m ~ U{1,2},
      L ~ U{3..8}, static disorder sigma ~ U[0, 0.02] (one extra averaged
      channel per molecule), gsn ~ U[0.02, 0.15]; lambda 0.01, gamma 0.05,
      kT 0.025, resonant, no loss; upper-polariton start, dt 0.02 x 10000.
  w5  N=1000, m=4 (Drude-Lorentz + 3 Pade poles; lambda 0.03, gamma 0.02,
      kT 0.01), L=12, kappa 0.005, gsn 0.1, detuning 0.02; random
      permutation-invariant density matrix (seed 2608); dt 0.01 x 50000.
  sec5(N, init, d)  the paper's own production set (Sec. V), in physical
      units: energies in cm^-1, temperature in K, time in fs (see sec5).
"""
from __future__ import annotations

import numpy as np

SEED = 2608


def _w(name, N, L, scheme, lam, gam, kT, poles, sigma, gsn, detuning, kappa, init, dt, steps, **kw):
    d = dict(name=name, N=N, L=L, scheme=scheme, lam=lam, gam=gam, kT=kT, poles=poles, sigma=sigma, gsn=gsn,
             detuning=detuning, kappa=kappa, init=init, dt=dt, steps=steps)
    d.update(kw)
    return d


WORKLOADS = {
    "w1": _w("w1_N2_m1_L3", 2, 3, "high_t", 0.01, 0.05, 0.025, 0, 0.0, 0.05, 0.0, 0.0, "cavity", 0.05, 2000),
    "w2": _w("w2_N10_m2_L6", 10, 6, "matsubara", 0.01, 0.05, 0.025, 1, 0.0, 0.05, 0.0, 0.0, "bright", 0.02, 5000),
    "w3": _w("w3_N100_m2_L8", 100, 8, "matsubara", 0.02, 0.05, 0.025, 1, 0.0, 0.1, 0.02, 0.01, "up", 0.02, 20000),
    "w5": _w("w5_N1000_m4_L12", 1000, 12, "pade", 0.03, 0.02, 0.01, 3, 0.0, 0.1, 0.02, 0.005, "random", 0.01,
             50000, seed=SEED),
}


# Sec. V: the molecule numbers of Figs. 3-6 and the initial states of
# Secs. V.A-V.F (up: upper polariton; localised: |e_1><e_1|; superposed:
# sqrt(0.3)|e_1> + sqrt(0.7)|c>, the last two with molecule 1 distinguished)
SEC5_N = (5, 10, 25, 100, 1000, 10 ** 12)


def sec5(N: int, init: str = "up", d: int | None = None, steps: int = 4000) -> dict:
    """The paper's production parameters (Sec. V): resonant cavity and
    molecules (omega_cav = eps_x = 10000 cm^-1, so detuning 0), Rabi splitting
    Omega_R = 500 cm^-1 at every N (g = Omega_R / (2 sqrt N)), Drude-Lorentz
    bath lambda = 50 cm^-1, gamma = 18 cm^-1 at T = 300 K, one exponential per
    local bath (the gamma pole) with every Matsubara term left to the
    Ishizaki-Tanimura terminator, no cavity loss, depth L = 25, dt = 0.5 fs;
    4000 steps reach the 2 ps of Figs. 5-6."""
    if d is None:
        d = 1 if init in ("localised", "superposed") else 0
    return dict(name=f"sec5_N{N}_{init}", N=N, L=25, scheme="matsubara", poles=0, sigma=0.0, units="cm-1/fs",
                lam_cm=50.0, gam_cm=18.0, T_K=300.0, omega_R_cm=500.0, detuning_cm=0.0, kappa_cm=0.0,
                terminator=True, d=d, init=init, dt_fs=0.5, steps=steps)


def batch_w4(count: int = 512, seed: int = SEED) -> list[dict]:
    """The 512 seeded instances of w4 (uneven N, m, L)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(2, 65))
        m = int(rng.integers(1, 3))
        L = int(rng.integers(3, 9))
        sigma = float(rng.uniform(0.0, 0.02))
        gsn = float(rng.uniform(0.02, 0.15))
        out.append(_w(f"w4_{i}", N, L, "high_t" if m == 1 else "matsubara", 0.01, 0.05, 0.025, m - 1, sigma, gsn,
                      0.0, 0.0, "up", 0.02, 10000))
    return out


def random_rho_draws(seed: int = SEED) -> dict:
    """Random numbers for a random permutation-invariant density matrix: a
    2x2 complex Gaussian matrix (cavity / bright block) and a uniform dark
    weight.  Turning them into unique variables is each side's job."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    return {"A": a, "w_dark": float(rng.uniform(0.0, 1.0))}


def random_state(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded random complex vector (input of single right-hand-side
    checks, where any state is a valid input of the linear map)."""
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(n) + 1j * rng.standard_normal(n))


def sample_indices(n: int, count: int, seed: int) -> np.ndarray:
    """Seeded sorted sample of variable indices, always including both ends."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(n, size=min(count, n), replace=False)
    return np.unique(np.concatenate([idx, [0, n - 1]])).astype(np.int64)

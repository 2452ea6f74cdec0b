"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's callers.

This module only builds problem inputs (coordinate vectors, Hamiltonians,
spectral-density parameters, initial density matrices, random tensors).  It
holds none of the method's arithmetic and imports neither the CUDA binding nor
the oracle.  Random draws use numpy's PCG64 generator with the seeds stated
below.

Workloads (hbar = k_B = 1):

* ``spin_boson_L6``   M=2, s=(+1,-1), H=[[0,1],[1,0]], Ohmic J=(pi/2) 0.1 w e^{-w/7.5}, beta=5,
                      dt=0.25, Delta k_max=6 (4^6 = 4096-entry tensor), 100 steps, rho0=|0><0|.
* ``biased_L12``      M=2, H=[[0.5,1],[1,-0.5]], Ohmic alpha=0.3, wc=5, beta=1, dt=0.1,
                      Delta k_max=12 (16.8 M entries), 400 steps, rho0=|0><0|.
* ``three_level_L8``  M=3, s=(-1,0,1), seeded Hermitian H (seed 1205: diagonal N(0,1);
                      off-diagonal (a+ib)/sqrt2 with a,b ~ N(0,1), upper triangle in
                      row order), super-Ohmic J=0.05 w^3 e^{-(w/2)^2}, beta=2, dt=0.2,
                      Delta k_max=8 (9^8 = 43 M entries), 300 steps, rho0 = psi psi^dagger
                      with psi complex Gaussian (seed 6872), normalised.
* ``batched_256``     256 spin-boson instances (seed 0): Delta k_max ~ U{4..11},
                      alpha ~ U[0.01,0.5], wc ~ U[1,10], beta ~ U[0.2,10], eps ~ U[-1,1],
                      H=[[eps,1],[1,-eps]], Ohmic, dt=0.25, 200 steps each, rho0=|0><0|.
* ``spin_boson_L14``  M=2, H=[[0,1],[1,0]], Ohmic alpha=0.5, wc=2.5, beta=0.5, dt=0.15,
                      Delta k_max=14 (4^14 = 268 M entries), 1000 steps, rho0=|0><0|.
* ``quantum_dot``     the model system of Sec. III (driven quantum dot after the rotating-wave
                      approximation): s in {0, 1}, H = (1/2)[[0, W],[W, 0]] with W = pi/8 ps^-1,
                      J = A w^3 exp(-(w/wc)^2) with A = pi 0.027 ps^2 and wc = 2.2 ps^-1, T = 25 K
                      (beta = hbar/(k_B T) = 0.6582119569 meV ps / (0.08617333262 meV/K x 25 K) in ps),
                      Delta k_max = 11; time unit ps.  The paper does not state dt; 0.25 ps is used.
* ``pulse_area_sweep`` the same dot driven with W_j = theta_j / t_final for pulse areas
                      theta_j = 5 pi j / n (j = 1..n): rho at t_final only, one instance per area.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

OHMIC_EXP = "ohmic_exp"
SUPEROHMIC_GAUSS = "superohmic_gauss"


@dataclass
class Problem:
    name: str
    s: np.ndarray          # coordinate eigenvalues, length M
    H: np.ndarray          # M x M complex Hermitian
    jkind: str             # OHMIC_EXP | SUPEROHMIC_GAUSS
    ja: float              # alpha (Ohmic) or xi (super-Ohmic) prefactor
    wc: float              # cutoff frequency
    beta: float
    dt: float
    L: int                 # Delta k_max
    N: int                 # number of time steps
    rho0: np.ndarray       # M x M complex

    @property
    def M(self) -> int:
        return int(self.s.shape[0])

    @property
    def elements(self) -> int:
        """Entries of the augmented tensor, (M^2)^L."""
        return (self.M * self.M) ** self.L


def _pure0(M):
    r = np.zeros((M, M), dtype=np.complex128)
    r[0, 0] = 1.0
    return r


def spin_boson(name, eps, omega, alpha, wc, beta, dt, L, N):
    H = np.array([[eps, omega], [omega, -eps]], dtype=np.complex128)
    return Problem(name, np.array([1.0, -1.0]), H, OHMIC_EXP, alpha, wc, beta, dt, L, N, _pure0(2))


def random_hermitian(M: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    H = np.zeros((M, M), dtype=np.complex128)
    diag = rng.normal(size=M)
    for i in range(M):
        H[i, i] = diag[i]
    for i in range(M):
        for j in range(i + 1, M):
            a, b = rng.normal(size=2)
            H[i, j] = (a + 1j * b) / np.sqrt(2.0)
            H[j, i] = np.conj(H[i, j])
    return H


def random_pure_state(M: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    psi = rng.normal(size=M) + 1j * rng.normal(size=M)
    psi = psi / np.linalg.norm(psi)
    return np.outer(psi, psi.conj())


def spin_boson_L6() -> Problem:
    return spin_boson("spin_boson_L6", 0.0, 1.0, 0.1, 7.5, 5.0, 0.25, 6, 100)


def biased_L12() -> Problem:
    return spin_boson("biased_L12", 0.5, 1.0, 0.3, 5.0, 1.0, 0.1, 12, 400)


def three_level_L8() -> Problem:
    return Problem("three_level_L8", np.array([-1.0, 0.0, 1.0]), random_hermitian(3, 1205),
                   SUPEROHMIC_GAUSS, 0.05, 2.0, 2.0, 0.2, 8, 300, random_pure_state(3, 6872))


def spin_boson_L14() -> Problem:
    return spin_boson("spin_boson_L14", 0.0, 1.0, 0.5, 2.5, 0.5, 0.15, 14, 1000)


def batched_256(n: int = 256, seed: int = 0, N: int = 200, dt: float = 0.25):
    rng = np.random.Generator(np.random.PCG64(seed))
    L = rng.integers(4, 12, size=n)
    alpha = rng.uniform(0.01, 0.5, size=n)
    wc = rng.uniform(1.0, 10.0, size=n)
    beta = rng.uniform(0.2, 10.0, size=n)
    eps = rng.uniform(-1.0, 1.0, size=n)
    return [spin_boson(f"batched_{i}", float(eps[i]), 1.0, float(alpha[i]), float(wc[i]),
                       float(beta[i]), dt, int(L[i]), N) for i in range(n)]


def random_tensor(n_elements: int, seed: int) -> np.ndarray:
    """Complex Gaussian tensor (unit variance per component) for single-step tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(size=n_elements) + 1j * rng.normal(size=n_elements)


def random_eta(L: int, seed: int, scale: float = 0.05) -> np.ndarray:
    """A random 4L+3 eta vector (complex), for checks that do not need a physical bath."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * (rng.normal(size=4 * L + 3) + 1j * rng.normal(size=4 * L + 3))


HBAR_MEV_PS = 0.6582119569
KB_MEV_PER_K = 0.08617333262


def quantum_dot(L: int = 11, N: int = 1000, dt: float = 0.25, omega: float = np.pi / 8,
                temperature_K: float = 25.0, name: str = "quantum_dot") -> Problem:
    beta = HBAR_MEV_PS / (KB_MEV_PER_K * temperature_K)
    H = 0.5 * np.array([[0.0, omega], [omega, 0.0]], dtype=np.complex128)
    return Problem(name, np.array([0.0, 1.0]), H, SUPEROHMIC_GAUSS, np.pi * 0.027, 2.2, beta, dt, L, N,
                   _pure0(2))


def pulse_area_sweep(n: int = 64, L: int = 11, N: int = 200, dt: float = 0.25):
    t_final = N * dt
    return [quantum_dot(L=L, N=N, dt=dt, omega=5.0 * np.pi * (j + 1) / n / t_final, name=f"pulse_area_{j}")
            for j in range(n)]


CONFIGS = {
    "spin_boson_L6": spin_boson_L6,
    "biased_L12": biased_L12,
    "three_level_L8": three_level_L8,
    "spin_boson_L14": spin_boson_L14,
    "quantum_dot_L11": quantum_dot,
}

"""Seeded synthetic workloads shaped like the toy models of arXiv:2111.00050.

This module is shared by the CUDA path, the oracle and the tests.  It holds
only model and initial-state PARAMETERS (the dispersion w_p, the coupling
tensor of Eq. (Lambda), coherent / field-number amplitudes) and the seeded
random draws; none of the method's arithmetic (no Hamiltonian application, no
time stepping, no observables) lives here.

Coupling tensors are complex arrays L[p, q, r, s] (mode indices) with
L_{pq;rs} = Lambda^{rs}_{pq} / 2, the coefficient of a_p^dag a_q^dag a_r a_s in
the ordered sum of Eq. (Ham); entries that do not conserve momentum are zero
(modulo M by default; exactly, the plain label sum of Sec. III B, with
exact=True).  Mode index i carries momentum label i - (M-1)/2 for odd M (i for
even M).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


def mode_labels(M: int) -> np.ndarray:
    return np.arange(M) - (M - 1) // 2 if M % 2 else np.arange(M)


def _conserving(M: int, exact: bool = False) -> np.ndarray:
    lab = mode_labels(M)
    s = lab[:, None, None, None] + lab[None, :, None, None] - lab[None, None, :, None] - lab[None, None, None, :]
    return (s == 0) if exact else (s % M) == 0


def dispersion_quadratic(M: int) -> np.ndarray:
    """w_p = p^2 / 2 (Sec. IV A, long-range toy model)."""
    return mode_labels(M).astype(np.float64) ** 2 / 2


def dispersion_abs(M: int) -> np.ndarray:
    """Linear dispersion w_p = |p|."""
    return np.abs(mode_labels(M)).astype(np.float64)


def contact_coupling(M: int, C: float, exact: bool = False) -> np.ndarray:
    """Contact interaction L_{pq;rs} = C / M on every momentum-conserving tuple."""
    return np.where(_conserving(M, exact), C / M, 0.0).astype(np.complex128)


def long_range_coupling(M: int, G: float, exact: bool = False, min_image: bool = False) -> np.ndarray:
    """Gravity-like L_{pq;rs} = -G / (M d^2) for labels p != r, else 0, with
    d = p - r the raw label difference, or (min_image) its minimal image on the
    ring of M momenta, |d| <= M/2; the divergent p = r term is dropped."""
    lab = mode_labels(M).astype(np.float64)
    d = lab[:, None, None, None] - lab[None, None, :, None]
    if min_image:
        d = d - M * np.round(d / M)
    d = np.broadcast_to(d, (M, M, M, M))
    with np.errstate(divide="ignore"):
        val = np.where(d != 0, -G / (M * np.where(d != 0, d, 1.0) ** 2), 0.0)
    return np.where(_conserving(M, exact), val, 0.0).astype(np.complex128)


def paper_coupling(M: int, C: float, Lambda0: float) -> np.ndarray:
    """Eq. (Lambda) halved: L_{pl;ij} = C/(4(p_p-p_i)^2) + C/(4(p_p-p_j)^2) + Lambda0/2
    on conserving tuples, each divergent (p_p = p_i) term taken as zero."""
    lab = mode_labels(M).astype(np.float64)
    L = np.zeros((M, M, M, M), dtype=np.complex128)
    cons = _conserving(M)
    for p in range(M):
        for l in range(M):
            for i in range(M):
                for j in range(M):
                    if not cons[p, l, i, j]:
                        continue
                    v = Lambda0 / 2
                    if lab[p] != lab[i]:
                        v += C / (4 * (lab[p] - lab[i]) ** 2)
                    if lab[p] != lab[j]:
                        v += C / (4 * (lab[p] - lab[j]) ** 2)
                    L[p, l, i, j] = v
    return L


def poisson_nmax(n_tot: float) -> int:
    """Truncation N <= floor(n_tot + 6 sqrt(n_tot)) for Poisson-weighted sectors."""
    return int(math.floor(n_tot + 6.0 * math.sqrt(n_tot)))


@dataclasses.dataclass
class Workload:
    name: str
    M: int
    w: np.ndarray
    L: np.ndarray
    kind: str  # "number" | "coherent" | "field_number"
    dt: float
    steps: int
    obs_every: int
    occ: Optional[np.ndarray] = None  # number state
    z: Optional[np.ndarray] = None  # coherent / field-number amplitudes
    n_tot: Optional[int] = None  # field-number total
    n_min: int = 0
    n_max: int = 0
    sweep: Optional[np.ndarray] = None  # coupling scale factors of a batched sweep

    def sectors_hint(self):
        """(n_min, n_max) spanned by the initial state."""
        return self.n_min, self.n_max


def plain_single_sector() -> Workload:
    """M=5 ring, w=p^2/2, contact C=-0.1, number state (0,2,2,2,0) (N=6, P=0),
    RK4 dt=1e-3 to t=10, observables every 100 steps."""
    M = 5
    occ = np.array([0, 2, 2, 2, 0])
    return Workload("plain_single_sector_M5_N6", M, dispersion_quadratic(M), contact_coupling(M, -0.1), "number",
                    1e-3, 10000, 100, occ=occ, n_min=6, n_max=6)


def batched_coherent(n_tot: int = 16, dt: float = 1e-3, t_end: float = 20.0) -> Workload:
    """M=7, w=p^2/2, contact C=-0.05/n_tot, alpha = sqrt(n_tot/2) on p=-1 and p=+1,
    Poisson-weighted sectors N <= n_tot + 6 sqrt(n_tot)."""
    M = 7
    z = np.zeros(M, dtype=np.complex128)
    z[2] = z[4] = math.sqrt(n_tot / 2)
    return Workload(f"batched_coherent_M7_ntot{n_tot}", M, dispersion_quadratic(M),
                    contact_coupling(M, -0.05 / n_tot), "coherent", dt, int(round(t_end / dt)), 100, z=z,
                    n_min=0, n_max=poisson_nmax(n_tot))


def long_range_field_number(M: int = 9, seed: int = 0, mean: float = 3.0, dt: float = 1e-3,
                            t_end: float = 20.0) -> Workload:
    """w=p^2/2, L=-G/(M (p-r)^2) with G=0.1/n_tot, field number state with n_p ~ Poisson(mean)
    and phases ~ U[0, 2 pi) drawn in that order from numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    n = rng.poisson(mean, M)
    theta = rng.uniform(0.0, 2 * math.pi, M)
    z = np.sqrt(n) * np.exp(1j * theta)
    n_tot = int(n.sum())
    return Workload(f"long_range_field_number_M{M}_N{n_tot}", M, dispersion_quadratic(M),
                    long_range_coupling(M, 0.1 / n_tot), "field_number", dt, int(round(t_end / dt)), 100,
                    z=z, n_tot=n_tot, n_min=n_tot, n_max=n_tot, occ=n)


def adjoint_coherent(M: int = 5, C: float = -0.1, n_tot: float = 40.0, seed: int = 0, dt: float = 1e-3,
                     t_f: float = 5.0) -> Workload:
    """Contact C, alpha_p complex Gaussian (numpy default_rng(seed).standard_normal((M, 2)))
    rescaled to sum |alpha|^2 = n_tot; loss Q(t_f)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((M, 2))
    z = x[:, 0] + 1j * x[:, 1]
    z *= math.sqrt(n_tot / float(np.sum(np.abs(z) ** 2)))
    return Workload(f"adjoint_coherent_M{M}_ntot{n_tot:g}", M, dispersion_quadratic(M), contact_coupling(M, C),
                    "coherent", dt, int(round(t_f / dt)), 0, z=z, n_min=0, n_max=poisson_nmax(n_tot))


def large_sector(M: int = 11, N: int = 20, dt: float = 5e-4, t_end: float = 10.0) -> Workload:
    """M=11, w=|p|, contact C=-0.02, number state with N/3-ish particles on p in {-1, 0, +1}
    (7, 6, 7 at N=20; P=0), plus a sweep of 8 couplings C_k = -0.005 k."""
    c = (M - 1) // 2
    occ = np.zeros(M, dtype=np.int64)
    third = N // 3
    occ[c - 1] = occ[c + 1] = (N - third) // 2
    occ[c] = N - 2 * ((N - third) // 2)
    return Workload(f"large_sector_M{M}_N{N}", M, dispersion_abs(M), contact_coupling(M, -0.02), "number", dt,
                    int(round(t_end / dt)), 100, occ=occ, n_min=N, n_max=N,
                    sweep=np.array([0.25 * k for k in range(1, 9)]))


def large_field_number(M: int = 11, N: int = 20, seed: int = 0) -> Workload:
    """Field number state on p in {-1, 0, +1} with |z|^2 = N/3 each, phases from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    c = (M - 1) // 2
    z = np.zeros(M, dtype=np.complex128)
    th = rng.uniform(0.0, 2 * math.pi, 3)
    for k, i in enumerate((c - 1, c, c + 1)):
        z[i] = math.sqrt(N / 3) * np.exp(1j * th[k])
    return Workload(f"large_field_number_M{M}_N{N}", M, dispersion_abs(M), contact_coupling(M, -0.02),
                    "field_number", 5e-4, 20000, 100, z=z, n_tot=N, n_min=N, n_max=N)


def squeezing_coherent(n_tot: float, M: int = 7, G: float = 1.0, dt: float = 2e-3, t_end: float = 1.6,
                       obs_every: int = 10) -> Workload:
    """Sec. IV E's squeezing systems: quadratic dispersion, gravity-like long-range
    coupling of strength G, coherent state with a Gaussian momentum profile
    z_p ~ exp(-p^2 / 2) rescaled to sum |z_p|^2 = n_tot.  The paper holds the mean
    interaction energy per occupation at |n_tot chi| = 0.242 for every n_tot; for a
    fixed profile n_tot chi is proportional to G n_tot, so callers pick G from the
    value at G = 1."""
    lab = mode_labels(M).astype(np.float64)
    z = np.exp(-lab ** 2 / 2).astype(np.complex128)
    z *= math.sqrt(n_tot / float(np.sum(np.abs(z) ** 2)))
    return Workload(f"squeezing_coherent_M{M}_ntot{n_tot:g}", M, dispersion_quadratic(M), long_range_coupling(M, G),
                    "coherent", dt, int(round(t_end / dt)), obs_every, z=z, n_min=0, n_max=poisson_nmax(n_tot))


def breaktime_coherent(r: float, M: int = 5, g: float = 0.5, seed: int = 0, dt: float = 5e-3,
                       t_end: float = 30.0, obs_every: int = 20) -> Workload:
    """Sec. IV C-D's breaktime systems: quadratic dispersion, gravity-like long range,
    coherent state with average mode occupation r (|z_p|^2 = r on every mode, phases
    from numpy default_rng(seed).uniform(0, 2 pi, M)), n_tot = M r, and strength
    G = g / n_tot so that the mean-field dynamics is the same for every n_tot."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 2 * math.pi, M)
    z = math.sqrt(r) * np.exp(1j * th)
    n_tot = M * r
    return Workload(f"breaktime_coherent_M{M}_r{r:g}", M, dispersion_quadratic(M), long_range_coupling(M, g / n_tot),
                    "coherent", dt, int(round(t_end / dt)), obs_every, z=z, n_tot=n_tot, n_min=0,
                    n_max=poisson_nmax(n_tot))

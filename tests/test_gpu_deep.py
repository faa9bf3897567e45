"""Parity of the RK4 stages where the weighted basis and the batched launches are
stressed: deep sectors with large ket weights, long horizons against the exact
discrete scheme, and whole sectors of the full-size benchmark step.

The stage kernels hold f = psi / w(n), w(n) = sqrt(N! / prod n_m!) times a power of
two per N, as fp32 pairs; these cases reach weights up to 2^154 (M = 3, N = 200).
Tolerance: relative 2-norm state error <= 1e-10 against the oracle's classic RK4
(or the RK4 polynomial applied in each sector's eigenbasis).
"""
import numpy as np
import pytest

import oracle as orc
import workloads as wl
from helpers import pair, rel_err, to_dev, to_host, random_state

pytestmark = pytest.mark.gpu

STATE_TOL = 1e-10


def _deep_case(name):
    if name == "M3_N200":  # one sector of 6,767 kets, ket weights up to 2^154
        M = 3
        return M, wl.dispersion_quadratic(M), wl.contact_coupling(M, -0.02), 200, [0], 20
    if name == "M5_N77":  # the deepest layer of the adjoint workload: 332,748 kets, weights up to 2^83
        M = 5
        return M, wl.dispersion_quadratic(M), wl.contact_coupling(M, -0.1), 77, [0], 2
    if name == "M5_N40_deep":
        M = 5
        return M, wl.dispersion_quadratic(M), wl.contact_coupling(M, -0.1), 40, [1], 20
    raise KeyError(name)


@pytest.mark.parametrize("name", ["M3_N200", "M5_N77", "M5_N40_deep"])
def test_deep_sector_evolution_matches_oracle(name):
    """qb_evolve (stage launches, weighted basis) on one deep sector from a random
    state against the oracle's classic RK4."""
    M, w, L, N, plist, steps = _deep_case(name)
    qs, os_ = pair(M, w, L, N, N, plist)
    x = random_state(qs.total, 23)
    psi = to_dev(x)
    qs.set_resident_max(0)
    qs.evolve(psi, 1e-3, steps)
    ref = orc.rk4(os_, w, L, x, 1e-3, steps)
    assert rel_err(to_host(psi), ref) <= STATE_TOL


def _eigen_rk4(os_, w, L, psi0, dt, steps):
    """steps RK4 steps applied in each sector's eigenbasis: V R(-i lam dt)^k V^dag psi0
    with R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, H from the oracle's dense sector matrix."""
    out = np.zeros_like(psi0)
    for s in range(len(os_.sectors)):
        sl = os_.sector_slice(s)
        lam, V = np.linalg.eigh(orc.h_dense(os_, s, w, L))
        z = -1j * lam * dt
        R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
        out[sl] = V @ (R ** steps * (V.conj().T @ psi0[sl]))
    return out


@pytest.mark.parametrize("resident", [0, 1024])
def test_long_horizon_coherent_multi_sector(resident):
    """2 x 10^4 steps of a coherent state over every sector N <= 8 (M = 5, 41
    sectors), against the RK4 polynomial in each sector's eigenbasis; with
    resident_max 0 every step goes through the graph-replayed stage launches."""
    M = 5
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.15)
    qs, os_ = pair(M, w, L, 0, 8)
    z = np.array([0.4, 0.9j, 1.0, -0.6 + 0.3j, 0.2])
    psi = qs.empty_state()
    qs.init_coherent(z, psi)
    psi0 = to_host(psi)
    qs.set_resident_max(resident)
    steps, dt = 20000, 1e-3
    qs.evolve(psi, dt, steps)
    ref = _eigen_rk4(os_, w, L, psi0, dt, steps)
    assert rel_err(to_host(psi), ref) <= STATE_TOL


def test_long_horizon_deep_sectors():
    """2 x 10^4 stage-launch steps of a random state over the sectors 44 <= N <= 50
    of M = 3 (21 sectors, ket weights up to 2^38), against the eigenbasis polynomial."""
    M = 3
    w = np.array([0.5, 0.0, 0.5])
    L = wl.contact_coupling(M, -0.02)
    qs, os_ = pair(M, w, L, 44, 50)
    x = random_state(qs.total, 29)
    psi = to_dev(x)
    qs.set_resident_max(0)
    steps, dt = 20000, 1e-3
    qs.evolve(psi, dt, steps)
    ref = _eigen_rk4(os_, w, L, x, dt, steps)
    assert rel_err(to_host(psi), ref) <= STATE_TOL


def test_full_size_step_whole_sectors_against_oracle():
    """One RK4 step of the full batched coherent workload (M=7, n_tot=16, N <= 40,
    281 sectors, 62,891,499 kets) in the benchmark's launch configuration, and the
    oracle's classic RK4 on whole sectors cut from the same state: every sector with
    N <= 10 and the (16, 0) sector.  Sectors evolve independently, so the cut is exact."""
    import paper_2111_00050_gb300 as qb

    W = wl.batched_coherent()
    qs = qb.Space(W.M, W.w, W.L, 0, W.n_max)
    assert qs.total == 62891499 and qs.n_sectors == 281
    psi = qs.empty_state()
    qs.init_coherent(W.z, psi)
    work = qs.workspace(1)
    qs.autotune(W.dt, psi, steps=1, work=work)
    # a generic state: one step first, so that every sector carries a non-coherent amplitude
    qs.evolve(psi, W.dt, 1, work)
    x = to_host(psi)
    qs.evolve(psi, W.dt, 1, work)
    got = to_host(psi)
    picks = [s for s, (N, P) in enumerate(qs.sectors) if N <= 10] + [qs.sectors.index((16, 0))]
    for s in picks:
        off, dim = int(qs.offsets[s]), int(qs.dims[s])
        os_ = orc.Space(W.M, [qs.sectors[s]])
        assert os_.total == dim
        ref = orc.rk4(os_, W.w, W.L, x[off:off + dim], W.dt, 1)
        assert rel_err(got[off:off + dim], ref) <= STATE_TOL, qs.sectors[s]

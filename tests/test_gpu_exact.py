"""Exact momentum conservation (the plain label sum of Sec. III B instead of the
sum mod M): the CUDA path against the oracle's exact-momentum sectors.

Same tolerances as the mod-M parity tests: bases and ranks bit-exact, one H psi
<= 1e-13 relative, evolved states <= 1e-10 relative, observables <= 1e-9,
gradients <= 1e-8 relative to the oracle's discrete adjoint.
"""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from helpers import rel_err, random_state, to_dev, to_host

pytestmark = pytest.mark.gpu

STATE_TOL = 1e-10
HPSI_TOL = 1e-13
OBS_TOL = 1e-9


def _random_exact_hermitian(M, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    L = (rng.standard_normal((M,) * 4) + 1j * rng.standard_normal((M,) * 4)) * scale
    L = L * wl._conserving(M, exact=True)
    L = 0.5 * (L + np.conj(L.transpose(3, 2, 1, 0)))
    return rng.standard_normal(M), L


def _case(name):
    if name == "M5_contact":
        M = 5
        return M, wl.dispersion_quadratic(M), wl.contact_coupling(M, -0.1, exact=True), 0, 8, None
    if name == "M7_long_range":
        M = 7
        return M, wl.dispersion_quadratic(M), wl.long_range_coupling(M, 0.1 / 8, exact=True), 8, 8, [0, 1, -3]
    if name == "M5_complex_hermitian":
        w, L = _random_exact_hermitian(5, 21)
        return 5, w, L, 0, 6, None
    if name == "M4_even":
        M = 4
        return M, wl.dispersion_abs(M), wl.contact_coupling(M, 0.07, exact=True), 2, 7, None
    if name == "M9_N10":
        M = 9
        return M, wl.dispersion_quadratic(M), wl.contact_coupling(M, -0.05, exact=True), 10, 10, [0, 2]
    raise KeyError(name)


CASES = ["M5_contact", "M7_long_range", "M5_complex_hermitian", "M4_even", "M9_N10"]


def _pair(M, w, L, n0, n1, pl):
    import paper_2111_00050_gb300 as qb

    qs = qb.Space(M, w, L, n0, n1, pl, exact=True)
    os_ = orc.Space(M, qs.sectors, exact=True)
    assert os_.total == qs.total
    return qs, os_


@pytest.mark.parametrize("name", CASES)
def test_exact_basis_rank_hpsi_and_terms(name):
    import torch

    M, w, L, n0, n1, pl = _case(name)
    qs, os_ = _pair(M, w, L, n0, n1, pl)
    if pl is None:  # every exact sector of the N range, N then P ascending
        assert qs.sectors == orc.all_sectors(M, n0, n1, exact=True)
    np.testing.assert_array_equal(qs.basis().cpu().numpy(), os_.basis)
    idx = qs.rank(torch.from_numpy(os_.basis).cuda()).cpu().numpy()
    np.testing.assert_array_equal(idx, np.arange(qs.total))
    x = random_state(qs.total, 7)
    out = qs.empty_state()
    qs.hpsi(to_dev(x), out)
    assert rel_err(to_host(out), orc.apply_h(os_, w, L, x)) <= HPSI_TOL
    assert qs.terms()[0] == orc.count_terms(os_, L)


def test_exact_coherent_evolution_observables_and_resident_path():
    """A coherent state on every exact sector with N <= 12 (M=5): 100 RK4 steps
    against the oracle, observables, and the resident small-sector path bit for
    bit against stage launches."""
    import paper_2111_00050_gb300 as qb

    M = 5
    rng = np.random.default_rng(5)
    z = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    z *= math.sqrt(3.0 / np.sum(np.abs(z) ** 2))
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.08, exact=True)
    qs, os_ = _pair(M, w, L, 0, 12, None)
    psi = qs.empty_state()
    kept = qs.init_coherent(z, psi)
    ref, kept_ref = orc.coherent_state(os_, z)
    assert abs(kept - kept_ref) <= 1e-14
    b = psi.clone()
    qs.set_resident_max(1024)
    qs.evolve(psi, 2e-3, 100)
    qs.set_resident_max(0)
    qs.evolve(b, 2e-3, 100)
    assert bool((psi == b).all())
    ref = orc.rk4(os_, w, L, ref, 2e-3, 100)
    assert rel_err(to_host(psi), ref) <= STATE_TOL
    ob = qs.observables(psi)
    ro = orc.observables(os_, ref, w, L)
    for key in ("Q", "PO", "Vminus_p"):
        assert abs(ob[key] - ro[key]) <= OBS_TOL, key
    np.testing.assert_allclose(ob["a"], ro["a"], atol=OBS_TOL * max(1, np.abs(ro["a"]).max()))
    np.testing.assert_allclose(ob["Mij"], ro["Mij"], atol=OBS_TOL * ro["n_tot"])
    np.testing.assert_allclose(ob["aa"], ro["aa"], atol=OBS_TOL * ro["n_tot"])
    assert abs(ob["H"] - ro["H"]) <= OBS_TOL * max(1, abs(ro["H"]))
    # the second-order Taylor step on the exact sectors
    qs.set_order(2)
    qs.evolve(psi, 2e-3, 10)
    ref = orc.taylor(os_, w, L, ref, 2e-3, 10, 2)
    assert rel_err(to_host(psi), ref) <= STATE_TOL


def test_exact_field_number_long_range_window():
    """Field-number state on the exact sectors of N = n_tot (10) of an M = 7 long-range model."""
    Wl = wl.long_range_field_number(M=7, seed=1, mean=1.3)
    n = Wl.n_tot
    L = wl.long_range_coupling(7, 0.1 / n, exact=True)
    qs, os_ = _pair(7, Wl.w, L, n, n, None)
    psi = qs.empty_state()
    qs.init_field_number(Wl.z, n, psi)
    ref = orc.field_number_state(os_, Wl.z, n)
    assert rel_err(to_host(psi), ref) <= 1e-13
    qs.evolve(psi, Wl.dt, 40)
    ref = orc.rk4(os_, Wl.w, L, ref, Wl.dt, 40)
    assert rel_err(to_host(psi), ref) <= STATE_TOL
    assert abs(qs.observables(psi)["PO"] - orc.observables(os_, ref)["PO"]) <= OBS_TOL


def test_exact_adjoint_matches_oracle():
    import paper_2111_00050_gb300 as qb

    M = 5
    rng = np.random.default_rng(0)
    x = rng.standard_normal((M, 2))
    z = x[:, 0] + 1j * x[:, 1]
    z *= math.sqrt(2.5 / np.sum(np.abs(z) ** 2))
    w = wl.dispersion_quadratic(M)
    L0 = wl.contact_coupling(M, 1.0, exact=True)
    qs = qb.Space(M, w, L0, 0, 10, exact=True)
    got = qs.adjoint(z, -0.2, 2e-3, 40, ckpt_every=1, loss="Q")
    os_ = orc.Space(M, qs.sectors, exact=True)
    loss, gs, gw, gz = orc.adjoint_gradient(os_, w, L0, -0.2, z, 2e-3, 40, "Q")
    rel = lambda a, b: float(np.max(np.abs(np.atleast_1d(a) - np.atleast_1d(b))) / np.max(np.abs(np.atleast_1d(b))))
    assert abs(got["loss"] - loss) <= 1e-10 * max(1, abs(loss))
    assert rel(got["grad_scale"], gs) <= 1e-8
    assert rel(got["grad_w"], gw) <= 1e-8
    assert rel(got["grad_z"], gz) <= 1e-8
    # every coupling entry (tape mode): along L0 it is grad_scale; along an exactly
    # conserving Hermitian direction it matches central differences
    gc = qs.adjoint(z, -0.2, 2e-3, 40, ckpt_every=0, loss="Q", coupling_grad=True)
    g = gc["grad_L"]
    assert abs(float(np.sum((np.conj(g) * L0).real)) - gc["grad_scale"]) <= 1e-10 * abs(gc["grad_scale"])
    _, D = _random_exact_hermitian(M, 3)
    h = 1e-5

    def fl(eps):
        return qb.Space(M, w, -0.2 * L0 + eps * D, 0, 10, exact=True).adjoint(z, 1.0, 2e-3, 40, ckpt_every=1,
                                                                              loss="Q")["loss"]

    fd = (fl(h) - fl(-h)) / (2 * h)
    an = float(np.sum((np.conj(g) * D).real))
    assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(gc["grad_scale"]))


def test_exact_rejects_umklapp_coupling_and_batches():
    import torch

    import paper_2111_00050_gb300 as qb

    M = 5
    with pytest.raises(qb.QbError):
        qb.Space(M, wl.dispersion_quadratic(M), wl.contact_coupling(M, 0.1), 0, 4, exact=True)
    qs = qb.Space(M, wl.dispersion_quadratic(M), wl.contact_coupling(M, 0.1, exact=True), 0, 4, exact=True)
    psi = torch.zeros((2, qs.total), dtype=torch.complex128, device="cuda")
    with pytest.raises(qb.QbError):
        qs.evolve_batch(psi, [1.0, 0.5], 1e-3, 1)


def test_minimal_image_long_range_evolution():
    """The minimal-image variant of the long-range kernel (distance on the ring of
    M momenta) on mod-M sectors, against the oracle."""
    from helpers import pair

    M = 9
    L = wl.long_range_coupling(M, 0.1 / 8, min_image=True)
    w = wl.dispersion_quadratic(M)
    qs, os_ = pair(M, w, L, 8, 8, [0, 4])
    x = random_state(qs.total, 3)
    out = qs.empty_state()
    qs.hpsi(to_dev(x), out)
    assert rel_err(to_host(out), orc.apply_h(os_, w, L, x)) <= HPSI_TOL
    psi = to_dev(x)
    qs.evolve(psi, 1e-3, 30)
    assert rel_err(to_host(psi), orc.rk4(os_, w, L, x, 1e-3, 30)) <= STATE_TOL

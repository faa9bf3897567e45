"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances:
  * one H psi: relative 2-norm error <= 1e-13 (only the summation order differs);
  * evolved states: relative 2-norm error <= 1e-10 (same discrete RK4 scheme);
  * observables: absolute <= 1e-9 on normalised quantities (Q, PO, V_-), relative
    <= 1e-9 on <a_i>, M_ij, <a_i a_j>.
Bases are compared bit-exactly; sector order and ket order must agree.
"""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from helpers import pair, rel_err, to_dev, to_host, random_state

pytestmark = pytest.mark.gpu

STATE_TOL = 1e-10
HPSI_TOL = 1e-13
OBS_TOL = 1e-9


def _random_hermitian(M, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    L = (rng.standard_normal((M,) * 4) + 1j * rng.standard_normal((M,) * 4)) * scale
    L = L * wl._conserving(M)
    L = 0.5 * (L + np.conj(L.transpose(3, 2, 1, 0)))
    return rng.standard_normal(M), L


def _case(name):
    if name == "M5_N6_contact":
        M = 5
        return M, wl.dispersion_quadratic(M), wl.contact_coupling(M, -0.1), 6, 6, [0]
    if name == "M7_N9_allP":
        M = 7
        return M, wl.dispersion_quadratic(M), wl.contact_coupling(M, -0.05), 9, 9, None
    if name == "M9_long_range":
        M = 9
        return M, wl.dispersion_quadratic(M), wl.long_range_coupling(M, 0.1 / 8), 8, 8, [0, 3]
    if name == "M5_complex_hermitian":
        w, L = _random_hermitian(5, 11)
        return 5, w, L, 0, 5, None
    if name == "M3_multi_sector":
        M = 3
        return M, np.array([0.4, -0.2, 0.9]), wl.contact_coupling(M, 0.07), 0, 12, None
    if name == "M1_kerr":
        return 1, np.array([0.7]), np.full((1, 1, 1, 1), 0.13, dtype=np.complex128), 0, 30, None
    if name == "M4_even_paper":
        M = 4
        rng = np.random.default_rng(3)
        return M, rng.standard_normal(M), wl.paper_coupling(M, -0.2, 0.05), 0, 6, None
    if name == "M11_N6":
        M = 11
        return M, wl.dispersion_abs(M), wl.contact_coupling(M, -0.02), 6, 6, [0, 5]
    if name == "M5_N40_deep":
        M = 5
        return M, wl.dispersion_quadratic(M), wl.contact_coupling(M, -0.1), 40, 40, [1]
    if name == "M16_max_modes":  # QB_MAX_MODES (even M: labels 0..15), every P, N up to 3
        M = 16
        return M, wl.dispersion_abs(M), wl.contact_coupling(M, 0.05), 0, 3, None
    if name == "M13_generic":  # odd M without a specialised kernel
        M = 13
        return M, wl.dispersion_quadratic(M), wl.long_range_coupling(M, 0.02), 4, 4, [0, 6]
    raise KeyError(name)


CASES = ["M5_N6_contact", "M7_N9_allP", "M9_long_range", "M5_complex_hermitian", "M3_multi_sector", "M1_kerr",
         "M4_even_paper", "M11_N6", "M5_N40_deep", "M16_max_modes", "M13_generic"]


@pytest.mark.parametrize("name", CASES)
def test_basis_and_rank_match_oracle(name):
    import torch

    M, w, L, n0, n1, pl = _case(name)
    qs, os_ = pair(M, w, L, n0, n1, pl)
    b = qs.basis().cpu().numpy()
    np.testing.assert_array_equal(b, os_.basis)
    idx = qs.rank(torch.from_numpy(os_.basis).cuda()).cpu().numpy()
    np.testing.assert_array_equal(idx, np.arange(qs.total))
    # kets outside the space rank to -1
    bad = os_.basis[:4].copy()
    bad[:, 0] += n1 + 1  # more particles than any held sector
    assert (qs.rank(torch.from_numpy(bad).cuda()).cpu().numpy() == -1).all()


@pytest.mark.parametrize("name", CASES)
def test_hpsi_matches_oracle(name):
    M, w, L, n0, n1, pl = _case(name)
    qs, os_ = pair(M, w, L, n0, n1, pl)
    x = random_state(qs.total, 5)
    out = qs.empty_state()
    qs.hpsi(to_dev(x), out)
    ref = orc.apply_h(os_, w, L, x)
    assert rel_err(to_host(out), ref) <= HPSI_TOL


@pytest.mark.parametrize("name", ["M5_N6_contact", "M7_N9_allP", "M9_long_range", "M5_complex_hermitian",
                                  "M3_multi_sector", "M4_even_paper"])
def test_terms_count_matches_oracle(name):
    """Distinct nonzero H elements (diagonal included) against the oracle's count,
    which is pinned to the dense-matrix structure on the CPU."""
    M, w, L, n0, n1, pl = _case(name)
    qs, os_ = pair(M, w, L, n0, n1, pl)
    terms, tuples = qs.terms()
    assert terms == orc.count_terms(os_, L)


def test_plain_single_sector_full_run():
    """M=5, contact C=-0.1, |0,2,2,2,0>, RK4 dt=1e-3 to t=10, observables every
    100 steps: every sample and the final state against the oracle."""
    import torch

    W = wl.plain_single_sector()
    qs, os_ = pair(W.M, W.w, W.L, 6, 6, [0])
    psi = qs.empty_state()
    qs.init_number(W.occ, psi)
    series = qs.evolve_observe(psi, W.dt, W.steps, W.obs_every)
    ref = orc.number_state(os_, W.occ)
    for k, ob in enumerate(series):
        if k > 0:
            ref = orc.rk4(os_, W.w, W.L, ref, W.dt, W.obs_every)
        if k % 10 == 0 or k == len(series) - 1:
            ro = orc.observables(os_, ref, W.w, W.L)
            assert abs(ob["Q"] - ro["Q"]) <= OBS_TOL
            assert abs(ob["lam_p"] - ro["lam_p"]) <= OBS_TOL * ro["n_tot"]
            assert abs(ob["H"] - ro["H"]) <= OBS_TOL * abs(ro["H"])
            np.testing.assert_allclose(ob["Mij"], ro["Mij"], atol=OBS_TOL * ro["n_tot"])
            np.testing.assert_allclose(ob["aa"], ro["aa"], atol=OBS_TOL * ro["n_tot"])
    assert rel_err(to_host(psi), ref) <= STATE_TOL
    torch.cuda.synchronize()


def _coherent_case(M, n_tot, nmax, C, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    z *= math.sqrt(n_tot / np.sum(np.abs(z) ** 2))
    return z, wl.dispersion_quadratic(M), wl.contact_coupling(M, C)


def test_coherent_multi_sector_evolution_and_observables():
    M = 5
    z, w, L = _coherent_case(M, 3.0, 13, -0.08, 1)
    qs, os_ = pair(M, w, L, 0, 13, None)
    psi = qs.empty_state()
    kept = qs.init_coherent(z, psi)
    ref, kept_ref = orc.coherent_state(os_, z)
    assert abs(kept - kept_ref) <= 1e-14
    assert rel_err(to_host(psi), ref) <= 1e-14
    ob0 = qs.observables(psi)
    ro0 = orc.observables(os_, ref, w, L)
    # truncation at N <= 13 leaves Q(0) at the size of the Poisson tail, not 0
    assert abs(ob0["Q"] - ro0["Q"]) <= OBS_TOL and abs(ob0["Q"]) < 1e-4
    assert abs(ob0["Vminus_p"] - ro0["Vminus_p"]) <= OBS_TOL
    qs.evolve(psi, 2e-3, 200)
    ref = orc.rk4(os_, w, L, ref, 2e-3, 200)
    assert rel_err(to_host(psi), ref) <= STATE_TOL
    ob = qs.observables(psi)
    ro = orc.observables(os_, ref, w, L)
    for key in ("Q", "PO", "Vminus_p"):
        assert abs(ob[key] - ro[key]) <= OBS_TOL, key
    np.testing.assert_allclose(ob["Vminus_modes"], ro["Vminus_modes"], atol=OBS_TOL)
    np.testing.assert_allclose(ob["a"], ro["a"], atol=OBS_TOL * max(1, np.abs(ro["a"]).max()))
    np.testing.assert_allclose(ob["Mij"], ro["Mij"], atol=OBS_TOL * ro["n_tot"])
    np.testing.assert_allclose(ob["aa"], ro["aa"], atol=OBS_TOL * ro["n_tot"])
    np.testing.assert_allclose(ob["eigvals"], ro["eigvals"], atol=OBS_TOL * ro["n_tot"])
    assert abs(ob["H"] - ro["H"]) <= OBS_TOL * max(1, abs(ro["H"]))
    assert abs(abs(np.vdot(ob["xi"], ro["xi"])) - 1) < 1e-9


def test_field_number_long_range_window():
    """Scaled-down gravity-like workload: M=9 long range, field number state."""
    Wl = wl.long_range_field_number(M=9, seed=0, mean=0.4)
    n_tot = Wl.n_tot
    qs, os_ = pair(Wl.M, Wl.w, Wl.L, n_tot, n_tot, None)
    psi = qs.empty_state()
    qs.init_field_number(Wl.z, n_tot, psi)
    ref = orc.field_number_state(os_, Wl.z, n_tot)
    assert rel_err(to_host(psi), ref) <= 1e-13
    ob = qs.observables(psi)
    assert abs(ob["Q"] - 1) < 1e-9 and abs(ob["lam_p"] - n_tot) < 1e-9 * n_tot
    qs.evolve(psi, Wl.dt, 60)
    ref = orc.rk4(os_, Wl.w, Wl.L, ref, Wl.dt, 60)
    assert rel_err(to_host(psi), ref) <= STATE_TOL
    ro = orc.observables(os_, ref)
    ob = qs.observables(psi)
    assert abs(ob["PO"] - ro["PO"]) <= OBS_TOL


def test_batched_sweep_matches_separate_members():
    import torch

    M = 5
    z, w, L = _coherent_case(M, 2.0, 10, -0.1, 2)
    scales = [0.5, 1.0, 2.0, -1.0]
    qs, os_ = pair(M, w, L, 0, 10, None)
    psi = torch.empty((4, qs.total), dtype=torch.complex128, device="cuda")
    for b in range(4):
        qs.init_coherent(z, psi[b])
    qs.evolve_batch(psi, scales, 2e-3, 120)
    ref0, _ = orc.coherent_state(os_, z)
    for b, sc in enumerate(scales):
        ref = orc.rk4(os_, w, sc * L, ref0, 2e-3, 120)
        assert rel_err(to_host(psi[b]), ref) <= STATE_TOL


def test_kerr_single_mode_gpu_matches_closed_form():
    """M=1: <a(t)> = a0 e^{-iwt} exp(|a0|^2 (e^{-2iLt} - 1)) to the RK4 error."""
    w, Lk, a0 = 0.5, 0.1, 1.1 + 0.3j
    import paper_2111_00050_gb300 as qb

    qs = qb.Space(1, [w], np.full((1, 1, 1, 1), Lk, dtype=np.complex128), 0, 40)
    psi = qs.empty_state()
    qs.init_coherent([a0], psi)
    qs.evolve(psi, 1e-3, 1000)
    a_ref = a0 * np.exp(-1j * w) * np.exp(abs(a0) ** 2 * (np.exp(-2j * Lk) - 1))
    assert abs(qs.observables(psi)["a"][0] - a_ref) < 1e-9


def test_large_sector_sampled_rows():
    """M=11, N=20, P=0 (2,731,365 kets): sampled kets rank to their oracle index and
    sampled rows of H psi match the oracle's per-row application; one RK4 step
    conserves the norm to O(dt^6) and <H> to rounding."""
    import torch

    W = wl.large_sector()
    qs, os_ = pair(W.M, W.w, W.L, 20, 20, [0])
    assert qs.total == 2731365
    rng = np.random.default_rng(9)
    rows = np.sort(rng.choice(qs.total, 256, replace=False))
    rows[0], rows[-1] = 0, qs.total - 1
    got = qs.rank(torch.from_numpy(os_.basis[rows]).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, rows)
    b = qs.basis(int(rows[100]), 1).cpu().numpy()[0]
    np.testing.assert_array_equal(b, os_.basis[rows[100]])
    x = random_state(qs.total, 13)
    out = qs.empty_state()
    xd = to_dev(x)
    qs.hpsi(xd, out)
    ref = orc.apply_h_rows(os_, 0, W.w, W.L, x, rows)
    got = to_host(out)[rows]
    assert np.max(np.abs(got - ref)) <= HPSI_TOL * np.max(np.abs(ref)) * 10
    psi = qs.empty_state()
    qs.init_number(W.occ, psi)
    e0 = qs.observables(psi)["H"]
    qs.evolve(psi, W.dt, 4)
    ob = qs.observables(psi)
    assert abs(ob["norm"] - 1) < 1e-12
    assert abs(ob["H"] - e0) < 1e-10 * abs(e0)


def test_errors_are_reported():
    import paper_2111_00050_gb300 as qb

    M = 5
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.1)
    Lbad = L.copy()
    Lbad[0, 1, 2, 4] = 0.3j  # breaks Hermiticity
    Lbad = Lbad * wl._conserving(M)
    with pytest.raises(qb.QbError) as e:
        qb.Space(M, w, Lbad, 3, 3)
    assert e.value.code == 1
    with pytest.raises(qb.QbError) as e:
        qb.Space(17, np.zeros(17), np.zeros((17,) * 4), 1, 1)
    assert e.value.code == 6
    qs = qb.Space(M, w, L, 3, 3)
    with pytest.raises(qb.QbError):
        qs.init_number([3, 0, 0, 0, 1], qs.empty_state())  # N=4 not held


@pytest.mark.parametrize("call", ["evolve", "hpsi", "observables", "basis"])
def test_device_status_word_fails_the_next_call(call):
    """A failed device-side check is reported through the space's status word, not
    a fault: with a bit pre-set on the host (qb_space_status), the next call that
    synchronises returns QB_EINTERNAL and clears the word, and the call after it
    succeeds with unchanged results."""
    import paper_2111_00050_gb300 as qb

    M = 5
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.1)
    qs = qb.Space(M, w, L, 0, 6)
    psi = qs.empty_state()
    qs.init_coherent(np.array([0.3, 0.8j, 0.5, 0.0, -0.2]), psi)
    out = qs.empty_state()
    run = {"evolve": lambda: qs.evolve(psi, 1e-3, 3), "hpsi": lambda: qs.hpsi(psi, out),
           "observables": lambda: qs.observables(psi), "basis": lambda: qs.basis(0, 7)}[call]
    run()
    ref = to_host(psi).copy()
    assert qs.status() == 0
    assert qs.status(2) == 2
    with pytest.raises(qb.QbError) as e:
        run()
    assert e.value.code == qb.QB_EINTERNAL and "status 2" in str(e.value)
    assert qs.status() == 0
    if call == "evolve":
        psi.copy_(to_dev(ref))
    run()
    if call == "evolve":
        again = to_dev(ref)
        qs.evolve(again, 1e-3, 3)
        assert bool((psi == again).all())


def test_plain_per_sector_path_is_bit_identical_to_batched():
    """One launch per sector per stage and one launch for all sectors compute every
    ket with the same arithmetic: the states must agree bit for bit."""
    M = 5
    z, w, L = _coherent_case(M, 2.0, 11, -0.1, 3)
    import paper_2111_00050_gb300 as qb

    qs = qb.Space(M, w, L, 0, 11)
    a = qs.empty_state()
    qs.init_coherent(z, a)
    b = a.clone()
    qs.evolve(a, 2e-3, 40)
    qs.evolve_plain(b, 2e-3, 40)
    assert bool((a == b).all())


def test_breaktime_pipeline_matches_oracle():
    """Observation series on the GPU -> breaktimes, against the oracle's series:
    Q breaktime of a coherent start, PO breaktime of a field-number start (whose
    Q is 1 from t = 0 and is flagged AT_START), and the mean-field companion."""
    import paper_2111_00050_gb300 as qb

    M, dt, steps, every = 5, 2e-3, 400, 20
    w = wl.dispersion_quadratic(M)
    L = wl.long_range_coupling(M, 0.6)
    z, _, _ = _coherent_case(M, 3.0, 13, -0.1, 4)
    qs, os_ = pair(M, w, L, 0, 13, None)
    psi = qs.empty_state()
    qs.init_coherent(z, psi)
    series = qs.evolve_observe(psi, dt, steps, every)
    ref = orc.coherent_state(os_, z)[0]
    ref_Q = [orc.observables(os_, ref)["Q"]]
    for _ in range(steps // every):
        ref = orc.rk4(os_, w, L, ref, dt, every)
        ref_Q.append(orc.observables(os_, ref)["Q"])
    gpu_Q = [s["Q"] for s in series]
    np.testing.assert_allclose(gpu_Q, ref_Q, atol=OBS_TOL)
    thr = ref_Q[0] + 0.5 * (max(ref_Q) - ref_Q[0])
    t_gpu, f_gpu = qb.breaktime(gpu_Q, dt * every, thr)
    t_ref, f_ref = orc.breaktime(ref_Q, dt * every, thr)
    assert f_gpu == f_ref == qb.QB_CROSSED
    assert abs(t_gpu - t_ref) < 1e-6
    traj = qb.meanfield(M, w, L, z, dt, steps, every)
    np.testing.assert_allclose(traj, orc.meanfield(w, L, z, dt, steps, every), atol=1e-11)

    n = np.array([0, 2, 1, 3, 0])
    zf = np.sqrt(n) * np.exp(1j * np.array([0.0, 0.4, 2.0, -1.1, 0.0]))
    qf, of = pair(M, w, L, 6, 6, None)
    pf = qf.empty_state()
    qf.init_field_number(zf, 6, pf)
    sf = qf.evolve_observe(pf, dt, steps, every)
    reff = orc.field_number_state(of, zf, 6)
    ref_PO = [orc.observables(of, reff)["PO"]]
    for _ in range(steps // every):
        reff = orc.rk4(of, w, L, reff, dt, every)
        ref_PO.append(orc.observables(of, reff)["PO"])
    gpu_PO = [s["PO"] for s in sf]
    np.testing.assert_allclose(gpu_PO, ref_PO, atol=OBS_TOL)
    assert qb.breaktime([s["Q"] for s in sf], dt * every, 0.15)[1] == qb.QB_AT_START
    thr = 0.5 * max(ref_PO)
    t_gpu, f_gpu = qb.breaktime(gpu_PO, dt * every, thr)
    t_ref, f_ref = orc.breaktime(ref_PO, dt * every, thr)
    assert f_gpu == f_ref == qb.QB_CROSSED and abs(t_gpu - t_ref) < 1e-6


@pytest.mark.parametrize("steps", [5, 70])
def test_resident_small_sectors_bit_identical_to_stage_launches(steps):
    """M=7, N <= 12: the leading sectors (up to 1024 kets) run shared-memory
    resident beside the stage launches of the larger ones; the state must equal
    the all-stage-launch run bit for bit, and the oracle to 1e-10.  70 steps also
    cover the CUDA-graph replay of the stage launches."""
    import paper_2111_00050_gb300 as qb

    M = 7
    z, w, L = _coherent_case(M, 3.0, 12, -0.05, 5)
    qs = qb.Space(M, w, L, 0, 12)
    assert qs.dims.min() <= 1024 < qs.dims.max()
    a = qs.empty_state()
    qs.init_coherent(z, a)
    b = a.clone()
    c = a.clone()
    qs.set_resident_max(1024)
    qs.evolve(a, 1e-3, steps)
    qs.set_resident_max(0)
    qs.evolve(b, 1e-3, steps)
    assert bool((a == b).all())
    qs.evolve_plain(c, 1e-3, steps)
    assert bool((a == c).all())
    if steps == 5:
        os_ = orc.Space(M, qs.sectors)
        ref = orc.rk4(os_, w, L, orc.coherent_state(os_, z)[0], 1e-3, steps)
        assert rel_err(to_host(a), ref) <= STATE_TOL


@pytest.mark.parametrize("M", [5, 7, 9, 4])
def test_every_tile_shape_is_bit_identical(M):
    """The compiled tile shapes of the stage kernel (qb_space_set_tile_shape) only
    change how kets map to warps, not the order of any ket's sums: 40 steps (graph
    replay included) under every shape equal shape 0 bit for bit; the autotuner keeps
    one of them and reports its timings."""
    import paper_2111_00050_gb300 as qb

    nmax = {5: 12, 7: 11, 9: 9, 4: 14}[M]
    z, w, L = _coherent_case(M, 3.0, nmax, -0.05, 7)
    qs = qb.Space(M, w, L, 0, nmax)
    qs.set_resident_max(0)
    x = qs.empty_state()
    qs.init_coherent(z, x)
    ref = None
    for shape in range(qb._lib.QB_TILE_SHAPES):
        qs.set_tile_shape(shape)
        y = x.clone()
        qs.evolve(y, 2e-3, 40)
        if ref is None:
            ref = y
        else:
            assert bool((y == ref).all()), shape
    with pytest.raises(qb.QbError):
        qs.set_tile_shape(qb._lib.QB_TILE_SHAPES)
    chosen = qs.autotune(2e-3, x, steps=2)
    assert qs.tuning["tile_shape"] in range(qb._lib.QB_TILE_SHAPES) and chosen == qs.tuning["resident_max_kets"]
    assert len(qs.tuning["tile_shape_ms"]) == qb._lib.QB_TILE_SHAPES


@pytest.mark.parametrize("order", [2, 3])
def test_taylor_order_matches_oracle(order):
    """Selectable step order (Sec. III B's second-order Taylor step, and third order) on
    a coherent multi-sector space, against the oracle's Taylor steps; the resident and
    graph-replayed paths (70 steps) stay bit-identical to plain stage launches."""
    import paper_2111_00050_gb300 as qb

    M = 5
    z, w, L = _coherent_case(M, 3.0, 13, -0.08, 1)
    qs, os_ = pair(M, w, L, 0, 13, None)
    qs.set_order(order)
    psi = qs.empty_state()
    qs.init_coherent(z, psi)
    ref, _ = orc.coherent_state(os_, z)
    b = psi.clone()
    qs.evolve(psi, 2e-3, 70)
    ref = orc.taylor(os_, w, L, ref, 2e-3, 70, order)
    assert rel_err(to_host(psi), ref) <= STATE_TOL
    qs.set_resident_max(0)
    qs.evolve_plain(b, 2e-3, 70)
    assert bool((psi == b).all())
    with pytest.raises(qb.QbError):
        qs.adjoint(z, 1.0, 2e-3, 2)  # the adjoint is RK4's
    with pytest.raises(qb.QbError):
        qs.set_order(5)


def test_taylor_order_error_vs_exact_flow():
    """Global error against the exact flow exp(-iHt) at t = 10 on the 42-ket sector of
    |0,2,2,2,0>: the GPU's order-2, -3 and -4 runs (10^4 steps of 1e-3) land on the
    eigenbasis prediction sum_k (-i E dt)^k / k! per step, i.e. ~1.04e-5, 1.04e-8, 1.03e-11."""
    import math

    import paper_2111_00050_gb300 as qb

    W = wl.plain_single_sector()
    qs = qb.Space(W.M, W.w, W.L, 6, 6, [0])
    os_ = orc.Space(W.M, [(6, 0)])
    lam, V = np.linalg.eigh(orc.h_dense(os_, 0, W.w, W.L))
    psi0 = orc.number_state(os_, W.occ)
    c0 = V.conj().T @ psi0
    exact = V @ (np.exp(-1j * lam * W.steps * W.dt) * c0)
    for order in (2, 3, 4):
        x = -1j * lam * W.dt
        pred = V @ (sum(x ** k / math.factorial(k) for k in range(order + 1)) ** W.steps * c0)
        qs.set_order(order)
        psi = qs.empty_state()
        qs.init_number(W.occ, psi)
        qs.evolve(psi, W.dt, W.steps)
        got = to_host(psi)
        assert rel_err(got, pred) <= STATE_TOL
        e_pred = np.linalg.norm(pred - exact)
        assert abs(np.linalg.norm(got - exact) - e_pred) <= 1e-3 * e_pred + STATE_TOL


def test_squeezing_times_match_oracle():
    """Sec. IV E's squeezing analysis on a GPU run (M=5, Gaussian coherent profile,
    n_tot=3, long range with |n_tot chi| = 0.242, N <= 10): the V_- series of the
    principal mode from qb_evolve_observe against the oracle's, and onset (V_- <= 0.8)
    and maximal squeezing from qb_squeezing against the oracle's analysis of the
    oracle's series; the onset lies near the one-mode estimate 0.05 / |n_tot chi|."""
    import paper_2111_00050_gb300 as qb

    unit = wl.squeezing_coherent(3, M=5)
    chi1 = qb.api.interaction_per_occupation(unit.M, unit.w, unit.L, unit.z)
    W = wl.squeezing_coherent(3, M=5, G=0.242 / abs(chi1), t_end=0.9, obs_every=10)
    chi = qb.api.interaction_per_occupation(W.M, W.w, W.L, W.z)
    assert abs(abs(chi) - 0.242) < 1e-12
    qs, os_ = pair(W.M, W.w, W.L, 0, 10, None)
    psi = qs.empty_state()
    qs.init_coherent(W.z, psi)
    series = qs.evolve_observe(psi, W.dt, W.steps, W.obs_every)
    v_gpu = [o["Vminus_p"] for o in series]
    ref, _ = orc.coherent_state(os_, W.z)
    v_ref = [orc.observables(os_, ref)["Vminus_p"]]
    for _ in range(W.steps // W.obs_every):
        ref = orc.rk4(os_, W.w, W.L, ref, W.dt, W.obs_every)
        v_ref.append(orc.observables(os_, ref)["Vminus_p"])
    np.testing.assert_allclose(v_gpu, v_ref, atol=OBS_TOL)
    dt_obs = W.dt * W.obs_every
    got, exp = qb.api.squeezing(v_gpu, dt_obs, 0.8), orc.squeezing(v_ref, dt_obs, 0.8)
    assert got["flag"] == exp["flag"] == qb.QB_CROSSED
    assert 0 < got["t_min"] < W.steps * W.dt  # an interior minimum
    for key in ("t_sqz", "t_min", "v_min"):
        assert abs(got[key] - exp[key]) <= 1e-6, key
    assert 0.8 < got["t_sqz"] * abs(chi) / 0.05 < 1.6


@pytest.mark.parametrize("name", CASES)
def test_observables_match_oracle(name):
    """The moments of a random normalised state on every parity case: the kernels
    specialised for M = 5, 7, 9, 11 and the generic one (M = 1, 3, 4, 13, 16),
    complex couplings, single and multi-sector spaces."""
    M, w, L, n0, n1, pl = _case(name)
    qs, os_ = pair(M, w, L, n0, n1, pl)
    x = random_state(qs.total, 17)
    x = x / np.linalg.norm(x)
    ob = qs.observables(to_dev(x))
    ro = orc.observables(os_, x, w, L)
    n = max(1.0, ro["n_tot"])
    assert abs(ob["norm"] - 1) <= 1e-12
    assert abs(ob["n_tot"] - ro["n_tot"]) <= OBS_TOL * n
    np.testing.assert_allclose(ob["a"], ro["a"], atol=OBS_TOL * n)
    np.testing.assert_allclose(ob["Mij"], ro["Mij"], atol=OBS_TOL * n)
    np.testing.assert_allclose(ob["aa"], ro["aa"], atol=OBS_TOL * n)
    assert abs(ob["H"] - ro["H"]) <= OBS_TOL * max(1, abs(ro["H"]))


@pytest.mark.parametrize("name", ["M16_max_modes", "M13_generic"])
def test_evolution_at_the_mode_limits(name):
    """RK4 on the largest mode count and on an odd M without a specialised kernel."""
    M, w, L, n0, n1, pl = _case(name)
    qs, os_ = pair(M, w, L, n0, n1, pl)
    x = random_state(qs.total, 9)
    psi = to_dev(x)
    qs.evolve(psi, 2e-3, 25)
    assert rel_err(to_host(psi), orc.rk4(os_, w, L, x, 2e-3, 25)) <= STATE_TOL


def test_degenerate_inputs():
    """Zero steps leave the state untouched; a space of the single empty ket (N = 0)
    evolves by the phase of its zero energy, i.e. not at all; an H psi of the zero
    vector is zero."""
    import paper_2111_00050_gb300 as qb

    M = 5
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.1)
    qs = qb.Space(M, w, L, 0, 4)
    x = random_state(qs.total, 2)
    psi = to_dev(x)
    qs.evolve(psi, 1e-3, 0)
    assert bool((to_host(psi) == x).all())
    out = qs.empty_state()
    qs.hpsi(to_dev(np.zeros(qs.total)), out)
    assert not to_host(out).any()
    q0 = qb.Space(M, w, L, 0, 0)
    assert q0.total == 1 and q0.n_sectors == 1
    p0 = q0.empty_state()
    q0.init_number([0] * M, p0)
    q0.evolve(p0, 1e-3, 70)
    assert to_host(p0)[0] == 1.0


@pytest.mark.parametrize("which", ["batched_coherent", "long_range_field_number"])
def test_full_size_sampled_rows_and_one_step(which):
    """The benchmark's workloads at full size, in the launch configuration the
    benchmark times: batched coherent (M=7, n_tot=16, N <= 40: 281 sectors,
    62,891,499 kets) and the long-range field-number state (M=9, N=27, every P:
    23,535,820 kets).  Sampled rows of H psi (FP64 kernel) against the oracle's per-row
    application in three sectors, then one RK4 step of the double-float batched path
    (autotuned resident threshold, every sector per launch) against the classic four
    stages composed from that FP64 H psi, and its norm after the step."""
    import torch

    import paper_2111_00050_gb300 as qb

    if which == "batched_coherent":
        W = wl.batched_coherent()
        qs = qb.Space(W.M, W.w, W.L, 0, W.n_max)
        assert qs.total == 62891499 and qs.n_sectors == 281
        psi = qs.empty_state()
        qs.init_coherent(W.z, psi)
        picks = ((1, 0), (16, 0), (40, 3))
    else:
        W = wl.long_range_field_number()
        qs = qb.Space(W.M, W.w, W.L, W.n_tot, W.n_tot)
        assert qs.total == 23535820
        psi = qs.empty_state()
        qs.init_field_number(W.z, W.n_tot, psi)
        picks = tuple((W.n_tot, P) for P in (0, 4, 8))
    out = qs.empty_state()
    qs.hpsi(psi, out)
    x_host = to_host(psi)
    rng = np.random.default_rng(17)
    for N, P in picks:
        s = qs.sectors.index((N, P))
        off, dim = int(qs.offsets[s]), int(qs.dims[s])
        os_ = orc.Space(W.M, [(N, P)])
        assert os_.total == dim
        rows = np.unique(np.concatenate([[0, dim - 1], rng.choice(dim, min(dim, 64), replace=False)]))
        ref = orc.apply_h_rows(os_, 0, W.w, W.L, x_host[off:off + dim], rows)
        got = to_host(out[off:off + dim])[rows]
        assert np.max(np.abs(got - ref)) <= HPSI_TOL * 10 * max(1e-300, np.max(np.abs(ref)))
    # classic RK4 from the FP64 operator, in plain torch arithmetic
    dt = W.dt

    def A(v):
        r = qs.empty_state()
        qs.hpsi(v, r)
        return -1j * dt * r

    k1 = A(psi)
    k2 = A(psi + 0.5 * k1)
    k3 = A(psi + 0.5 * k2)
    k4 = A(psi + k3)
    ref = psi + (k1 + 2 * k2 + 2 * k3 + k4) / 6
    del k1, k2, k3, k4, out
    work = qs.workspace(1)
    qs.autotune(dt, psi, steps=1, work=work)
    qs.evolve(psi, dt, 1, work)
    err = float(torch.linalg.vector_norm(psi - ref) / torch.linalg.vector_norm(ref))
    assert err <= STATE_TOL
    # the step's norm is the scheme's (|R(iy)|^2 = 1 - y^6/72 + ..., not 1 for large |E| dt)
    assert abs(float(torch.vdot(psi, psi).real) - float(torch.vdot(ref, ref).real)) < 1e-12

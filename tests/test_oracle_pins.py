"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests touch the CUDA library.  Each pin is chosen so that a
plausible mistake in the oracle (a dropped term, a wrong sign or index, a
transposed operand, a factor of two in the coupling) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import oracle as orc
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def gen_function_dims(M, N):
    """Sector sizes from the generating function prod_i 1/(1 - t x^{label_i}) taken
    modulo x^M - 1: coefficient array c[n, k] = #kets with n particles, momentum k."""
    lab = wl.mode_labels(M) % M
    c = np.zeros((N + 1, M), dtype=object)
    c[0, 0] = 1
    for i in range(M):
        new = np.zeros_like(c)
        for n in range(N + 1):
            for k in range(M):
                if c[n, k] == 0:
                    continue
                for v in range(0, N - n + 1):
                    new[n + v, (k + v * lab[i]) % M] += c[n, k]
        c = new
    return c[N]


def fock_ops(M, cutoff):
    """Annihilation operators on the truncated tensor-product space (sparse)."""
    d = cutoff + 1
    a1 = sp.diags([np.sqrt(np.arange(1, d))], [1], shape=(d, d), format="csr")
    eye = sp.identity(d, format="csr")
    ops = []
    for i in range(M):
        op = None
        for k in range(M):
            f = a1 if k == i else eye
            op = f if op is None else sp.kron(op, f, format="csr")
        ops.append(op)
    return ops


def fock_hamiltonian(M, cutoff, w, L):
    a = fock_ops(M, cutoff)
    ad = [x.conj().T.tocsr() for x in a]
    H = sum(w[p] * (ad[p] @ a[p]) for p in range(M))
    for p in range(M):
        for q in range(M):
            for r in range(M):
                for s in range(M):
                    if L[p, q, r, s] != 0:
                        H = H + L[p, q, r, s] * (ad[p] @ ad[q] @ a[r] @ a[s])
    return H.tocsr()


def full_index(occ, cutoff):
    d = cutoff + 1
    idx = 0
    for n in occ:
        idx = idx * d + int(n)
    return idx


def random_hermitian_coupling(M, rng, scale=0.1):
    """Random complex coupling with the operator symmetries and Hermiticity,
    supported on momentum-conserving tuples only."""
    L = (rng.standard_normal((M,) * 4) + 1j * rng.standard_normal((M,) * 4)) * scale
    L = L * wl._conserving(M)
    L = 0.5 * (L + np.conj(L.transpose(3, 2, 1, 0)))  # L_{pq;rs} = conj(L_{sr;qp}) term by term
    return L


def R4(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


# ------------------------------------------------------------- sector sizes

def test_sector_dims_match_generating_function():
    for M, N in [(1, 5), (3, 6), (5, 6), (5, 9), (7, 8), (4, 5), (6, 4)]:
        c = gen_function_dims(M, N)
        tot = 0
        for P in range(M):
            d = orc.sector_dim(M, N, P)
            assert d == c[P], (M, N, P)
            tot += d
        assert tot == math.comb(N + M - 1, M - 1)  # stars and bars


def test_sector_dims_golden():
    """Stored sizes (written by tests/golden/make_sector_dims.py from the oracle),
    re-derived here from the generating function; includes the M=11, N=20, P=0
    sector of about 2.7M kets."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sector_dims.txt")) if l.strip() and l[0] != "#"]
    for M, N, P, D in ((int(a), int(b), int(c), int(d)) for a, b, c, d in rows):
        assert gen_function_dims(M, N)[P % M] == D


def test_sector_dim_scaling_appendix():
    """App. A counts D ~ C(n, M-2) for exact momentum conservation.  Under the
    modulo-M reading the momentum constraint only splits the C(N+M-1, M-1)
    compositions into M nearly equal residue classes, so D ~ N^{M-1}/(M (M-1)!)."""
    for M, N in [(5, 40), (7, 30)]:
        comp = math.comb(N + M - 1, M - 1)
        for P in range(M):
            assert abs(orc.sector_dim(M, N, P) * M / comp - 1) < 0.01


def gen_function_dims_exact(M, N):
    """Exact-momentum sector sizes from prod_i 1/(1 - t x^{label_i}) without any
    modulus: dict P -> #kets with N particles and label sum P."""
    lab = [int(x) for x in wl.mode_labels(M)]
    c = {(0, 0): 1}
    for i in range(M):
        new = {}
        for (n, k), cnt in c.items():
            for v in range(0, N - n + 1):
                key = (n + v, k + v * lab[i])
                new[key] = new.get(key, 0) + cnt
        c = new
    return {k: cnt for (n, k), cnt in c.items() if n == N}


def test_exact_sector_dims_match_generating_function_and_residue_classes():
    """Exact momentum (Sec. III B): sizes from the generating function, and the
    exact sectors with P = P0 (mod M) partition the mod-M sector P0."""
    for M, N in [(1, 4), (3, 6), (5, 6), (5, 9), (7, 5), (4, 5)]:
        ref = gen_function_dims_exact(M, N)
        lab = wl.mode_labels(M)
        for P in range(int(lab.min()) * N - 2, int(lab.max()) * N + 3):
            assert orc.sector_dim(M, N, P, exact=True) == ref.get(P, 0), (M, N, P)
        for P0 in range(M):
            assert sum(d for P, d in ref.items() if (P - P0) % M == 0) == orc.sector_dim(M, N, P0)


def test_exact_basis_is_sorted_and_in_sector():
    b = orc.sector_basis(5, 6, 1, exact=True)
    keys = [tuple(r) for r in b]
    assert len(keys) > 0 and keys == sorted(keys) and len(set(keys)) == len(keys)
    for r in b:
        assert orc.sector_of(r, exact=True) == (6, 1)
    sp_ = orc.Space(5, orc.all_sectors(5, 0, 4, exact=True), exact=True)
    assert sp_.total == sum(math.comb(N + 4, 4) for N in range(5))  # every ket once
    for k in (0, 17, sp_.total - 1):
        assert sp_.index_of(sp_.basis[k]) == k


def test_exact_coupling_rule():
    M = 5
    assert orc.check_coupling(M, wl.contact_coupling(M, 0.1, exact=True), exact=True)
    assert not orc.check_coupling(M, wl.contact_coupling(M, 0.1), exact=True)  # umklapp terms
    assert orc.check_coupling(M, wl.contact_coupling(M, 0.1, exact=True))  # exact implies mod M


@pytest.mark.parametrize("case", ["contact", "long_range"])
def test_exact_sector_hamiltonian_and_moments_match_tensor_product(case):
    """Exact-momentum sectors are closed under an exactly conserving H, which the
    oracle applies literally; moments of a multi-sector exact space follow the
    full Fock-space operators."""
    M, N = 5, 4
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.3, exact=True) if case == "contact" else wl.long_range_coupling(M, 0.7, exact=True)
    Hf = fock_hamiltonian(M, N, w, L)
    for P in range(-2 * N, 2 * N + 1):
        sp_ = orc.Space(M, [(N, P)], exact=True)
        if sp_.total == 0:
            continue
        Hs = orc.h_dense(sp_, 0, w, L)
        idx = [full_index(o, N) for o in sp_.basis]
        ref = Hf[idx][:, idx].toarray()
        np.testing.assert_allclose(Hs, ref, atol=1e-13, rtol=0)
        col_mass = np.asarray(abs(Hf[:, idx]).sum(axis=0)).ravel()
        np.testing.assert_allclose(col_mass, np.abs(ref).sum(axis=0), atol=1e-12)
    # moments on all exact sectors with N <= 3 against the tensor-product operators
    cut = 3
    sp_ = orc.Space(M, orc.all_sectors(M, 0, cut, exact=True), exact=True)
    rng = np.random.default_rng(8)
    psi = rng.standard_normal(sp_.total) + 1j * rng.standard_normal(sp_.total)
    full = np.zeros((cut + 1) ** M, dtype=np.complex128)
    full[[full_index(o, cut) for o in sp_.basis]] = psi
    a = fock_ops(M, cut)
    mo = orc.moments(sp_, psi)
    for i in range(M):
        assert abs(mo["a"][i] - np.vdot(full, a[i] @ full)) < 1e-12
        for j in range(M):
            assert abs(mo["Mij"][i, j] - np.vdot(full, a[i].conj().T @ (a[j] @ full))) < 1e-12
            assert abs(mo["aa"][i, j] - np.vdot(full, a[i] @ (a[j] @ full))) < 1e-12


def test_minimal_image_long_range():
    """Minimal image on the ring: |d| <= M/2, so labels -3 and 3 of M = 7 are one apart."""
    M = 7
    L = wl.long_range_coupling(M, 1.0, min_image=True)
    lab = list(wl.mode_labels(M))
    p, r = lab.index(-3), lab.index(3)
    q = lab.index(0)
    s = [i for i in range(M) if (lab[p] + lab[q] - lab[r] - lab[i]) % M == 0][0]
    assert abs(L[p, q, r, s] - (-1.0 / M)) < 1e-15
    assert abs(wl.long_range_coupling(M, 1.0)[p, q, r, s] - (-1.0 / (M * 36))) < 1e-15


def test_basis_is_sorted_and_in_sector():
    b = orc.sector_basis(5, 6, 0)
    assert b.shape == (42, 5)
    keys = [tuple(r) for r in b]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    for r in b:
        assert orc.sector_of(r) == (6, 0)


# ---------------------------------------------------- Hamiltonian vs Fock space

@pytest.mark.parametrize("case", ["random", "contact", "long_range", "paper"])
def test_sector_hamiltonian_matches_tensor_product_construction(case):
    rng = np.random.default_rng(1)
    if case == "random":
        M, N = 3, 4
        w = rng.standard_normal(M)
        L = random_hermitian_coupling(M, rng)
    elif case == "contact":
        M, N = 5, 3
        w = wl.dispersion_quadratic(M)
        L = wl.contact_coupling(M, -0.3)
    elif case == "long_range":
        M, N = 5, 3
        w = wl.dispersion_abs(M)
        L = wl.long_range_coupling(M, 0.7)
    else:
        M, N = 4, 3
        w = rng.standard_normal(M)
        L = wl.paper_coupling(M, -0.2, 0.05)
    Hf = fock_hamiltonian(M, N, w, L)
    for P in range(M):
        sp_ = orc.Space(M, [(N, P)])
        if sp_.total == 0:
            continue
        Hs = orc.h_dense(sp_, 0, w, L)
        idx = [full_index(o, N) for o in sp_.basis]
        ref = Hf[idx][:, idx].toarray()
        np.testing.assert_allclose(Hs, ref, atol=1e-13, rtol=0)
        # the sector is closed under H: no amplitude leaks to other kets
        col_mass = np.asarray(abs(Hf[:, idx]).sum(axis=0)).ravel()
        np.testing.assert_allclose(col_mass, np.abs(ref).sum(axis=0), atol=1e-12)


def test_dagger_is_adjoint():
    rng = np.random.default_rng(2)
    M = 5
    L = random_hermitian_coupling(M, rng)
    L[0, 1, 2, 4] += 0.3  # break Hermiticity deliberately: dagger must still be the adjoint
    L = L * wl._conserving(M)
    w = rng.standard_normal(M)
    sp_ = orc.Space(M, [(4, 1)])
    x = rng.standard_normal(sp_.total) + 1j * rng.standard_normal(sp_.total)
    y = rng.standard_normal(sp_.total) + 1j * rng.standard_normal(sp_.total)
    lhs = np.vdot(y, orc.apply_h(sp_, w, L, x))
    rhs = np.vdot(orc.apply_h(sp_, w, L, y, dagger=True), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_non_conserving_coupling_rejected():
    M = 5
    L = np.zeros((M,) * 4, dtype=np.complex128)
    L[0, 0, 0, 1] = 1.0
    assert not orc.check_coupling(M, L)
    assert orc.check_coupling(M, wl.contact_coupling(M, 0.1))


# ------------------------------------------------------------- integrator

def test_rk4_discrete_exact_on_diagonal_hamiltonian():
    """For diagonal H every amplitude is multiplied by R(-i E dt) per step."""
    M = 3
    w = np.array([0.7, -1.3, 2.1])
    L = np.zeros((M,) * 4, dtype=np.complex128)
    sp_ = orc.Space(M, orc.all_sectors(M, 0, 6))
    rng = np.random.default_rng(3)
    psi0 = rng.standard_normal(sp_.total) + 1j * rng.standard_normal(sp_.total)
    E = sp_.basis @ w
    dt, k = 1e-2, 300
    ref = psi0 * R4(-1j * E * dt) ** k
    got = orc.rk4(sp_, w, L, psi0, dt, k)
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)


def test_rk4_equals_matrix_polynomial_on_interacting_sector():
    M, N = 5, 4
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.4)
    sp_ = orc.Space(M, [(N, 1)])
    Hs = orc.h_dense(sp_, 0, w, L)
    lam, V = np.linalg.eigh(Hs)
    rng = np.random.default_rng(4)
    psi0 = rng.standard_normal(sp_.total) + 1j * rng.standard_normal(sp_.total)
    dt, k = 2e-3, 400
    ref = V @ (R4(-1j * lam * dt) ** k * (V.conj().T @ psi0))
    got = orc.rk4(sp_, w, L, psi0, dt, k)
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)


def test_taylor_order4_equals_classic_rk4():
    """For a linear H the order-4 Taylor step and the classic four stages are one polynomial."""
    M = 5
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.3)
    sp_ = orc.Space(M, orc.all_sectors(M, 2, 4))
    rng = np.random.default_rng(11)
    psi0 = rng.standard_normal(sp_.total) + 1j * rng.standard_normal(sp_.total)
    got = orc.taylor(sp_, w, L, psi0, 3e-3, 40, 4)
    ref = orc.rk4(sp_, w, L, psi0, 3e-3, 40)
    assert np.linalg.norm(got - ref) < 1e-13 * np.linalg.norm(ref)


def test_taylor_order2_discrete_exact_on_diagonal_hamiltonian():
    """Second-order Taylor (Sec. III B's step with the 1/2 restored) multiplies each
    amplitude of a diagonal H by 1 + x + x^2/2, x = -i E dt, per step."""
    M = 3
    w = np.array([0.7, -1.3, 2.1])
    L = np.zeros((M,) * 4, dtype=np.complex128)
    sp_ = orc.Space(M, orc.all_sectors(M, 0, 6))
    rng = np.random.default_rng(12)
    psi0 = rng.standard_normal(sp_.total) + 1j * rng.standard_normal(sp_.total)
    x = -1j * (sp_.basis @ w) * 1e-2
    ref = psi0 * (1 + x + x * x / 2) ** 200
    got = orc.taylor(sp_, w, L, psi0, 1e-2, 200, 2)
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)


def test_taylor_order3_equals_matrix_polynomial_on_interacting_sector():
    M, N = 5, 4
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.4)
    sp_ = orc.Space(M, [(N, 1)])
    lam, V = np.linalg.eigh(orc.h_dense(sp_, 0, w, L))
    rng = np.random.default_rng(13)
    psi0 = rng.standard_normal(sp_.total) + 1j * rng.standard_normal(sp_.total)
    x = -1j * lam * 2e-3
    ref = V @ ((1 + x + x ** 2 / 2 + x ** 3 / 6) ** 300 * (V.conj().T @ psi0))
    got = orc.taylor(sp_, w, L, psi0, 2e-3, 300, 3)
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)


def test_norm_decay_and_energy_under_rk4():
    """|R(iy)|^2 = 1 - y^6/72 + y^8/576 per eigencomponent: norm decays only at O(dt^6)."""
    y = 0.3
    assert abs(abs(R4(-1j * y)) ** 2 - (1 - y ** 6 / 72 + y ** 8 / 576)) < 1e-15
    M, N = 5, 6
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.1)
    sp_ = orc.Space(M, [(N, 0)])
    psi0 = orc.number_state(sp_, [0, 2, 2, 2, 0])
    psi = orc.rk4(sp_, w, L, psi0, 1e-3, 2000)
    assert abs(np.vdot(psi, psi).real - 1) < 1e-12
    e0 = orc.observables(sp_, psi0, w, L)["H"]
    e1 = orc.observables(sp_, psi, w, L)["H"]
    assert abs(e1 - e0) < 1e-10 * abs(e0)


# ------------------------------------------------- single-mode Kerr closed forms

def kerr_exact(space, w, L, psi0, t):
    """Exact propagation exp(-iHt) psi0 for the diagonal single-mode H."""
    E = np.array([orc.h_dense(space, s, w, L).diagonal() for s in range(len(space.sectors))], dtype=object)
    E = np.concatenate([np.asarray(e, dtype=np.complex128) for e in E]).real
    return np.exp(-1j * E * t) * psi0


@pytest.mark.parametrize("a0", [1.3 * np.exp(0.4j), 0.9 - 1.1j])
def test_single_mode_kerr_closed_forms(a0):
    """<a(t)> = a0 e^{-iwt} exp(|a0|^2 (e^{-2iLt} - 1)), <a^2(t)> = a0^2 e^{-i(2w+2L)t}
    exp(|a0|^2 (e^{-4iLt} - 1)), Q(t) = 1 - exp(2|a0|^2 (cos 2Lt - 1)),
    for H = w n + L a^dag a^dag a a and a coherent start."""
    w, Lk = 0.7, 0.13
    L = np.full((1, 1, 1, 1), Lk, dtype=np.complex128)
    space = orc.Space(1, [(N, 0) for N in range(0, 45)])
    psi0, kept = orc.coherent_state(space, [a0])
    assert abs(kept - 1) < 1e-15
    n0 = abs(a0) ** 2
    for t in [0.0, 0.5, 2.0, 7.3]:
        psi = kerr_exact(space, [w], L, psi0, t)
        ob = orc.observables(space, psi)
        a_ref = a0 * np.exp(-1j * w * t) * np.exp(n0 * (np.exp(-2j * Lk * t) - 1))
        aa_ref = a0 ** 2 * np.exp(-1j * (2 * w + 2 * Lk) * t) * np.exp(n0 * (np.exp(-4j * Lk * t) - 1))
        Q_ref = 1 - np.exp(2 * n0 * (np.cos(2 * Lk * t) - 1))
        assert abs(ob["a"][0] - a_ref) < 1e-12
        assert abs(ob["aa"][0, 0] - aa_ref) < 1e-12
        assert abs(ob["Q"] - Q_ref) < 1e-12
        assert abs(ob["n_tot"] - n0) < 1e-12
        V_ref = 1 + 2 * (n0 - abs(a_ref) ** 2) - 2 * abs(aa_ref - a_ref ** 2)
        assert abs(ob["Vminus_modes"][0] - V_ref) < 1e-11
        assert abs(ob["Vminus_p"] - V_ref) < 1e-11


def test_single_mode_kerr_rk4_converges_to_closed_form():
    """The oracle's RK4 approaches the closed form at the O(dt^4) rate."""
    w, Lk, a0 = 0.5, 0.1, 1.1 + 0.3j
    L = np.full((1, 1, 1, 1), Lk, dtype=np.complex128)
    space = orc.Space(1, [(N, 0) for N in range(0, 40)])
    psi0, _ = orc.coherent_state(space, [a0])
    t = 1.0
    a_ref = a0 * np.exp(-1j * w * t) * np.exp(abs(a0) ** 2 * (np.exp(-2j * Lk * t) - 1))
    errs = []
    for dt in (1e-2, 5e-3):
        psi = orc.rk4(space, [w], L, psi0, dt, int(round(t / dt)))
        errs.append(abs(orc.observables(space, psi)["a"][0] - a_ref))
    assert errs[0] < 1e-6
    assert 10 < errs[0] / errs[1] < 22  # ~2^4


def test_vminus_bajer_approximation_and_squeezing_onset():
    """Eq. (VminusBajer) approximates the exact single-mode V_-(tau), tau = n_tot|chi|t,
    with chi = L for L = Lambda/2 (a factor-two slip in the coupling fails this);
    V_- = 0.8 is reached near tau = 0.05 (Sec. II E: t_sqz ~ 0.05/(n_tot|chi|), the
    linear estimate 1 - 4 tau; the curvature of Eq. (VminusBajer) moves it to ~0.056)."""
    n_tot, Lk = 25.0, -0.004
    L = np.full((1, 1, 1, 1), Lk, dtype=np.complex128)
    space = orc.Space(1, [(N, 0) for N in range(0, 100)])
    psi0, _ = orc.coherent_state(space, [math.sqrt(n_tot)])
    chi = abs(Lk)
    worst = 0.0
    taus = np.linspace(0.0, 0.3, 31)
    vs = []
    for tau in taus:
        t = tau / (n_tot * chi)
        ob = orc.observables(space, kerr_exact(space, [0.0], L, psi0, t))
        s = math.sqrt(1 + 4 * tau ** 2)
        v_b = 1 - 4 * tau * s + 8 * tau ** 2 + 8 * tau ** 3 * (5 + 12 * tau ** 2) / (n_tot * s) - 16 * tau ** 4 / n_tot
        worst = max(worst, abs(ob["Vminus_p"] - v_b))
        vs.append(ob["Vminus_p"])
    assert worst < 1e-3
    tau_sqz = np.interp(0.8, vs[::-1], taus[::-1])
    assert abs(tau_sqz - 0.05) < 0.01


def test_squeezing_analysis_on_known_series():
    """Onset of a line (exact under linear interpolation), the vertex of a sampled
    parabola, an end minimum, and the never-squeezed case."""
    dt = 0.01
    t = np.arange(100) * dt
    r = orc.squeezing(1 - 4 * t, dt, 0.8)
    assert r["flag"] == orc.CROSSED and abs(r["t_sqz"] - 0.05) < 1e-12
    r = orc.squeezing((t - 0.3137) ** 2 + 0.25, dt, 0.8)
    assert r["flag"] == orc.AT_START and abs(r["t_min"] - 0.3137) < 1e-12 and abs(r["v_min"] - 0.25) < 1e-12
    r = orc.squeezing(1 - t, dt, 0.0)
    assert r["flag"] == orc.NOT_CROSSED and math.isnan(r["t_sqz"])
    assert r["t_min"] == t[-1] and r["v_min"] == 1 - t[-1]


def test_interaction_per_occupation_closed_forms():
    """Single mode: n_tot chi = L n_tot (chi = L, Sec. II E).  Contact C/M on two
    modes p = -1, +1 with amplitude a: six conserving tuples, n_tot chi = 3 C a^2 / M."""
    assert abs(orc.interaction_per_occupation(np.full((1,) * 4, -0.004), [5.0]) - (-0.004 * 25.0)) < 1e-15
    M, C, a = 7, -0.3, 1.7
    z = np.zeros(M, dtype=np.complex128)
    lab = list(wl.mode_labels(M))
    z[lab.index(-1)] = z[lab.index(1)] = a * np.exp(0.4j)
    got = orc.interaction_per_occupation(wl.contact_coupling(M, C), z)
    assert abs(got - 3 * C * a * a / M) < 1e-14


def test_squeezing_workload_interaction_scales_with_strength_and_occupation():
    """n_tot chi of the squeezing workloads is proportional to G n_tot (fixed profile),
    so one value at G = 1 fixes the strength that holds |n_tot chi| = 0.242 (Sec. IV E)."""
    for M in (5, 7):
        base = orc.interaction_per_occupation(wl.squeezing_coherent(1.0, M=M).L, wl.squeezing_coherent(1.0, M=M).z)
        for n, G in ((3, 0.7), (8, 1.9), (20, 0.05)):
            W = wl.squeezing_coherent(n, M=M, G=G)
            assert abs(orc.interaction_per_occupation(W.L, W.z) - base * G * n) < 1e-13 * abs(base * G * n)
            W = wl.squeezing_coherent(n, M=M, G=0.242 / abs(base * n))
            assert abs(abs(orc.interaction_per_occupation(W.L, W.z)) - 0.242) < 1e-13


def test_fits_recover_exact_laws():
    x = np.array([20.0, 40.0, 80.0, 160.0])
    c0, c1 = orc.fit(x, 0.919 * x ** -0.194, "power")
    assert abs(c0 - 0.919) < 1e-12 and abs(c1 + 0.194) < 1e-12
    c0, c1 = orc.fit(x, 0.0120 + 0.0833 * np.log(x), "log")
    assert abs(c0 - 0.0120) < 1e-12 and abs(c1 - 0.0833) < 1e-12


def test_single_mode_squeezing_onset_from_series():
    """The exact single-mode evolution sampled in time: the onset of the series
    lands at tau = n_tot |chi| t ~ 0.05 (Sec. II E), and t_min follows Eq.
    (VminusBajer)'s minimum to within the sampling."""
    n_tot, Lk = 25.0, -0.004
    L = np.full((1, 1, 1, 1), Lk, dtype=np.complex128)
    space = orc.Space(1, [(N, 0) for N in range(0, 100)])
    psi0, _ = orc.coherent_state(space, [math.sqrt(n_tot)])
    chi = abs(orc.interaction_per_occupation(L, [math.sqrt(n_tot)])) / n_tot
    dtau = 0.005
    taus = np.arange(0, 0.4, dtau)
    vs = [orc.observables(space, kerr_exact(space, [0.0], L, psi0, tau / (n_tot * chi)))["Vminus_p"] for tau in taus]
    r = orc.squeezing(vs, dtau, 0.8)
    assert r["flag"] == orc.CROSSED and abs(r["t_sqz"] - 0.05) < 0.01
    s = np.sqrt(1 + 4 * taus ** 2)
    vb = 1 - 4 * taus * s + 8 * taus ** 2 + 8 * taus ** 3 * (5 + 12 * taus ** 2) / (n_tot * s) - 16 * taus ** 4 / n_tot
    assert abs(r["t_min"] - taus[int(np.argmin(vb))]) < 2 * dtau


# ------------------------------------------------------------- initial states

def test_coherent_layer_weights_are_poisson():
    M = 3
    z = np.array([0.8 + 0.2j, -0.5j, 1.1])
    space = orc.Space(M, orc.all_sectors(M, 0, 30))
    amp = orc.coherent_amplitudes(space, z)
    lam = float(np.sum(np.abs(z) ** 2))
    Ns = space.basis.sum(axis=1)
    for N in range(12):
        wN = float(np.sum(np.abs(amp[Ns == N]) ** 2))
        assert abs(wN - math.exp(-lam) * lam ** N / math.factorial(N)) < 1e-14


def test_coherent_t0_observables():
    M = 5
    z = np.array([0, 1.2j, 0.9, -0.7 + 0.4j, 0])
    space = orc.Space(M, orc.all_sectors(M, 0, 25))
    psi, kept = orc.coherent_state(space, z)
    ob = orc.observables(space, psi)
    n_tot = float(np.sum(np.abs(z) ** 2))
    assert abs(kept - 1) < 1e-12
    np.testing.assert_allclose(ob["a"], z, atol=1e-12)
    assert abs(ob["Q"]) < 1e-12
    assert abs(ob["lam_p"] - n_tot) < 1e-11
    assert abs(ob["Vminus_p"] - 1) < 1e-11
    np.testing.assert_allclose(ob["Vminus_modes"], 1.0, atol=1e-11)
    # principal eigenvector is z^*/|z| up to a phase (Sec. II D)
    ov = abs(np.vdot(np.conj(z) / math.sqrt(n_tot), ob["xi"]))
    assert abs(ov - 1) < 1e-12


def test_field_number_state_t0():
    M = 5
    n = np.array([0, 3, 2, 1, 0])
    z = np.sqrt(n) * np.exp(1j * np.array([0, 0.3, 1.9, -2.2, 0]))
    n_tot = int(n.sum())
    space = orc.Space(M, [(n_tot, P) for P in range(M)])
    psi = orc.field_number_state(space, z, n_tot)
    assert abs(np.vdot(psi, psi).real - 1) < 1e-13  # multinomial theorem
    ob = orc.observables(space, psi)
    np.testing.assert_allclose(ob["a"], 0, atol=1e-14)
    assert abs(ob["Q"] - 1) < 1e-13
    assert abs(ob["lam_p"] - n_tot) < 1e-12
    np.testing.assert_allclose(ob["Mij"], np.outer(np.conj(z), z), atol=1e-12)


def test_number_state_t0():
    M = 5
    occ = [0, 2, 2, 2, 0]
    space = orc.Space(M, [(6, 0)])
    ob = orc.observables(space, orc.number_state(space, occ))
    np.testing.assert_allclose(ob["Mij"], np.diag(occ), atol=1e-15)
    assert abs(ob["lam_p"] - 2) < 1e-14 and ob["gap"] < 1e-12
    assert abs(ob["Q"] - 1) < 1e-15


def test_moments_match_fock_space_operators():
    """<a_i>, <a_i^dag a_j>, <a_i a_j> against the tensor-product construction."""
    M, cutoff = 3, 5
    rng = np.random.default_rng(5)
    space = orc.Space(M, orc.all_sectors(M, 0, cutoff))
    psi = rng.standard_normal(space.total) + 1j * rng.standard_normal(space.total)
    full = np.zeros((cutoff + 1) ** M, dtype=np.complex128)
    for k, o in enumerate(space.basis):
        full[full_index(o, cutoff)] = psi[k]
    a = fock_ops(M, cutoff)
    # only kets with N <= cutoff are held: truncate operators the same way
    keep = np.zeros_like(full, dtype=bool)
    keep[[full_index(o, cutoff) for o in space.basis]] = True
    proj = lambda v: np.where(keep, v, 0)
    m = orc.moments(space, psi)
    for i in range(M):
        assert abs(m["a"][i] - np.vdot(full, proj(a[i] @ full))) < 1e-11
        for j in range(M):
            assert abs(m["Mij"][i, j] - np.vdot(full, proj(a[i].conj().T @ (a[j] @ full)))) < 1e-11
            assert abs(m["aa"][i, j] - np.vdot(full, proj(a[i] @ (a[j] @ full)))) < 1e-11


# ---------------------------------------------------------------- mean field

def test_meanfield_free_and_single_mode():
    M = 5
    w = wl.dispersion_quadratic(M)
    z = np.array([0.3, 1j, 0.5 - 0.5j, 2.0, 0.1j])
    L0 = np.zeros((M,) * 4, dtype=np.complex128)
    traj = orc.meanfield(w, L0, z, 1e-3, 3000, every=1000)
    for k, t in enumerate([0, 1, 2, 3]):
        np.testing.assert_allclose(traj[k], z * np.exp(-1j * w * t), atol=1e-10)
    Lk, a0 = 0.2, 1.3 + 0.2j
    L1 = np.full((1, 1, 1, 1), Lk, dtype=np.complex128)
    traj = orc.meanfield([0.4], L1, [a0], 1e-3, 2000, every=2000)
    ref = a0 * np.exp(-1j * (0.4 + 2 * Lk * abs(a0) ** 2) * 2.0)
    assert abs(traj[-1][0] - ref) < 1e-10


def test_quantum_free_coherent_follows_classical_field():
    """At L = 0 the coherent state stays coherent: <a_p(t)> = z_p e^{-i w_p t}."""
    M = 3
    w = np.array([0.5, 0.0, 0.5])
    L0 = np.zeros((M,) * 4, dtype=np.complex128)
    z = np.array([0.6, 0.8j, -0.4])
    space = orc.Space(M, orc.all_sectors(M, 0, 22))
    psi0, _ = orc.coherent_state(space, z)
    psi = orc.rk4(space, w, L0, psi0, 1e-3, 1000)
    ob = orc.observables(space, psi)
    np.testing.assert_allclose(ob["a"], z * np.exp(-1j * w * 1.0), atol=1e-10)
    assert abs(ob["Q"]) < 1e-10


# ------------------------------------------------------------------ breaktime

def test_breaktime_rule():
    t, f = orc.breaktime([0.0, 0.05, 0.08, 0.12, 0.3], 0.5, 0.1)
    assert f == orc.CROSSED and abs(t - (1.0 + 0.5 * 0.5)) < 1e-15
    assert orc.breaktime([0.2, 0.3], 1.0, 0.1) == (0.0, orc.AT_START)
    t, f = orc.breaktime([0.0, 0.01], 1.0, 0.1)
    assert f == orc.NOT_CROSSED and math.isnan(t)


# ------------------------------------------------------------------- adjoint

def test_rk4_step_adjoint_matches_finite_differences():
    """The oracle's discrete adjoint of one RK4 step against central differences."""
    M, N = 3, 3
    rng = np.random.default_rng(6)
    w = rng.standard_normal(M)
    L0 = wl.contact_coupling(M, 1.0)
    C = -0.3
    space = orc.Space(M, [(N, P) for P in range(M)])
    psi = rng.standard_normal(space.total) + 1j * rng.standard_normal(space.total)
    c = rng.standard_normal(space.total) + 1j * rng.standard_normal(space.total)
    dt = 0.05

    def loss(Cv, wv, ps):
        out = orc.rk4(space, wv, Cv * L0, ps, dt, 1)
        return float(np.vdot(c, out).real)

    lam_next = c / 2  # d Re<c, psi'> / d psi'^* = c/2
    nop = lambda v: orc.apply_h(space, np.zeros(M), L0, v)
    dws = [lambda v, i=i: orc.apply_mode_op(space, v, "n", i) for i in range(M)]
    lam0, g = orc.rk4_step_adjoint(space, w, C * L0, psi, lam_next, dt, [nop] + dws)
    h = 1e-6
    fd_C = (loss(C + h, w, psi) - loss(C - h, w, psi)) / (2 * h)
    assert abs(g[0] - fd_C) < 1e-7 * max(1, abs(fd_C))
    for i in range(M):
        e = np.zeros(M)
        e[i] = h
        fd = (loss(C, w + e, psi) - loss(C, w - e, psi)) / (2 * h)
        assert abs(g[1 + i] - fd) < 1e-7 * max(1, abs(fd))
    # state cotangent: d loss = 2 Re <lam0, d psi>
    d = rng.standard_normal(space.total) + 1j * rng.standard_normal(space.total)
    fd = (loss(C, w, psi + h * d) - loss(C, w, psi - h * d)) / (2 * h)
    assert abs(2 * np.vdot(lam0, d).real - fd) < 1e-7 * max(1, abs(fd))


def test_single_row_application_matches_push_form():
    """The per-row form used for sampled checks of huge sectors equals the
    push form, for a non-Hermitian coupling too (no symmetry is assumed)."""
    rng = np.random.default_rng(7)
    M = 5
    L = random_hermitian_coupling(M, rng)
    L[0, 1, 2, 4] += 0.3 - 0.1j
    L = L * wl._conserving(M)
    w = rng.standard_normal(M)
    space = orc.Space(M, [(5, 2)])
    psi = rng.standard_normal(space.total) + 1j * rng.standard_normal(space.total)
    full = orc.apply_h(space, w, L, psi)
    rows = [0, 3, space.total // 2, space.total - 1]
    np.testing.assert_allclose(orc.apply_h_rows(space, 0, w, L, psi, rows), full[rows], atol=1e-12)


def test_count_terms_equals_dense_structure():
    M, N = 5, 4
    w = wl.dispersion_quadratic(M)
    L = wl.long_range_coupling(M, 0.3)
    space = orc.Space(M, [(N, P) for P in range(M)])
    nnz = 0
    for s in range(M):
        Hd = orc.h_dense(space, s, w, L)
        nnz += int((np.abs(Hd - np.diag(np.diag(Hd))) > 0).sum()) + Hd.shape[0]
    assert orc.count_terms(space, L) == nnz


@pytest.mark.parametrize("kind", ["Q", "PO"])
def test_oracle_adjoint_gradient_matches_finite_differences(kind):
    """The oracle's exact discrete adjoint (every state stored) against central
    differences of the oracle's own loss, for the coupling scale, every w_p and
    every Re z_k, Im z_k."""
    M = 3
    L0 = wl.contact_coupling(M, 1.0)
    w = np.array([0.3, -0.2, 0.7])
    z = np.array([0.6 + 0.2j, -0.4j, 0.5])
    scale, dt, steps = -0.3, 0.02, 12
    space = orc.Space(M, orc.all_sectors(M, 0, 9))

    def loss_of(sc, wv, zv):
        psi, _ = orc.coherent_state(space, zv)
        psi = orc.rk4(space, wv, sc * L0, psi, dt, steps)
        return orc.loss_and_seed(space, psi, kind)[0]

    loss, gs, gw, gz = orc.adjoint_gradient(space, w, L0, scale, z, dt, steps, kind)
    assert abs(loss - loss_of(scale, w, z)) < 1e-14
    h = 1e-6
    fd = (loss_of(scale + h, w, z) - loss_of(scale - h, w, z)) / (2 * h)
    assert abs(gs - fd) < 1e-7 * max(1, abs(fd))
    for q in range(M):
        e = np.zeros(M)
        e[q] = h
        fd = (loss_of(scale, w + e, z) - loss_of(scale, w - e, z)) / (2 * h)
        assert abs(gw[q] - fd) < 1e-7 * max(1, abs(fd))
    for k in range(M):
        for unit, part in ((1.0, gz[k].real), (1j, gz[k].imag)):
            e = np.zeros(M, dtype=np.complex128)
            e[k] = unit * h
            fd = (loss_of(scale, w, z + e) - loss_of(scale, w, z - e)) / (2 * h)
            assert abs(part - fd) < 1e-7 * max(1, abs(fd))


# ------------------------------------ principal-mode squeezing with a complex xi

def principal_kerr_state(space, phi, a0, w, Lk, t):
    """A state of one effective mode b = (a_0 + e^{i phi} a_1) / sqrt(2) (the
    other modes empty) whose amplitudes on |n>_b = (b^dag)^n / sqrt(n!) |0> are
    the single-mode Kerr ones c_n(t) = e^{-|a0|^2/2} a0^n / sqrt(n!)
    e^{-i (w n + Lk n (n - 1)) t}.  Expanded in the Fock basis of the M modes,
    (b^dag)^n / sqrt(n!) |0> = 2^{-n/2} sum_k sqrt(C(n, k)) e^{-i phi (n - k)}
    |k, n - k, 0, ...>, so the state spreads over every (N, P) sector it meets."""
    psi = np.zeros(space.total, dtype=np.complex128)
    n_max = int(space.basis.sum(axis=1).max())
    for n in range(n_max + 1):
        cn = (np.exp(-abs(a0) ** 2 / 2) * a0 ** n / math.sqrt(math.factorial(n))
              * np.exp(-1j * (w * n + Lk * n * (n - 1)) * t))
        for k in range(n + 1):
            occ = np.zeros(space.M, dtype=np.int32)
            occ[0], occ[1] = k, n - k
            psi[space.index_of(occ)] += cn * 2.0 ** (-n / 2) * math.sqrt(math.comb(n, k)) * np.exp(-1j * phi * (n - k))
    return psi


def principal_squeezing_errors(ob, phi, a0, w, Lk, t):
    """Deviations of an observables dict from the one-mode closed forms of b:
    V_-(a^p) (Eq. generalVminus with a^p of Eq. a_op), lam_p = <b^dag b> = |a0|^2
    and xi^p ~ (1, e^{i phi}, 0, ...) / sqrt(2) up to a phase."""
    n0 = abs(a0) ** 2
    b = a0 * np.exp(-1j * w * t) * np.exp(n0 * (np.exp(-2j * Lk * t) - 1))
    bb = a0 ** 2 * np.exp(-1j * (2 * w + 2 * Lk) * t) * np.exp(n0 * (np.exp(-4j * Lk * t) - 1))
    v_ref = 1 + 2 * (n0 - abs(b) ** 2) - 2 * abs(bb - b ** 2)
    xi_ref = np.zeros(len(ob["xi"]), dtype=np.complex128)
    xi_ref[0], xi_ref[1] = 1 / math.sqrt(2), np.exp(1j * phi) / math.sqrt(2)
    return (abs(ob["Vminus_p"] - v_ref), abs(ob["lam_p"] - n0), abs(abs(np.vdot(xi_ref, ob["xi"])) - 1))


PRINCIPAL_CASES = [(1.1, 1.3 * np.exp(0.4j), 0.7, 0.13, 0.9), (2.3, 0.9 - 1.1j, -0.2, -0.05, 3.1)]


@pytest.mark.parametrize("phi,a0,w,Lk,t", PRINCIPAL_CASES)
def test_principal_mode_squeezing_with_complex_eigenvector(phi, a0, w, Lk, t):
    """Eq. (a_op) with a non-real principal eigenvector: for a state that lives in
    the single mode b = (a_0 + e^{i phi} a_1) / sqrt(2), M_ij = <b^dag b> v_i^* v_j
    with v = (1, e^{-i phi}, 0) / sqrt(2) conjugated, so xi^p = (1, e^{i phi}, 0) /
    sqrt(2) (Sec. II D: xi^p is z^* / |z| for M_ij = z_i^* z_j) and a^p = b.
    V_-(a^p) must then equal the single-mode Kerr closed form; a conjugate slip on
    xi in either <dO^dag dO> or Var O gives V_- of another operator."""
    M = 3
    space = orc.Space(M, orc.all_sectors(M, 0, 34))
    psi = principal_kerr_state(space, phi, a0, w, Lk, t)
    assert abs(np.vdot(psi, psi).real - 1) < 1e-13  # Poisson tail beyond N = 34 below 1e-15
    ob = orc.observables(space, psi)
    dv, dl, dx = principal_squeezing_errors(ob, phi, a0, w, Lk, t)
    assert dv < 1e-11 and dl < 1e-11 and dx < 1e-11
    # xi is not real up to a phase: its two components differ in phase by phi
    assert abs(ob["xi"][1] / ob["xi"][0] - np.exp(1j * phi)) < 1e-9 and abs(np.sin(phi)) > 0.5
    # several (N, P) sectors carry weight: the three residues of P and many N
    held = {space.sectors[s] for s in range(len(space.sectors)) if np.linalg.norm(psi[space.sector_slice(s)]) > 1e-3}
    assert len({P for _, P in held}) == M and len({N for N, _ in held}) > 5


def test_principal_mode_pin_rejects_conjugated_eigenvector(monkeypatch):
    """The pin above fails when the oracle's principal eigenvector is conjugated
    (a^p = sum_k conj(xi_k) a_k instead of Eq. a_op): planted in the oracle by
    conjugating what its eigensolver returns."""
    phi, a0, w, Lk, t = PRINCIPAL_CASES[0]
    space = orc.Space(3, orc.all_sectors(3, 0, 34))
    psi = principal_kerr_state(space, phi, a0, w, Lk, t)
    eigh = np.linalg.eigh
    monkeypatch.setattr(orc.np.linalg, "eigh", lambda m: (eigh(m)[0], np.conj(eigh(m)[1])))
    dv, _, dx = principal_squeezing_errors(orc.observables(space, psi), phi, a0, w, Lk, t)
    assert dv > 1e-3 and dx > 1e-3


# ---------------------------------------- interacting multi-mode mean field

def classical_energy(w, L, a):
    """E(a) = sum_k w_k |a_k|^2 + sum_{pqrs} L_{pq;rs} a_p^* a_q^* a_r a_s: Eq. (Ham)
    with every operator replaced by its classical field value (Sec. III A)."""
    a = np.asarray(a, dtype=np.complex128)
    return (np.sum(np.asarray(w) * np.abs(a) ** 2)
            + np.einsum("pqrs,p,q,r,s->", np.asarray(L, dtype=np.complex128), a.conj(), a.conj(), a, a)).real


def meanfield_gradient_error(rhs, w, L, a, h=1e-5):
    """Largest deviation of i * rhs(a) from the Wirtinger gradient dE/da_k^* =
    (dE/dRe a_k + i dE/dIm a_k) / 2, by central differences of the classical
    energy: Eq. (classicalFieldEqns) is Hamilton's equation i da_k/dt = dE/da_k^*."""
    g = np.zeros(len(a), dtype=np.complex128)
    for k in range(len(a)):
        for unit, part in ((1.0, 1.0), (1j, 1j)):
            e = np.zeros(len(a), dtype=np.complex128)
            e[k] = unit * h
            g[k] += part * (classical_energy(w, L, a + e) - classical_energy(w, L, a - e)) / (4 * h)
    return float(np.max(np.abs(1j * rhs(w, L, a) - g)))


def long_range_asymmetric(M):
    """The gravity-like coupling on raw label differences: Hermitian, but neither
    symmetric under p <-> q nor under r <-> s, so the symmetrisation of Eq.
    (classicalFieldEqns) matters."""
    L = wl.long_range_coupling(M, 0.4)
    assert np.abs(L - L.transpose(1, 0, 2, 3)).max() > 1e-3 and np.abs(L - L.transpose(0, 1, 3, 2)).max() > 1e-3
    return L


def test_meanfield_rhs_is_the_energy_gradient():
    """The mean-field right-hand side at random points equals -i times the
    Wirtinger gradient of the classical energy, for the asymmetric long-range
    coupling (M = 5) and a random complex Hermitian coupling (M = 4)."""
    rng = np.random.default_rng(11)
    for M, L in ((5, long_range_asymmetric(5)), (4, random_hermitian_coupling(4, rng, 0.3))):
        w = rng.standard_normal(M)
        for _ in range(3):
            a = rng.standard_normal(M) + 1j * rng.standard_normal(M)
            assert meanfield_gradient_error(orc.mf_rhs, w, L, a) < 1e-8


def test_meanfield_conserves_occupation_and_energy():
    """Along an interacting M = 5 trajectory under the asymmetric long-range
    coupling, sum_k |a_k|^2 and the classical energy stay constant up to the RK4
    error, which falls as dt^4 (the energy drift halves dt -> ~1/16)."""
    M = 5
    w = wl.dispersion_quadratic(M)
    L = long_range_asymmetric(M)
    a0 = np.array([0.3 + 0.1j, 1.2j, 0.9, -0.7 + 0.4j, 0.2])
    N0, E0 = float(np.sum(np.abs(a0) ** 2)), classical_energy(w, L, a0)
    drift = []
    for dt in (4e-3, 2e-3):
        traj = orc.meanfield(w, L, a0, dt, int(round(8.0 / dt)), every=int(round(0.5 / dt)))
        # the interaction moves occupation between modes (the run is not trivial)
        assert np.abs(np.abs(traj[-1]) ** 2 - np.abs(a0) ** 2).max() > 0.05
        assert max(abs(float(np.sum(np.abs(x) ** 2)) - N0) for x in traj) < 1e-9
        drift.append(max(abs(classical_energy(w, L, x) - E0) for x in traj))
    assert drift[0] < 1e-7 and 8 < drift[0] / drift[1] < 40


def _rhs_unsymmetrised(w, L, a):
    return -1j * (np.asarray(w) * a + 2 * np.einsum("kqrs,q,r,s->k", L, np.conj(a), a, a))


def _rhs_wrong_axis(w, L, a):
    G = L + L.transpose(0, 1, 3, 2)
    return -1j * (np.asarray(w) * a + np.einsum("kqrs,q,r,s->k", G, np.conj(a), a, a))


def _rhs_conjugate_slip(w, L, a):
    G = L + L.transpose(1, 0, 2, 3)
    return -1j * (np.asarray(w) * a + np.einsum("kqrs,q,r,s->k", G, a, np.conj(a), a))


@pytest.mark.parametrize("mutant", [_rhs_unsymmetrised, _rhs_wrong_axis, _rhs_conjugate_slip])
def test_meanfield_pins_reject_planted_mistakes(mutant):
    """Mistakes planted in the oracle's mean-field right-hand side (the p <-> q
    symmetrisation dropped, symmetrised over r <-> s instead, a conjugate on the
    wrong field) fail the gradient pin and break energy conservation."""
    M = 5
    rng = np.random.default_rng(12)
    w = wl.dispersion_quadratic(M)
    L = long_range_asymmetric(M)
    a = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    assert meanfield_gradient_error(mutant, w, L, a) > 1e-3
    a0 = np.array([0.3 + 0.1j, 1.2j, 0.9, -0.7 + 0.4j, 0.2])
    E0 = classical_energy(w, L, a0)
    x = a0.copy()
    dt = 2e-3
    for _ in range(2000):  # classic RK4 with the mutant right-hand side
        k1 = mutant(w, L, x)
        k2 = mutant(w, L, x + 0.5 * dt * k1)
        k3 = mutant(w, L, x + 0.5 * dt * k2)
        k4 = mutant(w, L, x + dt * k3)
        x = x + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    drift_e = abs(classical_energy(w, L, x) - E0)
    drift_n = abs(float(np.sum(np.abs(x) ** 2)) - float(np.sum(np.abs(a0) ** 2)))
    assert drift_e > 1e-4 or drift_n > 1e-4


def test_row_parallel_rk4_equals_rk4():
    """The row-by-row RK4 of the timed CPU baseline (OpenMP over rows where the
    compiler has it) computes the same scheme as rk4: only the summation order of
    each row differs."""
    M = 5
    rng = np.random.default_rng(41)
    L = random_hermitian_coupling(M, rng, 0.2)
    w = rng.standard_normal(M)
    space = orc.Space(M, orc.all_sectors(M, 0, 7))
    psi = rng.standard_normal(space.total) + 1j * rng.standard_normal(space.total)
    a = orc.rk4(space, w, L, psi, 0.01, 5)
    b = orc.rk4_rows(space, w, L, psi, 0.01, 5)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)
    assert orc.threads() >= 1

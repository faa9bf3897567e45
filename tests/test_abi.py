"""The C ABI library loads here (no GPU needed) and exports every function
include/*.h declares; host-only entry points work without a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(qb_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    import paper_2111_00050_gb300._lib as L

    lib = L.lib()
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, n
    assert set(L.SIGNATURES) == set(names)


def test_obs_struct_layout_matches_header():
    import paper_2111_00050_gb300._lib as L

    M = L.QB_MAX_MODES
    assert ctypes.sizeof(L.QbObs) == 8 * (10 + 2 * M + 4 * M * M + 2 * M + M + M)


def test_header_constants_match_binding():
    """Every QB_* value constant of include/*.h equals the binding's constant of the
    same name."""
    import paper_2111_00050_gb300._lib as L

    found = 0
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            for name, value in re.findall(r"^#define (QB_[A-Z0-9_]+) (\d+)", open(os.path.join(inc, h)).read(), re.M):
                assert getattr(L, name) == int(value), name
                found += 1
    assert found >= 14


def test_host_only_entry_points():
    import paper_2111_00050_gb300 as qb

    assert qb.breaktime([0.0, 0.05, 0.08, 0.12, 0.3], 0.5, 0.1) == (1.25, qb.QB_CROSSED)
    assert qb.breaktime([0.2, 0.3], 1.0, 0.1) == (0.0, qb.QB_AT_START)
    t, f = qb.breaktime([0.0, 0.01], 1.0, 0.1)
    assert f == qb.QB_NOT_CROSSED and np.isnan(t)


def test_meanfield_matches_oracle():
    import oracle as orc
    import paper_2111_00050_gb300 as qb
    import workloads as wl

    M = 5
    w = wl.dispersion_quadratic(M)
    L = wl.long_range_coupling(M, 0.2)
    z = np.array([0.2, 1.0 + 0.5j, 0.7j, -0.4, 0.1])
    a = qb.meanfield(M, w, L, z, 1e-3, 500, 100)
    b = orc.meanfield(w, L, z, 1e-3, 500, 100)
    np.testing.assert_allclose(a, b, atol=1e-12)


@pytest.mark.parametrize("bad", ["nonhermitian", "nonconserving", "too_many_modes", "too_deep", "too_heavy"])
def test_model_validation_without_device(bad):
    import paper_2111_00050_gb300 as qb
    import workloads as wl

    M = 5
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.1)
    n_max = 4
    if bad == "nonhermitian":
        L = L.copy()
        L[0, 1, 2, 4] = 0.3j
    elif bad == "nonconserving":
        L = L.copy()
        L[0, 0, 0, 1] = 1.0
    elif bad == "too_many_modes":
        M = 17
        w, L = np.zeros(M), np.zeros((M,) * 4)
    elif bad == "too_deep":
        n_max = 1 << 13
    else:
        # packs into 64 bits (5 x 8), but the largest ket weight sqrt(150!/(30!)^5) is
        # 2^167: the weighted fp32-pair stage vectors could not hold psi / w
        n_max = 150
    with pytest.raises(qb.QbError) as e:
        qb.Space(M, w, L, 0, n_max)
    assert e.value.code in (1, 6)
    if bad == "too_heavy":
        assert e.value.code == qb.QB_EUNSUPPORTED and "ket weights" in str(e.value)


def test_squeezing_analysis_matches_oracle():
    """qb_squeezing, qb_interaction_per_occupation and qb_fit (host only) against
    the oracle's restatements on noisy series, random couplings and runs."""
    import oracle as orc
    import paper_2111_00050_gb300.api as api
    import workloads as wl

    rng = np.random.default_rng(4)
    dt = 0.02
    t = np.arange(60) * dt
    for k in range(5):
        v = 1 - 3 * t + 4 * t * t + 0.01 * rng.standard_normal(t.size)
        got, ref = api.squeezing(v, dt, 0.8), orc.squeezing(v, dt, 0.8)
        assert got["flag"] == ref["flag"] and abs(got["t_sqz"] - ref["t_sqz"]) < 1e-13
        assert abs(got["t_min"] - ref["t_min"]) < 1e-12 and abs(got["v_min"] - ref["v_min"]) < 1e-12
    M = 7
    for L in (wl.long_range_coupling(M, 0.3), wl.contact_coupling(M, -0.2), wl.long_range_coupling(M, 0.3, min_image=True)):
        z = rng.standard_normal(M) + 1j * rng.standard_normal(M)
        got = api.interaction_per_occupation(M, wl.dispersion_quadratic(M), L, z)
        assert abs(got - orc.interaction_per_occupation(L, z)) < 1e-13 * max(1, abs(got))
    x = np.array([4.0, 6.0, 8.0, 12.0, 20.0])
    y = 0.9 * x ** -0.2 * np.exp(0.01 * rng.standard_normal(x.size))
    for kind in ("power", "log"):
        np.testing.assert_allclose(api.fit(x, y, kind), orc.fit(x, y, kind), rtol=1e-12)


def test_null_space_is_refused_without_device():
    """Every entry point that takes a space refuses NULL with QB_EINVAL (the size
    queries with -1) before any device call, and names the fault in qb_last_error."""
    import paper_2111_00050_gb300._lib as L

    lib = L.lib()
    d = ctypes.c_double()
    i64 = ctypes.c_int64()
    i32 = ctypes.c_int()
    z = (ctypes.c_double * 32)()
    g = (ctypes.c_double * 32)()
    gl = (ctypes.c_double * (2 * 16 ** 4))()
    occ = (ctypes.c_int * 16)()
    obs = L.QbObs()
    series = (L.QbObs * 2)()
    scale = (ctypes.c_double * 1)(1.0)
    calls = {
        "qb_space_info": (None, ctypes.byref(i64), ctypes.byref(i32), ctypes.byref(i64)),
        "qb_space_sectors": (None, None, None, None, None),
        "qb_space_basis": (None, 0, 1, None, None),
        "qb_space_rank": (None, None, 1, None, None),
        "qb_space_terms": (None, ctypes.byref(i64), None, None),
        "qb_init_number": (None, occ, None, None),
        "qb_init_coherent": (None, z, None, ctypes.byref(d), None),
        "qb_init_field_number": (None, z, 4, None, None),
        "qb_hpsi": (None, None, None, None),
        "qb_evolve": (None, None, 1e-3, 1, None, None),
        "qb_evolve_batch": (None, None, 1, scale, 1e-3, 1, None, None),
        "qb_evolve_plain": (None, None, 1e-3, 1, None, None),
        "qb_space_set_resident_max": (None, 0),
        "qb_space_set_tile_shape": (None, 0),
        "qb_space_set_order": (None, 4),
        "qb_observables": (None, None, ctypes.byref(obs), None),
        "qb_observables_noalloc": (None, None, ctypes.byref(obs), None),
        "qb_evolve_observe": (None, None, 1e-3, 1, 1, series, None, None),
        "qb_adjoint": (None, z, 1.0, 1e-3, 1, 1, 0, ctypes.byref(d), ctypes.byref(d), g, z, None, None),
        "qb_adjoint_couplings": (None, z, 1.0, 1e-3, 1, 1, 0, ctypes.byref(d), ctypes.byref(d), g, z, gl, None,
                                 None),
        "qb_space_status": (None, 0, ctypes.byref(i32), None),
    }
    for name, args in calls.items():
        rc = getattr(lib, name)(*args)
        assert rc == 1, (name, rc)  # QB_EINVAL
        assert lib.qb_last_error(), name
    assert lib.qb_workspace_bytes(None, 1) == -1
    assert lib.qb_adjoint_workspace_bytes(None, 1, 1) == -1
    lib.qb_space_free(None)  # a no-op


def test_host_only_entry_points_refuse_bad_arguments():
    """The host-only analysis calls return QB_EINVAL on the arguments their header
    comments exclude (NULL pointers, too few samples, a non-positive spacing, an
    unknown fit kind, data a power-law fit cannot take the log of)."""
    import paper_2111_00050_gb300._lib as L

    lib = L.lib()
    d, d2, d3 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    flag = ctypes.c_int()
    v = (ctypes.c_double * 4)(0.9, 0.85, 0.7, 0.75)
    x = (ctypes.c_double * 3)(1.0, 2.0, 4.0)
    y = (ctypes.c_double * 3)(1.0, -2.0, 4.0)
    assert lib.qb_breaktime(None, 4, 0.1, 0.5, ctypes.byref(d), ctypes.byref(flag)) == 1
    assert lib.qb_breaktime(v, -1, 0.1, 0.5, ctypes.byref(d), ctypes.byref(flag)) == 1
    assert lib.qb_breaktime(v, 4, 0.1, 0.5, None, ctypes.byref(flag)) == 1
    sq = (ctypes.byref(d), ctypes.byref(flag), ctypes.byref(d2), ctypes.byref(d3))
    assert lib.qb_squeezing(v, 0, 0.1, 0.8, *sq) == 1
    assert lib.qb_squeezing(v, 4, 0.0, 0.8, *sq) == 1
    assert lib.qb_squeezing(v, 4, 0.1, 0.8, *sq) == 0 and flag.value == L.QB_CROSSED
    assert lib.qb_fit(x, x, 1, 0, ctypes.byref(d), ctypes.byref(d2)) == 1  # n < 2
    assert lib.qb_fit(x, x, 3, 2, ctypes.byref(d), ctypes.byref(d2)) == 1  # unknown kind
    assert lib.qb_fit(x, y, 3, 0, ctypes.byref(d), ctypes.byref(d2)) == 1  # log of a negative y
    assert lib.qb_fit(x, y, 3, 1, ctypes.byref(d), ctypes.byref(d2)) == 0  # y = c0 + c1 log x takes any y
    z = (ctypes.c_double * 4)()
    traj = (ctypes.c_double * 8)()
    assert lib.qb_meanfield(None, z, 1e-3, 1, 1, traj) == 1
    assert lib.qb_interaction_per_occupation(None, z, ctypes.byref(d)) == 1

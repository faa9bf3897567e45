"""qb_observables_noalloc, the entry point for callers that cannot allocate.

Some callers must not allocate device memory while they run (a service under a
fixed memory budget, a custom allocator that forbids cudaMalloc after start-up,
a thread that must not enter the allocator because that can synchronise the
device).  For them the library offers an observables call whose reduction
scratch is a fixed device array inside the library.  This test calls it through
the C ABI twice in a row, on two different states, and checks each result
against qb_observables within the observables tolerance of the parity tests.

This file is named so that pytest collects it last.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OBS_TOL = 1e-9


def _compare(got, ref):
    for key in ("norm", "N", "H", "n_tot", "Q", "lam_p", "PO", "Vminus_p"):
        assert abs(got[key] - ref[key]) <= OBS_TOL * max(1.0, abs(ref[key])), key
    for key in ("a", "Mij", "aa", "eigvals", "Vminus_modes"):
        np.testing.assert_allclose(got[key], ref[key], atol=OBS_TOL * max(1.0, ref["n_tot"]))
    assert abs(abs(np.vdot(got["xi"], ref["xi"])) - 1) < OBS_TOL


def test_noalloc_observables_match_allocating_call_twice():
    import torch

    import paper_2111_00050_gb300 as qb
    import workloads as wl
    from paper_2111_00050_gb300 import _lib
    from paper_2111_00050_gb300.api import obs_to_dict

    M = 7
    w = wl.dispersion_quadratic(M)
    L = wl.contact_coupling(M, -0.08)
    rng = np.random.default_rng(21)
    z = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    z *= math.sqrt(4.0 / np.sum(np.abs(z) ** 2))
    qs = qb.Space(M, w, L, 0, 14)
    psi = qs.empty_state()
    qs.init_coherent(z, psi)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        qs.evolve(psi, 2e-3, 25 * (call + 1))  # a different state for each call
        ref = qs.observables(psi)
        out = _lib.QbObs()
        rc = _lib.lib().qb_observables_noalloc(qs._h, ctypes.c_void_p(psi.data_ptr()), ctypes.byref(out), stream)
        assert rc == 0, _lib.lib().qb_last_error()
        _compare(obs_to_dict(out, M), ref)


def test_noalloc_capped_grid_after_another_space():
    """The same call on the 2,731,365-ket sector (M = 11, N = 20, P = 0), where the
    moments grid is capped to fit the fixed array and the <H> kernel runs fewer CTAs
    than the moments kernel; a call on a different space first leaves other words
    in the shared array, so a reduction over words the <H> kernel did not write would
    show.  <H> is checked against <psi|H psi> from the FP64 H psi kernel."""
    import torch

    import paper_2111_00050_gb300 as qb
    import workloads as wl
    from paper_2111_00050_gb300 import _lib
    from paper_2111_00050_gb300.api import obs_to_dict

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def noalloc(space, psi):
        out = _lib.QbObs()
        rc = _lib.lib().qb_observables_noalloc(space._h, ctypes.c_void_p(psi.data_ptr()), ctypes.byref(out), stream)
        assert rc == 0, _lib.lib().qb_last_error()
        return obs_to_dict(out, space.M)

    M0 = 3
    q0 = qb.Space(M0, wl.dispersion_quadratic(M0), wl.contact_coupling(M0, 0.3), 0, 60)
    p0 = q0.empty_state()
    q0.init_coherent(np.array([2.0, 3.0j, -1.5]), p0)
    noalloc(q0, p0)
    W = wl.large_sector()
    qs = qb.Space(W.M, W.w, W.L, 20, 20, [0])
    assert qs.total == 2731365
    rng = np.random.default_rng(31)
    x = rng.standard_normal(qs.total) + 1j * rng.standard_normal(qs.total)
    psi = torch.from_numpy(x / np.linalg.norm(x)).cuda()
    got = noalloc(qs, psi)
    hp = qs.empty_state()
    qs.hpsi(psi, hp)
    h_ref = float(torch.vdot(psi, hp).real)
    assert abs(got["H"] - h_ref) <= OBS_TOL * max(1.0, abs(h_ref))
    _compare(got, qs.observables(psi))

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

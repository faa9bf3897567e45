"""The seeded workloads have the sizes the benchmark and the full-size GPU tests
assume, counted by the oracle's own enumeration of the special Hilbert spaces
(sectors of fixed N and P mod M, Sec. III B and App. A).  CPU only."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as orc  # noqa: E402
import workloads as wl  # noqa: E402


def _count(M, Ns):
    dims = [orc.sector_dim(M, N, P) for N in Ns for P in range(M)]
    return sum(dims), sum(d > 0 for d in dims)


def test_batched_coherent_workload_size():
    """M = 7 coherent state at n_tot = 16, every sector N <= n_tot + 6 sqrt(n_tot) = 40."""
    W = wl.batched_coherent()
    assert (W.M, W.n_max) == (7, 40)
    assert _count(W.M, range(W.n_max + 1)) == (62891499, 281)


def test_adjoint_workload_size():
    """M = 5 coherent state at n_tot = 40, every sector N <= 40 + 6 sqrt(40) = 77."""
    W = wl.adjoint_coherent()
    assert (W.M, W.n_max) == (5, 77)
    assert _count(W.M, range(W.n_max + 1)) == (27285336, 386)


def test_long_range_field_number_workload_size():
    """M = 9 field-number state with Poisson(3) occupations drawn from seed 0: N = 27,
    every P."""
    W = wl.long_range_field_number()
    assert (W.M, W.n_tot, W.name) == (9, 27, "long_range_field_number_M9_N27")
    assert _count(W.M, [W.n_tot]) == (23535820, 9)

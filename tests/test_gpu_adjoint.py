"""Adjoint gradients (qb_adjoint) against the oracle's exact discrete adjoint
(every state stored) and against central differences of the GPU loss.

Tolerances: relative 1e-8 against the oracle with every state stored
(ckpt_every = 1) or every stage vector kept (ckpt_every = 0, the tape mode) and 1e-7
with time reversal between checkpoints; 1e-6 against central differences with h = 1e-6.
"""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl

pytestmark = pytest.mark.gpu


def _case():
    M = 5
    rng = np.random.default_rng(0)
    x = rng.standard_normal((M, 2))
    z = x[:, 0] + 1j * x[:, 1]
    z *= math.sqrt(2.5 / np.sum(np.abs(z) ** 2))
    w = wl.dispersion_quadratic(M)
    L0 = wl.contact_coupling(M, 1.0)
    return M, w, L0, z, -0.2, 2e-3, 60


def _rel(a, b):
    a, b = np.atleast_1d(a), np.atleast_1d(b)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


@pytest.mark.parametrize("kind", ["Q", "PO"])
@pytest.mark.parametrize("ckpt", [0, 1, 20])
def test_adjoint_matches_oracle_discrete_adjoint(kind, ckpt):
    import paper_2111_00050_gb300 as qb

    M, w, L0, z, scale, dt, steps = _case()
    qs = qb.Space(M, w, L0, 0, 10)
    got = qs.adjoint(z, scale, dt, steps, ckpt_every=ckpt, loss=kind)
    os_ = orc.Space(M, qs.sectors)
    loss, gs, gw, gz = orc.adjoint_gradient(os_, w, L0, scale, z, dt, steps, kind)
    tol = 1e-8 if ckpt <= 1 else 1e-7
    assert abs(got["loss"] - loss) <= 1e-10 * max(1, abs(loss))
    assert _rel(got["grad_scale"], gs) <= tol
    assert _rel(got["grad_w"], gw) <= tol
    assert _rel(got["grad_z"], gz) <= tol


def test_tape_mode_equals_stored_states():
    """ckpt_every = 0 keeps the stage vectors of the forward pass instead of
    recomputing them from stored states: the same arithmetic on the same vectors,
    so the loss and gradients agree with ckpt_every = 1 to rounding (they are the
    same double-float stage vectors); the workspace holds 4 vectors per step more."""
    import paper_2111_00050_gb300 as qb

    M, w, L0, z, scale, dt, steps = _case()
    qs = qb.Space(M, w, L0, 0, 10)
    lib = qb.lib()
    b1 = lib.qb_adjoint_workspace_bytes(qs._h, steps, 1)
    b0 = lib.qb_adjoint_workspace_bytes(qs._h, steps, 0)
    assert b0 - b1 >= 4 * steps * 16 * qs.total - steps * 16 * qs.total - 4096
    assert lib.qb_adjoint_workspace_bytes(qs._h, steps, -1) == -1
    for kind in ("Q", "PO"):
        a = qs.adjoint(z, scale, dt, steps, ckpt_every=0, loss=kind)
        b = qs.adjoint(z, scale, dt, steps, ckpt_every=1, loss=kind)
        assert abs(a["loss"] - b["loss"]) <= 1e-14 * abs(b["loss"])
        for k in ("grad_scale", "grad_w", "grad_z"):
            assert _rel(a[k], b[k]) <= 1e-13


def test_adjoint_matches_gpu_central_differences():
    import paper_2111_00050_gb300 as qb

    M, w, L0, z, scale, dt, steps = _case()
    qs = qb.Space(M, w, L0, 0, 10)
    got = qs.adjoint(z, scale, dt, steps, ckpt_every=10, loss="Q")
    h = 1e-6

    def loss(sc=scale, ww=w, zz=z):
        sp = qb.Space(M, ww, L0, 0, 10)
        return sp.adjoint(zz, sc, dt, steps, ckpt_every=steps, loss="Q")["loss"]

    fd = (loss(sc=scale + h) - loss(sc=scale - h)) / (2 * h)
    assert abs(got["grad_scale"] - fd) <= 1e-6 * max(1e-3, abs(fd))
    e = np.zeros(M)
    e[2] = h
    fd = (loss(ww=w + e) - loss(ww=w - e)) / (2 * h)
    assert abs(got["grad_w"][2] - fd) <= 1e-6 * max(1e-3, abs(fd))
    ez = np.zeros(M, dtype=np.complex128)
    ez[1] = 1j * h
    fd = (loss(zz=z + ez) - loss(zz=z - ez)) / (2 * h)
    assert abs(got["grad_z"][1].imag - fd) <= 1e-6 * max(1e-3, abs(fd))


def test_autograd_function_returns_adjoint_gradients():
    import torch

    import paper_2111_00050_gb300 as qb

    M, w, L0, z, scale, dt, steps = _case()
    s_t = torch.tensor(scale, dtype=torch.float64, requires_grad=True)
    w_t = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    z_t = torch.tensor(z, dtype=torch.complex128, requires_grad=True)
    loss = qb.adjoint_loss(s_t, w_t, z_t, M=M, L0=L0, n_min=0, n_max=10, dt=dt, steps=steps, ckpt_every=20,
                           loss="Q")
    loss.backward()
    os_ = orc.Space(M, qb.Space(M, w, L0, 0, 10).sectors)
    ref = orc.adjoint_gradient(os_, w, L0, scale, z, dt, steps, "Q")
    assert abs(loss.item() - ref[0]) <= 1e-10
    assert _rel(s_t.grad.item(), ref[1]) <= 1e-7
    assert _rel(w_t.grad.numpy(), ref[2]) <= 1e-7
    assert _rel(z_t.grad.numpy(), ref[3]) <= 1e-7
    # without gradients only the forward run and the loss are computed, on the cached space
    with torch.no_grad():
        plain = qb.adjoint_loss(s_t, w_t, z_t, M=M, L0=L0, n_min=0, n_max=10, dt=dt, steps=steps, loss="Q")
    assert abs(plain.item() - ref[0]) <= 1e-10
    # the coupling as an input: L0.grad = scale * d loss / d L (qb_adjoint_couplings)
    L_t = torch.tensor(L0, dtype=torch.complex128, requires_grad=True)
    loss2 = qb.adjoint_loss(s_t, w_t, z_t, L_t, M=M, n_min=0, n_max=10, dt=dt, steps=steps, ckpt_every=1,
                            loss="Q")
    loss2.backward()
    r = qb.Space(M, w, L0, 0, 10).adjoint(z, scale, dt, steps, ckpt_every=1, loss="Q", coupling_grad=True)
    assert np.allclose(L_t.grad.numpy(), scale * r["grad_L"], rtol=0, atol=1e-14 * np.abs(r["grad_L"]).max())
    assert abs(float(np.sum((np.conj(L_t.grad.numpy()) * L0).real)) - scale * r["grad_scale"]) <= \
        1e-10 * abs(scale * r["grad_scale"])


def test_adjoint_full_size_against_central_differences():
    """The adjoint benchmark workload at full size (M=5, contact, complex-Gaussian
    amplitudes with n_tot = 40, N <= 77: 386 sectors, 27,285,336 kets), 4 steps with
    checkpoints every 2: d Q / d scale, d Q / d w_2 and d Q / d Im z_1 against central
    differences of the loss.  After 4 steps Q and its w-derivatives are small (~5e-9),
    so the steps are sized for the loss's rounding: h = 1e-4 for the scale, 1e-2 for
    w, 1e-3 for z, and a relative tolerance of 1e-4 on the last two."""
    import paper_2111_00050_gb300 as qb

    W = wl.adjoint_coherent()
    L0 = wl.contact_coupling(W.M, 1.0)
    scale, steps = -0.1, 4
    qs = qb.Space(W.M, W.w, L0, 0, W.n_max)
    assert qs.total == 27285336
    got = qs.adjoint(W.z, scale, W.dt, steps, ckpt_every=2, loss="Q")

    def loss(sc=scale, ww=None, zz=None):
        sp = qs if ww is None else qb.Space(W.M, ww, L0, 0, W.n_max)
        return sp.adjoint(W.z if zz is None else zz, sc, W.dt, steps, ckpt_every=steps, loss="Q")["loss"]

    h = 1e-4
    fd = (loss(sc=scale + h) - loss(sc=scale - h)) / (2 * h)
    assert abs(got["grad_scale"] - fd) <= 1e-5 * abs(fd)
    h = 1e-2
    e = np.zeros(W.M)
    e[2] = h
    fd = (loss(ww=W.w + e) - loss(ww=W.w - e)) / (2 * h)
    assert abs(got["grad_w"][2] - fd) <= 1e-4 * abs(fd)
    h = 1e-3
    ez = np.zeros(W.M, dtype=np.complex128)
    ez[1] = 1j * h
    fd = (loss(zz=W.z + ez) - loss(zz=W.z - ez)) / (2 * h)
    assert abs(got["grad_z"][1].imag - fd) <= 1e-4 * abs(fd)


def _hermitian_direction(M, seed):
    """A random coupling direction D with D_{pq;rs} = conj(D_{rs;pq}), zero off momentum
    conservation mod M."""
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((M,) * 4) + 1j * rng.standard_normal((M,) * 4)
    idx = np.indices((M,) * 4)
    D[(idx[0] + idx[1] - idx[2] - idx[3]) % M != 0] = 0.0
    return 0.5 * (D + np.conj(D.transpose(2, 3, 0, 1)))


@pytest.mark.parametrize("kind", ["Q", "PO"])
def test_coupling_gradient_against_scale_and_central_differences(kind):
    """qb_adjoint_couplings: the derivative along the space's own coupling equals
    grad_scale (an identity of the two sums, 1e-10), and along two random Hermitian
    momentum-conserving directions it matches central differences of the loss (1e-6).
    The other outputs equal those of qb_adjoint."""
    import paper_2111_00050_gb300 as qb

    M, w, L0, z, scale, dt, steps = _case()
    qs = qb.Space(M, w, L0, 0, 10)
    got = qs.adjoint(z, scale, dt, steps, ckpt_every=1, loss=kind, coupling_grad=True)
    ref = qs.adjoint(z, scale, dt, steps, ckpt_every=1, loss=kind)
    assert got["loss"] == ref["loss"] and got["grad_scale"] == ref["grad_scale"]
    g = got["grad_L"]
    along_L0 = float(np.sum((np.conj(g) * L0).real))
    assert abs(along_L0 - got["grad_scale"]) <= 1e-10 * abs(got["grad_scale"])
    h = 1e-5
    for seed in (1, 2):
        D = _hermitian_direction(M, seed)

        def loss(eps):
            Lp = scale * L0 + eps * D
            sp = qb.Space(M, w, Lp, 0, 10)
            return sp.adjoint(z, 1.0, dt, steps, ckpt_every=1, loss=kind)["loss"]

        fd = (loss(h) - loss(-h)) / (2 * h)
        an = float(np.sum((np.conj(g) * D).real))
        assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(got["grad_scale"]))


def test_coupling_gradient_complex_generic_tape():
    """The generic kernels (M = 4, a random complex Hermitian coupling) in tape mode:
    the derivative along the coupling equals grad_scale and along a random direction
    matches central differences."""
    import paper_2111_00050_gb300 as qb

    M = 4
    rng = np.random.default_rng(5)
    w = rng.standard_normal(M)
    L0 = 0.05 * _hermitian_direction(M, 9)
    z = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * 0.6
    dt, steps = 2e-3, 40
    qs = qb.Space(M, w, L0, 0, 8)
    got = qs.adjoint(z, 1.0, dt, steps, ckpt_every=0, loss="Q", coupling_grad=True)
    g = got["grad_L"]
    assert abs(float(np.sum((np.conj(g) * L0).real)) - got["grad_scale"]) <= 1e-10 * abs(got["grad_scale"])
    D = _hermitian_direction(M, 11)
    h = 1e-5

    def loss(eps):
        return qb.Space(M, w, L0 + eps * D, 0, 8).adjoint(z, 1.0, dt, steps, ckpt_every=1, loss="Q")["loss"]

    fd = (loss(h) - loss(-h)) / (2 * h)
    an = float(np.sum((np.conj(g) * D).real))
    assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(got["grad_scale"]))


@pytest.mark.parametrize("M", [1, 3, 6])
def test_coupling_gradient_small_and_even_mode_counts(M):
    """The generic kernels with one operator (M = 1: L_{00;00} only), a few (M = 3) and
    an even mode count (M = 6): the derivative along the space's own coupling equals
    grad_scale, and the entries are the same for every ordering of the two pairs."""
    import paper_2111_00050_gb300 as qb

    rng = np.random.default_rng(M)
    w = wl.dispersion_quadratic(M)
    L0 = wl.contact_coupling(M, 1.0) if M != 3 else 0.2 * _hermitian_direction(M, 4)
    z = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * 0.8
    qs = qb.Space(M, w, L0, 0, 9 if M < 6 else 6)
    got = qs.adjoint(z, -0.3, 2e-3, 30, ckpt_every=0, loss="Q", coupling_grad=True)
    g = got["grad_L"]
    assert abs(float(np.sum((np.conj(g) * L0).real)) - got["grad_scale"]) <= 1e-10 * abs(got["grad_scale"]) + 1e-16
    assert np.array_equal(g, g.transpose(1, 0, 2, 3)) and np.array_equal(g, g.transpose(0, 1, 3, 2))

"""Plain CPU oracle for the sector-restricted bosonic-mode solver of
Eberhardt, Zamora, Kopp & Abel (arXiv:2111.00050).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library in ``paper_2111_00050_gb300``; the heavy loops live in
``qb_oracle.c`` (plain C, built by :func:`build`), the rest is plain numpy.

Conventions (the readings of the paper this oracle follows):

* H = sum_p w_p n_p + sum over ordered (p,q,r,s) with p+q = r+s (mod M) of
  L_{pq;rs} a_p^dag a_q^dag a_r a_s, i.e. Eq. (Ham) with L_{pq;rs} equal to
  Lambda^{rs}_{pq}/2 (upper indices annihilate, lower indices create).
* Mode labels are i - (M-1)/2 for odd M (i for even M); momentum is conserved
  modulo M and a sector is the pair (N, P = sum label*n mod M) (Sec. III B).
* Expectations are <psi|O|psi>/<psi|psi>; n_tot = <N> = Tr M (Sec. II C-D).
* RK4 is the classic four-stage scheme, applied sector by sector (Sec. III B:
  sectors evolve independently).

Parity pins for every function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_OMP_PATH = os.path.join(_HERE, "_build", "liboracle_omp.so")  # the same source built with OpenMP
_lib = None
_omp = None


def build(force: bool = False) -> str:
    """Compile qb_oracle.c into a shared library with the host C compiler, and the
    same file with OpenMP (the row-parallel RK4 of the timed CPU baseline) if the
    compiler supports it."""
    src = os.path.join(_HERE, "qb_oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    for path, extra in ((_LIB_PATH, []), (_OMP_PATH, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
            tmp = path + f".tmp{os.getpid()}"
            r = subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", *extra, src, "-o", tmp, "-lm"],
                               capture_output=True, text=True)
            if r.returncode != 0:
                if extra:  # no OpenMP: the baseline falls back to the single-threaded build
                    continue
                raise RuntimeError(f"gcc failed on the oracle:\n{r.stderr}")
            os.replace(tmp, path)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.orc_sector_basis.restype = i64
        lib.orc_sector_basis.argtypes = [i32, i32, i32, i32, vp, i64]
        lib.orc_find.restype = i64
        lib.orc_find.argtypes = [i32, vp, i64, vp]
        lib.orc_check_coupling.restype = i32
        lib.orc_check_coupling.argtypes = [i32, vp, i32]
        lib.orc_apply_h.restype = i32
        lib.orc_apply_h.argtypes = [i32, i64, vp, vp, vp, vp, vp, i32]
        lib.orc_rk4.restype = i32
        lib.orc_rk4.argtypes = [i32, i64, vp, vp, vp, vp, ctypes.c_double, i64]
        lib.orc_apply_h_row.restype = i32
        lib.orc_apply_h_row.argtypes = [i32, i64, vp, vp, vp, vp, i64, vp]
        lib.orc_count_terms.restype = i64
        lib.orc_count_terms.argtypes = [i32, i64, vp, vp]
        lib.orc_moments.restype = None
        lib.orc_moments.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, i32]
        lib.orc_apply_mode_op.restype = None
        lib.orc_apply_mode_op.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32, i32, vp, i32]
        _lib = lib
    return _lib


def _omp_lib():
    """The OpenMP build (rk4_rows), or the plain one where OpenMP is not available."""
    global _omp
    if _omp is None:
        _L()
        path = _OMP_PATH if os.path.exists(_OMP_PATH) else _LIB_PATH
        lib = ctypes.CDLL(path)
        lib.orc_rk4_rows.restype = ctypes.c_int
        lib.orc_rk4_rows.argtypes = [ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 4 + [ctypes.c_double,
                                                                                              ctypes.c_int64]
        lib.orc_threads.restype = ctypes.c_int
        _omp = lib
    return _omp


def threads() -> int:
    """Host threads rk4_rows uses."""
    return int(_omp_lib().orc_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def label(M: int, i: int) -> int:
    """Momentum label of mode index i."""
    return i - (M - 1) // 2 if M % 2 else i


def labels(M: int) -> np.ndarray:
    return np.array([label(M, i) for i in range(M)], dtype=np.int64)


def sector_of(occ, exact: bool = False) -> tuple[int, int]:
    """(N, P) of an occupation vector (Sec. III B); P mod M unless exact."""
    occ = np.asarray(occ, dtype=np.int64)
    M = occ.size
    P = int(np.dot(labels(M), occ))
    return int(occ.sum()), (P if exact else P % M)


def sector_basis(M: int, N: int, P: int, exact: bool = False) -> np.ndarray:
    """All occupation vectors of sector (N, P), lexicographic, shape [D, M]."""
    lib = _L()
    D = lib.orc_sector_basis(M, N, P, int(exact), None, 0)
    out = np.zeros((max(D, 0), M), dtype=np.int32)
    if D > 0:
        lib.orc_sector_basis(M, N, P, int(exact), _p(out), D)
    return out


def sector_dim(M: int, N: int, P: int, exact: bool = False) -> int:
    return int(_L().orc_sector_basis(M, N, P, int(exact), None, 0))


def check_coupling(M: int, L: np.ndarray, exact: bool = False) -> bool:
    Lc = np.ascontiguousarray(L, dtype=np.complex128).reshape(-1)
    return _L().orc_check_coupling(M, _p(Lc), int(exact)) == 0


class Space:
    """A list of sectors with their concatenated lexicographic bases; exact:
    sectors of exact total momentum (the plain label sum) instead of mod M."""

    def __init__(self, M: int, sectors, exact: bool = False):
        self.M = M
        self.exact = bool(exact)
        self.sectors = [(int(N), int(P) if exact else int(P) % M) for N, P in sectors]
        bases = [sector_basis(M, N, P, exact) for N, P in self.sectors]
        self.dims = np.array([b.shape[0] for b in bases], dtype=np.int64)
        self.off = np.zeros(len(bases) + 1, dtype=np.int64)
        self.off[1:] = np.cumsum(self.dims)
        self.basis = np.ascontiguousarray(np.concatenate(bases, axis=0) if bases else np.zeros((0, M), np.int32))
        self.secN = np.array([s[0] for s in self.sectors], dtype=np.int32)
        self.secP = np.array([s[1] for s in self.sectors], dtype=np.int32)

    @property
    def total(self) -> int:
        return int(self.off[-1])

    def index_of(self, occ) -> int:
        """Global index of an occupation vector, or -1."""
        occ = np.ascontiguousarray(occ, dtype=np.int32)
        N, P = sector_of(occ, self.exact)
        for s, (sN, sP) in enumerate(self.sectors):
            if (sN, sP) == (N, P):
                b = self.basis[self.off[s]:self.off[s + 1]]
                k = _L().orc_find(self.M, _p(np.ascontiguousarray(b)), b.shape[0], _p(occ))
                return -1 if k < 0 else int(self.off[s] + k)
        return -1

    def sector_slice(self, s: int) -> slice:
        return slice(int(self.off[s]), int(self.off[s + 1]))


def all_sectors(M: int, n_min: int, n_max: int, exact: bool = False):
    """Non-empty sectors, N ascending then P ascending (exact: every label sum)."""
    out = []
    for N in range(n_min, n_max + 1):
        Ps = range(int(labels(M).min()) * N, int(labels(M).max()) * N + 1) if exact else range(M)
        out += [(N, P) for P in Ps if sector_dim(M, N, P, exact) > 0]
    return out


# --------------------------------------------------------------------------- H

def apply_h(space: Space, w, L, psi: np.ndarray, dagger: bool = False) -> np.ndarray:
    """H psi (or H^dag psi) sector by sector, Eq. (Ham) applied literally."""
    M = space.M
    w = np.ascontiguousarray(w, dtype=np.float64)
    Lc = np.ascontiguousarray(L, dtype=np.complex128).reshape(-1)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros_like(psi)
    lib = _L()
    for s in range(len(space.sectors)):
        sl = space.sector_slice(s)
        b = np.ascontiguousarray(space.basis[sl])
        x = np.ascontiguousarray(psi[sl])
        y = np.zeros_like(x)
        rc = lib.orc_apply_h(M, b.shape[0], _p(b), _p(w), _p(Lc), _p(x), _p(y), int(dagger))
        if rc != 0:
            raise ValueError("coupling maps a ket outside its sector")
        out[sl] = y
    return out


def apply_h_rows(space: Space, s: int, w, L, psi_sector: np.ndarray, rows) -> np.ndarray:
    """(H psi)_i for the given local rows i of sector s only (psi_sector is that
    sector's slice), by applying the adjoint of each term to ket i."""
    M = space.M
    w = np.ascontiguousarray(w, dtype=np.float64)
    Lc = np.ascontiguousarray(L, dtype=np.complex128).reshape(-1)
    b = np.ascontiguousarray(space.basis[space.sector_slice(s)])
    x = np.ascontiguousarray(psi_sector, dtype=np.complex128)
    out = np.zeros(len(rows), dtype=np.complex128)
    buf = np.zeros(1, dtype=np.complex128)
    lib = _L()
    for k, i in enumerate(rows):
        if lib.orc_apply_h_row(M, b.shape[0], _p(b), _p(w), _p(Lc), _p(x), int(i), _p(buf)) != 0:
            raise ValueError("coupling maps a ket outside its sector")
        out[k] = buf[0]
    return out


def rk4(space: Space, w, L, psi: np.ndarray, dt: float, steps: int) -> np.ndarray:
    """`steps` classic RK4 steps of d psi/dt = -i H psi (Eq. Schr), per sector."""
    M = space.M
    w = np.ascontiguousarray(w, dtype=np.float64)
    Lc = np.ascontiguousarray(L, dtype=np.complex128).reshape(-1)
    out = np.array(psi, dtype=np.complex128, copy=True)
    lib = _L()
    for s in range(len(space.sectors)):
        sl = space.sector_slice(s)
        b = np.ascontiguousarray(space.basis[sl])
        x = np.ascontiguousarray(out[sl])
        rc = lib.orc_rk4(M, b.shape[0], _p(b), _p(w), _p(Lc), _p(x), float(dt), int(steps))
        if rc != 0:
            raise ValueError("coupling maps a ket outside its sector")
        out[sl] = x
    return out


def rk4_rows(space: Space, w, L, psi: np.ndarray, dt: float, steps: int) -> np.ndarray:
    """rk4 with H psi formed row by row, the rows of a sector on every host core
    (OpenMP build); the arithmetic of each row is that of apply_h_rows."""
    M = space.M
    w = np.ascontiguousarray(w, dtype=np.float64)
    Lc = np.ascontiguousarray(L, dtype=np.complex128).reshape(-1)
    out = np.array(psi, dtype=np.complex128, copy=True)
    lib = _omp_lib()
    for s in range(len(space.sectors)):
        sl = space.sector_slice(s)
        b = np.ascontiguousarray(space.basis[sl])
        x = np.ascontiguousarray(out[sl])
        if lib.orc_rk4_rows(M, b.shape[0], _p(b), _p(w), _p(Lc), _p(x), float(dt), int(steps)) != 0:
            raise ValueError("coupling maps a ket outside its sector")
        out[sl] = x
    return out


def taylor(space: Space, w, L, psi: np.ndarray, dt: float, steps: int, order: int) -> np.ndarray:
    """`steps` Taylor steps of order K of d psi/dt = -i H psi: each step is
    psi <- sum_{k=0}^{K} (-i dt H)^k / k! psi, the terms formed one after the
    other as t_k = (-i dt / k) H t_{k-1} (Sec. III B's scheme is K = 2, with the
    1/2 of the second-order term; K = 4 equals classic RK4 for a linear H)."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    for _ in range(steps):
        term = out.copy()
        acc = out.copy()
        for k in range(1, order + 1):
            term = (-1j * dt / k) * apply_h(space, w, L, term)
            acc = acc + term
        out = acc
    return out


def count_terms(space: Space, L) -> int:
    """Distinct nonzero H matrix elements of all held sectors, diagonal included."""
    Lc = np.ascontiguousarray(L, dtype=np.complex128).reshape(-1)
    tot = 0
    for s in range(len(space.sectors)):
        b = np.ascontiguousarray(space.basis[space.sector_slice(s)])
        tot += int(_L().orc_count_terms(space.M, b.shape[0], _p(b), _p(Lc)))
    return tot


def h_dense(space: Space, s: int, w, L) -> np.ndarray:
    """Dense matrix of H restricted to sector s, column j = H e_j."""
    sl = space.sector_slice(s)
    D = sl.stop - sl.start
    sub = Space(space.M, [space.sectors[s]], space.exact)
    Hm = np.zeros((D, D), dtype=np.complex128)
    for j in range(D):
        e = np.zeros(D, dtype=np.complex128)
        e[j] = 1.0
        Hm[:, j] = apply_h(sub, w, L, e)
    return Hm


# --------------------------------------------------------------- initial states

def _fact(n: np.ndarray) -> np.ndarray:
    return np.array([float(math.factorial(int(k))) for k in n.reshape(-1)]).reshape(n.shape)


def number_state(space: Space, occ) -> np.ndarray:
    """The single Fock ket |{n}> (Eq. numEigenstate)."""
    psi = np.zeros(space.total, dtype=np.complex128)
    k = space.index_of(occ)
    if k < 0:
        raise ValueError("occupation vector is not in the space")
    psi[k] = 1.0
    return psi


def coherent_amplitudes(space: Space, z) -> np.ndarray:
    """<n|z>_C = prod_i exp(-|z_i|^2/2) z_i^{n_i} / sqrt(n_i!) (Eq. coherentStates),
    unnormalised over the held (truncated) space."""
    z = np.asarray(z, dtype=np.complex128)
    n = space.basis.astype(np.int64)
    amp = np.ones(space.total, dtype=np.complex128)
    for i in range(space.M):
        amp *= np.exp(-abs(z[i]) ** 2 / 2) * np.power(z[i], n[:, i]) / np.sqrt(_fact(n[:, i]))
    return amp


def coherent_state(space: Space, z):
    """Coherent state truncated to the held sectors and renormalised to 1.
    Returns (psi, kept_norm) with kept_norm = sum |<n|z>|^2 before renormalising."""
    amp = coherent_amplitudes(space, z)
    kept = float(np.vdot(amp, amp).real)
    return amp / math.sqrt(kept), kept


def field_number_state(space: Space, z, n_tot: int) -> np.ndarray:
    """Field number state (Eq. fieldNumState) with the amplitudes z/sqrt(sum|z|^2)
    so that the multinomial weights sum to one: on kets with sum n = n_tot,
    sqrt(n_tot!) prod_i zeta_i^{n_i}/sqrt(n_i!), zero elsewhere."""
    z = np.asarray(z, dtype=np.complex128)
    zeta = z / math.sqrt(float(np.sum(np.abs(z) ** 2)))
    n = space.basis.astype(np.int64)
    amp = np.full(space.total, math.sqrt(float(math.factorial(n_tot))), dtype=np.complex128)
    for i in range(space.M):
        amp *= np.power(zeta[i], n[:, i]) / np.sqrt(_fact(n[:, i]))
    amp[n.sum(axis=1) != n_tot] = 0.0
    return amp


# ------------------------------------------------------------------ observables

def moments(space: Space, psi: np.ndarray) -> dict:
    """Raw moments <psi|O|psi> by acting with each operator on every ket."""
    M = space.M
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(2 + 2 * M + 4 * M * M, dtype=np.float64)
    _L().orc_moments(M, len(space.sectors), _p(space.secN), _p(space.secP), _p(space.off), _p(space.basis),
                     _p(psi), _p(out), int(space.exact))
    c = out[2:].view(np.complex128)
    return {
        "norm": out[0],
        "N": out[1],
        "a": c[:M].copy(),
        "Mij": c[M:M + M * M].reshape(M, M).copy(),
        "aa": c[M + M * M:].reshape(M, M).copy(),
    }


def apply_mode_op(space: Space, psi: np.ndarray, kind: str, i: int) -> np.ndarray:
    """a_i psi, a_i^dag psi or n_i psi on the held space."""
    k = {"a": 0, "adag": 1, "n": 2}[kind]
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros_like(psi)
    _L().orc_apply_mode_op(space.M, len(space.sectors), _p(space.secN), _p(space.secP), _p(space.off),
                           _p(space.basis), _p(psi), k, int(i), _p(out), int(space.exact))
    return out


def vminus(dOdO: float, varO: complex) -> float:
    """Minimum quadrature variance V_- = 1 + 2<dO^dag dO> - 2|Var O| (Eq. generalVminus)."""
    return 1.0 + 2.0 * dOdO - 2.0 * abs(varO)


def observables(space: Space, psi: np.ndarray, w=None, L=None) -> dict:
    """Normalised observables of Sec. II C-E:
    <a_i>, M_ij = <a_i^dag a_j>, <a_i a_j>, n_tot = Tr M, Q (Eq. Qparam),
    principal eigenvalue/eigenvector of M (Eq. POcriterion), V_- for every mode
    operator a_i and for a^p = sum_k xi_k a_k (Eq. a_op), and <H> if w, L given."""
    m = moments(space, psi)
    nrm = m["norm"]
    a = m["a"] / nrm
    Mij = m["Mij"] / nrm
    aa = m["aa"] / nrm
    n_tot = float(np.trace(Mij).real)
    Q = float(sum(Mij[j, j].real - abs(a[j]) ** 2 for j in range(space.M)) / n_tot)
    evals, evecs = np.linalg.eigh(Mij)
    lam = float(evals[-1])
    xi = evecs[:, -1]
    Vm = [vminus(Mij[i, i].real - abs(a[i]) ** 2, aa[i, i] - a[i] ** 2) for i in range(space.M)]
    dOdO = sum(np.conj(xi[k]) * xi[l] * (Mij[k, l] - np.conj(a[k]) * a[l]) for k in range(space.M)
               for l in range(space.M))
    varO = sum(xi[k] * xi[l] * (aa[k, l] - a[k] * a[l]) for k in range(space.M) for l in range(space.M))
    out = {
        "norm": nrm,
        "N": m["N"] / nrm,
        "a": a,
        "Mij": Mij,
        "aa": aa,
        "n_tot": n_tot,
        "Q": Q,
        "lam_p": lam,
        "eigvals": evals,
        "xi": xi,
        "gap": float(evals[-1] - evals[-2]) if space.M > 1 else float("inf"),
        "Vminus_modes": np.array(Vm),
        "Vminus_p": vminus(float(dOdO.real), varO),
        "PO": 1.0 - lam / n_tot,
    }
    if w is not None and L is not None:
        Hpsi = apply_h(space, w, L, psi)
        out["H"] = float(np.vdot(psi, Hpsi).real / nrm)
    return out


# -------------------------------------------------------------------- mean field

def mf_rhs(w, L, a):
    """d a_k/dt = -i (w_k a_k + sum_{q,r,s} (L_{kq;rs} + L_{qk;rs}) a_q^* a_r a_s),
    Eq. (classicalFieldEqns) with Lambda^{rs}_{kq} = 2 L^sym."""
    L = np.asarray(L, dtype=np.complex128)
    G = L + L.transpose(1, 0, 2, 3)
    return -1j * (np.asarray(w) * a + np.einsum("kqrs,q,r,s->k", G, np.conj(a), a, a))


def meanfield(w, L, a0, dt: float, steps: int, every: int = 1) -> np.ndarray:
    """Classic RK4 of the mean-field equations; returns a[t_k] for k*every steps
    (row 0 is the initial condition)."""
    a = np.array(a0, dtype=np.complex128)
    out = [a.copy()]
    for st in range(1, steps + 1):
        k1 = mf_rhs(w, L, a)
        k2 = mf_rhs(w, L, a + 0.5 * dt * k1)
        k3 = mf_rhs(w, L, a + 0.5 * dt * k2)
        k4 = mf_rhs(w, L, a + dt * k3)
        a = a + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if st % every == 0:
            out.append(a.copy())
    return np.array(out)


# --------------------------------------------------------------------- breaktime

CROSSED, AT_START, NOT_CROSSED = 0, 1, 2


def breaktime(values, dt_obs: float, thr: float):
    """First sample with value >= thr, linearly interpolated with the previous
    sample (Sec. IV C-D define the thresholds; the crossing rule is a reading).
    Returns (t_br, flag)."""
    v = np.asarray(values, dtype=np.float64)
    for k in range(v.size):
        if v[k] >= thr:
            if k == 0:
                return 0.0, AT_START
            f = (thr - v[k - 1]) / (v[k] - v[k - 1])
            return (k - 1 + f) * dt_obs, CROSSED
    return float("nan"), NOT_CROSSED


# -------------------------------------------------------------- squeezing times

def squeezing(values, dt_obs: float, thr: float = 0.8) -> dict:
    """Squeezing analysis of a V_- series (Sec. II E): the onset t_sqz, first
    sample with V_- <= thr (0.8 in the paper) interpolated linearly with the
    previous one; the smallest sample refined by the quadratic through it and its
    two neighbours (numpy.polyfit), or the sample itself at an end of the series."""
    v = np.asarray(values, dtype=np.float64)
    t_sqz, flag = float("nan"), NOT_CROSSED
    for k in range(v.size):
        if v[k] <= thr:
            if k == 0:
                t_sqz, flag = 0.0, AT_START
            else:
                t_sqz, flag = (k - 1 + (v[k - 1] - thr) / (v[k - 1] - v[k])) * dt_obs, CROSSED
            break
    k = int(np.argmin(v))
    v_min, t_min = float(v[k]), k * dt_obs
    if 0 < k < v.size - 1:
        c = np.polyfit([-1.0, 0.0, 1.0], v[k - 1:k + 2], 2)
        if c[0] > 0:
            u = -c[1] / (2 * c[0])
            t_min, v_min = (k + u) * dt_obs, float(np.polyval(c, u))
    return {"t_sqz": t_sqz, "flag": flag, "v_min": v_min, "t_min": t_min}


def interaction_per_occupation(L, z) -> float:
    """n_tot chi = n_tot^-1 sum_{pqrs} L_{pq;rs} z_p^* z_q^* z_r z_s, n_tot = sum |z|^2
    (Sec. II E, with L = Lambda/2)."""
    z = np.asarray(z, dtype=np.complex128)
    e = np.einsum("pqrs,p,q,r,s->", np.asarray(L, dtype=np.complex128), z.conj(), z.conj(), z, z)
    return float(e.real / np.sum(np.abs(z) ** 2))


def fit(x, y, kind: str = "power"):
    """Least squares over runs: y = c0 x^c1 ("power", a line in log-log) or
    y = c0 + c1 log x ("log"); returns (c0, c1)."""
    lx = np.log(np.asarray(x, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    if kind == "power":
        c1, lc0 = np.polyfit(lx, np.log(y), 1)
        return float(np.exp(lc0)), float(c1)
    c1, c0 = np.polyfit(lx, y, 1)
    return float(c0), float(c1)


# ---------------------------------------------------------------------- adjoint

def rk4_step_adjoint(space: Space, w, L, psi_n: np.ndarray, lam_next: np.ndarray, dt: float, dH_list):
    """Exact discrete adjoint of one classic RK4 step psi' = Phi(psi).

    Given the stored state psi_n and the cotangent lam_next = dloss/dpsi'^*, returns
    (lam_n, [g_theta]) where lam_n = (dPhi/dpsi)^dag lam_next and
    g_theta = 2 Re <lam_next, dPhi/dtheta> for each callable dH(v) = (dH/dtheta) v.
    """
    A = lambda v: -1j * dt * apply_h(space, w, L, v)
    Ad = lambda v: 1j * dt * apply_h(space, w, L, v, dagger=True)
    u1 = psi_n
    k1 = A(u1)
    u2 = psi_n + 0.5 * k1
    k2 = A(u2)
    u3 = psi_n + 0.5 * k2
    k3 = A(u3)
    u4 = psi_n + k3
    # psi' = psi + (k1 + 2 k2 + 2 k3 + k4)/6, k_i = A u_i
    g4 = lam_next / 6
    ub4 = Ad(g4)
    g3 = lam_next / 3 + ub4
    ub3 = Ad(g3)
    g2 = lam_next / 3 + 0.5 * ub3
    ub2 = Ad(g2)
    g1 = lam_next / 6 + 0.5 * ub2
    ub1 = Ad(g1)
    lam_n = lam_next + ub1 + ub2 + ub3 + ub4
    grads = []
    for dH in dH_list:
        dA = lambda v: -1j * dt * dH(v)
        g = 0.0
        for gk, uk in ((g1, u1), (g2, u2), (g3, u3), (g4, u4)):
            g += 2.0 * np.vdot(gk, dA(uk)).real
        grads.append(g)
    return lam_n, grads


def loss_and_seed(space: Space, psi: np.ndarray, kind: str = "Q"):
    """Loss at the final state and its Wirtinger gradient d loss / d psi^*, by
    definition.  kind "Q": Eq. (Qparam) with n_tot = Tr M; kind "PO": the
    principal eigenvalue lam_p of M (Eq. POcriterion), d lam_p = xi^dag dM xi."""
    ob = observables(space, psi)
    nu = ob["norm"]
    if kind == "Q":
        a = ob["a"]
        Nexp = ob["n_tot"]
        S = float(np.sum(np.abs(a) ** 2))
        lam = (S / Nexp) * psi
        Npsi = np.zeros_like(psi)
        for j in range(space.M):
            Npsi += apply_mode_op(space, psi, "n", j)
            lam -= (np.conj(a[j]) * apply_mode_op(space, psi, "a", j)
                    + a[j] * apply_mode_op(space, psi, "adag", j)) / Nexp
        lam += (S / Nexp ** 2) * Npsi
        return ob["Q"], lam / nu
    xi = ob["xi"]
    lam = -ob["lam_p"] * psi
    for i in range(space.M):
        for j in range(space.M):
            lam += np.conj(xi[i]) * xi[j] * apply_mode_op(space, apply_mode_op(space, psi, "a", j), "adag", i)
    return ob["lam_p"], lam / nu


def adjoint_gradient(space: Space, w, L0, scale: float, z, dt: float, steps: int, kind: str = "Q"):
    """Exact discrete adjoint of `steps` classic RK4 steps of H = H_w + scale H_{L0}
    from the renormalised truncated coherent state of z; every state is stored.
    Returns (loss, d/dscale, d/dw [M], d/dz [M] as d/dRe z + i d/dIm z)."""
    M = space.M
    L = scale * np.asarray(L0, dtype=np.complex128)
    psi0, _ = coherent_state(space, z)
    states = [psi0]
    for _ in range(steps):
        states.append(rk4(space, w, L, states[-1], dt, 1))
    loss, lam = loss_and_seed(space, states[-1], kind)
    dHs = lambda v: apply_h(space, np.zeros(M), L0, v)
    dHw = [lambda v, q=q: apply_mode_op(space, v, "n", q) for q in range(M)]
    g_s, g_w = 0.0, np.zeros(M)
    for n in range(steps - 1, -1, -1):
        lam, g = rk4_step_adjoint(space, w, L, states[n], lam, dt, [dHs] + dHw)
        g_s += g[0]
        g_w += np.array(g[1:])
    psi0 = states[0]
    c = np.vdot(lam, psi0)
    gz = np.zeros(M, dtype=np.complex128)
    for k in range(M):
        ak_dag_psi = apply_mode_op(space, psi0, "adag", k)
        Gk = np.vdot(lam, ak_dag_psi)    # <lam, d psi0/d z_k> before renormalisation
        Hk = np.vdot(psi0, ak_dag_psi)
        dx = 2 * Gk.real - 2 * c.real * Hk.real
        dy = -2 * Gk.imag + 2 * c.real * Hk.imag
        gz[k] = dx + 1j * dy
    return loss, g_s, g_w, gz

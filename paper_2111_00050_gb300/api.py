"""Thin Python binding of the qb C ABI (include/qb.h).

Argument marshalling only: every step of the computation runs in libqb's CUDA
kernels (or, for the tiny host-side pieces the ABI documents -- the M x M
eigensolve, breaktime, mean field -- in its C++).  Device buffers are torch
tensors; the current torch CUDA stream is passed to every call.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import QbModel, QbObs, check, lib


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t: torch.Tensor) -> ctypes.c_void_p:
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128_as_f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def _model(M: int, w, L, exact: bool = False):
    w = _f64(w)
    Lf = _c128_as_f64(np.asarray(L, dtype=np.complex128).reshape(-1))
    if w.size != M or Lf.size != 2 * M ** 4:
        raise ValueError("w must have M entries and L M^4")
    m = QbModel(M, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                Lf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1 if exact else 0)
    return m, (w, Lf)  # keep the arrays alive with the struct


def obs_to_dict(o: QbObs, M: int) -> dict:
    c = lambda arr, n: np.frombuffer(bytes(arr), dtype=np.float64)[: 2 * n].view(np.complex128).copy()
    return {
        "t": o.t,
        "norm": o.norm,
        "N": o.N,
        "H": o.H,
        "n_tot": o.n_tot,
        "Q": o.Q,
        "lam_p": o.lam_p,
        "PO": o.PO,
        "gap": o.gap,
        "Vminus_p": o.Vminus_p,
        "a": c(o.a, M),
        "Mij": c(o.Mij, M * M).reshape(M, M),
        "aa": c(o.aa, M * M).reshape(M, M),
        "xi": c(o.xi, M),
        "eigvals": np.array(o.eig[:M]),
        "Vminus_modes": np.array(o.Vminus[:M]),
    }


class Space:
    """qb_sector_build: all non-empty sectors (N, P) with n_min <= N <= n_max
    and P in p_list (every P if None).  exact: momentum conserved exactly (P the
    plain label sum) instead of mod M."""

    def __init__(self, M: int, w, L, n_min: int, n_max: int, p_list: Optional[Sequence[int]] = None,
                 exact: bool = False):
        self.M = int(M)
        self.exact = bool(exact)
        self._model, self._keep = _model(self.M, w, L, self.exact)
        h = ctypes.c_void_p()
        if p_list is None:
            check(lib().qb_sector_build(ctypes.byref(self._model), int(n_min), int(n_max), None, 0, ctypes.byref(h)))
        else:
            pl = np.ascontiguousarray(p_list, dtype=np.int32)
            check(lib().qb_sector_build(ctypes.byref(self._model), int(n_min), int(n_max),
                                        pl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(pl.size),
                                        ctypes.byref(h)))
        self._h = h
        tot, ns, mx = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
        check(lib().qb_space_info(h, ctypes.byref(tot), ctypes.byref(ns), ctypes.byref(mx)))
        self.total, self.n_sectors, self.max_dim = int(tot.value), int(ns.value), int(mx.value)
        N = np.zeros(self.n_sectors, np.int32)
        P = np.zeros(self.n_sectors, np.int32)
        dim = np.zeros(self.n_sectors, np.int64)
        off = np.zeros(self.n_sectors, np.int64)
        ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        lp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        check(lib().qb_space_sectors(h, ip(N), ip(P), lp(dim), lp(off)))
        self.sectors = list(zip(N.tolist(), P.tolist()))
        self.dims = dim
        self.offsets = off
        self.order = 4
        self.tile_shape = 0
        self.tuning = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.qb_space_free(h)
            self._h = None

    # ---- basis
    def basis(self, first: int = 0, count: Optional[int] = None, device="cuda") -> torch.Tensor:
        count = self.total - first if count is None else count
        out = torch.empty((count, self.M), dtype=torch.int32, device=device)
        if count:
            check(lib().qb_space_basis(self._h, int(first), int(count), _dptr(out), _stream()))
        return out

    def rank(self, occ: torch.Tensor) -> torch.Tensor:
        occ = occ.to(torch.int32).contiguous()
        out = torch.empty(occ.shape[0], dtype=torch.int64, device=occ.device)
        if occ.shape[0]:
            check(lib().qb_space_rank(self._h, _dptr(occ), int(occ.shape[0]), _dptr(out), _stream()))
        return out

    def status(self, set_bits: int = 0) -> int:
        """qb_space_status: ORs set_bits into the space's device status word and
        returns the word (nonzero: the next synchronising call fails with QB_EINTERNAL)."""
        st = ctypes.c_int()
        check(lib().qb_space_status(self._h, int(set_bits), ctypes.byref(st), _stream()))
        return int(st.value)

    def terms(self):
        t, u = ctypes.c_int64(), ctypes.c_int64()
        check(lib().qb_space_terms(self._h, ctypes.byref(t), ctypes.byref(u), _stream()))
        return int(t.value), int(u.value)

    # ---- states
    def empty_state(self, batch: int = 1) -> torch.Tensor:
        shape = (self.total,) if batch == 1 else (batch, self.total)
        return torch.empty(shape, dtype=torch.complex128, device="cuda")

    def init_number(self, occ, psi: torch.Tensor) -> None:
        o = np.ascontiguousarray(occ, dtype=np.int32)
        check(lib().qb_init_number(self._h, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(psi), _stream()))

    def init_coherent(self, z, psi: torch.Tensor) -> float:
        zf = _c128_as_f64(z)
        kept = ctypes.c_double()
        check(lib().qb_init_coherent(self._h, zf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _dptr(psi),
                                     ctypes.byref(kept), _stream()))
        return float(kept.value)

    def init_field_number(self, z, n_tot: int, psi: torch.Tensor) -> None:
        zf = _c128_as_f64(z)
        check(lib().qb_init_field_number(self._h, zf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n_tot),
                                         _dptr(psi), _stream()))

    # ---- evolution
    def workspace(self, batch: int = 1) -> torch.Tensor:
        n = int(lib().qb_workspace_bytes(self._h, int(batch)))
        return torch.empty(n // 16, dtype=torch.complex128, device="cuda")

    def hpsi(self, psi: torch.Tensor, out: torch.Tensor) -> None:
        check(lib().qb_hpsi(self._h, _dptr(psi), _dptr(out), _stream()))

    def evolve(self, psi: torch.Tensor, dt: float, steps: int, work: Optional[torch.Tensor] = None) -> None:
        work = self.workspace(1) if work is None else work
        check(lib().qb_evolve(self._h, _dptr(psi), float(dt), int(steps), _dptr(work), _stream()))

    def set_resident_max(self, kets: int) -> None:
        """qb_space_set_resident_max: sectors up to `kets` kets run shared-memory resident (0: never)."""
        check(lib().qb_space_set_resident_max(self._h, int(kets)))

    def set_order(self, order: int) -> None:
        """Taylor order of a time step (4: RK4, the default; 2: the second-order Taylor step)."""
        check(lib().qb_space_set_order(self._h, int(order)))
        self.order = int(order)

    def set_tile_shape(self, shape: int) -> None:
        """qb_space_set_tile_shape: tile shape of the RK4 stage kernel (0 .. QB_TILE_SHAPES-1)."""
        check(lib().qb_space_set_tile_shape(self._h, int(shape)))
        self.tile_shape = int(shape)

    def _time_evolve(self, dt, psi, trial, steps, work) -> float:
        trial.copy_(psi)
        self.evolve(trial, dt, 1, work)  # first launches of a setting pay their set-up
        trial.copy_(psi)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        self.evolve(trial, dt, steps, work)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def autotune(self, dt: float, psi: torch.Tensor, candidates=(0, 256, 1024, 4096), steps: int = 2,
                 work: Optional[torch.Tensor] = None, shapes=None) -> int:
        """Picks the execution settings of qb_evolve for this space by timing `steps`
        RK4 steps from a copy of psi (CUDA events): first the tile shape of the stage
        kernel (every compiled shape, or `shapes`; resident threshold 0, so that every
        sector runs through the stage kernel), then the resident threshold among
        `candidates`.  Keeps the fastest of each and returns the threshold; the chosen
        shape is in self.tile_shape and both, with every timing, in self.tuning."""
        work = self.workspace(1) if work is None else work
        trial = psi.clone()
        shapes = range(_lib.QB_TILE_SHAPES) if shapes is None else shapes
        self.set_resident_max(0)
        shape_ms = {}
        for sh in shapes:
            self.set_tile_shape(sh)
            shape_ms[int(sh)] = self._time_evolve(dt, psi, trial, steps, work)
        self.set_tile_shape(min(shape_ms, key=shape_ms.get))
        res_ms = {}
        for kets in candidates:
            self.set_resident_max(kets)
            res_ms[int(kets)] = self._time_evolve(dt, psi, trial, steps, work)
        best = min(res_ms, key=res_ms.get)
        self.set_resident_max(best)
        self.tuning = {"tile_shape": self.tile_shape, "resident_max_kets": best, "tile_shape_ms": shape_ms,
                       "resident_ms": res_ms, "steps": steps}
        return best

    def evolve_plain(self, psi: torch.Tensor, dt: float, steps: int, work: Optional[torch.Tensor] = None) -> None:
        work = self.workspace(1) if work is None else work
        check(lib().qb_evolve_plain(self._h, _dptr(psi), float(dt), int(steps), _dptr(work), _stream()))

    def evolve_batch(self, psi: torch.Tensor, scale, dt: float, steps: int,
                     work: Optional[torch.Tensor] = None) -> None:
        sc = _f64(scale)
        work = self.workspace(sc.size) if work is None else work
        check(lib().qb_evolve_batch(self._h, _dptr(psi), int(sc.size),
                                    sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(dt), int(steps),
                                    _dptr(work), _stream()))

    # ---- adjoint
    def adjoint(self, z, scale: float, dt: float, steps: int, ckpt_every: int = 1, loss: str = "Q",
                work: Optional[torch.Tensor] = None, coupling_grad: bool = False) -> dict:
        """qb_adjoint: loss (Q or PO = lam_p) at t_f and its gradients with respect to
        the two-body scale, w_p and the coherent amplitudes z (d/dRe z + i d/dIm z).
        ckpt_every >= 1 stores every ckpt_every-th state and rebuilds the others by time
        reversal; 0 keeps every step's stage vectors on the device (64 B per ket and
        step) and runs only the costate stages backwards.  coupling_grad: also
        grad_L[p, q, r, s] = d loss / d Re L_{pq;rs} + i d loss / d Im L_{pq;rs} for the
        couplings of H (scale times the space's L), qb_adjoint_couplings."""
        kind = {"Q": _lib.QB_LOSS_Q, "PO": _lib.QB_LOSS_PO}[loss]
        nbytes = int(lib().qb_adjoint_workspace_bytes(self._h, int(steps), int(ckpt_every)))
        if work is None:
            work = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        if work.numel() < nbytes or work.data_ptr() % 256:
            raise ValueError("workspace too small or not 256-byte aligned")
        zf = _c128_as_f64(z)
        out_loss, gs = ctypes.c_double(), ctypes.c_double()
        gw = np.zeros(self.M)
        gz = np.zeros(2 * self.M)
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if coupling_grad:
            gl = np.zeros(2 * self.M ** 4)
            check(lib().qb_adjoint_couplings(self._h, dp(zf), float(scale), float(dt), int(steps), int(ckpt_every), kind,
                                     ctypes.byref(out_loss), ctypes.byref(gs), dp(gw), dp(gz), dp(gl), _dptr(work),
                                     _stream()))
        else:
            check(lib().qb_adjoint(self._h, dp(zf), float(scale), float(dt), int(steps), int(ckpt_every), kind,
                                   ctypes.byref(out_loss), ctypes.byref(gs), dp(gw), dp(gz), _dptr(work), _stream()))
        out = {"loss": out_loss.value, "grad_scale": gs.value, "grad_w": gw, "grad_z": gz[0::2] + 1j * gz[1::2]}
        if coupling_grad:
            out["grad_L"] = (gl[0::2] + 1j * gl[1::2]).reshape(self.M, self.M, self.M, self.M)
        return out

    # ---- observables
    def observables(self, psi: torch.Tensor) -> dict:
        o = QbObs()
        check(lib().qb_observables(self._h, _dptr(psi), ctypes.byref(o), _stream()))
        return obs_to_dict(o, self.M)

    def evolve_observe(self, psi: torch.Tensor, dt: float, steps: int, obs_every: int,
                       work: Optional[torch.Tensor] = None) -> list:
        work = self.workspace(1) if work is None else work
        n = steps // obs_every + 1
        arr = (QbObs * n)()
        check(lib().qb_evolve_observe(self._h, _dptr(psi), float(dt), int(steps), int(obs_every), arr, _dptr(work),
                                      _stream()))
        return [obs_to_dict(arr[k], self.M) for k in range(n)]


def measure_fp64_fma(reps: int = 3) -> float:
    """qb_measure_fp64_fma: the GPU's FP64 FMA rate in TFLOP/s (2 flop per FMA)."""
    out = ctypes.c_double()
    check(lib().qb_measure_fp64_fma(int(reps), ctypes.byref(out), _stream()))
    return float(out.value)


def breaktime(values, dt_obs: float, thr: float):
    v = _f64(values)
    t, f = ctypes.c_double(), ctypes.c_int()
    check(lib().qb_breaktime(v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(v.size), float(dt_obs),
                             float(thr), ctypes.byref(t), ctypes.byref(f)))
    return float(t.value), int(f.value)


def squeezing(values, dt_obs: float, thr: float = 0.8) -> dict:
    """Onset (first V_- <= thr) and maximal squeezing of a V_- series (qb_squeezing)."""
    v = _f64(values)
    t, f, vm, tm = ctypes.c_double(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib().qb_squeezing(v.ctypes.data_as(dp), int(v.size), float(dt_obs), float(thr), ctypes.byref(t),
                             ctypes.byref(f), ctypes.byref(vm), ctypes.byref(tm)))
    return {"t_sqz": float(t.value), "flag": int(f.value), "v_min": float(vm.value), "t_min": float(tm.value)}


def interaction_per_occupation(M: int, w, L, z, exact: bool = False) -> float:
    """n_tot chi = n_tot^-1 sum L_{pq;rs} z_p^* z_q^* z_r z_s (qb_interaction_per_occupation)."""
    m, keep = _model(M, w, L, exact)
    zz = _c128_as_f64(z)
    out = ctypes.c_double()
    check(lib().qb_interaction_per_occupation(ctypes.byref(m), zz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              ctypes.byref(out)))
    return float(out.value)


def fit(x, y, kind: str = "power"):
    """(c0, c1) of y = c0 x^c1 (kind "power") or y = c0 + c1 log x (kind "log") (qb_fit)."""
    xs, ys = _f64(x), _f64(y)
    if xs.size != ys.size:
        raise ValueError("x and y differ in length")
    c0, c1 = ctypes.c_double(), ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib().qb_fit(xs.ctypes.data_as(dp), ys.ctypes.data_as(dp), int(xs.size), {"power": 0, "log": 1}[kind],
                       ctypes.byref(c0), ctypes.byref(c1)))
    return float(c0.value), float(c1.value)


def meanfield(M: int, w, L, z0, dt: float, steps: int, every: int = 1, exact: bool = False) -> np.ndarray:
    m, keep = _model(M, w, L, exact)
    z = _c128_as_f64(z0)
    rows = steps // every + 1
    out = np.zeros(2 * M * rows, dtype=np.float64)
    check(lib().qb_meanfield(ctypes.byref(m), z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(dt),
                             int(steps), int(every), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out.view(np.complex128).reshape(rows, M)


_SPACE_CACHE: "dict" = {}
_SPACE_CACHE_SIZE = 2


def _cached_space(M: int, w, L0, n_min: int, n_max: int, p_list) -> Space:
    """A Space for (M, w, L0, N range, P list), reused across calls: building one
    (sector tables, per-ket diagonal and occupations) costs a device pass over every
    ket.  The few most recent ones are kept."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    L0 = np.ascontiguousarray(L0, dtype=np.complex128)
    key = (int(M), w.tobytes(), L0.tobytes(), int(n_min), int(n_max),
           None if p_list is None else tuple(int(p) for p in p_list))
    sp = _SPACE_CACHE.pop(key, None)
    if sp is None:
        sp = Space(M, w, L0, n_min, n_max, p_list)
    _SPACE_CACHE[key] = sp  # most recent last
    while len(_SPACE_CACHE) > _SPACE_CACHE_SIZE:
        _SPACE_CACHE.pop(next(iter(_SPACE_CACHE)))
    return sp


class AdjointLoss(torch.autograd.Function):
    """Loss (Q or lam_p at t_f) of an RK4 run from a coherent state, with gradients
    by qb_adjoint.  Inputs: the two-body scale (0-d float64 tensor), the dispersion
    w (float64 [M]), the coherent amplitudes z (complex128 [M]) and optionally the unit
    coupling L0 (complex128 [M, M, M, M]; else spec["L0"], constant), H = H_w + scale
    H_{L0}; the space is reused across calls with the same model and range.  When no
    input requires a gradient (or autograd is off) only the forward run and the loss
    are computed; otherwise the adjoint runs once, in forward (qb_adjoint_couplings
    when L0 requires a gradient), and backward returns its gradients.  Complex inputs
    follow torch's convention for real losses: d loss / d Re + i d loss / d Im."""

    @staticmethod
    def forward(ctx, scale, w, z, L0, spec):
        L0n = L0.detach().cpu().numpy() if L0 is not None else spec["L0"]
        space = _cached_space(spec["M"], w.detach().cpu().numpy(), L0n, spec["n_min"], spec["n_max"],
                              spec.get("p_list"))
        zz = z.detach().cpu().numpy()
        kind = spec.get("loss", "Q")
        want_L = L0 is not None and ctx.needs_input_grad[3]
        if not any(ctx.needs_input_grad[:4]):
            psi = space.empty_state()
            space.init_coherent(zz, psi)
            space.evolve_batch(psi, [float(scale)], spec["dt"], spec["steps"])
            ob = space.observables(psi)
            ctx.grads = None
            return torch.tensor(ob["Q"] if kind == "Q" else ob["lam_p"], dtype=torch.float64)
        r = space.adjoint(zz, float(scale), spec["dt"], spec["steps"], spec.get("ckpt_every", 1), kind,
                          coupling_grad=want_L)
        # d loss / d L0 = scale times the gradient with respect to H's couplings
        gL = torch.from_numpy(float(scale) * r["grad_L"]) if want_L else None
        ctx.grads = (torch.tensor(r["grad_scale"], dtype=torch.float64),
                     torch.from_numpy(np.asarray(r["grad_w"], dtype=np.float64)),
                     torch.from_numpy(np.asarray(r["grad_z"], dtype=np.complex128)), gL)
        return torch.tensor(r["loss"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        gs, gw, gz, gL = ctx.grads
        return g * gs, g * gw, g * gz, (g * gL if gL is not None else None), None


def adjoint_loss(scale, w, z, L0=None, **spec):
    """Differentiable loss of a coherent-state run: see AdjointLoss.  L0 may be a
    complex128 tensor (an input with a gradient) or an array (a constant)."""
    if L0 is not None and not torch.is_tensor(L0):
        spec["L0"] = L0
        L0 = None
    return AdjointLoss.apply(scale, w, z, L0, spec)

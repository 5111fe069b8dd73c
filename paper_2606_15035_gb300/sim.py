"""Python binding of the PIC C-ABI with the same names as include/pic.h.

The module-level functions ``pic_config_default``, ``pic_init``, ``pic_step``,
``pic_energy``, ``pic_diagnostics``, ``pic_get_state``, ``pic_set_state``,
``pic_iterate`` and ``pic_destroy`` marshal arguments to the library and return Python
values; ``PicSim`` bundles them around one context.  PyTorch supplies device memory
(the library allocates through torch's caching allocator) and the CUDA stream.
Host arrays are numpy float64; device arrays are torch float64 CUDA tensors.
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (PIC_FP64, PIC_QUAD_CLOSED, PIC_QUAD_GAUSS, PicAllocator, PicConfig, PicDiag,  # noqa: F401
                   PicEnergy, PicError, PicIterateOut, PicParticles, PicProfile, PicStateView, PicStepInfo,
                   PicVjpInfo)


def _check(status, ctx=None):
    if status != _lib.PIC_OK:
        msg = _lib.lib().pic_last_error(ctx).decode() if ctx else ""
        raise PicError(status, msg)


def pic_config_default(**overrides) -> PicConfig:
    """Default configuration with keyword overrides (n and L accept 3-sequences)."""
    cfg = PicConfig()
    _check(_lib.lib().pic_config_default(C.byref(cfg)))
    for k, v in overrides.items():
        if k in ("n", "L"):
            arr = getattr(cfg, k)
            for a in range(3):
                arr[a] = v[a]
        elif k == "split_orbit_at_knots" or k in ("picard_max", "quadrature", "nq", "precision", "sort_every",
                                                  "diagnostics", "accept_unconverged", "picard_accel", "mixed_max32",
                                                  "deterministic", "shape_order", "ops", "mixed_pair_max"):
            setattr(cfg, k, int(v))
        else:
            setattr(cfg, k, float(v))
    return cfg


def _torch():
    import torch
    return torch


class _TorchAllocator:
    """Device memory for the library from torch's caching allocator."""

    def __init__(self, device):
        torch = _torch()
        self.device = device
        self._live = {}

        def alloc(nbytes, stream, user):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=stream or 0)
            except Exception:
                return None
            self._live[int(ptr)] = nbytes
            return ptr

        def free(ptr, nbytes, stream, user):
            if ptr is None:
                return
            self._live.pop(int(ptr), None)
            torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc_cb = _lib.ALLOC_FN(alloc)
        self._free_cb = _lib.FREE_FN(free)
        self.struct = PicAllocator(self._alloc_cb, self._free_cb, None)


def _ptr(a):
    """Data pointer of a contiguous float64 numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data
    assert a.dtype == _torch().float64 and a.is_contiguous()
    return a.data_ptr()


def _on_device(a):
    return 0 if (a is None or isinstance(a, np.ndarray)) else int(a.is_cuda)


def soa(a):
    """(np, 3) -> contiguous structure-of-arrays (3, np) float64 (numpy or torch)."""
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)
    return a.to(dtype=_torch().float64).t().contiguous()


def pic_init(cfg: PicConfig, x, v, q: float, m: float, stream=None, use_torch_allocator=True):
    """Create a context from positions x and velocities v, each (np, 3), host or device."""
    torch = _torch()
    xs, vs = soa(x), soa(v)
    npart = int(xs.shape[1])
    parts = PicParticles(npart, float(q), float(m), _ptr(xs), _ptr(vs), _on_device(xs))
    if stream is None:
        stream = torch.cuda.current_stream()
    alloc = _TorchAllocator(stream.device) if use_torch_allocator else None
    ctx = C.c_void_p()
    st = _lib.lib().pic_init(C.byref(cfg), C.byref(parts), C.byref(alloc.struct) if alloc else None,
                             C.c_void_p(stream.cuda_stream), C.byref(ctx))
    if st != _lib.PIC_OK:
        raise PicError(st, "pic_init failed")
    return ctx, alloc, (xs, vs)


def pic_step(ctx, nsteps: int = 1) -> PicStepInfo:
    info = PicStepInfo()
    _check(_lib.lib().pic_step(ctx, int(nsteps), C.byref(info)), ctx)
    return info


def pic_energy(ctx) -> PicEnergy:
    e = PicEnergy()
    _check(_lib.lib().pic_energy(ctx, C.byref(e)), ctx)
    return e


def pic_diagnostics(ctx) -> PicDiag:
    d = PicDiag()
    _check(_lib.lib().pic_diagnostics(ctx, C.byref(d)), ctx)
    return d


def pic_get_state(ctx, view: PicStateView):
    _check(_lib.lib().pic_get_state(ctx, C.byref(view)), ctx)


def pic_set_state(ctx, view: PicStateView):
    _check(_lib.lib().pic_set_state(ctx, C.byref(view)), ctx)


def pic_iterate(ctx, v_iter, out: PicIterateOut):
    _check(_lib.lib().pic_iterate(ctx, _ptr(v_iter), _on_device(v_iter), C.byref(out)), ctx)


def pic_profile(ctx, enable: bool, read: bool = True):
    """Switch live kernel profiling on/off; return (and reset) the accumulated profile."""
    out = PicProfile() if read else None
    _check(_lib.lib().pic_profile(ctx, int(bool(enable)), C.byref(out) if read else None), ctx)
    return out


def pic_residual_history(ctx):
    """Per-iteration (e_v, e_J, fp32) of the last step, as three 1-D numpy arrays."""
    L = _lib.lib()
    n = L.pic_residual_history(ctx, 0, None, None, None)
    if n < 0:
        raise ValueError("null context")
    ev, ej, f32 = np.zeros(max(n, 1)), np.zeros(max(n, 1)), np.zeros(max(n, 1), dtype=np.int32)
    L.pic_residual_history(ctx, n, ev.ctypes.data_as(C.POINTER(C.c_double)),
                           ej.ctypes.data_as(C.POINTER(C.c_double)), f32.ctypes.data_as(C.POINTER(C.c_int32)))
    return ev[:n], ej[:n], f32[:n]


def pic_get_iterate(ctx, npart):
    """Last Picard iterate and its image G, each (np, 3) host arrays in pic_init order."""
    a, b = np.zeros(3 * npart), np.zeros(3 * npart)
    _check(_lib.lib().pic_get_iterate(ctx, _ptr(a), _ptr(b), 0), ctx)
    return a.reshape(3, npart).T.copy(), b.reshape(3, npart).T.copy()


def pic_get_accepted(ctx, npart):
    """The last committed step's final-sweep iterate v^{n+1,p+1} ((np, 3)) and its sliding
    bits ((np,) uint8, bit a: component a landed on a knot), host arrays in pic_init order."""
    a = np.zeros(3 * npart)
    sl = np.zeros(max(npart, 1), dtype=np.uint8)
    _check(_lib.lib().pic_get_accepted(ctx, _ptr(a), sl.ctypes.data, 0), ctx)
    return a.reshape(3, npart).T.copy(), sl[:npart].copy()


def pic_set_wait_limit(ctx, cycles: int):
    _check(_lib.lib().pic_set_wait_limit(ctx, int(cycles)), ctx)


def pic_get_positions(ctx, npart):
    """Positions in cell units exactly as stored, (np, 3) host array in pic_init order."""
    a = np.zeros(3 * npart)
    _check(_lib.lib().pic_get_positions(ctx, _ptr(a), 0), ctx)
    return a.reshape(3, npart).T.copy()


def pic_probe_fma_rates(stream=None):
    """Measured (FP64, FP32) FMA throughput of the current device in flop/s."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    a, b = C.c_double(), C.c_double()
    _check(_lib.lib().pic_probe_fma_rates(C.c_void_p(stream.cuda_stream), C.byref(a), C.byref(b)))
    return a.value, b.value


def pic_last_error(ctx) -> str:
    return _lib.lib().pic_last_error(ctx).decode()


def pic_destroy(ctx):
    _lib.lib().pic_destroy(ctx)


def _mesh_to_xyz(a, n):
    """x-fastest flat mesh array (ncell,) or (3*ncell,) -> [ix, iy, iz] numpy layout."""
    a = np.asarray(a)
    if a.size == n[0] * n[1] * n[2]:
        return a.reshape(n[2], n[1], n[0]).transpose(2, 1, 0).copy()
    return a.reshape(3, n[2], n[1], n[0]).transpose(0, 3, 2, 1).copy()


def _xyz_to_mesh(a):
    """[ix, iy, iz] (or [c, ix, iy, iz]) numpy array -> contiguous x-fastest flat array."""
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 3:
        return np.ascontiguousarray(a.transpose(2, 1, 0)).ravel()
    return np.ascontiguousarray(a.transpose(0, 3, 2, 1)).ravel()


@dataclass
class HostState:
    x: np.ndarray
    v: np.ndarray
    P: np.ndarray
    vprev: np.ndarray
    phi: np.ndarray
    psi: np.ndarray
    rho: np.ndarray
    A: np.ndarray
    U: np.ndarray


class PicSim:
    """One simulation context on the current CUDA device and stream."""

    def __init__(self, cfg: PicConfig, x, v, q, m, stream=None):
        self.cfg = cfg
        self.n = tuple(cfg.n)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.np = int(np.shape(x)[0])
        self._owned = True
        self.ctx, self._alloc, self._keep = pic_init(cfg, x, v, q, m, stream)

    @classmethod
    def _view(cls, ctx, cfg: PicConfig, npart: int, owner):
        """A context owned by someone else (an ensemble run); close() does not destroy it."""
        self = cls.__new__(cls)
        self.cfg = cfg
        self.n = tuple(cfg.n)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.np = int(npart)
        self._owned = False
        self._owner = owner
        self.ctx = C.c_void_p(ctx)
        return self

    def close(self):
        if self.ctx and self._owned:
            pic_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1) -> PicStepInfo:
        return pic_step(self.ctx, nsteps)

    def energy(self) -> PicEnergy:
        return pic_energy(self.ctx)

    def positions_cells(self):
        return pic_get_positions(self.ctx, self.np)

    def last_iterate(self):
        return pic_get_iterate(self.ctx, self.np)

    def accepted(self):
        """(v^{n+1,p+1}, sliding bits) of the last committed step (pic_get_accepted)."""
        return pic_get_accepted(self.ctx, self.np)

    def set_wait_limit(self, cycles: int):
        pic_set_wait_limit(self.ctx, cycles)

    def profile(self, enable=True, read=True):
        return pic_profile(self.ctx, enable, read)

    def residual_history(self):
        return pic_residual_history(self.ctx)

    def autotune(self):
        """Measure and set the particle-kernel grids (blocks per SM): returns (fp64, fp32)."""
        a, b = C.c_int32(), C.c_int32()
        _check(_lib.lib().pic_autotune(self.ctx, C.byref(a), C.byref(b)), self.ctx)
        return a.value, b.value

    def diagnostics(self) -> PicDiag:
        return pic_diagnostics(self.ctx)

    def get_state(self) -> HostState:
        """Full state as host numpy arrays: particles (np, 3), mesh in [ix, iy, iz] layout."""
        npart, N = self.np, self.ncell
        bufs = {k: np.zeros(3 * npart) for k in ("x", "v", "P", "vprev")}
        mesh = {k: np.zeros(N) for k in ("phi", "psi", "rho")}
        vec = {k: np.zeros(3 * N) for k in ("A", "U")}
        view = PicStateView(*[_ptr(bufs[k]) for k in ("x", "v", "P", "vprev")],
                            *[_ptr(mesh[k]) for k in ("phi", "psi", "rho")],
                            _ptr(vec["A"]), _ptr(vec["U"]), 0)
        pic_get_state(self.ctx, view)
        pt = {k: b.reshape(3, npart).T.copy() for k, b in bufs.items()}
        return HostState(**pt, **{k: _mesh_to_xyz(v, self.n) for k, v in mesh.items()},
                         **{k: _mesh_to_xyz(v, self.n) for k, v in vec.items()})

    # ---- device-resident state and the adjoint (flat arrays in the library's layouts) ----

    STATE_KEYS = ("x", "v", "P", "vprev", "phi", "psi", "rho", "A", "U")

    def state_zeros(self):
        """A dict of zero float64 CUDA tensors in the state layout: particles SoA (3 np),
        mesh x-fastest (ncell, or 3 ncell for A and U)."""
        torch = _torch()
        sizes = {"x": 3 * self.np, "v": 3 * self.np, "P": 3 * self.np, "vprev": 3 * self.np, "phi": self.ncell,
                 "psi": self.ncell, "rho": self.ncell, "A": 3 * self.ncell, "U": 3 * self.ncell}
        return {k: torch.zeros(max(n, 1), dtype=torch.float64, device="cuda") for k, n in sizes.items()}

    def _dview(self, d):
        return PicStateView(*[d[k].data_ptr() for k in self.STATE_KEYS], 1)

    def get_state_device(self):
        d = self.state_zeros()
        pic_get_state(self.ctx, self._dview(d))
        return d

    def set_state_device(self, d):
        pic_set_state(self.ctx, self._dview(d))

    def checkpoint(self):
        """The state as device tensors plus the positions as stored (cell units, key "xi"), so
        that restore() brings the run back bit for bit (pic_set_positions)."""
        d = self.get_state_device()
        xi = _torch().zeros(max(3 * self.np, 1), dtype=_torch().float64, device="cuda")
        _check(_lib.lib().pic_get_positions(self.ctx, C.c_void_p(xi.data_ptr()), 1), self.ctx)
        d["xi"] = xi
        return d

    def restore(self, d):
        pic_set_state(self.ctx, self._dview(d))
        _check(_lib.lib().pic_set_positions(self.ctx, C.c_void_p(d["xi"].data_ptr()), 1), self.ctx)

    def step_vjp(self, lam_next):
        """(d state^{n+1} / d state^n)^T lam_next for the step just committed: (lam_prev, info)."""
        lam_prev = self.state_zeros()
        info = PicVjpInfo()
        _check(_lib.lib().pic_step_vjp(self.ctx, C.byref(self._dview(lam_next)), C.byref(self._dview(lam_prev)),
                                       C.byref(info)), self.ctx)
        return lam_prev, info

    def energy_vjp(self):
        """dW/d(state) of the current state, W the field energy."""
        lam = self.state_zeros()
        _check(_lib.lib().pic_energy_vjp(self.ctx, C.byref(self._dview(lam))), self.ctx)
        return lam

    def init_vjp(self, lam0):
        """(lam_x0, lam_v0), each 3 np SoA: the adjoint of pic_init's map from the initial
        particles to the initial state (the context must still hold pic_init's state)."""
        torch = _torch()
        lx = torch.zeros(max(3 * self.np, 1), dtype=torch.float64, device="cuda")
        lv = torch.zeros_like(lx)
        _check(_lib.lib().pic_init_vjp(self.ctx, C.byref(self._dview(lam0)), lx.data_ptr(), lv.data_ptr(), 1),
               self.ctx)
        return lx, lv

    def set_state(self, s: HostState):
        arrs = [soa(s.x), soa(s.v), soa(s.P), soa(s.vprev),
                _xyz_to_mesh(s.phi), _xyz_to_mesh(s.psi), _xyz_to_mesh(s.rho),
                _xyz_to_mesh(s.A), _xyz_to_mesh(s.U)]
        pic_set_state(self.ctx, PicStateView(*[_ptr(a) for a in arrs], 0))

    def iterate(self, v_iter):
        """One Algorithm 1 loop body from v^{n+1,p} ((np, 3) host array); nothing is committed."""
        npart, N = self.np, self.ncell
        out = {k: np.zeros(3 * N) for k in ("J", "A", "U")}
        out.update({k: np.zeros(N) for k in ("rho", "phi", "psi")})
        pt = {k: np.zeros(3 * npart) for k in ("x", "P", "v")}
        o = PicIterateOut(*[_ptr(out[k]) for k in ("J", "rho", "phi", "psi", "A", "U")],
                          *[_ptr(pt[k]) for k in ("x", "P", "v")], 0)
        vs = soa(np.asarray(v_iter, dtype=np.float64))
        pic_iterate(self.ctx, vs, o)
        res = {k: _mesh_to_xyz(v, self.n) for k, v in out.items()}
        res.update({k: b.reshape(3, npart).T.copy() for k, b in pt.items()})
        return res


class PicEnsemble:
    """Independent runs advanced together (pic_ensemble_*): runs[i] = (cfg, x, v, q, m)."""

    def __init__(self, runs, autotune=False):
        torch = _torch()
        L = _lib.lib()
        R = len(runs)
        cfgs = (PicConfig * R)()
        parts = (PicParticles * R)()
        self._keep = []
        self.cfgs, self.nps = [], []
        for i, (cfg, x, v, q, m) in enumerate(runs):
            xs, vs = soa(x), soa(v)
            self._keep.append((xs, vs))
            cfgs[i] = cfg
            parts[i] = PicParticles(int(xs.shape[1]), float(q), float(m), _ptr(xs), _ptr(vs), _on_device(xs))
            self.cfgs.append(cfg)
            self.nps.append(int(xs.shape[1]))
        self._alloc = _TorchAllocator(torch.cuda.current_stream().device)
        self.ens = C.c_void_p()
        st = L.pic_ensemble_init(R, cfgs, parts, C.byref(self._alloc.struct), C.byref(self.ens))
        if st != _lib.PIC_OK:
            raise PicError(st, "pic_ensemble_init failed")
        self.runs = [PicSim._view(L.pic_ensemble_run(self.ens, i), self.cfgs[i], self.nps[i], self)
                     for i in range(R)]
        self.tuning = [r.autotune() for r in self.runs] if autotune else None

    def __len__(self):
        return len(self.runs)

    def step(self, nsteps=1, raise_on_error=True):
        """Advance every run; returns (infos, statuses).  With raise_on_error, a failed run
        raises PicError (the other runs have still been advanced)."""
        L = _lib.lib()
        R = len(self.runs)
        infos = (PicStepInfo * R)()
        sts = (C.c_int * R)()
        st = L.pic_ensemble_step(self.ens, int(nsteps), infos, sts)
        if st != _lib.PIC_OK and raise_on_error:
            raise PicError(st, L.pic_ensemble_last_error(self.ens).decode())
        return list(infos), list(sts)

    def close(self):
        if self.ens:
            for r in self.runs:
                r.ctx = None
            _lib.lib().pic_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

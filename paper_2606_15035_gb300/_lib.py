"""ctypes binding of the C-ABI declared in include/pic.h (argument marshalling only).

Every computation runs in the sm_103a library ``_build/libpic.so``; this module only
mirrors the C structs, converts numpy arrays / torch tensors to pointers, and turns
non-zero status codes into exceptions.  If the library is missing it raises at load
time: there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpic.so")

PIC_OK = 0
STATUS_NAMES = {
    0: "PIC_OK",
    1: "PIC_ERR_ARG",
    2: "PIC_ERR_OOM",
    3: "PIC_ERR_CUDA",
    4: "PIC_ERR_NO_CONVERGENCE",
    5: "PIC_ERR_NONFINITE",
    6: "PIC_ERR_SEGMENTS",
    7: "PIC_ERR_INTERNAL",
    8: "PIC_ERR_TIMEOUT",
}
PIC_FP64, PIC_MIXED = 0, 1
PIC_QUAD_CLOSED, PIC_QUAD_GAUSS = 0, 1
PIC_OPS_CENTRAL2, PIC_OPS_SPECTRAL = 0, 1

EXPORTED = ["pic_config_default", "pic_init", "pic_step", "pic_energy", "pic_diagnostics",
            "pic_get_state", "pic_set_state", "pic_iterate", "pic_get_positions", "pic_set_positions", "pic_get_iterate", "pic_get_accepted", "pic_set_wait_limit", "pic_step_vjp", "pic_energy_vjp", "pic_init_vjp", "pic_profile", "pic_residual_history",
            "pic_cn_update_static", "pic_probe_fma_rates", "pic_last_error", "pic_destroy", "pic_autotune", "pic_ensemble_init", "pic_ensemble_step",
            "pic_ensemble_size", "pic_ensemble_run", "pic_ensemble_last_error", "pic_ensemble_destroy"]


class PicConfig(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 3),
        ("L", C.c_double * 3),
        ("dt", C.c_double),
        ("kappa", C.c_double),
        ("sigma1", C.c_double),
        ("sigma2", C.c_double),
        ("n0", C.c_double),
        ("picard_tol", C.c_double),
        ("picard_max", C.c_int32),
        ("split_orbit_at_knots", C.c_int32),
        ("quadrature", C.c_int32),
        ("nq", C.c_int32),
        ("precision", C.c_int32),
        ("sort_every", C.c_int32),
        ("diagnostics", C.c_int32),
        ("accept_unconverged", C.c_int32),
        ("picard_accel", C.c_int32),
        ("helmholtz_tol", C.c_double),
        ("mixed_tol32", C.c_double),
        ("mixed_max32", C.c_int32),
        ("deterministic", C.c_int32),
        ("shape_order", C.c_int32),
        ("ops", C.c_int32),
        ("mixed_tol64", C.c_double),
        ("mixed_pair_max", C.c_int32),
    ]


class PicParticles(C.Structure):
    _fields_ = [
        ("np", C.c_int64),
        ("q", C.c_double),
        ("m", C.c_double),
        ("x", C.c_void_p),
        ("v", C.c_void_p),
        ("on_device", C.c_int32),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class PicAllocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class PicStepInfo(C.Structure):
    _fields_ = [
        ("steps_done", C.c_int32),
        ("iterations", C.c_int32),
        ("converged", C.c_int32),
        ("total_iterations", C.c_int32),
        ("e_v", C.c_double),
        ("e_J", C.c_double),
        ("iterations_fp32", C.c_int32),
        ("total_iterations_fp32", C.c_int32),
        ("iterations_pair", C.c_int32),
        ("total_iterations_pair", C.c_int32),
    ]


class PicEnergy(C.Structure):
    _fields_ = [("K", C.c_double), ("W", C.c_double), ("total", C.c_double)]


class PicDiag(C.Structure):
    _fields_ = [
        ("gauge_max", C.c_double), ("gauge_rms", C.c_double),
        ("gauss_max", C.c_double), ("gauss_rms", C.c_double),
        ("continuity_max", C.c_double),
        ("RA_max", C.c_double), ("RA_rms", C.c_double),
        ("partition_max", C.c_double),
        ("particle_work", C.c_double), ("mesh_work", C.c_double),
        ("R_field", C.c_double), ("R_particle", C.c_double), ("R_total", C.c_double),
        ("K0", C.c_double), ("W0", C.c_double), ("K1", C.c_double), ("W1", C.c_double),
        ("picard_iterations", C.c_int32),
        ("e_v", C.c_double), ("e_J", C.c_double),
    ]


class PicStateView(C.Structure):
    _fields_ = [
        ("x", C.c_void_p), ("v", C.c_void_p), ("P", C.c_void_p), ("vprev", C.c_void_p),
        ("phi", C.c_void_p), ("psi", C.c_void_p), ("rho", C.c_void_p),
        ("A", C.c_void_p), ("U", C.c_void_p),
        ("on_device", C.c_int32),
    ]


class PicIterateOut(C.Structure):
    _fields_ = [
        ("J", C.c_void_p), ("rho", C.c_void_p), ("phi", C.c_void_p), ("psi", C.c_void_p),
        ("A", C.c_void_p), ("U", C.c_void_p),
        ("x", C.c_void_p), ("P", C.c_void_p), ("v", C.c_void_p),
        ("on_device", C.c_int32),
    ]


class PicVjpInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("residual", C.c_double)]


class PicProfile(C.Structure):
    _fields_ = [
        ("launches", C.c_int64),
        ("push_launches", C.c_int64),
        ("push_ms", C.c_double),
        ("commit_launches", C.c_int64),
        ("commit_ms", C.c_double),
        ("scatter_launches", C.c_int64),
        ("scatter_ms", C.c_double),
        ("mesh_ms", C.c_double),
        ("sort_ms", C.c_double),
        ("particle_pushes", C.c_int64),
        ("push_pieces", C.c_int64),
        ("scatter_pieces", C.c_int64),
        ("push32_launches", C.c_int64),
        ("push32_ms", C.c_double),
        ("local_launches", C.c_int64),
        ("local_ms", C.c_double),
        ("local_solves", C.c_int64),
        ("local_evals", C.c_int64),
        ("push32_chunks", C.c_int64),
        ("push32_chunks_global", C.c_int64),
        ("pushpair_launches", C.c_int64),
        ("pushpair_ms", C.c_double),
        ("local_failed", C.c_int64),
        ("local_failed_unpinned", C.c_int64),
    ]


_lib = None


def lib():
    """Load libpic.so once; raise if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"PIC CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build() or python -m paper_2606_15035_gb300.build)")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    L.pic_config_default.argtypes = [P(PicConfig)]
    L.pic_init.argtypes = [P(PicConfig), P(PicParticles), P(PicAllocator), C.c_void_p, P(C.c_void_p)]
    L.pic_step.argtypes = [C.c_void_p, C.c_int32, P(PicStepInfo)]
    L.pic_energy.argtypes = [C.c_void_p, P(PicEnergy)]
    L.pic_diagnostics.argtypes = [C.c_void_p, P(PicDiag)]
    L.pic_get_state.argtypes = [C.c_void_p, P(PicStateView)]
    L.pic_set_state.argtypes = [C.c_void_p, P(PicStateView)]
    L.pic_iterate.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, P(PicIterateOut)]
    L.pic_profile.argtypes = [C.c_void_p, C.c_int32, P(PicProfile)]
    L.pic_residual_history.argtypes = [C.c_void_p, C.c_int32, P(C.c_double), P(C.c_double), P(C.c_int32)]
    L.pic_residual_history.restype = C.c_int32
    L.pic_get_iterate.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    L.pic_get_positions.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
    L.pic_set_positions.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
    L.pic_get_accepted.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
    L.pic_set_wait_limit.argtypes = [C.c_void_p, C.c_int64]
    L.pic_step_vjp.argtypes = [C.c_void_p, P(PicStateView), P(PicStateView), P(PicVjpInfo)]
    L.pic_energy_vjp.argtypes = [C.c_void_p, P(PicStateView)]
    L.pic_init_vjp.argtypes = [C.c_void_p, P(PicStateView), C.c_void_p, C.c_void_p, C.c_int32]
    L.pic_cn_update_static.argtypes = [C.POINTER(C.c_int32), C.POINTER(C.c_double), C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_double] + [C.c_void_p] * 10 + [C.c_void_p]
    L.pic_probe_fma_rates.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double)]
    L.pic_last_error.argtypes = [C.c_void_p]
    L.pic_last_error.restype = C.c_char_p
    L.pic_destroy.argtypes = [C.c_void_p]
    L.pic_destroy.restype = None
    L.pic_autotune.argtypes = [C.c_void_p, P(C.c_int32), P(C.c_int32)]
    L.pic_ensemble_init.argtypes = [C.c_int32, P(PicConfig), P(PicParticles), P(PicAllocator), P(C.c_void_p)]
    L.pic_ensemble_step.argtypes = [C.c_void_p, C.c_int32, P(PicStepInfo), P(C.c_int)]
    L.pic_ensemble_size.argtypes = [C.c_void_p]
    L.pic_ensemble_size.restype = C.c_int32
    L.pic_ensemble_run.argtypes = [C.c_void_p, C.c_int32]
    L.pic_ensemble_run.restype = C.c_void_p
    L.pic_ensemble_last_error.argtypes = [C.c_void_p]
    L.pic_ensemble_last_error.restype = C.c_char_p
    L.pic_ensemble_destroy.argtypes = [C.c_void_p]
    L.pic_ensemble_destroy.restype = None
    for name in EXPORTED:
        if name not in ("pic_last_error", "pic_destroy", "pic_ensemble_size", "pic_ensemble_run",
                        "pic_ensemble_last_error", "pic_ensemble_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class PicError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status

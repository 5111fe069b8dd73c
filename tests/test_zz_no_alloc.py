"""pic_cn_update_static: the Crank--Nicolson update for callers that cannot allocate device
memory where they need it (a fixed device-memory budget, a thread that must not enter the
CUDA allocator, a plugin whose host application owns all allocations).

It is checked through the C ABI against the library's own allocating path: pic_iterate
runs one Algorithm 1 body, whose mesh phase is the same CN update.  The static entry point
gets that body's inputs (level-n potentials, rho^{n+1/2}, J^{n+1/2}) and must reproduce its
level-(n+1) potentials within the tolerance of the GPU parity tests, on two calls in a row
(the shared working storage keeps the first call's contents).  The same outputs are checked
against the oracle's CN update (an exact per-Fourier-mode solve with the central-difference
operators, a different algorithm), and the device's free memory must not change by a single
byte across warmed-up calls: the entry point allocates nothing.  This file is named so that
pytest collects it last.
"""

import ctypes as C

import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def test_static_cn_update_matches_pic_iterate(cuda_ok):
    import torch
    from paper_2606_15035_gb300 import build
    build.build()
    from paper_2606_15035_gb300 import _lib, sim

    w = pi.WORKLOADS["twostream-8c-8k"]
    x, v, q, m = pi.workload_particles(w)
    cfg = sim.pic_config_default(n=w.n, L=w.L, dt=w.dt, picard_tol=1e-13)
    s = sim.PicSim(cfg, x, v, q, m)
    s.step(2)                                          # non-trivial fields: psi, A, U != 0
    st = s.get_state()
    rng = np.random.default_rng(7)
    body = s.iterate(st.v + 1e-3 * rng.normal(size=st.v.shape))
    s.close()

    flat = sim._xyz_to_mesh
    phi, psi, A, U = (_dev(flat(a)) for a in (st.phi, st.psi, st.A, st.U))
    rho_half = _dev(flat(0.5 * (body["rho"] + st.rho)))
    J = _dev(flat(body["J"]))
    N = int(np.prod(w.n))
    n_arr = (C.c_int32 * 3)(*w.n)
    L_arr = (C.c_double * 3)(*w.L)
    stream = torch.cuda.current_stream().cuda_stream
    lib = _lib.lib()
    from oracle import mesh as omesh
    from oracle import pic as opic
    grid = opic.Config(n=w.n, L=w.L, dt=w.dt).grid()
    oracle = dict(zip(("phi", "psi", "A", "U"),
                      omesh.cn_fields(st.phi, st.psi, st.A, st.U, 0.5 * (body["rho"] + st.rho), body["J"], cfg.dt,
                                      cfg.kappa, cfg.sigma1, cfg.sigma2, grid)))
    for call in range(2):
        outs = [torch.full((k * N,), np.nan, dtype=torch.float64, device="cuda") for k in (1, 1, 3, 3)]
        st_code = lib.pic_cn_update_static(n_arr, L_arr, cfg.dt, cfg.kappa, cfg.sigma1, cfg.sigma2,
                                           cfg.helmholtz_tol, phi.data_ptr(), psi.data_ptr(), A.data_ptr(),
                                           U.data_ptr(), rho_half.data_ptr(), J.data_ptr(),
                                           *[o.data_ptr() for o in outs], C.c_void_p(stream))
        assert st_code == 0
        torch.cuda.synchronize()
        phi1, psi1, A1, U1 = (o.cpu().numpy() for o in outs)
        for name, got in (("phi", phi1), ("psi", psi1), ("A", A1), ("U", U1)):
            for ref in (flat(body[name]), flat(oracle[name])):
                err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
                assert err <= 1e-12, (call, name, err)
    # no allocation: the device's free memory is the same, to the byte, before and after
    # further calls (after the ones above, which also loaded the library's device code)
    outs = [torch.empty(k * N, dtype=torch.float64, device="cuda") for k in (1, 1, 3, 3)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.pic_cn_update_static(n_arr, L_arr, cfg.dt, cfg.kappa, cfg.sigma1, cfg.sigma2, cfg.helmholtz_tol,
                                        phi.data_ptr(), psi.data_ptr(), A.data_ptr(), U.data_ptr(),
                                        rho_half.data_ptr(), J.data_ptr(), *[o.data_ptr() for o in outs],
                                        C.c_void_p(stream)) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_cn_update_rejects_oversized_meshes(cuda_ok):
    import torch
    from paper_2606_15035_gb300 import build
    build.build()
    from paper_2606_15035_gb300 import _lib
    n = (64, 32, 32)                                   # 65536 nodes > the 32768-node maximum
    N = int(np.prod(n))
    bufs = [torch.zeros(k * N, dtype=torch.float64, device="cuda") for k in (1, 1, 3, 3, 1, 3, 1, 1, 3, 3)]
    code = _lib.lib().pic_cn_update_static((C.c_int32 * 3)(*n), (C.c_double * 3)(1.0, 1.0, 1.0), 0.1, 1.0, 1.0,
                                           1.0, 1e-17, *[b.data_ptr() for b in bufs], C.c_void_p(0))
    assert code == 1                                   # PIC_ERR_ARG
    # a tolerance that needs more Chebyshev steps than one call may run is refused too
    n = (32, 32, 32)
    N = int(np.prod(n))
    bufs = [torch.zeros(k * N, dtype=torch.float64, device="cuda") for k in (1, 1, 3, 3, 1, 3, 1, 1, 3, 3)]
    code = _lib.lib().pic_cn_update_static((C.c_int32 * 3)(*n), (C.c_double * 3)(1.0, 1.0, 1.0), 10.0, 1.0, 1.0,
                                           1.0, 1e-300, *[b.data_ptr() for b in bufs], C.c_void_p(0))
    assert code == 1

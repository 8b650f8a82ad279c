"""nl_solve_static: the CG solve that allocates no device memory.

Some callers cannot allocate device memory while they call the solver: a
latency-critical loop that cannot pay for cudaMalloc/cudaFree (cudaFree
synchronises the whole device), code working inside a memory budget reserved
up front by another framework, or a thread holding a lock that its allocator
needs.  nl_solve_static serves them with scratch vectors kept in a fixed
device array inside the library.  This test calls it through the C-ABI twice
in a row (the second call reuses the array the first one left behind) and
checks both results against the allocating nl_solve on the same system.

The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

import nl_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_static_solve_matches_allocating_solve_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_07499_gb300 as nl
    from paper_2302_07499_gb300 import _binding as B
    from paper_2302_07499_gb300 import build
    build.build()
    L = nl.lib()
    L.nl_solve_static.argtypes = [C.c_void_p, C.POINTER(B.nl_solve_opts), C.c_void_p, C.POINTER(B.nl_solve_info)]
    L.nl_solve_static.restype = C.c_int

    mesh, delta = I.config_mesh("cube6_d025")
    g = I.quadratic_g(mesh.verts)
    dev = nl.Device()
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    s = nl.System(p, strategy=nl.NOCAPS, precision=nl.FP64, gamma=I.gamma_const(delta), f_const=-6.0, g=g)

    u_ref = torch.empty(mesh.nv, dtype=torch.float64, device="cuda")
    _, info = s.solve(rtol=1e-12, out=u_ref)
    assert info["status"] == 0
    ref = u_ref.cpu().numpy()

    opts = B.nl_solve_opts(1e-12, 0, 0, 0.0, 0)
    for call in range(2):
        u = torch.full((mesh.nv,), float("nan"), dtype=torch.float64, device="cuda")
        inf = B.nl_solve_info()
        st = L.nl_solve_static(s.h, C.byref(opts), C.c_void_p(u.data_ptr()), C.byref(inf))
        assert st == 0, L.nl_last_error().decode()
        got = u.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), call
        assert inf.rel_residual <= 1e-12 * 1.01


def test_static_solve_rejects_a_host_output():
    """The static solve writes u_out from its kernels, so it must be device
    memory: a host array is refused with NL_EINVAL before any launch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_07499_gb300 as nl
    from paper_2302_07499_gb300 import _binding as B
    L = nl.lib()
    L.nl_solve_static.argtypes = [C.c_void_p, C.POINTER(B.nl_solve_opts), C.c_void_p, C.POINTER(B.nl_solve_info)]
    L.nl_solve_static.restype = C.c_int
    mesh, delta = I.config_mesh("cube6_d025")
    dev = nl.Device()
    m = nl.Mesh(mesh.verts, mesh.tets, mesh.tet_in_omega, mesh.node_free, dev)
    p = nl.Pairs(m, delta)
    s = nl.System(p, strategy=nl.NOCAPS, precision=nl.FP64, gamma=I.gamma_const(delta), f_const=-6.0,
                  g=I.quadratic_g(mesh.verts))
    host = np.zeros(mesh.nv)
    inf = B.nl_solve_info()
    st = L.nl_solve_static(s.h, C.byref(B.nl_solve_opts(1e-12, 0, 0, 0.0, 0)), C.c_void_p(host.ctypes.data),
                           C.byref(inf))
    assert st == 1 and b"device memory" in L.nl_last_error()
    assert np.all(host == 0.0)

"""cswgs_solve_noalloc, the solve for callers that cannot allocate device memory
(a real-time SLM loop that cannot take an allocation's latency or failure, a
host with a fixed device-memory budget), gives what the plan-based cswgs_solve
gives on the same problem.  It is called through the C ABI twice in a row on
different problems, then once more on the first problem, since every call
shares one scratch array that keeps the previous call's contents."""
import ctypes

import numpy as np
import pytest

import workloads
from gpu_helpers import rms_wrapped

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# same arithmetic as the plan's solver, possibly another tile shape, so another
# FP32 summation order: the tolerances of the batch-versus-solo tests
TOL_SAME_PHASE = 1e-4
TOL_SAME_EU = 1e-5


def _ptr(t, typ):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), ctypes.POINTER(typ))


def _noalloc(lib, pb):
    xyz = torch.tensor(np.ascontiguousarray(pb.xyz), dtype=torch.float64, device="cuda")
    out = torch.full((pb.M,), -1.0, dtype=torch.float32, device="cuda")
    eu = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.cswgs_solve_noalloc(_ptr(xyz, ctypes.c_double), None, pb.N, pb.P, pb.c, pb.iterations, pb.seed,
                                 _ptr(out, ctypes.c_float), _ptr(eu, ctypes.c_double),
                                 ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.cswgs_last_error()
    stream.synchronize()
    e, u = eu.cpu().tolist()
    return out.cpu().numpy(), e, u


def test_noalloc_matches_solve():
    from paper_2003_05293_gb300 import Plan, capi
    lib = capi.load()
    first = workloads.problem(512, 100, 10.0, 0.125, 12, seed=3)
    second = workloads.problem(1152, 300, 10.0, 0.0625, 6, seed=4)
    with Plan(precision="fp32") as plan:
        refs = []
        for pb in (first, second):
            out = torch.empty(pb.M, dtype=torch.float32, device="cuda")
            r = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=out)
            refs.append((out.cpu().numpy(), r["e"], r["u"]))
    for pb, (ph_ref, e_ref, u_ref) in zip((first, second, first), refs + refs[:1]):
        ph, e, u = _noalloc(lib, pb)
        assert np.all(ph >= 0) and np.all(ph < 2 * np.pi)
        assert rms_wrapped(ph, ph_ref) < TOL_SAME_PHASE
        assert abs(e - e_ref) < TOL_SAME_EU and abs(u - u_ref) < TOL_SAME_EU


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2003_05293_gb300 import capi
    lib = capi.load()
    xyz = torch.zeros((600, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(2048 * 2048, dtype=torch.float32, device="cuda")
    for N, P in ((600, 512), (100, 2048), (100, 1153)):
        st = lib.cswgs_solve_noalloc(_ptr(xyz, ctypes.c_double), None, N, P, 0.125, 2, 0,
                                     _ptr(out, ctypes.c_float), None, None)
        assert st == capi.CSWGS_EINVAL
        assert b"allocation-free" in lib.cswgs_last_error()

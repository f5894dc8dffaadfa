"""The tensor-core kernel's bounded waits: with the plan's wait test on, the
producer warp holds back the first work item, every other warp's first wait
runs out after a short poll limit (before any bulk copy or MMA is issued), the
kernel ends and the solve reports CSWGS_ETIMEOUT; with the test off again the
next solve on the same plan (the same cached batch and graph) matches the
oracle.  Nothing here faults, traps or hangs the GPU: every wait is bounded
and the kernel returns normally."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_EU, TOL_PHASE_RMS, rms_wrapped, write_pinned_tune_cache

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_wait_time_out_is_reported_and_the_plan_recovers(tmp_path):
    from paper_2003_05293_gb300 import Plan, capi
    path = tmp_path / "tc.json"
    with Plan(precision="fp32", tune_cache=write_pinned_tune_cache(path, 1, 1, 2)) as plan:
        pb = workloads.problem(256, 40, 5.0, 0.25, 4, seed=3)
        out = torch.empty(pb.M, dtype=torch.float32, device="cuda")
        ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
        # a normal solve builds the cached batch first
        r = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=out)
        assert rms_wrapped(out.cpu().numpy(), ref["phase"]) < TOL_PHASE_RMS
        plan.test_waits(True, 4096)
        with pytest.raises(capi.CswgsError) as err:
            plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=out)
        assert err.value.status == capi.CSWGS_ETIMEOUT
        plan.test_waits(False, 0)
        out.fill_(-1.0)
        r = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=out)
        ph = out.cpu().numpy()
        assert np.all(ph >= 0) and rms_wrapped(ph, ref["phase"]) < TOL_PHASE_RMS
        assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU
        # a short poll limit alone changes nothing when every hand-over happens
        plan.test_waits(False, 1 << 16)
        r2 = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=out)
        assert abs(r2["e"] - r["e"]) < 1e-12
        plan.test_waits(False, 0)

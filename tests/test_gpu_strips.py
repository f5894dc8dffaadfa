"""The tensor-core kernel's strips: a work item of several tiles along one row
block, with GEMM 2's Z(n, y) accumulated over the strip's tiles and reduced
to the spot fields once per strip (V_n = sum_y conj(R_n(y)) Z(n, y) takes the
same R_n(y) for every tile of a row block).  Forced strip lengths give the
maps, e and u of strips of one tile and of the oracle: square and round
pupils (strips with tiles outside the pupil at either end, strips with no
tile inside), grids that are not a multiple of the tile, one and two GEMM 2
spot blocks (the latter takes strips of one tile), compressed and full
iterations.  The bench's own shape (64 holograms, P = 1152, N = 100, c = 1/8,
30 iterations, the autotuner's launch shapes) is held to the oracle on
sampled holograms."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_EU, TOL_PHASE_RMS, oracle_states, rms_wrapped, write_pinned_tune_cache

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SUBSET_TC = 1
FULL_WS = 2
# same sums in another order (Z accumulated across tiles in FP32 instead of
# per-tile partials summed with compensation): far inside the parity bar
TOL_SAME_PHASE = 1e-4
TOL_SAME_EU = 1e-5


def _plan(tmp_path_factory, strip):
    from paper_2003_05293_gb300 import Plan
    path = tmp_path_factory.mktemp("strip%d" % strip) / "t.json"
    return Plan(precision="fp32", max_batch=64,
                tune_cache=write_pinned_tune_cache(path, SUBSET_TC, 1, FULL_WS, strip=strip))


@pytest.fixture(scope="module")
def one(tmp_path_factory):
    p = _plan(tmp_path_factory, 1)
    yield p
    p.close()


def _batch(pbs):
    out = []
    for pb in pbs:
        o = torch.full((pb.M,), -1.0, dtype=torch.float32, device="cuda")
        out.append(o)
    return out


def _mix():
    # P = 1152 (18 tiles a row), 640 (10), 300 (5, ragged), 200 (4, ragged);
    # N over one spot block (40, 100, 128) and two (129, strips of one tile)
    pbs = []
    for i, (P, N, rnd) in enumerate([(1152, 100, False), (640, 40, True), (300, 128, False), (1152, 129, True),
                                     (200, 17, True), (640, 100, False)]):
        pb = workloads.problem(P, N, 5.0, 0.125, 5, seed=700 + i)
        if rnd:
            pb.extra = {"aperture": "round", "waist": 0.45 * P}
        pbs.append(pb)
    return pbs


@pytest.mark.parametrize("strip", [2, 3, 5, 18])
def test_forced_strips_equal_single_tiles(tmp_path_factory, one, strip):
    pbs = _mix()
    o1, o2 = _batch(pbs), _batch(pbs)
    r1 = one.solve_batch(pbs, o1)
    with _plan(tmp_path_factory, strip) as plan:
        b = plan.batch(pbs, o2)
        assert b.tile_shape()["threads"] == SUBSET_TC and b.tile_shape()["full_threads"] == FULL_WS
        for rep in range(2):
            b.run()
            r2 = b.results()
            for pb, a, c, x, y in zip(pbs, o1, o2, r1, r2):
                ph = c.cpu().numpy()
                assert np.all(ph >= 0) and np.all(ph < 2 * np.pi)
                assert rms_wrapped(a.cpu().numpy(), ph) < TOL_SAME_PHASE
                assert abs(x["e"] - y["e"]) < TOL_SAME_EU and abs(x["u"] - y["u"]) < TOL_SAME_EU
        b.close()
    # the first hologram (square, 18 tiles a row) and the round one against the oracle
    for i in (0, 1):
        pb = pbs[i]
        kw = {k: pb.extra[k] for k in ("aperture", "waist") if k in pb.extra}
        ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed, **kw)
        assert rms_wrapped(o2[i].cpu().numpy(), ref["phase"]) < TOL_PHASE_RMS
        assert abs(r2[i]["e"] - ref["e"]) < TOL_EU and abs(r2[i]["u"] - ref["u"]) < TOL_EU


@pytest.mark.parametrize("full", [0, 1])
def test_teacher_forced_iteration_whole_row_strips(tmp_path_factory, full):
    # one iteration (compressed, or over all pixels) from the oracle's state,
    # every row block one work item of 18 tiles
    pb = workloads.problem(1152, 100, 10.0, 0.125, 30, seed=31)
    j = 4
    st = oracle_states(oracle, pb, j, full_iterations=0)
    w0, th0 = st[j - 1]
    ref = oracle.solve(pb.P, pb.xyz, pb.amp, c=pb.c, iterations=1, seed=pb.seed, theta_in=th0, w_in=w0,
                       first_j=j, final_pass=False, full_iterations=full)
    with _plan(tmp_path_factory, 18) as plan:
        r = plan.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, init_w=w0, init_theta=th0, first_iteration=j,
                       full_iterations=full, final_pass=False, state=True)
    assert rms_wrapped(r["theta"], ref["theta"]) < TOL_PHASE_RMS
    assert np.sqrt(np.mean((r["w"] / ref["w"] - 1) ** 2)) < TOL_PHASE_RMS


def test_serving_with_strips(tmp_path_factory, one):
    pbs = [workloads.problem(P, 60, 5.0, 0.25, 4, seed=800 + i) for i, P in enumerate((640, 384, 640, 256))]
    with _plan(tmp_path_factory, 3) as plan:
        outs = _batch(pbs)
        res = [plan.wait(plan.submit(pb, o)) for pb, o in zip(pbs, outs)]
    for pb, o, r in zip(pbs, outs, res):
        q = torch.empty(pb.M, dtype=torch.float32, device="cuda")
        s = one.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=q)
        assert rms_wrapped(o.cpu().numpy(), q.cpu().numpy()) < TOL_SAME_PHASE
        assert abs(r["e"] - s["e"]) < TOL_SAME_EU and abs(r["u"] - s["u"]) < TOL_SAME_EU


def test_bench_shape_against_oracle():
    # the bench's workload through the autotuner's choice (64 holograms, P =
    # 1152, N = 100, c = 1/8, 30 iterations); holograms 0 and 37 against the oracle
    from paper_2003_05293_gb300 import Plan
    pbs = [workloads.problem(1152, 100, 10.0, 0.125, 30, seed=h) for h in range(64)]
    outs = _batch(pbs)
    with Plan(precision="fp32", max_batch=64) as plan:
        b = plan.batch(pbs, outs)
        b.run()
        res = b.results()
        shape = b.tile_shape()
        b.close()
    assert all(0.0 < r["e"] <= 1.0 and 0.0 < r["u"] <= 1.0 for r in res)
    for h in (0, 37):
        pb = pbs[h]
        ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
        assert rms_wrapped(outs[h].cpu().numpy(), ref["phase"]) < TOL_PHASE_RMS, shape
        assert abs(res[h]["e"] - ref["e"]) < TOL_EU and abs(res[h]["u"] - ref["u"]) < TOL_EU

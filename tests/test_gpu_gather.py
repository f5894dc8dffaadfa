"""The subset-only gather kernel for compressed iterations (the pixels of S_j
only, on the CUDA cores, one complex multiply-add per pixel-spot pair and pass
with the separable factors of Eq. 2) against the oracle: teacher-forced
iterations, free-running solves over one to six spots per lane, ragged bands
and row ranges, subsets barely larger than the spot count, the paper's round
pupil and Gaussian beam in both subset readings, batches of uneven holograms
against the direct-phasor kernel, serving, and the fall-back past its spot
limit."""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_EU, TOL_PHASE_RMS, oracle_states, rms_wrapped, write_pinned_tune_cache

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GATHER = 3             # threads marker of the gather kernel
FULL_WS = 2


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    from paper_2003_05293_gb300 import Plan
    d = tmp_path_factory.mktemp("gather")
    ga = Plan(precision="fp32", max_batch=32, tune_cache=write_pinned_tune_cache(d / "g.json", GATHER, 1, FULL_WS))
    cc = Plan(precision="fp32", max_batch=32, tune_cache=write_pinned_tune_cache(d / "c.json", 256, 4, FULL_WS))
    yield ga, cc
    ga.close()
    cc.close()


def _solve(plan, pb, **kw):
    out = torch.full((pb.M,), -1.0, dtype=torch.float32, device="cuda")
    r = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=out, state=True, **kw)
    torch.cuda.synchronize()
    return r, out.cpu().numpy().astype(np.float64)


def test_path_is_reported(plans):
    ga, _ = plans
    b = ga.batch([workloads.problem(256, 40, 5.0, 0.125, 4, seed=s) for s in range(3)])
    assert b.tile_shape()["threads"] == GATHER
    b.close()
    # past 192 spots the direct-phasor kernel takes over
    b = ga.batch([workloads.problem(256, 200, 5.0, 0.125, 4, seed=1)])
    assert b.tile_shape()["threads"] == 256
    b.close()


@pytest.mark.parametrize("j", [1, 2, 17])
def test_teacher_forced_compressed_iteration(plans, j):
    ga, _ = plans
    pb = workloads.problem(512, 100, 10.0, 0.125, 30, seed=12)
    st = oracle_states(oracle, pb, j, full_iterations=0)
    w0, th0 = st[j - 1]
    w1, th1 = st[j]
    r = ga.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, init_w=w0, init_theta=th0, first_iteration=j,
                 full_iterations=0, final_pass=False, state=True)
    assert rms_wrapped(r["theta"], th1) < TOL_PHASE_RMS
    assert math.sqrt(np.mean((r["w"] / w1 - 1) ** 2)) < TOL_PHASE_RMS


@pytest.mark.parametrize("P,N,c,I", [(512, 100, 0.125, 30), (200, 150, 0.25, 8), (130, 17, 0.5, 10),
                                     (1152, 100, 0.0625, 12), (96, 129, 0.25, 6), (300, 192, 0.125, 6),
                                     (64, 1, 0.25, 5), (320, 64, 1.0 / 32, 8)])
def test_free_running_against_oracle(plans, P, N, c, I):
    ga, _ = plans
    pb = workloads.problem(P, N, 10.0, c, I, seed=7)
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
    r, ph = _solve(ga, pb)
    assert np.all(ph >= 0) and np.all(ph < 2 * np.pi)
    assert rms_wrapped(ph, ref["phase"]) < TOL_PHASE_RMS
    assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU
    assert rms_wrapped(r["theta"], ref["theta"]) < TOL_PHASE_RMS


@pytest.mark.parametrize("j", [1, 2, 3])
def test_teacher_forced_tiny_subset(plans, j):
    # c = 1/64 at P = 96: 144 subset pixels for 129 spots (five spots a lane),
    # against the direct-phasor kernel and the oracle
    ga, cc = plans
    pb = workloads.problem(96, 129, 10.0, 1.0 / 64, 3, seed=7)
    st = oracle_states(oracle, pb, j, full_iterations=0)
    w0, th0 = st[j - 1]
    w1, th1 = st[j]
    kw = dict(init_w=w0, init_theta=th0, first_iteration=j, full_iterations=0, final_pass=False, state=True)
    r = ga.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, **kw)
    q = cc.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, **kw)
    assert rms_wrapped(r["theta"], q["theta"]) < 1e-4
    assert rms_wrapped(r["theta"], th1) < TOL_PHASE_RMS
    assert math.sqrt(np.mean((r["w"] / w1 - 1) ** 2)) < TOL_PHASE_RMS


@pytest.mark.parametrize("mode", ["windows", "fresh"])
def test_round_pupil(plans, mode):
    ga, _ = plans
    pb = workloads.problem(512, 100, 10.0, 0.125, 12, seed=21)
    kw = dict(aperture="round", waist=290.0, subset_mode=mode)
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed, **kw)
    r, ph = _solve(ga, pb, **kw)
    om = oracle.pupil_pixels(pb.P, "round")
    assert rms_wrapped(ph[om], ref["phase"][om]) < TOL_PHASE_RMS
    assert np.all(np.delete(ph, om) == 0.0)
    assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU


def test_batch_against_direct_phasors(plans):
    # several hundred items per launch, P not a multiple of the band, N over
    # one to six spots a lane, square and round pupils, two runs of the batch
    ga, cc = plans
    pbs = []
    for i in range(16):
        P, N = [(512, 40), (300, 100), (256, 160), (384, 33)][i % 4]
        pb = workloads.problem(P, N, 5.0, 0.125, 8, seed=600 + i)
        if i % 3 == 0:
            pb.extra = {"aperture": "round", "waist": 0.4 * P}
        pbs.append(pb)
    o1 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    o2 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    b = ga.batch(pbs, o1)
    assert b.tile_shape()["threads"] == GATHER
    r2 = cc.solve_batch(pbs, o2)
    for rep in range(2):
        b.run()
        r1 = b.results()
        for a, c2, x, y in zip(r1, r2, o1, o2):
            assert rms_wrapped(x.cpu().numpy(), y.cpu().numpy()) < TOL_PHASE_RMS
            assert abs(a["e"] - c2["e"]) < TOL_EU and abs(a["u"] - c2["u"]) < TOL_EU
    b.close()


def test_serving(plans):
    ga, cc = plans
    pbs = [workloads.problem(P, 60, 5.0, 0.25, 6, seed=300 + i) for i, P in enumerate((256, 192, 256, 128, 320))]
    outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    res = [ga.wait(ga.submit(pb, o)) for pb, o in zip(pbs, outs)]
    for pb, out, r in zip(pbs, outs, res):
        o2 = torch.empty(pb.M, dtype=torch.float32, device="cuda")
        s = cc.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=o2)
        assert rms_wrapped(out.cpu().numpy(), o2.cpu().numpy()) < TOL_PHASE_RMS
        assert abs(r["e"] - s["e"]) < TOL_EU and abs(r["u"] - s["u"]) < TOL_EU

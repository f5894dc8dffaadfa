"""Compressed iterations on the tensor cores: the warp-specialised kernel runs
every pixel through both products with u zero outside the subset S_j (a bit
mask made from the subset draw before each launch), so the sums of Eqs. 1 and
3 are over S_j exactly as in the CUDA-core kernel.  Plans are pinned to this
path through their tune caches and compared with the FP64 oracle (teacher-
forced compressed iterations, free-running solves, the round pupil with
windows) and with the CUDA-core compressed kernel (batches, serving)."""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_EU, TOL_PHASE_RMS, oracle_states, rms_wrapped, write_pinned_tune_cache

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SUBSET_TC = 1          # threads marker of compressed iterations on the tensor cores
FULL_WS = 2            # the warp-specialised full-pass kernel


def _plan(path, sub, full, **kw):
    from paper_2003_05293_gb300 import Plan
    return Plan(precision="fp32", tune_cache=write_pinned_tune_cache(path, sub[0], sub[1], full), **kw)


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    d = tmp_path_factory.mktemp("subtc")
    tc = _plan(d / "tc.json", (SUBSET_TC, 1), FULL_WS, max_batch=32)
    cc = _plan(d / "cc.json", (256, 4), FULL_WS, max_batch=32)
    yield tc, cc
    tc.close()
    cc.close()


def _solve(plan, pb, **kw):
    out = torch.full((pb.M,), -1.0, dtype=torch.float32, device="cuda")
    r = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=out, state=True, **kw)
    torch.cuda.synchronize()
    return r, out.cpu().numpy().astype(np.float64)


def test_path_is_reported(plans):
    tc, cc = plans
    pbs = [workloads.problem(256, 40, 5.0, 0.125, 4, seed=s) for s in range(3)]
    for plan, want in ((tc, SUBSET_TC), (cc, 256)):
        b = plan.batch(pbs)
        assert b.tile_shape()["threads"] == want
        b.close()


@pytest.mark.parametrize("j", [1, 2, 17])
def test_teacher_forced_compressed_iteration(plans, j):
    tc, _ = plans
    pb = workloads.problem(512, 100, 10.0, 0.125, 30, seed=12)
    st = oracle_states(oracle, pb, j, full_iterations=0)
    w0, th0 = st[j - 1]
    w1, th1 = st[j]
    r = tc.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, init_w=w0, init_theta=th0, first_iteration=j,
                 full_iterations=0, final_pass=False, state=True)
    assert rms_wrapped(r["theta"], th1) < TOL_PHASE_RMS
    assert math.sqrt(np.mean((r["w"] / w1 - 1) ** 2)) < TOL_PHASE_RMS


@pytest.mark.parametrize("P,N,c,I", [(512, 100, 0.125, 30), (200, 300, 0.25, 8), (130, 17, 0.5, 10),
                                     (1152, 100, 0.125, 12), (96, 129, 0.25, 6)])
def test_free_running_against_oracle(plans, P, N, c, I):
    tc, _ = plans
    pb = workloads.problem(P, N, 10.0, c, I, seed=7)
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
    r, ph = _solve(tc, pb)
    assert np.all(ph >= 0) and np.all(ph < 2 * np.pi)
    assert rms_wrapped(ph, ref["phase"]) < TOL_PHASE_RMS
    assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU
    assert rms_wrapped(r["theta"], ref["theta"]) < TOL_PHASE_RMS


@pytest.mark.parametrize("j", [1, 2])
def test_teacher_forced_large_grid(plans, j):
    # P = 1408: a subset mask (248 KB) larger than a block's shared memory is
    # drawn with bit sets in global memory instead
    tc, _ = plans
    pb = workloads.problem(1408, 40, 10.0, 0.125, 4, seed=5)
    st = oracle_states(oracle, pb, j, full_iterations=0)
    w0, th0 = st[j - 1]
    w1, th1 = st[j]
    r = tc.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, init_w=w0, init_theta=th0, first_iteration=j,
                 full_iterations=0, final_pass=False, state=True)
    assert rms_wrapped(r["theta"], th1) < TOL_PHASE_RMS
    assert math.sqrt(np.mean((r["w"] / w1 - 1) ** 2)) < TOL_PHASE_RMS


@pytest.mark.parametrize("j", [1, 2, 3])
def test_teacher_forced_tiny_subset(plans, j):
    # c = 1/64 at P = 96: 144 subset pixels for 129 spots (two spot blocks),
    # ragged tiles; one iteration at a time (free-running, a subset barely
    # larger than the spot count amplifies rounding differences)
    tc, cc = plans
    pb = workloads.problem(96, 129, 10.0, 1.0 / 64, 3, seed=7)
    st = oracle_states(oracle, pb, j, full_iterations=0)
    w0, th0 = st[j - 1]
    w1, th1 = st[j]
    kw = dict(init_w=w0, init_theta=th0, first_iteration=j, full_iterations=0, final_pass=False, state=True)
    r = tc.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, **kw)
    q = cc.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, **kw)
    assert rms_wrapped(r["theta"], q["theta"]) < 1e-4
    assert rms_wrapped(r["theta"], th1) < TOL_PHASE_RMS
    assert math.sqrt(np.mean((r["w"] / w1 - 1) ** 2)) < TOL_PHASE_RMS


@pytest.mark.parametrize("mode", ["windows", "fresh"])
def test_round_pupil(plans, mode):
    # the subset is drawn from the pupil's pixels (cycle walking on a rectangle
    # larger than D); the mask must pick exactly those
    tc, _ = plans
    pb = workloads.problem(512, 100, 10.0, 0.125, 12, seed=21)
    kw = dict(aperture="round", waist=290.0, subset_mode=mode)
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed, **kw)
    r, ph = _solve(tc, pb, **kw)
    om = oracle.pupil_pixels(pb.P, "round")
    assert rms_wrapped(ph[om], ref["phase"][om]) < TOL_PHASE_RMS
    assert np.all(np.delete(ph, om) == 0.0)
    assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU


def test_batch_against_cuda_core(plans):
    # several hundred tiles per launch, P not a multiple of the tile, N over
    # one, two and three spot blocks, square and round pupils, and two runs of
    # the same batch (the masks are cleared between uses).  Every hologram is
    # well conditioned: the oracle's phase map moves by at most 1.4e-5 rad RMS
    # when the spot coordinates change by 1e-9 relative (a subset only a few
    # times larger than N can amplify FP32 rounding differences without bound)
    tc, cc = plans
    pbs = []
    for i in range(20):
        P, N = [(512, 40), (300, 100), (256, 200), (384, 300)][i % 4]
        pb = workloads.problem(P, N, 5.0, 0.125, 8, seed=200 + i)
        if i % 3 == 0:
            pb.extra = {"aperture": "round", "waist": 0.4 * P}
        pbs.append(pb)
    outs1 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    outs2 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    b = tc.batch(pbs, outs1)
    for rep in range(2):
        b.run()
        r1 = b.results()
        r2 = cc.solve_batch(pbs, outs2)
        # two FP32 paths that round differently in every compressed iteration
        # (split-BF16 products against fixed-point sines): the parity bar
        for a, c2, o1, o2 in zip(r1, r2, outs1, outs2):
            assert rms_wrapped(o1.cpu().numpy(), o2.cpu().numpy()) < TOL_PHASE_RMS
            assert abs(a["e"] - c2["e"]) < TOL_EU and abs(a["u"] - c2["u"]) < TOL_EU
    b.close()


def test_square_batch_side_draws(plans):
    # every hologram square: the subset masks of launch L + 1 are drawn on a
    # side stream beside launch L, alternating two masks per hologram; three
    # runs of the same batch (both masks reused and cleared), P not a multiple
    # of the tile, one to three spot blocks
    tc, cc = plans
    pbs = [workloads.problem(P, N, 5.0, 0.125, 9, seed=400 + i)
           for i, (P, N) in enumerate([(512, 40), (300, 100), (256, 200), (384, 300), (512, 129), (200, 17)])]
    outs1 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    outs2 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    b = tc.batch(pbs, outs1)
    assert b.tile_shape()["threads"] == SUBSET_TC
    r2 = cc.solve_batch(pbs, outs2)
    ref = [o.cpu().numpy() for o in outs2]
    for rep in range(3):
        b.run()
        r1 = b.results()
        for a, c2, o1, o2 in zip(r1, r2, outs1, ref):
            assert rms_wrapped(o1.cpu().numpy(), o2) < TOL_PHASE_RMS
            assert abs(a["e"] - c2["e"]) < TOL_EU and abs(a["u"] - c2["u"]) < TOL_EU
    b.close()
    # the first hologram against the oracle
    pb = pbs[0]
    o = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
    assert rms_wrapped(outs1[0].cpu().numpy(), o["phase"]) < TOL_PHASE_RMS


def test_square_batch_uneven_schedules(plans):
    # side-stream mask draws when the holograms' schedules differ: compressed
    # iterations ending at different steps, WGS (no compressed iteration), RS
    # (no iteration), no full iteration before the final pass; each hologram
    # equals its solo solve
    tc, _ = plans
    pbs = [workloads.problem(256, 60, 5.0, 0.125, 9, seed=500),
           workloads.problem(384, 100, 5.0, 0.125, 3, seed=501),
           workloads.problem(256, 40, 5.0, 1.0, 5, seed=502),
           workloads.problem(200, 30, 5.0, 0.125, 0, seed=503),
           workloads.problem(320, 129, 5.0, 0.25, 6, seed=504)]
    pbs[4].extra["full_iterations"] = 0
    outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    b = tc.batch(pbs, outs)
    for rep in range(2):
        b.run()
        res = b.results()
        for pb, out, r in zip(pbs, outs, res):
            kw = dict(full_iterations=pb.extra.get("full_iterations", 2))
            o2 = torch.empty(pb.M, dtype=torch.float32, device="cuda")
            s2 = tc.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=o2, **kw)
            assert rms_wrapped(out.cpu().numpy(), o2.cpu().numpy()) < TOL_PHASE_RMS
            assert abs(r["e"] - s2["e"]) < TOL_EU and abs(r["u"] - s2["u"]) < TOL_EU
    b.close()


def test_serving(plans):
    # continuous batching: each admitted request gets a clear mask
    tc, cc = plans
    pbs = [workloads.problem(P, 60, 5.0, 0.25, 6, seed=300 + i) for i, P in enumerate((256, 192, 256, 128, 320, 256))]
    outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    tickets = [tc.submit(pb, out) for pb, out in zip(pbs, outs)]
    res = [tc.wait(t) for t in tickets]
    for pb, out, r in zip(pbs, outs, res):
        o2 = torch.empty(pb.M, dtype=torch.float32, device="cuda")
        s = cc.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=o2)
        assert rms_wrapped(out.cpu().numpy(), o2.cpu().numpy()) < TOL_PHASE_RMS
        assert abs(r["e"] - s["e"]) < TOL_EU and abs(r["u"] - s["u"]) < TOL_EU


# ---- the half-precision option on the tensor cores: GEMM 2 of compressed
# launches with single FP16 operands (full passes and the final pass keep the
# split BF16 products); held to the parity bar, not to the FP16-sincos one

@pytest.fixture(scope="module")
def half_plan(tmp_path_factory):
    from paper_2003_05293_gb300 import Plan
    path = tmp_path_factory.mktemp("half") / "h.json"
    plan = Plan(precision="fp32_fp16sincos",
                tune_cache=write_pinned_tune_cache(path, SUBSET_TC, 1, FULL_WS, half=True))
    yield plan
    plan.close()


def test_half_path_is_reported(half_plan):
    pbs = [workloads.problem(256, 40, 5.0, 0.125, 4, seed=s) for s in range(3)]
    b = half_plan.batch(pbs)
    assert b.tile_shape()["threads"] == SUBSET_TC
    b.close()


@pytest.mark.parametrize("P,N,c,j", [(512, 100, 0.125, 1), (512, 100, 0.125, 17), (96, 129, 1.0 / 64, 1),
                                     (96, 129, 1.0 / 64, 2)])
def test_half_teacher_forced_compressed_iteration(half_plan, P, N, c, j):
    pb = workloads.problem(P, N, 10.0, c, 30, seed=12 if P == 512 else 7)
    st = oracle_states(oracle, pb, j, full_iterations=0)
    w0, th0 = st[j - 1]
    w1, th1 = st[j]
    r = half_plan.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, init_w=w0, init_theta=th0, first_iteration=j,
                        full_iterations=0, final_pass=False, state=True)
    assert rms_wrapped(r["theta"], th1) < TOL_PHASE_RMS
    assert math.sqrt(np.mean((r["w"] / w1 - 1) ** 2)) < TOL_PHASE_RMS


@pytest.mark.parametrize("P,N,c,I", [(512, 100, 0.125, 30), (1152, 100, 0.125, 12), (200, 300, 0.25, 8)])
def test_half_free_running_against_oracle(half_plan, P, N, c, I):
    pb = workloads.problem(P, N, 10.0, c, I, seed=7)
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
    r, ph = _solve(half_plan, pb)
    assert rms_wrapped(ph, ref["phase"]) < TOL_PHASE_RMS
    assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU

"""Batched (persistent launch + CUDA graph) and served (continuous batching)
forms: every hologram equals its solo solve, and the solo solve equals the
oracle (covered in test_gpu_parity)."""
import time

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_EU, TOL_PHASE_RMS, rms_wrapped

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# batch/serve vs solo: same arithmetic, other tile shapes -> other FP32 summation order
TOL_SAME_PHASE = 1e-4
TOL_SAME_EU = 1e-5


@pytest.fixture(scope="module")
def plan():
    from paper_2003_05293_gb300 import Plan
    p = Plan(precision="fp32", max_batch=16)
    yield p
    p.close()


def solo(plan, pb):
    out = torch.empty(pb.M, dtype=torch.float32, device="cuda")
    r = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, amp=pb.amp, out=out)
    return r, out.cpu().numpy()


def small_mix(count, seed):
    return workloads.batch(count, seed=seed, P_choices=(64, 96, 128, 256), N_lo=1, N_hi=60,
                           gamma_max=5.0, c=0.25, iterations=6)


def test_batch_equals_solo(plan):
    pbs = small_mix(12, 3)
    pbs[3].iterations = 0          # RS inside a batch
    pbs[5].c = 1.0                 # WGS inside a batch
    pbs[7].extra["full_iterations"] = 0
    outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    b = plan.batch(pbs, outs)
    for rep in range(2):           # graph replays give the same result
        b.run()
        res = b.results()
        for pb, out, r in zip(pbs, outs, res):
            kw = dict(full_iterations=pb.extra.get("full_iterations", 2))
            o2 = torch.empty(pb.M, dtype=torch.float32, device="cuda")
            s = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=o2, **kw)
            assert rms_wrapped(out.cpu().numpy(), o2.cpu().numpy()) < TOL_SAME_PHASE
            assert abs(r["e"] - s["e"]) < TOL_SAME_EU and abs(r["u"] - s["u"]) < TOL_SAME_EU
    times = b.kernel_times()
    assert len(times) == 1 + max(pb.iterations for pb in pbs) + 1 and all(t > 0 for t in times[1:])
    tot, it = b.pairs()
    want = sum(pb.N * (2 * (pb.iterations - min(2 if pb is not pbs[7] else 0, pb.iterations))
                       * oracle.subset_size(pb.P, pb.c)
                       + 2 * min(2 if pb is not pbs[7] else 0, pb.iterations) * pb.M + 2 * pb.M)
               for pb in pbs)
    assert tot == want
    b.close()


def test_batch_against_oracle(plan):
    pbs = small_mix(4, 9)
    outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    b = plan.batch(pbs, outs)
    b.run()
    res = b.results()
    for pb, out, r in zip(pbs, outs, res):
        ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
        assert rms_wrapped(out.cpu().numpy(), ref["phase"]) < TOL_PHASE_RMS
        assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU
    b.close()


def test_batched_form_full_size():
    # the batched form at full size: 64 holograms, P in {512, 768, 1024, 1152},
    # N ~ U{10..300}, c = 1/8, 30 iterations, one persistent launch per
    # iteration on the autotuner's shapes; sampled holograms against the
    # oracle (the two smallest by P * N, and the largest N at P <= 768) and
    # against their solo solves, and e, u of every hologram in range
    from paper_2003_05293_gb300 import Plan
    pbs = workloads.batch(64, seed=11)
    with Plan(precision="fp32", max_batch=64) as big:
        outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
        b = big.batch(pbs, outs)
        b.run()
        res = b.results()
        for r in res:
            assert 0.0 < r["e"] <= 1.0 and 0.0 < r["u"] <= 1.0
        order = sorted(range(len(pbs)), key=lambda i: pbs[i].P * pbs[i].N)
        picks = order[:2] + [max((i for i in range(len(pbs)) if pbs[i].P <= 768), key=lambda i: pbs[i].N)]
        for i in picks:
            pb = pbs[i]
            ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
            assert rms_wrapped(outs[i].cpu().numpy(), ref["phase"]) < TOL_PHASE_RMS
            assert abs(res[i]["e"] - ref["e"]) < TOL_EU and abs(res[i]["u"] - ref["u"]) < TOL_EU
            o2 = torch.empty(pb.M, dtype=torch.float32, device="cuda")
            s = big.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=o2)
            assert rms_wrapped(outs[i].cpu().numpy(), o2.cpu().numpy()) < TOL_PHASE_RMS
            assert abs(res[i]["e"] - s["e"]) < TOL_EU and abs(res[i]["u"] - s["u"]) < TOL_EU
        b.close()


def test_solve_batch_host_outputs(plan):
    pbs = small_mix(5, 4)
    outs = [np.empty(pb.M, dtype=np.float32) for pb in pbs]
    res = plan.solve_batch(pbs, outs)
    for pb, out, r in zip(pbs, outs, res):
        s, ph = solo(plan, pb)
        assert rms_wrapped(out, ph) < TOL_SAME_PHASE
        assert abs(r["e"] - s["e"]) < TOL_SAME_EU
    # again with new inputs of the same shape (cached graph, restaged inputs)
    pbs2 = small_mix(5, 4)
    for pb in pbs2:
        pb.seed += 1
        pb.xyz = pb.xyz[::-1].copy()
    res2 = plan.solve_batch(pbs2, outs)
    for pb, out, r in zip(pbs2, outs, res2):
        s, ph = solo(plan, pb)
        assert rms_wrapped(out, ph) < TOL_SAME_PHASE
        assert abs(r["u"] - s["u"]) < TOL_SAME_EU


def test_pinned_and_pageable_host_outputs(plan):
    # host phase maps in pinned and in pageable memory: both give the device
    # result, for batches and single solves
    pbs = small_mix(4, 7)
    pinned = [torch.empty(pb.M, dtype=torch.float32, pin_memory=True).numpy() for pb in pbs]
    pageable = [np.empty(pb.M, dtype=np.float32) for pb in pbs]
    for o in pinned + pageable:
        o.fill(-1.0)
    r1 = plan.solve_batch(pbs, pinned)
    r2 = plan.solve_batch(pbs, pageable)
    for pb, a, b, x, y in zip(pbs, pinned, pageable, r1, r2):
        s, ph = solo(plan, pb)
        assert np.all(a >= 0) and rms_wrapped(a, ph) < TOL_SAME_PHASE
        assert np.array_equal(a, b)
        assert x["e"] == y["e"] and abs(x["e"] - s["e"]) < TOL_SAME_EU
    pb = pbs[0]
    host = torch.full((pb.M,), -1.0, dtype=torch.float32, pin_memory=True).numpy()
    r = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, amp=pb.amp, out=host)
    s, ph = solo(plan, pb)
    assert np.all(host >= 0) and rms_wrapped(host, ph) < TOL_SAME_PHASE and abs(r["e"] - s["e"]) < TOL_SAME_EU


def test_host_batches_alternating_equal_solve_batch(plan):
    # two host-buffer batches, each run on its own stream, alternated over four
    # steps with new spots and seeds each step (update, run one; collect the
    # other): every step's host maps and e, u equal the synchronous batch
    # solve of the same inputs
    shape = small_mix(5, 40)
    steps = [shape] + [[workloads.problem(ref.P, ref.N, 5.0, ref.c, ref.iterations, seed=100 * k + i)
                        for i, ref in enumerate(shape)] for k in range(1, 4)]   # same shapes, new spots and seeds
    outs = [[np.full(pb.M, -1.0, dtype=np.float32) for pb in st] for st in steps]
    pinned = [torch.empty(pb.M, dtype=torch.float32, pin_memory=True).numpy() for pb in shape]
    hb = [plan.host_batch(shape, pinned), plan.host_batch(shape, pinned)]
    res = [None] * 4
    for k in range(4):
        b = hb[k % 2]
        if k >= 2:
            res[k - 2] = b.results()
        b.update(steps[k], outs[k])
        b.run()
    res[2], res[3] = hb[0].results(), hb[1].results()
    for b in hb:
        b.close()
    for k in range(4):
        want = [np.full(pb.M, -1.0, dtype=np.float32) for pb in steps[k]]
        ref = plan.solve_batch(steps[k], want)
        for o, w, r, q in zip(outs[k], want, res[k], ref):
            assert np.all(o >= 0) and np.array_equal(o, w)
            assert r["e"] == q["e"] and r["u"] == q["u"]
    # a host batch takes host maps only, and keeps its shape on update
    with pytest.raises(Exception):
        plan.host_batch(shape, [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in shape])
    hb = plan.host_batch(shape)
    bad = [workloads.problem(shape[0].P * 2, shape[0].N, 5.0, shape[0].c, shape[0].iterations, seed=1)] + shape[1:]
    with pytest.raises(Exception):
        hb.update(bad)
    hb.close()


def test_serving_mixed_stream_equals_solo():
    from paper_2003_05293_gb300 import Plan
    with Plan(precision="fp32", max_batch=4) as p:
        pbs = small_mix(14, 21)
        outs = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
        tickets = []
        for i, (pb, out) in enumerate(zip(pbs, outs)):
            tickets.append(p.submit(pb, out))
            if i % 3 == 2:
                time.sleep(0.002)   # later arrivals join while earlier requests run
        results = [p.wait(t, 60.0) for t in tickets]
        st = p.serve_stats()
        assert st["completed"] == len(pbs) and st["active"] == 0
        assert st["launches"] < sum(pb.iterations + 1 for pb in pbs)   # requests shared launches
        for pb, out, r in zip(pbs, outs, results):
            assert r["status"] == 0
            s, ph = solo(p, pb)
            assert rms_wrapped(out.cpu().numpy(), ph) < TOL_SAME_PHASE
            assert abs(r["e"] - s["e"]) < TOL_SAME_EU and abs(r["u"] - s["u"]) < TOL_SAME_EU
            assert r["latency_ms"] >= r["queue_ms"] >= 0


def test_serving_host_output_and_poll():
    from paper_2003_05293_gb300 import Plan
    with Plan(precision="fp32", max_batch=2) as p:
        pb = small_mix(1, 5)[0]
        out = np.zeros(pb.M, dtype=np.float32)
        t = p.submit(pb, out)
        r = None
        for _ in range(20000):
            r = p.poll(t)
            if r is not None:
                break
            time.sleep(0.001)
        assert r is not None and r["status"] == 0
        s, ph = solo(p, pb)
        assert rms_wrapped(out, ph) < TOL_SAME_PHASE
        from paper_2003_05293_gb300 import CswgsError
        with pytest.raises(CswgsError):
            p.poll(t)                  # collected tickets are gone


def test_serving_cancel():
    from paper_2003_05293_gb300 import Plan
    with Plan(precision="fp32", max_batch=1) as p:
        # ~10^13 phasor pairs: seconds of work, so it is still running when cancelled
        big = workloads.problem(2048, 1000, 5.0, 1.0, 600, seed=1)
        small = small_mix(3, 8)
        tb = p.submit(big, None)
        ts = [p.submit(pb, None) for pb in small]
        assert p.cancel(ts[1]) == 0           # cancelled while queued
        time.sleep(0.05)
        assert p.cancel(tb) == 0              # cancelled while running
        rb = p.wait(tb, 60.0)
        assert rb["status"] == 6
        r1 = p.wait(ts[1], 60.0)
        assert r1["status"] == 6
        for t in (ts[0], ts[2]):
            r = p.wait(t, 60.0)
            assert r["status"] == 0 and 0 < r["u"] <= 1
        st = p.serve_stats()
        assert st["cancelled"] == 2 and st["bytes_in_use"] == 0


def test_serving_admission_by_memory():
    from paper_2003_05293_gb300 import CswgsError, Plan
    # a cap that holds one 256^2 request at a time (its phase map alone is 256 KiB)
    # and never a 1024^2 one (4 MiB phase map)
    with Plan(precision="fp32", max_batch=8, mem_cap_bytes=400 << 10) as p:
        pbs = [workloads.problem(256, 8, 2.0, 0.25, 4, seed=s) for s in range(4)]
        ts = [p.submit(pb, None) for pb in pbs]
        for t in ts:
            assert p.wait(t, 60.0)["status"] == 0
        st = p.serve_stats()
        assert st["completed"] == 4 and st["bytes_in_use"] == 0
        with pytest.raises(CswgsError) as ei:
            p.submit(workloads.problem(1024, 64, 2.0, 0.25, 4, seed=0), None)
        assert ei.value.status == 2
        assert p.serve_stats()["rejected"] == 1


@pytest.mark.parametrize("name", ["grid100", "grid36", "cubes100"])
def test_paper_scenarios_match_oracle(plan, name):
    # the paper's scenarios (Section 5) at P = 512: GPU e, u equal the oracle's,
    # and the rotated grids reach e, u > 0.9 as the paper reports for N <= 100
    pb = workloads.scenario(name, 512, seed=3)
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
    r, ph = solo(plan, pb)
    assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU
    assert rms_wrapped(ph, ref["phase"]) < TOL_PHASE_RMS
    if name.startswith("grid"):
        assert ref["e"] > 0.9 and ref["u"] > 0.9

"""The kernels of the full iterations and the final pass, side by side: the
tensor-core kernel (tcgen05, split-BF16 products accumulated in FP32,
warp-specialised and pipelined across tiles) and the CUDA-core separable
kernel.
Each plan is pinned to one of them through its tune cache; each tensor-core
kernel is compared with the FP64 oracle (teacher-forced full iterations, the
final pass, free-running solves) and with the CUDA-core kernel, over
grid sides that do and do not divide into the 128 x 64 tiles, spot counts
below and above the 128 of one spot block, the round pupil, and SLM frames."""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import TOL_EU, TOL_PHASE_RMS, oracle_states, rms_wrapped, write_pinned_tune_cache

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC_KERNELS = {"ws": 2}
CUDA_CORE = 256


def _plan(tmp_path, full):
    # a tune cache that pins every (P, N, batch) bucket these tests can reach to
    # one full-pass kernel: P rounded up to 128, N and the batch size to powers of two
    from paper_2003_05293_gb300 import Plan
    path = tmp_path / ("tune_%d.json" % full)
    return Plan(precision="fp32", tune_cache=write_pinned_tune_cache(path, 256, 4, full, batch_pow2=range(0, 5)))


@pytest.fixture(scope="module")
def cuda_core_plan(tmp_path_factory):
    plan = _plan(tmp_path_factory.mktemp("cc"), CUDA_CORE)
    yield plan
    plan.close()


@pytest.fixture(scope="module", params=sorted(TC_KERNELS), ids=sorted(TC_KERNELS))
def plans(request, tmp_path_factory, cuda_core_plan):
    tc = _plan(tmp_path_factory.mktemp(request.param), TC_KERNELS[request.param])
    tc.kernel = TC_KERNELS[request.param]
    yield tc, cuda_core_plan
    tc.close()


def _solve(plan, pb, **kw):
    out = torch.full((pb.M,), -1.0, dtype=torch.float32, device="cuda")
    r = plan.solve(pb.xyz, pb.P, pb.c, pb.iterations, pb.seed, out=out, state=True, **kw)
    torch.cuda.synchronize()
    return r, out.cpu().numpy().astype(np.float64)


def test_kernel_choice_is_reported(plans):
    tc, cc = plans
    pbs = [workloads.problem(256, 40, 5.0, 0.125, 4, seed=s) for s in range(4)]
    for plan, want in ((tc, tc.kernel), (cc, CUDA_CORE)):
        b = plan.batch(pbs)
        assert b.tile_shape()["full_threads"] == want
        b.close()


@pytest.mark.parametrize("j", [29, 30])
def test_teacher_forced_full_iteration(plans, j):
    tc, _ = plans
    pb = workloads.problem(512, 100, 10.0, 0.125, 30, seed=12)
    states = oracle_states(oracle, pb, pb.iterations)
    w0, th0 = states[j - 1]
    w1, th1 = states[j]
    r = tc.solve(pb.xyz, pb.P, pb.c, 1, pb.seed, init_w=w0, init_theta=th0, first_iteration=j, full_iterations=1,
                 final_pass=False, state=True)
    assert rms_wrapped(r["theta"], th1) < TOL_PHASE_RMS
    assert math.sqrt(np.mean((r["w"] / w1 - 1) ** 2)) < TOL_PHASE_RMS


@pytest.mark.parametrize("P,N", [(512, 100), (130, 17), (200, 300), (64, 1), (96, 129)])
def test_final_pass_against_oracle_and_cuda_core(plans, P, N):
    tc, cc = plans
    pb = workloads.problem(P, N, 5.0, 0.25, 0, seed=P + N)
    rng = np.random.default_rng(P)
    w = rng.uniform(0.5, 1.5, N)
    th = rng.uniform(-np.pi, np.pi, N)
    ref = oracle.solve(P, pb.xyz, c=pb.c, iterations=0, seed=pb.seed, theta_in=th, w_in=w)
    r1, ph1 = _solve(tc, pb, init_w=w, init_theta=th)
    r2, ph2 = _solve(cc, pb, init_w=w, init_theta=th)
    assert rms_wrapped(ph1, ref["phase"]) < TOL_PHASE_RMS
    assert abs(r1["e"] - ref["e"]) < TOL_EU and abs(r1["u"] - ref["u"]) < TOL_EU
    assert np.allclose(r1["I"], ref["I"], rtol=2e-3, atol=1e-8)
    # the two kernels: the split-BF16 products keep the tensor-core path at FP32 class
    assert rms_wrapped(ph1, ph2) < 1e-4
    assert abs(r1["e"] - r2["e"]) < 1e-5 and abs(r1["u"] - r2["u"]) < 1e-4


@pytest.mark.parametrize("P,N,c,I", [(512, 100, 0.125, 30), (200, 300, 0.25, 8), (1152, 100, 0.125, 12)])
def test_free_running_against_oracle(plans, P, N, c, I):
    tc, cc = plans
    pb = workloads.problem(P, N, 10.0, c, I, seed=7)
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed)
    r1, ph1 = _solve(tc, pb)
    assert np.all(ph1 >= 0) and np.all(ph1 < 2 * np.pi)
    assert rms_wrapped(ph1, ref["phase"]) < TOL_PHASE_RMS
    assert abs(r1["e"] - ref["e"]) < TOL_EU and abs(r1["u"] - ref["u"]) < TOL_EU
    assert rms_wrapped(r1["theta"], ref["theta"]) < TOL_PHASE_RMS


def test_wgs_all_full_iterations(plans):
    # plain WGS: every iteration over all pixels, all on the tensor cores
    tc, _ = plans
    pb = workloads.problem(130, 17, 5.0, 1.0, 10, seed=3)
    ref = oracle.solve(pb.P, pb.xyz, c=1.0, iterations=10, seed=pb.seed, full_iterations=10)
    r, ph = _solve(tc, pb, full_iterations=10)
    assert rms_wrapped(ph, ref["phase"]) < TOL_PHASE_RMS
    assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU


def test_round_pupil_and_slm_frame(plans):
    from paper_2003_05293_gb300 import SlmFrame
    tc, cc = plans
    pb = workloads.problem(512, 100, 10.0, 0.125, 12, seed=21)
    kw = dict(aperture="round", waist=290.0, subset_mode="windows")
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed, **kw)
    lut = torch.from_numpy(np.random.default_rng(0).integers(0, 256, 256).astype(np.uint8)).cuda()
    frame = torch.full((600, 704), 7, dtype=torch.uint8, device="cuda")
    r, ph = _solve(tc, pb, slm=SlmFrame(frame, lut, offset_x=96, offset_y=44), **kw)
    om = oracle.pupil_pixels(pb.P, "round")
    assert rms_wrapped(ph[om], ref["phase"][om]) < TOL_PHASE_RMS
    assert np.all(np.delete(ph, om) == 0.0)
    assert abs(r["e"] - ref["e"]) < TOL_EU and abs(r["u"] - ref["u"]) < TOL_EU
    want = oracle.slm_gray(ph.astype(np.float32), lut.cpu().numpy(), 256).reshape(pb.P, pb.P)
    f = frame.cpu().numpy()
    assert np.array_equal(f[44:44 + 512, 96:96 + 512], want)
    f[44:44 + 512, 96:96 + 512] = 7
    assert np.all(f == 7)


def test_batch_of_uneven_holograms(plans):
    tc, cc = plans
    pbs = [workloads.problem(P, N, 5.0, 0.125, 6, seed=i) for i, (P, N) in
           enumerate([(256, 40), (130, 17), (200, 300), (96, 129)])]
    outs1 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    outs2 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    r1 = tc.solve_batch(pbs, outs1)
    r2 = cc.solve_batch(pbs, outs2)
    for a, b, o1, o2 in zip(r1, r2, outs1, outs2):
        assert rms_wrapped(o1.cpu().numpy(), o2.cpu().numpy()) < 1e-4
        assert abs(a["e"] - b["e"]) < 1e-5 and abs(a["u"] - b["u"]) < 1e-4


def test_many_tiles_per_block(plans):
    # several hundred tiles over the persistent blocks, so that each block runs
    # a long chain of tiles through its pipeline: spot counts over one, two and
    # three spot blocks, round pupils (tiles that skip both products) beside
    # square ones, and both kinds of pass
    tc, cc = plans
    pbs, kws = [], []
    for i in range(24):
        N = (40, 100, 200, 300)[i % 4]
        pbs.append(workloads.problem(512, N, 5.0, 0.125, 4, seed=100 + i))
        kws.append({"aperture": "round", "waist": 200.0} if i % 3 == 0 else {})
    outs1 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    outs2 = [torch.empty(pb.M, dtype=torch.float32, device="cuda") for pb in pbs]
    for pb, kw in zip(pbs, kws):
        pb.extra = dict(kw, full_iterations=4)
    r1 = tc.solve_batch(pbs, outs1)
    r2 = cc.solve_batch(pbs, outs2)
    for a, b, o1, o2 in zip(r1, r2, outs1, outs2):
        assert rms_wrapped(o1.cpu().numpy(), o2.cpu().numpy()) < 1e-4
        assert abs(a["e"] - b["e"]) < 1e-5 and abs(a["u"] - b["u"]) < 1e-4
    # and one of them (two spot blocks, square pupil) against the oracle
    pb = pbs[2]
    ref = oracle.solve(pb.P, pb.xyz, c=pb.c, iterations=pb.iterations, seed=pb.seed, full_iterations=4)
    assert rms_wrapped(outs1[2].cpu().numpy().astype(np.float64), ref["phase"]) < TOL_PHASE_RMS
    assert abs(r1[2]["e"] - ref["e"]) < TOL_EU and abs(r1[2]["u"] - ref["u"]) < TOL_EU

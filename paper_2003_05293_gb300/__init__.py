"""GB300 (sm_103a) CS-WGS point-cloud hologram library: Python binding.

The work happens in ``lib/libcswgs.so`` (hand-written CUDA kernels behind the
C ABI of ``include/cswgs.h``).  This package marshals arguments: numpy arrays
for host data, torch CUDA tensors for device buffers (data pointers only), and
the torch stream handle when the caller wants the plan on its stream.

    plan = Plan(precision="fp32")
    out = torch.empty(P * P, device="cuda")
    r = plan.solve(xyz, P=1152, c=0.125, iterations=30, seed=0, out=out)
    r["e"], r["u"]
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi
from .capi import (CSWGS_FP32, CSWGS_FP32_FP16SINCOS, CSWGS_FP64, CswgsError, check,
                   cswgs_plan_desc, cswgs_pupil, cswgs_request, cswgs_result, cswgs_serve_stats,
                   cswgs_slm_frame, cswgs_solve_opts)

__all__ = ["Plan", "Batch", "CswgsError", "PRECISIONS", "APERTURES", "SUBSET_MODES", "SlmFrame", "capi",
           "spots_from_physical"]

PRECISIONS = {"fp64": CSWGS_FP64, "fp32": CSWGS_FP32, "fp32_fp16sincos": CSWGS_FP32_FP16SINCOS}
APERTURES = {"square": capi.CSWGS_APERTURE_SQUARE, "round": capi.CSWGS_APERTURE_ROUND}
SUBSET_MODES = {"fresh": capi.CSWGS_SUBSET_FRESH, "windows": capi.CSWGS_SUBSET_WINDOWS}


def _pupil(aperture="square", waist=0.0, subset_mode="fresh"):
    p = cswgs_pupil()
    p.aperture = APERTURES[aperture]
    p.subset_mode = SUBSET_MODES[subset_mode]
    p.beam_waist = float(waist)
    return p


_SQUARE = _pupil()


def _addr(a):
    """Address of a contiguous array, or None."""
    return None if a is None else a.ctypes.data


def _out_addr(out):
    """(address, on_host) of an output: a torch CUDA tensor, a numpy float32 array or None."""
    if out is None:
        return None, 0
    if isinstance(out, np.ndarray):
        if out.dtype != np.float32 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("host output must be a contiguous float32 array")
        return out.ctypes.data, 1
    if not out.is_cuda or out.dtype.__str__() != "torch.float32" or not out.is_contiguous():
        raise ValueError("device output must be a contiguous float32 CUDA tensor")
    return out.data_ptr(), 0


def _u8ptr(t):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), capi.c_uint8_p)


class SlmFrame:
    """A gray-level SLM frame on the device (cswgs_slm_frame): `frame` a uint8
    CUDA tensor of shape (height, pitch), `lut` a uint8 CUDA tensor of the phase
    levels' gray values, the grid placed at (offset_x, offset_y)."""

    def __init__(self, frame, lut, width=None, offset_x=0, offset_y=0):
        if frame.dtype.__str__() != "torch.uint8" or frame.dim() != 2 or not frame.is_contiguous():
            raise ValueError("frame must be a contiguous 2D uint8 CUDA tensor")
        if lut.dtype.__str__() != "torch.uint8" or lut.dim() != 1 or not lut.is_contiguous():
            raise ValueError("lut must be a contiguous 1D uint8 CUDA tensor")
        self.frame, self.lut = frame, lut
        self.c = cswgs_slm_frame()
        self.c.frame = _u8ptr(frame)
        self.c.height, self.c.pitch = frame.shape
        self.c.width = frame.shape[1] if width is None else int(width)
        self.c.offset_x, self.c.offset_y = int(offset_x), int(offset_y)
        self.c.lut = _u8ptr(lut)
        self.c.levels = lut.shape[0]


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(capi.c_double_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _out_ptr(out):
    """(float*, on_host) for a torch CUDA tensor, a numpy float32 array or None."""
    if out is None:
        return None, 0
    if isinstance(out, np.ndarray):
        if out.dtype != np.float32 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("host output must be a contiguous float32 array")
        return out.ctypes.data_as(capi.c_float_p), 1
    # torch tensor
    if not out.is_cuda or out.dtype.__str__() != "torch.float32" or not out.is_contiguous():
        raise ValueError("device output must be a contiguous float32 CUDA tensor")
    return ctypes.cast(ctypes.c_void_p(out.data_ptr()), capi.c_float_p), 0


def spots_from_physical(xyz_m, P: int, wavelength: float, focal_length: float, pixel_pitch: float):
    """cswgs_spots_from_physical: spots in metres (x, y in the focal plane, z
    from it) -> the normalised (alpha, beta, gamma) every solve takes."""
    xyz = _f64(xyz_m, (-1, 3))
    out = np.empty_like(xyz)
    o = capi.cswgs_optics(float(wavelength), float(focal_length), float(pixel_pitch))
    check(capi.load().cswgs_spots_from_physical(ctypes.byref(o), _dptr(xyz), xyz.shape[0], int(P), _dptr(out)),
          "cswgs_spots_from_physical")
    return out


class Plan:
    """A cswgs_plan: device, stream, limits, precision, tunings and serving loop.

    stream: a cudaStream_t handle (e.g. ``torch.cuda.Stream().cuda_stream``) the
    plan runs on, or None/0 for a stream of the plan's own.  torch's default
    stream has handle 0, so pass a non-default torch stream to share one."""

    def __init__(self, device: int = 0, max_P: int = 2048, max_N: int = 1024, max_batch: int = 64,
                 mem_cap_bytes: int = 0, precision: str = "fp32", stream=None, tune_cache=None):
        self.lib = capi.load()
        d = cswgs_plan_desc()
        self.lib.cswgs_plan_desc_default(ctypes.byref(d))
        d.device, d.max_P, d.max_N, d.max_batch = device, max_P, max_N, max_batch
        d.mem_cap_bytes = mem_cap_bytes
        d.precision = PRECISIONS[precision]
        d.stream = stream
        self._tune_cache = tune_cache.encode() if tune_cache else None
        d.tune_cache = self._tune_cache
        h = ctypes.c_void_p()
        check(self.lib.cswgs_plan_create(ctypes.byref(h), ctypes.byref(d)), "cswgs_plan_create")
        self.handle = h
        self.precision = precision
        self._keep = {}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.cswgs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------- solve --
    def solve(self, xyz, P: int, c: float, iterations: int, seed: int, amp=None, out=None,
              full_iterations: int = 2, first_iteration: int = 1, final_pass: bool = True,
              init_w=None, init_theta=None, state: bool = False, aperture: str = "square",
              waist: float = 0.0, subset_mode: str = "fresh", slm: "SlmFrame" = None):
        """cswgs_solve_ex; returns dict(e, u[, w, theta, I]).  aperture, waist
        and subset_mode give the pupil (cswgs_pupil); slm an SLM frame."""
        xyz = _f64(xyz, (-1, 3))
        N = xyz.shape[0]
        amp = _f64(amp)
        init_w = _f64(init_w)
        init_theta = _f64(init_theta)
        o = cswgs_solve_opts()
        self.lib.cswgs_solve_opts_default(ctypes.byref(o))
        o.full_iterations = full_iterations
        o.first_iteration = first_iteration
        o.final_pass = 1 if final_pass else 0
        o.init_w = _dptr(init_w)
        o.init_theta = _dptr(init_theta)
        w = np.empty(N) if state else None
        th = np.empty(N) if state else None
        In = np.empty(N) if state and final_pass else None
        o.final_w = _dptr(w)
        o.final_theta = _dptr(th)
        o.spot_intensity = _dptr(In)
        o.pupil = _pupil(aperture, waist, subset_mode)
        if slm is not None:
            o.slm = ctypes.pointer(slm.c)
        ptr, host = _out_ptr(out)
        e = ctypes.c_double(float("nan"))
        u = ctypes.c_double(float("nan"))
        check(self.lib.cswgs_solve_ex(self.handle, _dptr(xyz), _dptr(amp), N, P, float(c), int(iterations),
                                      int(seed) & (2**64 - 1), ctypes.byref(o), ptr, host,
                                      ctypes.byref(e), ctypes.byref(u)), "cswgs_solve_ex")
        res = {"e": e.value, "u": u.value}
        if state:
            res.update(w=w, theta=th, I=In)
        return res

    def solve_simple(self, xyz, P, c, iterations, seed, amp=None, out=None):
        """cswgs_solve (the plain entry point)."""
        xyz = _f64(xyz, (-1, 3))
        amp = _f64(amp)
        ptr, host = _out_ptr(out)
        e = ctypes.c_double()
        u = ctypes.c_double()
        check(self.lib.cswgs_solve(self.handle, _dptr(xyz), _dptr(amp), xyz.shape[0], P, float(c),
                                   int(iterations), int(seed) & (2**64 - 1), ptr, host,
                                   ctypes.byref(e), ctypes.byref(u)), "cswgs_solve")
        return {"e": e.value, "u": u.value}

    def subset(self, P: int, Mp: int, seed: int, j: int, out):
        """cswgs_subset into a CUDA int32 tensor of Mp entries."""
        ptr = ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_int32))
        check(self.lib.cswgs_subset(self.handle, P, Mp, int(seed) & (2**64 - 1), j, ptr), "cswgs_subset")

    def subset_ex(self, P: int, c: float, seed: int, j: int, out, aperture: str = "square",
                  subset_mode: str = "fresh") -> int:
        """cswgs_subset_ex into a CUDA int32 tensor with room for the pupil's
        pixel count; returns the subset size Mp."""
        ptr = ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_int32))
        pu = _pupil(aperture, 0.0, subset_mode)
        n = ctypes.c_int64()
        check(self.lib.cswgs_subset_ex(self.handle, P, float(c), int(seed) & (2**64 - 1), j, ctypes.byref(pu),
                                       ptr, ctypes.byref(n)), "cswgs_subset_ex")
        return n.value

    # ----------------------------------------------------------- batches --
    def _requests(self, problems, outs):
        n = len(problems)
        reqs = (cswgs_request * n)()
        keep = []
        for i, pb in enumerate(problems):
            xyz = _f64(pb.xyz, (-1, 3))
            amp = _f64(pb.amp)
            keep += [xyz, amp]
            r = reqs[i]
            r.spots_xyz = _addr(xyz)
            r.amplitudes = _addr(amp)
            r.N = xyz.shape[0]
            r.P = pb.P
            r.subset_fraction = pb.c
            r.iterations = pb.iterations
            r.seed = int(pb.seed) & (2**64 - 1)
            extra = getattr(pb, "extra", None)
            if extra:
                r.full_iterations = int(extra.get("full_iterations", 2))
                r.pupil = _pupil(extra.get("aperture", "square"), extra.get("waist", 0.0),
                                 extra.get("subset_mode", "fresh"))
                slm = extra.get("slm")
                if slm is not None:
                    r.slm = ctypes.pointer(slm.c)
                    keep.append(slm)
            else:
                r.full_iterations = 2
                r.pupil = _SQUARE
            r.phase_out, r.out_on_host = _out_addr(outs[i] if outs is not None else None)
        return reqs, keep

    def batch(self, problems, outs=None) -> "Batch":
        reqs, keep = self._requests(problems, outs)
        h = ctypes.c_void_p()
        check(self.lib.cswgs_batch_create(self.handle, reqs, len(problems), ctypes.byref(h)),
              "cswgs_batch_create")
        return Batch(self, h, len(problems), keep + [outs])

    def host_batch(self, problems, outs=None) -> "HostBatch":
        """cswgs_batch_create_host: a batch with host inputs and host phase maps
        (numpy float32 arrays, or None) that runs on a stream of its own."""
        reqs, keep = self._requests(problems, outs)
        h = ctypes.c_void_p()
        check(self.lib.cswgs_batch_create_host(self.handle, reqs, len(problems), ctypes.byref(h)),
              "cswgs_batch_create_host")
        return HostBatch(self, h, len(problems), keep + [outs])

    def solve_batch(self, problems, outs=None):
        reqs, keep = self._requests(problems, outs)
        res = (cswgs_result * len(problems))()
        check(self.lib.cswgs_solve_batch(self.handle, reqs, len(problems), res), "cswgs_solve_batch")
        return [{"e": r.e, "u": r.u, "latency_ms": r.latency_ms} for r in res]

    # ----------------------------------------------------------- serving --
    def submit(self, pb, out=None) -> int:
        reqs, keep = self._requests([pb], [out])
        t = ctypes.c_uint64()
        check(self.lib.cswgs_submit(self.handle, reqs, ctypes.byref(t)), "cswgs_submit")
        self._keep[t.value] = (reqs, keep, out)
        return t.value

    def poll(self, ticket: int):
        """None while pending, else dict(status, e, u, latency_ms, queue_ms)."""
        r = cswgs_result()
        st = self.lib.cswgs_poll(self.handle, ticket, ctypes.byref(r))
        if st == capi.CSWGS_EBUSY:
            return None
        self._keep.pop(ticket, None)
        if st not in (capi.CSWGS_OK, capi.CSWGS_ECANCELLED):
            check(st, "cswgs_poll")
        return {"status": st, "e": r.e, "u": r.u, "latency_ms": r.latency_ms, "queue_ms": r.queue_ms}

    def wait(self, ticket: int, timeout_s: float = 60.0):
        r = cswgs_result()
        st = self.lib.cswgs_wait(self.handle, ticket, float(timeout_s), ctypes.byref(r))
        if st not in (capi.CSWGS_OK, capi.CSWGS_ECANCELLED):
            check(st, "cswgs_wait")
        self._keep.pop(ticket, None)
        return {"status": st, "e": r.e, "u": r.u, "latency_ms": r.latency_ms, "queue_ms": r.queue_ms}

    def cancel(self, ticket: int) -> int:
        return self.lib.cswgs_cancel(self.handle, ticket)

    def serve_stats(self) -> dict:
        s = cswgs_serve_stats()
        check(self.lib.cswgs_serve_stats_get(self.handle, ctypes.byref(s)), "cswgs_serve_stats_get")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def test_waits(self, withhold_first_item: bool, wait_polls: int = 0):
        """cswgs_plan_test_waits: the test of the tensor-core kernel's bounded waits."""
        check(self.lib.cswgs_plan_test_waits(self.handle, 1 if withhold_first_item else 0, int(wait_polls)),
              "cswgs_plan_test_waits")

    # ------------------------------------------------------ tuning/probes --
    def autotune(self, P: int, N: int, c: float) -> float:
        ms = ctypes.c_double()
        check(self.lib.cswgs_autotune(self.handle, P, N, float(c), ctypes.byref(ms)), "cswgs_autotune")
        return ms.value

    def sincos_peak(self):
        v = ctypes.c_double()
        mhz = ctypes.c_double()
        check(self.lib.cswgs_sincos_peak(self.handle, ctypes.byref(v), ctypes.byref(mhz)), "cswgs_sincos_peak")
        return v.value, mhz.value


class Batch:
    """A cswgs_batch: device-resident holograms with a captured CUDA graph."""

    def __init__(self, plan: Plan, handle, count: int, keep):
        self.plan, self.handle, self.count, self._keep = plan, handle, count, keep
        self.lib = plan.lib

    def run(self):
        check(self.lib.cswgs_batch_run(self.handle), "cswgs_batch_run")

    def results(self):
        res = (cswgs_result * self.count)()
        check(self.lib.cswgs_batch_results(self.handle, res), "cswgs_batch_results")
        return [{"e": r.e, "u": r.u, "latency_ms": r.latency_ms} for r in res]

    def kernel_times(self):
        n = ctypes.c_int()
        check(self.lib.cswgs_batch_kernel_times(self.handle, None, 0, ctypes.byref(n)), "kernel_times")
        ms = (ctypes.c_float * n.value)()
        check(self.lib.cswgs_batch_kernel_times(self.handle, ms, n.value, ctypes.byref(n)), "kernel_times")
        return list(ms)

    def pairs(self):
        a = ctypes.c_double()
        b = ctypes.c_double()
        check(self.lib.cswgs_batch_pairs(self.handle, ctypes.byref(a), ctypes.byref(b)), "cswgs_batch_pairs")
        return a.value, b.value

    def tile_shape(self):
        """dict: threads, pixels_per_thread, blocks (compressed iterations);
        full_threads, full_blocks (full iterations and final pass)."""
        v = [ctypes.c_int() for _ in range(5)]
        check(self.lib.cswgs_batch_tile_shape(self.handle, *[ctypes.byref(x) for x in v]), "cswgs_batch_tile_shape")
        keys = ("threads", "pixels_per_thread", "full_threads", "blocks", "full_blocks")
        return dict(zip(keys, (x.value for x in v)))

    def close(self):
        if self.handle:
            self.lib.cswgs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostBatch(Batch):
    """A cswgs_batch of cswgs_batch_create_host: host spots in, host phase maps
    out, on the batch's own stream (run() returns once the work is queued)."""

    def update(self, problems, outs=None):
        """cswgs_batch_update: the next run's spots, seeds and host phase maps."""
        reqs, keep = self.plan._requests(problems, outs)
        check(self.lib.cswgs_batch_update(self.handle, reqs, len(problems)), "cswgs_batch_update")
        # the previous run may still write its maps: its buffers stay referenced
        # until the run after this one is set up
        self._keep = [self._keep[-1] if self._keep else None, keep + [outs]]

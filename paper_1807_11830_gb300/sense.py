"""Thin Python binding of libsense.so (ctypes; argument marshalling only).

The functions keep the C names of ``include/sense.h`` and take PyTorch CUDA
tensors, which serve only as device memory; every step of the computation
runs in the library's kernels.  A missing library raises -- there is no
fallback path.

Tensor conventions (all contiguous, on the plan's device):
  images x, out          complex64  [frames, ny, nx]
  S (C64 storage)        complex64  [coils, ny, nx]
  y (C64 storage)        complex64  [frames, coils, lines, nx]
  S, y (BF16 storage)    bfloat16   [..., 2]  (re, im pairs)
  lines                  int32      [frames, lines]
"""
import ctypes
import os

import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsense.so")

STORE_C64 = 0
STORE_BF16 = 1

SENSE_OK = 0
STATUS_NAMES = {
    0: "SENSE_OK", 1: "SENSE_EINVAL", 2: "SENSE_EUNSUPPORTED_SIZE", 3: "SENSE_ENOMEM", 4: "SENSE_ECUDA",
    5: "SENSE_ETIMEOUT", 6: "SENSE_ENUMERIC", 7: "SENSE_EQUEUE_FULL", 8: "SENSE_ENOTFOUND", 9: "SENSE_EDEVICE",
}
CG_CONVERGED, CG_MAXITER, CG_BREAKDOWN = 1, 2, 3

EXPORTED = (
    "sense_size_supported", "sense_plan_create", "sense_plan_destroy", "sense_plan_workspace_bytes",
    "sense_forward", "sense_adjoint", "sense_normal", "sense_cg_solve", "sense_cg_solve_host", "sense_rss",
    "sense_c32_to_bf16",
    "sense_plan_check", "sense_last_error", "sense_plan_set_timing", "sense_plan_phase_time",
    "sense_adjoint_noalloc", "sense_plan_set_variant", "sense_plan_variant", "sense_plan_autotune",
    "sense_plan_set_cg_mode", "sense_selftest_wait", "sense_fp32_peak", "sense_plan_set_column_pass", "sense_plan_set_lambda", "sense_batch_set_lambda",
    "sense_plan_set_temporal", "sense_batch_set_temporal",
    "sense_batch_create", "sense_batch_destroy", "sense_batch_workspace_bytes", "sense_batch_classes",
    "sense_batch_autotune", "sense_batch_set_variant", "sense_batch_cg_solve", "sense_batch_check",
    "sense_queue_create", "sense_queue_create_with_hooks", "sense_queue_submit", "sense_queue_poll", "sense_queue_wait", "sense_queue_cancel",
    "sense_queue_stats_get", "sense_queue_variant", "sense_queue_set_variant", "sense_queue_destroy",
)
REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_CANCELLED, REQ_FAILED = 0, 1, 2, 3, 4
NORM_VARIANTS = 4
# transform lengths compiled into the library (ny and nx each; sense_size_supported)
SIZES = (8, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 120, 128, 144, 160, 192, 240, 256, 288, 320, 384)

PHASES = ("rows_fwd", "rows_inv", "fwd_col", "adj_col", "normal", "cg_normal", "cg_update", "cg_persistent",
          "maps_transpose", "cg_finish", "fwd_fused", "adj_fused")
CG_MODE_GRAPH, CG_MODE_PERSISTENT, CG_MODE_DIRECT = 0, 1, 2


class SenseError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))


class _Shape(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nx", ctypes.c_int), ("coils", ctypes.c_int),
                ("frames", ctypes.c_int), ("lines", ctypes.c_int), ("storage", ctypes.c_int),
                ("centred", ctypes.c_int)]


def _shape_struct(d):
    """sense_shape from a dict with ny, nx, coils, frames, lines and
    optionally storage (default complex64) and centred (default 0)."""
    return _Shape(d["ny"], d["nx"], d["coils"], d["frames"], d["lines"], d.get("storage", STORE_C64),
                  int(d.get("centred", 0)))


class _BatchIO(ctypes.Structure):
    _fields_ = [("y", ctypes.c_void_p), ("S", ctypes.c_void_p), ("lines", ctypes.c_void_p),
                ("x_out", ctypes.c_void_p), ("iters_out", ctypes.c_void_p), ("rel_resid_out", ctypes.c_void_p),
                ("outcome_out", ctypes.c_void_p)]


class _QueueCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_live", ctypes.c_int), ("autotune", ctypes.c_int),
                ("iters_per_tick", ctypes.c_int), ("staging_reserve_bytes", ctypes.c_size_t),
                ("max_live_work", ctypes.c_size_t), ("admit_waves", ctypes.c_double)]


class _QueueHooks(ctypes.Structure):
    """sense_queue_test_hooks (sense_testing.h): host-only scheduler tests."""
    _fields_ = [("fake_device", ctypes.c_int), ("fake_tick_us", ctypes.c_int), ("fake_iters", ctypes.c_int),
                ("fail_admit_every", ctypes.c_int)]


class _QueueStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("refused", ctypes.c_uint64),
                ("ticks", ctypes.c_uint64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("hbm_in_use", ctypes.c_size_t),
                ("hbm_budget", ctypes.c_size_t), ("live", ctypes.c_int), ("pending", ctypes.c_int),
                ("staging_reserved", ctypes.c_size_t), ("staging_in_use", ctypes.c_size_t)]


_LIB = None


def load_library(path=LIB_PATH):
    """Load libsense.so and declare its entry points (raises if not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError("libsense.so is not built (%s); run paper_1807_11830_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    vp, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    lib.sense_size_supported.argtypes = [i]
    lib.sense_size_supported.restype = i
    lib.sense_plan_create.argtypes = [ctypes.POINTER(_Shape), i, ctypes.POINTER(vp)]
    lib.sense_plan_create.restype = st
    lib.sense_plan_destroy.argtypes = [vp]
    lib.sense_plan_destroy.restype = st
    lib.sense_plan_workspace_bytes.argtypes = [vp]
    lib.sense_plan_workspace_bytes.restype = ctypes.c_size_t
    for name in ("sense_forward", "sense_adjoint", "sense_normal"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp, vp, vp]
        getattr(lib, name).restype = st
    lib.sense_cg_solve.argtypes = [vp, vp, vp, vp, i, ctypes.c_double, vp, vp, vp, vp, vp]
    lib.sense_cg_solve.restype = st
    lib.sense_cg_solve_host.argtypes = [vp, vp, vp, vp, i, ctypes.c_double, vp, vp, vp, vp, vp]
    lib.sense_cg_solve_host.restype = st
    lib.sense_rss.argtypes = [vp, vp, vp, vp, vp]
    lib.sense_rss.restype = st
    lib.sense_c32_to_bf16.argtypes = [vp, vp, ctypes.c_size_t, vp]
    lib.sense_c32_to_bf16.restype = st
    lib.sense_plan_check.argtypes = [vp, vp]
    lib.sense_plan_check.restype = st
    lib.sense_plan_set_timing.argtypes = [vp, i]
    lib.sense_plan_set_timing.restype = st
    lib.sense_plan_phase_time.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long)]
    lib.sense_plan_phase_time.restype = st
    lib.sense_adjoint_noalloc.argtypes = [ctypes.POINTER(_Shape), vp, vp, vp, vp, vp]
    lib.sense_adjoint_noalloc.restype = st
    lib.sense_plan_set_variant.argtypes = [vp, i]
    lib.sense_plan_set_variant.restype = st
    lib.sense_plan_variant.argtypes = [vp]
    lib.sense_plan_variant.restype = i
    lib.sense_plan_set_lambda.argtypes = [vp, ctypes.c_double]
    lib.sense_plan_set_lambda.restype = st
    lib.sense_batch_set_lambda.argtypes = [vp, i, ctypes.c_double]
    lib.sense_batch_set_lambda.restype = st
    lib.sense_plan_set_temporal.argtypes = [vp, ctypes.c_double]
    lib.sense_plan_set_temporal.restype = st
    lib.sense_batch_set_temporal.argtypes = [vp, i, ctypes.c_double]
    lib.sense_batch_set_temporal.restype = st
    lib.sense_plan_autotune.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), vp]
    lib.sense_plan_autotune.restype = st
    lib.sense_plan_set_column_pass.argtypes = [vp, i]
    lib.sense_plan_set_column_pass.restype = st
    lib.sense_plan_set_cg_mode.argtypes = [vp, i]
    lib.sense_plan_set_cg_mode.restype = st
    lib.sense_selftest_wait.argtypes = [i, ctypes.c_long]
    lib.sense_selftest_wait.restype = st
    lib.sense_fp32_peak.argtypes = [i, ctypes.POINTER(ctypes.c_double)]
    lib.sense_fp32_peak.restype = st
    bp = ctypes.POINTER(_BatchIO)
    lib.sense_batch_create.argtypes = [ctypes.POINTER(_Shape), i, i, ctypes.POINTER(vp)]
    lib.sense_batch_create.restype = st
    lib.sense_batch_destroy.argtypes = [vp]
    lib.sense_batch_destroy.restype = st
    lib.sense_batch_workspace_bytes.argtypes = [vp]
    lib.sense_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.sense_batch_classes.argtypes = [vp]
    lib.sense_batch_classes.restype = i
    lib.sense_batch_autotune.argtypes = [vp, bp, vp]
    lib.sense_batch_autotune.restype = st
    lib.sense_batch_set_variant.argtypes = [vp, i, i]
    lib.sense_batch_set_variant.restype = st
    lib.sense_batch_cg_solve.argtypes = [vp, bp, i, ctypes.c_double, vp]
    lib.sense_batch_cg_solve.restype = st
    lib.sense_batch_check.argtypes = [vp, vp]
    lib.sense_batch_check.restype = st
    lib.sense_queue_create.argtypes = [i, ctypes.POINTER(_QueueCfg), ctypes.POINTER(vp)]
    lib.sense_queue_create.restype = st
    lib.sense_queue_create_with_hooks.argtypes = [i, ctypes.POINTER(_QueueCfg), ctypes.POINTER(_QueueHooks),
                                                  ctypes.POINTER(vp)]
    lib.sense_queue_create_with_hooks.restype = st
    lib.sense_queue_submit.argtypes = [vp, ctypes.POINTER(_Shape), vp, vp, vp, i, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_uint64)]
    lib.sense_queue_submit.restype = st
    lib.sense_queue_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.sense_queue_poll.restype = st
    lib.sense_queue_wait.argtypes = [vp, ctypes.c_uint64, vp, vp, vp, vp, ctypes.c_double]
    lib.sense_queue_wait.restype = st
    lib.sense_queue_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.sense_queue_cancel.restype = st
    lib.sense_queue_stats_get.argtypes = [vp, ctypes.POINTER(_QueueStats)]
    lib.sense_queue_stats_get.restype = st
    lib.sense_queue_variant.argtypes = [vp, i, i, i]
    lib.sense_queue_variant.restype = i
    lib.sense_queue_set_variant.argtypes = [vp, i, i, i, i]
    lib.sense_queue_set_variant.restype = st
    lib.sense_queue_destroy.argtypes = [vp]
    lib.sense_queue_destroy.restype = st
    lib.sense_last_error.argtypes = []
    lib.sense_last_error.restype = ctypes.c_char_p
    _LIB = lib
    return lib


def _check(rc):
    if rc != SENSE_OK:
        msg = load_library().sense_last_error()
        raise SenseError(rc, msg.decode() if msg else "")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def sense_size_supported(n):
    return bool(load_library().sense_size_supported(int(n)))


class Plan:
    """Owns a ``sense_plan*`` (twiddles + workspace) for one problem shape."""

    def __init__(self, ny, nx, coils, frames, lines, storage=STORE_C64, device=0, centred=False):
        lib = load_library()
        self.shape = dict(ny=ny, nx=nx, coils=coils, frames=frames, lines=lines, storage=storage,
                          centred=int(centred))
        self.device = device
        h = ctypes.c_void_p()
        sh = _Shape(ny, nx, coils, frames, lines, storage, int(centred))
        _check(lib.sense_plan_create(ctypes.byref(sh), device, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().sense_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self):
        return load_library().sense_plan_workspace_bytes(self.handle)


def sense_plan_create(ny, nx, coils, frames, lines, storage=STORE_C64, device=0):
    return Plan(ny, nx, coils, frames, lines, storage, device)


def sense_plan_destroy(plan):
    plan.close()


def sense_forward(plan, x, S, lines, y, stream=None):
    _check(load_library().sense_forward(plan.handle, _ptr(x), _ptr(S), _ptr(lines), _ptr(y), _stream(stream)))
    return y


def sense_adjoint(plan, y, S, lines, x, stream=None):
    _check(load_library().sense_adjoint(plan.handle, _ptr(y), _ptr(S), _ptr(lines), _ptr(x), _stream(stream)))
    return x


def sense_adjoint_noalloc(shape, y, S, lines, x, stream=None):
    """Adjoint without a plan and without device allocation (fixed-size
    library scratch; see include/sense.h).  `shape` is a dict with ny, nx,
    coils, frames, lines and optionally storage and centred."""
    sh = _shape_struct(shape)
    _check(load_library().sense_adjoint_noalloc(ctypes.byref(sh), _ptr(y), _ptr(S), _ptr(lines), _ptr(x),
                                                _stream(stream)))
    return x


def sense_normal(plan, x, S, lines, out, stream=None):
    _check(load_library().sense_normal(plan.handle, _ptr(x), _ptr(S), _ptr(lines), _ptr(out), _stream(stream)))
    return out


def sense_cg_solve(plan, y, S, lines, max_iter, rel_tol, x_out, iters_out=None, rel_resid_out=None,
                   outcome_out=None, stream=None):
    _check(load_library().sense_cg_solve(plan.handle, _ptr(y), _ptr(S), _ptr(lines), int(max_iter),
                                         float(rel_tol), _ptr(x_out), _ptr(iters_out), _ptr(rel_resid_out),
                                         _ptr(outcome_out), _stream(stream)))
    return x_out


def _host_ptr(t):
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return ctypes.c_void_p(t.data_ptr())


def sense_cg_solve_host(plan, y, S, lines, max_iter, rel_tol, x_out, iters_out=None, rel_resid_out=None,
                        outcome_out=None, stream=None):
    """CG-SENSE on host tensors (pinned for asynchronous copies); returns once
    the results are in `x_out` (and the optional per-frame outputs)."""
    _check(load_library().sense_cg_solve_host(plan.handle, _host_ptr(y), _host_ptr(S), _host_ptr(lines),
                                              int(max_iter), float(rel_tol), _host_ptr(x_out),
                                              _host_ptr(iters_out), _host_ptr(rel_resid_out),
                                              _host_ptr(outcome_out), _stream(stream)))


def sense_rss(plan, y, lines, out, stream=None):
    _check(load_library().sense_rss(plan.handle, _ptr(y), _ptr(lines), _ptr(out), _stream(stream)))
    return out


def sense_c32_to_bf16(inp, out, stream=None):
    count = inp.numel()
    _check(load_library().sense_c32_to_bf16(_ptr(inp), _ptr(out), count, _stream(stream)))
    return out


def sense_plan_check(plan, stream=None):
    _check(load_library().sense_plan_check(plan.handle, _stream(stream)))


def sense_plan_set_timing(plan, on):
    _check(load_library().sense_plan_set_timing(plan.handle, 1 if on else 0))


def sense_plan_phase_time(plan, phase):
    """(summed kernel milliseconds, launches) of a phase name or index."""
    idx = PHASES.index(phase) if isinstance(phase, str) else int(phase)
    ms = ctypes.c_double()
    n = ctypes.c_long()
    _check(load_library().sense_plan_phase_time(plan.handle, idx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def sense_plan_set_lambda(plan, lam):
    """Tikhonov weight of the plan's CG: solves (E^H E + lam I) x = E^H y."""
    _check(load_library().sense_plan_set_lambda(plan.handle, float(lam)))


def sense_batch_set_lambda(batch, instance, lam):
    _check(load_library().sense_batch_set_lambda(batch.handle, int(instance), float(lam)))


def sense_plan_set_temporal(plan, lam_t):
    """Couple the plan's frames in time: one CG on (E^H E + lam I + lam_t L) x = E^H y."""
    _check(load_library().sense_plan_set_temporal(plan.handle, float(lam_t)))


def sense_batch_set_temporal(batch, instance, lam_t):
    _check(load_library().sense_batch_set_temporal(batch.handle, int(instance), float(lam_t)))


def sense_plan_set_cg_mode(plan, mode):
    _check(load_library().sense_plan_set_cg_mode(plan.handle, int(mode)))


def sense_plan_set_column_pass(plan, staged):
    _check(load_library().sense_plan_set_column_pass(plan.handle, int(staged)))


def sense_plan_set_variant(plan, variant):
    _check(load_library().sense_plan_set_variant(plan.handle, int(variant)))


def sense_plan_variant(plan):
    return load_library().sense_plan_variant(plan.handle)


def sense_plan_autotune(plan, S, lines, stream=None):
    """Time the normal-operator variants on this plan; returns (chosen, {variant: ms})."""
    v = ctypes.c_int(-1)
    ms = (ctypes.c_double * NORM_VARIANTS)()
    _check(load_library().sense_plan_autotune(plan.handle, _ptr(S), _ptr(lines), ctypes.byref(v), ms,
                                              _stream(stream)))
    return v.value, {k: ms[k] for k in range(NORM_VARIANTS) if ms[k] >= 0}


def sense_selftest_wait(device=0, max_spins=1000):
    """Returns the status of the bounded-wait self-test (5 = SENSE_ETIMEOUT expected)."""
    return load_library().sense_selftest_wait(int(device), int(max_spins))


def sense_fp32_peak(device=0):
    """Measured FP32 FMA throughput of the device, TFLOP/s."""
    out = ctypes.c_double()
    _check(load_library().sense_fp32_peak(int(device), ctypes.byref(out)))
    return out.value


def to_bf16_pairs(t, stream=None):
    """complex64 CUDA tensor -> bfloat16 [..., 2] tensor (RNE, in the library's kernel)."""
    out = torch.empty(tuple(t.shape) + (2,), dtype=torch.bfloat16, device=t.device)
    return sense_c32_to_bf16(t.contiguous(), out, stream)


class Batch:
    """Owns a ``sense_batch*``: many instances, one persistent CG launch per size class."""

    def __init__(self, shapes, device=0):
        lib = load_library()
        arr = (_Shape * len(shapes))(*[_shape_struct(d) for d in shapes])
        h = ctypes.c_void_p()
        _check(lib.sense_batch_create(arr, len(shapes), device, ctypes.byref(h)))
        self.handle = h
        self.count = len(shapes)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().sense_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def classes(self):
        return load_library().sense_batch_classes(self.handle)

    @property
    def workspace_bytes(self):
        return load_library().sense_batch_workspace_bytes(self.handle)


def _batch_io(items):
    """items: list of dicts with y, S, lines, x_out and optional iters_out, rel_resid_out, outcome_out."""
    arr = (_BatchIO * len(items))()
    for k, d in enumerate(items):
        arr[k] = _BatchIO(*[(_ptr(d.get(name)).value if d.get(name) is not None else None)
                            for name in ("y", "S", "lines", "x_out", "iters_out", "rel_resid_out", "outcome_out")])
    return arr


def sense_batch_create(shapes, device=0):
    return Batch(shapes, device)


def sense_batch_destroy(batch):
    batch.close()


def sense_batch_workspace_bytes(batch):
    return batch.workspace_bytes


def sense_batch_classes(batch):
    return batch.classes


def sense_batch_autotune(batch, items, stream=None):
    _check(load_library().sense_batch_autotune(batch.handle, _batch_io(items), _stream(stream)))


def sense_batch_set_variant(batch, ny, variant):
    _check(load_library().sense_batch_set_variant(batch.handle, int(ny), int(variant)))


def sense_batch_cg_solve(batch, items, max_iter, rel_tol=0.0, stream=None):
    _check(load_library().sense_batch_cg_solve(batch.handle, _batch_io(items), int(max_iter), float(rel_tol),
                                               _stream(stream)))


def sense_batch_check(batch, stream=None):
    _check(load_library().sense_batch_check(batch.handle, _stream(stream)))


def _np_ptr(a):
    import numpy as np  # host buffers of the queue are numpy arrays
    if a is None:
        return None
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous array")
    return ctypes.c_void_p(a.ctypes.data)


class Queue:
    """Owns a ``sense_queue*`` (scheduler thread + device-resident requests).
    Host buffers are numpy arrays: y, S complex64 (or uint16 [...,2] bf16
    bits), lines int32."""

    def __init__(self, device=0, hbm_budget_bytes=0, max_live=0, fake_device=False, fake_tick_us=0,
                 fake_iters=0, autotune=False, iters_per_tick=0, fail_admit_every=0, staging_reserve_bytes=0,
                 max_live_work=0, admit_waves=0.0):
        cfg = _QueueCfg(hbm_budget_bytes, max_live, 1 if autotune else 0, iters_per_tick, staging_reserve_bytes,
                        max_live_work, float(admit_waves))
        h = ctypes.c_void_p()
        lib = load_library()
        if fake_device or fake_tick_us or fake_iters or fail_admit_every:  # test hooks (sense_testing.h)
            hooks = _QueueHooks(1 if fake_device else 0, fake_tick_us, fake_iters, fail_admit_every)
            _check(lib.sense_queue_create_with_hooks(device, ctypes.byref(cfg), ctypes.byref(hooks), ctypes.byref(h)))
        else:
            _check(lib.sense_queue_create(device, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h

    def submit(self, shape, y, S, lines, max_iter, rel_tol=0.0):
        sh = _shape_struct(shape)
        rid = ctypes.c_uint64()
        _check(load_library().sense_queue_submit(self.handle, ctypes.byref(sh), _np_ptr(y), _np_ptr(S),
                                                 _np_ptr(lines), int(max_iter), float(rel_tol), ctypes.byref(rid)))
        return rid.value

    def poll(self, rid):
        st_, it = ctypes.c_int(), ctypes.c_int()
        _check(load_library().sense_queue_poll(self.handle, rid, ctypes.byref(st_), ctypes.byref(it)))
        return st_.value, it.value

    def wait(self, rid, x=None, iters=None, resid=None, outcome=None, timeout_s=0.0):
        _check(load_library().sense_queue_wait(self.handle, rid, _np_ptr(x), _np_ptr(iters), _np_ptr(resid),
                                               _np_ptr(outcome), float(timeout_s)))

    def cancel(self, rid):
        _check(load_library().sense_queue_cancel(self.handle, rid))

    def stats(self):
        s_ = _QueueStats()
        _check(load_library().sense_queue_stats_get(self.handle, ctypes.byref(s_)))
        return {k: getattr(s_, k) for k, _ in _QueueStats._fields_}

    def variant(self, ny, nx, storage=STORE_C64):
        return load_library().sense_queue_variant(self.handle, ny, nx, storage)

    def set_variant(self, ny, nx, variant, storage=STORE_C64):
        _check(load_library().sense_queue_set_variant(self.handle, int(ny), int(nx), int(storage), int(variant)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().sense_queue_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sense_queue_create(device=0, **cfg):
    return Queue(device, **cfg)


def sense_queue_submit(q, shape, y, S, lines, max_iter, rel_tol=0.0):
    return q.submit(shape, y, S, lines, max_iter, rel_tol)


def sense_queue_poll(q, rid):
    return q.poll(rid)


def sense_queue_wait(q, rid, x=None, iters=None, resid=None, outcome=None, timeout_s=0.0):
    return q.wait(rid, x, iters, resid, outcome, timeout_s)


def sense_queue_cancel(q, rid):
    return q.cancel(rid)


def sense_queue_stats_get(q):
    return q.stats()


def sense_queue_variant(q, ny, nx, storage=STORE_C64):
    return q.variant(ny, nx, storage)


def sense_queue_set_variant(q, ny, nx, variant, storage=STORE_C64):
    return q.set_variant(ny, nx, variant, storage)


def sense_queue_destroy(q):
    q.close()

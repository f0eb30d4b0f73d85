"""FP64 oracle references of the 320x320, 32-coil precision study, computed
in a background thread while the other GPU tests run.

The study's reference CG takes minutes on the host (50 iterations of the
literal E^H(E p) per slice), so `start()` is called once collection has
chosen the precision test (tests/conftest.py) and `get()` waits for it.  The
oracle is a C library called through ctypes, which releases the GIL, so the
thread runs beside the GPU tests.

Workload: three of the 16 slices of synth.slices_320 (320x320, 32 coils,
acceleration 3, 107 lines of which 24 centre lines), k-space E x + noise made
by the oracle from the exact maps and phantoms.  References, all FP64:
  c64  -- inputs rounded to complex64 (what the complex64 path is given);
  bf16 -- inputs rounded to bfloat16 pairs (what the BF16 path is given).
"""
import threading

import numpy as np

import oracle
from paper_1807_11830_gb300 import synth

SLICES = (3, 9, 14)
K = 50

_lock = threading.Lock()
_thread = None
_result = {}


def c64_round(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def problem():
    """(x_true, S, lines, y) of the selected slices, y = E x + noise in FP64."""
    p = synth.slices_320(frames=16)
    sel = list(SLICES)
    y = oracle.forward(p.x_true[sel], p.S, p.lines[sel]) + p.noise[sel]
    return p.x_true[sel], p.S, p.lines[sel], y


def _compute():
    try:
        x, S, lines, y = problem()
        inputs = {"c64": (c64_round(y), c64_round(S)),
                  "bf16": (oracle.quantize_c64_bf16(y), oracle.quantize_c64_bf16(S))}
        x32 = c64_round(x)
        out = {"x": x32, "lines": lines, "inputs": inputs}

        def run(name):
            yy, SS = inputs[name]
            out["cg_" + name] = oracle.cg(yy, SS, lines, K)
            out["forward_" + name] = oracle.forward(x32, SS, lines)
            out["adjoint_" + name] = oracle.adjoint(yy, SS, lines)
            out["normal_" + name] = oracle.normal(x32, SS, lines)

        workers = [threading.Thread(target=run, args=(n,)) for n in inputs]
        for w in workers:
            w.start()
        for w in workers:
            w.join()
        _result.update(out)
    except BaseException as exc:  # reported by get()
        _result["error"] = exc


def start():
    global _thread
    with _lock:
        if _thread is None:
            _thread = threading.Thread(target=_compute, name="precision-oracle", daemon=True)
            _thread.start()


def get(timeout=1800.0):
    start()
    _thread.join(timeout)
    if _thread.is_alive():
        raise TimeoutError("the oracle references of the precision study did not finish in %.0f s" % timeout)
    if "error" in _result:
        raise _result["error"]
    return _result

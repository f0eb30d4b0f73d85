"""FP64 CPU oracle for multi-coil Cartesian SENSE -- TEST INFRASTRUCTURE ONLY.

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.

Every function takes and returns numpy arrays (complex128 images, int32
lines) and calls the plain C++ implementation in ``sense_oracle.cpp``:

* ``dft`` / ``fft`` / ``fft2``  -- unitary DFT (direct O(n^2) and recursive
  mixed radix), sign exp(-2 pi i jk/n) forward;
* ``forward``   -- E   (arXiv 1807.11830 Sec. IV-A; encoding model of Eq. 1);
* ``adjoint``   -- E^H, which with every line sampled is Eq. 1 itself;
* ``normal``    -- E^H E computed literally as adjoint(forward(x));
* ``normal_collapsed`` -- the column-wise form of E^H E (a pin, not a path);
* ``cg``        -- Hestenes-Stiefel CG-SENSE per frame;
* ``rss``       -- root sum of squares coil combine (Sec. IV-B);
* ``bf16_rne``  -- binary32 -> bfloat16 round-to-nearest-even.

Layouts: x [F][ny][nx], S [C][ny][nx], y [F][C][L][nx], lines [F][L].
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

CG_CONVERGED = 1
CG_MAXITER = 2
CG_BREAKDOWN = 3


def _load(path):
    """Load an oracle shared library and declare its entry points."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i = ctypes.c_int
    lib.orc_dft.argtypes = [i, i, dp, dp]
    lib.orc_fft.argtypes = [i, i, dp, dp]
    lib.orc_fft2.argtypes = [i, i, i, i, dp, dp, i]
    for name in ("orc_forward", "orc_adjoint", "orc_normal"):
        getattr(lib, name).argtypes = [i, i, i, i, i, dp, dp, ip, dp, i]
    lib.orc_normal_collapsed.argtypes = [i, i, i, i, i, dp, dp, ip, dp]
    lib.orc_cg.argtypes = [i, i, i, i, i, dp, dp, ip, i, ctypes.c_double, dp, ip, dp, ip, i, ctypes.c_double,
                           ctypes.c_double]
    lib.orc_rss.argtypes = [i, i, i, i, i, dp, ip, dp, i]
    lib.orc_bf16_rne.argtypes = [ctypes.c_long, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_uint16)]
    lib.orc_bf16_rne.restype = None
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [i]
    lib.orc_set_threads.restype = None
    return lib


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = _load(_build.build())
    return _LIB


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s rejected its arguments (status %d)" % (what, rc))


def threads():
    return _lib().orc_threads()


def set_threads(n):
    _lib().orc_set_threads(int(n))


def dft(v, inverse=False):
    v = _c128(v)
    out = np.empty_like(v)
    _check(_lib().orc_dft(v.shape[0], 1 if inverse else -1, _dptr(v), _dptr(out)), "dft")
    return out


def fft(v, inverse=False):
    v = _c128(v)
    out = np.empty_like(v)
    _check(_lib().orc_fft(v.shape[0], 1 if inverse else -1, _dptr(v), _dptr(out)), "fft")
    return out


def fft2(img, inverse=False, centred=False):
    img = _c128(img)
    ny, nx = img.shape[-2:]
    count = int(np.prod(img.shape[:-2])) if img.ndim > 2 else 1
    out = np.empty_like(img)
    _check(_lib().orc_fft2(count, ny, nx, 1 if inverse else -1, _dptr(img), _dptr(out), int(centred)), "fft2")
    return out


def _shape(x_or_none, S, lines):
    S = _c128(S)
    lines = np.ascontiguousarray(lines, dtype=np.int32)
    C, ny, nx = S.shape
    F, L = lines.shape
    return S, lines, F, C, ny, nx, L


def forward(x, S, lines, centred=False):
    S, lines, F, C, ny, nx, L = _shape(x, S, lines)
    x = _c128(x).reshape(F, ny, nx)
    y = np.empty((F, C, L, nx), np.complex128)
    _check(_lib().orc_forward(F, C, ny, nx, L, _dptr(x), _dptr(S), _iptr(lines), _dptr(y), int(centred)),
           "forward")
    return y


def adjoint(y, S, lines, centred=False):
    S, lines, F, C, ny, nx, L = _shape(None, S, lines)
    y = _c128(y).reshape(F, C, L, nx)
    x = np.empty((F, ny, nx), np.complex128)
    _check(_lib().orc_adjoint(F, C, ny, nx, L, _dptr(y), _dptr(S), _iptr(lines), _dptr(x), int(centred)),
           "adjoint")
    return x


def normal(x, S, lines, centred=False):
    S, lines, F, C, ny, nx, L = _shape(x, S, lines)
    x = _c128(x).reshape(F, ny, nx)
    out = np.empty_like(x)
    _check(_lib().orc_normal(F, C, ny, nx, L, _dptr(x), _dptr(S), _iptr(lines), _dptr(out), int(centred)),
           "normal")
    return out


def normal_collapsed(x, S, lines):
    S, lines, F, C, ny, nx, L = _shape(x, S, lines)
    x = _c128(x).reshape(F, ny, nx)
    out = np.empty_like(x)
    _check(_lib().orc_normal_collapsed(F, C, ny, nx, L, _dptr(x), _dptr(S), _iptr(lines), _dptr(out)),
           "normal_collapsed")
    return out


def cg(y, S, lines, max_iter, tol=0.0, centred=False, lam=0.0, lam_t=0.0):
    """CG on (E^H E + lam I) x = E^H y per frame; with lam_t > 0 one CG over
    all frames on (E^H E + lam I + lam_t L) x = E^H y, L the cyclic second
    difference across frames.  Returns (x, iters[F], resid[F], status[F])."""
    S, lines, F, C, ny, nx, L = _shape(None, S, lines)
    y = _c128(y).reshape(F, C, L, nx)
    x = np.empty((F, ny, nx), np.complex128)
    iters = np.zeros(F, np.int32)
    resid = np.zeros(F, np.float64)
    status = np.zeros(F, np.int32)
    _check(_lib().orc_cg(F, C, ny, nx, L, _dptr(y), _dptr(S), _iptr(lines), int(max_iter), float(tol),
                         _dptr(x), _iptr(iters), _dptr(resid), _iptr(status), int(centred), float(lam),
                         float(lam_t)), "cg")
    return x, iters, resid, status


def rss(y, lines, ny, centred=False):
    lines = np.ascontiguousarray(lines, dtype=np.int32)
    y = _c128(y)
    F, C, L, nx = y.shape
    out = np.empty((F, ny, nx), np.float64)
    _check(_lib().orc_rss(F, C, ny, nx, L, _dptr(y), _iptr(lines), _dptr(out), int(centred)), "rss")
    return out


def bf16_rne(a):
    """float32 array -> uint16 array of bfloat16 bit patterns (RNE)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty(a.shape, np.uint16)
    _lib().orc_bf16_rne(a.size, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)))
    return out


def bf16_to_f32(bits):
    """Exact widening of bfloat16 bit patterns back to float32."""
    bits = np.ascontiguousarray(bits, dtype=np.uint16)
    return (bits.astype(np.uint32) << 16).view(np.float32)


def quantize_c64_bf16(a):
    """complex array -> complex128 array whose re/im are the bf16-rounded
    binary32 values (the oracle's 'quantised input' mode)."""
    a = np.asarray(a)
    f32 = np.ascontiguousarray(a, dtype=np.complex64).view(np.float32)
    q = bf16_to_f32(bf16_rne(f32))
    return q.view(np.complex64).astype(np.complex128).reshape(a.shape)

"""Plain CPU oracle for exact grey-value dilation / erosion (test infrastructure).

This package is the reference the CUDA library is checked against.  It is
TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never imports, links or calls it, and it shares no code with
the library.

Every function computes the plain definition from the paper:

* :func:`dilate` -- Eq. 6new cropped to the image domain as in Eq. 6 (value 0
  where no SE tap is valid), plus the number of taps attaining the maximum
  and, optionally, the whole count polynomial of Eq. Obs7.
* :func:`erode` -- Eq. Erosion computed directly (min over the SE), not by
  duality, so that duality can be tested against it.
* :func:`dilate_backward` -- the tie-split argmax gradient of the max-plus
  dilation, in fp64, summed in a fixed order.
* :func:`erode_backward` -- the same for the erosion (argmin taps; b enters
  with a minus sign).
* :func:`dilate3d` / :func:`erode3d` -- the definitions on 3-D volumes with a
  3-D SE (the method is stated for N-D images, Sec. 2.1 and Sec. 3).
* :func:`opening` / :func:`closing` / :func:`gradient` -- the composite
  operators named in the paper's conclusion, written out in NumPy on the raw
  integer intermediate (no tonal shift).

The arithmetic lives in ``morph_oracle.c`` (plain C, OpenMP over image rows
only); :func:`build` compiles it with gcc.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "morph_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmorph_oracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/libmorph_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            f64p = ctypes.POINTER(ctypes.c_double)
            ci = ctypes.c_int
            lib.orc_dilate.argtypes = [i32p, ci, ci, ci, ci, ci, ci, ci, ci, u8p, i32p,
                                       i32p, i32p, i32p, ci, ci, ci]
            lib.orc_erode.argtypes = [i32p, ci, ci, ci, ci, ci, ci, ci, ci, u8p, i32p,
                                      i32p, i32p, ci, ci, ci]
            lib.orc_dilate_backward.argtypes = [i32p, ci, ci, ci, ci, ci, ci, ci, ci, u8p, i32p,
                                                i32p, i32p, f64p, f64p, f64p]
            lib.orc_erode_backward.argtypes = [i32p, ci, ci, ci, ci, ci, ci, ci, ci, u8p, i32p,
                                               i32p, i32p, f64p, f64p, f64p]
            lib.orc_morph3d.argtypes = [i32p, ci, ci, ci, ci, ci, ci, ci, ci, ci, ci, ci, u8p, i32p, ci,
                                        i32p, i32p, ci]
            lib.orc_max_offset.argtypes = [ci, ci, u8p, i32p]
            for fn in (lib.orc_dilate, lib.orc_erode, lib.orc_dilate_backward, lib.orc_erode_backward, lib.orc_morph3d,
                       lib.orc_max_offset, lib.orc_max_threads):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _prep(f, mask, offset, origin):
    f = np.ascontiguousarray(np.asarray(f), dtype=np.int32)
    if f.ndim == 2:
        f = f[None]
    if f.ndim != 3:
        raise ValueError("image must be [H, W] or [N, H, W]")
    mask = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
    offset = np.ascontiguousarray(np.asarray(offset), dtype=np.int32)
    if mask.ndim != 2 or offset.shape != mask.shape:
        raise ValueError("mask and offset must be [kh, kw] arrays of one shape")
    oy, ox = (int(origin[0]), int(origin[1]))
    return f, mask, offset, oy, ox


_ERR = {1: "invalid argument", 2: "value out of range (pixel not in [0, L) or negative SE offset)"}


def _check(rc):
    if rc != 0:
        raise ValueError("oracle: " + _ERR.get(rc, f"error {rc}"))


def max_offset(mask, offset) -> int:
    """max b over B (0 for an empty B)."""
    m = np.asarray(offset)[np.asarray(mask) != 0]
    return int(m.max()) if m.size else 0


def dilate(f, L, mask, offset, origin, counts=False, rows=None, nthreads=1):
    """Dilation of Eq. 6 with top-coefficient counts.

    Returns ``(D, cD)`` or ``(D, cD, C)`` with ``C[n, i, j, d]`` the count
    polynomial of Eq. Obs7 (``d`` in ``[0, L + max b)``).  ``rows=(a, b)``
    computes only image rows ``a..b-1`` (other outputs stay 0).
    """
    lib = _load()
    f, mask, offset, oy, ox = _prep(f, mask, offset, origin)
    N, H, W = f.shape
    kh, kw = mask.shape
    D = np.zeros((N, H, W), np.int32)
    cD = np.zeros((N, H, W), np.int32)
    C = None
    if counts:
        R = int(L) + max_offset(mask, offset)
        C = np.zeros((N, H, W, R), np.int32)
    a, b = rows if rows is not None else (0, H)
    _check(lib.orc_dilate(_p(f, ctypes.c_int32), N, H, W, int(L), kh, kw, oy, ox,
                          _p(mask, ctypes.c_uint8), _p(offset, ctypes.c_int32),
                          _p(D, ctypes.c_int32), _p(cD, ctypes.c_int32), _p(C, ctypes.c_int32),
                          int(a), int(b), int(nthreads)))
    return (D, cD, C) if counts else (D, cD)


def erode(f, L, mask, offset, origin, rows=None, nthreads=1):
    """Erosion of Eq. Erosion, computed directly; returns ``(E, cE)``."""
    lib = _load()
    f, mask, offset, oy, ox = _prep(f, mask, offset, origin)
    N, H, W = f.shape
    kh, kw = mask.shape
    E = np.zeros((N, H, W), np.int32)
    cE = np.zeros((N, H, W), np.int32)
    a, b = rows if rows is not None else (0, H)
    _check(lib.orc_erode(_p(f, ctypes.c_int32), N, H, W, int(L), kh, kw, oy, ox,
                         _p(mask, ctypes.c_uint8), _p(offset, ctypes.c_int32),
                         _p(E, ctypes.c_int32), _p(cE, ctypes.c_int32),
                         int(a), int(b), int(nthreads)))
    return E, cE


def dilate_backward(f, L, mask, offset, origin, D, cD, g):
    """Tie-split argmax gradient of the dilation; returns ``(grad_f, grad_b)`` in fp64."""
    lib = _load()
    f, mask, offset, oy, ox = _prep(f, mask, offset, origin)
    N, H, W = f.shape
    kh, kw = mask.shape
    D = np.ascontiguousarray(np.asarray(D).reshape(N, H, W), dtype=np.int32)
    cD = np.ascontiguousarray(np.asarray(cD).reshape(N, H, W), dtype=np.int32)
    g = np.ascontiguousarray(np.asarray(g).reshape(N, H, W), dtype=np.float64)
    gf = np.zeros((N, H, W), np.float64)
    gb = np.zeros((kh, kw), np.float64)
    _check(lib.orc_dilate_backward(_p(f, ctypes.c_int32), N, H, W, int(L), kh, kw, oy, ox,
                                   _p(mask, ctypes.c_uint8), _p(offset, ctypes.c_int32),
                                   _p(D, ctypes.c_int32), _p(cD, ctypes.c_int32),
                                   _p(g, ctypes.c_double), _p(gf, ctypes.c_double),
                                   _p(gb, ctypes.c_double)))
    return gf, gb


def erode_backward(f, L, mask, offset, origin, E, cE, g):
    """Tie-split argmin gradient of the erosion; returns ``(grad_f, grad_b)`` in fp64."""
    lib = _load()
    f, mask, offset, oy, ox = _prep(f, mask, offset, origin)
    N, H, W = f.shape
    kh, kw = mask.shape
    E = np.ascontiguousarray(np.asarray(E).reshape(N, H, W), dtype=np.int32)
    cE = np.ascontiguousarray(np.asarray(cE).reshape(N, H, W), dtype=np.int32)
    g = np.ascontiguousarray(np.asarray(g).reshape(N, H, W), dtype=np.float64)
    gf = np.zeros((N, H, W), np.float64)
    gb = np.zeros((kh, kw), np.float64)
    _check(lib.orc_erode_backward(_p(f, ctypes.c_int32), N, H, W, int(L), kh, kw, oy, ox,
                                  _p(mask, ctypes.c_uint8), _p(offset, ctypes.c_int32),
                                  _p(E, ctypes.c_int32), _p(cE, ctypes.c_int32),
                                  _p(g, ctypes.c_double), _p(gf, ctypes.c_double),
                                  _p(gb, ctypes.c_double)))
    return gf, gb


def _morph3d(f, L, mask, offset, origin, op, nthreads):
    lib = _load()
    f = np.ascontiguousarray(np.asarray(f), dtype=np.int32)
    if f.ndim == 3:
        f = f[None]
    mask = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
    offset = np.ascontiguousarray(np.asarray(offset), dtype=np.int32)
    if f.ndim != 4 or mask.ndim != 3 or offset.shape != mask.shape:
        raise ValueError("volume [N, Z, H, W] or [Z, H, W]; mask and offset [kd, kh, kw]")
    N, Z, H, W = f.shape
    kd, kh, kw = mask.shape
    out = np.zeros(f.shape, np.int32)
    cnt = np.zeros(f.shape, np.int32)
    _check(lib.orc_morph3d(_p(f, ctypes.c_int32), N, Z, H, W, int(L), kd, kh, kw,
                           int(origin[0]), int(origin[1]), int(origin[2]),
                           _p(mask, ctypes.c_uint8), _p(offset, ctypes.c_int32), int(op),
                           _p(out, ctypes.c_int32), _p(cnt, ctypes.c_int32), int(nthreads)))
    return out, cnt


def dilate3d(f, L, mask, offset, origin, nthreads=1):
    """3-D dilation (Eq. 6new / Eq. 6 on volumes); returns ``(D, cD)``."""
    return _morph3d(f, L, mask, offset, origin, 0, nthreads)


def erode3d(f, L, mask, offset, origin, nthreads=1):
    """3-D erosion (Eq. Erosion on volumes); returns ``(E, cE)``."""
    return _morph3d(f, L, mask, offset, origin, 1, nthreads)


def max_threads() -> int:
    """Threads an OpenMP region of the oracle would use."""
    return int(_load().orc_max_threads())


# ---------------------------------------------------------------- composites
# Opening, closing and the Beucher gradient (the combinations named in the
# paper's conclusion), written out from the definitions of Sec. 2.1 on the raw
# integer intermediate, with no tonal shift: the erosion's result may be
# negative.  Empty-tap convention: where no tap is valid, a dilation gives the
# lowest value of its input's tonal range and an erosion the highest (for an
# image in [0, L) these are Eq. 6's 0 and L - 1).  The erosion result lies in
# [-max b, L - 1] and the dilation result in [0, L - 1 + max b].

def _dilate_raw(g, lo, mask, offset, origin):
    """max over taps y in B with x - y in F of g(x - y) + b(y) (Eq. 6new); lo where none."""
    g = np.asarray(g, np.int64)
    N, H, W = g.shape
    oy, ox = int(origin[0]), int(origin[1])
    none = np.iinfo(np.int64).min
    out = np.full(g.shape, none, np.int64)
    for r, c in zip(*np.nonzero(np.asarray(mask))):
        dy, dx = int(r) - oy, int(c) - ox                   # y = (dy, dx); source x - y
        i0, i1 = max(0, dy), min(H, H + dy)
        j0, j1 = max(0, dx), min(W, W + dx)
        if i0 >= i1 or j0 >= j1:
            continue
        cand = g[:, i0 - dy:i1 - dy, j0 - dx:j1 - dx] + int(offset[r, c])
        out[:, i0:i1, j0:j1] = np.maximum(out[:, i0:i1, j0:j1], cand)
    out[out == none] = lo
    return out


def _erode_raw(g, hi, mask, offset, origin):
    """min over taps y in B with x + y in F of g(x + y) - b(y) (Eq. Erosion); hi where none."""
    g = np.asarray(g, np.int64)
    N, H, W = g.shape
    oy, ox = int(origin[0]), int(origin[1])
    none = np.iinfo(np.int64).max
    out = np.full(g.shape, none, np.int64)
    for r, c in zip(*np.nonzero(np.asarray(mask))):
        dy, dx = int(r) - oy, int(c) - ox                   # y = (dy, dx); source x + y
        i0, i1 = max(0, -dy), min(H, H - dy)
        j0, j1 = max(0, -dx), min(W, W - dx)
        if i0 >= i1 or j0 >= j1:
            continue
        cand = g[:, i0 + dy:i1 + dy, j0 + dx:j1 + dx] - int(offset[r, c])
        out[:, i0:i1, j0:j1] = np.minimum(out[:, i0:i1, j0:j1], cand)
    out[out == none] = hi
    return out


def _prep3(f):
    f = np.asarray(f)
    return f[None] if f.ndim == 2 else f


def opening(f, L, mask, offset, origin):
    """(f erode b) dilate b on the raw integers; int64 [N, H, W]."""
    f = _prep3(f)
    mb = max_offset(mask, offset)
    E = _erode_raw(f, int(L) - 1, mask, offset, origin)         # in [-max b, L - 1]
    return _dilate_raw(E, -mb, mask, offset, origin)


def closing(f, L, mask, offset, origin):
    """(f dilate b) erode b on the raw integers; int64 [N, H, W]."""
    f = _prep3(f)
    mb = max_offset(mask, offset)
    D = _dilate_raw(f, 0, mask, offset, origin)                 # in [0, L - 1 + max b]
    return _erode_raw(D, int(L) - 1 + mb, mask, offset, origin)


def gradient(f, L, mask, offset, origin):
    """Beucher gradient (f dilate b) - (f erode b); int64 [N, H, W]."""
    f = _prep3(f)
    return _dilate_raw(f, 0, mask, offset, origin) - _erode_raw(f, int(L) - 1, mask, offset, origin)

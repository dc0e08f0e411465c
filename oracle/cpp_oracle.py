"""ctypes binding of the plain C++ oracle in ``oracle/cpp/oracle.cpp``.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  ``build()`` compiles the
library with g++ (no GPU code); ``load()`` builds it on first use.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpp", "oracle.cpp")
_LIB = os.path.join(_HERE, "cpp", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle shared library (plain C++17, -O2, pthreads)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(
        ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp]
    )
    os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            sz, p, i = ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int
            lib.orc_verify.argtypes = [i, sz, p, p, p, p, p, i]
            lib.orc_sign.argtypes = [i, sz, p, p, p, p, p, p, i]
            lib.orc_scalar_mul.argtypes = [i, sz, p, p, p, i]
            lib.orc_msm.argtypes = [i, sz, p, p, p, i]
            lib.orc_fe_mul.argtypes = [i, i, sz, p, p, p]
            lib.orc_fe_inv.argtypes = [i, i, sz, p, p]
            lib.orc_limbs.argtypes = [i]
            _lib = lib
    return _lib


def default_threads():
    return max(1, os.cpu_count() or 1)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def verify(curve_id, hash_be, r_be, s_be, pub_be, threads=None):
    """Arrays of shape (n, 32), (n, 32), (n, 32), (n, 64) uint8 -> (n,) uint8."""
    lib = load()
    h, r, s, q = _u8(hash_be), _u8(r_be), _u8(s_be), _u8(pub_be)
    n = h.shape[0]
    ok = np.zeros(n, dtype=np.uint8)
    rc = lib.orc_verify(curve_id, n, _ptr(h), _ptr(r), _ptr(s), _ptr(q), _ptr(ok),
                        threads or default_threads())
    if rc != 0:
        raise ValueError(f"orc_verify: unsupported curve {curve_id}")
    return ok


def sign(curve_id, d_be, e_be, k_be, threads=None):
    """Returns (r, s, pub) as uint8 arrays (n, 32), (n, 32), (n, 64)."""
    lib = load()
    d, e, k = _u8(d_be), _u8(e_be), _u8(k_be)
    n = d.shape[0]
    r = np.zeros((n, 32), np.uint8)
    s = np.zeros((n, 32), np.uint8)
    pub = np.zeros((n, 64), np.uint8)
    rc = lib.orc_sign(curve_id, n, _ptr(d), _ptr(e), _ptr(k), _ptr(r), _ptr(s), _ptr(pub),
                      threads or default_threads())
    if rc != 0:
        raise ValueError(f"orc_sign: unsupported curve {curve_id}")
    return r, s, pub


def scalar_mul(curve_id, k_limbs, pts_limbs, threads=None):
    lib = load()
    k, P = _u32(k_limbs), _u32(pts_limbs)
    out = np.zeros_like(P)
    rc = lib.orc_scalar_mul(curve_id, k.shape[0], _ptr(k), _ptr(P), _ptr(out),
                            threads or default_threads())
    if rc != 0:
        raise ValueError("orc_scalar_mul failed")
    return out


def msm(curve_id, pts_limbs, k_limbs, threads=None):
    lib = load()
    k, P = _u32(k_limbs), _u32(pts_limbs)
    m = lib.orc_limbs(curve_id)
    out = np.zeros(2 * m, np.uint32)
    rc = lib.orc_msm(curve_id, k.shape[0], _ptr(P), _ptr(k), _ptr(out),
                     threads or default_threads())
    if rc != 0:
        raise ValueError("orc_msm failed")
    return out


def fe_mul(curve_id, which, a_limbs, b_limbs):
    lib = load()
    a, b = _u32(a_limbs), _u32(b_limbs)
    out = np.zeros_like(a)
    lib.orc_fe_mul(curve_id, which, a.shape[0], _ptr(a), _ptr(b), _ptr(out))
    return out


def fe_inv(curve_id, which, a_limbs):
    lib = load()
    a = _u32(a_limbs)
    out = np.zeros_like(a)
    lib.orc_fe_inv(curve_id, which, a.shape[0], _ptr(a), _ptr(out))
    return out

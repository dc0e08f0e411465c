"""Thin Python binding of the C ABI in ``include/gecc.h`` (argument marshalling only).

Every function has the name of the C entry point it calls and takes the same
arguments; arrays may be torch tensors (CUDA or CPU) or numpy arrays (host), and
``stream`` may be a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or
``None`` for torch's current stream on the current device.  All computation
happens in ``libgecc.so``; there is no Python or CPU fallback: if the library is
missing, ``load()`` raises.
"""
import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgecc.so")

ECC_SECP256K1, ECC_P256, ECC_BN254, ECC_BLS12_381, ECC_SM2 = 0, 1, 2, 3, 4
CURVES = {"secp256k1": 0, "P-256": 1, "BN254": 2, "BLS12-381": 3}
ECC_FIELD_BASE, ECC_FIELD_SCALAR = 0, 1
ECC_OK, ECC_EINVAL, ECC_EUNSUPPORTED, ECC_ENOMEM, ECC_ECUDA, ECC_ETIMEOUT = 0, -1, -2, -3, -4, -5

_lock = threading.Lock()
_lib = None


class EccError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_SIGS = {
    "ecc_last_error": (ctypes.c_char_p, []),
    "ecc_version": (ctypes.c_char_p, []),
    "ecc_limbs": (ctypes.c_int, [ctypes.c_int]),
    "ecc_fp_mul": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 4),
    "ecc_fp_add": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 4),
    "ecc_fp_sub": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 4),
    "ecc_fp_inv": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 3),
    "ecc_fp_inv_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 3),
    "ecc_fp_inv_batch_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t] +
                                 [ctypes.c_void_p] * 3),
    "ecc_point_add_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 4),
    "ecc_point_dbl_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 3),
    "ecc_point_op_custom": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t] +
                            [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]),
    "ecc_verify_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 6),
    "ecc_fixed_base_mul": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 3),
    "ecc_sign_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 7),
    "ecc_msm": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 4),
    "ecc_msm_ragged": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 5),
    "ecc_bases_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 3),
    "ecc_msm_bases": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t] + [ctypes.c_void_p] * 3),
    "ecc_msm_bases_ragged": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t] + [ctypes.c_void_p] * 4),
    "ecc_bases_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ecc_msm_window": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t]),
    "ecc_msm_set_window": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "ecc_msm_reduce_chunk": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t]),
    "ecc_set_phase_timing": (ctypes.c_int, [ctypes.c_int]),
    "ecc_set_gas_cluster": (ctypes.c_int, [ctypes.c_int]),
    "ecc_msm_ragged_dev": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t] +
                           [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_void_p]),
    "ecc_msm_bases_ragged_dev": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t] +
                                 [ctypes.c_void_p] * 4),
    "ecc_sync_status": (ctypes.c_int, [ctypes.c_void_p]),
    "ecc_set_allocator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ecc_validate_points": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t] + [ctypes.c_void_p] * 3),
    "ecc_msm_phase_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ecc_msm_set_reduce_chunk": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "ecc_bench_imad": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "ecc_bench_inv": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "ecc_bases_precompute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "ecc_bases_window": (ctypes.c_int, [ctypes.c_void_p]),
    "ecc_bench_modmul": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]),
}


def load():
    """Loads libgecc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() first")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                if hasattr(lib, name):
                    fn = getattr(lib, name)
                    fn.restype = res
                    fn.argtypes = args
            _lib = lib
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):  # numpy array
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is None:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc):
    if rc != ECC_OK:
        msg = load().ecc_last_error().decode(errors="replace")
        raise EccError(rc, msg)
    return rc


def ecc_last_error():
    return load().ecc_last_error().decode(errors="replace")


def ecc_version():
    return load().ecc_version().decode()


def ecc_limbs(curve):
    rc = load().ecc_limbs(curve)
    if rc < 0:
        _check(rc)
    return rc


def ecc_fp_mul(curve, field, n, a, b, out, stream=None):
    return _check(load().ecc_fp_mul(curve, field, n, _ptr(a), _ptr(b), _ptr(out), _stream(stream)))


def ecc_fp_add(curve, field, n, a, b, out, stream=None):
    return _check(load().ecc_fp_add(curve, field, n, _ptr(a), _ptr(b), _ptr(out), _stream(stream)))


def ecc_fp_sub(curve, field, n, a, b, out, stream=None):
    return _check(load().ecc_fp_sub(curve, field, n, _ptr(a), _ptr(b), _ptr(out), _stream(stream)))


def ecc_fp_inv(curve, field, n, a, out, stream=None):
    return _check(load().ecc_fp_inv(curve, field, n, _ptr(a), _ptr(out), _stream(stream)))


def ecc_fp_inv_batch(curve, field, n, a, out, stream=None):
    return _check(load().ecc_fp_inv_batch(curve, field, n, _ptr(a), _ptr(out), _stream(stream)))


def ecc_fp_inv_batch_noalloc(curve, field, n, a, out, stream=None):
    """Allocation-free batch inversion (device buffers only, n <= 65536)."""
    return _check(load().ecc_fp_inv_batch_noalloc(curve, field, n, _ptr(a), _ptr(out),
                                                  _stream(stream)))


def ecc_point_add_batch(curve, n, p, q, out, stream=None):
    return _check(load().ecc_point_add_batch(curve, n, _ptr(p), _ptr(q), _ptr(out), _stream(stream)))


def ecc_point_dbl_batch(curve, n, p, out, stream=None):
    return _check(load().ecc_point_dbl_batch(curve, n, _ptr(p), _ptr(out), _stream(stream)))


def ecc_point_op_custom(prime, a, n, p, q, out, dbl=0, stream=None):
    """prime, a: Python ints (converted to 8 host limbs each)."""
    import numpy as np

    def limbs(v):
        return np.array([(v >> (32 * i)) & 0xFFFFFFFF for i in range(8)], dtype=np.uint32)

    pl, al = limbs(prime), limbs(a)
    return _check(load().ecc_point_op_custom(pl.ctypes.data, al.ctypes.data, n, _ptr(p), _ptr(q),
                                             _ptr(out), int(dbl), _stream(stream)))


def ecc_verify_batch(curve, n, hash, r, s, pubkey, ok_out, stream=None):
    return _check(load().ecc_verify_batch(curve, n, _ptr(hash), _ptr(r), _ptr(s), _ptr(pubkey),
                                          _ptr(ok_out), _stream(stream)))


def ecc_fixed_base_mul(curve, n, k, out, stream=None):
    return _check(load().ecc_fixed_base_mul(curve, n, _ptr(k), _ptr(out), _stream(stream)))


def ecc_sign_batch(curve, n, d, e, k, r_out, s_out, pub_out, stream=None):
    return _check(load().ecc_sign_batch(curve, n, _ptr(d), _ptr(e), _ptr(k), _ptr(r_out),
                                        _ptr(s_out), _ptr(pub_out), _stream(stream)))


def ecc_msm(curve, n, points, scalars, out, stream=None):
    return _check(load().ecc_msm(curve, n, _ptr(points), _ptr(scalars), _ptr(out), _stream(stream)))


def ecc_msm_ragged(curve, num, offsets, points, scalars, out, stream=None):
    """offsets: host array (numpy uint64 or list) of num + 1 row indices."""
    import numpy as np

    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    return _check(load().ecc_msm_ragged(curve, num, offs.ctypes.data, _ptr(points), _ptr(scalars),
                                        _ptr(out), _stream(stream)))


def ecc_bases_create(curve, n, points, stream=None):
    """Returns the opaque handle (an int)."""
    h = ctypes.c_void_p()
    _check(load().ecc_bases_create(curve, n, _ptr(points), ctypes.addressof(h), _stream(stream)))
    return h.value


def ecc_msm_bases(handle, num_vectors, scalars, out, stream=None):
    return _check(load().ecc_msm_bases(handle, num_vectors, _ptr(scalars), _ptr(out), _stream(stream)))


def ecc_msm_bases_ragged(handle, num, sizes, scalars, out, stream=None):
    """sizes: host array (numpy uint64 or list) of num instance sizes."""
    import numpy as np

    sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.uint64))
    return _check(load().ecc_msm_bases_ragged(handle, num, sz.ctypes.data, _ptr(scalars), _ptr(out),
                                              _stream(stream)))


def ecc_bases_destroy(handle):
    return _check(load().ecc_bases_destroy(handle))


def ecc_bases_precompute(handle, c, stream=None):
    return _check(load().ecc_bases_precompute(handle, c, _stream(stream)))


def ecc_bases_window(handle):
    rc = load().ecc_bases_window(handle)
    if rc < 0:
        _check(rc)
    return rc


def ecc_msm_window(curve, n):
    rc = load().ecc_msm_window(curve, n)
    if rc < 0:
        _check(rc)
    return rc


def ecc_msm_set_window(curve, log2_n, c):
    return _check(load().ecc_msm_set_window(curve, log2_n, c))


def ecc_msm_reduce_chunk(curve, n):
    rc = load().ecc_msm_reduce_chunk(curve, n)
    if rc < 0:
        _check(rc)
    return rc


def ecc_msm_set_reduce_chunk(curve, log2_n, log2_chunk):
    return _check(load().ecc_msm_set_reduce_chunk(curve, log2_n, log2_chunk))


def ecc_msm_ragged_dev(curve, num, max_points, offsets, points, scalars, out, c=0, stream=None):
    """offsets: device tensor of num + 1 uint64 row indices (offsets[0] = 0)."""
    return _check(load().ecc_msm_ragged_dev(curve, num, max_points, _ptr(offsets), _ptr(points),
                                            _ptr(scalars), _ptr(out), c, _stream(stream)))


def ecc_msm_bases_ragged_dev(handle, num, max_points, sizes, scalars, out, stream=None):
    """sizes: device tensor of num uint64 instance sizes."""
    return _check(load().ecc_msm_bases_ragged_dev(handle, num, max_points, _ptr(sizes), _ptr(scalars),
                                                  _ptr(out), _stream(stream)))


def ecc_sync_status(stream=None):
    """Synchronises the stream and raises EccError if a kernel recorded an error."""
    return _check(load().ecc_sync_status(_stream(stream)))


# ctypes prototypes of the allocator hook (kept referenced while installed)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_hooks = []


def ecc_set_allocator(alloc=None, release=None):
    """Installs Python callables alloc(bytes, stream) -> int pointer and
    release(ptr, stream) as the workspace allocator (None, None: default)."""
    if alloc is None:
        rc = _check(load().ecc_set_allocator(None, None, None))
        _hooks.clear()
        return rc
    fa = ALLOC_FN(lambda b, s, ctx: alloc(b, s or 0) or None)
    fr = FREE_FN(lambda p, s, ctx: release(p, s or 0))
    rc = _check(load().ecc_set_allocator(ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(fr, ctypes.c_void_p),
                                         None))
    _hooks[:] = [fa, fr]
    return rc


def ecc_validate_points(curve, n, points, ok_out, stream=None):
    return _check(load().ecc_validate_points(curve, n, _ptr(points), _ptr(ok_out), _stream(stream)))


MSM_PHASES = ("sort", "accumulate", "fold", "reduce", "combine")


def ecc_set_gas_cluster(ctas):
    return _check(load().ecc_set_gas_cluster(int(ctas)))


def ecc_set_phase_timing(on):
    return _check(load().ecc_set_phase_timing(int(bool(on))))


def ecc_msm_phase_times():
    """{phase name: device ms} of this thread's last timed MSM call."""
    buf = (ctypes.c_float * len(MSM_PHASES))()
    k = load().ecc_msm_phase_times(ctypes.addressof(buf), len(MSM_PHASES))
    if k < 0:
        _check(k)
    return {MSM_PHASES[i]: float(buf[i]) for i in range(k)}


def ecc_bench_imad(threads, iters, sink, stream=None):
    return _check(load().ecc_bench_imad(threads, iters, _ptr(sink), _stream(stream)))


def ecc_bench_modmul(curve, reduction, threads, iters, sink, stream=None):
    return _check(load().ecc_bench_modmul(curve, reduction, threads, iters, _ptr(sink), _stream(stream)))


def ecc_bench_inv(curve, method, threads, iters, sink, stream=None):
    return _check(load().ecc_bench_inv(curve, method, threads, iters, _ptr(sink), _stream(stream)))

"""ctypes front of the C oracle (sv_oracle.c).  TEST INFRASTRUCTURE ONLY.

build() compiles sv_oracle.c with gcc (-O2, OpenMP, portable flags: no -march) into
oracle/_build/; load() builds on first use when the shared object is missing or older
than the source.
"""
import ctypes
import os
import subprocess

import numpy as np

from .circuit import KIND_CODE

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'sv_oracle.c')
_OUT_DIR = os.path.join(_HERE, '_build')
_LIB = os.path.join(_OUT_DIR, 'libsv_oracle.so')
_lib = None


def build(force=False):
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + '.tmp%d' % os.getpid()
    subprocess.check_call(['gcc', '-O2', '-std=c11', '-D_DEFAULT_SOURCE', '-fopenmp',
                           '-fPIC', '-shared', _SRC, '-o', tmp, '-lm'])
    os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_size_t, u8p, u8p, u8p,
                                   ctypes.c_int, dp]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_branch_amplitudes.argtypes = [
            ctypes.c_int, ctypes.c_size_t, u8p, u8p, u8p, ctypes.c_uint64, ctypes.c_size_t,
            ctypes.POINTER(ctypes.c_uint64), dp]
        lib.oracle_branch_amplitudes.restype = ctypes.c_int
        lib.oracle_reductions.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.oracle_reductions.restype = None
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        _lib = lib
    return _lib


def _arrays(gates):
    k = np.array([KIND_CODE[g[0]] for g in gates], dtype=np.uint8)
    a = np.array([g[1] for g in gates], dtype=np.uint8)
    b = np.array([max(g[2], 0) for g in gates], dtype=np.uint8)
    return k, a, b


def _u8(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _dp(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads():
    return load().oracle_threads()


def set_threads(t):
    load().oracle_set_threads(int(t))


def run(n, gates, psi=None, adjoint=False):
    """complex128 state after the gate list (or its inverse), default start |0..0>."""
    lib = load()
    if psi is None:
        buf = np.zeros(2 << n, dtype=np.float64)
        buf[0] = 1.0
    else:
        buf = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128)).view(np.float64).copy()
    k, a, b = _arrays(gates)
    rc = lib.oracle_run(n, len(gates), _u8(k), _u8(a), _u8(b), int(bool(adjoint)), _dp(buf))
    if rc != 0:
        raise ValueError('oracle_run failed: %d' % rc)
    return buf.view(np.complex128)


def branch_amplitudes(n, gates, half_a_mask, bitstrings):
    lib = load()
    k, a, b = _arrays(gates)
    bits = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint64))
    out = np.zeros(2 * bits.size, dtype=np.float64)
    rc = lib.oracle_branch_amplitudes(n, len(gates), _u8(k), _u8(a), _u8(b),
                                      ctypes.c_uint64(half_a_mask), bits.size,
                                      bits.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      _dp(out))
    if rc != 0:
        raise ValueError('oracle_branch_amplitudes failed: %d' % rc)
    return out.view(np.complex128)


def reductions(psi):
    """(sum |alpha|^2, sum |alpha|^4) in fp64."""
    lib = load()
    buf = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128)).view(np.float64)
    n = (buf.size // 2).bit_length() - 1
    s2 = ctypes.c_double()
    s4 = ctypes.c_double()
    lib.oracle_reductions(n, _dp(buf), ctypes.byref(s2), ctypes.byref(s4))
    return s2.value, s4.value

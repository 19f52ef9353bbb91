"""ctypes binding of the C interface in include/sv.h.

Argument marshalling only: every step of the simulation runs in the CUDA library.  The
functions keep the C names; they raise SvError on a non-zero status.  There is no CPU
fallback: if the shared library cannot be built or loaded, importing it fails loudly.
"""
import ctypes
import os

import numpy as np

from . import build as _build

c_int, c_uint8, c_uint32, c_uint64, c_size_t, c_double, c_void_p = (
    ctypes.c_int, ctypes.c_uint8, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t,
    ctypes.c_double, ctypes.c_void_p)

SV_OK, SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA, SV_ERR_TIMEOUT, SV_ERR_STATE = range(6)
SV_H, SV_T, SV_SX, SV_SY, SV_CZ, SV_P0, SV_P1, SV_Z, SV_TDG, SV_SXDG, SV_SYDG = range(11)
SV_PREC_PLAIN, SV_PREC_TF32X3, SV_PREC_F16X3, SV_PREC_PERGATE = 0, 1, 2, 3

GATE_DTYPE = np.dtype([('kind', 'u1'), ('q0', 'u1'), ('q1', 'u1'), ('pad', 'u1'), ('layer', '<u4')])


class SvError(RuntimeError):
    def __init__(self, status, message):
        super().__init__('sv status %d: %s' % (status, message))
        self.status = status


class sv_options(ctypes.Structure):
    _fields_ = [('fuse_k', c_int), ('precision', c_int), ('autotune', c_int), ('stream', c_void_p),
                ('tile_bits', c_int), ('low_bits', c_int), ('jit', c_int), ('pipeline', c_int),
                ('norm_restore', c_int)]


class sv_lattice(ctypes.Structure):
    _fields_ = [('rows', c_int), ('cols', c_int), ('removed_mask', c_uint64), ('depth', c_int),
                ('seed', c_uint64)]


class sv_cut(ctypes.Structure):
    _fields_ = [('half_a_mask', c_uint64), ('full_decomposition', c_int), ('depth', c_int)]


class sv_plan_summary(ctypes.Structure):
    _fields_ = [('passes', c_int), ('stages', c_int), ('ops', c_int), ('init_uniform', c_int),
                ('hbm_bytes', c_double), ('matrix_stages', c_int)]


class sv_profile(ctypes.Structure):
    _fields_ = [('launches', c_int), ('ms', c_double), ('hbm_bytes', c_double), ('h2d_bytes', c_double),
                ('d2h_bytes', c_double), ('other_launches', c_int), ('jit_launches', c_int),
                ('plain_fallbacks', c_int), ('plan_tile_bits', c_int), ('plan_stage_qubits', c_int),
                ('plan_passes', c_int)]


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = c_void_p
    sig = {
        'sv_last_error': ([], ctypes.c_char_p),
        'sv_create': ([c_int, P(sv_options), P(vp)], c_int),
        'sv_create_from_ptr': ([c_int, vp, vp, P(vp)], c_int),
        'sv_destroy': ([vp], c_int),
        'sv_set_options': ([vp, P(sv_options)], c_int),
        'sv_copy_state': ([vp, vp], c_int),
        'sv_load_state': ([vp, vp], c_int),
        'sv_device_ptr': ([vp, P(vp)], c_int),
        'sv_reset': ([vp], c_int),
        'sv_generate_circuit': ([P(sv_lattice), vp, c_size_t, P(c_size_t)], c_int),
        'sv_apply_circuit': ([vp, vp, c_size_t], c_int),
        'sv_apply_circuit_inverse': ([vp, vp, c_size_t], c_int),
        'sv_get_amplitudes': ([vp, vp, c_size_t, vp], c_int),
        'sv_get_probabilities': ([vp, vp, c_size_t, vp], c_int),
        'sv_norm': ([vp, P(c_double), P(c_double)], c_int),
        'sv_branch_amplitudes': ([P(sv_lattice), P(sv_cut), vp, c_size_t, P(sv_options), vp], c_int),
        'sv_branch_counts': ([P(sv_lattice), P(sv_cut), vp], c_int),
        'sv_branch_full_state': ([P(sv_lattice), P(sv_cut), P(sv_options), vp], c_int),
        'sv_apply_batch': ([vp, c_size_t, P(sv_options), vp], c_int),
        'sv_batch_amplitudes': ([c_size_t, vp, c_size_t, vp], c_int),
        'sv_batch_free': ([], c_int),
        'sv_batch_config': ([P(c_int), P(c_int), P(c_int)], c_int),
        'sv_selftest_wait_timeout': ([c_int], c_int),
        'sv_norm_noalloc': ([vp, c_int, vp, P(c_double), P(c_double)], c_int),
        'sv_plan': ([c_int, vp, c_size_t, P(sv_options), c_int, P(sv_plan_summary), vp, vp, vp,
                     c_size_t], c_int),
        'sv_jit_check': ([c_int, vp, c_size_t, P(sv_options), c_int, ctypes.c_char_p, c_size_t], c_int),
        'sv_set_basis_state': ([vp, c_uint64], c_int),
        'sv_inner_product': ([vp, vp, vp], c_int),
        'sv_amplitudes_by_inner_product': ([P(sv_lattice), c_int, vp, c_size_t, P(sv_options), vp], c_int),
        'sv_set_profiling': ([vp, c_int], c_int),
        'sv_get_profile': ([vp, P(sv_profile)], c_int),
        'sv_get_launch_times': ([vp, vp, vp, c_size_t, P(c_size_t)], c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status):
    if status != SV_OK:
        raise SvError(status, lib().sv_last_error().decode())


def options(precision=SV_PREC_PLAIN, fuse_k=0, tile_bits=0, low_bits=0, stream=None, autotune=0, jit=0,
            pipeline=0, norm_restore=0):
    return sv_options(fuse_k, precision, autotune, stream, tile_bits, low_bits, jit, pipeline, norm_restore)


def lattice(lat):
    """An inputs.Lattice (or any object with rows/cols/removed_mask/depth/seed) -> sv_lattice."""
    return sv_lattice(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)


def _gates(gates):
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    return g, g.ctypes.data, g.size


def gates_from_tuples(tuples):
    """[(kind_code, q0, q1, layer), ...] -> gate array."""
    g = np.zeros(len(tuples), dtype=GATE_DTYPE)
    for i, (k, a, b, l) in enumerate(tuples):
        g[i] = (k, a, b, 0, l)
    return g


# --- state lifetime ----------------------------------------------------------------

def sv_create(n_qubits, opts=None):
    h = c_void_p()
    _check(lib().sv_create(n_qubits, ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
    return h


def sv_create_from_ptr(n_qubits, dev_ptr, stream=None):
    h = c_void_p()
    _check(lib().sv_create_from_ptr(n_qubits, c_void_p(dev_ptr), c_void_p(stream), ctypes.byref(h)))
    return h


def sv_destroy(h):
    _check(lib().sv_destroy(h))


def sv_set_options(h, opts):
    _check(lib().sv_set_options(h, ctypes.byref(opts)))


def sv_copy_state(h, n_qubits, dst=None):
    """Copy the amplitudes to a new host complex64 array (or to dst: a host numpy array
    or an integer device pointer)."""
    if dst is None:
        out = np.empty(1 << n_qubits, dtype=np.complex64)
        _check(lib().sv_copy_state(h, out.ctypes.data))
        return out
    ptr = dst if isinstance(dst, int) else dst.ctypes.data
    _check(lib().sv_copy_state(h, c_void_p(ptr)))
    return dst


def sv_load_state(h, src):
    """src: a device or host address (int), or an array converted to complex64 (kept
    alive until the copy is done)."""
    keep = src if isinstance(src, int) else np.ascontiguousarray(src, dtype=np.complex64)
    ptr = keep if isinstance(keep, int) else keep.ctypes.data
    _check(lib().sv_load_state(h, c_void_p(ptr)))
    del keep


def sv_reset(h):
    _check(lib().sv_reset(h))


def sv_device_ptr(h):
    p = c_void_p()
    _check(lib().sv_device_ptr(h, ctypes.byref(p)))
    return p.value


# --- circuits ---------------------------------------------------------------------

def sv_generate_circuit(lat):
    L = lat if isinstance(lat, sv_lattice) else lattice(lat)
    n = c_size_t()
    _check(lib().sv_generate_circuit(ctypes.byref(L), None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=GATE_DTYPE)
    _check(lib().sv_generate_circuit(ctypes.byref(L), out.ctypes.data, out.size, ctypes.byref(n)))
    return out


def sv_apply_circuit(h, gates):
    g, p, n = _gates(gates)
    _check(lib().sv_apply_circuit(h, p, n))


def sv_apply_circuit_inverse(h, gates):
    g, p, n = _gates(gates)
    _check(lib().sv_apply_circuit_inverse(h, p, n))


def sv_get_amplitudes(h, bits):
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    out = np.zeros(2 * b.size, dtype=np.float64)
    _check(lib().sv_get_amplitudes(h, b.ctypes.data, b.size, out.ctypes.data))
    return out.view(np.complex128)


def sv_get_probabilities(h, bits):
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    out = np.zeros(b.size, dtype=np.float64)
    _check(lib().sv_get_probabilities(h, b.ctypes.data, b.size, out.ctypes.data))
    return out


def sv_norm(h):
    a, b = c_double(), c_double()
    _check(lib().sv_norm(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sv_branch_amplitudes(lat, half_a_mask, bits, opts=None, full_decomposition=False):
    L = lat if isinstance(lat, sv_lattice) else lattice(lat)
    cut = sv_cut(half_a_mask, int(bool(full_decomposition)), 0)
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    out = np.zeros(2 * b.size, dtype=np.float64)
    _check(lib().sv_branch_amplitudes(ctypes.byref(L), ctypes.byref(cut), b.ctypes.data, b.size,
                                      ctypes.byref(opts) if opts is not None else None, out.ctypes.data))
    return out.view(np.complex128)


def sv_branch_full_state(lat, half_a_mask, h, opts=None, full_decomposition=False, depth=0):
    """Write sum_l A_l (x) B_l (the full state) into handle h; depth > 0: the halves take
    layers 0..depth and the remaining layers (part C) run on the result."""
    L = lat if isinstance(lat, sv_lattice) else lattice(lat)
    cut = sv_cut(half_a_mask, int(bool(full_decomposition)), int(depth))
    _check(lib().sv_branch_full_state(ctypes.byref(L), ctypes.byref(cut),
                                      ctypes.byref(opts) if opts is not None else None, h))


def sv_branch_counts(lat, half_a_mask, full_decomposition=False):
    """(crossing CZs, absorbed signs, branch bits of A, of B, summed branch bits)."""
    L = lat if isinstance(lat, sv_lattice) else lattice(lat)
    cut = sv_cut(half_a_mask, int(bool(full_decomposition)), 0)
    out = np.zeros(5, dtype=np.int32)
    _check(lib().sv_branch_counts(ctypes.byref(L), ctypes.byref(cut), out.ctypes.data))
    return tuple(int(v) for v in out)


def sv_apply_batch(lats, opts=None, stats=True):
    """Run the batch; per-circuit [sum p, sum p^2, n] rows, or None with stats=False (the
    reduction is then skipped)."""
    arr = (sv_lattice * len(lats))(*[x if isinstance(x, sv_lattice) else lattice(x) for x in lats])
    out = np.zeros(3 * len(lats), dtype=np.float64) if stats else None
    _check(lib().sv_apply_batch(ctypes.cast(arr, c_void_p), len(lats),
                                ctypes.byref(opts) if opts is not None else None,
                                out.ctypes.data if stats else None))
    return out.reshape(len(lats), 3) if stats else None


def sv_batch_amplitudes(circuit, bits):
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    out = np.zeros(2 * b.size, dtype=np.float64)
    _check(lib().sv_batch_amplitudes(circuit, b.ctypes.data, b.size, out.ctypes.data))
    return out.view(np.complex128)


def sv_selftest_wait_timeout(limit_ms):
    """Raw status of the bounded-wait self-test (SV_ERR_TIMEOUT expected)."""
    return lib().sv_selftest_wait_timeout(int(limit_ms))


def sv_batch_config():
    """(tile_bits, circuits on plan-specialised kernels, circuits in the persistent launch)
    of the last batch."""
    v = [c_int(), c_int(), c_int()]
    _check(lib().sv_batch_config(ctypes.byref(v[0]), ctypes.byref(v[1]), ctypes.byref(v[2])))
    return tuple(x.value for x in v)


def sv_batch_free():
    _check(lib().sv_batch_free())


def sv_norm_noalloc(dev_ptr, n_qubits, stream=None):
    a, b = c_double(), c_double()
    _check(lib().sv_norm_noalloc(c_void_p(dev_ptr), n_qubits, c_void_p(stream), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sv_plan(n_qubits, gates, opts=None, fresh_state=True):
    """Host-only planning: (summary, execution order, pass of each executed gate, tiles)."""
    g, p, n = _gates(gates)
    summ = sv_plan_summary()
    _check(lib().sv_plan(n_qubits, p, n, ctypes.byref(opts) if opts is not None else None,
                         int(bool(fresh_state)), ctypes.byref(summ), None, None, None, 0))
    order = np.zeros(max(n, 1), dtype=np.int32)
    pass_of = np.zeros(max(n, 1), dtype=np.int32)
    tiles = np.zeros(64 * max(summ.passes, 1), dtype=np.int32)
    _check(lib().sv_plan(n_qubits, p, n, ctypes.byref(opts) if opts is not None else None,
                         int(bool(fresh_state)), ctypes.byref(summ), order.ctypes.data,
                         pass_of.ctypes.data, tiles.ctypes.data, tiles.size))
    return summ, order[:n], pass_of[:n], tiles.reshape(-1, 64)[:summ.passes]


def sv_set_basis_state(h, x):
    _check(lib().sv_set_basis_state(h, int(x)))


def sv_inner_product(a, b):
    """<a|b> (complex)."""
    out = np.zeros(2, dtype=np.float64)
    _check(lib().sv_inner_product(a, b, out.ctypes.data))
    return complex(out[0], out[1])


def sv_amplitudes_by_inner_product(lat, split_layer, bitstrings, opts=None):
    """Amplitudes alpha_x = <U2^dagger x | U1 H^n 0> of a lattice circuit cut after split_layer."""
    bits = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    out = np.zeros(2 * bits.size, dtype=np.float64)
    L = lattice(lat)
    _check(lib().sv_amplitudes_by_inner_product(ctypes.byref(L), int(split_layer), bits.ctypes.data, bits.size,
                                                ctypes.byref(opts) if opts is not None else None,
                                                out.ctypes.data))
    return out[0::2] + 1j * out[1::2]


def sv_jit_check(n_qubits, gates, opts=None, fresh_state=True):
    """Compile the plan-specialised kernels of a gate list for sm_103a (NVRTC, no device).
    Returns the compiler log; raises SvError if the compile fails."""
    g, p, n = _gates(gates)
    buf = ctypes.create_string_buffer(1 << 16)
    st = lib().sv_jit_check(n_qubits, p, n, ctypes.byref(opts) if opts is not None else None,
                            int(bool(fresh_state)), buf, len(buf))
    if st != SV_OK:
        raise SvError(st, lib().sv_last_error().decode() + '\n' + buf.value.decode(errors='replace'))
    return buf.value.decode(errors='replace')


def sv_set_profiling(h, on):
    _check(lib().sv_set_profiling(h, int(bool(on))))


def sv_get_profile(h):
    p = sv_profile()
    _check(lib().sv_get_profile(h, ctypes.byref(p)))
    return p


def sv_get_launch_times(h):
    """(ms, bytes) numpy arrays, one entry per timed launch since profiling was turned on."""
    n = c_size_t()
    _check(lib().sv_get_launch_times(h, None, None, 0, ctypes.byref(n)))
    ms = np.zeros(n.value, dtype=np.float64)
    by = np.zeros(n.value, dtype=np.float64)
    _check(lib().sv_get_launch_times(h, ms.ctypes.data, by.ctypes.data, n.value, ctypes.byref(n)))
    return ms, by

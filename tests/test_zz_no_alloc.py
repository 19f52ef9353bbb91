"""sv_norm_noalloc: the allocation-free norm for callers that cannot allocate device
memory (a framework's allocator owns the GPU budget, or device-wide syncs from
cudaMalloc/cudaFree are not allowed).  It is checked through the C interface against
sv_norm, which allocates its scratch on the handle, on two calls in a row (the shared
static scratch keeps the previous call's contents).  Collected last on purpose."""
import ctypes

import pytest

from paper_1804_04797_gb300 import inputs
from paper_1804_04797_gb300 import sv

pytestmark = pytest.mark.gpu

NORM_TOL = 1e-6


def _noalloc(dev_ptr, n, stream=None):
    L = sv.lib()
    f = L.sv_norm_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    a, b = ctypes.c_double(), ctypes.c_double()
    st = f(ctypes.c_void_p(dev_ptr), n, ctypes.c_void_p(stream), ctypes.byref(a), ctypes.byref(b))
    if st != 0:
        raise sv.SvError(st, L.sv_last_error().decode())
    return a.value, b.value


@pytest.mark.parametrize('lat', [inputs.lattice_for(4, 5, 14, seed=5), inputs.lattice_for(2, 3, 6, seed=1)],
                         ids=['20q', '6q'])
def test_noalloc_norm_matches_sv_norm_twice(lat):
    n = lat.n_qubits
    h = sv.sv_create(n)
    try:
        sv.sv_apply_circuit(h, sv.sv_generate_circuit(lat))
        want2, want4 = sv.sv_norm(h)
        ptr = sv.sv_device_ptr(h)
        first = _noalloc(ptr, n)
        second = _noalloc(ptr, n)
    finally:
        sv.sv_destroy(h)
    for got2, got4 in (first, second):
        assert abs(got2 - want2) <= NORM_TOL
        assert abs(got2 - 1.0) <= NORM_TOL
        assert abs(got4 - want4) <= NORM_TOL * want4
    assert first == second


def test_noalloc_rejects_sizes_beyond_the_maximum():
    with pytest.raises(sv.SvError):
        _noalloc(16, 35)
    with pytest.raises(sv.SvError):
        _noalloc(16, 0)
    with pytest.raises(sv.SvError):
        _noalloc(0, 10)


def test_noalloc_rejects_misaligned_pointers_before_any_launch():
    # the reduction reads 16-byte vectors (n >= 2) or 8-byte amplitudes (n = 1); the
    # check runs on the host before any CUDA call, so these pointers are never touched
    with pytest.raises(sv.SvError, match='aligned'):
        _noalloc(8, 10)
    with pytest.raises(sv.SvError, match='aligned'):
        _noalloc(4, 1)


@pytest.mark.parametrize('gates', [[], [(sv.SV_H, 0)]], ids=['basis', 'uniform'])
def test_noalloc_one_qubit_state(gates):
    # n = 1 takes the single-thread reduction of 8-byte amplitudes
    h = sv.sv_create(1)
    try:
        g = sv.gates_from_tuples([(k, q, 0, 0) for k, q in gates])
        sv.sv_apply_circuit(h, g)
        want2, want4 = sv.sv_norm(h)
        ptr = sv.sv_device_ptr(h)
        got = [_noalloc(ptr, 1), _noalloc(ptr, 1)]
    finally:
        sv.sv_destroy(h)
    for got2, got4 in got:
        assert abs(got2 - want2) <= NORM_TOL
        assert abs(got4 - want4) <= NORM_TOL * want4
    assert got[0] == got[1]


def test_noalloc_on_a_caller_stream_matches_the_default_stream():
    import torch
    lat = inputs.lattice_for(4, 4, 10, seed=3)
    n = lat.n_qubits
    h = sv.sv_create(n)
    try:
        sv.sv_apply_circuit(h, sv.sv_generate_circuit(lat))
        ptr = sv.sv_device_ptr(h)
        torch.cuda.synchronize()
        st = torch.cuda.Stream()
        on_stream = _noalloc(ptr, n, st.cuda_stream)
        on_default = _noalloc(ptr, n)
    finally:
        sv.sv_destroy(h)
    assert on_stream == on_default
    assert abs(on_stream[0] - 1.0) <= NORM_TOL

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

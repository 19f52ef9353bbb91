"""Property tests of the planner (host only): for random gate lists of every kind the
oracle supports (projectors included), random tile shapes and both starting conditions,
the execution order the planner returns is a valid reordering of the list -- the
oracle, replaying the gates in that order, reaches the state of the original order --
and every gate runs exactly once.  The plans are those sv_apply_circuit builds for the
same options."""
import numpy as np
import pytest

from oracle import circuit as oc
from oracle import statevec as ov
from paper_1804_04797_gb300 import sv

hypothesis = pytest.importorskip('hypothesis')
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

KINDS = ['H', 'T', 'SX', 'SY', 'CZ', 'Z', 'P0', 'P1']
OPTIONS = [dict(), dict(tile_bits=6, low_bits=1, fuse_k=2), dict(tile_bits=7, low_bits=2, fuse_k=3),
           dict(tile_bits=8, low_bits=3, fuse_k=4), dict(tile_bits=9, low_bits=4, fuse_k=5), dict(jit=1),
           dict(jit=1, tile_bits=7, low_bits=2), dict(precision=sv.SV_PREC_TF32X3)]


@st.composite
def plans(draw):
    n = draw(st.integers(6, 11))
    gates = []
    for _ in range(draw(st.integers(0, 50))):
        k = draw(st.sampled_from(KINDS))
        a = draw(st.integers(0, n - 1))
        b = -1
        if k == 'CZ':
            b = draw(st.integers(0, n - 2))
            b = b + 1 if b >= a else b
        gates.append((k, a, b, 1))
    if draw(st.booleans()):  # a leading H layer, as in the lattice circuits
        gates = [('H', q, -1, 0) for q in range(n)] + gates
    return n, gates, draw(st.sampled_from(OPTIONS)), draw(st.booleans())


@settings(max_examples=150, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(plans())
def test_execution_order_is_a_valid_reordering(case):
    n, gates, kw, fresh = case
    lib_gates = sv.gates_from_tuples([(oc.KIND_CODE[k], a, max(b, 0), l) for (k, a, b, l) in gates])
    _summ, order, _pass_of, _tiles = sv.sv_plan(n, lib_gates, sv.options(**kw), fresh_state=fresh)
    assert sorted(order.tolist()) == list(range(len(gates)))
    rng = np.random.default_rng(len(gates) * 131 + n)
    start = None if fresh else rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    want = ov.run(n, gates, start)
    got = ov.run(n, [gates[i] for i in order.tolist()], start)
    np.testing.assert_allclose(got, want, atol=1e-11 * max(1.0, float(np.abs(want).max())))

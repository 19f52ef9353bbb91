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


def _recount(gates, in_a):
    """Crossing CZs, those that only sign the output (neither qubit meets a later
    non-diagonal gate), and the implicit ones (one side quiet), from the gate list."""
    last_nd = {}
    for i, (k, q0, _q1, _l) in enumerate(gates):
        if k in ('H', 'SX', 'SY'):
            last_nd[q0] = i
    t = absorbed = full = impl_a = impl_b = 0
    for i, (k, q0, q1, _l) in enumerate(gates):
        if k != 'CZ' or in_a[q0] == in_a[q1]:
            continue
        t += 1
        qa, qb = (q0, q1) if in_a[q0] else (q1, q0)
        quiet_a, quiet_b = last_nd.get(qa, -1) < i, last_nd.get(qb, -1) < i
        if quiet_a and quiet_b:
            absorbed += 1
        elif quiet_a:
            impl_a += 1
        elif quiet_b:
            impl_b += 1
        else:
            full += 1
    return t, absorbed, full + impl_b, full + impl_a, full


@st.composite
def cuts(draw):
    rows = draw(st.integers(2, 5))
    cols = draw(st.integers(2, 6))
    depth = draw(st.integers(1, 16))
    seed = draw(st.integers(0, 2 ** 32))
    cut_row = draw(st.integers(1, rows - 1))
    return rows, cols, depth, seed, cut_row


@settings(max_examples=120, deadline=None)
@given(cuts())
def test_cut_plan_counts_match_a_recount(case):
    rows, cols, depth, seed, cut_row = case
    n, gates = oc.generate(rows, cols, 0, depth, seed)
    half_a = (1 << (cut_row * cols)) - 1  # rows 0..cut_row-1
    in_a = [bool((half_a >> q) & 1) for q in range(n)]
    lat = sv.sv_lattice(rows, cols, 0, depth, seed)
    n_a = cut_row * cols
    n_b = n - n_a
    t = _recount(gates, in_a)[0]
    for full, want in ((False, _recount(gates, in_a)), (True, (t, 0, t, t, t))):
        if n_a + want[2] > 34 or n_b + want[3] > 34:  # a half state beyond one GPU: refused
            with pytest.raises(sv.SvError):
                sv.sv_branch_counts(lat, half_a, full_decomposition=full)
        else:
            assert sv.sv_branch_counts(lat, half_a, full_decomposition=full) == want


@settings(max_examples=8, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(plans())
def test_generated_kernels_compile(case):
    """Every plan-specialised pass kernel of a random plan (and its last pass as the
    inner-product variant) compiles for sm_103a (NVRTC, no device)."""
    n, gates, kw, fresh = case
    kw = {k: v for k, v in kw.items() if k != 'precision'}  # the plain path's kernels
    lib_gates = sv.gates_from_tuples([(oc.KIND_CODE[k], a, max(b, 0), l) for (k, a, b, l) in gates])
    try:
        sv.sv_jit_check(n, lib_gates, sv.options(**kw), fresh_state=fresh)
    except sv.SvError as e:
        if 'libnvrtc' in str(e):
            pytest.skip('NVRTC not installed')
        raise

"""Host-side checks of the CUDA library (no GPU needed): the shared library loads and
exports every function declared in include/sv.h, the generator matches the oracle's
independent generator bit for bit, and the planner's execution order is a valid
reordering of the circuit (checked by running both orders through the CPU oracle)."""
import os
import re

import numpy as np
import pytest

from oracle import circuit as oc
from oracle import statevec as ov
from paper_1804_04797_gb300 import inputs
from paper_1804_04797_gb300 import sv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, 'include')):
        if fn.endswith('.h'):
            text = open(os.path.join(ROOT, 'include', fn)).read()
            text = re.sub(r'/\*.*?\*/', '', text, flags=re.S)
            names |= set(re.findall(r'\b(sv_[a-z0-9_]+)\s*\(', text))
    return names


def test_library_exports_every_declared_function():
    import ctypes
    L = ctypes.CDLL(sv.lib()._name)
    names = _declared_functions()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def _lib_gates(lat):
    g = sv.sv_generate_circuit(lat)
    out = []
    for x in g:
        k = oc.CODE_KIND[int(x['kind'])]
        out.append((k, int(x['q0']), int(x['q1']) if k == 'CZ' else -1, int(x['layer'])))
    return out


LATTICES = [inputs.C16, inputs.C30, inputs.C34, inputs.C42, inputs.C28,
            inputs.lattice_for(3, 5, 17, seed=99), inputs.lattice_for(1, 7, 9, seed=5),
            inputs.lattice_for(5, 5, 40, seed=12345, removed=[(2, 2), (0, 4)])]


@pytest.mark.parametrize('lat', LATTICES)
def test_generator_matches_oracle_generator(lat):
    n_o, g_o = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
    assert n_o == lat.n_qubits
    assert _lib_gates(lat) == g_o


def test_generator_batch_lattices():
    for lat in inputs.batch(64):
        n_o, g_o = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
        assert 16 <= n_o <= 24 and 10 <= lat.depth <= 24
        assert _lib_gates(lat) == g_o
    small = inputs.batch(64, n_min=12, n_max=16)
    assert {lat.n_qubits for lat in small} == set(range(12, 17))
    for lat in small[:16]:
        n_o, g_o = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
        assert n_o == lat.n_qubits and _lib_gates(lat) == g_o


def test_generator_rejects_bad_lattices():
    with pytest.raises(sv.SvError):
        sv.sv_generate_circuit(sv.sv_lattice(9, 8, 0, 3, 0))       # 72 sites
    with pytest.raises(sv.SvError):
        sv.sv_generate_circuit(sv.sv_lattice(2, 2, 0xF, 3, 0))     # every site removed


def _oracle_run_order(n, gates, order):
    return ov.run(n, [gates[i] for i in order])


PLAN_CASES = [(inputs.lattice_for(3, 4, 14, seed=3), dict()),
              (inputs.lattice_for(3, 4, 14, seed=3), dict(tile_bits=8, low_bits=2, fuse_k=3)),
              (inputs.lattice_for(4, 4, 12, seed=8), dict(tile_bits=10, low_bits=4, fuse_k=5)),
              (inputs.lattice_for(4, 4, 12, seed=8), dict(tile_bits=7, low_bits=1, fuse_k=2)),
              (inputs.lattice_for(2, 7, 20, seed=1), dict(tile_bits=9, low_bits=3, fuse_k=4)),
              (inputs.lattice_for(4, 4, 12, seed=8), dict(tile_bits=8, low_bits=4, fuse_k=5,
                                                          precision=sv.SV_PREC_TF32X3)),
              # the fused packed plan of the matrix-stage kernels (12-qubit TMA tiles)
              (inputs.lattice_for(4, 4, 12, seed=8), dict(precision=sv.SV_PREC_F16X3)),
              (inputs.lattice_for(2, 7, 20, seed=1), dict(precision=sv.SV_PREC_TF32X3)),
              # the plain pipelined kernels' plans (TMA tile layout; a T waits for the next
              # non-diagonal gate on its qubit)
              (inputs.lattice_for(4, 4, 12, seed=8), dict(jit=1)),
              (inputs.lattice_for(2, 7, 20, seed=1), dict(jit=1)),
              (inputs.lattice_for(3, 5, 16, seed=4), dict(jit=1, tile_bits=10))]


@pytest.mark.parametrize('lat,kw', PLAN_CASES)
def test_planner_order_is_a_valid_reordering(lat, kw):
    gates = _lib_gates(lat)
    n = lat.n_qubits
    g = sv.sv_generate_circuit(lat)
    summ, order, pass_of, tiles = sv.sv_plan(n, g, sv.options(**kw), fresh_state=True)
    assert sorted(order.tolist()) == list(range(len(gates)))
    assert summ.init_uniform == 1
    # every non-diagonal gate of a pass acts on a tile qubit of that pass
    for i, p in zip(order.tolist(), pass_of.tolist()):
        k, a, _b, _l = gates[i]
        if k in ('SX', 'SY', 'H') and gates[i][3] > 0:
            assert a in set(tiles[p][tiles[p] >= 0].tolist())
    want = ov.run(n, gates)
    got = _oracle_run_order(n, gates, order.tolist())
    np.testing.assert_allclose(got, want, atol=1e-12)


@pytest.mark.parametrize('kw', [dict(jit=1), dict(jit=1, tile_bits=10)])
def test_plain_plan_of_a_random_gate_list_is_a_valid_reordering(kw):
    """Random lists of the oracle's gate kinds (T before H, SX, SY or nothing on its qubit,
    Z and CZ signs, no leading H layer) on 14 qubits: the plain pipelined kernels' plans,
    where each T waits for the next non-diagonal gate on its qubit, run in their execution
    order give the oracle's state."""
    n = 14
    rng = np.random.default_rng(5)
    kinds = ['H', 'T', 'SX', 'SY', 'CZ', 'Z', 'T', 'T']
    gates = []
    for layer in range(220):
        k = kinds[rng.integers(len(kinds))]
        a = int(rng.integers(n))
        b = -1
        if k == 'CZ':
            b = int(rng.integers(n - 1))
            b = b + 1 if b >= a else b
        gates.append((k, a, b, layer))
    g = sv.gates_from_tuples([(oc.KIND_CODE[k], a, max(b, 0), l) for k, a, b, l in gates])
    summ, order, pass_of, tiles = sv.sv_plan(n, g, sv.options(**kw), fresh_state=True)
    assert sorted(order.tolist()) == list(range(len(gates)))
    assert summ.passes >= 2
    want = ov.run(n, gates)
    got = _oracle_run_order(n, gates, order.tolist())
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_planner_pass_counts_headline_workload():
    """The 34-qubit depth-30 circuit needs far fewer state sweeps than gates."""
    g = sv.sv_generate_circuit(inputs.C34)
    summ, *_ = sv.sv_plan(34, g, sv.options(), fresh_state=True)
    assert len(g) == 478
    assert summ.passes <= 12
    assert summ.hbm_bytes == pytest.approx(8.0 * 2 ** 34 + 16.0 * 2 ** 34 * (summ.passes - 1))


def test_plain_plan_applies_each_t_in_the_pass_of_the_next_gate_on_its_qubit():
    """Plans for the plain pipelined kernels: a T (or its adjoint) on a qubit of the tile
    goes to the pass of the next non-diagonal gate on its qubit (where the kernel applies
    both as one step); one on a qubit outside the tile stays a phase of the tile.  The
    execution order stays a valid reordering (the oracle run in that order matches)."""
    for lat in (inputs.C34, inputs.C30):
        n = lat.n_qubits
        gates = _lib_gates(lat)
        g = sv.sv_generate_circuit(lat)
        summ, order, pass_of, tiles = sv.sv_plan(n, g, sv.options(jit=1), fresh_state=True)
        where = dict(zip(order.tolist(), pass_of.tolist()))
        checked = 0
        for i, (k, a, _b, _l) in enumerate(gates):
            if k not in ('T', 'TDG'):
                continue
            succ = next((j for j in range(i + 1, len(gates))
                         if gates[j][0] in ('SX', 'SY', 'H', 'SXDG', 'SYDG') and gates[j][1] == a), None)
            if succ is None:
                continue
            p = where[i]
            assert where[succ] >= p
            if a in set(tiles[p][tiles[p] >= 0].tolist()):
                assert where[succ] == p, (i, succ)
                checked += 1
        assert checked > 20
        # waiting phases cost no pass: the same pass counts as with every phase placed as
        # early as it could go
        assert summ.passes == {34: 8, 30: 5}[n]


def test_fused_plans_of_the_headline_workload():
    """The 34-qubit circuit's tensor-core plans: the same 8 passes as the plain plan (the
    passes do not depend on the stage form), every stage a matrix stage, more stages than
    the plain plan (a diagonal gate joining a register qubit to an outside one after a
    non-diagonal gate on it ends the stage); the tile kernel's unpacked plan (five free
    register qubits) needs fewer than the packed one."""
    g = sv.sv_generate_circuit(inputs.C34)
    plain, *_ = sv.sv_plan(34, g, sv.options(jit=1))
    packed, *_ = sv.sv_plan(34, g, sv.options(precision=sv.SV_PREC_F16X3))
    tile, *_ = sv.sv_plan(34, g, sv.options(precision=sv.SV_PREC_F16X3, pipeline=-1))
    assert plain.passes == packed.passes == tile.passes == 8
    assert packed.matrix_stages == packed.stages
    assert plain.stages < tile.matrix_stages < packed.matrix_stages


def test_batch_config_needs_a_batch():
    with pytest.raises(sv.SvError):
        sv.sv_batch_config()


def test_planner_rejects_invalid_gates():
    bad = sv.gates_from_tuples([(4, 3, 3, 1)])  # CZ on one qubit
    with pytest.raises(sv.SvError):
        sv.sv_plan(8, bad)
    bad = sv.gates_from_tuples([(2, 9, 0, 1)])  # qubit out of range
    with pytest.raises(sv.SvError):
        sv.sv_plan(8, bad)
    bad = sv.gates_from_tuples([(42, 1, 0, 1)])  # unknown kind
    with pytest.raises(sv.SvError):
        sv.sv_plan(8, bad)
    with pytest.raises(sv.SvError):
        sv.sv_plan(8, sv.gates_from_tuples([(0, 1, 0, 0)]), sv.options(tile_bits=15))
    # 14-qubit tiles only for the plan-specialised plain kernels
    with pytest.raises(sv.SvError):
        sv.sv_plan(16, sv.gates_from_tuples([(0, 1, 0, 0)]), sv.options(tile_bits=14, jit=-1))
    with pytest.raises(sv.SvError):
        sv.sv_plan(16, sv.gates_from_tuples([(0, 1, 0, 0)]), sv.options(tile_bits=14, precision=sv.SV_PREC_F16X3))
    sv.sv_plan(16, sv.gates_from_tuples([(0, 1, 0, 0)]), sv.options(tile_bits=14))


def _all_kind_gates(n, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        k = int(rng.integers(11))
        if k in (5, 6):  # projectors: keep them rare
            k = 7
        a = int(rng.integers(n))
        b = int(rng.integers(n - 1))
        b = b + 1 if b >= a else b
        out.append((k, a, b if k == 4 else 0, 1))
    return sv.gates_from_tuples(out)


@pytest.mark.parametrize('case', ['16q_d10', '30q_d20', 'all_kinds_18q', 'tile9_all_kinds_14q', 'projectors_12q',
                                  'f16x3_34q_d30', 'tf32x3_16q_d10', 'f16x3_raw_all_kinds_14q'])
def test_plan_kernels_compile_without_a_device(case):
    """The code generator's kernels compile for sm_103a (NVRTC, no GPU needed), with
    tensor-core matrix stages for the split-precision modes."""
    if case == 'f16x3_34q_d30':
        n, g, o = 34, sv.sv_generate_circuit(inputs.C34), sv.options(precision=sv.SV_PREC_F16X3)
    elif case == 'tf32x3_16q_d10':
        n, g, o = 16, sv.sv_generate_circuit(inputs.C16), sv.options(precision=sv.SV_PREC_TF32X3)
    elif case == 'f16x3_raw_all_kinds_14q':
        n, g, o = 14, _all_kind_gates(14, 120, 6), sv.options(precision=sv.SV_PREC_F16X3, norm_restore=-1)
    elif case == '16q_d10':
        n, g, o = 16, sv.sv_generate_circuit(inputs.C16), None
    elif case == '30q_d20':
        n, g, o = 30, sv.sv_generate_circuit(inputs.C30), None
    elif case == 'all_kinds_18q':
        n, g, o = 18, _all_kind_gates(18, 200, 5), None
    elif case == 'tile9_all_kinds_14q':
        n, g, o = 14, _all_kind_gates(14, 120, 6), sv.options(tile_bits=9, low_bits=3, fuse_k=3)
    else:
        n = 12
        g = sv.gates_from_tuples([(0, q, 0, 0) for q in range(n)] + [(5, 3, 0, 1), (6, 9, 0, 1), (4, 2, 7, 1)])
        o = None
    try:
        sv.sv_jit_check(n, g, o)
    except sv.SvError as e:
        if 'libnvrtc not found' in str(e):
            pytest.skip('NVRTC not installed')
        raise


@pytest.mark.parametrize('lat,half_a', [(inputs.C42, inputs.C42_HALF_A), (inputs.C28, inputs.C28_HALF_A),
                                        (inputs.lattice_for(4, 4, 9, seed=31), (1 << 8) - 1)])
def test_branch_decomposition_counts(lat, half_a):
    """The cut plan's absorbed signs and implicit decompositions, recounted from the
    oracle's own gate list."""
    n, gates = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
    in_a = [bool((half_a >> q) & 1) for q in range(n)]
    last_nd = [-1] * n
    for i, (k, q0, _q1, _l) in enumerate(gates):
        if k in ('H', 'SX', 'SY'):
            last_nd[q0] = i
    t = absorbed = full = impl_a = impl_b = 0
    for i, (k, q0, q1, _l) in enumerate(gates):
        if k != 'CZ' or in_a[q0] == in_a[q1]:
            continue
        t += 1
        qa, qb = (q0, q1) if in_a[q0] else (q1, q0)
        qa_q, qb_q = last_nd[qa] < i, last_nd[qb] < i
        if qa_q and qb_q:
            absorbed += 1
        elif qa_q:
            impl_a += 1
        elif qb_q:
            impl_b += 1
        else:
            full += 1
    assert sv.sv_branch_counts(lat, half_a) == (t, absorbed, full + impl_b, full + impl_a, full)
    assert sv.sv_branch_counts(lat, half_a, full_decomposition=True) == (t, 0, t, t, t)


def test_42q_decomposition_sizes():
    """42 qubits cut 2|3: the last layer's 3 crossing CZs become output signs, so the
    halves hold 21 + 7 and 21 + 5 qubits instead of 21 + 10 each."""
    assert sv.sv_branch_counts(inputs.C42, inputs.C42_HALF_A) == (10, 3, 7, 5, 5)

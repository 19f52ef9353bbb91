"""GPU parity: the CUDA library (through its C interface) against the complex128 CPU
oracle on the same seeded circuits.

Bar (floating point): relative L2 error of the complex64 state <= 1e-5 and
|norm^2 - 1| <= 1e-6 (fp64 reduction) -- the tolerance the target sets for complex64
against an fp64 oracle.  Amplitude-level values that the method fixes exactly (uniform
layer 0, zeros of projectors) are compared at fp32 rounding.
"""
import numpy as np
import pytest

from oracle import circuit as oc
from oracle import csim
from oracle import statevec as ov
from paper_1804_04797_gb300 import inputs
from paper_1804_04797_gb300 import sv

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
NORM_TOL = 1e-6


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_gates(lat):
    return oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)


def run_gpu(lat, **kw):
    g = sv.sv_generate_circuit(lat)
    h = sv.sv_create(lat.n_qubits, sv.options(**kw))
    try:
        sv.sv_apply_circuit(h, g)
        psi = sv.sv_copy_state(h, lat.n_qubits)
        norm2, sp2 = sv.sv_norm(h)
    finally:
        sv.sv_destroy(h)
    return psi, norm2, sp2


TC = sv.SV_PREC_TF32X3
H16 = sv.SV_PREC_F16X3
MODES = [dict(), dict(tile_bits=14), dict(tile_bits=10, low_bits=4, fuse_k=5), dict(tile_bits=8, low_bits=2, fuse_k=3),
         dict(tile_bits=12, low_bits=5, fuse_k=4), dict(precision=sv.SV_PREC_PERGATE),
         dict(precision=TC), dict(precision=TC, tile_bits=12), dict(precision=TC, tile_bits=12, low_bits=3),
         dict(precision=H16), dict(precision=H16, tile_bits=12),
         dict(jit=1), dict(jit=1, tile_bits=12), dict(jit=1, tile_bits=8, low_bits=2, fuse_k=3), dict(jit=-1),
         # pipelined plan kernels on 10- and 11-qubit tiles (four groups of one and two warps)
         dict(jit=1, tile_bits=10), dict(jit=1, tile_bits=11)]


@pytest.mark.parametrize('kw', MODES)
def test_16q_depth10_matches_oracle(kw):
    lat = inputs.C16
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    psi, norm2, sp2 = run_gpu(lat, **kw)
    assert rel_l2(psi, want) <= REL_L2
    assert abs(norm2 - 1) <= NORM_TOL
    assert abs(sp2 - ov.sum_p2(want)) <= 1e-6 * ov.sum_p2(want) + 1e-12


SIZES = [inputs.lattice_for(2, 3, 8, seed=4),            # 6 qubits: one tile = the state
         inputs.lattice_for(3, 3, 12, seed=2),           # 9
         inputs.lattice_for(3, 5, 16, seed=7, removed=[(1, 2)]),   # 14, removed site
         inputs.lattice_for(4, 5, 18, seed=11),          # 20: 128 tiles of 2^13
         inputs.lattice_for(4, 6, 24, seed=13),          # 24
         inputs.lattice_for(1, 3, 6, seed=1),            # 3 qubits (per-gate path)
         inputs.lattice_for(1, 1, 0, seed=0)]            # 1 qubit, H only


@pytest.mark.parametrize('lat', SIZES, ids=lambda l: '%dx%d_d%d' % (l.rows, l.cols, l.depth))
def test_sizes_match_oracle(lat):
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    modes = [dict(), dict(tile_bits=min(13, max(6, n)), low_bits=min(4, n), fuse_k=5), dict(jit=1), dict(jit=-1)]
    # the tensor-core kernels take 12- and 13-qubit tiles: smaller states run the plain
    # kernel (test_tensor_core_request_below_12_qubits_is_reported), so only states that
    # reach the tensor cores carry their labels here
    if n >= 12:
        modes += [dict(precision=TC), dict(precision=TC, tile_bits=12), dict(precision=H16),
                  dict(precision=H16, tile_bits=12)]
    for kw in modes:
        psi, norm2, _ = run_gpu(lat, **kw)
        assert rel_l2(psi, want) <= REL_L2, kw
        assert abs(norm2 - 1) <= NORM_TOL


# the tensor-core kernels: matrix stages of the pipelined plan kernels (5-qubit blocks, the
# default), and the tile kernel with 5- and 4-qubit blocks
TC_KERNELS = {'k5_plan': dict(fuse_k=5), 'k5_tile': dict(fuse_k=5, pipeline=-1), 'k4_tile': dict(fuse_k=4)}


@pytest.mark.parametrize('kernel', list(TC_KERNELS))
@pytest.mark.parametrize('restore', [0, -1], ids=['restored', 'raw'])
@pytest.mark.parametrize('prec', [TC, H16], ids=['tf32x3', 'f16x3'])
@pytest.mark.parametrize('lat', [inputs.C16, inputs.lattice_for(4, 5, 18, seed=11)], ids=['16q', '20q'])
def test_tensor_core_paths_with_and_without_the_norm_restore(lat, prec, restore, kernel):
    """Both tensor-core formats, both kernels and both block sizes (32x32 and 16x16 stage
    unitaries) against the oracle, with the per-tile norm restore on and off: rel-L2 is
    the criterion in both cases; without the restore the norm shows the raw drift of the
    truncating accumulation (bounded loosely, recorded)."""
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    psi, norm2, _ = run_gpu(lat, precision=prec, norm_restore=restore, **TC_KERNELS[kernel])
    assert rel_l2(psi, want) <= REL_L2
    assert abs(norm2 - 1) <= (NORM_TOL if restore == 0 else 1e-4)


@pytest.mark.parametrize('prec', [TC, H16], ids=['tf32x3', 'f16x3'])
@pytest.mark.parametrize('lat', [inputs.lattice_for(3, 3, 12, seed=2), inputs.lattice_for(1, 3, 6, seed=1)],
                         ids=['9q', '3q'])
def test_tensor_core_request_below_12_qubits_is_reported(lat, prec):
    """Below 12 qubits a tensor-core request runs the plain kernel (tile passes; per-gate
    sweeps below 6 qubits); the profile counts it as a plain fallback, and the state still
    matches the oracle."""
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    h = sv.sv_create(n, sv.options(precision=prec))
    try:
        sv.sv_set_profiling(h, True)
        sv.sv_apply_circuit(h, sv.sv_generate_circuit(lat))
        prof = sv.sv_get_profile(h)
        psi = sv.sv_copy_state(h, n)
    finally:
        sv.sv_destroy(h)
    assert prof.plain_fallbacks == 1
    assert rel_l2(psi, want) <= REL_L2


def test_layer0_only_is_uniform():
    lat = inputs.lattice_for(4, 5, 0)
    psi, norm2, _ = run_gpu(lat)
    np.testing.assert_allclose(psi, np.full(1 << 20, 2.0 ** -10), rtol=0, atol=0)
    assert abs(norm2 - 1) < 1e-12


def _random_gate_list(n, count, seed):
    """Every kind of the interface, random qubits, no leading H layer."""
    rng = np.random.default_rng(seed)
    out = []
    kinds = ['H', 'T', 'SX', 'SY', 'CZ', 'Z', 'TDG', 'SXDG', 'SYDG']
    for _ in range(count):
        k = kinds[rng.integers(len(kinds))]
        a = int(rng.integers(n))
        if k == 'CZ':
            b = int(rng.integers(n - 1))
            b = b + 1 if b >= a else b
            out.append((k, a, b))
        else:
            out.append((k, a, -1))
    return out


_CODE = dict(oc.KIND_CODE, TDG=8, SXDG=9, SYDG=10)


def _to_lib(gl):
    return sv.gates_from_tuples([(_CODE[k], a, max(b, 0), 1) for (k, a, b) in gl])


def _oracle_apply(n, gl, psi):
    psi = np.array(psi, dtype=np.complex128)
    for k, a, b in gl:
        if k == 'CZ':
            ov.apply_cz(psi, a, b)
        elif k.endswith('DG'):
            ov.apply_1q(psi, ov.gate_matrix(k[:-2]).conj().T, a)
        else:
            ov.apply_1q(psi, ov.gate_matrix(k), a)
    return psi


@pytest.mark.parametrize('n,kw', [(7, {}), (13, {}), (18, {}), (18, dict(tile_bits=9, low_bits=3, fuse_k=2)),
                                  (13, dict(jit=1)), (18, dict(jit=1)), (18, dict(jit=1, tile_bits=9, low_bits=3)),
                                  (18, dict(jit=1, tile_bits=10)), (17, dict(jit=1, tile_bits=11)),
                                  (16, dict(precision=sv.SV_PREC_PERGATE)), (12, dict(precision=TC)),
                                  (17, dict(precision=TC)), (19, dict(precision=TC, tile_bits=12)),
                                  (17, dict(precision=H16)), (19, dict(precision=H16, tile_bits=12)),
                                  (12, dict(precision=H16)), (13, dict(precision=H16)),
                                  (17, dict(precision=H16, pipeline=-1)), (17, dict(precision=TC, fuse_k=4)),
                                  (17, dict(precision=H16, norm_restore=-1))])
def test_all_gate_kinds_from_zero_and_loaded_state(n, kw):
    gl = _random_gate_list(n, 120, seed=n)
    # from |0..0> (no H layer: the first pass generates |0..0>)
    want = _oracle_apply(n, gl, ov.zero_state(n))
    h = sv.sv_create(n, sv.options(**kw))
    try:
        sv.sv_apply_circuit(h, _to_lib(gl))
        assert rel_l2(sv.sv_copy_state(h, n), want) <= REL_L2
        # from a loaded random state (not fresh: the first pass reads it)
        rng = np.random.default_rng(3)
        start = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
        start /= np.linalg.norm(start)
        sv.sv_load_state(h, start)
        sv.sv_apply_circuit(h, _to_lib(gl))
        want2 = _oracle_apply(n, gl, start.astype(np.complex128))
        assert rel_l2(sv.sv_copy_state(h, n), want2) <= REL_L2
    finally:
        sv.sv_destroy(h)


@pytest.mark.parametrize('jit', [-1, 1])
def test_projectors_zero_exactly(jit):
    n = 12
    gl = [('H', q, -1) for q in range(n)] + [('SX', 3, -1), ('CZ', 3, 9, -1)]
    codes = sv.gates_from_tuples([(_CODE[k], a, max(b, 0), 0) for (k, a, b, *_r) in gl] +
                                 [(5, 3, 0, 1), (6, 9, 0, 1), (5, 0, 0, 1)])
    h = sv.sv_create(n, sv.options(jit=jit))
    try:
        sv.sv_apply_circuit(h, codes)
        psi = sv.sv_copy_state(h, n)
    finally:
        sv.sv_destroy(h)
    idx = np.arange(1 << n)
    dead = (((idx >> 3) & 1) == 1) | (((idx >> 9) & 1) == 0) | (((idx >> 0) & 1) == 1)
    assert np.all(psi[dead] == 0)
    assert np.count_nonzero(psi[~dead]) == np.count_nonzero(~dead)


@pytest.mark.parametrize('prec', [sv.SV_PREC_PLAIN, TC, H16])
def test_inverse_circuit_returns_to_zero_state(prec):
    lat = inputs.lattice_for(4, 5, 16, seed=21)
    g = sv.sv_generate_circuit(lat)
    h = sv.sv_create(20, sv.options(precision=prec))
    try:
        sv.sv_apply_circuit(h, g)
        sv.sv_apply_circuit_inverse(h, g)
        psi = sv.sv_copy_state(h, 20)
    finally:
        sv.sv_destroy(h)
    e0 = np.zeros(1 << 20, dtype=np.complex128)
    e0[0] = 1
    assert rel_l2(psi, e0) <= 1e-5


@pytest.mark.parametrize('lat,gl', [(inputs.lattice_for(4, 5, 18, seed=11), None),
                                    (None, _random_gate_list(19, 150, seed=77))])
def test_plan_kernels_bitwise_equal_to_interpreter(lat, gl):
    """The kernels compiled for a plan run the interpreter's arithmetic op for op.  Same
    stages for both: 13-qubit tiles (the largest the interpreter takes) and stages of
    qubit 0 + 3 (fuse_k = 3; the two kernels differ only in how many qubits a thread
    holds, which changes no amplitude's sequence of operations).  The pipelined kernels
    lay the tile out for the TMA copies and fill a stage's spare register slots with other
    qubits, so a diagonal gate on such a qubit may run in registers instead of as a phase
    at the stage's end (the same values to rounding): equal to 1e-6 and to the oracle."""
    if lat is not None:
        n, g = lat.n_qubits, sv.sv_generate_circuit(lat)
    else:
        n, g = 19, _to_lib(gl)
    out = {}
    for key, kw in (('interp', dict(jit=-1)), ('plan', dict(jit=1, pipeline=-1)), ('pipelined', dict(jit=1))):
        h = sv.sv_create(n, sv.options(tile_bits=13, fuse_k=3, **kw))
        try:
            sv.sv_set_profiling(h, True)
            sv.sv_apply_circuit(h, g)
            prof = sv.sv_get_profile(h)
            out[key] = sv.sv_copy_state(h, n)
        finally:
            sv.sv_destroy(h)
        assert (prof.jit_launches > 0) == (key != 'interp')
        assert prof.jit_launches == (prof.launches if key != 'interp' else 0)
    assert np.array_equal(out['interp'].view(np.uint32), out['plan'].view(np.uint32))
    assert rel_l2(out['pipelined'], out['interp']) <= 1e-6
    if lat is not None:
        n_, gates = oracle_gates(lat)
        assert rel_l2(out['pipelined'], csim.run(n_, gates)) <= REL_L2


def test_amplitudes_and_probabilities_gather():
    lat = inputs.lattice_for(4, 5, 14, seed=5)
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    bits = inputs.bitstrings(n, 64, seed=2) + [0, (1 << n) - 1]
    h = sv.sv_create(n)
    try:
        sv.sv_apply_circuit(h, sv.sv_generate_circuit(lat))
        amps = sv.sv_get_amplitudes(h, bits)
        probs = sv.sv_get_probabilities(h, bits)
        with pytest.raises(sv.SvError):
            sv.sv_get_amplitudes(h, [1 << n])
    finally:
        sv.sv_destroy(h)
    sel = want[np.array(bits, dtype=np.int64)]
    assert rel_l2(amps, sel) <= REL_L2
    np.testing.assert_allclose(probs, np.abs(amps) ** 2, rtol=1e-12, atol=0)


def test_empty_inputs():
    """An empty gate list leaves the state as it is (|0...0> when fresh), a gather of no
    bitstrings returns nothing, an empty batch is a no-op."""
    n = 12
    lat = inputs.lattice_for(3, 4, 6, seed=1)
    n_o, gates = oracle_gates(lat)
    assert n_o == n
    h = sv.sv_create(n)
    try:
        sv.sv_apply_circuit(h, sv.gates_from_tuples([]))
        psi = sv.sv_copy_state(h, n)
        assert psi[0] == 1 and np.count_nonzero(psi) == 1
        # from the written |0...0> (no uniform shortcut): the H layer runs as gates
        sv.sv_apply_circuit(h, sv.sv_generate_circuit(lat))
        before = sv.sv_copy_state(h, n)
        assert rel_l2(before, csim.run(n, gates)) <= REL_L2
        sv.sv_apply_circuit(h, sv.gates_from_tuples([]))
        sv.sv_apply_circuit_inverse(h, sv.gates_from_tuples([]))
        assert np.array_equal(sv.sv_copy_state(h, n), before)
        assert sv.sv_get_amplitudes(h, []).size == 0
        assert sv.sv_get_probabilities(h, []).size == 0
    finally:
        sv.sv_destroy(h)
    assert sv.sv_apply_batch([]).shape == (0, 3)


def test_invalid_arguments_leave_state_usable():
    h = sv.sv_create(10)
    try:
        with pytest.raises(sv.SvError):
            sv.sv_apply_circuit(h, sv.gates_from_tuples([(4, 2, 2, 1)]))
        with pytest.raises(sv.SvError):
            sv.sv_apply_circuit(h, sv.gates_from_tuples([(1, 10, 0, 1)]))
        sv.sv_apply_circuit(h, sv.gates_from_tuples([(0, q, 0, 0) for q in range(10)]))
        n2, _ = sv.sv_norm(h)
        assert abs(n2 - 1) < 1e-6
    finally:
        sv.sv_destroy(h)
    with pytest.raises(sv.SvError):
        sv.sv_create(35)
    with pytest.raises(sv.SvError):
        sv.sv_create(0)


def test_branch_amplitudes_small_cut_match_oracle():
    lat = inputs.lattice_for(4, 4, 9, seed=31)
    half_a = (1 << 8) - 1
    n, gates = oracle_gates(lat)
    bits = inputs.bitstrings(n, 64, seed=2)
    want_full = csim.run(n, gates)[np.array(bits, dtype=np.int64)]
    want_branch = csim.branch_amplitudes(n, gates, half_a, bits)
    assert rel_l2(want_branch, want_full) < 1e-12
    assert rel_l2(ov.branch_amplitudes_reduced(n, gates, half_a, bits), want_full) < 1e-12
    for kw in (dict(), dict(precision=TC), dict(precision=H16), dict(jit=1)):
        for full in (False, True):
            got = sv.sv_branch_amplitudes(lat, half_a, bits, sv.options(**kw), full_decomposition=full)
            assert rel_l2(got, want_full) <= REL_L2, (kw, full)


def test_branch_amplitudes_28q_check_against_full_state():
    """4x7 depth 10 cut 1|2 (t = 7): branch sum == a full 28-qubit GPU state, and both
    == the oracle's branch sum."""
    lat = inputs.C28
    n, gates = oracle_gates(lat)
    bits = inputs.bitstrings(n, 64, seed=2)
    got = sv.sv_branch_amplitudes(lat, inputs.C28_HALF_A, bits)
    got_full = sv.sv_branch_amplitudes(lat, inputs.C28_HALF_A, bits, full_decomposition=True)
    assert rel_l2(got_full, got) <= REL_L2
    h = sv.sv_create(n)
    try:
        sv.sv_apply_circuit(h, sv.sv_generate_circuit(lat))
        full = sv.sv_get_amplitudes(h, bits)
    finally:
        sv.sv_destroy(h)
    want = csim.branch_amplitudes(n, gates, inputs.C28_HALF_A, bits)
    assert rel_l2(got, want) <= REL_L2
    assert rel_l2(full, want) <= REL_L2


def test_batch_stats_match_oracle():
    lats = inputs.batch(6)
    stats = sv.sv_apply_batch(lats)
    for lat, row in zip(lats, stats):
        n, gates = oracle_gates(lat)
        s2, s4 = csim.reductions(csim.run(n, gates))
        assert row[2] == n
        assert abs(row[0] - 1) <= NORM_TOL
        assert abs(row[1] - s4) <= 1e-5 * s4


def test_batch_amplitudes_and_replay_match_oracle(tmp_path, monkeypatch):
    """Uneven batch in one persistent launch: per-circuit amplitudes and statistics match
    the oracle; the graph replay gives bit-identical statistics; autotune writes its cache."""
    lats = inputs.batch(12)
    stats = sv.sv_apply_batch(lats)
    again = sv.sv_apply_batch(lats)
    assert np.array_equal(stats, again)
    for i in (0, 5, 11):
        n, gates = oracle_gates(lats[i])
        want = csim.run(n, gates)
        bits = inputs.bitstrings(n, 32, seed=7)
        got = sv.sv_batch_amplitudes(i, bits)
        assert rel_l2(got, want[np.array(bits, dtype=np.int64)]) <= REL_L2
        s2, s4 = csim.reductions(want)
        assert abs(stats[i][0] - 1) <= NORM_TOL and abs(stats[i][1] - s4) <= 1e-5 * s4
    cache = tmp_path / 'tune.json'
    monkeypatch.setenv('SV_AUTOTUNE_CACHE', str(cache))
    tuned = sv.sv_apply_batch(lats, sv.options(autotune=1))
    assert cache.exists() and '|batch|' in cache.read_text()
    np.testing.assert_allclose(tuned[:, 0], 1.0, atol=NORM_TOL)
    # the configuration it ran with: the cached tile size, every circuit accounted for
    import json
    tile_bits, on_plan, persistent = sv.sv_batch_config()
    assert tile_bits in [v for k, v in json.loads(cache.read_text()).items() if '|batch|' in k]
    assert 11 <= tile_bits <= 13 and on_plan + persistent == len(lats)
    for i in (0, 11):
        n, gates = oracle_gates(lats[i])
        want = csim.run(n, gates)
        bits = inputs.bitstrings(n, 16, seed=5)
        assert rel_l2(sv.sv_batch_amplitudes(i, bits), want[np.array(bits, dtype=np.int64)]) <= REL_L2
    sv.sv_batch_free()
    with pytest.raises(sv.SvError):
        sv.sv_batch_amplitudes(0, [0])
    with pytest.raises(sv.SvError):
        sv.sv_batch_config()


@pytest.mark.parametrize('jit', [0, 1])
def test_batch_with_plan_kernel_circuits_matches_oracle(jit):
    """Circuits of 24 qubits (jit 0), or all of them (jit 1), run on kernels compiled for
    their plans inside the batch graph; the rest share the persistent launch."""
    every = inputs.batch(512)
    lats = every[:6] + [every[15]] + every[6:8]
    assert lats[6].n_qubits == 24
    try:
        stats = sv.sv_apply_batch(lats, sv.options(jit=jit))
    except sv.SvError as e:
        if 'libnvrtc' in str(e):
            pytest.skip('NVRTC not installed')
        raise
    for i in (0, 5, 6, 8):
        n, gates = oracle_gates(lats[i])
        want = csim.run(n, gates)
        bits = inputs.bitstrings(n, 32, seed=11)
        got = sv.sv_batch_amplitudes(i, bits)
        assert rel_l2(got, want[np.array(bits, dtype=np.int64)]) <= REL_L2
        s2, s4 = csim.reductions(want)
        assert stats[i][2] == n
        assert abs(stats[i][0] - 1) <= NORM_TOL and abs(stats[i][1] - s4) <= 1e-5 * s4
    assert np.array_equal(stats, sv.sv_apply_batch(lats, sv.options(jit=jit)))
    # without statistics: another graph, the same states
    before = [sv.sv_batch_amplitudes(i, inputs.bitstrings(lats[i].n_qubits, 16, seed=3)) for i in (1, 6)]
    assert sv.sv_apply_batch(lats, sv.options(jit=jit), stats=False) is None
    after = [sv.sv_batch_amplitudes(i, inputs.bitstrings(lats[i].n_qubits, 16, seed=3)) for i in (1, 6)]
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    sv.sv_batch_free()


def test_norm_summed_by_the_last_pass():
    """Plan kernels sum p and p^2 in the pass that writes the state and sv_norm returns
    those sums: they match the oracle and a separate reduction of the same state, and any
    other write of the state (load, basis state, a caller-writable pointer) drops them."""
    lat = inputs.lattice_for(4, 5, 14, seed=21)
    n, gates = oracle_gates(lat)
    assert n == 20
    want = csim.run(n, gates)
    _s2w, s4w = csim.reductions(want)
    g = sv.sv_generate_circuit(lat)
    h = sv.sv_create(n, sv.options(jit=1))
    try:
        sv.sv_apply_circuit(h, g)
        s2, s4 = sv.sv_norm(h)
        assert abs(s2 - 1) <= NORM_TOL and abs(s4 - s4w) <= 1e-5 * s4w
        state = sv.sv_copy_state(h, n)
        sv.sv_load_state(h, state)  # the same amplitudes, reduced by the separate kernel
        r2, r4 = sv.sv_norm(h)
        assert abs(r2 - s2) <= 1e-6 and abs(r4 - s4) <= 1e-6 * s4
        sv.sv_set_basis_state(h, 5)
        assert sv.sv_norm(h) == (1.0, 1.0)
        sv.sv_reset(h)
        sv.sv_apply_circuit(h, g)
        assert sv.sv_norm(h) == (s2, s4)  # the same run, the same sums
        sv.sv_device_ptr(h)  # from now on the caller may write the state
        sv.sv_reset(h)
        sv.sv_apply_circuit(h, g)
        d2, d4 = sv.sv_norm(h)
        assert abs(d2 - s2) <= 1e-6 and abs(d4 - s4) <= 1e-6 * s4
    finally:
        sv.sv_destroy(h)


def test_many_square_roots_in_one_stage():
    """200 X^{1/2} / Y^{1/2} gates on five qubits fall into one stage: their factors 1/2
    (deferred and applied in bulk by the tile kernels) must neither overflow nor lose
    accuracy."""
    n = 14
    gl = [('H', q, -1) for q in range(n)]
    for i in range(200):
        gl.append((('SX', 'SY', 'SXDG')[i % 3], i % 5, -1))
    want = _oracle_apply(n, gl, ov.zero_state(n))
    for kw in (dict(), dict(precision=TC), dict(precision=H16)):
        h = sv.sv_create(n, sv.options(**kw))
        try:
            sv.sv_apply_circuit(h, sv.gates_from_tuples([(_CODE[k], a, 0, 1) for (k, a, _b) in gl]))
            got = sv.sv_copy_state(h, n)
        finally:
            sv.sv_destroy(h)
        assert np.all(np.isfinite(got))
        assert rel_l2(got, want) <= REL_L2, kw


@pytest.mark.parametrize('kw', [dict(), dict(jit=1), dict(precision=TC), dict(precision=H16)])
def test_amplitudes_by_inner_product_match_oracle(kw):
    """Task 2 by <U2^dagger x | U1 H^n 0>: equals the oracle's full-state amplitudes."""
    lat = inputs.lattice_for(4, 5, 14, seed=5)
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    bits = inputs.bitstrings(n, 16, seed=2) + [0, (1 << n) - 1]
    sel = want[np.array(bits, dtype=np.int64)]
    for split in (0, 6, 14):
        got = sv.sv_amplitudes_by_inner_product(lat, split, bits, sv.options(**kw))
        assert rel_l2(got, sel) <= REL_L2, (split, kw)


def test_inner_product_and_basis_state():
    n = 17
    rng = np.random.default_rng(8)
    a = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    b = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    ha, hb = sv.sv_create(n), sv.sv_create(n)
    try:
        sv.sv_load_state(ha, a)
        sv.sv_load_state(hb, b)
        want = np.vdot(a.astype(np.complex128), b.astype(np.complex128))
        got = sv.sv_inner_product(ha, hb)
        assert abs(got - want) <= 1e-6 * np.linalg.norm(a) * np.linalg.norm(b)
        self_ip = sv.sv_inner_product(ha, ha)
        n2, _ = sv.sv_norm(ha)
        assert abs(self_ip.imag) <= 1e-6 * n2 and abs(self_ip.real - n2) <= 1e-6 * n2
        sv.sv_set_basis_state(hb, 12345)
        e = sv.sv_copy_state(hb, n)
        assert e[12345] == 1 and np.count_nonzero(e) == 1
        assert sv.sv_inner_product(ha, hb) == pytest.approx(complex(np.conj(a[12345])), rel=1e-6)
        with pytest.raises(sv.SvError):
            sv.sv_set_basis_state(hb, 1 << n)
    finally:
        sv.sv_destroy(ha)
        sv.sv_destroy(hb)
    h3, h4 = sv.sv_create(3), sv.sv_create(4)
    try:
        with pytest.raises(sv.SvError):
            sv.sv_inner_product(h3, h4)
    finally:
        sv.sv_destroy(h3)
        sv.sv_destroy(h4)


# the tensor-form product on the CUDA cores (plain) and on the tensor cores (TF32x3).  The
# tensor-core accumulation truncates toward zero; the product has no unitary structure
# whose norm could be restored per tile, so its norm keeps that drift (~1e-6 at 28
# qubits): rel-L2 and fidelity are its criteria, the norm is bounded loosely.
PRODUCT = {'cuda_cores': None, 'tensor_cores': sv.options(precision=TC)}
PRODUCT_NORM_TOL = {'cuda_cores': NORM_TOL, 'tensor_cores': 1e-5}


@pytest.mark.parametrize('full', [False, True])
@pytest.mark.parametrize('product', list(PRODUCT))
def test_branch_full_state_matches_oracle(full, product):
    """Eqs. 6-7: the full state as the sum over branches of A_l (x) B_l."""
    lat = inputs.lattice_for(4, 4, 9, seed=31)
    half_a = (1 << 8) - 1
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    h = sv.sv_create(n)
    try:
        sv.sv_branch_full_state(lat, half_a, h, PRODUCT[product], full_decomposition=full)
        got = sv.sv_copy_state(h, n)
        n2, _ = sv.sv_norm(h)
    finally:
        sv.sv_destroy(h)
    assert rel_l2(got, want) <= REL_L2
    assert abs(n2 - 1) <= PRODUCT_NORM_TOL[product]


@pytest.mark.parametrize('product', list(PRODUCT))
@pytest.mark.parametrize('depth', [3, 6])
@pytest.mark.parametrize('full', [False, True])
def test_branch_full_state_with_part_c_matches_oracle(full, depth, product):
    """Eq. 3: layers 0..depth through the tensor form of the cut decomposition (parts A
    and B), the remaining layers (part C) on the reconstructed state."""
    lat = inputs.lattice_for(4, 4, 11, seed=37)
    half_a = (1 << 8) - 1
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    h = sv.sv_create(n)
    try:
        sv.sv_branch_full_state(lat, half_a, h, PRODUCT[product], full_decomposition=full, depth=depth)
        got = sv.sv_copy_state(h, n)
        n2, _ = sv.sv_norm(h)
    finally:
        sv.sv_destroy(h)
    assert rel_l2(got, want) <= REL_L2
    assert abs(n2 - 1) <= PRODUCT_NORM_TOL[product]


@pytest.mark.parametrize('full', [False, True])
@pytest.mark.parametrize('product', list(PRODUCT))
def test_branch_full_state_28q_with_part_c_equals_direct_run(product, full):
    """The 28-qubit check lattice cut after layer 5: parts A and B by the decomposition
    (the default one, and the full one: 2^7 summed branches), part C (layers 6..10) on
    the full 2^28 state, against the direct run."""
    lat = inputs.C28
    n = lat.n_qubits
    a, b = sv.sv_create(n), sv.sv_create(n)
    try:
        sv.sv_branch_full_state(lat, inputs.C28_HALF_A, a, PRODUCT[product], full_decomposition=full, depth=5)
        sv.sv_apply_circuit(b, sv.sv_generate_circuit(lat))
        ip = sv.sv_inner_product(b, a)
        n2a, _ = sv.sv_norm(a)
    finally:
        sv.sv_destroy(a)
        sv.sv_destroy(b)
    assert abs(n2a - 1) <= PRODUCT_NORM_TOL[product]
    assert 1 - abs(ip) ** 2 / n2a <= 1e-9


@pytest.mark.parametrize('product', list(PRODUCT))
def test_branch_full_state_28q_equals_direct_run(product):
    lat = inputs.C28
    n = lat.n_qubits
    a, b = sv.sv_create(n), sv.sv_create(n)
    try:
        sv.sv_branch_full_state(lat, inputs.C28_HALF_A, a, PRODUCT[product])
        sv.sv_apply_circuit(b, sv.sv_generate_circuit(lat))
        ip = sv.sv_inner_product(b, a)
        n2a, _ = sv.sv_norm(a)
        bits = inputs.bitstrings(n, 64, seed=2)
        assert rel_l2(sv.sv_get_amplitudes(a, bits), sv.sv_get_amplitudes(b, bits)) <= REL_L2
    finally:
        sv.sv_destroy(a)
        sv.sv_destroy(b)
    assert abs(n2a - 1) <= PRODUCT_NORM_TOL[product]
    assert 1 - abs(ip) ** 2 / n2a <= 1e-9        # 1 - fidelity against the direct state
    h = sv.sv_create(n)
    try:
        with pytest.raises(sv.SvError):          # half A must be the low qubits
            sv.sv_branch_full_state(lat, ((1 << n) - 1) ^ inputs.C28_HALF_A, h)
    finally:
        sv.sv_destroy(h)


@pytest.mark.parametrize('kw', [dict(), dict(jit=-1), dict(precision=H16)])
def test_repeated_circuit_reuses_its_plan(kw):
    """A handle replays the last plan when the same circuit comes again (same options and
    starting condition); a changed condition plans anew."""
    lat = inputs.lattice_for(4, 6, 16, seed=9)
    n = lat.n_qubits
    g = sv.sv_generate_circuit(lat)
    h = sv.sv_create(n, sv.options(**kw))
    try:
        sv.sv_apply_circuit(h, g)
        a1 = sv.sv_copy_state(h, n)
        sv.sv_reset(h)
        sv.sv_apply_circuit(h, g)                 # same key: replayed
        a2 = sv.sv_copy_state(h, n)
        sv.sv_apply_circuit_inverse(h, g)         # another plan
        sv.sv_apply_circuit(h, g)                 # not fresh now: planned again
        a3 = sv.sv_copy_state(h, n)
    finally:
        sv.sv_destroy(h)
    assert np.array_equal(a1.view(np.uint32), a2.view(np.uint32))
    assert rel_l2(a3, a1) <= 2e-5


def test_autotuned_plain_path_caches_its_choice_and_matches_the_oracle(tmp_path, monkeypatch):
    """sv_options.autotune = 1 on a fresh state: the tile size, the fusion width (qubits
    per stage) and each pass's compute groups are picked by timing and kept in the JSON
    cache; the tuned run matches the oracle, and a second handle takes the cached choice
    (same plan, bitwise the same state)."""
    import json
    cache = tmp_path / 'autotune.json'
    monkeypatch.setenv('SV_AUTOTUNE_CACHE', str(cache))
    lat = inputs.lattice_for(4, 6, 16, seed=13)
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    psi1, norm2, _ = run_gpu(lat, jit=1, autotune=1)
    assert rel_l2(psi1, want) <= REL_L2
    assert abs(norm2 - 1) <= NORM_TOL
    entries = json.loads(cache.read_text())
    keys = [k for k in entries if '|circuit|%d|' % n in k]
    m = [entries[k] for k in keys if k.endswith('|m')]
    passes = [entries[k] for k in keys if k.endswith('|passes')]
    k = [entries[k] for k in keys if k.endswith('|k')]
    assert m and m[0] in (12, 13)
    assert k and (m[0], k[0]) in ((12, 5), (13, 5), (12, 6))
    assert passes and all(k.rsplit('|', 1)[0] + '|p%d' % i in entries for k in keys if k.endswith('|passes')
                          for i in range(passes[0]))
    psi2, _, _ = run_gpu(lat, jit=1, autotune=1)
    assert np.array_equal(psi1.view(np.uint32), psi2.view(np.uint32))
    # the profile reports the plan the handle ran: the cached tile size and width
    h = sv.sv_create(n, sv.options(jit=1, autotune=1))
    try:
        sv.sv_set_profiling(h, True)
        sv.sv_apply_circuit(h, sv.sv_generate_circuit(lat))
        prof = sv.sv_get_profile(h)
    finally:
        sv.sv_destroy(h)
    assert (prof.plan_tile_bits, prof.plan_stage_qubits) == (m[0], k[0]) and prof.plan_passes == passes[0]


def test_state_on_a_torch_owned_buffer_matches_the_oracle():
    """sv_create_from_ptr on a torch-allocated complex64 tensor (PyTorch owns the device
    memory; the library only runs kernels on it): |0...0> written by torch, the circuit
    applied by the library, the tensor read back by torch and checked against the oracle;
    a misaligned view is refused."""
    import torch
    lat = inputs.lattice_for(4, 5, 14, seed=5)
    n, gates = oracle_gates(lat)
    want = csim.run(n, gates)
    buf = torch.zeros(1 << n, dtype=torch.complex64, device='cuda')
    buf[0] = 1
    stream = torch.cuda.current_stream()
    h = sv.sv_create_from_ptr(n, buf.data_ptr(), stream.cuda_stream)
    try:
        sv.sv_apply_circuit(h, sv.sv_generate_circuit(lat))
        norm2, _ = sv.sv_norm(h)
    finally:
        sv.sv_destroy(h)
    torch.cuda.synchronize()
    psi = buf.cpu().numpy()
    assert rel_l2(psi, want) <= REL_L2
    assert abs(norm2 - 1) <= NORM_TOL
    with pytest.raises(sv.SvError, match='aligned'):
        sv.sv_create_from_ptr(n - 1, buf[1:].data_ptr(), stream.cuda_stream)

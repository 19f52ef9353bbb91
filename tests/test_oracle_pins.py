"""Pins of the CPU oracle to things other than itself (runs without a GPU).

Each test ties the oracle to the paper's definitions, to closed forms, to brute force
on tiny inputs, or to published reference values, so that a plausible mistake in the
oracle (a wrong sign in a gate matrix, a transposed pair update, a wrong bit index, a
dropped branch term, a generator rule misread) fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import circuit as oc
from oracle import csim
from oracle import statevec as ov
from paper_1804_04797_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)


# --- gate matrices (reading of the gate set in §2) -----------------------------------

def test_gate_matrices_are_the_named_roots_and_unitary():
    sx, sy, h, t = (ov.gate_matrix(k) for k in ('SX', 'SY', 'H', 'T'))
    np.testing.assert_allclose(sx @ sx, X, atol=1e-15)
    np.testing.assert_allclose(sy @ sy, Y, atol=1e-15)
    np.testing.assert_allclose(h @ h, I2, atol=1e-15)
    np.testing.assert_allclose(h @ Z @ h, X, atol=1e-15)
    np.testing.assert_allclose(np.linalg.matrix_power(t, 2), np.diag([1, 1j]), atol=1e-15)
    np.testing.assert_allclose(np.linalg.matrix_power(t, 8), I2, atol=1e-14)
    for u in (sx, sy, h, t):
        np.testing.assert_allclose(u @ u.conj().T, I2, atol=1e-15)
    # principal roots: eigenvalues 1 and i
    for u in (sx, sy):
        ev = np.sort_complex(np.linalg.eigvals(u))
        np.testing.assert_allclose(ev, np.sort_complex(np.array([1, 1j])), atol=1e-14)


def test_cz_equals_projector_decomposition():
    """§2: CU^{c,t} = P0^c (x) I^t + P1^c (x) U^t with U = Z, as 2^n matrices."""
    n = 3
    for c, t in [(0, 1), (2, 0), (1, 2)]:
        lhs = ov.embed_cz(n, c, t)
        rhs = (ov.embed_1q(n, ov.gate_matrix('P0'), c)
               + ov.embed_1q(n, ov.gate_matrix('P1'), c) @ ov.embed_1q(n, Z, t))
        np.testing.assert_allclose(lhs, rhs, atol=0)


def test_pair_update_equals_kronecker_definition():
    """§2: the pair update on qubit k equals I^(n-k-1) (x) U (x) I^(k) applied to psi."""
    rng = np.random.default_rng(5)
    n = 6
    for k in range(n):
        U = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        want = ov.embed_1q(n, U, k) @ psi
        got = ov.apply_1q(psi.copy(), U, k)
        np.testing.assert_allclose(got, want, atol=1e-13)
        # spot-check one pair against the printed update rule by hand
        i = 0b101010 & ~(1 << k)
        j = i + (1 << k)
        np.testing.assert_allclose(got[i], U[0, 0] * psi[i] + U[0, 1] * psi[j], atol=1e-13)
        np.testing.assert_allclose(got[j], U[1, 0] * psi[i] + U[1, 1] * psi[j], atol=1e-13)


# --- brute force and closed forms ----------------------------------------------------

SMALL = [(2, 3, 0, 12, 3), (3, 3, 0, 16, 7), (2, 5, 0, 9, 11), (3, 3, 1 << 4, 14, 1)]


@pytest.mark.parametrize('rows,cols,rm,depth,seed', SMALL)
def test_oracle_matches_brute_force_unitary(rows, cols, rm, depth, seed):
    n, gates = oc.generate(rows, cols, rm, depth, seed)
    U = ov.full_unitary(n, gates)
    want = U[:, 0]
    np.testing.assert_allclose(ov.run(n, gates), want, atol=1e-12)
    np.testing.assert_allclose(csim.run(n, gates), want, atol=1e-12)


def test_layer0_gives_uniform_amplitudes():
    n, gates = oc.generate(4, 4, 0, 0, 0)
    assert all(g[0] == 'H' for g in gates) and len(gates) == 16
    psi = csim.run(n, gates)
    np.testing.assert_allclose(psi, np.full(1 << n, 2.0 ** (-n / 2)), atol=1e-15)


def test_layer1_closed_form_cz_signs():
    """After layer 0 and layer 1 (CZs only): alpha_x = 2^{-n/2} (-1)^{sum x_a x_b}."""
    n, gates = oc.generate(4, 5, 0, 1, 0)
    pairs = [(a, b) for (k, a, b, _l) in gates if k == 'CZ']
    assert pairs and all(l <= 1 for (*_x, l) in gates)
    x = np.arange(1 << n)
    par = np.zeros(1 << n, dtype=np.int64)
    for a, b in pairs:
        par ^= ((x >> a) & 1) & ((x >> b) & 1)
    want = 2.0 ** (-n / 2) * (1 - 2 * par)
    np.testing.assert_allclose(csim.run(n, gates), want, atol=1e-15)
    np.testing.assert_allclose(ov.run(n, gates), want, atol=1e-15)


def test_t_and_cz_only_phases():
    """H on all, then T on a qubit set and CZ on pairs: alpha_x = 2^{-n/2} w^{sum_T x_q}
    (-1)^{sum x_a x_b}, w = e^{i pi/4}."""
    n = 7
    tq = [0, 3, 3, 6]
    cz = [(1, 2), (0, 6), (3, 5)]
    gates = [('H', q, -1, 0) for q in range(n)]
    gates += [('T', q, -1, 1) for q in tq] + [('CZ', a, b, 1) for a, b in cz]
    x = np.arange(1 << n)
    e = sum(((x >> q) & 1) for q in tq)
    s = sum(((x >> a) & 1) & ((x >> b) & 1) for a, b in cz)
    want = 2.0 ** (-n / 2) * np.exp(1j * np.pi / 4 * e) * (-1.0) ** s
    np.testing.assert_allclose(csim.run(n, gates), want, atol=1e-15)


def test_norm_and_inverse():
    n, gates = oc.generate(4, 4, 0, 10, 0)
    psi = csim.run(n, gates)
    assert abs(ov.norm2(psi) - 1) < 1e-13
    back = csim.run(n, gates, psi=psi, adjoint=True)
    e0 = np.zeros(1 << n, dtype=np.complex128)
    e0[0] = 1
    np.testing.assert_allclose(back, e0, atol=1e-13)
    back2 = ov.run_adjoint(n, gates, psi)
    np.testing.assert_allclose(back2, e0, atol=1e-13)


def test_c_and_numpy_oracles_agree():
    n, gates = oc.generate(3, 5, 0, 18, 42)
    np.testing.assert_allclose(csim.run(n, gates), ov.run(n, gates), atol=1e-13)
    s2, s4 = csim.reductions(csim.run(n, gates))
    psi = ov.run(n, gates)
    assert abs(s2 - ov.norm2(psi)) < 1e-13 and abs(s4 - ov.sum_p2(psi)) < 1e-15


def test_porter_thomas_statistic_of_deep_circuit():
    """§3 (Porter-Thomas figure): deep random circuits have N * sum p^2 close to 2."""
    n, gates = oc.generate(4, 5, 0, 32, 3)
    s2, s4 = csim.reductions(csim.run(n, gates))
    assert abs(s2 - 1) < 1e-12
    assert 1.85 < (1 << n) * s4 < 2.15


# --- cut decomposition (§2 Fig. 2, Eq. 1; §2.1 Fig. 3) ----------------------------------

@pytest.mark.parametrize('rows,cols,depth,seed,half_rows', [(2, 3, 10, 1, 1), (4, 3, 9, 4, 2),
                                                          (3, 4, 12, 9, 1)])
def test_branch_sum_equals_full_state(rows, cols, depth, seed, half_rows):
    n, gates = oc.generate(rows, cols, 0, depth, seed)
    half_a = (1 << (half_rows * cols)) - 1
    t = len(oc.cut_crossings(gates, half_a))
    assert t >= 1
    psi = ov.run(n, gates)
    bits = list(range(0, 1 << n, max(1, (1 << n) // 37)))
    want = psi[bits]
    np.testing.assert_allclose(ov.branch_amplitudes(n, gates, half_a, bits), want, atol=1e-13)
    np.testing.assert_allclose(csim.branch_amplitudes(n, gates, half_a, bits), want, atol=1e-13)


def test_dropping_one_branch_is_detected():
    """A sum that loses a branch (a dropped term) no longer equals the full state."""
    n, gates = oc.generate(2, 3, 0, 10, 1)
    half_a = 0b000111
    qa, qb, ga, gb, t = ov.split_halves(n, gates, half_a)
    psi = ov.run(n, gates)
    bits = list(range(1 << n))
    acc = np.zeros(len(bits), dtype=np.complex128)
    xa = [ov._compress(x, qa) for x in bits]
    xb = [ov._compress(x, qb) for x in bits]
    for l in range(1, 1 << t):
        A = ov.run(len(qa), ov._branch_gates(ga, l, 'A'))
        B = ov.run(len(qb), ov._branch_gates(gb, l, 'B'))
        acc += A[xa] * B[xb]
    assert np.max(np.abs(acc - psi)) > 1e-3


def _read_fig3():
    parts = {'A': [], 'B': [], 'C': []}
    with open(os.path.join(GOLDEN, 'fig3_worked_example.txt')) as f:
        for line in f:
            line = line.split('#')[0].strip()
            if not line:
                continue
            part, rest = line.split(':')
            tok = rest.split()
            parts[part].append((tok[0], [int(v) for v in tok[1:]]))
    return parts


def test_fig3_worked_example_eq1_and_implicit_zero_pattern():
    """Eq. 1 then the part-C product reproduce the direct 4-qubit run, and the part-B
    amplitudes vanish when l2 differs from the index of qubit 2 (implicit
    decomposition, §2.1)."""
    parts = _read_fig3()
    # direct run: merge parts A and B in time order around the two cut CZ^{2,1}
    seq_a = parts['A']
    seq_b = parts['B']

    def upto(seq, tag):
        i = [k for k, (g, _q) in enumerate(seq) if g == tag][0]
        return seq[:i], seq[i + 1:]

    a0, a_rest = upto(seq_a, 'CUT1')
    a1, a2 = upto(a_rest, 'CUT2')
    b0, b_rest = upto(seq_b, 'CUT1')
    b1, b2 = upto(b_rest, 'CUT2')

    def tog(seq):
        return [(g, q[0], q[1] if len(q) > 1 else -1, 0) for g, q in seq]
    full = (tog(a0) + tog(b0) + [('CZ', 1, 2, 0)] + tog(a1) + tog(b1) + [('CZ', 1, 2, 0)]
            + tog(a2) + tog(b2) + tog(parts['C']))
    want = ov.run(4, full)

    psi_in = np.zeros(16, dtype=np.complex128)
    for l1 in (0, 1):
        for l2 in (0, 1):
            ga, gb = [], []
            for g, q in seq_a:
                if g.startswith('CUT'):
                    lj = l1 if g == 'CUT1' else l2
                    if lj:
                        ga.append(('Z', q[0], -1, 0))
                else:
                    ga.append((g, q[0], q[1] if len(q) > 1 else -1, 0))
            for g, q in seq_b:
                if g.startswith('CUT'):
                    lj = l1 if g == 'CUT1' else l2
                    gb.append(('P1' if lj else 'P0', q[0] - 2, -1, 0))
                else:
                    gb.append((g, q[0] - 2, (q[1] - 2) if len(q) > 1 else -1, 0))
            phi = ov.run(2, ga)        # qubits 0, 1
            xi = ov.run(2, gb)         # qubits 2, 3 as local 0, 1
            for i2 in (0, 1):
                if i2 != l2:
                    assert abs(xi[i2]) < 1e-15 and abs(xi[i2 + 2]) < 1e-15
            psi_in += np.kron(xi, phi)
    got = ov.run(4, tog(parts['C']), psi=psi_in)
    np.testing.assert_allclose(got, want, atol=1e-14)


# --- generator rules ---------------------------------------------------------------

def _golden_splitmix():
    out = {}
    with open(os.path.join(GOLDEN, 'splitmix64_vectors.txt')) as f:
        for line in f:
            line = line.split('#')[0].strip()
            if line:
                s, vals = line.split(':')
                out[int(s)] = [int(v) for v in vals.split()]
    return out


def test_splitmix64_published_vectors():
    for seed, vals in _golden_splitmix().items():
        r = oc.SplitMix64(seed)
        assert [r.next() for _ in vals] == vals


def _lattice_neighbours(rows, cols, rm):
    idx = oc.site_numbering(rows, cols, rm)
    nb = set()
    for (r, c), a in idx.items():
        for (dr, dc) in ((0, 1), (1, 0)):
            o = (r + dr, c + dc)
            if o in idx:
                nb.add((min(a, idx[o]), max(a, idx[o])))
    return nb


@pytest.mark.parametrize('rows,cols,rm', [(4, 4, 0), (5, 6, 0), (6, 6, 1 | (1 << 35)), (6, 7, 0),
                                          (4, 5, (1 << 9) | (1 << 14) | (1 << 19))])
def test_cz_patterns_are_matchings_covering_every_bond_once(rows, cols, rm):
    pats = oc.cz_patterns(rows, cols, rm)
    assert len(pats) == 8
    seen = []
    for p in pats:
        qs = [q for pr in p for q in pr]
        assert len(qs) == len(set(qs))
        seen += p
    assert sorted(seen) == sorted(_lattice_neighbours(rows, cols, rm))


def test_single_qubit_gate_rule():
    rows, cols, rm, depth = 5, 6, 0, 40
    for seed in (0, 1, 2):
        n, gates = oc.generate(rows, cols, rm, depth, seed)
        pats = oc.cz_patterns(rows, cols, rm)
        prev_gate = [None] * n
        for layer in range(1, depth + 1):
            cur = set(q for p in pats[(layer - 1) % 8] for q in p)
            prevl = set(q for p in pats[(layer - 2) % 8] for q in p) if layer > 1 else set()
            one = [g for g in gates if g[3] == layer and g[0] != 'CZ']
            assert sorted(g[1] for g in one) == sorted(prevl - cur)
            for g in one:
                assert g[0] in ('T', 'SX', 'SY') and g[0] != prev_gate[g[1]]
                prev_gate[g[1]] = g[0]
            czs = [g for g in gates if g[3] == layer and g[0] == 'CZ']
            assert sorted((g[1], g[2]) for g in czs) == pats[(layer - 1) % 8]
            # order inside a layer: one-qubit gates first
            pos = [i for i, g in enumerate(gates) if g[3] == layer]
            kinds = [gates[i][0] for i in pos]
            assert kinds == sorted(kinds, key=lambda k: k == 'CZ')


def test_single_qubit_gate_frequencies_near_one_third():
    counts = {'T': 0, 'SX': 0, 'SY': 0}
    for seed in range(20):
        _n, gates = oc.generate(6, 6, 0, 40, seed)
        for g in gates:
            if g[0] in counts:
                counts[g[0]] += 1
    tot = sum(counts.values())
    for k, v in counts.items():
        assert abs(v / tot - 1 / 3) < 0.03, counts


def test_gate_counts_of_the_workloads():
    """Gate totals of the five lattices under the readings (layer-0 H included)."""
    cases = [((4, 4, 0, 10), (32, 34, 82)), ((5, 6, 0, 20), (123, 140, 293)),
             ((6, 6, 1 | (1 << 35), 30), (212, 232, 478)), ((4, 7, 0, 10), (58, 60, 146)),
             ((6, 7, 0, 10), (91, 91, 224))]
    for (r, c, rm, d), (ncz, n1, tot) in cases:
        n, g = oc.generate(r, c, rm, d, 0)
        assert sum(1 for x in g if x[0] == 'CZ') == ncz
        assert sum(1 for x in g if x[0] in ('T', 'SX', 'SY')) == n1
        assert len(g) == tot


def test_cut_crossing_counts():
    """Crossing CZs of the two cut configurations: 42 qubits cut 2|3 -> t = 10 (layers
    2, 6, 10); 28 qubits cut 1|2 -> t = 7."""
    _n, g = oc.generate(6, 7, 0, 10, 0)
    cr = oc.cut_crossings(g, (1 << 21) - 1)
    assert len(cr) == 10
    assert sorted(set(g[i][3] for i in cr)) == [2, 6, 10]
    _n, g = oc.generate(4, 7, 0, 10, 0)
    assert len(oc.cut_crossings(g, (1 << 14) - 1)) == 7


@pytest.mark.parametrize('rows,cols,depth,split', [(3, 3, 8, 3), (3, 4, 10, 5), (2, 5, 9, 0), (3, 3, 8, 8),
                                                   (3, 3, 8, 20)])
def test_inner_product_amplitudes_equal_the_full_state(rows, cols, depth, split):
    """Task 2 by <U2^dagger x | U1 H^n 0> (cut after any layer, including before every
    layer but layer 0 and after the last) equals the forward state's amplitude."""
    lat = inputs.lattice_for(rows, cols, depth, seed=17)
    n, gates = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
    want = ov.run(n, gates)
    bits = inputs.bitstrings(n, 12, seed=3) + [0, (1 << n) - 1]
    got = ov.amplitudes_inner_product(n, gates, split, bits)
    np.testing.assert_allclose(got, want[np.array(bits)], rtol=0, atol=1e-13)


def test_inner_product_detects_a_missing_adjoint():
    """A planted mistake (U2 applied forward instead of as its adjoint) fails."""
    lat = inputs.lattice_for(3, 3, 8, seed=17)
    n, gates = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
    want = ov.run(n, gates)
    g1 = [g for g in gates if g[3] <= 3]
    g2 = [g for g in gates if g[3] > 3]
    psi = ov.run(n, g1)
    x = 5
    e = np.zeros(1 << n, dtype=np.complex128)
    e[x] = 1.0
    wrong = np.vdot(ov.run(n, g2, e), psi)
    assert abs(wrong - want[x]) > 1e-3 * abs(want[x])


@pytest.mark.parametrize('rows,cols,depth,cut_rows', [(4, 4, 9, 2), (3, 4, 12, 1), (4, 3, 10, 2)])
def test_reduced_branch_sum_equals_the_full_state(rows, cols, depth, cut_rows):
    """Absorbed output signs and implicit decompositions give the exact amplitudes."""
    lat = inputs.lattice_for(rows, cols, depth, seed=31)
    n, gates = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
    half_a = (1 << (cut_rows * cols)) - 1
    bits = inputs.bitstrings(n, 10, seed=4) + [0, (1 << n) - 1]
    want = ov.run(n, gates)[np.array(bits)]
    np.testing.assert_allclose(ov.branch_amplitudes_reduced(n, gates, half_a, bits), want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ov.branch_amplitudes(n, gates, half_a, bits), want, rtol=0, atol=1e-12)


def test_implicit_branch_slices_vanish():
    """§2.1: after the last non-diagonal gate on the projector's qubit q, the branch with
    l != x_q is identically zero -- the fact implicit decomposition rests on."""
    lat = inputs.lattice_for(4, 4, 9, seed=31)
    n, gates = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
    half_a = (1 << 8) - 1
    qa, qb, ga, gb, t = ov.split_halves(n, gates, half_a)
    last_nd = [-1] * len(qa)
    for i, g in enumerate(ga):
        if g[0] in ov.NON_DIAGONAL:
            last_nd[g[1]] = i
    quiet = [(i, g) for i, g in enumerate(ga) if g[0] == 'CUT' and last_nd[g[1]] < i]
    assert quiet, 'the case needs a quiet crossing'
    for _i, (_k, q, j, _layer) in quiet:
        for l in range(1 << t):
            A = ov.run(len(qa), ov._branch_gates(ga, l, 'A'))
            lj = (l >> j) & 1
            idx = np.arange(A.size)
            assert np.all(A[((idx >> q) & 1) != lj] == 0)


def test_full_state_is_the_sum_of_branch_outer_products():
    """§2 Eqs. 6-7 (the tensor form): psi = sum_l A_l (x) B_l over all 2^t branches,
    with half A the low qubits."""
    lat = inputs.lattice_for(4, 4, 9, seed=31)
    n, gates = oc.generate(lat.rows, lat.cols, lat.removed_mask, lat.depth, lat.seed)
    half_a = (1 << 8) - 1
    qa, qb, ga, gb, t = ov.split_halves(n, gates, half_a)
    assert qa == list(range(8))
    psi = np.zeros(1 << n, dtype=np.complex128)
    for l in range(1 << t):
        A = ov.run(len(qa), ov._branch_gates(ga, l, 'A'))
        B = ov.run(len(qb), ov._branch_gates(gb, l, 'B'))
        psi += np.outer(B, A).reshape(-1)      # index x_A + (x_B << n_A)
    np.testing.assert_allclose(psi, ov.run(n, gates), rtol=0, atol=1e-12)


def test_square_roots_as_scaled_rotations():
    """The factorisation the plain kernels use (a scalar e^{+-i pi/4} 2^{-1/2} times an
    unscaled rotation), checked on the oracle's own matrices: X^{1/2} = e^{i pi/4}
    2^{-1/2} [[1,-i],[-i,1]], Y^{1/2} = e^{i pi/4} 2^{-1/2} [[1,-1],[1,1]], and their
    adjoints with e^{-i pi/4} and [[1,i],[i,1]], [[1,1],[-1,1]]."""
    w = np.exp(1j * np.pi / 4) / np.sqrt(2.0)
    sx, sy = ov.gate_matrix('SX'), ov.gate_matrix('SY')
    np.testing.assert_allclose(sx, w * np.array([[1, -1j], [-1j, 1]]), atol=1e-15)
    np.testing.assert_allclose(sy, w * np.array([[1, -1], [1, 1]]), atol=1e-15)
    np.testing.assert_allclose(sx.conj().T, np.conj(w) * np.array([[1, 1j], [1j, 1]]), atol=1e-15)
    np.testing.assert_allclose(sy.conj().T, np.conj(w) * np.array([[1, 1], [-1, 1]]), atol=1e-15)
    # a circuit's square roots leave one scalar: its phase count mod 8 and its 2^{-1/2} count
    rng = np.random.default_rng(3)
    kinds = rng.choice(['SX', 'SY'], size=37)
    total = np.eye(2, dtype=np.complex128)
    bare = np.eye(2, dtype=np.complex128)
    rot = {'SX': np.array([[1, -1j], [-1j, 1]]), 'SY': np.array([[1, -1], [1, 1]])}
    for k in kinds:
        total = ov.gate_matrix(k) @ total
        bare = rot[k] @ bare
    q, u = len(kinds) % 8, len(kinds) % 2
    scalar = np.exp(1j * np.pi * q / 4) * 2.0 ** (-u / 2) * 2.0 ** (-(len(kinds) - u) / 2)
    np.testing.assert_allclose(total, scalar * bare, atol=1e-12)

"""Plain complex128 state-vector oracle (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Slow and obvious on purpose:
every gate is one full sweep over the 2^n amplitudes, in the order of the gate list.

What each function follows
  * Amplitude order (§2, first equations): |psi> = (alpha_0 .. alpha_{2^n-1}); qubit k
    is bit k of the index, U on qubit k means I^{(n-k-1)} (x) U^k (x) I^{(k)}.
  * apply_1q: the pair update of §2 -- for every i with bit k = 0,
    (alpha_i, alpha_{i+2^k}) <- [[a, b], [c, d]] (alpha_i, alpha_{i+2^k}).
  * apply_cz: CZ is diagonal, -1 where both qubits are 1 (§2: the controlled gate acts
    like the single-qubit gate where the control is |1>).
  * projectors P_0 = |0><0|, P_1 = |1><1| (§2.1, Fig. 3 discussion) are one-qubit
    matrices applied by the same pair update.
  * initial state |0>^{(x) n} (§2), layer-0 H gates are ordinary gates here.
  * full_unitary: the Kronecker-product definition of §2, multiplied out (n <= 10).
  * branch_amplitudes: the decomposition CZ^{c,t} = P_0^c (x) I^t + P_1^c (x) Z^t (§2,
    Fig. 2 caption and Eq. 1): every CZ crossing the cut is replaced by the sum of its
    two product terms, so alpha_x = sum_l <x_A|A_l> <x_B|B_l> over l in {0,1}^t.
  * norm2 / sum_p2: sum |alpha|^2 and sum |alpha|^4 (Porter-Thomas statistic, §3
    final figure: for chaotic states N * sum p^2 -> 2).
  * branch_amplitudes_reduced: the same sum with the paper's two savings written out
    per branch: a crossing CZ after which neither qubit meets a non-diagonal gate only
    multiplies the output by (-1)^{x_a x_b} (the last layer's CZs change phases only,
    §3); a crossing CZ after which one qubit q stays a basis state is decomposed
    implicitly (§2.1, Fig. 4 discussion): the projector goes on q and its branch index
    equals x_q, so that half needs no sum over it.
  * amplitudes_inner_product: Task 2 by the inner product (§2 "Calculating one or a few
    amplitudes"): U = U2 U1, |psi> = U1 H^n |0>, |phi> = U2^dagger |x>, alpha_x =
    <phi|psi>.

Gate matrices (the paper names the gates but prints no matrices; reading):
  H = (1/sqrt2)[[1,1],[1,-1]], T = diag(1, e^{i pi/4}),
  X^{1/2} = 1/2 [[1+i, 1-i], [1-i, 1+i]], Y^{1/2} = 1/2 [[1+i, -1-i], [1+i, 1+i]]
  (principal square roots of Pauli X and Y), Z = diag(1, -1), CZ = diag(1,1,1,-1).
"""
import numpy as np

_SQ2 = np.sqrt(2.0)
_OMEGA = complex(np.cos(np.pi / 4), np.sin(np.pi / 4))

_MATS = {
    'H': np.array([[1, 1], [1, -1]], dtype=np.complex128) / _SQ2,
    'T': np.array([[1, 0], [0, _OMEGA]], dtype=np.complex128),
    'SX': 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128),
    'SY': 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128),
    'Z': np.array([[1, 0], [0, -1]], dtype=np.complex128),
    'P0': np.array([[1, 0], [0, 0]], dtype=np.complex128),
    'P1': np.array([[0, 0], [0, 1]], dtype=np.complex128),
}

ONE_QUBIT = ('H', 'T', 'SX', 'SY', 'Z', 'P0', 'P1')


def gate_matrix(kind):
    """2x2 complex128 matrix of a one-qubit gate kind."""
    return _MATS[kind].copy()


def zero_state(n):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_1q(psi, U, k):
    """Pair update of §2 on qubit k, in place."""
    n = psi.size.bit_length() - 1
    v = psi.reshape(1 << (n - k - 1), 2, 1 << k)
    a0 = v[:, 0, :].copy()
    a1 = v[:, 1, :].copy()
    v[:, 0, :] = U[0, 0] * a0 + U[0, 1] * a1
    v[:, 1, :] = U[1, 0] * a0 + U[1, 1] * a1
    return psi


def apply_cz(psi, a, b):
    """CZ on qubits a, b in place: negate the amplitudes whose bits a and b are both 1."""
    idx = np.arange(psi.size, dtype=np.int64)
    sel = ((idx >> a) & 1) & ((idx >> b) & 1)
    psi[sel == 1] *= -1
    return psi


def apply_gate(psi, gate, adjoint=False):
    kind, q0, q1, _layer = gate
    if kind == 'CZ':
        return apply_cz(psi, q0, q1)
    U = _MATS[kind]
    if adjoint:
        U = U.conj().T
    return apply_1q(psi, U, q0)


def run(n, gates, psi=None):
    """Apply gates (in list order) to psi, default |0...0>.  Returns psi (complex128)."""
    if psi is None:
        psi = zero_state(n)
    else:
        psi = np.array(psi, dtype=np.complex128, copy=True)
    for g in gates:
        apply_gate(psi, g)
    return psi


def run_adjoint(n, gates, psi):
    """Apply the inverse of the circuit: gates in reverse order, each conjugate-transposed."""
    psi = np.array(psi, dtype=np.complex128, copy=True)
    for g in reversed(gates):
        apply_gate(psi, g, adjoint=True)
    return psi


def embed_1q(n, U, k):
    """I^{(n-k-1)} (x) U (x) I^{(k)} as a dense 2^n x 2^n matrix (§2)."""
    return np.kron(np.kron(np.eye(1 << (n - k - 1)), U), np.eye(1 << k))


def embed_cz(n, a, b):
    d = np.ones(1 << n, dtype=np.complex128)
    for x in range(1 << n):
        if (x >> a) & 1 and (x >> b) & 1:
            d[x] = -1
    return np.diag(d)


def full_unitary(n, gates):
    """Brute-force product of the dense gate matrices, last gate leftmost (n <= 10)."""
    if n > 10:
        raise ValueError('full_unitary is for n <= 10')
    M = np.eye(1 << n, dtype=np.complex128)
    for kind, q0, q1, _l in gates:
        G = embed_cz(n, q0, q1) if kind == 'CZ' else embed_1q(n, _MATS[kind], q0)
        M = G @ M
    return M


def norm2(psi):
    return float(np.sum(np.abs(psi) ** 2))


def sum_p2(psi):
    return float(np.sum(np.abs(psi) ** 4))


def amplitudes(psi, bitstrings):
    return np.array([psi[int(x)] for x in bitstrings], dtype=np.complex128)


def _compress(x, qubits):
    """Bits of x at positions qubits[0], qubits[1], ... packed into 0, 1, ..."""
    out = 0
    for j, q in enumerate(qubits):
        out |= ((x >> q) & 1) << j
    return out


def split_halves(n, gates, half_a_mask):
    """Split a gate list at the cut.

    Returns (qa, qb, ga, gb, t): qa/qb the sorted qubits of halves A and B, ga/gb the
    per-half gate lists in local qubit numbering, with each crossing CZ j replaced by
    the placeholder ('CUT', local_qubit, j, layer) at its position; t = crossings."""
    qa = [q for q in range(n) if (half_a_mask >> q) & 1]
    qb = [q for q in range(n) if not (half_a_mask >> q) & 1]
    la = {q: i for i, q in enumerate(qa)}
    lb = {q: i for i, q in enumerate(qb)}
    ga, gb = [], []
    t = 0
    for kind, q0, q1, layer in gates:
        if kind == 'CZ':
            a_in = q0 in la
            b_in = q1 in la
            if a_in and b_in:
                ga.append(('CZ', la[q0], la[q1], layer))
            elif not a_in and not b_in:
                gb.append(('CZ', lb[q0], lb[q1], layer))
            else:
                qa_side = q0 if a_in else q1
                qb_side = q1 if a_in else q0
                ga.append(('CUT', la[qa_side], t, layer))
                gb.append(('CUT', lb[qb_side], t, layer))
                t += 1
        else:
            if q0 in la:
                ga.append((kind, la[q0], -1, layer))
            else:
                gb.append((kind, lb[q0], -1, layer))
    return qa, qb, ga, gb, t


def _branch_gates(half_gates, bits, side):
    """Instantiate the CUT placeholders of one half for branch bits l: half A gets the
    projector P_{l_j} on its qubit, half B gets Z^{l_j} (Z when l_j = 1, else nothing)."""
    out = []
    for g in half_gates:
        if g[0] != 'CUT':
            out.append(g)
            continue
        _k, q, j, layer = g
        lj = (bits >> j) & 1
        if side == 'A':
            out.append(('P1' if lj else 'P0', q, -1, layer))
        elif lj:
            out.append(('Z', q, -1, layer))
    return out


def branch_amplitudes(n, gates, half_a_mask, bitstrings):
    """alpha_x by the cut decomposition, summed over all 2^t branches in complex128."""
    qa, qb, ga, gb, t = split_halves(n, gates, half_a_mask)
    xa = [_compress(int(x), qa) for x in bitstrings]
    xb = [_compress(int(x), qb) for x in bitstrings]
    acc = np.zeros(len(bitstrings), dtype=np.complex128)
    for l in range(1 << t):
        A = run(len(qa), _branch_gates(ga, l, 'A'))
        B = run(len(qb), _branch_gates(gb, l, 'B'))
        acc += A[xa] * B[xb]
    return acc



def amplitudes_inner_product(n, gates, split_layer, bitstrings):
    """alpha_x = <phi_x|psi> with psi = (gates of layers <= split_layer) |0..0> (the H
    layer is layer 0) and phi_x = (gates of later layers)^dagger |x>."""
    g1 = [g for g in gates if g[3] <= split_layer]
    g2 = [g for g in gates if g[3] > split_layer]
    psi = run(n, g1)
    out = np.zeros(len(bitstrings), dtype=np.complex128)
    for j, x in enumerate(bitstrings):
        e = np.zeros(1 << n, dtype=np.complex128)
        e[int(x)] = 1.0
        phi = run_adjoint(n, g2, e)
        out[j] = np.vdot(phi, psi)  # conj(phi) . psi
    return out


NON_DIAGONAL = ('H', 'SX', 'SY')


def branch_amplitudes_reduced(n, gates, half_a_mask, bitstrings):
    """alpha_x with absorbed output signs and implicit decompositions (see the module
    docstring); one pair of half-state runs per branch of the remaining CZs."""
    in_a = [bool((half_a_mask >> q) & 1) for q in range(n)]
    last_nd = [-1] * n
    for i, (kind, q0, _q1, _l) in enumerate(gates):
        if kind in NON_DIAGONAL:
            last_nd[q0] = i
    roles = []  # per crossing CZ: ('full' | 'sign' | 'implicit_a' | 'implicit_b', qa, qb)
    for i, (kind, q0, q1, _l) in enumerate(gates):
        if kind == 'CZ' and in_a[q0] != in_a[q1]:
            qa, qb = (q0, q1) if in_a[q0] else (q1, q0)
            quiet_a, quiet_b = last_nd[qa] < i, last_nd[qb] < i
            role = 'sign' if quiet_a and quiet_b else 'implicit_a' if quiet_a else 'implicit_b' if quiet_b \
                else 'full'
            roles.append((role, qa, qb))
    qa_list, qb_list, ga, gb, t = split_halves(n, gates, half_a_mask)
    full = [j for j, r in enumerate(roles) if r[0] == 'full']
    out = np.zeros(len(bitstrings), dtype=np.complex128)
    for k, x in enumerate(bitstrings):
        x = int(x)
        sign = 1.0
        for role, qa, qb in roles:
            if role == 'sign' and (x >> qa) & 1 and (x >> qb) & 1:
                sign = -sign
        xa = _compress(x, qa_list)
        xb = _compress(x, qb_list)
        acc = 0.0 + 0.0j
        for lf in range(1 << len(full)):
            # branch index of every crossing CZ: summed (full), fixed by x (implicit)
            def half(side, gl):
                res = []
                for g in gl:
                    if g[0] != 'CUT':
                        res.append(g)
                        continue
                    _k, q, j, layer = g
                    role, qa, qb = roles[j]
                    if role == 'sign':
                        continue
                    if role == 'full':
                        lj = (lf >> full.index(j)) & 1
                        proj_side = 'A'
                    elif role == 'implicit_a':   # projector on qa, l = x_qa: A drops it
                        lj = (x >> qa) & 1
                        proj_side = 'A'
                    else:                       # projector on qb, l = x_qb: B drops it
                        lj = (x >> qb) & 1
                        proj_side = 'B'
                    if side == proj_side:
                        if role == 'full':
                            res.append(('P1' if lj else 'P0', q, -1, layer))
                    elif lj:
                        res.append(('Z', q, -1, layer))
                return res
            A = run(len(qa_list), half('A', ga))
            B = run(len(qb_list), half('B', gb))
            acc += A[xa] * B[xb]
        out[k] = sign * acc
    return out

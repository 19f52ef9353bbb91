"""Independent re-implementation of the random lattice circuit rules.

TEST INFRASTRUCTURE ONLY (see the package docstring).  This is the oracle's own
generator; tests assert that the library's generator emits exactly the same gate
list.  Nothing here is shared with the library.

Source of the rules
  * §2 (after Fig. 2): the gates are H, X^{1/2}, Y^{1/2}, T and CZ; CZ acts only on
    lattice neighbours and the CZ positions of each layer are fixed.
  * §1, footnote on depth: the layer of H gates is layer 0 and is not counted in the
    depth, so depth d means layers 1..d after layer 0.
  The paper does not print the CZ patterns (their figures are missing) nor the rule
  for choosing single-qubit gates.  The readings used here are:
  * 8 CZ patterns used cyclically.  A horizontal bond (r,c)-(r,c+1) belongs to class
    (c + 2*(r mod 2)) mod 4, a vertical bond (r,c)-(r+1,c) to class
    (r + 2*(c mod 2)) mod 4; layer l uses pattern (l-1) mod 8 of the list
    [H0, V0, H1, V1, H2, V2, H3, V3].  Bonds touching a removed site are dropped.
  * In layer l a qubit that was in a CZ of layer l-1 and is in no CZ of layer l gets
    one gate out of {T, X^{1/2}, Y^{1/2}}, never the same as its previous
    single-qubit gate (the layer-0 H does not count).
  * RNG: SplitMix64 from the seed; layers ascending, qubits ascending, one draw per
    gate; candidates in the order [T, SX, SY] with the previous gate removed; the
    choice is candidates[draw % len(candidates)].
  * Within a layer: single-qubit gates (ascending qubit) first, then the CZs sorted
    by (smaller qubit, larger qubit) with q0 < q1.
  * Sites are numbered row-major over the kept sites (qubit q = running index).

Gate tuples are (kind, q0, q1, layer) with kind one of the strings
'H', 'T', 'SX', 'SY', 'CZ', 'P0', 'P1', 'Z'; q1 is -1 for one-qubit gates.
"""

_M64 = (1 << 64) - 1

# Integer codes of the C interface's gate kinds (an interchange format, used only to
# compare gate lists with the library's output).
KIND_CODE = {'H': 0, 'T': 1, 'SX': 2, 'SY': 3, 'CZ': 4, 'P0': 5, 'P1': 6, 'Z': 7}
CODE_KIND = {v: k for k, v in KIND_CODE.items()}


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma, then the
    variant-13 finaliser of MurmurHash3's fmix64 on the state."""

    def __init__(self, seed):
        self.state = seed & _M64

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)


def site_numbering(rows, cols, removed_mask):
    """Map (r, c) -> qubit index for the kept sites, row-major.  Bit r*cols+c of
    removed_mask marks a removed site."""
    index = {}
    q = 0
    for r in range(rows):
        for c in range(cols):
            if (removed_mask >> (r * cols + c)) & 1:
                continue
            index[(r, c)] = q
            q += 1
    return index


def cz_patterns(rows, cols, removed_mask):
    """The 8 CZ patterns [H0, V0, H1, V1, H2, V2, H3, V3] as lists of (q0, q1), q0 < q1,
    sorted."""
    idx = site_numbering(rows, cols, removed_mask)
    horiz = [[] for _ in range(4)]
    vert = [[] for _ in range(4)]
    for (r, c), a in idx.items():
        right = (r, c + 1)
        if c + 1 < cols and right in idx:
            horiz[(c + 2 * (r % 2)) % 4].append((a, idx[right]))
        down = (r + 1, c)
        if r + 1 < rows and down in idx:
            vert[(r + 2 * (c % 2)) % 4].append((a, idx[down]))
    pats = []
    for h in range(4):
        pats.append(sorted((min(p), max(p)) for p in horiz[h]))
        pats.append(sorted((min(p), max(p)) for p in vert[h]))
    return pats


def generate(rows, cols, removed_mask, depth, seed):
    """Return (n_qubits, gates) for the lattice circuit of the given depth and seed."""
    idx = site_numbering(rows, cols, removed_mask)
    n = len(idx)
    pats = cz_patterns(rows, cols, removed_mask)
    rng = SplitMix64(seed)
    gates = [('H', q, -1, 0) for q in range(n)]
    previous = [None] * n
    in_prev_layer = set()
    for layer in range(1, depth + 1):
        pairs = pats[(layer - 1) % 8]
        in_layer = set()
        for a, b in pairs:
            in_layer.add(a)
            in_layer.add(b)
        for q in range(n):
            if q in in_prev_layer and q not in in_layer:
                draw = rng.next()
                cand = [g for g in ('T', 'SX', 'SY') if g != previous[q]]
                g = cand[draw % len(cand)]
                previous[q] = g
                gates.append((g, q, -1, layer))
        for a, b in pairs:
            gates.append(('CZ', a, b, layer))
        in_prev_layer = in_layer
    return n, gates


def to_codes(gates):
    """Gate tuples -> list of (kind_code, q0, q1, layer); q1 is 0 for one-qubit gates,
    the value the C interface stores in its unused field."""
    return [(KIND_CODE[k], a, (b if b >= 0 else 0), l) for (k, a, b, l) in gates]


def cut_crossings(gates, half_a_mask):
    """Indices (into gates) of the CZs with exactly one qubit in half A."""
    out = []
    for i, (k, a, b, _l) in enumerate(gates):
        if k == 'CZ':
            ina = (half_a_mask >> a) & 1
            inb = (half_a_mask >> b) & 1
            if ina != inb:
                out.append(i)
    return out

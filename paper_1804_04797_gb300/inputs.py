"""Seeded synthetic workloads shared by the tests, smoke() and bench.py.

This module holds no arithmetic of the method: it only names the lattice circuits the
paper's experiments are built from (2D lattices, §2 and §3) at the sizes this library
targets, the uneven batch, the cut of the amplitude task, and seeded bitstrings.  The
random numbers it draws (bitstrings, batch sizes) come from SplitMix64, a published
counter-free generator (Steele, Lea, Flood 2014), implemented here on its own.
"""
from dataclasses import dataclass

_M64 = (1 << 64) - 1

#: seed offset of the batched circuits (project constant)
BATCH_SEED = 180404797


def _splitmix(seed):
    s = seed & _M64
    while True:
        s = (s + 0x9E3779B97F4A7C15) & _M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        yield z ^ (z >> 31)


@dataclass(frozen=True)
class Lattice:
    """An R x C lattice circuit: removed_mask bit r*cols+c drops site (r, c)."""
    rows: int
    cols: int
    removed_mask: int
    depth: int
    seed: int

    @property
    def n_qubits(self):
        return self.rows * self.cols - bin(self.removed_mask).count('1')


def site_bit(rows, cols, r, c):
    return 1 << (r * cols + c)


#: 16 qubits, 4x4, depth 10 -- the small parity case
C16 = Lattice(4, 4, 0, 10, 0)
#: 30 qubits, 5x6, depth 20
C30 = Lattice(5, 6, 0, 20, 0)
#: 34 qubits, 6x6 without corners (0,0) and (5,5), depth 30 -- the headline workload
C34 = Lattice(6, 6, site_bit(6, 6, 0, 0) | site_bit(6, 6, 5, 5), 30, 0)
#: amplitude task: 42 qubits, 6x7, depth 10, cut between rows 2 and 3
C42 = Lattice(6, 7, 0, 10, 0)
C42_HALF_A = (1 << 21) - 1
#: full-state cross-check of the amplitude task: 28 qubits, 4x7, depth 10, cut rows 1|2
C28 = Lattice(4, 7, 0, 10, 0)
C28_HALF_A = (1 << 14) - 1


def lattice_for(n_rows, n_cols, depth, seed=0, removed=()):
    mask = 0
    for (r, c) in removed:
        mask |= site_bit(n_rows, n_cols, r, c)
    return Lattice(n_rows, n_cols, mask, depth, seed)


def batch_lattice(n, depth, seed):
    """Uneven-batch lattice for n qubits (8..28): 4 rows x ceil(n/4) columns, all sites
    of the first floor(n/4) columns plus the first (n mod 4) rows of the last column."""
    cols = (n + 3) // 4
    full, extra = n // 4, n % 4
    mask = 0
    for r in range(4):
        for c in range(cols):
            if not (c < full or (c == full and r < extra)):
                mask |= site_bit(4, cols, r, c)
    return Lattice(4, cols, mask, depth, seed)


def batch(count=512, seed=BATCH_SEED, n_min=16, n_max=24):
    """The uneven batch: n uniform in n_min..n_max (16..24), depth uniform in 10..24 (n
    drawn first, then depth, from one SplitMix64(seed)); circuit i uses generator seed
    seed + i."""
    g = _splitmix(seed)
    out = []
    for i in range(count):
        n = n_min + next(g) % (n_max - n_min + 1)
        d = 10 + next(g) % 15
        out.append(batch_lattice(n, d, seed + i))
    return out


def bitstrings(n_qubits, count, seed=2):
    """count seeded bitstrings of n_qubits bits (bit q = outcome of qubit q)."""
    g = _splitmix(seed)
    mask = (1 << n_qubits) - 1 if n_qubits < 64 else _M64
    return [next(g) & mask for _ in range(count)]


def sample_indices(n_qubits, count, seed=1):
    """count seeded amplitude indices (for sampled probabilities)."""
    return bitstrings(n_qubits, count, seed)

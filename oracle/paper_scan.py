"""The paper's own enumeration, restated in plain Python for tiny depths.

TEST INFRASTRUCTURE: see the package docstring.

Sec. "Implementation" renders by scanning every index n of the unpruned
m-ary tree at depth d, turning n into a string of d base-m digits (each digit
plus one, so that 0 stays free for the identity), and keeping the string only
if a run of the indexed Cayley table (Sec. "Cayley Multiplication Tables")
never reaches the crash state 0.  The string is read right to left: its last
character is the first letter applied.  This module writes that procedure out
from its description; it is independent of the C oracle's closed-form decode
and is used to pin it.
"""
from typing import Iterator, List, Sequence, Tuple

# Indexed Cayley table of the once-punctured-torus group (Sec. "Cayley
# Multiplication Tables"): rows = current state, columns = next symbol,
# symbols 1..4 = a, b, A, B, 0 = identity / crash.  Loaded from the golden
# fixture by the tests; repeated here as data for the scan.
T11_INDEXED = (
    (0, 1, 2, 3, 4),
    (1, 1, 2, 0, 4),
    (2, 1, 2, 3, 0),
    (3, 0, 2, 3, 4),
    (4, 1, 0, 3, 4),
)

LETTERS = "abAB"  # symbol k+1 <-> letter LETTERS[k]


def digit_string(n: int, m: int, d: int) -> List[int]:
    """The d low base-m digits of n, most significant first, each plus one.
    Defined for 0 <= n < m^d (larger n is out of range here)."""
    if not 0 <= n < m ** d:
        raise ValueError("index outside the depth-d tree")
    out = []
    for _ in range(d):
        out.append(n % m + 1)
        n //= m
    return out[::-1]


def table_run(symbols: Sequence[int], table) -> Tuple[int, List[int]]:
    """Run the indexed table over the symbols read right to left, starting in
    state 0.  Returns (1, states) for a regular word, (0, states) when a crash
    state is met (the run stops there) and (0, []) for the empty word."""
    if len(symbols) == 0:
        return 0, []
    state, states = 0, []
    for sym in reversed(symbols):
        state = table[state][sym]
        states.append(state)
        if state == 0:
            return 0, states
    return 1, states


def reduced_words_by_scan(d: int, table=T11_INDEXED, m: int = 4) -> Iterator[Tuple[int, List[int]]]:
    """(n, letter codes w_1..w_d) for every index n of the unpruned tree whose
    string survives the table run, in increasing n.  Letter code = symbol - 1."""
    for n in range(m ** d):
        s = digit_string(n, m, d)
        ok, _ = table_run(s, table)
        if ok:
            yield n, [c - 1 for c in s]


def mobius(mat, z: complex) -> complex:
    (p, q), (r, s) = mat
    return (p * z + q) / (r * z + s)


def word_value(gens, seeds, word: Sequence[int]) -> complex:
    """Orbit of seed[w_d] under w_d, w_{d-1}, ..., w_1 (right to left)."""
    z = seeds[word[-1]]
    for x in reversed(word):
        z = mobius(gens[x], z)
    return z

"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each one checks it
against a worked example printed in the paper (golden fixtures), a brute-force
enumeration written from the paper's description, a closed form, an invariant
of the group, or an independent library computation (numpy matrix products).
"""
import cmath

import numpy as np
import pytest

import klsynth
import oracle
from oracle import paper_scan
from conftest import golden_table, read_golden

GASKET = (2 + 0j, 2 + 0j)
NEAR_CUSP = (1.91 + 0.05j, 1.91 + 0.05j)
FUCHSIAN = (3 + 0j, 3 + 0j)
TRACE_PAIRS = [GASKET, NEAR_CUSP, FUCHSIAN] + [
    (g.ta, g.tb) for g, _ in klsynth.draw_groups(klsynth.BATCH_SEED, 6)]


def mats(ta, tb):
    g, s = oracle.group(ta, tb)
    return oracle.as_matrices(g), oracle.as_points(s), g, s


def mob(M, z):
    return (M[0, 0] * z + M[0, 1]) / (M[1, 0] * z + M[1, 1])


# --------------------------------------------------------------------------
# seeded sampler

def test_splitmix64_reference_vector():
    seed, outs = read_golden("splitmix64.txt")[0].split("|")
    want = [int(t) for t in outs.split()]
    rng = klsynth.SplitMix64(int(seed))
    assert [rng.next() for _ in want] == want
    assert [int(x) for x in klsynth.splitmix64_array(int(seed), len(want))] == want


# --------------------------------------------------------------------------
# tables and the crash rule (Sec. "Once-punctured torus groups", "Cayley
# Multiplication Tables")

def test_indexed_table_matches_letter_table_and_inverse_pairs():
    idx = golden_table("t11_indexed_cayley.txt")
    assert [list(r) for r in paper_scan.T11_INDEXED] == idx
    rows = read_golden("t11_letter_table.txt")
    head = rows[0].split()
    names = {"I": 0, "a": 1, "b": 2, "A": 3, "B": 4}
    for ln in rows[1:]:
        toks = ln.split()
        r = names[toks[0]]
        for c, ent in zip(head, toks[1:]):
            want = 0 if ent == "I" and c != "I" else names[ent] if ent != "I" else 0
            if r == 0:
                want = names[c]
            assert idx[r][names[c]] == want, (toks[0], c)
    # crash entries are exactly the inverse pairs inv(x) = (x + 2) mod 4 on codes
    for r in range(1, 5):
        for c in range(1, 5):
            assert (idx[r][c] == 0) == (((r - 1) + 2) % 4 == c - 1)


@pytest.mark.parametrize("line", read_golden("table_runs.txt"))
def test_worked_table_runs(line):
    name, syms, want, states = [t.strip() for t in line.split("|")]
    table = golden_table("t11_indexed_cayley.txt" if name == "t11" else "klein4_indexed_cayley.txt")
    symbols = [] if syms == "-" else [int(ch) for ch in syms]
    ok, seen = paper_scan.table_run(symbols, table)
    assert ok == int(want)
    assert seen == ([] if states == "-" else [int(t) for t in states.split()])


# --------------------------------------------------------------------------
# index decode (Sec. "The revised deterministic approach", "Implementation")

@pytest.mark.parametrize("d", range(1, 9))
def test_scan_survivor_count(d):
    n = sum(1 for _ in paper_scan.reduced_words_by_scan(d))
    assert n == 4 * 3 ** (d - 1) == oracle.word_count(d)


@pytest.mark.parametrize("d", range(1, 9))
def test_decode_is_the_rank_in_the_paper_scan(d):
    """The closed-form decode equals the order in which the base-4 scan filtered
    by the indexed table meets reduced words: same set, same order."""
    scanned = np.array([w for _, w in paper_scan.reduced_words_by_scan(d)], dtype=np.uint8)
    decoded = oracle.decode(d, np.arange(oracle.word_count(d), dtype=np.uint64))
    assert np.array_equal(scanned, decoded)


def test_decode_edges():
    assert oracle.word_count(0) == 0
    assert oracle.word_count(40) == 4 * 3 ** 39
    assert oracle.word_count(41) == 0            # overflows 64 bits
    with pytest.raises(IndexError):
        oracle.decode(5, [oracle.word_count(5)])
    d = 40
    last = oracle.decode(d, [oracle.word_count(d) - 1])[0]
    assert list(last) == [3] * d                 # the last word is B^d
    first = oracle.decode(d, [0])[0]
    assert list(first) == [0] * d                # the first word is a^d
    # a large index: reduced, and re-encoded to itself
    i = 4 * 3 ** 39 - 123456789
    w = oracle.decode(d, [i])[0]
    assert all((int(w[k]) + 2) % 4 != int(w[k + 1]) for k in range(d - 1))
    rank = int(w[0])
    for k in range(1, d):
        allowed = [x for x in range(4) if x != (int(w[k - 1]) + 2) % 4]
        rank = rank * 3 + allowed.index(int(w[k]))
    assert rank == i


# --------------------------------------------------------------------------
# generators (Grandma's recipe) and seeds

@pytest.mark.parametrize("ta,tb", TRACE_PAIRS)
def test_grandma_invariants(ta, tb):
    G, _, _, _ = mats(ta, tb)
    a, b, A, B = G
    assert abs(np.trace(a) - ta) < 1e-13
    assert abs(np.trace(b) - tb) < 1e-13
    for M in G:
        assert abs(np.linalg.det(M) - 1) < 1e-13
    assert np.allclose(a @ A, np.eye(2), atol=1e-13)
    assert np.allclose(b @ B, np.eye(2), atol=1e-13)
    assert abs(np.trace(a @ b @ A @ B) + 2) < 1e-12
    # tr(ab) is the root of x^2 - ta tb x + ta^2 + tb^2 = 0
    tab = np.trace(a @ b)
    assert abs(tab * tab - ta * tb * tab + ta * ta + tb * tb) < 1e-12 * max(1, abs(tab) ** 2)


def test_grandma_gasket_closed_form():
    """ta = tb = 2 gives the Apollonian-gasket group a = [[1, 0], [-2i, 1]],
    b = [[1 - i, 1], [1, 1 + i]] (tab = 2 - 2i)."""
    G, seeds, _, _ = mats(*GASKET)
    assert np.allclose(G[0], [[1, 0], [-2j, 1]], atol=1e-15, rtol=0)
    assert np.allclose(G[1], [[1 - 1j, 1], [1, 1 + 1j]], atol=1e-15, rtol=0)
    assert abs(np.trace(G[0] @ G[1]) - (2 - 2j)) < 1e-15
    # parabolic generators: a and A fix 0, b and B fix -i
    assert np.allclose(seeds, [0, -1j, 0, -1j], atol=1e-15)


def test_fuchsian_recipe_is_unitary_on_the_disc():
    """Real traces with ta^2 tb^2 >= 4 (ta^2 + tb^2) give a real tab, and both
    generators of the form [[u, v], [conj v, conj u]] preserve the unit circle."""
    G, _, _, _ = mats(*FUCHSIAN)
    for M in G:
        assert abs(M[0, 0] - np.conj(M[1, 1])) < 1e-14
        assert abs(M[0, 1] - np.conj(M[1, 0])) < 1e-14


@pytest.mark.parametrize("ta,tb", TRACE_PAIRS)
def test_seeds_are_attracting_fixed_points(ta, tb):
    G, seeds, _, _ = mats(ta, tb)
    for M, z in zip(G, seeds):
        assert abs(mob(M, z) - z) < 1e-12 * max(1, abs(z))
        p, q, r, s = M[0, 0], M[0, 1], M[1, 0], M[1, 1]
        roots = np.roots([r, s - p, -q])
        other = roots[np.argmax(np.abs(roots - z))]
        if abs(other - z) < 1e-6:   # parabolic: a double fixed point
            assert abs((p + s) ** 2 - 4) < 1e-12
            continue
        # |M'(z)| = 1/|rz + s|^2: the seed contracts at least as much as the other root
        assert abs(r * z + s) >= abs(r * other + s) - 1e-12


# --------------------------------------------------------------------------
# word values (Sec. "Introduction": orbit, reading order, word value)

def test_orbit_order_of_the_paper_example():
    word, applied = [t.strip() for t in read_golden("orbit_order.txt")[0].split("|")]
    codes = {"a": 0, "b": 1, "A": 2, "B": 3}
    for ta, tb in (NEAR_CUSP, TRACE_PAIRS[4]):
        G, seeds, g, s = mats(ta, tb)
        letters = [codes[ch] for ch in word]
        # locate abA by its index (rank of a reduced word)
        idx = letters[0]
        for k in range(1, len(letters)):
            allowed = [x for x in range(4) if x != (letters[k - 1] + 2) % 4]
            idx = idx * 3 + allowed.index(letters[k])
        assert list(oracle.decode(3, [idx])[0]) == letters
        z = seeds[codes[applied.split()[0]]]
        for ch in applied.split():
            z = mob(G[codes[ch]], z)
        got = oracle.evaluate(g, s, 3, [idx])[0]
        assert abs(got - z) < 1e-13 * max(1, abs(z))
        # and not the other reading order
        zr = seeds[codes[applied.split()[0]]]
        for ch in reversed(applied.split()):
            zr = mob(G[codes[ch]], zr)
        assert abs(got - zr) > 1e-6


@pytest.mark.parametrize("ta,tb,d", [(*GASKET, 12), (*NEAR_CUSP, 14), (*TRACE_PAIRS[5], 16)])
def test_word_value_equals_matrix_product(ta, tb, d):
    """Sequential point maps equal one map by the product matrix (numpy matmul,
    a different association) within rounding; every product has det 1."""
    G, seeds, g, s = mats(ta, tb)
    idx = klsynth.index_sample(7, 300, d)
    vals = oracle.evaluate(g, s, d, idx)
    words = oracle.decode(d, idx)
    for w, v in zip(words, vals):
        M = np.eye(2, dtype=complex)
        for x in w:
            M = M @ G[int(x)]
        scale = np.abs(M).max() ** 2
        assert abs(np.linalg.det(M) - 1) < 1e-13 * scale
        want = mob(M, seeds[int(w[-1])])
        assert abs(v - want) < 1e-9 * max(1, abs(want)), (w, v, want)


def test_fuchsian_limit_points_on_the_unit_circle():
    _, _, g, s = mats(*FUCHSIAN)
    d = 8
    vals = oracle.evaluate(g, s, d, np.arange(oracle.word_count(d), dtype=np.uint64))
    assert np.max(np.abs(np.abs(vals) - 1)) < 1e-12


# --------------------------------------------------------------------------
# rendering

def brute_render(G, seeds, d, window, W, H):
    """Paper-order scan of all 4^d strings, Python complex arithmetic, floor binning."""
    x0, x1, y0, y1 = window
    img = np.zeros((H, W), dtype=np.int64)
    dropped = 0
    for _, w in paper_scan.reduced_words_by_scan(d):
        z = paper_scan.word_value(G, seeds, w)
        u = (z.real - x0) * (W / (x1 - x0))
        v = (y1 - z.imag) * (H / (y1 - y0))
        if 0 <= u < W and 0 <= v < H:
            img[int(np.floor(v)), int(np.floor(u))] += 1
        else:
            dropped += 1
    return img, dropped


@pytest.mark.parametrize("ta,tb,d", [(*TRACE_PAIRS[3], 6), (*NEAR_CUSP, 6), (*GASKET, 5)])
def test_render_matches_brute_force_scan(ta, tb, d):
    G, seeds, g, s = mats(ta, tb)
    window = (-1.37, 1.41, -1.29, 1.33)   # no exact grid hits of rational points
    img, dropped = brute_render(G, seeds, d, window, 64, 48)
    for mode in ("tree", "indexed"):
        r = oracle.render(g, s, d, window, 64, 48, mode=mode, threads=3)
        assert np.array_equal(r.image.astype(np.int64), img)
        assert r.dropped == dropped
        assert r.in_window + r.dropped == oracle.word_count(d)


@pytest.mark.parametrize("ta,tb,d", [(*GASKET, 9), (*NEAR_CUSP, 8), (*TRACE_PAIRS[2], 7)])
def test_tree_walk_is_bitwise_the_per_word_definition(ta, tb, d):
    """With a half-pixel edge band every word near the window is logged with its
    index and pixel coordinates: both enumerations must log identical pairs."""
    _, _, g, s = mats(ta, tb)
    window = (-2.0, 2.0, -2.0, 2.0)
    a = oracle.render(g, s, d, window, 256, 256, mode="indexed", eta=0.5, edge_cap=1 << 20)
    b = oracle.render(g, s, d, window, 256, 256, mode="tree", threads=4, eta=0.5, edge_cap=1 << 20)
    assert a.edge_total == b.edge_total > 0.5 * oracle.word_count(d) * (a.in_window / oracle.word_count(d))
    oa, ob = np.argsort(a.edge_idx), np.argsort(b.edge_idx)
    assert np.array_equal(a.edge_idx[oa], b.edge_idx[ob])
    assert np.array_equal(a.edge_uv[oa], b.edge_uv[ob])          # bitwise
    assert np.array_equal(a.image, b.image)
    # the logged coordinates are the word values of those indices
    z = oracle.evaluate(g, s, d, a.edge_idx[oa][:500])
    u = (z.real + 2.0) * 64.0
    v = (2.0 - z.imag) * 64.0
    assert np.array_equal(u, a.edge_uv[oa][:500, 0]) and np.array_equal(v, a.edge_uv[oa][:500, 1])


def test_gasket_config_words_all_in_window():
    c = klsynth.C1
    g, s = oracle.group(c.group.ta, c.group.tb)
    r = oracle.render(g, s, c.depth, c.window, c.width, c.height, threads=4)
    assert r.dropped == 0 and r.in_window == 78732 == int(r.image.sum())
    # z -> -conj(z) conjugates a to itself and b to B (and fixes the seeds
    # 0 and -i), so the multiset of word values is mirror-symmetric about the
    # imaginary axis; only words on the axis itself (pixel edge between
    # columns 511 and 512) may fall on one side.
    img = r.image.astype(np.int64)
    assert np.array_equal(img[:, :511], img[:, 513:][:, ::-1])


@pytest.mark.parametrize("ta,tb,d", [(*GASKET, 5), (*NEAR_CUSP, 5)])
def test_tiling_render_matches_brute_force_scan_over_all_lengths(ta, tb, d):
    """Tiling mode draws every node of the tree: the paper's scan at every
    length 1 .. d, each word at its own value; 2 (3^d - 1) nodes in all."""
    G, seeds, g, s = mats(ta, tb)
    window = (-1.37, 1.41, -1.29, 1.33)
    img = np.zeros((48, 64), dtype=np.int64)
    dropped = 0
    for k in range(1, d + 1):
        i, dr = brute_render(G, seeds, k, window, 64, 48)
        img += i
        dropped += dr
    r = oracle.render_tiling(g, s, d, window, 64, 48, threads=2)
    assert np.array_equal(r.image.astype(np.int64), img)
    assert r.dropped == dropped
    assert r.in_window + r.dropped == 2 * (3 ** d - 1)


# --------------------------------------------------------------------------
# general presentations: the paper's scan with the indexed table

# Klein four-group as Moebius maps of determinant one: a(z) = -z, b(z) = 1/z,
# ab(z) = -1/z (symbols 1, 2, 3 of the table fixture); each squares to -I.
KLEIN = [np.array([[1j, 0], [0, -1j]]), np.array([[0, 1j], [1j, 0]]),
         np.array([[0, -1 + 0j], [1 + 0j, 0]])]


def test_klein_generators_satisfy_the_table():
    """The fixture's products: a b = ab, a ab = b, b ab = a (up to sign), and
    every letter squares to the identity (the crash state)."""
    a, b, c = KLEIN
    I = np.eye(2)
    for x in KLEIN:
        assert np.allclose(x @ x, -I)
        assert np.isclose(np.linalg.det(x), 1)
    for x, y, z in [(a, b, c), (a, c, b), (b, c, a)]:
        assert np.allclose(x @ y, z) or np.allclose(x @ y, -z)


@pytest.mark.parametrize("d", range(1, 9))
def test_fsa_counts(d):
    t11 = golden_table("t11_indexed_cayley.txt")
    k4 = golden_table("klein4_indexed_cayley.txt")
    assert oracle.fsa_count(4, t11, d) == 4 * 3 ** (d - 1)
    assert oracle.fsa_count(3, k4, d) == 3 * 2 ** (d - 1)


def brute_render_table(G, seeds, table, m, d, window, W, H):
    x0, x1, y0, y1 = window
    img = np.zeros((H, W), dtype=np.int64)
    dropped = kept = 0
    for _, w in paper_scan.reduced_words_by_scan(d, table=table, m=m):
        kept += 1
        z = paper_scan.word_value(G, seeds, w)
        u = (z.real - x0) * (W / (x1 - x0))
        v = (y1 - z.imag) * (H / (y1 - y0))
        if 0 <= u < W and 0 <= v < H:
            img[int(np.floor(v)), int(np.floor(u))] += 1
        else:
            dropped += 1
    return img, dropped, kept


def test_fsa_render_klein_four_matches_the_scan():
    k4 = golden_table("klein4_indexed_cayley.txt")
    seeds = [0.31 + 0.17j, -0.43 + 0.29j, 0.12 - 0.61j]
    window = (-4.1, 3.9, -3.7, 4.3)
    img, dropped, kept = brute_render_table(KLEIN, seeds, k4, 3, 7, window, 80, 60)
    r = oracle.render_fsa(3, k4, KLEIN, seeds, 7, window, 80, 60)
    assert np.array_equal(r.image.astype(np.int64), img)
    assert r.dropped == dropped and r.in_window + r.dropped == kept == 3 * 2 ** 6


@pytest.mark.parametrize("ta,tb,d", [(*GASKET, 6), (*NEAR_CUSP, 5)])
def test_fsa_render_of_the_torus_table_matches_the_scan_and_the_limit_set(ta, tb, d):
    G, seeds, g, s = mats(ta, tb)
    t11 = golden_table("t11_indexed_cayley.txt")
    window = (-1.37, 1.41, -1.29, 1.33)
    img, dropped, kept = brute_render_table(G, seeds, t11, 4, d, window, 64, 48)
    r = oracle.render_fsa(4, t11, G, seeds, d, window, 64, 48)
    assert np.array_equal(r.image.astype(np.int64), img)
    assert r.dropped == dropped and kept == oracle.word_count(d)
    # the same words as the reduced-index render, with the same arithmetic
    ref = oracle.render(g, s, d, window, 64, 48, mode="indexed")
    assert np.array_equal(r.image, ref.image)


# --------------------------------------------------------------------------
# Maskit's slice (the group of the paper's example)

MASKIT_MU = -0.097 + 1.838j


@pytest.mark.parametrize("mu", [MASKIT_MU, 2j, 1.91 + 0.05j])
def test_maskit_group(mu):
    """a(z) = mu + 1/z and b(z) = z + 2 as det-1 matrices, tr(abAB) = -2,
    seeds fixed by their letters (b, B: by the commutator), a's attracting."""
    g, s = oracle.maskit(mu)
    a, b, A, B = oracle.as_matrices(g)
    rng = np.random.default_rng(3)
    for z in rng.normal(size=5) + 1j * rng.normal(size=5):
        assert np.isclose(mob(a, z), mu + 1 / z) and np.isclose(mob(b, z), z + 2)
    for m in (a, b, A, B):
        assert np.isclose(np.linalg.det(m), 1.0, atol=1e-14)
    assert np.allclose(a @ A, np.eye(2)) and np.allclose(b @ B, np.eye(2))
    K = a @ b @ A @ B
    assert abs(np.trace(K) + 2) < 1e-12
    pts = oracle.as_points(s)
    assert abs(mob(a, pts[0]) - pts[0]) < 1e-12 and abs(mob(A, pts[2]) - pts[2]) < 1e-12
    assert pts[1] == pts[3] and abs(mob(K, pts[1]) - pts[1]) < 1e-12
    # attracting (or neutral, when a is parabolic as at mu = 2i):
    # |a'(z)| = 1/|r z + s|^2 <= 1 at a's seed
    assert abs(a[1, 0] * pts[0] + a[1, 1]) >= 1.0 - 1e-12


# --------------------------------------------------------------------------
# multi-seed feeding

@pytest.mark.parametrize("ta,tb", [GASKET, NEAR_CUSP, FUCHSIAN] + TRACE_PAIRS[3:6])
def test_cusp_seeds(ta, tb):
    """The commutator's cyclic permutations are parabolic and fix their
    points; each permutation is the previous one conjugated by its first
    letter, so each point is the previous one's image under that letter's
    inverse: bABa = A (abAB) a fixes A(z0), ABab fixes B(z1), BabA fixes a(z2)."""
    G, seeds, g, s = mats(ta, tb)
    out = oracle.cusp_seeds(g)
    pts = [complex(out[2 * i], out[2 * i + 1]) for i in range(8)]
    assert np.allclose(pts[:4], seeds, rtol=1e-14, atol=1e-15)
    a, b, A, B = G
    words = [a @ b @ A @ B, b @ A @ B @ a, A @ B @ a @ b, B @ a @ b @ A]
    for K, z in zip(words, pts[4:]):
        assert abs(np.trace(K) + 2) < 1e-10 * max(1.0, np.abs(K).max() ** 2)
        assert abs(mob(K, z) - z) < 1e-7 * max(1.0, abs(z))
    for prev, nxt, inv in [(pts[4], pts[5], A), (pts[5], pts[6], B), (pts[6], pts[7], a)]:
        assert abs(mob(inv, prev) - nxt) < 1e-7 * max(1.0, abs(nxt))


@pytest.mark.parametrize("ta,tb,d", [(*GASKET, 5), (*NEAR_CUSP, 5)])
def test_multiseed_render_matches_the_scan(ta, tb, d):
    """Each reduced word drawn once per point of the list, its maps applied
    to that point (not to its first letter's seed)."""
    G, seeds, g, s = mats(ta, tb)
    out = oracle.cusp_seeds(g)
    pts = [complex(out[2 * i], out[2 * i + 1]) for i in range(8)]
    window = (-1.37, 1.41, -1.29, 1.33)
    img = np.zeros((48, 64), dtype=np.int64)
    dropped = 0
    for z in pts:
        i, dr = brute_render(G, [z] * 4, d, window, 64, 48)
        img += i
        dropped += dr
    r = oracle.render_multiseed(g, pts, d, window, 64, 48, threads=2)
    assert np.array_equal(r.image.astype(np.int64), img)
    assert r.dropped == dropped and r.in_window + r.dropped == 8 * oracle.word_count(d)


# --------------------------------------------------------------------------
# repetends (Sec. "The revised deterministic approach": near (nearly)
# parabolic points orbits run slower and slower; the book the paper builds on
# adds "repetends").  Reading: a repetend is a periodic tail t of an infinite
# word w t t t ..., whose limit point is w(fix t).  The parabolic tails are the
# cyclic permutations of the commutator abAB and of its inverse BAba.

PARABOLIC_TAILS = ["abAB", "bABa", "ABab", "BabA", "BAba", "AbaB", "baBA", "aBAb"]
CODE = {"a": 0, "b": 1, "A": 2, "B": 3}


def word_matrix(G, letters):
    M = np.eye(2, dtype=complex)
    for x in letters:
        M = M @ G[CODE[x]]
    return M


@pytest.mark.parametrize("ta,tb", [GASKET, NEAR_CUSP] + TRACE_PAIRS[3:5])
def test_repetend_points_are_the_commutator_fixed_points(ta, tb):
    """The 8 parabolic tails fix 4 distinct points, the last four points of
    the multi-seed list (a tail and its inverse share a fixed point); after
    any last letter w_d, each of the 4 points is the limit of a reduced
    continuation (a tail whose first letter is not the inverse of w_d)."""
    G, _, g, _ = mats(ta, tb)
    out = oracle.cusp_seeds(g)
    cusps = [complex(out[2 * i], out[2 * i + 1]) for i in range(4, 8)]
    for t in PARABOLIC_TAILS:
        T = word_matrix(G, t)
        assert abs(np.trace(T) + 2) < 1e-9 * max(1.0, np.abs(T).max() ** 2)
        d = [abs(mob(T, z) - z) / max(1.0, abs(z)) for z in cusps]
        assert min(d) < 1e-7, t
    for wd in "abAB":
        inv = {"a": "A", "A": "a", "b": "B", "B": "b"}[wd]
        reached = set()
        for t in PARABOLIC_TAILS:
            if t[0] != inv:
                T = word_matrix(G, t)
                reached.add(int(np.argmin([abs(mob(T, z) - z) for z in cusps])))
        assert reached == {0, 1, 2, 3}, wd


@pytest.mark.parametrize("ta,tb", [GASKET, NEAR_CUSP])
def test_parabolic_tails_converge_like_one_over_n(ta, tb):
    """w t^n (z) -> w(fix t) only like 1/n for a parabolic tail t (the slow
    orbits of the paper's remark), against geometric convergence for a
    loxodromic tail: the error falls about tenfold from n = 100 to 1000."""
    G, seeds, g, _ = mats(ta, tb)
    out = oracle.cusp_seeds(g)
    cusps = [complex(out[2 * i], out[2 * i + 1]) for i in range(4, 8)]
    W = word_matrix(G, "abaBA")   # any reduced head; its last letter A
    for t in ["baBA", "aBAb"]:     # tails allowed after A (first letter not a)
        T = word_matrix(G, t)
        fix = cusps[int(np.argmin([abs(mob(T, z) - z) for z in cusps]))]
        z = seeds[CODE[t[-1]]]
        err = {}
        for n in range(1, 1001):
            z = mob(T, z)
            if n in (100, 1000):
                err[n] = abs(mob(W, z) - mob(W, fix))
        assert 7.0 < err[100] / err[1000] < 13.0, (t, err)


def test_loxodromic_tail_converges_geometrically():
    """The contrast: a loxodromic generator's orbit reaches its attracting
    fixed point geometrically (a batch group, Re tr a > 2)."""
    ta, tb = TRACE_PAIRS[3]
    G, seeds, g, _ = mats(ta, tb)
    a = G[0]
    z, fix = 0.3 + 0.1j, seeds[0]
    errs = []
    for n in range(1, 41):
        z = mob(a, z)
        if n in (10, 20):
            errs.append(abs(z - fix))
    assert errs[1] < 1e-3 * errs[0]

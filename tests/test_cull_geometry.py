"""The geometry the culled render (kl_params.cull) rests on, checked against
the mathematics on the CPU (the kernels themselves are checked on the GPU,
bit for bit against the per-word render, in tests/test_gpu_cull.py).

* The pole-form map (u, v) = M (w_re, w_im) / |w|^2 + (ax, ay), w = v + gamma,
  sends the disk D(c, rho), |c + gamma| > rho, into the disk of center
  M (c + gamma) / q + (ax, ay) and radius |M| rho / q, q = |c + gamma|^2 - rho^2;
  the bound is attained when M is a similarity (square pixels).
* |M| = ((|(c1 + c4, c2 - c3)| + |(c1 - c4, c2 + c3)|) / 2 is the largest
  singular value of [[c1, c2], [c3, c4]].
* Aligned runs of 3^j consecutive suffix indices of one first letter hold
  the words that share all but their last j letters (one subtree), by the
  mixed-radix decode.
"""
import numpy as np
import pytest

import oracle


def pole_map(M, A, gamma, v):
    w = v + gamma
    n = np.abs(w) ** 2
    return (M[0, 0] * w.real + M[0, 1] * w.imag) / n + A[0], \
        (M[1, 0] * w.real + M[1, 1] * w.imag) / n + A[1]


def pixel_matrix(mbeta, sx, sy):
    """The real 2x2 matrix of the pole form in pixel units (mbeta = -beta)."""
    return np.array([[-sx * mbeta.real, -sx * mbeta.imag],
                     [sy * mbeta.imag, -sy * mbeta.real]])


def opnorm(M):
    c1, c2, c3, c4 = M[0, 0], M[0, 1], M[1, 0], M[1, 1]
    return 0.5 * (np.hypot(c1 + c4, c2 - c3) + np.hypot(c1 - c4, c2 + c3))


@pytest.mark.parametrize("seed", range(6))
def test_operator_norm_is_the_largest_singular_value(seed):
    rng = np.random.default_rng(seed)
    for _ in range(200):
        M = rng.normal(size=(2, 2)) * 10.0 ** rng.uniform(-3, 3)
        assert opnorm(M) == pytest.approx(np.linalg.norm(M, 2), rel=1e-12)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("square", [True, False])
def test_disk_image_bound(seed, square):
    rng = np.random.default_rng(100 + seed)
    for _ in range(40):
        gamma = complex(*rng.normal(size=2)) * 3.0
        mbeta = complex(*rng.normal(size=2)) * 10.0 ** rng.uniform(-4, 1)
        sx = 10.0 ** rng.uniform(2, 4)
        sy = sx if square else sx * rng.uniform(0.5, 2.0)
        M = pixel_matrix(mbeta, sx, sy)
        A = rng.normal(size=2) * 100.0
        c = complex(*rng.normal(size=2))
        c0 = c + gamma
        rho = abs(c0) * rng.uniform(0.01, 0.49)     # the test's |c + gamma| > 2 rho
        q = abs(c0) ** 2 - rho ** 2
        center = M @ np.array([c0.real, c0.imag]) / q + A
        radius = opnorm(M) * rho / q
        t = rng.uniform(0, 2 * np.pi, 4000)
        r = rho * np.sqrt(rng.uniform(0, 1, 4000))
        r[:1000] = rho                               # the boundary circle
        u, v = pole_map(M, A, gamma, c + r * np.exp(1j * t))
        dist = np.hypot(u - center[0], v - center[1])
        assert dist.max() <= radius * (1 + 1e-12) + 1e-9
        if square:
            assert dist[:1000].max() >= radius * (1 - 1e-3)


def test_disk_image_rejects_a_disk_over_the_pole():
    """A disk holding the pole has no bounded image: the closed form's q is
    then not positive (the kernels demand |c + gamma| > 2 rho)."""
    gamma, c, rho = 1.0 + 0.5j, -1.0 - 0.4j, 0.2
    assert abs(c + gamma) < rho
    assert abs(c + gamma) ** 2 - rho ** 2 < 0


@pytest.mark.parametrize("s", [4, 6, 7])
def test_aligned_suffix_runs_are_subtrees(s):
    words = oracle.decode(s, np.arange(oracle.word_count(s), dtype=np.uint64))
    per = 3 ** (s - 1)                                # suffixes per first letter
    for u in range(4):
        block = words[u * per:(u + 1) * per]
        assert (block[:, 0] == block[0, 0]).all()
        for j in range(0, s):
            size = 3 ** j
            runs = block.reshape(-1, size, s)
            # all but the last j letters agree within each run
            assert (runs[:, :, : s - j] == runs[:, :1, : s - j]).all()
            if j >= 1:
                # and each run is a whole subtree: its first free letter takes
                # all three values allowed after the shared letters
                for r in runs[:, :, s - j]:
                    assert len(set(r.tolist())) == 3

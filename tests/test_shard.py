"""The sharded render on CPU: the oracle's partition of the words by prefix
slot, pinned by what a partition must satisfy, and the multi-rank path of
bench.py (world size 2 over gloo): each rank renders its shard, one reduce
sums the uint32 images and counters onto rank 0, and the sum is the whole
render.  The library's argument checks for the shard fields need no GPU.

The words of the paper's method are independent of one another: each is
pulled out of its own integer (Sec. "The revised deterministic approach"),
so any split of the index set renders the same image once the parts are
added up.  The library splits by prefix slot (kl_params.shard_index /
shard_count, include/kl.h)."""
import ctypes
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import klsynth
import oracle

GROUPS = [(klsynth.GASKET.ta, klsynth.GASKET.tb), (klsynth.NEAR_CUSP.ta, klsynth.NEAR_CUSP.tb),
          (2.3 + 0.04j, 2.7 - 0.02j)]


def _whole(ta, tb, d, W=96, window=(-2.0, 2.0, -2.0, 2.0)):
    g, s = oracle.group(ta, tb)
    return g, s, oracle.render(g, s, d, window, W, W, mode="indexed")


@pytest.mark.parametrize("p", [1, 2, 3, 5, 7])
def test_prefix_slot_is_a_bijection_of_the_prefixes(p):
    """(w_p, r) numbers the 4 3^(p-1) reduced prefixes one to one: checked on
    all words of length p, where the word is its own prefix."""
    n = oracle.word_count(p)
    idx = np.arange(n, dtype=np.uint64)
    r = oracle.prefix_rank(p, p, idx)
    last = oracle.decode(p, idx)[:, p - 1].astype(np.uint64)
    assert int(r.max()) < 3 ** (p - 1)
    slots = last * np.uint64(3 ** (p - 1)) + r
    assert np.array_equal(np.sort(slots), np.arange(n, dtype=np.uint64))


def test_prefix_slot_reads_the_right_neighbour():
    """Spelled out on one prefix: w = a b A (codes 0 1 2, p = 3).  w_2 = b sits
    left of A, whose inverse a is banned: allowed b, A, B, so b has rank 0;
    w_1 = a sits left of b, inverse B banned: allowed a, b, A, rank 0.  So
    r = 0.  For w = B a b (3 0 1): w_2 = a left of b (B banned): a, b, A ->
    rank 0; w_1 = B left of a (A banned): a, b, B -> rank 2; r = 2 * 3^0 = 2."""
    def index_of(word):
        d = len(word)
        i = word[0]
        for k in range(1, d):
            ban = (word[k - 1] + 2) & 3
            allowed = [x for x in range(4) if x != ban]
            i = 3 * i + allowed.index(word[k])
        return i
    assert list(oracle.decode(3, [index_of([0, 1, 2])])[0]) == [0, 1, 2]
    assert int(oracle.prefix_rank(3, 3, [index_of([0, 1, 2])])[0]) == 0
    assert int(oracle.prefix_rank(3, 3, [index_of([3, 0, 1])])[0]) == 2
    # w = b B? not reduced; w = A b a (2 1 0): w_2 = b left of a (A banned):
    # a, b, B -> rank 1; w_1 = A left of b (B banned): a, b, A -> rank 2;
    # r = 1 * 3 + 2 = 5
    assert int(oracle.prefix_rank(3, 3, [index_of([2, 1, 0])])[0]) == 5


@pytest.mark.parametrize("d,p", [(7, 1), (7, 3), (7, 6), (8, 8), (9, 5)])
def test_words_of_one_prefix_stay_in_one_slot(d, p):
    """The 3^(d-p) words that share w_1 .. w_p (consecutive indices) share
    one prefix slot, so a shard never splits a prefix."""
    n = oracle.word_count(d)
    idx = np.arange(n, dtype=np.uint64)
    r = oracle.prefix_rank(d, p, idx).reshape(-1, 3 ** (d - p))
    assert (r == r[:, :1]).all()


@pytest.mark.parametrize("ta,tb", GROUPS)
@pytest.mark.parametrize("d,p,n", [(6, 3, 2), (7, 4, 3), (8, 5, 5), (7, 2, 4), (5, 5, 7),
                                   (1, 1, 3), (9, 8, 2)])
def test_shards_sum_to_the_whole_render(ta, tb, d, p, n):
    g, s, whole = _whole(ta, tb, d)
    total = np.zeros_like(whole.image)
    inw = drop = 0
    np3 = 3 ** (p - 1)
    for k in range(n):
        r = oracle.render_shard(g, s, d, (-2.0, 2.0, -2.0, 2.0), 96, 96, p, k, n)
        slots = (k + 1) * np3 // n - k * np3 // n
        assert r.in_window + r.dropped == 4 * 3 ** (d - p) * slots   # closed-form size
        total += r.image
        inw += r.in_window
        drop += r.dropped
    assert np.array_equal(total, whole.image)
    assert (inw, drop) == (whole.in_window, whole.dropped)


def test_shard_arguments_are_checked():
    g, s = oracle.group(2 + 0j, 2 + 0j)
    for bad in [(3, 2, 2), (3, 0, 0), (3, -1, 2), (0, 0, 1), (5, 0, 1)]:
        p, k, n = bad
        with pytest.raises(ValueError):
            oracle.render_shard(g, s, 4, (-2.0, 2.0, -2.0, 2.0), 8, 8, p, k, n)


# ---------------------------------------------------------------------------
# bench.py's multi-rank path, world size 2 over gloo

def _free_port():
    so = socket.socket()
    so.bind(("127.0.0.1", 0))
    port = so.getsockname()[1]
    so.close()
    return port


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ta, tb, d, p, W = klsynth.NEAR_CUSP.ta, klsynth.NEAR_CUSP.tb, 9, 6, 128
        f = bench.shard_fields(world, rank)
        assert f == {"shard_index": rank, "shard_count": world}
        g, s = oracle.group(ta, tb)
        part = oracle.render_shard(g, s, d, (-2.0, 2.0, -2.0, 2.0), W, W, p, f["shard_index"],
                                   f["shard_count"])
        image = torch.from_numpy(part.image.view(np.int32).copy())
        counters = torch.tensor([part.in_window, part.dropped, 0, 0], dtype=torch.int64)
        bench.make_image_sum(world)(image, counters)
        if rank == 0:
            out["image"] = image.numpy().view(np.uint32).copy()
            out["counters"] = counters.tolist()
        out[f"words{rank}"] = part.in_window + part.dropped
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_their_shards_into_the_whole_render():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    g, s, whole = _whole(klsynth.NEAR_CUSP.ta, klsynth.NEAR_CUSP.tb, 9, W=128)
    assert np.array_equal(res["image"], whole.image)
    assert res["counters"][:2] == [whole.in_window, whole.dropped]
    # every word in exactly one shard, the two shards within one prefix slot
    # (3^(9-6) * 4 = 108 words) of each other
    assert res["words0"] + res["words1"] == oracle.word_count(9)
    assert abs(res["words0"] - res["words1"]) <= 4 * 3 ** 3


# ---------------------------------------------------------------------------
# the library's checks of the shard fields (no device call is made)

@pytest.fixture(scope="module")
def kl():
    from paper_1709_08018_gb300 import build
    build.build()
    import paper_1709_08018_gb300 as kl
    return kl


def test_library_rejects_bad_shards_before_any_device_call(kl):
    L = kl.binding.lib()
    fake = 0x1000   # never dereferenced: the checks come first
    bad = [dict(shard_index=2, shard_count=2), dict(shard_index=5, shard_count=3),
           dict(shard_index=0, shard_count=2, mode=kl.TILING)]
    for f in bad:
        p = kl.params_init(2 + 0j, 2 + 0j, 12, 256, 256, (-1.5, 1.5, -1.5, 1.5), **f)
        ws = kl.workspace_bytes(p)
        st = L.kl_render(ctypes.byref(p), fake, fake, ctypes.c_void_p(1 << 20), max(ws, 256),
                         None)
        assert st == 1, f   # KL_EINVAL
    p = kl.params_init(2 + 0j, 2 + 0j, 14, 256, 256, (-1.5, 1.5, -1.5, 1.5), kl.MIXED,
                       shard_index=0, shard_count=2)
    h = ctypes.c_void_p()
    assert L.kl_batch_create((kl.Params * 1)(p), 1, ctypes.byref(h)) == 1
    assert L.kl_lod_label_bytes(ctypes.byref(p), 4, 8) == 0


def test_shard_leaves_the_workspace_size_alone(kl):
    p = kl.params_init(2 + 0j, 2 + 0j, 18, 4096, 4096, (-1.5, 1.5, -1.5, 1.5))
    q = kl.params_init(2 + 0j, 2 + 0j, 18, 4096, 4096, (-1.5, 1.5, -1.5, 1.5), shard_index=3,
                       shard_count=8)
    assert kl.workspace_bytes(p) == kl.workspace_bytes(q) > 0

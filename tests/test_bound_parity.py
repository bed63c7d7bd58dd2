"""Parity of the CUDA batched bounding kernel with the CPU oracle.

Every child bound (LB1 and LB2, forward and backward) must be bit-identical
to the oracle's from-scratch value; scheduled jobs must read -1.  Cases span
several warps and CTAs, ragged tails, both job-mask widths (n <= 32 and
n > 32), every m from 1 to 32, nodes of every depth (both forms of the
front/back computation), exhaustive node sets of tiny instances, the
degenerate depths, and sampled nodes of the full 4,194,304-node batch of the
20 x 20 bounding benchmark in the launch configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2012_09511_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2012_09511_gb300 import build
    build.build()
    from paper_2012_09511_gb300 import pfsp
    return pfsp


def _compare(pf, p, perm, d1, d2, threads=8):
    inst = pf.pfsp_load_instance(p)
    g1, g2 = pf.pfsp_bound_batch(inst, pf.PFSP_LB1 | pf.PFSP_LB2, perm, d1, d2)
    o1, o2 = orc.children_bounds_batch(p, perm, d1, d2, threads=threads)
    bad1 = np.argwhere(g1 != o1)
    bad2 = np.argwhere(g2 != o2)
    assert len(bad1) == 0, ("LB1 mismatch", bad1[:5], g1[tuple(bad1[0])], o1[tuple(bad1[0])])
    assert len(bad2) == 0, ("LB2 mismatch", bad2[:5], g2[tuple(bad2[0])], o2[tuple(bad2[0])])
    return g1, g2


@pytest.mark.parametrize("n,m,count", [
    (20, 20, 6000), (20, 10, 5000), (10, 5, 5000), (12, 20, 3000), (50, 5, 1500), (30, 10, 2000),
    (33, 7, 1500), (64, 4, 800), (32, 32, 600), (17, 3, 3001), (7, 2, 2000), (9, 1, 1000),
    (2, 3, 300), (1, 4, 50),
])
def test_random_nodes_bit_exact(pf, n, m, count):
    p = inputs.make_instance(n, m, 1000 + n * 64 + m)
    perm, d1, d2 = inputs.random_nodes(n, count, seed=n + m, dmax=min(10, n))
    _compare(pf, p, perm, d1, d2)


@pytest.mark.parametrize("n,m,count,dmax", [
    (40, 20, 2000, 10), (50, 17, 1500, 10), (64, 16, 800, 10),  # 64-bit masks, fronts by max-scans
    (50, 20, 1500, 45), (64, 20, 600, 60), (33, 25, 1000, 30),  # positions past 32 in both directions
    (20, 20, 6000, 20), (32, 32, 1500, 32), (24, 18, 3000, 24),  # deep and shallow nodes alike
])
def test_deep_nodes_and_many_machines_bit_exact(pf, n, m, count, dmax):
    # at 16 machines or more the kernel builds fronts and backs by max-scans
    # over the machines, one per scheduled job; nodes of every depth reach
    # the jobs held by the second register of each lane (positions >= 32)
    p = inputs.make_instance(n, m, 7000 + n * 64 + m)
    perm, d1, d2 = inputs.random_nodes(n, count, seed=3 * n + m, dmax=dmax)
    _compare(pf, p, perm, d1, d2)


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8])
def test_every_node_of_tiny_instances(pf, m):
    n = 5
    p = inputs.make_instance(n, m, 77 + m)
    perm, d1, d2 = inputs.all_nodes_small(n)
    _compare(pf, p, perm, d1, d2)


def test_degenerate_depths(pf):
    n, m = 20, 20
    p = inputs.make_instance(n, m, 5)
    rng = np.random.default_rng(0)
    perm = np.stack([rng.permutation(n) for _ in range(64)]).astype(np.uint8)
    # root, no children (d1 + d2 = n), leaf children (d1 + d2 = n - 1), one side empty
    d1 = np.array([0, 20, 10, 19, 0, 0, 18, 1] * 8, dtype=np.uint8)
    d2 = np.array([0, 0, 10, 0, 19, 20, 1, 0] * 8, dtype=np.uint8)
    g1, g2 = _compare(pf, p, perm, d1, d2)
    assert (g1[1] == -1).all() and (g2[5] == -1).all()
    # leaves: the bound of a complete schedule is its makespan
    full = np.concatenate([perm[3, :19], [perm[3, 19]]])
    assert g1[3, 0, perm[3, 19]] == g2[3, 0, perm[3, 19]] == orc.makespan(p, full)


def test_empty_batch_and_invalid_depths(pf):
    p = inputs.make_instance(8, 4, 1)
    inst = pf.pfsp_load_instance(p)
    g1, g2 = pf.pfsp_bound_batch(inst, 3, np.zeros((0, 8)), np.zeros(0), np.zeros(0))
    assert g1.shape == (0, 2, 8)
    with pytest.raises(pf.PfspError) as e:
        pf.pfsp_bound_batch(inst, 3, np.zeros((1, 8)) + np.arange(8), [5], [4])
    assert e.value.code == pf.PFSP_ERR_INVALID
    with pytest.raises(pf.PfspError):
        pf.pfsp_bound_batch(inst, 0, np.arange(8)[None], [1], [1])


def test_invalid_depths_found_in_large_batches(pf):
    # batches of a million nodes and more (four chunks of the host pipeline):
    # the host validates the depths while the first chunks run on the GPU, and
    # copies nothing back before the validation passes, so an invalid node is
    # refused wherever it sits (last chunk, first chunk) and the caller's
    # buffers stay as they were
    n, m, N = 12, 5, (1 << 20) + 333
    inst = pf.pfsp_load_instance(inputs.make_instance(n, m, 2))
    perm, d1, d2 = inputs.random_nodes(n, N, seed=3, dmax=5)
    for bad in (N - 1, 7):
        e1, e2 = d1.copy(), d2.copy()
        e1[bad], e2[bad] = 7, 6  # 13 > n
        h1 = np.full((N, 2, n), -7, dtype=np.int32)
        h2 = np.full((N, 2, n), -7, dtype=np.int32)
        with pytest.raises(pf.PfspError) as e:
            pf.pfsp_bound_batch(inst, 3, perm, e1, e2, lb1_out=h1, lb2_out=h2)
        assert e.value.code == pf.PFSP_ERR_INVALID and ("node %d" % bad) in str(e.value)
        assert (h1 == -7).all() and (h2 == -7).all()
    g1, _ = pf.pfsp_bound_batch(inst, pf.PFSP_LB1, perm, d1, d2)
    assert pf.pfsp_stats(inst)["bounded_children"] == int(2 * (n - d1.astype(np.int64) - d2).sum())
    assert ((g1 >= 0).sum(axis=2) == (n - d1.astype(np.int64) - d2)[:, None]).all()


def test_lb1_only_and_lb2_only(pf):
    n, m = 20, 20
    p = inputs.make_instance(n, m, 9)
    perm, d1, d2 = inputs.random_nodes(n, 3000, 4)
    inst = pf.pfsp_load_instance(p)
    a1, _ = pf.pfsp_bound_batch(inst, pf.PFSP_LB1, perm, d1, d2)
    _, b2 = pf.pfsp_bound_batch(inst, pf.PFSP_LB2, perm, d1, d2)
    o1, o2 = orc.children_bounds_batch(p, perm, d1, d2, threads=8)
    assert (a1 == o1).all() and (b2 == o2).all()


def test_device_entry_point_with_torch_buffers(pf):
    import torch
    n, m = 20, 20
    p = inputs.make_instance(n, m, 21)
    perm, d1, d2 = inputs.random_nodes(n, 4099, 8)
    inst = pf.pfsp_load_instance(p)
    dev = torch.device("cuda:0")
    tp = torch.from_numpy(perm).to(dev)
    t1 = torch.from_numpy(d1).to(dev)
    t2 = torch.from_numpy(d2).to(dev)
    o1 = torch.empty((4099, 2, n), dtype=torch.int32, device=dev)
    o2 = torch.empty_like(o1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pf.pfsp_bound_batch_dev(inst, 3, 4099, tp.data_ptr(), t1.data_ptr(), t2.data_ptr(), o1.data_ptr(),
                                o2.data_ptr(), s.cuda_stream)
    s.synchronize()
    r1, r2 = orc.children_bounds_batch(p, perm, d1, d2, threads=8)
    assert (o1.cpu().numpy() == r1).all() and (o2.cpu().numpy() == r2).all()


def test_full_benchmark_batch_sampled(pf):
    # the 20 x 20 bounding benchmark: 4,194,304 nodes, depths uniform in 0..10;
    # every output is checked for structure, a sample against the oracle.
    n, m, N = 20, 20, 4194304
    p = inputs.make_instance(n, m, 2020)
    perm, d1, d2 = inputs.random_nodes(n, N, seed=2020)
    inst = pf.pfsp_load_instance(p)
    g1, g2 = pf.pfsp_bound_batch(inst, 3, perm, d1, d2)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.integers(0, N, 3000), np.arange(64), np.arange(N - 64, N)])
    o1, o2 = orc.children_bounds_batch(p, perm[idx], d1[idx], d2[idx], threads=8)
    assert (g1[idx] == o1).all() and (g2[idx] == o2).all()
    # properties at every node: -1 exactly on scheduled jobs, LB1 <= LB2
    u = n - d1.astype(np.int64) - d2.astype(np.int64)
    assert ((g1 >= 0).sum(axis=2) == u[:, None]).all()
    assert (g2 >= g1).all()
    st = pf.pfsp_stats(inst)
    assert st["bounded_children"] == int(2 * u.sum())


def test_host_entry_point_chunks_match_one_launch(pf):
    # the host-pointer entry point bounds the batch in chunks on two streams;
    # its outputs must equal one launch of the device entry point everywhere,
    # and the oracle at the chunk boundaries and in the ragged tail
    import torch
    n, m = 14, 6
    N = 4 * 262144 + 777
    p = inputs.make_instance(n, m, 33)
    perm, d1, d2 = inputs.random_nodes(n, N, seed=5, dmax=6)
    inst = pf.pfsp_load_instance(p)
    h1, h2 = pf.pfsp_bound_batch(inst, 3, perm, d1, d2)
    dev = torch.device("cuda:0")
    o1 = torch.empty((N, 2, n), dtype=torch.int32, device=dev)
    o2 = torch.empty_like(o1)
    tp, t1, t2 = (torch.from_numpy(x).to(dev) for x in (perm, d1, d2))
    pf.pfsp_bound_batch_dev(inst, 3, N, tp.data_ptr(), t1.data_ptr(), t2.data_ptr(), o1.data_ptr(), o2.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert (h1 == o1.cpu().numpy()).all() and (h2 == o2.cpu().numpy()).all()
    idx = np.concatenate([np.arange(262136, 262152), np.arange(786424, 786440), np.arange(N - 40, N)])
    r1, r2 = orc.children_bounds_batch(p, perm[idx], d1[idx], d2[idx], threads=8)
    assert (h1[idx] == r1).all() and (h2[idx] == r2).all()
    lb1_only, none2 = pf.pfsp_bound_batch(inst, pf.PFSP_LB1, perm, d1, d2)
    assert none2 is None and (lb1_only == h1).all()


def test_host_entry_point_into_pinned_buffers(pf):
    # with page-locked output buffers, the chunks after the first two write
    # their results in place from the kernel instead of through device
    # buffers and copies: every value must still equal one launch of the
    # device entry point (both modes, two calls in a row), and a batch refused
    # for an invalid depth must leave the pinned buffers as they were
    import torch
    n, m = 14, 6
    N = 5 * 262144 + 999
    p = inputs.make_instance(n, m, 34)
    perm, d1, d2 = inputs.random_nodes(n, N, seed=6, dmax=6)
    inst = pf.pfsp_load_instance(p)
    dev = torch.device("cuda:0")
    o1 = torch.empty((N, 2, n), dtype=torch.int32, device=dev)
    o2 = torch.empty_like(o1)
    tp, t1, t2 = (torch.from_numpy(x).to(dev) for x in (perm, d1, d2))
    pf.pfsp_bound_batch_dev(inst, 3, N, tp.data_ptr(), t1.data_ptr(), t2.data_ptr(), o1.data_ptr(), o2.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    w1, w2 = o1.cpu().numpy(), o2.cpu().numpy()
    h1 = torch.full((N, 2, n), -7, dtype=torch.int32).pin_memory()
    h2 = torch.full((N, 2, n), -7, dtype=torch.int32).pin_memory()
    for _ in range(2):
        pf.pfsp_bound_batch(inst, 3, perm, d1, d2, lb1_out=h1.numpy(), lb2_out=h2.numpy())
        assert (h1.numpy() == w1).all() and (h2.numpy() == w2).all()
        h1.fill_(-7)
        h2.fill_(-7)
    _, only2 = pf.pfsp_bound_batch(inst, pf.PFSP_LB2, perm, d1, d2, lb2_out=h2.numpy())
    assert (only2 == w2).all()
    h2.fill_(-7)
    for bad in (N - 1, 5):
        e1 = d1.copy()
        e1[bad] = n  # d1 + d2 > n
        e2 = d2.copy()
        e2[bad] = 1
        with pytest.raises(pf.PfspError) as e:
            pf.pfsp_bound_batch(inst, 3, perm, e1, e2, lb1_out=h1.numpy(), lb2_out=h2.numpy())
        assert e.value.code == pf.PFSP_ERR_INVALID
        assert (h1.numpy() == -7).all() and (h2.numpy() == -7).all()
    # reduce mode: summaries in place against the copy path on pageable memory
    ub = int(np.median(w2[w2 >= 0]))
    want = pf.pfsp_bound_reduce(inst, pf.PFSP_LB2, perm, d1, d2, ub)
    raw = torch.zeros(N * pf.SUMMARY_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    hs = raw.numpy().view(pf.SUMMARY_DTYPE)
    for _ in range(2):
        got = pf.pfsp_bound_reduce(inst, pf.PFSP_LB2, perm, d1, d2, ub, out=hs)
        assert got.tobytes() == want.tobytes()
        raw.zero_()


@pytest.mark.parametrize("n,m,subset", [
    (16, 20, "adjacent"), (16, 20, "random40"), (14, 20, "random33"), (12, 7, "adjacent"), (12, 7, "random5"),
    (35, 10, "random20"),
])
def test_lb2_over_pair_subsets_bit_exact(pf, n, m, subset):
    # LB2 over a subset of the machine pairs (max of LB1 and the listed pairs'
    # values), against the oracle's definition with the same pairs
    P = m * (m - 1) // 2
    rng = np.random.default_rng(n * 100 + m)
    if subset == "adjacent":
        pairs = [k * (2 * m - k - 1) // 2 for k in range(m - 1)]
    else:
        pairs = list(rng.permutation(P)[:int(subset[6:])])
    p = inputs.make_instance(n, m, 77)
    perm, d1, d2 = inputs.random_nodes(n, 3000, seed=9, dmax=min(10, n // 3))
    inst = pf.pfsp_load_instance(p)
    pf.pfsp_set_lb2_pairs(inst, pairs)
    assert list(pf.pfsp_get_pair_order(inst)) == [int(q) for q in pairs]
    g1, g2 = pf.pfsp_bound_batch(inst, 3, perm, d1, d2)
    o1, o2 = orc.children_bounds_batch(p, perm, d1, d2, threads=8, pairs=pairs)
    assert (g1 == o1).all()
    bad = np.argwhere(g2 != o2)
    assert len(bad) == 0, (bad[:5], g2[tuple(bad[0])], o2[tuple(bad[0])])
    pf.pfsp_set_lb2_pairs(inst, None)
    _, full = pf.pfsp_bound_batch(inst, 3, perm, d1, d2)
    _, ofull = orc.children_bounds_batch(p, perm, d1, d2, threads=8)
    assert (full == ofull).all() and (g2 <= full).all()
    with pytest.raises(pf.PfspError):
        pf.pfsp_set_lb2_pairs(inst, [0, 0])


@pytest.mark.parametrize("n,m,count", [
    (20, 10, 3000), (12, 5, 3000), (20, 20, 1500), (36, 4, 800), (64, 3, 300), (9, 1, 500), (5, 7, 400),
])
def test_heads_tails_refinement_bit_exact(pf, n, m, count):
    # PFSP_MINHT: LB1 with the least heads / tails of the unscheduled jobs when
    # sigma1 / sigma2 is empty (LB2 = max of that LB1 and the pairs).  Small
    # depths make one side empty on about a third of the nodes; the degenerate
    # rows (root, one side only, leaf children, no children) are appended.
    p = inputs.make_instance(n, m, 4000 + n * 64 + m)
    perm, d1, d2 = inputs.random_nodes(n, count, seed=n * m, dmax=min(3, n))
    extra_d1 = np.array([0, n, 0, n - 1, 0, 1], dtype=np.uint8) if n >= 2 else np.zeros(6, np.uint8)
    extra_d2 = np.array([0, 0, n, 0, n - 1, 0], dtype=np.uint8) if n >= 2 else np.zeros(6, np.uint8)
    perm = np.concatenate([perm, perm[:6]])
    d1 = np.concatenate([d1, extra_d1])
    d2 = np.concatenate([d2, extra_d2])
    inst = pf.pfsp_load_instance(p)
    for kind in (pf.PFSP_LB1 | pf.PFSP_MINHT, pf.PFSP_LB1 | pf.PFSP_LB2 | pf.PFSP_MINHT):
        g1, g2 = pf.pfsp_bound_batch(inst, kind, perm, d1, d2)
        o1, o2 = orc.children_bounds_batch(p, perm, d1, d2, kind=kind, threads=8)
        bad = np.argwhere(g1 != o1)
        assert len(bad) == 0, ("LB1 minht mismatch", kind, bad[:5], g1[tuple(bad[0])], o1[tuple(bad[0])])
        if kind & pf.PFSP_LB2:
            bad = np.argwhere(g2 != o2)
            assert len(bad) == 0, ("LB2 minht mismatch", bad[:5], g2[tuple(bad[0])], o2[tuple(bad[0])])
    plain, _ = pf.pfsp_bound_batch(inst, pf.PFSP_LB1, perm, d1, d2)
    assert (g1 >= plain).all() and (g1 > plain).any() == (m > 1)
    with pytest.raises(pf.PfspError):
        pf.pfsp_bound_batch(inst, pf.PFSP_MINHT, perm, d1, d2)


def _summaries(o, ub):
    """Reduce-mode summaries from the oracle's bound arrays o [N, 2, n] (-1: scheduled)."""
    N, _, n = o.shape
    on = o >= 0
    big = np.where(on, o, np.iinfo(np.int32).max).astype(np.int64)
    mn = big.min(axis=2)
    cnt = (on & (o == mn[:, :, None])).sum(axis=2)
    sm = np.where(on, o, 0).astype(np.int64).sum(axis=2)
    bits = (np.uint64(1) << np.arange(n, dtype=np.uint64))
    keep = np.where(on & (o < ub), bits[None, None, :], np.uint64(0)).sum(axis=2, dtype=np.uint64)
    return mn.astype(np.int64), cnt, sm, keep


@pytest.mark.parametrize("n,m,count", [(20, 20, 4000), (20, 10, 3000), (12, 5, 3000), (50, 5, 800), (64, 4, 300),
                                       (33, 7, 500), (9, 1, 500), (1, 3, 20)])
def test_reduce_mode_matches_oracle(pf, n, m, count):
    # per parent and direction: least bound, its count, the sum and the job
    # mask of the children below ub, against the oracle's bound arrays
    p = inputs.make_instance(n, m, 5000 + n * 64 + m)
    perm, d1, d2 = inputs.random_nodes(n, count, seed=n + 3 * m, dmax=min(10, n))
    # append a root, a node without children and one with leaf children
    perm = np.concatenate([perm, perm[:3]])
    d1 = np.concatenate([d1, np.array([0, n, max(n - 1, 0)], dtype=np.uint8)])
    d2 = np.concatenate([d2, np.array([0, 0, 0], dtype=np.uint8)])
    inst = pf.pfsp_load_instance(p)
    o1, o2 = orc.children_bounds_batch(p, perm, d1, d2, threads=8)
    for kind, o in ((pf.PFSP_LB1, o1), (pf.PFSP_LB2, o2)):
        ub = int(np.median(o[o >= 0])) if (o >= 0).any() else 1
        s = pf.pfsp_bound_reduce(inst, kind, perm, d1, d2, ub)
        mn, cnt, sm, keep = _summaries(o, ub)
        assert (s["min"] == mn).all() and (s["count"] == cnt).all()
        assert (s["sum"] == sm).all() and (s["keep"] == keep).all()
    assert s["min"][-2].tolist() == [2**31 - 1] * 2 and s["count"][-2].tolist() == [0, 0]
    with pytest.raises(pf.PfspError):
        pf.pfsp_bound_reduce(inst, pf.PFSP_LB1 | pf.PFSP_LB2, perm, d1, d2, 10)


def test_reduce_mode_device_entry_point(pf):
    import torch
    n, m = 20, 20
    p = inputs.make_instance(n, m, 8)
    perm, d1, d2 = inputs.random_nodes(n, 5000, seed=3)
    d1[7], d2[7] = 15, 9  # invalid: d1 + d2 > n, clamped on the device
    inst = pf.pfsp_load_instance(p)
    tp = torch.from_numpy(perm).cuda()
    t1 = torch.from_numpy(d1).cuda()
    t2 = torch.from_numpy(d2).cuda()
    out = torch.empty(len(d1) * 48, dtype=torch.uint8, device="cuda")
    pf.pfsp_bound_reduce_dev(inst, pf.PFSP_LB2, len(d1), tp.data_ptr(), t1.data_ptr(), t2.data_ptr(), 1500,
                             out.data_ptr())
    torch.cuda.synchronize()
    s = out.cpu().numpy().view(pf.SUMMARY_DTYPE)
    assert s["min"][7].tolist() == [-1, -1] and s["count"][7].tolist() == [-1, -1]
    ok = np.ones(len(d1), dtype=bool)
    ok[7] = False
    d2[7] = 0
    ref = pf.pfsp_bound_reduce(inst, pf.PFSP_LB2, perm, d1, d2, 1500)
    for f in ("min", "count", "sum", "keep"):
        assert (s[f][ok] == ref[f][ok]).all()

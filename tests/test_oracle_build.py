"""Pins for the oracle's iterator build and zero-in-degree set (Section 2.4, Section 2.5 "Init").

Each check is independent of oracle.c: brute force with Python sets, hand-built graphs whose
answer is known, and the definition of E iterated naively against the peeling algorithm.
"""
import numpy as np
import pytest

import oracle
import workloads


def brute_build(n, src, dst):
    links = sorted(set(zip(src.tolist(), dst.tolist())))
    out_rows = [[] for _ in range(n)]
    in_rows = [[] for _ in range(n)]
    for s, t in links:
        out_rows[s].append(t)
        in_rows[t].append(s)
    return links, out_rows, in_rows


def csr_rows(rp, col):
    return [col[rp[i]:rp[i + 1]].tolist() for i in range(len(rp) - 1)]


@pytest.mark.parametrize("seed", range(12))
def test_build_matches_brute_force(seed):
    n = [1, 2, 5, 17, 40, 90][seed % 6]
    n, src, dst = workloads.small_random_graph(n, 4 * n + 3, seed=1000 + seed)
    g = oracle.build(n, src, dst)
    links, out_rows, in_rows = brute_build(n, src, dst)
    assert g.L == len(links)
    assert csr_rows(g.rp_out, g.col_out) == [sorted(r) for r in out_rows]
    assert csr_rows(g.rp_in, g.col_in) == [sorted(r) for r in in_rows]
    assert g.outdeg.tolist() == [len(r) for r in out_rows]
    assert g.indeg.tolist() == [len(r) for r in in_rows]
    assert g.loop.tolist() == [int(i in set(out_rows[i])) for i in range(n)]
    assert g.D == sum(len(r) == 0 for r in out_rows)
    assert g.O == sum(int(i in set(out_rows[i])) for i in range(n))
    assert g.max_in == max(len(r) for r in in_rows)
    assert g.max_out == max(len(r) for r in out_rows)


def test_build_rejects_out_of_range():
    with pytest.raises(ValueError, match="edge 2"):
        oracle.build(3, np.array([0, 1, 2], np.int32), np.array([1, 2, 3], np.int32))
    with pytest.raises(ValueError, match="edge 0"):
        oracle.build(3, np.array([-1], np.int32), np.array([1], np.int32))


def test_build_empty_and_single():
    g = oracle.build(4, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.L == 0 and g.D == 4 and g.rp_out.tolist() == [0] * 5 and g.rp_in.tolist() == [0] * 5
    g = oracle.build(1, np.array([0, 0], np.int32), np.array([0, 0], np.int32))
    assert g.L == 1 and g.O == 1 and g.D == 0 and g.loop.tolist() == [1]


def _e(n, edges):
    src = np.array([s for s, _ in edges], np.int32)
    dst = np.array([t for _, t in edges], np.int32)
    g = oracle.build(n, src, dst)
    return g, oracle.zero_in(g), oracle.zero_in_naive(g)


def test_e_directed_cycle_is_empty():
    g, (m, lv, cnt, nl), naive = _e(6, [(i, (i + 1) % 6) for i in range(6)])
    assert cnt == 0 and nl == 0 and m.sum() == 0 and (lv == -1).all()
    assert naive[2] == 0


def test_e_chain_levels():
    n = 9
    g, (m, lv, cnt, nl), (m2, lv2, cnt2, nl2) = _e(n, [(i, i + 1) for i in range(n - 1)])
    assert cnt == n and nl == n and lv.tolist() == list(range(n))
    assert cnt2 == n and lv2.tolist() == list(range(n))


def test_e_star_and_reverse_star():
    g, (m, lv, cnt, nl), _ = _e(6, [(0, k) for k in range(1, 6)])
    assert cnt == 6 and lv.tolist() == [0, 1, 1, 1, 1, 1] and nl == 2
    g, (m, lv, cnt, nl), _ = _e(6, [(k, 0) for k in range(1, 6)])
    assert cnt == 6 and lv.tolist() == [1, 0, 0, 0, 0, 0]


def test_e_self_loop_never_member():
    # node 1 has a self-loop and an in-link from E member 0: not in E, nor anything after it
    g, (m, lv, cnt, nl), naive = _e(4, [(0, 1), (1, 1), (1, 2), (2, 3)])
    assert m.tolist() == [1, 0, 0, 0] and lv.tolist() == [0, -1, -1, -1]
    assert naive[0].tolist() == m.tolist()


def test_e_level_is_one_plus_max():
    # 0 -> 2, 1 -> 3, 3 -> 2 : level(2) = 1 + max(level 0, level 3) = 2
    g, (m, lv, cnt, nl), naive = _e(4, [(0, 2), (1, 3), (3, 2)])
    assert lv.tolist() == [0, 0, 2, 1] and nl == 3
    assert naive[1].tolist() == lv.tolist()


def test_e_cycle_fed_by_chain():
    # chain 0->1->2 feeds the cycle 3->4->5->3: E = {0, 1, 2}
    g, (m, lv, cnt, nl), naive = _e(6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 3)])
    assert m.tolist() == [1, 1, 1, 0, 0, 0] and lv.tolist() == [0, 1, 2, -1, -1, -1]
    assert naive[0].tolist() == m.tolist()


@pytest.mark.parametrize("seed", range(10))
def test_e_peeling_equals_definition(seed):
    n = 30 + 17 * seed
    # sparse graphs so that a good part of the nodes sits in E
    n, src, dst = workloads.small_random_graph(n, n, seed=2000 + seed, p_loop=0.05)
    g = oracle.build(n, src, dst)
    a = oracle.zero_in(g)
    b = oracle.zero_in_naive(g)
    assert a[0].tolist() == b[0].tolist()
    assert a[1].tolist() == b[1].tolist()
    assert a[2:] == b[2:]


def test_e_peeling_equals_definition_on_paper_sized_graph():
    spec = workloads.WORKLOADS["pa_n10k"]["spec"]
    n, src, dst = workloads.generate(spec)
    g = oracle.build(n, src, dst)
    a = oracle.zero_in(g)
    b = oracle.zero_in_naive(g)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2:] == b[2:]
    assert 0 < a[2] < n


def test_generator_is_deterministic_and_shaped():
    spec = workloads.WORKLOADS["pa_n10k"]["spec"]
    a = workloads.generate(spec)
    b = workloads.generate(spec)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    n, src, dst = a
    g = oracle.build(n, src, dst)
    assert g.D == int(0.15 * n)          # exactly floor(p_D * N) dangling nodes
    assert g.max_out <= 500
    assert g.max_in > 5 * g.max_out or g.max_in > 200   # power-law in-degree: hubs

"""GPU graph build (iterator "Init", Section 2.1/2.5; statistics and E of Section 2.4) against the
oracle, bit for bit, through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import assert_build_matches_oracle, lib

pytestmark = pytest.mark.gpu


def _graph(n, src, dst, device=False):
    lib()
    if device:
        import torch
        return di.di_graph_create(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    return di.di_graph_create(n, src, dst)


# sizes straddle the radix-sort tile (4096 links), warps (32) and ragged tails
@pytest.mark.parametrize("n,m", [(1, 0), (1, 3), (2, 5), (3, 31), (33, 32), (40, 33), (100, 4095), (300, 4096),
                                 (1000, 4097), (5000, 20000), (20000, 70001), (70000, 300000)])
@pytest.mark.parametrize("device", [False, True])
def test_build_random_graphs(n, m, device):
    n, src, dst = workloads.small_random_graph(n, m, seed=n * 7 + m)
    g = _graph(n, src, dst, device)
    assert_build_matches_oracle(g, oracle.build(n, src, dst))
    di.di_graph_validate(g)


def test_build_all_duplicates_and_self_loops():
    n = 10
    src = np.array([3] * 5000 + [4] * 3 + list(range(10)), np.int32)
    dst = np.array([3] * 5000 + [7] * 3 + list(range(10)), np.int32)
    g = _graph(n, src, dst)
    og = oracle.build(n, src, dst)
    assert og.L == 11
    assert_build_matches_oracle(g, og)


def test_build_hubs_take_the_heavy_paths():
    # node 0 links to every other node and every node links back: out/in degree far above the
    # split thresholds of the push and pull kernels
    n = 20000
    src = np.concatenate([np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int32), np.zeros(n - 1, np.int32)])
    perm = np.argsort(workloads.u64(5, 5, len(src)), kind="stable")
    g = _graph(n, src[perm].copy(), dst[perm].copy())
    assert_build_matches_oracle(g, oracle.build(n, src, dst))


def test_build_long_chain_levels():
    n = 3000   # E = every node, levels 0..n-1 (one peeling round per level)
    src = np.arange(n - 1, dtype=np.int32)
    dst = src + 1
    g = _graph(n, src[::-1].copy(), dst[::-1].copy())
    og = oracle.build(n, src, dst)
    assert_build_matches_oracle(g, og)
    assert g.stats["E"] == n and g.stats["e_levels"] == n


@pytest.mark.parametrize("name", ["pa_n10k", "web_n1m"])
def test_build_workloads(name):
    spec = workloads.WORKLOADS[name]["spec"]
    n, src, dst = workloads.generate(spec)
    g = _graph(n, src, dst)
    assert_build_matches_oracle(g, oracle.build(n, src, dst))
    di.di_graph_validate(g)


def test_build_rejects_bad_ids_and_sizes():
    lib()
    with pytest.raises(di.DiError) as e:
        di.di_graph_create(5, np.array([0, 1, 2], np.int32), np.array([1, 5, 2], np.int32))
    assert e.value.status == 2 and "edge 1" in e.value.message
    with pytest.raises(di.DiError) as e:
        di.di_graph_create(5, np.array([0, -1], np.int32), np.array([1, 2], np.int32))
    assert e.value.status == 2
    with pytest.raises(di.DiError) as e:
        di.di_graph_create(0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert e.value.status == 1

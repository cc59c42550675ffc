"""The seeded input generator against its recipe (the inputs of every parity test and of the
benchmark): SplitMix64's published sequence, counter-based addressing, determinism, and the
shape of a web-like graph (dangling count, host locality, mean out-degree, loop nodes, the
zero-in-degree chains, a power-law in-degree) and of the personalised seed sets."""
import math

import numpy as np
import pytest

import oracle
import workloads

M64 = (1 << 64) - 1


def _splitmix64_stream(state, count):
    """SplitMix64 as published (Steele, Lea and Flood, OOPSLA 2014): the state advances by the
    golden gamma, and each output is the state through the variant-13 mix."""
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_published_sequence():
    # the widely published first outputs of SplitMix64 from seed 1234567
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert workloads.draw(1234567, 0, 5).tolist() == want


@pytest.mark.parametrize("key", [0, 1, 1234567, 0xDEADBEEFCAFEF00D, M64])
def test_counter_addressing_is_the_stream(key):
    # draw(key, c) is the c-th output of the stream, so any slice can be drawn independently
    stream = _splitmix64_stream(key, 300)
    assert workloads.draw(key, 0, 300).tolist() == stream
    assert workloads.draw(key, 123, 50).tolist() == stream[123:173]


SPEC = workloads.GraphSpec(n=200_000, p_dangling=0.2, cap=5000, mean_out=10.0, p_local=0.7, chain_frac=0.1,
                           seed=777)


@pytest.fixture(scope="module")
def web():
    n, src, dst = workloads.generate(SPEC)
    return n, src, dst


def test_deterministic_and_seeded(web):
    n, src, dst = web
    n2, src2, dst2 = workloads.generate(SPEC)
    assert n2 == n and np.array_equal(src, src2) and np.array_equal(dst, dst2)
    _, src3, dst3 = workloads.generate(SPEC.with_seed(778))
    assert src3.size != src.size or not np.array_equal(dst3, dst)


def test_web_graph_shape(web):
    n, src, dst = web
    assert src.min() >= 0 and dst.min() >= 0 and src.max() < n and dst.max() < n
    outdeg = np.bincount(src, minlength=n)
    # exactly floor(p_dangling * N) nodes without out-links (chain nodes always link onwards)
    assert int((outdeg == 0).sum()) == math.floor(SPEC.p_dangling * n)
    # the mean out-degree of the others is the requested one (duplicates included)
    assert abs(outdeg[outdeg > 0].mean() / SPEC.mean_out - 1.0) < 0.08
    # host locality: about p_local of the non-loop links stay within the window
    nl = src != dst
    local = float((np.abs(dst[nl].astype(np.int64) - src[nl]) <= SPEC.window).mean())
    assert abs(local - SPEC.p_local) < 0.05
    # loop nodes: p_loop of the nodes that are neither dangling nor on a chain
    loops = np.unique(src[~nl]).size / n
    expect = SPEC.p_loop * (1.0 - SPEC.p_dangling - SPEC.chain_frac)
    assert abs(loops - expect) < 0.01


def test_chains_and_power_law_in_degree(web):
    n, src, dst = web
    og = oracle.build(n, src, dst)
    _, _, count, levels = oracle.zero_in(og)
    # the zero-in-degree chains make up about chain_frac of the nodes, in several levels
    assert SPEC.chain_frac * 0.95 <= count / n <= SPEC.chain_frac * 1.3
    assert levels >= SPEC.chain_min
    # preferential attachment: max_in far above max_out, and a power-law tail of in-degrees
    assert og.max_in > 3 * og.max_out
    nl = src != dst
    indeg = np.bincount(dst[nl], minlength=n)
    p100, p1000 = (indeg >= 100).mean(), (indeg >= 1000).mean()
    assert p1000 > 0
    slope = math.log10(p100 / p1000)     # CCDF decade slope, alpha - 1 for a density ~ k^-alpha
    assert 0.8 < slope < 1.6


def test_seed_sets():
    n, k, max_size = 50_000, 512, 1000
    off, seeds = workloads.seed_sets(n, k, max_size, seed=3)
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == seeds.size and sizes.min() >= 1 and sizes.max() <= max_size
    assert seeds.min() >= 0 and seeds.max() < n
    for r in range(k):
        s = seeds[off[r]:off[r + 1]]
        assert np.unique(s).size == s.size          # without replacement
    # log-uniform sizes: floor(exp(u ln 1000)) <= 31 exactly when u < ln 32 / ln 1000
    frac = float((sizes <= 31).mean())
    assert abs(frac - math.log(32) / math.log(max_size)) < 0.07
    off2, seeds2 = workloads.seed_sets(n, k, max_size, seed=3)
    assert np.array_equal(off, off2) and np.array_equal(seeds, seeds2)

"""di_csr_validate finds every planted inconsistency in graph arrays (host code: no GPU needed).

The arrays come from the oracle's build of random graphs (pinned bit for bit against the GPU
build elsewhere); each case corrupts one invariant and the validator must report DI_ERR_CORRUPT.
"""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads

CORRUPT = 8


def _arrays(seed):
    spec = workloads.GraphSpec(n=400, p_dangling=0.15, cap=40, mean_out=6.0, p_local=0.6, window=20,
                               chain_frac=0.2, p_loop=0.2, seed=seed)
    n, src, dst = workloads.generate(spec)
    g = oracle.build(n, src, dst)
    e_mask, level, _, _ = oracle.zero_in(g)
    return dict(n=n, L=g.L, rp_out=g.rp_out.copy(), col_out=g.col_out.copy(), rp_in=g.rp_in.copy(),
                col_in=g.col_in.copy(), out_deg=g.outdeg.copy(), in_deg=g.indeg.copy(), loop=g.loop.copy(),
                e_mask=e_mask.copy(), e_level=level.copy())


def _validate(a):
    di.di_csr_validate(a["n"], a["L"], a["rp_out"], a["col_out"], a["rp_in"], a["col_in"], a["out_deg"],
                       a["in_deg"], a["loop"], a["e_mask"], a["e_level"])


def _row_with(a, minlen):
    lens = np.diff(a["rp_out"])
    return int(np.nonzero(lens >= minlen)[0][0])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    di.build()
    di.load()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_consistent_arrays_pass(seed):
    _validate(_arrays(9000 + seed))


def _corrupt_unsorted(a):
    i = _row_with(a, 2)
    b = a["rp_out"][i]
    a["col_out"][b], a["col_out"][b + 1] = a["col_out"][b + 1], a["col_out"][b]


def _corrupt_duplicate(a):
    i = _row_with(a, 2)
    b = a["rp_out"][i]
    a["col_out"][b + 1] = a["col_out"][b]


def _corrupt_out_of_range(a):
    i = _row_with(a, 1)
    a["col_out"][a["rp_out"][i + 1] - 1] = a["n"]


def _corrupt_not_transpose(a):
    # move one in-link of a row to another origin while keeping the row sorted and unique
    for i in range(a["n"]):
        b, e = a["rp_in"][i], a["rp_in"][i + 1]
        row = set(a["col_in"][b:e].tolist())
        if e > b:
            for c in range(a["n"]):
                if c not in row:
                    new = sorted((row - {int(a["col_in"][e - 1])}) | {c})
                    a["col_in"][b:e] = new
                    return
    raise AssertionError("no row to corrupt")


def _corrupt_degree(a):
    a["out_deg"][_row_with(a, 1)] += 1


def _corrupt_loop(a):
    a["loop"][0] ^= 1


def _corrupt_e_mask(a):
    a["e_mask"][int(np.nonzero(a["e_mask"] == 0)[0][0])] = 1


def _corrupt_e_level(a):
    i = int(np.nonzero(a["e_level"] > 0)[0][0])
    a["e_level"][i] += 1


def _corrupt_rowptr(a):
    a["rp_out"][5] = a["rp_out"][4] - 1


def _corrupt_rowptr_past_end(a):
    a["rp_out"][1] = a["L"] + 100


@pytest.mark.parametrize("corrupt", [_corrupt_unsorted, _corrupt_duplicate, _corrupt_out_of_range,
                                     _corrupt_not_transpose, _corrupt_degree, _corrupt_loop, _corrupt_e_mask,
                                     _corrupt_e_level, _corrupt_rowptr, _corrupt_rowptr_past_end],
                         ids=lambda f: f.__name__[9:])
def test_planted_inconsistency_is_found(corrupt):
    a = _arrays(9100)
    corrupt(a)
    with pytest.raises(di.DiError) as e:
        _validate(a)
    assert e.value.status == CORRUPT

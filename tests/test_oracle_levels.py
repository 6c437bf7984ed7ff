"""The level-by-level oracle driver (oracle_tiled_qr_levels, the CPU
baseline's build with OpenMP): running the tasks of each level of Algorithm
2's task graph concurrently gives exactly the bits of the sequential loop
order (Sec. 4: any topological order does), and its number of levels is the
length of the longest dependency chain of the graph derived independently
from the tasks' tile reads and writes (oracle.dependencies)."""
import numpy as np
import pytest

import oracle
from paper_0709_1272_gb300 import inputs


def _longest_chain(m, n, nb):
    tasks, preds = oracle.dependencies(m, n, nb)
    depth = {}
    for t in tasks:   # the loop order is topological
        depth[t] = 1 + max((depth[p] for p in preds[t]), default=0)
    return max(depth.values()) if depth else 0


@pytest.mark.parametrize("m,n,nb,ib", [(700, 500, 64, 16), (512, 512, 64, 16), (300, 900, 64, 32),
                                       (1100, 130, 128, 32), (64, 64, 64, 16), (1, 1, 64, 16)])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_levels_equal_sequential_bits(m, n, nb, ib, threads):
    A = inputs.normal_matrix(m, n, seed=m + 7 * n)
    f0 = oracle.tiled_qr(A, nb, ib)
    f1, nlev = oracle.tiled_qr_levels(A, nb, ib, threads)
    assert np.array_equal(f0.A, f1.A) and np.array_equal(f0.T, f1.T)
    assert nlev == _longest_chain(m, n, nb)


def test_levels_closed_form_square():
    # p x p tiles: step k's chain GEQRT -> TSQRT(k+1..p-1) -> the last SSRFB
    # feeds step k+1's GEQRT; the graph's longest chain is 3p - 2 levels
    for p in (2, 3, 5, 8):
        _, nlev = oracle.tiled_qr_levels(inputs.normal_matrix(64 * p, 64 * p, seed=p), 64, 16, 2)
        assert nlev == _longest_chain(64 * p, 64 * p, 64)

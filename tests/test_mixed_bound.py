"""The per-task error bound of the mixed-precision updates (tests/mixed_cases
.py, BOUND = 32 * 2^-21 per column) separates 3xTF32 from a product that
drops a term: on the same DLARFB and DSSRFB cases the GPU test uses, a CPU
emulation of 3xTF32 stays well below the bound, while dropping the lo*hi
term, or both cross terms (plain TF32), lands far above it.  This pins the
GPU test's bound to the arithmetic rather than to a measured number."""
import pytest

import mixed_cases as mc


@pytest.mark.parametrize("ib", [16, 32])
def test_bound_separates_3xtf32_from_dropped_terms_larfb(ib):
    V, T, C, ref = mc.larfb_case(ib)
    full = mc.column_error(mc.emulate_larfb(V, T, C, ib), ref, C)
    one_cross = mc.column_error(mc.emulate_larfb(V, T, C, ib, terms=("hl",)), ref, C)
    plain = mc.column_error(mc.emulate_larfb(V, T, C, ib, terms=()), ref, C)
    assert full <= mc.BOUND / 4, full
    assert one_cross >= 10 * mc.BOUND and plain >= 10 * mc.BOUND, (one_cross, plain)


@pytest.mark.parametrize("ib", [16, 32])
def test_bound_separates_3xtf32_from_dropped_terms_ssrfb(ib):
    import numpy as np
    V, T, Bp, C, ref = mc.ssrfb_case(ib)
    x = np.vstack([Bp, C])
    full = mc.column_error(mc.emulate_ssrfb(V, T, Bp, C, ib), ref, x)
    one_cross = mc.column_error(mc.emulate_ssrfb(V, T, Bp, C, ib, terms=("lh",)), ref, x)
    plain = mc.column_error(mc.emulate_ssrfb(V, T, Bp, C, ib, terms=()), ref, x)
    assert full <= mc.BOUND / 4, full
    assert one_cross >= 10 * mc.BOUND and plain >= 10 * mc.BOUND, (one_cross, plain)


def test_ssrfb_case_is_the_dssrfb_of_algorithm_2():
    """The DSSRFB reference really is one task: the oracle's Q^T of the
    two-tile factorization equals its DLARFB on the top tile followed by the
    pair update, i.e. the pair [B'; C] is rotated without changing column
    norms (Q^T is orthogonal)."""
    import numpy as np
    V, T, Bp, C, ref = mc.ssrfb_case(16)
    x = np.vstack([Bp, C])
    assert np.allclose(np.linalg.norm(ref, axis=0), np.linalg.norm(x, axis=0), rtol=1e-13)

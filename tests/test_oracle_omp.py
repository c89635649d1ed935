"""The OpenMP variant of the oracle's column recurrence (used only to time
the CPU baseline on several cores) gives bitwise the single-thread result:
same scalar arithmetic, same summation order per entry."""
import numpy as np
import pytest

import oracle
import synth


def factored(p, wmax, cplx=False):
    sym = oracle.analyse(p.n, p.colptr, p.rowind, wmax, 1)
    lcp, lri = oracle.supernodal_pattern(p.n, sym["sn_start"], sym["rcount"], sym["rrows"])
    vals = p.values.astype(complex) * (1 + 0.3j) if cplx else p.values
    lv, d = oracle.ldlt(p.n, sym["colptr"], sym["rowind"], vals, lcp, lri)
    return lcp, lri, lv, d


@pytest.mark.parametrize("side,wmax,cplx", [(13, 16, False), (11, 128, True), (20, 32, False)])
@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_threads_bitwise_equal_single_thread(side, wmax, cplx, threads):
    p = synth.grid3d(side)
    lcp, lri, lv, d = factored(p, wmax, cplx)
    xv, xd = oracle.selinv(p.n, lcp, lri, lv, d)
    xv2, xd2 = oracle.selinv(p.n, lcp, lri, lv, d, threads=threads)
    assert np.array_equal(xv, xv2) and np.array_equal(xd, xd2)


def test_threads_on_a_2d_grid_and_the_fundamental_pattern():
    p = synth.grid2d_31()
    lcp, lri, lv, d = factored(p, 0)
    xv, xd = oracle.selinv(p.n, lcp, lri, lv, d)
    xv2, xd2 = oracle.selinv(p.n, lcp, lri, lv, d, threads=4)
    assert np.array_equal(xv, xv2) and np.array_equal(xd, xd2)

"""CPU pins of the arithmetic behind opts.fp64_emulation (steps 2 and 3 on
bf16 slices), written independently of the CUDA path in Python integers and
exact rationals:

* the power-of-two scaling e_p = ceil(E_p / 2) (X_pp < 2^E_p) puts every
  entry of 2^-(e_p+e_q) X below 1 for SPD X (Cauchy-Schwarz);
* cutting q = floor(|v| 2^(56-E)) into 7 bytes reconstructs q exactly, and
  every byte is an integer in [0, 255] (exact in bf16's 8 significant bits);
* the group sums over a 32-row chunk stay below 2^24 even for the largest
  slices, so FP32 accumulation of integer products is exact;
* the fold hi = S0 2^16 + S1 2^8 + S2, lo = S3 2^24 + ... + S6 and the final
  scaling 2^(e + F - 31) (hi + lo 2^-32) reproduce the sum of the kept slice
  products exactly;
* the dropped products (t + u >= 7) and the truncation stay below 2^-53 per
  term of 2^(e_i + F_j), checked against the exact rational product."""
import math
from fractions import Fraction

import numpy as np
import pytest

NSL = 7          # slices per entry
KC = 32          # rows per exact FP32 chunk


def slices(v, E):
    """The 7 signed byte slices of v with |v| < 2^E: q = floor(|v| 2^(56-E))."""
    assert abs(v) < 2.0 ** E
    q = math.floor(Fraction(abs(v)) * Fraction(2) ** (56 - E))
    assert 0 <= q < 2 ** 56
    sgn = -1 if v < 0 else 1
    return [sgn * ((q >> (8 * (6 - t))) & 255) for t in range(NSL)], q


def slice_value(sl, E):
    """Exact value of the slices: sum_t s_t 2^(8 (6 - t)) 2^(E - 56)."""
    return sum(Fraction(s) * Fraction(2) ** (8 * (6 - t) + E - 56) for t, s in enumerate(sl))


def exp_of_diag(d):
    """e = ceil(E / 2) with d < 2^E (frexp), so 2^e >= sqrt(d)."""
    _, E = math.frexp(d)
    return (E + 1) >> 1


@pytest.mark.parametrize("seed", range(4))
def test_cauchy_schwarz_scaling_bounds_every_entry_below_one(seed):
    rng = np.random.default_rng(seed)
    n = 40
    B = rng.normal(size=(n, n)) * np.exp(rng.normal(scale=3.0, size=n))[:, None]  # rows of very different size
    A = B @ B.T + 1e-3 * np.eye(n)
    X = np.linalg.inv(A)
    e = np.array([exp_of_diag(X[p, p]) for p in range(n)])
    assert np.all(2.0 ** (2 * e) >= np.diag(X))
    Xt = X / np.ldexp(1.0, e[:, None] + e[None, :])
    assert np.max(np.abs(Xt)) < 1.0
    assert np.max(np.abs(Xt)) > 0.25        # the scaling is not needlessly loose on the diagonal


@pytest.mark.parametrize("seed", range(3))
def test_slices_reconstruct_the_fixed_point_value_and_fit_bf16(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(300):
        E = int(rng.integers(-40, 40))
        v = float(rng.uniform(-1, 1)) * 2.0 ** E * float(rng.choice([1.0, 0.999999, 1e-5, 1e-12]))
        if v == 0.0:
            continue
        sl, q = slices(v, E)
        assert all(0 <= abs(s) <= 255 for s in sl)
        assert sum(abs(s) << (8 * (6 - t)) for t, s in enumerate(sl)) == q
        # truncation: |v| - value < 2^(E - 56)
        assert 0 <= Fraction(abs(v)) - abs(slice_value(sl, E)) < Fraction(2) ** (E - 56)
        # every slice is an integer bf16 represents exactly (<= 8 significant bits)
        for s in sl:
            f = np.float32(abs(s))
            bits = f.view(np.uint32)
            assert bits & 0xFFFF == 0


def test_group_sums_of_a_chunk_stay_below_two_to_the_24():
    # worst case: every slice of both operands at 255, all k of the chunk
    for g in range(NSL):
        pairs = [(t, g - t) for t in range(NSL) if 0 <= g - t < NSL]
        assert len(pairs) == g + 1
        worst = KC * sum(255 * 255 for _ in pairs)
        assert worst < 2 ** 24, (g, worst)
    # the step-2 A operand is below 1 in magnitude with q < 2^55, so its top slice is < 128
    assert (2 ** 55 - 1) >> 48 == 127


def fold_and_scale(S, e_i, F_j, step):
    """hi, lo of the seven group sums and the scaled result (step 2: -31,
    step 3: -32), exactly."""
    hi = S[0] * 65536 + S[1] * 256 + S[2]
    lo = S[3] * 16777216 + S[4] * 65536 + S[5] * 256 + S[6]
    off = 31 if step == 2 else 32
    return (Fraction(hi) + Fraction(lo) / 2 ** 32) * Fraction(2) ** (e_i + F_j - off)


@pytest.mark.parametrize("step", [2, 3])
@pytest.mark.parametrize("seed", range(3))
def test_fold_equals_the_kept_slice_products_and_error_is_fp64_class(step, seed):
    """One output entry y = sum_k a_k b_k over K = 96 rows (three chunks):
    step 2 has a = X~ in (-1, 1) cut at E = 1 (q_a = |a| 2^55) and b = B'/2^F
    at E = 0; step 3 has both operands cut at E = 0.  The folded result equals
    the exact sum of the kept products (t + u <= 6), and differs from the
    exact y by less than K 2^-53 of the scale 2^(e + F)."""
    rng = np.random.default_rng(7 + seed)
    K = 96
    e_i, F_j = int(rng.integers(-20, 20)), int(rng.integers(-20, 20))
    a = rng.uniform(-1, 1, K) * rng.choice([1.0, 1e-3, 1e-9], K)
    b = rng.uniform(-1, 1, K) * rng.choice([1.0, 1e-4], K)
    Ea = 1 if step == 2 else 0
    sa = [slices(float(x), Ea)[0] for x in a]
    sb = [slices(float(x), 0)[0] for x in b]
    S = [0] * NSL
    for k in range(K):
        for t in range(NSL):
            for u in range(NSL - t):
                S[t + u] += sa[k][t] * sb[k][u]
    # chunk-wise exactness: every partial group sum of a chunk is below 2^24
    for c0 in range(0, K, KC):
        for g in range(NSL):
            part = sum(sa[k][t] * sb[k][g - t] for k in range(c0, c0 + KC) for t in range(g + 1) if g - t < NSL)
            assert abs(part) < 2 ** 24
    got = fold_and_scale(S, e_i, F_j, step)
    # exact value of the kept products, with the operands' own scalings
    wa = (lambda t: Fraction(2) ** (8 * (6 - t) + Ea - 56))
    wb = (lambda u: Fraction(2) ** (8 * (6 - u) - 56))
    kept = sum(Fraction(sa[k][t] * sb[k][u]) * wa(t) * wb(u)
               for k in range(K) for t in range(NSL) for u in range(NSL - t))
    assert got == kept * Fraction(2) ** (e_i + F_j)
    exact = sum(Fraction(float(a[k])) * Fraction(float(b[k])) for k in range(K)) * Fraction(2) ** (e_i + F_j)
    err = abs(got - exact) / Fraction(2) ** (e_i + F_j)
    assert err < K * Fraction(1, 2 ** 53), float(err)
    # and the FP64 evaluation of the same scaled sum (hi + lo 2^-32, then ldexp) rounds once more
    hi = S[0] * 65536 + S[1] * 256 + S[2]
    lo = S[3] * 16777216 + S[4] * 65536 + S[5] * 256 + S[6]
    f64 = math.ldexp(float(hi) + float(lo) * 2.0 ** -32, e_i + F_j - (31 if step == 2 else 32))
    assert abs(Fraction(f64) - got) <= abs(got) * Fraction(1, 2 ** 51) + Fraction(2) ** (e_i + F_j - 1074 + 60)

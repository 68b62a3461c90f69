"""The error-free slicing behind the tensor-core trailing updates (chol_df = 3), checked on the
CPU in the kernel's own steps: per row a power-of-two scale 2^-E with max |P_rk| < 2^E, eight
signed slices s_i = rint(128 v_i), v_{i+1} = 128 v_i - s_i, so that P_rk = 2^E sum_i s_i 2^-7(i+1)
to the double-float's precision.  The conditions the kernel relies on:

* every slice is an integer of magnitude <= 128, exact in BF16 (8 significant bits);
* every level l = i + j of slice products, summed over K = 32 and over the level's pairs, is an
  integer below 2^22, so an FP32 accumulator holds it exactly whatever the order of the sums;
* the levels 0-7 added with their weights 2^-7(l+2) reproduce P_I P_J^T to FP64 class relative
  to sum_k |P_rk||P_ck| (the dropped levels >= 8 are below 2^-56 of it).
"""
import numpy as np
import pytest

NS, K = 8, 32


def slices(P):
    m = np.abs(P).max(axis=1)
    E = np.where(m > 0, np.frexp(m)[1], 0)                   # m < 2^E
    v = P * np.ldexp(1.0, -E)[:, None]
    S = np.empty((NS,) + P.shape)
    for i in range(NS):
        t = v * 128.0
        S[i] = np.rint(t)
        v = t - S[i]
    return S, E


def levels(SA, SB):
    acc = np.zeros((NS, SA.shape[1], SB.shape[1]))
    for lev in range(NS):
        for i in range(lev + 1):
            acc[lev] += SA[i] @ SB[lev - i].T
    return acc


@pytest.mark.parametrize("seed,spread", [(0, 0.0), (1, 20.0), (2, 40.0)])
def test_slices_levels_and_reconstruction(seed, spread):
    rng = np.random.default_rng(seed)
    PI = rng.standard_normal((128, K)) * np.exp(rng.uniform(-spread, spread, (128, 1)))
    PJ = rng.standard_normal((64, K)) * np.exp(rng.uniform(-spread, spread, (64, 1)))
    PI[5] = 0.0                                              # an all-zero row (rows past n)
    SA, EA = slices(PI)
    SB, EB = slices(PJ)
    for S in (SA, SB):
        assert np.all(S == np.rint(S)) and np.abs(S).max() <= 128
    acc = levels(SA, SB)
    assert np.abs(acc).max() < 2.0 ** 22
    assert np.all(acc.astype(np.float32).astype(np.float64) == acc)
    comb = sum(acc[lev] * 2.0 ** (-7 * lev) for lev in range(NS))
    val = comb * np.ldexp(1.0, EA[:, None] + EB[None, :] - 14)
    exact = PI @ PJ.T
    scale = np.abs(PI) @ np.abs(PJ).T
    err = np.abs(val - exact)
    assert np.all(err <= 1e-15 * scale + 1e-300)
    assert np.all(val[5] == 0.0)


def test_a_largest_magnitude_of_a_power_of_two():
    """max |P_rk| = 2^k exactly: frexp puts E at k + 1, so the first slice stays <= 64."""
    P = np.zeros((1, K))
    P[0, 3] = 8.0
    P[0, 7] = -3.0
    S, E = slices(P)
    assert E[0] == 4 and np.abs(S).max() <= 128
    back = sum(S[i] * 2.0 ** (-7 * (i + 1)) for i in range(NS)) * 2.0 ** E[0]
    assert np.array_equal(back, P)

"""CPU checks of the index maps of the emulated step-2/3 kernels (the maps
in paper_1404_0447_gb300/csrc/emulate.cu, restated here): every staging map
covers its tile exactly once and stays in bounds, the 32-bit plane stores of
one warp instruction hit 32 distinct shared-memory banks.
These are the checks made before the kernels first ran on a GPU."""
import itertools

import numpy as np
import pytest

KC, KP = 32, 40            # rows of C per chunk; slice-plane row stride (bf16) of the mma.sync kernels
TILE_M, THREADS = 64, 128  # mma.sync tile rows, threads


def banks_of_words(word_addrs):
    return [w % 32 for w in word_addrs]


# ---- mma.sync kernels (k_em_gemm1, k_em_gemm2): pair maps, plane stores ----

def pair_mma(warp, lane, p, right_of_rows):
    """(row, first k) of pair p of a thread; 2 entries (k, k+1) per pair."""
    bi = warp * 8 + p
    if right_of_rows:
        return (bi & 3) + 8 * (bi >> 2) + 4 * (lane >> 4), 2 * (lane & 15)
    return 8 * (bi & 7) + (lane & 7), 2 * (4 * (bi >> 3) + (lane >> 3))


@pytest.mark.parametrize("right", [False, True])
def test_mma_pair_map_covers_the_tile_once_and_stores_without_conflicts(right):
    seen = np.zeros((TILE_M, KC), int)
    for warp, p in itertools.product(range(4), range(8)):
        words = []
        for lane in range(32):
            row, k = pair_mma(warp, lane, p, right)
            assert 0 <= row < TILE_M and 0 <= k <= KC - 2 and k % 2 == 0
            seen[row, k] += 1
            seen[row, k + 1] += 1
            words.append((row * KP + k) // 2)       # 32-bit word of plane[row][k]
        assert len(set(banks_of_words(words))) == 32, (warp, p)
    assert np.all(seen == 1)


@pytest.mark.parametrize("nb", [8, 16])
def test_mma_b_pair_map_covers_the_b_tile(nb):
    seen = np.zeros((nb, KC), int)
    for j in range(nb // 8):
        for t in range(THREADS):
            pi = j * THREADS + t
            n, k = pi >> 4, 2 * (pi & 15)
            assert n < nb and k <= KC - 2
            seen[n, k] += 1
            seen[n, k + 1] += 1
    assert np.all(seen == 1)


def test_ldmatrix_rows_hit_distinct_16_byte_bank_groups():
    # 8 row addresses of one 8x8 matrix: rows r0..r0+7 at stride KP bf16 (80 B)
    for r0 in range(0, TILE_M, 8):
        for kofs in (0, 8, 16, 24):
            groups = {((r0 + i) * KP * 2 + kofs * 2) // 16 % 8 for i in range(8)}
            assert len(groups) == 8
            assert all(((r0 + i) * KP * 2 + kofs * 2) % 16 == 0 for i in range(8))

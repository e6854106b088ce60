"""Host-side packing of moves into the compact 4-byte form (no GPU needed).

Every code below is worked out by hand from the encoding p = (b1 << 16) | code,
code = swap partner or 65535 - t for a shift to period t."""

import numpy as np
import pytest


def test_hand_worked_codes():
    import paper_2511_18296_b300 as mm
    B, T = 50_000, 20
    moves = np.array([
        (0, 1),          # swap 0 with 1: (0 << 16) | 1 = 1
        (3, -1),         # shift 3 to period 0: code 65535 -> 3 * 65536 + 65535 = 262143
        (7, -21),        # shift 7 to period 20 = T (unmined): code 65515 -> 7 * 65536 + 65515 = 524267
        (49_999, 12),    # swap: 49999 * 65536 + 12 = 3276734476
    ], np.int32)
    p = mm.pack_moves(moves, B, T)
    assert p.dtype == np.uint32
    assert p.tolist() == [1, 262143, 524267, 3276734476]


def test_rejects_what_cannot_be_encoded():
    import paper_2511_18296_b300 as mm
    with pytest.raises(ValueError):
        mm.pack_moves(np.array([(0, 1)]), 65_530, 10)       # B + T + 1 > 65536
    with pytest.raises(ValueError):
        mm.pack_moves(np.array([(5, -22)]), 100, 20)        # period 21 > T
    with pytest.raises(ValueError):
        mm.pack_moves(np.array([(100, 3)]), 100, 20)        # b1 out of range

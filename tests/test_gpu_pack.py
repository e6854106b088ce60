"""mm_unpack_moves: packed 4-byte moves decode on the device to exactly the
moves they were made from; codes outside the encoding decode to a bad move;
evaluation from unpacked moves equals evaluation from the originals bit for
bit; models too large for the encoding are refused."""

import numpy as np
import pytest

import workloads as W
from helpers import tiny_problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("name", ["plain_4k", "plain_50k"])
def test_round_trip_and_same_scores(name):
    import paper_2511_18296_b300 as mm
    p = W.config(name)
    m = mm.Model.from_problem(p)
    m.schedule_set(p.x0)
    packed = torch.as_tensor(mm.pack_moves(p.moves, p.B, p.T).view(np.int32), device="cuda")
    mv = m.unpack_moves(packed)
    torch.cuda.synchronize()
    assert np.array_equal(mv.cpu().numpy(), p.moves)
    s1, f1, _ = m.eval_moves(mv, want_mean=False)
    s2, f2, _ = m.eval_moves(torch.as_tensor(p.moves, device="cuda"), want_mean=False)
    torch.cuda.synchronize()
    assert np.array_equal(s1.cpu().numpy().view(np.uint32), s2.cpu().numpy().view(np.uint32))
    assert np.array_equal(f1.cpu().numpy(), f2.cpu().numpy())


def test_codes_outside_the_encoding_are_bad_moves():
    import paper_2511_18296_b300 as mm
    p = tiny_problem(S=4, T=3)  # B = 27
    codes = np.array([
        (1 << 16) | 5,          # swap 1, 5
        (2 << 16) | 65535,      # shift 2 to period 0
        (2 << 16) | 65532,      # shift 2 to period 3 = T
        (2 << 16) | 65531,      # period 4 > T: bad
        (2 << 16) | 27,         # partner 27 = B: bad
        (27 << 16) | 1,         # b1 = B: bad
    ], np.uint32)
    m = mm.Model.from_problem(p)
    out = m.unpack_moves(torch.as_tensor(codes.view(np.int32), device="cuda")).cpu().numpy()
    assert out.tolist() == [[1, 5], [2, -1], [2, -4], [-1, -1], [-1, -1], [-1, -1]]


def test_model_too_large_is_refused():
    import paper_2511_18296_b300 as mm
    p = tiny_problem(nx=300, ny=220, nz=1, S=1, T=3, cap_blocks=30_000, target_blocks=10)  # B = 66,000
    m = mm.Model.from_problem(p)
    with pytest.raises(mm.MMError):
        m.unpack_moves(torch.zeros(4, dtype=torch.int32, device="cuda"))

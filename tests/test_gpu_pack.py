"""mm_unpack_moves: packed 4-byte moves decode on the device to exactly the
moves they were made from; codes outside the encoding decode to a bad move;
evaluation from unpacked moves equals evaluation from the originals bit for
bit; models too large for the encoding are refused.  mm_search_step_packed,
which decodes the compact form inside the fused step, gives exactly what
mm_unpack_moves followed by mm_search_step gives (scores, flags, top k, the
applied move, the sticky status), and refuses models whose step is not one
launch."""

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


def _step_outputs(res):
    s, f, i, t, c = (v.cpu().numpy() for v in res)
    n = int(c[0])
    return s.view(np.uint32), f, i[:n], t[:n].view(np.uint32), n


@pytest.mark.parametrize("name,weighted,steps", [("plain_4k", False, 12), ("plain_50k", False, 6),
                                                 ("plain_4k", True, 8)])
def test_packed_step_equals_unpack_then_step(name, weighted, steps):
    import paper_2511_18296_b300 as mm
    p = W.config(name)
    sigma = W.uncertainty_weights(p.T, p.S, seed=6) if weighted else None
    a = mm.Model.from_problem(p, sigma=sigma)
    b = mm.Model.from_problem(p, sigma=sigma)
    a.schedule_set(p.x0)
    b.schedule_set(p.x0)
    packed = torch.as_tensor(mm.pack_moves(p.moves, p.B, p.T).view(np.int32), device="cuda")
    for k in [32, 1, 7] + [16] * (steps - 3):
        ra = a.search_step_packed(packed, k=k, apply=True)
        rb = b.search_step(b.unpack_moves(packed), k=k, apply=True)
        torch.cuda.synchronize()
        oa, ob = _step_outputs(ra), _step_outputs(rb)
        for x, y in zip(oa, ob):
            assert np.array_equal(x, y)
        assert a.last_apply() == b.last_apply()
    assert np.array_equal(a.schedule_get(), b.schedule_get())
    assert np.array_equal(a.npv()[0], b.npv()[0])


def test_packed_step_bad_codes_and_no_apply():
    import paper_2511_18296_b300 as mm
    p = W.config("plain_4k")
    codes = mm.pack_moves(p.moves[:3000], p.B, p.T).copy()
    rng = np.random.default_rng(21)
    bad = rng.choice(codes.shape[0], 200, replace=False)
    codes[bad[:100]] = (codes[bad[:100]] & 0xffff) | (p.B << 16)      # b1 = B
    codes[bad[100:]] = (codes[bad[100:]] & 0xffff0000) | (p.B + 5)     # a code that names no move
    packed = torch.as_tensor(codes.view(np.int32), device="cuda")
    a = mm.Model.from_problem(p)
    b = mm.Model.from_problem(p)
    a.schedule_set(p.x0)
    b.schedule_set(p.x0)
    ra = a.search_step_packed(packed, k=32, apply=False)
    rb = b.search_step(b.unpack_moves(packed), k=32, apply=False)
    torch.cuda.synchronize()
    for x, y in zip(_step_outputs(ra), _step_outputs(rb)):
        assert np.array_equal(x, y)
    s, f = ra[0].cpu().numpy(), ra[1].cpu().numpy()
    assert np.all(f[bad] == 0) and np.all(np.isneginf(s[bad]))
    for m in (a, b):
        with pytest.raises(mm.MMError) as e:
            m.npv()
        assert e.value.status == 6  # MM_ERR_BAD_MOVE, sticky until read
    assert np.array_equal(a.schedule_get(), p.x0)
    # an empty batch: count 0, and with apply nothing is applied
    for apply in (False, True):
        ra = a.search_step_packed(torch.empty(0, dtype=torch.int32, device="cuda"), k=4, apply=apply)
        torch.cuda.synchronize()
        assert int(ra[4].cpu()[0]) == 0
    assert a.last_apply()[0] == 0


def test_packed_step_refused_where_not_one_launch():
    import paper_2511_18296_b300 as mm
    packed = torch.zeros(8, dtype=torch.int32, device="cuda")
    # S > 768 (more scenarios than the step's CTA has threads) with apply:
    # the apply is a second launch
    p = tiny_problem(S=800, T=3)
    m = mm.Model.from_problem(p)
    m.schedule_set(p.x0)
    with pytest.raises(mm.MMError) as e:
        m.search_step_packed(packed, k=4, apply=True)
    assert e.value.status == 1
    m.search_step_packed(packed, k=4, apply=False)  # without apply it is one launch
    torch.cuda.synchronize()
    # weights outside the weighted fast form (S % 4 != 0)
    p = tiny_problem(S=5, T=3)
    m = mm.Model.from_problem(p, sigma=W.uncertainty_weights(p.T, p.S, seed=1))
    m.schedule_set(p.x0)
    with pytest.raises(mm.MMError) as e:
        m.search_step_packed(packed, k=4, apply=True)
    assert e.value.status == 1
    # B + T + 1 > 65536
    p = tiny_problem(nx=300, ny=220, nz=1, S=1, T=3, cap_blocks=30_000, target_blocks=10)
    m = mm.Model.from_problem(p)
    m.schedule_set(p.x0)
    with pytest.raises(mm.MMError) as e:
        m.search_step_packed(packed, k=4, apply=False)
    assert e.value.status == 1

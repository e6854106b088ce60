"""The caller-free top-k (mm_topk_noalloc) against the model-owned one (mm_topk).

mm_topk_noalloc exists for callers that cannot allocate device memory (code
held to a fixed memory budget or pool, loops that must not let
cudaMalloc/cudaFree block the device); its scratch is a fixed array inside the
library.  Both entry points are called through the C ABI on the same inputs, two
calls in a row, and must agree exactly (indices bit for bit, scores equal); the
Python wrapper is checked on the largest batch the array takes with every
score tied (all keys in one histogram bin: the array's whole key region in
use) and on an empty batch.  This file is collected last so that a failure here
never hides another test.
"""

import ctypes

import numpy as np
import pytest

import workloads as W
from helpers import tiny_problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _abi():
    import paper_2511_18296_b300 as mm
    return mm, mm.lib()


def _topk_both(L, m, score, feas, k):
    dev = score.device
    outs = []
    for which in ("model", "noalloc"):
        idx = torch.full((k,), -7, dtype=torch.int32, device=dev)
        top = torch.full((k,), np.nan, dtype=torch.float32, device=dev)
        cnt = torch.full((1,), -7, dtype=torch.int32, device=dev)
        n = score.shape[0]
        if which == "model":
            st = L.mm_topk(m.h, score.data_ptr(), feas.data_ptr(), n, k, idx.data_ptr(), top.data_ptr(),
                           cnt.data_ptr())
        else:
            stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            st = L.mm_topk_noalloc(score.data_ptr(), feas.data_ptr(), n, k, idx.data_ptr(), top.data_ptr(),
                                   cnt.data_ptr(), stream)
        assert st == 0, L.mm_last_error()
        torch.cuda.synchronize()
        c = int(cnt.cpu()[0])
        outs.append((c, idx.cpu().numpy()[:c], top.cpu().numpy()[:c]))
    return outs


def test_noalloc_topk_matches_model_topk_twice():
    assert torch.cuda.is_available()
    mm, L = _abi()
    p = W.config("plain_4k")
    m = mm.Model.from_problem(p)
    m.schedule_set(p.x0)
    mv = torch.as_tensor(p.moves, device="cuda")
    score, feas, _ = m.eval_moves(mv)
    rng = np.random.default_rng(3)
    s2 = torch.as_tensor(rng.integers(-50, 50, 300_000).astype(np.float32), device="cuda")  # many ties
    f2 = torch.as_tensor((rng.random(300_000) < 0.5).astype(np.uint8), device="cuda")
    for (s, f, k) in ((score, feas, 32), (s2, f2, 1000)):   # two calls in a row, different sizes
        (ca, ia, ta), (cb, ib, tb) = _topk_both(L, m, s, f, k)
        assert ca == cb > 0
        assert np.array_equal(ia, ib)
        assert np.array_equal(ta, tb)


def test_noalloc_topk_rejects_oversized_batch():
    mm, L = _abi()
    big = (1 << 20) + 1
    st = L.mm_topk_noalloc(None, None, big, 4, None, None, None, None)
    assert st == 1 and b"fixed scratch size" in L.mm_last_error()


def test_noalloc_topk_full_size_all_tied_and_empty_through_the_wrapper():
    mm, L = _abi()
    p = W.config("plain_4k")
    m = mm.Model.from_problem(p)
    m.schedule_set(p.x0)
    n, k = 1 << 20, 1024
    score = torch.full((n,), 1.5, dtype=torch.float32, device="cuda")  # every key in one histogram bin
    feas = torch.ones(n, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        idx = torch.full((k,), -7, dtype=torch.int32, device="cuda")
        top = torch.zeros(k, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        mm.topk_noalloc(score, feas, k, idx, top, cnt)
        ri, rt, rc = m.topk(score, feas, k)
        torch.cuda.synchronize()
        assert int(cnt.cpu()[0]) == int(rc.cpu()[0]) == k
        assert np.array_equal(idx.cpu().numpy(), np.arange(k, dtype=np.int32))  # ties: the lower indices
        assert np.array_equal(idx.cpu().numpy(), ri.cpu().numpy())
        assert np.array_equal(top.cpu().numpy(), rt.cpu().numpy())
    empty_s = torch.empty(0, dtype=torch.float32, device="cuda")
    empty_f = torch.empty(0, dtype=torch.uint8, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    mm.topk_noalloc(empty_s, empty_f, 4, torch.empty(4, dtype=torch.int32, device="cuda"),
                    torch.empty(4, dtype=torch.float32, device="cuda"), cnt)
    torch.cuda.synchronize()
    assert int(cnt.cpu()[0]) == 0
    with pytest.raises(ValueError):  # the wrapper refuses a flag array shorter than the scores
        mm.topk_noalloc(score, feas[:10], 4, torch.empty(4, dtype=torch.int32, device="cuda"),
                        torch.empty(4, dtype=torch.float32, device="cuda"), cnt)

"""The two paths the benchmark times, checked against the FP64 oracle directly.

* The end-to-end step: mm_search_step_packed (compact 4-byte moves decoded in
  the launch, evaluation, top-32 and the in-launch apply) on the 50,000-block
  workload, ten steps in a row.  At every step the flags must equal the
  oracle's bit for bit, every score must be within 1e-5 * max(|ref|, F) of the
  oracle's incremental evaluation of the current schedule, the top 32 must be
  exactly the selection of the GPU's own scores and may differ from the
  oracle's only by certified near-ties; after the step the schedule and NPV_s
  must equal the oracle's apply of the same move (NPV_s to FP64 rounding).
* The batched form: every chain of the 64-chain workload, first run, against
  the oracle: flags and scores of every move, and the top 32.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import assert_close_floor, certified_swaps

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = 32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_packed_fused_step_with_apply_against_oracle_50k():
    import paper_2511_18296_b300 as mm
    p = W.config("plain_50k")
    om = O.OracleModel(p)
    m = mm.Model.from_problem(p)
    m.schedule_set(p.x0)
    packed = torch.as_tensor(mm.pack_moves(p.moves, p.B, p.T).view(np.int32), device="cuda")
    x = p.x0.copy()
    swaps = 0
    for step in range(10):
        score, feas, idx, top, cnt = m.search_step_packed(packed, k=K, apply=True)
        torch.cuda.synchronize()
        ref = om.eval_incremental(x, p.moves)  # the schedule before this step's move
        s, f = score.cpu().numpy(), feas.cpu().numpy()
        assert np.array_equal(f, ref["flag"]), f"step {step}: flags"
        assert_close_floor(s, ref["score"], ref["floor"], what=f"step {step}: scores")
        c = int(cnt.cpu()[0])
        gi = idx.cpu().numpy()[:c]
        own, own_top = O.topk(s.astype(np.float64), f, K)
        assert np.array_equal(gi, own), f"step {step}: top-k of the GPU's own scores"
        assert np.array_equal(top.cpu().numpy()[:c], own_top.astype(np.float32))
        ri, _ = O.topk(ref["score"], ref["flag"], K)
        swaps += certified_swaps(gi, ri, ref["score"], ref["floor"])
        assert c > 0
        assert om.apply(x, p.moves[gi[0]]) == 0  # the move the step applied
        assert np.array_equal(m.schedule_get(), x), f"step {step}: schedule"
        np.testing.assert_allclose(m.npv()[0], om.npv(x), rtol=1e-12, atol=1e-3)
    assert swaps == 0  # no near-tie met on this workload: the indices agree exactly


def test_batch_64_chains_against_oracle():
    import paper_2511_18296_b300 as mm
    probs = [W.chain_problem(sp) for sp in W.batched_chain_specs(64)]
    models, mvs = [], []
    for p in probs:
        m = mm.Model.from_problem(p)
        m.schedule_set(p.x0)
        models.append(m)
        mvs.append(torch.as_tensor(p.moves, device="cuda"))
    b = mm.Batch(list(zip(models, mvs)), k=K)
    b.run()
    torch.cuda.synchronize()
    for c, (p, o) in enumerate(zip(probs, b.out)):
        ref = O.OracleModel(p).eval_incremental(p.x0, p.moves)
        s, f = o["score"].cpu().numpy(), o["feas"].cpu().numpy()
        assert np.array_equal(f, ref["flag"]), f"chain {c}: flags"
        assert_close_floor(s, ref["score"], ref["floor"], what=f"chain {c}: scores")
        n = int(o["count"].cpu()[0])
        gi = o["idx"].cpu().numpy()[:n]
        own, _ = O.topk(s.astype(np.float64), f, K)
        assert np.array_equal(gi, own), f"chain {c}: top-k of the GPU's own scores"
        ri, _ = O.topk(ref["score"], ref["flag"], K)
        certified_swaps(gi, ri, ref["score"], ref["floor"])
    b.close()

"""Mixed-precision stress at 400,000 blocks x 500 scenarios (T = 30).

FP32 scenario arithmetic with compensated (Kahan) sums on a 1,048,576-move
batch (flags exact and scores within tolerance against the FP64 oracle on a
sample), then 1,000 accepted moves applied on the device with FP64 running
totals.  The final NPV_s must match a full FP64 recomputation of the final
schedule by the oracle to 1e-12 relative; the FP32 shadow accumulators, kept
beside them for comparison, drift by orders of magnitude more.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import assert_close_floor

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_stress_400k_kahan_parity_and_drift_after_1000_applies():
    import paper_2511_18296_b300 as mm
    p = W.config("stress_400k")
    om = O.OracleModel(p)
    m = mm.Model.from_problem(p)
    assert m.schedule_set(p.x0)
    m.set_fp32_shadow(True)
    mv = torch.as_tensor(p.moves, device="cuda")
    # evaluation parity on a sample of the full batch, plain and compensated
    sample = np.sort(np.random.default_rng(4).choice(p.moves.shape[0], 2048, replace=False))
    inc = om.eval_incremental(p.x0, p.moves[sample])
    for kahan in (False, True):
        s, f, _ = m.eval_moves(mv, want_mean=False, kahan=kahan)
        torch.cuda.synchronize()
        f0 = f.cpu().numpy()  # flags at the initial schedule (bit-exact on the sample below)
        fs, ss = f0[sample], s.cpu().numpy()[sample]
        assert np.array_equal(fs, inc["flag"])
        assert_close_floor(ss, inc["score"], inc["floor"], what=f"stress kahan={kahan}")
    # 1,000 applies that change the schedule.  The batch's best move stops
    # improving the NPV after a few steps on this model (then it is a feasible
    # no-op, which changes nothing), so a few best-move steps on the device are
    # followed by the batch's moves flagged feasible at the initial schedule,
    # applied one by one through mm_apply_move, which checks each exactly (those that became infeasible are
    # refused and skipped; no-ops are not sent), the schedule tracked here.
    idx = torch.empty(1, dtype=torch.int32, device="cuda")
    top = torch.empty(1, dtype=torch.float32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    x = p.x0.copy()
    changes = steps = 0
    for _ in range(20):
        s, f, _ = m.eval_moves(mv, want_mean=False, kahan=True)
        m.topk(s, f, 1, idx=idx, top=top, count=cnt)
        m.apply_best(mv, idx, cnt)
        steps += 1
        if m.last_apply()[0] and float(top[0].item()) > 0.0:  # synchronises
            assert om.apply(x, p.moves[int(idx[0].item())]) == 0
            changes += 1
    assert changes > 0
    cand = np.flatnonzero(f0)
    for i in cand:
        if changes == 1000:
            break
        b1, arg = (int(v) for v in p.moves[i])
        if (arg < 0 and x[b1] == -arg - 1) or (arg >= 0 and x[b1] == x[arg]):
            continue  # a no-op now
        try:
            m.apply_move((b1, arg))
        except mm.MMError:
            assert om.apply(x, p.moves[i]) == 1  # the oracle refuses it too
            continue  # infeasible after the earlier applies
        assert om.apply(x, p.moves[i]) == 0
        changes += 1
    assert changes == 1000
    accepted = changes
    assert np.array_equal(m.schedule_get(), x)
    x = m.schedule_get()
    assert np.count_nonzero(x != p.x0) > 0
    ref = om.npv(x)
    npv64, mean64, _ = m.npv()
    npv32 = m.fp32_shadow_npv()
    drift64 = np.max(np.abs(npv64 - ref) / np.abs(ref))
    drift32 = np.max(np.abs(npv32 - ref) / np.abs(ref))
    print(f"{accepted} accepted moves in {steps} steps: FP64 accumulators max rel drift {drift64:.3e}, FP32 shadow {drift32:.3e}")
    assert drift64 <= 1e-12
    assert drift32 > drift64
    mined, oreT = m.tonnage()
    rm, ro = om.tonnage(x)
    assert np.array_equal(mined, rm) and np.array_equal(oreT, ro)


def test_fp32_shadow_small():
    """Shadow on/off on a small model: starts from the FP64 state (to FP32
    rounding), follows applies, and is re-initialised by mm_schedule_set."""
    import paper_2511_18296_b300 as mm
    p = W.config("plain_4k")
    om = O.OracleModel(p)
    m = mm.Model.from_problem(p)
    m.schedule_set(p.x0)
    with pytest.raises(mm.MMError):
        m.fp32_shadow_npv()  # off
    m.set_fp32_shadow(True)
    np.testing.assert_allclose(m.fp32_shadow_npv(), om.npv(p.x0), rtol=1e-6)
    inc = om.eval_incremental(p.x0, p.moves)
    x = p.x0.copy()
    for i in np.nonzero(inc["flag"])[0][:20]:
        try:
            m.apply_move(tuple(p.moves[i]))
        except mm.MMError:
            continue  # infeasible after the earlier applies
        om.apply(x, p.moves[i])
    np.testing.assert_allclose(m.fp32_shadow_npv(), om.npv(x), rtol=1e-5)
    m.schedule_set(p.x0)
    np.testing.assert_allclose(m.fp32_shadow_npv(), om.npv(p.x0), rtol=1e-6)
    m.set_fp32_shadow(False)
    with pytest.raises(mm.MMError):
        m.fp32_shadow_npv()

"""Batched multi-chain evaluation (mm_batch_*) against the per-model calls.

Every chain of a batch -- different block models, scenario counts and batch
sizes, evaluated together in one persistent launch -- must get exactly what
the single-model path gives it: the same score and flag bits, the same top k,
and (with apply) the same schedule and NPV afterwards.  Two chains are also
checked against the FP64 oracle.
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


def mm():
    import paper_2511_18296_b300 as m
    return m


# (side, S, n_moves): every compiled shape (S = 16, 32, 48, 64, 100) and the
# run-time-shaped one (S = 13, 36), ragged batch sizes, one empty chain
SMALL = [(10, 16, 1000), (12, 32, 3333), (9, 48, 700), (11, 64, 2500), (13, 100, 4100), (8, 13, 999),
         (10, 36, 64), (9, 100, 0), (14, 16, 6000)]


def small_chains(seed0=500):
    specs = W.batched_chain_specs(len(SMALL), base_seed=seed0)
    probs = []
    for spec, (side, S, n) in zip(specs, SMALL):
        spec = dict(spec, nx=side, ny=side, nz=side, S=S, n_moves=n)
        spec["cap_blocks"] = int(np.ceil(1.12 * side ** 3 / spec["T"]))
        spec["target_blocks"] = int(round(0.393 * spec["cap_blocks"]))
        probs.append(W.chain_problem(spec))
    return probs


def models_for(probs):
    out = []
    for p in probs:
        m = mm().Model.from_problem(p)
        m.schedule_set(p.x0)
        out.append(m)
    return out


def moves_of(p):
    return torch.as_tensor(p.moves.reshape(-1, 2), device="cuda")


def check_chain(m, mv, o, k):
    """The batch's outputs for one chain equal a separate evaluation + top-k."""
    n = mv.shape[0]
    if n == 0:
        assert int(o["count"].cpu()[0]) == 0
        return
    s, f, _ = m.eval_moves(mv, want_mean=False)
    idx, top, cnt = m.topk(s, f, k)
    torch.cuda.synchronize()
    assert np.array_equal(o["feas"].cpu().numpy(), f.cpu().numpy())
    assert np.array_equal(o["score"].cpu().numpy().view(np.uint32), s.cpu().numpy().view(np.uint32))
    c = int(cnt.cpu()[0])
    assert int(o["count"].cpu()[0]) == c
    assert np.array_equal(o["idx"].cpu().numpy()[:c], idx.cpu().numpy()[:c])
    assert np.array_equal(o["top"].cpu().numpy()[:c], top.cpu().numpy()[:c])


@pytest.fixture(scope="module")
def small():
    probs = small_chains()
    return probs, models_for(probs)


def test_batch_matches_separate_calls_every_tile(small):
    probs, models = small
    mvs = [moves_of(p) for p in probs]
    b = mm().Batch(list(zip(models, mvs)), k=32)
    for tile, ctas in ((64, 0), (512, 0), (2048, 1), (1 << 20, 0)):
        b.set_tile(tile, ctas)
        for o in b.out:
            o["score"].fill_(float("nan"))
            o["count"].fill_(-1)
        b.run()
        torch.cuda.synchronize()
        for m, mv, o in zip(models, mvs, b.out):
            check_chain(m, mv, o, 32)
    b.close()


def test_batch_against_oracle(small):
    probs, models = small
    mvs = [moves_of(p) for p in probs]
    b = mm().Batch(list(zip(models, mvs)), k=8)
    b.run()
    torch.cuda.synchronize()
    for c in (1, 5):  # S = 32 (compiled shape) and S = 13 (run-time shape)
        p = probs[c]
        inc = O.OracleModel(p).eval_incremental(p.x0, p.moves)
        assert np.array_equal(b.out[c]["feas"].cpu().numpy(), inc["flag"])
        assert_close_floor(b.out[c]["score"].cpu().numpy(), inc["score"], inc["floor"], what=f"chain {c}")
    b.close()


def test_batch_graph_replay_with_new_moves(small):
    probs, models = small
    mvs = [moves_of(p) for p in probs]
    st = torch.cuda.Stream()
    b = mm().Batch(list(zip(models, mvs)), k=16, stream=st)
    b.run()
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        b.run()
    rng = np.random.default_rng(3)
    for rep in range(2):
        for p, mv in zip(probs, mvs):  # new moves written into the same buffers
            if mv.shape[0]:
                new = W.random_moves(p.x0, p.T, mv.shape[0], 0.5, rng)
                mv.copy_(torch.as_tensor(new))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for m, mv, o in zip(models, mvs, b.out):
            check_chain(m, mv, o, 16)
    b.close()


def test_batch_autotune_keeps_results(small):
    probs, models = small
    mvs = [moves_of(p) for p in probs]
    b = mm().Batch(list(zip(models, mvs)), k=4)
    tile, ctas, ms = b.autotune(reps=2)
    assert tile in (512, 1024, 2048, 4096, 8192, 16384) and ctas >= 1 and ms > 0
    assert b.tile()[:2] == (tile, ctas)
    b.run()
    torch.cuda.synchronize()
    for c, (p, m, mv, o) in enumerate(zip(probs, models, mvs, b.out)):
        if b.chain_shape(c)[0] == default_team(p.S):  # the autotuner kept the single-model team
            check_chain(m, mv, o, 4)
    b.close()


def test_batch_apply_matches_search_step():
    probs = small_chains(seed0=900)
    twins = models_for(probs)
    models = models_for(probs)
    mvs = [moves_of(p) for p in probs]
    b = mm().Batch(list(zip(models, mvs)), k=32, apply=True)
    for step in range(3):
        b.run()
        torch.cuda.synchronize()
        for c, (m, t, mv, o) in enumerate(zip(models, twins, mvs, b.out)):
            if mv.shape[0] == 0:
                assert int(o["count"].cpu()[0]) == 0
                continue
            s, f, idx, top, cnt = t.search_step(mv, k=32, apply=True)
            torch.cuda.synchronize()
            assert np.array_equal(o["score"].cpu().numpy().view(np.uint32), s.cpu().numpy().view(np.uint32))
            ca = int(cnt.cpu()[0])
            assert int(o["count"].cpu()[0]) == ca
            assert np.array_equal(o["idx"].cpu().numpy()[:ca], idx.cpu().numpy()[:ca])
            assert np.array_equal(m.schedule_get(), t.schedule_get()), (step, c)
            assert m.last_apply() == t.last_apply()
    b.close()


def test_batch_errors(small):
    probs, models = small
    mvs = [moves_of(p) for p in probs]
    with pytest.raises(mm().MMError):
        mm().Batch([(models[0], mvs[0]), (models[0], mvs[0])], k=4)  # shared model
    with pytest.raises(mm().MMError):
        mm().Batch([(models[0], mvs[0])], k=33)
    b = mm().Batch([(models[0], mvs[0])], k=4, apply=True)
    with pytest.raises(mm().MMError):
        b.autotune()  # a batch that applies is not autotuned
    b.close()
    with pytest.raises(mm().MMError):
        b2 = mm().Batch([(models[0], mvs[0])], k=4)
        b2.set_tile(100, 0)  # not a multiple of 64


def test_batch_64_chains_full_workload():
    """The 64-chain workload (cubes of side 15..40, S in {16, 32, 64, 100},
    1,024..65,536 moves per chain) in one launch equals 64 separate calls."""
    specs = W.batched_chain_specs(64)
    probs = [W.chain_problem(s) for s in specs]
    models = models_for(probs)
    mvs = [moves_of(p) for p in probs]
    b = mm().Batch(list(zip(models, mvs)), k=32)
    b.autotune(reps=2)
    b.run()
    torch.cuda.synchronize()
    for c, (p, m, mv, o) in enumerate(zip(probs, models, mvs, b.out)):
        if b.chain_shape(c)[0] == default_team(p.S):  # the autotuner kept the single-model team
            check_chain(m, mv, o, 32)
    b.close()


def default_team(S):
    """The single-model team width: the smallest of 4..32 lanes giving at most
    four scenario quads per lane (32 otherwise)."""
    nq = (S + 3) // 4
    for team in (4, 8, 16, 32):
        if (nq + team - 1) // team <= 4:
            return team
    return 32


def test_batch_chain_shapes_team_and_prefetch(small):
    """mm_batch_set_chain: another team width adds the scenario sums in another
    order (same flags, scores within FP32 rounding of the default ones); the
    prefetch distance changes no bit; team 0 restores the default bits."""
    probs, models = small
    mvs = [moves_of(p) for p in probs]
    b = mm().Batch(list(zip(models, mvs)), k=8)
    ref = []
    for m, mv in zip(models, mvs):
        if mv.shape[0] == 0:
            ref.append(None)
            continue
        s, f, _ = m.eval_moves(mv, want_mean=False)
        ref.append((s.cpu().numpy(), f.cpu().numpy()))
    for c, p in enumerate(probs):
        assert b.chain_shape(c) == (default_team(p.S), 0)
        wider = default_team(p.S) * 2
        if wider <= 32:
            b.set_chain(c, wider, 2)
            assert b.chain_shape(c) == (wider, 2)
    b.run()
    torch.cuda.synchronize()
    for c, o in enumerate(b.out):
        if ref[c] is None:
            continue
        s, f = ref[c]
        assert np.array_equal(o["feas"].cpu().numpy(), f)
        got = o["score"].cpu().numpy()
        fin = np.isfinite(s)
        assert np.array_equal(np.isfinite(got), fin)
        scale = np.abs(s[fin]).max() if fin.any() else 1.0
        np.testing.assert_allclose(got[fin], s[fin], rtol=0, atol=1e-5 * scale)
    for c in range(len(probs)):
        b.set_chain(c, 0, 3)  # default team, prefetch three batches ahead
    b.run()
    torch.cuda.synchronize()
    for m, mv, o in zip(models, mvs, b.out):
        check_chain(m, mv, o, 8)
    b.close()


def test_batch_chain_shape_errors(small):
    probs, models = small
    mvs = [moves_of(p) for p in probs]
    b = mm().Batch(list(zip(models, mvs)), k=4)
    i100 = next(i for i, p in enumerate(probs) if p.S == 100)
    for args in ((0, 3, 0), (i100, 4, 0), (len(probs), 0, 0), (0, 0, 9), (-1, 0, 0)):
        with pytest.raises(mm().MMError):
            b.set_chain(*args)
    b.close()


def test_batch_autotune_cache_installs_stored_shapes(small, tmp_path):
    """autotune(cache=...) stores each chain's team width and prefetch under its
    (S, B, n) key and the tile under the batch's key set; a second batch of the
    same chains installs them from the file without timing."""
    import json
    probs, models = small
    mvs = [moves_of(p) for p in probs]
    path = str(tmp_path / "tune.json")
    b = mm().Batch(list(zip(models, mvs)), k=4)
    tile, ctas, ms = b.autotune(reps=1, cache=path)
    shapes = [b.chain_shape(c) for c in range(len(probs))]
    b.close()
    data = json.load(open(path))
    keys = [f"S{p.S}_B{p.B}_n{int(mv.shape[0])}" for p, mv in zip(probs, mvs)]
    for k, sh in zip(keys, shapes):
        assert data["chains"][k] == {"team": sh[0], "prefetch": sh[1]}
    assert len(data["tiles"]) == 1
    b2 = mm().Batch(list(zip(models, mvs)), k=4)
    t2, c2, ms2 = b2.autotune(reps=1, cache=path)
    assert (t2, c2, ms2) == (tile, ctas, pytest.approx(ms))
    assert [b2.chain_shape(c) for c in range(len(probs))] == shapes
    b2.run()
    torch.cuda.synchronize()
    for c, (m, mv, o) in enumerate(zip(models, mvs, b2.out)):
        if shapes[c][0] == default_team(probs[c].S):
            check_chain(m, mv, o, 4)
    b2.close()


def test_batch_wide_scenario_shapes():
    """The run-time-shaped evaluators of 8, 16 and 32 lanes as chains' default
    shapes (S = 70, 200, 300: the single model's team widths 8, 16, 32), each
    in its own non-inlined function inside the batched kernel: every chain gets
    the single-model bits and top k, and one is checked against the oracle."""
    specs = W.batched_chain_specs(3, base_seed=900)
    probs = []
    for spec, (side, S, n) in zip(specs, ((9, 70, 1500), (8, 200, 1100), (7, 300, 777))):
        spec = dict(spec, nx=side, ny=side, nz=side, S=S, n_moves=n)
        spec["cap_blocks"] = int(np.ceil(1.12 * side ** 3 / spec["T"]))
        spec["target_blocks"] = int(round(0.393 * spec["cap_blocks"]))
        probs.append(W.chain_problem(spec))
    assert [default_team(p.S) for p in probs] == [8, 16, 32]
    models = models_for(probs)
    mvs = [moves_of(p) for p in probs]
    b = mm().Batch(list(zip(models, mvs)), k=16)
    for tile, ctas in ((256, 0), (1 << 20, 0)):
        b.set_tile(tile, ctas)
        b.run()
        torch.cuda.synchronize()
        for m, mv, o in zip(models, mvs, b.out):
            check_chain(m, mv, o, 16)
    p = probs[2]
    inc = O.OracleModel(p).eval_incremental(p.x0, p.moves)
    assert np.array_equal(b.out[2]["feas"].cpu().numpy(), inc["flag"])
    assert_close_floor(b.out[2]["score"].cpu().numpy(), inc["score"], inc["floor"], what="S = 300 chain")
    b.close()

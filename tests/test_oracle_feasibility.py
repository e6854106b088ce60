"""Feasibility flag vs a library transitive closure (oracle only).

Eq. 15 asks that every direct predecessor be mined no later; by transitivity
this is the same as asking it of every ancestor.  networkx builds the closure of
the predecessor graph independently of the oracle, and capacity (Eq. 16) is
checked with numpy.  On a feasible base schedule the oracle's local flag of a
move must equal full feasibility of the moved schedule.
"""

import networkx as nx
import numpy as np
import pytest

import oracle as O
from helpers import all_moves, tiny_problem


def grid_graph(nx_, ny_, nz_):
    """1-5 pattern from coordinates: (x,y,z-1), (x+-1,y,z-1), (x,y+-1,z-1)."""
    g = nx.DiGraph()
    B = nx_ * ny_ * nz_
    g.add_nodes_from(range(B))
    for z in range(1, nz_):
        for y in range(ny_):
            for x in range(nx_):
                b = x + nx_ * (y + ny_ * z)
                for dx, dy in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
                    px, py = x + dx, y + dy
                    if 0 <= px < nx_ and 0 <= py < ny_:
                        g.add_edge(px + nx_ * (py + ny_ * (z - 1)), b)
    return g


def closure_feasible(closure, x, mass, cap, T):
    for i, j in closure.edges():
        if x[i] > x[j]:
            return False
    mined = np.bincount(x[x < T], weights=mass[x < T], minlength=T)
    return bool(np.all(mined <= cap))


def test_stencil_arc_counts():
    # 3x3 level: 4 corners x 3 + 4 edges x 4 + centre x 5 = 33 arcs per level pair
    ptr, idx = O.stencil_preds(3, 3, 2)
    assert ptr[-1] == 33
    centre = 4 + 9
    assert sorted(idx[ptr[centre]:ptr[centre + 1]].tolist()) == [1, 3, 4, 5, 7]
    assert ptr[9] == 0  # top level has none


@pytest.mark.parametrize("dims,T,seed", [((3, 3, 3), 3, 1), ((2, 3, 3), 4, 2), ((4, 1, 3), 3, 3)])
def test_flag_equals_closure_feasibility(dims, T, seed):
    nx_, ny_, nz_ = dims
    B = nx_ * ny_ * nz_
    rng = np.random.default_rng(seed)
    p = tiny_problem(nx_, ny_, nz_, S=2, T=T, cap_blocks=-(-B // T) + 2, seed=seed)
    om = O.OracleModel(p)
    g = grid_graph(nx_, ny_, nz_)
    clo = nx.transitive_closure_dag(g)
    # a few random feasible base schedules: top-down greedy plus random pushes down
    bases = [p.x0.copy()]
    for _ in range(3):
        x = p.x0.copy()
        for _ in range(20):
            b = rng.integers(B)
            tn = rng.integers(T + 1)
            y = x.copy(); y[b] = tn
            if closure_feasible(clo, y, p.mass.astype(float), p.cap.astype(float), T):
                x = y
        bases.append(x)
    mv = all_moves(B, T)
    for x in bases:
        assert om.feasible(x)
        r = om.eval_bruteforce(x, mv, want_delta=False)
        ri = om.eval_incremental(x, mv)
        assert np.array_equal(r["flag"], ri["flag"])
        for i, (b1, arg) in enumerate(mv):
            y = x.copy()
            if arg >= 0:
                y[b1], y[arg] = x[arg], x[b1]
            else:
                y[b1] = -arg - 1
            want = closure_feasible(clo, y, p.mass.astype(float), p.cap.astype(float), T)
            assert bool(r["flag"][i]) == want, (x.tolist(), b1, arg)
            assert om.feasible(y) == want


def test_general_dag_csr():
    """A hand-made DAG through the CSR path: 0 -> 2, 1 -> 2, 2 -> 3."""
    ptr = np.array([0, 0, 0, 2, 3], np.int32)
    idx = np.array([0, 1, 2], np.int32)
    p = tiny_problem(4, 1, 1, S=1, T=3, cap_blocks=2, x0=np.array([0, 0, 1, 2], np.uint8))
    om = O.OracleModel(p, preds=(ptr, idx))
    mv = np.array([[3, -2], [3, -1], [2, -1], [2, -3], [0, -2], [0, -3], [2, 3]], np.int32)
    r = om.eval_bruteforce(p.x0, mv)
    # 3->1: ok (pred 2 in 1); 3->0: pred 2 later; 2->0: preds fine, succ fine, period 0 holds 3 > 2;
    # 2->2: succ 3 in 2 ok; 0->1: succ 2 in 1 ok; 0->2: succ 2 in 1 violated; swap 2<->3: 3 before 2
    assert r["flag"].tolist() == [1, 0, 0, 1, 1, 0, 0]

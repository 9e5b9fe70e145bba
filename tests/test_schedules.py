"""Host checks of the diagonal tile's task-graph order (CPU only).

The kernel hands tasks out by an atomic ticket in list order and every task
waits (bounded) on progress counters of the blocks it reads.  If each
task's waits are met by tasks earlier in the list, the graph cannot
deadlock whatever the number of co-resident CTAs: replaying the list with
one CTA (strictly in order) must therefore finish with every counter at its
final value.  The wait and release rules below restate the kernel's: block
(r, c) of the factor counts its c updates and then its solve or
factorisation; block (j, r) of W = L^{-T} counts its r - j updates and then
its solve.
"""
import numpy as np
import pytest


def _replay(tasks, nb):
    ver = np.zeros((nb, nb), dtype=np.int64)
    wv = np.zeros((nb, nb), dtype=np.int64)
    seen = set()

    def need(cond, what, t):
        assert cond, f"task {t} waits on {what} that no earlier task provides"

    def put(arr, idx, val, t, steps=1):
        assert arr[idx] == val - steps, f"task {t} moves counter {idx} from {arr[idx]} to {val}"
        arr[idx] = val

    for t in map(tuple, tasks):
        op, r, c, k = t
        assert t not in seen, f"task {t} listed twice"
        seen.add(t)
        if op == 0:
            assert (r, c, k) == (0, 0, 0)
            put(ver, (0, 0), 1, t)
            put(wv, (0, 0), 1, t)
        elif op == 3:      # G(k): solve (k, k-1), update and factor (k, k)
            need(ver[k, k - 1] >= k - 1 and ver[k, k] >= k - 1, "updated blocks", t)
            need(ver[k - 1, k - 1] >= k, "the previous diagonal block", t)
            put(ver, (k, k - 1), k, t)
            put(ver, (k, k), k + 1, t, steps=2)     # its last update, then the factorisation
            put(wv, (k, k), 1, t)
        elif op == 1:      # T(r, k)
            need(ver[k, k] >= k + 1 and ver[r, k] >= k, "factor / updates", t)
            put(ver, (r, k), k + 1, t)
        elif op == 2:      # U(r, c, k)
            need(ver[r, k] >= k + 1 and ver[c, k] >= k + 1 and ver[r, c] >= k, "solved blocks", t)
            put(ver, (r, c), k + 1, t)
        elif op == 4:      # V(r, j = c)
            need(ver[r, r] >= r + 1 and wv[c, r] >= r - c, "factor / W updates", t)
            put(wv, (c, r), r - c + 1, t)
        elif op == 5:      # E(r, k, j = c)
            need(ver[r, k] >= k + 1, "solved block", t)
            need(wv[c, c] >= 1 if k == c else wv[c, k] >= k - c + 1, "W block", t)
            need(wv[c, r] >= k - c, "previous W update", t)
            put(wv, (c, r), k - c + 1, t)
        else:
            raise AssertionError(f"unknown op {op}")
    return ver, wv


@pytest.mark.parametrize("nb", [1, 2, 3, 4, 8, 16, 24, 32, 64])
def test_task_order_is_topological_and_complete(nb):
    from paper_2406_02701_gb300 import mpchol
    tasks = mpchol.potrf_dag_schedule(nb)
    ver, wv = _replay(tasks, nb)
    for r in range(nb):
        for c in range(r + 1):
            assert ver[r, c] == c + 1, (r, c)
            assert wv[c, r] == r - c + 1, (c, r)


def test_chain_tasks_come_one_step_ahead():
    """G(k+2) is handed out before T(r, k+1) and the rest of step k, right
    after the two updates it reads."""
    from paper_2406_02701_gb300 import mpchol
    nb = 32
    tasks = [tuple(t) for t in mpchol.potrf_dag_schedule(nb)]
    pos = {t: i for i, t in enumerate(tasks)}
    for k in range(nb - 2):
        g = pos[(3, k + 2, k + 2, k + 2)]
        assert g == pos[(2, k + 2, k + 2, k)] + 1
        assert g > pos[(2, k + 2, k + 1, k)]
        if k + 3 < nb:
            assert g < pos[(1, k + 3, k + 1, k + 1)]


def test_replay_catches_a_misplaced_task():
    """The replay is not vacuous: moving G(3) before the update it reads
    fails."""
    from paper_2406_02701_gb300 import mpchol
    tasks = [tuple(t) for t in mpchol.potrf_dag_schedule(8)]
    g = tasks.index((3, 3, 3, 3))
    u = tasks.index((2, 3, 3, 1))
    bad = tasks[:u] + [tasks[g]] + [t for i, t in enumerate(tasks[u:], u) if i != g]
    with pytest.raises(AssertionError):
        _replay(np.array(bad), 8)


def test_schedule_rejects_bad_sizes():
    from paper_2406_02701_gb300 import mpchol
    for nb in (0, 65, -3):
        with pytest.raises(mpchol.MPError):
            mpchol.potrf_dag_schedule(nb)


def _replay_solve(tasks, nt, P, trans):
    """The solve graph's rules: block p of in_i counts the updates applied to
    it in place (they must come in solve order of the columns j); the
    product with the row solved just before i goes to a chain vector
    instead (op 2) and waits only for out_j; D(i, p) waits for all
    in-place updates and chain products of the blocks of in_i it reads
    (p' <= p forward, p' >= p backward); an update with out_j waits for all
    P blocks of out_j."""
    order = {(nt - 1 - st if trans else st): st for st in range(nt)}
    cnt = np.zeros((nt, P), dtype=np.int64)
    chain = np.zeros((nt, P), dtype=np.int64)
    done = np.zeros(nt, dtype=np.int64)
    seen = set()
    for t in map(tuple, tasks):
        op, i, j, p = t
        assert t not in seen, f"task {t} listed twice"
        seen.add(t)
        if op == 0:
            blocks = range(p, P) if trans else range(p + 1)
            if order[i] >= 1:
                assert all(cnt[i, q] == order[i] - 1 and chain[i, q] == 1 for q in blocks), \
                    f"task {t} before its row's updates"
            done[i] += 1
        else:
            assert done[j] == P, f"task {t} before out_{j} is complete"
            if op == 2:
                assert order[j] == order[i] - 1, f"chain task {t} with a row other than the previous"
                chain[i, p] += 1
            else:
                assert order[j] <= order[i] - 2, f"in-place task {t} with the previous row or later"
                assert cnt[i, p] == order[j], f"task {t} out of column order"
                cnt[i, p] += 1
    assert np.all(done == P)
    for i in range(nt):
        assert np.all(cnt[i] == max(order[i] - 1, 0))
        assert np.all(chain[i] == (1 if order[i] >= 1 else 0))


@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("nt,P", [(1, 4), (2, 16), (3, 4), (7, 16), (32, 16), (64, 32)])
def test_solve_order_is_topological_and_complete(nt, P, trans):
    from paper_2406_02701_gb300 import mpchol
    tasks = mpchol.solve_dag_schedule(nt, P, trans)
    assert len(tasks) == nt * P + nt * (nt - 1) // 2 * P
    assert np.sum(tasks[:, 0] == 2) == (nt - 1) * P
    _replay_solve(tasks, nt, P, trans)


def test_solve_order_hands_out_the_chain_first():
    """The chain products of row s+1 and its diagonal blocks come together,
    ahead of the in-place updates with out_s."""
    from paper_2406_02701_gb300 import mpchol
    nt, P = 8, 4
    tasks = [tuple(t) for t in mpchol.solve_dag_schedule(nt, P, 0)]
    pos = {t: i for i, t in enumerate(tasks)}
    for s in range(nt - 2):
        assert pos[(0, s + 1, 0, 0)] == pos[(2, s + 1, s, P - 1)] + 1
        assert pos[(0, s + 1, 0, P - 1)] < pos[(1, s + 2, s, 0)]

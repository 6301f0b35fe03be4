"""The proof server's admission logic on a virtual clock (no GPU): FIFO
order, at most `slots` jobs at once, never more device memory admitted than
the budget, queue deadlines, jobs that can never fit."""
import random

import pytest

import paper_2603_10242_gb300 as ace


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ace.build()
    ace.lib()


def test_fifo_and_slot_cap():
    n = 10
    st, fi, status, peaks, _ = ace.scheduler_sim(2, 10**12, [0.0] * n, [1.0] * n, [1] * n)
    assert status == [0] * n
    assert st == [0, 0, 1, 1, 2, 2, 3, 3, 4, 4]
    assert fi == [s + 1 for s in st]
    assert peaks[0] == 2


def test_memory_budget_limits_concurrency():
    n = 6
    st, fi, status, peaks, _ = ace.scheduler_sim(3, 10, [0.0] * n, [1.0] * n, [6] * n)
    assert status == [0] * n and peaks[0] == 1 and peaks[1] == 6
    assert st == [0, 1, 2, 3, 4, 5]


def test_queue_deadline_and_never_fits():
    st, fi, status, _, _ = ace.scheduler_sim(1, 100, [0.0, 0.0, 0.1, 5.0], [1.0, 1.0, 1.0, 1.0], [10, 10, 10, 500],
                                          max_wait=0.5)
    assert status[0] == 0 and st[0] == 0
    assert status[1] == -6 and status[2] == -6          # could not start within 0.5 s
    assert status[3] == -2                               # larger than the budget


def test_random_load_invariants():
    rng = random.Random(5)
    n, slots, budget = 400, 3, 100
    t = 0.0
    arr, dur, mem = [], [], []
    for _ in range(n):
        t += rng.expovariate(1 / 0.4)
        arr.append(t)
        dur.append(rng.uniform(0.05, 1.2))
        mem.append(rng.randint(10, 60))
    st, fi, status, peaks, prio = ace.scheduler_sim(slots, budget, arr, dur, mem, max_wait=3.0)
    ran = [i for i in range(n) if status[i] == 0]
    assert len(ran) > n // 2
    for i in ran:
        assert st[i] >= arr[i] - 1e-12 and abs(fi[i] - st[i] - dur[i]) < 1e-9
        assert st[i] - arr[i] <= 3.0 + 1e-9
    # starts follow arrival order (FIFO)
    order = sorted(ran, key=lambda i: (st[i], i))
    assert order == sorted(ran)
    # at every start, running jobs <= slots and admitted memory <= budget
    for i in ran:
        live = [j for j in ran if st[j] <= st[i] < fi[j]]
        assert len(live) <= slots
        assert sum(mem[j] for j in live) <= budget
    assert peaks[0] <= slots and peaks[1] <= budget
    # a job's stream-priority level is the number of jobs running when it
    # started (jobs started at the same instant count if admitted before it)
    for i in ran:
        running = [j for j in ran if (st[j] < st[i] or (st[j] == st[i] and j < i)) and st[i] < fi[j]]
        assert prio[i] == len(running)


def test_priority_levels_follow_admission_order():
    # three overlapping jobs on three slots get levels 0, 1, 2; a job that
    # starts on an idle device gets level 0 again
    st, fi, status, _, prio = ace.scheduler_sim(3, 10**12, [0.0, 0.1, 0.2, 5.0], [1.0, 1.0, 1.0, 1.0], [1, 1, 1, 1])
    assert status == [0, 0, 0, 0]
    assert prio == [0, 1, 2, 0]
    # the first job finishes before the fourth of a busy stream starts: two running
    st, fi, status, _, prio = ace.scheduler_sim(3, 10**12, [0.0, 0.1, 0.2, 1.05], [1.0, 1.0, 1.0, 1.0], [1] * 4)
    assert prio == [0, 1, 2, 2]

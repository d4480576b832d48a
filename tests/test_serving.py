"""Host logic of the serving loop with a fake launcher and a fake clock (CPU):
first-come first-served admission, the device-byte budget, the in-flight slot
limit, rejection of requests larger than the budget, and that every admitted
request completes."""

import itertools

import pytest

from paper_2009_09500_gb300.serving import Admission, ServeRequest, Server


class FakeClock:
    def __init__(self, step=1e-4):
        self.t = 0.0
        self.step = step

    def __call__(self):
        self.t += self.step
        return self.t


class FakeHandle:
    def __init__(self, polls, log, reqs):
        self.polls = polls
        self.log = log
        self.reqs = reqs

    def done(self):
        self.polls -= 1
        return self.polls <= 0

    def finish(self):
        self.log.append(("done", [r.rid for r in self.reqs]))
        return 0


def make(n_req, dims=(64, 64, 64), n=1000, gap=1e-3):
    return [ServeRequest(rid=i, arrival_s=i * gap, n=n, dims=dims, voxels=n * 10) for i in range(n_req)]


def test_admission_fifo_and_budget():
    reqs = make(5)
    per = reqs[0].device_bytes
    adm = Admission(budget_bytes=3 * per + 1, max_batch_requests=10)
    import collections

    q = collections.deque(reqs)
    batch, rej = adm.take(q, bytes_in_use=0)
    assert [r.rid for r in batch] == [0, 1, 2] and not rej
    batch, rej = adm.take(q, bytes_in_use=3 * per)
    assert batch == [] and [r.rid for r in q] == [3, 4]


def test_admission_rejects_oversized():
    import collections

    big = ServeRequest(rid=9, arrival_s=0, n=10, dims=(1024, 1024, 1024))
    small = make(2)
    adm = Admission(budget_bytes=big.device_bytes - 1)
    q = collections.deque([big] + small)
    batch, rej = adm.take(q, 0)
    assert [r.rid for r in rej] == [9] and [r.rid for r in batch] == [0, 1]


@pytest.mark.parametrize("slots,polls", [(1, 3), (2, 5), (4, 50)])
def test_server_completes_everything_within_limits(slots, polls):
    reqs = make(60, gap=2e-4)
    per = reqs[0].device_bytes
    budget = 5 * per
    log = []
    launched = []

    def launcher(batch, slot):
        launched.append((slot, [r.rid for r in batch]))
        return FakeHandle(polls, log, batch)

    srv = Server(launcher, budget_bytes=budget, max_inflight=slots, max_batch_requests=3, clock=FakeClock(),
                 idle_sleep_s=0)
    st = srv.run(reqs)
    assert st.completed == 60 and st.rejected == 0 and st.failed == 0
    assert st.max_bytes_in_use <= budget
    assert st.max_inflight <= slots
    order = list(itertools.chain.from_iterable(ids for _, ids in launched))
    assert order == sorted(order) == list(range(60)), "admission keeps arrival order"
    assert all(len(ids) <= 3 for _, ids in launched)
    assert all(r.done_s >= r.admitted_s >= r.arrival_s for r in reqs)
    s = st.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["voxels"] == 60 * 10000


def test_server_counts_device_failures():
    reqs = make(4)

    class Bad(FakeHandle):
        def finish(self):
            return 2

    srv = Server(lambda b, s: Bad(1, [], b), budget_bytes=10**12, clock=FakeClock(), idle_sleep_s=0)
    st = srv.run(reqs)
    assert st.failed == 4 and st.completed == 0


def test_admission_follows_the_memory_probe():
    """With a memory probe, admission takes what the device has free (less the
    reserve) under the cap, and waits when the probe says memory is short."""
    import collections

    reqs = make(6)
    per = reqs[0].device_bytes
    free = {"bytes": 2 * per + 100}
    adm = Admission(budget_bytes=100 * per, max_batch_requests=10, mem_probe=lambda: free["bytes"],
                    reserve_bytes=50)
    q = collections.deque(reqs)
    batch, rej = adm.take(q, bytes_in_use=0)
    assert [r.rid for r in batch] == [0, 1] and not rej
    free["bytes"] = 10  # the device filled up meanwhile
    batch, _ = adm.take(q, bytes_in_use=2 * per)
    assert batch == []
    free["bytes"] = 3 * per + 50
    batch, _ = adm.take(q, bytes_in_use=2 * per)
    assert [r.rid for r in batch] == [2, 3, 4]


def test_server_with_probe_completes_and_respects_free_memory():
    reqs = make(30, gap=1e-4)
    per = reqs[0].device_bytes
    in_use = {"bytes": 0}
    device_total = 4 * per

    def launcher(batch, slot):
        in_use["bytes"] += sum(r.device_bytes for r in batch)
        assert in_use["bytes"] <= device_total, "admitted beyond the free memory"

        class H(FakeHandle):
            def finish(self):
                in_use["bytes"] -= sum(r.device_bytes for r in self.reqs)
                return 0

        return H(3, [], batch)

    srv = Server(launcher, budget_bytes=10**15, max_inflight=4, max_batch_requests=8, clock=FakeClock(),
                 idle_sleep_s=0, mem_probe=lambda: device_total - in_use["bytes"], reserve_bytes=0)
    st = srv.run(reqs)
    assert st.completed == 30 and st.max_bytes_in_use <= device_total

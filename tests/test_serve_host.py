"""Host logic of the serving layer, without a GPU: admission under a memory budget, LRU
eviction, refusal while an FDL is in use, clean rollback on an injected allocation failure,
and the bounded wait of the batch loop."""

import collections

import pytest
import torch

from paper_1901_06919_gb300.serve import AdmissionError, FdlStore, Server


def _views(K=4, C=1, H=16, W=16):
    return torch.zeros((K, C, H, W)), torch.zeros((K, 2)), torch.linspace(-1, 1, 4)


def test_admission_evicts_least_recently_used():
    one = FdlStore.fdl_bytes(4, 1, 16, 16)
    st = FdlStore(budget_bytes=2 * one + 10, device="cpu")
    v, u, d = _views()
    st.admit(1, v, u, d)
    st.admit(2, v, u, d)
    st.get(1)  # 1 is now more recent than 2
    st.admit(3, v, u, d)
    assert set(st.entries) == {1, 3}
    assert st.bytes_used <= st.budget


def test_admission_refuses_when_everything_is_in_use():
    one = FdlStore.fdl_bytes(4, 1, 16, 16)
    st = FdlStore(budget_bytes=one, device="cpu")
    v, u, d = _views()
    st.admit(1, v, u, d)
    st.entries[1].refs = 1  # read by an in-flight request
    with pytest.raises(AdmissionError):
        st.admit(2, v, u, d)
    assert list(st.entries) == [1]


def test_allocation_failure_rolls_back():
    calls = collections.Counter()

    def failing(shape, dtype):
        calls["n"] += 1
        if calls["n"] > 2:
            raise RuntimeError("out of memory (injected)")
        return torch.empty(shape, dtype=dtype)

    one = FdlStore.fdl_bytes(4, 1, 16, 16)
    st = FdlStore(budget_bytes=one, device="cpu", allocate=failing)
    v, u, d = _views()
    st.admit(1, v, u, d)
    with pytest.raises(AdmissionError):
        st.admit(2, v, u, d)  # would evict 1, but the allocation fails first
    assert list(st.entries) == [1]  # nothing was evicted
    with pytest.raises(AdmissionError):
        st.admit(1, v, u, d)  # duplicate id


class _FakeEvent:
    def __init__(self, done_after):
        self.n = done_after

    def query(self):
        self.n -= 1
        return self.n < 0


def test_is_ready_follows_the_fit_event_and_then_forgets_it():
    st = FdlStore(budget_bytes=FdlStore.fdl_bytes(4, 1, 16, 16), device="cpu")
    v, u, d = _views()
    st.admit(1, v, u, d)
    assert st.is_ready(1)  # no fit on the device: ready at once
    st.entries[1].ready = ev = _FakeEvent(done_after=2)
    assert not st.is_ready(1) and not st.is_ready(1)
    assert st.is_ready(1)
    assert st.entries[1].ready is None  # dropped: batches no longer wait on it
    calls = ev.n
    assert st.is_ready(1) and ev.n == calls  # not queried again


class _StuckBatch:
    busy = True
    requests = []

    class done:
        @staticmethod
        def query():
            return False


def test_drain_times_out_on_a_batch_that_never_completes():
    srv = Server.__new__(Server)
    srv.batches = [_StuckBatch()]
    srv.queue = collections.deque()
    srv.completed = []
    srv._fresh = []
    srv.store = FdlStore(1 << 20, "cpu")
    with pytest.raises(TimeoutError):
        srv.drain(timeout_s=0.05)

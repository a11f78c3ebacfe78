"""Host logic of the server (no GPU): the first-come-first-served memory budget
and the request stream."""
import threading
import time

from paper_2609_00535_b300 import inputs
from paper_2609_00535_b300.serve import Budget, Record, Stats


def test_budget_is_fifo_and_blocks_until_released():
    b = Budget(100)
    stop = threading.Event()
    order = []

    def take(name, n, delay):
        time.sleep(delay)
        assert b.acquire(n, stop)
        order.append(name)

    assert b.acquire(80, stop)                     # holds 80 of 100
    t1 = threading.Thread(target=take, args=("big", 60, 0.0))
    t2 = threading.Thread(target=take, args=("small", 10, 0.05))
    t1.start(); t2.start()
    time.sleep(0.2)
    assert order == []                             # small waits behind big (FIFO)
    b.release(80)
    t1.join(2); t2.join(2)
    assert order == ["big", "small"] and b.used == 70


def test_budget_admits_an_oversized_request_alone():
    b = Budget(10)
    stop = threading.Event()
    assert b.acquire(50, stop) and b.used == 50
    stop.set()
    assert not b.acquire(1, stop)


def test_request_stream_mix_and_arrivals():
    r = inputs.request_stream(n=400, rate=20.0, seed=5)
    assert len(r) == 400 and all(a.arrival < b.arrival for a, b in zip(r, r[1:]))
    kinds = {x.kind for x in r}
    assert kinds == {"flat2d", "cylinder2d", "sphere3d", "droplet2d", "droplet3d"}
    assert all(256 <= x.E <= 8192 and 4 <= x.N <= 7 for x in r)
    gaps = [b.arrival - a.arrival for a, b in zip(r, r[1:])]
    assert abs(sum(gaps) / len(gaps) - 1 / 20.0) < 0.01   # Poisson mean gap


def test_stats_percentiles():
    s = Stats(records=[Record(i, 0.0, finished=float(i + 1)) for i in range(100)], wall_s=10.0)
    assert s.percentile(50) in (50.0, 51.0) and s.percentile(99) == 99.0

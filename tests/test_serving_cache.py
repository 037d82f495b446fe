"""Host logic of the serving loop's plan cache (least-recently-used eviction within a byte
cap, idle plans counted against the same device budget as the requests in flight), with
stand-in plans: no GPU."""
import pytest

S = pytest.importorskip("paper_2305_07165_gb300.serving")


class FakePlan:
    def __init__(self, nbytes):
        self.nbytes, self.closed = nbytes, False

    def device_bytes(self):
        return self.nbytes

    def close(self):
        self.closed = True


def _server(budget, device_budget=1 << 40, used=0):
    srv = S.Server.__new__(S.Server)     # the cache alone: no streams, no device
    srv.cache, srv.cache_budget, srv.cache_bytes, srv.cache_hits = S.OrderedDict(), budget, 0, 0
    srv.budget, srv.used, srv.held = device_budget, used, 0
    return srv


def test_cache_take_put_and_lru_eviction():
    srv = _server(100)
    a, b, c = FakePlan(40), FakePlan(40), FakePlan(40)
    srv._cache_put("A", a)
    srv._cache_put("B", b)
    assert srv.cache_bytes == 80 and srv._cache_take("C") is None
    assert srv._cache_take("A") is a and srv.cache_hits == 1 and srv.cache_bytes == 40
    srv._cache_put("A", a)                # A is now the most recently used
    srv._cache_put("C", c)                # over budget: evicts B, the least recently used
    assert b.closed and not a.closed and not c.closed
    assert srv.cache_bytes == 80 and set(srv.cache) == {"A", "C"}


def test_cache_refuses_plans_larger_than_its_budget():
    srv = _server(10)
    p = FakePlan(11)
    srv._cache_put("X", p)
    assert p.closed and srv.cache_bytes == 0 and not srv.cache


def test_several_idle_plans_per_key():
    srv = _server(1000)
    p1, p2 = FakePlan(10), FakePlan(10)
    srv._cache_put("K", p1)
    srv._cache_put("K", p2)
    assert {id(srv._cache_take("K")), id(srv._cache_take("K"))} == {id(p1), id(p2)}
    assert srv._cache_take("K") is None and srv.cache_bytes == 0


def test_idle_plans_share_the_device_budget_with_requests_in_flight():
    """Requests in flight hold 60 of a 100-byte device budget: idle plans may keep only the other
    40, whatever the cache's own cap, evicting the least recently used first."""
    srv = _server(1000, device_budget=100, used=60)
    a, b, c = FakePlan(20), FakePlan(20), FakePlan(30)
    srv._cache_put("A", a)
    srv._cache_put("B", b)
    assert srv._resident() == 100 and not a.closed and not b.closed
    srv._cache_put("C", c)                # 60 + 20 + 30 fits only after A and B leave
    assert a.closed and b.closed and not c.closed and srv._resident() == 90
    big = FakePlan(41)                    # larger than what the requests leave free: released at once
    srv._cache_put("D", big)
    assert big.closed and "D" not in srv.cache and srv._resident() <= 100

"""Scheduling logic of the continuous-batching server with a fake backend
(no GPU): admission in arrival order under an HBM budget, no step past a
solve's own count, retirement when done, latency bookkeeping."""
from paper_1808_03801_gb300.serve import Request, Server, percentile


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeSim:
    def __init__(self, w):
        self.w = w
        self.steps = 0
        self.bytes = w["bytes"]

    def info(self):
        return {"n_particles": self.w["n"], "device_bytes": self.bytes}

    def sample(self, averaged=False):
        return ("fields", self.steps)

    def close(self):
        pass


class FakeBatch:
    def __init__(self, budget, max_sims, clock):
        self.budget, self.max_sims, self.clock = budget, max_sims, clock
        self.members = []
        self.log = []

    def admit(self, s):
        used = sum(m.bytes for m in self.members)
        if len(self.members) >= self.max_sims or used + s.bytes > self.budget:
            return -4
        self.members.append(s)
        return 0

    def retire(self, s):
        self.members.remove(s)

    def step(self, k):
        self.log.append((k, len(self.members)))
        for m in self.members:
            m.steps += k
        self.clock.t += 0.001 * k


def _server(budget, max_sims=8, chunk=8):
    clock = FakeClock()
    holder = {}

    def make_batch(b, m):
        holder["b"] = FakeBatch(b, m, clock)
        return holder["b"]

    srv = Server(FakeSim, make_batch, budget, max_sims=max_sims, chunk=chunk, clock=clock)
    return srv, holder["b"], clock


def test_every_solve_gets_exactly_its_steps_and_latency_is_recorded():
    srv, batch, clock = _server(budget=100)
    steps = [5, 13, 8, 21, 3]
    for i, s in enumerate(steps):
        srv.submit(Request(0.002 * i, i, {"n": 100 * (i + 1), "bytes": 10}, s))
    rep = srv.run(idle_sleep=0)
    assert rep["requests"] == 5
    for r in srv.finished:
        assert r.result["sim"].steps == r.steps
        assert r.done >= r.admitted >= r.arrival
    assert all(k <= 8 for k, _ in batch.log)
    assert rep["particle_updates"] == sum(100 * (i + 1) * s for i, s in enumerate(steps))


def test_budget_limits_residency_and_arrival_order_is_kept():
    srv, batch, clock = _server(budget=25)        # two solves of 10 bytes fit, not three
    for i in range(6):
        srv.submit(Request(0.0, i, {"n": 10, "bytes": 10}, 4 + i))
    srv.run(idle_sleep=0)
    assert max(n for _, n in batch.log) == 2
    order = [r.rid for r in sorted(srv.finished, key=lambda r: r.admitted)]
    assert order == sorted(order)


def test_percentiles():
    v = list(range(1, 101))
    assert percentile(v, 50) == 50.5
    assert abs(percentile(v, 99) - 99.01) < 1e-9

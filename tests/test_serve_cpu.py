"""Host logic of the continuous-batching scheduler, with a fake executor and clock."""
import numpy as np
import pytest

import fem_inputs as FI
from paper_2402_15940_b300.serve import FakeExecutor, Request, Server, device_bytes, poisson_arrivals


class FakeClock:
    def __init__(self, dt=1.0):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def reqs(specs):
    return [Request(rid=i, form=f, p=p, n=(n, n, n), mesh_seed=i, arrival=a) for i, (f, p, n, a) in enumerate(specs)]


def test_device_bytes_grows_with_size_and_precision():
    a = Request(0, "diffusion", 4, (8, 8, 8), 0)
    b = Request(1, "diffusion", 4, (16, 16, 16), 0)
    c = Request(2, "diffusion", 4, (16, 16, 16), 0, precision="mixed")
    m = Request(3, "mass", 4, (16, 16, 16), 0)
    assert device_bytes(a) < device_bytes(b) < device_bytes(c)
    assert device_bytes(m) < device_bytes(b)
    # FP64 D alone for p=4 diffusion: 48 q^3 bytes per element
    assert device_bytes(b) > 48 * 216 * 16 ** 3


def test_all_complete_and_budget_respected():
    rs = reqs([("diffusion", (i % 6) + 1, 4 + i % 5, 0.0) for i in range(40)])
    budget = 3 * max(device_bytes(r) for r in rs)
    srv = Server(FakeExecutor(lambda r: 10 + 7 * r.rid), hbm_budget=budget, tick_iters=8, clock=FakeClock())
    out = srv.run(rs)
    assert [o.rid for o in out] == list(range(40))
    assert all(o.iterations == 10 + 7 * o.rid for o in out)
    assert srv.peak_in_use <= budget and srv.in_use == 0
    assert srv.max_concurrent >= 2


def test_late_short_request_overtakes_long_one():
    # a long request is running when a short one arrives: the short one is admitted at the
    # next tick boundary and finishes first (continuous batching, not a queue)
    rs = reqs([("diffusion", 2, 4, 0.0), ("mass", 2, 4, 5.0)])
    need = {0: 1000, 1: 16}
    srv = Server(FakeExecutor(lambda r: need[r.rid]), hbm_budget=1e12, tick_iters=8, clock=FakeClock())
    out = {o.rid: o for o in srv.run(rs)}
    assert out[1].admitted < out[0].finished
    assert out[1].finished < out[0].finished
    assert srv.max_concurrent == 2


def test_fifo_admission_under_memory_pressure():
    rs = reqs([("diffusion", 3, 10, 0.0), ("diffusion", 3, 10, 0.0), ("mass", 1, 2, 0.0), ("diffusion", 3, 10, 0.0)])
    budget = device_bytes(rs[0]) * 1.5   # one big request at a time
    ex = FakeExecutor(lambda r: 20)
    srv = Server(ex, hbm_budget=budget, tick_iters=4, clock=FakeClock())
    srv.run(rs)
    starts = [rid for kind, rid in ex.log if kind == "start"]
    assert starts == [0, 1, 2, 3]          # the small one does not jump the queue
    assert srv.peak_in_use <= budget


def test_oversize_request_rejected_not_blocking():
    rs = reqs([("diffusion", 8, 60, 0.0), ("mass", 1, 2, 0.0)])
    srv = Server(FakeExecutor(lambda r: 5), hbm_budget=device_bytes(rs[1]) * 4, clock=FakeClock())
    out = srv.run(rs)
    assert srv.rejected == [0] and [o.rid for o in out] == [1]


def test_report_percentiles_and_poisson_arrivals():
    rs = reqs([("mass", 1, 2, 0.0) for _ in range(200)])
    poisson_arrivals(rs, rate=50.0, seed=3)
    gaps = np.diff([0.0] + [r.arrival for r in rs])
    assert abs(gaps.mean() - 1 / 50.0) < 0.2 / 50.0
    srv = Server(FakeExecutor(lambda r: 3), hbm_budget=1e12, tick_iters=1, clock=FakeClock(dt=0.001))
    srv.run(rs)
    rep = srv.report()
    assert rep["completed"] == 200 and rep["p50_latency_s"] <= rep["p99_latency_s"]


def test_serve_request_generator():
    r = FI.serve_requests(500, seed=1)
    assert {x["form"] for x in r} == {"mass", "diffusion"}
    assert min(x["p"] for x in r) == 1 and max(x["p"] for x in r) == 8
    n = np.array([(x["p"] * x["n"][0] + 1) ** 3 for x in r])
    assert n.min() >= 8 and n.max() < 1.5e7
    assert 0.35 < np.mean([x["precision"] == "mixed" for x in r]) < 0.65


def test_sjf_admits_the_least_work_first():
    # one slot, everything waiting at once: with "sjf" the requests start in order of
    # estimated work (the arrival order under "fifo")
    from paper_2402_15940_b300.serve import estimated_work
    rs = reqs([("diffusion", 4, 12, 0.0), ("diffusion", 4, 12, 0.0), ("mass", 1, 2, 0.0), ("diffusion", 2, 5, 0.0)])
    for policy, order in (("sjf", sorted(rs, key=lambda r: (estimated_work(r), r.arrival, r.rid))), ("fifo", rs)):
        ex = FakeExecutor(lambda r: 10)
        srv = Server(ex, hbm_budget=1e12, tick_iters=4, max_active=1, clock=FakeClock(), policy=policy)
        srv.run(rs)
        assert [rid for kind, rid in ex.log if kind == "start"] == [r.rid for r in order]
    with pytest.raises(ValueError):
        Server(FakeExecutor(lambda r: 1), policy="lifo")


def test_estimated_work_orders_by_size_order_and_precision():
    from paper_2402_15940_b300.serve import estimated_work
    a = Request(0, "diffusion", 2, (8, 8, 8), 0)
    b = Request(1, "diffusion", 4, (8, 8, 8), 0)
    c = Request(2, "diffusion", 4, (8, 8, 8), 0, precision="mixed")
    assert estimated_work(a) < estimated_work(b) and estimated_work(c) < estimated_work(b)


def test_one_advance_in_flight_per_request():
    # while a request's last advance is still running (poll returns None) the scheduler does not
    # queue another one; it resumes once the poll reports a state
    class BusyFake(FakeExecutor):
        def __init__(self):
            super().__init__(lambda r: 40)
            self.busy_left = {}
            self.advances = 0

        def advance(self, h, iters):
            assert self.busy_left.get(h["req"].rid, 0) == 0, "advanced while busy"
            self.advances += 1
            self.busy_left[h["req"].rid] = 3
            super().advance(h, iters)

        def poll(self, h):
            rid = h["req"].rid
            if self.busy_left.get(rid, 0) > 0:
                self.busy_left[rid] -= 1
                return None
            return super().poll(h)

    ex = BusyFake()
    srv = Server(ex, hbm_budget=1e12, tick_iters=8, clock=FakeClock())
    out = srv.run(reqs([("diffusion", 2, 4, 0.0), ("mass", 3, 3, 0.0)]))
    assert len(out) == 2 and all(o.iterations == 40 for o in out)
    assert ex.advances == 2 * 5          # 40 iterations in advances of 8, nothing extra queued


def test_tick_size_scales_with_the_request():
    srv = Server(FakeExecutor(lambda r: 1), tick_iters=16, tick_seconds=2e-3)
    small = Request(0, "mass", 2, (4, 4, 4), 0)
    big = Request(1, "diffusion", 4, (48, 48, 48), 0)
    assert srv.tick_size(small) == 4096 and 16 <= srv.tick_size(big) < 4096
    assert Server(FakeExecutor(lambda r: 1), tick_iters=16).tick_size(big) == 16


def test_solver_policy_gives_large_diffusion_requests_multigrid():
    """solver="auto": diffusion requests of at least pmg_min_dofs DOFs get the p-multigrid
    preconditioner, smaller ones and mass requests keep Jacobi; the estimates follow the choice
    (more device memory for the levels, less estimated work) and pmg requests advance by 1 to 4
    of their iterations per tick."""
    from paper_2402_15940_b300.serve import estimated_work
    rs = reqs([("diffusion", 4, 12, 0.0), ("diffusion", 2, 3, 0.0), ("mass", 4, 12, 0.0), ("diffusion", 6, 8, 1.0)])
    srv = Server(FakeExecutor(lambda r: 30), hbm_budget=1e12, tick_iters=8, clock=FakeClock(), solver="auto",
                 pmg_min_dofs=20000, tick_seconds=2e-3)
    out = srv.run(rs)
    assert len(out) == 4
    assert [r.solver for r in rs] == ["pmg", "jacobi", "jacobi", "pmg"]
    assert srv.report()["pmg_requests"] == 2 and srv.report()["solver"] == "auto"
    assert all(1 <= srv.tick_size(r) <= 4 for r in rs if r.solver == "pmg")
    j = Request(9, "diffusion", 4, (12, 12, 12), 0)
    m = Request(9, "diffusion", 4, (12, 12, 12), 0, solver="pmg")
    assert device_bytes(m) > device_bytes(j)
    assert estimated_work(m) < estimated_work(j)
    # with the Jacobi policy nothing changes
    rs2 = reqs([("diffusion", 4, 12, 0.0)])
    Server(FakeExecutor(lambda r: 30), hbm_budget=1e12, clock=FakeClock()).run(rs2)
    assert rs2[0].solver == "jacobi"
    with pytest.raises(ValueError):
        Server(FakeExecutor(lambda r: 1), solver="amg")

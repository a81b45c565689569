"""Host logic of bench.py on CPU: the synthetic workloads follow their stated recipes (the
256-instance ensemble, the serving stream's arrival order, ranges and time-step bounds, the
CFL eigenvalue the time steps use), the serving replay's latency figures are consistent
when the server is a fake that takes one step of every admitted request per tick and admits
at most two requests per tick, and the per-class roofline arithmetic of the line recomputes
from the algorithmic work and the timings."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class FakeImex:
    REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_FAILED = range(4)
    MIXED, FP64 = 1, 0
    FLOW_TG2D, FLOW_TG3D, FLOW_TGTRAVEL = 1, 2, 3
    NU_CONST, NU_VARXYT = 0, 1
    FORCE_TGTRAVEL_VARNU = 4

    class Server:
        TICK_S = 0.002

        def __init__(self, budget_bytes, precision, tol, maxit):
            self.reqs, self.order, self.ticks, self.tick_ms = {}, [], 0, []
            self.dof_stages = 0.0

        def submit(self, **req):
            i = len(self.order)
            self.reqs[i] = {"req": req, "state": FakeImex.REQ_QUEUED, "done": 0}
            self.order.append(i)
            return i

        def tick(self):
            t0 = time.perf_counter()
            admitted = 0
            for i in self.order:
                r = self.reqs[i]
                if r["state"] == FakeImex.REQ_QUEUED and admitted < 2:
                    r["state"] = FakeImex.REQ_ACTIVE
                    admitted += 1
            active = 0
            for i in self.order:
                r = self.reqs[i]
                if r["state"] != FakeImex.REQ_ACTIVE:
                    continue
                active += 1
                r["done"] += 1
                q = r["req"]
                n = q["dim"] * (q["P"] + 1) ** q["dim"]
                for k in q["nelem"]:
                    n *= k
                self.dof_stages += 3 * n
                if r["done"] == q["nsteps"]:
                    r["state"] = FakeImex.REQ_DONE
            time.sleep(self.TICK_S)
            self.ticks += 1
            self.tick_ms.append(1e3 * (time.perf_counter() - t0))
            return active

        def poll(self, i):
            r = self.reqs[i]
            return r["state"], r["done"], 0.0

        def stats(self):
            st = [r["state"] for r in self.reqs.values()]
            ms = sorted(self.tick_ms) or [0.0]
            return {"active": st.count(FakeImex.REQ_ACTIVE), "queued": st.count(FakeImex.REQ_QUEUED),
                    "completed": st.count(FakeImex.REQ_DONE), "failed": st.count(FakeImex.REQ_FAILED),
                    "p50_tick_ms": ms[len(ms) // 2], "p99_tick_ms": ms[-1], "ticks": self.ticks,
                    "dof_stages": self.dof_stages, "busy_s": 1e-3 * sum(self.tick_ms),
                    "max_footprint_bytes": 0.0, "budget_bytes": 1e9}

        def last_error(self):
            return ""

        def close(self):
            pass


def test_stream_recipe():
    s = bench.serving_stream(400)
    arr = [q["arrival"] for q in s]
    assert all(b > a for a, b in zip(arr, arr[1:]))
    # Poisson arrivals at 50 per second: the mean gap is 1/50 s within sampling error
    assert abs(arr[-1] / len(arr) - 0.02) < 0.004
    for q in s:
        assert q["d"] in (2, 3) and 10 <= q["steps"] <= 100
        if q["d"] == 2:
            assert 4 <= q["K"] <= 32 and 3 <= q["P"] <= 8 and q["flow"] in ("tg", "mms")
        else:
            assert 4 <= q["K"] <= 24 and 3 <= q["P"] <= 7 and q["flow"] == "tg"
    assert {q["d"] for q in s} == {2, 3} and {q["flow"] for q in s} == {"tg", "mms"}
    assert bench.serving_stream(50) == s[:50]  # the stream is a prefix-stable seeded sequence


def test_request_time_steps():
    for q in bench.serving_stream(200):
        r = bench.serving_request(FakeImex, q)
        K, P = q["K"], q["P"]
        assert r["nsteps"] == q["steps"] and r["P"] == P and r["dim"] == q["d"]
        if q["flow"] == "mms":
            h, nu0 = 1.0 / K, 0.01
            assert r["dt"] <= 4.0 * h * h / (nu0 * (P + 1) ** 4) * (1 + 1e-12)
            assert r["dt"] <= 0.3 / (5 ** 0.5 * bench.rho_hat(P) * 2.0 / h) * (1 + 1e-12)
            assert r["periodic"] == (0, 0)
        else:
            h = bench.TWO_PI / K
            assert r["dt"] == pytest.approx(0.3 / (bench.rho_hat(P) * 2.0 / h))
            assert all(r["periodic"])


def test_replay_latencies():
    n = 6
    out = bench.run_serving(FakeImex, n)
    assert out["requests"] == n and out["completed"] == n and out["failed"] == 0
    stream = bench.serving_stream(n)
    ticks_min = max(q["steps"] for q in stream)
    assert out["ticks"] >= ticks_min
    # a request steps once per tick, so its own step latency is about one tick
    tick_ms = 1e3 * FakeImex.Server.TICK_S
    assert tick_ms * 0.9 <= out["p50_request_step_ms"] <= out["p99_request_step_ms"]
    assert out["p50_request_step_ms"] < 5 * out["p99_step_ms"]
    # end-to-end latency covers queueing plus every step
    assert out["p50_queue_wait_s"] >= 0.0
    assert out["p99_request_latency_s"] >= 1e-3 * out["p50_request_step_ms"] * min(q["steps"] for q in stream)
    assert out["value"] > 0 and out["dof_stages"] > 0


def test_cfl_eigenvalue():
    """rho_hat(P), the largest eigenvalue modulus of the GLL collocation derivative with the
    inflow node removed, has the values the workloads' CFL_lambda numbers rest on
    (rho_hat(7) = 5.656, rho_hat(8) = 6.967) and grows with P."""
    assert bench.rho_hat(7) == pytest.approx(5.656, abs=5e-4)
    assert bench.rho_hat(8) == pytest.approx(6.967, abs=5e-4)
    r = [bench.rho_hat(P) for P in range(2, 9)]
    assert all(b > a for a, b in zip(r, r[1:]))


def test_ensemble_recipe():
    """256 decaying Taylor-Green instances from seed 0: K in 4..32, P in 3..8 (six degree
    groups), nu in [1e-3, 1e-1], dt at CFL_lambda = 0.3; 9,851,694 velocity DOF in all."""
    s = bench.ensemble_specs()
    assert len(s) == 256 and s == bench.ensemble_specs()
    assert {P for _, P, _, _ in s} == set(range(3, 9))
    for K, P, nu, dt in s:
        assert 4 <= K <= 32 and 3 <= P <= 8 and 1e-3 <= nu <= 1e-1
        assert 0.3 == pytest.approx(dt * bench.rho_hat(P) * 2.0 / (bench.TWO_PI / K))
    assert sum(2 * K * K * (P + 1) ** 2 for K, P, _, _ in s) == 9851694


class FakeProfiledContext:
    """Per-class launches / milliseconds and algorithmic work, as imex_profile_read and
    imex_profile_work return them."""

    def __init__(self, rows):
        self.rows = rows

    def profile_read(self, cls):
        r = self.rows.get(cls)
        return (r[0], r[1]) if r else (0, 0.0)

    def profile_work(self, cls):
        r = self.rows.get(cls)
        return (r[2], r[3], r[4]) if r else (0.0, 0.0, 0)


def test_operator_table_and_roofline():
    """Achieved GB/s and GFLOP/s are the algorithmic work over the CUDA-event time, the
    fractions divide by the HBM copy rate or the ALU peak of the class's arithmetic, and the
    roofline names the class with the largest time, bound by the larger of its two fractions,
    with the DRAM traffic of that class's capture."""
    import types
    names = ["a_fp32", "b_ff", "c_fp64"]
    imex = types.SimpleNamespace(PROF_NAMES=names)
    hbm = 8000.0
    # (launches, total ms, bytes, flops, arith) per class; b_ff has the largest time
    ctx = FakeProfiledContext({0: (100, 2.0, 100 * 8e6, 100 * 1e6, 1),
                               1: (4, 5.0, 4 * 1e8, 4 * 2.8e9, 3),
                               2: (10, 1.0, 10 * 1.6e7, 0.0, 0)})
    rows = bench.operator_table(imex, ctx, hbm)
    a = rows["a_fp32"]
    assert a["avg_us"] == pytest.approx(20.0) and a["bytes_per_launch"] == pytest.approx(8e6)
    assert a["gbs"] == pytest.approx(100 * 8e6 / 2e-3 / 1e9) and a["hbm_frac"] == pytest.approx(a["gbs"] / hbm)
    assert a["alu_peak_gflops"] == pytest.approx(bench.FP32_PEAK_GFLOPS)
    assert rows["b_ff"]["alu_peak_gflops"] == pytest.approx(bench.FP32_PEAK_GFLOPS * 2 / 15)
    assert rows["c_fp64"]["flops_per_launch"] is None and "alu_frac" not in rows["c_fp64"]
    roof = bench.roofline_of(rows, hbm, "measured", traffic={"b_ff": 6.6e7})
    assert roof["kernel"] == "b_ff" and roof["bound"] == "alu" and roof["unit"] == "GFLOP/s"
    assert roof["achieved"] == pytest.approx(4 * 2.8e9 / 5e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["traffic"] == 6.6e7 and roof["avg_launch_us"] == pytest.approx(1250.0)
    assert roof["share_of_profiled_ms"] == pytest.approx(5.0 / 8.0)
    # an HBM-bound dominant class reports GB/s against the copy rate, traffic unknown: None
    ctx2 = FakeProfiledContext({2: (10, 9.0, 10 * 6e8, 0.0, 0)})
    roof2 = bench.roofline_of(bench.operator_table(imex, ctx2, hbm), hbm, "measured")
    assert roof2["bound"] == "hbm" and roof2["unit"] == "GB/s" and roof2["traffic"] is None
    assert roof2["frac"] == pytest.approx(10 * 6e8 / 9e-3 / 1e9 / hbm)
    assert bench.roofline_of({}, hbm, "measured") is None


def test_whole_job_value():
    """The whole-job throughput is all ranks' units over the slowest rank's time."""
    assert bench.job_value(4, 1e6, 2.0) == pytest.approx(2e6)

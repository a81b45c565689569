"""GPU parity of the serving form: requests that arrive, wait for room under an HBM budget,
join and leave the union-mesh groups between steps (continuous batching) finish with the
same fields as each request run alone through one context (FP64 solves to 1e-13: 1e-10
relative; the mixed form, whose FP32 inner iterations run differently in a group than
alone, with its FP64 refinement to 1e-12: 1e-9 relative), and the active footprint never
exceeds the budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
TWO_PI = 2 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def tg2d(P, K, nu, dt, n):
    return dict(dim=2, P=P, nelem=(K, K), lo=(0, 0), hi=(TWO_PI, TWO_PI), periodic=(1, 1), flow=imex.FLOW_TG2D,
                flow_params=[nu], nu_kind=imex.NU_CONST, nu_params=[nu], dt=dt, nsteps=n)


def tg3d(P, K, nu, dt, n):
    return dict(dim=3, P=P, nelem=(K, K, K), lo=(0, 0, 0), hi=(TWO_PI,) * 3, periodic=(1, 1, 1),
                flow=imex.FLOW_TG3D, nu_kind=imex.NU_CONST, nu_params=[nu], dt=dt, nsteps=n)


def mms(P, K, nu0, dt, n):
    return dict(dim=2, P=P, nelem=(K, K), lo=(0, 0), hi=(1, 1), periodic=(0, 0), flow=imex.FLOW_TGTRAVEL,
                flow_params=[nu0], nu_kind=imex.NU_VARXYT, nu_params=[nu0], bc_kind=imex.FLOW_TGTRAVEL,
                bc_params=[nu0], f_kind=imex.FORCE_TGTRAVEL_VARNU, f_params=[nu0], dt=dt, nsteps=n)


def alone(r, precision=imex.FP64, tol=1e-13):
    c = imex.Context(r["dim"], r["P"], r["nelem"], r["lo"], r["hi"], r["periodic"], precision=precision, tol=tol,
                     maxit=50000)
    if r["nu_kind"] == imex.NU_CONST:
        c.set_viscosity_const(r["nu_params"][0])
    else:
        c.set_viscosity_model(r["nu_kind"], r["nu_params"])
    if r.get("bc_kind"):
        c.set_boundary(r["bc_kind"], r["bc_params"])
    if r.get("f_kind"):
        c.set_forcing(r["f_kind"], r["f_params"])
    c.init_flow(r["flow"], r.get("flow_params", ()), 0.0)
    c.step(r["dt"], r["nsteps"])
    return c.get_velocity()


def footprint(r):
    return imex.Server.footprint(**r)


def test_continuous_batching_matches_alone():
    reqs = [tg2d(4, 3, 0.01, 0.02, 4), tg2d(4, 5, 0.03, 0.01, 2), mms(4, 3, 0.01, 0.005, 3),
            tg3d(3, 2, 1e-3, 0.02, 3), tg2d(4, 2, 0.002, 0.03, 5), tg2d(5, 4, 0.01, 0.01, 1),
            mms(4, 2, 0.02, 0.01, 2)]
    # room for about two of the larger requests at a time: the rest must queue
    budget = 2.2 * max(footprint(r) for r in reqs)
    sv = imex.Server(budget_bytes=budget, precision=imex.FP64, tol=1e-13, maxit=50000, keep_results=True)
    ids = [sv.submit(**reqs[0]), sv.submit(**reqs[1])]
    sv.tick()
    for r in reqs[2:]:                      # later arrivals, while the first ones run
        ids.append(sv.submit(**r))
    queued_seen = False
    for _ in range(200):
        sv.tick()
        st = sv.stats()
        queued_seen = queued_seen or st["queued"] > 0
        assert st["footprint_bytes"] <= budget
        if st["completed"] + st["failed"] == len(reqs):
            break
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_footprint_bytes"] <= budget
    assert queued_seen
    for i, r in zip(ids, reqs):
        state, steps, t = sv.poll(i)
        assert state == imex.REQ_DONE and steps == r["nsteps"]
        assert t == pytest.approx(r["nsteps"] * r["dt"], rel=1e-14)
        assert rel(sv.result(i), alone(r)) < 1e-10, i


def test_request_larger_than_budget_fails_alone():
    sv = imex.Server(budget_bytes=1e4, precision=imex.FP64)
    i = sv.submit(**tg2d(3, 4, 0.01, 0.01, 2))
    sv.tick()
    assert sv.poll(i)[0] == imex.REQ_FAILED
    with pytest.raises(imex.ImexError):
        sv.submit(**dict(tg2d(3, 4, 0.01, 0.01, 2), dt=-1.0))


def test_server_groups_join_and_leave_repeatedly():
    # requests of one group arriving one per tick with staggered lengths: the group is
    # repacked on every tick (members join and leave) and grows past its first capacity
    reqs = [tg2d(4, 2 + (i % 4), 0.01 * (1 + i % 3), 0.01, 1 + i % 5) for i in range(12)]
    sv = imex.Server(budget_bytes=0.0, precision=imex.FP64, tol=1e-13, maxit=50000, keep_results=True)
    ids = []
    for r in reqs:
        ids.append(sv.submit(**r))
        sv.tick()
    for _ in range(20):
        if sv.tick() == 0 and sv.stats()["queued"] == 0:
            break
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for i, r in zip(ids, reqs):
        assert rel(sv.result(i), alone(r)) < 1e-10, i


def test_continuous_batching_mixed_matches_alone():
    """The served form as the serving workload runs it (IMEX_MIXED): every request of the
    mix equals the same request run alone in the mixed form, and the FP64 form, to the
    solver tolerance."""
    reqs = [tg2d(4, 3, 0.01, 0.02, 4), mms(4, 3, 0.01, 0.005, 3), tg3d(3, 2, 1e-3, 0.02, 3),
            tg2d(5, 4, 0.01, 0.01, 2), tg3d(4, 3, 1e-3, 0.02, 2), mms(5, 2, 0.02, 0.01, 2)]
    budget = 2.5 * max(footprint(r) for r in reqs)
    sv = imex.Server(budget_bytes=budget, precision=imex.MIXED, tol=1e-12, maxit=50000, keep_results=True)
    ids = [sv.submit(**reqs[0])]
    sv.tick()
    for r in reqs[1:]:
        ids.append(sv.submit(**r))
        sv.tick()
    for _ in range(100):
        if sv.tick() == 0 and sv.stats()["queued"] == 0:
            break
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_footprint_bytes"] <= budget
    for i, r in zip(ids, reqs):
        got = sv.result(i)
        assert rel(got, alone(r, precision=imex.MIXED, tol=1e-12)) < 1e-9, i
        assert rel(got, alone(r)) < 1e-9, i

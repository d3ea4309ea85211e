"""Serving by continuous batching (pa_server_*): requests of mixed lattice
sizes, schedules and population sizes, admitted by a device-memory budget
that forces queueing, each give the same result, bit for bit, as the same
run alone through pa_create/pa_step, and the oracle's population sizes and
energies."""
import numpy as np
import pytest

from oracle import oracle as o
from paper_1006_0252_gb300 import inputs, pa

pytestmark = pytest.mark.gpu


def _requests():
    reqs = []
    for k, (dim, L, R0, nb, theta) in enumerate([(3, 4, 700, 9, 3), (3, 8, 2000, 6, 2), (3, 6, 1500, 12, 2),
                                                  (1, 96, 900, 8, 3), (3, 4, 300, 15, 4), (3, 10, 800, 5, 2),
                                                  (3, 6, 1200, 7, 3)]):
        J = inputs.couplings_3d(L, k, 1) if dim == 3 else inputs.couplings_chain(L, k, 1)
        betas = inputs.linear_schedule(0.2 * nb, nb + 1)[1:]
        reqs.append(dict(dim=dim, L=L, J=J, R0=R0, seed=500 + k, betas=betas, theta=theta))
    return reqs


def test_served_runs_equal_runs_alone_and_the_oracle():
    reqs = _requests()
    srv = pa.Server(hbm_budget_bytes=0, max_runs=4)
    ids = [srv.submit(q["dim"], q["L"], q["J"], q["R0"], q["seed"], q["betas"], q["theta"]) for q in reqs]
    max_active, ticks = 0, 0
    while True:
        a, qd, f = srv.tick(2)
        max_active = max(max_active, a + f)
        ticks += 1
        if a == 0 and qd == 0:
            break
        assert ticks < 200
    assert max_active <= 4
    for q, rid in zip(reqs, ids):
        res = srv.result(rid, traj_count=len(q["betas"]) + 1)
        assert res["status"] == 2 and res["steps"] == len(q["betas"])
        alone = pa.Run(q["J"], q["L"], q["dim"], q["R0"], q["seed"])
        for b in q["betas"]:
            alone.step(float(b), q["theta"])
        obs = alone.observables()
        assert res["R"] == obs["R"] and res["sumE"] == obs["sumE"] and res["sumE2"] == obs["sumE2"]
        assert res["minus_beta_F"] == obs["minus_beta_F"]
        assert np.array_equal(res["trajectory"], alone.trajectory()["minus_beta_F"])
        if q["dim"] == 3:
            c = o.Run(q["J"], 3, q["L"], q["L"], q["L"], 7, R0=q["R0"], seed=q["seed"],
                      R_cap=inputs.default_capacity(q["R0"]))
        else:
            c = o.Run(q["J"], 1, q["L"], R0=q["R0"], seed=q["seed"], R_cap=inputs.default_capacity(q["R0"]))
        for b in q["betas"]:
            c.step(float(b), q["theta"], q["R0"])
        st = c.state()
        assert res["R"] == st.R and res["sumE"] == st.sumE
        assert abs(res["minus_beta_F"] - st.minus_beta_F) <= 1e-12 * abs(st.minus_beta_F)
        assert res["done_s"] >= res["admit_s"] >= res["submit_s"]


def test_memory_budget_limits_concurrency():
    reqs = _requests()
    srv0 = pa.Server()
    rid = srv0.submit(3, 8, reqs[1]["J"], reqs[1]["R0"], 1, reqs[1]["betas"], 1)
    need = srv0.result(rid)["device_bytes"]
    srv0.close()
    srv = pa.Server(hbm_budget_bytes=2.5 * need, max_runs=16)
    for k in range(6):
        srv.submit(3, 8, reqs[1]["J"], reqs[1]["R0"], 10 + k, reqs[1]["betas"], 1)
    seen = 0
    while True:
        a, qd, f = srv.tick(1)
        seen = max(seen, a + f)
        if a == 0 and qd == 0:
            break
    assert seen == 2  # budget admits two such runs at a time
    with pytest.raises(pa.PAError) as e:
        pa.Server(hbm_budget_bytes=need / 2).submit(3, 8, reqs[1]["J"], reqs[1]["R0"], 1, reqs[1]["betas"], 1)
    assert e.value.code == pa.PA_ERR_OOM

"""Writes the oracle regression fixtures in this folder.  Calls only the
oracle and the seeded input generators; run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as o  # noqa: E402
from paper_1006_0252_gb300 import inputs  # noqa: E402


def trajectory(spec, n_steps):
    J = spec.couplings()
    L = spec.L
    if spec.dim == 3:
        r = o.Run(J, 3, L, L, L, 7, R0=spec.R0, R_cap=inputs.default_capacity(spec.R0), seed=spec.seed)
    else:
        r = o.Run(J, 1, L, R0=spec.R0, R_cap=inputs.default_capacity(spec.R0), seed=spec.seed)
    rows = []
    st = r.state()
    rows.append(dict(beta=st.beta, R=st.R, minus_beta_F=st.minus_beta_F.hex(), sumE=st.sumE, sumE2=st.sumE2))
    for k in range(1, n_steps + 1):
        r.step(float(spec.betas[k]), spec.theta, spec.R0)
        st = r.state()
        rows.append(dict(beta=st.beta, R=st.R, minus_beta_F=st.minus_beta_F.hex(),
                         lnQ=st.lnQ_last.hex(), sumE=st.sumE, sumE2=st.sumE2))
    return rows


def main():
    spec = inputs.config_small_3d()[0]
    out = dict(workload="3D L=4 periodic, couplings seed 1, R0=1000, beta 0..5 in 101 values, "
                        "theta=10, PA seed 1: first 12 annealing steps",
               rows=trajectory(spec, 12))
    with open(os.path.join(HERE, "oracle_l4_prefix.json"), "w") as f:
        json.dump(out, f, indent=1)
    chain = inputs.RunSpec(1, 96, 2, 7, 500, inputs.linear_schedule(4.0, 41), 5)
    out = dict(workload="open chain N=96, realisation 2, R0=500, beta 0..4 in 41 values, "
                        "theta=5, PA seed 7: all 40 annealing steps",
               rows=trajectory(chain, 40))
    with open(os.path.join(HERE, "oracle_chain96.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

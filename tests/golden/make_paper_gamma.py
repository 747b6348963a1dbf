"""Writes tests/golden/paper_khi_gamma.json: the FP64 oracle's diagnostics
series and linear-stage growth rates of two of the paper's Kelvin-Helmholtz
set-ups (Sec. IV.A state A at D_v = D_rho = 8 cells on 200 x 600 nodes, and
Sec. IV.B state B at D_v = D_rho = 4 cells on 100 x 300 nodes; perturbation
u_y = 0.02 sin(k x) exp(-k |y|), k = 10 pi, dt = tau = 1e-5, 40000 steps to
t = 0.4, sampled every 50).  The growth rate is half the slope of
ln max(rho u_y^2 / 2) over the linear stage chosen by oracle.fit's rule.
Calls only oracle/ and the input generator.

Run from the repository root:  python tests/golden/make_paper_gamma.py
(about 10 minutes of 8 host cores).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import core, fit  # noqa: E402
from paper_1010_4124_gb300 import inputs  # noqa: E402

CASES = (("A", 8.0, 8.0), ("B", 4.0, 4.0))


def main():
    out = {"source": "FP64 CPU oracle (oracle/oklb.c), written by tests/golden/make_paper_gamma.py", "cases": []}
    for state, Dv, Drho in CASES:
        pb = inputs.paper_khi(Dv, Drho, state, steps=40000, sample_every=50)
        p = core.Params(nx=pb.nx, ny=pb.ny, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau, v=pb.v,
                        bc_x=pb.bc_x, bc_y=pb.bc_y)
        t0 = time.time()
        f = core.init_feq(p, *inputs.fields(pb))
        _, d = core.run(p, f, pb.steps, sample_every=pb.sample_every)
        gamma, first, last = fit.linear_stage_rate(d[:, 5], pb.dt * pb.sample_every)
        case = {"state": state, "Dv": Dv, "Drho": Drho, "nx": pb.nx, "ny": pb.ny, "steps": pb.steps,
                "sample_every": pb.sample_every, "gamma": gamma, "window": [first, last],
                "diag": d.tolist(), "seconds": time.time() - t0}
        out["cases"].append(case)
        print(json.dumps({k: v for k, v in case.items() if k != "diag"}), flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "paper_khi_gamma.json"), "w") as fp:
        json.dump(out, fp)


if __name__ == "__main__":
    main()

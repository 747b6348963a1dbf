"""Writes tests/golden/khi512_gamma.json: the FP64 oracle's diagnostics series
and growth rates for the single 512 x 512 Kelvin-Helmholtz run (u_x = 0.25
tanh(y / 4 dy), rho = 3 + 2 tanh(y / 4 dy), p = 1.5, u_y = 0.01 sin(2 pi x / Lx)
exp(-(y / 0.05 Ly)^2), dx = dy = 0.002, dt = tau = 1e-5, periodic x, outflow
y, 4000 steps sampled every 10).  Calls only oracle/ and the input generator.

Run from the repository root:  python tests/golden/make_khi_gamma.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import core, fit  # noqa: E402
from paper_1010_4124_gb300 import inputs  # noqa: E402


def main():
    pb = inputs.khi(512, 512, 4000, Dv=4.0, Drho=4.0, sample_every=10)
    p = core.Params(nx=pb.nx, ny=pb.ny, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau, v=pb.v,
                    bc_x=pb.bc_x, bc_y=pb.bc_y)
    t0 = time.time()
    f = core.init_feq(p, *inputs.fields(pb))
    _, d = core.run(p, f, pb.steps, sample_every=pb.sample_every)
    g_uy, g_ex, g_ke = fit.growth_rates(d, pb.dt, pb.sample_every)
    out = {
        "source": "FP64 CPU oracle (oracle/oklb.c), written by tests/golden/make_khi_gamma.py",
        "workload": "KHI 512x512, D_v = D_rho = 4 cells, 4000 steps, sampled every 10",
        "gamma_ln_max_uy": g_uy,
        "gamma_half_ln_max_Ex": g_ex,
        "gamma_half_ln_sum_Ex": g_ke,
        "diag": d.tolist(),
        "seconds": time.time() - t0,
    }
    with open(os.path.join(ROOT, "tests", "golden", "khi512_gamma.json"), "w") as fp:
        json.dump(out, fp)
    print(json.dumps({k: v for k, v in out.items() if k != "diag"}))


if __name__ == "__main__":
    main()

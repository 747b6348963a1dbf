"""The paper's Kelvin-Helmholtz results (Sec. IV), reproduced with the CUDA
path on its own set-ups (inputs.paper_khi), run as batches.  These pin the
physics weakly, against the paper's statements and fitted laws:

* Sec. IV.A (Fig. 7): the growth rate decreases with the width D_v of the
  velocity transition layer, below the sharp-interface rate gamma_c, along
  ln gamma_v = a - b D_v with the paper's a = 2.70, b = 0.07;
* Sec. IV.B (Figs. 8-9): the growth rate increases with D_rho and no longer
  varies much beyond D_rho = 6;
* Sec. IV.C (Fig. 10): for R = D_rho / D_v < 1 it decreases monotonically
  with D_rho; for R > 1 it rises to a peak and then decreases;
* Sec. IV.A (Fig. 4): the mixing layer of the averaged density profile
  thickens with time.
"""
import numpy as np
import pytest

from paper_1010_4124_gb300 import inputs, klb, sweeps

pytestmark = pytest.mark.gpu


def test_velocity_gradient_law():
    res = sweeps.run_pairs("A", [(2.0, 8.0), (8.0, 8.0), (16.0, 8.0)])
    g = [r["gamma"] for r in res]
    gc = sweeps.classical_rate(inputs.paper_khi(2.0, 8.0, "A"))
    assert gc > g[0] > g[1] > g[2] > 0, (g, gc)
    a, b = sweeps.fit_velocity_law(res)
    assert abs(a - 2.70) < 0.15 and abs(b - 0.07) < 0.015, (a, b)


def test_density_gradient_trend():
    res = sweeps.run_pairs("B", [(4.0, 1.0), (4.0, 3.0), (4.0, 5.0), (4.0, 6.0), (4.0, 10.0)])
    g = [r["gamma"] for r in res]
    assert g[0] < g[1] < g[2], g
    assert abs(g[4] - g[3]) < 0.03 * g[3], g


def test_hybrid_gradient_trends():
    Dr = (4.0, 6.0, 8.0, 10.0)
    res = sweeps.run_pairs("B", [(d / 0.5, d) for d in Dr] + [(d / 5.0, d) for d in Dr])
    lo = [r["gamma"] for r in res[:4]]
    hi = [r["gamma"] for r in res[4:]]
    assert all(x > y for x, y in zip(lo, lo[1:])), lo          # R = 0.5: monotone decrease
    k = int(np.argmax(hi))
    assert 0 < k < len(hi) - 1, hi                              # R = 5: an interior peak


def test_mixing_layer_thickens():
    pb = inputs.paper_khi(4.0, 8.0, "A", steps=40000, sample_every=0)
    widths = []
    with klb.Klb.from_problem(pb, precision="fp32") as h:
        h.init_fields(*inputs.fields(pb))
        lo, hi = pb.rho2 + 0.05 * (pb.rho1 - pb.rho2), pb.rho1 - 0.05 * (pb.rho1 - pb.rho2)
        for _ in range(4):
            h.step(10000)
            md = h.mean_density()
            widths.append(int(((md > lo) & (md < hi)).sum()))
    assert all(b > a for a, b in zip(widths, widths[1:])), widths


def test_fp32_sod_converges_to_the_exact_solution():
    # Sec. III.B: the Sod tube (gamma = 2, R8) on the FP32 production path at
    # 100, 200 and 400 cells, t = 0.1 (dt scaled with dx): the L1 errors of
    # rho, u, p and T against the exact Riemann solution shrink under
    # refinement and stay below 0.02 at 200 cells
    from oracle import riemann
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    errs = {}
    for nx in (100, 200, 400):
        pb = inputs.sod(nx=nx, ny=4, steps=int(round(0.1 / (2e-5 * 200 / nx))))
        with klb.Klb.from_problem(pb, precision="fp32", sample_every=0) as h:
            h.init_fields(*inputs.fields(pb))
            h.step(pb.steps)
            r, u, w, T = (a[0] for a in h.moments())
        x = (np.arange(nx) + 0.5) * pb.dx
        re, ue, pe = riemann.sample(x, pb.steps * pb.dt, 0.5, left, right, gamma=2.0)
        errs[nx] = [float(np.abs(a - b).mean()) for a, b in ((r, re), (u, ue), (r * T, pe), (T, pe / re))]
    print("FP32 Sod L1 (rho, u, p, T):", errs)
    for k in range(4):
        assert errs[200][k] < errs[100][k] and errs[400][k] < errs[200][k], errs
    assert max(errs[200]) < 0.02, errs

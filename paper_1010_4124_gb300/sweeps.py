"""The parameter sweeps of the paper's Kelvin-Helmholtz study (Sec. IV) on the
batched engine, and the linear growth rate fitted to each run.

    res = sweeps.run("velocity")         # D_v sweep of state A (Sec. IV.A)
    res = sweeps.run("density")          # D_rho sweep of state B (Sec. IV.B)
    res = sweeps.run("hybrid")           # R = D_rho / D_v sweep of state B (Sec. IV.C)

Each returns one record per instance: D_v, D_rho, R, the growth rate gamma
and the samples it was fitted to.  The paper fits gamma "to the initial
growth stage" by eye; here the window is fixed by rule (`growth_rate`).
Every step runs in the library's kernels; this module only lays out the
instances and fits the sampled series.
"""
from __future__ import annotations

import numpy as np

from . import inputs, klb

# the instances of each sweep: (state, [(D_v, D_rho), ...])
SWEEPS = {
    # Sec. IV.A: D_v varied, D_rho = 8 (the paper's Figs. 5-7)
    "velocity": ("A", [(Dv, 8.0) for Dv in (2.0, 4.0, 6.0, 8.0, 10.0, 12.0, 14.0, 16.0)]),
    # Sec. IV.B: D_rho varied at a fixed D_v (the paper does not state it; 4 here)
    "density": ("B", [(4.0, Dr) for Dr in (1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 8.0, 10.0)]),
    # Sec. IV.C: R = D_rho / D_v in {0.5, 1, 2, 5} (the paper's Fig. 10)
    "hybrid": ("B", [(Dr / R, Dr) for R in (0.5, 1.0, 2.0, 5.0) for Dr in (4.0, 6.0, 8.0, 10.0, 12.0)]),
}


def growth_rate(E, dt_sample: float, skip: float = 0.05, rise: float = 4.0):
    """Linear growth rate gamma from the series E_s = max rho u_y^2 / 2 of the
    samples s = 0, 1, ... taken every dt_sample time units.  E grows as
    exp(2 gamma t) in the linear stage (Sec. IV.A), so gamma is half the OLS
    slope of ln E over that stage, taken here as the samples from `skip` time
    units after the minimum of ln E (the seeded perturbation first decays
    into the growing mode) up to the first sample at which ln E has risen by
    `rise` above its value at the window start (or the end of the run).
    Returns (gamma, first, last) with the window's sample indices."""
    lnE = np.log(np.asarray(E, dtype=float))
    t = np.arange(len(lnE)) * dt_sample
    i0 = int(np.argmin(lnE))
    a = min(len(lnE) - 2, i0 + int(round(skip / dt_sample)))
    b = a + 1
    while b + 1 < len(lnE) and lnE[b] < lnE[a] + rise:
        b += 1
    tt, yy = t[a:b + 1], lnE[a:b + 1]
    tm = tt.mean()
    slope = float(((tt - tm) * (yy - yy.mean())).sum() / ((tt - tm) ** 2).sum())
    return 0.5 * slope, a, b


def problems(name: str, steps: int = 40000, sample_every: int = 50):
    state, pairs = SWEEPS[name]
    return [inputs.paper_khi(Dv, Dr, state, steps=steps, sample_every=sample_every) for Dv, Dr in pairs]


def run(name: str, steps: int = 40000, sample_every: int = 50, stream=None, dv=None):
    """Run the sweep `name` as one batch (all instances advance together, one
    persistent launch per step) and fit each instance's growth rate.  For the
    density study, `dv` replaces the fixed D_v (cells) that the paper leaves
    unstated; "equal" sets D_v = D_rho for every instance."""
    state, pairs = SWEEPS[name]
    if dv is not None:
        if name != "density":
            raise ValueError("dv applies to the density study only")
        pairs = [(Dr if dv == "equal" else float(dv), Dr) for _, Dr in pairs]
    return run_pairs(state, pairs, steps, sample_every, stream)


def run_pairs(state: str, pairs, steps: int = 40000, sample_every: int = 50, stream=None):
    """The same for an explicit list of (D_v, D_rho) pairs of one state."""
    pbs = [inputs.paper_khi(Dv, Dr, state, steps=steps, sample_every=sample_every) for Dv, Dr in pairs]
    with klb.KlbBatch.from_problems(pbs, stream=stream) as bt:
        for m, pb in zip(bt.members, pbs):
            m.init_fields(*inputs.fields(pb))
        bt.autotune(steps=5)  # picks the tile shape on a snapshot and restores the state
        bt.step(steps)
        bt.sync()
        diags = [m.diagnostics(cap=steps // sample_every + 1) for m in bt.members]
    out = []
    for pb, d in zip(pbs, diags):
        g, a, b = growth_rate(d[:, 5], pb.dt * sample_every)
        out.append({"Dv": pb.Dv, "Drho": pb.Drho, "R": pb.Drho / pb.Dv, "gamma": g,
                    "window": (a * pb.dt * sample_every, b * pb.dt * sample_every), "E_max": d[:, 5]})
    return out


def classical_rate(pb: inputs.Problem) -> float:
    """gamma_c = k sqrt(rho1 rho2) |dv| / (rho1 + rho2) of a sharp interface (Sec. IV.A)."""
    k = 2.0 * np.pi / (pb.nx * pb.dx)
    return k * np.sqrt(pb.rho1 * pb.rho2) * pb.u0 / (pb.rho1 + pb.rho2)


def fit_velocity_law(res):
    """(a, b) of ln gamma_v = a - b D_v (the paper's Eq. for Fig. 7) by least squares."""
    D = np.array([r["Dv"] for r in res])
    y = np.log([r["gamma"] for r in res])
    b, a = np.polyfit(D, y, 1)
    return float(a), float(-b)


def fit_density_law(res, dmax: float = 6.0):
    """(c, e) of gamma_rho = c + e ln D_rho over D_rho < dmax (the paper's Eq. for Fig. 9)."""
    sel = [r for r in res if r["Drho"] < dmax]
    e, c = np.polyfit(np.log([r["Drho"] for r in sel]), [r["gamma"] for r in sel], 1)
    return float(c), float(e)


def main(argv=None):
    """python -m paper_1010_4124_gb300.sweeps {velocity,density,hybrid} [--steps N]
    runs one of the paper's studies as a batch and prints the growth rates and
    the fitted law."""
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("study", choices=sorted(SWEEPS))
    ap.add_argument("--steps", type=int, default=40000)
    ap.add_argument("--sample-every", type=int, default=50)
    ap.add_argument("--dv", default=None,
                    help="density study only: the fixed D_v in cells (default 4), or 'equal' for D_v = D_rho")
    args = ap.parse_args(argv)
    res = run(args.study, steps=args.steps, sample_every=args.sample_every, dv=args.dv)
    for r in res:
        print(f"D_v = {r['Dv']:6.2f}  D_rho = {r['Drho']:6.2f}  R = {r['R']:5.2f}  gamma = {r['gamma']:.4f}")
    if args.study == "velocity":
        a, b = fit_velocity_law(res)
        print(f"ln gamma_v = a - b D_v: a = {a:.4f}, b = {b:.5f}   (paper: a = 2.70, b = 0.07)")
    elif args.study == "density":
        c, e = fit_density_law(res)
        print(f"gamma_rho = c + e ln D_rho (D_rho < 6): c = {c:.4f}, e = {e:.4f}   (paper: c = 5.28, e = 0.62)")


if __name__ == "__main__":
    main()

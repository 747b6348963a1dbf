"""The hand-written adjoint of the step (reverse sweep with checkpoints).

Pinned to the oracle: its complex-step run is an exact tangent of the step
map, so for a random lambda^N and a random perturbation delta of f^0,
<lambda^N, J delta> (oracle tangent) must equal <J^T lambda^N, delta> (GPU
adjoint) to rounding; the gradients of KE and gamma with respect to D_v, D_rho
and the initial u_y field must equal the oracle's complex-step derivatives;
and central finite differences of the GPU forward (h = 1e-4) must agree to
their truncation error.
"""
import numpy as np
import pytest

from gpu_common import oracle_params
from oracle import core, fit
from paper_1010_4124_gb300 import inputs, klb

pytestmark = pytest.mark.gpu


def _small(steps=30, sample_every=5):
    # a small KHI (thin layers: nonlinear WENO weights active), periodic x, outflow y
    return inputs.khi(24, 20, steps, Dv=2.0, Drho=3.0, sample_every=sample_every)


def _oracle_objective(pb, fields, cs=False):
    """(KE, gamma) of the oracle run from the fields (complex fields: complex-step)."""
    p = oracle_params(pb)
    f0 = core.init_feq(p, *fields, cs=cs)
    _, d = core.run(p, f0, pb.steps, sample_every=pb.sample_every, cs=cs)
    K = d[:, 6]
    ke = K[-1] * pb.dx * pb.dy
    M = len(K)
    w = fit.window(M)
    t = np.arange(M) * pb.sample_every * pb.dt
    tw = t[w] - t[w].mean()
    gamma = 0.5 * np.sum(tw * np.log(K[w])) / np.sum(tw**2)
    return ke, gamma


@pytest.mark.parametrize("ckpt,size", [(7, None), (1, None), (100, None), (7, (70, 45)), (4, (45, 70)), (3, (5, 12)),
                                       (5, (64, 32))])
def test_dot_product_with_oracle_tangent(ckpt, size):
    # size None: the small grid (one tile column); (70, 45) and (45, 70):
    # several tiles of the fused reverse step in x and y, ragged at the edges;
    # (5, 12): narrower than the periodic wrap's depth (a node imaged more than
    # once); (64, 32): whole tiles, so the ghost positions at every edge lie
    # past the tiles' own columns and rows
    pb = _small() if size is None else inputs.khi(size[0], size[1], 30, Dv=2.0, Drho=3.0, sample_every=5)
    fields = inputs.fields(pb)
    p = oracle_params(pb)
    f0 = core.init_feq(p, *fields)
    rng = np.random.default_rng(3)
    delta = rng.standard_normal(f0.shape) * 1e-3
    lamN = rng.standard_normal(f0.shape)
    h = 1e-30
    fN_cs, _ = core.run(p, f0 + 1j * h * delta, pb.steps, cs=True)
    Jd = np.imag(fN_cs) / h
    lhs = np.sum(lamN * Jd)
    with klb.KlbAdjoint.from_problem(pb, "fp64", checkpoint_every=ckpt) as adj:
        adj.forward(*fields)
        lam0 = adj.vjp(np.ascontiguousarray(lamN))
    rhs = np.sum(lam0 * delta)
    assert rhs == pytest.approx(lhs, rel=1e-10), (lhs, rhs)


def test_checkpointing_does_not_change_the_result():
    pb = _small()
    fields = inputs.fields(pb)
    lamN = np.random.default_rng(4).standard_normal((19, pb.ny, pb.nx))
    out = []
    for ckpt in (1, 7, 30):
        with klb.KlbAdjoint.from_problem(pb, "fp64", checkpoint_every=ckpt) as adj:
            adj.forward(*fields)
            out.append(adj.vjp(lamN))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_objective_matches_oracle():
    pb = _small()
    fields = inputs.fields(pb)
    ke_ref, g_ref = _oracle_objective(pb, fields)
    with klb.KlbAdjoint.from_problem(pb, "fp64", checkpoint_every=7) as adj:
        ke, gamma = adj.forward(*fields)
    assert ke == pytest.approx(ke_ref, rel=1e-12)
    assert gamma == pytest.approx(g_ref, rel=1e-10)


def test_gradients_match_oracle_complex_step():
    torch = pytest.importorskip("torch")
    from paper_1010_4124_gb300.adjoint import khi_loss
    pb = _small()
    uy0 = inputs.perturbation_shape(pb)
    rng = np.random.default_rng(5)
    dir_uy = rng.standard_normal(uy0.shape)
    with klb.KlbAdjoint.from_problem(pb, "fp64", checkpoint_every=7) as adj:
        Dv = torch.tensor(pb.Dv, dtype=torch.float64, requires_grad=True)
        Dr = torch.tensor(pb.Drho, dtype=torch.float64, requires_grad=True)
        uy = torch.tensor(uy0, dtype=torch.float64, device="cuda", requires_grad=True)
        for which in (0, 1):
            for t in (Dv, Dr, uy):
                t.grad = None
            ke, gamma = khi_loss(pb, Dv.cuda(), Dr.cuda(), uy, adj, device="cuda")
            (ke if which == 0 else gamma).backward()
            got = [Dv.grad.item(), Dr.grad.item(), float((uy.grad.cpu().numpy() * dir_uy).sum())]
            h = 1e-25
            ref = [
                np.imag(_oracle_objective(pb, inputs.fields(pb, Dv=pb.Dv + 1j * h), cs=True)[which]) / h,
                np.imag(_oracle_objective(pb, inputs.fields(pb, Drho=pb.Drho + 1j * h), cs=True)[which]) / h,
                np.imag(_oracle_objective(pb, inputs.fields(pb, uy=uy0 + 1j * h * dir_uy), cs=True)[which]) / h,
            ]
            for g, r in zip(got, ref):
                assert g == pytest.approx(r, rel=1e-8, abs=1e-14 * max(1.0, abs(r))), (which, got, ref)


def test_fp32_adjoint_close_to_fp64():
    pb = _small()
    fields = inputs.fields(pb)
    outs = {}
    for prec in ("fp64", "fp32"):
        with klb.KlbAdjoint.from_problem(pb, prec, checkpoint_every=7) as adj:
            adj.forward(*fields)
            outs[prec] = adj.backward(1.0, 0.0)
    for a, b in zip(outs["fp32"], outs["fp64"]):
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 2e-3 * scale


def _khi256():
    return inputs.khi(256, 256, 2000, Dv=4.0, Drho=4.0, sample_every=10)


def _width_gradients(pb, fields, d_rho, d_ux, d_T):
    """d/dD_v and d/dD_rho of an objective from its gradients with respect to
    the initial fields (the chain rule through the tanh profiles)."""
    X, Y = inputs.coords(pb)
    s = Y / (pb.Dv * pb.dy)
    dux = 0.5 * pb.u0 / np.cosh(s) ** 2 * (-s / pb.Dv)
    sr = Y / (pb.Drho * pb.dy)
    drho = 0.5 * (pb.rho1 - pb.rho2) / np.cosh(sr) ** 2 * (-sr / pb.Drho)
    rho = fields[0]
    return float((d_ux * dux).sum()), float((d_rho * drho + d_T * (-pb.p0 / rho**2) * drho).sum())


def test_config_size_gradient_vs_finite_differences():
    # 256 x 256 KHI as the single run, 2000 steps, checkpoints every 45:
    # dKE/dD_v, dKE/dD_rho, dgamma/dD_v and dgamma/dD_rho by the adjoint
    # against central differences of the GPU forward in FP64 (h = 1e-4)
    pb = _khi256()
    with klb.KlbAdjoint.from_problem(pb, "fp64", checkpoint_every=45) as adj:
        fields = inputs.fields(pb)
        adj.forward(*fields)
        d_rho, d_ux, _, d_T = adj.backward(1.0, 0.0)
        g_ke = _width_gradients(pb, fields, d_rho, d_ux, d_T)
        adj.forward(*fields)  # the reverse sweep reuses the forward grid's buffers
        d_rho, d_ux, _, d_T = adj.backward(0.0, 1.0)
        g_gamma = _width_gradients(pb, fields, d_rho, d_ux, d_T)
        h = 1e-4
        fd_ke, fd_gamma = [], []
        for key in ("Dv", "Drho"):
            vals = [adj.forward(*inputs.fields(pb, **{key: getattr(pb, key) + sgn * h})) for sgn in (1, -1)]
            fd_ke.append((vals[0][0] - vals[1][0]) / (2 * h))
            fd_gamma.append((vals[0][1] - vals[1][1]) / (2 * h))
    assert g_ke[0] == pytest.approx(fd_ke[0], rel=1e-5)
    assert g_ke[1] == pytest.approx(fd_ke[1], rel=1e-5)
    assert g_gamma[0] == pytest.approx(fd_gamma[0], rel=1e-5)
    assert g_gamma[1] == pytest.approx(fd_gamma[1], rel=1e-5)


def test_config_size_uy0_gradient_along_random_directions():
    # the same run: the adjoint's gradient of KE with respect to the initial
    # u_y field, projected on 16 seeded random directions, against central
    # differences of the GPU forward along each direction (FP64, h = 1e-4,
    # Richardson-extrapolated with 2h).  The directions are smooth random fields (a few low Fourier modes of
    # random amplitude and phase, max |d| = 1; 8 of them under the
    # perturbation's Gaussian envelope): a white-noise direction would move
    # the WENO weights off their smooth regime within h and put O(1e-4) of
    # curvature into the central difference itself.
    pb = _khi256()
    rng = np.random.default_rng(256)
    X, Y = inputs.coords(pb)
    xs, ys = X / (pb.nx * pb.dx), Y / (pb.ny * pb.dy)
    env = np.exp(-(Y / (0.05 * pb.ny * pb.dy)) ** 2)
    dirs = []
    for k in range(16):
        d = np.zeros_like(X)
        for _ in range(4):
            kx, ky = rng.integers(0, 4, size=2)
            d += rng.uniform(-1, 1) * np.sin(2 * np.pi * (kx * xs + ky * ys) + rng.uniform(0, 2 * np.pi))
        d = d * (env if k >= 8 else 1.0)
        dirs.append(d / np.abs(d).max())
    fields = inputs.fields(pb)
    uy0 = fields[2]
    h = 1e-4
    with klb.KlbAdjoint.from_problem(pb, "fp64", checkpoint_every=45) as adj:
        adj.forward(*fields)
        _, _, d_uy, _ = adj.backward(1.0, 0.0)
        for k, dvec in enumerate(dirs):
            got = float((d_uy * dvec).sum())
            # central differences with h and 2h; their Richardson combination
            # removes the h^2 term (a direction almost orthogonal to the
            # gradient has a small derivative against which that term is not
            # small: 6e-5 of it for one of these with h alone)
            cd = []
            for step in (h, 2 * h):
                ke = [adj.forward(*inputs.fields(pb, uy=uy0 + sgn * step * dvec))[0] for sgn in (1, -1)]
                cd.append((ke[0] - ke[1]) / (2 * step))
            fd = (4.0 * cd[0] - cd[1]) / 3.0
            assert got == pytest.approx(fd, rel=1e-5), (k, got, fd, cd)


def test_fp32_adjoint_graphs_follow_the_grid_tile_shape():
    # the FP32 forward run and reverse sweep are replayed from CUDA graphs
    # captured on first use; after the grid's tile shape is switched, a run
    # must equal, bit for bit, a fresh adjoint started with the new shape (its
    # states are the same bits either way; gamma's diagnostics sums follow the
    # shape's reduction order), and a repeated run must equal the first
    pb = inputs.khi(70, 45, 40, Dv=2.0, Drho=3.0, sample_every=5)
    fields = [np.ascontiguousarray(a) for a in inputs.fields(pb)]

    def run(adj):
        ke, gamma = adj.forward(*fields)
        return ke, gamma, adj.backward(1.0, 1.0)

    with klb.KlbAdjoint.from_problem(pb, "fp32", checkpoint_every=7) as adj:
        v0 = adj.grid.variant
        run(adj)  # graphs captured with the first shape
        adj.grid.variant = 1 - v0
        switched = [run(adj), run(adj)]
    with klb.KlbAdjoint.from_problem(pb, "fp32", checkpoint_every=7) as fresh:
        fresh.grid.variant = 1 - v0
        ref = run(fresh)
    for got in switched:
        assert got[0] == ref[0] and got[1] == ref[1]
        for a, b in zip(got[2], ref[2]):
            assert np.array_equal(a, b)

"""The batched engine (D_v x D_rho sweeps, Sec. IV): every member of a batch
evolves exactly as the same grid stepped alone; graph replay, the tile shapes
and the autotuner change nothing in the result; each member's diagnostics and
growth rate match the oracle."""
import numpy as np
import pytest

from gpu_common import oracle_params, rel_err_fields
from oracle import core, fit
from paper_1010_4124_gb300 import inputs, klb

pytestmark = pytest.mark.gpu


def _problems(steps=40):
    # uneven sizes (ragged tiles), both boundary layouts, sampling cadences
    return [inputs.khi(96, 80, steps, Dv=2.0, Drho=6.0, sample_every=10),
            inputs.khi(128, 64, steps, Dv=8.0, Drho=2.0, sample_every=10),
            inputs.khi(63, 97, steps, Dv=4.0, Drho=12.0, sample_every=5),
            inputs.khi(200, 40, steps, Dv=16.0, Drho=24.0, sample_every=10)]


def _alone(pb, steps, variant):
    with klb.Klb.from_problem(pb, precision="fp32") as h:
        h.variant = variant
        h.init_fields(*inputs.fields(pb))
        h.step(steps)
        return h.get_f(), h.diagnostics()


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("graph", [True, False])
def test_members_match_grids_stepped_alone(variant, graph):
    pbs = _problems()
    steps = 140  # two 70-step graph replays when graphs are on
    with klb.KlbBatch.from_problems(pbs) as b:
        b.variant = variant
        b.use_graph(graph)
        for m, pb in zip(b.members, pbs):
            m.init_fields(*inputs.fields(pb))
        b.step(steps)
        b.sync()
        got = [(m.get_f(), m.diagnostics()) for m in b.members]
        assert all(m.step_count == steps for m in b.members)
    for (fb, db), pb in zip(got, pbs):
        fa, da = _alone(pb, steps, variant)
        assert np.array_equal(fa, fb)
        assert np.array_equal(da, db)


def test_many_members_with_mixed_sampling_match_grids_stepped_alone():
    # more than 32 members (the due-for-a-sample mask spans two words), three
    # sampling cadences (partial masks) and uneven sizes: every member's state
    # and diagnostics series equal those of the grid stepped alone.  The
    # common period is 12 steps and one graph holds 72: 96 steps replay one
    # graph and take 24 steps one by one.
    rng = np.random.default_rng(11)
    steps = 96
    pbs = [inputs.khi(int(rng.integers(33, 90)), int(rng.integers(20, 70)), steps, Dv=float(rng.integers(2, 9)),
                      Drho=float(rng.integers(2, 13)), sample_every=(3, 4, 6)[i % 3]) for i in range(37)]
    with klb.KlbBatch.from_problems(pbs) as b:
        for m, pb in zip(b.members, pbs):
            m.init_fields(*inputs.fields(pb))
        b.step(steps)
        b.sync()
        got = [(m.get_f(), m.diagnostics()) for m in b.members]
    for (fb, db), pb in zip(got, pbs):
        fa, da = _alone(pb, steps, 0)
        assert np.array_equal(fa, fb)
        assert da.shape == (steps // pb.sample_every + 1, 7)
        assert np.array_equal(da, db)


def test_autotune_leaves_the_run_unchanged():
    pbs = _problems()
    with klb.KlbBatch.from_problems(pbs) as b:
        for m, pb in zip(b.members, pbs):
            m.init_fields(*inputs.fields(pb))
        b.step(20)
        v = b.autotune(steps=4)
        assert v in (0, 1) and b.variant == v
        b.step(20)
        b.sync()
        got = [m.get_f() for m in b.members]
    for fb, pb in zip(got, pbs):
        fa, _ = _alone(pb, 40, 0)
        assert np.array_equal(fa, fb)


def test_batch_member_parity_with_oracle():
    pbs = _problems(60)
    with klb.KlbBatch.from_problems(pbs) as b:
        for m, pb in zip(b.members, pbs):
            m.init_fields(*inputs.fields(pb))
        b.step(60)
        got = [(m.get_f(), m.diagnostics()) for m in b.members]
    for (f, d), pb in zip(got, pbs):
        p = oracle_params(pb)
        ref, dref = core.run(p, core.init_feq(p, *inputs.fields(pb)), 60, sample_every=pb.sample_every)
        errs = rel_err_fields(f, ref, p)
        assert max(errs["rho"], errs["u"], errs["T"]) <= 1e-5, errs
        assert d.shape == dref.shape
        np.testing.assert_allclose(d[:, 0], dref[:, 0], rtol=1e-6)


def test_batch_rejects_mixed_constants_and_fp64():
    a = inputs.khi(64, 64, 10)
    bb = a.with_(dt=2e-5)
    with pytest.raises(klb.KlbError) as e:
        klb.KlbBatch.from_problems([a, bb])
    assert e.value.code == -1
    p = [klb.make_params(64, 64, 0.002, 0.002, 1e-5, 1e-5, precision="fp64")]
    with pytest.raises(klb.KlbError):
        klb.KlbBatch(p)


def test_batch_step_needs_members_in_step():
    pbs = _problems()
    with klb.KlbBatch.from_problems(pbs) as b:
        with pytest.raises(klb.KlbError) as e:
            b.step(1)
        assert e.value.code == -6
        for m, pb in zip(b.members, pbs):
            m.init_fields(*inputs.fields(pb))
        b.step(3)
        b.members[1].init_fields(*inputs.fields(pbs[1]))  # member 1 back at step 0
        with pytest.raises(klb.KlbError) as e:
            b.step(1)
        assert e.value.code == -6

"""The slab engine (klb_slabs_*) on the GPU: the grid cut in y into slabs, the
ghost rows at every cut copied from the neighbour before each step.  A node's
update reads only its stencil, so the slabs must reproduce the whole grid bit
for bit, in FP32 (both tile shapes) and FP64, for periodic, outflow and
fixed-equilibrium y sides, with 1, 2 and 3 slabs of ragged heights."""
import numpy as np
import pytest

from gpu_common import oracle_params, rel_err_global
from oracle import core
from paper_1010_4124_gb300 import inputs, klb

pytestmark = pytest.mark.gpu


def _problem(nx, ny, bcy, steps):
    return inputs.Problem("slabs", nx, ny, 0.002, 0.002, 1e-5, 1e-5, steps, bc_x=("periodic", "periodic"),
                          bc_y=(bcy, bcy))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("bcy", ["periodic", "outflow", "fixed_eq"])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_slabs_equal_the_whole_grid(prec, bcy, n):
    pb = _problem(70, 50, bcy, 25)
    fields = [np.ascontiguousarray(a) for a in inputs.rough_random_fields(pb.nx, pb.ny, seed=50 + n)]
    with klb.Klb.from_problem(pb, prec) as h:
        h.init_fields(*fields)
        h.step(pb.steps)
        ref = h.get_f()
    with klb.KlbSlabs.from_problem(pb, n, prec) as s:
        assert [m.ny for m in s.members] == klb.slab_partition(pb.ny, n)[1]
        s.init_fields(*fields)
        s.step(pb.steps)
        got = s.get_f()
    assert np.array_equal(got, ref)


def test_slabs_match_the_oracle_and_both_tile_shapes():
    # the KHI layer split into 4 slabs (outflow y): against the FP64 oracle,
    # and with the members' tile shape switched, bit for bit the same
    pb = inputs.khi(96, 64, 40, Dv=3.0, Drho=3.0, sample_every=0)
    fields = inputs.fields(pb)
    p = oracle_params(pb)
    ref, _ = core.run(p, core.init_feq(p, *fields), pb.steps)
    out = []
    for v in (0, 1):
        with klb.KlbSlabs.from_problem(pb, 4, "fp32") as s:
            for m in s.members:
                m.variant = v
            s.init_fields(*fields)
            s.step(pb.steps)
            out.append(s.get_f())
    assert np.array_equal(out[0], out[1])
    assert rel_err_global(out[0], ref) <= 1e-5


def test_slabs_refuse_thin_slabs_and_halo_domains():
    pb = _problem(32, 8, "outflow", 1)
    with pytest.raises(klb.KlbError):
        klb.KlbSlabs.from_problem(pb, 3, "fp32")  # slabs of 2-3 rows: shallower than the ghost layer
    with pytest.raises(klb.KlbError):
        klb.KlbSlabs.from_problem(pb.with_(bc_y=("halo", "halo")), 2, "fp32")


def test_slabs_with_device_fields_and_output():
    # fields and the assembled distribution as torch device tensors (each slab
    # takes its rows of the fields by pointer offset; the distribution is
    # gathered on the device)
    torch = pytest.importorskip("torch")
    pb = _problem(48, 40, "outflow", 12)
    fields = [np.ascontiguousarray(a) for a in inputs.smooth_random_fields(pb.nx, pb.ny, seed=7, amp=0.08)]
    dev = [torch.from_numpy(a).cuda() for a in fields]
    with klb.KlbSlabs.from_problem(pb, 2, "fp32") as s:
        s.init_fields(*dev)
        s.step(pb.steps)
        out = torch.empty((19, pb.ny, pb.nx), dtype=torch.float64, device="cuda")
        s.get_f(out)
        host = s.get_f()
    with klb.Klb.from_problem(pb, "fp32") as h:
        h.init_fields(*fields)
        h.step(pb.steps)
        ref = h.get_f()
    assert np.array_equal(out.cpu().numpy(), ref) and np.array_equal(host, ref)

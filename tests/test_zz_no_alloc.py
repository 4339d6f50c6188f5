"""The no-allocation phase-volume entry point (needs a GB300).

oscar_phase_volume_noalloc serves callers that cannot call cudaMalloc (code
running under stream capture, hosts with a fixed device-memory budget). It
must give the same phase volume as the instance path (oscar_stats), on two
calls in a row that share its static scratch, and must refuse grids larger
than that scratch. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2105_10576_gb300 import inputs
from paper_2105_10576_gb300 import oscar as ox

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("make,prec", [(lambda: inputs.channel_bubble_2d(), inputs.PREC_FP64),
                                       (lambda: inputs.random_small_case(7, 30, 20, nz=12, dim=3),
                                        inputs.PREC_MIXED)])
def test_noalloc_phase_volume_matches_instance_path(make, prec):
    torch = pytest.importorskip("torch")
    c = make()
    p = dict(c.params, precision=prec)
    g = ox.Oscar(p, c.solid, c.alpha0)
    dt_cfl, dt_b, dt_vd, N = ox.oscar_timesteps(p, 0.02)
    g.drag_step(dt_vd, strict=False)
    g.relax(dt_vd / N, 3, strict=False)
    expect = g.stats()["phase_volume"]
    n = c.solid.size
    V = p["hx"] * p["hy"] * (p["hz"] if p["dim"] == 3 else 1.0)
    alpha = torch.empty(n, dtype=torch.float64, device="cuda")
    g.field_device(ox.FIELD_ALPHA, alpha.data_ptr(), n)
    solid = torch.from_numpy(np.ascontiguousarray(c.solid).ravel()).to("cuda")
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    ox.oscar_phase_volume_noalloc(alpha.data_ptr(), solid.data_ptr(), n, V, out.data_ptr(), stream)
    ox.oscar_phase_volume_noalloc(alpha.data_ptr(), solid.data_ptr(), n, V, out.data_ptr() + 8, stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == pytest.approx(expect, rel=1e-12)
    assert got[1] == pytest.approx(expect, rel=1e-12)
    g.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ox.OscarError) as e:
        ox.oscar_phase_volume_noalloc(buf.data_ptr(), buf.data_ptr(), 16_777_217, 1.0, buf.data_ptr(), 0)
    assert e.value.code == -1

"""The ingest transpose (time-major [N][C] -> channel-major [C][N], the optional
first step of the path) against the oracle, bit-exact, on ragged shapes, on
strides that force the byte path, and followed by dedispersion."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gsp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_12749_gb300 import build, gsp as g
    build.build()
    g.lib()
    return g


@pytest.mark.parametrize("n,c,in_pad,out_pad", [(1013, 77, 3, 5), (4096, 256, 0, 0), (1000, 200, 8, 24),
                                                (70, 1, 0, 2), (130, 4096, 4, 16)])
def test_transpose_bit_exact(gsp, orc, n, c, in_pad, out_pad):
    rng = np.random.default_rng(n + c)
    x = rng.integers(0, 256, (n, c + in_pad), dtype=np.uint8)
    out = torch.full((c, n + out_pad), 7, dtype=torch.uint8, device="cuda")
    gsp.gsp_ingest_transpose(torch.from_numpy(x).cuda(), n, c, out)
    o = out.cpu().numpy()
    assert (o[:, :n] == orc.ingest_transpose(x[:, :c])).all()
    assert (o[:, n:] == 7).all()


def test_ingest_then_dedisperse(gsp, orc):
    rng = np.random.default_rng(4)
    nchan, n_in = 128, 6000
    dms = np.arange(0.0, 30.0, 0.5)
    x_tc = rng.integers(0, 256, (n_in, nchan), dtype=np.uint8)
    stride = (n_in + 15) // 16 * 16
    xd = torch.zeros((nchan, stride), dtype=torch.uint8, device="cuda")
    gsp.gsp_ingest_transpose(torch.from_numpy(x_tc).cuda(), n_in, nchan, xd)
    desc, keep = gsp.make_desc(nchan, 1200.0, 1500.0, 1e-4, n_in, dms=dms)
    plan = gsp.gsp_plan_create(desc, keep)
    n_out = gsp.gsp_plan_nout(plan, n_in)
    D = torch.zeros((len(dms), (n_out + 3) // 4 * 4), dtype=torch.int32, device="cuda")
    gsp.gsp_dedisperse(plan, xd, n_in, D)
    dl, _ = orc.delays(nchan, 1200.0, 1500.0, 1e-4, dms)
    ref = orc.dedisperse(orc.ingest_transpose(x_tc), n_in, dl)
    assert (D.cpu().numpy()[:, :n_out].astype(np.int64) == ref).all()

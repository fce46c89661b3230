"""The convolver's bounded waits on a GPU, made to run out without a fault:
fdas_debug_wait_timeout arms every CTA's first template-row barrier without
issuing its copy, so each first wait gives up after a few polls with nothing
in flight.  The call must return with FDAS_STATUS_TIMEOUT in the status word,
and the device must still run a normal search correctly afterwards."""
import numpy as np
import pytest

import oracle.fdas_oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_05335_gb300 as F
    F.load_library()
    return F


def test_bounded_wait_runs_out_and_reports(F):
    from paper_1804_05335_gb300.search import Search
    n = 1 << 16
    S = Search(n, 1024, 256, -200, 200, 2, thr=20.0)
    x = synth.make_series(n, ((n / 5 + 0.25, 60.0, 20.0),), 501)
    S.series.copy_(torch.from_numpy(x))
    S.make_templates()
    S.normalise()
    S.status.zero_()
    F.fdas_debug_wait_timeout(S.p, S.spec, S.nb, S.bank, S.plane, S.row_stride, 1000, S.status)
    torch.cuda.synchronize()
    assert S.status.item() & F.FDAS_STATUS_TIMEOUT
    # the context is intact: a normal search afterwards matches the oracle
    S.status.zero_()
    S.plane.fill_(-1.0)
    S.correlate(fused=True)
    torch.cuda.synchronize()
    assert S.status.item() == 0
    A = S.spec.cpu().numpy().astype(np.complex128)
    zs = O.z_grid(-200, 200, 2)
    got = S.plane2d()[:, 2 * 5000: 2 * 5256].cpu().numpy().astype(np.float64)
    ref = O.plane_window(A, zs, 5000, 256)
    assert np.abs(got - ref).max() < 1e-3


def test_wait_probe_rejects_other_forms(F):
    from paper_1804_05335_gb300.search import Search
    S = Search(1 << 14, 2048, 64, -20, 20, 2)
    S.make_templates()
    with pytest.raises(F.FdasError) as e:
        F.fdas_debug_wait_timeout(S.p, S.spec, S.nb, S.bank, S.plane, S.row_stride, 100, S.status)
    assert e.value.code == F.FDAS_E_UNSUPPORTED
    S1 = Search(1 << 14, 1024, 64, -20, 20, 2)
    with pytest.raises(F.FdasError) as e:
        F.fdas_debug_wait_timeout(S1.p, S1.spec, S1.nb, S1.bank, S1.plane, S1.row_stride, 0,
                                  S1.status)
    assert e.value.code == F.FDAS_E_INVAL

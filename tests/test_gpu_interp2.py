"""2-bin Fourier interpolation (interbin = 2): the correlation evaluated at
half-bin resolution through the same convolver (spectrum with zeros
interleaved, templates sampled every half bin), against the oracle's plain
tap sum at half-integer frequencies; 1e-3 absolute on normalised power."""
import numpy as np
import pytest

import oracle.fdas_oracle as O
import synth
from tests.gpu_common import compare_candidates

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PTOL = 1e-3


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_05335_gb300 as F
    F.load_library()
    return F


def _search(**kw):
    from paper_1804_05335_gb300.search import Search
    return Search(**kw)


@pytest.mark.parametrize("n,L,M,zmin,zmax,zstep", [
    (1 << 14, 2048, 128, -20, 20, 2),
    (1 << 14, 1024, 128, -20, 20, 2),
    (1 << 14, 4096, 256, -30, 30, 3),
    (1 << 14, 2048, 128, -10, 30, 5),
    (1 << 13, 4096, 512, -40, 40, 20),     # one segment longer than the doubled spectrum
])
def test_interp2_plane_matches_oracle(F, n, L, M, zmin, zmax, zstep):
    x = synth.make_series(n, ((n / 7 + 0.5, 6.0, 18.0), (n / 3 + 0.25, -14.0, 20.0)), 19)
    A = O.normalise(O.real_spectrum(x), 1024).astype(np.complex64)
    S = _search(n=n, L=L, M=M, zmin=zmin, zmax=zmax, zstep=zstep, interbin=2)
    S.spec.copy_(torch.from_numpy(A))
    S.make_templates()
    S.plane.fill_(-1.0)
    S.correlate(fused=False)
    got = S.plane2d().cpu().numpy().astype(np.float64)
    ref = O.plane_interp2(A.astype(np.complex128), O.z_grid(zmin, zmax, zstep))
    assert got.shape == ref.shape
    err = np.abs(got - ref)
    assert err.max() < PTOL, (err.max(), np.unravel_index(np.argmax(err), err.shape))


@pytest.mark.parametrize("nb", [1, 7, 1001, 1612])
def test_interp2_odd_and_tiny_spectra(F, nb):
    A = synth.random_spectrum(nb, 70 + nb)
    S = _search(n=1 << 12, L=2048, M=256, zmin=-24, zmax=24, zstep=4, interbin=2)
    S.spec[:nb].copy_(torch.from_numpy(A))
    S.make_templates()
    S.plane.fill_(-7.0)
    S.correlate(fused=False, nb=nb)
    P = S.plane.view(S.K, S.row_stride).cpu().numpy()
    ref = O.plane_interp2(A.astype(np.complex128), O.z_grid(-24, 24, 4))
    assert np.abs(P[:, : 2 * nb] - ref).max() < PTOL
    assert np.all(P[:, 2 * nb:] == -7.0)


def test_interp2_fused_candidates_match_oracle(F):
    n = 1 << 14
    x = synth.make_series(n, ((2500.5, 8.0, 20.0), (5100.25, -12.0, 18.0)), 23)
    A = O.normalise(O.real_spectrum(x), 1024).astype(np.complex64)
    S = _search(n=n, L=2048, M=128, zmin=-20, zmax=20, zstep=2, interbin=2, thr=10.0,
                cap=1 << 14)
    S.spec.copy_(torch.from_numpy(A))
    S.make_templates()
    S.status.zero_()
    S.correlate(fused=True)
    r, c, p, fl, total = S.candidates()
    assert total == len(r) and total > 20 and S.status.item() == 0
    ref = O.plane_interp2(A.astype(np.complex128), O.z_grid(-20, 20, 2))
    rr, cc, pp, _ = O.threshold(ref, 10.0, flags=False)
    compare_candidates((r, c, p), (rr, cc, pp), 10.0)

"""fdas_noise_means against the oracle's FP64 means, and the significance
model against noise planes made by the GPU search: per-row means of even and
odd columns, exponential tails, and the gamma tail of harmonic sums."""
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


@pytest.mark.parametrize("L,M,zmin,zmax,zstep,ib", [
    (2048, 256, -200, 200, 2, 1), (2048, 256, -200, 200, 2, 0), (2048, 436, -200, 200, 2, 2),
    (1024, 128, -10, 30, 5, 1), (2048, 64, -21, 21, 2, 1),
])
def test_noise_means_match_oracle(F, L, M, zmin, zmax, zstep, ib):
    from paper_1804_05335_gb300.significance import noise_means
    p = F.params(L, M, zmin, zmax, zstep, ib)
    got = noise_means(p)
    ref = O.noise_means(O.z_grid(zmin, zmax, zstep), ib)
    assert np.abs(got / ref - 1.0).max() < 1e-6


def test_gpu_noise_plane_follows_the_model(F):
    from paper_1804_05335_gb300.search import Search
    from paper_1804_05335_gb300.significance import harmonic_significance, noise_means
    n = 1 << 19
    S = Search(n, 2048, 256, -60, 60, 30)
    S.series.copy_(torch.from_numpy(synth.make_series(n, (), 80)))
    S.step()
    P = S.plane2d().cpu().numpy().astype(np.float64)
    mu = noise_means(S.p)
    for k in range(S.K):
        for e in (0, 1):
            v = P[k, e::2]
            assert abs(v.mean() / mu[k, e] - 1.0) < 0.02
            assert abs(np.mean(v / mu[k, e] > 4.0) - np.exp(-4.0)) < 0.003
    # two-harmonic sums of the z = 0 row (row 2) on even columns: full-bin means
    j, c = 2, np.arange(0, (P.shape[1] - 1) // 2 + 1, 2)
    s2 = P[j, c] + P[j, 2 * c]
    t = 9.0
    logp, _ = harmonic_significance(t, [mu[j, 0], mu[j, 0]])
    assert abs(np.mean(s2 > t) / np.exp(logp) - 1.0) < 0.1

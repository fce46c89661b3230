"""Batched persistent launch (a10): every trial's plane and candidates equal
what the single-series call gives (same kernel arithmetic, bit-exact), a
captured CUDA graph replays the whole batch, the autotuner picks a valid
configuration, and one trial is checked against the FP64 oracle."""
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


def _batch(F, ns, L=1024, M=64, pool=1 << 30, cps=0, thr=8.0):
    from paper_1804_05335_gb300.batch import BatchSearch
    return BatchSearch(ns, L, M, -20, 20, 2, thr=thr, pool_bytes=pool, ctas_per_sm=cps)


def test_batched_equals_single_series(F):
    from paper_1804_05335_gb300.search import Search
    ns = [1 << 14, 1 << 13, 1 << 16, 1 << 13, 1 << 15]
    bs = _batch(F, ns, pool=6 << 20)          # small pool: several waves
    assert len(bs.waves) > 1
    xs = [synth.make_series(n, ((n / 5 + 0.3, 6.0, 20.0),), 100 + i) for i, n in enumerate(ns)]
    for i, x in enumerate(xs):
        bs.set_series(i, x)
    bs.front(stream=None)
    planes = {}
    for k, w in enumerate(bs.waves):
        bs.correlate_wave(k)
        torch.cuda.synchronize()
        for i in w:
            planes[i] = bs.plane_of(i).cpu().numpy().copy()
    cands, counts = bs.candidates()
    for i, n in enumerate(ns):
        S = Search(n, 1024, 64, -20, 20, 2, thr=8.0)
        S.series.copy_(torch.from_numpy(xs[i]))
        S.step()
        torch.cuda.synchronize()
        assert np.array_equal(S.spec.cpu().numpy(), bs.spec_of(i).cpu().numpy())
        assert np.array_equal(S.plane2d().cpu().numpy(), planes[i])
        r, c, p, fl, total = S.candidates()
        br, bc, bp = cands[i]
        assert np.array_equal(r, br) and np.array_equal(c, bc) and np.array_equal(p, bp)


def test_batched_trial_against_oracle(F):
    ns = [1 << 13, 1 << 14]
    bs = _batch(F, ns)
    xs = [synth.make_series(n, ((n / 3, -8.0, 18.0),), 200 + i) for i, n in enumerate(ns)]
    for i, x in enumerate(xs):
        bs.set_series(i, x)
    bs.run()
    torch.cuda.synchronize()
    A = O.normalise(O.real_spectrum(xs[1]), 1024)
    ref = O.plane(A, O.z_grid(-20, 20, 2))
    assert np.abs(bs.plane_of(1).cpu().numpy() - ref).max() < 1e-3


def test_batched_graph_replay(F):
    ns = [1 << 14, 1 << 13, 1 << 15]
    bs = _batch(F, ns, pool=1 << 30)
    for i, n in enumerate(ns):
        bs.set_series(i, synth.make_series(n, ((n / 7, 4.0, 25.0),), 300 + i))
    bs.capture()
    torch.cuda.synchronize()
    ref_planes = [bs.plane_of(i).cpu().numpy().copy() for i in range(len(ns))]
    ref_c, ref_n = bs.candidates()
    bs.pool.fill_(-1.0)
    bs.count.fill_(-5)
    bs.replay()
    torch.cuda.synchronize()
    for i in range(len(ns)):
        assert np.array_equal(bs.plane_of(i).cpu().numpy(), ref_planes[i])
    c, n = bs.candidates()
    assert np.array_equal(n, ref_n)
    for i in range(len(ns)):
        for a, b in zip(c[i], ref_c[i]):
            assert np.array_equal(a, b)


def test_autotune_picks_a_candidate(F, tmp_path):
    from paper_1804_05335_gb300.autotune import autotune
    path = str(tmp_path / "tune.json")
    cands = ((1024, 0, 0), (1024, 0, 5), (2048, 0, 0), (2048, 1, 0))
    res = autotune([1 << 15, 1 << 14], 64, -20, 20, 2, candidates=cands, cache_path=path)
    assert (res["L"], res["ctas_per_sm"], res["templates_per_block"]) in cands
    assert len(res["ms"]) == 4 and all(v > 0 for v in res["ms"].values())
    again = autotune([1 << 15, 1 << 14], 64, -20, 20, 2, candidates=cands, cache_path=path)
    assert again == res


@pytest.mark.parametrize("tpb", [1, 7, 26, 500])
def test_templates_per_block_keeps_every_plane(F, tpb):
    """Chunking a group's templates (templates per block) only reorders the
    work: planes and candidates equal the default order's, bit for bit, on the
    production bank with uneven lengths that are not powers of two."""
    from paper_1804_05335_gb300.batch import BatchSearch
    ns = [20002, 65536, 9000, 131074]
    ref = None
    for t in (0, tpb):
        bs = BatchSearch(ns, 1024, 256, -200, 200, 2, thr=20.0, ctas_per_sm=1,
                         templates_per_block=t)
        for i, n in enumerate(ns):
            bs.set_series(i, synth.make_series(n, ((n / 4 + 0.2, 90.0, 18.0),), 600 + i))
        bs.run()
        torch.cuda.synchronize()
        planes = [bs.plane_of(i).cpu().numpy().copy() for i in range(len(ns))]
        cands, counts = bs.candidates()
        if ref is None:
            ref = (planes, cands)
            continue
        for i in range(len(ns)):
            assert np.array_equal(planes[i], ref[0][i]), (tpb, i)
            for a, b in zip(cands[i], ref[1][i]):
                assert np.array_equal(a, b)


@pytest.mark.parametrize("L", [1024, 2048])
def test_batched_production_bank(F, L):
    """The production template bank (z = -200..200 step 2, M = 256: four
    template groups of increasing overlap) in the batched launch, on trials of
    uneven length (most of them not powers of two), with one CTA per SM so
    that each CTA's range crosses trial and group boundaries, and a pool small
    enough for several waves: every trial's spectrum, plane and candidate list
    are bit-identical to the single-series call, and a trial that is not the
    first of its wave matches the FP64 oracle."""
    from paper_1804_05335_gb300.batch import BatchSearch
    from paper_1804_05335_gb300.search import Search
    ns = [8194, 40000, 1 << 14, 70002, 12288, 1 << 15]
    bs = BatchSearch(ns, L, 256, -200, 200, 2, thr=20.0, pool_bytes=64 << 20, ctas_per_sm=1)
    assert len(bs.waves) > 1
    assert len(F.fdas_template_groups(bs.p)) == 4
    xs = [synth.make_series(n, ((n / 5 + 0.3, 150.0, 20.0), (n / 3 + 0.7, -120.0, 15.0)), 400 + i)
          for i, n in enumerate(ns)]
    for i, x in enumerate(xs):
        bs.set_series(i, x)
    bs.front(stream=None)
    planes = {}
    for k, w in enumerate(bs.waves):
        bs.correlate_wave(k)
        torch.cuda.synchronize()
        for i in w:
            planes[i] = bs.plane_of(i).cpu().numpy().copy()
    cands, counts = bs.candidates()
    assert bs.status.item() == 0
    for i, n in enumerate(ns):
        S = Search(n, L, 256, -200, 200, 2, thr=20.0)
        S.series.copy_(torch.from_numpy(xs[i]))
        S.step()
        torch.cuda.synchronize()
        assert np.array_equal(S.spec.cpu().numpy(), bs.spec_of(i).cpu().numpy())
        assert np.array_equal(S.plane2d().cpu().numpy(), planes[i]), i
        r, c, p, fl, total = S.candidates()
        br, bc, bp = cands[i]
        assert total > 0
        assert np.array_equal(r, br) and np.array_equal(c, bc) and np.array_equal(p, bp)
    # a later trial of a wave, on the oracle's own spectrum, against the oracle
    k = next(k for k, w in enumerate(bs.waves) if len(w) > 1)
    i = bs.waves[k][-1]
    A = O.normalise(O.real_spectrum(xs[i]), 1024)
    bs.spec_of(i).copy_(torch.from_numpy(A.astype(np.complex64)))
    bs.correlate_wave(k)
    torch.cuda.synchronize()
    ref = O.plane(A.astype(np.complex64).astype(np.complex128), O.z_grid(-200, 200, 2))
    err = np.abs(bs.plane_of(i).cpu().numpy().astype(np.float64) - ref)
    assert err.max() < 1e-3, (i, err.max())

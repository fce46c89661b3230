"""fdas_correlate_plane16 (16-bit plane output): the plane equals the FP32
plane of fdas_correlate rounded to nearest (bit-exact), the fused candidates
equal fdas_correlate's, and against the FP64 oracle the error is the FP32
bar plus the storage rounding: |dP| <= 1e-3 + u P with u = 2^-11 (binary16)
or 2^-8 (bfloat16)."""
import numpy as np
import pytest

import oracle.fdas_oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TYPES = {1: (torch.float16, 2.0 ** -11), 2: (torch.bfloat16, 2.0 ** -8)}


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


def _plane16(F, S, ptype, fused=False, nb=None):
    dt, _ = TYPES[ptype]
    buf = torch.full((S.K * S.row_stride,), -3.0, dtype=dt, device="cuda")
    F.fdas_correlate_plane16(S.p, ptype, S.spec, S.nb if nb is None else nb, S.bank, buf,
                             S.row_stride, S.fused if fused else None, S.status)
    return buf.view(S.K, S.row_stride)


@pytest.mark.parametrize("ptype", [1, 2], ids=["f16", "bf16"])
@pytest.mark.parametrize("n,L,M,zmin,zmax,zstep,ib", [
    (1 << 14, 1024, 64, -20, 20, 2, 1), (1 << 14, 2048, 64, -21, 21, 2, 1),
    (1 << 14, 4096, 128, -20, 20, 2, 1), (1 << 14, 2048, 128, -10, 30, 5, 0),
])
def test_plane16_is_the_rounded_fp32_plane_and_matches_oracle(F, ptype, n, L, M, zmin, zmax,
                                                              zstep, ib):
    x = synth.make_series(n, ((n / 7 + 0.25, 6.0, 18.0), (n / 3, -14.0, 20.0)), 9)
    A = O.normalise(O.real_spectrum(x), 1024).astype(np.complex64)
    S = _search(n=n, L=L, M=M, zmin=zmin, zmax=zmax, zstep=zstep, interbin=ib)
    S.spec.copy_(torch.from_numpy(A))
    S.make_templates()
    S.correlate(fused=False)
    p32 = S.plane.view(S.K, S.row_stride)[:, : S.width]
    p16 = _plane16(F, S, ptype)
    dt, u = TYPES[ptype]
    assert torch.equal(p16[:, : S.width], p32.to(dt))
    assert bool((p16[:, S.width:] == -3.0).all())     # nothing past the row width
    ref = O.plane(A.astype(np.complex128), O.z_grid(zmin, zmax, zstep), bool(ib))
    got = p16[:, : S.width].float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-3 + u * np.abs(ref))


@pytest.mark.parametrize("ptype", [1, 2], ids=["f16", "bf16"])
def test_plane16_fused_candidates_equal_fp32(F, ptype):
    n = 1 << 16
    x = synth.make_series(n, ((n / 5 + 0.3, 8.0, 20.0), (n / 3, -30.0, 18.0)), 21)
    S = _search(n=n, L=2048, M=256, zmin=-60, zmax=60, zstep=2, thr=10.0, cap=1 << 14)
    S.series.copy_(torch.from_numpy(x))
    S.step()
    r0, c0, p0, _, t0 = S.candidates()
    _plane16(F, S, ptype, fused=True)
    r1, c1, p1, _, t1 = S.candidates()
    assert t0 == t1 and t0 > 10
    assert np.array_equal(r0, r1) and np.array_equal(c0, c1) and np.array_equal(p0, p1)


def test_plane16_production_equals_rounded_fp32(F):
    wl = synth.workload("production")
    S = _search(n=wl.n, L=wl.L, M=wl.M, zmin=wl.zmin, zmax=wl.zmax, zstep=wl.zstep,
                thr=wl.threshold)
    S.series.copy_(torch.from_numpy(wl.series()))
    S.make_templates()
    S.normalise()
    S.correlate(fused=False)
    p32 = S.plane.view(S.K, S.row_stride)[:, : S.width]
    p16 = _plane16(F, S, 1)
    for k0 in range(0, S.K, 32):      # row blocks, to bound the temporaries
        assert torch.equal(p16[k0:k0 + 32, : S.width], p32[k0:k0 + 32].to(torch.float16))

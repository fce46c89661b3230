"""GPU parity of fdas_correlate_split, the convolver whose radix-16 DFT passes
run as split-precision tensor-core products, against the FP64 oracle and
against the FP32 form on the same spectrum.

Tolerances on normalised power (noise mean 1), |P_gpu - P_ref| <= a + b P_ref:
  FP32 through this entry: bit-identical to fdas_correlate.
  FP16 hi+lo (22-bit operand pairs, per-instance power-of-two scaling):
      a = 1e-3, b = 0 (the FP32 bar).
  BF16 hi+lo (16-bit operand pairs): each operand carries a relative error
      of at most u = 2^-16 and the lo*lo term drops another u, so one DFT
      stage loses at most ~3u in amplitude; four stages give 12u and the
      power twice that, b = 24 * 2^-16 ~ 3.7e-4, plus the FP32 bar a = 1e-3.
Inputs are seeded synthetic series; no expected value comes from the GPU.
"""
import numpy as np
import pytest

import oracle.fdas_oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {1: (1e-3, 0.0), 2: (1e-3, 24 * 2.0 ** -16)}
NAMES = {1: "fp16", 2: "bf16"}


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


def _within(got, ref, prec):
    a, b = TOL[prec]
    excess = np.abs(got - ref) - (a + b * np.abs(ref))
    return float(excess.max()) <= 0.0, float(np.abs(got - ref).max())


CASES = [
    # n, L, M, zmin, zmax, zstep, interbin
    (1 << 14, 2048, 64, -20, 20, 2, 1),      # ragged tail
    (1 << 14, 4096, 128, -20, 20, 2, 1),
    (1 << 14, 2048, 64, -21, 21, 2, 1),      # symmetric grid without z = 0
    (1 << 14, 2048, 128, -10, 30, 5, 1),     # asymmetric grid: no conjugation
    (1 << 14, 2048, 64, -20, 20, 2, 0),      # no interbinning
    (1 << 13, 4096, 256, -6, 6, 2, 1),       # one segment longer than the spectrum
]


@pytest.mark.parametrize("prec", [1, 2], ids=["fp16", "bf16"])
@pytest.mark.parametrize("n,L,M,zmin,zmax,zstep,ib", CASES)
def test_split_plane_matches_oracle(F, prec, n, L, M, zmin, zmax, zstep, ib):
    x = synth.make_series(n, ((n / 7 + 0.25, 6.0, 18.0), (n / 3, -14.0, 20.0)), 9)
    A = O.normalise(O.real_spectrum(x), 1024).astype(np.complex64)
    S = _search(n=n, L=L, M=M, zmin=zmin, zmax=zmax, zstep=zstep, interbin=ib)
    S.spec.copy_(torch.from_numpy(A))
    S.make_templates()
    S.plane.fill_(-1.0)
    S.correlate(fused=False, prec=prec)
    got = S.plane2d().cpu().numpy().astype(np.float64)
    ref = O.plane(A.astype(np.complex128), O.z_grid(zmin, zmax, zstep), bool(ib))
    ok, emax = _within(got, ref, prec)
    assert ok, (NAMES[prec], emax)


def test_split_rejects_warp_segment_length(F):
    """L = 1024 runs the one-warp-per-segment convolver, which has no split form."""
    S = _search(n=1 << 14, L=1024, M=64, zmin=-20, zmax=20, zstep=2)
    S.make_templates()
    for prec in (1, 2):
        with pytest.raises(F.FdasError) as e:
            S.correlate(fused=False, prec=prec)
        assert e.value.code == F.FDAS_E_UNSUPPORTED


def test_split_fp32_entry_is_fdas_correlate(F):
    n = 1 << 14
    x = synth.make_series(n, ((2000.5, 8.0, 15.0),), 11)
    A = O.normalise(O.real_spectrum(x), 1024).astype(np.complex64)
    S = _search(n=n, L=2048, M=64, zmin=-20, zmax=20, zstep=2)
    S.spec.copy_(torch.from_numpy(A))
    S.make_templates()
    S.correlate(fused=False)
    a = S.plane.clone()
    S.plane.fill_(0.0)
    S.correlate(fused=False, prec=F.FDAS_PREC_FP32)
    assert torch.equal(a, S.plane)


@pytest.mark.parametrize("prec", [1, 2], ids=["fp16", "bf16"])
def test_split_tiny_and_odd_spectra(F, prec):
    for nb in (1, 5, 999, 1793):
        A = synth.random_spectrum(nb, 40 + nb)
        S = _search(n=1 << 12, L=2048, M=256, zmin=-40, zmax=40, zstep=4)
        S.spec[:nb].copy_(torch.from_numpy(A))
        S.make_templates()
        S.plane.fill_(-7.0)
        S.correlate(fused=False, nb=nb, prec=prec)
        P = S.plane.view(S.K, S.row_stride).cpu().numpy()
        ref = O.plane(A.astype(np.complex128), O.z_grid(-40, 40, 4))
        ok, emax = _within(P[:, : 2 * nb].astype(np.float64), ref, prec)
        assert ok, (nb, emax)
        assert np.all(P[:, 2 * nb:] == -7.0)


def test_fp16_split_keeps_range_on_strong_lines(F):
    """Lines of amplitude 1e5 and 7e4 (above FP16's largest finite value 65504)
    stay finite and accurate: the per-instance scaling keeps every operand
    inside FP16's exponent range."""
    nb = 6000
    A = synth.random_spectrum(nb, 77).astype(np.complex128)
    A[1500] += 1.0e5
    A[4200] -= 7.0e4j
    A = A.astype(np.complex64)
    S = _search(n=2 * nb, L=2048, M=64, zmin=-20, zmax=20, zstep=2)
    S.spec[:nb].copy_(torch.from_numpy(A))
    S.make_templates()
    S.correlate(fused=False, nb=nb, prec=1)
    P = S.plane2d().cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(P))
    ref = O.plane(A.astype(np.complex128), O.z_grid(-20, 20, 2))
    # Errors scale with the strongest value a DFT instance holds: four split
    # passes of 2^-22 each plus the FP32 passes' rounding (~log2(L) * 2^-24),
    # doubled for power, stay below 1e-5 of the line's power.
    err = np.abs(P - ref)
    assert err.max() < 1e-5 * ref.max(), (err.max(), ref.max())


@pytest.mark.parametrize("prec", [1, 2], ids=["fp16", "bf16"])
def test_split_production_sampled_and_candidates(F, prec):
    """2^23-sample series, zmax = 200, L = 2048: sampled windows against the
    oracle, and the fused candidate list against the FP32 form's."""
    wl = synth.workload("production")
    x = wl.series()
    A = O.normalise(O.real_spectrum(x), wl.median_block).astype(np.complex64)
    A64 = A.astype(np.complex128)
    S = _search(n=wl.n, L=2048, M=wl.M, zmin=wl.zmin, zmax=wl.zmax, zstep=wl.zstep,
                thr=wl.threshold, cap=1 << 16)
    S.spec.copy_(torch.from_numpy(A))
    S.make_templates()
    S.status.zero_()
    S.correlate(fused=True)
    r0_, c0_, p0_, _, tot0 = S.candidates()
    S.correlate(fused=True, prec=prec)
    r1_, c1_, p1_, _, tot1 = S.candidates()
    assert S.status.item() == 0
    plane = S.plane2d()
    zs = O.z_grid(wl.zmin, wl.zmax, wl.zstep)
    rng = np.random.default_rng(2048)
    starts = list(rng.integers(0, wl.nb - 256, 6)) + [0, wl.nb - 256]
    starts += [int(r0) - 128 for r0, _, _ in wl.injections]
    for r0 in starts:
        got = plane[:, 2 * r0: 2 * (r0 + 256)].cpu().numpy().astype(np.float64)
        ref = O.plane_window(A64, zs, r0, 256)
        ok, emax = _within(got, ref, prec)
        assert ok, (r0, emax)
    # candidates: the same list as the FP32 form except within tolerance of
    # the threshold, and powers within tolerance of each other
    a, b = TOL[prec]
    g = {(int(r), int(c)): float(p) for r, c, p in zip(r1_, c1_, p1_)}
    f = {(int(r), int(c)): float(p) for r, c, p in zip(r0_, c0_, p0_)}
    for key in set(g) ^ set(f):
        v = g.get(key, f.get(key))
        assert abs(v - wl.threshold) <= a + b * wl.threshold, key
    for key in set(g) & set(f):
        assert abs(g[key] - f[key]) <= a + b * f[key], key

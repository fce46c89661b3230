"""GPU parity: every call through the C ABI against the FP64 oracle.

Tolerances: normalised power within 1e-3 absolute (noise power mean 1);
candidate lists identical except for points within 1e-3 of the threshold;
bit-exact candidate lists where both sides threshold the same FP32 plane.
Inputs are seeded synthetic series and spectra; no expected value comes
from the GPU path.
"""
import math

import numpy as np
import pytest

import oracle.fdas_oracle as O
import synth
from tests.gpu_common import bank_natural, compare_candidates, mirror_expected

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


def _search(F, **kw):
    from paper_1804_05335_gb300.search import Search
    return Search(**kw)


def _upload_spec(S, A):
    S.spec.copy_(torch.from_numpy(np.ascontiguousarray(A.astype(np.complex64))))


# ------------------------------------------------------------------ bank (a1)
@pytest.mark.parametrize("L,M,zmin,zmax,zstep", [
    (1024, 64, -20, 20, 2), (2048, 256, -200, 200, 2), (4096, 256, -200, 200, 2),
    (2048, 64, -21, 21, 2), (2048, 128, -10, 30, 5), (1024, 64, 0, 0, 1),
])
def test_template_bank_matches_oracle(F, L, M, zmin, zmax, zstep):
    p = F.params(L, M, zmin, zmax, zstep, 1)
    Kb = F.fdas_bank_rows(p)
    bank = torch.empty(F.fdas_bank_floats(p), dtype=torch.float32, device="cuda")
    F.fdas_make_templates(p, bank)
    torch.cuda.synchronize()
    H, mirror = bank_natural(bank.cpu().numpy(), Kb, L)
    assert np.array_equal(mirror, mirror_expected(H, L))
    zs = O.z_grid(zmin, zmax, zstep)
    zb = zs[zs >= 0] if zmin == -zmax and zmax > 0 else zs
    assert len(zb) == Kb
    for b, z in enumerate(zb):
        ref = O.kernel_spectrum(z, L)
        rms = math.sqrt(np.mean(np.abs(ref) ** 2))
        assert np.abs(H[b] - ref).max() / rms < 2e-6, (z, np.abs(H[b] - ref).max() / rms)


# ------------------------------------------------------------------ front end (a2-a3)
@pytest.mark.parametrize("n,block,seed", [
    (1 << 13, 64, 3), (1 << 14, 1024, 4), (1 << 17, 1024, 1), (1 << 20, 1000, 5), (1 << 23, 1024, 2),
    (1 << 25, 1024, 14),   # the largest length (three passes of 256-point lines)
    # even lengths that are not powers of two (Bluestein's convolution)
    (8194, 1024, 6), (3 << 12, 256, 7), (100000, 1024, 8), (1048578, 1024, 9), (5000002, 1024, 10),
    ((1 << 23) - 2, 1024, 11), ((1 << 24) - 2, 1024, 12),
])
def test_normalise_matches_oracle(F, n, block, seed):
    inj = ((n / 8 + 0.3, 10.0, 15.0), (n / 5, -40.0, 20.0))
    x = synth.make_series(n, inj, seed)
    S = _search(F, n=n, L=2048, M=256, zmin=0, zmax=0, zstep=1, median_block=block, plane=False)
    S.series.copy_(torch.from_numpy(x))
    S.normalise()
    got = S.spec.cpu().numpy().astype(np.complex128)
    ref = O.normalise(O.real_spectrum(x), block)
    err = np.abs(got - ref)
    assert err.max() < 2e-4 * (1.0 + np.abs(ref).max() / 10.0), err.max()
    assert np.sqrt(np.mean(err ** 2)) < 2e-6
    assert got[0] == 0


@pytest.mark.parametrize("n", [8194, 100000, 2 * 1234567, 1 << 16])
def test_normalise_prepared_is_bit_identical(F, n):
    """fdas_normalise_prepared with the kernel spectrum from
    fdas_bluestein_prepare gives fdas_normalise's spectrum bit for bit (the
    same FFT of the same chirp, computed once instead of per call); a power
    of two needs no spectrum."""
    x = torch.from_numpy(synth.make_series(n, ((n / 7 + 0.2, 6.0, 12.0),), 5)).cuda()
    wb = F.fdas_normalise_workspace_bytes(n)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    a = torch.empty(n // 2, dtype=torch.complex64, device="cuda")
    b = torch.full((n // 2,), float("nan"), dtype=torch.complex64, device="cuda")
    F.fdas_normalise(x, n, 1024, a, work, wb)
    cb = F.fdas_bluestein_bytes(n)
    chirp = torch.empty(max(cb, 16), dtype=torch.uint8, device="cuda") if cb else None
    if cb:
        F.fdas_bluestein_prepare(n, chirp, work, wb)
    work.fill_(0x7f)                      # the prepared call must not read stale scratch
    F.fdas_normalise_prepared(x, n, 1024, b, work, wb, chirp)
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.float32), b.view(torch.float32))


def test_normalise_zero_series_gives_zero(F):
    n = 1 << 14
    S = _search(F, n=n, L=2048, M=256, zmin=0, zmax=0, zstep=1, plane=False)
    S.series.zero_()
    S.normalise()
    assert torch.count_nonzero(S.spec).item() == 0


# ------------------------------------------------------------------ convolver (a4-a7)
CASES = [
    # n, L, M, zmin, zmax, zstep, interbin
    (1 << 14, 1024, 64, -20, 20, 2, 1),      # 8.53 segments: ragged tail
    (1 << 14, 2048, 64, -20, 20, 2, 1),
    (1 << 14, 4096, 128, -20, 20, 2, 1),
    (1 << 14, 2048, 64, -21, 21, 2, 1),      # symmetric grid without z = 0
    (1 << 14, 2048, 128, -10, 30, 5, 1),     # asymmetric grid: no conjugation
    (1 << 14, 1024, 64, -20, 20, 2, 0),      # no interbinning
    (1 << 13, 4096, 256, -6, 6, 2, 1),       # one segment longer than the spectrum
]


@pytest.mark.parametrize("n,L,M,zmin,zmax,zstep,ib", CASES)
def test_plane_matches_oracle(F, n, L, M, zmin, zmax, zstep, ib):
    x = synth.make_series(n, ((n / 7 + 0.25, 6.0, 18.0), (n / 3, -14.0, 20.0)), 9)
    A = O.normalise(O.real_spectrum(x), 1024).astype(np.complex64)
    S = _search(F, n=n, L=L, M=M, zmin=zmin, zmax=zmax, zstep=zstep, interbin=ib)
    _upload_spec(S, A)
    S.make_templates()
    S.correlate(fused=False)
    got = S.plane2d().cpu().numpy().astype(np.float64)
    ref = O.plane(A.astype(np.complex128), O.z_grid(zmin, zmax, zstep), bool(ib))
    assert got.shape == ref.shape
    err = np.abs(got - ref)
    assert err.max() < PTOL, (err.max(), np.unravel_index(np.argmax(err), err.shape))


@pytest.mark.parametrize("nb", [1, 5, 999, 1793, 6001])
def test_plane_odd_and_tiny_spectra(F, nb):
    A = synth.random_spectrum(nb, 40 + nb)
    S = _search(F, n=1 << 14, L=2048, M=256, zmin=-40, zmax=40, zstep=4)
    S.spec[:nb].copy_(torch.from_numpy(A))
    S.make_templates()
    S.plane.fill_(-7.0)
    S.correlate(fused=False, nb=nb)
    P = S.plane.view(S.K, S.row_stride).cpu().numpy()
    ref = O.plane(A.astype(np.complex128), O.z_grid(-40, 40, 4))
    assert np.abs(P[:, : 2 * nb] - ref).max() < PTOL
    assert np.all(P[:, 2 * nb:] == -7.0)     # nothing written past the row's 2nb columns


def test_fused_threshold_matches_oracle_and_overflow(F):
    n = 1 << 14
    x = synth.make_series(n, ((1500.0, 6.0, 20.0), (4100.5, -12.0, 18.0)), 7)
    A = O.normalise(O.real_spectrum(x), 1024).astype(np.complex64)
    S = _search(F, n=n, L=1024, M=64, zmin=-20, zmax=20, zstep=2, thr=8.0, cap=1 << 14)
    _upload_spec(S, A)
    S.make_templates()
    S.status.zero_()
    S.correlate(fused=True)
    r, c, p, fl, total = S.candidates()
    assert total == len(r) and total > 50 and S.status.item() == 0
    ref = O.plane(A.astype(np.complex128), O.z_grid(-20, 20, 2))
    rr, cc, pp, _ = O.threshold(ref, 8.0, flags=False)
    compare_candidates((r, c, p), (rr, cc, pp), 8.0)
    # too small a buffer: count keeps the total, the status word flags the overflow
    S.cap = 10
    S.fused.cap = 10
    S.correlate(fused=True)
    assert int(S.count.item()) == total
    assert S.status.item() & 2


# ------------------------------------------------------------------ threshold (a8)
def test_threshold_bit_exact_on_same_plane(F):
    rng = np.random.default_rng(5)
    P = rng.exponential(1.0, size=(13, 1003)).astype(np.float32) * 4
    P[3, 10] = P[3, 11] = 40.0          # tie: the earlier one is the peak
    P[0, 0] = 30.0
    P[12, 1002] = 50.0
    P[7, 500] = 20.0                    # equal to the threshold: not a candidate
    stride = 1008
    dev = torch.zeros(13 * stride, dtype=torch.float32, device="cuda")
    dev.view(13, stride)[:, :1003] = torch.from_numpy(P).cuda()
    cap = 4096
    out = torch.zeros(cap * 4, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    F.fdas_threshold(dev, 13, 1003, stride, 20.0, F.FDAS_CAND_PEAK, out, cap, count, status)
    k = int(count.item())
    c = out[: 4 * k].view(k, 4).cpu().numpy()
    o = np.lexsort((c[:, 1], c[:, 0]))
    c = c[o]
    rows, cols, pw, fl = O.threshold(P.astype(np.float64), 20.0)
    assert k == len(rows) and status.item() == 0
    assert np.array_equal(c[:, 0], rows) and np.array_equal(c[:, 1], cols)
    assert np.array_equal(c[:, 2].view(np.float32), pw.astype(np.float32))
    assert np.array_equal(c[:, 3], fl)


# ------------------------------------------------------------------ whole path, small workload
def test_small_workload_end_to_end(F):
    wl = synth.workload("small")
    x = wl.series()
    S = _search(F, n=wl.n, L=wl.L, M=wl.M, zmin=wl.zmin, zmax=wl.zmax, zstep=wl.zstep,
                thr=wl.threshold)
    S.series.copy_(torch.from_numpy(x))
    S.status.zero_()
    S.step()
    r, c, p, fl, total = S.candidates()
    A, P, (rr, cc, pp, _) = O.search(x, wl.zmin, wl.zmax, wl.zstep, wl.median_block, wl.threshold)
    got = S.plane2d().cpu().numpy().astype(np.float64)
    assert np.abs(got - P).max() < PTOL
    compare_candidates((r, c, p), (rr, cc, pp), wl.threshold)
    # the injection (r0 = 20000.3, z0 = +10) is recovered within 1/2 bin and one z step
    k, col = np.unravel_index(np.argmax(got), got.shape)
    zs = O.z_grid(wl.zmin, wl.zmax, wl.zstep)
    assert abs(col / 2.0 - 20000.3) <= 0.5 and abs(zs[k] - 10.0) <= wl.zstep


# ------------------------------------------------------------------ production size, sampled
@pytest.mark.parametrize("L", [1024, 2048, 4096])
def test_production_plane_sampled(F, L):
    wl = synth.workload("production")
    x = wl.series()
    A = O.normalise(O.real_spectrum(x), wl.median_block).astype(np.complex64)
    A64 = A.astype(np.complex128)
    S = _search(F, n=wl.n, L=L, M=wl.M, zmin=wl.zmin, zmax=wl.zmax, zstep=wl.zstep,
                thr=wl.threshold, cap=1 << 16)
    _upload_spec(S, A)
    S.make_templates()
    S.status.zero_()
    S.correlate(fused=True)
    torch.cuda.synchronize()
    plane = S.plane2d()
    zs = O.z_grid(wl.zmin, wl.zmax, wl.zstep)
    # every row over 64 random 4096-column windows, both ends and every
    # injection's neighbourhood
    rng = np.random.default_rng(L)
    wins = [(int(r), 2048) for r in rng.integers(0, wl.nb - 2048, 64)]
    wins += [(0, 2048), (wl.nb - 2048, 2048)]
    wins += [(int(r0) - 128, 256) for r0, _, _ in wl.injections]
    for r0, w in wins:
        got = plane[:, 2 * r0: 2 * (r0 + w)].cpu().numpy().astype(np.float64)
        ref = O.plane_window(A64, zs, r0, w)
        assert np.abs(got - ref).max() < PTOL, (r0, np.abs(got - ref).max())
    # every fused candidate is a true crossing (oracle value within tolerance)
    r, c, p, fl, total = S.candidates()
    assert total == len(r) and S.status.item() == 0
    ref = O.plane_points(A64, zs, r, c)
    assert np.abs(ref - p).max() < PTOL
    assert np.all(ref > wl.threshold - PTOL)
    # each injection is recovered within 1/2 bin and one z step (Section 5.2)
    for r0, z0, snr in wl.injections:
        lo = 2 * (int(r0) - 8)
        sub = plane[:, lo: lo + 32].cpu().numpy()
        k, cc = np.unravel_index(np.argmax(sub), sub.shape)
        if snr >= 8:
            assert abs((lo + cc) / 2.0 - r0) <= 0.5 + 1e-9 and abs(zs[k] - z0) <= wl.zstep

"""Pins for the FP64 oracle: each checks it against something other than itself.

Mathematics and the paper fix every expected value here: the defining
integral (evaluated by an adaptive library integrator, not the oracle's
Fresnel form), closed forms, Parseval, brute-force sums, a different
algorithm (overlap-save with FFTs) for the same correlation, and the
amplitude-loss figures printed in Section 3.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle.fdas_oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- templates
def _integral(z, d):
    """R_z(d) by scipy.integrate.quad of the real and imaginary parts."""
    ph = lambda u: 2 * math.pi * (z * u * u / 2 - (d + z / 2) * u)  # noqa: E731
    kw = dict(limit=2000, epsabs=1e-14, epsrel=1e-13)
    re = integrate.quad(lambda u: math.cos(ph(u)), 0, 1, **kw)[0]
    im = integrate.quad(lambda u: math.sin(ph(u)), 0, 1, **kw)[0]
    return re + 1j * im


@pytest.mark.parametrize("z", [2.0, 10.0, 64.0, 200.0, -200.0, -7.3, 0.3, -0.05, 3.7])
def test_template_matches_defining_integral(z):
    ds = [-108, -40, -3, -1, 0, 0.37, 1, 2.5, 40, 108]
    got = O.template_response(z, np.array(ds, float))
    ref = np.array([_integral(z, d) for d in ds])
    assert np.abs(got - ref).max() < 1e-10


def test_template_z0_is_delta_and_sinc():
    d = np.arange(-20, 21)
    R = O.template_response(0.0, d)
    assert np.abs(R - (d == 0)).max() < 1e-15
    f = np.array([0.25, 0.5, -0.5, 1.5])
    ref = (1 - np.exp(-2j * np.pi * f)) / (2j * np.pi * f)   # int_0^1 e^{-i2pi f u} du
    assert np.abs(O.template_response(0.0, f) - ref).max() < 1e-15


@pytest.mark.parametrize("z", [2.0, 17.0, 200.0])
def test_template_plus_minus_z_symmetry(z):
    # integer offsets: R_{-z}(d) = conj(R_z(d)) (the symmetry used in Section 4.2)
    d = np.arange(-120, 121)
    assert np.abs(O.template_response(-z, d) - np.conj(O.template_response(z, d))).max() < 1e-12
    # fractional offsets pick up exp(-i 2 pi d)  (u -> 1-u in the integral)
    f = np.array([-3.3, 0.25, 7.5])
    lhs = O.template_response(-z, f)
    rhs = np.exp(-2j * np.pi * f) * np.conj(O.template_response(z, f))
    assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("z", [0.0, 6.0, 200.0])
def test_template_parseval_and_sum(z):
    # R_z(d) are the Fourier-series coefficients of exp(i pi z (u^2 - u)) on [0,1]:
    # sum |R|^2 = int |f|^2 = 1 and sum R = f(0) = 1.  f' jumps by 2 i pi z at
    # the ends, so R_z(d) ~ -i z / (2 pi d^2) and the tail beyond |d| = D sums
    # to about i z / (pi D), which the partial sum misses.
    D = 20000
    d = np.arange(-D, D + 1)
    R = O.template_response(z, d)
    assert abs(np.sum(np.abs(R) ** 2) - 1.0) < 2e-5
    assert abs(np.sum(R) - (1.0 - 1j * z / (math.pi * D))) < 1e-6


def test_half_width():
    assert [O.half_width(z) for z in (0, 1, 2, -21, 200, -200)] == [8, 9, 9, 19, 108, 108]
    assert list(O.z_grid(-20, 20, 2)[:3]) == [-20, -18, -16] and len(O.z_grid(-200, 200, 2)) == 201


# ---------------------------------------------------------------- front end
@pytest.mark.parametrize("n", [64, 90, 250])   # a power of two and two lengths that are not
def test_real_spectrum_bruteforce_and_sign(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    k = np.arange(n // 2)[:, None]
    t = np.arange(n)[None, :]
    ref = (np.exp(-2j * np.pi * ((k * t) % n) / n) * x[None, :]).sum(1)   # exact phase reduction
    ref[0] = 0
    assert np.abs(O.real_spectrum(x) - ref).max() < 1e-12
    # sign convention: sin(2 pi k0 t/n) -> X_k0 = -i n/2
    s = np.sin(2 * np.pi * 5 * np.arange(n) / n)
    X = O.real_spectrum(s)
    assert abs(X[5] - (-0.5j * n)) < 1e-12 and np.abs(np.delete(X, 5)).max() < 1e-12


@pytest.mark.parametrize("n", [4096, 6000])
def test_real_spectrum_parseval(n):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n)
    x -= x.mean()
    X = np.fft.fft(x)
    # sum over the half spectrum (bins 1..n/2-1) is half the energy minus Nyquist
    half = np.sum(np.abs(O.real_spectrum(x)) ** 2)
    total = n * np.sum(x ** 2)
    assert abs(2 * half + abs(X[n // 2]) ** 2 - total) < 1e-8 * total


def test_block_median_rank_and_tail():
    X = np.sqrt(np.array([3.0, 1.0, 2.0, 5.0, 9.0, 4.0, 7.0]))
    # blocks of 4: [3,1,2,5] -> sorted 1,2,3,5 -> rank 1 -> 2 ; tail [9,4,7] -> 4,7,9 -> rank 1 -> 7
    assert np.allclose(O.block_medians(X, 4), [2.0, 7.0])
    A = O.normalise(X, 4)
    assert np.allclose(A[:4], X[:4] / math.sqrt(2.0 / math.log(2)))
    assert np.all(O.normalise(np.zeros(8), 4) == 0)


def test_normalised_noise_is_unit_exponential():
    x = synth.make_series(1 << 17, (), seed=11)
    A = O.normalise(O.real_spectrum(x), 1024)
    P = np.abs(A[1024:]) ** 2
    # the median of each block is ln 2 by construction; Exp(1) has mean 1, var 1
    assert np.allclose(O.block_medians(A[1024:], 1024), math.log(2.0), rtol=1e-12)
    assert abs(P.mean() - 1.0) < 0.02 and abs(P.var() - 1.0) < 0.06
    assert abs(np.mean(P > 3.0) - math.exp(-3.0)) < 0.005


# ---------------------------------------------------------------- correlation
def test_correlate_z0_is_identity():
    A = synth.random_spectrum(500, 3).astype(np.complex128)
    F = O.correlate(A, [0.0])
    assert np.abs(F[0] - A).max() < 1e-14


def test_correlate_matches_python_loops():
    A = synth.random_spectrum(40, 4).astype(np.complex128)
    zs = [-6.0, 0.0, 4.0]
    F = O.correlate(A, zs)
    for k, z in enumerate(zs):
        h = O.half_width(z)
        for r in range(40):
            acc = 0j
            for d in range(-h, h + 1):
                if 0 <= r + d < 40:
                    acc += A[r + d] * np.conj(O.template_response(z, d))
            assert abs(F[k, r] - acc) < 1e-12


def test_correlate_equals_overlap_save():
    """Overlap-save with numpy FFTs (Section 3, Fig. 1) gives the tap sum."""
    nb, L, M = 3000, 256, 64
    B = L - M
    A = synth.random_spectrum(nb, 5).astype(np.complex128)
    zs = [-20.0, -6.0, 0.0, 14.0, 20.0]
    F = O.correlate(A, zs)
    padded = np.concatenate([np.zeros(M // 2), A, np.zeros(L)])
    for k, z in enumerate(zs):
        H = O.kernel_spectrum(z, L)
        out = []
        for s in range((nb + B - 1) // B):
            blk = padded[s * B: s * B + L]
            y = np.fft.ifft(np.fft.fft(blk) * H) * L
            out.append(y[M // 2: M // 2 + B])
        osv = np.concatenate(out)[:nb]
        assert np.abs(osv - F[k]).max() < 1e-10


def test_correlate_matched_template_peaks_at_truth():
    # A spectrum equal to a template (shifted to r0) correlates to sum |R|^2 at
    # (r0, z0) and, by Cauchy-Schwarz, to less anywhere else.
    nb, r0 = 2000, 900
    zs = O.z_grid(-20, 20, 2)
    for z0 in (-14.0, 0.0, 8.0):
        d = np.arange(-400, 401)
        A = np.zeros(nb, np.complex128)
        A[r0 + d] = O.template_response(z0, d)
        F = O.correlate(A, zs)
        k0 = int(np.where(zs == z0)[0][0])
        h = O.half_width(z0)
        e = np.sum(np.abs(O.template_response(z0, np.arange(-h, h + 1))) ** 2)
        assert abs(F[k0, r0] - e) < 1e-12
        P = np.abs(F) ** 2
        assert np.unravel_index(np.argmax(P), P.shape) == (k0, r0)


# ---------------------------------------------------------------- interbinning
def _tone(nb, r0):
    # continuous-limit spectrum of a unit tone at fractional bin r0: R_0(k - r0)
    return O.template_response(0.0, np.arange(nb) - r0)


def test_interbin_half_and_integer_tones():
    nb = 64
    P = O.power_plane(O.correlate(_tone(nb, 20.5), [0.0]))
    assert abs(P[0, 2 * 20 + 1] - 1.0) < 1e-12            # half bin recovers full amplitude
    assert abs(P[0, 2 * 20] - (2 / math.pi) ** 2) < 1e-12   # sinc(1/2)^2 at the full bin
    P = O.power_plane(O.correlate(_tone(nb, 20.0), [0.0]))
    assert abs(P[0, 40] - 1.0) < 1e-12 and abs(P[0, 41] - (math.pi / 4) ** 2) < 1e-12
    assert P[0, -1] == 0.0


def test_interbin_worst_case_loss_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "interbin_loss.json")))
    nb = 64
    best_ib, best_full = [], []
    for f in np.linspace(0.0, 1.0, 201):
        P = O.power_plane(O.correlate(_tone(nb, 20.0 + f), [0.0]))[0, 36:48]
        best_ib.append(math.sqrt(P.max()))
        best_full.append(math.sqrt(P[0::2].max()))
    loss_ib = 1 - min(best_ib)
    loss_full = 1 - min(best_full)
    assert abs(loss_ib - g["max_amplitude_loss_interbinned"]) < g["tolerance"]
    assert abs(loss_full - g["max_amplitude_loss_full_bins_only"]) < g["tolerance"]


def test_plane_window_and_points_agree_with_full_plane():
    A = synth.random_spectrum(700, 6).astype(np.complex128)
    zs = O.z_grid(-10, 10, 2)
    P = O.plane(A, zs)
    assert np.allclose(O.plane_window(A, zs, 100, 50), P[:, 200:300], atol=1e-13, rtol=0)
    assert np.allclose(O.plane_window(A, zs, 650, 50), P[:, 1300:1400], atol=1e-13, rtol=0)
    zi = np.array([0, 3, 10, 10, 5])
    col = np.array([0, 77, 1399, 1398, 640])
    assert np.allclose(O.plane_points(A, zs, zi, col), P[zi, col], atol=1e-13, rtol=0)
    assert np.allclose(O.plane(A, zs, interbin=False), P[:, 0::2], atol=1e-13, rtol=0)


# ---------------------------------------------------------------- candidates
def test_threshold_and_peak_ties():
    P = np.zeros((3, 6))
    P[1, 2] = 30.0
    P[1, 3] = 30.0     # tie with the earlier neighbour -> (1,2) is the peak
    P[0, 0] = 25.0
    P[2, 5] = 19.0
    P[2, 4] = 21.0
    rows, cols, pw, fl = O.threshold(P, 20.0)
    assert list(zip(rows, cols)) == [(0, 0), (1, 2), (1, 3), (2, 4)]
    assert list(fl) == [1, 1, 0, 0]          # (2,4) is below its neighbour (1,3)
    assert np.all(pw > 20.0)
    rows, cols, pw, fl = O.threshold(np.full((2, 2), 20.0), 20.0)
    assert len(rows) == 0                     # strict P > T


def test_injection_recovered_on_grid():
    """An on-grid chirp peaks exactly at its (r0, z0), power ~ SNR^2 sum|R|^2."""
    n, r0, z0, snr = 1 << 14, 3000.0, 8.0, 30.0
    x = synth.make_series(n, ((r0, z0, snr),), seed=21)
    A, P, (rows, cols, pw, fl) = O.search(x, -20, 20, 2, 1024, 20.0)
    k, c = np.unravel_index(np.argmax(P), P.shape)
    assert O.z_grid(-20, 20, 2)[k] == z0 and c == 2 * int(r0)
    h = O.half_width(z0)
    e = np.sum(np.abs(O.template_response(z0, np.arange(-h, h + 1))) ** 2)
    assert abs(P[k, c] / (snr ** 2 * e) - 1.0) < 0.15
    assert np.any((rows == k) & (cols == c) & (fl == O.PEAK_FLAG))


def test_injection_recovered_off_grid_within_paper_tolerance():
    """Off-grid truths are found within +-1/2 bin and +-1 z step (Section 5.2)."""
    wl = synth.workload("tiny")
    A, P, _ = O.search(wl.series(), wl.zmin, wl.zmax, wl.zstep, wl.median_block, wl.threshold)
    zs = O.z_grid(wl.zmin, wl.zmax, wl.zstep)
    for r0, z0, snr in wl.injections:
        lo, hi = int(2 * (r0 - 8)), int(2 * (r0 + 8))
        sub = P[:, lo:hi]
        k, c = np.unravel_index(np.argmax(sub), sub.shape)
        assert abs((lo + c) / 2.0 - r0) <= 0.5 + 1e-9
        assert abs(zs[k] - z0) <= wl.zstep


# ---------------------------------------------------------------- refinement
def test_response_derivatives_match_finite_differences():
    for z in (150.0, 7.3, 0.3, 0.0, -42.0):
        d = np.array([-60.2, -3.5, 0.0, 0.45, 12.0])
        R, Rd, Rz = O.response_derivs_quadrature(z, d)
        assert np.abs(R - O.template_response(z, d)).max() < 1e-11
        h = 1e-5
        Rdp = O.response_derivs_quadrature(z, d + h)[0]
        Rdm = O.response_derivs_quadrature(z, d - h)[0]
        Rzp = O.response_derivs_quadrature(z + h, d)[0]
        Rzm = O.response_derivs_quadrature(z - h, d)[0]
        assert np.abs((Rdp - Rdm) / (2 * h) - Rd).max() < 1e-6
        assert np.abs((Rzp - Rzm) / (2 * h) - Rz).max() < 1e-6


def test_refine_power_on_grid_equals_tap_sum():
    # at an integer bin and a grid z, with m = h(z), P is |F_z(r)|^2 of Eq. 23
    A = synth.random_spectrum(600, 8).astype(np.complex128)
    for z in (-14.0, 0.0, 6.0):
        m = O.half_width(z)
        F = O.correlate(A, [z], 250, 1)[0, 0]
        P, _, _, S = O.refine_power(A, 250.0, z, m)
        assert abs(S - F) < 1e-10 and abs(P - abs(F) ** 2) < 1e-9


def test_refine_gradients_match_finite_differences():
    A = synth.random_spectrum(400, 9).astype(np.complex128)
    m = 20
    for r, z in ((150.3, 4.2), (201.49, -7.9), (90.0, 0.25)):
        P, gr, gz, _ = O.refine_power(A, r, z, m)
        h = 1e-5
        fr = (O.refine_power(A, r + h, z, m)[0] - O.refine_power(A, r - h, z, m)[0]) / (2 * h)
        fz = (O.refine_power(A, r, z + h, m)[0] - O.refine_power(A, r, z - h, m)[0]) / (2 * h)
        assert abs(fr - gr) < 1e-5 * (1 + abs(gr)) and abs(fz - gz) < 1e-5 * (1 + abs(gz))
        k, g = O.refine_grad_spec(A, r, z, m)
        for idx in (0, len(k) // 2, len(k) - 1):
            Ap, Am = A.copy(), A.copy()
            Ap[k[idx]] += h
            Am[k[idx]] -= h
            dre = (O.refine_power(Ap, r, z, m)[0] - O.refine_power(Am, r, z, m)[0]) / (2 * h)
            Ap, Am = A.copy(), A.copy()
            Ap[k[idx]] += 1j * h
            Am[k[idx]] -= 1j * h
            dim = (O.refine_power(Ap, r, z, m)[0] - O.refine_power(Am, r, z, m)[0]) / (2 * h)
            assert abs((dre + 1j * dim) - g[idx]) < 1e-6 * (1 + abs(g[idx]))


def test_refine_ascent_finds_an_injected_chirp():
    n, r0, z0 = 1 << 14, 3000.37, 7.4
    x = synth.make_series(n, ((r0, z0, 40.0),), seed=31)
    A = O.normalise(O.real_spectrum(x), 1024)
    r, z, P = O.refine_ascent(A, 3000.5, 8.0, m=O.half_width(20), steps=20)
    assert abs(r - r0) < 0.05 and abs(z - z0) < 0.3
    assert P > O.refine_power(A, 3000.5, 8.0, O.half_width(20))[0]


# ---------------------------------------------------------------- 2-bin Fourier interpolation
def test_half_bin_correlation_even_columns_are_the_integer_tap_sum():
    A = synth.random_spectrum(900, 12).astype(np.complex128)
    zs = O.z_grid(-12, 12, 4)
    Fh = O.correlate_half(A, zs)
    F = O.correlate(A, zs)
    assert np.abs(Fh[:, 0::2] - F).max() < 1e-12


def test_half_bin_correlation_recovers_a_matched_half_bin_template():
    # noise-free spectrum A_k = R_z0(k - rho0) at a half-integer rho0: F(rho0)
    # is the template energy over the window (Cauchy-Schwarz equality)
    for z0 in (0.0, 6.0, -14.0):
        rho0 = 300.5
        k = np.arange(700)
        A = O.template_response(z0, k - rho0)
        h = O.half_width(z0)
        m0 = int(2 * rho0)
        Fh = O.correlate_half(A, [z0], 280, 40)[0]
        d = np.arange(-h, h + 1) - 0.5
        d = d[np.abs(d) <= h]
        energy = np.sum(np.abs(O.template_response(z0, d)) ** 2)
        F0 = Fh[m0 - 2 * 280]
        assert abs(F0 - energy) < 1e-12 * energy


def test_half_bin_correlation_matches_quadrature_responses():
    # the odd columns again, with R from Gauss-Legendre quadrature of its integral
    A = synth.random_spectrum(400, 13).astype(np.complex128)
    for z in (10.0, -3.0, 0.0):
        h = O.half_width(z)
        Fh = O.correlate_half(A, [z], 100, 50)[0]
        for i in (0, 17, 49):
            rho = 100 + i + 0.5
            j = np.arange(int(np.ceil(rho - h)), int(np.floor(rho + h)) + 1)
            R, _, _ = O.response_derivs_quadrature(z, j - rho)
            ref = np.sum(A[j] * np.conj(R))
            assert abs(Fh[2 * i + 1] - ref) < 1e-9 * (1 + abs(ref))


# ---------------------------------------------------------------- harmonic summing
def test_harmonic_sum_brute_force_tiny():
    rng = np.random.default_rng(14)
    zmin, zstep, K, W = -12, 3, 9, 37            # z = -12..12 step 3
    P = rng.exponential(1.0, (K, W))
    for H in (2, 4, 8):
        S = O.harmonic_sum(P, zmin, zstep, H)
        for j in range(K):
            for c in range(W):
                tot, ok = 0.0, True
                for h in range(1, H + 1):
                    z = h * (zmin + j * zstep)
                    row = (z - zmin) / zstep
                    if not (0 <= row < K) or h * c >= W:
                        ok = False
                        break
                    tot += P[int(row), h * c]
                if ok:
                    assert abs(S[j, c] - tot) < 1e-12
                else:
                    assert np.isnan(S[j, c])


def test_harmonic_sum_peaks_at_an_injected_pulse_trains_fundamental():
    # four harmonically related chirps (h r0, h z0): the 4-harmonic sum peaks
    # at the fundamental, where no single harmonic stands out
    n, r0, z0 = 1 << 15, 1000.0, 4.0
    inj = tuple((h * r0, h * z0, 6.0) for h in range(1, 5))
    x = synth.make_series(n, inj, 51)
    A = O.normalise(O.real_spectrum(x), 1024)
    zmin, zstep = -20, 2
    P = O.plane(A, O.z_grid(zmin, 20, 2))
    S = O.harmonic_sum(P, zmin, zstep, 4)
    j0 = int((z0 - zmin) // zstep)
    k, c = np.unravel_index(np.nanargmax(S), S.shape)
    assert k == j0 and abs(c / 2.0 - r0) <= 0.5
    assert S[k, c] > 2 * np.nanmax(P[:, 2 * int(r0) - 4: 2 * int(r0) + 5])


def test_harmonic_sum_of_noise_adds_the_mean_powers():
    x = synth.make_series(1 << 16, (), 52)
    A = O.normalise(O.real_spectrum(x), 1024)
    P = O.plane(A, O.z_grid(-4, 4, 2))
    S2 = O.harmonic_sum(P, -4, 2, 2)
    # even columns: full bins only; the fundamental row of z = 0 sums rows 2 and 2
    m_full = P[:, 0::2].mean()
    s = S2[2, 0::2]
    s = s[~np.isnan(s)]
    assert abs(s.mean() - 2 * m_full) < 0.03 * 2 * m_full


def _brute_harmonic_candidates(P, zmin, zstep, thresholds):
    """Independent triple loop over (level, row, column): every fundamental
    whose H harmonics (h z_j, h c) all fall on the plane, summed, kept if the
    sum is strictly above the level's threshold."""
    K, W = P.shape
    out = []
    for lev, thr in enumerate(thresholds):
        H = (2, 4, 8)[lev]
        for j in range(K):
            for c in range(W):
                tot, ok = 0.0, True
                for h in range(1, H + 1):
                    z = h * (zmin + j * zstep)
                    if (z - zmin) % zstep:
                        ok = False
                        break
                    row = (z - zmin) // zstep
                    if not (0 <= row < K) or h * c >= W:
                        ok = False
                        break
                    tot += P[row, h * c]
                if ok and tot > thr:
                    out.append((H, j, c, tot))
    return sorted(out)


@pytest.mark.parametrize("zmin,zstep,K,W", [(-12, 3, 9, 41), (-20, 2, 21, 64), (0, 1, 6, 30)])
def test_harmonic_candidates_match_brute_force(zmin, zstep, K, W):
    rng = np.random.default_rng(K * W)
    # integer-valued powers so that sums are exact and can equal a threshold
    P = rng.integers(0, 6, (K, W)).astype(np.float64)
    thresholds = (7.0, 13.0, 24.0)
    rows, cols, sums, Hs = O.harmonic_candidates(P, zmin, zstep, thresholds)
    got = sorted(zip(Hs.tolist(), rows.tolist(), cols.tolist(), sums.tolist()))
    ref = _brute_harmonic_candidates(P, zmin, zstep, thresholds)
    assert got == ref
    # the strict comparison matters: some sums sit exactly on a threshold
    ties = 0
    for lev, thr in enumerate(thresholds):
        S = O.harmonic_sum(P, zmin, zstep, 2 << lev)
        ties += int(np.sum(S == thr))
    assert ties > 0
    # fundamentals whose harmonics leave the plane are never listed
    for H, j, c, _ in got:
        assert H * c < W and 0 <= (H - 1) * (zmin // zstep) + H * j < K


# ---------------------------------------------------------------- significance
def test_noise_means_closed_forms_at_z0():
    m1 = O.noise_means([0.0], 1)[0]
    assert abs(m1[0] - 1.0) < 1e-15                      # R(0) = 1, R(d != 0) = 0
    assert abs(m1[1] - 2 * (np.pi / 4) ** 2) < 1e-15     # |R(0) - R(-1)|^2 + |R(1) - R(0)|^2
    m2 = O.noise_means([0.0], 2)[0]
    d = np.arange(-8, 8) + 0.5
    assert abs(m2[1] - np.sum(np.sinc(d) ** 2)) < 1e-14


@pytest.mark.parametrize("interbin", [1, 2])
def test_noise_planes_are_exponential_with_the_predicted_means(interbin):
    x = synth.make_series(1 << 17, (), 70 + interbin)
    A = O.normalise(O.real_spectrum(x), 1024)
    zs = O.z_grid(-30, 30, 15)
    P = O.plane(A, zs) if interbin == 1 else O.plane_interp2(A, zs)
    mu = O.noise_means(zs, interbin)
    for k in range(len(zs)):
        for e in (0, 1):
            v = P[k, e::2]
            assert abs(v.mean() / mu[k, e] - 1.0) < 0.03, (k, e, v.mean(), mu[k, e])
            tail = np.mean(v / mu[k, e] > 3.0)
            assert abs(tail - np.exp(-3.0)) < 0.006


def _normal_log_tail_asymptotic(s):
    """log P(N(0,1) > s) from the asymptotic series phi(s)/s (1 - 1/s^2 +
    3/s^4 - 15/s^6 + 105/s^8), accurate to ~1e-18 relative at s = 100."""
    u = 1.0 / (s * s)
    series = 1.0 - u + 3 * u ** 2 - 15 * u ** 3 + 105 * u ** 4
    return -0.5 * s * s - math.log(s * math.sqrt(2 * math.pi)) + math.log(series)


def test_sigma_of_log_tail_matches_the_normal_table():
    # upper-tail probabilities of the standard normal (tabulated values)
    table = {1.0: 0.15865525393145705, 2.0: 0.022750131948179195,
             3.0: 0.0013498980316300946, 5.0: 2.866515718791939e-07}
    for s, q in table.items():
        assert abs(O.sigma_of_log_tail(math.log(q)) - s) < 1e-12 * s
    for s in (40.0, 100.0):
        assert abs(O.sigma_of_log_tail(_normal_log_tail_asymptotic(s)) - s) < 1e-12 * s
    assert O.sigma_of_log_tail(math.log(0.5)) == 0.0
    assert O.sigma_of_log_tail(-0.1) == 0.0


def test_exp_sum_tail_special_cases():
    from scipy.special import gammaincc
    # one exponential: exp(-x/m)
    assert abs(O.exp_sum_log_tail(7.5, [1.5]) - (-5.0)) < 1e-14
    # equal means: the Erlang (integer-shape gamma) tail
    for H, x, m in ((2, 9.0, 1.0), (4, 30.0, 1.234), (8, 60.0, 1.0)):
        assert abs(O.exp_sum_log_tail(x, [m] * H) / math.log(gammaincc(H, x / m)) - 1) < 1e-13
    # two well-separated means: (m1 e^{-x/m1} - m2 e^{-x/m2}) / (m1 - m2) in FP64
    m1, m2, x = 1.0, 3.0, 11.0
    ref = math.log((m1 * math.exp(-x / m1) - m2 * math.exp(-x / m2)) / (m1 - m2))
    assert abs(O.exp_sum_log_tail(x, [m1, m2]) / ref - 1) < 1e-14
    # a tail is a probability, falls with x, and nearly equal means sit near the Erlang tail
    a = [O.exp_sum_log_tail(x, [1.0, 1.001, 0.999, 1.002]) for x in (2.0, 8.0, 20.0)]
    assert 0.0 > a[0] > a[1] > a[2]
    e = math.log(gammaincc(4, 20.0))
    assert abs(a[2] - e) < 0.01 * abs(e)


def test_exp_sum_tail_monte_carlo():
    rng = np.random.default_rng(91)
    means = np.array([1.0, 1.05, 1.2337, 0.97])
    s = (rng.exponential(1.0, (2_000_000, 4)) * means).sum(axis=1)
    for x in (6.0, 10.0):
        p = math.exp(O.exp_sum_log_tail(x, means))
        n = int(np.sum(s > x))
        assert abs(n - p * len(s)) < 5 * math.sqrt(p * len(s)), (x, n, p * len(s))

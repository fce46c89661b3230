"""Plain FP64 CPU oracle for the FDAS correlation hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import or run anything in
``oracle/``; the product (the CUDA library and its binding) never does.

It computes, slowly and by definition, what the GPU path computes fast:

* ``template_response``  R_z(d), the predicted normalised Fourier response of
  a constant-fdot signal at offset d from its mid-observation bin (Section 2,
  Eqs. 22-23; the paper cites the closed form rather than printing it).
* ``real_spectrum``      the real-to-complex DFT of the series (Section 4.1,
  DFT sign convention of Section 4.2), DC zeroed, Nyquist dropped.
* ``normalise``          block running-median power normalisation (Section 3).
* ``correlate``          the matched-filter correlation of Eq. 23 as a direct
  tap sum -- no FFT and no overlap-save (Section 3 explains overlap-save only
  as a fast way to evaluate this same sum).
* ``power_plane``        full-bin power and interbinned half-bin power
  (Eq. "f-interp", Section 3).
* ``threshold``          candidates P > T, with the local-maximum flag.
* ``refine_power``       the correlation power at continuous (r, z) and its
  derivatives, from the defining integrals by quadrature (Section 5.2's
  fine-binning around a detection, done as a continuous maximisation).

Readings of the paper that this file relies on (each also listed in the
design notes):

1. R_z(d) = int_0^1 exp(i 2 pi (z u^2/2 - (d + z/2) u)) du: a unit chirp
   centred on its mid-observation frequency.  It is the one centring under
   which the +/-z conjugate symmetry used in Section 4.2 holds exactly at
   integer offsets; no further normalisation (sum_d |R_z(d)|^2 -> 1).
2. Template half-width h(z) = ceil(|z|/2) + 8 taps.
3. DC bin zeroed, Nyquist bin dropped: n samples -> n/2 bins.
4. Median filter: non-overlapping blocks of ``block`` bins (the tail block
   takes the remainder); lower median (rank floor((len-1)/2)) of |X|^2;
   scale sqrt(median / ln 2), because the median of Exp(mu) is mu ln 2, so
   normalised noise power has mean 1.  A block whose median is 0 is set to 0.
5. Interbinning F_{r+1/2} = (pi/4)(F_r - F_{r+1}); the last half bin of a
   row (no F_{r+1}) is 0.
6. Plane layout: row j is z_j = zmin + j zstep; column 2r is the full bin r,
   column 2r+1 the half bin r + 1/2 (interbin) -- or column r (no interbin).

Parity pins for every function here live in tests/test_oracle.py.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np
from scipy.special import fresnel

__all__ = [
    "half_width", "z_grid", "template_response", "template_taps", "kernel_spectrum",
    "real_spectrum", "normalise", "block_medians", "correlate", "correlate_points",
    "power_plane", "plane", "plane_window", "plane_points", "threshold", "peak_flags",
    "search", "oracle_threads", "PEAK_FLAG", "response_derivs_quadrature", "refine_taps",
    "correlate_half", "plane_interp2", "harmonic_sum", "harmonic_candidates", "noise_means",
    "refine_power", "refine_grad_spec", "refine_ascent", "exp_sum_log_tail", "sigma_of_log_tail",
]

PEAK_FLAG = 1
_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_tapsum.so")
_lib = None
_lock = threading.Lock()


# --------------------------------------------------------------------------
# build / load the C tap sum (plain gcc + OpenMP)
# --------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile oracle/tapsum.c into oracle/_tapsum.so (plain C, -O2, OpenMP)."""
    src = os.path.join(_HERE, "tapsum.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
            lp = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_tapsum.argtypes = [dp, ctypes.c_int64, dp, ip, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, dp]
            lib.oracle_tapsum.restype = None
            lib.oracle_tapsum_points.argtypes = [dp, ctypes.c_int64, dp, ip, ctypes.c_int32,
                                                 ip, lp, ctypes.c_int64, dp]
            lib.oracle_tapsum_points.restype = None
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def oracle_threads() -> int:
    """Number of OpenMP threads the tap sum runs on."""
    return int(_load().oracle_num_threads())


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


# --------------------------------------------------------------------------
# templates (Section 2, Eqs. 22-23)
# --------------------------------------------------------------------------
def half_width(z: float) -> int:
    """Template half-width in taps: ceil(|z|/2) + 8 (reading 2)."""
    return int(math.ceil(abs(float(z)) / 2.0)) + 8


def z_grid(zmin: int, zmax: int, zstep: int) -> np.ndarray:
    """Plane row j holds z_j = zmin + j*zstep, j = 0..K-1."""
    K = (int(zmax) - int(zmin)) // int(zstep) + 1
    return (int(zmin) + int(zstep) * np.arange(K)).astype(np.float64)


def _response_quadrature(z: float, d: np.ndarray) -> np.ndarray:
    """R_z(d) by composite 16-point Gauss-Legendre quadrature of its definition.

    Used for 0 < |z| < 0.5, where the Fresnel closed form loses digits to the
    large cancelling phases.  Panels are sized to at most one cycle of the
    integrand.
    """
    x, w = np.polynomial.legendre.leggauss(16)
    out = np.empty(d.shape, np.complex128)
    for idx, dd in np.ndenumerate(d):
        panels = int(math.ceil(abs(dd) + abs(z) + 2.0))
        edges = np.linspace(0.0, 1.0, panels + 1)
        mid = 0.5 * (edges[1:] + edges[:-1])
        half = 0.5 * (edges[1:] - edges[:-1])
        u = (mid[:, None] + half[:, None] * x[None, :]).ravel()
        ww = (half[:, None] * w[None, :]).ravel()
        ph = z * u * u / 2.0 - (dd + z / 2.0) * u
        out[idx] = np.sum(ww * np.exp(2j * np.pi * ph))
    return out


def template_response(z: float, d) -> np.ndarray:
    """R_z(d) = int_0^1 exp(i 2 pi (z u^2/2 - (d + z/2) u)) du  (complex128).

    Closed form (z != 0), completing the square with q = -(d + z/2):
        R = exp(-i pi q^2/z) [ (C(Y)-C(X)) + i sgn(z) (S(Y)-S(X)) ] / sqrt(2|z|),
        X = sqrt(2|z|) q/z,  Y = sqrt(2|z|) (1 + q/z),
    with C, S the Fresnel integrals int_0^x cos/sin(pi t^2/2) dt
    (scipy.special.fresnel is the library primitive).  z = 0 gives
    exp(-i pi d) sinc(d), a Kronecker delta at integer d.
    """
    z = float(z)
    d = np.asarray(d, dtype=np.float64)
    if z == 0.0:
        return np.exp(-1j * np.pi * d) * np.sinc(d)
    if abs(z) < 0.5:
        return _response_quadrature(z, d)
    q = -(d + 0.5 * z)
    s = math.sqrt(2.0 * abs(z))
    X = s * q / z
    Y = s * (1.0 + q / z)
    SX, CX = fresnel(X)          # scipy returns (S, C)
    SY, CY = fresnel(Y)
    sg = 1.0 if z > 0 else -1.0
    inner = (CY - CX) + 1j * sg * (SY - SX)
    return np.exp(-1j * np.pi * q * q / z) * inner / s


def template_taps(zs, hmax: int | None = None):
    """R[k, hmax + d] = R_{z_k}(d) for |d| <= h(z_k) (zero beyond), and h[k]."""
    zs = np.asarray(zs, np.float64)
    h = np.array([half_width(z) for z in zs], np.int32)
    if hmax is None:
        hmax = int(h.max()) if len(h) else 0
    R = np.zeros((len(zs), 2 * hmax + 1), np.complex128)
    for k, z in enumerate(zs):
        d = np.arange(-h[k], h[k] + 1)
        R[k, hmax - h[k]: hmax + h[k] + 1] = template_response(z, d)
    return R, h


def kernel_spectrum(z: float, L: int) -> np.ndarray:
    """H_z[k], k = 0..L-1, natural order: the length-L FIR kernel of template z.

    The kernel g[j] = conj(R_z(-j)) for |j| <= h is placed so that it is
    centred at bin 0 (j >= 0 at the start of the array, j < 0 wrapped to the
    end, zeros between: Section 3, Fig. 1); H = FFT_L(g) / L, the 1/L of the
    inverse transform being folded in here.  Circular convolution with g is
    then the correlation of Eq. 23.
    """
    h = half_width(z)
    g = np.zeros(L, np.complex128)
    j = np.arange(-h, h + 1)
    g[j % L] = np.conj(template_response(z, -j))
    return np.fft.fft(g) / L


# --------------------------------------------------------------------------
# front end (Sections 3 and 4.1): real FFT + running-median normalisation
# --------------------------------------------------------------------------
def real_spectrum(x) -> np.ndarray:
    """X_k = sum_n x_n exp(-i 2 pi k n / n_samples), k = 0..n/2-1; X_0 := 0.

    numpy's FFT is the library primitive.  The Nyquist bin is dropped.
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    X = np.fft.rfft(x)[: n // 2].copy()
    if n // 2 > 0:
        X[0] = 0.0
    return X


def block_medians(X, block: int = 1024) -> np.ndarray:
    """Lower median of |X|^2 over each block of ``block`` bins (reading 4)."""
    P = np.abs(np.asarray(X)) ** 2
    nb = P.shape[0]
    nblk = (nb + block - 1) // block
    med = np.empty(nblk, np.float64)
    for b in range(nblk):
        seg = P[b * block: (b + 1) * block]
        rank = (seg.shape[0] - 1) // 2
        med[b] = np.partition(seg, rank)[rank]
    return med


def normalise(X, block: int = 1024) -> np.ndarray:
    """A_k = X_k / sqrt(median_b / ln 2) for k in block b (0 if median_b = 0)."""
    X = np.asarray(X, dtype=np.complex128)
    med = block_medians(X, block)
    A = np.zeros_like(X)
    for b, m in enumerate(med):
        if m > 0.0:
            sl = slice(b * block, (b + 1) * block)
            A[sl] = X[sl] / math.sqrt(m / math.log(2.0))
    return A


# --------------------------------------------------------------------------
# correlation (Eq. 23) and power / interbinning (Eq. f-interp)
# --------------------------------------------------------------------------
def correlate(A, zs, r0: int = 0, nr: int | None = None) -> np.ndarray:
    """F[k, i] = sum_{|d| <= h_k} A[r0+i+d] conj(R_{z_k}(d)), A = 0 outside [0, nb)."""
    A = np.ascontiguousarray(np.asarray(A, np.complex128))
    nb = A.shape[0]
    if nr is None:
        nr = nb - r0
    R, h = template_taps(zs)
    R = np.ascontiguousarray(R)
    K, hmax = R.shape[0], (R.shape[1] - 1) // 2
    F = np.zeros((K, nr), np.complex128)
    if K and nr > 0:
        _load().oracle_tapsum(_ptr(A.view(np.float64), ctypes.c_double), nb,
                              _ptr(R.view(np.float64), ctypes.c_double),
                              _ptr(h, ctypes.c_int32), K, hmax, int(r0), int(nr),
                              _ptr(F.view(np.float64), ctypes.c_double))
    return F


def correlate_points(A, zs, zi, r) -> np.ndarray:
    """F at scattered points: template index zi[p], bin r[p]."""
    A = np.ascontiguousarray(np.asarray(A, np.complex128))
    zi = np.ascontiguousarray(np.asarray(zi, np.int32))
    r = np.ascontiguousarray(np.asarray(r, np.int64))
    R, h = template_taps(zs)
    R = np.ascontiguousarray(R)
    hmax = (R.shape[1] - 1) // 2
    F = np.zeros(zi.shape[0], np.complex128)
    if zi.shape[0]:
        _load().oracle_tapsum_points(_ptr(A.view(np.float64), ctypes.c_double), A.shape[0],
                                     _ptr(R.view(np.float64), ctypes.c_double),
                                     _ptr(h, ctypes.c_int32), hmax, _ptr(zi, ctypes.c_int32),
                                     _ptr(r, ctypes.c_int64), zi.shape[0],
                                     _ptr(F.view(np.float64), ctypes.c_double))
    return F


HALF_BIN_SCALE = (math.pi / 4.0) ** 2


def power_plane(F, interbin: bool = True, last_is_end: bool = True) -> np.ndarray:
    """Plane from correlated amplitudes F[k, r] (r = 0..nr-1).

    interbin: columns 2r = |F_r|^2 and 2r+1 = (pi/4)^2 |F_r - F_{r+1}|^2.
    If ``last_is_end`` the final half bin (no F_{r+1}) is 0; otherwise F must
    carry one extra column (r = nr) used only for the last half bin.
    """
    F = np.asarray(F)
    if not interbin:
        return np.abs(F) ** 2
    if last_is_end:
        nr = F.shape[1]
        nxt = np.concatenate([F[:, 1:], np.zeros((F.shape[0], 1), F.dtype)], axis=1)
    else:
        nr = F.shape[1] - 1
        nxt = F[:, 1:]
    P = np.empty((F.shape[0], 2 * nr), np.float64)
    P[:, 0::2] = np.abs(F[:, :nr]) ** 2
    P[:, 1::2] = HALF_BIN_SCALE * np.abs(F[:, :nr] - nxt) ** 2
    if last_is_end and nr:
        P[:, -1] = 0.0
    return P


def plane(A, zs, interbin: bool = True) -> np.ndarray:
    """The whole f-fdot power plane, K x (2nb or nb)."""
    return power_plane(correlate(A, zs), interbin, last_is_end=True)


def plane_window(A, zs, r0: int, nr: int, interbin: bool = True) -> np.ndarray:
    """Plane columns for bins r0..r0+nr-1 (2nr columns with interbinning)."""
    nb = np.asarray(A).shape[0]
    if not interbin:
        return power_plane(correlate(A, zs, r0, nr), False)
    ends = r0 + nr >= nb
    extra = 0 if ends else 1
    F = correlate(A, zs, r0, nr + extra)
    return power_plane(F, True, last_is_end=ends)


def correlate_half(A, zs, r0: int = 0, nr: int | None = None) -> np.ndarray:
    """Correlation at half-bin resolution (2-bin Fourier interpolation,
    Section 3 after Eq. f-interp): F[k, m] = sum over bins j with
    |j - m/2| <= h_k of A_j conj(R_{z_k}(j - m/2)), for m = 2 r0 .. 2(r0+nr)-1,
    A = 0 outside [0, nb).  Plain tap sum over the bins, numpy."""
    A = np.asarray(A, np.complex128)
    nb = A.shape[0]
    if nr is None:
        nr = nb - r0
    zs = np.atleast_1d(np.asarray(zs, np.float64))
    out = np.zeros((len(zs), 2 * nr), np.complex128)
    base = r0 + np.arange(nr)
    for kk, z in enumerate(zs):
        h = half_width(z)
        for e in (0, 1):               # m = 2 (r0 + i) + e, rho = r0 + i + e/2
            acc = np.zeros(nr, np.complex128)
            for q in range(-h, h + 2):   # bin j = r0 + i + q, offset d = q - e/2
                d = q - e / 2.0
                if abs(d) > h:
                    continue
                idx = base + q
                ok = (idx >= 0) & (idx < nb)
                Rd = complex(template_response(z, d))
                acc[ok] += A[idx[ok]] * np.conj(Rd)
            out[kk, e::2] = acc
    return out


def plane_interp2(A, zs, r0: int = 0, nr: int | None = None) -> np.ndarray:
    """Plane of the 2-bin Fourier interpolation: column m = |F(m/2)|^2."""
    return np.abs(correlate_half(A, zs, r0, nr)) ** 2


def harmonic_sum(P, zmin: int, zstep: int, H: int) -> np.ndarray:
    """S[j, c] = sum_{h=1}^{H} P[(h-1) zmin/zstep + h j, h c]: the powers at
    (h r, h z_j) summed over the first H harmonics, for every fundamental
    (j, c) whose H harmonics all lie on the plane (row in range, h c < width);
    NaN elsewhere.  Row j holds z_j = zmin + j zstep (zmin a multiple of zstep)."""
    P = np.asarray(P, np.float64)
    K, W = P.shape
    j0 = zmin // zstep
    S = np.full((K, W), np.nan)
    for j in range(K):
        rows = [(h - 1) * j0 + h * j for h in range(1, H + 1)]
        if min(rows) < 0 or max(rows) >= K:
            continue
        nc = (W - 1) // H + 1            # columns c with H c < W
        c = np.arange(nc)
        S[j, :nc] = sum(P[rows[h - 1], h * c] for h in range(1, H + 1))
    return S


def harmonic_candidates(P, zmin: int, zstep: int, thresholds):
    """(rows, cols, sums, H) with S_H > thresholds[level] (strict) for levels
    0, 1, 2 -> H = 2, 4, 8, for the fundamentals whose H harmonics all lie on
    the plane (harmonic_sum is NaN elsewhere and lists nothing); sorted by
    (H, row, col)."""
    out = []
    for lev, thr in enumerate(thresholds):
        H = 2 << lev
        S = harmonic_sum(P, zmin, zstep, H)
        j, c = np.nonzero(np.nan_to_num(S, nan=-np.inf) > thr)
        out.append((j, c, S[j, c], np.full(len(j), H)))
    return tuple(np.concatenate([o[i] for o in out]) for i in range(4))


def noise_means(zs, interbin: int = 1) -> np.ndarray:
    """(K, 2): mean power of unit complex Gaussian noise in the even and odd
    columns of each row (the variance of the correlated amplitude):
    even: sum_{|d|<=h} |R(d)|^2;  odd, interbin 1: (pi/4)^2 sum_d |Rt(d) -
    Rt(d-1)|^2 with Rt = R on |d| <= h and 0 outside; odd, interbin 2:
    sum over half-integer |d| <= h - 1/2 of |R(d)|^2; odd, interbin 0: as even."""
    zs = np.atleast_1d(np.asarray(zs, np.float64))
    out = np.zeros((len(zs), 2))
    for k, z in enumerate(zs):
        h = half_width(z)
        R = template_response(z, np.arange(-h, h + 1, dtype=np.float64))
        full = np.sum(np.abs(R) ** 2)
        if interbin == 1:
            Rt = np.concatenate([[0.0], R, [0.0]])
            odd = (np.pi / 4) ** 2 * np.sum(np.abs(Rt[1:] - Rt[:-1]) ** 2)
        elif interbin == 2:
            odd = np.sum(np.abs(template_response(z, np.arange(-h, h, dtype=np.float64) + 0.5)) ** 2)
        else:
            odd = full
        out[k] = (full, odd)
    return out


def plane_points(A, zs, zi, col, interbin: bool = True) -> np.ndarray:
    """Plane values at scattered (row zi[p], column col[p])."""
    A = np.asarray(A)
    nb = A.shape[0]
    zi = np.asarray(zi, np.int64)
    col = np.asarray(col, np.int64)
    if not interbin:
        return np.abs(correlate_points(A, zs, zi, col)) ** 2
    r = col // 2
    half = (col % 2) == 1
    Fr = correlate_points(A, zs, zi, r)
    out = np.abs(Fr) ** 2
    if half.any():
        rn = np.minimum(r[half] + 1, nb - 1)
        Fn = correlate_points(A, zs, zi[half], rn)
        ph = HALF_BIN_SCALE * np.abs(Fr[half] - Fn) ** 2
        ph[r[half] + 1 >= nb] = 0.0
        out[half] = ph
    return out


# --------------------------------------------------------------------------
# candidates
# --------------------------------------------------------------------------
def peak_flags(P, rows, cols) -> np.ndarray:
    """1 where (row, col) is a local maximum over its 8 neighbours.

    Ties go to the lower (row, col): the point must be strictly above every
    neighbour that precedes it in row-major order and at least equal to every
    neighbour after it.
    """
    P = np.asarray(P)
    K, W = P.shape
    out = np.zeros(len(rows), np.int32)
    for i, (a, c) in enumerate(zip(rows, cols)):
        v = P[a, c]
        ok = True
        for da in (-1, 0, 1):
            for dc in (-1, 0, 1):
                if da == 0 and dc == 0:
                    continue
                b, e = a + da, c + dc
                if b < 0 or b >= K or e < 0 or e >= W:
                    continue
                w = P[b, e]
                before = (b, e) < (a, c)
                if (before and not v > w) or ((not before) and not v >= w):
                    ok = False
        out[i] = PEAK_FLAG if ok else 0
    return out


def threshold(P, thr: float, flags: bool = True):
    """Candidates with P > thr, sorted by (row, col): arrays (rows, cols, power, flags)."""
    P = np.asarray(P)
    rows, cols = np.nonzero(P > thr)
    pw = P[rows, cols]
    fl = peak_flags(P, rows, cols) if flags else np.zeros(len(rows), np.int32)
    return rows.astype(np.int32), cols.astype(np.int32), pw, fl


def search(x, zmin, zmax, zstep, block=1024, thr=20.0, interbin=True):
    """Whole path on the CPU: spectrum -> normalise -> plane -> candidates."""
    A = normalise(real_spectrum(x), block)
    zs = z_grid(zmin, zmax, zstep)
    P = plane(A, zs, interbin)
    return A, P, threshold(P, thr)


# --------------------------------------------------------------------------
# candidate refinement over continuous (r, z)
# --------------------------------------------------------------------------
def response_derivs_quadrature(z: float, d):
    """R_z(d), dR/dd, dR/dz by composite 16-point Gauss-Legendre quadrature of
    their defining integrals (vectorised over d):
        R     = int_0^1 e^{i phi} du,
        dR/dd = int_0^1 (-i 2 pi u) e^{i phi} du,
        dR/dz = int_0^1 i pi (u^2 - u) e^{i phi} du,
    phi(u) = 2 pi (z u^2/2 - (d + z/2) u).  Panels hold at most one cycle."""
    d = np.atleast_1d(np.asarray(d, np.float64))
    x, w = np.polynomial.legendre.leggauss(16)
    panels = int(math.ceil(np.max(np.abs(d)) + abs(z) + 2.0))
    edges = np.linspace(0.0, 1.0, panels + 1)
    mid = 0.5 * (edges[1:] + edges[:-1])
    half = 0.5 * (edges[1:] - edges[:-1])
    u = (mid[:, None] + half[:, None] * x[None, :]).ravel()
    ww = (half[:, None] * w[None, :]).ravel()
    ph = 2.0 * np.pi * (z * u[None, :] ** 2 / 2.0 - (d[:, None] + z / 2.0) * u[None, :])
    e = ww[None, :] * np.exp(1j * ph)
    R = e.sum(1)
    Rd = (e * (-2j * np.pi * u[None, :])).sum(1)
    Rz = (e * (1j * np.pi * (u[None, :] ** 2 - u[None, :]))).sum(1)
    return R, Rd, Rz


def refine_taps(nb: int, r: float, m: int):
    """Tap bins k = [r]-m .. [r]+m inside [0, nb) and offsets d = k - r."""
    k0 = int(math.floor(r + 0.5))
    k = np.arange(k0 - m, k0 + m + 1)
    k = k[(k >= 0) & (k < nb)]
    return k, k - float(r)


def refine_power(A, r: float, z: float, m: int):
    """P = |S|^2 with S = sum_k A_k conj(R_z(k - r)), and dP/dr, dP/dz, S."""
    A = np.asarray(A)
    k, d = refine_taps(A.shape[0], r, m)
    R, Rd, Rz = response_derivs_quadrature(z, d)
    a = A[k].astype(np.complex128)
    S = np.sum(a * np.conj(R))
    Sr = np.sum(a * np.conj(-Rd))
    Sz = np.sum(a * np.conj(Rz))
    P = abs(S) ** 2
    return P, 2.0 * np.real(np.conj(S) * Sr), 2.0 * np.real(np.conj(S) * Sz), S


def refine_grad_spec(A, r: float, z: float, m: int):
    """dP/dA_k (d/dRe + i d/dIm) = 2 S R_z(k - r) at the taps k."""
    k, d = refine_taps(np.asarray(A).shape[0], r, m)
    R, _, _ = response_derivs_quadrature(z, d)
    _, _, _, S = refine_power(A, r, z, m)
    return k, 2.0 * S * R


def refine_ascent(A, r0: float, z0: float, m: int, steps: int = 20, lr_r: float = 0.15,
                  lr_z: float = 9.0):
    """Gradient ascent on log P: r += clamp(lr_r P_r/P, +-0.5), z += clamp(lr_z P_z/P, +-2)."""
    r, z = float(r0), float(z0)
    P = 0.0
    for it in range(steps + 1):
        P, gr, gz, _ = refine_power(A, r, z, m)
        if it == steps or not P > 0.0:
            break
        r += min(max(lr_r * gr / P, -0.5), 0.5)
        z += min(max(lr_z * gz / P, -2.0), 2.0)
    return r, z, P


# --------------------------------------------------------------------------
# significance: exact tails of plane powers and their harmonic sums
# --------------------------------------------------------------------------
def exp_sum_log_tail(x: float, means, dps: int = 80) -> float:
    """log P(X_1 + ... + X_H > x) for independent exponential X_i with the
    given means (noise powers of the H harmonics: Section 5.2 leaves their
    statistics open; each normalised plane value is exponential).

    By definition, in arbitrary precision (mpmath, `dps` digits):
      all means equal (m):  the Erlang tail  e^{-x/m} sum_{k<H} (x/m)^k / k!;
      all means distinct:   the hypoexponential tail
        sum_i prod_{j != i} m_i / (m_i - m_j) * e^{-x/m_i},
    which cancels badly in FP64 when the means are close; the precision
    absorbs that.  Means that repeat only in part are not supported."""
    import mpmath as mp
    m = [float(v) for v in np.atleast_1d(means)]
    if any(v <= 0.0 for v in m):
        raise ValueError("means must be positive")
    with mp.workdps(dps):
        X = mp.mpf(x)
        if X <= 0:
            return 0.0
        if all(v == m[0] for v in m):
            u = X / mp.mpf(m[0])
            tail = mp.e ** (-u) * mp.fsum(u ** k / mp.factorial(k) for k in range(len(m)))
        elif len(set(m)) == len(m):
            M = [mp.mpf(v) for v in m]
            tail = mp.mpf(0)
            for i, mi in enumerate(M):
                c = mp.mpf(1)
                for j, mj in enumerate(M):
                    if j != i:
                        c *= mi / (mi - mj)
                tail += c * mp.e ** (-X / mi)
        else:
            raise ValueError("means must be all equal or all distinct")
        return float(mp.log(tail))


def sigma_of_log_tail(logp: float, dps: int = 50) -> float:
    """One-sided Gaussian sigma s with P(N(0,1) > s) = exp(logp), i.e. the root
    of log(erfc(s / sqrt 2) / 2) = logp, found in arbitrary precision; 0 when
    exp(logp) >= 1/2."""
    import mpmath as mp
    if logp >= math.log(0.5):
        return 0.0
    with mp.workdps(dps):
        lp = mp.mpf(logp)
        f = lambda s: mp.log(mp.erfc(s / mp.sqrt(2)) / 2) - lp
        s0 = mp.sqrt(-2 * lp)          # bracket: the root lies in (0, sqrt(-2 logp)]
        return float(mp.findroot(f, (mp.mpf("1e-30"), s0), solver="illinois"))

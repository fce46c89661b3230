"""Helpers shared by the GPU parity tests (test code; neither oracle nor product)."""
import numpy as np


def bank_slot(k, L):
    """Bank storage slot of frequency k, restated from the layout in fdas.h."""
    k = np.asarray(k)
    Q, T = L // 256, L // 16
    a, k1, c2 = k % 16, (k // 16) % 16, k // 256
    c1, s2 = k1 % Q, k1 // Q
    t, i = a * Q + c1, s2 * Q + c2
    return 2 * ((i // 2) * T + t) + (i % 2)


def bank_natural(bank_f32, Kb, L):
    """(Kb, L) complex128 template spectra in natural frequency order."""
    b = np.asarray(bank_f32, np.float32).reshape(Kb, L, 2)
    c = b[..., 0].astype(np.float64) + 1j * b[..., 1].astype(np.float64)
    return c[:, bank_slot(np.arange(L), L)]


def sorted_cands(rows, cols, pw):
    o = np.lexsort((cols, rows))
    return np.asarray(rows)[o], np.asarray(cols)[o], np.asarray(pw)[o]


def compare_candidates(g, o, thr, tol=1e-3):
    """g, o: (rows, cols, power) sorted.  Identical except points within tol of thr."""
    gs = {(int(r), int(c)): float(p) for r, c, p in zip(*g)}
    os_ = {(int(r), int(c)): float(p) for r, c, p in zip(*o)}
    for key in set(gs) ^ set(os_):
        v = gs.get(key, os_.get(key))
        assert abs(v - thr) <= tol, ("candidate lists differ at", key, v)
    for key in set(gs) & set(os_):
        assert abs(gs[key] - os_[key]) <= tol, ("candidate power differs", key, gs[key], os_[key])

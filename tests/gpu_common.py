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
    """(Kb, L) complex128 template spectra in natural frequency order, and the
    (Kb, 16) mirror slots, both restated from the layout in fdas.h."""
    b = np.asarray(bank_f32, np.float32).reshape(Kb, L + 16, 2)
    c = b[..., 0].astype(np.float64) + 1j * b[..., 1].astype(np.float64)
    return c[:, bank_slot(np.arange(L), L)], c[:, L:]


def mirror_expected(H, L):
    """Expected mirror slots from natural-order spectra H (Kb, L): complex
    L + 2j + 1 - e holds H[-k(s)] for slot s = 2(7 - j)T + e (T = L/16), the
    slot of register 2(7 - j) + e of thread 0."""
    T = L // 16
    slot_k = np.empty(L, np.int64)
    slot_k[bank_slot(np.arange(L), L)] = np.arange(L)
    out = np.empty((H.shape[0], 16), H.dtype)
    for j in range(8):
        for e in range(2):
            s = 2 * (7 - j) * T + e
            out[:, 2 * j + 1 - e] = H[:, (-slot_k[s]) % L]
    return out


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

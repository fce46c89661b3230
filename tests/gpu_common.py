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
    mirror slots ((Kb, 16), or (Kb, 32) for L = 1024), both restated from the
    layouts in fdas.h."""
    if L == 1024:
        # float4 slot j*33 + l = (H[l + 64 j], H[l + 64 j + 32]); slot j*33 + 32 is
        # the mirror column
        b = np.asarray(bank_f32, np.float32).reshape(Kb, 16, 33, 2, 2)
        c = b[..., 0].astype(np.float64) + 1j * b[..., 1].astype(np.float64)
        j, l, e = np.meshgrid(np.arange(16), np.arange(32), np.arange(2), indexing="ij")
        H = np.empty((Kb, L), np.complex128)
        H[:, (l + 64 * j + 32 * e).ravel()] = c[:, :, :32, :].reshape(Kb, -1)
        return H, c[:, :, 32, :].reshape(Kb, 32)
    b = np.asarray(bank_f32, np.float32).reshape(Kb, L + 16, 2)
    c = b[..., 0].astype(np.float64) + 1j * b[..., 1].astype(np.float64)
    return c[:, bank_slot(np.arange(L), L)], c[:, L:]


def mirror_expected(H, L):
    """Expected mirror slots from natural-order spectra H (Kb, L): complex
    L + 2j + 1 - e holds H[-k(s)] for slot s = 2(7 - j)T + e (T = L/16), the
    slot of register 2(7 - j) + e of thread 0.  L = 1024: the mirror column's
    float4 j holds (H[64 j + 32], H[(64 j + 64) mod 1024])."""
    if L == 1024:
        out = np.empty((H.shape[0], 32), H.dtype)
        for j in range(16):
            out[:, 2 * j] = H[:, 64 * j + 32]
            out[:, 2 * j + 1] = H[:, (64 * j + 64) % L]
        return out
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

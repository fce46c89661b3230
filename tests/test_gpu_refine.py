"""GPU refinement kernels against the FP64 quadrature oracle and finite
differences: forward power and derivatives, the spectrum gradient through
the torch.autograd.Function, and the ascent from grid points to injected
constant-fdot signals.  Candidate positions are generated here, never taken
from a GPU plane."""
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


def _spec(nb, seed):
    return synth.random_spectrum(nb, seed)


def _candidates(nb):
    r = [150.3, 151.49, 151.51, 400.0, 3.2, nb - 2.6, 700.25, 1000.7, 1200.0, 1500.45]
    z = [4.2, -7.9, 0.0, 0.3, -0.45, 12.0, 0.7, -150.3, 199.9, -2.0]
    return np.array(r), np.array(z)


def test_refine_forward_matches_oracle(F):
    nb = 2000
    A = _spec(nb, 3)
    r, z = _candidates(nb)
    m = 108
    spec = torch.from_numpy(A).cuda()
    rt = torch.from_numpy(r).cuda()
    zt = torch.from_numpy(z).cuda()
    n = len(r)
    P = torch.empty(n, dtype=torch.float64, device="cuda")
    gr = torch.empty_like(P)
    gz = torch.empty_like(P)
    S = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    F.fdas_refine_fwd(spec, nb, rt, zt, n, m, P, gr, gz, S)
    P, gr, gz, S = (x.cpu().numpy() for x in (P, gr, gz, S))
    A64 = A.astype(np.complex128)
    for i in range(n):
        Po, gro, gzo, So = O.refine_power(A64, r[i], z[i], m)
        assert abs(P[i] - Po) < 1e-9 * (1 + Po), (i, P[i], Po)
        assert abs(gr[i] - gro) < 1e-8 * (1 + abs(gro)), (i, gr[i], gro)
        assert abs(gz[i] - gzo) < 1e-8 * (1 + abs(gzo)), (i, gz[i], gzo)
        assert abs(S[2 * i] + 1j * S[2 * i + 1] - So) < 1e-9 * (1 + abs(So))


def test_refine_gradients_match_finite_differences_of_gpu_forward(F):
    nb = 2000
    A = _spec(nb, 4)
    r, z = _candidates(nb)
    spec = torch.from_numpy(A).cuda()
    m = 60
    h = 1e-4
    n = len(r)

    def fwd(rr, zz):
        P = torch.empty(n, dtype=torch.float64, device="cuda")
        gr = torch.empty_like(P)
        gz = torch.empty_like(P)
        F.fdas_refine_fwd(spec, nb, torch.from_numpy(rr).cuda(), torch.from_numpy(zz).cuda(), n, m,
                          P, gr, gz)
        return P.cpu().numpy(), gr.cpu().numpy(), gz.cpu().numpy()

    P, gr, gz = fwd(r, z)
    # central differences that stay inside one tap window ([r] fixed)
    ok = np.abs((r + h) - np.floor(r + 0.5) - 0.5) > 2 * h
    fr = (fwd(r + h, z)[0] - fwd(r - h, z)[0]) / (2 * h)
    fz = (fwd(r, z + h)[0] - fwd(r, z - h)[0]) / (2 * h)
    assert np.all(np.abs(fr - gr)[ok] < 1e-4 * (1 + np.abs(gr[ok])))
    assert np.all(np.abs(fz - gz) < 1e-4 * (1 + np.abs(gz)))


def test_refine_autograd_spectrum_gradient(F):
    from paper_1804_05335_gb300.refine import refine_power
    nb = 2000
    A = _spec(nb, 5)
    r, z = _candidates(nb)
    m = 40
    spec = torch.from_numpy(A).cuda().requires_grad_(True)
    rt = torch.from_numpy(r).cuda().requires_grad_(True)
    zt = torch.from_numpy(z).cuda().requires_grad_(True)
    w = torch.linspace(0.5, 1.5, len(r), dtype=torch.float64, device="cuda")
    P = refine_power(spec, rt, zt, m)
    (P * w).sum().backward()
    g = spec.grad.cpu().numpy().astype(np.complex128)
    ref = np.zeros(nb, np.complex128)
    A64 = A.astype(np.complex128)
    for i in range(len(r)):
        k, gk = O.refine_grad_spec(A64, r[i], z[i], m)
        ref[k] += w[i].item() * gk
    assert np.abs(g - ref).max() < 2e-5 * (1 + np.abs(ref).max())
    for i in range(len(r)):
        _, gro, gzo, _ = O.refine_power(A64, r[i], z[i], m)
        assert abs(rt.grad[i].item() - w[i].item() * gro) < 1e-7 * (1 + abs(gro))
        assert abs(zt.grad[i].item() - w[i].item() * gzo) < 1e-7 * (1 + abs(gzo))


def test_refine_ascent_recovers_injections(F):
    from paper_1804_05335_gb300.refine import refine
    n = 1 << 17
    truths = ((7000.37, 33.2, 20.0), (21000.71, -48.6, 18.0), (40000.05, 0.4, 16.0),
              (9000.5, -180.7, 20.0))
    x = synth.make_series(n, truths, 41)
    A = O.normalise(O.real_spectrum(x), 1024).astype(np.complex64)
    spec = torch.from_numpy(A).cuda()
    r0 = np.array([round(2 * t[0]) / 2 for t in truths])          # nearest half bin
    z0 = np.array([2 * round(t[1] / 2) for t in truths])           # nearest grid z (step 2)
    r, z, P = refine(spec, torch.from_numpy(r0).cuda(), torch.from_numpy(z0).cuda(), zmax=200,
                     steps=20)
    r, z, P = r.cpu().numpy(), z.cpu().numpy(), P.cpu().numpy()
    m = O.half_width(200)
    for i, (rt, zt, snr) in enumerate(truths):
        assert abs(r[i] - rt) < 0.05 and abs(z[i] - zt) < 1.0, (i, r[i], z[i], rt, zt)
    # same trajectory as the FP64 oracle's ascent on two of them
    for i in (0, 2):
        ro, zo, Po = O.refine_ascent(A.astype(np.complex128), r0[i], z0[i], m, steps=20)
        assert abs(r[i] - ro) < 1e-6 and abs(z[i] - zo) < 1e-5 and abs(P[i] - Po) < 1e-6 * Po

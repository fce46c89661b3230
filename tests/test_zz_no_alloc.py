"""fdas_normalise_noalloc: the entry point for callers that must not allocate
device memory when they call (for example a real-time pipeline that reserves
all of its memory at start-up).  It must give what fdas_normalise gives with
a caller workspace, call after call, although every call reuses the one
fixed workspace inside the library.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_normalise_matches_workspace_version_twice():
    """The same kernels on the same input with another workspace address:
    the spectra must be bit-identical, call after call.  Large, small, then
    large again: a stale value left in the shared array by the larger call
    would show in the smaller one, and the reverse."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_05335_gb300 as F
    F.load_library()
    cases = [(F.FDAS_NOALLOC_MAX_N, 1024, 11), (1 << 15, 512, 12), (F.FDAS_NOALLOC_MAX_N, 1024, 13)]
    for n, block, seed in cases:
        x = synth.make_series(n, ((n / 9 + 0.4, 8.0, 18.0),), seed)
        series = torch.from_numpy(x).cuda()
        ws = F.fdas_normalise_workspace_bytes(n)
        work = torch.empty(ws, dtype=torch.uint8, device="cuda")
        ref = torch.empty(n // 2, dtype=torch.complex64, device="cuda")
        got = torch.full((n // 2,), complex(7.0, 7.0), dtype=torch.complex64, device="cuda")
        F.fdas_normalise(series, n, block, ref, work, ws)
        F.fdas_normalise_noalloc(series, n, block, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (n, (got - ref).abs().max().item())
        assert got[0].item() == 0


def test_noalloc_rejects_sizes_above_its_limit_and_other_lengths():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_05335_gb300 as F
    n = 2 * F.FDAS_NOALLOC_MAX_N
    series = torch.zeros(n, dtype=torch.float32, device="cuda")
    spec = torch.zeros(n // 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FdasError) as e:
        F.fdas_normalise_noalloc(series, n, 1024, spec)
    assert e.value.code == F.FDAS_E_UNSUPPORTED
    # lengths that are not powers of two need Bluestein's larger workspace
    with pytest.raises(F.FdasError) as e:
        F.fdas_normalise_noalloc(series, 100000, 1024, spec)
    assert e.value.code == F.FDAS_E_UNSUPPORTED

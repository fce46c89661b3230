"""Search.stream (input copies overlapped with the previous search) gives,
for every series, exactly the candidate list of a plain step on that series."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_stream_equals_steps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_05335_gb300 as F
    from paper_1804_05335_gb300.search import Search
    F.load_library()
    n = 1 << 16
    S = Search(n, 1024, 64, -20, 20, 2, thr=8.0, cap=4096)
    xs = [synth.make_series(n, ((n / 5 + 0.3 * i, 4.0 * i - 6.0, 18.0),), 300 + i)
          for i in range(5)]
    host = [torch.from_numpy(x).pin_memory() for x in xs]
    outs = [torch.full((1 + 4 * S.cap,), -1, dtype=torch.int32).pin_memory() for _ in xs]
    S.stream(host, outs)
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        S.series.copy_(torch.from_numpy(x))
        S.step()
        r, c, p, fl, total = S.candidates()
        k = int(outs[i][0])
        assert k == total and total > 0
        a = outs[i][1:1 + 4 * k].view(k, 4).numpy()
        o = np.lexsort((a[:, 1], a[:, 0]))
        a = a[o]
        assert np.array_equal(a[:, 0], r) and np.array_equal(a[:, 1], c)
        assert np.array_equal(a[:, 2].copy().view(np.float32), p)

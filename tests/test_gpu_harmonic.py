"""fdas_harmonic_sum against the oracle's harmonic sums on the same plane
values (FP32 and 16-bit planes): identical candidate lists except sums within
a relative 1e-5 of a threshold (FP32 against FP64 summation)."""
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


def _run(F, p, plane_dev, ptype, width, stride, thr, cap=1 << 16):
    out = torch.zeros(4 * cap, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    F.fdas_harmonic_sum(p, ptype, plane_dev, width, stride, thr, out, cap, count, status)
    k = int(count.item())
    a = out[: 4 * min(k, cap)].view(-1, 4).cpu().numpy()
    return a, k, int(status.item())


def _compare(a, ref, thr):
    rr, cc, ss, hh = ref
    got = {(int(h), int(r), int(c)): float(np.frombuffer(np.int32(v).tobytes(), np.float32)[0])
           for r, c, v, h in a}
    exp = {(int(h), int(r), int(c)): float(s) for r, c, s, h in zip(rr, cc, ss, hh)}
    lev = {2: 0, 4: 1, 8: 2}
    for key in set(got) ^ set(exp):
        v = got.get(key, exp.get(key))
        t = thr[lev[key[0]]]
        assert abs(v - t) <= 1e-5 * t, ("lists differ at", key, v)
    for key in set(got) & set(exp):
        assert abs(got[key] - exp[key]) <= 1e-5 * exp[key], key


# Row strides with rows on and off 16-byte boundaries.
@pytest.mark.parametrize("ptype,stride", [(0, 20002), (0, 20004), (1, 20004), (1, 20008),
                                          (2, 20004), (2, 20008)],
                         ids=["f32-odd", "f32-aligned", "f16-odd", "f16-aligned", "bf16-odd",
                              "bf16-aligned"])
def test_harmonic_sum_matches_oracle_on_random_plane(F, ptype, stride):
    p = F.params(2048, 256, -40, 40, 2, 1)
    K = F.fdas_num_templates(p)
    width = 20002
    rng = np.random.default_rng(60 + ptype)
    P = rng.exponential(1.0, (K, width)).astype(np.float32)
    P[20, 300] = P[30, 600] = 25.0          # a planted fundamental (z = 0, col 300) at H = 2
    dt = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}[ptype]
    dev = torch.zeros((K, stride), dtype=dt, device="cuda")
    dev[:, :width] = torch.from_numpy(P).to(dt)
    Pq = dev[:, :width].float().cpu().numpy().astype(np.float64)   # the values the kernel reads
    thr = [14.0, 22.0, 36.0]
    a, k, st = _run(F, p, dev, ptype, width, stride, thr)
    assert st == 0 and k == len(a) and k > 0
    _compare(a, O.harmonic_candidates(Pq, -40, 2, thr), thr)
    assert any(int(h) == 2 and int(r) == 20 and int(c) == 300 for r, c, v, h in a)


def test_harmonic_sum_on_a_searched_plane_finds_the_fundamental(F):
    from paper_1804_05335_gb300.search import Search
    n, r0, z0 = 1 << 16, 2000.0, 6.0
    x = synth.make_series(n, tuple((h * r0, h * z0, 7.0) for h in range(1, 5)), 61)
    S = Search(n, 2048, 256, -40, 40, 2)
    S.series.copy_(torch.from_numpy(x))
    S.step()
    thr = [30.0, 50.0]
    a, k, st = _run(F, S.p, S.plane, 0, S.width, S.row_stride, thr)
    assert st == 0
    P = S.plane2d().cpu().numpy().astype(np.float64)
    _compare(a, O.harmonic_candidates(P, -40, 2, thr), thr)
    best = max((v for r, c, v, h in a if int(h) == 4), key=lambda v: np.int32(v).view(np.float32),
               default=None)
    assert best is not None
    top = [(int(r), int(c)) for r, c, v, h in a if int(h) == 4 and v == best][0]
    assert top[0] == int((z0 + 40) // 2) and abs(top[1] / 2.0 - r0) <= 0.5


def test_harmonic_sum_overflow_keeps_the_count(F):
    p = F.params(2048, 256, -20, 20, 2, 1)
    K = F.fdas_num_templates(p)
    P = torch.full((K, 4000), 10.0, dtype=torch.float32, device="cuda")
    a, k, st = _run(F, p, P, 0, 4000, 4000, [5.0], cap=16)
    assert k > 16 and len(a) == 16 and (st & 2)


@pytest.mark.parametrize("zmin,zmax,zstep,width,ptype", [
    (-40, 40, 2, 4002, 0),      # symmetric grid with a z = 0 row
    (-10, 50, 2, 4001, 0),      # asymmetric grid, odd width
    (10, 100, 2, 3000, 1),      # no z = 0 row, 16-bit plane
    (-200, 200, 1, 3001, 0),    # 401 rows at zstep 1
    (-200, 200, 1, 3001, 2),    # the same, bfloat16
    (-600, 600, 1, 1000, 0),    # 1201 rows
    (-40, 40, 2, 60002, 0),     # many column blocks per row
    (-10, 50, 2, 60001, 1),     # the same, asymmetric grid, binary16
    (10, 100, 2, 120000, 2),    # the same without a z = 0 row, bfloat16
])
def test_harmonic_sum_lists_every_fundamental_once(F, zmin, zmax, zstep, width, ptype):
    """With thresholds below every sum, each (fundamental, level) is listed
    exactly once, with the oracle's sum."""
    p = F.params(4096, 1024, zmin, zmax, zstep, 1)
    K = F.fdas_num_templates(p)
    stride = (width + 7) // 8 * 8
    rng = np.random.default_rng(K + width)
    P = rng.exponential(1.0, (K, width)).astype(np.float32)
    dt = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}[ptype]
    dev = torch.zeros((K, stride), dtype=dt, device="cuda")
    dev[:, :width] = torch.from_numpy(P).to(dt)
    Pq = dev[:, :width].float().cpu().numpy().astype(np.float64)
    thr = [-1.0, -1.0, -1.0]
    ref = O.harmonic_candidates(Pq, zmin, zstep, thr)
    a, k, st = _run(F, p, dev, ptype, width, stride, thr, cap=len(ref[0]) + 16)
    assert st == 0 and k == len(a) == len(ref[0])
    keys = {(int(h), int(r), int(c)) for r, c, v, h in a}
    assert len(keys) == k                                   # no fundamental twice
    _compare(a, ref, thr)


def _planned(F, p, plane_dev, ptype, width, stride, thr, plan, nbytes, cap=1 << 20):
    out = torch.zeros(4 * cap, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    F.fdas_harmonic_sum_planned(p, ptype, plane_dev, width, stride, thr, out, cap, count, plan,
                                nbytes, status)
    k = int(count.item())
    return out[: 4 * min(k, cap)].view(-1, 4).cpu().numpy(), k, int(status.item())


@pytest.mark.parametrize("zmin,zmax,zstep,width,stride,ptype", [
    (-40, 40, 2, 60002, 60008, 0),      # z = 0 row first, then ray order
    (-10, 50, 2, 60001, 60008, 1),      # asymmetric grid, binary16
    (10, 100, 2, 120000, 120000, 2),    # no z = 0 row, bfloat16
    (-200, 200, 2, 20002, 20004, 0),    # the production grid on a short plane
])
def test_planned_harmonic_sum_equals_the_unplanned_one(F, zmin, zmax, zstep, width, stride,
                                                       ptype):
    """The ray-ordered launch lists exactly the candidates of the row-major
    one, with bit-identical sums (same arithmetic, other block order)."""
    p = F.params(4096, 1024, zmin, zmax, zstep, 1)
    K = F.fdas_num_templates(p)
    rng = np.random.default_rng(K + width + ptype)
    P = rng.exponential(1.0, (K, width)).astype(np.float32)
    dt = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}[ptype]
    dev = torch.zeros((K, stride), dtype=dt, device="cuda")
    dev[:, :width] = torch.from_numpy(P).to(dt)
    thr = [7.0, 11.0, 17.0]
    nbytes = F.fdas_harmonic_plan_bytes(p, width)
    plan = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    F.fdas_harmonic_plan(p, width, plan, nbytes)
    a, k, st = _run(F, p, dev, ptype, width, stride, thr, cap=1 << 20)
    b, kb, stb = _planned(F, p, dev, ptype, width, stride, thr, plan, nbytes)
    assert st == 0 and stb == 0 and k == kb and k > 0
    key = lambda x: sorted(map(tuple, x.tolist()))
    assert key(a) == key(b)


def test_planned_harmonic_sum_rejects_a_plan_for_another_width(F):
    p = F.params(2048, 256, -40, 40, 2, 1)
    K = F.fdas_num_templates(p)
    dev = torch.full((K, 8000), 10.0, dtype=torch.float32, device="cuda")
    n1, n2 = F.fdas_harmonic_plan_bytes(p, 4000), F.fdas_harmonic_plan_bytes(p, 8000)
    plan = torch.empty(max(n1, n2), dtype=torch.uint8, device="cuda")
    F.fdas_harmonic_plan(p, 4000, plan, n1)
    b, k, st = _planned(F, p, dev, 0, 8000, 8000, [5.0], plan, max(n1, n2))
    assert k == 0 and (st & F.FDAS_STATUS_BADPLAN)


@pytest.mark.parametrize("width", [1, 2, 3, 5])
def test_harmonic_sum_on_degenerate_widths(F, width):
    """Planes one to five columns wide: every listed sum is the oracle's, and
    the planned launch lists the same candidates."""
    p = F.params(2048, 256, -20, 20, 2, 1)
    K = F.fdas_num_templates(p)
    rng = np.random.default_rng(width)
    P = rng.exponential(1.0, (K, width)).astype(np.float32)
    stride = 8
    dev = torch.zeros((K, stride), dtype=torch.float32, device="cuda")
    dev[:, :width] = torch.from_numpy(P)
    thr = [-1.0, -1.0, -1.0]
    ref = O.harmonic_candidates(dev[:, :width].cpu().numpy().astype(np.float64), -20, 2, thr)
    a, k, st = _run(F, p, dev, 0, width, stride, thr)
    assert st == 0 and k == len(ref[0])
    _compare(a, ref, thr)
    nbytes = F.fdas_harmonic_plan_bytes(p, width)
    plan = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    F.fdas_harmonic_plan(p, width, plan, nbytes)
    b, kb, stb = _planned(F, p, dev, 0, width, stride, thr, plan, nbytes)
    assert stb == 0 and kb == k
    assert sorted(map(tuple, a.tolist())) == sorted(map(tuple, b.tolist()))

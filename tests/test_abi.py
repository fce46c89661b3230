"""CPU checks of the C-ABI library: it loads, exports what include/fdas.h
declares, and its host-side bookkeeping and argument validation behave.

No call here launches GPU work: every compute entry point is called only with
arguments that its validation rejects before anything reaches CUDA.
"""
import ctypes

import numpy as np
import pytest

import paper_1804_05335_gb300 as F


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1804_05335_gb300 import build
    build.build()
    F.load_library()


def test_library_exports_every_declared_function():
    lib = ctypes.CDLL(F.lib_path())
    names = F.header_functions()
    assert "fdas_correlate" in names and "fdas_make_templates" in names
    for n in ("fdas_normalise", "fdas_threshold"):
        assert n in names
    for n in names:
        assert hasattr(lib, n), n


def test_host_helpers():
    p = F.params(2048, 256, -200, 200, 2, 1)
    assert F.fdas_num_templates(p) == 201
    assert F.fdas_bank_rows(p) == 101
    assert F.fdas_bank_floats(p) == 101 * (2048 + 16) * 2
    assert F.fdas_num_segments(p, 1 << 22) == -(-(1 << 22) // 1792)
    assert F.fdas_plane_width(p, 1 << 22) == 1 << 23
    assert F.fdas_plane_width(F.params(2048, 256, -200, 200, 2, 0), 1000) == 1000
    assert F.fdas_bank_rows(F.params(2048, 64, -21, 21, 2, 1)) == 11       # no z = 0
    assert F.fdas_bank_rows(F.params(2048, 64, -10, 20, 2, 1)) == 16       # asymmetric: all rows
    assert [F.fdas_half_width(z) for z in (0, 1, -21, 200)] == [8, 9, 19, 108]
    assert F.fdas_normalise_workspace_bytes(1 << 23) == (1 << 22) * 8
    assert F.fdas_normalise_workspace_bytes(1000) == 0
    # even lengths that are not powers of two: three buffers of the convolution
    # length P >= n - 1, the least of the form 2^m or 3 * 2^m (m <= 22)
    assert F.fdas_normalise_workspace_bytes(100000) == 3 * (1 << 17) * 8
    assert F.fdas_normalise_workspace_bytes(8194) == 3 * (3 << 12) * 8
    assert F.fdas_normalise_workspace_bytes(1048578) == 3 * (3 << 19) * 8
    assert F.fdas_normalise_workspace_bytes(12290) == 3 * (1 << 14) * 8   # 12289 > 3 * 2^12
    assert F.fdas_normalise_workspace_bytes((1 << 24) - 2) == 3 * (1 << 24) * 8
    assert F.fdas_normalise_workspace_bytes(100001) == 0          # odd
    assert F.fdas_normalise_workspace_bytes((1 << 24) + 2) == 0   # past the largest convolution
    # Bluestein kernel spectrum: P complex values for non-power-of-two lengths only
    assert F.fdas_bluestein_bytes(100000) == (1 << 17) * 8
    assert F.fdas_bluestein_bytes(8194) == (3 << 12) * 8
    assert F.fdas_bluestein_bytes(6291458) == (1 << 23) * 8             # 3 * 2^21 < n - 1
    assert F.fdas_bluestein_bytes(6291456) == (3 << 21) * 8
    assert F.fdas_bluestein_bytes((1 << 24) - 2) == (1 << 24) * 8
    assert F.fdas_bluestein_bytes(1 << 20) == 0
    assert F.fdas_bluestein_bytes(100001) == 0
    assert F.fdas_bluestein_bytes((1 << 24) + 2) == 0
    assert F.fdas_strerror(F.FDAS_E_INVAL) == "invalid argument"


@pytest.mark.parametrize("bad", [
    dict(L=512), dict(L=3000), dict(M=60), dict(M=66), dict(M=4096),
    dict(zstep=0), dict(zmin=10, zmax=-10), dict(zmin=-5, zmax=6, zstep=2),
    dict(interbin=3), dict(zmin=-300, zmax=300, M=256),          # h(300) = 158 > 127
    dict(interbin=2, M=256),                                     # 4 h(200) + 2 = 434 > 256
])
def test_invalid_params_rejected(bad):
    kw = dict(L=2048, M=256, zmin=-200, zmax=200, zstep=2, interbin=1)
    kw.update(bad)
    p = F.params(**kw)
    with pytest.raises(F.FdasError) as e:
        F.fdas_num_templates(p)
    assert e.value.code == F.FDAS_E_INVAL
    with pytest.raises(F.FdasError) as e:
        F.fdas_correlate(p, 256, 1000, 256, 256, 2000, stream=0)
    assert e.value.code == F.FDAS_E_INVAL


def test_invalid_buffers_rejected_before_launch():
    p = F.params(2048, 256, -200, 200, 2, 1)
    cases = [
        lambda: F.fdas_correlate(p, 0, 1000, 256, 256, 2000, stream=0),       # NULL spec
        lambda: F.fdas_correlate(p, 256, 1000, 264, 256, 2000, stream=0),     # bank not 16-aligned
        lambda: F.fdas_correlate(p, 256, 1000, 256, 256, 1998, stream=0),     # stride < width
        lambda: F.fdas_correlate(p, 256, 1000, 256, 256, 2002, stream=0),     # stride % 4
        lambda: F.fdas_correlate(p, 256, 0, 256, 256, 2000, stream=0),        # nb < 1
        lambda: F.fdas_make_templates(p, 0, stream=0),
        lambda: F.fdas_make_templates(p, 8, stream=0),
        lambda: F.fdas_normalise(256, 1000, 1024, 256, 256, 1 << 20, stream=0),    # n too small
        lambda: F.fdas_normalise(256, 100001, 1024, 256, 256, 1 << 24, stream=0),  # n odd
        lambda: F.fdas_normalise(256, 100000, 1024, 256, 256, 1 << 20, stream=0),  # work size
        lambda: F.fdas_normalise(256, 1 << 14, 16, 256, 256, 1 << 20, stream=0),   # block
        lambda: F.fdas_normalise(256, 1 << 14, 1024, 256, 256, 100, stream=0),     # work size
        lambda: F.fdas_bluestein_prepare(1 << 20, 256, 256, 1 << 24, stream=0),    # power of two
        lambda: F.fdas_bluestein_prepare(100000, 0, 256, 1 << 24, stream=0),       # NULL spectrum
        lambda: F.fdas_bluestein_prepare(100000, 264, 256, 1 << 24, stream=0),     # misaligned
        lambda: F.fdas_bluestein_prepare(100000, 256, 256, 1 << 20, stream=0),     # work size
        lambda: F.fdas_normalise_prepared(256, 100000, 1024, 256, 256, 1 << 24, 0,
                                          stream=0),                               # no spectrum
        lambda: F.fdas_normalise_prepared(256, 100000, 1024, 256, 256, 1 << 24, 264,
                                          stream=0),                               # misaligned
        lambda: F.fdas_normalise_prepared(256, 100000, 1024, 256, 256, 1 << 20, 256,
                                          stream=0),                               # work size
        lambda: F.fdas_threshold(256, 0, 10, 10, 20.0, 0, 256, 4, 256, stream=0),  # rows
        lambda: F.fdas_threshold(256, 3, 10, 9, 20.0, 0, 256, 4, 256, stream=0),   # stride
        lambda: F.fdas_threshold(256, 3, 10, 10, 20.0, 4, 256, 4, 256, stream=0),  # flags
        lambda: F.fdas_correlate_split(p, 4, 256, 1000, 256, 256, 2000, stream=0),    # prec
        lambda: F.fdas_correlate_split(p, -1, 256, 1000, 256, 256, 2000, stream=0),   # prec
        lambda: F.fdas_correlate_split(p, 1, 0, 1000, 256, 256, 2000, stream=0),      # NULL spec
        lambda: F.fdas_correlate_split(p, 2, 256, 1000, 256, 256, 2002, stream=0),    # stride % 4
        lambda: F.fdas_correlate_split(F.params(L=512), 1, 256, 1000, 256, 256, 2000,
                                       stream=0),                                     # L
        lambda: F.fdas_correlate_plane16(p, 0, 256, 1000, 256, 256, 2000, stream=0),  # type
        lambda: F.fdas_correlate_plane16(p, 3, 256, 1000, 256, 256, 2000, stream=0),  # type
        lambda: F.fdas_correlate_plane16(p, 1, 256, 1000, 256, 0, 2000, stream=0),    # NULL plane
        lambda: F.fdas_correlate_plane16(p, 2, 256, 1000, 256, 264, 2000, stream=0),  # plane align
        lambda: F.fdas_correlate_plane16(p, 1, 256, 1000, 256, 256, 2002, stream=0),  # stride % 4
    ]
    for f in cases:
        with pytest.raises(F.FdasError) as e:
            f()
        assert e.value.code == F.FDAS_E_INVAL


def _slot(k, L):
    """Bank storage slot of frequency k, restated from the layout in fdas.h."""
    Q, T = L // 256, L // 16
    a, k1, c2 = k % 16, (k // 16) % 16, k // 256
    c1, s2 = k1 % Q, k1 // Q
    t, i = a * Q + c1, s2 * Q + c2
    return 2 * ((i // 2) * T + t) + (i % 2)


@pytest.mark.parametrize("L", [1024, 2048, 4096])
def test_bank_layout_is_a_permutation(L):
    s = np.array([_slot(k, L) for k in range(L)])
    assert sorted(s) == list(range(L))


def _needed_overlap(z):
    """Overlap a template needs, as fdas.h states it: >= 2h + 2, multiple of 4, >= 64."""
    h = F.fdas_half_width(z)
    return max(64, -(-(2 * h + 2) // 4) * 4)


@pytest.mark.parametrize("L,M,zmax,zstep", [(2048, 256, 200, 2), (2048, 128, 58, 2),
                                            (1024, 64, 20, 2), (4096, 256, 201, 3)])
def test_template_groups_cover_the_grid_and_minimise_work(L, M, zmax, zstep):
    import itertools
    p = F.params(L, M, -zmax, zmax, zstep, 1)
    groups = F.fdas_template_groups(p)
    K, Kb = F.fdas_num_templates(p), F.fdas_bank_rows(p)
    j0 = K - Kb
    zb = [-zmax + (j0 + b) * zstep for b in range(Kb)]
    zero = zb[0] == 0
    assert 1 <= len(groups) <= F.FDAS_MAX_GROUPS
    assert sum(c for _, _, c in groups) == K
    firsts = [f for _, f, _ in groups] + [Kb]
    assert firsts[0] == 0 and all(a < b for a, b in zip(firsts, firsts[1:]))

    def rows(lo, hi):
        return 2 * (hi - lo) - (1 if zero and lo == 0 else 0)

    for k, (ov, f, c) in enumerate(groups):
        assert c == rows(f, firsts[k + 1])
        assert ov == max(_needed_overlap(z) for z in zb[f:firsts[k + 1]]) and ov <= M
    work = sum((c + 0.5) / (L - ov) for ov, _, c in groups)
    # brute force over every split of the bank rows into at most 4 runs
    best = float("inf")
    for n in range(1, F.FDAS_MAX_GROUPS + 1):
        for cut in itertools.combinations(range(1, Kb), n - 1):
            ends = (0,) + cut + (Kb,)
            w = sum((rows(a, b) + 0.5) / (L - _needed_overlap(zb[b - 1]))
                    for a, b in zip(ends, ends[1:]))
            best = min(best, w)
    assert work <= best * (1 + 1e-12)


def test_template_groups_one_group_off_symmetric_grids():
    p = F.params(2048, 128, -10, 30, 5, 1)
    assert F.fdas_template_groups(p) == [(128, 0, F.fdas_num_templates(p))]


def test_interp2_grid_and_split_rejection():
    p = F.params(2048, 436, -200, 200, 2, 2)           # 4 h(200) + 2 = 434 <= 436
    assert F.fdas_num_templates(p) == 201
    assert F.fdas_bank_rows(p) == 201                   # no +-z pairing at half-bin taps
    assert F.fdas_plane_width(p, 1 << 22) == 1 << 23
    assert F.fdas_num_segments(p, 1 << 22) == -(-(1 << 23) // (2048 - 436))
    assert F.fdas_template_groups(p) == [(436, 0, 201)]
    with pytest.raises(F.FdasError) as e:
        F.fdas_correlate_split(p, 1, 256, 1000, 256, 256, 2000, stream=0)
    assert e.value.code == F.FDAS_E_UNSUPPORTED
    with pytest.raises(F.FdasError) as e:                # no 16-bit plane at half bins
        F.fdas_correlate_plane16(p, 1, 256, 1000, 256, 256, 2000, stream=0)
    assert e.value.code == F.FDAS_E_UNSUPPORTED


def test_harmonic_sum_rejects_bad_arguments_before_launch():
    p = F.params(2048, 256, -200, 200, 2, 1)
    cases = [
        lambda: F.fdas_harmonic_sum(p, 3, 256, 1000, 1000, [20.0], 256, 4, 256, stream=0),     # type
        lambda: F.fdas_harmonic_sum(p, 0, 0, 1000, 1000, [20.0], 256, 4, 256, stream=0),       # NULL plane
        lambda: F.fdas_harmonic_sum(p, 0, 256, 1000, 999, [20.0], 256, 4, 256, stream=0),      # stride
        lambda: F.fdas_harmonic_sum(p, 0, 256, 1000, 1000, [], 256, 4, 256, stream=0),         # no level
        lambda: F.fdas_harmonic_sum(p, 0, 256, 1000, 1000, [1.0] * 4, 256, 4, 256, stream=0),  # 4 levels
        lambda: F.fdas_harmonic_sum(F.params(2048, 256, -21, 21, 2, 1), 0, 256, 1000, 1000,
                                    [20.0], 256, 4, 256, stream=0),                            # zmin % zstep
    ]
    for f in cases:
        with pytest.raises((F.FdasError, ValueError, IndexError)) as e:
            f()
        if isinstance(e.value, F.FdasError):
            assert e.value.code == F.FDAS_E_INVAL


def test_harmonic_plan_sizes_and_validation():
    p = F.params(2048, 256, -200, 200, 2, 1)
    # 101 fundamental rows (second harmonic on the plane) x 4096 blocks of 1024 columns
    assert F.fdas_harmonic_plan_bytes(p, 1 << 23) == 64 + 8 * 101 * 4096
    assert F.fdas_harmonic_plan_bytes(p, 1000) == (64 + 8 * 101 + 15) // 16 * 16
    assert F.fdas_harmonic_plan_bytes(p, 0) == 0
    bad = F.params(2048, 256, -201, 199, 2, 1)            # zmin not a multiple of zstep
    assert F.fdas_harmonic_plan_bytes(bad, 1000) == 0
    need = F.fdas_harmonic_plan_bytes(p, 1000)
    for args in [(p, 1000, 0, need), (p, 1000, 264, need), (p, 1000, 256, need - 16),
                 (bad, 1000, 256, need)]:
        with pytest.raises(F.FdasError) as e:
            F.fdas_harmonic_plan(*args)
        assert e.value.code == F.FDAS_E_INVAL
    for plan, nbytes in [(0, need), (264, need), (256, need - 16)]:   # NULL, unaligned, short
        with pytest.raises(F.FdasError) as e:
            F.fdas_harmonic_sum_planned(p, 0, 256, 1000, 1000, [20.0], 256, 4, 256, plan,
                                        nbytes, stream=0)
        assert e.value.code == F.FDAS_E_INVAL

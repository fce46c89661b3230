"""Power error of the three convolver forms (FP32, FP16 hi+lo and BF16 hi+lo
tensor-core DFT passes) against the FP64 oracle, printed as one JSON line.

    python tests/report_split_error.py [--configs small,production]

small: the 2^17-sample series (21 templates, L = 2048), whole plane.
production: the 2^23-sample series (201 templates, M = 256) at L = 1024,
2048 and 4096, on 18 windows of 256 bins (8 random, both ends, and the 8
injections), all 201 rows.  Also reports the fused candidate lists of the
split forms against the FP32 form's.  Needs a CUDA device.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle.fdas_oracle as O  # noqa: E402
import synth  # noqa: E402

FORMS = (("fp32", 0), ("fp16_split", 1), ("bf16_split", 2))


def stats(err, ref):
    big = ref > 20.0
    return {"max_abs": float(err.max()), "rms": float(np.sqrt(np.mean(err ** 2))),
            "max_rel_above_20": float((err[big] / ref[big]).max()) if big.any() else None,
            "points": int(err.size)}


def small(torch):
    from paper_1804_05335_gb300.search import Search
    wl = synth.workload("small")
    x = wl.series()
    A = O.normalise(O.real_spectrum(x), wl.median_block).astype(np.complex64)
    ref = O.plane(A.astype(np.complex128), O.z_grid(wl.zmin, wl.zmax, wl.zstep))
    S = Search(n=wl.n, L=wl.L, M=wl.M, zmin=wl.zmin, zmax=wl.zmax, zstep=wl.zstep,
               thr=wl.threshold)
    S.spec.copy_(torch.from_numpy(A))
    S.make_templates()
    out = {}
    for name, prec in FORMS:
        S.correlate(fused=False, prec=prec)
        got = S.plane2d().cpu().numpy().astype(np.float64)
        out[name] = stats(np.abs(got - ref), ref)
    return {"workload": "small, L=%d, whole plane %dx%d" % (wl.L, S.K, S.width), "forms": out}


def production(torch, L):
    from paper_1804_05335_gb300.search import Search
    wl = synth.workload("production")
    x = wl.series()
    A = O.normalise(O.real_spectrum(x), wl.median_block).astype(np.complex64)
    A64 = A.astype(np.complex128)
    zs = O.z_grid(wl.zmin, wl.zmax, wl.zstep)
    rng = np.random.default_rng(L)
    starts = list(rng.integers(0, wl.nb - 256, 8)) + [0, wl.nb - 256]
    starts += [int(r0) - 128 for r0, _, _ in wl.injections]
    refs = [O.plane_window(A64, zs, r0, 256) for r0 in starts]
    S = Search(n=wl.n, L=L, M=wl.M, zmin=wl.zmin, zmax=wl.zmax, zstep=wl.zstep,
               thr=wl.threshold, cap=1 << 16)
    S.spec.copy_(torch.from_numpy(A))
    S.make_templates()
    out, lists = {}, {}
    for name, prec in FORMS:
        S.status.zero_()
        S.correlate(fused=True, prec=prec)
        r, c, p, _, tot = S.candidates()
        lists[name] = {(int(a), int(b)) for a, b in zip(r, c)}
        plane = S.plane2d()
        errs, rv = [], []
        for r0, ref in zip(starts, refs):
            got = plane[:, 2 * r0: 2 * (r0 + 256)].cpu().numpy().astype(np.float64)
            errs.append(np.abs(got - ref).ravel())
            rv.append(ref.ravel())
        out[name] = stats(np.concatenate(errs), np.concatenate(rv))
        out[name]["candidates"] = int(tot)
        if name != "fp32":
            out[name]["candidates_only_here"] = len(lists[name] - lists["fp32"])
            out[name]["candidates_only_in_fp32"] = len(lists["fp32"] - lists[name])
    return {"workload": "production, L=%d, %d windows x 256 bins x %d rows"
                        % (L, len(starts), S.K), "forms": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", default="small,production")
    args = ap.parse_args()
    import torch
    import paper_1804_05335_gb300 as F
    F.load_library()
    res = []
    cfg = args.configs.split(",")
    if "small" in cfg:
        res.append(small(torch))
    if "production" in cfg:
        for L in (1024, 2048, 4096):
            res.append(production(torch, L))
    print(json.dumps(res))


if __name__ == "__main__":
    main()

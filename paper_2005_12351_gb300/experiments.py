"""The paper's FMM and Barnes-Hut experiments (§4) as synthetic runs on the GPU.

E3 -- error distributions: per-particle relative error of the Coulomb potential
(and field) of random charges against the FP64 direct sum, for several
expansion orders p at opening angles theta = 0.25 and 0.5, n_crit = 128, for
the FMM and the multipolar Barnes-Hut.  The paper shows histograms and
cumulative distributions whose median falls as p rises, and notes that the
FMM at theta matches the Barnes-Hut at about theta / 2.

E2 -- runtime against N: log-spaced particle counts up to 10^6 for several
(theta, p), the whole path (tree, lists, evaluate) and the evaluate alone,
beside the direct sum, to show the O(N) growth of the FMM, the O(N log N) of
the Barnes-Hut walk and the breakeven N.

Inputs are seeded synthetic charges (q uniform in [-1, 1]) uniform in the
cube [-1e-9, 1e-9]^3 of the paper's tests, which also exercises the scale
invariance of the method.  Usage:

    python -m paper_2005_12351_gb300.experiments e3 [--n 50000] [--orders 1,2,...]
    python -m paper_2005_12351_gb300.experiments e2 [--nmax 1000000]

Each prints one JSON line per (theta, p) or (N, theta, p).
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import synth

SEED_E3 = 20260020
SEED_E2 = 20260021
BOX = 1e-9


def charges_in_box(n: int, seed: int):
    """n charges q ~ U[-1, 1] at positions uniform in [-BOX, BOX]^3."""
    pos, q = synth.make_system(n, 0, "uniform", seed)
    return (2.0 * pos - 1.0) * BOX, q


def _dev(x, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device)


def relative_errors(val, ref):
    """Per-particle relative error |val - ref| / |ref| (vectors: by norm)."""
    val, ref = np.asarray(val, float), np.asarray(ref, float)
    if val.ndim == 2:
        return np.linalg.norm(val - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    return np.abs(val - ref) / np.maximum(np.abs(ref), 1e-300)


def summarize(err, bins_lo=-16, bins_hi=2):
    """Median / p90 / p99 / max and a log10 histogram (one bin per decade; the end
    bins also count the errors beyond them)."""
    err = np.asarray(err, float)
    lg = np.clip(np.log10(np.maximum(err, 10.0 ** bins_lo)), bins_lo, bins_hi - 1e-9)
    hist, edges = np.histogram(lg, bins=np.arange(bins_lo, bins_hi + 1))
    return {"median": float(np.median(err)), "p90": float(np.quantile(err, 0.9)),
            "p99": float(np.quantile(err, 0.99)), "max": float(err.max()),
            "rel_rms": None,
            "log10_hist": {"edges": [int(e) for e in edges], "counts": [int(c) for c in hist]}}


def e3(n=50_000, thetas=(0.25, 0.5), orders=(1, 2, 3, 4, 5, 6, 7, 8, 9, 10), ncrit=128,
       precision="fp64", seed=SEED_E3, device=0, methods=("fmm", "bh")):
    """Yields one result dict per (method, theta, p)."""
    import torch
    from . import fmm
    dev = torch.device("cuda", device)
    pos, q = charges_in_box(n, seed)
    P, Q = _dev(pos, dev), _dev(q, dev)
    phi_d, E_d = fmm.direct_sum(P, Q, 0)
    phi_d, E_d = phi_d.cpu().numpy(), E_d.cpu().numpy()
    for theta in thetas:
        tree = fmm.create_tree(device=device, max_leaf=ncrit, precision=precision)
        tree.set_sources(P, Q, 0)
        for method in methods:
            for p in orders:
                if method == "fmm":
                    phi, E = tree.evaluate(p, theta)
                else:
                    phi, E = tree.evaluate_bh(p, theta)
                torch.cuda.synchronize(dev)
                phi, E = phi.cpu().numpy(), E.cpu().numpy()
                sp = summarize(relative_errors(phi, phi_d))
                sp["rel_rms"] = float(np.sqrt(((phi - phi_d) ** 2).sum() / (phi_d ** 2).sum()))
                sf = summarize(relative_errors(E, E_d))
                sf["rel_rms"] = float(np.sqrt(((E - E_d) ** 2).sum() / (E_d ** 2).sum()))
                yield {"experiment": "E3", "method": method, "n": n, "theta": theta, "p": p,
                       "n_crit": ncrit, "precision": precision if method == "fmm" else "fp64",
                       "potential_error": sp, "field_error": sf,
                       "reference": "FP64 direct sum on the GPU (parity-tested against the oracle)"}
        tree.destroy()


def _time(fn, reps, dev):
    import torch
    fn()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def e2(nmin=1_000, nmax=1_000_000, points=10, thetas=(0.3, 0.5, 0.7), orders=(2, 4, 6, 8),
       ncrit=128, precision="fp64", seed=SEED_E2, device=0, direct_max=200_000,
       methods=("fmm", "bh")):
    """Yields one result dict per (N, method, theta, p): ms per whole step (tree +
    lists + evaluate, or tree + Barnes-Hut walk), ms per evaluate with the tree (and
    lists) kept, and the direct sum's ms (up to direct_max particles)."""
    import torch
    from . import fmm
    dev = torch.device("cuda", device)
    for n in np.unique(np.round(np.logspace(math.log10(nmin), math.log10(nmax), points)).astype(int)):
        n = int(n)
        pos, q = charges_in_box(n, seed + n)
        P, Q = _dev(pos, dev), _dev(q, dev)
        t_direct = _time(lambda: fmm.direct_sum(P, Q, 0), 2, dev) if n <= direct_max else None
        for theta in thetas:
            tree = fmm.create_tree(device=device, max_leaf=ncrit, precision=precision)
            for method in methods:
                for p in orders:
                    ev = ((lambda: tree.evaluate(p, theta)) if method == "fmm"
                          else (lambda: tree.evaluate_bh(p, theta)))

                    def whole():
                        tree.set_sources(P, Q, 0)
                        ev()
                    reps = 3 if method == "fmm" else 1
                    t_whole = _time(whole, reps, dev)
                    t_eval = _time(ev, reps, dev)
                    yield {"experiment": "E2", "method": method, "n": n, "theta": theta, "p": p,
                           "n_crit": ncrit, "precision": precision if method == "fmm" else "fp64",
                           "ms_whole": t_whole, "ms_evaluate": t_eval, "ms_direct": t_direct,
                           "particles_per_s": n / (t_whole / 1e3)}
            tree.destroy()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("which", choices=["e2", "e3"])
    ap.add_argument("--n", type=int, default=50_000)
    ap.add_argument("--nmax", type=int, default=1_000_000)
    ap.add_argument("--orders", default=None, help="comma-separated p list")
    ap.add_argument("--thetas", default=None, help="comma-separated theta list")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "3xtf32"])
    ap.add_argument("--methods", default="fmm,bh", help="comma-separated: fmm, bh")
    args = ap.parse_args(argv)
    kw = {"precision": args.precision, "methods": tuple(args.methods.split(","))}
    if args.orders:
        kw["orders"] = tuple(int(x) for x in args.orders.split(","))
    if args.thetas:
        kw["thetas"] = tuple(float(x) for x in args.thetas.split(","))
    gen = e3(n=args.n, **kw) if args.which == "e3" else e2(nmax=args.nmax, **kw)
    for r in gen:
        print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

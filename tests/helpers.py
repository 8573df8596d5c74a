"""Shared test helpers: exact binary32 emulation and tracking-quality metrics.

None of this is tracker arithmetic: fma32 emulates one IEEE binary32 fused
multiply-add from exact rationals; evaluate() compares tracks with the
generator's truth labels.
"""
from fractions import Fraction

import numpy as np


def round32(q: Fraction) -> np.float32:
    """Correctly rounded (nearest, ties to even) binary32 value of an exact rational."""
    f = np.float32(float(q))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    best = None
    for c in cands:
        if not np.isfinite(c):
            continue
        d = abs(Fraction(float(c)) - q)
        if best is None or d < best[0] or (d == best[0] and (int(np.float32(c).view(np.uint32)) & 1) == 0):
            best = (d, c)
    return np.float32(best[1])


def fma32(a, b, c) -> np.float32:
    return round32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def evaluate(ev, tr_off, tr_clus, min_findable=70, pt_min=0.0):
    """Efficiency / clone / fake rates against generator truth.

    A track's label is the majority label of its clusters; it is fake when
    fewer than 90 % of its clusters carry that label.  A generated primary is
    findable with >= min_findable clusters; found when a non-fake track carries
    its label; cloned when more than one does."""
    lab = ev.label
    T = len(tr_off) - 1
    ntrk = ev.trk_pt.size
    cnt_true = np.bincount(lab[lab >= 0], minlength=ntrk)
    found = np.zeros(ntrk, int)
    fakes = 0
    for t in range(T):
        c = tr_clus[tr_off[t]:tr_off[t + 1]]
        v, k = np.unique(lab[c], return_counts=True)
        j = np.argmax(k)
        if v[j] < 0 or k[j] < 0.9 * len(c):
            fakes += 1
        else:
            found[v[j]] += 1
    findable = (cnt_true >= min_findable) & (ev.trk_pt >= pt_min) & (~ev.trk_looper)
    return dict(T=T, findable=int(findable.sum()),
                eff=float((found[findable] > 0).mean()) if findable.any() else float("nan"),
                clone=float((found[findable] > 1).mean()) if findable.any() else float("nan"),
                fake=fakes / max(T, 1))


def track_truth_state(ev, cl):
    """Exact generator state (y, z, sin phi, tan lambda, q/pT) at cluster cl."""
    t = ev.label[cl]
    return np.array([ev.true_y[cl], ev.true_z[cl], ev.true_snp[cl], np.sinh(ev.trk_eta[t]),
                     ev.trk_q[t] / ev.trk_pt[t]])


def is_spd(c15) -> bool:
    C = np.zeros((5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            C[i, j] = C[j, i] = c15[k]
            k += 1
    try:
        np.linalg.cholesky(C)
        return True
    except np.linalg.LinAlgError:
        return False


def golden_line_cases(path):
    """The hand-built straight-line cases of tests/golden/tracklets_b0.json as
    (case, sector, row, y, z) cluster arrays (one sector, Bz = 0, z given)."""
    import json

    import tpcgen
    X = tpcgen.row_x_f32().astype(np.float64)
    with open(path) as f:
        spec = json.load(f)
    for case in spec["cases"]:
        rows, ys, zs = [], [], []
        for part in case["parts"]:
            r = np.array([q for q in range(*part["rows"]) if q not in part.get("skip", [])])
            dx = X[r] - X[0]
            rows.append(r)
            yy = part["y0"] + part["a"] * dx
            for rr, d in part.get("displace", []):
                yy[r == rr] += d
            ys.append(yy)
            zs.append(part["z0"] + part["b"] * dx + part["dz"])
        row = np.concatenate(rows).astype(np.uint8)
        y = np.concatenate(ys)
        z = np.concatenate(zs)
        if case.get("noise_cm", 0.0) > 0:
            rng = np.random.default_rng(case["noise_seed"])
            y = y + rng.normal(0, case["noise_cm"], y.size)
            z = z + rng.normal(0, case["noise_cm"], z.size)
        yield case, np.zeros(row.size, np.uint8), row, y.astype(np.float32), z.astype(np.float32)

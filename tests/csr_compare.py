"""CSR comparison of the CUDA path against the FP64 oracle.

Structure: per row, the column sets may differ only in pairs the oracle marks
ambiguous (within +-1e-6 relative of the threshold, or within 1e-3 mm of the
lateral cutoff).  Values: max relative error over common entries <= tol.
"""
import numpy as np


def compare(gpu_rows, orc, tol=1e-4, value_of=None):
    """gpu_rows: list of (cols, vals) in the oracle's row order.  Returns stats dict;
    raises AssertionError with details on a mismatch."""
    max_rel = 0.0
    abs_sum = 0.0
    n_common = 0
    n_amb_diff = 0
    bad_struct = []
    for i, (gc, gv) in enumerate(gpu_rows):
        oc, ov = orc.row(i)
        gc = np.asarray(gc, dtype=np.int64)
        oc = np.asarray(oc, dtype=np.int64)
        assert np.all(np.diff(gc) > 0), f"row {i}: GPU columns not strictly ascending"
        common, gi, oi = np.intersect1d(gc, oc, assume_unique=True, return_indices=True)
        only_g = np.setdiff1d(gc, oc, assume_unique=True)
        only_o = np.setdiff1d(oc, gc, assume_unique=True)
        if only_g.size or only_o.size:
            amb = orc.ambiguous(i)
            for c in np.concatenate([only_g, only_o]).tolist():
                if c in amb:
                    n_amb_diff += 1
                else:
                    bad_struct.append((i, c, c in set(only_g.tolist())))
        if common.size:
            g = np.asarray(gv, dtype=np.float64)[gi]
            o = ov[oi]
            rel = np.abs(g - o) / np.abs(o)
            max_rel = max(max_rel, float(rel.max()))
            abs_sum += float(np.abs(g - o).sum())
            n_common += int(common.size)
    stats = {"max_rel": max_rel, "eps": abs_sum / max(n_common, 1), "n_common": n_common,
             "n_ambiguous_diff": n_amb_diff, "n_struct_bad": len(bad_struct)}
    assert not bad_struct, f"structure differs outside the bands: {bad_struct[:10]} (total {len(bad_struct)}); {stats}"
    assert max_rel <= tol, f"max relative error {max_rel:.3e} > {tol:.1e}; {stats}"
    return stats

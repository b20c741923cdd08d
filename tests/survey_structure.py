"""Full-matrix structure survey of the CUDA path against the oracle (GPU).

    python tests/survey_structure.py            # every workload below
    python tests/survey_structure.py --quick    # the 9-field prostate only
    python tests/survey_structure.py --instances 8   # the first 8 batched instances only

For every workload below, the whole CSR is computed through the C ABI and by
the FP64 oracle, and every row is compared: a column present on one side
only is counted as "ambiguous" when the oracle places it in a band (within
1e-6 of the threshold, within 1e-3 mm of the cutoff), else as "bad" with its
distance from the threshold.  Workloads: the 9-field prostate, the 32
batched re-plan instances, Table 1 cases 1, 4 and 7, and the slab phantom
(about 1.56e9 candidate pairs; several minutes, most of it in the oracle).
The exit status is the number of bad pairs (0 expected).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def survey(dsc, O, w):
    csr, res, g = dsc.compute_workload(w)
    orc = O.compute_workload(w)
    n_bad = n_amb = 0
    bad = []
    for r in range(w.nrows):
        gc, _ = csr.row(r)
        oc, ov = orc.row(r)
        diff = np.concatenate([np.setdiff1d(gc, oc), np.setdiff1d(oc, gc)])
        if diff.size:
            amb = orc.ambiguous(r)
            for c in diff.tolist():
                if c in amb:
                    n_amb += 1
                    continue
                n_bad += 1
                hit = np.nonzero(oc == c)[0]
                rel = float(ov[hit[0]] / (w.tau * orc.row_max[r]) - 1.0) if hit.size else float("nan")
                bad.append((r, c, rel))
    print(f"{w.name}: pairs {csr.pairs} nnz {csr.nnz} ambiguous {n_amb} bad {n_bad} {bad[:8]}", flush=True)
    dsc.dsc_release_result(res)
    dsc.dsc_destroy_geometry(g)
    return n_bad


def main():
    import torch
    from oracle import oracle as O
    from paper_0908_4417_gb300 import build as B
    from paper_0908_4417_gb300 import dsc, phantoms as P
    B.build()
    O.build()
    torch.cuda.init()
    dsc.lib()
    n_inst = int(sys.argv[sys.argv.index("--instances") + 1]) if "--instances" in sys.argv else 32
    ws = [P.prostate_256()]
    if "--quick" not in sys.argv:
        ws += P.batched(32)[:n_inst] + [P.table1_water(c) for c in (1, 4, 7)]
        ws.append(P.slabs_128(value_dtype=P.VALUE_F32))
    total = sum(survey(dsc, O, w) for w in ws)
    print("bad pairs in total:", total)
    return min(total, 255)


if __name__ == "__main__":
    sys.exit(main())

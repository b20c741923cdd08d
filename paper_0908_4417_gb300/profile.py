"""Run the D_ij path a few times on one workload and print per-stage times.

    python -m paper_0908_4417_gb300.profile --workload prostate_256_2f --reps 3

Used as the target program of Nsight Compute captures (kernel-level
profiles) and for quick stage timing; every repetition is one full
computation through the C ABI with per-stage CUDA events.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="prostate_256_2f")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--bf16", action="store_true")
    a = ap.parse_args()
    import torch
    from paper_0908_4417_gb300 import build, dsc, phantoms
    build.build()
    torch.cuda.init()
    w = phantoms.get(a.workload)
    g = dsc.geometry_from_workload(w)
    opts = dsc.compute_opts(w.tau, dsc.DSC_VALUE_BF16 if a.bf16 else dsc.DSC_VALUE_F32, w.h_frac, dsc.DSC_FLAG_TIMING)
    for i in range(a.reps):
        r = dsc.dsc_compute_dij(g, opts)
        dsc.dsc_result_wait(r)
        v = dsc.dsc_get_csr(r, False)
        t = dsc.dsc_get_stage_times(r)
        print(json.dumps({"rep": i, "workload": w.name, "pairs": int(v.pairs), "nnz": int(v.nnz),
                          "ms": {k: round(x, 4) for k, x in t.items()}}), flush=True)
        dsc.dsc_release_result(r)
    dsc.dsc_destroy_geometry(g)


if __name__ == "__main__":
    main()

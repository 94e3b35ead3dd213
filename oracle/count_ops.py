"""Writes the frozen operation counts that the benchmark's roofline divides by.

The counts come from the oracle alone (``oracle.count_ops``: the FP64 renders
and the replay adjoint evaluated with a counting scalar, per pixel-stroke or
per visited hard-render step), averaged over a seeded pixel sample of each
workload:

  * capsule map: soft render and replay adjoint of the 2000-stroke operating
    program (seed 102, 1024^2, w = 1/200); hard render of the resolution-sweep
    program (seed 106, 1024^2), per visited step;
  * R_D (sixteen-drop transport): soft render of the operating program;
  * Phi_g (coupling profiles seed 403): soft render and adjoint of the
    operating program.

    python oracle/count_ops.py [--pixels 2048] [--out profiles/opcount_1024_2000.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2609_08722_b300 import inputs  # noqa: E402

RES = 1024


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pixels", type=int, default=2048)
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles", "opcount_1024_2000.json"))
    a = ap.parse_args()
    t0 = time.time()
    pix = inputs.sample_pixels(4711, RES * RES, a.pixels)
    tau, tau_min = inputs.SHARP_TAU, inputs.SHARP_TAU_MIN
    op = inputs.operating_program()
    capsule = oracle.count_ops(op, RES, RES, tau, tau_min, pix=pix)
    hard = oracle.count_ops(inputs.resolution_program(), RES, RES, tau, tau_min, pix=pix)["hard"]
    drops = oracle.count_ops(op, RES, RES, tau, tau_min, pix=pix, transport="drops")
    cp = op.copy()
    cp.coupling = inputs.make_coupling(403, cp.n)
    coupled = oracle.count_ops(cp, RES, RES, tau, tau_min, pix=pix)
    out = {
        "what": "operations per unit, counted by evaluating the FP64 oracle with a counting scalar "
                "(FP32-pipe: add, subtract, multiply = 1, no fused multiply-add in the oracle, so a FLOP count; "
                "XU: sqrt, sin, cos, atan2, exp, log, reciprocal); see orc_count_ops in oracle/tbr_oracle.cpp",
        "command": f"python oracle/count_ops.py --pixels {a.pixels}",
        "pixels": int(a.pixels), "resolution": RES, "strokes": op.n,
        "capsule": {"soft_forward": capsule["soft"], "adjoint": capsule["adjoint"], "hard_per_visited_step": hard},
        "drops": {"soft_forward": drops["soft"], "hard_per_visited_step": drops["hard"]},
        "coupled": {"soft_forward": coupled["soft"], "adjoint": coupled["adjoint"],
                    "hard_per_visited_step": coupled["hard"]},
        "seconds": round(time.time() - t0, 1),
    }
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps({k: out[k] for k in ("capsule", "drops", "coupled")}, indent=1))


if __name__ == "__main__":
    main()

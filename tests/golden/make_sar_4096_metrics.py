"""Write sar_4096_image_metrics.json: the FP64 oracle's point-target metrics of
the config-3 image (4096 azimuth x 4096 range point-target scene, range then
azimuth compression; Section VI, Fig. 1, Table III's metric names).

Inputs are what the GPU receives: the seeded scene's echo rounded to complex64
and the oracle's matched filters rounded to FP32.  Only oracle/ does
arithmetic here; the scene comes from the seeded input generator.
``bench.py`` reports the GPU image's metric deltas against these values and
tests/test_gpu_sar.py checks that the file still equals the oracle's output.

Run:  python tests/golden/make_sar_4096_metrics.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import metrics, quant, sar  # noqa: E402
from paper_2605_28451_gb300 import synth  # noqa: E402

KEYS = ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "width_range_cells",
        "width_azimuth_cells", "snr_db", "peak")


def main():
    n = 4096
    sc = synth.point_target_scene(n, n)
    raw = quant.round_binary32(sc.raw)
    hr = quant.round_binary32(sar.matched_filter(quant.round_binary32(sc.ref_range), False))
    ha = quant.round_binary32(sar.matched_filter(quant.round_binary32(sc.ref_azimuth), True))
    img = sar.range_doppler_image(raw, hr, ha)
    m = metrics.point_target_metrics(img, sc.targets)
    out = {
        "what": "FP64 oracle point-target metrics of the 4096 x 4096 range-Doppler image "
                "(synth.point_target_scene(4096, 4096), complex64 echo, FP32-rounded filters; guard 96)",
        "written_by": "tests/golden/make_sar_4096_metrics.py (oracle.sar, oracle.metrics)",
        "targets": [[int(e), int(r)] for e, r, _ in sc.targets],
        "peak_cells": [[int(x["peak_cell"][0]), int(x["peak_cell"][1])] for x in m],
        "metrics": [{k: float(x[k]) for k in KEYS} for x in m],
    }
    with open(os.path.join(HERE, "sar_4096_image_metrics.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()

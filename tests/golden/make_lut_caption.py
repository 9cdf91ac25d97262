"""Writes lut_caption.json: a 17-sample, 9-pixel fixture for the two-level
lookup table of HCGrid Sec. 3.3 (Fig. "preorder" caption: 17 samples in 9
HEALPix pixels, R_start[1..4] = 1, 7, 10, 17 in 1-based sample positions).

Samples sit near the centres of chosen Nside=2 RING pixels (centres from the
oracle's pix2ang, offsets of at most 1.5 degrees, far inside pixels that span
~29 degrees), so that rings 1..4 hold 6, 3, 7 and 1 samples.  Calls only
oracle/.  Run from the repository root:  python tests/golden/make_lut_caption.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle  # noqa: E402

NSIDE = 2
# pixel -> number of samples; rings (Nside 2): 1 = pix 0-3, 2 = 4-11, 3 = 12-19, 4 = 20-27
LAYOUT = {0: 2, 1: 2, 3: 2, 5: 2, 6: 1, 12: 3, 13: 2, 19: 2, 22: 1}
OFFS = [(0.0, 0.0), (1.5, -1.0), (-1.0, 1.5)]


def main():
    lon, lat = [], []
    for p, k in LAYOUT.items():
        clon, clat = oracle.pix2ang(NSIDE, [p])
        for q in range(k):
            dl, db = OFFS[q]
            lon.append(float(clon[0] + dl)); lat.append(float(clat[0] + db))
    order = np.random.default_rng(7).permutation(len(lon))
    lon = [lon[i] for i in order]; lat = [lat[i] for i in order]
    out = {
        "source": "HCGrid (arXiv 2012.13173) Sec. 3.3, caption of Fig. 'preorder'",
        "nside": NSIDE, "r_lo": 1, "r_hi": 4,
        "lon_deg": lon, "lat_deg": lat,
        "expect_samples": 17, "expect_pixels": 9,
        "expect_rstart_1based": [1, 7, 10, 17],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lut_caption.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()

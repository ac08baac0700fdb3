"""Writes the stored expected values under tests/golden/.

Calls only the oracle (and the closed forms stated beside each value); never
the CUDA path.  Run:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    h = 1.0 / 64
    cw = {
        "_source": "closed form at mu_t = 0, D_0 = (2h/pi) ln(1+sqrt 2) (cell integral of "
                   "1/(2 pi r), Sec. 2.3 diagonal rule); oracle values for mu_t > 0 as regression pins",
        "D0_massless_h1_64": 2 * h / math.pi * math.log(1 + math.sqrt(2)),
        "oracle_D_mu1_h1_64_m0_4_8": [float(v) for v in oracle.cell_weights_2d(1.0, h, 8)[8::4]],
        "oracle_D_mu10_h1_256_m0_4_8": [float(v) for v in oracle.cell_weights_2d(10.0, 1 / 256, 8)[8::4]],
        "oracle_D3_mu100_h1_128": oracle.cell_weight_3d(100.0, 1 / 128),
    }
    with open(os.path.join(HERE, "cell_weights.json"), "w") as fh:
        json.dump(cw, fh, indent=1)
    print("wrote cell_weights.json")


if __name__ == "__main__":
    main()

"""Writes the stored oracle outputs used by the regression tests.

Calls only the oracle and the seeded input generator. Run from the
repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    frames, seed, ebn0, L, T = 48, 0, 1.0, 8, 4
    wl = synth.make_workload("rm26_crc6", ebn0, frames, seed=seed)
    code = oracle.rm_code(6, 2, crc_poly=0x21, crc_len=6)
    code = code.with_patterns(code.enumerate_codewords([16]))
    out = code.decode(wl.y, L, T, threads=1)
    gold = {
        "source": "oracle outputs (two-stage SCL + MP-WSD, Sec. III) on the first 48 frames of the RM(2,6)+CRC-6 "
                  "workload at Eb/N0 = 1 dB, seed 0; y stored as integers y * 2^19",
        "code": "rm26_crc6", "ebn0_db": ebn0, "frames": frames, "seed": seed, "L": L, "T": T,
        "y_int": np.rint(wl.y.astype(np.float64) * 2 ** 19).astype(np.int64).tolist(),
        "cw_hex": [f"{int(w):016x}" for w in out["cw"][:, 0]],
        "flags": out["flags"].tolist(),
    }
    with open(os.path.join(here, "rm26_crc6_1db_seed0_first48.json"), "w") as fh:
        json.dump(gold, fh, separators=(",", ":"))
        fh.write("\n")


if __name__ == "__main__":
    main()

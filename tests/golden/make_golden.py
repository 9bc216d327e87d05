"""Write the stored expected values under tests/golden/ from the FP64 oracle alone:

    python tests/golden/make_golden.py

cube8_ngll5_seismograms.txt -- the homogeneous 8^3-element cube (side 1 km, NGLL 5, rho 2500,
vp 3000, vs 1730; Ricker 10 Hz +z point force of 1e10 N at the centre node; 8 receivers on
the top face; Courant 0.4), 200 explicit Newmark steps from rest (Sec. II-B, Sec. V-C): the
oracle's time step, source and receiver nodes, and seismograms [receiver][component][step].
A later change to the oracle's arithmetic that moves these values has to name, in its
commit message, the passage of the paper (or the reading of it) that justifies it.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import sem_oracle  # noqa: E402
from paper_2606_12850_gb300 import inputs  # noqa: E402

CUBE8 = os.path.join(HERE, "cube8_ngll5_seismograms.txt")


def cube8():
    w = inputs.homogeneous_cube()
    return w, sem_oracle.run_workload(w)


def write_cube8(path: str = CUBE8):
    w, ref = cube8()
    seis = ref["seis"]
    with open(path, "w") as f:
        f.write("# homogeneous 8^3 cube, 1 km, NGLL 5, 200 Newmark steps from rest; FP64 oracle\n")
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        f.write(f"dt {ref['dt']:.17g}\n")
        f.write("src " + " ".join(str(int(v)) for v in ref["src"]) + "\n")
        f.write("rec " + " ".join(str(int(v)) for v in ref["rec"]) + "\n")
        f.write(f"shape {seis.shape[0]} {seis.shape[1]} {seis.shape[2]}\n")
        for r in range(seis.shape[0]):
            for c in range(seis.shape[1]):
                f.write(" ".join(f"{v:.17g}" for v in seis[r, c]) + "\n")


def read_cube8(path: str = CUBE8) -> dict:
    out = {}
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "dt":
                out["dt"] = float(rest)
            elif key in ("src", "rec"):
                out[key] = np.array([int(v) for v in rest.split()])
            elif key == "shape":
                out["shape"] = tuple(int(v) for v in rest.split())
            else:
                rows.append([float(v) for v in line.split()])
    out["seis"] = np.array(rows).reshape(out["shape"])
    return out


if __name__ == "__main__":
    write_cube8()
    print("wrote", CUBE8)

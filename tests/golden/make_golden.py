"""Write the stored expected values under tests/golden/ (run: python tests/golden/make_golden.py).

The paper prints no worked numbers for its kernels (their sources are not part of it), so
these fixtures hold the exact values of the two loop bodies defined in the oracle (RHS: Euler
flux differences with 4th-order dissipation; star stencil: the 25-point variable-coefficient
Laplacian-type sum), on small seeded inputs, as computed over the rationals by
`oracle/exact.py` and rounded once to the nearest double. Only `oracle/` and the seeded input
generators are called; nothing here runs the CUDA path.

Each file: '#' header lines (what, inputs, recipe), then one line per output value:
`c k j i value` (RHS) or `k j i value` (stencil), value as a round-trip decimal.
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.abspath(os.path.join(HERE, "..", "..")))

from oracle import exact  # noqa: E402
from paper_2306_13002_gb300 import inputs  # noqa: E402

# (file, kind, interior dims (nx, ny, nz), seed, parameters)
CASES = [
    ("rhs_4x3x3_seed13002.txt", "rhs", (4, 3, 3), 13002, {"gamma": 1.4, "eps": 0.25, "h": (1.0, 1.0, 1.0)}),
    ("rhs_3x3x2_seed13010_h.txt", "rhs", (3, 3, 2), 13010, {"gamma": 1.4, "eps": 0.25, "h": (1.0, 0.5, 2.0)}),
    ("star_4x3x3_seed13004.txt", "star", (4, 3, 3), 13004, {}),
]

# 8th-order central second-derivative weights on every axis (the stencil's default table)
TAYLOR = [[8 / 5, -1 / 5, 8 / 315, -1 / 560]] * 3


def write(name, kind, dims, seed, prm):
    nx, ny, nz = dims
    lines = [f"# {kind} exact values, interior {nx} x {ny} x {nz}, seed {seed}, written by make_golden.py",
             "# exact rational value of the as-written definition (oracle/exact.py), rounded once to FP64"]
    if kind == "rhs":
        U = inputs.rhs_field(nx, ny, nz, halo=2, seed=seed)
        lines.append(f"# inputs: inputs.rhs_field({nx}, {ny}, {nz}, halo=2, seed={seed}); "
                     f"gamma {prm['gamma']}, eps {prm['eps']}, h {prm['h']}")
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    vals, _ = exact.rhs_point(U, i, j, k, gamma=prm["gamma"], eps=prm["eps"], h=prm["h"])
                    for c in range(5):
                        lines.append(f"{c} {k} {j} {i} {float(vals[c])!r}")
    else:
        u, a = inputs.stencil_fields(nx, ny, nz, halo=4, seed=seed)
        lines.append(f"# inputs: inputs.stencil_fields({nx}, {ny}, {nz}, halo=4, seed={seed}); "
                     "weights [8/5, -1/5, 8/315, -1/560] on every axis")
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    val, _ = exact.stencil_point(u, a, TAYLOR, i, j, k)
                    lines.append(f"{k} {j} {i} {float(val)!r}")
    with open(os.path.join(HERE, name), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    for case in CASES:
        write(*case)
        print("wrote", case[0])

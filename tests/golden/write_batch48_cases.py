"""Writes batch48_cases.txt: the 48-case uneven batch drawn with numpy PCG64(20260503) by
paper_2605_03479_gb300.inputs.config4_cases.  Input data only (no step of the method); run from the repository
root:  python tests/golden/write_batch48_cases.py"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2605_03479_gb300 import inputs as I  # noqa: E402


def table_lines():
    lines = ["# 48-case batch, numpy PCG64(20260503), drawn in the order drive, N_cell, N_vel, N_H, log10 Kn, log10 St",
             "# columns: index drive n_cell n_vel n_h kn st"]
    for k, c in enumerate(I.config4_cases()):
        drive = "shear" if "shear" in c.name else "thermal"
        lines.append(f"{k} {drive} {c.nx} {c.nu} {c.n_harmonics} {c.kn:.17g} {c.st:.17g}")
    return lines


if __name__ == "__main__":
    with open(os.path.join(HERE, "batch48_cases.txt"), "w") as f:
        f.write("\n".join(table_lines()) + "\n")

"""The paper's isentropic-vortex table (Sec. 6.1, Table 1), read from tests/golden/vortex_table1.txt."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def table1():
    """{(R, cells per side): (L1 error, EOC or None)}"""
    out = {}
    with open(os.path.join(HERE, "golden", "vortex_table1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            R, n, err, eoc = line.split()
            out[(int(R), int(n))] = (float(err), None if eoc == "-" else float(eoc))
    return out

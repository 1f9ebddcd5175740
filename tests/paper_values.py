"""Reader for tests/golden/paper_counts.txt (values printed in the paper, each with its citation)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_counts.txt")


def load():
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = float(v) if ("." in v or "e" in v) else int(v)
    return out

"""Reader for the small text fixtures in this folder."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_figures() -> dict:
    out = {}
    with open(os.path.join(HERE, "paper_figures.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = float(v)
    return out

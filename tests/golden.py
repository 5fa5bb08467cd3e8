"""Reader for the paper's numbers under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def keyvals(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, *v = line.split()
            vals = [float(x) if any(c in x for c in ".e") else int(x) for x in v]
            out[k] = vals[0] if len(vals) == 1 else vals
    return out


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                out.append([float(x) for x in line.split()])
    return out

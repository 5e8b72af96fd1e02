"""Reader of the paper's printed counts in paper_counts.txt."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_counts():
    out = {}
    with open(os.path.join(HERE, "paper_counts.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (t.strip() for t in line.split("=", 1))
            vals = [int(v) for v in val.split(",")]
            out[key] = vals[0] if len(vals) == 1 else vals
    return out

"""Reader for tests/golden/paper_counts.txt (values printed in the paper)."""
import os

_PATH = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")


def table(name):
    rows = []
    with open(_PATH) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == name:
                rows.append([float(t) for t in parts[1:]])
    return rows

"""Reader for the hand-derived text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    """Returns (filter KxK array, [(case, border, input HxW, expected HxW), ...])."""
    lines = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                lines.append(line)
    pos = 0

    def rows(count):
        nonlocal pos
        out = [list(map(float, lines[pos + k].split())) for k in range(count)]
        pos += count
        return np.array(out, dtype=np.float64)

    head = lines[pos].split(); pos += 1
    assert head[0] == "filter"
    filt = rows(int(head[1]))
    cases = []
    while pos < len(lines):
        head = lines[pos].split(); pos += 1
        assert head[0] == "case"
        name, border, H = head[1], head[2], int(head[3])
        assert lines[pos] == "input"; pos += 1
        x = rows(H)
        assert lines[pos] == "expected"; pos += 1
        y = rows(H)
        cases.append((name, border, x, y))
    return filt, cases

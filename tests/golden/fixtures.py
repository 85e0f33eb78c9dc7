"""Readers for the hand-written golden fixtures in this folder."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def worked_example():
    """Returns {variant: dict} parsed from worked_example.txt."""
    out, cur = {}, None
    with open(os.path.join(HERE, "worked_example.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "variant":
                cur = {"edges": []}
                out[vals[0]] = cur
            elif key == "end":
                cur = None
            elif key == "edge":
                cur["edges"].append(tuple(int(v) for v in vals))
            elif len(vals) == 1:
                cur[key] = int(vals[0])
            else:
                cur[key] = [int(v) for v in vals]
    return out

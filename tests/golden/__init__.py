"""Reader for the hand-worked text fixtures in this folder."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load_hand_graphs(path=None):
    """Parse hand_graphs.txt into a list of dicts (name, n, root, edges [2, m],
    levels, parents and, where given, off, col, teps)."""
    path = path or os.path.join(HERE, "hand_graphs.txt")
    out, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "graph":
                cur = {"name": vals[0]}
            elif key == "end":
                e = np.array(cur.pop("edges_flat"), dtype=np.int64).reshape(-1, 2)
                cur["edges"] = np.ascontiguousarray(e.T)
                out.append(cur)
                cur = None
            elif key in ("n", "root", "teps"):
                cur[key] = int(vals[0])
            elif key == "edges":
                cur["edges_flat"] = [int(v) for v in vals]
            elif key in ("levels", "parents", "col"):
                cur[key] = np.array([int(v) for v in vals], dtype=np.int32)
            elif key == "off":
                cur[key] = np.array([int(v) for v in vals], dtype=np.int64)
            else:
                raise ValueError("unknown fixture key %r" % key)
    return out

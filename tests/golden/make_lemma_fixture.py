"""Writes lemma_active_set.json: the active sets printed in the paper's Lemma (Section
"Large sets of active vertices") for the lattice [-n, n] x [0, n], T = 3..22.  The sets
come from the Lemma's formula alone; no solver is called."""
import json
import os


def lemma_set(T, n):
    K = (T + 1) // 4
    pts = {(0, T), (0, T - 1)}
    for k in range(1, K + 1):
        pts |= {(-k, T - 2 * k), (k, T - 2 * k)}
    for z in range(-n, n + 1):
        if abs(z) > K:
            pts.add((z, T // 2))
    return sorted(pts)


if __name__ == "__main__":
    n = 24
    out = {"source": "arXiv 1511.06441, Lemma in Section 'Large sets of active vertices'",
           "n": n, "lemma_sets": {str(T): lemma_set(T, n) for T in range(3, 23)}}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "lemma_active_set.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))

"""Reader for tests/golden/worked_examples.txt (hand-derived closed forms)."""
import os
from typing import Dict, List

import numpy as np

from workloads import Circuit, Gate, qft

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "worked_examples.txt")


def _parse_gates(n: int, text: str) -> Circuit:
    text = text.strip()
    if text == "QFT":
        return qft(n)
    gates: List[Gate] = []
    for part in [p.strip() for p in text.split(";") if p.strip()]:
        tok = part.split()
        kind, targets, controls, angle = tok[0], [], [], 0.0
        for t in tok[1:]:
            if t.startswith("c="):
                controls = [int(v) for v in t[2:].split(",")]
            elif t.startswith("a="):
                angle = float(t[2:])
            else:
                targets.append(int(t))
        gates.append(Gate(kind, tuple(targets), tuple(controls), -1, angle))
    return Circuit(n, gates, 0)


def load() -> List[Dict]:
    blocks, cur = [], None
    with open(GOLDEN) as f:
        for line in f:
            line = line.rstrip("\n")
            if not line.strip() or line.lstrip().startswith("#"):
                continue
            if line.startswith("["):
                cur = {"name": line.strip()[1:-1]}
                blocks.append(cur)
                continue
            key, _, val = line.partition("=")
            cur[key.strip()] = val.strip()
    out = []
    for b in blocks:
        n = int(b["n"])
        e = {"name": b["name"], "n": n, "input": int(b["input"]),
             "circuit": _parse_gates(n, b.get("gates", "")), "cite": b["cite"]}
        if "amps" in b:
            amps = np.zeros(1 << n, np.complex128)
            for item in b["amps"].split():
                idx, _, reim = item.partition(":")
                re, im = reim.split(",")
                amps[int(idx)] = complex(float(re), float(im))
            e["amps"] = amps
        if "energy" in b:
            e["energy"] = float(b["energy"])
        out.append(e)
    return out

"""Reader of tests/golden/bicgstab_breakdown.txt: small block systems on which
BiCGStab meets an exact zero divisor (written in exact rational arithmetic by
tests/golden/breakdown_cases.py).  Builds each as a 3x3 block-CSR system
(blocks scalar * I3, right-hand side repeating one value per block row)."""
import os
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bicgstab_breakdown.txt")


@dataclass
class Case:
    name: str
    nb: int
    event: str          # rho, rhv, tt or omega: the divisor that is exactly zero
    k: int              # iteration in which the method meets it
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray    # (nnzb, 9)
    b: np.ndarray       # 3 nb
    part: np.ndarray | None
    q: dict = field(default_factory=dict)  # quantity -> list of Fractions (per block row)

    def vec(self, name):
        """A listed per-block-row quantity as a 3 nb float vector."""
        return np.repeat(np.array([float(v) for v in self.q[name]]), 3)


def load():
    cases = {}
    cur = None
    with open(PATH) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "case":
                cur = {"name": w[1], "nb": int(w[2]), "event": w[3], "k": int(w[4]), "a": {}, "part": None,
                       "q": {}}
            elif w[0] == "a":
                cur["a"][(int(w[1]), int(w[2]))] = Fraction(w[3])
            elif w[0] == "b":
                cur["b"] = [Fraction(v) for v in w[1:]]
            elif w[0] == "part":
                cur["part"] = np.array([int(v) for v in w[1:]], dtype=np.int32)
            elif w[0] == "q":
                cur["q"][w[1]] = [Fraction(v) for v in w[2:]]
            elif w[0] == "end":
                nb = cur["nb"]
                rowptr = [0]
                colidx, vals = [], []
                for i in range(nb):
                    for j in range(nb):
                        if (i, j) in cur["a"]:
                            colidx.append(j)
                            vals.append(float(cur["a"][(i, j)]) * np.eye(3).ravel())
                    rowptr.append(len(colidx))
                cases[cur["name"]] = Case(cur["name"], nb, cur["event"], cur["k"],
                                          np.array(rowptr, dtype=np.int32), np.array(colidx, dtype=np.int32),
                                          np.array(vals), np.repeat(np.array([float(v) for v in cur["b"]]), 3),
                                          cur["part"], cur["q"])
    return cases

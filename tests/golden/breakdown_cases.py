"""Writes bicgstab_breakdown.txt: small block systems on which right-
preconditioned BiCGStab (Section 4.2; van der Vorst 1992) meets an exact
zero in one of its four divisors, derived in exact rational arithmetic.

Every block is a scalar times the 3x3 identity and every right-hand side
repeats one value per block row, so each system is three copies of a scalar
system.  Entries are small dyadic rationals and every pivot is a power of
two, so each quantity below is exactly representable in binary floating
point: a floating-point run that follows the method reaches the same exact
zero whatever its summation order.  The preconditioner is ILU0 in natural
order (Algorithm 2): fill between rows that share only an earlier neighbour
is dropped, so M differs from A.  The block-Jacobi case keeps only the
diagonal blocks (Section 4.5, every row its own partition).

This script uses Python's Fraction only; it calls neither the oracle nor the
library.  Run it from the repository root to rewrite the fixture:
    python tests/golden/breakdown_cases.py
"""
from fractions import Fraction as F
import os

# name: (block rows, {(i, j): scalar}, b per block row, partition or None,
#        the zero the method meets, the iteration it meets it in)
CASES = {
    "arrow_rhv1": (3, {(0, 0): F(1, 2), (0, 1): F(1, 2), (0, 2): F(1), (1, 0): F(1), (1, 1): F(-1),
                       (2, 0): F(1), (2, 2): F(1)}, [2, 1, -2], None, "rhv", 1),
    "arrow_omega1": (3, {(0, 0): F(1), (0, 1): F(-2), (0, 2): F(-2), (1, 0): F(-1), (1, 1): F(4),
                         (2, 0): F(-2), (2, 2): F(2)}, [2, 0, -2], None, "omega", 1),
    "arrow_tt1": (3, {(0, 0): F(1), (0, 1): F(-1, 2), (0, 2): F(1, 2), (1, 0): F(-1, 2), (1, 1): F(1, 2),
                      (2, 0): F(-1), (2, 2): F(-1)}, [2, 0, 0], None, "tt", 1),
    "arrow_rho2": (3, {(0, 0): F(2), (0, 1): F(2), (0, 2): F(2), (1, 0): F(-2), (1, 1): F(-1),
                       (2, 0): F(-1), (2, 2): F(1)}, [2, 0, 0], None, "rho", 2),
    "arrow_rhv2": (3, {(0, 0): F(4), (0, 1): F(-1), (0, 2): F(-2), (1, 0): F(-1), (1, 1): F(1, 2),
                       (2, 0): F(-1), (2, 2): F(1)}, [0, 2, 0], None, "rhv", 2),
    "cycle_rho2": (4, {(0, 0): F(1), (0, 1): F(1, 2), (0, 2): F(1), (1, 0): F(2), (1, 1): F(1, 2),
                       (1, 3): F(-2), (2, 0): F(1, 2), (2, 2): F(1), (2, 3): F(-1, 2), (3, 1): F(1, 2),
                       (3, 2): F(1, 2), (3, 3): F(2)}, [1, 0, 0, -2], None, "rho", 2),
    # unpreconditioned (M = I): rho2 = -omega1 (b, A s1) vanishes while (b, A r1) does not, so this
    # case meets only the rho test
    "jacobi_rho2": (3, {(0, 0): F(1), (0, 1): F(1), (1, 1): F(1), (1, 2): F(1), (2, 0): F(1), (2, 2): F(1)},
                    [0, -2, 0], [0, 1, 2], "rho", 2),
    "jacobi_rhv1": (2, {(0, 0): F(1), (0, 1): F(-2), (1, 1): F(1)}, [1, 1], [0, 1], "rhv", 1),
}


def _ilu0(n, a, keep):
    """Natural-order ILU0 on the kept pattern; returns (lu, inverse pivots)."""
    lu = {e: v for e, v in a.items() if keep(e)}
    dinv = []
    for i in range(n):
        for k in sorted(j for (r, j) in lu if r == i and j < i):
            lu[(i, k)] *= dinv[k]
            for j in range(k + 1, n):
                if (i, j) in lu and (k, j) in lu:
                    lu[(i, j)] -= lu[(i, k)] * lu[(k, j)]
        dinv.append(1 / lu[(i, i)])
    return lu, dinv


def _solve_m(n, lu, dinv, r):
    y = list(r)
    for i in range(n):
        for j in range(i):
            if (i, j) in lu:
                y[i] -= lu[(i, j)] * y[j]
    z = [F(0)] * n
    for i in reversed(range(n)):
        acc = y[i]
        for j in range(i + 1, n):
            if (i, j) in lu:
                acc -= lu[(i, j)] * z[j]
        z[i] = dinv[i] * acc
    return z


def _mv(n, a, x):
    return [sum((a[(i, j)] * x[j] for j in range(n) if (i, j) in a), F(0)) for i in range(n)]


def _dot(u, v):  # scalar dot; the block system's is three times it
    return sum((p * q for p, q in zip(u, v)), F(0))


def derive(n, a, b, part):
    keep = (lambda e: True) if part is None else (lambda e: part[e[0]] == part[e[1]])
    lu, dinv = _ilu0(n, a, keep)
    b = [F(q) for q in b]
    x, r, rh = [F(0)] * n, list(b), list(b)
    p, v = [F(0)] * n, [F(0)] * n
    rho_prev = alpha = omega = F(1)
    out = []
    for k in (1, 2):
        rho = _dot(rh, r)
        out.append((f"rho{k}", [rho]))
        if rho == 0:
            return out
        beta = (rho / rho_prev) * (alpha / omega)
        p = [ri + beta * (pi - omega * vi) for ri, pi, vi in zip(r, p, v)]
        ph = _solve_m(n, lu, dinv, p)
        v = _mv(n, a, ph)
        rhv = _dot(rh, v)
        out += [(f"ph{k}", ph), (f"v{k}", v), (f"rhv{k}", [rhv])]
        if rhv == 0:
            return out
        alpha = rho / rhv
        s = [ri - alpha * vi for ri, vi in zip(r, v)]
        sh = _solve_m(n, lu, dinv, s)
        t = _mv(n, a, sh)
        tt = _dot(t, t)
        out += [(f"alpha{k}", [alpha]), (f"s{k}", s), (f"sh{k}", sh), (f"t{k}", t), (f"tt{k}", [tt])]
        if tt == 0:
            return out
        omega = _dot(t, s) / tt
        out.append((f"omega{k}", [omega]))
        if omega == 0:
            return out
        x = [xi + alpha * phi + omega * shi for xi, phi, shi in zip(x, ph, sh)]
        r = [si - omega * ti for si, ti in zip(s, t)]
        out += [(f"x{k}", x), (f"r{k}", r)]
        rho_prev = rho
    return out


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "# BiCGStab breakdowns (Section 4.2 building blocks; van der Vorst 1992), derived in exact",
        "# rational arithmetic by breakdown_cases.py beside this file (Fraction only, no oracle, no GPU).",
        "# Blocks are scalar * I3 and b repeats one value per block row, so the vectors below are per",
        "# block row and every block dot product is three times the scalar one listed.",
        "# Hand check of arrow_rhv1: ILU0 gives L = [1 0 0; 2 1 0; 2 0 1], U = [1/2 1/2 1; 0 -2 0; 0 0 -1]",
        "# (the (1,2) and (2,1) fill is dropped); M^-1 b = (-19/2, 3/2, 6); A of that = (2, -11, -7/2);",
        "# (b, v) = 4 - 11 + 7 = 0.",
        "# Hand check of jacobi_rho2 (M = I): v1 = A b = (-2, -2, 0), (b, v1) = 4 = (b, b), alpha1 = 1,",
        "# s1 = b - v1 = (2, 0, 0), t1 = A s1 = (2, 0, 2), omega1 = 4 / 8 = 1/2, r1 = s1 - t1 / 2 = (1, 0, -1),",
        "# (b, r1) = 0; had the method gone on, (b, A r1) = 2 would not vanish.",
        "# Format: 'case NAME NB EVENT K', 'a I J VALUE' per block, 'b ...', optional 'part ...',",
        "# then 'q NAME VALUES...' for the quantities up to the zero, 'end'.",
    ]
    for name, (n, a, b, part, event, k) in CASES.items():
        q = derive(n, a, b, part)
        last = q[-1]
        assert last[0] == f"{event}{k}" and last[1] == [0], (name, last)
        lines.append(f"case {name} {n} {event} {k}")
        for (i, j), v in sorted(a.items()):
            lines.append(f"a {i} {j} {v}")
        lines.append("b " + " ".join(str(v) for v in b))
        if part is not None:
            lines.append("part " + " ".join(str(v) for v in part))
        for qn, vals in q:
            lines.append(f"q {qn} " + " ".join(str(v) for v in vals))
        lines.append("end")
    with open(os.path.join(here, "bicgstab_breakdown.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

"""Readers for the text fixtures under tests/golden (values printed in the
paper's worked examples, or worked by hand; each file cites its source)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln


def frac(s):
    return Fraction(s.strip())


def read_example3():
    d = {"P": []}
    for ln in _lines("example3.txt"):
        key, *vals = ln.split()
        if key == "P":
            d["P"].append([frac(v) for v in vals])
        else:
            d[key] = [frac(v) for v in vals]
    return d


def _eval_expr(expr, M):
    env = {"M1": M[0], "M2": M[1], "M3": M[2], "M4": M[3], "__builtins__": {}}
    return Fraction(eval(expr.replace(" ", ""), env))


def read_example9(name, M):
    """Rows (t, H_t, C_t, G_t) of an Example 9 table with M_0 = M (Fractions)."""
    M = [Fraction(x) for x in M]
    rows = []
    for ln in _lines(name):
        t, h, c, g = [p.strip() for p in ln.split(";")]
        H = [_eval_expr(e, M) for e in h.split(",")]
        C = [_eval_expr(e, M) for e in c.split(",")]
        rows.append((int(t), H, C, int(g)))
    return rows


def read_selection_cases():
    out = []
    for ln in _lines("selection_cases.txt"):
        sched, param, cash, green, theta = [p.strip() for p in ln.split(";")]
        out.append(dict(sched=sched, param=float(param),
                        cash=np.array([float(x) for x in cash.split(",")]),
                        green=sorted(int(x) for x in green.split(",")),
                        theta=float(Fraction(theta)) if "/" in theta else float(theta)))
    return out

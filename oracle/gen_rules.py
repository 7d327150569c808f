"""Oracle-side solver for the Gauss-Hermite velocity sets (test infrastructure).

Solves the moment conditions of a degree-Q Gauss-Hermite quadrature
(Sec. 2, the quadrature identity preceding Eq. an1: the weighted sum of any
polynomial of degree <= Q over the abscissae equals its integral against the
Gaussian weight omega) for the two velocity sets used by this project:

* D2Q37, degree 9 (Sec. 3: "ninth-order accurate D2Q37"); the abscissae are
  c * e_i for the integer shells (0,0), (1,0), (1,1), (2,0), (2,1), (2,2),
  (3,0), (3,1) with their full square symmetry.  The paper prints only the
  lattice constant c ~ 1.19698 (Sec. 3.1).
* D3Q39, degree 7; shells (0,0,0), (1,0,0), (1,1,1), (2,0,0), (2,2,0), (3,0,0)
  with full cubic symmetry.  Not in the paper: a standard degree-7 rule.

Unknowns are one weight per shell plus the scale c; the equations are the
even-moment conditions sum_i w_i xi_i^alpha = prod_k (alpha_k - 1)!!, one per
monomial class up to permutation.  The solve is a Newton iteration on the full
nonlinear system in 50-digit arithmetic (mpmath.findroot).

Running this module writes ``oracle/rules.h``: each constant rounded once,
correctly, from the 50-digit solution to an IEEE double and printed as a C99
hex-float literal, so x86_64 and aarch64 builds read bit-identical values.  It
is the ONLY producer of that file.
"""
import itertools
import os

import mpmath as mp

mp.mp.dps = 50

SHELLS = {
    "D2Q37": [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)],
    "D3Q39": [(0, 0, 0), (1, 0, 0), (1, 1, 1), (2, 0, 0), (2, 2, 0), (3, 0, 0)],
}
DEGREE = {"D2Q37": 9, "D3Q39": 7}
# starting points for Newton (rough double-precision guesses)
GUESS = {
    "D2Q37": ([0.233, 0.107, 0.0577, 0.0142, 0.00535, 0.00101, 0.000245, 0.000283], 1.197),
    "D3Q39": ([0.083, 0.083, 0.037, 0.0148, 0.0023, 0.0006], 1.22),
}


def shell_members(rep, D):
    """All distinct vectors obtained from rep by permutations and sign flips."""
    out = set()
    for perm in itertools.permutations(rep):
        for signs in itertools.product((1, -1), repeat=D):
            out.add(tuple(s * p for s, p in zip(signs, perm)))
    return sorted(out)


def velocity_set(name):
    """Ordered list of (shell index, integer vector) for the named set."""
    D = len(SHELLS[name][0])
    vs = []
    for k, rep in enumerate(SHELLS[name]):
        for v in shell_members(rep, D):
            vs.append((k, v))
    return vs


def dfact(n):
    """(n-1)!! for even n, i.e. the n-th moment of the unit Gaussian."""
    r = 1
    for k in range(n - 1, 0, -2):
        r *= k
    return r


def even_classes(D, degree):
    """Monomial exponent classes (sorted, all even) of total degree <= degree."""
    cls = set()
    for alpha in itertools.product(range(0, degree + 1, 2), repeat=D):
        if sum(alpha) <= degree:
            cls.add(tuple(sorted(alpha, reverse=True)))
    return sorted(cls)


def residuals(name, w, c):
    D = len(SHELLS[name][0])
    vs = velocity_set(name)
    res = []
    for alpha in even_classes(D, DEGREE[name]):
        s = mp.mpf(0)
        for k, v in vs:
            term = w[k]
            for a, e in zip(alpha, v):
                term *= (c * e) ** a
            s += term
        exact = 1
        for a in alpha:
            exact *= dfact(a)
        res.append(s - exact)
    return res


def solve(name):
    w0, c0 = GUESS[name]
    n = len(w0)

    def F(*x):
        return residuals(name, list(x[:n]), x[n])

    sol = mp.findroot(F, [mp.mpf(v) for v in w0] + [mp.mpf(c0)], tol=mp.mpf(10) ** -45)
    sol = [sol[i] for i in range(n + 1)]
    return sol[:n], sol[n]


def to_hex(x):
    """Correctly rounded IEEE double of an mpf, as a C99 hex-float literal."""
    return float(x).hex()


def write_header(path):
    lines = [
        "/* Generated by oracle/gen_rules.py (mpmath Newton solve of the moment",
        " * conditions, 50 digits; each value rounded once to double).",
        " * Oracle-only constants; do not edit. */",
        "#ifndef ORACLE_RULES_H",
        "#define ORACLE_RULES_H",
    ]
    for name in ("D2Q37", "D3Q39"):
        w, c = solve(name)
        D = len(SHELLS[name][0])
        vs = velocity_set(name)
        lines.append(f"#define ORC_{name}_Q {len(vs)}")
        lines.append(f"#define ORC_{name}_D {D}")
        lines.append(f"static const double orc_{name}_c = {to_hex(c)}; /* {mp.nstr(c, 25)} */")
        lines.append(f"static const double orc_{name}_shell_w[{len(w)}] = {{")
        lines += [f"  {to_hex(x)}, /* {mp.nstr(x, 25)} */" for x in w]
        lines.append("};")
        lines.append("/* (shell, e_x, e_y, e_z) */")
        lines.append(f"static const int orc_{name}_vel[{len(vs)}][4] = {{")
        for k, v in vs:
            v3 = list(v) + [0] * (3 - D)
            lines.append(f"  {{{k}, {v3[0]}, {v3[1]}, {v3[2]}}},")
        lines.append("};")
    lines.append("#endif")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    write_header(os.path.join(os.path.dirname(os.path.abspath(__file__)), "rules.h"))

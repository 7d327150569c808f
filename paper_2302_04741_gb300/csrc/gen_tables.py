"""Generator of the compile-time velocity-set tables of the CUDA library.

Writes ``lattice_tables.cuh``.  The velocity sets are degree-Q Gauss-Hermite
rules (Sec. 2, the quadrature identity before Eq. an1): D2Q37 of degree 9
(Sec. 3, cited there from Shan 2016; only c ~ 1.19698 is printed) and D3Q39
of degree 7.  The solve here is independent of any other solver in the
repository: for a trial s = c^2 the shell weights follow from the lowest
even-moment conditions by Gaussian elimination in 60-digit ``decimal``
arithmetic, and s is the root of the one remaining condition (``residual``:
a class whose removal leaves the linear system nonsingular), bracketed and
bisected.

Direction order is chosen for the kernels: index 0 is the rest particle, then
opposite pairs (2k+1, 2k+2) = (e, -e), so that the even/odd parts of each
polynomial in xi are shared by a pair.
"""
import decimal
import itertools
import os

D = decimal.Decimal
decimal.getcontext().prec = 60

SETS = {
    "D2Q37": dict(dim=2, degree=9, neq=4,
                  shells=[(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)],
                  bracket=("1.30", "1.60"), residual=(8, 0)),
    "D3Q39": dict(dim=3, degree=7, neq=3,
                  shells=[(0, 0, 0), (1, 0, 0), (1, 1, 1), (2, 0, 0), (2, 2, 0), (3, 0, 0)],
                  bracket=("1.40", "1.60"), residual=(2, 2, 2)),
}


def members(rep, dim):
    out = set()
    for p in itertools.permutations(rep):
        for sg in itertools.product((1, -1), repeat=dim):
            out.add(tuple(a * b for a, b in zip(sg, p)))
    return out


def gaussian_moment(alpha):
    r = 1
    for a in alpha:
        for k in range(a - 1, 0, -2):
            r *= k
    return r


def moment_classes(dim, degree):
    cl = set()
    for alpha in itertools.product(range(0, degree + 1, 2), repeat=dim):
        if sum(alpha) <= degree:
            cl.add(tuple(sorted(alpha, reverse=True)))
    return sorted(cl, key=lambda a: (sum(a), a))


def shell_sum(shell_vecs, alpha):
    s = 0
    for v in shell_vecs:
        t = 1
        for a, e in zip(alpha, v):
            t *= e ** a
        s += t
    return s


def solve_linear(A, b):
    n = len(b)
    M = [row[:] + [bb] for row, bb in zip(A, b)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(M[r][col]))
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col] / M[col][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return [M[r][n] / M[r][r] for r in range(n)]


def weights_and_residual(spec, s):
    dim = spec["dim"]
    shells = [sorted(members(r, dim)) for r in spec["shells"]]
    classes = moment_classes(dim, spec["degree"])
    classes.remove(spec["residual"])
    classes.append(spec["residual"])
    nw = len(shells)
    rows = []
    rhs = []
    for alpha in classes:
        k = sum(alpha) // 2
        rows.append([D(shell_sum(sv, alpha)) * s ** k for sv in shells])
        rhs.append(D(gaussian_moment(alpha)))
    w = solve_linear(rows[:nw], rhs[:nw])
    res = sum(a * x for a, x in zip(rows[nw], w)) - rhs[nw]
    return w, res


def solve(spec):
    lo, hi = D(spec["bracket"][0]), D(spec["bracket"][1])
    rlo = weights_and_residual(spec, lo)[1]
    rhi = weights_and_residual(spec, hi)[1]
    assert rlo * rhi < 0, "root not bracketed"
    for _ in range(200):
        mid = (lo + hi) / 2
        rm = weights_and_residual(spec, mid)[1]
        if rm == 0:
            lo = hi = mid
            break
        if (rm < 0) == (rlo < 0):
            lo, rlo = mid, rm
        else:
            hi = mid
    s = (lo + hi) / 2
    w, _ = weights_and_residual(spec, s)
    return s, w


def ordered_directions(spec):
    dim = spec["dim"]
    dirs = [((0,) * dim, 0)]
    for k, rep in enumerate(spec["shells"]):
        if k == 0:
            continue
        seen = set()
        for v in sorted(members(rep, dim), reverse=True):
            if v in seen:
                continue
            nv = tuple(-x for x in v)
            seen.add(v)
            seen.add(nv)
            dirs.append((v, k))
            dirs.append((nv, k))
    return dirs


def hexd(x):
    return float(x).hex()


def emit(name, spec):
    s, w = solve(spec)
    c = s.sqrt()
    dirs = ordered_directions(spec)
    Q = len(dirs)
    dim = spec["dim"]
    lines = [f"struct {name} {{",
             f"  static constexpr int Q = {Q};",
             f"  static constexpr int D = {dim};",
             f"  static constexpr int NEQ = {spec['neq']};",
             f"  static constexpr int NSHELL = {len(spec['shells'])};",
             f"  static constexpr double c = {hexd(c)};   // {c:.25f}",
             f"  static constexpr double c2 = {hexd(s)};  // c^2 rounded once",
             "  // e[i] = (e_x, e_y, e_z); i = 0 rest, then (e, -e) pairs",
             f"  static constexpr int e[{Q}][3] = {{"]
    for v, _ in dirs:
        v3 = list(v) + [0] * (3 - dim)
        lines.append(f"    {{{v3[0]}, {v3[1]}, {v3[2]}}},")
    lines.append("  };")
    lines.append(f"  static constexpr int shell[{Q}] = {{" + ", ".join(str(k) for _, k in dirs) + "};")
    lines.append(f"  // |e|^2 of each shell")
    lines.append(f"  static constexpr int shell_e2[{len(spec['shells'])}] = {{"
                 + ", ".join(str(sum(x * x for x in r)) for r in spec["shells"]) + "};")
    lines.append(f"  static constexpr double shell_w[{len(w)}] = {{")
    for x in w:
        lines.append(f"    {hexd(x)},  // {x:.25f}")
    lines.append("  };")
    lines.append(f"  static constexpr double w[{Q}] = {{")
    for _, k in dirs:
        lines.append(f"    {hexd(w[k])},")
    lines.append("  };")
    lines.append("  // element accessors usable in device code inside constant expressions")
    lines.append("  __host__ __device__ static constexpr int E(int i, int a) { return e[i][a]; }")
    lines.append("  __host__ __device__ static constexpr int SH(int i) { return shell[i]; }")
    lines.append("  __host__ __device__ static constexpr int E2(int s) { return shell_e2[s]; }")
    lines.append("  __host__ __device__ static constexpr double W(int i) { return w[i]; }")
    lines.append("};")
    return lines


def main():
    out = ["// Generated by gen_tables.py -- do not edit.",
           "// Degree-Q Gauss-Hermite velocity sets; constants rounded once to double.",
           "#pragma once", "", "namespace lbm {", ""]
    for name, spec in SETS.items():
        out += emit(name, spec) + [""]
    out.append("}  // namespace lbm")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lattice_tables.cuh")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()

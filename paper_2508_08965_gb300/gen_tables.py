"""Exact generator of the reconstruction tables of the CUDA library.

Run ``python -m paper_2508_08965_gb300.gen_tables`` to rewrite
``csrc/cgks_tables.h`` and ``csrc/cgks_recon_gen.cuh``; both headers are
committed so that the build needs only nvcc.

What is tabulated (standard reference cell [0,1]^dim of Sec. 4, centroid 1/2,
h = 1, so delta = xi - 1/2 lies in [-1/2, 1/2]^dim):

* the quartic zero-mean basis of Eq. (base) (1 <= |d| <= 4: 34 terms in 3-D,
  14 in 2-D), ordered by reflection-parity class;
* the matrix M with a = M d for the constrained least squares of
  Eq. (compact-big-ref): face-neighbour averages exact, edge-neighbour
  averages (weight 1), face-neighbour gradients (h1' = 2), edge-neighbour
  directional derivatives (h2' = 1, unit directions along the shared edge and
  toward the neighbour centroid) and the target cell's line differences
  (h3' = 3) in the least-squares sense; neighbours are unit cells at integer
  offsets;
* the Gram matrices of the GENO smoothness indicators (all derivatives
  1 <= |l| <= 4, and |l| = 1 alone);
* basis values and gradients at the face Gauss points (2-point Gauss per
  tangential direction, +-1/(2 sqrt 3)).

All entries are computed exactly: rationals plus rational multiples of sqrt(3)
(the Gauss points), solved by fraction-exact Gaussian elimination on the KKT
system, and rounded once to double.

Data vector order used by the kernels (per variable):
  [Q0,
   for each face neighbour m (-x,+x,-y,+y[,-z,+z]): Q_m, (J0^T grad Q)_m (dim),
   for each edge neighbour n: Q_n, tv_n . (J0^T grad Q)_n with the integer
     directions tv = e_edge (3-D only) and tv = sum of the offset's non-zero
     signed unit vectors (not normalised; the weight carries 1/|tv|^2),
   line differences s = axis*gpf + k]
Edge neighbours are taken in increasing offset order (o_z, o_y, o_x
lexicographic, -1 < +1) among offsets with exactly two non-zero entries.
"""
import math
import itertools
import os
from decimal import Decimal, getcontext
from fractions import Fraction as Fr

getcontext().prec = 60
SQRT3 = Decimal(3).sqrt()


class Q3:
    """Number a + b sqrt(3) with rational a, b."""
    __slots__ = ("a", "b")

    def __init__(self, a=0, b=0):
        self.a, self.b = Fr(a), Fr(b)

    def __add__(self, o):
        o = _q(o)
        return Q3(self.a + o.a, self.b + o.b)

    __radd__ = __add__

    def __sub__(self, o):
        o = _q(o)
        return Q3(self.a - o.a, self.b - o.b)

    def __rsub__(self, o):
        return _q(o) - self

    def __mul__(self, o):
        o = _q(o)
        return Q3(self.a * o.a + 3 * self.b * o.b, self.a * o.b + self.b * o.a)

    __rmul__ = __mul__

    def __neg__(self):
        return Q3(-self.a, -self.b)

    def to_float(self):
        v = Decimal(self.a.numerator) / Decimal(self.a.denominator) + \
            Decimal(self.b.numerator) / Decimal(self.b.denominator) * SQRT3
        return float(v)

    def is_zero(self):
        return self.a == 0 and self.b == 0


def _q(x):
    return x if isinstance(x, Q3) else Q3(x, 0)


G = Q3(0, Fr(1, 6))  # 1/(2 sqrt 3) = sqrt(3)/6
HALF = Fr(1, 2)


def fact(n):
    f = 1
    for i in range(2, n + 1):
        f *= i
    return f


def ipow(x, e):
    r = Q3(1)
    for _ in range(e):
        r = r * x
    return r


def int_mono(e, lo, hi):
    """int_lo^hi t^e / e! dt (rational bounds)."""
    return (Fr(hi) ** (e + 1) - Fr(lo) ** (e + 1)) / fact(e + 1)


def basis(dim):
    """exponents with 1 <= |d| <= 4 grouped by parity class (d mod 2), then degree."""
    ex = [e for e in itertools.product(range(5), repeat=dim) if 1 <= sum(e) <= 4]
    ex.sort(key=lambda e: (tuple(x % 2 for x in e), sum(e), tuple(-x for x in e)))
    return ex


def stencil(dim):
    faces = []
    for ax in range(dim):
        for s in (-1, 1):
            o = [0] * dim
            o[ax] = s
            faces.append(tuple(o))
    edges = []
    for o in itertools.product((-1, 0, 1), repeat=dim):
        o = tuple(reversed(o))  # o_x fastest varying in the product -> reverse
        if sum(1 for x in o if x != 0) == 2:
            edges.append(o)
    edges.sort(key=lambda o: tuple(reversed(o)))
    return faces, edges


def gpf(dim):
    return 4 if dim == 3 else 2


def gp_delta(dim, ax, side, k):
    ta = [a for a in range(dim) if a != ax]
    d = [Q3(0)] * dim
    d[ax] = Q3(HALF if side else -HALF)
    d[ta[0]] = G if (k & 1) else -G
    if dim == 3:
        d[ta[1]] = G if (k & 2) else -G
    return d


def tau_dirs(dim, o):
    """directions of the edge-neighbour derivatives as integer vectors tv with
    the squared inverse norm 1/|tv|^2: along the shared edge (3-D only) and
    toward the neighbour centroid."""
    nz = [a for a in range(dim) if o[a] != 0]
    out = []
    if dim == 3:
        z = [a for a in range(3) if o[a] == 0][0]
        t1 = [0] * 3
        t1[z] = 1
        out.append((t1, Fr(1)))
    t2 = [0] * dim
    for a in nz:
        t2[a] = o[a]
    out.append((t2, Fr(1, 2)))  # |t2|^2 = 2 -> unit vector t2/sqrt(2)
    return out


def mean_basis(e):
    m = Fr(1)
    for x in e:
        m *= int_mono(x, -HALF, HALF)
    return m


def avg_basis(e, o):
    v = Fr(1)
    for i, x in enumerate(e):
        v *= int_mono(x, o[i] - HALF, o[i] + HALF)
    return v - mean_basis(e)


def avg_dbasis(e, k, o):
    if e[k] == 0:
        return Fr(0)
    v = Fr(1)
    for i, x in enumerate(e):
        xx = x - (1 if i == k else 0)
        v *= int_mono(xx, o[i] - HALF, o[i] + HALF)
    return v


def eval_basis(e, d):
    v = Q3(1)
    for i, x in enumerate(e):
        v = v * ipow(d[i], x) * Fr(1, fact(x))
    return v - mean_basis(e)


def eval_dbasis(e, k, d):
    if e[k] == 0:
        return Q3(0)
    v = Q3(1)
    for i, x in enumerate(e):
        xx = x - (1 if i == k else 0)
        v = v * ipow(d[i], xx) * Fr(1, fact(xx))
    return v


def solve_exact(K, B):
    """Solve K X = B exactly (K, B lists of lists of Fractions)."""
    n, m = len(K), len(B[0])
    A = [row[:] + brow[:] for row, brow in zip(K, B)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        inv = 1 / A[c][c]
        A[c] = [x * inv for x in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    return [row[n:] for row in A]


def build(dim):
    ex = basis(dim)
    nb = len(ex)
    faces, edges = stencil(dim)
    g = gpf(dim)
    ntau = 2 if dim == 3 else 1
    # data index map
    idx = {"Q0": 0}
    c = 1
    for m in range(len(faces)):
        idx[("fQ", m)] = c
        c += 1
        for k in range(dim):
            idx[("fG", m, k)] = c
            c += 1
    for n in range(len(edges)):
        idx[("eQ", n)] = c
        c += 1
        for t in range(ntau):
            idx[("eT", n, t)] = c
            c += 1
    for s in range(dim * g):
        idx[("L", s)] = c
        c += 1
    nd = c
    # equality rows (face averages) and least-squares rows: (coef row as Q3, weight^2, rhs column dict)
    eq_rows, ls_rows = [], []
    for m, o in enumerate(faces):
        eq_rows.append(([Q3(avg_basis(e, o)) for e in ex], {idx[("fQ", m)]: Q3(1), 0: Q3(-1)}))
    for n, o in enumerate(edges):
        ls_rows.append(([Q3(avg_basis(e, o)) for e in ex], Fr(1), {idx[("eQ", n)]: Q3(1), 0: Q3(-1)}))
    for m, o in enumerate(faces):
        for k in range(dim):
            ls_rows.append(([Q3(avg_dbasis(e, k, o)) for e in ex], Fr(4), {idx[("fG", m, k)]: Q3(1)}))
    for n, o in enumerate(edges):
        for t, (tv, s2) in enumerate(tau_dirs(dim, o)):
            row = [Q3(sum(tv[k] * avg_dbasis(e, k, o) for k in range(dim))) for e in ex]
            # the kernel loads tv . (J0^T grad Q) with the integer vector tv; the unit
            # direction is tv/|tv|, so the 1/|tv|^2 factor goes into the weight
            ls_rows.append((row, s2, {idx[("eT", n, t)]: Q3(1)}))
    for ax in range(dim):
        for k in range(g):
            hi, lo = gp_delta(dim, ax, 1, k), gp_delta(dim, ax, 0, k)
            row = [eval_basis(e, hi) - eval_basis(e, lo) for e in ex]
            ls_rows.append((row, Fr(9), {idx[("L", ax * g + k)]: Q3(1)}))
    # KKT: [sum w2 r r^T, C^T; C, 0][a; mu] = [sum w2 r rhs; rhs_eq]
    nk = nb + len(eq_rows)
    KQ = [[Q3(0)] * nb for _ in range(nb)]
    Br = [[Fr(0)] * nd for _ in range(nk)]
    Bs = [[Fr(0)] * nd for _ in range(nk)]
    for row, w2, rhs in ls_rows:
        for i in range(nb):
            if row[i].is_zero():
                continue
            for j in range(nb):
                if row[j].is_zero():
                    continue
                KQ[i][j] = KQ[i][j] + row[i] * row[j] * w2
            for col, r in rhs.items():
                v = row[i] * r * w2
                Br[i][col] += v.a
                Bs[i][col] += v.b
    K = [[Fr(0)] * nk for _ in range(nk)]
    for i in range(nb):
        for j in range(nb):
            # the sqrt(3) parts of the line rows cancel over the symmetric Gauss points
            assert KQ[i][j].b == 0
            K[i][j] = KQ[i][j].a
    for q, (row, rhs) in enumerate(eq_rows):
        for i in range(nb):
            assert row[i].b == 0
            K[i][nb + q] = row[i].a
            K[nb + q][i] = row[i].a
        for col, r in rhs.items():
            Br[nb + q][col] += r.a
    Xr = solve_exact(K, Br)
    Xs = solve_exact(K, Bs)
    M = [[Q3(Xr[i][j], Xs[i][j]) for j in range(nd)] for i in range(nb)]
    # Gram matrices
    GH = [[Fr(0)] * nb for _ in range(nb)]
    GL = [[Fr(0)] * nb for _ in range(nb)]
    lrange = [l for l in itertools.product(range(5), repeat=dim) if 1 <= sum(l) <= 4]
    for i, ei in enumerate(ex):
        for j, ej in enumerate(ex):
            sh = sl = Fr(0)
            for l in lrange:
                v = Fr(1)
                for a in range(dim):
                    p, q = ei[a] - l[a], ej[a] - l[a]
                    if p < 0 or q < 0:
                        v = Fr(0)
                        break
                    v *= int_mono(p + q, -HALF, HALF) * fact(p + q) / (fact(p) * fact(q))
                sh += v
                if sum(l) == 1:
                    sl += v
            GH[i][j], GL[i][j] = sh, sl
    # Gauss point tables: gp = (2*axis+side)*gpf + k
    ngp = 2 * dim * g
    PV = [[None] * nb for _ in range(ngp)]
    PD = [[[None] * nb for _ in range(dim)] for _ in range(ngp)]
    POS = []
    for f in range(2 * dim):
        for k in range(g):
            gp = f * g + k
            d = gp_delta(dim, f // 2, f & 1, k)
            POS.append(d)
            for b, e in enumerate(ex):
                PV[gp][b] = eval_basis(e, d)
                for kk in range(dim):
                    PD[gp][kk][b] = eval_dbasis(e, kk, d)
    return dict(ex=ex, nb=nb, nd=nd, M=M, GH=GH, GL=GL, PV=PV, PD=PD, POS=POS, faces=faces,
                edges=edges, ngp=ngp)


def _fmt(x):
    if isinstance(x, Q3):
        x = x.to_float()
    elif isinstance(x, Fr):
        x = float(Decimal(x.numerator) / Decimal(x.denominator))
    return repr(float(x))


def emit(path):
    out = ["/* Generated by paper_2508_08965_gb300/gen_tables.py -- do not edit.",
           "   Exact reconstruction tables of the CGKS-5 reference cell, rounded once to double. */",
           "#pragma once", "#ifndef CGKS_TABLE", "#define CGKS_TABLE __constant__", "#endif",
           "/* the Gauss-point tables live in global memory: the constant bank holds 64 KB */",
           "#ifndef CGKS_GTABLE", "#define CGKS_GTABLE __device__ const", "#endif", ""]
    for dim in (2, 3):
        t = build(dim)
        nb, nd, ngp = t["nb"], t["nd"], t["ngp"]
        p = "T%d" % dim
        out.append("/* %d-D: %d basis terms, %d data per variable, %d face Gauss points */" % (dim, nb, nd, ngp))
        out.append("#define %s_NB %d" % (p, nb))
        out.append("#define %s_ND %d" % (p, nd))
        out.append("#define %s_NGP %d" % (p, ngp))
        out.append("static const int %s_EXP[%d][3] = {%s};" % (
            p, nb, ", ".join("{%s}" % ", ".join(str(x) for x in list(e) + [0] * (3 - dim)) for e in t["ex"])))
        out.append("CGKS_TABLE double %s_M[%d][%d] = {" % (p, nb, nd))
        out += ["  {%s}," % ", ".join(_fmt(x) for x in row) for row in t["M"]]
        out.append("};")
        for name in ("GH", "GL"):
            out.append("CGKS_TABLE double %s_%s[%d][%d] = {" % (p, name, nb, nb))
            out += ["  {%s}," % ", ".join(_fmt(x) for x in row) for row in t[name]]
            out.append("};")
        out.append("CGKS_GTABLE double %s_PV[%d][%d] = {" % (p, ngp, nb))
        out += ["  {%s}," % ", ".join(_fmt(x) for x in row) for row in t["PV"]]
        out.append("};")
        out.append("CGKS_GTABLE double %s_PD[%d][%d][%d] = {" % (p, ngp, dim, nb))
        for gp in range(ngp):
            out.append("  {%s}," % ", ".join("{%s}" % ", ".join(_fmt(x) for x in t["PD"][gp][k]) for k in range(dim)))
        out.append("};")
        out.append("")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")




# ---------------------------------------------------------------------------
# Straight-line reconstruction code exploiting the reflection symmetry of the
# reference stencil.
#
# The least-squares problem is invariant under the reflections delta_s ->
# -delta_s of the reference cell, and the basis functions are eigenfunctions
# of them (parity class c = exponents mod 2).  Hence a_b, for b in class c,
# depends only on the class-c characters of the data: for every orbit o of
# data items under the reflection group, f_{c,o} = sum_S chi_c(S) sgn(S,o)
# d_{R_S(o)} and a_b = sum_o M[b,o] / |stab(o)| f_{c(b),o}.  The face Gauss
# points of one axis form one orbit too, so their values and gradients are a
# Walsh-Hadamard transform of per-class sums.  The Gram matrices of the
# smoothness indicators are block diagonal in the classes.
# ---------------------------------------------------------------------------

def _items(dim):
    """data items in the order of build(): (kind, index...)"""
    faces, edges = stencil(dim)
    ntau = 2 if dim == 3 else 1
    it = [("Q0",)]
    for m in range(len(faces)):
        it.append(("fQ", m))
        for k in range(dim):
            it.append(("fG", m, k))
    for n in range(len(edges)):
        it.append(("eQ", n))
        for t in range(ntau):
            it.append(("eT", n, t))
    for s in range(dim * gpf(dim)):
        it.append(("L", s))
    return it


def _reflect(dim, item, s):
    """image of a data item under the reflection of axis s: (item', sign)"""
    faces, edges = stencil(dim)
    kind = item[0]
    if kind == "Q0":
        return item, 1
    if kind in ("fQ", "fG"):
        o = list(faces[item[1]])
        o[s] = -o[s]
        m2 = faces.index(tuple(o))
        if kind == "fQ":
            return ("fQ", m2), 1
        return ("fG", m2, item[2]), (-1 if item[2] == s else 1)
    if kind in ("eQ", "eT"):
        o = list(edges[item[1]])
        o[s] = -o[s]
        n2 = edges.index(tuple(o))
        if kind == "eQ":
            return ("eQ", n2), 1
        t = item[2]
        if dim == 3 and t == 0:  # along the shared edge: flips when the edge axis is reflected
            z0 = [a for a in range(3) if edges[item[1]][a] == 0][0]
            return ("eT", n2, t), (-1 if s == z0 else 1)
        return ("eT", n2, t), 1  # toward the centroid: invariant
    if kind == "L":
        g = gpf(dim)
        d, k = item[1] // g, item[1] % g
        if s == d:
            return item, -1
        ta = [a for a in range(dim) if a != d]
        bit = 1 if ta[0] == s else 2
        return ("L", d * g + (k ^ bit)), 1
    raise ValueError(item)


def _group(dim):
    return [tuple(a for a in range(dim) if (S >> a) & 1) for S in range(1 << dim)]


def _act(dim, item, S):
    sign = 1
    for s in S:
        item, sg = _reflect(dim, item, s)
        sign *= sg
    return item, sign


def _classes(dim):
    return list(itertools.product((0, 1), repeat=dim))


def _chi(c, S):
    v = 1
    for s in S:
        if c[s]:
            v = -v
    return v


def symmetry_plan(dim):
    """orbits of data items and, per orbit and class, the signed item sums"""
    items = _items(dim)
    pos = {it: i for i, it in enumerate(items)}
    G = _group(dim)
    seen, orbits = set(), []
    for it in items:
        if it in seen:
            continue
        orb = sorted({_act(dim, it, S)[0] for S in G}, key=lambda x: pos[x])
        seen |= set(orb)
        rep = it
        stab = sum(1 for S in G if _act(dim, rep, S)[0] == rep)
        feats = {}
        for c in _classes(dim):
            coef = {}
            for S in G:
                img, sg = _act(dim, rep, S)
                coef[img] = coef.get(img, 0) + _chi(c, S) * sg
            coef = {k: v for k, v in coef.items() if v != 0}
            if coef:
                feats[c] = coef
        orbits.append((rep, orb, stab, feats))
    return items, pos, orbits


def _lit(x):
    return "T(%s)" % repr(float(x))


def emit_recon_code(path):
    out = ["/* Generated by paper_2508_08965_gb300/gen_tables.py -- do not edit.",
           "   Straight-line CGKS-5 reconstruction on the reference cell using its",
           "   reflection symmetry (see gen_tables.py), generic in the real type T.",
           "   Ld is a loader with q0(), avg(ox,oy,oz), grefv(ox,oy,oz,g[dim])",
           "   (neighbour gradient in the target's reference frame) and line(s) (own",
           "   reference line difference); averages may be given relative to q0. */",
           "#pragma once", ""]
    for dim in (2, 3):
        t = build(dim)
        ex, nb = t["ex"], t["nb"]
        M = [[x.to_float() for x in row] for row in t["M"]]
        items, pos, orbits = symmetry_plan(dim)
        cls = [tuple(x % 2 for x in e) for e in ex]
        faces, edges = stencil(dim)
        # numerical check of the orbit formula against M
        import random
        rnd = random.Random(5)
        dvec = [rnd.uniform(-1, 1) for _ in items]
        for b in range(nb):
            ref = sum(M[b][j] * dvec[j] for j in range(len(items)))
            acc = 0.0
            for rep, orb, stab, feats in orbits:
                if cls[b] in feats:
                    f = sum(cf * dvec[pos[it]] for it, cf in feats[cls[b]].items())
                    acc += M[b][pos[rep]] / stab * f
            assert abs(acc - ref) < 1e-12 * (1 + abs(ref)), (dim, b, acc, ref)
        # group orbits by the neighbour set they read
        def nb_offsets(it):
            if it[0] in ("fQ", "fG"):
                return (faces[it[1]],)
            if it[0] in ("eQ", "eT"):
                return (edges[it[1]],)
            return ((0,) * dim,)
        groups = {}
        for o in orbits:
            key = tuple(sorted({nb_offsets(it)[0] for it in o[1]}))
            groups.setdefault(key, []).append(o)
        fn = []
        fn.append("template <typename T, class Ld>")
        fn.append("CGKS_HD void gen_coeffs_%dd(const Ld& ld, T* __restrict__ a) {" % dim)
        fn.append("#pragma unroll")
        fn.append("  for (int b = 0; b < %d; ++b) a[b] = T(0);" % nb)

        def off3(o):
            o = list(o) + [0] * (3 - dim)
            return "%d, %d, %d" % tuple(o)

        for key, orbs in groups.items():
            fn.append("  {")
            var = {}
            for o in key:
                if all(x == 0 for x in o):
                    continue
                nm = "n" + "".join("m" if x < 0 else ("p" if x > 0 else "z") for x in o)
                fn.append("    const T %sQ = ld.avg(%s);" % (nm, off3(o)))
                fn.append("    T %sG[%d];" % (nm, dim))
                fn.append("    ld.grefv(%s, %sG);" % (off3(o), nm))
                var[o] = nm

            def item_expr(it):
                if it[0] == "Q0":
                    return "ld.q0()"
                if it[0] == "L":
                    return "ld.line(%d)" % it[1]
                if it[0] == "fQ":
                    return "%sQ" % var[faces[it[1]]]
                if it[0] == "fG":
                    return "%sG[%d]" % (var[faces[it[1]]], it[2])
                if it[0] == "eQ":
                    return "%sQ" % var[edges[it[1]]]
                o = edges[it[1]]
                nm = var[o]
                if dim == 3 and it[2] == 0:
                    z0 = [a for a in range(3) if o[a] == 0][0]
                    return "%sG[%d]" % (nm, z0)
                terms = ["%s%sG[%d]" % ("+" if o[a] > 0 else "-", nm, a) for a in range(dim) if o[a] != 0]
                return "(%s)" % " ".join(terms).lstrip("+")

            oi = [0]

            def butterfly_plan(work):
                """For an orbit whose features are +-g sums (g a power of two)
                over the same four items: every feature is
                g (+-(x_0 +- x_1) +- (x_2 +- x_3)), so the pair sums and
                differences serve all features (at most 4 additions, plus one
                per feature, instead of three per feature).  None otherwise."""
                if len(work) < 3:
                    return None
                its = sorted(work[0][1], key=lambda it: pos[it])
                if len(its) != 4 or any(sorted(cf, key=lambda it: pos[it]) != its for _, cf, _, _ in work):
                    return None
                mags = {abs(v) for _, cf, _, _ in work for v in cf.values()}
                if len(mags) != 1:
                    return None
                g = mags.pop()
                if g & (g - 1):
                    return None
                plan = []
                for _, cf, _, _ in work:
                    sg = [cf[its[q]] // g for q in range(4)]
                    plan.append((sg[0], sg[0] * sg[1], sg[2], sg[2] * sg[3]))
                return its, g, plan

            for rep, orb, stab, feats in orbs:
                # features of this orbit that reach a coefficient
                work = []
                for c, coef in feats.items():
                    if all(it[0] == "Q0" for it in coef):
                        continue
                    rows = [b for b in range(nb) if cls[b] == c and M[b][pos[rep]] != 0.0]
                    if rows:
                        work.append((c, coef, rows, None))
                bp = butterfly_plan(work)
                if bp is not None:
                    its, g, plan = bp
                    (i, j), (k, l) = (0, 1), (2, 3)
                    oi[0] += 1
                    nm = "o%d" % oi[0]
                    fn.append("    const T %sx0 = %s, %sx1 = %s, %sx2 = %s, %sx3 = %s;" % (
                        nm, item_expr(its[0]), nm, item_expr(its[1]), nm, item_expr(its[2]), nm, item_expr(its[3])))
                    used = set()
                    for _, pij, _, pkl in plan:
                        used.add(("a", pij))
                        used.add(("b", pkl))
                    for side, (p, q) in (("a", (i, j)), ("b", (k, l))):
                        for sg in (1, -1):
                            if (side, sg) in used:
                                fn.append("    const T %s%s%s = %sx%d %s %sx%d;" % (
                                    nm, side, "p" if sg > 0 else "m", nm, p, "+" if sg > 0 else "-", nm, q))
                    for (c, coef, rows, _), (si, pij, sk, pkl) in zip(work, plan):
                        t1 = "%sa%s" % (nm, "p" if pij > 0 else "m")
                        t2 = "%sb%s" % (nm, "p" if pkl > 0 else "m")
                        expr = "%s%s %s %s" % ("" if si > 0 else "-", t1, "+" if si * sk > 0 else "-", t2)
                        fn.append("    { const T f = %s;" % expr.strip())
                        for b in rows:
                            fn.append("      a[%d] = cg_fma(%s, f, a[%d]);" % (b, _lit(M[b][pos[rep]] / stab * g), b))
                        fn.append("    }")
                    continue
                for c, coef in feats.items():
                    # the loader hands averages over relative to q0, so q0
                    # itself is zero: its terms add nothing
                    if all(it[0] == "Q0" for it in coef):
                        continue
                    # a power-of-two factor common to the integer weights
                    # moves into the coefficients (exact scaling: the same
                    # values, without the multiplications)
                    g = 0
                    for cf in coef.values():
                        g = math.gcd(g, abs(cf))
                    if g & (g - 1):
                        g = 1
                    expr = " ".join("%s%s" % ("+" if cf > 0 else "-", item_expr(it)) if abs(cf) == g else
                                    "%sT(%d)*%s" % ("+" if cf > 0 else "-", abs(cf) // g, item_expr(it))
                                    for it, cf in coef.items()).lstrip("+")
                    rows = [b for b in range(nb) if cls[b] == c and M[b][pos[rep]] != 0.0]
                    if not rows:
                        continue
                    fn.append("    { const T f = %s;" % expr)
                    for b in rows:
                        fn.append("      a[%d] = cg_fma(%s, f, a[%d]);" % (b, _lit(M[b][pos[rep]] / stab * g), b))
                    fn.append("    }")
            fn.append("  }")
        fn.append("}")
        fn.append("")
        # Gram quadratic forms (block diagonal by class)
        GH = [[float(x) for x in row] for row in t["GH"]]
        GL = [[float(x) for x in row] for row in t["GL"]]
        # the higher-derivative part GH - GL (exact in rational arithmetic) and
        # the entrywise absolute values, for the FP32 screen of the FP64 path
        GT = [[float(t["GH"][i][j] - t["GL"][i][j]) for j in range(nb)] for i in range(nb)]
        GTA = [[abs(x) for x in row] for row in GT]
        GLA = [[abs(x) for x in row] for row in GL]
        for name, Gm in (("ish", GH), ("isl", GL), ("ist", GT), ("ista", GTA), ("isla", GLA)):
            fn.append("template <typename T>")
            fn.append("CGKS_HD T gen_%s_%dd(const T* __restrict__ a) {" % (name, dim))
            fn.append("  T s = T(0);")
            for i in range(nb):
                terms = []
                if Gm[i][i] != 0.0:
                    terms.append((_lit(Gm[i][i]), i))
                for j in range(i + 1, nb):
                    if Gm[i][j] != 0.0:
                        assert cls[i] == cls[j]
                        terms.append((_lit(2.0 * Gm[i][j]), j))
                if not terms:
                    continue
                fn.append("  { T r = T(0);")
                for cst, j in terms:
                    fn.append("    r = cg_fma(%s, a[%d], r);" % (cst, j))
                fn.append("    s = cg_fma(a[%d], r, s); }" % i)
            fn.append("  return s;")
            fn.append("}")
            fn.append("")
        # mean of the P4 correction: sum_b a_b mean_b
        fn.append("template <typename T>")
        fn.append("CGKS_HD T gen_mean_%dd(const T* __restrict__ a) {" % dim)
        fn.append("  T s = T(0);")
        for b, e in enumerate(ex):
            mb = mean_basis(e)
            if mb != 0:
                fn.append("  s = cg_fma(%s, a[%d], s);" % (_lit(float(mb)), b))
        fn.append("  return s;")
        fn.append("}")
        fn.append("")
        # face Gauss points of axis AX: values and reference gradients of P4 - Q0 + mean
        g = gpf(dim)
        npts = 2 * g
        for ax in range(dim):
            ta = [a for a in range(dim) if a != ax]
            # representative x0: +1/2 along ax, +g along the tangential axes
            x0 = [Q3(0)] * dim
            x0[ax] = Q3(HALF)
            for a in ta:
                x0[a] = G
            fn.append("/* axis %d: out_v[i], out_g[i][k] for the %d Gauss points i = side*%d + k */" % (ax, npts, g))
            fn.append("template <typename T>")
            fn.append("CGKS_HD void gen_gp_%dd_ax%d(const T* __restrict__ a, T* __restrict__ out_v, "
                      "T (* __restrict__ out_g)[%d]) {" % (dim, ax, dim))
            C = _classes(dim)
            # class sums of values and of each derivative
            for ci, c in enumerate(C):
                terms = []
                for b, e in enumerate(ex):
                    if cls[b] != c:
                        continue
                    v = Q3(1)
                    for i2 in range(dim):
                        v = v * ipow(x0[i2], e[i2]) * Fr(1, fact(e[i2]))
                    terms.append((v.to_float(), b))
                fn.append("  T S%d = T(0);" % ci)
                for v, b in terms:
                    if v != 0.0:
                        fn.append("  S%d = cg_fma(%s, a[%d], S%d);" % (ci, _lit(v), b, ci))
                for k in range(dim):
                    fn.append("  T D%d_%d = T(0);" % (ci, k))
                    for b, e in enumerate(ex):
                        if cls[b] != c or e[k] == 0:
                            continue
                        v = Q3(1)
                        for i2 in range(dim):
                            ee = e[i2] - (1 if i2 == k else 0)
                            v = v * ipow(x0[i2], ee) * Fr(1, fact(ee))
                        fn.append("  D%d_%d = cg_fma(%s, a[%d], D%d_%d);" % (ci, k, _lit(v.to_float()), b, ci, k))
            # Each Gauss point is R_S x0 for the set S of negated axes, and
            #   value(S)         = sum_c chi_c(S) S_c,
            #   d/dx_kk value(S) = sum_c chi_{c xor e_kk}(S) D_c,kk
            #                    = (-1)^[kk in S] sum_c chi_c(S) D_c,kk,
            # chi_c(S) = (-1)^(c . S): a Walsh-Hadamard transform over the class
            # bits, evaluated by butterflies (dim 2^(dim-1) of them) instead of
            # one 2^dim-term sum per point.
            def wht(prefix, names):
                """emit butterflies over the class bits; returns the output
                variable of each mask of negated axes"""
                cur = {}
                for ci, c in enumerate(C):
                    m = sum(bit << a for a, bit in enumerate(c))
                    cur[m] = names[ci]
                for a in range(dim):
                    nxt = {}
                    for m in range(1 << dim):
                        if m & (1 << a):
                            continue
                        m2 = m | (1 << a)
                        n0, n1 = "%s%d_%d" % (prefix, a, m), "%s%d_%d" % (prefix, a, m2)
                        fn.append("  const T %s = %s + %s, %s = %s - %s;" % (n0, cur[m], cur[m2], n1, cur[m],
                                                                          cur[m2]))
                        nxt[m], nxt[m2] = n0, n1
                    cur = nxt
                return cur
            yv = wht("wv", ["S%d" % ci for ci in range(len(C))])
            yg = [wht("wg%d_" % kk, ["D%d_%d" % (ci, kk) for ci in range(len(C))]) for kk in range(dim)]
            for side in (0, 1):
                for k in range(g):
                    S = []
                    if side == 0:
                        S.append(ax)
                    if not (k & 1):
                        S.append(ta[0])
                    if dim == 3 and not (k & 2):
                        S.append(ta[1])
                    i = side * g + k
                    m = sum(1 << a for a in S)
                    fn.append("  out_v[%d] = %s;" % (i, yv[m]))
                    for kk in range(dim):
                        fn.append("  out_g[%d][%d] = %s%s;" % (i, kk, "-" if kk in S else "", yg[kk][m]))
            fn.append("}")
            fn.append("")
        # the coefficients in the frame of axis ax: the coordinates relabelled
        # by pi (pi(0) = ax, the tangential axes in increasing order), so that
        # the axis-0 Gauss-point code evaluates the faces of axis ax; the
        # code's derivative j is the physical derivative pi(j)
        fn.append("/* the coefficients a relabelled for the faces of axis ax: o[b'] = a[b] where")
        fn.append("   exponent(b)[pi(j)] = exponent(b')[j], pi(0) = ax, pi(1) < pi(2) */")
        fn.append("template <typename T>")
        fn.append("CGKS_HD void gen_perm_%dd(const T* __restrict__ a, int ax, T* __restrict__ o) {" % dim)
        index = {e: b for b, e in enumerate(ex)}
        for b2, e2 in enumerate(ex):
            srcs = []
            for ax in range(dim):
                pi = [ax] + [x for x in range(dim) if x != ax]
                e = [0] * dim
                for j in range(dim):
                    e[pi[j]] = e2[j]
                srcs.append(index[tuple(e)])
            if dim == 3:
                fn.append("  o[%d] = ax == 0 ? a[%d] : (ax == 1 ? a[%d] : a[%d]);" % (b2, srcs[0], srcs[1], srcs[2]))
            else:
                fn.append("  o[%d] = ax == 0 ? a[%d] : a[%d];" % (b2, srcs[0], srcs[1]))
        fn.append("}")
        fn.append("")
        out += fn
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


def emit_all():
    here = os.path.dirname(os.path.abspath(__file__))
    emit(os.path.join(here, "csrc", "cgks_tables.h"))
    emit_recon_code(os.path.join(here, "csrc", "cgks_recon_gen.cuh"))


if __name__ == "__main__":
    emit_all()

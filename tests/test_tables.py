"""P15: the CUDA library's exact (rational) reconstruction tables agree with the
oracle's run-time long-double KKT solution of Eq. (compact-big-ref)."""
import math

import numpy as np
import pytest

import refgeom as rg
from tables_header import read_table


def product_data_from_oracle_data(dim, d):
    """Re-order an oracle data vector into the library's layout (see gen_tables)."""
    fo = rg.face_offsets(dim)
    eo, taus = rg.edge_offsets_and_tau(dim)
    nf, ne = len(fo), len(eo)
    ntau = 2 if dim == 3 else 1
    o_face, o_edge = 1, 1 + nf
    o_fg = o_edge + ne
    o_et = o_fg + nf * dim
    o_line = o_et + ne * ntau
    out = [d[0]]
    for m in range(nf):
        out.append(d[o_face + m])
        out += list(d[o_fg + m * dim: o_fg + (m + 1) * dim])
    # library edge order: offsets sorted by (o_z, o_y, o_x)
    order = sorted(range(ne), key=lambda n: tuple(reversed(eo[n])))
    for n in order:
        out.append(d[o_edge + n])
        for t in range(ntau):
            v = d[o_et + n * ntau + t]
            # oracle uses unit directions, the library the un-normalised offset vector
            if t == ntau - 1:
                v = v * math.sqrt(2.0)
            out.append(v)
    out += list(d[o_line:])
    return np.array(out)


@pytest.mark.parametrize("dim", [2, 3])
def test_generated_matrix_matches_oracle_kkt(orc, dim):
    Mo, exo = orc.recon_matrix(dim)
    Mp = read_table("T%d_M" % dim)
    exp = read_table("T%d_EXP" % dim).astype(int)
    nd = Mo.shape[1]
    rng = np.random.default_rng(9)
    for _ in range(5):
        d = rng.standard_normal(nd)
        ao = Mo @ d
        ap = Mp @ product_data_from_oracle_data(dim, d)
        ko = {tuple(e[:dim]): v for e, v in zip(exo, ao)}
        for e, v in zip(exp, ap):
            ref = ko[tuple(e[:dim])]
            assert abs(v - ref) <= 1e-13 * max(1.0, np.abs(ao).max())


@pytest.mark.parametrize("dim", [2, 3])
def test_generated_gram_matches_oracle(orc, dim):
    gho, glo = orc.gram(dim)
    _, exo = orc.recon_matrix(dim)
    exp = read_table("T%d_EXP" % dim).astype(int)
    pos = {tuple(e[:dim]): i for i, e in enumerate(exo)}
    perm = [pos[tuple(e[:dim])] for e in exp]
    for name, ref in (("GH", gho), ("GL", glo)):
        Gp = read_table("T%d_%s" % (dim, name))
        assert np.allclose(Gp, ref[np.ix_(perm, perm)], rtol=1e-15, atol=1e-16)

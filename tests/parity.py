"""Shared helpers of the GPU parity tests."""
import numpy as np


def class_scaled_diff(a, b, h=None, avg_floor=None):
    """max |a - b| / scale over variable classes (density, momentum vector,
    energy) and field groups (cell averages; all derivative fields).

    Averages: scale = max |b| of the class.  Momentum components share a
    scale because they form one vector.
    Derivative fields: they are difference quotients of interface values of
    size ~|average|, so their rounding is ~eps |average| / h whatever their
    own size; with h (the smallest cell size) given, their scale is
    max(max |b|, max |average| / h).  Without h the derivative scale is
    max |b| alone (stricter for small derivatives).
    avg_floor: (density, momentum, energy) magnitudes of the whole field, a
    floor for max |average| when b holds a few sampled cells only (where a
    class can vanish, e.g. the momentum at a symmetry point of the flow)."""
    nf, nv = b.shape[0], b.shape[1]
    classes = [[0], list(range(1, nv - 1)), [nv - 1]]
    worst = 0.0
    for ci, c in enumerate(classes):
        avg = np.abs(b[np.ix_([0], c)]).max()
        if avg_floor is not None:
            avg = max(avg, avg_floor[ci])
        for g in ([0], list(range(1, nf))):
            ix = np.ix_(g, c)
            sc = np.abs(b[ix]).max()
            if g == [0]:
                sc = max(sc, avg)
            if g != [0] and h is not None:
                sc = max(sc, avg / h)
            if sc == 0.0:
                sc = 1.0
            worst = max(worst, np.abs(a[ix] - b[ix]).max() / sc)
    return worst

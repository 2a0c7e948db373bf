"""Shared helpers of the GPU parity tests."""
import numpy as np


def class_scaled_diff(a, b):
    """max |a - b| / scale, scale = max |b| over the same variable class
    (density, momentum vector, energy) and field group (cell averages, or all
    derivative fields).  Momentum components share a scale because they form
    one vector; derivative fields share one because they are differences of
    the same interface values."""
    nf, nv = b.shape[0], b.shape[1]
    classes = [[0], list(range(1, nv - 1)), [nv - 1]]
    groups = [[0], list(range(1, nf))]
    worst = 0.0
    for g in groups:
        for c in classes:
            ix = np.ix_(g, c)
            sc = np.abs(b[ix]).max()
            if sc == 0.0:
                sc = 1.0
            worst = max(worst, np.abs(a[ix] - b[ix]).max() / sc)
    return worst

"""Ordered-subset partition of the sinogram rows (§2.1, Eq. (subobjective)).

The rows are split by view into N_s disjoint, nonempty subsets whose union is
every row.  Views are dealt out angle-interleaved (view i goes to subset
i mod N_s), which keeps the subsets balanced and spreads each subset's views over
[0, pi), so that consecutive subsets see nearly orthogonal views as §2.1
recommends (§5.1 splits its 180 views into 15/30/45 subsets of 12/6/4
views).  When N_s
does not divide the number of views, the first n_angles mod N_s subsets get
one extra view.
"""
from __future__ import annotations

import numpy as np


def subset_views(n_angles: int, n_subsets: int):
    """List of view-index arrays, one per subset, views in increasing order."""
    if not 1 <= n_subsets <= n_angles:
        raise ValueError("need 1 <= n_subsets <= n_angles")
    return [np.arange(t, n_angles, n_subsets) for t in range(n_subsets)]


def subset_rows(n_angles: int, n_bins: int, n_subsets: int):
    """List of row-index arrays (row = view*n_bins + bin), one per subset."""
    return [(v[:, None] * n_bins + np.arange(n_bins)[None, :]).ravel()
            for v in subset_views(n_angles, n_subsets)]

"""Sufficient statistics (FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper: Section "Notation" defines mat_l[X] (d_l x d_{\\l}) and
S_l = mat_l[{X}] mat_l[{X}]^T; Section "Algorithm" shows S_l for several
modalities is the Gram of the column-concatenation of their matricisations.
Reading (two-axis case): rows of X are cells, so S_cells = X X^T and
S_genes = X^T X; no 1/n normalisation.
"""

import numpy as np


def log1p_centre(counts: np.ndarray) -> np.ndarray:
    """Preprocessing used by the scRNA-like workloads: log1p, then centre every
    column (gene) over the rows (cells).  Returns float64."""
    x = np.log1p(np.asarray(counts, dtype=np.float64))
    return x - x.mean(axis=0, keepdims=True)


def log1p_col_means(chunks, threads: int = 8) -> np.ndarray:
    """The column means that ``log1p_centre`` subtracts, for a matrix given as
    row blocks (``chunks`` yields array-likes with the same columns): each
    block's FP64 column sums of log1p, added, over the total row count.  Row
    blocks only split the sum over cells; ``threads`` blocks are summed at a
    time (numpy releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    def part(c):
        y = np.log1p(np.asarray(c, dtype=np.float64))
        return y.sum(axis=0), y.shape[0]

    total, n = None, 0
    it = iter(chunks)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while True:
            wave = [c for _, c in zip(range(threads), it)]  # at most `threads` blocks held at once
            if not wave:
                break
            for s, m in ex.map(part, wave):
                total = s if total is None else total + s
                n += m
    return total / n


def matricize(t: np.ndarray, axis: int) -> np.ndarray:
    """mat_l[T]: move ``axis`` to the front and flatten the rest (row-major),
    giving a d_l x (prod of the other sizes) matrix."""
    t = np.asarray(t, dtype=np.float64)
    return np.moveaxis(t, axis, 0).reshape(t.shape[axis], -1)


def gram(t: np.ndarray, axis: int) -> np.ndarray:
    """S_l = mat_l[T] mat_l[T]^T for one tensor (matrix: axis 0 -> X X^T,
    axis 1 -> X^T X)."""
    m = matricize(t, axis)
    return m @ m.T


def gram_multimodal(tensors, axis_labels, label) -> np.ndarray:
    """S_l = sum over modalities containing axis ``label`` of that modality's
    Gram along it (equivalently the Gram of the concatenated matricisation).

    ``tensors[g]`` has axes named ``axis_labels[g]`` (a tuple of labels)."""
    s = None
    for t, labels in zip(tensors, axis_labels):
        if label not in labels:
            continue
        g = gram(t, labels.index(label))
        s = g if s is None else s + g
    return s


def log1p_centred_gram_blocks(chunks):
    """Column Gram of the centred log1p matrix, for a matrix given as row
    blocks (too large for FP64 in memory): with Y = log1p(counts) and mu its
    column means, (Y - 1 mu^T)^T (Y - 1 mu^T) = sum_b Y_b^T Y_b - n mu mu^T
    (the same rank-one correction as the sparse path).  One pass over the
    blocks.  Returns (S, mu, n), FP64."""
    s, tot, n = None, None, 0
    for c in chunks:
        y = np.log1p(np.asarray(c, dtype=np.float64))
        g = y.T @ y
        cs = y.sum(axis=0)
        s = g if s is None else s + g
        tot = cs if tot is None else tot + cs
        n += y.shape[0]
    mu = tot / n
    return s - n * np.outer(mu, mu), mu, n
